"""The C ABI library builds for sm_103a, loads, and exports every function include/petgem.h
declares (no compute calls: these run without a GPU)."""
import ctypes
import os

import pytest

from paper_1808_00186_gb300 import api
from paper_1808_00186_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib_path():
    return libbuild.build()


def test_header_declares_the_boundary():
    names = api.header_functions()
    for required in ("petgem_create", "petgem_destroy", "petgem_mesh_edges", "petgem_assemble", "petgem_solve",
                     "petgem_receivers", "petgem_status_string", "petgem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in api.header_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(api.header_functions()) == set(api._SIGNATURES)


def test_status_strings_without_gpu(lib_path):
    L = api.load(lib_path)
    assert L.petgem_status_string(0) == b"ok"
    assert L.petgem_status_string(api.ERR_NOT_CONVERGED) == b"not converged"
    assert L.petgem_last_error(None) == b"null context"
    # A null context is rejected before any CUDA call.
    assert L.petgem_solve(None, None, None, None) == api.ERR_INVALID_ARG
    assert L.petgem_destroy(None) == api.OK
    # the batch solver and the frequency re-assembly check their arguments on the host too
    assert L.petgem_solve_batch(None, 0, None, None, None) == api.OK  # nothing to do
    assert L.petgem_solve_batch(None, 1, None, None, None) == api.ERR_INVALID_ARG
    assert L.petgem_assemble_frequency(None, 1.0, 1, None) == api.ERR_INVALID_ARG
    # the SSOR ordering and preconditioner entry points
    assert L.petgem_colouring(None, None, None, None) == api.ERR_INVALID_ARG
    assert L.petgem_ssor_apply(None, 1.0, None, None) == api.ERR_INVALID_ARG


def test_solve_opts_layout_matches_the_header():
    # the omega field closes the struct: int32 x4, double x2, int64, int32 x4, double = 64 bytes
    assert ctypes.sizeof(api.petgem_solve_opts) == 64
    assert api.petgem_solve_opts.omega.offset == 56
    o = api.solve_opts(precond=api.PRECOND_SSOR, method=api.METHOD_SQMR, omega=1.2)
    assert (o.precond, o.method, o.omega) == (2, 2, 1.2)


def test_no_cpu_fallback_when_library_missing(tmp_path):
    saved = api._lib
    api._lib = None
    try:
        with pytest.raises(RuntimeError):
            api.load(str(tmp_path / "missing.so"))
    finally:
        api._lib = saved


def test_noalloc_limit_matches_header_and_is_checked_on_the_host(lib_path):
    import re
    text = open(api.HEADER).read()
    assert int(re.search(r"#define PETGEM_NOALLOC_MAX_VOXELS (\d+)", text).group(1)) == api.NOALLOC_MAX_VOXELS
    L = api.load(lib_path)
    fake = ctypes.c_void_p(256)  # never dereferenced: the sizes are rejected before any CUDA call
    assert L.petgem_nn_conv3d_wgrad_noalloc(None, 64, 64, 33, 16, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d_wgrad_noalloc(None, 8, 8, 8, 24, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d_wgrad_noalloc(None, 0, 8, 8, 16, 16, fake, fake, fake) == api.ERR_INVALID_ARG


def test_conv_grids_whose_voxel_count_wraps_are_rejected_on_the_host(lib_path):
    """Dimensions whose product overflows 64 bits (2^21 + 1 cubed wraps negative) or exceeds the
    kernels' 32-bit voxel indexing are refused before any CUDA call, with nothing written."""
    L = api.load(lib_path)
    fake = ctypes.c_void_p(256)  # never dereferenced
    big = 2 ** 21 + 1
    assert L.petgem_nn_conv3d_wgrad_noalloc(None, big, big, big, 16, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d_wgrad_noalloc(None, 131073, 1, 1, 16, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d_wgrad(None, big, big, big, 16, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d_wgrad(None, 1024, 1024, 64, 16, 16, fake, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d(None, big, big, big, 16, 16, fake, fake, fake, 0, fake, 1) == api.ERR_UNSUPPORTED
    assert L.petgem_nn_conv3d(None, 4, 4, 4, 16, 24, fake, fake, fake, 0, fake, 1) == api.ERR_UNSUPPORTED
    odd = ctypes.c_void_p(264)  # 8-byte aligned only
    assert L.petgem_nn_conv3d(None, 4, 4, 4, 16, 16, odd, fake, fake, 0, fake, 1) == api.ERR_INVALID_ARG
    assert L.petgem_nn_conv3d(None, 4, 4, 4, 16, 16, fake, fake, fake, 0, odd, 1) == api.ERR_INVALID_ARG


def test_layered_primary_field_checks_its_arguments_on_the_host(lib_path):
    L = api.load(lib_path)
    d = api.petgem_dipole(0.0, 0.0, 50.0, 1.0, 0, 0)
    dz = api.petgem_dipole(0.0, 0.0, 50.0, 1.0, 2, 0)
    zi = (ctypes.c_double * 2)(0.0, -100.0)
    zbad = (ctypes.c_double * 2)(0.0, 10.0)
    sg = (ctypes.c_double * 3)(3.3, 1.0, 0.01)
    sneg = (ctypes.c_double * 3)(3.3, -1.0, 0.01)
    fake = ctypes.c_void_p(256)  # never dereferenced
    assert L.petgem_primary_layered(None, 3, zi, sg, 1.0, ctypes.byref(d), 0, None, None) == api.OK
    assert L.petgem_primary_layered(None, 3, zbad, sg, 1.0, ctypes.byref(d), 4, fake, fake) == api.ERR_INVALID_ARG
    assert L.petgem_primary_layered(None, 3, zi, sneg, 1.0, ctypes.byref(d), 4, fake, fake) == api.ERR_INVALID_ARG
    assert L.petgem_primary_layered(None, 3, zi, sg, 0.0, ctypes.byref(d), 4, fake, fake) == api.ERR_INVALID_ARG
    assert L.petgem_primary_layered(None, 3, zi, sg, 1.0, ctypes.byref(dz), 4, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_primary_layered(None, 9, zi, sg, 1.0, ctypes.byref(d), 4, fake, fake) == api.ERR_UNSUPPORTED
    assert L.petgem_primary_layered(None, 3, zi, sg, 1.0, ctypes.byref(d), 4, None, fake) == api.ERR_INVALID_ARG
