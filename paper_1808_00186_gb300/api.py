"""Thin Python binding of the petgem C ABI (include/petgem.h).

Argument marshalling only: every step of the computation runs in libpetgem.so's CUDA
kernels.  Device buffers are torch CUDA tensors (torch is used for memory and streams);
the functions take and return them with the layouts petgem.h documents.

load() raises when the library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpetgem.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "petgem.h")

OK, ERR_INVALID_ARG, ERR_BAD_MESH, ERR_DEGENERATE_TET, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_NOT_CONVERGED, \
    ERR_BREAKDOWN, ERR_RECEIVER_OUTSIDE, ERR_UNSUPPORTED, ERR_TIMEOUT = range(11)
PREC_C128, PREC_MIXED = 0, 1
ORTH_CGS2, ORTH_CGS, ORTH_CGS_IFNEEDED = 0, 1, 2
PRECOND_JACOBI, PRECOND_LEARNED, PRECOND_SSOR = 0, 1, 2
METHOD_GMRES, METHOD_COCG, METHOD_SQMR = 0, 1, 2


class petgem_dipole(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("z", ctypes.c_double),
                ("moment", ctypes.c_double), ("axis", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class petgem_solve_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("precision", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_iters", ctypes.c_int64), ("orth", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("method", ctypes.c_int32), ("spmv_lanes", ctypes.c_int32), ("omega", ctypes.c_double)]


class petgem_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int64), ("refinements", ctypes.c_int64),
                ("true_rel_residual", ctypes.c_double), ("status", ctypes.c_int32), ("reorth", ctypes.c_int32),
                ("fell_back", ctypes.c_int32), ("spmv_lanes", ctypes.c_int32)]


_P, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_SIGNATURES = {
    "petgem_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "petgem_destroy": (ctypes.c_int, [_P]),
    "petgem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "petgem_last_error": (ctypes.c_char_p, [_P]),
    "petgem_mesh_edges": (ctypes.c_int, [_P, _I64, _P, _I64, _P, ctypes.POINTER(_I64)]),
    "petgem_get_topology": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "petgem_assemble": (ctypes.c_int, [_P, _D, _P, _D, _I32, ctypes.POINTER(petgem_dipole)]),
    "petgem_assemble_frequency": (ctypes.c_int, [_P, _D, _I32, ctypes.POINTER(petgem_dipole)]),
    "petgem_get_system": (ctypes.c_int, [_P, ctypes.POINTER(_I64), _P, _P, _P, _P, _P]),
    "petgem_get_elements": (ctypes.c_int, [_P, _P, _P, _P]),
    "petgem_solve": (ctypes.c_int, [_P, ctypes.POINTER(petgem_solve_opts), _P, ctypes.POINTER(petgem_solve_info)]),
    "petgem_solve_batch": (ctypes.c_int, [ctypes.POINTER(_P), _I32, ctypes.POINTER(petgem_solve_opts),
                                          ctypes.POINTER(_P), ctypes.POINTER(petgem_solve_info)]),
    "petgem_spmv": (ctypes.c_int, [_P, _P, _P]),
    "petgem_colouring": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "petgem_ssor_apply": (ctypes.c_int, [_P, _D, _P, _P]),
    "petgem_receivers": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "petgem_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "petgem_kernel_stats": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(_I64), ctypes.POINTER(_D),
                                           ctypes.POINTER(_D)]),
    "petgem_launch_count": (_I64, [_P]),
    "petgem_learned_create": (ctypes.c_int, [_P, _I32, _I32, _I32]),
    "petgem_learned_params": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(_I64)]),
    "petgem_learned_train_step": (ctypes.c_int, [_P, _I32, _P, ctypes.c_float, ctypes.POINTER(_D)]),
    "petgem_learned_apply": (ctypes.c_int, [_P, _P, _P]),
    "petgem_nn_conv3d": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _P, _P, _P, _I32, _P, _I32]),
    "petgem_nn_conv3d_wgrad": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _P, _P, _P]),
    "petgem_nn_conv3d_wgrad_noalloc": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _P, _P, _P]),
    "petgem_primary_layered": (ctypes.c_int, [_P, _I32, _P, _P, _D, ctypes.POINTER(petgem_dipole), _I32, _P, _P]),
    "petgem_assemble_layered": (ctypes.c_int, [_P, _D, _P, _I32, _P, _P, _I32, ctypes.POINTER(petgem_dipole)]),
}

_lib = None


def header_functions() -> list:
    """Names of the functions include/petgem.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*\*?\s*(petgem_\w+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH):
    """Load libpetgem.so (built by paper_1808_00186_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libpetgem.so is not built (run __graft_entry__.build()); no fallback exists")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PetgemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (load().petgem_status_string(status).decode(), status, msg))
        self.status = status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous CUDA tensor")
        return t.data_ptr()
    raise TypeError("expected a torch CUDA tensor")


# ------------------------------------------------------------------ same-name wrappers
def petgem_create(device: int = 0, stream=None):
    h = _P()
    st = load().petgem_create(ctypes.byref(h), device, stream)
    if st != OK:
        raise PetgemError(st, "petgem_create failed")
    return h


def petgem_destroy(ctx) -> int:
    return load().petgem_destroy(ctx)


def _check(ctx, st, allowed=(OK,)):
    if st not in allowed:
        raise PetgemError(st, load().petgem_last_error(ctx).decode())
    return st


def petgem_mesh_edges(ctx, nodes, tets) -> int:
    n = _I64(0)
    _check(ctx, load().petgem_mesh_edges(ctx, nodes.shape[0], _ptr(nodes), tets.shape[0], _ptr(tets), ctypes.byref(n)))
    return n.value


def petgem_get_topology(ctx, edges=None, tet_edges=None, signs=None, boundary=None):
    _check(ctx, load().petgem_get_topology(ctx, _ptr(edges), _ptr(tet_edges), _ptr(signs), _ptr(boundary)))


def dipoles(sources) -> ctypes.Array:
    arr = (petgem_dipole * len(sources))()
    for i, s in enumerate(sources):
        arr[i] = petgem_dipole(s.x, s.y, s.z, s.moment, s.axis, 0)
    return arr


def petgem_assemble(ctx, freq, sigma, sigma_p, sources):
    arr = dipoles(sources)
    _check(ctx, load().petgem_assemble(ctx, float(freq), _ptr(sigma), float(sigma_p), len(sources), arr))


def petgem_assemble_frequency(ctx, freq, sources):
    arr = dipoles(sources)
    _check(ctx, load().petgem_assemble_frequency(ctx, float(freq), len(sources), arr))


def petgem_get_system(ctx, row_ptr=None, col=None, val=None, b=None, diag=None) -> int:
    nnz = _I64(0)
    _check(ctx, load().petgem_get_system(ctx, ctypes.byref(nnz), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b),
                                         _ptr(diag)))
    return nnz.value


def petgem_get_elements(ctx, K21=None, M21=None, vol=None):
    _check(ctx, load().petgem_get_elements(ctx, _ptr(K21), _ptr(M21), _ptr(vol)))


def solve_opts(restart=50, precision=PREC_C128, tol=1e-8, inner_tol=1e-4, max_iters=200000, batch=1,
               orth=ORTH_CGS, use_graphs=0, precond=PRECOND_JACOBI, method=METHOD_GMRES,
               spmv_lanes=0, omega=0.0) -> petgem_solve_opts:
    return petgem_solve_opts(restart, precision, precond, batch, tol, inner_tol, max_iters, orth, use_graphs, method,
                             spmv_lanes, omega)


def petgem_solve(ctx, x, n_src, opts=None, allow_not_converged=False):
    info = (petgem_solve_info * n_src)()
    o = opts if opts is not None else solve_opts()
    allowed = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
    st = _check(ctx, load().petgem_solve(ctx, ctypes.byref(o), _ptr(x), info), allowed)
    return st, _info_dicts(info)


def _info_dicts(info):
    return [dict(iters=i.iters, restarts=i.restarts, refinements=i.refinements,
                 true_rel_residual=i.true_rel_residual, status=i.status, reorth=i.reorth,
                 fell_back=i.fell_back, spmv_lanes=i.spmv_lanes) for i in info]


def petgem_solve_batch(ctxs, xs, n_srcs, opts=None, allow_not_converged=False):
    """Solve the systems of several contexts together (COCG); xs[k] is context k's solution tensor."""
    n = len(ctxs)
    arr = (_P * max(n, 1))(*[c for c in ctxs])
    xarr = (_P * max(n, 1))(*[_ptr(x) for x in xs])
    info = (petgem_solve_info * max(sum(n_srcs), 1))()
    o = opts if opts is not None else solve_opts(method=METHOD_COCG)
    allowed = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
    st = load().petgem_solve_batch(arr, n, ctypes.byref(o), xarr, info)
    if st not in allowed:
        raise PetgemError(st, load().petgem_last_error(ctxs[0]).decode() if n else "")
    return st, _info_dicts(info)[:sum(n_srcs)]


def petgem_spmv(ctx, x, y):
    _check(ctx, load().petgem_spmv(ctx, _ptr(x), _ptr(y)))


def petgem_colouring(ctx, colour=None):
    """Returns (number of colours, rounds); colour: optional device int32[E] tensor to fill."""
    nc, nr = _I32(0), _I32(0)
    _check(ctx, load().petgem_colouring(ctx, _ptr(colour), ctypes.byref(nc), ctypes.byref(nr)))
    return nc.value, nr.value


def petgem_ssor_apply(ctx, omega, r, z):
    _check(ctx, load().petgem_ssor_apply(ctx, omega, _ptr(r), _ptr(z)))


def petgem_receivers(ctx, rx, x, out, allow_outside=False) -> int:
    allowed = (OK, ERR_RECEIVER_OUTSIDE) if allow_outside else (OK,)
    return _check(ctx, load().petgem_receivers(ctx, rx.shape[0], _ptr(rx), _ptr(x), _ptr(out)), allowed)


def petgem_profile(ctx, enable: bool):
    _check(ctx, load().petgem_profile(ctx, 1 if enable else 0))


def petgem_kernel_stats(ctx, name: str):
    n, ms, by = _I64(0), _D(0.0), _D(0.0)
    _check(ctx, load().petgem_kernel_stats(ctx, name.encode(), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return n.value, ms.value, by.value


def petgem_learned_create(ctx, nx, ny, nz):
    _check(ctx, load().petgem_learned_create(ctx, nx, ny, nz))


def petgem_learned_params(ctx, set_params=None, get=False, grad=False):
    """Set (host float32 array) and/or get the network parameters (and the last mean gradient).
    Returns the parameter count, or the requested arrays."""
    n = _I64(0)
    _check(ctx, load().petgem_learned_params(ctx, None, None, None, ctypes.byref(n)))
    src = None
    if set_params is not None:
        src = np.ascontiguousarray(set_params, dtype=np.float32)
        if src.size != n.value:
            raise ValueError("expected %d parameters" % n.value)
    out = np.zeros(n.value, np.float32) if get else None
    gout = np.zeros(n.value, np.float32) if grad else None
    _check(ctx, load().petgem_learned_params(ctx, None if src is None else src.ctypes.data,
                                             None if out is None else out.ctypes.data,
                                             None if gout is None else gout.ctypes.data, ctypes.byref(n)))
    if get and grad:
        return out, gout
    if get:
        return out
    if grad:
        return gout
    return n.value


def petgem_learned_train_step(ctx, x_iters, lr) -> float:
    loss = _D(0.0)
    _check(ctx, load().petgem_learned_train_step(ctx, x_iters.shape[0], _ptr(x_iters), ctypes.c_float(lr),
                                                  ctypes.byref(loss)))
    return loss.value


def petgem_learned_apply(ctx, r, z):
    _check(ctx, load().petgem_learned_apply(ctx, _ptr(r), _ptr(z)))


def petgem_nn_conv3d(stream, grid, cin, cout, x, w, bias, relu, y, y_fp32):
    st = load().petgem_nn_conv3d(stream, grid[0], grid[1], grid[2], cin, cout, _ptr(x), _ptr(w), _ptr(bias),
                                 1 if relu else 0, _ptr(y), 1 if y_fp32 else 0)
    if st != OK:
        raise PetgemError(st, "petgem_nn_conv3d")


def petgem_nn_conv3d_wgrad(stream, grid, cin, cout, x, dy, dw):
    st = load().petgem_nn_conv3d_wgrad(stream, grid[0], grid[1], grid[2], cin, cout, _ptr(x), _ptr(dy), _ptr(dw))
    if st != OK:
        raise PetgemError(st, "petgem_nn_conv3d_wgrad")


# Largest grid (voxels) petgem_nn_conv3d_wgrad_noalloc accepts: the size of its fixed scratch.
NOALLOC_MAX_VOXELS = 131072


def petgem_nn_conv3d_wgrad_noalloc(stream, grid, cin, cout, x, dy, dw):
    """petgem_nn_conv3d_wgrad without any device allocation (fixed library scratch; calls on one
    device must not overlap in time)."""
    st = load().petgem_nn_conv3d_wgrad_noalloc(stream, grid[0], grid[1], grid[2], cin, cout, _ptr(x), _ptr(dy),
                                               _ptr(dw))
    if st != OK:
        raise PetgemError(st, "petgem_nn_conv3d_wgrad_noalloc")


def petgem_primary_layered(stream, z_interfaces, sigma_layers, freq, src, pts, out):
    """Primary field of a horizontal dipole in a layered Earth at device points pts [n, 3] into the
    device complex128 tensor out [n, 3] (enqueued on stream).  z_interfaces decreasing (host
    sequence), sigma_layers one longer; src: a synth.Dipole-like object."""
    zi = np.ascontiguousarray(z_interfaces, dtype=np.float64)
    sg = np.ascontiguousarray(sigma_layers, dtype=np.float64)
    d = petgem_dipole(src.x, src.y, src.z, src.moment, src.axis, 0)
    n = 0 if pts is None else int(pts.shape[0])
    st = load().petgem_primary_layered(stream, len(sg), zi.ctypes.data_as(_P) if zi.size else None,
                                       sg.ctypes.data_as(_P), freq, ctypes.byref(d), n, _ptr(pts), _ptr(out))
    if st != OK:
        raise PetgemError(st, "petgem_primary_layered")


def petgem_assemble_layered(ctx, freq, sigma, z_interfaces, sigma_layers, sources):
    """Assembly with a layered background (host sequences z_interfaces, sigma_layers)."""
    zi = np.ascontiguousarray(z_interfaces, dtype=np.float64)
    sg = np.ascontiguousarray(sigma_layers, dtype=np.float64)
    arr = dipoles(sources)
    _check(ctx, load().petgem_assemble_layered(ctx, freq, _ptr(sigma), len(sg), zi.ctypes.data_as(_P) if zi.size else None,
                                               sg.ctypes.data_as(_P), len(sources), arr))


def petgem_launch_count(ctx) -> int:
    return load().petgem_launch_count(ctx)


# ------------------------------------------------------------------ convenience
@dataclass
class Forward:
    """Device-resident results of one forward run (see run_forward)."""
    n_edges: int
    x: object          # complex128 [n_src, E]
    rcv: object        # complex128 [n_src, n_rcv, 3, 3]
    info: list
    status: int


def solve_batch(contexts, xs=None, **opts):
    """petgem_solve_batch over Context objects (COCG); returns (xs, info, status)."""
    import torch
    if xs is None:
        xs = [torch.zeros((c.n_src, c.n_edges), dtype=torch.complex128, device=c.nodes.device) for c in contexts]
    allow = opts.pop("allow_not_converged", False)
    opts.setdefault("method", METHOD_COCG)
    st, info = petgem_solve_batch([c.h for c in contexts], xs, [c.n_src for c in contexts], solve_opts(**opts),
                                  allow_not_converged=allow)
    return xs, info, st


class Context:
    """Owns a petgem context on the current torch CUDA device and stream."""

    def __init__(self, device=None, stream=None):
        import torch
        self.torch = torch
        dev = torch.cuda.current_device() if device is None else device
        st = torch.cuda.current_stream(dev) if stream is None else stream
        self.device = dev
        self.stream = st
        self.h = petgem_create(dev, ctypes.c_void_p(st.cuda_stream))

    def close(self):
        if getattr(self, "h", None):
            petgem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def tensor(self, a, dtype=None):
        t = self.torch.as_tensor(np.ascontiguousarray(a), device="cuda:%d" % self.device)
        return t if dtype is None else t.to(dtype)

    def mesh(self, nodes, tets) -> int:
        self.nodes = nodes if hasattr(nodes, "data_ptr") else self.tensor(nodes, self.torch.float64)
        self.tets = tets if hasattr(tets, "data_ptr") else self.tensor(tets, self.torch.int32)
        self.n_edges = petgem_mesh_edges(self.h, self.nodes, self.tets)
        return self.n_edges

    def topology(self):
        T, E = self.tets.shape[0], self.n_edges
        tt = self.torch
        out = (tt.empty((E, 2), dtype=tt.int32, device=self.nodes.device),
               tt.empty((T, 6), dtype=tt.int32, device=self.nodes.device),
               tt.empty((T, 6), dtype=tt.int8, device=self.nodes.device),
               tt.empty(E, dtype=tt.uint8, device=self.nodes.device))
        petgem_get_topology(self.h, *out)
        return out

    def assemble(self, freq, sigma, sigma_p, sources):
        self.sigma = sigma if hasattr(sigma, "data_ptr") else self.tensor(sigma, self.torch.float64)
        self.n_src = len(sources)
        petgem_assemble(self.h, freq, self.sigma, sigma_p, sources)

    def assemble_layered(self, freq, sigma, z_interfaces, sigma_layers, sources):
        self.sigma = sigma if hasattr(sigma, "data_ptr") else self.tensor(sigma, self.torch.float64)
        self.n_src = len(sources)
        petgem_assemble_layered(self.h, freq, self.sigma, z_interfaces, sigma_layers, sources)

    def assemble_frequency(self, freq, sources):
        self.n_src = len(sources)
        petgem_assemble_frequency(self.h, freq, sources)

    def system(self):
        tt = self.torch
        E = self.n_edges
        nnz = petgem_get_system(self.h)
        d = self.nodes.device
        rp = tt.empty(E + 1, dtype=tt.int64, device=d)
        col = tt.empty(nnz, dtype=tt.int32, device=d)
        val = tt.empty(nnz, dtype=tt.complex128, device=d)
        b = tt.empty((self.n_src, E), dtype=tt.complex128, device=d)
        dg = tt.empty(E, dtype=tt.complex128, device=d)
        petgem_get_system(self.h, rp, col, val, b, dg)
        return rp, col, val, b, dg

    def elements(self):
        tt = self.torch
        T = self.tets.shape[0]
        K = tt.empty((21, T), dtype=tt.float64, device=self.nodes.device)
        M = tt.empty((21, T), dtype=tt.float64, device=self.nodes.device)
        v = tt.empty(T, dtype=tt.float64, device=self.nodes.device)
        petgem_get_elements(self.h, K, M, v)
        return K, M, v

    def solve(self, x=None, **opts):
        tt = self.torch
        if x is None:
            x = tt.zeros((self.n_src, self.n_edges), dtype=tt.complex128, device=self.nodes.device)
        allow = opts.pop("allow_not_converged", False)
        st, info = petgem_solve(self.h, x, self.n_src, solve_opts(**opts), allow_not_converged=allow)
        return x, info, st

    def colouring(self):
        """(colour int32[E] device tensor, number of colours, rounds) of the SSOR ordering."""
        tt = self.torch
        colour = tt.empty(self.n_edges, dtype=tt.int32, device=self.nodes.device)
        nc, nr = petgem_colouring(self.h, colour)
        return colour, nc, nr

    def ssor_apply(self, r, omega=1.0):
        """z = M^{-1} r for the SSOR preconditioner (r: device complex128[E])."""
        z = self.torch.empty_like(r)
        petgem_ssor_apply(self.h, omega, r, z)
        return z

    def receivers(self, rx, x, allow_outside=False):
        tt = self.torch
        rxt = rx if hasattr(rx, "data_ptr") else self.tensor(rx, tt.float64)
        out = tt.empty((self.n_src, rxt.shape[0], 3, 3), dtype=tt.complex128, device=self.nodes.device)
        st = petgem_receivers(self.h, rxt, x, out, allow_outside=allow_outside)
        return out, st
