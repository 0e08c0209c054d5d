"""CPU oracle (FP64, C++17) for the secondary-field CSEM forward problem.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
reference legs may import this package.  It shares no code with the CUDA library in
paper_1808_00186_gb300/ and the library never calls it.

build() compiles oracle.cpp with g++ into liboracle.so beside it; the wrappers below marshal
numpy arrays through ctypes.  Every wrapper names the part of the paper it follows in
oracle.cpp.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

OK, BAD_INPUT, DEGENERATE, NOT_CONVERGED, OUTSIDE, SINGULAR = range(6)

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "orc_element": (I, [P, P, P, P, P]),
            "orc_geometry": (I, [P, P, P, P, P]),
            "orc_primary_field": (I, [I64, P, P, D, D, P]),
            "orc_quadrature": (I, [P]),
            "orc_build": (P, [I64, P, I64, P, P, D, D, I64, P, P, ctypes.POINTER(I)]),
            "orc_topology": (P, [I64, I64, P, ctypes.POINTER(I)]),
            "orc_free": (None, [P]),
            "orc_sizes": (I, [P, P]),
            "orc_get_topology": (I, [P, P, P, P, P]),
            "orc_get_system": (I, [P, P, P, P, P]),
            "orc_solve": (I, [P, I, D, I64, P, P]),
            "orc_spmv": (I, [P, P, P]),
            "orc_receivers": (I, [P, P, I64, P, P]),
            "orc_dense_solve": (I, [I64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def element(p: np.ndarray, signs: np.ndarray):
    """K^e, M^e (6x6) and volume of one tet (Appendix B eqs. B.14-B.15)."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(4, 3)
    s = np.ascontiguousarray(signs, dtype=np.int8).reshape(6)
    K = np.zeros((6, 6))
    M = np.zeros((6, 6))
    v = np.zeros(1)
    st = lib().orc_element(_p(p), _p(s), _p(K), _p(M), _p(v))
    if st != OK:
        raise ValueError("orc_element status %d" % st)
    return K, M, float(v[0])


def geometry(p: np.ndarray):
    """Barycentric constants c0[4], gradients [4][3], edge lengths [6], volume of one tet."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(4, 3)
    c0, g, ln, v = np.zeros(4), np.zeros((4, 3)), np.zeros(6), np.zeros(1)
    st = lib().orc_geometry(_p(p), _p(c0), _p(g), _p(ln), _p(v))
    if st != OK:
        raise ValueError("orc_geometry status %d" % st)
    return c0, g, ln, float(v[0])


def primary_field(pts: np.ndarray, src, sigma_p: float, freq: float) -> np.ndarray:
    """Whole-space dipole field (Appendix A) at pts [n, 3]; src = (x, y, z, axis, moment)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(src, dtype=np.float64).reshape(5)
    out = np.zeros((pts.shape[0], 3), dtype=np.complex128)
    lib().orc_primary_field(pts.shape[0], _p(pts), _p(s), sigma_p, freq, _p(out))
    return out


def quadrature() -> np.ndarray:
    q = np.zeros((4, 4))
    lib().orc_quadrature(_p(q))
    return q


class System:
    """Assembled forward problem (edges, boundary, CSR with Dirichlet rows, right-hand sides)."""

    def __init__(self, nodes, tets, sigma=None, sigma_p=1.0, freq=1.0, sources=None, g=None,
                 topology_only=False):
        self.nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        st = ctypes.c_int(0)
        if topology_only:
            h = lib().orc_topology(self.nodes.shape[0], self.tets.shape[0], _p(self.tets), ctypes.byref(st))
        else:
            self.sigma = np.ascontiguousarray(sigma, dtype=np.float64)
            self.src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 5)
            gg = None if g is None else np.ascontiguousarray(g, dtype=np.complex128)
            h = lib().orc_build(self.nodes.shape[0], _p(self.nodes), self.tets.shape[0], _p(self.tets),
                                _p(self.sigma), sigma_p, freq, self.src.shape[0], _p(self.src),
                                _p(gg), ctypes.byref(st))
        if not h:
            raise ValueError("oracle build failed with status %d" % st.value)
        self.h = h
        sizes = np.zeros(3, dtype=np.int64)
        lib().orc_sizes(h, _p(sizes))
        self.n_edges, self.nnz, self.n_src = (int(v) for v in sizes)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    def topology(self):
        E, T = self.n_edges, self.tets.shape[0]
        edges = np.zeros((E, 2), np.int32)
        te = np.zeros((T, 6), np.int32)
        sg = np.zeros((T, 6), np.int8)
        bd = np.zeros(E, np.uint8)
        lib().orc_get_topology(self.h, _p(edges), _p(te), _p(sg), _p(bd))
        return edges, te, sg, bd

    def system(self):
        E = self.n_edges
        rp = np.zeros(E + 1, np.int64)
        col = np.zeros(self.nnz, np.int32)
        val = np.zeros(self.nnz, np.complex128)
        b = np.zeros((self.n_src, E), np.complex128)
        lib().orc_get_system(self.h, _p(rp), _p(col), _p(val), _p(b))
        return rp, col, val, b

    def solve(self, restart=50, tol=1e-8, maxit=100000, x0=None):
        x = np.zeros((self.n_src, self.n_edges), np.complex128) if x0 is None else \
            np.ascontiguousarray(x0, dtype=np.complex128).copy()
        info = np.zeros((self.n_src, 3))
        st = lib().orc_solve(self.h, restart, tol, maxit, _p(x), _p(info))
        return x, info, st

    def spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros(self.n_edges, np.complex128)
        lib().orc_spmv(self.h, _p(x), _p(y))
        return y

    def receivers(self, x, rx):
        x = np.ascontiguousarray(x, dtype=np.complex128).reshape(self.n_src, self.n_edges)
        rx = np.ascontiguousarray(rx, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((self.n_src, rx.shape[0], 3, 3), np.complex128)
        st = lib().orc_receivers(self.h, _p(x), rx.shape[0], _p(rx), _p(out))
        return out, st


def dense_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros(b.shape[0], np.complex128)
    st = lib().orc_dense_solve(A.shape[0], _p(A), _p(b), _p(x))
    if st != OK:
        raise ValueError("orc_dense_solve status %d" % st)
    return x
