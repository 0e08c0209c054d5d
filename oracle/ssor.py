"""FP64 CPU oracle of the multicolour symmetric SOR preconditioner of the SQMR solver (the
paper's Section 5.3 solves its adapted meshes with SQMR preconditioned by SOR).

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU legs may use it; the CUDA library never does.

Reading of the paper: it names SOR without a relaxation factor or sweep type.  SQMR needs a
complex-symmetric preconditioner, so the sweep is the symmetric one (a forward then a backward
Gauss-Seidel sweep, SSOR), with omega = 1 unless given (symmetric Gauss-Seidel).  A sequential
sweep has no parallelism, so the rows are ordered by a colouring of the matrix graph: rows of one
colour share no entry, the sweep takes the colours in order and the rows of a colour at once.

Colouring (Jones and Plassmann, SIAM J. Sci. Comput. 14, 1993): every row i gets the priority
key (splitmix64(i), i), compared lexicographically; splitmix64 is the output function of
Steele, Lea and Flood's SplitMix64 generator (OOPSLA 2014) for the state i.  In each round, every
uncoloured row whose key exceeds the keys of all its uncoloured neighbours takes the smallest
colour that none of its already coloured neighbours holds.  Neighbours are the off-diagonal
entries of the CSR pattern (explicit zeros included).

SSOR (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Section 10.2): with A = D + L
+ U split in the colour order (L: entries a_ij whose column has a lower colour than the row, U:
a higher one; rows of one colour share no entry, so nothing else is off the diagonal),
    M = (D + omega L) D^{-1} (D + omega U),
complex symmetric because U = L^T.  SQMR uses it split as M = M1 M2 with M1 = (D + omega L)
D^{-1/2} and M2 = M1^T:  M1^{-1} v = D^{1/2} F v,  M2^{-1} t = B D^{1/2} t, where F = (D + omega
L)^{-1} is the forward sweep and B = (D + omega U)^{-1} the backward one (so that
M2^{-1} M1^{-1} r = B D F r = M^{-1} r; D^{1/2} is the principal root).  omega = 0 gives M = D,
the Jacobi preconditioner.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state) -> np.ndarray:
    """The generator's output for state s: z = s + gamma, then the two xor-shift-multiply rounds
    and a final xor-shift, all modulo 2^64 (numpy's uint64 arithmetic wraps)."""
    z = np.asarray(state, dtype=np.uint64) + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def priority_rank(n: int) -> np.ndarray:
    """rank[i] = position of row i when the rows are sorted by (splitmix64(i), i)."""
    idx = np.arange(n, dtype=np.int64)
    order = np.lexsort((idx, splitmix64(idx.astype(np.uint64))))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = idx
    return rank


def jp_colouring(indptr, indices):
    """Returns (colour int32[n], rounds) of the Jones-Plassmann colouring described above."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    n = len(indptr) - 1
    rank = priority_rank(n)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    off = rows != indices
    rows, cols = rows[off], indices[off]
    colour = np.full(n, -1, dtype=np.int64)
    rounds = 0
    while (colour < 0).any():
        uncoloured = colour < 0
        # a row waits while an uncoloured neighbour has a higher key
        waits = np.zeros(n, dtype=bool)
        m = uncoloured[rows] & uncoloured[cols] & (rank[cols] > rank[rows])
        waits[rows[m]] = True
        chosen = uncoloured & ~waits
        # colours held by the chosen rows' neighbours, coloured in earlier rounds
        used = np.zeros(n, dtype=np.uint64)
        m = chosen[rows] & (colour[cols] >= 0)
        if (colour[cols[m]] >= 64).any():
            raise ValueError("more than 64 colours")
        np.bitwise_or.at(used, rows[m], np.left_shift(np.uint64(1), colour[cols[m]].astype(np.uint64)))
        free = ~used[chosen] & (used[chosen] + np.uint64(1))  # lowest clear bit
        colour[chosen] = np.log2(free.astype(np.float64)).astype(np.int64)
        rounds += 1
    return colour.astype(np.int32), rounds


class SSOR:
    """M = (D + omega L) D^{-1} (D + omega U) in the colour order of `colours` (any int array whose
    equal entries mark rows that share no entry of A)."""

    def __init__(self, A, colours, omega: float = 1.0):
        A = sp.csr_matrix(A, dtype=np.complex128)
        self.n = A.shape[0]
        self.omega = float(omega)
        self.colours = np.asarray(colours, dtype=np.int64)
        self.d = np.asarray(A.diagonal(), dtype=np.complex128)
        C = A.tocoo()
        cr, cc = self.colours[C.row], self.colours[C.col]
        if ((cr == cc) & (C.row != C.col)).any():
            raise ValueError("two rows of one colour share an entry")
        lo, hi = cc < cr, cc > cr
        self.L = sp.csr_matrix((C.data[lo], (C.row[lo], C.col[lo])), shape=A.shape)
        self.U = sp.csr_matrix((C.data[hi], (C.row[hi], C.col[hi])), shape=A.shape)
        self.order = [np.flatnonzero(self.colours == k) for k in np.unique(self.colours)]

    def forward(self, v):
        """F v = (D + omega L)^{-1} v: colours ascending; a colour's rows read only lower colours."""
        v = np.asarray(v, dtype=np.complex128)
        y = np.zeros(self.n, dtype=np.complex128)
        for rows in self.order:
            y[rows] = (v[rows] - self.omega * (self.L[rows] @ y)) / self.d[rows]
        return y

    def backward(self, w):
        """B w = (D + omega U)^{-1} w: colours descending."""
        w = np.asarray(w, dtype=np.complex128)
        z = np.zeros(self.n, dtype=np.complex128)
        for rows in reversed(self.order):
            z[rows] = (w[rows] - self.omega * (self.U[rows] @ z)) / self.d[rows]
        return z

    def minv(self, r):
        """M^{-1} r = B D F r."""
        return self.backward(self.d * self.forward(r))

    def m1inv(self, v):
        """M1^{-1} v = D^{1/2} F v."""
        return np.sqrt(self.d) * self.forward(v)

    def m2inv(self, t):
        """M2^{-1} t = B D^{1/2} t."""
        return self.backward(np.sqrt(self.d) * t)
