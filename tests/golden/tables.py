"""Readers for the small text fixtures in this folder (each file states its citation)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def local_edge_table() -> np.ndarray:
    """[6, 2] zero-based (a, b) node pairs of W_ab (Appendix B eqs. B.1-B.6)."""
    rows = [list(map(int, l.split())) for l in open(os.path.join(HERE, "local_edge_table.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array([[r[1] - 1, r[2] - 1] for r in rows], dtype=np.int64)
