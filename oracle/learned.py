"""FP64 CPU oracle of the learned preconditioner's network and of its grid maps.

TEST INFRASTRUCTURE (like the rest of oracle/): used only by tests/ and the benchmark's CPU
legs.  The paper has no learned part; what this file fixes is the design the CUDA library
implements, written plainly so that its kernels can be checked element by element, and pinned
by finite differences (tests/test_oracle_learned.py).

Conventions shared with the CUDA kernels (by definition, not by code):
  * grid tensors are numpy arrays [Z, Y, X, C], so the flat voxel index is v = x + X (y + Y z)
    (the node numbering of the Kuhn lattice) with the channels innermost;
  * a 3x3x3 convolution with zero "same" padding has weights W[t][co][ci], tap
    t = (dx + 1) + 3 (dy + 1) + 9 (dz + 1), and bias b[co]:
        y[v][co] = b[co] + sum_t sum_ci W[t][co][ci] x[v + (dx, dy, dz)][ci];
  * pooling averages the (up to 8) fine voxels 2 c + {0, 1} of a coarse voxel c that exist
    (coarse size ceil(G / 2)); upsampling copies a coarse voxel to its fine children.
"""
from __future__ import annotations

import numpy as np

OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap order t


def shift(x: np.ndarray, d) -> np.ndarray:
    """x[v + d] for d = (dx, dy, dz), zeros outside the grid; x is [Z, Y, X, C]."""
    out = np.zeros_like(x)
    sl_dst, sl_src = [], []
    for a, n in zip((d[2], d[1], d[0]), x.shape[:3]):
        if a >= 0:
            sl_dst.append(slice(0, n - a))
            sl_src.append(slice(a, n))
        else:
            sl_dst.append(slice(-a, n))
            sl_src.append(slice(0, n + a))
    out[tuple(sl_dst)] = x[tuple(sl_src)]
    return out


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [Z,Y,X,Cin], W [27, Cout, Cin], b [Cout] -> [Z,Y,X,Cout]."""
    y = np.zeros(x.shape[:3] + (W.shape[1],)) + b
    for t, d in enumerate(OFFS):
        y += shift(x, d) @ W[t].T
    return y


def conv3d_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of sum(dy * conv3d(x, W, b)) w.r.t. x, W and b."""
    dx = np.zeros_like(x, dtype=np.float64)
    dW = np.zeros_like(W, dtype=np.float64)
    for t, d in enumerate(OFFS):
        xs = shift(x, d)
        dW[t] = np.einsum("zyxo,zyxi->oi", dy, xs)
        dx += shift(dy @ W[t], tuple(-a for a in d))
    db = dy.sum(axis=(0, 1, 2))
    return dx, dW, db


def pool(x: np.ndarray) -> np.ndarray:
    X, Y, Z, C = x.shape  # (axis sizes; the averaging is the same along every axis)
    cX, cY, cZ = (X + 1) // 2, (Y + 1) // 2, (Z + 1) // 2
    s = np.zeros((cX, cY, cZ, C))
    n = np.zeros((cX, cY, cZ, 1))
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                part = x[ox::2, oy::2, oz::2]
                s[:part.shape[0], :part.shape[1], :part.shape[2]] += part
                n[:part.shape[0], :part.shape[1], :part.shape[2]] += 1
    return s / n


def pool_backward(dy: np.ndarray, fine_shape) -> np.ndarray:
    X, Y, Z, C = fine_shape
    cX, cY, cZ = dy.shape[:3]
    n = np.zeros((cX, cY, cZ, 1))
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                n[:len(range(ox, X, 2)), :len(range(oy, Y, 2)), :len(range(oz, Z, 2))] += 1
    g = dy / n
    dx = np.zeros(fine_shape)
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                tgt = dx[ox::2, oy::2, oz::2]
                tgt += g[:tgt.shape[0], :tgt.shape[1], :tgt.shape[2]]
    return dx


def upsample(x: np.ndarray, fine_shape) -> np.ndarray:
    X, Y, Z = fine_shape[:3]
    out = np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)
    return out[:X, :Y, :Z]


def upsample_backward(dy: np.ndarray, coarse_shape) -> np.ndarray:
    dx = np.zeros(coarse_shape)
    X, Y, Z = dy.shape[:3]
    for ox in (0, 1):
        for oy in (0, 1):
            for oz in (0, 1):
                part = dy[ox::2, oy::2, oz::2]
                dx[:part.shape[0], :part.shape[1], :part.shape[2]] += part
    return dx


# ---------------------------------------------------------------- the network
# name: (in channels, out channels, relu).  Level 0 is the node grid, level l + 1 the pooling of
# level l; the number of levels grows with the grid (levels()): poolings continue until the
# coarsest grid has at most 3 nodes along every axis (at least 3 levels), so the coarsest level
# spans the whole domain at every resolution.  c1 / c7 act on level 0, c2 / c6 on level 1, c4 on
# the coarsest level, and c3 / c5 on every level in between (weights shared between those
# levels, as a multigrid cycle uses one smoother on every level).  Decoder levels add the
# upsampled coarse features to the encoder's.
LAYERS = [("c1", 16, 16, True), ("c2", 16, 32, True), ("c3", 32, 32, True), ("c4", 32, 32, True),
          ("c5", 32, 32, True), ("c6", 32, 16, True), ("c7", 16, 16, False)]
N_IN, N_OUT = 16, 14


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through float32, returned as float64: the
    storage format of the network's activations, gradients and weights on the GPU."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def levels(shape) -> int:
    """Number of levels for a grid of `shape` nodes (any axis order)."""
    dims, L = list(shape[:3]), 1
    while max(dims) > 3:
        dims = [(d + 1) // 2 for d in dims]
        L += 1
    return max(3, L)


def init_params(seed: int = 0, scale: float = 1.0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co, _ in LAYERS:
        std = scale * np.sqrt(2.0 / (27 * ci))
        p[name + ".W"] = rng.normal(size=(27, co, ci)) * std
        p[name + ".b"] = rng.normal(size=co) * 0.01
    p["c7.W"][:, N_OUT:, :] = 0.0   # output channels 14, 15 are padding
    p["c7.b"][N_OUT:] = 0.0
    return p


def forward(p: dict, x: np.ndarray, round_bf16: bool = False):
    """x [Z,Y,X,16] -> (y [Z,Y,X,16], cache).  With round_bf16 the weights and every stored
    activation (encoder inputs and outputs, decoder inputs and hidden outputs) are rounded to
    bfloat16 where the GPU kernels store them; arithmetic stays FP64."""
    relu = lambda a: np.maximum(a, 0.0)
    rnd = bf16 if round_bf16 else (lambda a: a)
    L = levels(x.shape)
    conv = lambda name, a: conv3d(a, rnd(p[name + ".W"]), p[name + ".b"])
    enc_name = lambda l: "c1" if l == 0 else "c2" if l == 1 else "c4" if l == L - 1 else "c3"
    dec_name = lambda l: "c7" if l == 0 else "c6" if l == 1 else "c5"
    q, e = {0: rnd(x)}, {}
    for l in range(L):
        if l > 0:
            q[l] = rnd(pool(e[l - 1]))
        e[l] = rnd(relu(conv(enc_name(l), q[l])))
    d, sk = {L - 1: e[L - 1]}, {}
    for l in range(L - 2, -1, -1):
        sk[l] = rnd(upsample(d[l + 1], e[l].shape) + e[l])
        out = conv(dec_name(l), sk[l])
        d[l] = out if l == 0 else rnd(relu(out))
    return d[0], dict(L=L, q=q, e=e, d=d, s=sk, round_bf16=round_bf16)


def backward(p: dict, cache: dict, dy: np.ndarray) -> dict:
    """Gradients of sum(dy * forward(p, x)) with respect to every parameter (shared weights
    collect the gradients of every level they act on).  When the forward pass rounded to
    bfloat16, dy and every stored gradient tensor are rounded where the GPU stores them."""
    L, q, e, d, sk = cache["L"], cache["q"], cache["e"], cache["d"], cache["s"]
    rnd = bf16 if cache.get("round_bf16") else (lambda a: a)
    enc_name = lambda l: "c1" if l == 0 else "c2" if l == 1 else "c4" if l == L - 1 else "c3"
    dec_name = lambda l: "c7" if l == 0 else "c6" if l == 1 else "c5"
    g = {k: np.zeros_like(v) for k, v in p.items()}

    def conv_back(name, inp, dz):
        dx, dW, db = conv3d_backward(inp, rnd(p[name + ".W"]), dz)
        g[name + ".W"] += dW
        g[name + ".b"] += db
        return rnd(dx)

    de = {}
    dd = rnd(dy)                              # gradient at d[0] = y (no ReLU on the output)
    for l in range(0, L - 1):
        dz = dd if l == 0 else dd * (d[l] > 0)
        ds = conv_back(dec_name(l), sk[l], dz)
        de[l] = ds.copy()                     # skip path into e[l]
        dd = rnd(upsample_backward(ds, d[l + 1].shape))
    de[L - 1] = dd                            # d[L-1] = e[L-1]
    for l in range(L - 1, -1, -1):
        dz = de[l] * (e[l] > 0)
        dq = conv_back(enc_name(l), q[l], dz)
        if l > 0:
            de[l - 1] = rnd(de[l - 1] + pool_backward(dq, e[l - 1].shape))
    return g


def loss(p: dict, x: np.ndarray, target: np.ndarray):
    """Mean squared error over the 14 output channels: 0.5 * mean((y - t)^2); returns (L, dL/dy)."""
    y, cache = forward(p, x)
    diff = np.zeros_like(y)
    diff[..., :N_OUT] = y[..., :N_OUT] - target[..., :N_OUT]
    cnt = np.prod(y.shape[:3]) * N_OUT
    return 0.5 * float((diff ** 2).sum()) / cnt, diff / cnt, cache


# ---------------------------------------------------------------- edge <-> grid
# Edge classes of a Kuhn-split lattice, by the step from the edge's low node to its high node.
CLASSES = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def edge_grid_index(edges: np.ndarray, n: int) -> np.ndarray:
    """Grid slot (voxel * 7 + class) of every edge (low, high) of a Kuhn lattice with n cells a side
    and node id i + (n+1) (j + (n+1) k); -1 if the edge is not a lattice step."""
    s = n + 1
    lo, hi = edges[:, 0].astype(np.int64), edges[:, 1].astype(np.int64)
    li, lj, lk = lo % s, (lo // s) % s, lo // (s * s)
    hi_i, hi_j, hi_k = hi % s, (hi // s) % s, hi // (s * s)
    d = np.stack([hi_i - li, hi_j - lj, hi_k - lk], axis=1)
    out = np.full(edges.shape[0], -1, np.int64)
    for c, step in enumerate(CLASSES):
        m = np.all(d == np.array(step), axis=1)
        out[m] = lo[m] * 7 + c
    return out


# ---------------------------------------------------------------- residual-angle training loss
def edges_to_grid(v_edges: np.ndarray, slot: np.ndarray, n_nodes: int, scale: float = 1.0) -> np.ndarray:
    """[n_nodes, 16] grid with Re / Im of an edge vector on channels c / 7 + c of its slot."""
    g = np.zeros((n_nodes, 16))
    v, c = slot // 7, slot % 7
    g[v, c] = v_edges.real * scale
    g[v, 7 + c] = v_edges.imag * scale
    return g


def grid_to_edges(g: np.ndarray, slot: np.ndarray) -> np.ndarray:
    v, c = slot // 7, slot % 7
    return g[v, c] + 1j * g[v, 7 + c]


def angle_loss(y_grid: np.ndarray, r: np.ndarray, slot: np.ndarray, spmv, diag: np.ndarray):
    """L = 1 - |<r, Ahat z>|^2 / (|r|^2 |Ahat z|^2) for z = the network output on the edges and
    Ahat = A D^{-1} (A complex symmetric, so Ahat^H g = conj(D)^{-1} conj(A) g).  Returns
    (L, dL/dy on the grid): the gradient of the real loss with respect to Re y and Im y."""
    z = grid_to_edges(y_grid, slot)
    w = spmv(z / diag)
    a = np.vdot(r, w)
    b = np.vdot(w, w).real
    c = np.vdot(r, r).real
    L = 1.0 - abs(a) ** 2 / (b * c)
    gw = -2.0 * (a * r / (c * b) - abs(a) ** 2 * w / (c * b * b))      # dL/dRe w + i dL/dIm w
    gz = np.conj(spmv(np.conj(gw))) / np.conj(diag)                    # Ahat^H gw = conj(D)^-1 conj(A) gw
    gy = np.zeros_like(y_grid)
    v, cc = slot // 7, slot % 7
    gy[v, cc] = gz.real
    gy[v, 7 + cc] = gz.imag
    return L, gy


# ---------------------------------------------------------------- auxiliary-space preconditioner
# The network acts through the two auxiliary spaces of lowest-order edge elements (the
# Hiptmair-Xu decomposition): nodal gradients G phi, on which the curl-curl term vanishes, and
# nodal vector fields Pi w.  With phi and w on the lattice nodes,
#     z = D^{-1} r + G phi + Pi w,
# where phi, w are the nodal values of a scalar and a vector field, interpolated linearly, and
# phi, w are zero on nodes of the outer boundary (Dirichlet condition, Section 2).  With the
# exact auxiliary solutions phi = (G^T A G)^{-1} G^T r, w = (Pi^T A Pi)^{-1} Pi^T r this is the
# additive auxiliary-space preconditioner; the network approximates both solves.  The edge
# degrees of freedom of the basis of eqs. B.8-B.13 (scaled by the edge length) are tangential
# components, E . t_e / |t_e|, so both maps carry a factor 1 / |t_e|:
#     (G phi)_e = (phi_hi - phi_lo) / |t_e|,    (Pi w)_e = (w_lo + w_hi) . t_e / (2 |t_e|).
#
# Network input (grid [V, 16], V = lattice nodes): with sg = |diag(G^T A G)|^{-1/2},
# sp = |diag(Pi^T A Pi)|^{-1/2} (per node and component, zero on boundary nodes),
#     fg = sg * (G^T r),  fp = sp * (Pi^T r),
#     s  = sqrt((sum |fg|^2 + sum |fp|^2) / (4 n_interior))   (1 when r = 0),
#     channels 0, 1 = Re, Im fg / s;  2..4 = Re fp / s (x, y, z);  5..7 = Im fp / s;
#     8, 9 = the node features;  10..15 = 0.
# Network output y [V, 16]: phi = s sg (y0 + i y1), w_a = s sp_a (y_{2+a} + i y_{5+a}).
AUX_IN = 8


def _cells(n):
    return (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)


def interior_nodes(n) -> np.ndarray:
    """Nodes of a lattice of n = (nx, ny, nz) cells (or n^3) off the outer boundary: bool over the
    (nx+1)(ny+1)(nz+1) nodes, node i + (nx+1)(j + (ny+1) k)."""
    nx, ny, nz = _cells(n)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    inner = (i >= 1) & (i <= nx - 1) & (j >= 1) & (j <= ny - 1) & (k >= 1) & (k <= nz - 1)
    return inner.reshape(-1)


def aux_operators(edges: np.ndarray, nodes: np.ndarray, n):
    """(G [E x V], Pi [E x 3V]) as scipy CSR matrices for a lattice of n = (nx, ny, nz) cells (or
    n^3); columns of boundary nodes are empty."""
    import scipy.sparse as sp
    nx, ny, nz = _cells(n)
    E, V = edges.shape[0], (nx + 1) * (ny + 1) * (nz + 1)
    inner = interior_nodes(n)
    lo, hi = edges[:, 0].astype(np.int64), edges[:, 1].astype(np.int64)
    t = nodes[hi] - nodes[lo]
    ell = np.linalg.norm(t, axis=1)
    rows, cols, vals = [], [], []
    for end, sign in ((lo, -1.0), (hi, 1.0)):
        keep = inner[end]
        rows.append(np.nonzero(keep)[0])
        cols.append(end[keep])
        vals.append(sign / ell[keep])
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(E, V))
    rows, cols, vals = [], [], []
    for end in (lo, hi):
        keep = inner[end]
        for a in range(3):
            rows.append(np.nonzero(keep)[0])
            cols.append(3 * end[keep] + a)
            vals.append(0.5 * t[keep, a] / ell[keep])
    Pi = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(E, 3 * V))
    return G, Pi


def aux_scales(G, Pi, A):
    """sg [V] = |diag(G^T A G)|^{-1/2}, sp [V, 3] = |diag(Pi^T A Pi)|^{-1/2}; zero where the
    diagonal is zero (boundary nodes).  A: scipy CSR of the assembled system."""
    dg = np.abs((G.T @ A @ G).diagonal())
    dp = np.abs((Pi.T @ A @ Pi).diagonal())
    sg = np.where(dg > 0, 1.0 / np.sqrt(np.where(dg > 0, dg, 1.0)), 0.0)
    spp = np.where(dp > 0, 1.0 / np.sqrt(np.where(dp > 0, dp, 1.0)), 0.0)
    return sg, spp.reshape(-1, 3)


def node_features(sigma: np.ndarray, cells, sigma_p: float, freq: float, h: float) -> np.ndarray:
    """[V, 2]: log10(sigma / sigma_p) and log10(w mu0 sigma h^2) of the cell whose lowest corner is
    the node (clamped to the last cell), sigma of a cell = the mean over its six tets 6c .. 6c+5."""
    nx, ny, nz = cells
    sig = sigma.reshape(nz, ny, nx, 6).mean(axis=3)
    ix, iy, iz = (np.minimum(np.arange(m + 1), m - 1) for m in (nx, ny, nz))
    sc = sig[np.ix_(iz, iy, ix)].reshape(-1)
    w = 2.0 * np.pi * freq * 4e-7 * np.pi
    return np.stack([np.log10(sc / sigma_p), np.log10(w * sc * h * h)], axis=1)


def hx_input(r: np.ndarray, G, Pi, sg: np.ndarray, sp_: np.ndarray, feat: np.ndarray):
    """Network input grid [V, 16] and the scale s for the residual r (complex [E])."""
    V = G.shape[1]
    fg = sg * (G.T @ r)
    fp = sp_ * (Pi.T @ r).reshape(-1, 3)
    n_in = int(np.count_nonzero(sg))
    tot = (np.abs(fg) ** 2).sum() + (np.abs(fp) ** 2).sum()
    s = float(np.sqrt(tot / (4 * n_in))) if n_in and tot > 0 else 1.0
    x = np.zeros((V, 16))
    x[:, 0], x[:, 1] = fg.real / s, fg.imag / s
    x[:, 2:5], x[:, 5:8] = fp.real / s, fp.imag / s
    x[:, 8:10] = feat
    return x, s


def hx_direction(y: np.ndarray, r: np.ndarray, s: float, G, Pi, sg, sp_, diag: np.ndarray) -> np.ndarray:
    """z = D^{-1} r + G phi + Pi w for the network output y [V, 16]."""
    phi = s * sg * (y[:, 0] + 1j * y[:, 1])
    w = s * sp_ * (y[:, 2:5] + 1j * y[:, 5:8])
    return r / diag + G @ phi + Pi @ w.reshape(-1)


def hx_angle_loss(y: np.ndarray, r: np.ndarray, s: float, G, Pi, sg, sp_, diag, spmv):
    """L = 1 - |<r, A z>|^2 / (|r|^2 |A z|^2) for z = hx_direction(y, ...): zero when one step
    along z removes the whole residual.  Returns (L, dL/dy [V, 16]), the gradient with respect to
    the real output channels (channels 8..15 get zero)."""
    z = hx_direction(y, r, s, G, Pi, sg, sp_, diag)
    w = spmv(z)
    a = np.vdot(r, w)
    b = np.vdot(w, w).real
    c = np.vdot(r, r).real
    L = 1.0 - abs(a) ** 2 / (b * c)
    gw = -2.0 * (a * r / (c * b) - abs(a) ** 2 * w / (c * b * b))   # dL/dRe w + i dL/dIm w
    gz = np.conj(spmv(np.conj(gw)))                                 # A^H gw (A complex symmetric)
    gphi = G.T @ gz                                                 # real G: dL/dRe phi + i dL/dIm phi
    gwn = (Pi.T @ gz).reshape(-1, 3)
    gy = np.zeros_like(y)
    gy[:, 0], gy[:, 1] = s * sg * gphi.real, s * sg * gphi.imag
    gy[:, 2:5], gy[:, 5:8] = s * sp_ * gwn.real, s * sp_ * gwn.imag
    return L, gy
