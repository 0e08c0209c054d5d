"""Training and use of the learned preconditioner (network and kernels in the CUDA library).

Parameter layout of the flat vector the library exposes (petgem_learned_params): for each of the
seven convolutions c1..c7 in order, W[27][cout][cin] then b[cout], with (cin, cout) =
(16,16), (16,32), (32,32), (32,32), (32,32), (32,16), (16,16).  Output channels 14, 15 of c7 are
padding and stay zero.

Training samples come from the plain solver: the iterate x_k at the start of every GMRES cycle; the
library turns each into its residual and trains the network's direction on the residual angle.
"""
from __future__ import annotations

import time

import numpy as np

from . import api, synth

LAYERS = [(16, 16), (16, 32), (32, 32), (32, 32), (32, 32), (32, 16), (16, 16)]
N_OUT = 14


def layout():
    """[(name, w_offset, b_offset, cin, cout)] of the flat parameter vector."""
    out, off = [], 0
    for i, (ci, co) in enumerate(LAYERS):
        w = off
        off += 27 * co * ci
        b = off
        off += co
        out.append(("c%d" % (i + 1), w, b, ci, co))
    return out, off


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases; the output layer starts small."""
    rng = np.random.default_rng(seed)
    lay, n = layout()
    p = np.zeros(n, np.float32)
    for name, w, b, ci, co in lay:
        scale = 0.1 if name == "c7" else 1.0
        wv = rng.normal(size=(27, co, ci)) * np.sqrt(2.0 / (27 * ci)) * scale
        if name == "c7":
            wv[:, N_OUT:, :] = 0.0
        p[w:w + 27 * co * ci] = wv.reshape(-1)
    return p


def unflatten(p: np.ndarray) -> dict:
    lay, _ = layout()
    d = {}
    for name, w, b, ci, co in lay:
        d[name + ".W"] = p[w:w + 27 * co * ci].reshape(27, co, ci).astype(np.float64)
        d[name + ".b"] = p[b:b + co].astype(np.float64)
    return d


def random_block_model(n: int, seed: int) -> synth.Model:
    """Training / evaluation model: the cube [-1000, 1000]^3 m with n cells a side, 1 S/m background,
    1-4 axis-aligned blocks of log-uniform conductivity in [0.01, 10] S/m, frequency log-uniform in
    [0.1, 5] Hz, one x-directed dipole near the centre (outside every block)."""
    rng = np.random.default_rng(seed)
    mesh = synth.kuhn_mesh(n, (-1000.0,) * 3, (1000.0,) * 3)
    cen = mesh.centroids()
    sigma = np.ones(mesh.n_tets)
    for _ in range(int(rng.integers(1, 5))):
        lo = rng.uniform(-900, 500, 3)
        hi = lo + rng.uniform(150, 700, 3)
        inside = np.all((cen >= lo) & (cen <= hi), axis=1)
        sigma[inside] = 10.0 ** rng.uniform(-2, 1)
    src = synth.Dipole(1.0, 1.0, 1.0, 0, 1.0)
    # keep the dipole's own tet in the background so the right-hand side stays integrable
    near = np.linalg.norm(cen - np.array([1.0, 1.0, 1.0]), axis=1) < 2000.0 / n * 1.5
    sigma[near] = 1.0
    freq = float(10.0 ** rng.uniform(np.log10(0.1), np.log10(5.0)))
    rx = np.stack([np.linspace(-500, 500, 11), np.zeros(11), np.full(11, -100.0)], axis=1)
    return synth.Model("blocks_n%d_s%d" % (n, seed), mesh, sigma, 1.0, freq, [src], rx)


def solver_pairs(ctx: api.Context, restart: int = 50, max_cycles: int = 400, precision=api.PREC_MIXED):
    """Run the plain solver one cycle at a time on the context's assembled system (source 0);
    returns (iterates [k, E] at the start of every cycle, converged solution [E], cycles)."""
    import torch
    x = torch.zeros((1, ctx.n_edges), dtype=torch.complex128, device=ctx.nodes.device)
    iterates = []
    for k in range(max_cycles):
        iterates.append(x[0].clone())
        st, info = api.petgem_solve(ctx.h, x, 1, api.solve_opts(restart=restart, precision=precision,
                                                               max_iters=restart), allow_not_converged=True)
        if st == api.OK:
            break
    return torch.stack(iterates), x[0].clone(), len(iterates)


def train(n: int = 32, models: int = 200, epochs: int = 2, lr: float = 1e-3, seed: int = 0, samples_per_model: int = 12,
          params: np.ndarray | None = None, log=None):
    """Train the network on residual / correction pairs of the plain solver over random block models.
    Returns (params, history)."""
    import torch
    ctx = api.Context()
    data = []
    t0 = time.time()
    for m in range(models):
        mdl = random_block_model(n, seed * 100000 + m)
        ctx.mesh(mdl.mesh.nodes, mdl.mesh.tets)
        ctx.assemble(mdl.freq, mdl.sigma, mdl.sigma_p, mdl.sources)
        its, xstar, cyc = solver_pairs(ctx)
        if its.shape[0] > samples_per_model:
            idx = np.linspace(0, its.shape[0] - 1, samples_per_model).round().astype(int)
            its = its[idx]
        data.append((mdl, its, xstar))
    gen_s = time.time() - t0
    history = []
    p = init_params(seed) if params is None else params
    first = True
    t0 = time.time()
    for ep in range(epochs):
        order = np.random.default_rng(seed + ep).permutation(len(data))
        losses = []
        for i in order:
            mdl, its, xstar = data[i]
            ctx.mesh(mdl.mesh.nodes, mdl.mesh.tets)
            ctx.assemble(mdl.freq, mdl.sigma, mdl.sigma_p, mdl.sources)
            api.petgem_learned_create(ctx.h, n, n, n)
            if first:
                api.petgem_learned_params(ctx.h, set_params=p)
                first = False
            losses.append(api.petgem_learned_train_step(ctx.h, its.contiguous(), lr))
        history.append(float(np.mean(losses)))
        if log:
            log("epoch %d loss %.4e" % (ep, history[-1]))
    p = api.petgem_learned_params(ctx.h, get=True)
    ctx.close()
    return p, {"loss": history, "generate_s": gen_s, "train_s": time.time() - t0, "models": models, "n": n}
