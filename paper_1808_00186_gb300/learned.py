"""Training and use of the learned preconditioner (network and kernels in the CUDA library).

The preconditioner is z = D^{-1} r + G phi + Pi w: Jacobi plus the two auxiliary spaces of the
edge elements (nodal gradients and nodal vector fields), with the two nodal solves replaced by a
3-D convolutional network on the node lattice (include/petgem.h, "learned preconditioner").

Parameter layout of the flat vector the library exposes (petgem_learned_params): for each of the
seven convolutions c1..c7 in order, W[27][cout][cin] then b[cout], with (cin, cout) =
(16,16), (16,32), (32,32), (32,32), (32,32), (32,16), (16,16).  Output channels 8..15 of c7 are
unused and stay zero.

Training samples come from the plain solver: the iterate x_k at the start of every GMRES cycle; the
library turns each into its residual and trains the network on the residual angle of one step
along z.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import api, synth

LAYERS = [(16, 16), (16, 32), (32, 32), (32, 32), (32, 32), (32, 16), (16, 16)]
# the network trained by train_learned at the 2000-model 32^3 scale (its run record beside it)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "learned_n32.npy")
N_OUT = 8


def levels(grid) -> int:
    """Levels of the network on a node grid (poolings until the coarsest grid has at most 3 nodes
    per axis, at least 3 levels), as the library builds it."""
    dims, L = list(grid), 1
    while max(dims) > 3:
        dims = [(d + 1) // 2 for d in dims]
        L += 1
    return max(3, L)


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


def solve_samples(ctx: api.Context, samples: int, restart: int = 50, max_cycles: int = 400,
                  precision=api.PREC_MIXED):
    """Iterates at `samples` cycle starts, spread evenly over the plain solve of the context's
    assembled system (source 0), as a device tensor [k, E]; and the number of cycles it took."""
    its, _, cyc = solver_pairs(ctx, restart=restart, max_cycles=max_cycles, precision=precision)
    if its.shape[0] > samples:
        idx = np.linspace(0, its.shape[0] - 1, samples).round().astype(int)
        its = its[idx]
    return its, cyc


def train(n: int = 32, models: int = 200, epochs: int = 2, lr: float = 1e-3, seed: int = 0, samples_per_model: int = 8,
          params: np.ndarray | None = None, log=None, lr_final: float | None = None, max_cycles: int = 400):
    """Train the network on residuals of the plain solver over random block models on one n^3 cube
    lattice (models differ in conductivity and frequency only, so the mesh is built once).
    The learning rate decays geometrically from lr to lr_final (default lr / 10) over the epochs.
    Returns (params, history)."""
    ctx = api.Context()
    mdl0 = random_block_model(n, seed * 100000)
    ctx.mesh(mdl0.mesh.nodes, mdl0.mesh.tets)
    api.petgem_learned_create(ctx.h, n, n, n)
    data = []
    t0 = time.time()
    cycles = []
    for m in range(models):
        mdl = random_block_model(n, seed * 100000 + m)
        ctx.assemble(mdl.freq, mdl.sigma, mdl.sigma_p, mdl.sources)
        its, cyc = solve_samples(ctx, samples_per_model, max_cycles=max_cycles)
        cycles.append(cyc)
        data.append((mdl.freq, mdl.sigma, mdl.sigma_p, mdl.sources, its))
        if log and (m + 1) % 200 == 0:
            log("data: %d models, %.0f s" % (m + 1, time.time() - t0))
    gen_s = time.time() - t0
    history = []
    p = init_params(seed) if params is None else params
    api.petgem_learned_params(ctx.h, set_params=p)
    lr_final = lr / 10.0 if lr_final is None else lr_final
    t0 = time.time()
    steps = 0
    for ep in range(epochs):
        order = np.random.default_rng(seed + ep).permutation(len(data))
        lr_ep = lr * (lr_final / lr) ** (ep / max(1, epochs - 1))
        losses = []
        for i in order:
            freq, sigma, sigma_p, sources, its = data[i]
            ctx.assemble(freq, sigma, sigma_p, sources)
            losses.append(api.petgem_learned_train_step(ctx.h, its.contiguous(), lr_ep))
            steps += 1
        history.append(float(np.mean(losses)))
        if log:
            log("epoch %d lr %.2e loss %.4e (%.0f s)" % (ep, lr_ep, history[-1], time.time() - t0))
    p = api.petgem_learned_params(ctx.h, get=True)
    ctx.close()
    return p, {"loss": history, "generate_s": gen_s, "train_s": time.time() - t0, "models": models, "n": n,
               "samples_per_model": samples_per_model, "epochs": epochs, "steps": steps,
               "mean_cycles": float(np.mean(cycles))}


def evaluate(params: np.ndarray, n: int, seeds, precision=api.PREC_MIXED, tol: float = 1e-8, log=None,
             use_graphs: int = 1):
    """Learned FGMRES against plain Jacobi GMRES(50) on unseen random block models of n^3 cells:
    [{seed, iters_jacobi, iters_learned, s_jacobi, s_learned, fell_back, relres}] (times from
    CUDA events around each solve, assembly excluded)."""
    import torch
    out = []
    ctx = api.Context()
    try:
        for k, sd in enumerate(seeds):
            mdl = random_block_model(n, sd)
            if k == 0:
                ctx.mesh(mdl.mesh.nodes, mdl.mesh.tets)
                api.petgem_learned_create(ctx.h, n, n, n)
                api.petgem_learned_params(ctx.h, set_params=params)
            ctx.assemble(mdl.freq, mdl.sigma, mdl.sigma_p, mdl.sources)
            rec = {"seed": int(sd), "freq": mdl.freq}
            for name, pc in (("jacobi", api.PRECOND_JACOBI), ("learned", api.PRECOND_LEARNED)):
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                ev0.record()
                x, info, st = ctx.solve(precision=precision, precond=pc, tol=tol, allow_not_converged=True,
                                        use_graphs=use_graphs)
                ev1.record()
                torch.cuda.synchronize()
                rec["iters_" + name] = int(info[0]["iters"])
                rec["s_" + name] = ev0.elapsed_time(ev1) / 1e3
                rec["relres_" + name] = float(info[0]["true_rel_residual"])
                rec["status_" + name] = int(st)
                if name == "learned":
                    rec["fell_back"] = int(info[0]["fell_back"])
            out.append(rec)
            if log:
                log("eval n=%d seed %d f=%.2f: jacobi %d its %.3f s, learned %d its %.3f s (fell back %d)"
                    % (n, sd, mdl.freq, rec["iters_jacobi"], rec["s_jacobi"], rec["iters_learned"],
                       rec["s_learned"], rec["fell_back"]))
    finally:
        ctx.close()
    return out
