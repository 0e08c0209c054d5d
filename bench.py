"""Benchmark: time-to-solution per source of the CSEM forward hot path on one GB300.

One step = the whole path on the marine model (64^3 Kuhn cells, 1.57 M tets, 1.87 M edges,
one x-directed dipole at 1 Hz): global edge numbering, assembly of matrix and right-hand
side, the Jacobi-GMRES(50) solve to a relative residual of 1e-8, and the receiver fields.
The headline runs the mixed-precision solver (complex64 Krylov vectors and matrix, FP64
residuals and solution); the plain complex128 solver is timed beside it.

Prints one JSON line.  --impl reference times the CPU oracle on a bounded sample of the same
workload instead.  Synthetic inputs: seeded, generated by paper_1808_00186_gb300.synth.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
METRIC = "time-to-solution per source at rel-residual 1e-8 (learned + mixed c64/FP64-refined FGMRES vs plain)"
sys.path.insert(0, ROOT)

import numpy as np

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=64, help="cells per axis of the marine model")
    p.add_argument("--no-plain", action="store_true", help="skip the complex128 comparison run")
    p.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle throughput leg")
    p.add_argument("--no-ssor", action="store_true", help="skip the SSOR-preconditioned SQMR comparison")
    p.add_argument("--block-sources", type=int, default=32, help="sources of the multi-source block solve (0 = skip)")
    p.add_argument("--freq-sources", type=int, default=64,
                   help="sources of the three-frequency block solve on the bench mesh (0 = skip)")
    p.add_argument("--bathy-n", type=int, default=96, help="cells per axis of the bathymetry case (0 = skip)")
    p.add_argument("--bathy-sources", type=int, default=4, help="sources of the bathymetry case solved with the network")
    p.add_argument("--bathy-block-sources", type=int, default=32,
                   help="sources of the bathymetry case in one learned block solve (0 = skip)")
    p.add_argument("--profile-step", action="store_true",
                   help="run one untimed step of the hot path and exit (the command profilers capture)")
    p.add_argument("--precision", default="mixed", choices=["mixed", "c128"], help="solver of --profile-step")
    p.add_argument("--solver", default="gmres", choices=["gmres", "cocg", "ssor", "learned"],
                   help="Krylov method of --profile-step / --profile-block (ssor: SQMR with the SSOR preconditioner)")
    p.add_argument("--no-cocg", action="store_true", help="skip the COCG measurement")
    p.add_argument("--no-batch", action="store_true", help="skip the batch of uneven meshes")
    p.add_argument("--no-graded", action="store_true", help="skip the graded-mesh measurement")
    p.add_argument("--no-general", action="store_true", help="skip the randomly numbered mesh")
    p.add_argument("--profile-block", type=int, default=0, metavar="ITERS",
                   help="run only the 32-source block solve, capped at ITERS iterations (for ncu)")
    return p.parse_args()


# DRAM traffic per launch / algorithmic bytes per launch, from one ncu capture of each kernel at
# 48^3 (the marine model, Arnoldi step j = 20): these kernels stream
# their vectors once, so the traffic of a bench launch is this ratio times its algorithmic bytes.
TRAFFIC_RATIO = {"spmv_c64": 1.0013, "mdot_c64": 1.0301, "cgs_upd_c64": 0.9860}
# DRAM traffic per launch of kernels whose algorithmic unit is FLOPs, from one ncu capture of the
# same workload (the 11 convolution layers of one network application on the 65^3 lattice:
# 22.46 MB read, 0 written, over 11 launches; each layer's input is read once, its output stays
# in L2 for the next layer).
TRAFFIC_BYTES = {"conv3d_fwd": 2042205}


def tensor_peak():
    """Dense BF16 tensor peak (burst): measured, else the fallback figure."""
    try:
        return float(json.load(open(MEASURED))["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def fp64_peak(device):
    """FP64 FMA peak of the CUDA cores from unit counts: SMs x 2 FP64 FMA/clk x 2 flops x the
    maximum SM clock (measured, else the GB300's 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = 2070.0
    try:
        with open(MEASURED) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return round(sms * 2 * 2 * mhz * 1e6 / 1e12, 3), "%d SMs x 2 FP64 FMA/clk x 2 x %.0f MHz" % (sms, mhz)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device="cpu"):
    """Largest x over the ranks of the process group (all-reduce MAX); x itself for one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_source(t_max_s, sources_per_rank, world):
    """Whole-job time per source of the replicas: the slowest rank's time over every source that all
    ranks solved together (each rank solves its own sources_per_rank)."""
    return t_max_s / (sources_per_rank * world)


def peaks():
    try:
        d = json.load(open(MEASURED))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import torch

    from paper_1808_00186_gb300 import api, synth
    from paper_1808_00186_gb300 import build as libbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    libbuild.build()
    api.load()

    # Replicas: every rank solves its own copy of the model (the path does not shard).
    m = synth.marine_model(args.n, n_src=1)
    S = len(m.sources)
    ctx = api.Context(local)
    dev = torch.device("cuda", local)
    nodes = torch.as_tensor(m.mesh.nodes, device=dev)
    tets = torch.as_tensor(m.mesh.tets, device=dev)
    sigma = torch.as_tensor(m.sigma, device=dev)
    rx = torch.as_tensor(m.receivers, device=dev)

    n_edges = [0]

    def step(precision, method=api.METHOD_GMRES, graphs=1, precond=api.PRECOND_JACOBI):
        E = api.petgem_mesh_edges(ctx.h, nodes, tets)
        n_edges[0] = E
        if precond == api.PRECOND_LEARNED:  # slot map of the new mesh; the weights stay loaded
            api.petgem_learned_create(ctx.h, args.n, args.n, args.n)
        api.petgem_assemble(ctx.h, m.freq, sigma, m.sigma_p, m.sources)
        x = torch.zeros((S, E), dtype=torch.complex128, device=dev)
        st, info = api.petgem_solve(ctx.h, x, S, api.solve_opts(precision=precision, tol=1e-8, method=method,
                                                                use_graphs=graphs, precond=precond))
        out = torch.empty((S, rx.shape[0], 3, 3), dtype=torch.complex128, device=dev)
        api.petgem_receivers(ctx.h, rx, x, out)
        return info, out

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    step_ms = []  # per-step times of the last timed() call (CUDA events between steps)

    def timed(precision, steps, warmup, profile=False, clocks=None, method=api.METHOD_GMRES, graphs=1,
              precond=api.PRECOND_JACOBI):
        for _ in range(warmup):
            step(precision, method, graphs, precond)
        barrier()
        if profile:
            api.petgem_profile(ctx.h, True)
        launches0 = api.petgem_launch_count(ctx.h)
        if clocks:
            clocks.start()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record()
        infos = []
        for k in range(steps):
            infos.append(step(precision, method, graphs, precond)[0])
            evs[k + 1].record()
        barrier()
        cl = clocks.stop() if clocks else None
        ms = evs[0].elapsed_time(evs[-1]) / steps
        step_ms[:] = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
        launches = (api.petgem_launch_count(ctx.h) - launches0) // steps
        return max_over_ranks(ms, world, dev), infos[-1], launches, cl

    if args.profile_block:
        mb = synth.marine_model(args.n, n_src=32)
        Eb = api.petgem_mesh_edges(ctx.h, nodes, tets)
        api.petgem_assemble(ctx.h, mb.freq, sigma, mb.sigma_p, mb.sources)
        xb = torch.zeros((len(mb.sources), Eb), dtype=torch.complex128, device=dev)
        _, binfo = api.petgem_solve(ctx.h, xb, len(mb.sources),
                                    api.solve_opts(precision=api.PREC_MIXED, tol=1e-8, batch=0,
                                                   max_iters=args.profile_block,
                                                   method=api.METHOD_COCG if args.solver == "cocg" else api.METHOD_GMRES),
                                    allow_not_converged=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_block": True, "n": args.n, "edges": Eb, "iters": max(i["iters"] for i in binfo),
                          "launches": api.petgem_launch_count(ctx.h)}))
        ctx.close()
        return None

    if args.profile_block and args.solver == "ssor":
        raise SystemExit("--profile-block runs GMRES or COCG")
    if args.profile_step:
        method = {"gmres": api.METHOD_GMRES, "cocg": api.METHOD_COCG, "ssor": api.METHOD_SQMR,
                  "learned": api.METHOD_GMRES}[args.solver]
        pc = {"ssor": api.PRECOND_SSOR, "learned": api.PRECOND_LEARNED}.get(args.solver, api.PRECOND_JACOBI)
        if pc == api.PRECOND_LEARNED:
            from paper_1808_00186_gb300 import learned as PL
            api.petgem_mesh_edges(ctx.h, nodes, tets)
            api.petgem_learned_create(ctx.h, args.n, args.n, args.n)
            api.petgem_learned_params(ctx.h, set_params=np.load(PL.WEIGHTS))
        info, _ = step(api.PREC_MIXED if args.precision == "mixed" else api.PREC_C128, method, precond=pc)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "n": args.n, "edges": n_edges[0], "info": info,
                          "launches": api.petgem_launch_count(ctx.h)}))
        ctx.close()
        return None

    hbm, peak_kind = peaks()
    bf16_peak = tensor_peak()
    clocks = ClockSampler(local)
    # The learned auxiliary-space preconditioner: the network trained at the 2000-model 32^3 scale
    # (paper_1808_00186_gb300/weights), fully convolutional, applied here on the 65^3 node grid.
    from paper_1808_00186_gb300 import learned as PL
    api.petgem_mesh_edges(ctx.h, nodes, tets)
    api.petgem_learned_create(ctx.h, args.n, args.n, args.n)
    api.petgem_learned_params(ctx.h, set_params=np.load(PL.WEIGHTS))
    LEARNED = api.PRECOND_LEARNED
    # The step time is taken without per-kernel events (an event pair around each launch of a
    # solve costs several percent) and with each FGMRES cycle replayed as a CUDA graph; the
    # per-kernel times come from one more step of the same workload with the events on (direct
    # launches), right after.
    ms_mixed, info_mixed, launches, cl = timed(api.PREC_MIXED, args.steps, args.warmup, clocks=clocks,
                                               precond=LEARNED)
    head_steps = list(step_ms)
    ms_median = max_over_ranks(statistics.median(head_steps), world, dev)
    ms_events, _, _, _ = timed(api.PREC_MIXED, 1, 0, profile=True, precond=LEARNED)
    # Dominant kernel over that step (CUDA events around each launch on the ctx stream): memory
    # kernels carry algorithmic bytes, the convolutions floating-point operations.
    kstats = {}
    for name in ("spmv_c64", "mdot_c64", "cgs_dot2_c64", "cgs_upd_c64", "cgs_upd2_c64", "cycle_init_c64",
                 "xupdate_c64", "residual_c128", "hx_in_c64", "hx_out_c64", "conv3d_fwd",
                 "element", "matrix_gather", "rhs", "rcv_locate"):
        n, kms, by = api.petgem_kernel_stats(ctx.h, name)
        if n:
            flops = name.startswith("conv3d")
            kstats[name] = {"launches": n, "ms": kms, "bytes": by, "unit": "flop" if flops else "byte",
                            "rate": by / (kms * 1e-3) / (1e12 if flops else 1e9)}
    n_apply, ms_apply, _ = api.petgem_kernel_stats(ctx.h, "learned_apply")
    api.petgem_profile(ctx.h, False)
    # The same solve with every kernel launched directly (no CUDA-graph replay of the cycles).
    ms_direct, _, _, _ = timed(api.PREC_MIXED, args.steps, 1, graphs=0, precond=LEARNED)
    # The same precision with Jacobi alone (mixed Jacobi-GMRES(50)), the method without the network.
    ms_jac, info_jac, _, _ = timed(api.PREC_MIXED, min(args.steps, 3), 1)
    mixed_jacobi = {"ms_per_step": round(ms_jac, 3), "s_per_source": round(ms_jac / 1e3 / S, 6),
                    "iters": info_jac[0]["iters"], "cycles": info_jac[0]["restarts"],
                    "true_rel_residual": info_jac[0]["true_rel_residual"]}
    plain = None
    if not args.no_plain:
        ms_plain, info_plain, _, _ = timed(api.PREC_C128, 1, 1)
        plain = {"ms_per_step": ms_plain, "s_per_source": ms_plain / 1e3 / S, "iters": info_plain[0]["iters"],
                 "true_rel_residual": info_plain[0]["true_rel_residual"]}
        # Its Gram-Schmidt kernels are bound by the FP64 pipe (ncu: 87-95 % busy, DRAM 11-26 %), so
        # their roofline is FP64 arithmetic: one more step with per-kernel events, FLOPs from the
        # timed bytes (projections over j + 1 vectors: (j + 2) 16 n bytes, 8 (j + 1) n + 4 n FLOP;
        # update: (j + 3) 16 n bytes, 8 (j + 1) n + 4 n FLOP), peak from the unit counts.
        timed(api.PREC_C128, 1, 0, profile=True)
        n_e = n_edges[0]
        pk = {}
        for name, extra in (("mdot_c128", 4.0), ("cgs_upd_c128", 12.0)):
            nl, kms, by = api.petgem_kernel_stats(ctx.h, name)
            if nl:
                pk[name] = {"launches": nl, "ms": round(kms, 3), "tflops": (by / 2.0 - extra * n_e * nl) / (kms * 1e-3) / 1e12,
                            "gbs": round(by / (kms * 1e-3) / 1e9, 1)}
        api.petgem_profile(ctx.h, False)
        if pk:
            kname, kd = max(pk.items(), key=lambda kv: kv[1]["ms"])
            fp64 = fp64_peak(local)
            plain["roofline"] = {"kernel": kname, "bound": "alu", "achieved": round(kd["tflops"], 3), "peak": fp64[0],
                                 "unit": "TFLOP/s (FP64)", "frac": round(kd["tflops"] / fp64[0], 4),
                                 "peak_source": fp64[1], "hbm_gbs": kd["gbs"], "hbm_frac": round(kd["gbs"] / hbm, 4)}
            plain["kernels"] = {k: {kk: (round(vv, 3) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                                for k, v in pk.items()}

    # COCG (short-recurrence complex-symmetric solver), same workload and tolerance: mixed
    # precision timed like the headline, then one step with per-kernel events.
    cocg = None
    if not args.no_cocg:
        ms_cg, info_cg, _, _ = timed(api.PREC_MIXED, args.steps, 1, method=api.METHOD_COCG)
        timed(api.PREC_MIXED, 1, 0, profile=True, method=api.METHOD_COCG)
        cks = {}
        for name in ("cg_inner_c64", "cg_residual_c128"):
            n_, kms, by = api.petgem_kernel_stats(ctx.h, name)
            if n_:
                cks[name] = {"launches": n_, "ms": round(kms, 3), "gbs": round(by / (kms * 1e-3) / 1e9, 1)}
        api.petgem_profile(ctx.h, False)
        cocg = {"precision": "mixed", "ms_per_step": round(ms_cg, 3), "s_per_source": round(ms_cg / 1e3 / S, 6),
                "iters": info_cg[0]["iters"], "inner_solves": info_cg[0]["restarts"],
                "true_rel_residual": info_cg[0]["true_rel_residual"], "kernels": cks}
        # SQMR (the paper's Section 5.3 solver): COCG's recurrences with the QMR-smoothed iterate
        ms_q, info_q, _, _ = timed(api.PREC_MIXED, args.steps, 1, method=api.METHOD_SQMR)
        cocg["sqmr"] = {"precision": "mixed", "ms_per_step": round(ms_q, 3), "s_per_source": round(ms_q / 1e3 / S, 6),
                        "iters": info_q[0]["iters"], "inner_solves": info_q[0]["restarts"],
                        "true_rel_residual": info_q[0]["true_rel_residual"]}
        # SQMR with the multicolour SSOR preconditioner (the paper's SQMR + SOR runs): mixed
        # precision timed like the headline, then one step with per-kernel events; FP64 beside the
        # Jacobi-split SQMR in FP64.  A step includes the colouring (the mesh is renumbered).
        if not args.no_ssor:
            ms_s, info_s, _, _ = timed(api.PREC_MIXED, args.steps, 1, method=api.METHOD_SQMR,
                                       precond=api.PRECOND_SSOR)
            timed(api.PREC_MIXED, 1, 0, profile=True, method=api.METHOD_SQMR, precond=api.PRECOND_SSOR)
            sks = {}
            for name in ("ssor_spmv_c64", "ssor_forward_c64", "ssor_backward_c64", "ssor_residual_c128"):
                n_, kms, by = api.petgem_kernel_stats(ctx.h, name)
                if n_:
                    sks[name] = {"timed_scopes": n_, "ms": round(kms, 3), "gbs": round(by / (kms * 1e-3) / 1e9, 1)}
            api.petgem_profile(ctx.h, False)
            nc, nr = api.petgem_colouring(ctx.h)
            ms_s128, info_s128, _, _ = timed(api.PREC_C128, 1, 1, method=api.METHOD_SQMR, precond=api.PRECOND_SSOR)
            ms_j, info_j, _, _ = timed(api.PREC_C128, 1, 1, method=api.METHOD_SQMR)
            cocg["sqmr_ssor"] = {
                "precision": "mixed", "ms_per_step": round(ms_s, 3), "s_per_source": round(ms_s / 1e3 / S, 6),
                "iters": info_s[0]["iters"], "inner_solves": info_s[0]["restarts"],
                "true_rel_residual": info_s[0]["true_rel_residual"], "omega": 1.0, "colours": nc,
                "colouring_rounds": nr, "kernels": sks,
                "c128": {"ms_per_step": round(ms_s128, 3), "iters": info_s128[0]["iters"],
                         "true_rel_residual": info_s128[0]["true_rel_residual"]},
                "jacobi_sqmr_c128": {"ms_per_step": round(ms_j, 3), "iters": info_j[0]["iters"],
                                     "true_rel_residual": info_j[0]["true_rel_residual"]}}

    # Multi-source block solve (all sources of one frequency in one SpMM-based solve): the marine
    # mesh with args.block_sources dipoles along x in [-4, 4] km; timed once after a warm-up.
    block = None
    if args.block_sources > 1:
        mb = synth.marine_model(args.n, n_src=args.block_sources)
        Sb = len(mb.sources)

        def block_step(method):
            Eb = api.petgem_mesh_edges(ctx.h, nodes, tets)
            api.petgem_assemble(ctx.h, mb.freq, sigma, mb.sigma_p, mb.sources)
            xb = torch.zeros((Sb, Eb), dtype=torch.complex128, device=dev)
            st, info = api.petgem_solve(ctx.h, xb, Sb, api.solve_opts(precision=api.PREC_MIXED, tol=1e-8, batch=0,
                                                                      method=method))
            return info

        def block_run(method, names):
            block_step(method)
            barrier()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record()
            binfo = block_step(method)
            b1.record()
            barrier()
            api.petgem_profile(ctx.h, True)  # per-kernel times: one more solve with events on
            block_step(method)
            barrier()
            bks = {}
            for name in names:
                n_, kms, by = api.petgem_kernel_stats(ctx.h, name)
                if n_:
                    bks[name] = {"launches": n_, "ms": round(kms, 3), "gbs": round(by / (kms * 1e-3) / 1e9, 1)}
            api.petgem_profile(ctx.h, False)
            bms = b0.elapsed_time(b1)
            return {"sources": Sb, "ms_per_step": round(bms, 3), "s_per_source": round(bms / 1e3 / Sb, 6),
                    "iters_max": max(i["iters"] for i in binfo),
                    "worst_true_rel_residual": max(i["true_rel_residual"] for i in binfo), "kernels": bks}

        block = block_run(api.METHOD_GMRES, ("bspmm_c64", "bmdot_c64", "bmupdate_c64", "bresidual_c128"))
        if not args.no_cocg:
            block["cocg"] = block_run(api.METHOD_COCG, ("bcg_spmm_c64", "bcg_pq_c64", "bcg_update_c64", "bcg_dir_c64",
                                                        "bcg_residual_c128"))

    # Learned preconditioner (tcgen05 convolutions): the network on this mesh's parent grid
    # ((n+1)^3 nodes), apply time and the convolutions' throughput against the BF16 tensor peak.
    # Frequency reuse: the bench system re-assembled from 1 Hz to 3 Hz (one of the batched
    # configuration's frequencies) from the kept K and M_sigma, against a full assembly at 3 Hz.
    freq_reuse = None
    if not args.no_batch:
        api.petgem_mesh_edges(ctx.h, nodes, tets)

        def t_of(fn, reps=5):
            fn()
            best = float("inf")
            for _ in range(reps):
                barrier()
                t0 = time.perf_counter()
                fn()
                barrier()
                best = min(best, time.perf_counter() - t0)
            return best

        t_full = t_of(lambda: api.petgem_assemble(ctx.h, 3.0, sigma, m.sigma_p, m.sources))
        api.petgem_assemble(ctx.h, 1.0, sigma, m.sigma_p, m.sources)
        t_reuse = t_of(lambda: api.petgem_assemble_frequency(ctx.h, 3.0, m.sources))
        freq_reuse = {"from_hz": 1.0, "to_hz": 3.0, "assemble_ms": round(t_full * 1e3, 3),
                      "assemble_frequency_ms": round(t_reuse * 1e3, 3), "speedup": round(t_full / t_reuse, 2)}

    # Frequency-adapted graded meshes (Section 5.3's spacing rules) against uniform meshes at equal
    # accuracy: the marine two-half-space model (seawater 3.3 S/m over 1 S/m sediment, no
    # reservoir) with the homogeneous seawater background, so that E_s = E_layered - E_whole(3.3)
    # is known exactly (petgem_primary_layered) and the right-hand side lives in the sediment only,
    # away from the source.  Domain top at 3 km (truncation of the seawater field ~e^-10).  Error:
    # relative L2 error of the inline E_s,x and of E_total at the 101 seafloor receivers 1 m into
    # the sediment with offsets >= 500 m; mixed COCG to 1e-8.
    graded = None
    if not args.no_graded:
        f_g = 1.0
        rxg = np.stack([np.linspace(-4000.0, 4000.0, 101), np.zeros(101), np.full(101, -1.0)], axis=1)
        keep = np.abs(rxg[:, 0]) >= 500.0
        src_g = synth.Dipole(0.0, 0.0, 50.0, 0, 1.0)
        rxg_t = torch.as_tensor(rxg, device=dev)
        e_lay = torch.empty((101, 3), dtype=torch.complex128, device=dev)
        e_ws = torch.empty_like(e_lay)
        cs = torch.cuda.current_stream(dev).cuda_stream
        api.petgem_primary_layered(cs, [0.0], [3.3, 1.0], f_g, src_g, rxg_t, e_lay)
        api.petgem_primary_layered(cs, [], [3.3], f_g, src_g, rxg_t, e_ws)
        es_x = (e_lay - e_ws).cpu().numpy()[keep, 0]
        et_ex = e_lay.cpu().numpy()[keep]

        def score(mesh, label):
            cen = mesh.centroids()
            sg = np.where(cen[:, 2] > 0.0, 3.3, 1.0)
            gc = api.Context(local)
            try:
                E = gc.mesh(mesh.nodes, mesh.tets)
                gc.assemble(f_g, sg, 3.3, [src_g])
                barrier()
                t0 = time.perf_counter()
                xg, ginfo, gst = gc.solve(precision=api.PREC_MIXED, method=api.METHOD_COCG, tol=1e-8,
                                          allow_not_converged=True)
                barrier()
                t_s = time.perf_counter() - t0
                og, _ = gc.receivers(rxg, xg)
                og = og[0].cpu().numpy()
            finally:
                gc.close()
            ex_err = np.linalg.norm(og[keep, 1, 0] - es_x) / np.linalg.norm(es_x)
            et_err = np.linalg.norm(og[keep, 2, :] - et_ex) / np.linalg.norm(et_ex)
            return {"mesh": label, "cells": list(mesh.n), "edges": E, "iters": ginfo[0]["iters"], "status": gst,
                    "solve_ms": round(t_s * 1e3, 3), "err_Es_x": round(float(ex_err), 5),
                    "err_E_total": round(float(et_err), 5)}

        runs = []
        for N in (49, 63, 91):
            axx = np.linspace(-5000.0, 5000.0, N + 1)
            runs.append(score(synth.kuhn_mesh_axes([axx, axx, np.linspace(-4000.0, 3000.0, N + 1)]),
                              "uniform %d^3" % N))
        for rd in (1.0, 2.0, 3.0):
            gm = synth.graded_marine_model(f_g, L_s=1200.0, r_delta=rd, reservoir=False, z_surface=3000.0)
            runs.append(score(gm.mesh, "graded r_delta=%g L_s=1200" % rd))
        graded = {"model": "seawater 3.3 / sediment 1.0 half-spaces, background 3.3, x-HED 50 m above seafloor",
                  "freq_hz": f_g, "receivers": "101 at z = -1 m, offsets >= 500 m", "runs": runs}

    # Batch of uneven meshes: eight marine models from 16^3 to 48^3 cells (one source each) solved
    # together by petgem_solve_batch (COCG, mixed precision, one persistent launch per refinement
    # round, the rounds replayed as CUDA graphs, SpMV lanes per row autotuned), against the same
    # eight solved one after the other with petgem_solve (COCG, mixed).
    uneven = None
    if not args.no_batch:
        sizes = (16, 20, 24, 28, 32, 36, 40, 48)
        bctx = []
        for nn in sizes:
            mm = synth.marine_model(nn, n_src=1)
            cc = api.Context(local)
            cc.mesh(mm.mesh.nodes, mm.mesh.tets)
            cc.assemble(mm.freq, mm.sigma, mm.sigma_p, mm.sources)
            bctx.append(cc)
        xs = [torch.zeros((1, cc.n_edges), dtype=torch.complex128, device=dev) for cc in bctx]

        def batch_once():
            for xx in xs:
                xx.zero_()
            return api.solve_batch(bctx, xs, precision=api.PREC_MIXED, tol=1e-8, use_graphs=1)[1]

        def seq_once():
            infos = []
            for cc, xx in zip(bctx, xs):
                xx.zero_()
                infos.append(cc.solve(xx, precision=api.PREC_MIXED, tol=1e-8, method=api.METHOD_COCG)[1][0])
            return infos

        def best_of(fn, reps=3):
            fn()
            best, out = float("inf"), None
            for _ in range(reps):
                barrier()
                t0 = time.perf_counter()
                out = fn()
                barrier()
                best = min(best, time.perf_counter() - t0)
            return best, out

        t_b, ib = best_of(batch_once)
        t_s, isq = best_of(seq_once)
        uneven = {"meshes": ["%d^3" % nn for nn in sizes], "edges": [cc.n_edges for cc in bctx],
                  "batch_ms": round(t_b * 1e3, 3), "sequential_ms": round(t_s * 1e3, 3),
                  "speedup": round(t_s / t_b, 3), "spmv_lanes": ib[0]["spmv_lanes"],
                  "iters_batch": [i["iters"] for i in ib], "iters_sequential": [i["iters"] for i in isq],
                  "worst_true_rel_residual": max(i["true_rel_residual"] for i in ib)}
        for cc in bctx:
            cc.close()

    # A general mesh: the bench model with its node ids and tets in random order (seeded), so that
    # the numbering carries none of the lattice's locality.  The SELL-32 layout needs at most 64
    # distinct edge node-id differences and so falls back to the CSR product; mixed Jacobi-GMRES(50),
    # timed like the headline, then one step with per-kernel events for the SpMV's rate.
    general = None
    if not args.no_general:
        mg = synth.relabel(m)
        gc = api.Context(local)

        def gen_step(profile=False):
            gc.mesh(mg.mesh.nodes, mg.mesh.tets)
            gc.assemble(mg.freq, mg.sigma, mg.sigma_p, mg.sources)
            if profile:
                api.petgem_profile(gc.h, True)
            _, gi, gst = gc.solve(precision=api.PREC_MIXED, tol=1e-8, use_graphs=1)
            return gi

        gen_step()
        barrier()
        t0 = time.perf_counter()
        gi = gen_step()
        barrier()
        t_g = time.perf_counter() - t0
        gen_step(profile=True)
        nl, kms, by = api.petgem_kernel_stats(gc.h, "spmv_c64")
        api.petgem_profile(gc.h, False)
        general = {"mesh": "marine 64^3, node ids and tets randomly permuted", "edges": gc.n_edges,
                   "s_per_source": round(t_g / S, 6), "iters": gi[0]["iters"],
                   "true_rel_residual": gi[0]["true_rel_residual"],
                   "spmv_c64": {"launches": nl, "avg_us": round(kms / max(nl, 1) * 1e3, 2),
                                "gbs": round(by / (kms * 1e-3) / 1e9, 1) if kms else None,
                                "frac_of_hbm": round(by / (kms * 1e-3) / 1e9 / hbm, 4) if kms else None,
                                "layout": "CSR (no SELL-32 on this numbering)"}}
        gc.close()

    # Many sources at several frequencies on the bench mesh (64 x-HEDs along x in [-4, 4] km at
    # 0.25, 1 and 3 Hz): the first frequency assembled in full, the others re-formed from the kept K
    # and M_sigma; each frequency's sources solved together by block COCG in mixed precision (the
    # launch unit is a group of up to 32 interleaved sources).  One short solve first as a warm-up.
    multi_freq = None
    if args.freq_sources > 0:
        mf = synth.marine_model(args.n, n_src=args.freq_sources)
        Sf = len(mf.sources)
        Ef = api.petgem_mesh_edges(ctx.h, nodes, tets)
        xf = torch.zeros((Sf, Ef), dtype=torch.complex128, device=dev)
        freqs = (0.25, 1.0, 3.0)
        api.petgem_assemble(ctx.h, freqs[0], sigma, mf.sigma_p, mf.sources)
        api.petgem_solve(ctx.h, xf, Sf, api.solve_opts(precision=api.PREC_MIXED, tol=1e-8, batch=0, max_iters=20,
                                                       method=api.METHOD_COCG), allow_not_converged=True)
        barrier()
        per_f = []
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * len(freqs) + 1)]
        ev[0].record()
        infos_f = []
        for k, f in enumerate(freqs):
            if k == 0:
                api.petgem_assemble(ctx.h, f, sigma, mf.sigma_p, mf.sources)
            else:
                api.petgem_assemble_frequency(ctx.h, f, mf.sources)
            ev[2 * k + 1].record()
            xf.zero_()
            _, inf_f = api.petgem_solve(ctx.h, xf, Sf, api.solve_opts(precision=api.PREC_MIXED, tol=1e-8, batch=0,
                                                                       method=api.METHOD_COCG, max_iters=60000),
                                        allow_not_converged=True)
            ev[2 * k + 2].record()
            infos_f.append(inf_f)
        barrier()
        for k, f in enumerate(freqs):
            t_as = ev[2 * k].elapsed_time(ev[2 * k + 1])
            t_so = ev[2 * k + 1].elapsed_time(ev[2 * k + 2])
            per_f.append({"freq_hz": f, "assemble_ms": round(t_as, 3), "solve_ms": round(t_so, 3),
                          "s_per_source": round((t_as + t_so) / 1e3 / Sf, 6),
                          "iters_max": max(i["iters"] for i in infos_f[k]),
                          "not_converged": [j for j, i in enumerate(infos_f[k]) if i["status"] != api.OK],
                          "worst_true_rel_residual": max(i["true_rel_residual"] for i in infos_f[k])})
        total = ev[0].elapsed_time(ev[-1])
        multi_freq = {"sources": Sf, "frequencies_hz": list(freqs), "method": "block COCG, mixed precision",
                      "launch_unit_sources": min(Sf, 32), "total_ms": round(total, 3),
                      "s_per_source_per_frequency": round(total / 1e3 / (Sf * len(freqs)), 6), "per_frequency": per_f}
        del xf

    # The largest case: the 96^3 bathymetry model (sinusoidal seafloor, two resistive bodies) with
    # 32 x-HEDs at 0.5 Hz.  Mesh and assembly, then the learned + mixed FGMRES on the first
    # --bathy-sources sources one after the other, and on source 0 the same precision without the
    # network (mixed Jacobi GMRES) and the short-recurrence mixed COCG.  Block COCG over all 32
    # sources runs as long as its slowest source and is not timed here.
    bathy = None
    if args.bathy_n > 0:
        nb_ = args.bathy_n
        m4 = synth.bathymetry_model(nb_, n_src=32, freq=0.5)
        c4 = api.Context(local)
        t0 = time.perf_counter()
        E4 = c4.mesh(m4.mesh.nodes, m4.mesh.tets)
        api.petgem_learned_create(c4.h, nb_, nb_, nb_)
        c4.assemble(m4.freq, m4.sigma, m4.sigma_p, m4.sources[:args.bathy_sources])
        barrier()
        t_setup = time.perf_counter() - t0
        api.petgem_learned_params(c4.h, set_params=np.load(PL.WEIGHTS))
        bathy = {"workload": "bathymetry_n%d_0.5Hz" % nb_, "tets": int(m4.mesh.n_tets), "edges": E4,
                 "mesh_and_assembly_ms": round(t_setup * 1e3, 3)}
        xs4 = torch.zeros((args.bathy_sources, E4), dtype=torch.complex128, device=dev)
        c4.solve(xs4, precision=api.PREC_MIXED, precond=LEARNED, tol=1e-8, use_graphs=1, max_iters=60,
                 allow_not_converged=True)
        barrier()
        t0 = time.perf_counter()
        xs4.zero_()
        _, il, _ = c4.solve(xs4, precision=api.PREC_MIXED, precond=LEARNED, tol=1e-8, use_graphs=1,
                            allow_not_converged=True, max_iters=60000)
        barrier()
        dt = time.perf_counter() - t0
        bathy["learned_fgmres_mixed"] = {"sources": args.bathy_sources, "s_per_source": round(dt / args.bathy_sources, 6),
                                         "iters": [i["iters"] for i in il], "fell_back": [i["fell_back"] for i in il],
                                         "worst_true_rel_residual": max(i["true_rel_residual"] for i in il),
                                         "not_converged": [j for j, i in enumerate(il) if i["status"] != api.OK]}
        del xs4
        # All sources in one learned block solve (flexible GMRES on interleaved block vectors, the
        # network applied to each source's column, one SpMM per step), mixed precision, to 1e-8.
        # A short solve first sizes the block workspace and runs the SpMM autotuner.
        if args.bathy_block_sources > 0:
            nbs = min(args.bathy_block_sources, len(m4.sources))
            c4.assemble(m4.freq, m4.sigma, m4.sigma_p, m4.sources[:nbs])
            xb4 = torch.zeros((nbs, E4), dtype=torch.complex128, device=dev)
            c4.solve(xb4, precision=api.PREC_MIXED, precond=LEARNED, tol=1e-8, batch=0, max_iters=60,
                     allow_not_converged=True)
            barrier()
            t0 = time.perf_counter()
            xb4.zero_()
            _, ibl, _ = c4.solve(xb4, precision=api.PREC_MIXED, precond=LEARNED, tol=1e-8, batch=0,
                                 allow_not_converged=True, max_iters=60000)
            barrier()
            dt = time.perf_counter() - t0
            bathy["learned_block_mixed"] = {"sources": nbs, "s_per_source": round(dt / nbs, 6),
                                            "iters_max": max(i["iters"] for i in ibl),
                                            "iters": [i["iters"] for i in ibl],
                                            "fell_back": [i["fell_back"] for i in ibl],
                                            "worst_true_rel_residual": max(i["true_rel_residual"] for i in ibl),
                                            "not_converged": [j for j, i in enumerate(ibl) if i["status"] != api.OK]}
            del xb4
        c4.assemble(m4.freq, m4.sigma, m4.sigma_p, m4.sources[:1])
        x1 = torch.zeros((1, E4), dtype=torch.complex128, device=dev)
        for name, kw in (("jacobi_gmres_mixed", dict(use_graphs=1)), ("cocg_mixed", dict(method=api.METHOD_COCG))):
            c4.solve(x1, precision=api.PREC_MIXED, tol=1e-8, max_iters=60, allow_not_converged=True, **kw)
            barrier()
            t0 = time.perf_counter()
            x1.zero_()
            _, i1, st1 = c4.solve(x1, precision=api.PREC_MIXED, tol=1e-8, allow_not_converged=True, max_iters=60000, **kw)
            barrier()
            dt = time.perf_counter() - t0
            bathy[name] = {"s_per_source": round(dt, 6), "iters": i1[0]["iters"], "status": st1,
                           "true_rel_residual": i1[0]["true_rel_residual"]}
        c4.close()
        del x1

    # The learned preconditioner in the headline step: apply time and the convolutions' rates
    # (all levels on the tensor cores, against the BF16 peak).
    learned = None
    if n_apply:
        conv = kstats.get("conv3d_fwd")
        learned = {"grid": [args.n + 1] * 3, "levels": PL.levels((args.n + 1,) * 3),
                   "weights": os.path.relpath(PL.WEIGHTS, ROOT),
                   "applies": n_apply, "apply_us": round(ms_apply / n_apply * 1e3, 1),
                   "iters": info_mixed[0]["iters"], "fell_back": info_mixed[0]["fell_back"],
                   "iters_jacobi": info_jac[0]["iters"],
                   "iteration_ratio": round(info_mixed[0]["iters"] / max(1, info_jac[0]["iters"]), 3),
                   "speedup_vs_mixed_jacobi": round(ms_jac / ms_mixed, 3)}
        if conv:
            learned["conv3d_tensor_core"] = {"launches": conv["launches"], "ms": round(conv["ms"], 3),
                                             "tflops": round(conv["rate"], 2),
                                             "frac_of_bf16_peak": round(conv["rate"] / bf16_peak[0], 4)}

    # End to end through the public API from pinned host buffers, results read back each step.
    h_nodes = torch.as_tensor(m.mesh.nodes).pin_memory()
    h_tets = torch.as_tensor(m.mesh.tets).pin_memory()
    h_sigma = torch.as_tensor(m.sigma).pin_memory()
    h_rx = torch.as_tensor(m.receivers).pin_memory()
    h_out = torch.empty((S, m.receivers.shape[0], 3, 3), dtype=torch.complex128).pin_memory()

    def e2e_step():
        nodes.copy_(h_nodes, non_blocking=True)
        tets.copy_(h_tets, non_blocking=True)
        sigma.copy_(h_sigma, non_blocking=True)
        rx.copy_(h_rx, non_blocking=True)
        info, out = step(api.PREC_MIXED, precond=LEARNED)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        return info

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        e2e_step()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / max(1, args.steps), world, dev)
    h2d = sum(t.numel() * t.element_size() for t in (h_nodes, h_tets, h_sigma, h_rx))
    d2h = h_out.numel() * h_out.element_size()

    result = None
    if rank == 0:
        dom = max(kstats.items(), key=lambda kv: kv[1]["ms"]) if kstats else None
        roof = None
        if dom:
            name, ks = dom
            achieved = ks["rate"]
            flops = ks["unit"] == "flop"
            bound = "tensor" if flops else "hbm"
            peak = bf16_peak[0] if flops else hbm
            roof = {"kernel": name, "bound": bound, "achieved": round(achieved, 2),
                    "peak": peak, "unit": "TFLOP/s" if flops else "GB/s", "frac": round(achieved / peak, 4),
                    "peak_source": bf16_peak[1] if flops else peak_kind,
                    "traffic": (round(TRAFFIC_RATIO[name] * ks["bytes"] / ks["launches"]) if name in TRAFFIC_RATIO
                                else TRAFFIC_BYTES.get(name)),
                    "traffic_unit": "bytes per launch (ncu DRAM read+write)",
                    "launches": ks["launches"], "avg_launch_us": round(ks["ms"] / ks["launches"] * 1e3, 2),
                    ("algorithmic_flops_per_launch" if flops else "algorithmic_bytes_per_launch"):
                        ks["bytes"] / ks["launches"]}
        result = {
            "metric": METRIC,
            "value": round(job_seconds_per_source(ms_mixed / 1e3, S, world), 6),
            "unit": "s/source",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_mixed, 3),
            "ms_per_step_median": round(ms_median, 3),
            "ms_per_step_each": [round(x, 3) for x in head_steps],
            "ms_per_step_with_kernel_events": round(ms_events, 3),
            "ms_per_step_without_graphs": round(ms_direct, 3),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "c64+f64",
            "data": "synthetic (seeded Kuhn mesh, marine layered model)",
            "config": {"workload": "marine_n%d_1src_1Hz" % args.n, "tets": m.mesh.n_tets,
                       "edges": n_edges[0], "sources": S, "restart": 50, "tol": 1e-8, "precision": "mixed",
                       "preconditioner": "learned auxiliary-space (Jacobi + network on the node lattice)",
                       "orth": "cgs, second pass when the norm fell below 1/sqrt(10)",
                       "l2": "working set > L2 (no flush needed)", "parallelism": "replicas" if world > 1 else "single"},
            "iters": info_mixed[0]["iters"], "cycles": info_mixed[0]["restarts"],
            "reorth_steps": info_mixed[0]["reorth"],
            "true_rel_residual": info_mixed[0]["true_rel_residual"],
            "mixed_jacobi_gmres": mixed_jacobi,
            "plain_c128": plain,
            "cocg": cocg,
            "block_multi_source": block,
            "uneven_batch": uneven,
            "general_mesh": general,
            "graded_mesh": graded,
            "frequency_reuse": freq_reuse,
            "learned_network": learned,
            "multi_frequency_64src": multi_freq,
            "bathymetry_96": bathy,
            "speedup_vs_plain": round(plain["ms_per_step"] / ms_mixed, 3) if plain else None,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            ("tflops" if v["unit"] == "flop" else "gbs"): round(v["rate"], 2)}
                        for k, v in kstats.items()},
            "roofline": roof,
            "clocks": cl,
            "e2e": {"value": round(job_seconds_per_source(e2e_s, S, world), 6), "unit": "s/source",
                    "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
        }
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def oracle_sample(n, gpu_iters=None):
    """Oracle on the host: full assembly of the workload + 10 GMRES iterations, scaled to a
    time-to-solution with the iteration count (measured here or given)."""
    import oracle
    from paper_1808_00186_gb300 import synth
    oracle.build()
    m = synth.marine_model(n, n_src=1)
    src = synth.sources_array(m.sources)
    t0 = time.perf_counter()
    s = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    t_asm = time.perf_counter() - t0
    k = 10
    t0 = time.perf_counter()
    s.solve(restart=50, tol=1e-8, maxit=k)
    t_it = (time.perf_counter() - t0) / k
    iters = gpu_iters if gpu_iters else 2000
    return {"t_assembly_s": t_asm, "t_iter_s": t_it, "iters_scaled_to": iters,
            "value": t_asm + t_it * iters, "cores": 1,
            "sample": "full oracle assembly of the %d^3 marine model + %d GMRES(50) iterations; value = "
                      "assembly + per-iteration time x %d iterations" % (n, k, iters)}


def _oracle_worker(job):
    n, iters = job
    return oracle_sample(n, gpu_iters=iters)


def host_info():
    """nproc and the CPU model of the host the oracle runs on (/proc/cpuinfo, else lscpu, which
    names Arm cores that /proc/cpuinfo gives only as part numbers)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            model = next((l.split(":", 1)[1].strip() for l in f if l.lower().startswith("model name")), None)
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            model = next((l.split(":", 1)[1].strip() for l in out.splitlines() if l.startswith("Model name:")), None)
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": len(os.sched_getaffinity(0)), "cpu_model": model}


def oracle_all_cores(n, iters, per_proc_bytes=3.0e9):
    """The unmodified single-threaded oracle on all host cores: one independent single-source
    sample per process, as many processes as cores, bounded so that they hold at most half of
    the host's available memory.  Throughput per source = median per-process time / processes."""
    import multiprocessing as mp
    P = len(os.sched_getaffinity(0))
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable:"))
        P = max(1, min(P, int(0.5 * avail // per_proc_bytes)))
    except (OSError, StopIteration):
        P = 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(P) as pool:  # spawn: the parent holds a CUDA context
        rs = pool.map(_oracle_worker, [(n, iters)] * P)
    wall = time.perf_counter() - t0
    per = statistics.median(r["value"] for r in rs)
    return {"value": per / P, "processes": P, "per_process_s": per, "wall_s": wall}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        samples = [oracle_sample(args.n) for _ in range(max(1, args.steps))]
        samp = samples[-1]
        v = statistics.median(x["value"] for x in samples)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s/source",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                          "config": {"workload": "marine_n%d_1src_1Hz" % args.n},
                          "cpu_baseline": {"value": round(v, 3), "unit": "s/source", "cores": 1, "kind": "oracle",
                                           "sample": samp["sample"], **host_info()},
                          "e2e": {"value": round(v, 3), "unit": "s/source", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0},
                          "wall_s": round(time.perf_counter() - t0, 1)}))
        return
    res = run_ours(args)
    if rank == 0 and res is not None:
        iters = (res["plain_c128"] or {}).get("iters") or res["iters"]
        cpu = oracle_sample(args.n, gpu_iters=iters)
        res["cpu_baseline"] = {"value": round(cpu["value"], 3), "unit": "s/source", "cores": cpu["cores"],
                               "kind": "oracle", "sample": cpu["sample"], **host_info()}
        if not args.no_all_cores:
            allc = oracle_all_cores(args.n, iters)
            res["cpu_baseline"]["all_cores"] = {
                "value": round(allc["value"], 3), "unit": "s/source", "processes": allc["processes"],
                "per_process_s": round(allc["per_process_s"], 3), "wall_s": round(allc["wall_s"], 1),
                "sample": "the same sample in %d concurrent single-threaded oracle processes; value = median "
                          "per-process time / processes" % allc["processes"]}
        print(json.dumps(res))


if __name__ == "__main__":
    main()
