"""Train the learned auxiliary-space preconditioner on the GPU and write its weights.

    python -m paper_1808_00186_gb300.train_learned --n 32 --models 2000 --epochs 8 \
        --out paper_1808_00186_gb300/weights/learned_n32.npy

Training data (the library's plain solver on random block models, learned.random_block_model):
the iterates at `--samples` cycle starts spread over the first `--max-cycles` cycles of mixed
Jacobi-GMRES(50) on models seeds 0 .. models-1 of an n^3 cube lattice.  The network is trained
with the library's own tensor-core forward and backward kernels (petgem_learned_train_step).
Then it is evaluated against plain Jacobi GMRES(50) on unseen models (seeds 10000+) of the
evaluation sizes.  Beside the weights (float32, the flat layout of learned.layout()) a JSON file
records the run: data, loss per epoch, times, and the evaluation.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--models", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--samples", type=int, default=6)
    ap.add_argument("--max-cycles", type=int, default=48)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init", default=None, help="start from these weights (.npy)")
    ap.add_argument("--eval-n", type=int, nargs="*", default=[32, 64])
    ap.add_argument("--eval-models", type=int, default=3)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)

    import torch

    from . import api, build
    from . import learned as PL
    build.build()
    api.load()
    torch.cuda.set_device(0)
    log = lambda s: print(s, flush=True)
    init = np.load(a.init) if a.init else None
    t0 = time.time()
    p, hist = PL.train(n=a.n, models=a.models, epochs=a.epochs, lr=a.lr, lr_final=a.lr_final, seed=a.seed,
                       samples_per_model=a.samples, params=init, log=log, max_cycles=a.max_cycles)
    log("trained: generate %.0f s, train %.0f s" % (hist["generate_s"], hist["train_s"]))
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, p.astype(np.float32))
    ev = {}
    for ne in a.eval_n:
        ev[str(ne)] = PL.evaluate(p, ne, list(range(10000, 10000 + a.eval_models)), log=log)
    rec = {"command": "python -m paper_1808_00186_gb300.train_learned " + " ".join(argv or __import__("sys").argv[1:]),
           "train": hist, "eval": ev, "wall_s": time.time() - t0,
           "gpu": torch.cuda.get_device_name(0)}
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
