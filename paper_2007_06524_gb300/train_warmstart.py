"""Trains the learned warm start on method-generated correctors and saves the weights.

  python -m paper_2007_06524_gb300.train_warmstart [--train N] [--epochs E] [--out PATH]

Workload: L=16, n=4 (N=64), Bernoulli(1/2) on {1,10}; training seeds
1000..1000+N-1 (default 4096), held-out evaluation seeds 6000.. (default 512).
Prints one JSON line: training time and loss, then zero start vs learned start
on the evaluation seeds (FP64 and FP32 + refinement: iterations, solves/s) and
the learned guess's initial relative residual and relative energy error.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--eval", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--loss", type=int, default=1,
                    help="0: squared error, 1: energy norm e.Ae, 2: residual norm |A y - b|^2")
    ap.add_argument("--conv", choices=["tc", "mma"], default="tc",
                    help="32-channel convolutions on tcgen05 (tc) or mma.sync (mma)")
    args = ap.parse_args()
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2007_06524_gb300 as sq
    from paper_2007_06524_gb300 import warmstart, workloads

    sq.sq_set_option(sq.SQ_OPT_CONV_TC, 1 if args.conv == "tc" else 0)
    wl = workloads.WARM_N64
    seeds = wl["train_seeds"][: args.train]
    targets, gen_iters = warmstart.generate_targets(torch, wl, seeds)
    net, losses, secs = warmstart.train(torch, wl, targets, seeds, epochs=args.epochs, batch=args.batch, lr=args.lr,
                                        log_every=64, loss_type=args.loss)
    out = args.out or warmstart.DEFAULT_WEIGHTS
    N = wl["L"] * wl["n"]
    warmstart.save(net, out, N, float(targets.std()),
                   {"train_seeds": np.array([seeds[0], seeds[-1]]), "epochs": args.epochs, "final_loss": losses[-1],
                    "loss_type": args.loss})
    evs = wl["eval_seeds"][: args.eval]
    ev = {"fp64": warmstart.evaluate(torch, wl, warmstart.load(out), evs, sq.SQ_FP64),
          "fp32_refine": warmstart.evaluate(torch, wl, warmstart.load(out), evs, sq.SQ_FP32_REFINE, quality=False)}
    print(json.dumps({"train_samples": len(seeds), "epochs": args.epochs, "train_seconds": round(secs, 1),
                      "steps": len(losses), "loss": args.loss, "loss_first": float(np.mean(losses[:16])),
                      "loss_last": float(np.mean(losses[-16:])), "gen_iters_mean": float(np.mean(gen_iters)),
                      "eval": ev, "weights": out}))


if __name__ == "__main__":
    main()
