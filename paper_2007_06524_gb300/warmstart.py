"""Training and evaluation of the learned warm start (sq_net_* in libsq).

The net is trained on correctors the method itself computes: for each
training seed the batched solver (sq_pcg_solve_batched) returns psi_1..3,
which become the targets of sq_net_train_step. At solve time sq_net_predict
supplies x0 to sq_pcg_solve, which keeps the guess only if it lowers the
residual. All arithmetic runs in libsq; this module sequences the calls.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import sq as _sq

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_n64.npz")


def generate_targets(torch, wl, seeds, chunk=256, tol=1e-10, stream=None):
    """Correctors of every seed's realization (3 per seed), as float64 CUDA
    tensors [len(seeds), 3, N^3], from the batched FP32+FP64 solver."""
    L, n = wl["L"], wl["n"]
    N = L * n
    pc = _sq.sq_precond_setup(N, 0)
    out = torch.empty((len(seeds), 3, N ** 3), dtype=torch.float64, device="cuda")
    k = min(chunk, len(seeds))
    pool = [_sq.sq_build_coeffs(L, n, seeds[0], wl["p_hi"], wl["a_lo"], wl["a_hi"]) for _ in range(k)]
    bufs = [[torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)] for _ in range(k)]
    batch = _sq.sq_batch_create([(pool[j], i, bufs[j][i]) for j in range(k) for i in range(3)], [pc] * (3 * k))
    iters = []
    for s0 in range(0, len(seeds), k):
        part = seeds[s0:s0 + k]
        for j, sd in enumerate(part):
            _sq.sq_coeffs_regenerate(pool[j], sd, wl["p_hi"], stream)
        for j in range(len(part), k):      # tail: repeat the last seed (results discarded)
            _sq.sq_coeffs_regenerate(pool[j], part[-1], wl["p_hi"], stream)
        infos = _sq.sq_pcg_solve_batched(batch, tol, 4000, stream)
        iters += [inf["iters"] for inf in infos[:3 * len(part)]]
        for j in range(len(part)):
            for i in range(3):
                out[s0 + j, i].copy_(bufs[j][i])
    return out, iters


def train(torch, wl, targets, seeds, epochs=4, batch=8, lr=2e-3, seed=1, log_every=0, stream=None, loss_type=1):
    """Adam on the energy norm of the error (loss_type 1; 0 = squared error,
    2 = residual norm of the prediction); returns (net, losses, seconds)."""
    L, n = wl["L"], wl["n"]
    N = L * n
    scale = float(targets.std())
    net = _sq.sq_net_create(N, batch, seed, scale)
    pool = [_sq.sq_build_coeffs(L, n, seeds[0], wl["p_hi"], wl["a_lo"], wl["a_hi"]) for _ in range(batch)]
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    nstep = 0
    total_steps = epochs * (len(seeds) // batch)
    for ep in range(epochs):
        order = rng.permutation(len(seeds))
        for b0 in range(0, len(order) - batch + 1, batch):
            idx = order[b0:b0 + batch]
            for j, k in enumerate(idx):
                _sq.sq_coeffs_regenerate(pool[j], seeds[k], wl["p_hi"], stream)
            tg = [[targets[k, i] for i in range(3)] for k in idx]
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * nstep / max(1, total_steps)))  # cosine decay
            losses.append(_sq.sq_net_train_step(net, pool, tg, lr_t, stream, loss_type))
            nstep += 1
            if log_every and nstep % log_every == 0:
                print(f"epoch {ep} step {nstep} loss {np.mean(losses[-log_every:]):.4e}", flush=True)
    torch.cuda.synchronize()
    return net, losses, time.perf_counter() - t0


def save(net, path, N, scale, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=_sq.sq_net_params(net), N=N, scale=scale, **(meta or {}))


def load(path, batch=1):
    d = np.load(path)
    net = _sq.sq_net_create(int(d["N"]), batch, 0, float(d["scale"]))
    _sq.sq_net_set_params(net, d["params"])
    return net


def evaluate(torch, wl, net, seeds, precision, tol=1e-8, stream=None, quality=True):
    """Zero start vs learned start on the given seeds: per-solve iterations and
    solves/s of each (the learned figure includes the net's inference)."""
    L, n = wl["L"], wl["n"]
    N = L * n
    pc = _sq.sq_precond_setup(N, 0)
    w = _sq.sq_workspace_create(N, precision)
    c = _sq.sq_build_coeffs(L, n, seeds[0], wl["p_hi"], wl["a_lo"], wl["a_hi"])
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {}
    for mode in ("zero", "learned"):
        its, used = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sd in seeds:
            _sq.sq_coeffs_regenerate(c, sd, wl["p_hi"], stream)
            if mode == "learned":
                _sq.sq_net_predict(net, c, *g, stream=stream)
            for i in range(3):
                inf = _sq.sq_pcg_solve(c, pc, w, i, tol, 4000, precision, g[i] if mode == "learned" else None, psi,
                                       stream)
                its.append(inf["iters"])
                used += inf["used_guess"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[mode] = {"solves_per_s": round(3 * len(seeds) / dt, 2), "iters_mean": round(float(np.mean(its)), 2),
                     "iters_p50": float(np.percentile(its, 50)), "iters_p99": float(np.percentile(its, 99)),
                     "guesses_kept": used}
    if quality:
        res["guess_quality"] = guess_quality(torch, wl, net, seeds, stream)
    return res


def guess_quality(torch, wl, net, seeds, stream=None, tol=1e-10):
    """How good the learned guess x0 is before any iteration (untimed): the
    mean over seeds and correctors of ||b - A x0|| / ||b|| (the stopping
    rule's norm; zero start gives 1) and of the relative energy-norm error
    sqrt(e.Ae / psi.b), e = x0 - psi, psi the solve's result (zero start
    gives 1). Operator, right-hand side and solve run in libsq; the norms
    and dot products of the resulting fields are taken with torch."""
    L, n = wl["L"], wl["n"]
    N = L * n
    pc = _sq.sq_precond_setup(N, 0)
    w = _sq.sq_workspace_create(N, _sq.SQ_FP64)
    c = _sq.sq_build_coeffs(L, n, seeds[0], wl["p_hi"], wl["a_lo"], wl["a_hi"])
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    psi, b, ax = (torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3))
    rr, ee = [], []
    for sd in seeds:
        _sq.sq_coeffs_regenerate(c, sd, wl["p_hi"], stream)
        _sq.sq_net_predict(net, c, *g, stream=stream)
        for i in range(3):
            _sq.sq_rhs(c, i, b, stream)
            _sq.sq_apply_operator(c, g[i], ax, stream)
            rr.append(float(torch.linalg.norm(b - ax) / torch.linalg.norm(b)))
            _sq.sq_pcg_solve(c, pc, w, i, tol, 4000, _sq.SQ_FP64, None, psi, stream)
            e = g[i] - psi
            _sq.sq_apply_operator(c, e.contiguous(), ax, stream)
            ee.append(float(torch.sqrt(torch.dot(e, ax) / torch.dot(psi, b))))
    return {"init_relres_mean": round(float(np.mean(rr)), 4), "init_relres_max": round(float(np.max(rr)), 4),
            "energy_err_mean": round(float(np.mean(ee)), 4), "samples": len(rr)}
