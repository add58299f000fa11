"""Tile autotuner: times candidate tile shapes through the C ABI and installs
the fastest per grid size with sq_set_tiles (single solves), or returns the
fastest per grid size of a batch for sq_batch_create (tune_batch).

Tuned per N: the number of complex pencils of a Hartley-pass tile (FP32 passes;
2P real pencils, 2P * 4 bytes per row segment), jointly the node rows per
thread and the x1-planes per work item of the FP32 operator, and the tile of the
last pass of a PCG iteration (x3 transform with the x and p updates, which
stages p and x in shared memory). Each candidate is timed with CUDA events over
a few repetitions of the call it drives (sq_apply_precond_f32 for the passes,
sq_apply_operator_f32 for the operator, 24 inner iterations of an FP32 solve for
the last pass), each after an L2 flush; results are cached in a JSON file keyed
by N and the device name.
"""
from __future__ import annotations

import json
import os

from . import sq as _sq

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "tiles.json")


_FLUSH = {}


def _time(torch, fn, reps=5):
    """Median time of fn over reps runs, each after writing 256 MB (twice the
    L2 size) so that the inputs come from HBM, as they do inside a solve."""
    dev = torch.cuda.current_device()
    if dev not in _FLUSH:
        _FLUSH[dev] = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    flush = _FLUSH[dev]
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def tune(torch, N, L=None, n=None, cache=DEFAULT_CACHE, reps=5):
    """Returns (dht_pencils, stencil_planes, stencil_rows, dht_pencils_e) for
    grid N and installs them with sq_set_tiles."""
    dev = torch.cuda.get_device_name()
    key = f"{dev}:{N}"
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except Exception:
            table = {}
    if key in table and "dht_pencils_e" in table[key]:
        e = table[key]
        tile = (e["dht_pencils"], e["stencil_planes"], e["stencil_rows"], e["dht_pencils_e"])
        _sq.sq_set_tiles([(N,) + tile])
        return tile
    if L is None:
        n = 8 if N % 8 == 0 else 4
        L = N // n
    c = _sq.sq_build_coeffs(L, n, 1, 0.5, 1.0, 100.0)
    pc = _sq.sq_precond_setup(N, 0)
    w = _sq.sq_workspace_create(N, _sq.SQ_FP32_REFINE)
    r = torch.randn(N ** 3, dtype=torch.float32, device="cuda")
    z = torch.empty_like(r)
    times_p = {}
    for P in (2, 4, 8, 16):
        if N % (2 * P) != 0:
            continue
        try:
            _sq.sq_set_tiles([(N, P, 0)])
        except _sq.SqError:
            continue
        times_p[P] = _time(torch, lambda: _sq.sq_apply_precond_f32(pc, w, r, z), reps)
    bestP = min(times_p, key=times_p.get)
    times_z = {}
    for rows in (1, 2, 4, 8):
        if N % (32 if rows == 8 else rows) != 0:
            continue
        for zc in ((0,) if rows == 8 else (4, 8, 16, 32)):  # the staged kernel's runs are tuned in solves below
            if zc > N:
                continue
            try:
                _sq.sq_set_tiles([(N, bestP, zc, rows)])
            except _sq.SqError:
                continue
            times_z[(rows, zc)] = _time(torch, lambda: _sq.sq_apply_operator_f32(c, r, z), reps)
    bestR, bestZ = min(times_z, key=times_z.get)
    # the last pass of an iteration, inside 24 inner iterations of an FP32
    # solve (tol 1e-30: the iteration cap ends it; the FP64 sweeps around the
    # inner solve are the same for every candidate)
    wr = _sq.sq_workspace_create(N, _sq.SQ_FP32_REFINE)
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    times_e = {}
    for Pe in sorted({bestP, bestP // 2, bestP // 4}):
        if Pe < 2 or N % (2 * Pe) != 0:
            continue
        try:
            _sq.sq_set_tiles([(N, bestP, bestZ, bestR, Pe)])
        except _sq.SqError:
            continue
        times_e[Pe] = _time(torch, lambda: _sq.sq_pcg_solve(c, pc, wr, 0, 1e-30, 24, _sq.SQ_FP32_REFINE, None, psi),
                            reps)
    bestE = min(times_e, key=times_e.get)
    # The staged operator's plane run per block, also inside solves: its
    # default fills one wave of blocks, and shorter or longer runs trade the
    # per-block set-up against the block count. (Timed alone after an L2
    # flush, the ranking did not carry over into solves.)
    times_s = {}
    if bestR == 8:
        times_s[0] = times_e[bestE]
        for zc in (N // 8, N // 4, N // 2):
            if zc < 4:
                continue
            _sq.sq_set_tiles([(N, bestP, zc, bestR, bestE)])
            times_s[zc] = _time(torch, lambda: _sq.sq_pcg_solve(c, pc, wr, 0, 1e-30, 24, _sq.SQ_FP32_REFINE, None,
                                                                psi), reps)
        bestZ = min(times_s, key=times_s.get)
    _sq.sq_set_tiles([(N, bestP, bestZ, bestR, bestE)])
    table[key] = {"dht_pencils": bestP, "stencil_planes": bestZ, "stencil_rows": bestR, "dht_pencils_e": bestE,
                  "precond_ms": {str(k): round(v, 4) for k, v in times_p.items()},
                  "operator_ms": {f"{k[0]}x{k[1]}": round(v, 4) for k, v in times_z.items()},
                  "solve24_ms": {str(k): round(v, 4) for k, v in times_e.items()},
                  "staged_runs_solve24_ms": {str(k): round(v, 4) for k, v in times_s.items()}}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        json.dump(table, open(cache, "w"), indent=1)
    return bestP, bestZ, bestR, bestE


def tune_batch(torch, descs, precs, tol, max_iter=2000, pencils=(4, 8, 16), planes=None, stream=None):
    """Tile shapes for a batch, per grid size: for each N the batch holds, the
    sub-batch of its solves with that N is planned with every candidate tile
    (Hartley pencils P with 2P dividing N; operator planes per work item, by
    default N/8, N/4 and N/2) and solved once after a warm-up solve; the
    fastest (CUDA events on the launching stream) is kept. Returns the list of
    (N, dht_pencils, stencil_planes) entries for sq_batch_create and the
    per-candidate times in ms."""
    byN = {}
    for d, p in zip(descs, precs):
        _, _, N = _sq.sq_coeffs_shape(d[0])
        byN.setdefault(N, ([], []))
        byN[N][0].append(d)
        byN[N][1].append(p)
    chosen, times = [], {}
    for N, (ds, ps) in sorted(byN.items()):
        cands = []
        for P in pencils:
            if N % (2 * P):
                continue
            for zc in (planes or sorted({max(2, N // 8), max(2, N // 4), max(2, N // 2)})):
                cands.append((P, zc))
        best, best_ms = None, float("inf")
        for P, zc in cands:
            try:
                b = _sq.sq_batch_create(ds, ps, tiles=[(N, P, zc)])
            except _sq.SqError:
                continue
            _sq.sq_pcg_solve_batched(b, tol, max_iter, stream)  # warm-up: graph capture, first touch
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = stream or torch.cuda.current_stream()
            e0.record(s)
            _sq.sq_pcg_solve_batched(b, tol, max_iter, stream)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            times[f"{N}:{P}x{zc}"] = round(ms, 3)
            del b
            if ms < best_ms:
                best, best_ms = (N, P, zc), ms
        if best is not None:
            chosen.append(best)
    return chosen, times
