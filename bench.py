#!/usr/bin/env python3
"""Corrector solves per second to rel. residual 1e-8 on the N=256 random
checkerboard (L=32 cells per side, n=8 points per cell, Bernoulli(1/2) on
{1,100}), three correctors e_1..e_3 and the full 3x3 homogenized matrix per
realization, FP64 PCG with the rank-8 canonical Laplacian preconditioner.

One step = one realization through the whole hot path: cell phases from the
seed, three PCG solves (RHS, iterations, mean projection, true-residual
check) and A_hom. `value` is measured with CUDA events on the launching
stream, inputs resident in HBM; `e2e` repeats the step through the public C
ABI with the cell phases copied from pinned host memory and A_hom read back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank runs independent realizations (replicas,
weak scaling); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "corrector solves/s to rel-res 1e-8 (N=256), % HBM peak, plain vs learned start"
UNIT = "corrector solves/s"


def _peaks():
    """HBM peak: the measured STREAM-style copy bandwidth of this GPU type
    (MEASURED_PEAKS.json) where present, else the fallback figure of one
    earlier GB300 measurement."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured (MEASURED_PEAKS.json copy)"}
    return {"hbm_gbs": 6800.0, "src": "fallback (6.8 TB/s, an earlier GB300 copy measurement)"}


# nominal rates, used only where no probe ran (host-only tests)
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x max clock


def default_peaks():
    """Peaks without a GPU probe: HBM as _peaks(), FMA rates nominal."""
    pk = _peaks()
    return {"hbm_gbs": pk["hbm_gbs"], "hbm_src": pk["src"],
            "fp64_tflops": FP64_NOMINAL_TFLOPS, "fp64_src": "nominal FP64 rate of GB300 (1.25 TFLOP/s)",
            "fp32_tflops": FP32_NOMINAL_TFLOPS, "fp32_src": "nominal: 152 SMs x 128 FMA x 2.07 GHz"}


def measure_peaks(sq, torch):
    """The roofline denominators measured on this GPU by the library's probes:
    FP64 and FP32 fused multiply-add throughput (eight independent chains per
    thread, a full grid) and a copy of 2 x 2 GiB (HBM) and of 2 x 16 MiB (L2)
    buffers. The HBM peak stays the MEASURED_PEAKS.json figure where present;
    the probe's copy figure is reported beside it (the fallback is used where
    that file is absent)."""
    pk = default_peaks()
    fp64, _ = sq.sq_probe_fma(0)
    fp32, _ = sq.sq_probe_fma(1)
    pk.update({"fp64_tflops": round(fp64, 4), "fp64_src": "measured: FP64 FMA probe (sq_probe_fma)",
               "fp32_tflops": round(fp32, 3), "fp32_src": "measured: FP32 FMA probe (sq_probe_fma)"})
    big = 2 << 30
    a = torch.empty(big // 4, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    pk["copy_hbm_gbs"] = round(sq.sq_probe_copy(a, b, 5), 1)
    del a, b
    small = 16 << 20
    a = torch.empty(small // 4, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    pk["copy_l2_gbs"] = round(sq.sq_probe_copy(a, b, 500), 1)
    del a, b
    return pk


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

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
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def workload_config(args, ws):
    """The `config` object of both arms: the N=256 workload and its settings."""
    from paper_2007_06524_gb300 import workloads

    wl = workloads.PLAIN_N256
    L, n = wl["L"], wl["n"]
    N = L * n
    elem = 8 if args.precision == "fp64" else 4
    return {"workload": f"plain L={L} n={n} N={N}, Bernoulli(1/2) on {{1,100}}, 3 correctors + A_hom, "
                        f"rank-{args.rank} preconditioner, tol {wl['tol']:g}, {args.precision}",
            "L": L, "n": n, "N": N, "rank": args.rank, "tol": wl["tol"], "precision": args.precision,
            "seeds": f"rank + {ws} k, k < {args.steps}",
            "l2": "inputs larger than L2 (4 working fields of %d MB each)" % (N ** 3 * elem // 2 ** 20),
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def replica_seeds(rank, ws, count, offset=0):
    """Realization seeds of one rank, disjoint across ranks for any count:
    offset + rank + ws * k, k < count."""
    return [offset + rank + ws * k for k in range(count)]


def aggregate(t_ms, steps, ws, device):
    """The slowest rank's timed region (max over ranks) and the whole-job
    corrector solves/s: 3 solves per realization, `steps` realizations per
    rank. Needs an initialised process group when ws > 1."""
    if ws > 1:
        import torch
        import torch.distributed as dist

        tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    return t_ms, 3 * steps * ws / (t_ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _algorithmic(N, elem, rank_r, table=None):
    """Per-launch algorithmic bytes and flops of each kernel class (one PCG iteration).

    bytes: the fields each kernel must read and write once (N^3 elements of
    `elem` bytes); flops: one real 1D Hartley pass = 2.5 log2 N + 3 per point
    (half-length complex FFT convention + the Hartley combine). The FP64
    passes B and D take the complex x2 route (no combine): 2.5 log2 N. Pass C
    does two transforms with no combine (the scaling is applied to the complex
    spectrum): 2 x 2.5 log2 N, plus 6 for the scaling and the r.z sum, plus
    the multiplier where it is evaluated per mode (2R, or 4 for the exact
    1/x); on grids N <= 256 pass C reads it from the precomputed table
    instead, except FP32 with the exact diagonal (table=None: that default)."""
    n3 = N ** 3
    f = 2.5 * math.log2(N) + 3.0
    if table is None:
        table = N <= 256 and (elem == 8 or rank_r > 0)
    scale = 6 if table else ((2 * rank_r + 6) if rank_r else 10)
    return {
        "stencil_matvec": (2 * elem * n3, 15 * n3),
        "dht_x3_in": (4 * elem * n3, (f + 4) * n3),
        "dht_x2": (2 * elem * n3, (f - 3.0 if elem == 8 else f) * n3),
        "dht_x1_scale": (2 * elem * n3, (2 * (f - 3.0) + scale) * n3),
        "dht_x3_out": (5 * elem * n3, (f + 4) * n3),
    }


# dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu --set full,
# N = 256, rank 8): profiles/dht_x1_scale_fp64_n256.md (multiplier table) and
# profiles/dht_x3_pass_e_fp32_n256.md (8-pencil tiles). Part of each kernel's
# writes is still in L2 when it ends, so traffic can read below the
# algorithmic bytes.
PROFILED_TRAFFIC = {("dht_x1_scale", 8): 151.53e6 + 79.04e6, ("dht_x3_out", 4): 201.35e6 + 76.52e6}


def kernel_table(work, prof, N, elem, R, t_ms, peaks=None):
    """Per-class table and the dominant class's roofline from the library's
    event profile: achieved = algorithmic bytes (flops) per launch x launches
    that did work / their summed duration (launches that returned at entry,
    their solve having stopped, excluded by sq_profile_work). The bound is the
    larger of the HBM and FMA-pipe fractions; both are reported."""
    alg = _algorithmic(N, elem, R)
    pk = peaks or default_peaks()
    kernels = {}
    for name, (ms, cnt) in prof.items():
        if ms <= 0:
            continue
        k = {"ms": round(ms, 3), "launches": cnt, "share": round(ms / t_ms, 4)}
        wms, wn = work.get(name, (0.0, 0))
        if name in alg and wn > 0 and wms > 0:
            b, f = alg[name]
            k.update({"work_launches": wn, "us_per_work_launch": round(wms / wn * 1e3, 1),
                      "GBps": round(b * wn / (wms / 1e3) / 1e9, 1), "GFLOPps": round(f * wn / (wms / 1e3) / 1e9, 1)})
        kernels[name] = k
    dom = max((k for k in kernels if "GBps" in kernels[k]), key=lambda k: kernels[k]["ms"])
    kd = kernels[dom]
    fp_peak, fp_src = (pk["fp64_tflops"], pk["fp64_src"]) if elem == 8 else (pk["fp32_tflops"], pk["fp32_src"])
    frac_hbm = kd["GBps"] / pk["hbm_gbs"]
    frac_alu = kd["GFLOPps"] / (fp_peak * 1e3)
    if frac_alu > frac_hbm:
        roof = {"kernel": dom, "bound": "alu", "achieved": round(kd["GFLOPps"] / 1e3, 4), "peak": fp_peak,
                "unit": "TFLOP/s", "frac": round(frac_alu, 4), "peak_src": fp_src,
                "hbm_frac": round(frac_hbm, 4), "hbm_peak_gbs": pk["hbm_gbs"]}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kd["GBps"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(frac_hbm, 4), "peak_src": pk["hbm_src"], "alu_frac": round(frac_alu, 4)}
    # DRAM bytes per launch (read + write) from the ncu capture of this kernel
    # at N = 256 (profiles/); None where no capture of the current kernel exists
    tr = PROFILED_TRAFFIC.get((dom, elem)) if N == 256 else None
    roof["traffic"] = tr
    if tr is not None:
        roof["traffic_alg"] = alg[dom][0]
    return kernels, roof


def run_native(args):
    import numpy as np
    import torch

    import __graft_entry__

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_2007_06524_gb300 as sq
    from paper_2007_06524_gb300 import workloads

    wl = dict(workloads.PLAIN_N256)
    L, n = wl["L"], wl["n"]
    N = L * n
    R = args.rank
    prec = sq.SQ_FP64 if args.precision == "fp64" else sq.SQ_FP32_REFINE
    tol, max_iter = wl["tol"], 1000
    stream = torch.cuda.current_stream()

    from paper_2007_06524_gb300 import autotune

    if args.no_graphs:  # the same kernels, launched one by one (for profilers that cannot replay graph nodes)
        sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, 0)
    if args.tiles:
        tiles = tuple(int(v) for v in args.tiles.split(","))
        if len(tiles) == 3:
            tiles = tiles + (0,)
        sq.sq_set_tiles([(N,) + tiles])
    else:
        tiles = autotune.tune(torch, N, L, n, cache=None)  # FP32 pass tile and operator planes for this grid
    c = sq.sq_build_coeffs(L, n, 0, wl["p_hi"], wl["a_lo"], wl["a_hi"])
    pc = sq.sq_precond_setup(N, R)
    w = sq.sq_workspace_create(N, prec)
    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]

    def step(seed, upload=None):
        if upload is None:
            sq.sq_coeffs_regenerate(c, seed, wl["p_hi"])
        else:
            sq.sq_coeffs_upload(c, upload)
        infos = [sq.sq_pcg_solve(c, pc, w, i, tol, max_iter, prec, None, psis[i]) for i in range(3)]
        A, _ = sq.sq_homogenized_matrix(c, *psis, energy=False)  # edge form (Eq. 21); the energy cross-check is not timed
        return infos, A

    seeds = replica_seeds(rank, ws, args.steps)
    for sd in replica_seeds(rank, ws, args.warmup, offset=10 ** 6):
        step(sd)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    # --- the timed region: K realizations, no profiling events
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    launches0 = sq.sq_launch_count()
    e0.record(stream)
    all_infos, As = [], []
    for sd in seeds:
        infos, A = step(sd)
        all_infos += infos
        As.append(A)
    e1.record(stream)
    torch.cuda.synchronize()
    gpu_launches = sq.sq_launch_count() - launches0
    clocks = sampler.stop()
    t_ms, value = aggregate(e0.elapsed_time(e1), args.steps, ws, "cuda")
    iters = [i["iters"] for i in all_infos]
    ok = all(i["status"] == sq.SQ_OK and i["relres_true"] <= tol for i in all_infos)
    elem = 8 if prec == sq.SQ_FP64 else 4

    # --- end to end through the C ABI with pinned host inputs
    e2e = None
    rng = np.random.default_rng(12345 + rank)
    if not args.no_e2e:
        host = [torch.from_numpy(rng.integers(0, 2, L ** 3, dtype=np.uint8)).pin_memory() for _ in range(args.steps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(None, upload=host[k])
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": round(3 * args.steps / t_e2e, 4), "unit": UNIT, "h2d_bytes_per_step": L ** 3,
               "d2h_bytes_per_step": 2 * 9 * 8}

    # --- per-kernel profile from one more realization (untimed: the event
    # pairs around every launch would slow the timed steps), and the measured
    # roofline denominators
    peaks = measure_peaks(sq, torch)
    sq.sq_coeffs_regenerate(c, replica_seeds(rank, ws, 1, offset=10 ** 7)[0], wl["p_hi"])
    sq.sq_profile_enable(True)
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    for i in range(3):
        sq.sq_pcg_solve(c, pc, w, i, tol, max_iter, prec, None, psis[i])
    sq.sq_homogenized_matrix(c, *psis, energy=False)
    ep1.record(stream)
    torch.cuda.synchronize()
    prof = sq.sq_profile_read()
    sq.sq_profile_enable(False)
    kernels, roof = kernel_table(sq.sq_profile_work(), prof, N, elem, R, ep0.elapsed_time(ep1), peaks)

    # whole-solve HBM fraction: the fused iteration's 17 field passes (operator
    # 2, x3 in 4, x2 2 + 2, x1 2, x3 out 5) of s-byte words per PCG iteration,
    # against the solve's wall time (setup passes, residual recomputations
    # and A_hom are not counted: a lower bound on the bytes moved)
    def solve_hbm(its_mean, solves_per_s, s_bytes):
        gbs = 17 * s_bytes * N ** 3 * its_mean * solves_per_s / 1e9
        return {"algorithmic_GBps": round(gbs, 1), "peak": peaks["hbm_gbs"], "peak_src": peaks["hbm_src"],
                "frac": round(gbs / peaks["hbm_gbs"], 4), "bytes_per_iteration": 17 * s_bytes * N ** 3}

    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if elem == 8 else "f32+f64",
           "data": "synthetic",
           "config": workload_config(args, ws),
           "clocks": clocks, "gpu_launches": gpu_launches, "roofline": roof}
    if e2e:
        out["e2e"] = e2e
    out.update({"peaks": peaks, "kernels": kernels,
                "iters": {"mean": round(statistics.mean(iters), 2), "min": min(iters), "max": max(iters)},
                "solve_hbm": solve_hbm(statistics.mean(iters), value / max(ws, 1), elem),
                "converged": ok, "tiles": {"dht_pencils_fp32": tiles[0], "stencil_planes": tiles[1],
                                           "stencil_rows_fp32": tiles[2], "dht_pencils_e_fp32": tiles[3]}})

    # --- variants on the same workload (2 steps each)
    want = None if args.variants is None else set(args.variants.split(","))

    def on(name):
        return want is None or name in want

    if not args.no_variants and rank == 0:
        variants = {}
        for label, rr, pp in (("fp32_refine_exact", 0, sq.SQ_FP32_REFINE), ("fp32_refine_rank8", 8, sq.SQ_FP32_REFINE),
                              ("fp64_exact", 0, sq.SQ_FP64), ("fp64_rank4", 4, sq.SQ_FP64),
                              ("fp64_rank16", 16, sq.SQ_FP64)):
            if not on(label):
                continue
            pcv = sq.sq_precond_setup(N, rr)
            wv = sq.sq_workspace_create(N, pp) if pp != prec else w
            sq.sq_coeffs_regenerate(c, 7, wl["p_hi"])
            for i in range(3):
                sq.sq_pcg_solve(c, pcv, wv, i, tol, max_iter, pp, None, psis[i])
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            its = []
            nst = 2
            for k in range(nst):
                sq.sq_coeffs_regenerate(c, replica_seeds(rank, ws, nst)[k], wl["p_hi"])
                for i in range(3):
                    inf = sq.sq_pcg_solve(c, pcv, wv, i, tol, max_iter, pp, None, psis[i])
                    its.append(inf["iters"])
                sq.sq_homogenized_matrix(c, *psis, energy=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            tv = ev0.elapsed_time(ev1)
            variants[label] = {"solves_per_s": round(3 * nst / (tv / 1e3), 3), "iters_mean": round(statistics.mean(its), 1),
                               "solve_hbm": solve_hbm(statistics.mean(its), 3 * nst / (tv / 1e3),
                                                      4 if pp == sq.SQ_FP32_REFINE else 8)}
            if label == "fp32_refine_rank8":
                # per-kernel table from one more, profiled realization
                sq.sq_coeffs_regenerate(c, replica_seeds(rank, ws, 1, offset=10 ** 7)[0], wl["p_hi"])
                sq.sq_profile_enable(True)
                evp0, evp1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                evp0.record(stream)
                for i in range(3):
                    sq.sq_pcg_solve(c, pcv, wv, i, tol, max_iter, pp, None, psis[i])
                evp1.record(stream)
                torch.cuda.synchronize()
                pv = sq.sq_profile_read()
                sq.sq_profile_enable(False)
                kv, rv = kernel_table(sq.sq_profile_work(), pv, N, 4, rr, evp0.elapsed_time(evp1), peaks)
                variants[label]["kernels"] = kv
                variants[label]["iteration_hbm"] = fused_iteration_hbm(kv, N, 4, peaks["hbm_gbs"])
                variants[label]["iteration_slope"] = iteration_by_slope(sq, torch, c, pcv, wv, N, stream,
                                                                        peaks["hbm_gbs"])
                out["roofline_fp32_refine"] = rv
            del pcv
        out["variants"] = variants
        del w
        torch.cuda.empty_cache()
        legs = (("refine_error_n128", lambda: run_refine_error_n128(sq, torch)),
                ("batch_768_mixed", lambda: run_batch(sq, torch, stream, peaks=peaks)),
                ("warm_start_n64", lambda: run_warm_start(sq, torch)),
                ("refine_n512", lambda: run_refine_n512(sq, torch, stream, peaks["hbm_gbs"])),
                ("ensemble", lambda: run_ensemble(sq, torch)),
                ("inclusions_alpha_quarter", lambda: run_inclusions(sq, torch, stream)),
                ("two_contrasts_alpha_quarter", lambda: run_two_contrasts(sq, torch, stream)),
                ("precond_routes_n256", lambda: run_precond_routes(sq, torch, stream)),
                ("table_2d_alpha_quarter", lambda: run_2d_table(sq, torch, stream)))
        for name, leg in legs:
            if on(name):
                variants[name] = leg()

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(R)
    if rank == 0:
        out["summary"] = summarize(out)
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def fused_iteration_hbm(kernels, N, elem, hbm_gbs):
    """One fused PCG iteration from the per-class times of launches that did
    work: operator + x3-in + 2 x x2 + x1 + x3-out, 17 field passes of
    elem-byte words, against the HBM peak."""
    need = ("stencil_matvec", "dht_x3_in", "dht_x2", "dht_x1_scale", "dht_x3_out")
    if not all(k in kernels and "us_per_work_launch" in kernels[k] for k in need):
        return None
    us = sum(kernels[k]["us_per_work_launch"] for k in need) + kernels["dht_x2"]["us_per_work_launch"]
    b = 17 * elem * N ** 3
    return {"us": round(us, 1), "bytes": b, "GBps": round(b / (us * 1e-6) / 1e9, 1),
            "frac": round(b / (us * 1e-6) / 1e9 / hbm_gbs, 4)}


def summarize(out):
    """The figures a reader needs first, repeated at the end of the line."""
    v = out.get("variants", {})
    sm = {"fp64_rank8_solves_per_s": out["value"], "e2e": (out.get("e2e") or {}).get("value"),
          "roofline": {k: out["roofline"].get(k) for k in ("kernel", "bound", "frac", "peak", "peak_src", "hbm_frac")},
          "peaks": {k: out.get("peaks", {}).get(k) for k in ("fp64_tflops", "fp32_tflops", "hbm_gbs", "copy_hbm_gbs",
                                                              "copy_l2_gbs")}}
    if "fp32_refine_rank8" in v:
        sm["fp32_refine_rank8_solves_per_s"] = v["fp32_refine_rank8"]["solves_per_s"]
        sm["fp32_iteration_hbm"] = v["fp32_refine_rank8"].get("iteration_hbm")
        sm["fp32_iteration_slope"] = v["fp32_refine_rank8"].get("iteration_slope")
        sm["fp32_solve_hbm_frac"] = v["fp32_refine_rank8"]["solve_hbm"]["frac"]
    if "fp32_refine_exact" in v:
        sm["fp32_refine_exact_solves_per_s"] = v["fp32_refine_exact"]["solves_per_s"]
    if "roofline_fp32_refine" in out:
        r = out["roofline_fp32_refine"]
        sm["roofline_fp32_refine"] = {k: r.get(k) for k in ("kernel", "bound", "frac")}
    if "batch_768_mixed" in v:
        b = v["batch_768_mixed"]
        sm["batch"] = {k: b.get(k) for k in ("solves_per_s", "iters_p50", "iters_p99", "hbm_frac")}
        sm["batch"]["inner_busy_frac"] = (b.get("inner_loop") or {}).get("busy_frac")
    if "warm_start_n64" in v:
        sm["warm_start"] = v["warm_start_n64"].get("summary")
    if "refine_error_n128" in v:
        sm["refine_error_n128"] = v["refine_error_n128"].get("max_rel_err")
    if "cpu_baseline" in out:
        sm["cpu_baseline"] = out["cpu_baseline"]["value"]
    return sm


def run_refine_error_n128(sq, torch, seeds=(0, 1, 2, 3)):
    """The precision configuration's subsample (L = 16, n = 8, N = 128,
    Bernoulli(1/2) on {1,100}): FP32 PCG inside FP64 refinement to 1e-10
    against the FP64 PCG solve to 1e-12 on the same GPU, per corrector and
    preconditioner (exact, rank 8): rel. L2 difference of psi and max
    difference of A_hom relative to its largest entry. (The FP64 solve itself
    matches the CPU oracle to 1e-9 in the parity tests.)"""
    import numpy as np

    L, n, N = 16, 8, 128
    c = sq.sq_build_coeffs(L, n, 0, 0.5, 1.0, 100.0)
    w64, w32 = sq.sq_workspace_create(N, sq.SQ_FP64), sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    p64 = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    p32 = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    res, worst = {}, 0.0
    for rank in (0, 8):
        pc = sq.sq_precond_setup(N, rank)
        rows = []
        for sd in seeds:
            sq.sq_coeffs_regenerate(c, sd, 0.5)
            errs = []
            for i in range(3):
                sq.sq_pcg_solve(c, pc, w64, i, 1e-12, 4000, sq.SQ_FP64, None, p64[i])
                sq.sq_pcg_solve(c, pc, w32, i, 1e-10, 4000, sq.SQ_FP32_REFINE, None, p32[i])
                errs.append(float(torch.linalg.norm(p32[i] - p64[i]) / torch.linalg.norm(p64[i])))
            A64, _ = sq.sq_homogenized_matrix(c, *p64, energy=False)
            A32, _ = sq.sq_homogenized_matrix(c, *p32, energy=False)
            ea = float(np.abs(A32 - A64).max() / np.abs(A64).max())
            rows.append({"seed": sd, "psi": [float(f"{e:.3g}") for e in errs], "A_hom": float(f"{ea:.3g}")})
            worst = max(worst, max(errs), ea)
        res[f"rank{rank}"] = rows
    res["max_rel_err"] = float(f"{worst:.3g}")
    return res


def batch_algorithmic(Ns, iters, seconds, hbm_gbs):
    """Algorithmic traffic of a batch: 17 FP32 field passes (4 N^3 bytes each)
    per inner PCG iteration of every solve, over the batch's wall time, and
    that rate against the HBM peak. Every kernel of the batch sweeps all its
    solves, whose fields (5 N^3 floats per solve) together far exceed L2, so
    these passes are HBM traffic."""
    b = float(sum(17 * 4 * int(N) ** 3 * int(it) for N, it in zip(Ns, iters)))
    ws = float(sum(5 * 4 * int(N) ** 3 for N in Ns))
    gbs = b / seconds / 1e9
    return {"algorithmic_bytes": b, "algorithmic_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm_gbs, 4),
            "working_set_GB": round(ws / 1e9, 2),
            "algorithmic_note": "17 FP32 field passes per inner iteration / wall time; working set far above L2"}


def batch_busy(t_graph, t_profiled, prof):
    """Kernel busy fraction of the batch's graph-replayed inner loops:
    the inner-iteration kernels' summed event time (profiled solve) over the
    inner loops' wall time in the graph solve, t_graph - (t_profiled -
    profiled inner-loop time). 1 - busy bounds what a persistent kernel could
    gain by removing kernel boundaries."""
    k_ms, k_n = prof.get("batch_inner", (0.0, 0))
    loop_ms, _ = prof.get("batch_inner_loop", (0.0, 0))
    outside = t_profiled - loop_ms / 1e3
    graph_loop = t_graph - outside
    return {"kernel_s": round(k_ms / 1e3, 5), "kernel_launches": int(k_n), "graph_loop_s": round(graph_loop, 5),
            "profiled_loop_s": round(loop_ms / 1e3, 5),
            "busy_frac": round(k_ms / 1e3 / graph_loop, 4) if graph_loop > 0 else None}


def run_batch(sq, torch, stream, nseeds=256, peaks=None):
    """768 corrector solves (256 realizations x e_1..e_3) in one batch: L drawn
    from {8,12,16,24} per seed, n=4 (N = 32..96), Bernoulli(1/2) on {1,10},
    exact preconditioner, FP32 PCG in FP64 refinement to 1e-8; tiles per N
    from the batch autotuner (each N's sub-batch timed per candidate)."""
    import numpy as np

    from paper_2007_06524_gb300 import autotune, workloads

    wl = workloads.BATCH_MIXED
    precs, descs, pl, coeffs, Ns = {}, [], [], [], []
    for seed in range(nseeds):
        L = wl["Ls"][workloads.batch_L_index(seed)]
        N = L * wl["n"]
        c = sq.sq_build_coeffs(L, wl["n"], seed, wl["p_hi"], wl["a_lo"], wl["a_hi"])
        coeffs.append(c)
        if N not in precs:
            precs[N] = sq.sq_precond_setup(N, 0)
        for i in range(3):
            descs.append((c, i, torch.empty(N ** 3, dtype=torch.float64, device="cuda")))
            pl.append(precs[N])
            Ns.append(N)
    t0 = time.perf_counter()
    tiles, tune_ms = autotune.tune_batch(torch, descs, pl, wl["tol"])
    tune_s = time.perf_counter() - t0
    res = {}
    for label, tl in (("default_tiles", None), ("tuned_tiles", tiles)):
        b = sq.sq_batch_create(descs, pl, tiles=tl)
        sq.sq_pcg_solve_batched(b, wl["tol"], 2000)  # warm-up (graph capture, first touch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = sq.sq_pcg_solve_batched(b, wl["tol"], 2000)
        e1.record(stream)
        torch.cuda.synchronize()
        del b
        res[label] = (e0.elapsed_time(e1) / 1e3, infos)
    # kernel busy time of the inner loop: one more solve with the library's
    # event profile, which launches the graph's kernels one by one with an
    # event pair each and times each whole inner loop. The graph-replayed inner
    # loop's wall time is the graph solve's time minus the profiled solve's
    # time outside its inner loops (the same launches in both).
    b = sq.sq_batch_create(descs, pl, tiles=tiles)
    sq.sq_pcg_solve_batched(b, wl["tol"], 2000)
    torch.cuda.synchronize()
    sq.sq_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sq.sq_pcg_solve_batched(b, wl["tol"], 2000)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sq.sq_profile_read()
    sq.sq_profile_enable(False)
    del b
    busy = batch_busy(res["tuned_tiles"][0], e0.elapsed_time(e1) / 1e3, prof)
    t, infos = res["tuned_tiles"]
    its = np.array([i["iters"] for i in infos])
    ok = all(i["status"] == sq.SQ_OK for i in infos)
    unknowns = sum(d[2].numel() for d in descs)
    out = {"solves": len(descs), "solves_per_s": round(len(descs) / t, 1), "seconds": round(t, 4),
           "iters_p50": float(np.percentile(its, 50)), "iters_p99": float(np.percentile(its, 99)),
           "unknowns": unknowns, "converged": ok, "tiles": [list(x) for x in tiles],
           "default_tiles_solves_per_s": round(len(descs) / res["default_tiles"][0], 1),
           "tune_seconds": round(tune_s, 2), "tune_ms": tune_ms, "inner_loop": busy}
    out.update(batch_algorithmic(Ns, its, t, (peaks or default_peaks())["hbm_gbs"]))
    return out


def run_warm_start(sq, torch, nseeds=512):
    """Zero start vs learned start (committed weights, trained on seeds 1000..5095)
    on held-out seeds 6000.. at L=16, n=4 (N=64), Bernoulli(1/2) on {1,10},
    exact preconditioner, tol 1e-8: FP32+FP64 refinement and plain FP64."""
    from paper_2007_06524_gb300 import warmstart, workloads

    if not os.path.exists(warmstart.DEFAULT_WEIGHTS):
        return {"unavailable": "no trained weights"}
    wl = workloads.WARM_N64
    net = warmstart.load(warmstart.DEFAULT_WEIGHTS)
    seeds = wl["eval_seeds"][:nseeds]
    res = {"eval_seeds": f"{seeds[0]}..{seeds[-1]} ({len(seeds)})"}
    res["fp32_refine"] = warmstart.evaluate(torch, wl, net, seeds, sq.SQ_FP32_REFINE, quality=False)
    res["fp64"] = warmstart.evaluate(torch, wl, net, seeds, sq.SQ_FP64)
    base = res["fp64"]["zero"]["solves_per_s"]
    res["summary"] = {"seeds": len(seeds), "plain_fp64_zero": base,
                      "fp64_learned": res["fp64"]["learned"]["solves_per_s"],
                      "fp32_refine_zero": res["fp32_refine"]["zero"]["solves_per_s"],
                      "fp32_refine_learned": res["fp32_refine"]["learned"]["solves_per_s"],
                      "iters_fp64_zero_learned": [res["fp64"]["zero"]["iters_mean"], res["fp64"]["learned"]["iters_mean"]],
                      "iters_fp32_zero_learned": [res["fp32_refine"]["zero"]["iters_mean"],
                                                  res["fp32_refine"]["learned"]["iters_mean"]],
                      "guess": res["fp64"].get("guess_quality")}
    return res


def run_ensemble(sq, torch, M=32):
    """Ensemble statistics of A_hom (Sec. 5): M realizations at each period
    L in {8, 16, 32} (n = 4, N = 32..128), Bernoulli(1/2) on {1,10}, exact
    preconditioner, FP32 + FP64 refinement to 1e-8; the diagonal spread
    sigma^M_L and its fitted exponent in L (theory: -3/2, Eq. var)."""
    import numpy as np

    res, Ls, sig = {}, [8, 16, 32], []
    for L in Ls:
        seeds = list(range(5000, 5000 + M))
        sq.sq_ensemble_ahom(L, 4, seeds[:2], 0.5, 1.0, 10.0)  # warm-up (graph capture, first touch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sq.sq_ensemble_ahom(L, 4, seeds, 0.5, 1.0, 10.0, tol=1e-8)
        dt = time.perf_counter() - t0
        s = float(np.mean(np.diag(r["sigma"])))
        sig.append(s)
        res[f"L{L}"] = {"realizations_per_s": round(M / dt, 2), "seconds": round(dt, 3),
                        "mean_diag": round(float(np.mean(np.diag(r["mean"]))), 6), "sigma_diag": round(s, 6),
                        "converged": r["status"] == sq.SQ_OK}
    res["sigma_exponent"] = round(float(np.polyfit(np.log(Ls), np.log(sig), 1)[0]), 3)
    res["M"] = M
    return res


def run_inclusions(sq, torch, stream):
    """The paper's experiment setting (Sec. 5): sub-cell inclusions with
    alpha = 1/4 (a centred cube of n/2 grid intervals per cell), lambda = 0.4
    (a in {0.4, 1.0}), Bernoulli(1/2) cells, L = 32, n = 8 (N = 256), three
    correctors + A_hom per realization, tol 1e-8: FP64 PCG (rank 8) and FP32
    + FP64 refinement (exact)."""
    import numpy as np

    L, n, sub, N = 32, 8, 4, 256
    c = sq.sq_build_coeffs(L, n, 0, 0.5, 0.4, 1.0)
    sq.sq_coeffs_set_subcell(c, sub)
    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {}
    for label, rank, prec in (("fp64_rank8", 8, sq.SQ_FP64), ("fp32_refine_exact", 0, sq.SQ_FP32_REFINE)):
        pc = sq.sq_precond_setup(N, rank)
        w = sq.sq_workspace_create(N, prec)
        for i in range(3):
            sq.sq_pcg_solve(c, pc, w, i, 1e-8, 1000, prec, None, psis[i])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, ok, As = [], True, []
        for sd in (11, 12):
            sq.sq_coeffs_regenerate(c, sd, 0.5)
            for i in range(3):
                inf = sq.sq_pcg_solve(c, pc, w, i, 1e-8, 1000, prec, None, psis[i])
                its.append(inf["iters"])
                ok = ok and inf["status"] == sq.SQ_OK
            As.append(sq.sq_homogenized_matrix(c, *psis, energy=False)[0])
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res[label] = {"solves_per_s": round(6 / t, 3), "iters_mean": round(float(np.mean(its)), 1), "converged": ok,
                      "A_hom_diag_mean": round(float(np.mean([np.diag(A) for A in As])), 6)}
    return res


def run_two_contrasts(sq, torch, stream):
    """Varying contrast (Sec. 2): alpha = 1/4 inclusions on half of the cells,
    lambda = 0.4, each inclusion with contrast beta = 0.3 or 0.6 (levels
    {0.4, 0.7, 1.0}), L = 32, n = 8 (N = 256), three correctors + A_hom per
    realization, tol 1e-8. "random": the contrast drawn per cell (probabilities
    1/2, 1/4, 1/4); "layers": the contrast set per layer of four cell planes
    along x1 (alternating), inclusion cells drawn with probability 1/2."""
    import numpy as np

    L, n, sub, N = 32, 8, 4, 256
    vals, probs = (0.4, 0.7, 1.0), (0.5, 0.25, 0.25)
    layer = (1 + (np.arange(L) // 4) % 2).astype(np.uint8)[:, None, None]

    def layered(seed):
        ph, _ = sq.sq_coeffs_cells(sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 2.0))
        return ph * layer

    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {}
    for kind in ("random", "layers"):
        if kind == "random":
            cs = [sq.sq_build_coeffs_levels(L, n, sd, probs, vals) for sd in (11, 12)]
        else:
            cs = [sq.sq_coeffs_from_host_levels(L, n, layered(sd).ravel(), vals) for sd in (11, 12)]
        for c in cs:
            sq.sq_coeffs_set_subcell(c, sub)
        for label, rank, prec in (("fp64_rank8", 8, sq.SQ_FP64), ("fp32_refine_exact", 0, sq.SQ_FP32_REFINE)):
            pc = sq.sq_precond_setup(N, rank)
            w = sq.sq_workspace_create(N, prec)
            for i in range(3):
                sq.sq_pcg_solve(cs[0], pc, w, i, 1e-8, 1000, prec, None, psis[i])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its, ok, As = [], True, []
            for c in cs:
                for i in range(3):
                    inf = sq.sq_pcg_solve(c, pc, w, i, 1e-8, 1000, prec, None, psis[i])
                    its.append(inf["iters"])
                    ok = ok and inf["status"] == sq.SQ_OK
                As.append(sq.sq_homogenized_matrix(c, *psis, energy=False)[0])
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            res[f"{kind}_{label}"] = {"solves_per_s": round(6 / t, 3), "iters_mean": round(float(np.mean(its)), 1),
                                      "converged": ok,
                                      "A_hom_diag": [round(float(v), 6) for v in np.mean([np.diag(A) for A in As], 0)]}
    return res


def run_precond_routes(sq, torch, stream):
    """Canonical preconditioners on the headline workload (L = 32, n = 8,
    N = 256, Bernoulli(1/2) on {1, 100}, FP64 PCG to 1e-8, three correctors):
    the exponential sum (rank 8), the same sum written as the 2R + 1 terms of
    Lemma 4.2 (without the mean projection's shortcut), and the paper's route
    (Sec. 4.2): HOSVD of G+ with Tucker rank r, then Tucker-to-canonical with
    core-slice eigenvalues below tol * max dropped. Per route: canonical
    rank, max relative error of the preconditioner over the nonzero modes,
    host setup time, iterations, solves/s."""
    import numpy as np

    L, n, N = 32, 8, 256
    c = sq.sq_build_coeffs(L, n, 0, 0.5, 1.0, 100.0)
    w = sq.sq_workspace_create(N, sq.SQ_FP64)
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")

    def split_factors(pc, R):
        t, wts = sq.sq_precond_factors(pc, R)
        lam = 4.0 * np.sin(np.pi * np.arange(N) / N) ** 2
        E = np.exp(-np.outer(t, lam))
        d0 = np.zeros(N)
        d0[0] = 1.0
        F1 = np.vstack([wts[:, None] * E, wts[:, None] * d0, [-wts.sum() * d0]])
        F1[:R, 0] = 0.0
        F23 = np.vstack([E, E, [d0]])
        return F1, F23, F23

    routes = [("expsum_r8", lambda: sq.sq_precond_setup(N, 8)),
              ("lemma_split_r8", lambda: sq.sq_precond_setup_canonical(N, *split_factors(sq.sq_precond_setup(N, 8), 8))),
              ("tucker_r8", lambda: sq.sq_precond_setup_tucker(N, 8, 0.0)),
              ("tucker_r10_tol1e-4", lambda: sq.sq_precond_setup_tucker(N, 10, 1e-4)),
              ("tucker_r12", lambda: sq.sq_precond_setup_tucker(N, 12, 0.0))]
    res = {}
    for name, make in routes:
        t0 = time.perf_counter()
        pc = make()
        setup_s = time.perf_counter() - t0
        R, err = sq.sq_precond_info(pc)
        sq.sq_pcg_solve(c, pc, w, 0, 1e-8, 2000, sq.SQ_FP64, None, psi)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [sq.sq_pcg_solve(c, pc, w, i, 1e-8, 2000, sq.SQ_FP64, None, psi) for i in range(3)]
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res[name] = {"rank": R, "max_rel_err": float(f"{err:.4g}"), "setup_s": round(setup_s, 3),
                     "iters_mean": round(float(np.mean([i["iters"] for i in infos])), 1),
                     "solves_per_s": round(3 / t, 3), "converged": all(i["status"] == sq.SQ_OK for i in infos)}
    return res


def run_2d_table(sq, torch, stream):
    """The paper's 2D experiment (Sec. 5, its tables of 2D solve times): n0 = 4
    grid intervals per cell, alpha = 1/4 inclusions (a centred 2 x 2 voxel
    square per cell), lambda = 0.4 (a in {0.4, 1.0}), Bernoulli(1/2) cells,
    L = 64 .. 512 (N = 256 .. 2048), FP64 PCG to 1e-8 with the exact and the
    rank-8 preconditioner, both correctors + A_hom of one realization (seed
    0). Per L: ms per corrector solve, iterations, and A_hom[0, 0]."""
    import numpy as np

    res = {}
    for L in (64, 128, 256, 512):
        n = 4
        N = L * n
        c = sq.sq2d_build_coeffs(L, n, 0, 0.5, 0.4, 1.0)
        sq.sq2d_coeffs_set_subcell(c, 2)
        w = sq.sq2d_workspace_create(N)
        psis = [torch.empty(N * N, dtype=torch.float64, device="cuda") for _ in range(2)]
        row = {}
        for rank in (0, 8):
            pc = sq.sq2d_precond_setup(N, rank)
            sq.sq2d_pcg_solve(c, pc, w, 0, 1e-8, 3000, psis[0])  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = [sq.sq2d_pcg_solve(c, pc, w, i, 1e-8, 3000, psis[i]) for i in range(2)]
            H, _ = sq.sq2d_homogenized_matrix(c, *psis)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[f"rank{rank}"] = {"ms_per_solve": round(ms / 2, 3), "iters": [i["iters"] for i in infos],
                                  "converged": all(i["status"] == sq.SQ_OK for i in infos),
                                  "A_hom_00": round(float(H[0, 0]), 6)}
        res[f"L{L}_N{N}"] = row
    return res


def run_refine_n512(sq, torch, stream, hbm_gbs):
    """L=64, n=8 (N=512, 134 M unknowns), Bernoulli(1/2) on {1,100}, three
    correctors: FP32 PCG inside FP64 refinement to rel. residual 1e-10, exact
    and rank-8 preconditioners (one realization, seed 0)."""
    from paper_2007_06524_gb300 import autotune, workloads

    wl = workloads.REFINE_N512
    L, n = wl["L"], wl["n"]
    N = L * n
    autotune.tune(torch, N, L, n, cache=None)
    c = sq.sq_build_coeffs(L, n, 0, wl["p_hi"], wl["a_lo"], wl["a_hi"])
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    res = {}
    for rank in wl["ranks"]:
        pc = sq.sq_precond_setup(N, rank)
        sq.sq_pcg_solve(c, pc, w, 0, wl["tol"], 4000, sq.SQ_FP32_REFINE, None, psi)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [sq.sq_pcg_solve(c, pc, w, i, wl["tol"], 4000, sq.SQ_FP32_REFINE, None, psi) for i in range(3)]
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res[f"rank{rank}"] = {"solves_per_s": round(3 / t, 3), "iters_mean": round(statistics.mean(i["iters"] for i in infos), 1),
                              "outer_steps": [i["outer_steps"] for i in infos],
                              "relres_true_max": max(i["relres_true"] for i in infos),
                              "converged": all(i["status"] == sq.SQ_OK for i in infos),
                              "iteration_slope": iteration_by_slope(sq, torch, c, pc, w, N, stream,
                                                                    hbm_gbs, reps=3)}
        del pc
    return res


def iteration_by_slope(sq, torch, c, pc, w, N, stream, hbm_gbs, Ks=(4, 8, 12, 16, 20), reps=5):
    """The FP32 PCG iteration as solves run it (graph-replayed, the gaps
    between kernels included), event-timed: FP32-refinement solves capped at
    K inner iterations (tol 1e-30, so the cap ends the first inner solve, all
    K iterations in one inner PCG), timed for several K; the slope of the
    median times is one iteration. The per-kernel event pairs of the
    profiled run time each launch with its own start and drain, so their sum
    reads a few us per kernel above this."""
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    ts = []
    for K in Ks:
        sq.sq_pcg_solve(c, pc, w, 0, 1e-30, K, sq.SQ_FP32_REFINE, None, psi)  # warm (graph capture)
        rt = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf = sq.sq_pcg_solve(c, pc, w, 0, 1e-30, K, sq.SQ_FP32_REFINE, None, psi)
            e1.record(stream)
            torch.cuda.synchronize()
            if inf["iters"] != K:
                return None  # the inner solve converged before the cap: no clean slope
            rt.append(e0.elapsed_time(e1))
        ts.append(statistics.median(rt))
    return slope_fit(Ks, ts, N, hbm_gbs)


def slope_fit(Ks, ts_ms, N, hbm_gbs):
    """One FP32 iteration from solve times t(K) (ms) capped at K iterations:
    the least-squares slope, its worst fit residual, and the 17 field passes
    of 4-byte words it moves against the HBM peak."""
    import numpy as np

    slope, icpt = np.polyfit(list(Ks), list(ts_ms), 1)
    resid = max(abs(t - (slope * k + icpt)) for k, t in zip(Ks, ts_ms))
    b = 17 * 4 * N ** 3
    gbps = b / (slope * 1e-3) / 1e9
    return {"us": round(slope * 1e3, 1), "fit_residual_us": round(resid * 1e3, 1), "bytes": b,
            "GBps": round(gbps, 1), "frac": round(gbps / hbm_gbs, 4), "Ks": list(Ks)}


def _oracle_precond(N, R, workers):
    """The oracle's preconditioner with the same construction as the GPU path
    (the exact diagonal, or the least-squares exponential sum), its FFTs on
    `workers` threads."""
    from oracle import precond

    G = precond.core_tensor_exact(N) if R == 0 else precond.core_tensor_from_nodes(N, *precond.lsq_nodes(N, R))
    return lambda r: precond.apply_precond(G, r.reshape(N, N, N), workers).ravel()


def _oracle_iterations(R, workers):
    """The oracle's own PCG iteration count on this workload's cells at a size
    it solves in seconds: L = 8, n = 8 (N = 64), Bernoulli(1/2) on {1,100},
    seed 0, e_1, tol 1e-8 (counts are nearly flat in N, Lemma 4.1)."""
    from oracle import pcg, problem

    re = problem.realization(8, 8, 0, 1.0, 100.0)
    _, it, _ = pcg.pcg(re.A, re.b[0], _oracle_precond(re.N, R, workers), tol=1e-8)
    return it


def _oracle_sample(R, workers, n_iter_sample=3):
    """Times the oracle (FP64 scipy CSR SpMV + scipy.fft PCG on `workers`
    threads) on one N=256 realization: assembly + RHS, then `n_iter_sample`
    PCG iterations of e_1; a solve is the oracle's own iteration count at
    N = 64 (see _oracle_iterations) plus one preconditioner apply."""
    from oracle import pcg, problem
    from paper_2007_06524_gb300 import workloads

    wl = workloads.PLAIN_N256
    its = _oracle_iterations(R, workers)
    t0 = time.perf_counter()
    re = problem.realization(wl["L"], wl["n"], 0, wl["a_lo"], wl["a_hi"])
    t_setup = time.perf_counter() - t0
    P = _oracle_precond(re.N, R, workers)
    t0 = time.perf_counter()
    pcg.pcg(re.A, re.b[0], P, tol=1e-30, maxit=n_iter_sample)
    t_it = (time.perf_counter() - t0) / (n_iter_sample + 1)  # + initial preconditioner apply
    t_solve = t_setup / 3.0 + (its + 1) * t_it
    return t_setup, t_it, t_solve, its


def _host_cpu(cpuinfo="/proc/cpuinfo"):
    """CPU model of this host (x86 'model name', else the Arm implementer/part
    codes) and the cores this process may use."""
    info = {}
    try:
        with open(cpuinfo) as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip().lower(), v.strip()
                if v and k in ("model name", "cpu implementer", "cpu part") and k not in info:
                    info[k] = v
    except OSError:
        pass
    if "model name" in info:
        model = info["model name"]
    elif "cpu part" in info:
        model = f"{platform.machine()} (CPU implementer {info.get('cpu implementer', '?')}, part {info['cpu part']})"
    else:
        model = platform.machine()
    return {"cpu_model": model, "cores_available": len(os.sched_getaffinity(0))}


def cpu_baseline(R):
    workers = len(os.sched_getaffinity(0))
    t_setup, t_it, t_solve, its = _oracle_sample(R, workers)
    return {"value": round(1.0 / t_solve, 6), "unit": UNIT, "cores": workers, "kind": "oracle", **_host_cpu(),
            "sample": f"oracle at N=256 (L=32, n=8, seed 0): assembly+RHS {t_setup:.1f} s (shared by 3 correctors) "
                      f"+ {t_it:.2f} s per PCG iteration (rank-{R}), measured on 3 iterations, times the oracle's "
                      f"own {its} iterations (its PCG at N=64, same cells and tolerance); FFTs on {workers} threads "
                      f"(scipy.fft), CSR SpMV single-threaded"}


def run_reference(args):
    """The oracle as the reference arm, on this arm's workload and metric:
    each step times one oracle PCG iteration at N = 256; a solve is the
    oracle's own iteration count at N = 64 plus the assembly's share."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import pcg, problem
    from paper_2007_06524_gb300 import workloads

    wl = workloads.PLAIN_N256
    R = args.rank
    workers = len(os.sched_getaffinity(0))
    its = _oracle_iterations(R, workers)
    t0 = time.perf_counter()
    re = problem.realization(wl["L"], wl["n"], 0, wl["a_lo"], wl["a_hi"])
    t_setup = time.perf_counter() - t0
    P = _oracle_precond(re.N, R, workers)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pcg.pcg(re.A, re.b[k % 3], P, tol=1e-30, maxit=1)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt / 2)  # one preconditioner apply before + one PCG iteration
    t_it = statistics.mean(times)
    t_solve = t_setup / 3.0 + (its + 1) * t_it
    value = 1.0 / t_solve
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_it * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(args, _dist()[0]),
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": workers, "kind": "oracle", **_host_cpu(),
                            "sample": f"step = one PCG iteration of the oracle at N=256 ({t_it:.2f} s; FFTs on "
                                      f"{workers} threads, CSR SpMV single-threaded); assembly {t_setup:.1f} s "
                                      f"once; a solve = the oracle's own {its} iterations (its PCG at N=64, same "
                                      f"cells and tolerance)"},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--rank", type=int, default=8, help="preconditioner rank (0 = exact Fourier diagonal)")
    ap.add_argument("--precision", choices=["fp64", "fp32_refine"], default="fp64")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variants", default=None,
                    help="comma-separated subset of the variant legs to run (default: all), e.g. batch_768_mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the PCG iterations' kernels one by one instead of replaying iteration graphs "
                         "(same kernels; for profiling tools)")
    ap.add_argument("--tiles", default=None,
                    help="fixed FP32 tile shape 'P,planes,rows[,Pe]' (Hartley pencils, operator planes per item, "
                         "operator rows per thread, pencils of the last pass of an iteration) instead of the autotuner")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
