"""Host-side logic that needs no GPU: workload presets, the batch size recipe,
binding argument checks and the committed warm-start weights file."""
import os

import numpy as np
import pytest

from paper_2007_06524_gb300 import workloads


def test_batch_lattice_draw_is_seeded_and_covers_all_sizes():
    idx = [workloads.batch_L_index(s) for s in range(256)]
    assert idx == [workloads.batch_L_index(s) for s in range(256)]
    assert set(idx) == {0, 1, 2, 3}
    Ns = {workloads.BATCH_MIXED["Ls"][i] * workloads.BATCH_MIXED["n"] for i in idx}
    assert Ns == {32, 48, 64, 96}


def test_presets_match_the_measured_configurations():
    assert workloads.PLAIN_N16["L"] * workloads.PLAIN_N16["n"] == 16
    assert workloads.PLAIN_N256["L"] * workloads.PLAIN_N256["n"] == 256
    assert workloads.REFINE_N512["L"] * workloads.REFINE_N512["n"] == 512
    assert workloads.WARM_N64["L"] * workloads.WARM_N64["n"] == 64
    assert len(workloads.WARM_N64["train_seeds"]) == 4096 and len(workloads.WARM_N64["eval_seeds"]) == 512
    assert not set(workloads.WARM_N64["train_seeds"]) & set(workloads.WARM_N64["eval_seeds"])


def test_binding_rejects_bad_buffers_before_calling_the_library():
    torch = pytest.importorskip("torch")
    from paper_2007_06524_gb300 import sq

    with pytest.raises(ValueError):
        sq._ptr(torch.zeros(4, dtype=torch.float64))            # not a CUDA tensor
    with pytest.raises(ValueError):
        sq.sq_coeffs_upload(None, torch.zeros(8, dtype=torch.uint8))   # not pinned


def test_warm_start_weights_file():
    from paper_2007_06524_gb300 import warmstart

    path = warmstart.DEFAULT_WEIGHTS
    assert os.path.exists(path)
    d = np.load(path)
    # 6 layers: 1->32, 4 x 32->32, 32->3, 3x3x3 taps, plus biases
    n = 27 * 1 * 32 + 32 + 4 * (27 * 32 * 32 + 32) + 27 * 32 * 3 + 3
    assert d["params"].shape == (n,) and d["params"].dtype == np.float32
    assert int(d["N"]) == 64 and float(d["scale"]) > 0
    assert np.all(np.isfinite(d["params"]))


def test_bench_algorithmic_model():
    import bench

    N, R = 256, 8
    alg = bench._algorithmic(N, 4, R)
    n3 = N ** 3
    # the fused iteration moves 17 field passes of 4-byte words
    assert sum(b for b, _ in alg.values()) + alg["dht_x2"][0] == 17 * 4 * n3
    # pass C: two transforms without combines, scaling and r.z; the multiplier
    # is a table lookup at N <= 256 (except FP32 exact), else the rank-R sum or
    # the exact 1/x
    assert alg["dht_x1_scale"][1] == (2 * 2.5 * 8 + 6) * n3
    assert bench._algorithmic(N, 8, R)["dht_x1_scale"][1] == (2 * 2.5 * 8 + 6) * n3
    assert bench._algorithmic(N, 4, 0)["dht_x1_scale"][1] == (2 * 2.5 * 8 + 10) * n3
    assert bench._algorithmic(N, 8, R, table=False)["dht_x1_scale"][1] == (2 * 2.5 * 8 + 2 * R + 6) * n3
    assert bench._algorithmic(N, 8, 0, table=False)["dht_x1_scale"][1] == (2 * 2.5 * 8 + 10) * n3
    assert bench._algorithmic(512, 4, 0)["dht_x1_scale"][1] == (2 * 2.5 * 9 + 10) * 512 ** 3
    # the x2 passes: a Hartley transform (FFT + combine) in FP32, the FFT alone
    # on the FP64 complex route
    assert alg["dht_x2"][1] == (2.5 * 8 + 3) * n3
    assert bench._algorithmic(N, 8, R)["dht_x2"][1] == 2.5 * 8 * n3


def test_new_bindings_reject_bad_arguments_before_calling_the_library():
    from paper_2007_06524_gb300 import sq

    with pytest.raises(ValueError):
        sq.sq_build_coeffs_levels(4, 8, 0, (0.5, 0.5), (1.0, 2.0, 3.0))   # probs and values differ in length
    with pytest.raises(ValueError):
        sq.sq_coeffs_set_levels(None, (1.0,))                               # fewer than 2 levels
    with pytest.raises(ValueError):
        sq.sq_coeffs_set_levels(None, (1.0,) * 5)                           # more than 4 levels
    with pytest.raises(ValueError):
        sq.sq_coeffs_from_host_levels(4, 8, np.zeros(10, np.uint8), (1.0, 2.0))  # not L^3 bytes
    with pytest.raises(ValueError):
        sq.sq_precond_setup_canonical(32, np.ones((3, 32)), np.ones((4, 32)))     # factor shapes differ
    with pytest.raises(ValueError):
        sq.sq2d_coeffs_from_host(4, 4, np.zeros(15, np.uint8), 1.0, 2.0)         # not L^2 bytes


def test_bench_host_cpu_description(tmp_path):
    import bench

    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Example Xeon 1234\n\n"
                   "processor\t: 1\nmodel name\t: Example Xeon 1234\n")
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU architecture: 8\n"
                   "CPU part\t: 0xd4f\n\nprocessor\t: 1\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    a = bench._host_cpu(str(x86))
    assert a["cpu_model"] == "Example Xeon 1234" and a["cores_available"] >= 1
    b = bench._host_cpu(str(arm))
    assert "implementer 0x41" in b["cpu_model"] and "part 0xd4f" in b["cpu_model"]
    c = bench._host_cpu(str(tmp_path / "missing"))
    assert c["cpu_model"] and c["cores_available"] >= 1


def test_bench_batch_leg_on_fakes(monkeypatch):
    """run_batch end to end against stand-ins for the library, the batch
    autotuner and torch (no GPU): the 768 descriptors, their grid sizes, the
    tuned tiles handed to the batch and the algorithmic traffic."""
    import types

    import bench
    from paper_2007_06524_gb300 import autotune, workloads

    tuned = [(32, 8, 8), (48, 8, 12), (64, 16, 16), (96, 16, 24)]
    monkeypatch.setattr(autotune, "tune_batch", lambda torch, descs, pl, tol: (tuned, {"32:8x8": 1.0}))

    class Buf:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 250.0  # ms

    calls = {}
    fake_sq = types.SimpleNamespace(
        SQ_OK=0,
        sq_build_coeffs=lambda L, n, seed, p, lo, hi: ("coeffs", L, n, seed),
        sq_precond_setup=lambda N, r: ("precond", N, r),
        sq_batch_create=lambda descs, pl, tiles=None: calls.setdefault(tiles is not None, (list(descs), list(pl),
                                                                                          tiles)),
        sq_pcg_solve_batched=lambda b, tol, mi: [{"iters": 20, "status": 0} for _ in b[0]],
        sq_profile_enable=lambda on: None,
        sq_profile_read=lambda: {"batch_inner": (200.0, 600), "batch_inner_loop": (230.0, 3)},
    )
    fake_torch = types.SimpleNamespace(
        float64="f64", empty=lambda n, dtype=None, device=None: Buf(n),
        cuda=types.SimpleNamespace(synchronize=lambda: None, Event=Event))
    out = bench.run_batch(fake_sq, fake_torch, stream=None)
    descs, pl, tiles = calls[True]
    assert tiles == tuned and calls[False][2] is None and out["tiles"] == [list(t) for t in tuned]
    Ns = [workloads.BATCH_MIXED["Ls"][workloads.batch_L_index(s)] * 4 for s in range(256) for _ in range(3)]
    assert out["solves"] == 768 and [p[1] for p in pl] == Ns
    assert [d[2].numel() for d in descs] == [N ** 3 for N in Ns]
    assert out["converged"] and out["iters_p50"] == 20.0 and out["seconds"] == 0.25
    want = sum(17 * 4 * N ** 3 * 20 for N in Ns)
    assert out["algorithmic_bytes"] == want
    assert abs(out["algorithmic_GBps"] - want / 0.25 / 1e9) <= 0.05
    assert 0 < out["hbm_frac"] < 10 and "L2" in out["algorithmic_note"]
    assert out["working_set_GB"] == round(sum(20 * N ** 3 for N in Ns) / 1e9, 2)
    # every fake solve takes 250 ms; the profiled one spends 230 ms in its inner
    # loops, of which 200 ms in kernels: the graph's inner loops take 230 ms
    assert out["inner_loop"]["graph_loop_s"] == 0.23 and out["inner_loop"]["busy_frac"] == round(0.2 / 0.23, 4)


def test_bench_roofline_selection():
    """kernel_table: the dominant class by time, ALU- or HBM-bound by the larger
    fraction, achieved = algorithmic bytes (flops) x working launches / their
    time, and the ncu traffic attached only where a capture of that kernel at
    N = 256 exists."""
    import bench

    N, R = 256, 8
    names = ("stencil_matvec", "dht_x3_in", "dht_x2", "dht_x1_scale", "dht_x3_out")
    # FP64: pass C dominates and is ALU-bound
    us64 = {"stencil_matvec": 262.0, "dht_x3_in": 597.0, "dht_x2": 481.0, "dht_x1_scale": 1103.0, "dht_x3_out": 562.0}
    prof = {k: (us64[k] * 100 / 1e3, 100) for k in names}
    work = {k: (us64[k] * 90 / 1e3, 90) for k in names}
    kernels, roof = bench.kernel_table(work, prof, N, 8, R, t_ms=400.0)
    flops = bench._algorithmic(N, 8, R)["dht_x1_scale"][1]
    assert roof["kernel"] == "dht_x1_scale" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["achieved"] - flops / 1103e-6 / 1e12) <= 1e-3
    assert abs(roof["frac"] - roof["achieved"] / bench.FP64_NOMINAL_TFLOPS) <= 1e-3
    # a measured peak replaces the nominal one
    pk = dict(bench.default_peaks(), fp64_tflops=1.0, fp64_src="measured")
    _, roof_m = bench.kernel_table(work, prof, N, 8, R, t_ms=400.0, peaks=pk)
    assert roof_m["peak"] == 1.0 and roof_m["peak_src"] == "measured"
    assert abs(roof_m["frac"] - roof["achieved"] / 1.0) <= 1e-3 and "hbm_frac" in roof_m
    assert roof["traffic"] == bench.PROFILED_TRAFFIC.get(("dht_x1_scale", 8))
    assert kernels["dht_x2"]["us_per_work_launch"] == 481.0
    # FP32: pass E dominates and is HBM-bound
    us32 = {"stencil_matvec": 41.0, "dht_x3_in": 52.0, "dht_x2": 24.5, "dht_x1_scale": 53.5, "dht_x3_out": 58.8}
    prof = {k: (us32[k] * 100 / 1e3, 100) for k in names}
    work = {k: (us32[k] * 90 / 1e3, 90) for k in names}
    kernels, roof = bench.kernel_table(work, prof, N, 4, R, t_ms=30.0)
    b = bench._algorithmic(N, 4, R)["dht_x3_out"][0]
    assert roof["kernel"] == "dht_x3_out" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["achieved"] - b / 58.8e-6 / 1e9) <= 0.1
    assert roof["traffic"] == bench.PROFILED_TRAFFIC[("dht_x3_out", 4)]
    # no capture at other sizes
    _, roof = bench.kernel_table(work, prof, 128, 4, R, t_ms=30.0)
    assert roof["traffic"] is None


def _complex_x2_route(r, G, scale):
    """The FP64 preconditioner's five passes as numpy array operations: x3
    Hartley transforms (2 H per pass) around an x2 FFT of packed column pairs
    with no Hartley combine, the x1 scaling W = s Z(k) + d conj Z(-k) over
    mirror modes (-k1, -k2) with the multiplier as 8 G, and the inverse x2
    transform read from index N - j. Returns z and the pass-C r.z sum."""
    import numpy as np

    N = r.shape[0]

    def hartley2(x):  # 2 H along x3 (real in, real out)
        F = np.fft.fft(x, axis=2)
        return 2 * (F.real - F.imag)

    Y = hartley2(r)
    Z = np.fft.fft(Y[:, :, 0::2] + 1j * Y[:, :, 1::2], axis=1)
    Z = np.fft.fft(Z, axis=0)
    m = (-np.arange(N)) % N
    Zm = Z[m][:, m]  # Z(-k1, -k2)
    ga, gb = 8 * scale * G[:, :, 0::2], 8 * scale * G[:, :, 1::2]
    s4, d4 = ga + gb, ga - gb
    W = s4 * Z + d4 * np.conj(Zm)
    rz = float(np.sum((np.conj(Z) * W).real))  # Re(conj Z W) summed over every mode
    V = np.conj(np.fft.fft(np.conj(W), axis=0))
    D = np.fft.fft(V, axis=1)[:, m, :]
    Y2 = np.empty_like(Y)
    Y2[:, :, 0::2], Y2[:, :, 1::2] = D.real, D.imag
    return hartley2(Y2), rz


@pytest.mark.parametrize("N", [8, 12, 16])
def test_complex_x2_route_is_the_fourier_multiplier(N):
    """The FP64 route through passes B, C, D applies z = F^-1 G F r for a
    multiplier even in every index, and its r.z sum is r . z (Parseval):
    checked against numpy's 3D FFT for the exact diagonal and a rank-2
    canonical G (Sec. 4.2, Eq. 31 and Eq. 34)."""
    import numpy as np

    rng = np.random.default_rng(N)
    r = rng.standard_normal((N, N, N))
    k = np.arange(N)
    lam = 4 * np.sin(np.pi * k / N) ** 2
    with np.errstate(divide="ignore"):
        exact = 1.0 / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :])
    exact[0, 0, 0] = 0.0
    u = [np.exp(-t * lam) for t in (0.3, 1.7)]
    rank2 = sum(w * ui[:, None, None] * ui[None, :, None] * ui[None, None, :] for w, ui in zip((0.8, 0.5), u))
    rank2[0, 0, 0] = 0.0
    for G in (exact, rank2):
        z, rz = _complex_x2_route(r, G, 1.0 / (64 * N ** 3))
        zref = np.fft.ifftn(G * np.fft.fftn(r)).real
        assert np.abs(z - zref).max() <= 1e-13 * np.abs(zref).max()
        assert abs(rz - float(np.sum(r * zref))) <= 1e-12 * abs(float(np.sum(r * zref)))


def test_bench_slope_fit():
    """The FP32 iteration from capped-solve times: a solve of K iterations
    taking c + K t gives t back whatever the fixed cost c, with the 17 FP32
    field passes of one iteration as its bytes."""
    import bench

    N, t_us, c_ms = 256, 226.0, 1.9
    Ks = (4, 8, 12, 16, 20)
    r = bench.slope_fit(Ks, [c_ms + k * t_us / 1e3 for k in Ks], N, 6690.5)
    assert r["us"] == t_us and r["fit_residual_us"] == 0.0
    assert r["bytes"] == 17 * 4 * N ** 3
    assert abs(r["GBps"] - r["bytes"] / (t_us * 1e-6) / 1e9) < 0.1
    assert abs(r["frac"] - r["GBps"] / 6690.5) < 1e-4
    # a noisy point shows up as the fit residual
    ts = [c_ms + k * t_us / 1e3 for k in Ks]
    ts[2] += 0.005
    assert bench.slope_fit(Ks, ts, N, 6690.5)["fit_residual_us"] > 2.0
