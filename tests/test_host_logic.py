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
