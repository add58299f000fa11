"""Learned warm start: the conv net kernels against a plain PyTorch FP32
reference of the same ops (periodic 3x3x3 convolutions, GELU), with the BF16
roundings of the kernels emulated; then the warm start inside the solver."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_NET = 32


@pytest.fixture(scope="module")
def sq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2007_06524_gb300 as pkg

    return pkg


def _layers():
    cin = [1, 32, 32, 32, 32, 32]
    cout = [32, 32, 32, 32, 32, 3]
    offs, o = [], 0
    for ci, co in zip(cin, cout):
        offs.append((o, o + 27 * ci * co, ci, co))
        o += 27 * ci * co + co
    return offs, o


def _bf16(x):
    import torch

    return x + (x.to(torch.bfloat16).to(torch.float32) - x).detach()


def _reference(params, feats, out_scale):
    """feats: (B,1,N,N,N) float32 -> (B,3,N,N,N); params: torch tensor (requires_grad ok)."""
    import torch
    import torch.nn.functional as F

    offs, _ = _layers()
    x = feats
    for l, (wo, bo, ci, co) in enumerate(offs):
        W = params[wo:wo + 27 * ci * co].reshape(3, 3, 3, co, ci).permute(3, 4, 0, 1, 2)
        if l > 0:
            W = _bf16(W)
        b = params[bo:bo + co]
        z = F.conv3d(F.pad(x, (1, 1, 1, 1, 1, 1), mode="circular"), W) + b[None, :, None, None, None]
        if l < 5:
            x = _bf16(F.gelu(z))
        else:
            return out_scale * z


def _features(sq, c, L, n):
    ph, _ = sq.sq_coeffs_cells(c)
    V = np.repeat(np.repeat(np.repeat(ph, n, 0), n, 1), n, 2)
    return np.where(V > 0, 1.0, -1.0).astype(np.float32)


def test_forward_matches_reference(sq):
    import torch

    L, n = 8, 4
    net = sq.sq_net_create(N_NET, 2, seed=7, out_scale=1.5)
    p = sq.sq_net_params(net)
    # bring the output layer to full scale so every layer matters
    offs, _ = _layers()
    wo, bo, ci, co = offs[5]
    p[wo:bo] *= 10.0
    p[bo:bo + co] = [0.1, -0.2, 0.3]
    sq.sq_net_set_params(net, p)
    c = sq.sq_build_coeffs(L, n, 11, 0.5, 1.0, 10.0)
    outs = [torch.empty(N_NET ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    sq.sq_net_predict(net, c, *outs)
    torch.cuda.synchronize()
    got = np.stack([o.cpu().numpy().reshape(N_NET, N_NET, N_NET) for o in outs])
    f = torch.from_numpy(_features(sq, c, L, n))[None, None]
    ref = _reference(torch.from_numpy(p), f, 1.5)[0].detach().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-2, err


@pytest.mark.parametrize("N,L,seeds", [(N_NET, 8, (21, 22)), (96, 24, (23,))])
def test_gradients_match_reference(sq, N, L, seeds):
    """Every weight and bias gradient of a training step against autograd of
    the reference. N = 96: the weight-gradient chunks (about 8192 voxels) must
    be whole 4-row tiles, 4 N = 384 voxels, which 8192 is not."""
    import torch

    n = 4
    B = len(seeds)
    net = sq.sq_net_create(N, B, seed=3, out_scale=2.0)
    p = sq.sq_net_params(net)
    offs, _ = _layers()
    wo, bo, ci, co = offs[5]
    p[wo:bo] *= 10.0
    sq.sq_net_set_params(net, p)
    cs = [sq.sq_build_coeffs(L, n, s, 0.5, 1.0, 10.0) for s in seeds]
    rng = np.random.default_rng(0)
    tg = [[torch.from_numpy(rng.standard_normal(N ** 3)).cuda() for _ in range(3)] for _ in cs]
    loss = sq.sq_net_train_step(net, cs, tg, 1e-3, loss_type=0)
    g_gpu = sq.sq_net_grads(net).astype(np.float64)
    P = torch.from_numpy(p).requires_grad_(True)
    feats = torch.from_numpy(np.stack([_features(sq, c, L, n) for c in cs]))[:, None]
    y = _reference(P, feats, 2.0)
    t = torch.from_numpy(np.stack([np.stack([x.cpu().numpy().reshape(N, N, N) for x in tri])
                                   for tri in tg]).astype(np.float32))
    lref = (((y - t) / 2.0) ** 2).sum()
    lref.backward()
    g_ref = P.grad.numpy().astype(np.float64)
    assert np.isfinite(g_gpu).all()
    assert abs(loss - lref.item() / (3 * B * N ** 3)) <= 1e-3 * abs(loss)
    for l, (wo, bo, ci, co) in enumerate(offs):
        for a, b in ((wo, bo), (bo, bo + co)):
            e = np.linalg.norm(g_gpu[a:b] - g_ref[a:b]) / max(np.linalg.norm(g_ref[a:b]), 1e-30)
            assert e <= 5e-2, (l, a == bo, e)


def test_training_and_warm_start_guess_handling(sq):
    import torch

    L, n = 8, 4
    N = L * n
    pc = sq.sq_precond_setup(N, 0)
    seeds = list(range(100, 108))
    cs = [sq.sq_build_coeffs(L, n, s, 0.5, 1.0, 10.0) for s in seeds]
    tg = [[torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)] for _ in cs]
    b = sq.sq_batch_create([(c, i, tg[k][i]) for k, c in enumerate(cs) for i in range(3)], [pc] * 24)
    sq.sq_pcg_solve_batched(b, 1e-10, 2000)
    scale = float(torch.stack([t.std() for tri in tg for t in tri]).mean())
    net = sq.sq_net_create(N, 4, seed=1, out_scale=scale)
    losses = []
    for step in range(120):
        k = (4 * step) % len(cs)
        losses.append(sq.sq_net_train_step(net, cs[k:k + 4], tg[k:k + 4], 3e-3, loss_type=1))
    assert np.mean(losses[-8:]) < 0.5 * np.mean(losses[:4]), (losses[:4], losses[-8:])
    # warm start on a training realization: the guess lowers the initial
    # residual (so the solver keeps it) and the solve reaches the same corrector
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    sq.sq_net_predict(net, cs[0], *g)
    bvec = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    Ag = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    for i in range(3):
        sq.sq_rhs(cs[0], i, bvec)
        sq.sq_apply_operator(cs[0], g[i], Ag)
        rel0 = float(torch.linalg.norm(bvec - Ag) / torch.linalg.norm(bvec))
        assert rel0 < 1.0, rel0
        psi0 = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        psiw = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        i0 = sq.sq_pcg_solve(cs[0], pc, w, i, 1e-8, 2000, sq.SQ_FP32_REFINE, None, psi0)
        iw = sq.sq_pcg_solve(cs[0], pc, w, i, 1e-8, 2000, sq.SQ_FP32_REFINE, g[i], psiw)
        assert iw["status"] == sq.SQ_OK and iw["used_guess"] == 1 and iw["relres_true"] <= 1e-8
        assert float(torch.linalg.norm(psiw - psi0) / torch.linalg.norm(psi0)) <= 1e-5
    # a useless guess is rejected by its residual and the solve starts from zero
    bad = torch.from_numpy(1e3 * np.random.default_rng(1).standard_normal(N ** 3)).cuda()
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    ib = sq.sq_pcg_solve(cs[1], pc, w, 0, 1e-8, 2000, sq.SQ_FP32_REFINE, bad, psi)
    assert ib["used_guess"] == 0 and ib["status"] == sq.SQ_OK
    wf = sq.sq_workspace_create(N, sq.SQ_FP64)
    ib = sq.sq_pcg_solve(cs[1], pc, wf, 0, 1e-8, 2000, sq.SQ_FP64, bad, psi)
    assert ib["used_guess"] == 0 and ib["status"] == sq.SQ_OK


def test_energy_loss_value_matches_oracle_operator(sq):
    """loss_type 1 reports mean(e . A e) with e = (prediction - target)/out_scale;
    checked with the oracle's matrix-free operator on the same fields."""
    import torch

    from oracle import assembly, rng

    L, n, seed = 8, 4, 31
    N = L * n
    scale = 1.7
    net = sq.sq_net_create(N, 1, seed=5, out_scale=scale)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 10.0)
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    sq.sq_net_predict(net, c, *g)
    tg = [torch.from_numpy(np.random.default_rng(i).standard_normal(N ** 3)).cuda() for i in range(3)]
    loss = sq.sq_net_train_step(net, [c], [tg], 1e-4, loss_type=1)
    a = assembly.edge_coefficients(rng.cell_values(rng.cell_phases(L, seed), 1.0, 10.0), n)
    ref = 0.0
    for i in range(3):
        e = ((g[i].cpu().numpy() - tg[i].cpu().numpy()) / scale).reshape(N, N, N)
        ref += float(np.sum(e * assembly.apply_stencil(a, e)))
    ref /= 3 * N ** 3
    assert abs(loss - ref) <= 1e-2 * abs(ref), (loss, ref)


def test_residual_loss_value_matches_oracle_operator(sq):
    """loss_type 2 reports mean(r . r) with r = (A prediction - b_i)/out_scale,
    the residual norm of the guess (targets not read); checked with the
    oracle's operator and right-hand sides. One training step with it moves
    the weights."""
    import torch

    from oracle import assembly, rng

    L, n, seed = 8, 4, 32
    N = L * n
    scale = 1.3
    net = sq.sq_net_create(N, 1, seed=9, out_scale=scale)
    p0 = sq.sq_net_params(net)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 10.0)
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    sq.sq_net_predict(net, c, *g)
    dummy = [torch.zeros(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    loss = sq.sq_net_train_step(net, [c], [dummy], 1e-3, loss_type=2)
    a = assembly.edge_coefficients(rng.cell_values(rng.cell_phases(L, seed), 1.0, 10.0), n)
    ref = 0.0
    for i in range(3):
        y = g[i].cpu().numpy().reshape(N, N, N)
        r = (assembly.apply_stencil(a, y).ravel() - assembly.rhs(a, i)) / scale
        ref += float(r @ r)
    ref /= 3 * N ** 3
    assert abs(loss - ref) <= 1e-2 * abs(ref), (loss, ref)
    assert np.abs(sq.sq_net_params(net) - p0).max() > 0


@pytest.mark.parametrize("N,L,n", [(32, 8, 4), (64, 16, 4), (96, 24, 4)])
def test_tcgen05_convolutions_match_mma_sync(sq, N, L, n):
    """The 32 -> 32 convolutions on tcgen05 (tensor memory accumulator; tile
    depth 2 and 4, SQ_OPT_CONV_TC = 2 / 4) and on mma.sync (0) take the same
    BF16 inputs: predictions agree to FP32 rounding of the accumulation order,
    and so do the gradients of a training step (forward and data-gradient
    convolutions both switch). N = 96 leaves the CTAs uneven tile counts."""
    import torch

    outs = {}
    for opt in (0, 2, 4):
        try:
            sq.sq_set_option(sq.SQ_OPT_CONV_TC, opt)
            net = sq.sq_net_create(N, 2, seed=13, out_scale=1.2)
            p = sq.sq_net_params(net)
            offs, _ = _layers()
            wo, bo, ci, co = offs[5]
            p[wo:bo] *= 10.0
            sq.sq_net_set_params(net, p)
            c = sq.sq_build_coeffs(L, n, 41, 0.5, 1.0, 10.0)
            g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
            sq.sq_net_predict(net, c, *g)
            cs = [c, sq.sq_build_coeffs(L, n, 42, 0.5, 1.0, 10.0)]
            rng = np.random.default_rng(5)
            tg = [[torch.from_numpy(rng.standard_normal(N ** 3)).cuda() for _ in range(3)] for _ in cs]
            loss = sq.sq_net_train_step(net, cs, tg, 1e-3, loss_type=0)
            outs[opt] = (np.stack([x.cpu().numpy() for x in g]), loss, sq.sq_net_grads(net))
        finally:
            sq.sq_set_option(sq.SQ_OPT_CONV_TC, 1)
    y0, l0, g0 = outs[0]
    g0 = g0.astype(np.float64)  # gradients reach 1e20 at N = 96: their squares overflow FP32
    for opt in (2, 4):
        y1, l1, g1 = outs[opt]
        g1 = g1.astype(np.float64)
        assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) <= 1e-3, opt
        assert abs(l1 - l0) <= 1e-3 * abs(l0), opt
        assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) <= 2e-2, opt


def test_tcgen05_bounded_wait_gives_up_cleanly(sq):
    """SQ_OPT_WAIT_POLLS = 0 makes the tensor-core convolution give up on its
    first MMA-completion wait: it stops issuing, waits for the MMAs it issued,
    frees its tensor memory and the prediction reports SQ_ETIMEOUT; the next
    prediction with the default limit is clean and matches mma.sync."""
    import torch

    N, L, n = 32, 8, 4
    net = sq.sq_net_create(N, 1, seed=2, out_scale=1.0)
    c = sq.sq_build_coeffs(L, n, 3, 0.5, 1.0, 10.0)
    g = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    try:
        sq.sq_set_option(sq.SQ_OPT_WAIT_POLLS, 0)
        with pytest.raises(sq.SqError) as e:
            sq.sq_net_predict(net, c, *g)
        assert e.value.status == sq.SQ_ETIMEOUT
    finally:
        sq.sq_set_option(sq.SQ_OPT_WAIT_POLLS, 1 << 22)
    sq.sq_net_predict(net, c, *g)
    y1 = np.stack([x.cpu().numpy() for x in g])
    try:
        sq.sq_set_option(sq.SQ_OPT_CONV_TC, 0)
        sq.sq_net_predict(net, c, *g)
    finally:
        sq.sq_set_option(sq.SQ_OPT_CONV_TC, 1)
    y0 = np.stack([x.cpu().numpy() for x in g])
    assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) <= 1e-3
