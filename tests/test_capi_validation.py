"""CPU-side checks of the C ABI's argument validation: every call here passes
an argument the library must reject before it touches the GPU (bad grid
size, rank, probability, coefficient, tolerance, precision or option), so
the status comes back as SQ_EINVAL with no device present. Grid sizes are
checked against the rule stated in include/sq.h (even, 8 <= N <= 512 in 3D
and <= 2048 in 2D, of the form 2^a or 2^a * 3), enumerated here."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def sq():
    from paper_2007_06524_gb300 import build

    build.build()
    import paper_2007_06524_gb300 as pkg

    return pkg


# Entry points that take a stream get the null stream (0), so that the binding
# does not ask torch for the current CUDA stream on a machine without a GPU.
def _einval(sq, fn, *args):
    with pytest.raises(sq.SqError) as e:
        fn(*args)
    assert e.value.status == sq.SQ_EINVAL, str(e.value)


def _supported(N, nmax):
    if N < 8 or N > nmax or N % 2:
        return False
    m = N
    while m % 2 == 0:
        m //= 2
    return m in (1, 3)


def test_supported_grid_sizes_rule():
    ok = [N for N in range(1, 600) if _supported(N, 512)]
    assert ok == [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]


@pytest.mark.parametrize("N", [0, 4, 6, 7, 9, 10, 18, 20, 36, 40, 72, 100, 144, 510, 514, 768, 1024])
def test_unsupported_grid_sizes_rejected(sq, N):
    assert not _supported(N, 512)
    _einval(sq, sq.sq_precond_setup, N, 0)
    _einval(sq, sq.sq_precond_setup, N, 8)
    _einval(sq, sq.sq_workspace_create, N, sq.SQ_FP64)
    _einval(sq, sq.sq_workspace_create, N, sq.SQ_FP32_REFINE)
    _einval(sq, sq.sq_precond_setup_tucker, N, 4, 0.0)
    if N > 0 and N % 4 == 0:
        _einval(sq, sq.sq_build_coeffs, N // 4, 4, 0, 0.5, 1.0, 10.0, 0)
    if not _supported(N, 2048):
        _einval(sq, sq.sq2d_precond_setup, N, 0)
        _einval(sq, sq.sq2d_workspace_create, N)


def test_unsupported_2d_grid_sizes_rejected(sq):
    for N in (2050, 3072, 4096, 6144):
        assert not _supported(N, 2048)
        _einval(sq, sq.sq2d_precond_setup, N, 0)
        _einval(sq, sq.sq2d_workspace_create, N)
        if N % 4 == 0:  # L n = N with n = 4
            _einval(sq, sq.sq2d_build_coeffs, N // 4, 4, 0, 0.5, 1.0, 10.0, 0)


@pytest.mark.parametrize("rank", [-1, 1, 65, 1000])
def test_exponential_sum_rank_range(sq, rank):
    # rank 0 (exact) or 2..64 terms; 1 term cannot fit 1/x
    _einval(sq, sq.sq_precond_setup, 64, rank)
    _einval(sq, sq.sq2d_precond_setup, 64, rank)


def test_workspace_precision(sq):
    for prec in (-1, 2, 7):
        _einval(sq, sq.sq_workspace_create, 64, prec)


@pytest.mark.parametrize("args", [
    (0, 4, 0.5, 1.0, 10.0),            # L < 1
    (8, 1, 0.5, 1.0, 10.0),            # n < 2
    (8, 4, -0.1, 1.0, 10.0),           # p_hi outside [0, 1]
    (8, 4, 1.5, 1.0, 10.0),
    (8, 4, math.nan, 1.0, 10.0),
    (8, 4, 0.5, 0.0, 10.0),            # coefficients must be positive and finite
    (8, 4, 0.5, 1.0, -2.0),
    (8, 4, 0.5, math.inf, 10.0),
    (8, 4, 0.5, 1.0, math.nan),
])
def test_build_coeffs_arguments(sq, args):
    L, n, p, lo, hi = args
    _einval(sq, sq.sq_build_coeffs, L, n, 0, p, lo, hi, 0)
    _einval(sq, sq.sq2d_build_coeffs, L, n, 0, p, lo, hi, 0)


def test_level_media_arguments(sq):
    # probabilities must lie in [0, 1] and sum to 1; values positive and finite
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [0.5, 0.6], [1.0, 10.0], 0)
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [1.2, -0.2], [1.0, 10.0], 0)
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [0.5, 0.5], [1.0, 0.0], 0)
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [0.5, 0.5], [1.0, math.inf], 0)
    # every value is checked before anything is allocated, the upper levels too
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [0.4, 0.3, 0.3], [1.0, 10.0, -5.0], 0)
    _einval(sq, sq.sq_build_coeffs_levels, 8, 4, 0, [0.4, 0.2, 0.2, 0.2], [1.0, 10.0, 20.0, math.nan], 0)
    lv = np.zeros(8 ** 3, dtype=np.uint8)
    _einval(sq, sq.sq_coeffs_from_host_levels, 8, 4, lv, [1.0, 10.0, 0.0], 0)
    _einval(sq, sq.sq_coeffs_from_host_levels, 8, 4, lv, [1.0, math.inf, 3.0], 0)
    with pytest.raises(ValueError):  # 2 to 4 levels, checked by the binding
        sq.sq_build_coeffs_levels(8, 4, 0, [1.0], [1.0])
    with pytest.raises(ValueError):
        sq.sq_build_coeffs_levels(8, 4, 0, [0.2] * 5, [1.0] * 5)


def test_tucker_route_arguments(sq):
    N = 64
    M = N // 2 + 1
    for r, tol in ((0, 0.0), (-3, 0.0), (M + 1, 0.0), (65, 0.0), (4, -1e-3), (4, 1.0), (4, math.nan)):
        _einval(sq, sq.sq_precond_setup_tucker, N, r, tol)


def test_canonical_factors_must_be_even(sq):
    # every factor row f(k) must equal f(N - k): the multiplier is applied on
    # the half spectrum [0, N/2] of each axis
    N, R = 32, 3
    m = np.minimum(np.arange(N), N - np.arange(N))  # f(k) = g(min(k, N - k)): exactly even
    even = np.stack([np.cos(2 * np.pi * (r + 1) * m / N) + 2.0 for r in range(R)])
    odd = even.copy()
    odd[1, 3] += 0.5
    _einval(sq, sq.sq_precond_setup_canonical, N, odd)
    _einval(sq, sq.sq_precond_setup_canonical, N, even, odd)
    _einval(sq, sq.sq_precond_setup_canonical, N, even, None, odd)
    _einval(sq, sq.sq_precond_setup_canonical, 30, np.ones((R, 30)))  # unsupported N
    with pytest.raises(ValueError):  # shapes checked by the binding
        sq.sq_precond_setup_canonical(N, even, np.ones((R + 1, N)))


def test_options_ranges_and_defaults(sq):
    try:
        for key, bad in ((sq.SQ_OPT_STRIDED_TWO_STAGE, (-1, 3)), (sq.SQ_OPT_STENCIL_ROWS, (-1, 3, 5, 16)),
                         (sq.SQ_OPT_INNER_TOL_EXP, (0, 1, 8, 12))):
            for v in bad:
                _einval(sq, sq.sq_set_option, key, v)
        for v in (0, 1, 2):
            sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, v)
        for v in (0, 1, 2, 4, 8):
            sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, v)
        for v in range(2, 8):
            sq.sq_set_option(sq.SQ_OPT_INNER_TOL_EXP, v)
        for key in (0, 8, 99):
            _einval(sq, sq.sq_set_option, key, 1)
        for v in (0, 1):
            sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, v)
        for v in (-1, 2):
            _einval(sq, sq.sq_set_option, sq.SQ_OPT_PCG_GRAPHS, v)
        for v in (0, 2, 4, 1):
            sq.sq_set_option(sq.SQ_OPT_CONV_TC, v)
        for v in (-1, 3, 8):
            _einval(sq, sq.sq_set_option, sq.SQ_OPT_CONV_TC, v)
        for v in (-1, 2):
            _einval(sq, sq.sq_set_option, sq.SQ_OPT_MULTIPLIER_TABLE, v)
    finally:  # the documented defaults
        sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, 1)
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, 0)
        sq.sq_set_option(sq.SQ_OPT_INNER_TOL_EXP, 5)
        sq.sq_set_option(sq.SQ_OPT_MULTIPLIER_TABLE, 1)
        sq.sq_set_option(sq.SQ_OPT_CONV_TC, 1)
        sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, 1)


def test_tile_overrides_reject_bad_entries(sq):
    try:
        _einval(sq, sq.sq_set_tiles, [(100, 8, 0)])      # unsupported N
        _einval(sq, sq.sq_set_tiles, [(64, 5, 0)])       # pencils: a power of two dividing N / 2
        _einval(sq, sq.sq_set_tiles, [(64, 0, 0, 3)])    # rows per thread: 1, 2, 4 or 8
        with pytest.raises(ValueError):
            sq.sq_set_tiles([(64, 8)])
    finally:
        sq.sq_set_tiles([])


def test_status_strings(sq):
    codes = (sq.SQ_OK, sq.SQ_EINVAL, sq.SQ_ENOMEM, sq.SQ_ECUDA, sq.SQ_ENOCONV, sq.SQ_ETIMEOUT, sq.SQ_EBADGUESS)
    names = [sq.sq_strerror(c) for c in codes]
    assert all(names) and len(set(names)) == len(names)
    assert sq.sq_strerror(99) and sq.sq_strerror(99) not in names[1:]


@pytest.mark.parametrize("a_lo,a_hi", [(float("inf"), 10.0), (1.0, float("inf")), (float("nan"), 1.0), (0.0, 1.0),
                                       (1.0, -2.0)])
def test_noalloc_rejects_bad_coefficients(sq, a_lo, a_hi):
    """The allocation-free A_hom checks its coefficients like sq_build_coeffs
    (finite and positive) before it looks at the device. The pointers are
    never dereferenced on a rejected call, so placeholders stand in for them."""
    import ctypes as C

    lib = sq.load_library()
    ptr = C.c_void_p(256)
    st = lib.sq_homogenized_matrix_noalloc(4, 4, ptr, C.c_double(a_lo), C.c_double(a_hi), ptr, ptr, ptr, ptr,
                                           C.c_void_p(0))
    assert st == sq.SQ_EINVAL


def test_wait_polls_option_range(sq):
    """SQ_OPT_WAIT_POLLS accepts 0 .. 2^24 and restores its default."""
    for bad in (-1, (1 << 24) + 1):
        _einval(sq, sq.sq_set_option, sq.SQ_OPT_WAIT_POLLS, bad)
    for ok in (0, 1, 1 << 24, 1 << 22):
        sq.sq_set_option(sq.SQ_OPT_WAIT_POLLS, ok)


def test_pass_e_tile_override(sq):
    """dht_pencils_e: a power of two with 2 P dividing N (0 = as dht_pencils)."""
    try:
        _einval(sq, sq.sq_set_tiles, [(64, 16, 0, 0, 5)])
        _einval(sq, sq.sq_set_tiles, [(48, 16, 0, 0, 32)])
        sq.sq_set_tiles([(64, 16, 0, 0, 8)])
        sq.sq_set_tiles([(256, 16, 0, 8, 0)])
        with pytest.raises(ValueError):
            sq.sq_set_tiles([(64, 16, 0, 0, 8, 1)])
    finally:
        sq.sq_set_tiles([])
