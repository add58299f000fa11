"""ctypes binding of libsq with the C ABI's names (include/sq.h).

Device buffers are torch CUDA tensors (contiguous, float64 unless the call is
an *_f32 one); streams default to torch's current stream. Handles are small
owner objects whose destructor calls the matching sq_*_destroy.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

SQ_OK, SQ_EINVAL, SQ_ENOMEM, SQ_ECUDA, SQ_ENOCONV, SQ_ETIMEOUT, SQ_EBADGUESS = range(7)
SQ_FP64, SQ_FP32_REFINE = 0, 1
SQ_OPT_STRIDED_TWO_STAGE = 1
SQ_OPT_STENCIL_ROWS = 2
SQ_OPT_INNER_TOL_EXP = 3
SQ_OPT_WAIT_POLLS = 4
SQ_OPT_MULTIPLIER_TABLE = 5
SQ_OPT_CONV_TC = 6
SQ_OPT_PCG_GRAPHS = 7

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "libsq.so")


class SqError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {sq_strerror(status)} (status {status})")
        self.status = status


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_steps", C.c_int), ("status", C.c_int), ("used_guess", C.c_int),
                ("relres", C.c_double), ("relres_true", C.c_double)]


class SolveDesc(C.Structure):
    _fields_ = [("coeffs", C.c_void_p), ("dir", C.c_int), ("psi", C.c_void_p)]


class TileConfig(C.Structure):
    _fields_ = [("N", C.c_int), ("dht_pencils", C.c_int), ("stencil_planes", C.c_int), ("stencil_rows", C.c_int),
                ("dht_pencils_e", C.c_int)]


def _tile_array(tl):
    """(N, dht_pencils, stencil_planes[, stencil_rows[, dht_pencils_e]]) tuples
    -> TileConfig array."""
    arr = (TileConfig * max(1, len(tl)))()
    for k, t in enumerate(tl):
        if len(t) not in (3, 4, 5):
            raise ValueError("tile entries are (N, dht_pencils, stencil_planes[, stencil_rows[, dht_pencils_e]])")
        arr[k].N, arr[k].dht_pencils, arr[k].stencil_planes = int(t[0]), int(t[1]), int(t[2])
        arr[k].stencil_rows = int(t[3]) if len(t) >= 4 else 0
        arr[k].dht_pencils_e = int(t[4]) if len(t) == 5 else 0
    return arr


def load_library():
    """Loads libsq.so (built by paper_2007_06524_gb300.build). Raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libsq.so not found at {path}: run paper_2007_06524_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, d, u64, p = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.POINTER
    sig = {
        "sq_build_coeffs": (i, [i, i, u64, d, d, d, vp, p(vp)]),
        "sq_coeffs_from_host": (i, [i, i, vp, d, d, vp, p(vp)]),
        "sq_coeffs_cells": (i, [vp, vp, p(C.c_int64)]),
        "sq_coeffs_regenerate": (i, [vp, u64, d, vp]),
        "sq_coeffs_upload": (i, [vp, vp, vp]),
        "sq_profile_enable": (i, [i]),
        "sq_profile_read": (i, [vp, vp, i]),
        "sq_profile_work": (i, [vp, vp, i]),
        "sq_profile_class_name": (C.c_char_p, [i]),
        "sq_launch_count": (C.c_int64, []),
        "sq_probe_fma": (i, [i, p(d), p(C.c_float), vp]),
        "sq_probe_copy": (i, [vp, vp, C.c_size_t, i, p(d), vp]),
        "sq_coeffs_shape": (i, [vp, p(i), p(i), p(i)]),
        "sq_coeffs_destroy": (None, [vp]),
        "sq_coeffs_set_subcell": (i, [vp, i]),
        "sq_coeffs_set_levels": (i, [vp, i, vp]),
        "sq_build_coeffs_levels": (i, [i, i, u64, i, vp, vp, vp, p(vp)]),
        "sq_coeffs_regenerate_levels": (i, [vp, u64, i, vp, vp]),
        "sq_coeffs_from_host_levels": (i, [i, i, vp, i, vp, vp, p(vp)]),
        "sq_precond_setup": (i, [i, i, p(vp)]),
        "sq_precond_destroy": (None, [vp]),
        "sq_precond_factors": (i, [vp, vp, vp]),
        "sq_precond_setup_canonical": (i, [i, i, vp, vp, vp, p(vp)]),
        "sq_precond_setup_tucker": (i, [i, i, d, p(vp)]),
        "sq_precond_info": (i, [vp, p(i), p(d)]),
        "sq_workspace_create": (i, [i, i, p(vp)]),
        "sq_workspace_destroy": (None, [vp]),
        "sq_pcg_solve": (i, [vp, vp, vp, i, d, i, i, vp, vp, p(SolveInfo), vp]),
        "sq_homogenized_matrix": (i, [vp, vp, vp, vp, vp, vp, vp]),
        "sq_homogenized_matrix_noalloc": (i, [i, i, vp, d, d, vp, vp, vp, vp, vp]),
        "sq_apply_operator": (i, [vp, vp, vp, vp]),
        "sq_apply_operator_f32": (i, [vp, vp, vp, vp]),
        "sq_rhs": (i, [vp, i, vp, vp]),
        "sq_apply_precond": (i, [vp, vp, vp, vp, vp]),
        "sq_apply_precond_f32": (i, [vp, vp, vp, vp, vp]),
        "sq_strerror": (C.c_char_p, [i]),
        "sq_batch_create": (i, [i, p(SolveDesc), p(vp), p(TileConfig), i, p(vp)]),
        "sq_net_create": (i, [i, i, u64, d, p(vp)]),
        "sq_net_destroy": (None, [vp]),
        "sq_net_params": (i, [vp, vp, p(C.c_int64)]),
        "sq_net_set_params": (i, [vp, vp, C.c_int64]),
        "sq_net_grads": (i, [vp, vp, C.c_int64]),
        "sq_net_predict": (i, [vp, vp, vp, vp, vp, vp]),
        "sq_net_train_step": (i, [vp, i, p(vp), p(vp), C.c_float, i, p(d), vp]),
        "sq_batch_destroy": (None, [vp]),
        "sq_pcg_solve_batched": (i, [vp, d, i, p(SolveInfo), vp]),
        "sq_set_tiles": (i, [p(TileConfig), i]),
        "sq_ensemble_ahom": (i, [i, i, vp, i, d, d, d, i, d, i, i, vp, vp, vp, vp, vp]),
        "sq_set_option": (i, [i, i]),
        "sq2d_build_coeffs": (i, [i, i, u64, d, d, d, vp, p(vp)]),
        "sq2d_coeffs_from_host": (i, [i, i, vp, d, d, vp, p(vp)]),
        "sq2d_coeffs_set_subcell": (i, [vp, i]),
        "sq2d_coeffs_cells": (i, [vp, vp]),
        "sq2d_coeffs_destroy": (None, [vp]),
        "sq2d_precond_setup": (i, [i, i, p(vp)]),
        "sq2d_precond_factors": (i, [vp, vp, vp]),
        "sq2d_precond_destroy": (None, [vp]),
        "sq2d_workspace_create": (i, [i, p(vp)]),
        "sq2d_workspace_destroy": (None, [vp]),
        "sq2d_pcg_solve": (i, [vp, vp, vp, i, d, i, vp, p(SolveInfo), vp]),
        "sq2d_homogenized_matrix": (i, [vp, vp, vp, vp, vp]),
        "sq2d_apply_operator": (i, [vp, vp, vp, vp]),
        "sq2d_rhs": (i, [vp, i, vp, vp]),
        "sq2d_apply_precond": (i, [vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def sq_strerror(status: int) -> str:
    return load_library().sq_strerror(int(status)).decode()


def _check(st: int, where: str, allow=()):
    if st != SQ_OK and st not in allow:
        raise SqError(st, where)
    return st


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t, dtype_name="float64"):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor")
    return C.c_void_p(t.data_ptr())


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(load_library(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Coeffs(_Handle):
    _destroy = "sq_coeffs_destroy"


class Precond(_Handle):
    _destroy = "sq_precond_destroy"


class Workspace(_Handle):
    _destroy = "sq_workspace_destroy"


class Net(_Handle):
    _destroy = "sq_net_destroy"


class Coeffs2D(_Handle):
    _destroy = "sq2d_coeffs_destroy"

    def __init__(self, ptr, L):
        super().__init__(ptr)
        self.L = L


class Precond2D(_Handle):
    _destroy = "sq2d_precond_destroy"


class Workspace2D(_Handle):
    _destroy = "sq2d_workspace_destroy"


class Batch(_Handle):
    _destroy = "sq_batch_destroy"

    def __init__(self, ptr, count, keep):
        super().__init__(ptr)
        self.count = count
        self._keep = keep  # coefficient handles, solution tensors and preconditioners stay alive


def sq_build_coeffs(L, n, seed, p_hi, a_lo, a_hi, stream=None) -> Coeffs:
    out = C.c_void_p()
    _check(load_library().sq_build_coeffs(int(L), int(n), int(seed) & (2**64 - 1), float(p_hi), float(a_lo),
                                          float(a_hi), _stream(stream), C.byref(out)), "sq_build_coeffs")
    return Coeffs(out)


def sq_coeffs_from_host(L, n, host_phase, a_lo, a_hi, stream=None) -> Coeffs:
    arr = np.ascontiguousarray(host_phase, dtype=np.uint8)
    if arr.size != L ** 3:
        raise ValueError("host_phase must hold L^3 bytes")
    out = C.c_void_p()
    _check(load_library().sq_coeffs_from_host(int(L), int(n), arr.ctypes.data_as(C.c_void_p), float(a_lo),
                                              float(a_hi), _stream(stream), C.byref(out)), "sq_coeffs_from_host")
    return Coeffs(out)


def sq_coeffs_set_subcell(c: Coeffs, sub: int):
    """Sub-cell inclusions: a centred cube of side `sub` grid intervals per cell
    carries the cell's value (sub = n: the checkerboard)."""
    _check(load_library().sq_coeffs_set_subcell(c, int(sub)), "sq_coeffs_set_subcell")


def _f64_array(vals, name):
    arr = np.ascontiguousarray(np.asarray(vals, dtype=np.float64).ravel())
    if arr.size < 2 or arr.size > 4:
        raise ValueError(f"{name}: 2 to 4 levels")
    return arr


def sq_coeffs_set_levels(c: Coeffs, values):
    """Multi-level medium: phase byte v reads level min(v, K-1) with value
    values[level] (K = len(values), 2..4); voxels outside the inclusion cube
    take values[0]."""
    arr = _f64_array(values, "values")
    _check(load_library().sq_coeffs_set_levels(c, int(arr.size), arr.ctypes.data_as(C.c_void_p)),
           "sq_coeffs_set_levels")


def sq_build_coeffs_levels(L, n, seed, probs, values, stream=None) -> Coeffs:
    """K-level cells drawn with probabilities probs (nested thresholds on the
    SplitMix64 stream of sq_build_coeffs) and coefficient values `values`."""
    pa, va = _f64_array(probs, "probs"), _f64_array(values, "values")
    if pa.size != va.size:
        raise ValueError("probs and values must have the same length")
    out = C.c_void_p()
    _check(load_library().sq_build_coeffs_levels(int(L), int(n), int(seed) & (2**64 - 1), int(pa.size),
                                                 pa.ctypes.data_as(C.c_void_p), va.ctypes.data_as(C.c_void_p),
                                                 _stream(stream), C.byref(out)), "sq_build_coeffs_levels")
    return Coeffs(out)


def sq_coeffs_from_host_levels(L, n, host_level, values, stream=None) -> Coeffs:
    """K-level handle from L^3 host cell levels (bytes >= K read as K - 1)."""
    arr = np.ascontiguousarray(host_level, dtype=np.uint8)
    if arr.size != L ** 3:
        raise ValueError("host_level must hold L^3 bytes")
    va = _f64_array(values, "values")
    out = C.c_void_p()
    _check(load_library().sq_coeffs_from_host_levels(int(L), int(n), arr.ctypes.data_as(C.c_void_p), int(va.size),
                                                     va.ctypes.data_as(C.c_void_p), _stream(stream), C.byref(out)),
           "sq_coeffs_from_host_levels")
    return Coeffs(out)


def sq_coeffs_regenerate_levels(c: Coeffs, seed, probs, stream=None):
    pa = _f64_array(probs, "probs")
    _check(load_library().sq_coeffs_regenerate_levels(c, int(seed) & (2**64 - 1), int(pa.size),
                                                      pa.ctypes.data_as(C.c_void_p), _stream(stream)),
           "sq_coeffs_regenerate_levels")


def sq_coeffs_regenerate(c: Coeffs, seed, p_hi, stream=None):
    _check(load_library().sq_coeffs_regenerate(c, int(seed) & (2**64 - 1), float(p_hi), _stream(stream)),
           "sq_coeffs_regenerate")


def sq_coeffs_upload(c: Coeffs, host_phase, stream=None):
    """host_phase: a PINNED torch uint8 CPU tensor of L^3 phases (0 / 1, or the
    cell levels of a multi-level handle)."""
    if host_phase.is_cuda or not host_phase.is_pinned() or str(host_phase.dtype) != "torch.uint8":
        raise ValueError("expected a pinned uint8 CPU tensor")
    _check(load_library().sq_coeffs_upload(c, C.c_void_p(host_phase.data_ptr()), _stream(stream)),
           "sq_coeffs_upload")


def sq_profile_enable(enable: bool):
    _check(load_library().sq_profile_enable(1 if enable else 0), "sq_profile_enable")


def sq_profile_read() -> dict:
    """{class name: (total ms, launches)} of the launches recorded since enable."""
    lib = load_library()
    ms = (C.c_double * 64)()
    cnt = (C.c_int64 * 64)()
    k = lib.sq_profile_read(ms, cnt, 64)
    if k < 0:
        raise SqError(-k, "sq_profile_read")
    return {lib.sq_profile_class_name(i).decode(): (ms[i], cnt[i]) for i in range(k)}


def sq_profile_work() -> dict:
    """{class name: (ms, launches)} of the launches that did work, from the last
    sq_profile_read (launches of at least half of the class median)."""
    lib = load_library()
    ms = (C.c_double * 64)()
    cnt = (C.c_int64 * 64)()
    k = lib.sq_profile_work(ms, cnt, 64)
    return {lib.sq_profile_class_name(i).decode(): (ms[i], cnt[i]) for i in range(k)}


def sq_profile_class_name(k: int) -> str:
    return load_library().sq_profile_class_name(int(k)).decode()


def sq_launch_count() -> int:
    """Kernel launches of the single-solve path since the library was loaded."""
    return int(load_library().sq_launch_count())


def sq_probe_fma(precision: int, stream=None):
    """(TFLOP/s, ms) of the FMA throughput probe: precision 0 = FP64, 1 = FP32."""
    tf, ms = C.c_double(0.0), C.c_float(0.0)
    _check(load_library().sq_probe_fma(int(precision), C.byref(tf), C.byref(ms), _stream(stream)), "sq_probe_fma")
    return tf.value, ms.value


def sq_probe_copy(src, dst, reps: int, stream=None) -> float:
    """GB/s (read + write) of dst <- src repeated `reps` times; src and dst are
    CUDA tensors of the same number of bytes (a multiple of 16)."""
    if not (src.is_cuda and dst.is_cuda and src.is_contiguous() and dst.is_contiguous()):
        raise ValueError("expected contiguous CUDA tensors")
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nbytes:
        raise ValueError("src and dst differ in size")
    g = C.c_double(0.0)
    _check(load_library().sq_probe_copy(C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()), nbytes, int(reps),
                                        C.byref(g), _stream(stream)), "sq_probe_copy")
    return g.value


def sq_coeffs_shape(c: Coeffs):
    L, n, N = C.c_int(), C.c_int(), C.c_int()
    _check(load_library().sq_coeffs_shape(c, C.byref(L), C.byref(n), C.byref(N)), "sq_coeffs_shape")
    return L.value, n.value, N.value


def sq_coeffs_cells(c: Coeffs):
    L, _, _ = sq_coeffs_shape(c)
    ph = np.empty(L ** 3, dtype=np.uint8)
    nhi = C.c_int64()
    _check(load_library().sq_coeffs_cells(c, ph.ctypes.data_as(C.c_void_p), C.byref(nhi)), "sq_coeffs_cells")
    return ph.reshape(L, L, L), nhi.value


def sq_precond_setup(N, rank) -> Precond:
    out = C.c_void_p()
    _check(load_library().sq_precond_setup(int(N), int(rank), C.byref(out)), "sq_precond_setup")
    return Precond(out)


def sq_precond_setup_canonical(N, f1, f2=None, f3=None) -> Precond:
    """Canonical preconditioner from host factors, each (R, N) FP64 with even
    rows; f2 / f3 None repeat f1."""
    arrs = [None if f is None else np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in (f1, f2, f3)]
    R = arrs[0].shape[0]
    for a in arrs:
        if a is not None and a.shape != (R, N):
            raise ValueError("factors must have shape (R, N)")
    ptrs = [None if a is None else a.ctypes.data_as(C.c_void_p) for a in arrs]
    out = C.c_void_p()
    _check(load_library().sq_precond_setup_canonical(int(N), int(R), ptrs[0], ptrs[1], ptrs[2], C.byref(out)),
           "sq_precond_setup_canonical")
    return Precond(out)


def sq_precond_setup_tucker(N, r, tol=0.0) -> Precond:
    """The paper's route: HOSVD of G+ with rank r, then Tucker-to-canonical
    dropping core-slice eigenvalues at or below tol * max."""
    out = C.c_void_p()
    _check(load_library().sq_precond_setup_tucker(int(N), int(r), float(tol), C.byref(out)),
           "sq_precond_setup_tucker")
    return Precond(out)


def sq_precond_info(pc: Precond):
    """(canonical rank, max relative error over the nonzero modes)."""
    R, e = C.c_int(), C.c_double()
    _check(load_library().sq_precond_info(pc, C.byref(R), C.byref(e)), "sq_precond_info")
    return R.value, e.value


def sq_precond_factors(pc: Precond, rank: int):
    """(t, w): the exponential-sum nodes and weights of a rank-R preconditioner."""
    t = np.zeros(max(rank, 1))
    w = np.zeros(max(rank, 1))
    _check(load_library().sq_precond_factors(pc, t.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)),
           "sq_precond_factors")
    return t[:rank], w[:rank]


def sq_workspace_create(N, precision) -> Workspace:
    out = C.c_void_p()
    _check(load_library().sq_workspace_create(int(N), int(precision), C.byref(out)), "sq_workspace_create")
    return Workspace(out)


def sq_pcg_solve(c, pc, w, dir, tol, max_iter, precision, x0, psi, stream=None) -> dict:
    """Solves into psi (float64 CUDA tensor, N^3); returns the solve info.
    SQ_ENOCONV and SQ_ETIMEOUT (a bounded device wait gave up; the solve still
    completed) are reported in info['status'], other errors raise."""
    info = SolveInfo()
    st = load_library().sq_pcg_solve(c, pc, w, int(dir), float(tol), int(max_iter), int(precision), _ptr(x0),
                                     _ptr(psi), C.byref(info), _stream(stream))
    _check(st, "sq_pcg_solve", allow=(SQ_ENOCONV, SQ_ETIMEOUT))
    return {k: getattr(info, k) for k, _ in SolveInfo._fields_}


def sq_homogenized_matrix(c, psi0, psi1, psi2, stream=None, energy=True):
    """(A_hom edge form, energy form); energy=False skips the energy form
    (returned as None), which is most of the kernel's FP64 work."""
    A = np.zeros(9)
    E = np.zeros(9) if energy else None
    _check(load_library().sq_homogenized_matrix(c, _ptr(psi0), _ptr(psi1), _ptr(psi2),
                                                A.ctypes.data_as(C.c_void_p),
                                                E.ctypes.data_as(C.c_void_p) if energy else None,
                                                _stream(stream)), "sq_homogenized_matrix")
    return A.reshape(3, 3), (E.reshape(3, 3) if energy else None)


def sq_homogenized_matrix_noalloc(L, n, phase, a_lo, a_hi, psi0, psi1, psi2, out, stream=None):
    """A_hom with no allocation inside the library: phase is a CUDA uint8 tensor
    (L^3), psi_i CUDA float64 tensors (N^3), out a CUDA float64 tensor of 18
    (edge form then energy form). Asynchronous on the stream."""
    _check(load_library().sq_homogenized_matrix_noalloc(int(L), int(n), _ptr(phase, "uint8"), float(a_lo), float(a_hi),
                                                        _ptr(psi0), _ptr(psi1), _ptr(psi2), _ptr(out),
                                                        _stream(stream)), "sq_homogenized_matrix_noalloc")


def sq_apply_operator(c, x, y, stream=None):
    _check(load_library().sq_apply_operator(c, _ptr(x), _ptr(y), _stream(stream)), "sq_apply_operator")


def sq_apply_operator_f32(c, x, y, stream=None):
    _check(load_library().sq_apply_operator_f32(c, _ptr(x, "float32"), _ptr(y, "float32"), _stream(stream)),
           "sq_apply_operator_f32")


def sq_rhs(c, dir, b, stream=None):
    _check(load_library().sq_rhs(c, int(dir), _ptr(b), _stream(stream)), "sq_rhs")


def sq_apply_precond(pc, w, r, z, stream=None):
    _check(load_library().sq_apply_precond(pc, w, _ptr(r), _ptr(z), _stream(stream)), "sq_apply_precond")


def sq_apply_precond_f32(pc, w, r, z, stream=None):
    _check(load_library().sq_apply_precond_f32(pc, w, _ptr(r, "float32"), _ptr(z, "float32"), _stream(stream)),
           "sq_apply_precond_f32")


def sq_batch_create(descs, precs, tiles=None) -> Batch:
    """descs: list of (Coeffs, dir, psi) with psi a float64 CUDA tensor of N^3;
    precs: one Precond per solve (same N); tiles: optional list of
    (N, dht_pencils, stencil_planes)."""
    n = len(descs)
    arr = (SolveDesc * n)()
    for k, (c, d, psi) in enumerate(descs):
        arr[k].coeffs = c.ptr
        arr[k].dir = int(d)
        arr[k].psi = _ptr(psi).value
    parr = (C.c_void_p * n)(*[p.ptr.value if isinstance(p.ptr, C.c_void_p) else p.ptr for p in precs])
    tl = list(tiles or [])
    tarr = _tile_array(tl)
    out = C.c_void_p()
    _check(load_library().sq_batch_create(n, arr, parr, tarr if tl else None, len(tl), C.byref(out)), "sq_batch_create")
    return Batch(out, n, (list(descs), list(precs)))


def sq_pcg_solve_batched(b: Batch, tol, max_iter, stream=None) -> list:
    """Solves the batch; returns one info dict per solve (SQ_ENOCONV is reported
    per solve, other errors raise)."""
    infos = (SolveInfo * b.count)()
    st = load_library().sq_pcg_solve_batched(b, float(tol), int(max_iter), infos, _stream(stream))
    _check(st, "sq_pcg_solve_batched", allow=(SQ_ENOCONV,))
    return [{k: getattr(inf, k) for k, _ in SolveInfo._fields_} for inf in infos]


def sq_net_create(N, max_batch, seed, out_scale) -> Net:
    out = C.c_void_p()
    _check(load_library().sq_net_create(int(N), int(max_batch), int(seed) & (2**64 - 1), float(out_scale),
                                        C.byref(out)), "sq_net_create")
    return Net(out)


def sq_net_params(net: Net) -> np.ndarray:
    n = C.c_int64()
    _check(load_library().sq_net_params(net, None, C.byref(n)), "sq_net_params")
    a = np.empty(n.value, dtype=np.float32)
    _check(load_library().sq_net_params(net, a.ctypes.data_as(C.c_void_p), C.byref(n)), "sq_net_params")
    return a


def sq_net_set_params(net: Net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(load_library().sq_net_set_params(net, a.ctypes.data_as(C.c_void_p), a.size), "sq_net_set_params")


def sq_net_grads(net: Net) -> np.ndarray:
    n = C.c_int64()
    _check(load_library().sq_net_params(net, None, C.byref(n)), "sq_net_params")
    a = np.empty(n.value, dtype=np.float32)
    _check(load_library().sq_net_grads(net, a.ctypes.data_as(C.c_void_p), a.size), "sq_net_grads")
    return a


def sq_net_predict(net: Net, c, psi0, psi1, psi2, stream=None):
    _check(load_library().sq_net_predict(net, c, _ptr(psi0), _ptr(psi1), _ptr(psi2), _stream(stream)),
           "sq_net_predict")


def sq_net_train_step(net: Net, coeffs, targets, lr, stream=None, loss_type=0) -> float:
    """coeffs: list of B Coeffs; targets: list of B triples of float64 CUDA
    tensors (psi_1..3); loss_type 0 = squared error, 1 = energy norm e.Ae, 2 = residual
    norm of the prediction (targets not read).
    Returns the loss of the forward pass."""
    B = len(coeffs)
    carr = (C.c_void_p * B)(*[c.ptr.value for c in coeffs])
    tarr = (C.c_void_p * (3 * B))(*[_ptr(t).value for tri in targets for t in tri])
    loss = C.c_double()
    _check(load_library().sq_net_train_step(net, B, carr, tarr, C.c_float(lr), int(loss_type), C.byref(loss),
                                            _stream(stream)),
           "sq_net_train_step")
    return loss.value


def sq_set_tiles(tiles):
    """tiles: list of (N, dht_pencils, stencil_planes[, stencil_rows[, dht_pencils_e]]);
    0 = default; [] restores every default."""
    tl = list(tiles)
    arr = _tile_array(tl)
    _check(load_library().sq_set_tiles(arr if tl else None, len(tl)), "sq_set_tiles")


def sq_ensemble_ahom(L, n, seeds, p_hi, a_lo, a_hi, rank=0, tol=1e-8, max_iter=2000, chunk=0, stream=None):
    """Empirical average and sample standard deviation of the edge-form A_hom
    over the realizations `seeds` (M >= 2). Returns a dict with mean (3x3),
    sigma (3x3), per_realization (M x 3 x 3), iters (M x 3) and status
    (SQ_OK or SQ_ENOCONV; other errors raise)."""
    sd = np.ascontiguousarray([int(x) & (2 ** 64 - 1) for x in seeds], dtype=np.uint64)
    M = sd.size
    mean, sigma = np.zeros(9), np.zeros(9)
    per = np.zeros(9 * max(M, 1))
    its = np.zeros(3 * max(M, 1), dtype=np.int32)
    st = load_library().sq_ensemble_ahom(int(L), int(n), sd.ctypes.data_as(C.c_void_p), int(M), float(p_hi),
                                         float(a_lo), float(a_hi), int(rank), float(tol), int(max_iter), int(chunk),
                                         mean.ctypes.data_as(C.c_void_p), sigma.ctypes.data_as(C.c_void_p),
                                         per.ctypes.data_as(C.c_void_p), its.ctypes.data_as(C.c_void_p),
                                         _stream(stream))
    _check(st, "sq_ensemble_ahom", allow=(SQ_ENOCONV,))
    return {"mean": mean.reshape(3, 3), "sigma": sigma.reshape(3, 3), "per_realization": per[:9 * M].reshape(M, 3, 3),
            "iters": its[:3 * M].reshape(M, 3), "status": st}


def sq_set_option(key, value):
    _check(load_library().sq_set_option(int(key), int(value)), "sq_set_option")


# ----------------------------------------------------------------------- 2D
def sq2d_build_coeffs(L, n, seed, p_hi, a_lo, a_hi, stream=None) -> Coeffs2D:
    out = C.c_void_p()
    _check(load_library().sq2d_build_coeffs(int(L), int(n), int(seed) & (2**64 - 1), float(p_hi), float(a_lo),
                                            float(a_hi), _stream(stream), C.byref(out)), "sq2d_build_coeffs")
    return Coeffs2D(out, int(L))


def sq2d_coeffs_from_host(L, n, host_phase, a_lo, a_hi, stream=None) -> Coeffs2D:
    arr = np.ascontiguousarray(host_phase, dtype=np.uint8)
    if arr.size != L * L:
        raise ValueError("host_phase must hold L^2 bytes")
    out = C.c_void_p()
    _check(load_library().sq2d_coeffs_from_host(int(L), int(n), arr.ctypes.data_as(C.c_void_p), float(a_lo),
                                                float(a_hi), _stream(stream), C.byref(out)), "sq2d_coeffs_from_host")
    return Coeffs2D(out, int(L))


def sq2d_coeffs_set_subcell(c: Coeffs2D, sub: int):
    _check(load_library().sq2d_coeffs_set_subcell(c, int(sub)), "sq2d_coeffs_set_subcell")


def sq2d_coeffs_cells(c: Coeffs2D) -> np.ndarray:
    ph = np.empty(c.L * c.L, dtype=np.uint8)
    _check(load_library().sq2d_coeffs_cells(c, ph.ctypes.data_as(C.c_void_p)), "sq2d_coeffs_cells")
    return ph.reshape(c.L, c.L)


def sq2d_precond_setup(N, rank) -> Precond2D:
    out = C.c_void_p()
    _check(load_library().sq2d_precond_setup(int(N), int(rank), C.byref(out)), "sq2d_precond_setup")
    return Precond2D(out)


def sq2d_precond_factors(pc: Precond2D, rank: int):
    t = np.zeros(max(rank, 1))
    w = np.zeros(max(rank, 1))
    _check(load_library().sq2d_precond_factors(pc, t.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)),
           "sq2d_precond_factors")
    return t[:rank], w[:rank]


def sq2d_workspace_create(N) -> Workspace2D:
    out = C.c_void_p()
    _check(load_library().sq2d_workspace_create(int(N), C.byref(out)), "sq2d_workspace_create")
    return Workspace2D(out)


def sq2d_pcg_solve(c, pc, w, dir, tol, max_iter, psi, stream=None) -> dict:
    """Solves corrector dir (0, 1) into psi (float64 CUDA tensor, N^2)."""
    info = SolveInfo()
    st = load_library().sq2d_pcg_solve(c, pc, w, int(dir), float(tol), int(max_iter), _ptr(psi), C.byref(info),
                                       _stream(stream))
    _check(st, "sq2d_pcg_solve", allow=(SQ_ENOCONV,))
    return {k: getattr(info, k) for k, _ in SolveInfo._fields_}


def sq2d_homogenized_matrix(c, psi0, psi1):
    A = np.zeros(4)
    E = np.zeros(4)
    _check(load_library().sq2d_homogenized_matrix(c, _ptr(psi0), _ptr(psi1), A.ctypes.data_as(C.c_void_p),
                                                  E.ctypes.data_as(C.c_void_p)), "sq2d_homogenized_matrix")
    return A.reshape(2, 2), E.reshape(2, 2)


def sq2d_apply_operator(c, x, y, stream=None):
    _check(load_library().sq2d_apply_operator(c, _ptr(x), _ptr(y), _stream(stream)), "sq2d_apply_operator")


def sq2d_rhs(c, dir, b, stream=None):
    _check(load_library().sq2d_rhs(c, int(dir), _ptr(b), _stream(stream)), "sq2d_rhs")


def sq2d_apply_precond(pc, w, r, z, stream=None):
    _check(load_library().sq2d_apply_precond(pc, w, _ptr(r), _ptr(z), _stream(stream)), "sq2d_apply_precond")
