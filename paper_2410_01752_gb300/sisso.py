"""Thin ctypes binding of the C ABI in ``include/sisso.h`` (argument marshalling only).

Every computation happens in the CUDA library; this module only converts arguments.
Arrays may be numpy arrays (host memory) or CUDA tensors (device memory, passed by
pointer).  If the shared library is missing, loading it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsisso_gb300.so")

# operator bits and enums of include/sisso.h
OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_EXP, OP_LOG, OP_SQRT, OP_SQ, OP_INV, OP_SIN, OP_CUBE, OP_EXPNEG = (
    1 << i for i in range(12))
PREC_FP64, PREC_FP32, PREC_MIXED_BF16, PREC_MIXED_FP16 = 0, 1, 2, 3
GRAMMAR_EQ2, GRAMMAR_NEW_X_PREV = 0, 1
PRESCREEN_NONE, PRESCREEN_MI, PRESCREEN_SPEARMAN = 0, 1, 2
SCREEN_AUTO, SCREEN_CORES, SCREEN_TENSOR = 0, 1, 2
GRAM_AUTO, GRAM_FP64, GRAM_TF32X3 = 0, 1, 2
MAX_DIM, MAX_SIS, MAX_RUNG = 5, 1024, 3
STATUS = {0: "SISSO_OK", -1: "SISSO_ERR_ARG", -2: "SISSO_ERR_OOM", -3: "SISSO_ERR_CUDA",
          -4: "SISSO_ERR_NUMERIC", -5: "SISSO_ERR_TIMEOUT", -6: "SISSO_ERR_STATE",
          -7: "SISSO_ERR_CAPACITY"}

# every entry point the header declares (checked by the tests)
EXPORTS = [
    "sisso_default_opts", "sisso_create", "sisso_fit", "sisso_get_n_dims", "sisso_get_descriptor",
    "sisso_get_sis", "sisso_feature_count", "sisso_feature_expr", "sisso_get_stats",
    "sisso_last_error", "sisso_destroy", "sisso_eval_features", "sisso_score_all",
    "sisso_sis_step", "sisso_l0_search", "sisso_space_sizes", "sisso_space_expr",
    "sisso_l0_search_noalloc", "sisso_gram_tc",
    "sisso_batch_create", "sisso_batch_create_error", "sisso_batch_set_tune", "sisso_batch_get_tune",
    "sisso_batch_autotune", "sisso_batch_load", "sisso_batch_run", "sisso_batch_results",
    "sisso_batch_timing", "sisso_batch_get_stats", "sisso_batch_last_error", "sisso_batch_destroy",
    "sisso_fit_batch", "sisso_subspace_gram",
    "sisso_mlp_create", "sisso_mlp_destroy", "sisso_mlp_get_params", "sisso_mlp_set_params", "sisso_mlp_forward",
    "sisso_mlp_gradients", "sisso_mlp_train", "sisso_prefix_features", "sisso_prefix_labels", "sisso_l0_learned",
    "sisso_set_proposal", "sisso_get_primaries", "sisso_prescreen", "sisso_prefix_training",
    "sisso_batch_set_wait_limit", "sisso_l0_learned_certified", "sisso_set_proposal_ex",
    "sisso_bilinear_tc", "sisso_measure_alu_peak", "sisso_release_memory",
]
MLP_IN, MLP_HIDDEN = 20, 256
MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1
NOALLOC_MAX_N = 256
NOALLOC_MAX_BAND = 65536


class SissoError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("grammar", C.c_int), ("survivors", C.c_int),
                ("band_rel", C.c_double), ("max_band", C.c_int64), ("cuda_stream", C.c_void_p),
                ("device", C.c_int), ("sis_threshold", C.c_double), ("stop_rmse", C.c_double),
                ("prescreen", C.c_int), ("prescreen_quantile", C.c_double), ("wait_limit_ns", C.c_int64),
                ("units", C.c_void_p), ("screen", C.c_int), ("gram", C.c_int), ("whiten", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("candidates_scored", C.c_int64), ("subsets_fit", C.c_int64),
                ("subsets_refit", C.c_int64), ("survivors_rescored", C.c_int64),
                ("window_grown", C.c_int), ("window_saturated", C.c_int), ("launches", C.c_int),
                ("ms_screen", C.c_double), ("ms_screen_pair", C.c_double),
                ("screen_pair_launches", C.c_int), ("ms_select", C.c_double),
                ("ms_radix", C.c_double), ("ms_rescore", C.c_double), ("ms_sort", C.c_double),
                ("ms_walk", C.c_double), ("walk_visited", C.c_int64), ("walk_dup_checks", C.c_int64),
                ("ms_gram", C.c_double), ("ms_l0", C.c_double), ("ms_refit", C.c_double),
                ("ms_fit", C.c_double), ("ms_l0_enum", C.c_double), ("l0_enum_launches", C.c_int),
                ("l0_candidates", C.c_int64), ("certified_prefixes", C.c_int64),
                ("screen_tc", C.c_int), ("tc_keys_raised", C.c_int64), ("pm_keys_direct", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Task(C.Structure):
    _fields_ = [("X", C.c_void_p), ("y", C.c_void_p), ("N", C.c_int), ("d", C.c_int)]


class TaskResult(C.Structure):
    _fields_ = [("status", C.c_int), ("n_dims", C.c_int),
                ("ids", (C.c_int64 * MAX_DIM) * MAX_DIM),
                ("coef", (C.c_double * (MAX_DIM + 1)) * MAX_DIM),
                ("rmse", C.c_double * MAX_DIM), ("r2", C.c_double * MAX_DIM)]


class BatchTune(C.Structure):
    _fields_ = [("score_units", C.c_int), ("enum_items", C.c_int), ("gram_rows", C.c_int),
                ("ctas_per_sm", C.c_int), ("window", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchStats(C.Structure):
    _fields_ = [("ms_run", C.c_double), ("candidates_scored", C.c_int64), ("subsets_fit", C.c_int64),
                ("subsets_refit", C.c_int64), ("windows_grown", C.c_int), ("windows_saturated", C.c_int),
                ("tasks_failed", C.c_int), ("grid", C.c_int), ("walk_visits", C.c_int64),
                ("walk_checks", C.c_int64), ("stage_ms", C.c_double * 16),
                ("stage_max_ms", C.c_double * 16), ("stage_count", C.c_int64 * 16)]

    def as_dict(self) -> dict:
        return {f: (list(getattr(self, f)) if f.startswith("stage_") else getattr(self, f)) for f, _ in self._fields_}


_lib = None


def load() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_01752_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    L.sisso_default_opts.argtypes = [C.POINTER(Opts)]
    L.sisso_default_opts.restype = None
    L.sisso_create.argtypes = [vp, vp, C.c_int, C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int,
                               C.POINTER(Opts), C.POINTER(vp)]
    L.sisso_fit.argtypes = [vp]
    L.sisso_get_n_dims.argtypes = [vp, C.POINTER(C.c_int)]
    L.sisso_get_descriptor.argtypes = [vp, C.c_int, i64p, dp, dp, dp]
    L.sisso_get_sis.argtypes = [vp, C.c_int, i64p, C.c_int, C.POINTER(C.c_int)]
    L.sisso_get_primaries.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    L.sisso_prescreen.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, C.c_double, dp, C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]
    L.sisso_feature_count.argtypes = [vp, i64p, i64p]
    L.sisso_feature_expr.argtypes = [vp, C.c_int64, C.c_char_p, C.c_size_t]
    L.sisso_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.sisso_last_error.argtypes = [vp]
    L.sisso_last_error.restype = C.c_char_p
    L.sisso_destroy.argtypes = [vp]
    L.sisso_destroy.restype = None
    L.sisso_eval_features.argtypes = [vp, vp, C.c_int64, C.c_int, vp]
    L.sisso_score_all.argtypes = [vp, vp, C.c_int, vp]
    L.sisso_sis_step.argtypes = [vp, vp, vp, C.c_int, C.c_int, i64p, C.POINTER(C.c_int)]
    L.sisso_l0_search.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.c_int, vp, C.c_int,
                                  C.POINTER(C.c_int), dp, i64p]
    L.sisso_space_sizes.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, i64p]
    L.sisso_gram_tc.argtypes = [vp, vp, C.c_double, C.c_int, C.c_int, C.c_int, vp, vp]
    L.sisso_bilinear_tc.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
    L.sisso_measure_alu_peak.argtypes = [C.c_int, C.POINTER(C.c_double)]
    L.sisso_release_memory.argtypes = [C.c_int]
    L.sisso_l0_search_noalloc.argtypes = [vp, vp, C.c_double, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp,
                                          C.POINTER(C.c_int), dp, i64p]
    L.sisso_space_expr.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int64, C.c_char_p, C.c_size_t]
    L.sisso_batch_create.argtypes = [vp, C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int, C.POINTER(Opts),
                                     C.POINTER(vp)]
    L.sisso_batch_create_error.argtypes = []
    L.sisso_batch_create_error.restype = C.c_char_p
    L.sisso_batch_set_tune.argtypes = [vp, C.POINTER(BatchTune)]
    L.sisso_batch_get_tune.argtypes = [vp, C.POINTER(BatchTune)]
    L.sisso_batch_autotune.argtypes = [vp, C.c_int, C.c_char_p, C.POINTER(BatchTune)]
    L.sisso_batch_load.argtypes = [vp, vp, C.c_int]
    L.sisso_batch_run.argtypes = [vp, C.c_int]
    L.sisso_batch_results.argtypes = [vp, vp, C.c_int]
    L.sisso_batch_timing.argtypes = [vp, dp, dp, C.c_int]
    L.sisso_batch_get_stats.argtypes = [vp, C.POINTER(BatchStats)]
    L.sisso_batch_last_error.argtypes = [vp]
    L.sisso_batch_last_error.restype = C.c_char_p
    L.sisso_batch_destroy.argtypes = [vp]
    L.sisso_batch_destroy.restype = None
    L.sisso_fit_batch.argtypes = [vp, C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int, C.POINTER(Opts), vp]
    L.sisso_subspace_gram.argtypes = [vp, vp, C.c_int, vp, vp, dp]
    L.sisso_mlp_create.argtypes = [C.c_uint64, C.POINTER(vp)]
    L.sisso_mlp_destroy.argtypes = [vp]
    L.sisso_mlp_destroy.restype = None
    L.sisso_mlp_get_params.argtypes = [vp, vp]
    L.sisso_mlp_set_params.argtypes = [vp, vp]
    L.sisso_mlp_forward.argtypes = [vp, vp, C.c_int64, vp]
    L.sisso_mlp_gradients.argtypes = [vp, vp, vp, C.c_int, C.POINTER(C.c_float), vp]
    L.sisso_mlp_train.argtypes = [vp, vp, vp, C.c_int64, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                  C.POINTER(C.c_float)]
    L.sisso_prefix_features.argtypes = [vp, vp, C.c_double, C.c_int, vp, vp, vp]
    L.sisso_prefix_labels.argtypes = [vp, vp, C.c_double, C.c_int, C.c_int, vp]
    L.sisso_prefix_training.argtypes = [vp, vp, C.c_double, C.c_int, C.c_int, vp, vp, vp]
    L.sisso_batch_set_wait_limit.argtypes = [vp, C.c_int64]
    L.sisso_set_proposal_ex.argtypes = [vp, vp, C.c_double, C.c_int]
    L.sisso_l0_learned_certified.argtypes = [vp, vp, vp, C.c_double, C.c_int, vp, vp, C.c_double, C.POINTER(C.c_int),
                                             dp, i64p, i64p, i64p]
    L.sisso_l0_learned.argtypes = [vp, vp, vp, C.c_double, C.c_int, vp, vp, C.c_double, C.POINTER(C.c_int), dp,
                                   i64p, i64p]
    L.sisso_set_proposal.argtypes = [vp, vp, C.c_double]
    for name in EXPORTS:
        if name not in ("sisso_default_opts", "sisso_last_error", "sisso_destroy", "sisso_batch_create_error",
                        "sisso_batch_last_error", "sisso_batch_destroy", "sisso_mlp_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a, dtype):
    """(pointer, keep-alive) for a numpy array or a CUDA tensor of the given dtype."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        want = {np.float64: torch.float64, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            a = a.to(want).contiguous()
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), arr


def space_sizes(d: int, op_set: int, rung: int, grammar: int = GRAMMAR_EQ2) -> list[int]:
    """|phi_l| for l = 0..rung (host only)."""
    out = np.zeros(rung + 1, dtype=np.int64)
    st = load().sisso_space_sizes(d, op_set, rung, grammar, out.ctypes.data_as(C.POINTER(C.c_int64)))
    if st:
        raise SissoError(st, "space_sizes")
    return [int(v) for v in out]


def space_expr(d: int, op_set: int, rung: int, grammar: int, fid: int) -> str:
    """Expression of feature ``fid`` (host only)."""
    buf = C.create_string_buffer(8192)
    st = load().sisso_space_expr(d, op_set, rung, grammar, fid, buf, 8192)
    if st:
        raise SissoError(st, "space_expr")
    return buf.value.decode()


def prescreen(X, y, method: int, quantile: float = 1.0):
    """(scores, keep flags) of the primaries (§3.1): method PRESCREEN_MI or PRESCREEN_SPEARMAN."""
    L = load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    d = X.shape[1]
    sc = np.zeros(d)
    keep = np.zeros(d, dtype=np.int32)
    n = C.c_int()
    st = L.sisso_prescreen(C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data), X.shape[0], d, int(method),
                           float(quantile), sc.ctypes.data_as(C.POINTER(C.c_double)),
                           keep.ctypes.data_as(C.POINTER(C.c_int)), C.byref(n))
    if st != 0:
        raise SissoError(st, "sisso_prescreen")
    return sc, keep.astype(bool)


def gram_tc(Z, yc, sdy: float, kind: int = PREC_MIXED_BF16):
    """Z Z^T / N and Z yc / N on the tensor cores (sisso_gram_tc): 16-bit operands for the
    mixed kinds, 3xTF32 split products for kind PREC_FP32."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    yc = np.ascontiguousarray(yc, dtype=np.float64)
    n, N = Z.shape
    G = np.zeros((n, n), dtype=np.float32)
    b = np.zeros(n, dtype=np.float32)
    st = load().sisso_gram_tc(C.c_void_p(Z.ctypes.data), C.c_void_p(yc.ctypes.data), float(sdy), n, N, kind,
                              C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data))
    if st:
        raise SissoError(st, "gram_tc")
    return G, b


def bilinear_tc(Lrows, Rrows, kind: int = PREC_MIXED_FP16):
    """sum_s L[i, s] R[j, s] from split 16-bit tensor-core products (sisso_bilinear_tc)."""
    Lrows = np.ascontiguousarray(Lrows, dtype=np.float64)
    Rrows = np.ascontiguousarray(Rrows, dtype=np.float64)
    m, N = Lrows.shape
    n = Rrows.shape[0]
    assert Rrows.shape[1] == N
    out = np.zeros((m, n), dtype=np.float64)
    st = load().sisso_bilinear_tc(C.c_void_p(Lrows.ctypes.data), C.c_void_p(Rrows.ctypes.data), m, n, N, kind,
                                  C.c_void_p(out.ctypes.data))
    if st:
        raise SissoError(st, "bilinear_tc")
    return out


ALU_FP32, ALU_FP32X2, ALU_FP64 = 0, 1, 2


def release_memory(device: int = 0) -> None:
    """Hand the device memory the library keeps for later contexts back to the device
    (sisso_release_memory)."""
    st = load().sisso_release_memory(int(device))
    if st:
        raise SissoError(st, "release_memory")


def measure_alu_peak(kind: int = ALU_FP32) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (sisso_measure_alu_peak)."""
    v = C.c_double()
    st = load().sisso_measure_alu_peak(int(kind), C.byref(v))
    if st:
        raise SissoError(st, "measure_alu_peak")
    return v.value


def l0_search_noalloc(G, b, syy: float, N: int, D: int, gid, precision: int = PREC_FP32, stream=None):
    """Exhaustive l0 over every D-subset of len(b) standardised features without a context
    and without allocating device memory (sisso_l0_search_noalloc): for callers that may
    not allocate.  Returns (positions, RSS, subsets examined)."""
    n = int(b.shape[0])
    gp, G = _ptr(G, np.float64)          # host arrays or CUDA tensors
    bp, b = _ptr(b, np.float64)
    ip, gid = _ptr(gid, np.int64)
    pos = np.zeros(D, dtype=np.int32)
    rss, ex = C.c_double(), C.c_int64()
    st = load().sisso_l0_search_noalloc(gp, bp, float(syy), int(N), n, D, ip, precision,
                                        C.c_void_p(getattr(stream, "cuda_stream", stream)) if stream else None,
                                        pos.ctypes.data_as(C.POINTER(C.c_int)), C.byref(rss), C.byref(ex))
    if st:
        raise SissoError(st, "l0_search_noalloc")
    return [int(p) for p in pos], rss.value, ex.value


@dataclass
class Descriptor:
    ids: list[int]
    coef: list[float]        # [intercept, c_1, ..., c_t] aligned with ids
    rmse: float
    r2: float


class Sisso:
    """One SISSO problem on one GPU: ``Sisso(X, y, ...).fit()``."""

    def __init__(self, X, y, op_set: int, rung: int, sis_size: int, max_dim: int,
                 precision: int = PREC_FP32, grammar: int = GRAMMAR_EQ2, survivors: int = 0,
                 max_band: int = 0, band_rel: float = 0.0, stream=None, device: int = 0,
                 sis_threshold: float = 0.0, stop_rmse: float = 0.0, units=None, prescreen=None,
                 screen: int = 0, gram: int = 0, whiten=None):
        L = load()
        self._ctx = C.c_void_p()
        N, d = int(X.shape[0]), int(X.shape[1])
        xp, self._x = _ptr(X, np.float64)
        yp, self._y = _ptr(y, np.float64)
        o = Opts()
        L.sisso_default_opts(C.byref(o))
        o.precision, o.grammar, o.survivors = precision, grammar, survivors
        o.max_band, o.band_rel, o.device = max_band, band_rel, device
        o.sis_threshold, o.stop_rmse = sis_threshold, stop_rmse
        o.screen = int(screen)          # SCREEN_AUTO, SCREEN_CORES or SCREEN_TENSOR (mixed forms)
        o.gram = int(gram)              # GRAM_AUTO, GRAM_FP64 or GRAM_TF32X3 (FP32 precision)
        wmat = None
        if whiten is not None:          # W (N x N): SISSO on W y and W Phi (FP64 precision)
            wmat = np.ascontiguousarray(np.asarray(whiten, dtype=np.float64))
            if wmat.shape != (N, N):
                raise ValueError("whiten: W must be N x N")
            o.whiten = C.c_void_p(wmat.ctypes.data)
        if prescreen is not None:    # (SISSO_PRESCREEN_MI or _SPEARMAN, quantile kept)
            o.prescreen, o.prescreen_quantile = int(prescreen[0]), float(prescreen[1])
        ulab = None
        if units is not None:        # one label per primary (-1: dimensionless); copied by sisso_create
            ulab = np.ascontiguousarray(np.asarray(units, dtype=np.int32))
            o.units = C.c_void_p(ulab.ctypes.data)
        if stream is not None:
            o.cuda_stream = C.c_void_p(getattr(stream, "cuda_stream", stream))
        st = L.sisso_create(xp, yp, N, d, op_set, rung, sis_size, max_dim, C.byref(o), C.byref(self._ctx))
        if st != 0:
            raise SissoError(st, "sisso_create")
        self.N, self.d, self.max_dim = N, d, max_dim
        self._x = self._y = None

    def _check(self, st: int, what: str):
        if st != 0:
            raise SissoError(st, f"{what}: {load().sisso_last_error(self._ctx).decode()}")

    def fit(self) -> list[Descriptor]:
        self._check(load().sisso_fit(self._ctx), "sisso_fit")
        return self.descriptors()

    def descriptors(self) -> list[Descriptor]:
        L = load()
        n = C.c_int()
        self._check(L.sisso_get_n_dims(self._ctx, C.byref(n)), "get_n_dims")
        out = []
        for t in range(1, n.value + 1):
            ids = np.zeros(t, dtype=np.int64)
            coef = np.zeros(t + 1, dtype=np.float64)
            rmse, r2 = C.c_double(), C.c_double()
            self._check(L.sisso_get_descriptor(self._ctx, t, ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                               coef.ctypes.data_as(C.POINTER(C.c_double)),
                                               C.byref(rmse), C.byref(r2)), "get_descriptor")
            out.append(Descriptor([int(v) for v in ids], [float(v) for v in coef], rmse.value, r2.value))
        return out

    def primaries(self) -> list[int]:
        """Original indices of the primaries the context was built on (pre-screening)."""
        L = load()
        n = C.c_int()
        self._check(L.sisso_get_primaries(self._ctx, None, 0, C.byref(n)), "get_primaries")
        idx = np.zeros(max(n.value, 1), dtype=np.int32)
        self._check(L.sisso_get_primaries(self._ctx, idx.ctypes.data_as(C.POINTER(C.c_int)), n.value, C.byref(n)),
                    "get_primaries")
        return [int(v) for v in idx[: n.value]]

    def sis(self, step: int) -> list[int]:
        buf = np.zeros(MAX_SIS, dtype=np.int64)
        n = C.c_int()
        self._check(load().sisso_get_sis(self._ctx, step, buf.ctypes.data_as(C.POINTER(C.c_int64)),
                                         MAX_SIS, C.byref(n)), "get_sis")
        return [int(v) for v in buf[: n.value]]

    def feature_count(self) -> tuple[int, list[int]]:
        n = C.c_int64()
        sizes = np.zeros(MAX_RUNG + 1, dtype=np.int64)
        self._check(load().sisso_feature_count(self._ctx, C.byref(n), sizes.ctypes.data_as(C.POINTER(C.c_int64))),
                    "feature_count")
        return n.value, [int(v) for v in sizes]

    def expr(self, fid: int) -> str:
        buf = C.create_string_buffer(8192)
        self._check(load().sisso_feature_expr(self._ctx, fid, buf, 8192), "feature_expr")
        return buf.value.decode()

    def stats(self) -> dict:
        s = Stats()
        self._check(load().sisso_get_stats(self._ctx, C.byref(s)), "get_stats")
        return s.as_dict()

    # ---- kernel-level entry points ----
    def eval_features(self, ids, precision: int = PREC_FP64) -> np.ndarray:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        out = np.zeros((ids.size, self.N), dtype=np.float64)
        self._check(load().sisso_eval_features(self._ctx, C.c_void_p(ids.ctypes.data), ids.size, precision,
                                               C.c_void_p(out.ctypes.data)), "eval_features")
        return out

    def score_all(self, target, precision: int = PREC_FP32) -> np.ndarray:
        n, _ = self.feature_count()
        out = np.zeros(n, dtype=np.float32)
        tp, keep = _ptr(target, np.float64)
        self._check(load().sisso_score_all(self._ctx, tp, precision, C.c_void_p(out.ctypes.data)), "score_all")
        del keep
        return out

    def sis_step(self, target, S_prev, k: int) -> list[int]:
        tp, keep = _ptr(target, np.float64)
        Sp = np.ascontiguousarray(np.asarray(S_prev, dtype=np.int64).reshape(-1))
        acc = np.zeros(k, dtype=np.int64)
        n = C.c_int()
        self._check(load().sisso_sis_step(self._ctx, tp, C.c_void_p(Sp.ctypes.data) if Sp.size else None,
                                          Sp.size, k, acc.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(n)),
                    "sis_step")
        del keep
        return [int(v) for v in acc[: n.value]]

    def l0_search(self, G, b, syy: float, D: int, gid, precision: int = PREC_FP32):
        G = np.ascontiguousarray(G, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        gid = np.ascontiguousarray(gid, dtype=np.int64)
        pos = np.zeros(D, dtype=np.int32)
        rss, ex = C.c_double(), C.c_int64()
        self._check(load().sisso_l0_search(self._ctx, C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data),
                                           float(syy), b.size, D, C.c_void_p(gid.ctypes.data), precision,
                                           pos.ctypes.data_as(C.POINTER(C.c_int)), C.byref(rss), C.byref(ex)),
                    "l0_search")
        return [int(p) for p in pos], rss.value, ex.value

    def subspace_gram(self, ids):
        """FP64 (G, b, syy) of the standardised features ids against y."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        n = ids.size
        G = np.zeros((n, n), dtype=np.float64)
        b = np.zeros(n, dtype=np.float64)
        syy = C.c_double()
        self._check(load().sisso_subspace_gram(self._ctx, C.c_void_p(ids.ctypes.data), n, C.c_void_p(G.ctypes.data),
                                               C.c_void_p(b.ctypes.data), C.byref(syy)), "subspace_gram")
        return G, b, syy.value

    def l0_learned(self, G, b, syy: float, gid, mlp: "MLP", frac: float):
        """D = 5 search over the prefixes the network ranks best (frac of all subsets)."""
        G = np.ascontiguousarray(G, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        gid = np.ascontiguousarray(gid, dtype=np.int64)
        pos = np.zeros(5, dtype=np.int32)
        rss, ex, npre = C.c_double(), C.c_int64(), C.c_int64()
        self._check(load().sisso_l0_learned(self._ctx, C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data),
                                            float(syy), b.size, C.c_void_p(gid.ctypes.data), mlp._m, float(frac),
                                            pos.ctypes.data_as(C.POINTER(C.c_int)), C.byref(rss), C.byref(ex),
                                            C.byref(npre)), "l0_learned")
        return [int(p) for p in pos], rss.value, ex.value, npre.value

    def l0_learned_certified(self, G, b, syy: float, gid, mlp: "MLP", frac: float):
        """The learned D = 5 search and its certificate: the exhaustive search's winner.
        Returns (positions, rss, subsets solved, prefixes proposed, prefixes the certificate kept)."""
        G = np.ascontiguousarray(G, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        gid = np.ascontiguousarray(gid, dtype=np.int64)
        pos = np.zeros(5, dtype=np.int32)
        rss, ex, npre, kept = C.c_double(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(load().sisso_l0_learned_certified(self._ctx, C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data),
                                                      float(syy), b.size, C.c_void_p(gid.ctypes.data), mlp._m,
                                                      float(frac), pos.ctypes.data_as(C.POINTER(C.c_int)),
                                                      C.byref(rss), C.byref(ex), C.byref(npre), C.byref(kept)),
                    "l0_learned_certified")
        return [int(p) for p in pos], rss.value, ex.value, npre.value, kept.value

    def set_proposal(self, mlp, frac: float = 0.01, certify: bool = True):
        """Learned search at the fit's D = 5 step; certify: followed by its certificate (exact)."""
        self._proposal = mlp
        self._check(load().sisso_set_proposal_ex(self._ctx, mlp._m if mlp is not None else None, float(frac),
                                                 int(bool(certify))), "set_proposal")

    def close(self):
        if self._ctx:
            load().sisso_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _task_array(problems):
    """ctypes array of sisso_task over host float64 copies (kept alive by the caller)."""
    keep = []
    arr = (Task * len(problems))()
    for i, (X, y) in enumerate(problems):
        Xa = np.ascontiguousarray(X, dtype=np.float64)
        ya = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        keep += [Xa, ya]
        arr[i].X, arr[i].y = Xa.ctypes.data, ya.ctypes.data
        arr[i].N, arr[i].d = int(Xa.shape[0]), int(Xa.shape[1])
    return arr, keep


def _results(res, n: int) -> list:
    out = []
    for i in range(n):
        r = res[i]
        dims = []
        for t in range(1, r.n_dims + 1):
            dims.append(Descriptor([int(r.ids[t - 1][j]) for j in range(t)],
                                   [float(r.coef[t - 1][j]) for j in range(t + 1)],
                                   float(r.rmse[t - 1]), float(r.r2[t - 1])))
        out.append((int(r.status), dims))
    return out


class Batch:
    """Many independent problems in one persistent launch (CUDA graph): ``Batch(problems, ...).run()``.

    problems: list of (X, y) host arrays; every task shares op_set, rung, sis_size, max_dim.
    """

    def __init__(self, problems, op_set: int, rung: int, sis_size: int, max_dim: int,
                 grammar: int = GRAMMAR_EQ2, max_band: int = 0, stream=None, device: int = 0):
        L = load()
        self._b = C.c_void_p()
        self.n = len(problems)
        arr, keep = _task_array(problems)
        o = Opts()
        L.sisso_default_opts(C.byref(o))
        o.precision, o.grammar, o.max_band, o.device = PREC_FP32, grammar, max_band, device
        if stream is not None:
            o.cuda_stream = C.c_void_p(getattr(stream, "cuda_stream", stream))
        st = L.sisso_batch_create(arr, self.n, op_set, rung, sis_size, max_dim, C.byref(o), C.byref(self._b))
        del keep
        if st != 0:
            raise SissoError(st, "sisso_batch_create: " + L.sisso_batch_create_error().decode())

    def _check(self, st: int, what: str):
        if st != 0:
            raise SissoError(st, f"{what}: {load().sisso_batch_last_error(self._b).decode()}")

    def load(self, problems):
        arr, keep = _task_array(problems)
        self._check(load().sisso_batch_load(self._b, arr, len(problems)), "batch_load")
        del keep

    def tune(self, **kw) -> dict:
        t = BatchTune(**kw)
        self._check(load().sisso_batch_set_tune(self._b, C.byref(t)), "batch_set_tune")
        return self.get_tune()

    def set_wait_limit(self, ns: int):
        """No-progress limit of the persistent kernel's work-queue wait (0: the default)."""
        self._check(load().sisso_batch_set_wait_limit(self._b, int(ns)), "batch_set_wait_limit")

    def get_tune(self) -> dict:
        t = BatchTune()
        self._check(load().sisso_batch_get_tune(self._b, C.byref(t)), "batch_get_tune")
        return t.as_dict()

    def autotune(self, reps: int = 2, cache_path: str | None = None) -> dict:
        t = BatchTune()
        self._check(load().sisso_batch_autotune(self._b, reps, cache_path.encode() if cache_path else None,
                                                C.byref(t)), "batch_autotune")
        return t.as_dict()

    def run(self, copies: bool = True):
        self._check(load().sisso_batch_run(self._b, 1 if copies else 0), "batch_run")

    def results(self) -> list:
        """Per task: (status, [Descriptor for t = 1..n_dims])."""
        res = (TaskResult * self.n)()
        self._check(load().sisso_batch_results(self._b, res, self.n), "batch_results")
        return _results(res, self.n)

    def timing(self) -> tuple[np.ndarray, np.ndarray]:
        """Per-task start and end (ms from the launch's first CTA)."""
        a = np.zeros(self.n, dtype=np.float64)
        e = np.zeros(self.n, dtype=np.float64)
        self._check(load().sisso_batch_timing(self._b, a.ctypes.data_as(C.POINTER(C.c_double)),
                                              e.ctypes.data_as(C.POINTER(C.c_double)), self.n), "batch_timing")
        return a, e

    def stats(self) -> dict:
        s = BatchStats()
        self._check(load().sisso_batch_get_stats(self._b, C.byref(s)), "batch_stats")
        return s.as_dict()

    def close(self):
        if self._b:
            load().sisso_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def fit_batch(problems, op_set: int, rung: int, sis_size: int, max_dim: int, grammar: int = GRAMMAR_EQ2) -> list:
    """One-shot sisso_fit_batch: per task (status, [Descriptor ...])."""
    L = load()
    arr, keep = _task_array(problems)
    o = Opts()
    L.sisso_default_opts(C.byref(o))
    o.precision, o.grammar = PREC_FP32, grammar
    res = (TaskResult * len(problems))()
    st = L.sisso_fit_batch(arr, len(problems), op_set, rung, sis_size, max_dim, C.byref(o), res)
    del keep
    if st != 0:
        raise SissoError(st, "sisso_fit_batch: " + L.sisso_batch_create_error().decode())
    return _results(res, len(problems))


class MLP:
    """The proposal network (20 -> 256 -> 256 -> 1, BF16 on the tensor cores) on the current device."""

    def __init__(self, seed: int = 0):
        self._m = C.c_void_p()
        st = load().sisso_mlp_create(int(seed), C.byref(self._m))
        if st != 0:
            raise SissoError(st, "sisso_mlp_create")

    def _check(self, st: int, what: str):
        if st != 0:
            raise SissoError(st, what)

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(load().sisso_mlp_get_params(self._m, C.c_void_p(p.ctypes.data)), "mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == MLP_PARAMS
        self._check(load().sisso_mlp_set_params(self._m, C.c_void_p(p.ctypes.data)), "mlp_set_params")

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
        out = np.zeros(X.shape[0], dtype=np.float32)
        self._check(load().sisso_mlp_forward(self._m, C.c_void_p(X.ctypes.data), X.shape[0],
                                             C.c_void_p(out.ctypes.data)), "mlp_forward")
        return out

    def gradients(self, X, t):
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = C.c_float()
        self._check(load().sisso_mlp_gradients(self._m, C.c_void_p(X.ctypes.data), C.c_void_p(t.ctypes.data),
                                               X.shape[0], C.byref(loss), C.c_void_p(g.ctypes.data)), "mlp_gradients")
        return loss.value, g

    def train(self, X, t, epochs: int = 5, batch: int = 2048, lr: float = 1e-3, seed: int = 0) -> float:
        X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1)
        loss = C.c_float()
        self._check(load().sisso_mlp_train(self._m, C.c_void_p(X.ctypes.data), C.c_void_p(t.ctypes.data),
                                           X.shape[0], epochs, batch, float(lr), int(seed), C.byref(loss)),
                    "mlp_train")
        return loss.value

    def close(self):
        if self._m:
            load().sisso_mlp_destroy(self._m)
            self._m = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prefix_features(G, b, syy: float):
    """(inputs C(n,3) x 20, prefixes C(n,3) x 3, base scores C(n,3)) of every 3-prefix, colex order."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.size
    npre = n * (n - 1) * (n - 2) // 6
    X = np.zeros((npre, MLP_IN), dtype=np.float32)
    P = np.zeros((npre, 3), dtype=np.int32)
    base = np.zeros(npre, dtype=np.float32)
    st = load().sisso_prefix_features(C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data), float(syy), n,
                                      C.c_void_p(X.ctypes.data), C.c_void_p(P.ctypes.data),
                                      C.c_void_p(base.ctypes.data))
    if st != 0:
        raise SissoError(st, "prefix_features")
    return X, P, base


def prefix_training(G, b, syy: float, N: int):
    """(inputs C(n,3) x 20, labels C(n,3), targets C(n,3)) of every 3-prefix, colex order: the
    network's inputs, the lowest RSS/SST of the prefix's extensions and the training target
    (its log10 minus the greedy completion's), all computed by the library."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.size
    npre = n * (n - 1) * (n - 2) // 6
    X = np.zeros((npre, MLP_IN), dtype=np.float32)
    lab = np.zeros(npre, dtype=np.float32)
    tgt = np.zeros(npre, dtype=np.float32)
    st = load().sisso_prefix_training(C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data), float(syy), int(N), n,
                                      C.c_void_p(X.ctypes.data), C.c_void_p(lab.ctypes.data), C.c_void_p(tgt.ctypes.data))
    if st != 0:
        raise SissoError(st, "prefix_training")
    return X, lab, tgt


def prefix_labels(G, b, syy: float, N: int) -> np.ndarray:
    """Per 3-prefix: the lowest RSS/SST over its 5-subset extensions (+inf: none)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.size
    out = np.zeros(n * (n - 1) * (n - 2) // 6, dtype=np.float32)
    st = load().sisso_prefix_labels(C.c_void_p(G.ctypes.data), C.c_void_p(b.ctypes.data), float(syy), int(N), n,
                                    C.c_void_p(out.ctypes.data))
    if st != 0:
        raise SissoError(st, "prefix_labels")
    return out
