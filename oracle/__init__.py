"""Python access to the plain FP64 CPU SISSO oracle (``oracle/sisso_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle states, slowly and plainly, what the GPU library
computes (arXiv 2410.01752 §2.1-§2.3).  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` import this module; the library never does, and the
two share no code.

``build()`` compiles the C file with gcc; every other function loads the shared object
and calls it through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sisso_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

# operator bits: the order of the operator table (binary first, then unary)
ADD, SUB, MUL, DIV, EXP, LOG, SQRT, SQ, INV, SIN, CUBE, EXPNEG = range(12)
OP_NAMES = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1", "sin", "^3", "exp-"]
GRAMMAR_EQ2, GRAMMAR_NEW_X_PREV = 0, 1
MAX_DIM = 8


def opmask(*ops: int) -> int:
    m = 0
    for o in ops:
        m |= 1 << o
    return m


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, pthreads)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, SRC, "-lm"], cwd=HERE)
        os.replace(tmp, LIB)
    return LIB


class _Result(C.Structure):
    _fields_ = [
        ("n_dims", C.c_int),
        ("n_sis", C.c_int * MAX_DIM),
        ("sis_ids", C.c_int64 * (MAX_DIM * 1024)),
        ("ids", (C.c_int64 * MAX_DIM) * MAX_DIM),
        ("coef", (C.c_double * (MAX_DIM + 1)) * MAX_DIM),
        ("rmse", C.c_double * MAX_DIM),
        ("r2", C.c_double * MAX_DIM),
        ("rss_gram", C.c_double * MAX_DIM),
        ("subsets", C.c_int64 * MAX_DIM),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        i64p = C.POINTER(C.c_int64)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.oracle_space_sizes.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, i64p]
        L.oracle_section_count.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int]
        L.oracle_section_count.restype = C.c_int64
        L.oracle_decode.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int64, ip, ip, i64p, i64p]
        L.oracle_pair_allowed.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int64]
        L.oracle_expr.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int64, C.c_char_p, C.c_int]
        L.oracle_eval.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, dp, C.c_int, C.c_int64, dp]
        L.oracle_scores.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, dp, C.c_int, dp, i64p,
                                    C.c_int64, dp, ip, C.c_int]
        L.oracle_scores_all.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, ip, dp, C.c_int, dp, dp, ip,
                                        C.c_int]
        L.oracle_units.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, ip, C.c_int64, ip]
        L.oracle_sis.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, dp, C.c_int, dp, i64p, C.c_int,
                                 C.c_int, i64p, C.c_int]
        L.oracle_sis_ex.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_int, ip, dp, C.c_int, dp, i64p, C.c_int,
                                    C.c_int, C.c_double, i64p, C.c_int]
        L.oracle_fit_ex.argtypes = [dp, dp, C.c_int, C.c_int, C.c_uint32, C.c_int, C.c_int, ip, C.c_int,
                                    C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(_Result)]
        L.oracle_fit_w.argtypes = [dp, dp, C.c_int, C.c_int, C.c_uint32, C.c_int, C.c_int, ip, dp, C.c_int,
                                   C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(_Result)]
        L.oracle_mi_kde.argtypes = [dp, C.c_int, C.c_int, dp, dp]
        L.oracle_spearman.argtypes = [dp, C.c_int, C.c_int, dp, dp]
        L.oracle_prescreen_keep.argtypes = [dp, C.c_int, C.c_double, ip]
        L.oracle_l0.argtypes = [dp, dp, C.c_double, C.c_int, C.c_int, C.c_int, i64p, ip, dp, C.c_int]
        L.oracle_l0.restype = C.c_int64
        L.oracle_fit.argtypes = [dp, dp, C.c_int, C.c_int, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                 C.c_int, C.c_int, C.POINTER(_Result)]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i64p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


@dataclass
class Space:
    """The expanded feature space phi_rung of §2.1 (Eq. 2).  units: one unit label per
    primary (equal labels share units, -1 dimensionless) for the dimensional analysis of
    §2.1 / §3.3, or None."""
    d: int
    ops: int
    rung: int
    grammar: int = GRAMMAR_EQ2
    units: tuple | None = None

    @property
    def args(self):
        return (self.d, self.ops, self.rung, self.grammar)

    def _units_ptr(self):
        if self.units is None:
            return None, None
        u = np.ascontiguousarray(np.asarray(self.units, dtype=np.int32))
        if u.size != self.d or u.min() < -1 or u.max() >= self.d:
            raise ValueError("units: one label in -1..d-1 per primary")
        return u.ctypes.data_as(C.POINTER(C.c_int)), u

    def units_of(self, fid: int):
        """(consistent, exponents over the unit labels in sixteenths) of feature fid."""
        up, keep = self._units_ptr()
        if up is None:
            raise ValueError("space without units")
        e = np.zeros(self.d, dtype=np.int32)
        ok = lib().oracle_units(*self.args, up, fid, e.ctypes.data_as(C.POINTER(C.c_int)))
        if ok < 0:
            raise ValueError("oracle_units failed")
        return bool(ok), e

    def sizes(self) -> list[int]:
        out = np.zeros(self.rung + 1, dtype=np.int64)
        if lib().oracle_space_sizes(*self.args, _i64p(out)):
            raise ValueError("bad feature space")
        return [int(v) for v in out]

    @property
    def n_features(self) -> int:
        return self.sizes()[-1]

    def section_count(self, level: int, op: int) -> int:
        return int(lib().oracle_section_count(*self.args, level, op))

    def decode(self, fid: int) -> tuple[int, int, int, int]:
        lv, op, a, b = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        if lib().oracle_decode(*self.args, fid, C.byref(lv), C.byref(op), C.byref(a), C.byref(b)):
            raise IndexError(fid)
        return lv.value, op.value, a.value, b.value

    def expr(self, fid: int) -> str:
        buf = C.create_string_buffer(8192)
        if lib().oracle_expr(*self.args, fid, buf, 8192) < 0:
            raise IndexError(fid)
        return buf.value.decode()

    def eval(self, X: np.ndarray, fid: int) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = np.empty(X.shape[0], dtype=np.float64)
        if lib().oracle_eval(*self.args, _dp(X), X.shape[0], fid, _dp(out)):
            raise IndexError(fid)
        return out

    def scores(self, X, target, ids=None, nthreads: int = 0):
        """(|rho|, valid) for each id (all ids when ``ids`` is None)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        if ids is None:
            ids = np.arange(self.n_features, dtype=np.int64)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        sc = np.zeros(ids.size, dtype=np.float64)
        va = np.zeros(ids.size, dtype=np.int32)
        rc = lib().oracle_scores(*self.args, _dp(X), X.shape[0], _dp(target), _i64p(ids), ids.size,
                                 _dp(sc), va.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
        if rc:
            raise ValueError(f"oracle_scores failed ({rc})")
        return sc, va.astype(bool)

    def scores_all(self, X, target, nthreads: int = 0):
        """(|rho|, valid) for every id, the features of phi_{rung-1} evaluated once and kept
        (the whole-space form the SIS step uses; equal to ``scores`` bit for bit)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        n = self.n_features
        sc = np.zeros(n, dtype=np.float64)
        va = np.zeros(n, dtype=np.int32)
        up, keep = self._units_ptr()
        rc = lib().oracle_scores_all(*self.args, up, _dp(X), X.shape[0], _dp(target), _dp(sc),
                                     va.ctypes.data_as(C.POINTER(C.c_int)), nthreads)
        if rc:
            raise ValueError(f"oracle_scores_all failed ({rc})")
        return sc, va.astype(bool)

    def sis(self, X, target, S_prev, k: int, nthreads: int = 0, threshold: float = 0.0) -> list[int]:
        """One SIS step (§2.2): up to k ids, only scores above `threshold` when it is > 0."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        Sp = np.ascontiguousarray(np.asarray(S_prev, dtype=np.int64).reshape(-1))
        acc = np.zeros(k, dtype=np.int64)
        up, keep = self._units_ptr()
        n = lib().oracle_sis_ex(*self.args, up, _dp(X), X.shape[0], _dp(target), _i64p(Sp), Sp.size, k,
                                float(threshold), _i64p(acc), nthreads)
        if n < 0:
            raise ValueError(f"oracle_sis failed ({n})")
        return [int(v) for v in acc[:n]]


def l0(G, b, syy: float, N: int, D: int, gid, nthreads: int = 0):
    """Exhaustive l0 (§2.3): (winning positions, RSS, subsets examined)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    gid = np.ascontiguousarray(gid, dtype=np.int64)
    n = b.size
    pos = np.zeros(D, dtype=np.int32)
    rss = C.c_double()
    ex = lib().oracle_l0(_dp(G), _dp(b), float(syy), int(N), n, D, _i64p(gid),
                         pos.ctypes.data_as(C.POINTER(C.c_int)), C.byref(rss), nthreads)
    if ex < 0:
        raise ValueError(f"oracle_l0 failed ({ex})")
    return [int(p) for p in pos], rss.value, int(ex)


@dataclass
class Descriptor:
    ids: list[int]
    coef: list[float]          # [intercept, c_1, ..., c_t] aligned with ids
    rmse: float
    r2: float
    rss_gram: float
    subsets: int


@dataclass
class FitResult:
    dims: list[Descriptor] = field(default_factory=list)
    sis: list[list[int]] = field(default_factory=list)   # ids accepted at each step


def fit(X, y, space: Space, k: int, max_dim: int, nthreads: int = 0, sis_threshold: float = 0.0,
        stop_rmse: float = 0.0, W=None) -> FitResult:
    """The SISSO iteration of §2.3 (Eq. 8) on the feature space of §2.1; sis_threshold > 0:
    the threshold variant of SIS (§2.2), stop_rmse > 0: stop once a step's RMSE is at or
    below it (§2.3, "low enough error"); W (N x N): SISSO on the whitened data W y, W Phi
    (§2.4)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    r = _Result()
    up, keep = space._units_ptr()
    if W is None:
        rc = lib().oracle_fit_ex(_dp(X), _dp(y), X.shape[0], X.shape[1], space.ops, space.rung,
                                 space.grammar, up, k, max_dim, float(sis_threshold), float(stop_rmse), nthreads,
                                 C.byref(r))
    else:
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (X.shape[0], X.shape[0])
        rc = lib().oracle_fit_w(_dp(X), _dp(y), X.shape[0], X.shape[1], space.ops, space.rung,
                                space.grammar, up, _dp(W), k, max_dim, float(sis_threshold), float(stop_rmse),
                                nthreads, C.byref(r))
    if rc:
        raise ValueError(f"oracle_fit failed ({rc})")
    out = FitResult()
    off = 0
    for t in range(max_dim):
        n = r.n_sis[t]
        if n == 0 and t >= r.n_dims:
            break
        out.sis.append([int(r.sis_ids[off + q]) for q in range(n)])
        off += n
    for t in range(r.n_dims):
        out.dims.append(Descriptor(ids=[int(r.ids[t][j]) for j in range(t + 1)],
                                   coef=[float(r.coef[t][j]) for j in range(t + 2)],
                                   rmse=float(r.rmse[t]), r2=float(r.r2[t]),
                                   rss_gram=float(r.rss_gram[t]), subsets=int(r.subsets[t])))
    return out


def mi_kde(X, y) -> np.ndarray:
    """MI(y; x_i) of every primary by Gaussian kernel density estimates (§3.1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(X.shape[1])
    if lib().oracle_mi_kde(_dp(X), X.shape[0], X.shape[1], _dp(y), _dp(out)):
        raise ValueError("oracle_mi_kde failed")
    return out


def spearman(X, y) -> np.ndarray:
    """Spearman rank correlation of every primary with y (§3.3)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(X.shape[1])
    if lib().oracle_spearman(_dp(X), X.shape[0], X.shape[1], _dp(y), _dp(out)):
        raise ValueError("oracle_spearman failed")
    return out


def prescreen_keep(score, q: float) -> np.ndarray:
    """Flags of the primaries whose score is in the top quantile q (§3.3)."""
    score = np.ascontiguousarray(score, dtype=np.float64)
    keep = np.zeros(score.size, dtype=np.int32)
    if lib().oracle_prescreen_keep(_dp(score), score.size, float(q), keep.ctypes.data_as(C.POINTER(C.c_int))) < 0:
        raise ValueError("oracle_prescreen_keep failed")
    return keep.astype(bool)
