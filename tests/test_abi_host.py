"""Host-side checks of the CUDA library (no GPU needed): the shared object loads and
exports every entry point include/sisso.h declares, the closed-form id <-> feature map
matches the oracle's loop-based decode, and argument errors are reported as statuses."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ALL9 = ["+", "-", "*", "/", "exp", "log", "sqrt", "^2", "^-1"]


@pytest.fixture(scope="module")
def lib():
    from paper_2410_01752_gb300 import build, sisso
    build.build()
    return sisso


def _mask(orc, names):
    return orc.opmask(*[orc.OP_NAMES.index(n) for n in names])


def test_exports_every_declared_symbol(lib):
    decl = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            decl |= set(re.findall(r"^\s*(?:sisso_status|void|const char\*)\s+(sisso_\w+)\s*\(", txt, re.M))
    assert decl, "no declarations found"
    L = lib.load()
    for name in decl:
        assert hasattr(L, name), name
    assert decl == set(lib.EXPORTS)


@pytest.mark.parametrize("d,names,rung,g", [
    (2, ["+", "*"], 3, 0), (2, ["+", "*"], 3, 1), (3, ALL9, 2, 0), (5, ALL9, 2, 0), (4, ALL9, 3, 1),
    (3, ["-", "/", "log", "^2", "sin", "^3", "exp-"], 3, 0), (10, ALL9, 2, 0), (12, ALL9, 2, 1),
    (1, ["sqrt", "exp"], 3, 0), (3, ["/"], 3, 1)])
def test_space_matches_oracle(orc, lib, d, names, rung, g):
    m = _mask(orc, names)
    sizes = lib.space_sizes(d, m, rung, g)
    sp = orc.Space(d, m, rung, g)
    assert sizes == sp.sizes()
    n = sizes[-1]
    ids = range(n) if n <= 4000 else np.random.default_rng(d).integers(0, n, 1500)
    for i in ids:
        assert lib.space_expr(d, m, rung, g, int(i)) == sp.expr(int(i))


def test_large_space_boundaries(orc, lib):
    """Section and row boundaries of the 2.9e8-feature space (d=10, rung 3, one rung-3
    operand from phi_1): first/last ids of every section and random ids."""
    m = _mask(orc, ALL9)
    sp = orc.Space(10, m, 3, orc.GRAMMAR_NEW_X_PREV)
    sizes = sp.sizes()
    assert lib.space_sizes(10, m, 3, 1) == sizes
    probes = set()
    base = sizes[2]
    for op in range(12):
        c = sp.section_count(3, op)
        if c > 0:
            probes |= {base, base + 1, base + c - 2, base + c - 1, base + c // 2}
            base += c
    probes |= set(int(v) for v in np.random.default_rng(5).integers(sizes[1], sizes[3], 300))
    for i in sorted(probes):
        assert lib.space_expr(10, m, 3, 1, i) == sp.expr(i)


def test_eq2_rung3_triangle_unranking(orc, lib):
    """Deep ids of the eq.-2 rung-3 space (triangle rows decoded by a square root)."""
    m = _mask(orc, ["+", "-", "*", "/", "sqrt"])
    sp = orc.Space(4, m, 3)
    sizes = sp.sizes()
    rng = np.random.default_rng(9)
    for i in list(rng.integers(sizes[2], sizes[3], 400)) + [sizes[3] - 1, sizes[2]]:
        assert lib.space_expr(4, m, 3, 0, int(i)) == sp.expr(int(i))


@pytest.mark.parametrize("kw,bad", [
    (dict(op_set=0), "empty op mask"), (dict(rung=4), "rung > 3"), (dict(rung=0), "rung 0"),
    (dict(max_dim=6), "max_dim > 5"), (dict(sis_size=0), "k = 0"), (dict(sis_size=2000), "k > 1024"),
    (dict(N=3), "N < max_dim + 1"), (dict(precision=7), "precision"), (dict(grammar=3), "grammar"),
    (dict(gram=3), "gram option"), (dict(gram=2, precision=0), "3xTF32 Gram with FP64 precision"),
    (dict(gram=2, precision=2), "3xTF32 Gram with a mixed form"),
    (dict(whiten=True, precision=1), "whitening needs FP64 precision")])
def test_argument_errors(lib, kw, bad):
    args = dict(N=20, d=3, op_set=lib.OP_ADD | lib.OP_MUL, rung=2, sis_size=5, max_dim=3, precision=1, grammar=0,
                gram=0, whiten=False)
    args.update(kw)
    L = lib.load()
    X = np.ones((max(args["N"], 1), args["d"]))
    y = np.arange(float(max(args["N"], 1)))
    o = lib.Opts()
    L.sisso_default_opts(C.byref(o))
    o.precision, o.grammar, o.gram = args["precision"], args["grammar"], args["gram"]
    W = np.eye(max(args["N"], 1))
    if args["whiten"]:
        o.whiten = C.c_void_p(W.ctypes.data)
    ctx = C.c_void_p()
    st = L.sisso_create(C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data), args["N"], args["d"],
                        args["op_set"], args["rung"], args["sis_size"], args["max_dim"], C.byref(o),
                        C.byref(ctx))
    assert st == -1, bad
    assert not ctx.value


def test_null_and_state_errors(lib):
    L = lib.load()
    assert L.sisso_fit(None) == -1
    assert L.sisso_release_memory(-1) == -1
    n = C.c_int()
    assert L.sisso_get_n_dims(None, C.byref(n)) == -1
    assert L.sisso_space_sizes(3, 0, 2, 0, None) == -1
    L.sisso_destroy(None)


@pytest.mark.parametrize("case,msg", [
    ("nan_x", "non-finite X"), ("nan_y", "non-finite y"), ("const_y", "constant y"),
    ("small_n", "N >= max_dim + 1"), ("k_dim", "max_dim * sis_size"), ("prec", "FP32"),
])
def test_batch_argument_errors(lib, case, msg):
    """The batched form validates every task on the host before touching a GPU."""
    rng = np.random.default_rng(0)
    probs = [(rng.uniform(1, 2, size=(30, 3)), rng.normal(size=30)) for _ in range(3)]
    k, D, prec = 10, 3, lib.PREC_FP32
    if case == "nan_x":
        probs[1][0][4, 2] = np.nan
    elif case == "nan_y":
        probs[2][1][7] = np.inf
    elif case == "const_y":
        probs[1] = (probs[1][0], np.full(30, 2.5))
    elif case == "small_n":
        probs[2] = (probs[2][0][:3], probs[2][1][:3])
    elif case == "k_dim":
        k = 200
    L = lib.load()
    arr, keep = lib._task_array(probs)
    o = lib.Opts()
    L.sisso_default_opts(C.byref(o))
    if case == "prec":
        o.precision = lib.PREC_FP64
    b = C.c_void_p()
    st = L.sisso_batch_create(arr, len(probs), lib.OP_ADD | lib.OP_MUL, 2, k, D, C.byref(o), C.byref(b))
    assert st == -1
    assert not b.value
    err = L.sisso_batch_create_error().decode()
    assert msg in err
    if case in ("nan_x", "const_y"):
        assert err.startswith("task 1:")


def test_batch_null_arguments(lib):
    L = lib.load()
    assert L.sisso_batch_run(None, 1) == -1
    assert L.sisso_batch_results(None, None, 0) == -1
    assert L.sisso_batch_set_tune(None, None) == -1
    L.sisso_batch_destroy(None)
    b = C.c_void_p()
    assert L.sisso_batch_create(None, 0, 1, 2, 5, 2, None, C.byref(b)) == -1


def test_learned_api_argument_errors(lib):
    """The learned-proposal entry points reject NULL pointers and out-of-range sizes with
    SISSO_ERR_ARG before they touch a device."""
    L = lib.load()
    f = np.zeros(lib.MLP_PARAMS, dtype=np.float32)
    X = np.zeros((256, lib.MLP_IN), dtype=np.float32)
    fp = C.c_void_p(f.ctypes.data)
    xp = C.c_void_p(X.ctypes.data)
    assert L.sisso_mlp_create(7, None) == -1
    assert L.sisso_mlp_get_params(None, fp) == -1
    assert L.sisso_mlp_set_params(None, fp) == -1
    assert L.sisso_mlp_forward(None, xp, 256, fp) == -1
    assert L.sisso_mlp_gradients(None, xp, fp, 256, None, fp) == -1
    assert L.sisso_mlp_train(None, xp, fp, 256, 1, 128, 1e-3, 0, None) == -1
    L.sisso_mlp_destroy(None)
    n = 12
    G = np.eye(n)
    b = np.full(n, 0.1)
    out = np.zeros(n ** 3, dtype=np.float32)
    Gp, bp, op = (C.c_void_p(a.ctypes.data) for a in (G, b, out))
    assert L.sisso_prefix_features(None, bp, 1.0, n, op, None, None) == -1
    assert L.sisso_prefix_features(Gp, bp, 1.0, 2, op, None, None) == -1       # fewer than 3 features
    assert L.sisso_prefix_features(Gp, bp, 1.0, 4096, op, None, None) == -1    # above 4095
    assert L.sisso_prefix_features(Gp, bp, 0.0, n, op, None, None) == -1       # syy must be > 0
    assert L.sisso_prefix_labels(Gp, bp, 1.0, 100, 4, op) == -1                # fewer than 5 features
    assert L.sisso_prefix_labels(Gp, bp, 1.0, 100, 1401, op) == -1             # above 1400
    assert L.sisso_prefix_labels(Gp, bp, 1.0, 0, n, op) == -1                  # N >= 1
    assert L.sisso_prefix_labels(Gp, None, 1.0, 100, n, op) == -1
    gid = np.arange(n, dtype=np.int64)
    pos = (C.c_int * 5)()
    rss = C.c_double()
    ex, npre = C.c_int64(), C.c_int64()
    assert L.sisso_l0_learned(None, Gp, bp, 1.0, n, C.c_void_p(gid.ctypes.data), None, 0.01, pos, C.byref(rss),
                              C.byref(ex), C.byref(npre)) == -1
    assert L.sisso_set_proposal(None, None, 0.01) == -1
    assert L.sisso_subspace_gram(None, C.c_void_p(gid.ctypes.data), n, Gp, bp, C.byref(rss)) == -1
