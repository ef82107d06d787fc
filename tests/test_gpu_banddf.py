"""The double-FP32 form of the assembled band product (op_form "assembled_df")
against the FP64 oracle: operators row by row within the bound of the arithmetic,
exact homogeneity under power-of-two scaling, launch configurations, steps, graph
replay, batches and the full-size patch.

Error bound: coefficients and inputs are held to 48 significant bits and every
product and addition of a row is error-free up to the rounding of the second FP32
accumulator, so |y_i - (A x)_i| <= C 2^-48 sum_j |A_ij| |x_j| with C a small
multiple of the number of terms' rounding steps seen in practice; C = 64 below.
Terms of tiny slots (every coefficient of the slot below 2^-24 of the matrix's
largest) are one FP32 multiply-add of the high parts, each within 2^-23 |A_ij x_j|
(2^-22 below, as slack), which adds 2^-22 sum over those slots of |A_ij| |x_j|."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import net
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
C_BOUND = 64 * 2.0 ** -48
TINY_BOUND = 2.0 ** -22


def _tiny_slots(A, cut=2.0 ** -23):
    """The slots the library may treat as tiny, as a superset: its cut is 2^-24 on the FP32
    high parts of its own band (assembled by probing, scaled so that the largest entry lies
    in [1, 2)); cut > 2^-24 here keeps every such slot whatever the roundoff of either band."""
    scale = 2.0 ** np.floor(np.log2(np.abs(A).max()))
    return (np.abs(A).max(axis=0) / scale < cut).astype(np.float64)


def _bound(P, rows, A, X, tiny):
    return (C_BOUND * P.band_rows_times(rows, np.abs(A), np.abs(X))
            + TINY_BOUND * P.band_rows_times(rows, np.abs(A) * tiny[None, :], np.abs(X)))

CASES = {
    "2d_p23": W.Workload("t", 2, (4, 5), (2, 3), 0.1, 1, 0.5, 1),
    "3d_mixed_p": W.small(d=3, nel=(3, 4, 5), p=(2, 3, 2), amp=0.12),
    "3d_p4": W.small(d=3, nel=(5, 4, 3), p=4, amp=0.1),
    "3d_p1": W.small(d=3, nel=4, p=1, amp=0.1),
    "3d_ragged_p3": W.small(d=3, nel=(11, 9, 13), p=3, amp=0.1),
    "3d_smallest": W.Workload("s2", 3, (1, 1, 1), (2, 2, 2), 0.1, 2, 0.5, 3),
    "2d_p1": W.Workload("s4", 2, (3, 2), (1, 1), 0.1, 2, 0.5, 3),
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _np(t):
    return t.cpu().numpy()


def _gpu(w, **kw):
    return iga.Patch(w.p, w.knots, w.ctrl(), **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_df_operators_within_the_arithmetic_bound(name):
    w = CASES[name]
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    Mr, Kr = P.assemble()
    rows = np.arange(P.N)
    g = _gpu(w, op_form="assembled_df")
    rng = np.random.default_rng(3)
    X = np.stack([rng.standard_normal(P.N), 1.0 + 0.1 * rng.standard_normal(P.N), rng.uniform(-1e3, 1e3, P.N)])
    y = torch.empty(3 * P.N, dtype=torch.float64, device=DEV)
    for A, apply in ((Mr, g.apply_M), (Kr, g.apply_K)):
        apply(_t(X.ravel()), y, 3)
        Y = _np(y).reshape(3, P.N)
        tiny = _tiny_slots(A)
        for v in range(3):
            ref = P.band_rows_times(rows, A, X[v])
            bound = _bound(P, rows, A, X[v], tiny)
            assert np.all(np.abs(Y[v] - ref) <= bound), (v, np.max(np.abs(Y[v] - ref) / bound))
    g.close()


@pytest.mark.parametrize("e", [300, -300, 0])
def test_df_product_is_exactly_homogeneous(e):
    """The per-vector scale is a power of two: x 2^e gives exactly (A x) 2^e."""
    w = CASES["3d_ragged_p3"]
    g = _gpu(w, op_form="assembled_df")
    X = np.random.default_rng(5).standard_normal((2, g.N))
    y0 = torch.empty(2 * g.N, dtype=torch.float64, device=DEV)
    y1 = torch.empty_like(y0)
    for apply in (g.apply_M, g.apply_K):
        apply(_t(X.ravel()), y0, 2)
        apply(_t(np.ldexp(X, e).ravel()), y1, 2)
        assert np.array_equal(_np(y1), np.ldexp(_np(y0), e))
    z = torch.zeros_like(y0)
    g.apply_M(z, y1, 2)
    assert torch.count_nonzero(y1).item() == 0
    g.close()


@pytest.mark.parametrize("threads", [64, 96, 128, 256, 512])
@pytest.mark.parametrize("nv", [1, 2, 3, 4])
def test_df_configs_are_bitwise_equal(threads, nv):
    w = W.small(d=3, nel=(9, 7, 6), p=3, amp=0.1)
    g = _gpu(w, op_form="assembled_df")
    x = _t(np.random.default_rng(1).standard_normal(5 * g.N))
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    g.apply_M(x, y0, nvec=5)
    g.set_band_config(threads, nv)
    g.apply_M(x, y1, nvec=5)
    assert torch.equal(y0, y1)
    g.apply_K(x, y1, nvec=5)
    g.set_band_config(0, 0)
    g.apply_K(x, y0, nvec=5)
    assert torch.equal(y0, y1)
    g.close()


def test_df_switching_forms_keeps_both_products():
    """assembled_df releases the FP64 band; switching back re-assembles it."""
    w = W.small(d=3, nel=(5, 6, 4), p=3, amp=0.1)
    g = _gpu(w, op_form="assembled")
    x = _t(np.random.default_rng(2).standard_normal(g.N))
    y64 = torch.empty_like(x)
    ydf = torch.empty_like(x)
    y = torch.empty_like(x)
    g.apply_K(x, y64)
    g.set_op_form("assembled_df")
    g.apply_K(x, ydf)
    g.set_op_form("assembled")
    g.apply_K(x, y)
    assert torch.equal(y, y64)
    g.set_op_form("assembled_df")
    g.apply_K(x, y)
    assert torch.equal(y, ydf)
    assert (ydf - y64).abs().max().item() <= 1e-12 * y64.abs().max().item()
    g.close()


def _dt(ops, rho, frac=0.5):
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    return frac * math.sqrt(oracle.theta_crit(rho) / lmax)


@pytest.mark.parametrize("precond", ["fp64", "banded", "banded32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_df_steps_match_oracle(k, precond):
    w = W.small(d=3, nel=(5, 4, 6), p=3, amp=0.1, k=k, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    st = oracle.Stepper(ops, k, w.rho, tol=1e-12)
    U0, V0 = w.initial()
    Xo = st.init(U0, V0)
    for _ in range(10):
        Xo = st.step(Xo, dt)
    g = _gpu(w, tol=1e-12, op_form="assembled_df", precond=precond)
    state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(k, _t(U0), _t(V0), state)
    s = g.step(state, k, w.rho, dt, 10)
    Xg = _np(state).reshape(3 * k, g.N)
    for row in (0, 1):
        err = np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row])
        assert err < 1e-9, (row, err)
    assert s.max_relres <= 1e-12
    g.close()


@pytest.mark.parametrize("guess", ["zero", "extrap", "learned"])
def test_df_graph_replay_equals_host_loop(guess):
    w = W.small(d=3, nel=(6, 5, 7), p=3, amp=0.1, k=2, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    U0, V0 = w.initial()
    out = []
    theta = net.bf16_round(np.random.default_rng(10).uniform(-0.2, 0.2, net.NPARAM)) if guess == "learned" else None
    for graphs in (False, True):
        g = _gpu(w, tol=1e-11, op_form="assembled_df", precond="banded32", guess=guess)
        if theta is not None:
            g.ws_set_params(theta)
        g.set_graphs(graphs)
        state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
        g.state_init(w.k, _t(U0), _t(V0), state)
        st = g.step(state, w.k, w.rho, dt, 4)
        st = g.step(state, w.k, w.rho, dt, 6, st)
        out.append((_np(state), st.iters, st.max_iters, st.steps))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_df_cfl_matches_dense_eigenvalue():
    w = CASES["3d_mixed_p"]
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    g = _gpu(w, tol=1e-10, op_form="assembled_df", precond="banded32")
    lam, tc = g.cfl(0.5, iters=min(ops.N, 200))
    g.close()
    assert abs(lam - lmax) <= 1e-8 * lmax


def test_df_batch_equals_patches_stepped_alone():
    rng = np.random.default_rng(4)
    ws = []
    for r in range(3):
        nel = tuple(int(v) for v in rng.integers(3, 7, size=3))
        p = (2, 3, 4)[r]
        ws.append(W.Workload("b%d" % r, 3, nel, (p, p, p), 0.1, 2, 0.5, 4, init="random", seed=r))
    pats, states, dts, inits = [], [], [], []
    for w in ws:
        g = _gpu(w, tol=1e-10, op_form="assembled_df", precond="banded32")
        lam, tc = g.cfl(w.rho, iters=100)
        U0, V0 = w.initial()
        pats.append(g)
        states.append(torch.zeros(6 * g.N, dtype=torch.float64, device=DEV))
        dts.append(0.5 * tc)
        inits.append((_t(U0), _t(V0)))
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(2, u0, v0, st)
    b = iga.Batch(pats)
    b.step(states, 2, 0.5, dts, 5)
    batched = [_np(s).copy() for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.set_time(0.0)
        g.state_init(2, u0, v0, st)
        g.step(st, 2, 0.5, dt, 5)
        assert np.array_equal(_np(st), batched[i]), i
    b.close()
    for g in pats:
        g.close()


def test_df_cube64_sampled_rows():
    """Full size (3-D deformed cube, p=3, 64^3 elements, N = 274625), two vectors in
    one launch as in the stage solves: sampled rows within the arithmetic bound."""
    w = W.config("cube64_p3")
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    rows = W.sample_indices(P.N, 300, seed=6)
    Mr, Kr = P.assemble(rows)
    g = _gpu(w, op_form="assembled_df")
    g.autotune(nvec=2, reps=2)
    rng = np.random.default_rng(2)
    X = np.stack([rng.standard_normal(P.N), np.sin(np.arange(P.N) * 1e-3)])
    y = torch.empty(2 * P.N, dtype=torch.float64, device=DEV)
    for A, apply in ((Mr, g.apply_M), (Kr, g.apply_K)):
        apply(_t(X.ravel()), y, 2)
        Y = _np(y).reshape(2, P.N)
        tiny = _tiny_slots(A, cut=2.0 ** -20)  # sampled rows: their largest entry may be below the band's
        for v in range(2):
            ref = P.band_rows_times(rows, A, X[v])
            bound = _bound(P, rows, A, X[v], tiny)
            assert np.all(np.abs(Y[v][rows] - ref) <= bound)
    g.close()


@pytest.mark.parametrize("decades", [15, 200])
def test_df_split_paths_wide_dynamic_range(decades):
    """Inputs spanning 10^-decades .. 10^decades with zeros and negative zeros: the
    split's integer path, its FP64 fallback (entries whose scaled value leaves FP32's
    normal range) and zero handling. Bound: the relative term of the arithmetic plus
    the absolute floor of a per-vector power-of-two scale, 2^-130 max|x| sum_j |a_ij|
    per term (entries that far below the largest are carried to that absolute
    precision only). The reference is the FP64 product of the same assembled band:
    with inputs spread over 10^400 a small coefficient's assembly roundoff (probing
    against the oracle's direct quadrature, ~1e-16 of the row's larger terms) times a
    10^200 entry is not the arithmetic under test; at 10^+-15 the oracle's rows serve
    as well."""
    w = CASES["3d_ragged_p3"]
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    Mr, Kr = P.assemble()
    rows = np.arange(P.N)
    rng = np.random.default_rng(8)
    X = rng.standard_normal(P.N) * 10.0 ** rng.uniform(-decades, decades, P.N)
    X[rng.integers(0, P.N, 40)] = 0.0
    X[rng.integers(0, P.N, 40)] = -0.0
    gdf = _gpu(w, op_form="assembled_df")
    g64 = _gpu(w, op_form="assembled")
    y = torch.empty(P.N, dtype=torch.float64, device=DEV)
    y64 = torch.empty_like(y)
    for A, adf, a64 in ((Mr, gdf.apply_M, g64.apply_M), (Kr, gdf.apply_K, g64.apply_K)):
        adf(_t(X), y)
        a64(_t(X), y64)
        absA = P.band_rows_times(rows, np.abs(A), np.ones(P.N))
        bound = _bound(P, rows, A, X, _tiny_slots(A)) + 343 * 2.0 ** -130 * np.abs(X).max() * absA
        assert np.all(np.abs(_np(y) - _np(y64)) <= bound)
        if decades <= 15:
            assert np.all(np.abs(_np(y) - P.band_rows_times(rows, A, X)) <= bound)
    gdf.close()
    g64.close()


@pytest.mark.parametrize("k", [1, 2])
def test_df_steps_2d_match_oracle(k):
    """2-D patch (mixed degrees 2, 3, deformed): double-FP32 steps against the oracle."""
    w = W.Workload("t2", 2, (9, 7), (2, 3), 0.1, k, 0.5, 12, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    st = oracle.Stepper(ops, k, w.rho, tol=1e-12)
    U0, V0 = w.initial()
    Xo = st.init(U0, V0)
    for _ in range(12):
        Xo = st.step(Xo, dt)
    g = _gpu(w, tol=1e-12, op_form="assembled_df", precond="banded32")
    state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(k, _t(U0), _t(V0), state)
    g.step(state, k, w.rho, dt, 12)
    Xg = _np(state).reshape(3 * k, g.N)
    for row in (0, 1):
        assert np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row]) < 1e-9
    g.close()


def test_df_strips_cover_every_row():
    """p = 4 on 66 x 66 x 8 elements: the blocks walk two strips of 34 lines of direction
    1, plane after plane, in windows that start at even rows. Every row of M x and K x
    (3 vectors) matches the FP64 band product, and every launch shape gives the same
    bits as every other."""
    w = W.Workload("t", 3, (66, 66, 8), (4, 4, 4), 0.1, 3, 0.5, 1)
    g = _gpu(w, op_form="assembled")
    nvec = 3
    x = _t(np.random.default_rng(9).standard_normal(nvec * g.N))
    ref = {}
    for name, apply in (("M", g.apply_M), ("K", g.apply_K)):
        y = torch.empty_like(x)
        apply(x, y, nvec)
        ref[name] = _np(y)
    g.set_op_form("assembled_df")
    first = {}
    for threads in (96, 128, 64, 256):
        for nv in (1, 2, 3, 4):
            g.set_band_config(threads, nv)
            for name, apply in (("M", g.apply_M), ("K", g.apply_K)):
                y = torch.full_like(x, float("nan"))
                apply(x, y, nvec)
                Y = _np(y)
                r = ref[name]
                assert np.all(np.isfinite(Y)), (threads, nv, name)
                # M rows have terms of one sign; K rows cancel (bound relative to the largest entry)
                assert np.abs(Y - r).max() <= 1e-12 * np.abs(r).max(), (threads, nv, name, np.abs(Y - r).max())
                if name not in first:
                    first[name] = Y
                assert np.array_equal(Y, first[name]), (threads, nv, name)
    g.close()


def _tiny_share(P, A):
    """The share of an interior row's terms in tiny slots as the library forms them:
    slots whose largest coefficient is below 2^-24 after the power-of-two scaling that
    puts the matrix's largest in [1, 2), taken at the two ends of each run of slots with
    equal offsets along directions 1 and 2 (both ends tiny, working inwards)."""
    offs = P.slot_offsets()
    p = P.p
    smax = np.abs(A).max(axis=0) / 2.0 ** np.floor(np.log2(np.abs(A).max()))
    ratio = smax / 2.0 ** -24
    assert not np.any(np.abs(ratio - 1.0) < 1e-6)  # no slot at the cut (the probed band may round either way)
    tiny = smax < 2.0 ** -24
    m0 = 2 * p[0] + 1
    cheap, total = 0, 1
    for o2 in range(0, p[2] + 1):
        for o1 in range(-p[1], p[1] + 1):
            if (o2, o1) < (0, 0):
                continue
            o0s = list(range(1, p[0] + 1)) if (o1, o2) == (0, 0) else list(range(-p[0], p[0] + 1))
            total += 2 * len(o0s)
            if (o1, o2) == (0, 0):
                continue
            sl = [int(np.where((offs[:, 0] == a) & (offs[:, 1] == o1) & (offs[:, 2] == o2))[0][0]) for a in o0s]
            m = 0
            while m < (m0 + 1) // 2 and tiny[sl[m]] and tiny[sl[m0 - 1 - m]]:
                m += 1
            cheap += 2 * min(2 * m, m0)
    return cheap / total


@pytest.mark.parametrize("p", [2, 3, 4])
def test_df_tiny_share_matches_the_slot_magnitudes(p):
    """iga_band_df_tiny against the oracle band's slot magnitudes: none at p = 2, about a
    fifth of M's terms at p = 4."""
    w = W.small(d=3, nel=(8, 7, 6), p=p, amp=0.1)
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    Mr, Kr = P.assemble()
    g = _gpu(w, op_form="assembled_df")
    fm, fk = g.band_df_tiny()
    g.close()
    assert fm == pytest.approx(_tiny_share(P, Mr), abs=1e-12)
    assert fk == pytest.approx(_tiny_share(P, Kr), abs=1e-12)
    if p == 2:
        assert fm == 0.0 and fk == 0.0
    if p == 4:
        assert fm > 0.15 and fk > 0.1
