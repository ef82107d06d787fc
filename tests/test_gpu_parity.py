"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs.

Tolerances (FP64 on both sides; only the summation order differs):
  * operators: max |y_gpu - y_oracle| <= 1e-12 max |y_oracle| (M, P^{-1}), 1e-11 (K,
    whose rows sum terms of both signs);
  * PCG solves at tol 1e-13: relative L2 difference <= 1e-10, iteration counts within 1;
  * time stepping at tol 1e-13: relative L2 of U and V <= 1e-10 after the whole run.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _gpu(w, **kw):
    return iga.Patch(w.p, w.knots, w.ctrl(), **kw)


OPERATOR_CASES = {
    "2d_p23": W.Workload("t", 2, (4, 5), (2, 3), 0.1, 1, 0.5, 1),
    "3d_mixed_p": W.small(d=3, nel=(3, 4, 5), p=(2, 3, 2), amp=0.12),
    "3d_p4": W.small(d=3, nel=(5, 4, 3), p=4, amp=0.1),
    "3d_p1": W.small(d=3, nel=4, p=1, amp=0.1),
    "3d_ragged_p3": W.small(d=3, nel=(11, 9, 13), p=3, amp=0.1),
    "3d_identity_p2": W.small(d=3, nel=(6, 5, 7), p=2, amp=0.0),
    "2d_square32_p2": W.config("square32_p2"),
}


@pytest.fixture(scope="module", params=sorted(OPERATOR_CASES))
def case(request):
    w = OPERATOR_CASES[request.param]
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    g = _gpu(w, tol=1e-13)
    yield w, ops, g
    g.close()


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_operators_match_oracle(case):
    w, ops, g = case
    N = ops.N
    nvec = 3
    X = np.random.default_rng(7).standard_normal((nvec, N))
    x = _t(X)
    y = torch.empty_like(x)
    g.apply_M(x, y, nvec)
    Y = _np(y).reshape(nvec, N)
    for v in range(nvec):
        assert _maxrel(Y[v], ops.apply_M(X[v])) < 1e-12
    g.apply_K(x, y, nvec)
    Y = _np(y).reshape(nvec, N)
    for v in range(nvec):
        assert _maxrel(Y[v], ops.apply_K(X[v])) < 1e-11
    g.apply_Pinv(x, y, nvec)
    Y = _np(y).reshape(nvec, N)
    for v in range(nvec):
        assert _maxrel(Y[v], ops.apply_Pinv(X[v])) < 1e-12


def test_assembled_operators_match_oracle(case):
    """The assembled band form (probed from the matrix-free operators) against the
    oracle's Gauss-quadrature band rows."""
    w, ops, g = case
    g.set_op_form("assembled")
    try:
        N = ops.N
        X = np.random.default_rng(8).standard_normal((3, N))
        x = _t(X)
        y = torch.empty_like(x)
        g.apply_M(x, y, 3)
        Y = _np(y).reshape(3, N)
        for v in range(3):
            assert _maxrel(Y[v], ops.apply_M(X[v])) < 1e-12
        g.apply_K(x, y, 3)
        Y = _np(y).reshape(3, N)
        for v in range(3):
            assert _maxrel(Y[v], ops.apply_K(X[v])) < 1e-11
    finally:
        g.set_op_form("matrix_free")


def test_pcg_matches_oracle(case):
    w, ops, g = case
    N = ops.N
    B = np.random.default_rng(11).standard_normal((2, N))
    x = torch.zeros(2 * N, dtype=torch.float64, device=DEV)
    its, rel = g.solve_M(_t(B), x, nvec=2)
    Xg = _np(x).reshape(2, N)
    for v in range(2):
        xr, it_r, _ = oracle.pcg(ops.apply_M, ops.apply_Pinv, B[v], tol=1e-13)
        assert np.linalg.norm(Xg[v] - xr) / np.linalg.norm(xr) < 1e-10
        assert abs(its[v] - it_r) <= 1 and rel[v] <= 1e-13
    if w.amp == 0.0:  # identity map: the preconditioner is M itself
        assert max(its) <= 2


def test_identity_map_first_iteration_is_exact():
    w = W.small(d=3, nel=(6, 5, 7), p=3, amp=0.0)
    g = _gpu(w, tol=0.0, max_iter=1)
    b = torch.randn(g.N, dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(0))
    x = torch.zeros_like(b)
    with pytest.raises(iga.IgaError) as e:  # one iteration cannot reach tol 0, but gets to rounding level
        g.solve_M(b, x)
    assert e.value.status == iga.ENOT_CONVERGED
    y = torch.empty_like(b)
    g.apply_M(x, y)
    assert float(torch.linalg.norm(y - b) / torch.linalg.norm(b)) < 1e-11
    g.close()


def _oracle_run(w, ops, steps, dt, tol, guess="zero"):
    U0, V0 = w.initial()
    st = oracle.Stepper(ops, w.k, w.rho, tol=tol, guess=guess)
    X = st.init(U0, V0)
    for _ in range(steps):
        X = st.step(X, dt)
    return X, st.iters


def _gpu_run(w, steps, dt, tol, guess="zero", precond="fp64", op_form="matrix_free"):
    U0, V0 = w.initial()
    g = _gpu(w, tol=tol, guess=guess, precond=precond, op_form=op_form)
    state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(w.k, _t(U0), _t(V0), state)
    st = g.step(state, w.k, w.rho, dt, steps)
    out = _np(state).reshape(3 * w.k, g.N)
    g.close()
    return out, st


def _dt(ops, rho, frac=0.5):
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    return frac * math.sqrt(oracle.theta_crit(rho) / lmax)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_step_matches_oracle(k, rho):
    w = W.small(d=3, nel=(4, 3, 5), p=2, amp=0.1, k=k, rho=rho)
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, rho)
    steps = 12
    Xo, _ = _oracle_run(w, ops, steps, dt, 1e-13)
    Xg, st = _gpu_run(w, steps, dt, 1e-13)
    assert st.steps == steps and st.solves == k * steps
    for row in (0, 1):
        err = np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row])
        assert err < 1e-10, (row, err)


@pytest.mark.parametrize("precond", ["fp64", "fp32", "banded"])
@pytest.mark.parametrize("k", [2, 3])
def test_assembled_step_matches_oracle(k, precond):
    w = W.small(d=3, nel=(5, 4, 6), p=3, amp=0.1, k=k, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    Xo, _ = _oracle_run(w, ops, 10, dt, 1e-13)
    Xg, _ = _gpu_run(w, 10, dt, 1e-13, precond=precond, op_form="assembled")
    for row in (0, 1):
        err = np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row])
        print("assembled form, precond %s, k=%d, row %d: rel L2 %.3e" % (precond, k, row, err))
        assert err < 1e-10, (row, err)


@pytest.mark.parametrize("guess", ["prev", "extrap", "taylor"])
def test_guesses_match_oracle(guess):
    w = W.small(d=3, nel=(5, 4, 4), p=3, amp=0.1, k=2, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    Xo, it_o = _oracle_run(w, ops, 8, dt, 1e-12, guess=guess)
    Xg, st = _gpu_run(w, 8, dt, 1e-12, guess=guess)
    for row in (0, 1):
        assert np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row]) < 1e-9
    assert abs(st.iters - sum(sum(i) for i in it_o)) <= 8


def test_square32_full_run():
    """2-D unit square, identity map, p=2, 32x32 elements, k=1, rho=0.5, dt = 0.5 tau_crit, 100 steps."""
    w = W.config("square32_p2")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    Xo, _ = _oracle_run(w, ops, w.steps, dt, 1e-13)
    Xg, st = _gpu_run(w, w.steps, dt, 1e-13)
    for row in (0, 1):
        err = np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row])
        assert err < 1e-10, (row, err)
    # identity map: every solve takes one iteration (two when rounding sits at the threshold)
    assert st.max_iters <= 2


def test_nonuniform_repeated_knots():
    U = np.array([0, 0, 0, 0, 0.15, 0.3, 0.3, 0.55, 0.8, 1, 1, 1, 1.0])
    V = np.array([0, 0, 0, 0.25, 0.4, 0.4, 0.7, 1, 1, 1.0])
    Wk = W.open_uniform_knots(4, 2)
    knots, p = [U, V, Wk], [3, 2, 2]
    ctrl = W.control_net(knots, p, 0.08)
    P = oracle.Patch(p, knots, ctrl)
    ops = oracle.Operators(P)
    g = iga.Patch(p, knots, ctrl, tol=1e-13)
    X = np.random.default_rng(3).standard_normal(ops.N)
    y = torch.empty(ops.N, dtype=torch.float64, device=DEV)
    g.apply_M(_t(X), y)
    assert _maxrel(_np(y), ops.apply_M(X)) < 1e-12
    g.apply_K(_t(X), y)
    assert _maxrel(_np(y), ops.apply_K(X)) < 1e-11
    g.apply_Pinv(_t(X), y)
    assert _maxrel(_np(y), ops.apply_Pinv(X)) < 1e-12
    g.close()


@pytest.mark.parametrize("form", [("matrix_free", "fp64", "zero"), ("assembled", "fp32", "zero"),
                                  ("assembled", "fp64", "extrap"), ("assembled", "bf16", "taylor"),
                                  ("assembled", "fp16", "zero"), ("assembled", "banded", "zero"),
                                  ("assembled", "banded32", "zero")])
def test_graph_replay_equals_host_loop(form):
    """The captured step (PCG loop on the device) and the host-driven loop run the same
    kernels in the same order: bitwise equal states and equal iteration counts."""
    op, prec, guess = form
    w = W.small(d=3, nel=(6, 5, 7), p=3, amp=0.1, k=2, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    U0, V0 = w.initial()
    out = []
    for graphs in (False, True):
        g = _gpu(w, tol=1e-11, op_form=op, precond=prec, guess=guess)
        g.set_graphs(graphs)
        state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
        g.state_init(w.k, _t(U0), _t(V0), state)
        st = g.step(state, w.k, w.rho, dt, 4)
        st = g.step(state, w.k, w.rho, dt, 6, st)  # a second call replays the cached graph
        out.append((_np(state), st.iters, st.max_iters, st.steps))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_deterministic_bitwise():
    w = W.small(d=3, nel=(6, 5, 4), p=3, amp=0.1, k=2)
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    a, _ = _gpu_run(w, 5, dt, 1e-10)
    b, _ = _gpu_run(w, 5, dt, 1e-10)
    assert np.array_equal(a, b)


def test_folded_geometry_is_rejected():
    w = W.small(d=3, nel=3, p=2, amp=2.5)
    with pytest.raises(iga.IgaError) as e:
        _gpu(w)
    assert e.value.status == iga.EGEOMETRY


def test_max_iter_reports_not_converged():
    w = W.small(d=3, nel=5, p=3, amp=0.15)
    g = _gpu(w, tol=1e-14, max_iter=1)
    b = torch.ones(g.N, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    with pytest.raises(iga.IgaError) as e:
        g.solve_M(b, x)
    assert e.value.status == iga.ENOT_CONVERGED
    g.close()


@pytest.mark.parametrize("name", list(OPERATOR_CASES))
def test_banded_preconditioner_matches_oracle(name):
    """FP64 Kronecker solve by band Cholesky along each direction: the same operator
    as the oracle's (LAPACK band Cholesky) to FP64 rounding."""
    w = OPERATOR_CASES[name]
    pre = oracle.Preconditioner(oracle.Patch(w.p, w.knots, w.ctrl()))
    g = _gpu(w, precond="banded")
    X = np.random.default_rng(3).standard_normal((3, pre.N))
    y = torch.empty(3 * pre.N, dtype=torch.float64, device=DEV)
    g.apply_Pinv(_t(X), y, 3)
    Y = _np(y).reshape(3, pre.N)
    for v in range(3):
        assert _maxrel(Y[v], pre.apply_Pinv(X[v])) < 1e-12
    g.close()


def test_banded_preconditioner_iterations_equal_fp64_fd():
    """Both FP64 preconditioners apply the same operator: the same PCG iteration counts."""
    w = W.small(d=3, nel=(7, 6, 5), p=3, amp=0.1, k=2, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    _, sa = _gpu_run(w, 6, dt, 1e-11, precond="fp64", op_form="assembled")
    _, sb = _gpu_run(w, 6, dt, 1e-11, precond="banded", op_form="assembled")
    assert sa.iters == sb.iters and sa.max_iters == sb.max_iters


# FP32 mode products: FP32 rounding; BF16 (tensor cores): 8-bit significand operands
# (unit roundoff 2^-9), FP32 accumulation over six mode products -> about 1e-2
# norm-wise; FP16: 11-bit significand (unit roundoff 2^-11, 4x smaller) after an
# exact per-line power-of-two scaling.
PRECOND_TOL = {"fp32": 1e-5, "bf16": 5e-2, "fp16": 5e-2 / 4, "banded32": 1e-5}


@pytest.mark.parametrize("precond", ["fp32", "bf16", "fp16", "banded32"])
@pytest.mark.parametrize("name", ["3d_mixed_p", "3d_ragged_p3", "2d_square32_p2", "3d_p4"])
def test_low_precision_preconditioner_close_to_oracle(name, precond):
    """Norm-wise relative error of P^{-1} r against the FP64 oracle at the arithmetic's level."""
    w = OPERATOR_CASES[name]
    pre = oracle.Preconditioner(oracle.Patch(w.p, w.knots, w.ctrl()))
    g = _gpu(w, precond=precond)
    X = np.random.default_rng(2).standard_normal((2, pre.N))
    y = torch.empty(2 * pre.N, dtype=torch.float64, device=DEV)
    g.apply_Pinv(_t(X), y, 2)
    Y = _np(y).reshape(2, pre.N)
    for v in range(2):
        ref = pre.apply_Pinv(X[v])
        err = np.linalg.norm(Y[v] - ref) / np.linalg.norm(ref)
        assert err < PRECOND_TOL[precond], err
    g.close()


@pytest.mark.parametrize("precond", ["bf16", "fp16"])
def test_tensor_core_preconditioner_cube64(precond):
    """The tensor-core forms at full size (n = 65 per direction, 2146 line tiles per mode)."""
    w = W.config("cube64_p3")
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    pre = oracle.Preconditioner(P)
    g = _gpu(w, precond=precond)
    X = np.random.default_rng(6).standard_normal(P.N)
    y = torch.empty(P.N, dtype=torch.float64, device=DEV)
    g.apply_Pinv(_t(X), y)
    ref = pre.apply_Pinv(X)
    assert np.linalg.norm(_np(y) - ref) / np.linalg.norm(ref) < PRECOND_TOL[precond]
    g.close()


@pytest.mark.parametrize("precond", ["bf16", "fp16"])
@pytest.mark.parametrize("e", [60, -60])
def test_tensor_core_preconditioner_is_exactly_homogeneous(precond, e):
    """Scaling the input by 2^e scales the output by 2^e bitwise: FP16's per-line
    power-of-two scaling is exact, and neither form under- or overflows."""
    w = OPERATOR_CASES["3d_ragged_p3"]
    g = _gpu(w, precond=precond)
    X = np.random.default_rng(12).standard_normal(2 * g.N)
    X[: g.N // 3] *= 1e-9  # lines of very different magnitudes
    y0 = torch.empty(2 * g.N, dtype=torch.float64, device=DEV)
    y1 = torch.empty_like(y0)
    g.apply_Pinv(_t(X), y0, 2)
    g.apply_Pinv(_t(np.ldexp(X, e)), y1, 2)
    assert np.array_equal(np.ldexp(_np(y0), e), _np(y1))
    g.close()


@pytest.mark.parametrize("precond", ["fp32", "bf16", "fp16", "banded32"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_step_with_low_precision_preconditioner_matches_fp64_oracle(k, precond):
    """Flexible PCG with an FP32 or BF16 preconditioner reaches the same FP64 tolerance, so
    the trajectory matches the FP64 oracle to the solver tolerance."""
    w = W.small(d=3, nel=(5, 4, 6), p=3, amp=0.1, k=k, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    Xo, it_o = _oracle_run(w, ops, 10, dt, 1e-12)
    Xg, st = _gpu_run(w, 10, dt, 1e-12, precond=precond)
    for row in (0, 1):
        err = np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row])
        assert err < 1e-9, (row, err)
    extra = 2 if precond in ("fp32", "banded32") else 6
    assert st.iters <= sum(sum(i) for i in it_o) + extra * st.solves


def test_cube64_sampled_rows_and_preconditioner():
    """Full size (3-D deformed cube, p=3, 64^3 elements, N = 274625): M x and K x on a
    seeded sample of rows against the oracle's Gauss-quadrature rows, and the full
    preconditioner against the oracle's banded-Cholesky Kronecker solve."""
    w = W.config("cube64_p3")
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    rows = W.sample_indices(P.N, 300, seed=5)
    Mr, Kr = P.assemble(rows)
    g = _gpu(w)
    X = np.random.default_rng(1).standard_normal(P.N)
    y = torch.empty(P.N, dtype=torch.float64, device=DEV)
    g.apply_M(_t(X), y)
    ym = _np(y)[rows]
    ref = P.band_rows_times(rows, Mr, X)
    assert np.abs(ym - ref).max() < 1e-12 * np.abs(ref).max()
    g.apply_K(_t(X), y)
    yk = _np(y)[rows]
    ref = P.band_rows_times(rows, Kr, X)
    assert np.abs(yk - ref).max() < 1e-11 * np.abs(ref).max()
    pre = oracle.Preconditioner(P)
    g.apply_Pinv(_t(X), y)
    assert _maxrel(_np(y), pre.apply_Pinv(X)) < 1e-11
    g.close()


SMALLEST = [W.Workload("s1", 3, (1, 3, 2), (2, 2, 2), 0.1, 2, 0.5, 3, init="random"),
            W.Workload("s2", 3, (1, 1, 1), (2, 2, 2), 0.1, 2, 0.5, 3, init="random"),
            W.Workload("s3", 3, (2, 1, 3), (3, 2, 2), 0.1, 1, 0.5, 3, init="random"),
            W.Workload("s4", 2, (3, 2), (1, 1), 0.1, 2, 0.5, 3, init="random")]


@pytest.mark.parametrize("precond", ["fp64", "fp32", "bf16", "fp16", "banded", "banded32"])
@pytest.mark.parametrize("wi", range(len(SMALLEST)))
def test_smallest_patches(wi, precond):
    """Degenerate sizes: one interior function in some directions (N = 1 for one element
    of degree 2 per direction); operators, preconditioner and steps against the oracle."""
    w = SMALLEST[wi]
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    g = _gpu(w, tol=1e-12, precond=precond, op_form="assembled")
    X = np.random.default_rng(13).standard_normal(ops.N)
    y = torch.empty(ops.N, dtype=torch.float64, device=DEV)
    g.apply_M(_t(X), y)
    assert _maxrel(_np(y), ops.apply_M(X)) < 1e-12
    g.apply_K(_t(X), y)
    assert _maxrel(_np(y), ops.apply_K(X)) < 1e-11
    g.apply_Pinv(_t(X), y)
    assert _maxrel(_np(y), ops.apply_Pinv(X)) < (1e-12 if precond in ("fp64", "banded") else 5e-2)
    g.close()
    dt = _dt(ops, w.rho)
    Xo, _ = _oracle_run(w, ops, w.steps, dt, 1e-12)
    Xg, st = _gpu_run(w, w.steps, dt, 1e-12, precond=precond, op_form="assembled")
    for row in (0, 1):
        den = max(np.linalg.norm(Xo[row]), 1e-300)
        assert np.linalg.norm(Xg[row] - Xo[row]) / den < 1e-9, (row,)
    if ops.N == 1:
        assert st.max_iters <= 1  # the preconditioner is the exact inverse of a 1 x 1 mass matrix


@pytest.mark.parametrize("case", ["3d_mixed_p", "2d_p23"])
@pytest.mark.parametrize("form", [("matrix_free", "fp64"), ("assembled", "banded32"), ("assembled", "bf16")])
def test_cfl_lambda_max_matches_dense_eigenvalue(case, form):
    """iga_cfl's Lanczos estimate of lambda_max(M^{-1} K) against the dense generalised
    eigenvalue, and tau_crit = sqrt(Theta_crit / lambda_max) with Theta_crit the stability
    limit of the characteristic equation."""
    w = OPERATOR_CASES[case]
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    g = _gpu(w, tol=1e-10, op_form=form[0], precond=form[1])
    lam, tc = g.cfl(0.5, iters=min(ops.N, 200))
    g.close()
    assert abs(lam - lmax) <= 1e-8 * lmax
    assert abs(tc - math.sqrt(oracle.theta_crit(0.5) / lmax)) <= 1e-8 * tc
