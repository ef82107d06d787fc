"""Pins of the CPU oracle to facts fixed by the paper and by mathematics, independent
of the oracle's own formulas: library routines (numpy Gauss rule, scipy B-splines,
scipy adaptive quadrature, dense LAPACK solves and eigendecompositions), closed forms,
the paper's printed amplification blocks and characteristic polynomials
(tests/golden/), a textbook special case (Hulbert-Chung explicit generalized-alpha)
and brute force on tiny meshes."""
import cmath
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.interpolate
import scipy.linalg

import oracle
import workloads as W
from conftest import read_golden

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


# ----------------------------------------------------------------------------- quadrature, basis
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-14, rtol=0) and np.allclose(w, wr, atol=1e-14, rtol=0)
    for deg in range(2 * n):
        exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
        assert abs(np.sum(w * x ** deg) - exact) < 1e-13


def _knot_cases():
    yield 1, W.open_uniform_knots(5, 1)
    yield 2, W.open_uniform_knots(6, 2)
    yield 3, W.open_uniform_knots(7, 3)
    yield 4, W.open_uniform_knots(5, 4)
    yield 3, np.array([0, 0, 0, 0, 0.1, 0.35, 0.35, 0.6, 0.9, 1, 1, 1, 1.0])  # non-uniform, repeated knot
    yield 2, np.array([0, 0, 0, 0.2, 0.2, 0.5, 0.7, 1, 1, 1.0])


@pytest.mark.parametrize("case", list(range(6)))
def test_basis_matches_scipy_bspline(case):
    p, U = list(_knot_cases())[case]
    m = len(U) - p - 1
    xs = np.random.default_rng(case).uniform(0, 1, 25)
    for x in xs:
        val, der = oracle.basis(p, U, x)
        for i in range(m):
            c = np.zeros(m)
            c[i] = 1.0
            spl = scipy.interpolate.BSpline(U, c, p, extrapolate=False)
            assert abs(val[i] - spl(x)) < 1e-13
            if p > 0:
                assert abs(der[i] - spl.derivative()(x)) < 1e-11
        assert abs(val.sum() - 1.0) < 1e-14  # partition of unity (eq. partition_unity)
        assert abs(der.sum()) < 1e-10


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_greville_reproduces_linear(p):
    U = W.open_uniform_knots(6, p)
    g = W.greville(U, p)
    for x in np.linspace(0, 1, 13):
        val, der = oracle.basis(p, U, x)
        assert abs(val @ g - x) < 1e-14
        assert abs(der @ g - 1.0) < 1e-12


# ----------------------------------------------------------------------------- 1-D matrices
def test_mass_1d_p1_closed_form():
    nel = 8
    q = oracle.Quad1D(1, W.open_uniform_knots(nel, 1), 2)
    h = 1.0 / nel
    M = q.mass_interior()
    n = nel - 1
    ref = h / 6 * (4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))
    assert np.abs(M - ref).max() < 1e-15


def _scipy_gram(p, U, deriv):
    m = len(U) - p - 1
    spl = []
    for i in range(1, m - 1):
        c = np.zeros(m)
        c[i] = 1
        s = scipy.interpolate.BSpline(U, c, p, extrapolate=False)
        spl.append(s.derivative() if deriv else s)
    n = len(spl)
    breaks = np.unique(U)
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - p), min(n, i + p + 1)):
            tot = 0.0
            for a, b in zip(breaks[:-1], breaks[1:]):
                tot += scipy.integrate.quad(lambda x: np.nan_to_num(spl[i](x)) * np.nan_to_num(spl[j](x)), a, b,
                                            epsabs=1e-15, epsrel=1e-13)[0]
            G[i, j] = tot
    return G


@pytest.mark.parametrize("case", [1, 2, 3, 4])
def test_mass_and_stiffness_1d_match_adaptive_quadrature(case):
    p, U = list(_knot_cases())[case]
    q = oracle.Quad1D(p, U, p + 1)
    assert np.abs(q.mass_interior() - _scipy_gram(p, U, False)).max() < 1e-13
    assert np.abs(q.stiffness_interior() - _scipy_gram(p, U, True)).max() < 1e-10


@pytest.mark.parametrize("p", [2, 3, 4])
def test_interior_mass_stencil_is_cardinal_spline_autocorrelation(p):
    # int N_p(x) N_p(x + k) dx = N_{2p+1}(p + 1 + k) for the cardinal B-spline N_p on [0, p+1]
    nel = 4 * p + 8
    h = 1.0 / nel
    q = oracle.Quad1D(p, W.open_uniform_knots(nel, p), p + 1)
    M = q.mass_interior()
    Kst = q.stiffness_interior()
    N2 = scipy.interpolate.BSpline.basis_element(np.arange(2 * p + 3), extrapolate=False)
    i = M.shape[0] // 2
    for k in range(0, p + 1):
        assert abs(M[i, i + k] / h - N2(p + 1 + k)) < 1e-13
        assert abs(Kst[i, i + k] * h + N2.derivative(2)(p + 1 + k)) < 1e-11


# ----------------------------------------------------------------------------- 2-D/3-D operators
def _patch(w):
    return oracle.Patch(w.p, w.knots, w.ctrl())


@pytest.mark.parametrize("d,nel,p", [(2, (4, 5), (2, 3)), (3, (3, 4, 3), (2, 2, 3)), (3, (3, 3, 3), (1, 1, 1))])
def test_identity_map_is_kronecker(d, nel, p):
    w = W.Workload("t", d, nel, p, 0.0, 1, 0.5, 1)
    P = _patch(w)
    M, K = P.assemble()
    Md, Kd = P.band_to_dense(M), P.band_to_dense(K)
    Mh = [q.mass_interior() for q in P.q1]
    Kh = [q.stiffness_interior() for q in P.q1]
    kron = lambda mats: mats[0] if len(mats) == 1 else np.kron(kron(mats[1:]), mats[0])  # co-lex
    Mref = kron(Mh)
    Kref = np.zeros_like(Mref)
    for a in range(d):
        Kref += kron([Kh[b] if b == a else Mh[b] for b in range(d)])
    assert np.abs(Md - Mref).max() < 1e-14 * np.abs(Mref).max() * 10
    assert np.abs(Kd - Kref).max() < 1e-12 * np.abs(Kref).max()


def _brute_entries(w, pairs):
    """M_ij and K_ij recomputed in numpy from scipy B-splines, same Gauss rule (brute force)."""
    d = w.d
    knots = w.knots
    ctrl = w.ctrl()
    mfull = w.m
    xg, wg = np.polynomial.legendre.leggauss(max(w.p) + 1)
    pts, wts = [], []
    for a in range(d):
        br = np.unique(knots[a])
        xa, wa = [], []
        for lo, hi in zip(br[:-1], br[1:]):
            xa += list(lo + (hi - lo) * (xg + 1) / 2)
            wa += list((hi - lo) / 2 * wg)
        pts.append(np.array(xa))
        wts.append(np.array(wa))
    tabs = []
    for a in range(d):
        B = np.zeros((len(pts[a]), mfull[a]))
        dB = np.zeros_like(B)
        for i in range(mfull[a]):
            c = np.zeros(mfull[a])
            c[i] = 1
            s = scipy.interpolate.BSpline(knots[a], c, w.p[a])
            B[:, i] = s(pts[a])
            dB[:, i] = s.derivative()(pts[a])
        tabs.append((B, dB))
    grid = ctrl.reshape(tuple(reversed(mfull)) + (d,))  # [i_{d-1}..i_0, coord]
    # DF at every quadrature point: DF[c, b] = sum_i C_ic dB_i/dxi_b
    out = []
    for (i, j) in pairs:
        ni = np.unravel_index(i, tuple(reversed(w.n)))[::-1]
        nj = np.unravel_index(j, tuple(reversed(w.n)))[::-1]
        Mij = 0.0
        Kij = 0.0
        for qs in np.ndindex(*[len(pts[a]) for a in range(d)]):
            vals_i = [tabs[a][0][qs[a], ni[a] + 1] for a in range(d)]
            vals_j = [tabs[a][0][qs[a], nj[a] + 1] for a in range(d)]
            if np.prod(vals_i) == 0 and all(tabs[a][1][qs[a], ni[a] + 1] == 0 for a in range(d)):
                continue
            J = np.zeros((d, d))
            for b in range(d):
                fac = [tabs[a][1][qs[a]] if a == b else tabs[a][0][qs[a]] for a in range(d)]
                for c in range(d):
                    t = grid[..., c]
                    for a in range(d):  # the last axis is i_0, then i_1, ...
                        t = t @ fac[a]
                    J[c, b] = t
            wq = np.prod([wts[a][qs[a]] for a in range(d)])
            det = np.linalg.det(J)
            gi = np.array([np.prod([tabs[a][1 if a == b else 0][qs[a], ni[a] + 1] for a in range(d)]) for b in range(d)])
            gj = np.array([np.prod([tabs[a][1 if a == b else 0][qs[a], nj[a] + 1] for a in range(d)]) for b in range(d)])
            Ji = np.linalg.inv(J)
            Mij += np.prod(vals_i) * np.prod(vals_j) * abs(det) * wq
            Kij += gi @ (Ji @ Ji.T) @ gj * abs(det) * wq
        out.append((Mij, Kij))
    return out


def test_deformed_entries_match_brute_force():
    w = W.Workload("t", 3, (3, 3, 3), (2, 2, 2), 0.12, 1, 0.5, 1)
    P = _patch(w)
    M, K = P.assemble()
    Md, Kd = P.band_to_dense(M), P.band_to_dense(K)
    rng = np.random.default_rng(3)
    pairs = [(0, 0), (P.N - 1, P.N - 1), (0, 1), (5, 13)]
    pairs += [tuple(int(v) for v in rng.integers(0, P.N, 2)) for _ in range(4)]
    ref = _brute_entries(w, pairs)
    for (i, j), (m_ref, k_ref) in zip(pairs, ref):
        assert abs(Md[i, j] - m_ref) < 1e-14 + 1e-12 * abs(m_ref)
        assert abs(Kd[i, j] - k_ref) < 1e-12 + 1e-10 * abs(k_ref)
    # symmetric positive definite
    assert np.abs(Md - Md.T).max() < 1e-16 + 1e-14 * np.abs(Md).max()
    assert np.linalg.eigvalsh(Md).min() > 0 and np.linalg.eigvalsh(Kd).min() > 0


def test_deformed_2d_entries_match_brute_force():
    w = W.Workload("t", 2, (4, 3), (3, 2), 0.1, 1, 0.5, 1)
    P = _patch(w)
    M, K = P.assemble()
    Md, Kd = P.band_to_dense(M), P.band_to_dense(K)
    pairs = [(0, 0), (1, 6), (P.N - 1, P.N - 2), (7, 7)]
    for (i, j), (m_ref, k_ref) in zip(pairs, _brute_entries(w, pairs)):
        assert abs(Md[i, j] - m_ref) < 1e-14 + 1e-12 * abs(m_ref)
        assert abs(Kd[i, j] - k_ref) < 1e-12 + 1e-10 * abs(k_ref)


def test_sampled_rows_equal_full_assembly():
    w = W.small(d=3, nel=4, p=3, amp=0.1)
    P = _patch(w)
    M, K = P.assemble()
    rows = W.sample_indices(P.N, 9, seed=1)
    Ms, Ks = P.assemble(rows)
    assert np.array_equal(Ms, M[rows]) and np.array_equal(Ks, K[rows])


def test_mass_diagonal_equals_assembled_diagonal():
    for w in (W.small(d=3, nel=(3, 4, 5), p=(2, 3, 2), amp=0.1), W.small(d=2, nel=(5, 4), p=3, amp=0.1)):
        P = _patch(w)
        M, _ = P.assemble(stiffness=False)
        assert np.abs(P.mass_diagonal() - M[:, P.nslots // 2]).max() < 1e-15 * np.abs(M).max() * 10


def test_rejects_folded_geometry():
    w = W.Workload("t", 3, (3, 3, 3), (2, 2, 2), 2.5, 1, 0.5, 1)
    with pytest.raises(ValueError):
        _patch(w)


def test_band_matvec_equals_dense():
    w = W.small(d=3, nel=(3, 4, 5), p=(2, 3, 2), amp=0.1)
    P = _patch(w)
    M, K = P.assemble()
    x = np.random.default_rng(0).standard_normal(P.N)
    assert np.allclose(P.band_matvec(M, x), P.band_to_dense(M) @ x, rtol=0, atol=1e-15)
    assert np.allclose(P.band_matvec(K, x), P.band_to_dense(K) @ x, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- preconditioner, PCG
def test_preconditioner_is_inverse_of_dense_definition():
    w = W.small(d=3, nel=(3, 4, 3), p=(2, 3, 2), amp=0.1)
    P = _patch(w)
    ops = oracle.Operators(P)
    Mh = [q.mass_interior() for q in P.q1]
    Mhat = np.kron(np.kron(Mh[2], Mh[1]), Mh[0])
    Dhat = np.diag(np.diag(Mhat))
    D = np.diag(np.diag(P.band_to_dense(ops.M)))
    s = lambda A, e: np.diag(np.diag(A) ** e)
    Pm = s(D, .5) @ s(Dhat, -.5) @ Mhat @ s(Dhat, -.5) @ s(D, .5)  # def:single_patch_prec
    r = np.random.default_rng(1).standard_normal(P.N)
    assert np.allclose(ops.apply_Pinv(r), np.linalg.solve(Pm, r), rtol=1e-12, atol=0)


@pytest.mark.parametrize("d,p", [(2, 2), (3, 3), (3, 4)])
def test_identity_map_pcg_converges_in_one_iteration(d, p):
    # F = identity => D = Dhat and M = Mhat, so the preconditioner is M itself: one PCG
    # iteration leaves only rounding (about eps * cond(M), cond ~ 2e5 for p = 4 in 3-D),
    # while on a deformed map one iteration is far from converged.
    b = np.random.default_rng(2).standard_normal(int(np.prod([5 + p - 2] * d)))
    rr = {}
    for amp in (0.0, 0.1):
        ops = oracle.Operators(_patch(W.small(d=d, nel=5, p=p, amp=amp)))
        _, it, rr[amp] = oracle.pcg(ops.apply_M, ops.apply_Pinv, b, tol=0.0, max_iter=1)
        assert it == 1
    assert rr[0.0] < 1e-10 and rr[0.1] > 1e-4


def test_pcg_matches_dense_solve():
    w = W.small(d=3, nel=4, p=2, amp=0.15)
    ops = oracle.Operators(_patch(w))
    Md = ops.patch.band_to_dense(ops.M)
    b = np.random.default_rng(5).standard_normal(ops.N)
    x, it, rr = oracle.pcg(ops.apply_M, ops.apply_Pinv, b, tol=1e-14)
    xr = scipy.linalg.solve(Md, b, assume_a="pos")
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-12
    assert 1 < it < 30


# ----------------------------------------------------------------------------- time scheme
def _eval(expr, a, b, g, T):
    return eval(expr, {"a": a, "b": b, "g": g, "T": T})


@pytest.mark.parametrize("k", [2, 3, 4])
def test_amplification_blocks_match_printed(k):
    gold = read_golden("amplification_blocks.txt")
    rng = np.random.default_rng(k)
    for _ in range(5):
        prm = [(rng.uniform(0.5, 2), rng.uniform(0, 1), rng.uniform(0, 2), 0.0) for _ in range(k)]
        T = rng.uniform(0.1, 3)
        G = oracle.scalar_amplification(k, 0.0, T, params=prm)
        for j in range(k):
            a, b, g, _ = prm[j]
            sec = "block j=k" if j == k - 1 else "block j<k"
            ref = np.array([[_eval(e, a, b, g, T) for e in row] for row in gold[sec]]) / a
            assert np.abs(G[3 * j:3 * j + 3, 3 * j:3 * j + 3] - ref).max() < 1e-13
            assert np.abs(G[3 * j + 3:, 3 * j:3 * j + 3]).max() == 0.0 if j < k - 1 else True  # block upper-triangular


def test_characteristic_polynomials_match_printed():
    gold = read_golden("characteristic_polynomials.txt")
    rng = np.random.default_rng(0)
    for _ in range(5):
        prm = [(rng.uniform(0.5, 2), rng.uniform(0, 1), rng.uniform(0, 2), 0.0) for _ in range(2)]
        T = rng.uniform(0.1, 3)
        G = oracle.scalar_amplification(2, 0.0, T, params=prm)
        for j, sec in enumerate(["block j<k", "block j=k"]):
            a, b, g, _ = prm[j]
            c = np.array([_eval(e, a, b, g, T) for e in gold[sec][0]])
            ev = np.linalg.eigvals(G[3 * j:3 * j + 3, 3 * j:3 * j + 3])
            assert np.abs(np.polyval(c / c[0], ev)).max() < 1e-10


def test_last_block_is_hulbert_chung():
    # Hulbert-Chung explicit generalized-alpha (textbook): alpha_m = (2 rho - 1)/(1 + rho),
    # beta = (5 - 3 rho)/((1 + rho)^2 (2 - rho)), gamma = 3/2 - alpha_m; the paper's
    # alpha = 1 - alpha_m (it weights the new acceleration).
    for rho in [0.0, 0.3, 0.5, 0.8, 1.0]:
        a, b, g, af = oracle.galpha_params(1, rho)[0]
        am = (2 * rho - 1) / (1 + rho)
        assert abs(a - (1 - am)) < 1e-15
        assert abs(b - (5 - 3 * rho) / ((1 + rho) ** 2 * (2 - rho))) < 1e-15
        assert abs(g - (1.5 - am)) < 1e-15 and af == 0.0


def test_k1_trajectory_equals_hulbert_chung():
    w = W.small(d=2, nel=4, p=2, amp=0.1, k=1)
    ops = oracle.Operators(_patch(w))
    Md, Kd = ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K)
    U0, V0 = w.initial()
    rho, tau = 0.4, 0.002
    st = oracle.Stepper(ops, 1, rho, tol=1e-15)
    X = st.init(U0, V0)
    am = (2 * rho - 1) / (1 + rho)
    beta = (5 - 3 * rho) / ((1 + rho) ** 2 * (2 - rho))
    gam = 1.5 - am
    d, v = U0.copy(), V0.copy()
    a = np.linalg.solve(Md, -Kd @ d)
    for _ in range(20):
        X = st.step(X, tau)
        # M ((1 - am) a1 + am a0) = -K d_n
        a1 = (np.linalg.solve(Md, -Kd @ d) - am * a) / (1 - am)
        d = d + tau * v + tau ** 2 * ((0.5 - beta) * a + beta * a1)
        v = v + tau * ((1 - gam) * a + gam * a1)
        a = a1
    assert np.linalg.norm(X[0] - d) / np.linalg.norm(d) < 1e-12
    assert np.linalg.norm(X[1] - v) / np.linalg.norm(v) < 1e-11


def test_theta_crit_is_the_minus_one_root_of_printed_polynomial():
    gold = read_golden("characteristic_polynomials.txt")
    for rho in [0.0, 0.25, 0.5, 0.75, 1.0]:
        a, b, g, _ = oracle.galpha_params(1, rho)[0]
        T = oracle.theta_crit(rho)
        c = np.array([_eval(e, a, b, g, T) for e in gold["block j=k"][0]])
        assert abs(np.polyval(c, -1.0)) < 1e-12
    assert abs(oracle.theta_crit(1.0) - 4.0) < 1e-15  # central-difference limit (Sec. 3.2)
    assert abs(oracle.theta_crit(0.0) - 2.4) < 1e-15


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9, 1.0])
def test_stability_limit_independent_of_k(rho):
    Tc = oracle.theta_crit(rho)
    for k in (1, 2, 3):
        sr_in = max(abs(np.linalg.eigvals(oracle.scalar_amplification(k, rho, Tc * 0.999))))
        sr_out = max(abs(np.linalg.eigvals(oracle.scalar_amplification(k, rho, Tc * 1.01))))
        assert sr_in <= 1 + 1e-6 and sr_out > 1 + 1e-4


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_spectral_radius_at_bifurcation_equals_rho(rho):
    # Omega_b = 2 + 2 rho_b + rho_s - rho_s rho_b^2 (boxed formulas) at rho_b = rho_s = rho:
    # all roots of each block equal -rho there, so the spectral radius is rho for every k.
    Ob = 2 + 3 * rho - rho ** 3
    for k in (1, 2, 3):
        G = oracle.scalar_amplification(k, rho, Ob)
        for j in range(k):
            ev = np.linalg.eigvals(G[3 * j:3 * j + 3, 3 * j:3 * j + 3])
            assert abs(max(abs(ev)) - rho) < 2e-5


def _modal_error(k, rho, n, lam=1.0, T=1.0):
    st = oracle.Stepper(oracle.ScalarOps(lam), k, rho, tol=0.0)
    w = math.sqrt(lam)
    X = np.zeros((3 * k, 1))
    for r in range(3 * k):  # derivatives of cos(w t) at 0
        X[r, 0] = (-1) ** (r // 2) * w ** r if r % 2 == 0 else 0.0
    eu = ev = 0.0
    for s in range(1, n + 1):  # max over the time grid (robust to zero crossings of the error)
        X = st.step(X, T / n)
        t = s * T / n
        eu = max(eu, abs(X[0, 0] - math.cos(w * t)))
        ev = max(ev, abs(X[1, 0] + w * math.sin(w * t)))
    return eu, ev


@pytest.mark.parametrize("k,ns,minorder", [(1, (40, 80), 1.9), (2, (20, 40), 3.85), (3, (16, 32), 5.5)])
@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_modal_order_is_2k(k, ns, minorder, rho):
    e1 = _modal_error(k, rho, ns[0], lam=4.0)
    e2 = _modal_error(k, rho, ns[1], lam=4.0)
    for a, b in zip(e1, e2):
        assert math.log2(a / b) > minorder


@pytest.mark.parametrize("k", [1, 2, 3])
def test_semidiscrete_temporal_order(k):
    w = W.small(d=3, nel=3, p=2, amp=0.1, k=k)
    ops = oracle.Operators(_patch(w))
    Md, Kd = ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K)
    U0, V0 = w.initial()
    lmax = oracle.lambda_max_dense(Md, Kd)
    tau0 = 0.4 * math.sqrt(oracle.theta_crit(0.5) / lmax)
    errs = []
    for n in (16, 32):
        T = 16 * tau0
        st = oracle.Stepper(ops, k, 0.5, tol=1e-15)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        Ue, Ve = oracle.exact_semidiscrete(Md, Kd, U0, V0, T)
        errs.append(np.linalg.norm(X[0] - Ue) / np.linalg.norm(Ue))
    order = math.log2(errs[0] / errs[1])
    assert order > 2 * k - 0.35, (errs, order)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cfl_limit_independent_of_k_on_mesh(k):
    w = W.small(d=2, nel=6, p=2, amp=0.1, k=k)
    ops = oracle.Operators(_patch(w))
    Md, Kd = ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K)
    lmax = oracle.lambda_max_dense(Md, Kd)
    rho = 0.5
    tc = math.sqrt(oracle.theta_crit(rho) / lmax)
    U0 = np.random.default_rng(0).standard_normal(ops.N)
    V0 = np.zeros(ops.N)

    def energy(X):
        return 0.5 * X[1] @ Md @ X[1] + 0.5 * X[0] @ Kd @ X[0]

    # The block upper-triangular amplification matrix is non-normal, so the energy can
    # rise transiently (by a few times for k = 3) before the dissipative decay; stability
    # means no sustained growth.
    out = []
    for frac in (0.98, 1.03):
        st = oracle.Stepper(ops, k, rho, tol=1e-14)
        X = st.init(U0, V0)
        e0 = energy(X)
        hist = []
        for _ in range(800):
            X = st.step(X, frac * tc)
            hist.append(energy(X) / e0)
        out.append(hist)
    stable, unstable = out
    mid = lambda h: max(h[200:400])
    late = lambda h: max(h[600:800])
    assert late(stable) <= mid(stable) * 1.001
    assert late(unstable) > 1e2 * mid(unstable)


# -- general model M U'' + C U' + K U = F: Rayleigh damping and harmonic forcing ----------
def _osc_exact(lam, c, terms, u0, v0):
    """Closed form of u'' + c u' + lam u = sum_m g_m sin(w_m t + p_m), u(0) = u0, u'(0) = v0
    (characteristic roots plus one particular solution per term); returns a function
    (t, m) -> m-th derivative of u at t."""
    parts = []
    for g, w, p in terms:  # particular: P sin(w t + p) + Q cos(w t + p)
        a, b = lam - w * w, c * w
        det = a * a + b * b
        parts.append((g * a / det, -g * b / det, w, p))

    def part(t, m):
        s = 0.0
        for P, Q, w, p in parts:
            ph = w * t + p + m * math.pi / 2
            s += w ** m * (P * math.sin(ph) + Q * math.cos(ph))
        return s

    r1 = (-c + cmath.sqrt(c * c - 4 * lam)) / 2
    r2 = (-c - cmath.sqrt(c * c - 4 * lam)) / 2
    h0, h1 = u0 - part(0.0, 0), v0 - part(0.0, 1)
    B = (h1 - r1 * h0) / (r2 - r1)
    A = h0 - B

    def u(t, m=0):
        return (A * r1 ** m * cmath.exp(r1 * t) + B * r2 ** m * cmath.exp(r2 * t)).real + part(t, m)

    return u


def _forcing_fn(G, terms):
    def F(s, t):
        return sum(g * G[i] * w ** s * math.sin(w * t + p + s * math.pi / 2) for i, (g, w, p) in enumerate(terms))
    return F


def _osc_error(k, rho, n, lam, aM, aK, terms, T=1.0):
    c = aM + aK * lam
    u = _osc_exact(lam, c, terms, 1.0, 0.0)
    forcing = _forcing_fn([np.ones(1)] * len(terms), terms) if terms else None
    st = oracle.Stepper(oracle.ScalarOps(lam), k, rho, tol=0.0,
                        damping=(aM, aK) if (aM or aK) else None, forcing=forcing)
    X = st.init(np.array([1.0]), np.array([0.0]))
    eu = ev = 0.0
    for s in range(1, n + 1):
        X = st.step(X, T / n)
        t = s * T / n
        eu = max(eu, abs(X[0, 0] - u(t)))
        ev = max(ev, abs(X[1, 0] - u(t, 1)))
    return eu, ev


OSC_CASES = {"damped": (0.8, 0.0, []), "stiffness_damped": (0.3, 0.1, []), "forced": (0.0, 0.0, [(1.0, 3.0, 0.0)]),
             "damped_forced": (0.5, 0.075, [(1.0, 3.0, 0.4), (0.5, 1.3, -0.7)])}


@pytest.mark.parametrize("k,ns,minorder", [(1, (40, 80), 1.9), (2, (80, 160), 3.7), (3, (32, 64), 5.4)])
@pytest.mark.parametrize("rho", [0.5, 1.0])
@pytest.mark.parametrize("case", list(OSC_CASES))
def test_damped_forced_modal_order_is_2k(k, ns, minorder, rho, case):
    """With C acting on the block's velocity-like predictor and F^{(s_j)} at t_{n+alpha_fj},
    the scheme keeps order 2k on the damped, forced oscillator (exact closed form)."""
    aM, aK, terms = OSC_CASES[case]
    e1 = _osc_error(k, rho, ns[0], 4.0, aM, aK, terms)
    e2 = _osc_error(k, rho, ns[1], 4.0, aM, aK, terms)
    for a, b in zip(e1, e2):
        assert math.log2(a / b) > minorder, (e1, e2)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_init_gives_the_exact_initial_derivatives(k):
    """X_a = M^{-1}(F^{(a)}(0) - K X_{a-2} - C X_{a-1}) are the derivatives u^{(a+2)}(0)."""
    lam, aM, aK = 4.0, 0.5, 0.075
    terms = [(1.0, 3.0, 0.4), (0.5, 1.3, -0.7)]
    u = _osc_exact(lam, aM + aK * lam, terms, 1.0, -0.3)
    st = oracle.Stepper(oracle.ScalarOps(lam), k, 0.5, tol=0.0, damping=(aM, aK),
                        forcing=_forcing_fn([np.ones(1)] * 2, terms))
    X = st.init(np.array([1.0]), np.array([-0.3]))
    for r in range(3 * k):
        assert abs(X[r, 0] - u(0.0, r)) < 1e-11 * max(1.0, abs(u(0.0, r))), r


def test_damped_forced_semidiscrete_order():
    """A small isogeometric system with Rayleigh damping and two harmonic loads against its
    exact modal solution (generalized eigenvectors of (K, M) decouple C = aM M + aK K)."""
    w = W.small(d=2, nel=4, p=2, amp=0.1, k=2)
    ops = oracle.Operators(_patch(w))
    Md, Kd = ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K)
    lam, Phi = scipy.linalg.eigh(Kd, Md)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((2, ops.N))
    terms = [(1.0, 7.0, 0.2), (1.0, 2.5, -1.0)]
    aM, aK = 0.6, 2e-4
    U0, V0 = rng.standard_normal(ops.N), np.zeros(ops.N)
    a0, b0 = Phi.T @ (Md @ U0), Phi.T @ (Md @ V0)
    g = Phi.T @ G.T  # modal loads [mode][term]
    T = 0.2
    exact = []
    for i in range(ops.N):
        u = _osc_exact(lam[i], aM + aK * lam[i], [(g[i, m], terms[m][1], terms[m][2]) for m in range(2)],
                       a0[i], b0[i])
        exact.append(u(T))
    Ue = Phi @ np.array(exact)
    tau0 = 0.4 * math.sqrt(oracle.theta_crit(0.5) / lam[-1])
    errs = []
    for n in (int(np.ceil(T / tau0)) * 2, int(np.ceil(T / tau0)) * 4):
        st = oracle.Stepper(ops, 2, 0.5, tol=1e-15, damping=(aM, aK), forcing=_forcing_fn(G, terms))
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        errs.append(np.linalg.norm(X[0] - Ue) / np.linalg.norm(Ue))
    assert math.log2(errs[0] / errs[1]) > 3.6, errs


@pytest.mark.parametrize("d,nel,p,amp", [(2, 8, 2, 0.1), (3, 4, 3, 0.12), (3, (5, 3, 4), 2, 0.0)])
def test_lanczos_lambda_max_equals_dense_eigenvalue(d, nel, p, amp):
    w = W.small(d=d, nel=nel, p=p, amp=amp)
    ops = oracle.Operators(_patch(w))
    Md, Kd = ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K)
    ref = oracle.lambda_max_dense(Md, Kd)
    lam = oracle.lambda_max_lanczos(ops, iters=min(ops.N, 80))
    assert abs(lam - ref) <= 1e-9 * ref, (lam, ref)
    # a few steps already bound it from below
    lam5 = oracle.lambda_max_lanczos(ops, iters=5)
    assert lam5 <= ref * (1 + 1e-12)


@pytest.mark.parametrize("Omega", [0.1, 0.7, 1.4, 1.99])
def test_modal_response_k1_rho1_is_central_difference(Omega):
    """k = 1 at rho_inf = 1 is the central-difference scheme: with U0 = 1, V0 = 0 the first
    step gives 1 - Omega^2/2 = cos(theta), and U_{s+1} = (2 - Omega^2) U_s - U_{s-1}
    makes U_s = cos(s theta), theta = arccos(1 - Omega^2/2) (stable for Omega < 2)."""
    lam = 3.7
    tau = Omega / math.sqrt(lam)
    U = oracle.modal_response(1, 1.0, lam, tau, 60)
    theta = math.acos(1 - Omega ** 2 / 2)
    assert np.allclose(U, np.cos(np.arange(61) * theta), rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_modal_response_dissipation_follows_rho(k):
    """At rho_inf = 1 nothing is damped; below it the response decays, the more the
    smaller rho_inf, with the same frequency for every k to leading order."""
    lam, tau, n = 1.0, 1.2, 400
    amp = {rho: np.abs(oracle.modal_response(k, rho, lam, tau, n)[-40:]).max() for rho in (1.0, 0.5, 0.0)}
    assert amp[1.0] > 0.99
    assert amp[1.0] > amp[0.5] > amp[0.0]


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8, 1.0])
def test_stability_diagram_is_independent_of_the_order(rho):
    """The amplification matrix is block triangular with every block's roots those of
    the second-order block (eq. HOampblock with the reading rho_bj = rho_sj = -rho_inf),
    so the spectral radius at every Omega is the same for k = 1, 2, 3: at most 1 below
    sqrt(Theta_crit) and equal to 1 there for rho_inf = 1."""
    lim = math.sqrt(oracle.theta_crit(rho))
    for Om in np.linspace(0.05, 0.999 * lim, 9):
        r = [oracle.spectral_radius(k, rho, Om) for k in (1, 2, 3)]
        assert max(r) - min(r) < 1e-7
        assert r[0] <= 1 + 1e-9
        if rho == 1.0:
            assert abs(r[0] - 1) < 1e-9


def test_thin_patch_is_the_1d_problem():
    """The dispersion study's stand-in for (0, 1) (paper_2102_11536_gb300.dispersion): the
    thin 2-D patch's generalised eigenvalues equal those of the 1-D B-spline
    discretisation on (0, 1) (the oracle's univariate mass and stiffness, identity map)
    up to the O(stretch^-2) shift, and the lowest ones are (j pi)^2 to the spline error."""
    import scipy.linalg
    from paper_2102_11536_gb300 import dispersion

    nel, p = 24, 4
    deg, knots, ctrl = dispersion.thin_patch_geometry(nel, p)
    P = oracle.Patch(list(deg), knots, ctrl)
    ops = oracle.Operators(P)
    lam2 = scipy.linalg.eigh(P.band_to_dense(ops.K), P.band_to_dense(ops.M), eigvals_only=True)
    q = oracle.Quad1D(p, knots[0], p + 1)
    lam1 = scipy.linalg.eigh(q.stiffness_interior(), q.mass_interior(), eigvals_only=True)
    assert len(lam1) == len(lam2)
    assert np.max(np.abs(lam2 / lam1 - 1)) < 1e-9
    for j in (1, 2, 3):
        assert abs(lam1[j - 1] / (j * math.pi) ** 2 - 1) < 1e-8


@pytest.mark.parametrize("p", [2, 3])
def test_preconditioner_is_asymptotically_exact(p):
    """Sec. 5.3: kappa(P^{-1} M) -> 1 as h -> 0 for the diagonal-scaled Kronecker
    preconditioner on a deformed patch; measured, kappa - 1 about halves with every
    refinement (O(h))."""
    excess = []
    for nel in (8, 16, 32):
        kn = [W.open_uniform_knots(nel, p)] * 2
        P = oracle.Patch([p, p], kn, W.control_net(kn, [p, p], 0.1))
        ops = oracle.Operators(P)
        Md = P.band_to_dense(ops.M)
        Pinv = np.column_stack([ops.apply_Pinv(e) for e in np.eye(ops.N)])
        ev = np.sort(np.real(np.linalg.eigvals(Pinv @ Md)))
        excess.append(ev[-1] / ev[0] - 1.0)
    assert excess[1] < 0.65 * excess[0] and excess[2] < 0.65 * excess[1], excess
    assert excess[2] < 0.03


def test_preconditioner_is_robust_in_p():
    """Sec. 5.3: kappa(P^{-1} M) grows slowly with the degree (measured on a deformed
    16 x 16 patch: 1.008 at p = 1 to 1.141 at p = 6)."""
    ks = []
    for p in range(1, 7):
        kn = [W.open_uniform_knots(16, p)] * 2
        P = oracle.Patch([p, p], kn, W.control_net(kn, [p, p], 0.1))
        ops = oracle.Operators(P)
        Md = P.band_to_dense(ops.M)
        Pinv = np.column_stack([ops.apply_Pinv(e) for e in np.eye(ops.N)])
        ev = np.sort(np.real(np.linalg.eigvals(Pinv @ Md)))
        ks.append(ev[-1] / ev[0])
    assert all(a < b for a, b in zip(ks, ks[1:])), ks
    assert ks[-1] < 1.2 and max(b - a for a, b in zip(ks, ks[1:])) < 0.06, ks


def test_preconditioner_tolerates_distorted_maps():
    """Sec. 5.3: the preconditioner stays good on distorted parametrisations. On a 16 x 16
    cubic patch kappa(P^{-1} M) is 1 on the identity map (M = P there) and grows to 1.25 at
    deformation amplitude 0.25, while diagonal scaling alone leaves kappa near 343."""
    p, nel = 3, 16
    ks = []
    for amp in (0.0, 0.1, 0.25):
        kn = [W.open_uniform_knots(nel, p)] * 2
        P = oracle.Patch([p, p], kn, W.control_net(kn, [p, p], amp))
        ops = oracle.Operators(P)
        Md = P.band_to_dense(ops.M)
        Pinv = np.column_stack([ops.apply_Pinv(e) for e in np.eye(ops.N)])
        ev = np.sort(np.real(np.linalg.eigvals(Pinv @ Md)))
        ks.append(ev[-1] / ev[0])
        D = np.diag(Md)
        evj = np.linalg.eigvalsh(Md / np.sqrt(np.outer(D, D)))
        assert evj[-1] / evj[0] > 300
    assert abs(ks[0] - 1.0) < 1e-10 and ks[0] < ks[1] < ks[2] < 1.3, ks
