"""Spatial accuracy of the oracle's discretisation with a forced, exactly known solution
(the O(h^{p+1}) L2 convergence of Sec. 6, here on the deformed unit square and cube,
whose boundary the deformation keeps), and pins of the quadrature helpers it uses."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import manufactured as mf


def _patch(d, nel, p, amp=0.1):
    kn = [W.open_uniform_knots(nel, p)] * d
    ctrl = W.control_net(kn, [p] * d, amp)
    return kn, ctrl


@pytest.mark.parametrize("d,p,amp", [(2, 2, 0.0), (2, 3, 0.1), (3, 2, 0.1)])
def test_quadrature_weights_integrate_the_domain(d, p, amp):
    """int S^2 over the unit square / cube is 2^-d whatever the (boundary-preserving) map."""
    kn, ctrl = _patch(d, 5, p, amp)
    q = mf.PatchQuadrature([p] * d, kn, ctrl, p + 4)
    assert abs(q.l2_error(np.zeros(int(np.prod(q.n))), mf.standing_profile(q.x)) ** 2 - 0.5 ** d) < 1e-9


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3), (3, 2)])
def test_integrate_of_evaluate_is_the_c_oracle_mass_product(d, p):
    """With the oracle's own rule (p + 1 points), int (sum_j U_j B_j) B_i is (M U)_i."""
    kn, ctrl = _patch(d, 4, p)
    q = mf.PatchQuadrature([p] * d, kn, ctrl, p + 1)
    ops = oracle.Operators(oracle.Patch([p] * d, kn, ctrl))
    U = np.random.default_rng(1).standard_normal(ops.N)
    ref = ops.apply_M(U)
    assert np.abs(q.integrate(q.evaluate(U).reshape(-1)) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_time_factor_derivatives():
    kn, ctrl = _patch(2, 3, 2)
    fw = mf.ForcedWave(mf.PatchQuadrature([2, 2], kn, ctrl, 3), 3.0)
    h = 1e-5
    for s in range(5):
        for t in (0.0, 0.37):
            fd = (fw.time_factor(s, t + h) - fw.time_factor(s, t - h)) / (2 * h)
            assert abs(fd - fw.time_factor(s + 1, t)) <= 1e-7 * 3.0 ** (s + 1)


@pytest.mark.parametrize("d,p,nels,rate", [(2, 2, (4, 8, 16), 2.8), (2, 3, (4, 8, 16), 3.7), (3, 2, (3, 6), 2.7)])
def test_forced_wave_converges_at_order_p_plus_1(d, p, nels, rate):
    """L2 error at T = 0.1 of the fourth-order scheme (k = 2, rho_inf = 0.5, tau <= T/20 and
    half the critical step) on the deformed patch: O(h^{p+1})."""
    errs = []
    for nel in nels:
        kn, ctrl = _patch(d, nel, p)
        ops = oracle.Operators(oracle.Patch([p] * d, kn, ctrl))
        q = mf.PatchQuadrature([p] * d, kn, ctrl, p + 3)
        fw = mf.ForcedWave(q, 2 * math.pi)
        U0, V0 = fw.initial(lambda b: oracle.pcg(ops.apply_M, ops.apply_Pinv, b, tol=1e-14)[0])
        lam = oracle.lambda_max_lanczos(ops, iters=100)
        T = 0.1
        n = max(20, int(math.ceil(T / (0.5 * math.sqrt(oracle.theta_crit(0.5) / lam)))))
        st = oracle.Stepper(ops, 2, 0.5, tol=1e-13, forcing=fw.forcing)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        errs.append(q.l2_error(X[0], fw.exact(T)))
    assert math.log2(errs[-2] / errs[-1]) > rate, errs


@pytest.mark.parametrize("p,rate", [(2, 2.8), (3, 3.7)])
def test_forced_wave_on_glued_patches_converges_at_order_p_plus_1(p, rate):
    """Optimal L2 convergence also on a multi-patch domain (Sec. 6): a 2 x 2 grid of
    deformed patches glued into [0, 2]^2 (N_adj = 4, the additive Schwarz preconditioner in
    the solves), S = sin(pi x / 2) sin(pi y / 2)."""
    from oracle import multipatch as mp
    from workloads import multipatch as WM
    errs = []
    for nsub in (4, 8):
        pts = WM.grid_of_patches((2, 2), nsub, p, amp=0.1)
        g = mp.GluedPatches(pts)
        fw = mf.GluedForcedWave(pts, g, (2.0, 2.0), 2 * math.pi, p + 3)
        U0, V0 = fw.initial(lambda b: oracle.pcg(g.apply_M, g.apply_Pinv, b, tol=1e-14)[0])
        lam = oracle.lambda_max_lanczos(g, iters=min(g.N, 200))
        T = 0.1
        n = max(20, int(math.ceil(T / (0.5 * math.sqrt(oracle.theta_crit(0.5) / lam)))))
        st = oracle.Stepper(g, 2, 0.5, tol=1e-13, forcing=fw.forcing)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        errs.append(fw.l2_error(X[0], T))
    assert math.log2(errs[0] / errs[1]) > rate, errs


def test_forced_wave_on_glued_3d_patches_converges_at_order_p_plus_1():
    """The same on a 3-D domain of 2 x 1 x 2 glued deformed patches ([0, 2] x [0, 1] x [0, 2],
    N_adj = 4), p = 2."""
    from oracle import multipatch as mp
    from workloads import multipatch as WM
    errs = []
    for nsub in (3, 6):
        pts = WM.grid_of_patches((2, 1, 2), nsub, 2, amp=0.1)
        g = mp.GluedPatches(pts)
        fw = mf.GluedForcedWave(pts, g, (2.0, 1.0, 2.0), 2 * math.pi, 4)
        U0, V0 = fw.initial(lambda b: oracle.pcg(g.apply_M, g.apply_Pinv, b, tol=1e-14)[0])
        lam = oracle.lambda_max_lanczos(g, iters=min(g.N, 200))
        T = 0.1
        n = max(20, int(math.ceil(T / (0.5 * math.sqrt(oracle.theta_crit(0.5) / lam)))))
        st = oracle.Stepper(g, 2, 0.5, tol=1e-13, forcing=fw.forcing)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        errs.append(fw.l2_error(X[0], T))
    assert math.log2(errs[0] / errs[1]) > 2.7, errs
