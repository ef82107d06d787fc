"""Fields at the Gauss points through the library (iga_gauss_points, iga_evaluate,
iga_integrate) against the oracle's quadrature, and the spatial accuracy the paper
measures in Sec. 6 reproduced through them: the forced wave u = S(x)(cos wt + sin wt),
S = prod_a sin(pi x_a), on the deformed unit square / cube, its load vector integrated by
the library, its initial data projected by the library's PCG, the load applied as one
harmonic term (cos wt + sin wt = sqrt(2) sin(wt + pi/4)), the fourth-order steps on the
GPU, and the L2 error evaluated at the library's Gauss points -- equal to the oracle's
error on the same mesh, dt and quadrature, and converging at O(h^{p+1}).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W
from oracle import manufactured as mf

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _patch(d, nel, p, amp=0.1):
    kn = [W.open_uniform_knots(nel, p)] * d
    ctrl = W.control_net(kn, [p] * d, amp)
    return kn, ctrl


@pytest.mark.parametrize("d,p,nel", [(2, 3, 5), (3, 2, 4)])
def test_points_evaluate_integrate_match_the_oracle(d, p, nel):
    kn, ctrl = _patch(d, nel, p)
    g = iga.Patch([p] * d, kn, ctrl)
    q = mf.PatchQuadrature([p] * d, kn, ctrl, p + 1)  # the library's default rule
    try:
        qt, Q = g.npoints()
        assert qt == q.W.size and Q == [nel * (p + 1)] * d
        x = torch.empty(d * qt, dtype=torch.float64, device=DEV)
        w = torch.empty(qt, dtype=torch.float64, device=DEV)
        g.gauss_points(x, w)
        X = x.cpu().numpy().reshape(d, qt)
        assert np.abs(X - q.x.reshape(d, -1)).max() <= 1e-14
        assert np.abs(w.cpu().numpy() - q.W.reshape(-1)).max() <= 1e-14 * q.W.max()
        nvec = 2
        U = np.random.default_rng(3).standard_normal((nvec, g.N))
        gv = torch.empty(nvec * qt, dtype=torch.float64, device=DEV)
        g.evaluate(torch.from_numpy(U.ravel()).to(DEV), gv, nvec)
        Gv = gv.cpu().numpy().reshape(nvec, qt)
        for v in range(nvec):
            ref = q.evaluate(U[v]).reshape(-1)
            assert np.abs(Gv[v] - ref).max() <= 1e-13 * np.abs(ref).max()
        F = np.random.default_rng(4).standard_normal((nvec, qt))
        b = torch.empty(nvec * g.N, dtype=torch.float64, device=DEV)
        g.integrate(torch.from_numpy(F.ravel()).to(DEV), b, nvec)
        B = b.cpu().numpy().reshape(nvec, g.N)
        for v in range(nvec):
            ref = q.integrate(F[v])
            assert np.abs(B[v] - ref).max() <= 1e-13 * np.abs(ref).max()
    finally:
        g.close()


def _gpu_forced_wave(d, nel, p, dt, n, omega, T):
    kn, ctrl = _patch(d, nel, p)
    g = iga.Patch([p] * d, kn, ctrl, tol=1e-13)
    try:
        qt, _ = g.npoints()
        x = torch.empty(d * qt, dtype=torch.float64, device=DEV)
        w = torch.empty(qt, dtype=torch.float64, device=DEV)
        g.gauss_points(x, w)
        S = torch.prod(torch.sin(math.pi * x.view(d, qt)), dim=0)
        G = torch.empty(g.N, dtype=torch.float64, device=DEV)
        g.integrate(S, G)
        U0 = torch.zeros_like(G)
        g.solve_M(G, U0)
        V0 = omega * U0
        amp = d * math.pi ** 2 - omega ** 2
        g.set_forcing((amp * math.sqrt(2.0)) * G, [omega], [math.pi / 4])
        g.set_time(0.0)
        k = 2
        state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
        g.state_init(k, U0, V0, state)
        g.step(state, k, 0.5, dt, n)
        uh = torch.empty(qt, dtype=torch.float64, device=DEV)
        g.evaluate(state[:g.N], uh)
        exact = S * (math.cos(omega * T) + math.sin(omega * T))
        return math.sqrt(float(torch.sum(w * (uh - exact) ** 2)))
    finally:
        g.close()


def _oracle_forced_wave(d, nel, p, omega, T):
    kn, ctrl = _patch(d, nel, p)
    ops = oracle.Operators(oracle.Patch([p] * d, kn, ctrl))
    q = mf.PatchQuadrature([p] * d, kn, ctrl, p + 1)
    fw = mf.ForcedWave(q, omega)
    U0, V0 = fw.initial(lambda b: oracle.pcg(ops.apply_M, ops.apply_Pinv, b, tol=1e-14)[0])
    lam = oracle.lambda_max_lanczos(ops, iters=100)
    n = max(20, int(math.ceil(T / (0.5 * math.sqrt(oracle.theta_crit(0.5) / lam)))))
    st = oracle.Stepper(ops, 2, 0.5, tol=1e-13, forcing=fw.forcing)
    X = st.init(U0, V0)
    for _ in range(n):
        X = st.step(X, T / n)
    return q.l2_error(X[0], fw.exact(T)), T / n, n


@pytest.mark.parametrize("d,p,nels,rate", [(2, 3, (6, 12), 3.7), (3, 2, (4, 8), 2.7)])
def test_forced_wave_through_the_library_converges_at_order_p_plus_1(d, p, nels, rate):
    omega, T = 2 * math.pi, 0.1
    errs = []
    for nel in nels:
        err_o, dt, n = _oracle_forced_wave(d, nel, p, omega, T)
        err_g = _gpu_forced_wave(d, nel, p, dt, n, omega, T)
        print("forced wave d=%d p=%d nel=%d: L2 error GPU %.6e, oracle %.6e" % (d, p, nel, err_g, err_o))
        assert abs(err_g - err_o) <= 1e-6 * err_o
        errs.append(err_g)
    r = math.log2(errs[0] / errs[1])
    print("forced wave d=%d p=%d: rate %.2f" % (d, p, r))
    assert r > rate, errs
