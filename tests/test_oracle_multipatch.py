"""Pins of the multi-patch oracle (oracle/multipatch.py: conforming patches, Sec. 5.1, and
the additive Schwarz preconditioner of Sec. 5.4, def:asp) against facts independent of
it: the oracle's C assembly, the single-patch preconditioner, the equivalence of glued
patches with one patch carrying a p-fold knot, the paper's conditioning bound, and the
scheme's temporal order on the glued system."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import multipatch as mp


@pytest.mark.parametrize("p", [2, 3])
def test_patch_assembly_equals_the_c_oracle_on_interior_functions(p):
    deg, knots, ctrl = mp.row_of_patches(1, 5, p, amp=0.12)[0]
    M, K, _, (m0, m1) = mp.patch_full_matrices(deg, knots, ctrl)
    P = oracle.Patch(list(deg), knots, ctrl)
    ops = oracle.Operators(P)
    inner = [j * m0 + i for j in range(1, m1 - 1) for i in range(1, m0 - 1)]
    Md, Kd = P.band_to_dense(ops.M), P.band_to_dense(ops.K)
    assert np.abs(M[np.ix_(inner, inner)] - Md).max() <= 1e-13 * np.abs(Md).max()
    assert np.abs(K[np.ix_(inner, inner)] - Kd).max() <= 1e-13 * np.abs(Kd).max()


def test_one_patch_schwarz_is_the_single_patch_preconditioner():
    pat = mp.row_of_patches(1, 6, 3, amp=0.1)[0]
    g = mp.GluedPatches([pat])
    pre = oracle.Preconditioner(oracle.Patch(list(pat[0]), pat[1], pat[2]))
    r = np.random.default_rng(0).standard_normal(g.N)
    z1, z2 = g.apply_Pinv(r), pre.apply_Pinv(r)
    assert np.abs(z1 - z2).max() <= 1e-12 * np.abs(z2).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_glued_patches_equal_one_patch_with_a_p_fold_knot(p):
    """Two unit patches glued along x = 1 span the C^0 space of one patch on [0, 2] x [0, 1]
    whose knot vector repeats the middle knot p times; with the affine geometries the
    global M and K are that patch's up to the order of the functions, so the spectra of
    M and of the pencil (K, M) coincide."""
    nel = 4
    g = mp.GluedPatches(mp.row_of_patches(2, nel, p, amp=0.0))
    kx = np.array([0.0] * (p + 1) + [i / (2 * nel) for i in range(1, nel)] + [0.5] * p
                  + [0.5 + i / (2 * nel) for i in range(1, nel)] + [1.0] * (p + 1))
    ky = np.array([0.0] * (p + 1) + [i / nel for i in range(1, nel)] + [1.0] * (p + 1))

    def greville(kn):
        m = len(kn) - p - 1
        return np.array([kn[i + 1:i + p + 1].mean() for i in range(m)])

    ctrl = np.array([(2 * x, y) for y in greville(ky) for x in greville(kx)])
    P = oracle.Patch([p, p], [kx, ky], ctrl)
    ops = oracle.Operators(P)
    Md, Kd = P.band_to_dense(ops.M), P.band_to_dense(ops.K)
    assert P.N == g.N
    ev_m = np.sort(np.linalg.eigvalsh(Md))
    assert np.allclose(np.sort(np.linalg.eigvalsh(g.M)), ev_m, rtol=1e-10, atol=1e-14 * ev_m[-1])
    ev = scipy.linalg.eigh(Kd, Md, eigvals_only=True)
    assert np.allclose(scipy.linalg.eigh(g.K, g.M, eigvals_only=True), ev, rtol=1e-9, atol=0)


def test_schwarz_conditioning_is_bounded_independently_of_h():
    """kappa(P_ad^{-1} M) <= C N_adj^2 with C independent of h and of the number of
    patches (Sec. 5.4): a row of 2 or 3 deformed patches at 3, 6, 12 elements per side."""
    kap = {}
    for npch in (2, 3):
        for nel in (3, 6, 12):
            g = mp.GluedPatches(mp.row_of_patches(npch, nel, 3, amp=0.1))
            assert g.n_adj == 2
            ev = np.sort(np.real(np.linalg.eigvals(g.dense_Pinv() @ g.M)))
            assert ev[0] > 0
            kap[(npch, nel)] = ev[-1] / ev[0]
    assert max(kap.values()) < 2.0 * 2 ** 2
    assert max(kap.values()) / min(kap.values()) < 1.2


def test_pcg_with_schwarz_reaches_the_dense_solution():
    g = mp.GluedPatches(mp.row_of_patches(3, 6, 3, amp=0.1))
    b = np.random.default_rng(3).standard_normal(g.N)
    x, it, rel = oracle.pcg(g.apply_M, g.apply_Pinv, b, tol=1e-12)
    xd = np.linalg.solve(g.M, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert it <= 25


@pytest.mark.parametrize("k", [1, 2, 3])
def test_scheme_on_glued_patches_has_order_2k(k):
    g = mp.GluedPatches(mp.row_of_patches(2, 4, 2, amp=0.1))
    rng = np.random.default_rng(5)
    lam = scipy.linalg.eigh(g.K, g.M, eigvals_only=True)
    U0 = rng.standard_normal(g.N)
    V0 = np.zeros(g.N)
    tau0 = 0.4 * math.sqrt(oracle.theta_crit(0.5) / lam[-1])
    T = 16 * tau0
    errs = []
    for n in (16, 32):
        st = oracle.Stepper(g, k, 0.5, tol=1e-15)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        Ue, _ = oracle.exact_semidiscrete(g.M, g.K, U0, V0, T)
        errs.append(np.linalg.norm(X[0] - Ue) / np.linalg.norm(Ue))
    assert math.log2(errs[0] / errs[1]) > 2 * k - 0.35, errs
