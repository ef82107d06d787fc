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
import workloads as W
from oracle import multipatch as mp
from workloads import multipatch as WM


@pytest.mark.parametrize("shape,nel,p", [((1, 1), 5, 2), ((1, 1), 5, 3), ((1, 1, 1), 3, 2)])
def test_patch_assembly_equals_the_c_oracle_on_interior_functions(shape, nel, p):
    deg, knots, ctrl = WM.grid_of_patches(shape, nel, p, amp=0.12)[0]
    M, K, _, m = mp.patch_full_matrices(deg, knots, ctrl)
    P = oracle.Patch(list(deg), knots, ctrl)
    ops = oracle.Operators(P)
    rng = [range(1, n - 1) for n in m] + [range(1)] * (3 - len(m))
    m3 = list(m) + [1] * (3 - len(m))
    inner = [i0 + m3[0] * (i1 + m3[1] * i2) for i2 in rng[2] for i1 in rng[1] for i0 in rng[0]]
    Md, Kd = P.band_to_dense(ops.M), P.band_to_dense(ops.K)
    assert np.abs(M[np.ix_(inner, inner)] - Md).max() <= 1e-13 * np.abs(Md).max()
    assert np.abs(K[np.ix_(inner, inner)] - Kd).max() <= 1e-13 * np.abs(Kd).max()


@pytest.mark.parametrize("shape,nel,p", [((1, 1), 6, 3), ((1, 1, 1), 4, 2)])
def test_one_patch_schwarz_is_the_single_patch_preconditioner(shape, nel, p):
    pat = WM.grid_of_patches(shape, nel, p, amp=0.1)[0]
    g = mp.GluedPatches([pat])
    pre = oracle.Preconditioner(oracle.Patch(list(pat[0]), pat[1], pat[2]))
    r = np.random.default_rng(0).standard_normal(g.N)
    z1, z2 = g.apply_Pinv(r), pre.apply_Pinv(r)
    assert np.abs(z1 - z2).max() <= 1e-12 * np.abs(z2).max()


def _pfold_patch(shape, nel, p):
    """One patch on [0, shape_0] x ... whose knot vector in direction a joins shape_a blocks
    of nel uniform elements with the knots between blocks repeated p times (C^0 there); the
    affine geometry x_a = shape_a xi_a (control points at the Greville abscissae)."""
    kns = []
    for s in shape:
        inner = []
        for b in range(s):
            inner += [(b + i / nel) / s for i in range(1, nel)]
            if b < s - 1:
                inner += [(b + 1) / s] * p
        kns.append(np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1)))
    g = [W.greville(kn, p) * s for kn, s in zip(kns, shape)]
    d = len(shape)
    import itertools
    ctrl = np.array([[g[a][ix[d - 1 - a]] for a in range(d)]
                     for ix in itertools.product(*[range(len(gg)) for gg in reversed(g)])])
    return oracle.Patch([p] * d, kns, ctrl)


def _same_spectra(g, P):
    ops = oracle.Operators(P)
    Md, Kd = P.band_to_dense(ops.M), P.band_to_dense(ops.K)
    assert P.N == g.N
    ev_m = np.sort(np.linalg.eigvalsh(Md))
    assert np.allclose(np.sort(np.linalg.eigvalsh(g.M)), ev_m, rtol=1e-10, atol=1e-14 * ev_m[-1])
    ev = scipy.linalg.eigh(Kd, Md, eigvals_only=True)
    assert np.allclose(scipy.linalg.eigh(g.K, g.M, eigvals_only=True), ev, rtol=1e-9, atol=0)


@pytest.mark.parametrize("shape,nel,p", [((2, 1), 4, 1), ((2, 1), 4, 2), ((2, 1), 4, 3), ((2, 2), 3, 2),
                                         ((3, 2), 2, 3), ((2, 1, 1), 2, 2), ((2, 2, 2), 2, 2)])
def test_glued_patches_equal_one_patch_with_p_fold_knots(shape, nel, p):
    """A grid of unit patches glued face to face spans the C^0 space of one patch on the
    union whose knot vectors repeat the knots between patches p times; with the affine
    geometries the global M and K are that patch's up to the order of the functions, so the
    spectra of M and of the pencil (K, M) coincide. The grids of 2 x 2 and 2 x 2 x 2 patches
    share functions among 4 and 8 patches."""
    g = mp.GluedPatches(WM.grid_of_patches(shape, nel, p, amp=0.0))
    _same_spectra(g, _pfold_patch(shape, nel, p))
    assert g.n_adj == 2 ** sum(1 for s in shape if s > 1)


@pytest.mark.parametrize("p,amp", [(1, 0.0), (2, 0.1), (3, 0.1)])
def test_l_shape_is_the_grid_without_the_functions_of_the_removed_patch(p, amp):
    """The space of the L (the 2 x 2 grid without patch 3) with homogeneous Dirichlet data is
    the subspace of the grid's space of the functions that vanish on patch 3: the grid's
    global functions with no copy in patch 3 (def:mp_basis; local B-splines are linearly
    independent). Their integrals over the grid and over the L agree, so the L's M and K
    are principal blocks of the grid's. The function at the re-entrant corner touches the
    removed patch and must not be in the L's space."""
    grid = WM.grid_of_patches((2, 2), 3, p, amp=amp)
    g4 = mp.GluedPatches(grid)
    gl = mp.GluedPatches(grid[:3])
    S = np.setdiff1d(np.arange(g4.N), g4.local[3]["ids"])
    assert gl.N == S.size
    ev = np.sort(np.linalg.eigvalsh(g4.M[np.ix_(S, S)]))
    assert np.allclose(np.sort(np.linalg.eigvalsh(gl.M)), ev, rtol=1e-11, atol=1e-15 * ev[-1])
    evk = scipy.linalg.eigh(g4.K[np.ix_(S, S)], g4.M[np.ix_(S, S)], eigvals_only=True)
    assert np.allclose(scipy.linalg.eigh(gl.K, gl.M, eigvals_only=True), evk, rtol=1e-9, atol=0)


@pytest.mark.parametrize("perm,flip", [((0, 1), (0,)), ((0, 1), (0, 1)), ((1, 0), ()), ((1, 0), (1,))])
def test_numbering_is_independent_of_the_patches_orientation(perm, flip):
    """Renaming or reversing the parameter directions of some patches leaves the glued space,
    hence the spectra of M and of (K, M), unchanged (reversal makes det DF < 0)."""
    base = WM.grid_of_patches((2, 2), 3, 2, amp=0.1)
    g0 = mp.GluedPatches(base)
    g1 = mp.GluedPatches([WM.reorient(pt, perm, flip) if r in (1, 2) else pt for r, pt in enumerate(base)])
    assert g1.N == g0.N and g1.n_adj == g0.n_adj == 4
    assert np.allclose(np.sort(np.linalg.eigvalsh(g1.M)), np.sort(np.linalg.eigvalsh(g0.M)), rtol=1e-11, atol=0)
    assert np.allclose(scipy.linalg.eigh(g1.K, g1.M, eigvals_only=True),
                       scipy.linalg.eigh(g0.K, g0.M, eigvals_only=True), rtol=1e-9, atol=0)


def test_reoriented_preconditioner_is_the_same_operator():
    """P_ad^{-1} M has the same spectrum whatever the orientation of each patch: the local
    Kronecker factors follow the renamed directions."""
    base = WM.l_shape(4, 3, amp=0.1)
    g0 = mp.GluedPatches(base)
    g1 = mp.GluedPatches([WM.reorient(base[0], (1, 0), (0,)), base[1], WM.reorient(base[2], (0, 1), (0, 1))])
    e0 = np.sort(np.real(np.linalg.eigvals(g0.dense_Pinv() @ g0.M)))
    e1 = np.sort(np.real(np.linalg.eigvals(g1.dense_Pinv() @ g1.M)))
    assert np.allclose(e1, e0, rtol=1e-9, atol=0)


@pytest.mark.parametrize("layout,sizes", [
    (lambda n: WM.row_of_patches(2, n, 3, amp=0.1), (3, 6, 12)),
    (lambda n: WM.row_of_patches(3, n, 3, amp=0.1), (3, 6, 12)),
    (lambda n: WM.l_shape(n, 3, amp=0.1), (3, 6, 12)),
    (lambda n: WM.grid_of_patches((2, 2), n, 3, amp=0.1), (3, 6, 12)),
    (lambda n: WM.grid_of_patches((2, 2, 2), n, 2, amp=0.1), (2, 4)),
])
def test_schwarz_conditioning_is_bounded_independently_of_h(layout, sizes):
    """kappa(P_ad^{-1} M) <= C N_adj^2 with C independent of h and of the number of
    patches (Sec. 5.4): rows, an L, 2 x 2 and 2 x 2 x 2 grids of deformed patches (N_adj =
    2, 2, 4, 8) at several mesh sizes. The paper gives no value of C; measured, kappa / N_adj^2
    lies between 1.3 and 2.4 here (the L's re-entrant corner gives the largest), and kappa
    varies by < 10 % with h."""
    kap = []
    for nel in sizes:
        g = mp.GluedPatches(layout(nel))
        ev = np.sort(np.real(np.linalg.eigvals(g.dense_Pinv() @ g.M)))
        assert ev[0] > 0
        kap.append(ev[-1] / ev[0])
        assert kap[-1] < 2.5 * g.n_adj ** 2, (nel, g.n_adj, kap)
    assert max(kap) / min(kap) < 1.1, kap


@pytest.mark.parametrize("layout", [lambda: WM.row_of_patches(3, 6, 3, amp=0.1), lambda: WM.l_shape(6, 3, amp=0.1),
                                    lambda: WM.grid_of_patches((2, 2), 6, 3, amp=0.1)])
def test_pcg_with_schwarz_reaches_the_dense_solution(layout):
    g = mp.GluedPatches(layout())
    b = np.random.default_rng(3).standard_normal(g.N)
    x, it, rel = oracle.pcg(g.apply_M, g.apply_Pinv, b, tol=1e-12)
    xd = np.linalg.solve(g.M, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert it <= 40


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("layout", [lambda: WM.row_of_patches(2, 4, 2, amp=0.1), lambda: WM.l_shape(3, 2, amp=0.1)])
def test_scheme_on_glued_patches_has_order_2k(k, layout):
    g = mp.GluedPatches(layout())
    rng = np.random.default_rng(5)
    lam = scipy.linalg.eigh(g.K, g.M, eigvals_only=True)
    U0 = rng.standard_normal(g.N)
    V0 = np.zeros(g.N)
    tau0 = 0.4 * math.sqrt(oracle.theta_crit(0.5) / lam[-1])
    T = 16 * tau0
    errs = []
    for n in (32, 64):
        st = oracle.Stepper(g, k, 0.5, tol=1e-15)
        X = st.init(U0, V0)
        for _ in range(n):
            X = st.step(X, T / n)
        Ue, _ = oracle.exact_semidiscrete(g.M, g.K, U0, V0, T)
        errs.append(np.linalg.norm(X[0] - Ue) / np.linalg.norm(Ue))
    assert math.log2(errs[0] / errs[1]) > 2 * k - 0.35, errs


@pytest.mark.parametrize("layout", [lambda: WM.l_shape(4, 3, amp=0.1), lambda: WM.grid_of_patches((2, 1, 2), 3, 2, amp=0.1)])
def test_lanczos_critical_step_on_glued_patches(layout):
    """The oracle's Lanczos estimate of lambda_max(M^{-1} K), the critical step's input,
    on glued patches (with P_ad in its solves) equals the dense generalised eigenvalue."""
    g = mp.GluedPatches(layout())
    ref = scipy.linalg.eigh(g.K, g.M, eigvals_only=True)[-1]
    est = oracle.lambda_max_lanczos(g, iters=g.N)
    assert abs(est - ref) <= 1e-9 * ref


@pytest.mark.parametrize("patch", [lambda: WM.grid_of_patches((1, 1), 4, 2, amp=0.12)[0],
                                   lambda: WM.reorient(WM.grid_of_patches((1, 1), 3, 3, amp=0.1)[0], (1, 0), (0,)),
                                   lambda: WM.grid_of_patches((1, 1, 1), 3, 2, amp=0.12)[0]])
def test_row_assembly_equals_the_dense_patch_matrices(patch):
    """patch_rows integrates over the row function's support only; every row of M and K
    (boundary functions included) equals the dense assembly's."""
    deg, kn, ctrl = patch()
    M, K, _, m = mp.patch_full_matrices(deg, kn, ctrl)
    rows = mp.patch_rows(deg, kn, ctrl, range(M.shape[0]))
    Mr, Kr = np.zeros_like(M), np.zeros_like(K)
    for i, row in enumerate(rows):
        for j, (mij, kij) in row.items():
            Mr[i, j], Kr[i, j] = mij, kij
    assert np.abs(Mr - M).max() <= 1e-13 * np.abs(M).max()
    assert np.abs(Kr - K).max() <= 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("layout", [lambda: WM.l_shape(3, 3, amp=0.1), lambda: WM.grid_of_patches((2, 2), 3, 2, amp=0.1),
                                    lambda: WM.grid_of_patches((2, 1, 2), 2, 2, amp=0.1)])
def test_sampled_glued_products_equal_the_global_matrices(layout):
    """glued_rows (per-row assembly through the copies of each global function, for
    full-size sampled checks) equals the dense global M x and K x on every row."""
    patches = layout()
    g = mp.GluedPatches(patches)
    x = np.random.default_rng(4).standard_normal(g.N)
    Mx, Kx = mp.glued_rows(patches, g.local, list(range(g.N)), x)
    assert np.abs(Mx - g.M @ x).max() <= 1e-13 * np.abs(g.M @ x).max()
    assert np.abs(Kx - g.K @ x).max() <= 1e-12 * np.abs(g.K @ x).max()


def test_oracle_refuses_a_non_matching_interface():
    """Assumption ass:conformity: a refined neighbour shares the face region but not its
    functions; the oracle refuses it like the library does."""
    left = WM.row_of_patches(2, 3, 2, amp=0.0)[0]
    right = WM.row_of_patches(2, 4, 2, amp=0.0)[1]
    with pytest.raises(ValueError, match="not conforming"):
        mp.glue([left, right])


def test_schwarz_iterations_grow_with_p_and_fall_with_refinement():
    """Table Fan_its (Sec. 6): the mean PCG iterations with the additive Schwarz
    preconditioner grow with the degree and fall as the patches are refined; here on a
    2 x 2 grid of deformed patches at the table's tau = 5e-5, T = 64 tau, tol 1e-12."""
    from oracle.multipatch_table import mean_iterations
    its = {(n, p): mean_iterations(WM.grid_of_patches((2, 2), n, p, amp=0.1))[0] for n in (4, 8) for p in (1, 2, 3)}
    for n in (4, 8):
        assert its[(n, 1)] < its[(n, 2)] < its[(n, 3)], its
    for p in (1, 2, 3):
        assert its[(8, p)] < its[(4, p)], its
    assert max(its.values()) < 30
