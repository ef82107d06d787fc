"""Parity of the multi-patch system (iga_mp_create: conforming patches, Sec. 5.1, with the
additive Schwarz preconditioner, Sec. 5.4) with the multi-patch oracle on the same seeded
layouts: three deformed quadratic patches in a row (N_adj = 2), an L of three patches (a
re-entrant corner), a 2 x 2 grid of cubic patches (N_adj = 4) and a 2 x 2 x 2 grid of
quadratic patches (N_adj = 8); every operator form, PCG, the critical step, the time
steps (initial data and k = 2 steps) from the host loop, the captured step, the
patches on concurrent streams, and the per-patch access, tuning and profiling calls.

Tolerances: FP64 forms as for one patch (operators 1e-12 of max|y| for M and P_ad^{-1},
1e-11 for K; solves at tol 1e-13 within 1e-10 relative, iteration counts within 1 of the
oracle's PCG; steps at tol 1e-13 within 1e-10 in U and V); the double-FP32 band products
within 64 * 2^-48 (|A| |x|) + 1e-15 max|y| per entry, and its steps (FP32 Kronecker local
preconditioners, tol 1e-10) within 1e-8; lambda_max within 1e-8 of the dense generalised
eigenvalue; captured and concurrent steps bitwise equal to the host loop."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
from oracle import multipatch as mp
from workloads import multipatch as WM

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

LAYOUTS = {
    "row3_p2": lambda: WM.row_of_patches(3, 4, 2, amp=0.1),
    "l3_p2": lambda: WM.l_shape(4, 2, amp=0.1),
    "grid2x2_p3": lambda: WM.grid_of_patches((2, 2), 4, 3, amp=0.1),
    "grid2x2x2_p2": lambda: WM.grid_of_patches((2, 2, 2), 2, 2, amp=0.1),
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module", params=sorted(LAYOUTS))
def layout(request):
    patches = LAYOUTS[request.param]()
    return patches, mp.GluedPatches(patches)


@pytest.mark.parametrize("form", ["matrix_free", "assembled", "assembled_df"])
def test_operators_match_the_oracle(layout, form):
    patches, g = layout
    sys_ = iga.MultiPatch(patches, op_form=form, tol=1e-13)
    try:
        assert sys_.N == g.N and sys_.n_adj == g.n_adj and sys_.npatch == len(patches)
        nvec = 3
        X = np.random.default_rng(11).standard_normal((nvec, g.N))
        x = _t(X)
        y = torch.empty_like(x)
        for name, A in (("M", g.M), ("K", g.K)):
            getattr(sys_, "apply_" + name)(x, y, nvec)
            Y = _np(y).reshape(nvec, g.N)
            for v in range(nvec):
                ref = A @ X[v]
                if form == "assembled_df":
                    # + 2^-22 |a x| for couplings a patch may hold in tiny slots (one FP32
                    # multiply-add: every coefficient below 2^-24 of that patch's largest)
                    At = np.abs(A)
                    small = At * (At < 2.0 ** -18 * At.max())
                    bound = (64 * 2.0 ** -48 * (At @ np.abs(X[v])) + 2.0 ** -22 * (small @ np.abs(X[v]))
                             + 1e-15 * np.abs(ref).max())
                    assert np.all(np.abs(Y[v] - ref) <= bound), name
                else:
                    assert _maxrel(Y[v], ref) < (1e-12 if name == "M" else 1e-11), name
        sys_.apply_Pinv(x, y, nvec)
        Y = _np(y).reshape(nvec, g.N)
        for v in range(nvec):
            assert _maxrel(Y[v], g.apply_Pinv(X[v])) < 1e-12
    finally:
        sys_.close()


def test_pcg_matches_the_oracle(layout):
    patches, g = layout
    sys_ = iga.MultiPatch(patches, tol=1e-13)
    try:
        B = np.random.default_rng(2).standard_normal((2, g.N))
        b = _t(B)
        x = torch.zeros_like(b)
        its, rel = sys_.solve_M(b, x, 2)
        Xg = _np(x).reshape(2, g.N)
        for v in range(2):
            xd = np.linalg.solve(g.M, B[v])
            assert np.linalg.norm(Xg[v] - xd) <= 1e-10 * np.linalg.norm(xd)
            _, it_o, _ = oracle.pcg(g.apply_M, g.apply_Pinv, B[v], tol=1e-13)
            assert abs(its[v] - it_o) <= 1
            assert rel[v] <= 1e-13
    finally:
        sys_.close()


def _dt(g, rho):
    return 0.5 * np.sqrt(oracle.theta_crit(rho) / oracle.lambda_max_dense(g.M, g.K))


def test_cfl_matches_the_oracle(layout):
    patches, g = layout
    sys_ = iga.MultiPatch(patches, tol=1e-13)
    try:
        lam, tau = sys_.cfl(0.5, iters=200)
        ref = oracle.lambda_max_dense(g.M, g.K)
        print("multi-patch lambda_max: GPU %.12g, dense %.12g" % (lam, ref))
        assert abs(lam - ref) <= 1e-8 * ref
        assert abs(tau - np.sqrt(oracle.theta_crit(0.5) / lam)) <= 1e-12 * tau
    finally:
        sys_.close()


@pytest.mark.parametrize("form", [("matrix_free", "fp64", 1e-13, 1e-10), ("assembled_df", "banded32", 1e-10, 1e-8)])
def test_steps_match_the_oracle(layout, form):
    op_form, precond, tol, bound = form
    patches, g = layout
    k, rho, nsteps = 2, 0.5, 8
    dt = _dt(g, rho)
    rng = np.random.default_rng(6)
    U0 = rng.standard_normal(g.N)
    V0 = 0.3 * rng.standard_normal(g.N)
    st = oracle.Stepper(g, k, rho, tol=1e-13)
    X = st.init(U0, V0)
    for _ in range(nsteps):
        X = st.step(X, dt)
    sys_ = iga.MultiPatch(patches, tol=tol, op_form=op_form, precond=precond)
    try:
        state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
        sys_.state_init(k, _t(U0), _t(V0), state)
        sg = sys_.step(state, k, rho, dt, nsteps)
        assert sg.steps == nsteps and sg.max_relres <= tol
        Xg = _np(state).reshape(3 * k, g.N)
        for row, var in ((0, "U"), (1, "V")):
            err = np.linalg.norm(Xg[row] - X[row]) / np.linalg.norm(X[row])
            print("multi-patch steps (%s, %s) vs oracle, %s: %.3e" % (op_form, precond, var, err))
            assert err <= bound, (var, err)
    finally:
        sys_.close()


def test_captured_and_concurrent_steps_equal_the_host_loop(layout):
    patches, g = layout
    k, rho, nsteps = 2, 0.5, 5
    dt = _dt(g, rho)
    U0 = np.random.default_rng(8).standard_normal(g.N)
    V0 = np.zeros(g.N)
    finals = {}
    for name, graphs, conc in (("host", False, False), ("graph", True, False), ("concurrent", False, True),
                               ("graph_concurrent", True, True)):
        sys_ = iga.MultiPatch(patches, tol=1e-12, op_form="assembled_df", precond="banded32")
        try:
            sys_.set_graphs(graphs)
            if conc:
                sys_.set_concurrent(True)
            state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
            sys_.state_init(k, _t(U0), _t(V0), state)
            st = sys_.step(state, k, rho, dt, nsteps)
            assert st.steps == nsteps
            finals[name] = _np(state)
        finally:
            sys_.close()
    for name in ("graph", "concurrent", "graph_concurrent"):
        assert np.array_equal(finals[name], finals["host"]), name


def test_per_patch_access_and_tuning(layout):
    """iga_mp_patch / iga_mp_patch_io against the layout's global ids: the gather copies each
    box entry's global value (zero where the entry is no degree of freedom), the adds sum
    the patches' copies in patch order; a lent patch handle has its box's size; the
    system's autotune and profile calls run through every patch."""
    patches, _ = layout
    lay = iga.multipatch_layout(patches)
    sys_ = iga.MultiPatch(patches, op_form="assembled", precond="fp64")
    try:
        N = sys_.N
        rng = np.random.default_rng(5)
        x = rng.standard_normal(N)
        y = torch.zeros(N, dtype=torch.float64, device=DEV)
        want_y = np.zeros(N)
        for r in range(len(patches)):
            gid = np.asarray(lay["gid"][r]).reshape(-1)
            assert sys_.patch(r).N == gid.size
            box = torch.full((gid.size,), np.nan, dtype=torch.float64, device=DEV)
            sys_.patch_gather(r, _t(x), box)
            want = np.where(gid >= 0, x[np.maximum(gid, 0)], 0.0)
            assert np.array_equal(_np(box), want), r
            b = rng.standard_normal(gid.size)
            sys_.patch_scatter_add(r, _t(b), y)
            for e in np.nonzero(gid >= 0)[0]:  # the patch's copies, in the order of the patches
                want_y[gid[e]] += b[e]
        torch.cuda.synchronize()
        assert np.array_equal(_np(y), want_y)
        cfg = sys_.autotune(nvec=2, reps=1)
        assert len(cfg) == 2 and cfg[0] > 0
        out = torch.empty_like(y)
        sys_.profile("band_mass")
        sys_.apply_M(_t(x), out)
        ms, launches, _, _ = sys_.profile_read()
        sys_.profile("off")
        assert launches >= len(patches) and ms > 0.0
    finally:
        sys_.close()
