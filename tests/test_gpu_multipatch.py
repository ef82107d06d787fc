"""Parity of the multi-patch system (iga_mp_create: conforming patches, Sec. 5.1, with the
additive Schwarz preconditioner, Sec. 5.4) with the multi-patch oracle on the same seeded
layout: three deformed quadratic patches in a row (N_adj = 2), every operator form.

Tolerances: FP64 forms as for one patch (operators 1e-12 of max|y| for M and P_ad^{-1},
1e-11 for K; solves at tol 1e-13 within 1e-10 relative, iteration counts within 1 of the
oracle's PCG); the double-FP32 band products within 64 * 2^-48 (|A| |x|) + 1e-15 max|y|
per entry."""

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
                    bound = 64 * 2.0 ** -48 * (np.abs(A) @ np.abs(X[v])) + 1e-15 * np.abs(ref).max()
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
