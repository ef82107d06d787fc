"""The dispersion study (Sec. 6.2) on the GPU: the scheme's response on discrete modes
of the thin patch that stands in for (0, 1), against the oracle's modal analysis of the
same scheme (oracle.modal_response), from the lowest mode to one at the stability
limit, for k = 1..3 and rho_inf in {0, 0.5, 1}; and the study's order effect."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2102_11536_gb300 import dispersion

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def thin():
    tp = dispersion.ThinPatch(nel=48, p=4)
    yield tp
    tp.close()


def test_thin_patch_modes_are_the_1d_modes(thin):
    """The lowest modes are sin(j pi x) up to the spline error: their eigenvalues are
    (j pi)^2 to high relative accuracy (p = 4 on 48 elements)."""
    for j in (1, 2, 3, 4):
        assert abs(thin.lam[j - 1] / (j * math.pi) ** 2 - 1) < 1e-7


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_gpu_modal_response_matches_analysis(thin, k, rho):
    tau = 0.95 * thin.critical_step(rho)
    n = 60
    for j in (0, thin.N // 3, thin.N - 1):
        c, st = thin.run(j, k, rho, tau, n)
        ref = oracle.modal_response(k, rho, thin.lam[j], tau, n)[-1]
        assert abs(c - ref) <= 1e-8, (j, c, ref, tau * math.sqrt(thin.lam[j]))


def test_study_shows_the_order_effect(thin):
    """At tau = 1e-3 the fourth-order scheme's error on the low modes is far below the
    second-order one's; every configuration run is stable."""
    rows = dispersion.study(taus=(1e-3,), ks=(1, 2), rhos=(0.5,), js=(1, 2), t_end=0.5, thin=thin)
    err = {(r["j"], r["k"]): r["err_semidiscrete"] for r in rows}
    assert all(r["stable"] for r in rows)
    for j in (1, 2):
        assert err[(j, 2)] < 1e-2 * err[(j, 1)]
