"""Mean PCG iterations of the multi-patch scheme with the additive Schwarz preconditioner
(the quantity of the paper's Table Fan_its, Sec. 6, on its multi-patch fan), here on a
2 x 2 grid of deformed patches (N_adj = 4) -- oracle, plain FP64; test infrastructure.

Setting as in that table: tau = 5e-5, T = 64 tau, PCG tolerance 1e-12 from the null guess;
k = 2, rho_inf = 0.5; initial displacement prod_a sin(pi x_a / 2) at the global functions'
control points, zero velocity. Rows: elements per patch side n_sub; columns: p = 1..4.

Usage: python -m oracle.multipatch_table [--nsub 4 8 16 32]
"""
from __future__ import annotations

import argparse

import numpy as np

from . import Stepper
from .multipatch import GluedPatches


def mean_iterations(patches, tau=5e-5, nsteps=64, k=2, rho=0.5, tol=1e-12):
    """Mean PCG iterations per solve over nsteps steps of the glued system."""
    g = GluedPatches(patches)
    d = g.d
    X = np.zeros((g.N, d))
    for (deg, kn, ctrl), loc in zip(patches, g.local):
        X[loc["ids"]] = np.asarray(ctrl).reshape(-1, d)[loc["keep"]]
    U0 = np.prod(np.sin(np.pi * X / 2.0), axis=1)
    st = Stepper(g, k, rho, tol=tol)
    state = st.init(U0, np.zeros(g.N))
    for _ in range(nsteps):
        state = st.step(state, tau)
    return float(np.mean(np.array(st.iters, dtype=float))), g.N


def main():
    from workloads import multipatch as WM

    ap = argparse.ArgumentParser()
    ap.add_argument("--nsub", type=int, nargs="+", default=[4, 8, 16, 32])
    a = ap.parse_args()
    print("| n_sub | p=1 | p=2 | p=3 | p=4 |")
    print("|---|---|---|---|---|")
    for nsub in a.nsub:
        vals = [mean_iterations(WM.grid_of_patches((2, 2), nsub, p, amp=0.1))[0] for p in (1, 2, 3, 4)]
        print("| %d | %s |" % (nsub, " | ".join("%.1f" % v for v in vals)), flush=True)


if __name__ == "__main__":
    main()
