"""Dispersion study of the explicit generalized-alpha schemes, run through the GPU steps
(Sec. 6.2: u(x, t) = sin(j pi x) cos(pi t) on (0, 1) with wave speed omega = 1/j, N = 400
elements of degree 4 and regularity C^3, final time 5, tau = 0.05 and 1e-3, second
against fourth order and the role of rho_inf).

The library's patches are 2-D or 3-D, so the 1-D problem is a thin 2-D patch: the
elements of degree p across x, one quadratic element across y (a single interior
function there) and y stretched by `stretch`. Its mass and stiffness are L (M_x (x) m)
and L (K_x (x) m) + (M_x (x) k) / L, so its modes are the 1-D ones with eigenvalues
shifted by (k/m) / L^2 (10^-12 for L = 10^6).

The wave speed is a time scale: the scheme on M U'' + omega^2 K U = 0 with step tau is
the scheme on M U'' + K U = 0 with step omega tau. Each run starts from a discrete mode
phi_j (a generalized eigenvector of (K, M), M-normalised, the j-th from the bottom, whose
shape is sin(j pi x) for j well below N) with V0 = 0, so the discrete solution stays that
mode times the scheme's modal response. A run reports the mode's coefficient
c = phi_j^T M U at the final time against the exact cos(pi t) and the semi-discrete
cos(omega sqrt(lambda_j) t). A run whose fastest mode is beyond the stability limit
(omega tau > the library's critical step) is reported as unstable and not run: rounding
would excite that mode and it would grow.

Usage: python -m paper_2102_11536_gb300.dispersion [--nel 400] [--degree 4]
"""
from __future__ import annotations

import argparse
import math

import numpy as np


def _open_knots(nel, p):
    return np.array([0.0] * (p + 1) + [i / nel for i in range(1, nel)] + [1.0] * (p + 1))


def _greville(knots, p):
    m = len(knots) - p - 1
    return np.array([knots[i + 1:i + p + 1].mean() for i in range(m)])


def thin_patch_geometry(nel=400, p=4, stretch=1e6):
    """(degrees, knots, control net) of the thin 2-D patch standing in for (0, 1)."""
    kx, ky = _open_knots(nel, p), _open_knots(1, 2)
    gx, gy = _greville(kx, p), _greville(ky, 2) * stretch
    ctrl = np.array([(x, y) for y in gy for x in gx])  # direction 0 fastest
    return (p, 2), [kx, ky], ctrl


def dense_operators(patch):
    """M and K as dense host matrices, column by column through the library's products
    (small patches only)."""
    import torch

    N = patch.N
    M = np.zeros((N, N))
    K = np.zeros((N, N))
    for c0 in range(0, N, 8):
        nv = min(8, N - c0)
        E = np.zeros((nv, N))
        E[np.arange(nv), c0 + np.arange(nv)] = 1.0
        x = torch.from_numpy(E.reshape(-1)).cuda()
        y = torch.empty_like(x)
        patch.apply_M(x, y, nv)
        M[:, c0:c0 + nv] = y.cpu().numpy().reshape(nv, N).T
        patch.apply_K(x, y, nv)
        K[:, c0:c0 + nv] = y.cpu().numpy().reshape(nv, N).T
    return 0.5 * (M + M.T), 0.5 * (K + K.T)


class ThinPatch:
    """The thin patch on the GPU with its dense operators and modes."""

    def __init__(self, nel=400, p=4, stretch=1e6, tol=1e-13, op_form="assembled", precond="fp64"):
        import scipy.linalg

        from . import Patch

        deg, knots, ctrl = thin_patch_geometry(nel, p, stretch)
        self.patch = Patch(deg, knots, ctrl, tol=tol, op_form=op_form, precond=precond)
        self.N = self.patch.N
        self.M, self.K = dense_operators(self.patch)
        self.lam, self.Phi = scipy.linalg.eigh(self.K, self.M)  # ascending, M-orthonormal

    def run(self, j, k, rho, tau_eff, nsteps):
        """c = phi_j^T M U after nsteps steps of length tau_eff from U0 = phi_j, V0 = 0."""
        import torch

        phi = self.Phi[:, j]
        dev = torch.device("cuda", torch.cuda.current_device())
        state = torch.zeros(3 * k * self.N, dtype=torch.float64, device=dev)
        self.patch.state_init(k, torch.from_numpy(np.ascontiguousarray(phi)).to(dev),
                              torch.zeros(self.N, dtype=torch.float64, device=dev), state)
        self.patch.set_time(0.0)
        st = self.patch.step(state, k, rho, tau_eff, nsteps)
        U = state[:self.N].cpu().numpy()
        return float(phi @ (self.M @ U)), st

    def critical_step(self, rho):
        return self.patch.cfl(rho, iters=min(self.N, 300))[1]

    def close(self):
        self.patch.close()


def study(nel=400, p=4, taus=(0.05, 1e-3), ks=(1, 2), rhos=(0.0, 0.5, 1.0),
          js=(1, 2, 4, 8, 16, 32, 64, 128, 256), t_end=5.0, thin=None):
    """Rows (tau, j, k, rho, stable, c, error against cos(pi t), semi-discrete error)."""
    own = thin is None
    tp = thin or ThinPatch(nel, p)
    rows = []
    crit = {rho: tp.critical_step(rho) for rho in rhos}
    for tau in taus:
        n = int(round(t_end / tau))
        t = n * tau
        for j in js:
            if j > tp.N:
                continue
            omega = 1.0 / j
            semi = math.cos(omega * math.sqrt(tp.lam[j - 1]) * t)
            for k in ks:
                for rho in rhos:
                    stable = omega * tau <= 0.999 * crit[rho]
                    c = float("nan")
                    if stable:
                        c, _ = tp.run(j - 1, k, rho, omega * tau, n)
                    rows.append({"tau": tau, "j": j, "k": k, "rho": rho, "stable": stable,
                                 "Omega": omega * tau * math.sqrt(tp.lam[j - 1]), "c": c,
                                 "err_exact": abs(c - math.cos(math.pi * t)),
                                 "err_semidiscrete": abs(c - semi),
                                 "spatial": abs(semi - math.cos(math.pi * t))})
    if own:
        tp.close()
    return rows


def table(rows):
    """A markdown table of the study rows."""
    out = ["| tau | j | Omega = tau sqrt(lambda_j)/j | spatial error | k | rho_inf | "
           "error vs cos(pi t) | error vs semi-discrete |",
           "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        if not r["stable"]:
            out.append("| %g | %d | %.3g | %.2e | %d | %g | unstable (fastest mode beyond the limit) | |" % (
                r["tau"], r["j"], r["Omega"], r["spatial"], r["k"], r["rho"]))
        else:
            out.append("| %g | %d | %.3g | %.2e | %d | %g | %.3e | %.3e |" % (
                r["tau"], r["j"], r["Omega"], r["spatial"], r["k"], r["rho"], r["err_exact"],
                r["err_semidiscrete"]))
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nel", type=int, default=400)
    ap.add_argument("--degree", type=int, default=4)
    a = ap.parse_args()
    print(table(study(nel=a.nel, p=a.degree)))


if __name__ == "__main__":
    main()
