"""Conforming multi-patch discretisation and the additive Schwarz mass preconditioner
(Sec. 5.1 "Multi-patch B-splines", Sec. 5.4, def:asp) -- oracle, plain FP64 numpy.

Test infrastructure, like the rest of `oracle/`: only the tests use it.

Scope: 2-D patches of one degree p in a row along direction 0, patch r glued to patch
r+1 along its face i0 = m0 - 1 (the face i0 = 0 of patch r+1), both faces with the same
knot vector in direction 1 and the same control points (Assumption ass:conformity);
homogeneous Dirichlet conditions on the outer boundary.

- Local functions of patch r: its tensor-product B-splines that do not lie on an outer
  face (per direction a range of indices: 1..m-2, extended to 0 or m-1 where that face is
  an interface).
- Global functions: the local ones with the interface functions of both sides identified
  (G^(r) of Sec. 5.1); global M and K are sums over the patches of their local matrices
  (integrals over the patch) scattered through G^(r).
- Additive Schwarz (def:asp): P_ad^{-1} = sum_r R^(r)T P^(r)^{-1} R^(r), R^(r) the selection
  of patch r's global functions, P^(r) = D^(r)^{1/2} Dhat^(r)^{-1/2} Mhat^(r) Dhat^(r)^{-1/2}
  D^(r)^{1/2} (def:loc_forms2) with Mhat^(r) the Kronecker product of the univariate
  parametric mass matrices over the local index ranges, Dhat^(r) its diagonal and D^(r) the
  diagonal of the patch's own mass matrix M^(r) (def:loc_matrices; the reading: the patch's
  integral, not the global diagonal restricted to the patch).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import Quad1D


def patch_full_matrices(degrees, knots, ctrl, nq=None):
    """Mass and stiffness matrices of one 2-D patch over ALL its tensor-product functions
    (index j * m0 + i for function (i, j), direction 0 fastest), by Gauss quadrature
    (nq points per element and direction, default p + 1) with the geometry of the control
    net ctrl (shape (m0 m1, 2), direction 0 fastest): M = int N_a N_b |det J|,
    K = int grad N_a . grad N_b |det J| (Sec. 2)."""
    p0, p1 = degrees
    nq = nq or max(p0, p1) + 1
    q0, q1 = Quad1D(p0, knots[0], nq), Quad1D(p1, knots[1], nq)
    B0, dB0 = q0.dense(), q0.dense(True)  # (Q0, m0)
    B1, dB1 = q1.dense(), q1.dense(True)  # (Q1, m1)
    m0, m1 = q0.m, q1.m
    C = np.asarray(ctrl, dtype=np.float64).reshape(m1, m0, 2)
    Cx, Cy = C[:, :, 0], C[:, :, 1]
    # geometry at the points (q1, q0)
    x_xi = B1 @ Cx @ dB0.T
    x_eta = dB1 @ Cx @ B0.T
    y_xi = B1 @ Cy @ dB0.T
    y_eta = dB1 @ Cy @ B0.T
    det = x_xi * y_eta - x_eta * y_xi
    if np.min(det) <= 0:
        raise ValueError("det DF <= 0 at a quadrature point")
    w = np.outer(q1.qw, q0.qw) * det  # |det J| times the weights
    # J^{-1} J^{-T} |det J|: with J = [[x_xi, x_eta], [y_xi, y_eta]],
    # J^{-1} = [[y_eta, -x_eta], [-y_xi, x_xi]] / det
    g00 = np.outer(q1.qw, q0.qw) * (y_eta ** 2 + x_eta ** 2) / det
    g01 = np.outer(q1.qw, q0.qw) * (-(y_eta * y_xi) - (x_eta * x_xi)) / det
    g11 = np.outer(q1.qw, q0.qw) * (y_xi ** 2 + x_xi ** 2) / det
    M = np.einsum("ab,aj,bi,al,bk->jilk", w, B1, B0, B1, B0, optimize=True).reshape(m0 * m1, m0 * m1)
    # d/dxi of N_(i,j) = B1_j dB0_i, d/deta = dB1_j B0_i
    K = (np.einsum("ab,aj,bi,al,bk->jilk", g00, B1, dB0, B1, dB0, optimize=True)
         + np.einsum("ab,aj,bi,al,bk->jilk", g01, B1, dB0, dB1, B0, optimize=True)
         + np.einsum("ab,aj,bi,al,bk->jilk", g01, dB1, B0, B1, dB0, optimize=True)
         + np.einsum("ab,aj,bi,al,bk->jilk", g11, dB1, B0, dB1, B0, optimize=True)).reshape(m0 * m1, m0 * m1)
    Mhat = (q0.dense().T @ (q0.qw[:, None] * q0.dense()), q1.dense().T @ (q1.qw[:, None] * q1.dense()))
    return M, K, Mhat, (m0, m1)


class GluedPatches:
    """Patches in a row along direction 0, glued conformingly (see the module docstring)."""

    def __init__(self, patches, nq=None):
        """patches: list of (degrees, knots, ctrl), patch r's face i0 = m0 - 1 glued to the
        face i0 = 0 of patch r + 1."""
        self.P = len(patches)
        self.local = []  # per patch: kept ranges, global ids of the kept functions, matrices
        gid = {}
        nglob = 0
        for r, (deg, knots, ctrl) in enumerate(patches):
            M, K, Mhat, (m0, m1) = patch_full_matrices(deg, knots, ctrl, nq)
            lo0 = 0 if r > 0 else 1
            hi0 = m0 - 1 if r < self.P - 1 else m0 - 2
            lo1, hi1 = 1, m1 - 2
            ids = []
            for j in range(lo1, hi1 + 1):
                for i in range(lo0, hi0 + 1):
                    key = (r, i, j)
                    if r > 0 and i == 0:  # the left patch's face i0 = m0 - 1, same j
                        key = (r - 1, self.local[r - 1]["m"][0] - 1, j)
                    if key not in gid:
                        gid[key] = nglob
                        nglob += 1
                    ids.append(gid[key])
            keep = [j * m0 + i for j in range(lo1, hi1 + 1) for i in range(lo0, hi0 + 1)]
            Ml, Kl = M[np.ix_(keep, keep)], K[np.ix_(keep, keep)]
            Mh0 = Mhat[0][lo0:hi0 + 1, lo0:hi0 + 1]
            Mh1 = Mhat[1][lo1:hi1 + 1, lo1:hi1 + 1]
            self.local.append({"m": (m0, m1), "ids": np.array(ids), "M": Ml, "K": Kl, "Mhat": (Mh0, Mh1),
                               "n": (hi0 - lo0 + 1, hi1 - lo1 + 1)})
        self.N = nglob
        self.M = np.zeros((nglob, nglob))
        self.K = np.zeros((nglob, nglob))
        for loc in self.local:
            ix = np.ix_(loc["ids"], loc["ids"])
            self.M[ix] += loc["M"]
            self.K[ix] += loc["K"]
        # multiplicity n_l of each global function (def:n_l) and N_adj (def:N_patch)
        self.mult = np.zeros(nglob, dtype=int)
        for loc in self.local:
            self.mult[loc["ids"]] += 1
        self.n_adj = int(self.mult.max())
        # local preconditioners P^(r): Cholesky factors of the univariate Mhat, the scalings
        for loc in self.local:
            Mh0, Mh1 = loc["Mhat"]
            loc["cho"] = (scipy.linalg.cho_factor(Mh0), scipy.linalg.cho_factor(Mh1))
            dhat = np.kron(np.diag(Mh1), np.diag(Mh0))  # direction 0 fastest
            loc["scale"] = np.sqrt(dhat / np.diag(loc["M"]))  # D^(r)^{-1/2} Dhat^(r)^{1/2}

    def local_Pinv(self, r, v):
        """P^(r)^{-1} v = D^{-1/2} Dhat^{1/2} (Mhat_1 (x) Mhat_0)^{-1} Dhat^{1/2} D^{-1/2} v."""
        loc = self.local[r]
        n0, n1 = loc["n"]
        t = (loc["scale"] * v).reshape(n1, n0)
        t = scipy.linalg.cho_solve(loc["cho"][0], t.T).T  # direction 0
        t = scipy.linalg.cho_solve(loc["cho"][1], t)  # direction 1
        return loc["scale"] * t.reshape(-1)

    # Operators-like interface (oracle.pcg, oracle.Stepper)
    def apply_M(self, x):
        return self.M @ x

    def apply_K(self, x):
        return self.K @ x

    def apply_Pinv(self, r):
        """The additive Schwarz preconditioner (def:asp): sum_r R^(r)T P^(r)^{-1} R^(r) r."""
        z = np.zeros(self.N)
        for q, loc in enumerate(self.local):
            z[loc["ids"]] += self.local_Pinv(q, r[loc["ids"]])
        return z

    def dense_Pinv(self):
        return np.column_stack([self.apply_Pinv(e) for e in np.eye(self.N)])


def row_of_patches(npatch, nel, p, amp=0.0):
    """npatch unit-square patches side by side along x ([r, r+1] x [0, 1]), nel x nel
    elements of degree p each, control points at the Greville abscissae moved by the
    smooth map (x, y) -> (x + amp sin(pi x / npatch) sin(pi y), y + amp sin(pi x / npatch)
    sin(pi y)); interface control points coincide, so the patches are conforming."""
    def knots_(n):
        return np.array([0.0] * (p + 1) + [i / n for i in range(1, n)] + [1.0] * (p + 1))

    def greville(kn):
        m = len(kn) - p - 1
        return np.array([kn[i + 1:i + p + 1].mean() for i in range(m)])

    kx = ky = knots_(nel)
    gx, gy = greville(kx), greville(ky)
    out = []
    for r in range(npatch):
        pts = []
        for y in gy:
            for x in gx:
                X = r + x
                b = amp * np.sin(np.pi * X / npatch) * np.sin(np.pi * y)
                pts.append((X + b, y + b))
        out.append(((p, p), [kx, ky], np.array(pts)))
    return out
