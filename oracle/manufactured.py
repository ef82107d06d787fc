"""Manufactured solutions for the spatial accuracy of the discretisation (the O(h^{p+1})
L2 convergence the paper measures in Sec. 6 with a forced, exactly known solution) --
oracle, plain FP64 numpy.

Test infrastructure, like the rest of `oracle/`: only the tests use it.

The solution is u(x, t) = S(x) (cos wt + sin wt) with S = prod_a sin(pi x_a) on the unit
square or cube, which vanishes on the boundary (homogeneous Dirichlet conditions, the
only ones the discretisation carries). With unit wave speed, u_tt - Lap u = f for
f = (d pi^2 - w^2) S (cos wt + sin wt), so the semi-discrete problem is
M U'' + K U = F(t) with F(t) = (d pi^2 - w^2) (cos wt + sin wt) G, G_i = int S B_i; the
initial data are the L2 projections of u(0) = S and u_t(0) = w S.

Integrals over a patch use the tensor Gauss rule of nq points per element and direction:
x(xi) = sum_i C_i B_i(xi) over the full control net, weights w |det DF|, and the interior
B-splines (the first and last of each direction carry the Dirichlet condition).
"""
from __future__ import annotations

import math

import numpy as np

from . import Quad1D


def _contract(tables, A):
    """sum over the functions of A (array axis d-1-a is direction a) against tables[a]
    (Q_a, n_a): the values at the tensor points, same axis order."""
    d = len(tables)
    for a in range(d):
        ax = d - 1 - a
        A = np.moveaxis(np.tensordot(tables[a], A, axes=(1, ax)), 0, ax)
    return A


class PatchQuadrature:
    """Physical Gauss points, weights w |det DF| and interior basis tables of one patch."""

    def __init__(self, degrees, knots, ctrl, nq, lo=None, n=None):
        """The functions are the box lo_a .. lo_a + n_a - 1 per direction (default: the
        interior functions 1 .. m_a - 2)."""
        self.d = d = len(degrees)
        quads = [Quad1D(p, kn, nq) for p, kn in zip(degrees, knots)]
        self.m = [q.m for q in quads]
        full = [q.dense() for q in quads]
        dfull = [q.dense(True) for q in quads]
        lo = lo if lo is not None else [1] * d
        n = n if n is not None else [self.m[a] - 2 for a in range(d)]
        self.B = [full[a][:, lo[a]:lo[a] + n[a]] for a in range(d)]
        self.n = [t.shape[1] for t in self.B]
        net = np.asarray(ctrl, dtype=np.float64).reshape(list(reversed(self.m)) + [d])
        # x_c and its derivatives along each direction at the points
        self.x = np.stack([_contract(full, net[..., c]) for c in range(d)])
        J = np.empty(self.x.shape[1:] + (d, d))
        for b in range(d):
            tabs = [dfull[a] if a == b else full[a] for a in range(d)]
            for c in range(d):
                J[..., c, b] = _contract(tabs, net[..., c])
        det = np.linalg.det(J)
        w = quads[0].qw
        for a in range(1, d):  # tensor product of the weights, array axis d-1-a is direction a
            w = np.multiply.outer(quads[a].qw, w)
        self.W = w * np.abs(det)

    def integrate(self, g):
        """b_i = int g B_i over the patch, g given at the points (flat with direction 0 fastest,
        or shaped like W)."""
        tabs = [t.T for t in self.B]  # (n_a, Q_a)
        return _contract(tabs, self.W * np.asarray(g, dtype=np.float64).reshape(self.W.shape)).reshape(-1)

    def evaluate(self, U):
        """sum_i U_i B_i at the points."""
        return _contract(self.B, np.asarray(U, dtype=np.float64).reshape(list(reversed(self.n))))

    def l2_error(self, U, exact):
        """|| sum_i U_i B_i - exact ||_L2 with exact given at the points."""
        return math.sqrt(float(np.sum(self.W * (self.evaluate(U) - exact) ** 2)))


def standing_profile(x, lengths=None):
    """S(x) = prod_a sin(pi x_a / L_a) at points x of shape (d, ...) (L_a = 1 by default)."""
    L = np.ones(x.shape[0]) if lengths is None else np.asarray(lengths, dtype=np.float64)
    return np.prod(np.sin(np.pi * x / L.reshape((-1,) + (1,) * (x.ndim - 1))), axis=0)


class ForcedWave:
    """u = S(x) (cos wt + sin wt) and its semi-discrete data on one patch (see the module
    docstring). ops supplies apply_M and apply_K (oracle.Operators); quad integrates."""

    def __init__(self, quad: PatchQuadrature, omega: float):
        self.quad, self.omega = quad, omega
        self.S = standing_profile(quad.x)
        self.G = quad.integrate(self.S)
        self.amp = quad.d * math.pi ** 2 - omega ** 2

    def time_factor(self, s, t):
        """s-th derivative of cos wt + sin wt: w^s (cos(wt + s pi/2) + sin(wt + s pi/2))."""
        w = self.omega
        return w ** s * (math.cos(w * t + s * math.pi / 2) + math.sin(w * t + s * math.pi / 2))

    def forcing(self, s, t):
        """F^{(s)}(t), the loads of oracle.Stepper."""
        return self.amp * self.time_factor(s, t) * self.G

    def exact(self, t):
        return self.S * self.time_factor(0, t)

    def initial(self, solve_M):
        """L2 projections of u(0) = S and u_t(0) = w S: M U0 = G, V0 = w U0."""
        U0 = solve_M(self.G)
        return U0, self.omega * U0


class GluedForcedWave:
    """The forced wave u = S(x) (cos wt + sin wt), S = prod_a sin(pi x_a / L_a), on glued
    patches covering the box prod_a [0, L_a] (Sec. 5.1: V_h on the union): the global load
    G = sum_r R^(r)T int S B^(r), the L2 projections, and the L2 error summed over the
    patches. f = (sum_a (pi / L_a)^2 - w^2) S (cos wt + sin wt)."""

    def __init__(self, patches, glued, lengths, omega, nq):
        self.omega = omega
        self.quads, self.S = [], []
        d = len(lengths)
        G = np.zeros(glued.N)
        for (deg, kn, ctrl), loc in zip(patches, glued.local):
            q = PatchQuadrature(deg, kn, ctrl, nq, lo=loc["lo"], n=loc["n"])
            S = standing_profile(q.x, lengths)
            G[loc["ids"]] += q.integrate(S)[loc["mask"]]
            self.quads.append((q, loc))
            self.S.append(S)
        self.G = G
        self.amp = sum((math.pi / L) ** 2 for L in lengths) - omega ** 2
        self.d = d

    def time_factor(self, s, t):
        w = self.omega
        return w ** s * (math.cos(w * t + s * math.pi / 2) + math.sin(w * t + s * math.pi / 2))

    def forcing(self, s, t):
        return self.amp * self.time_factor(s, t) * self.G

    def initial(self, solve_M):
        U0 = solve_M(self.G)
        return U0, self.omega * U0

    def l2_error(self, U, t):
        tot = 0.0
        for (q, loc), S in zip(self.quads, self.S):
            box = np.zeros(loc["mask"].size)
            box[loc["mask"]] = U[loc["ids"]]
            tot += q.l2_error(box, S * self.time_factor(0, t)) ** 2
        return math.sqrt(tot)
