"""Conforming multi-patch discretisation and the additive Schwarz mass preconditioner
(Sec. 5.1 "Multi-patch B-splines", Sec. 5.4, def:asp) -- oracle, plain FP64 numpy.

Test infrastructure, like the rest of `oracle/`: only the tests use it.

Scope: 2-D or 3-D patches glued face to face in any layout (rows, grids, L-shapes; any
relative orientation of the parameter directions), each interface face shared by exactly
two patches with the same knots and the same control points (Assumption ass:conformity);
homogeneous Dirichlet conditions on every face that is not an interface.

- Interfaces: a face of a patch is an interface when its control points are, as a set,
  those of a face of another patch. Conformity makes the functions on the two faces equal
  one by one, and each pair has coincident control points, so the gluing G^(r) of Sec. 5.1
  is read off the control points: whatever the orientation of the two patches.
- Global functions (def:mp_basis): the patches' tensor-product B-splines, those on
  interfaces identified through their control points; a global function is kept unless one
  of its copies lies on an outer face (it would not vanish on the Dirichlet boundary: at a
  re-entrant corner that removes a function whose other copies lie on interfaces only).
- Local functions of patch r: the copies of kept global functions. They lie in the tensor
  range of indices 1..m-2 per direction, widened to 0 or m-1 where that face is an
  interface; the range is the whole local set except next to re-entrant corners.
- Global M and K are sums over the patches of their local matrices (integrals over the
  patch) scattered through G^(r).
- Additive Schwarz (def:asp): P_ad^{-1} = sum_r R^(r)T P^(r)^{-1} R^(r), R^(r) the selection
  of patch r's global functions, P^(r) = D^(r)^{1/2} Dhat^(r)^{-1/2} Mhat^(r) Dhat^(r)^{-1/2}
  D^(r)^{1/2} (def:loc_forms2) with Mhat^(r) the Kronecker product of the univariate
  parametric mass matrices over the local index ranges, Dhat^(r) its diagonal and D^(r) the
  diagonal of the patch's own mass matrix M^(r) (def:loc_matrices; the reading: the patch's
  integral, not the global diagonal restricted to the patch). Where the local set is the
  tensor range minus some functions, P^(r)^{-1} is the Kronecker inverse over the range
  with those entries zero on input and dropped on output (the reading that keeps the
  Kronecker solve; a principal block of an SPD inverse, so still SPD).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg

from . import Quad1D


def _tensor(tables):
    """Kronecker product of per-direction tables with direction 0 fastest: tables[a] is
    (Q_a, m_a); the result has row q_0 + Q_0 (q_1 + Q_1 q_2) and column i_0 + m_0 (i_1 + ...)."""
    T = np.ones((1, 1))
    for t in tables:
        T = np.kron(t, T)
    return T


def patch_full_matrices(degrees, knots, ctrl, nq=None):
    """Mass and stiffness matrices of one patch over ALL its tensor-product functions (index
    i_0 + m_0 (i_1 + m_1 i_2), direction 0 fastest), by Gauss quadrature (nq points per
    element and direction, default max p + 1) with the geometry of the control net ctrl
    (shape (prod m, d), same order): M = int N_a N_b |det J|, K = int grad N_a . grad N_b
    |det J| (Sec. 2), with grad = J^{-T} grad_xi. Also the univariate parametric mass
    matrices over all functions and the counts m."""
    d = len(degrees)
    nq = nq or max(degrees) + 1
    quads = [Quad1D(p, kn, nq) for p, kn in zip(degrees, knots)]
    m = [q.m for q in quads]
    B = _tensor([q.dense() for q in quads])  # (Q, N) values at the tensor points
    dB = [_tensor([q.dense(c == a) for c, q in enumerate(quads)]) for a in range(d)]
    w = _tensor([q.qw[:, None] for q in quads])[:, 0]
    P = np.asarray(ctrl, dtype=np.float64).reshape(-1, d)
    J = np.stack([dB[a] @ P for a in range(d)], axis=2)  # J[q, c, a] = d x_c / d xi_a
    det = np.linalg.det(J)
    if not (np.all(det > 0) or np.all(det < 0)):
        raise ValueError("det DF vanishes or changes sign in the patch")
    Jinv = np.linalg.inv(J)  # Jinv[q, a, c] = d xi_a / d x_c
    G = Jinv @ np.transpose(Jinv, (0, 2, 1))  # G[q, a, b] = grad xi_a . grad xi_b
    wd = w * np.abs(det)
    M = B.T @ (wd[:, None] * B)
    K = sum(dB[a].T @ ((wd * G[:, a, b])[:, None] * dB[b]) for a in range(d) for b in range(d))
    Mhat = [q.dense().T @ (q.qw[:, None] * q.dense()) for q in quads]
    return M, K, Mhat, m


def _key(pt):
    return tuple(np.round(np.asarray(pt, dtype=np.float64), 10) + 0.0)


def _face_flat(m, a, side):
    """Flat indices (direction 0 fastest) of the functions on the face i_a = 0 (side 0) or
    i_a = m_a - 1 (side 1)."""
    rng = [range(n) for n in m]
    rng[a] = [0] if side == 0 else [m[a] - 1]
    return [_flat(ix, m) for ix in itertools.product(*reversed(rng))]


def _flat(ix_rev, m):
    """Flat index of the multi-index given last direction first."""
    f = 0
    for i, n in zip(ix_rev, reversed(m)):
        f = f * n + i
    return f


class GluedPatches:
    """Conforming patches glued face to face (see the module docstring)."""

    def __init__(self, patches, nq=None):
        """patches: list of (degrees, knots, ctrl)."""
        self.P = len(patches)
        self.d = len(patches[0][0])
        d = self.d
        full = []
        for deg, knots, ctrl in patches:
            M, K, Mhat, m = patch_full_matrices(deg, knots, ctrl, nq)
            full.append((M, K, Mhat, m, np.asarray(ctrl, dtype=np.float64).reshape(-1, d)))
        # interface faces: equal control-point sets on two different patches
        owners = {}
        for r, (_, _, _, m, pts) in enumerate(full):
            for a in range(d):
                for side in (0, 1):
                    fk = frozenset(_key(pts[f]) for f in _face_flat(m, a, side))
                    owners.setdefault(fk, []).append((r, a, side))
        self.interfaces = []
        iface = set()
        for fk, own in owners.items():
            if len(own) > 2 or (len(own) == 2 and own[0][0] == own[1][0]):
                raise ValueError("a face is shared by more than two patch faces: not conforming")
            if len(own) == 2:
                self.interfaces.append(tuple(own))
                iface.update(own)
        # identification: every function of every patch gets a key (functions on interfaces:
        # their control point); a key is outer when one of its copies lies on an outer face
        keys, outer = [], set()
        for r, (M, K, Mhat, m, pts) in enumerate(full):
            kr = {}
            for ix_rev in itertools.product(*[range(n) for n in reversed(m)]):
                f = _flat(ix_rev, m)
                ix = ix_rev[::-1]
                faces = [(a, 0) for a in range(d) if ix[a] == 0] + [(a, 1) for a in range(d) if ix[a] == m[a] - 1]
                on_iface = any((r, a, s_) in iface for a, s_ in faces)
                kr[f] = ("iface", _key(pts[f])) if on_iface else ("own", r, f)
                if any((r, a, s_) not in iface for a, s_ in faces):
                    outer.add(kr[f])
            keys.append(kr)
        self.local = []
        gid = {}
        nglob = 0
        for r, (M, K, Mhat, m, pts) in enumerate(full):
            lo = [0 if (r, a, 0) in iface else 1 for a in range(d)]
            hi = [m[a] - 1 if (r, a, 1) in iface else m[a] - 2 for a in range(d)]
            keep, ids, mask = [], [], []
            for ix_rev in itertools.product(*[range(lo[a], hi[a] + 1) for a in reversed(range(d))]):
                f = _flat(ix_rev, m)
                key = keys[r][f]
                mask.append(key not in outer)
                if key in outer:
                    continue
                if key not in gid:
                    gid[key] = nglob
                    nglob += 1
                keep.append(f)
                ids.append(gid[key])
            n = [hi[a] - lo[a] + 1 for a in range(d)]
            self.local.append({"m": m, "lo": lo, "n": n, "ids": np.array(ids, dtype=int), "mask": np.array(mask),
                               "M": M[np.ix_(keep, keep)], "K": K[np.ix_(keep, keep)],
                               "Mhat": [Mhat[a][lo[a]:hi[a] + 1, lo[a]:hi[a] + 1] for a in range(d)]})
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
            loc["cho"] = [scipy.linalg.cho_factor(Mh) for Mh in loc["Mhat"]]
            dhat = _tensor([np.diag(Mh)[:, None] for Mh in loc["Mhat"]])[:, 0][loc["mask"]]
            loc["scale"] = np.sqrt(dhat / np.diag(loc["M"]))  # D^(r)^{-1/2} Dhat^(r)^{1/2}

    def local_Pinv(self, r, v):
        """P^(r)^{-1} v = D^{-1/2} Dhat^{1/2} (Mhat_{d-1} (x) ... (x) Mhat_0)^{-1} Dhat^{1/2} D^{-1/2} v."""
        loc = self.local[r]
        d = self.d
        t = np.zeros(loc["mask"].size)
        t[loc["mask"]] = loc["scale"] * v
        t = t.reshape(list(reversed(loc["n"])))  # array axis d-1-a is direction a
        for a in range(d):
            ax = d - 1 - a
            u = np.moveaxis(t, ax, 0)
            sh = u.shape
            u = scipy.linalg.cho_solve(loc["cho"][a], u.reshape(sh[0], -1)).reshape(sh)
            t = np.moveaxis(u, 0, ax)
        return loc["scale"] * t.reshape(-1)[loc["mask"]]

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
