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


def _einsum_rows(S, facs):
    """sum over the tensor points of S (array axes: direction d-1 first) times, per direction
    a, the table facs[a] (|S_a|, c_a): the array of shape (c_{d-1}, ..., c_0)."""
    d = len(facs)
    pts = "".join(chr(ord("a") + k) for k in range(d))          # point axes, direction d-1 first
    outs = "".join(chr(ord("n") + k) for k in range(d))         # candidate axes, same order
    terms = [pts] + [pts[d - 1 - a] + outs[d - 1 - a] for a in range(d)]
    return np.einsum(",".join(terms) + "->" + outs, S, *facs, optimize=True)


def patch_rows(degrees, knots, ctrl, rows, nq=None):
    """Rows of one patch's M and K over ALL its functions (flat index i_0 + m_0 (i_1 + ...)),
    for the functions `rows` (flat indices), integrated by the Gauss rule (nq points, default
    max p + 1) over the elements in each row function's support only: for each row a dict
    {column: (M_ij, K_ij)} over the columns with |j_a - i_a| <= p_a. The geometry comes from
    the whole control net at the support points (Sec. 2: M_ij = int B_i B_j |det J|,
    K_ij = int grad B_i . grad B_j |det J|)."""
    d = len(degrees)
    nq = nq or max(degrees) + 1
    quads = [Quad1D(p, kn, nq) for p, kn in zip(degrees, knots)]
    m = [q.m for q in quads]
    B = [q.dense() for q in quads]
    dB = [q.dense(True) for q in quads]
    net = np.asarray(ctrl, dtype=np.float64).reshape(list(reversed(m)) + [d])
    wq = [q.qw for q in quads]
    out = []
    for i in rows:
        ia, f = [], int(i)
        for a in range(d):
            ia.append(f % m[a])
            f //= m[a]
        S = [np.nonzero(B[a][:, ia[a]])[0] for a in range(d)]          # support points per direction
        cand = [np.arange(max(0, ia[a] - degrees[a]), min(m[a], ia[a] + degrees[a] + 1)) for a in range(d)]
        # geometry at the support points
        J = np.empty([len(S[a]) for a in reversed(range(d))] + [d, d])
        for b in range(d):
            tabs = [(dB[a] if a == b else B[a])[S[a], :] for a in range(d)]
            for c in range(d):
                A = net[..., c]
                for a in range(d):
                    ax = d - 1 - a
                    A = np.moveaxis(np.tensordot(tabs[a], A, axes=(1, ax)), 0, ax)
                J[..., c, b] = A
        det = np.linalg.det(J)
        w = wq[0][S[0]]
        for a in range(1, d):
            w = np.multiply.outer(wq[a][S[a]], w)
        W = w * np.abs(det)
        Jinv = np.linalg.inv(J)
        G = np.einsum("...ac,...bc->...ab", Jinv, Jinv)
        # the row function and its parametric gradient at the support points
        def tensor(vecs):
            T = vecs[0]
            for a in range(1, d):
                T = np.multiply.outer(vecs[a], T)
            return T
        Ni = tensor([B[a][S[a], ia[a]] for a in range(d)])
        dNi = [tensor([(dB[a] if a == b else B[a])[S[a], ia[a]] for a in range(d)]) for b in range(d)]
        Mrow = _einsum_rows(W * Ni, [B[a][np.ix_(S[a], cand[a])] for a in range(d)])
        Krow = np.zeros_like(Mrow)
        for b in range(d):
            for c in range(d):
                Krow += _einsum_rows(W * G[..., b, c] * dNi[b],
                                     [(dB[a] if a == c else B[a])[np.ix_(S[a], cand[a])] for a in range(d)])
        row = {}
        for jr in itertools.product(*[range(len(cand[a])) for a in reversed(range(d))]):
            ja = [cand[a][jr[d - 1 - a]] for a in range(d)]
            j = 0
            for a in reversed(range(d)):
                j = j * m[a] + int(ja[a])
            row[j] = (float(Mrow[jr]), float(Krow[jr]))
        out.append(row)
    return out


def glued_rows(patches, local, rows, x, nq=None):
    """(M x)_g and (K x)_g of the glued system for the global functions `rows`, x a global
    vector: the sums over the copies (r, i) of global function g of patch r's rows over its
    local functions, sum_j M^(r)_ij x_gid(r, j) (Sec. 5.1: M = sum_r R^(r)T M^(r) R^(r)).
    local: the first result of glue(patches)."""
    copies = {}
    for r, loc in enumerate(local):
        for f, g in loc["to_gid"].items():
            copies.setdefault(g, []).append((r, f))
    Mx, Kx = np.zeros(len(rows)), np.zeros(len(rows))
    for k, g in enumerate(rows):
        for r, f in copies[g]:
            deg, knots, ctrl = patches[r]
            (row,) = patch_rows(deg, knots, ctrl, [f], nq)
            to_gid = local[r]["to_gid"]
            for j, (mij, kij) in row.items():
                if j in to_gid:
                    Mx[k] += mij * x[to_gid[j]]
                    Kx[k] += kij * x[to_gid[j]]
    return Mx, Kx


def glue(patches):
    """The numbering of Sec. 5.1 for conforming patches (see the module docstring), without
    matrices: per patch its function counts m, index box (lo, n), the flat full indices of
    its local functions (keep, box order), their global ids (ids), the box mask, and a dict
    full index -> global id; plus the number of global functions."""
    d = len(patches[0][0])
    nets = []
    for deg, knots, ctrl in patches:
        m = [len(kn) - p - 1 for p, kn in zip(deg, knots)]
        nets.append((m, np.asarray(ctrl, dtype=np.float64).reshape(-1, d)))
    # interface faces: equal control-point sets on two different patches
    owners = {}
    for r, (m, pts) in enumerate(nets):
        for a in range(d):
            for side in (0, 1):
                fk = frozenset(_key(pts[f]) for f in _face_flat(m, a, side))
                owners.setdefault(fk, []).append((r, a, side))
    interfaces, iface = [], set()
    for fk, own in owners.items():
        if len(own) > 2 or (len(own) == 2 and own[0][0] == own[1][0]):
            raise ValueError("a face is shared by more than two patch faces: not conforming")
        if len(own) == 2:
            interfaces.append(tuple(own))
            iface.update(own)
    # faces that cover the same region (equal bounding boxes) without equal control-point sets:
    # a non-conforming interface (Assumption ass:conformity), not two Dirichlet faces
    boxes = {}
    for fk, own in owners.items():
        if len(own) == 1:
            pts_f = np.array(sorted(fk))
            bb = (_key(pts_f.min(axis=0)), _key(pts_f.max(axis=0)))
            if bb in boxes and boxes[bb][0] != own[0][0]:
                raise ValueError("two faces cover the same region with different control points: not conforming")
            boxes[bb] = own[0]
    # identification: every function of every patch gets a key (functions on interfaces:
    # their control point); a key is outer when one of its copies lies on an outer face
    keys, outer = [], set()
    for r, (m, pts) in enumerate(nets):
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
    local, gid, nglob = [], {}, 0
    for r, (m, pts) in enumerate(nets):
        lo = [0 if (r, a, 0) in iface else 1 for a in range(d)]
        hi = [m[a] - 1 if (r, a, 1) in iface else m[a] - 2 for a in range(d)]
        keep, ids, mask, to_gid = [], [], [], {}
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
            to_gid[f] = gid[key]
        local.append({"m": m, "lo": lo, "n": [hi[a] - lo[a] + 1 for a in range(d)], "keep": keep,
                      "ids": np.array(ids, dtype=int), "mask": np.array(mask), "to_gid": to_gid})
    return local, nglob, interfaces


class GluedPatches:
    """Conforming patches glued face to face (see the module docstring)."""

    def __init__(self, patches, nq=None):
        """patches: list of (degrees, knots, ctrl)."""
        self.P = len(patches)
        self.d = d = len(patches[0][0])
        self.local, nglob, self.interfaces = glue(patches)
        for loc, (deg, knots, ctrl) in zip(self.local, patches):
            M, K, Mhat, m = patch_full_matrices(deg, knots, ctrl, nq)
            keep, lo, n = loc["keep"], loc["lo"], loc["n"]
            loc["M"], loc["K"] = M[np.ix_(keep, keep)], K[np.ix_(keep, keep)]
            loc["Mhat"] = [Mhat[a][lo[a]:lo[a] + n[a], lo[a]:lo[a] + n[a]] for a in range(d)]
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
