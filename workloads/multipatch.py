"""Seeded synthetic layouts of conforming patches (multi-patch inputs). Input generation
only: knot vectors and control nets, none of the method's arithmetic.

Recipe. The paper's multi-patch geometry (the fan of Sec. 6) is not published, so grids of
unit patches stand in for it: patch r covers [r_0, r_0 + 1] x ... on a grid of shape[a]
patches per direction, with nel uniform elements of degree p per direction (open knot
vectors, maximal regularity), control points at the Greville abscissae, and every
coordinate moved by b(X) = amp prod_a sin(pi X_a / shape_a), which vanishes on the outer
boundary of the grid. Neighbouring patches get the same control points on their common
face (the same formula at the same points), so they are conforming. An L is the 2 x 2
grid without its patch at [1, 2] x [1, 2]; `reorient` renames or reverses a patch's
parameter directions without changing its geometry.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import greville, open_uniform_knots


def grid_of_patches(shape, nel, p, amp=0.0):
    """List of (degrees, knots, ctrl) for the grid `shape`; patch index r_0 + shape_0 (r_1 +
    shape_1 r_2); ctrl has shape (prod m, d), direction 0 fastest."""
    d = len(shape)
    kn = open_uniform_knots(nel, p)
    g = greville(kn, p)
    out = []
    for r_rev in itertools.product(*[range(s) for s in reversed(shape)]):
        r = r_rev[::-1]
        pts = []
        for ix_rev in itertools.product(*[range(len(g))] * d):
            X = np.array([r[a] + g[ix_rev[d - 1 - a]] for a in range(d)])
            b = amp
            for a in range(d):
                b = b * np.sin(np.pi * X[a] / shape[a])
            pts.append(X + b)
        out.append(((p,) * d, [kn] * d, np.array(pts)))
    return out


def row_of_patches(npatch, nel, p, amp=0.0):
    """npatch unit-square patches side by side along x ([r, r+1] x [0, 1])."""
    return grid_of_patches((npatch, 1), nel, p, amp)


def l_shape(nel, p, amp=0.0):
    """Three unit squares forming an L: the 2 x 2 grid without its patch at [1, 2] x [1, 2]."""
    return [pt for r, pt in enumerate(grid_of_patches((2, 2), nel, p, amp)) if r != 3]


def reorient(patch, perm=None, flip=()):
    """The same patch with its parameter directions renamed and reversed: new direction a is
    the old direction perm[a], reversed if a is in flip."""
    degrees, knots, ctrl = patch
    d = len(degrees)
    perm = list(perm) if perm is not None else list(range(d))
    m = [len(kn) - p - 1 for p, kn in zip(degrees, knots)]
    net = np.asarray(ctrl, dtype=np.float64).reshape(list(reversed(m)) + [d])
    net = np.transpose(net, [d - 1 - perm[a] for a in reversed(range(d))] + [d])
    kn2 = [np.asarray(knots[perm[a]], dtype=np.float64) for a in range(d)]
    for a in flip:
        net = np.flip(net, axis=d - 1 - a)
        kn2[a] = (kn2[a][0] + kn2[a][-1]) - kn2[a][::-1]
    return tuple(degrees[perm[a]] for a in range(d)), kn2, np.ascontiguousarray(net).reshape(-1, d)
