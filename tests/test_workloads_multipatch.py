"""The multi-patch input generators (workloads/multipatch.py): neighbouring patches share
their interface control points bit for bit (conforming, as the gluing needs), the
deformation keeps the outer boundary, and reorienting a patch twice by inverse maps
returns it unchanged."""
import numpy as np
import pytest

from workloads import multipatch as WM


def _net(patch):
    deg, kn, ctrl = patch
    d = len(deg)
    m = [len(k) - p - 1 for p, k in zip(deg, kn)]
    return np.asarray(ctrl).reshape(list(reversed(m)) + [d])


@pytest.mark.parametrize("shape", [(2, 1), (2, 3), (2, 2, 2)])
def test_neighbours_share_interface_control_points(shape):
    pts = WM.grid_of_patches(shape, 3, 2, amp=0.13)
    d = len(shape)
    idx = lambda r: [(r // int(np.prod(shape[:a]))) % shape[a] for a in range(d)]
    for r in range(len(pts)):
        for s in range(len(pts)):
            ir, is_ = idx(r), idx(s)
            diff = [b - a for a, b in zip(ir, is_)]
            if sorted(map(abs, diff)) != [0] * (d - 1) + [1] or sum(diff) != 1:
                continue
            a = diff.index(1)  # s follows r along direction a
            ax = d - 1 - a
            face_r = np.take(_net(pts[r]), -1, axis=ax)
            face_s = np.take(_net(pts[s]), 0, axis=ax)
            assert np.array_equal(face_r, face_s)


@pytest.mark.parametrize("d", [2, 3])
def test_deformation_keeps_the_outer_boundary(d):
    """Every outer face of the grid lies on its plane x_a = 0 or x_a = shape_a (the
    deformation's sine factor vanishes there; sin(pi) in floating point leaves 1e-16)."""
    shape = (2,) * d
    pts = WM.grid_of_patches(shape, 3, 2, amp=0.2)
    for r, pt in enumerate(pts):
        ir = [(r // int(np.prod(shape[:a]))) % shape[a] for a in range(d)]
        net = _net(pt)
        for a in range(d):
            ax = d - 1 - a
            if ir[a] == 0:
                assert np.abs(np.take(net, 0, axis=ax)[..., a]).max() <= 1e-15
            if ir[a] == shape[a] - 1:
                assert np.abs(np.take(net, -1, axis=ax)[..., a] - shape[a]).max() <= 1e-15


@pytest.mark.parametrize("perm,flip", [((1, 0), (0,)), ((0, 1), (0, 1)), ((1, 0), ())])
def test_reorient_is_undone_by_its_inverse(perm, flip):
    pt = WM.grid_of_patches((1, 1), 3, 3, amp=0.1)[0]
    once = WM.reorient(pt, perm, flip)
    inv = [perm.index(b) for b in range(len(perm))]
    back = WM.reorient(once, inv, tuple(b for b in range(len(perm)) if inv[b] in flip))
    assert back[0] == pt[0]
    # a reversed knot vector is a + b - U reversed: twice gives U up to rounding
    assert all(np.allclose(a, b, rtol=0, atol=1e-15) for a, b in zip(back[1], pt[1]))
    assert np.array_equal(back[2], pt[2])  # control points are only permuted
