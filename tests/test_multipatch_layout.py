"""The library's gluing of conforming patches (iga_mp_layout, host only; Sec. 5.1,
def:mp_basis, def:N_patch) against the multi-patch oracle: the same index boxes, global
numbering, number of functions and N_adj on rows, grids, an L and patches with renamed or
reversed directions; and its rejection of non-conforming input."""
import numpy as np
import pytest

import paper_2102_11536_gb300 as iga
from oracle import multipatch as mp
from workloads import multipatch as WM


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2102_11536_gb300 import build as gb
    gb.build()


def _oracle_boxes(g):
    out = []
    for loc in g.local:
        box = np.full(loc["mask"].size, -1, dtype=np.int64)
        box[loc["mask"]] = loc["ids"]
        out.append(box.reshape(list(reversed(loc["n"]))))
    return out


LAYOUTS = {
    "single": lambda: WM.grid_of_patches((1, 1), 4, 2, amp=0.1),
    "row3": lambda: WM.row_of_patches(3, 3, 3, amp=0.1),
    "grid2x2": lambda: WM.grid_of_patches((2, 2), 3, 2, amp=0.1),
    "grid3x2": lambda: WM.grid_of_patches((3, 2), 2, 3, amp=0.05),
    "L": lambda: WM.l_shape(3, 2, amp=0.1),
    "L_p1": lambda: WM.l_shape(2, 1),
    "grid2x2x2": lambda: WM.grid_of_patches((2, 2, 2), 2, 2, amp=0.1),
    "row3d": lambda: WM.grid_of_patches((1, 1, 3), 2, 3, amp=0.1),
    "reoriented2d": lambda: [WM.reorient(pt, *o) for pt, o in zip(WM.grid_of_patches((2, 2), 3, 2, amp=0.1),
                                                                    [((0, 1), ()), ((1, 0), (0,)), ((0, 1), (0, 1)),
                                                                     ((1, 0), ())])],
    "reorientedL": lambda: [WM.reorient(pt, *o) for pt, o in zip(WM.l_shape(3, 3, amp=0.1),
                                                                   [((1, 0), (1,)), ((0, 1), (0,)), ((1, 0), (0, 1))])],
    "reoriented3d": lambda: [WM.reorient(pt, *o) for pt, o in zip(WM.grid_of_patches((2, 2, 1), 2, 2, amp=0.1),
                                                                    [((0, 1, 2), ()), ((2, 0, 1), (1,)),
                                                                     ((1, 2, 0), (0, 2)), ((0, 2, 1), (0, 1, 2))])],
}


@pytest.mark.parametrize("name", sorted(LAYOUTS))
def test_layout_matches_the_oracle(name):
    patches = LAYOUTS[name]()
    g = mp.GluedPatches(patches)
    lay = iga.multipatch_layout(patches)
    assert lay["nglob"] == g.N
    assert lay["n_adj"] == g.n_adj
    for r, loc in enumerate(g.local):
        assert lay["lo"][r].tolist() == list(loc["lo"])
        assert (lay["hi"][r] - lay["lo"][r] + 1).tolist() == list(loc["n"])
    for a, b in zip(lay["gid"], _oracle_boxes(g)):
        assert a.shape == b.shape
        assert np.array_equal(a, b)


def test_re_entrant_corner_function_is_not_a_degree_of_freedom():
    lay = iga.multipatch_layout(WM.l_shape(3, 2))
    # patch 0 ([0, 1]^2) has interfaces on both of its upper faces: its box reaches the
    # corner (1, 1), which lies on the boundary of the L
    assert lay["gid"][0][-1, -1] == -1
    assert (lay["gid"][0] >= 0).sum() == lay["gid"][0].size - 1
    assert lay["n_adj"] == 2


def test_n_adj_counts_the_patches_at_a_vertex():
    assert iga.multipatch_layout(WM.grid_of_patches((2, 2), 2, 2))["n_adj"] == 4
    assert iga.multipatch_layout(WM.grid_of_patches((2, 2, 2), 2, 2))["n_adj"] == 8
    assert iga.multipatch_layout(WM.grid_of_patches((3, 1), 2, 2))["n_adj"] == 2


def test_tolerance_identifies_nearly_equal_control_points():
    patches = WM.row_of_patches(2, 3, 2, amp=0.1)
    deg, kn, ctrl = patches[1]
    patches[1] = (deg, kn, ctrl + 1e-13)
    assert iga.multipatch_layout(patches)["n_adj"] == 2
    patches[1] = (deg, kn, ctrl + 1e-6)
    lay = iga.multipatch_layout(patches)
    assert lay["n_adj"] == 1  # no interface: two separate clamped patches
    assert iga.multipatch_layout(patches, tol=1e-5)["n_adj"] == 2


def test_non_conforming_knots_are_rejected():
    patches = WM.row_of_patches(2, 3, 2, amp=0.0)
    deg, kn, ctrl = patches[1]
    kn2 = [kn[0], np.array([0, 0, 0, 0.25, 2 / 3, 1, 1, 1.0])]  # same count, other interior knots
    patches[1] = (deg, kn2, ctrl)
    with pytest.raises(iga.IgaError) as e:
        iga.multipatch_layout(patches)
    assert e.value.status == iga.EINVAL and "not conforming" in str(e.value)


def test_a_non_matching_interface_is_rejected():
    """Two patches that share a face region but not its control points (the right one
    refined): a non-conforming interface, not two Dirichlet faces."""
    left = WM.row_of_patches(2, 3, 2, amp=0.0)[0]
    right = WM.row_of_patches(2, 4, 2, amp=0.0)[1]
    with pytest.raises(iga.IgaError) as e:
        iga.multipatch_layout([left, right])
    assert e.value.status == iga.EINVAL and "not conforming" in str(e.value)


def test_a_face_shared_by_three_patches_is_rejected():
    patches = WM.row_of_patches(2, 2, 2, amp=0.0)
    with pytest.raises(iga.IgaError) as e:
        iga.multipatch_layout(patches + [patches[1]])
    assert "more than one other face" in str(e.value)


@pytest.mark.parametrize("bad", ["degree", "knots", "open", "nan"])
def test_bad_arguments_are_rejected(bad):
    patches = WM.row_of_patches(2, 2, 2, amp=0.0)
    deg, kn, ctrl = patches[0]
    if bad == "degree":
        patches[0] = ((7, 2), kn, ctrl)
    elif bad == "knots":
        patches[0] = (deg, [kn[0][::-1], kn[1]], ctrl)
    elif bad == "open":
        patches[0] = (deg, [np.array([0, 0, 0.1, 0.5, 1, 1, 1.0]), kn[1]], ctrl[:16])
    else:
        c = ctrl.copy()
        c[3, 0] = np.nan
        patches[0] = (deg, kn, c)
    with pytest.raises(iga.IgaError) as e:
        iga.multipatch_layout(patches)
    assert e.value.status == iga.EINVAL


# iga_mp_create checks its arguments and the gluing before it touches a device, so its
# refusals are host logic.

def test_multipatch_handle_refuses_the_learned_guess():
    with pytest.raises(iga.IgaError) as e:
        iga.MultiPatch(WM.row_of_patches(2, 2, 2), guess="learned", stream=None)
    assert e.value.status == iga.EINVAL and "learned" in str(e.value)


def test_multipatch_handle_refuses_non_conforming_patches():
    patches = WM.row_of_patches(2, 3, 2)
    deg, kn, ctrl = patches[1]
    patches[1] = (deg, [kn[0], np.array([0, 0, 0, 0.25, 2 / 3, 1, 1, 1.0])], ctrl)
    with pytest.raises(iga.IgaError) as e:
        iga.MultiPatch(patches, stream=None)
    assert e.value.status == iga.EINVAL and "not conforming" in str(e.value)


def test_multipatch_info_refuses_a_null_handle():
    assert iga.lib().iga_mp_info(None, None, None, None) == iga.EINVAL


def test_multipatch_handle_without_a_device_fails_cleanly():
    """On a machine without a GPU the gluing succeeds and the device set-up fails with
    IGA_ECUDA; the partly built system is released without touching a device."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the handle would be created")
    with pytest.raises(iga.IgaError) as e:
        iga.MultiPatch(WM.l_shape(3, 2, amp=0.1), stream=None)
    assert e.value.status == iga.ECUDA
