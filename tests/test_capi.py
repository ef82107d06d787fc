"""CPU-side checks of the C ABI: the library loads, exports every entry point that
include/*.h declares, and its host-only logic (parameters, status strings, argument
validation that fails before any device call) agrees with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
import paper_2102_11536_gb300 as iga
from paper_2102_11536_gb300 import build as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:(?:const|unsigned|signed|long|short)\s+)*\w+\s*\*?\s*(iga_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    gb.build()
    return iga.lib()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 18
    raw = ctypes.CDLL(iga.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(raw, name), name
    assert set(iga.exported_symbols()) <= declared


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("rho", [0.0, 0.25, 0.5, 0.9, 1.0])
def test_params_match_oracle(lib, k, rho):
    a, b, g = iga.galpha_params(k, rho)
    ref = oracle.galpha_params(k, rho)
    for j in range(k):
        assert abs(a[j] - ref[j][0]) < 1e-15
        assert abs(b[j] - ref[j][1]) < 1e-14
        assert abs(g[j] - ref[j][2]) < 1e-15


def test_params_reject_bad_arguments(lib):
    with pytest.raises(iga.IgaError):
        iga.galpha_params(5, 0.5)
    with pytest.raises(iga.IgaError):
        iga.galpha_params(2, 1.5)


def test_status_strings(lib):
    for code in range(8):
        assert lib.iga_status_string(code)


def test_create_rejects_bad_knots_before_device_use(lib):
    # open knot vectors are required; the check happens on the host
    bad = [np.array([0, 0.1, 0.5, 1, 1, 1.0]), np.array([0, 0, 0, 1, 1, 1.0])]
    with pytest.raises(iga.IgaError) as e:
        iga.Patch([2, 2], bad, np.zeros((9, 2)))
    assert e.value.status == iga.EINVAL
    with pytest.raises(iga.IgaError) as e:
        iga.Patch([9, 2], [np.zeros(20), np.zeros(6)], np.zeros((9, 2)))
    assert e.value.status == iga.EINVAL


def test_network_entry_points_validate_before_any_device_work(lib):
    assert lib.iga_net_forward(0, 4, 4, 1, None, None, None, None, None) == iga.EINVAL
    assert lib.iga_net_forward(4, 4, 4, 0, 1, 1, 1, 1, None) == iga.EINVAL
    assert lib.iga_net_forward(4, 4, 4, 1, None, 1, 1, 1, None) == iga.EINVAL
    assert lib.iga_net_workspace_bytes(0, 1, 1, 1) == 0
    # dh [nb][16][N] floats plus per-block partials (1312 + 433 floats per 16x16x4 tile)
    n1, n2, n3 = 19, 21, 9
    blocks = 2 * 2 * 3
    assert lib.iga_net_workspace_bytes(n1, n2, n3, 1) == 4 * (16 * n1 * n2 * n3 + blocks * (1312 + 433))
    assert lib.iga_net_backward(4, 4, 4, 1, 1, 1, 1, 1, 1, 1, 10, None) == iga.EINVAL  # work too small
    assert lib.iga_net_adam(0, 1, 1, 1, 1, 1, 1e-3, None) == iga.EINVAL
    assert lib.iga_net_adam(8, 1, 1, 1, 1, 0, 1e-3, None) == iga.EINVAL
    assert lib.iga_net_adam(8, 1, 1, 1, 1, 1, 0.0, None) == iga.EINVAL
    assert iga.GUESSES["learned"] == 4 and iga.NET_NPARAM == 1745


def test_tuning_and_batch_entry_points_validate(lib):
    out = ctypes.c_void_p()
    assert lib.iga_batch_create(0, None, ctypes.byref(out)) == iga.EINVAL
    assert lib.iga_batch_create(1, None, ctypes.byref(out)) == iga.EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.iga_batch_create(1, arr, ctypes.byref(out)) == iga.EINVAL
    assert lib.iga_batch_step(None, None, 2, 0.5, None, 1, None) == iga.EINVAL
    assert lib.iga_batch_last_error(None) == b""
    assert lib.iga_set_band_config(None, 256, 2) == iga.EINVAL
    assert lib.iga_autotune(None, 2, 3, None, None) == iga.EINVAL
    assert lib.iga_band_df_tiny(None, None, None) == iga.EINVAL


def test_create_rejects_patches_without_interior_dofs(lib):
    # one linear element per direction: 2 basis functions, both carry the Dirichlet condition
    k1 = np.array([0, 0, 1, 1.0])
    with pytest.raises(iga.IgaError) as e:
        iga.Patch([1, 1, 1], [k1, k1, k1], np.zeros((8, 3)))
    assert e.value.status == iga.EINVAL


def test_every_declared_entry_point_is_documented():
    """Each entry point in include/*.h comes right after a comment block (argument meaning,
    layout, ownership, errors and the passage it follows); a group of related calls may
    share one block."""
    for hdr in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        lines = open(hdr).read().split("\n")
        last_end = -100
        for i, line in enumerate(lines):
            if "*/" in line:
                last_end = i
            m = re.match(r"^\s*(?:(?:const|unsigned|signed|long|short)\s+)*\w+\s*\*?\s*(iga_\w+)\s*\(", line)
            if m:
                assert i - last_end <= 8, (os.path.basename(hdr), m.group(1))


def test_binding_declares_argument_types_for_every_call():
    """Every entry point the headers declare, and every one the binding calls, has ctypes
    argument and result types in the binding (an undeclared call would pass 64-bit pointers
    as C ints)."""
    src = open(os.path.join(ROOT, "paper_2102_11536_gb300", "__init__.py")).read()
    typed = set(re.findall(r'"(iga_\w+)": \(', src))
    called = set(re.findall(r"\.(iga_\w+)\(", src))
    assert _declared() <= typed, sorted(_declared() - typed)
    assert called <= typed, sorted(called - typed)
