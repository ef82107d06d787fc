"""The library's univariate tables (host_setup.cpp, compiled here with the host compiler)
over function boxes: the parametric mass matrix of the box equals the oracle's univariate
mass matrix restricted to the box (def:matrices_1 in one direction, over the box of a
patch in a multi-patch system, Sec. 5.4), the operators' window start is the box index
of each point's first function plus one, and each function's quadrature range is where
it is nonzero. The interior box 1..m-2 is the single-patch case."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_11536_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "cuda.h")):
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path_factory.mktemp("host") / "box_tables")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + cuda_inc, "-I" + CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "host", "box_tables.cpp"), os.path.join(CSRC, "host_setup.cpp")],
                   check=True, capture_output=True)
    return exe


def _run(exe, p, lo, hi, knots, nq=None):
    out = subprocess.run([exe, str(p), str(lo), str(hi), str(nq or p + 1)] + ["%.17g" % k for k in knots],
                         capture_output=True, text=True)
    lines = out.stdout.split("\n")
    if lines[0].startswith("ERR"):
        return lines[0]
    n, Q, m, lo_t = map(int, lines[0].split())
    mh = np.array([float(v) for v in lines[1:1 + n * n]]).reshape(n, n)
    fl = np.array([[int(v) for v in s.split()] for s in lines[1 + n * n:1 + n * n + n]])
    qq = np.array([[int(v) for v in s.split()] for s in lines[1 + n * n + n:1 + n * n + n + Q]])
    return n, m, lo_t, mh, fl, qq


KNOTS = {
    "uniform": lambda p: np.array([0.0] * (p + 1) + [i / 5 for i in range(1, 5)] + [1.0] * (p + 1)),
    "graded": lambda p: np.array([0.0] * (p + 1) + [0.05, 0.2, 0.45, 0.8] + [1.0] * (p + 1)),
    "repeated": lambda p: np.array([0.0] * (p + 1) + [0.3] * p + [0.7] + [1.0] * (p + 1)),
    "one_element": lambda p: np.array([0.0] * (p + 1) + [1.0] * (p + 1)),
}


@pytest.mark.parametrize("kind", sorted(KNOTS))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_box_tables_match_the_oracle(driver, kind, p):
    kn = KNOTS[kind](p)
    m = len(kn) - p - 1
    q = oracle.Quad1D(p, kn, p + 1)
    B = q.dense()
    Mfull = B.T @ (q.qw[:, None] * B)
    for lo, hi in [(0, m - 1), (0, m - 2), (1, m - 1), (1, m - 2)]:
        if hi < lo or (lo, hi) == (1, m - 2) and m < 3:
            continue
        res = _run(driver, p, lo, hi, kn)
        assert not isinstance(res, str), res
        n, mm, lo_t, mh, fl, qq = res
        assert (n, mm, lo_t) == (hi - lo + 1, m, lo)
        ref = Mfull[lo:hi + 1, lo:hi + 1]
        assert np.abs(mh - ref).max() <= 1e-14 * np.abs(ref).max()
        assert np.array_equal(qq[:, 1], qq[:, 0] - lo + 1)
        for i in range(n):
            support = [k for k in range(len(qq)) if qq[k, 0] <= i + lo <= qq[k, 0] + p]
            assert (fl[i, 0], fl[i, 1]) == (support[0], support[-1] + 1)


def test_interior_box_is_the_default(driver):
    kn = KNOTS["graded"](3)
    a = _run(driver, 3, 1, -1, kn)
    b = _run(driver, 3, 1, len(kn) - 3 - 1 - 2, kn)
    assert a[0] == b[0] and np.array_equal(a[3], b[3]) and np.array_equal(a[5], b[5])
    q = oracle.Quad1D(3, kn, 4)
    assert np.abs(a[3] - q.mass_interior()).max() <= 1e-14 * np.abs(a[3]).max()


@pytest.mark.parametrize("lo,hi", [(-1, 3), (0, 9), (3, 2)])
def test_bad_boxes_are_rejected(driver, lo, hi):
    res = _run(driver, 2, lo, hi, KNOTS["uniform"](2))
    assert isinstance(res, str) and res.startswith("ERR")
