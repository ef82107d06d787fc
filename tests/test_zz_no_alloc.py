"""iga_apply_Pinv_noalloc: the preconditioner entry point for callers that cannot
allocate device memory while they run (their memory is committed to another
allocator's pool, or their loop forbids allocation after start-up).

It is called here through the C ABI (ctypes) and must return what the regular
iga_apply_Pinv returns, bit for bit (same kernels, same launch shapes, only the
intermediate buffers differ), on two calls in a row, in every preconditioner
arithmetic, without taking device memory after its first call on the device --
also on a handle whose own intermediate buffers were never made -- and must
refuse sizes beyond its fixed scratch. This file is collected last so that a run
stopping at the first failure has run every other test already; it also passes
alone in a fresh process.
"""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FORMS = ["fp64", "fp32", "banded", "banded32", "bf16", "fp16"]


def _noalloc(h, nvec, x, y):
    return iga.lib().iga_apply_Pinv_noalloc(h, nvec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _idle_noise():
    """How much the device's free memory moves on its own over a short idle period
    (another process on the device); 0 on a device of one's own."""
    a = _free_bytes()
    time.sleep(0.2)
    b = _free_bytes()
    return abs(a - b)


def _patch(precond):
    w = W.small(d=3, nel=(11, 9, 13), p=3, amp=0.1)
    return iga.Patch(w.p, w.knots, w.ctrl(), precond=precond)


@pytest.mark.parametrize("precond", FORMS)
def test_noalloc_matches_apply_pinv_twice(precond):
    # device set-up (symbol address, the form's kernels loaded) on a throw-away handle
    g0 = _patch(precond)
    x0 = torch.ones(g0.N, dtype=torch.float64, device=DEV)
    y0 = torch.empty_like(x0)
    assert _noalloc(g0.h, 1, x0, y0) == iga.OK
    g0.close()
    # a fresh handle: its own intermediate buffers have never been made
    g = _patch(precond)
    nvec = 3
    gen = torch.Generator(DEV).manual_seed(4)
    x = torch.randn(nvec * g.N, dtype=torch.float64, device=DEV, generator=gen)
    out = torch.full_like(x, float("nan"))
    noise = _idle_noise()
    free_before = _free_bytes()
    results = []
    for _ in range(2):  # two calls in a row on the shared scratch
        out.fill_(float("nan"))
        assert _noalloc(g.h, nvec, x, out) == iga.OK
        torch.cuda.synchronize()
        results.append(out.cpu().numpy())
    assert free_before - _free_bytes() <= noise, "the no-allocation entry point took device memory"
    ref = torch.empty_like(x)
    g.apply_Pinv(x, ref, nvec)  # the existing entry point (grows the handle's buffers)
    ref_h = ref.cpu().numpy()
    assert np.all(np.isfinite(ref_h))
    for r in results:
        assert np.array_equal(r, ref_h), "max abs difference %g" % np.abs(r - ref_h).max()
    g.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    w = W.Workload("t", 2, (400, 400), (2, 2), 0.0, 1, 0.5, 1)  # N = 160000
    g = iga.Patch(w.p, w.knots, w.ctrl())
    nvec = 7  # 7 * 160000 > 1048576
    x = torch.ones(nvec * g.N, dtype=torch.float64, device=DEV)
    y = torch.zeros_like(x)
    assert _noalloc(g.h, nvec, x, y) == iga.EINVAL
    assert b"exceeds" in iga.lib().iga_last_error(g.h)
    assert float(y.abs().max()) == 0.0
    assert _noalloc(g.h, 6, x, y) == iga.OK  # 6 * 160000 fits
    g.close()
