"""iga_apply_Pinv_noalloc: the preconditioner entry point for callers that cannot
allocate device memory while they run (their memory is committed to another
allocator's pool, or their loop forbids allocation after start-up).

It is called here through the C ABI (ctypes) and must return what the regular
iga_apply_Pinv returns, on two calls in a row, within the operator tolerance of
the parity tests (1e-12 relative), without taking device memory after its first
call on the device, and must refuse sizes beyond its fixed scratch. This file
is collected last so that a run stopping at the first failure has run every
other test already; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _noalloc(h, nvec, x, y):
    return iga.lib().iga_apply_Pinv_noalloc(h, nvec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))


@pytest.mark.parametrize("precond", ["fp64", "fp32"])
def test_noalloc_matches_apply_pinv_twice(precond):
    w = W.small(d=3, nel=(11, 9, 13), p=3, amp=0.1)
    g = iga.Patch(w.p, w.knots, w.ctrl(), precond=precond)
    nvec = 2
    gen = torch.Generator(DEV).manual_seed(4)
    x = torch.randn(nvec * g.N, dtype=torch.float64, device=DEV, generator=gen)
    ref = torch.empty_like(x)
    g.apply_Pinv(x, ref, nvec)  # the existing entry point
    ref_h = ref.cpu().numpy()
    out = torch.full_like(x, float("nan"))
    assert _noalloc(g.h, nvec, x, out) == iga.OK  # first call on the device: set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    results = []
    for _ in range(2):  # two calls in a row on the shared scratch
        out.fill_(float("nan"))
        assert _noalloc(g.h, nvec, x, out) == iga.OK
        torch.cuda.synchronize()
        results.append(out.cpu().numpy())
    assert torch.cuda.mem_get_info()[0] == free_before
    for r in results:
        assert np.all(np.isfinite(r))
        assert np.abs(r - ref_h).max() <= 1e-12 * np.abs(ref_h).max()
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
