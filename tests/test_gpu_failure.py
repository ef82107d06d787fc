"""Failure detection on the device without a GPU fault.

The double-FP32 band product splits its input vectors in one cooperative launch
whose blocks meet at a grid barrier with a bounded wait. Here the wait is made to
run out (a poll limit of 0: a block that has to wait gives up at once), and the
test checks what a caller sees: the kernel ends, the next checked call returns
IGA_ECUDA with a message, the error word and the barrier's words are reset by that
report, and the calls after it give the same products, bit for bit, as before.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_grid_barrier_timeout_is_reported_then_cleared():
    # N = 67 * 51 * 43 = 146 931: the split runs on 2 blocks per SM, all of which meet
    w = W.small(d=3, nel=(64, 48, 40), p=3, amp=0.1)
    g = iga.Patch(w.p, w.knots, w.ctrl(), op_form="assembled_df", precond="banded32", tol=1e-10)
    g.assemble()
    nvec = 2
    gen = torch.Generator(DEV).manual_seed(11)
    x = torch.randn(nvec * g.N, dtype=torch.float64, device=DEV, generator=gen)
    ref = torch.empty_like(x)
    z = torch.empty_like(x)
    g.apply_M(x, ref, nvec)  # the product at the default limit
    assert iga.lib().iga_apply_Pinv(g.h, nvec, _ptr(x), _ptr(z)) == iga.OK
    torch.cuda.synchronize()

    g.set_barrier_limit(0)
    y = torch.empty_like(x)
    status, msg = iga.OK, b""
    for _ in range(20):  # the first arriving block has to wait: one product suffices in practice
        g.apply_M(x, y, nvec)  # asynchronous; a time-out is recorded on the device
        status = iga.lib().iga_apply_Pinv(g.h, nvec, _ptr(x), _ptr(z))  # a checked call reports it
        if status != iga.OK:
            msg = iga.lib().iga_last_error(g.h)
            break
    assert status == iga.ECUDA, status
    assert b"timed out" in msg and b"grid" in msg, msg
    torch.cuda.synchronize()  # the context is still usable

    # the report cleared the error word and reset the barrier: normal calls succeed again
    g.set_barrier_limit(-1)
    y.zero_()
    g.apply_M(x, y, nvec)
    assert iga.lib().iga_apply_Pinv(g.h, nvec, _ptr(x), _ptr(z)) == iga.OK
    assert np.array_equal(y.cpu().numpy(), ref.cpu().numpy())
    # and a PCG solve, whose every iteration passes the barrier, converges
    xs = torch.zeros_like(x)
    its, rel = g.solve_M(ref, xs, nvec)
    assert max(rel) <= 1e-10
    assert np.abs(xs.cpu().numpy() - x.cpu().numpy()).max() <= 1e-4 * np.abs(x.cpu().numpy()).max()
    g.close()
