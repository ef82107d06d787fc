"""The persistent batch step (iga_batch_set_persistent): one cooperative launch per
step advances every patch of a batch of independent, uneven patches (FP64 band
operators; band-Cholesky Kronecker or BF16 fast-diagonalisation preconditioner).

  * three small patches of degrees 2, 3, 4 at PCG tol 1e-13: every patch after 6 steps
    within 1e-10 (relative L2 of U and V) of the oracle's Stepper on the same inputs,
    and of the patch stepped alone through the library; the same for k = 1 and k = 3;
  * the FP32 Kronecker solve (flexible PCG) at tol 1e-10: within 1e-8 of the same patches
    stepped alone with it;
  * the 48-patch batch (16^3..96^3 elements, p in {2, 3, 4}) for 3 steps: every patch
    within 1e-8 of that patch stepped alone, one launch per batch step;
  * the BF16 fast diagonalisation (flexible PCG) at tol 1e-10: within 1e-8 of the oracle
    and of the patches stepped alone with the tensor-core BF16 preconditioner;
  * a second persistent run equals the first bit for bit (fixed-order reductions);
  * the launch variants (three blocks per SM and two slots per band pass, or two blocks and
    four slots) give bitwise the same states, and the automatic choice times both;
  * the phase clock (iga_batch_phase_times): the products and the preconditioner are timed,
    the times add up to no more than the call, and a batch without a persistent step has none;
  * refusals: a form the persistent step does not compute gives IGA_EINVAL and the batch
    keeps its graph path.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _small_patches():
    out = []
    for r, (nel, p, amp) in enumerate([((5, 4, 6), 2, (0.1, 0.05, 0.12)), ((4, 5, 3), 3, (0.08, 0.1, 0.02)),
                                       ((3, 4, 4), 4, (0.05, 0.1, 0.1))]):
        w = W.Workload("pb%d" % r, 3, nel, (p, p, p), 0.0, 2, 0.5, 6, init="random", seed=r)
        w.amp = amp
        out.append(w)
    return out


def _setup(ws, precond, tol):
    pats, states, inits = [], [], []
    for w in ws:
        g = iga.Patch(w.p, w.knots, w.ctrl(), tol=tol, op_form="assembled", precond=precond)
        U0, V0 = w.initial()
        pats.append(g)
        inits.append((_t(U0), _t(V0)))
        states.append(torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV))
    return pats, states, inits


def test_persistent_batch_matches_oracle_and_patches_alone():
    ws = _small_patches()
    k, rho, nsteps = 2, 0.5, 6
    pats, states, inits = _setup(ws, "banded", 1e-13)
    dts = []
    refs = []
    for w in ws:
        ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
        lam = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
        dt = 0.5 * math.sqrt(oracle.theta_crit(rho) / lam)
        st = oracle.Stepper(ops, k, rho, tol=1e-13)
        U0, V0 = w.initial()
        X = st.init(U0, V0)
        for _ in range(nsteps):
            X = st.step(X, dt)
        dts.append(dt)
        refs.append(X)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    with pytest.raises(iga.IgaError) as e:  # no persistent step yet
        b.phase_times()
    assert e.value.status == iga.EINVAL
    b.set_persistent(True)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    stats = b.step(states, k, rho, dts, nsteps)
    t1.record()
    t1.synchronize()
    assert stats[0].launches == nsteps  # one launch per batch step
    # the device-side phase clock: every kind of phase ran, and the phases add up to the call
    ph = b.phase_times()
    total = sum(ph.values())
    print("persistent batch phases (ms over %d steps): %s; call %.3f ms" % (
        nsteps, ", ".join("%s %.3f" % kv for kv in ph.items()), t0.elapsed_time(t1)))
    assert all(v >= 0.0 for v in ph.values()) and ph["M product"] > 0.0 and ph["preconditioner"] > 0.0, ph
    assert total <= t0.elapsed_time(t1) * 1.01 + 0.05
    batched = [s.cpu().numpy().reshape(3 * k, -1) for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        assert stats[i].steps == nsteps and stats[i].solves == k * nsteps and stats[i].max_relres <= 1e-13
        g.state_init(k, u0, v0, st)
        g.step(st, k, rho, dt, nsteps)
        alone = st.cpu().numpy().reshape(3 * k, -1)
        for row, var in ((0, "U"), (1, "V")):
            e_o = _rel(batched[i][row], refs[i][row])
            e_a = _rel(batched[i][row], alone[row])
            print("persistent batch, patch %d (p=%d), %s: vs oracle %.3e, vs alone %.3e" % (i, ws[i].p[0], var, e_o, e_a))
            assert e_o <= 1e-10 and e_a <= 1e-10, (i, var, e_o, e_a)
    b.close()
    for g in pats:
        g.close()


@pytest.mark.parametrize("k", [1, 3])
def test_persistent_batch_other_orders_match_oracle(k):
    """The persistent step for k = 1 (second order) and k = 3 (sixth order): every patch
    within 1e-10 of the oracle's Stepper and of the patch stepped alone (FP64 Kronecker
    solve, tol 1e-13)."""
    ws = _small_patches()
    rho, nsteps = 0.5, 4
    pats, states, inits = [], [], []
    for w in ws:
        g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-13, op_form="assembled", precond="banded")
        U0, V0 = w.initial()
        pats.append(g)
        inits.append((_t(U0), _t(V0)))
        states.append(torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV))
    dts, refs = [], []
    for w in ws:
        ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
        lam = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
        dt = 0.5 * math.sqrt(oracle.theta_crit(rho) / lam)
        st = oracle.Stepper(ops, k, rho, tol=1e-13)
        U0, V0 = w.initial()
        X = st.init(U0, V0)
        for _ in range(nsteps):
            X = st.step(X, dt)
        dts.append(dt)
        refs.append(X)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    b.set_persistent(True)
    stats = b.step(states, k, rho, dts, nsteps)
    assert stats[0].launches == nsteps
    batched = [s.cpu().numpy().reshape(3 * k, -1) for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        assert stats[i].solves == k * nsteps and stats[i].max_relres <= 1e-13
        g.state_init(k, u0, v0, st)
        g.step(st, k, rho, dt, nsteps)
        alone = st.cpu().numpy().reshape(3 * k, -1)
        for row, var in ((0, "U"), (1, "V")):
            e_o = _rel(batched[i][row], refs[i][row])
            e_a = _rel(batched[i][row], alone[row])
            print("persistent batch k=%d, patch %d, %s: vs oracle %.3e, vs alone %.3e" % (k, i, var, e_o, e_a))
            assert e_o <= 1e-10 and e_a <= 1e-10, (k, i, var, e_o, e_a)
    b.close()
    for g in pats:
        g.close()


def test_persistent_batch_fp32_kronecker_and_reproducibility():
    ws = _small_patches()
    k, rho, nsteps = 2, 0.5, 5
    pats, states, inits = _setup(ws, "banded32", 1e-10)
    dts = []
    for g in pats:
        lam, tc = g.cfl(rho, iters=60)
        dts.append(0.5 * tc)
    b = iga.Batch(pats)
    b.set_persistent(True)
    runs = []
    for _ in range(2):
        for g, st, (u0, v0) in zip(pats, states, inits):
            g.state_init(k, u0, v0, st)
        stats = b.step(states, k, rho, dts, nsteps)
        assert all(s.max_relres <= 1e-10 for s in stats)
        runs.append([s.cpu().numpy().reshape(3 * k, -1) for s in states])
    for i in range(len(pats)):
        assert np.array_equal(runs[0][i], runs[1][i]), i
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.state_init(k, u0, v0, st)
        g.step(st, k, rho, dt, nsteps)
        alone = st.cpu().numpy().reshape(3 * k, -1)
        for row in (0, 1):
            assert _rel(runs[0][i][row], alone[row]) <= 1e-8, (i, row)
    b.close()
    for g in pats:
        g.close()


def test_persistent_batch_of_48_patches():
    ws = W.multipatch_batch()
    k, rho, nsteps = 2, 0.5, 3
    pats, states, dts, inits = [], [], [], []
    for w in ws:
        g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-10, op_form="assembled", precond="banded32")
        lam, tc = g.cfl(rho, iters=20)
        U0, V0 = w.initial()
        pats.append(g)
        dts.append(0.5 * tc)
        inits.append((_t(U0), _t(V0)))
        states.append(torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV))
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    b.set_persistent(True)
    stats = b.step(states, k, rho, dts, nsteps)
    assert stats[0].launches == nsteps
    assert all(s.max_relres <= 1e-10 for s in stats)
    batched = [s.cpu().numpy() for s in states]
    worst = 0.0
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.state_init(k, u0, v0, st)
        g.step(st, k, rho, dt, nsteps)
        alone = st.cpu().numpy().reshape(3 * k, -1)
        bt = batched[i].reshape(3 * k, -1)
        for row in (0, 1):
            e = _rel(bt[row], alone[row])
            worst = max(worst, e)
            assert e <= 1e-8, (i, row, e)
    print("48-patch persistent batch: largest relative L2 difference to the patches stepped alone %.3e" % worst)
    b.close()
    for g in pats:
        g.close()


def test_persistent_batch_bf16_fast_diagonalisation():
    ws = _small_patches()
    k, rho, nsteps = 2, 0.5, 5
    pats, states, inits = _setup(ws, "bf16", 1e-10)
    dts, refs = [], []
    for w in ws:
        ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
        lam = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
        dt = 0.5 * math.sqrt(oracle.theta_crit(rho) / lam)
        st = oracle.Stepper(ops, k, rho, tol=1e-13)
        U0, V0 = w.initial()
        X = st.init(U0, V0)
        for _ in range(nsteps):
            X = st.step(X, dt)
        dts.append(dt)
        refs.append(X)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    b.set_persistent(True)
    stats = b.step(states, k, rho, dts, nsteps)
    assert all(s.max_relres <= 1e-10 for s in stats)
    batched = [s.cpu().numpy().reshape(3 * k, -1) for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.state_init(k, u0, v0, st)
        sa = g.step(st, k, rho, dt, nsteps)
        alone = st.cpu().numpy().reshape(3 * k, -1)
        print("persistent BF16 batch, patch %d: %.2f iterations per solve (tensor-core form alone: %.2f)" % (
            i, stats[i].iters / stats[i].solves, sa.iters / sa.solves))
        for row, var in ((0, "U"), (1, "V")):
            e_o = _rel(batched[i][row], refs[i][row])
            e_a = _rel(batched[i][row], alone[row])
            print("  %s: vs oracle %.3e, vs alone %.3e" % (var, e_o, e_a))
            assert e_o <= 1e-8 and e_a <= 1e-8, (i, var, e_o, e_a)
    b.close()
    for g in pats:
        g.close()


def test_persistent_variants_agree_bitwise_and_are_timed():
    ws = _small_patches()
    k, rho, nsteps = 2, 0.5, 4
    pats, states, inits = _setup(ws, "banded", 1e-12)
    dts = [0.5 * g.cfl(rho, iters=60)[1] for g in pats]
    b = iga.Batch(pats)
    b.set_persistent(True)
    runs = []
    for v in (0, 1):
        b.set_persistent_variant(v)
        for g, st, (u0, v0) in zip(pats, states, inits):
            g.state_init(k, u0, v0, st)
        stats = b.step(states, k, rho, dts, nsteps)
        assert stats[0].launches == nsteps
        assert b.persistent_variant()[0] == v
        runs.append([s.cpu().numpy() for s in states])
    for i in range(len(pats)):
        assert np.array_equal(runs[0][i], runs[1][i]), i
    # the automatic choice: each variant timed twice over the first single steps
    b.set_persistent_variant(-1)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    for _ in range(4):
        b.step(states, k, rho, dts, 1)
    v, ms = b.persistent_variant()
    print("persistent variants: chosen %d, fastest step %.3f / %.3f ms" % (v, ms[0], ms[1]))
    assert v in (0, 1) and ms[0] > 0.0 and ms[1] > 0.0 and ms[v] == min(ms)
    for i, st in enumerate(states):  # the steps taken while timing are the same steps
        assert np.array_equal(st.cpu().numpy(), runs[0][i]), i
    with pytest.raises(iga.IgaError) as e:
        b.set_persistent_variant(2)
    assert e.value.status == iga.EINVAL
    b.close()
    for g in pats:
        g.close()


def test_persistent_batch_refuses_other_forms():
    ws = _small_patches()
    pats, states, inits = _setup(ws, "fp32", 1e-10)
    b = iga.Batch(pats)
    with pytest.raises(iga.IgaError) as e:
        b.set_persistent(True)
    assert e.value.status == iga.EINVAL and "preconditioner" in str(e.value)
    b.close()
    for g in pats:
        g.close()
