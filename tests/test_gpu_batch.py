"""Batches of independent patches (one graph launch per batch step) and the band
product's launch configurations: every configuration gives bitwise the same
products, a batch step gives bitwise what stepping each patch alone gives, and the
batched patches match the FP64 oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _uneven(npatch=4, seed=3):
    """Small uneven 3-D patches: sizes, degrees 2..4 and deformations differ."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(npatch):
        nel = tuple(int(v) for v in rng.integers(3, 8, size=3))
        p = int((2, 3, 4)[r % 3])
        w = W.Workload("b%d" % r, 3, nel, (p, p, p), 0.0, 2, 0.5, 6, init="random", seed=r)
        w.amp = tuple(float(v) for v in rng.uniform(0.02, 0.15, size=3))
        out.append(w)
    return out


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("nv", [1, 2, 3, 4])
def test_band_configs_are_bitwise_equal(threads, nv):
    w = W.small(d=3, nel=(9, 7, 6), p=3, amp=0.1)
    g = iga.Patch(w.p, w.knots, w.ctrl(), op_form="assembled")
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(5 * g.N)).to(DEV)
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    g.apply_M(x, y0, nvec=5)
    g.set_band_config(threads, nv)
    g.apply_M(x, y1, nvec=5)
    assert torch.equal(y0, y1)
    g.apply_K(x, y0, nvec=5)
    g.set_band_config(0, 0)
    g.apply_K(x, y1, nvec=5)
    assert torch.equal(y0, y1)
    g.close()


def test_autotune_picks_a_candidate_and_keeps_results():
    w = W.small(d=3, nel=(12, 10, 9), p=2, amp=0.1)
    g = iga.Patch(w.p, w.knots, w.ctrl(), op_form="assembled")
    x = torch.from_numpy(np.random.default_rng(2).standard_normal(2 * g.N)).to(DEV)
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    g.apply_M(x, y0, nvec=2)
    t, v = g.autotune(nvec=2, reps=3)
    assert t in (64, 128, 256, 512) and v in (1, 2)
    g.apply_M(x, y1, nvec=2)
    assert torch.equal(y0, y1)
    with pytest.raises(iga.IgaError):
        g.set_band_config(100, 1)
    g.close()


def _setup(ws, **opts):
    pats, states, dts, inits = [], [], [], []
    for w in ws:
        g = iga.Patch(w.p, w.knots, w.ctrl(), **opts)
        lam, tc = g.cfl(w.rho, iters=20)
        U0, V0 = w.initial()
        st = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
        pats.append(g)
        states.append(st)
        dts.append(0.5 * tc)
        inits.append((torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV)))
    return pats, states, dts, inits


@pytest.mark.parametrize("opts", [dict(op_form="assembled", precond="bf16"),
                                  dict(op_form="matrix_free", precond="fp64"),
                                  dict(op_form="assembled", precond="fp32", guess="extrap")])
def test_batch_step_equals_patches_stepped_alone(opts):
    ws = _uneven()
    k, rho, nsteps = 2, 0.5, 6
    pats, states, dts, inits = _setup(ws, tol=1e-10, **opts)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    stb = b.step(states, k, rho, dts, nsteps)
    batched = [s.cpu().numpy().copy() for s in states]
    alone = []
    for g, st, (u0, v0), dt in zip(pats, states, inits, dts):
        g.state_init(k, u0, v0, st)
        sa = g.step(st, k, rho, dt, nsteps)
        alone.append((st.cpu().numpy().copy(), sa))
    for i in range(len(ws)):
        assert np.array_equal(batched[i], alone[i][0]), i
        assert stb[i].iters == alone[i][1].iters and stb[i].steps == nsteps
        assert stb[i].max_relres <= 1e-10
    # a second call replays the captured batch graph
    stb2 = b.step(states, k, rho, dts, 2)
    assert all(s.steps == 2 for s in stb2)
    b.close()
    for g in pats:
        g.close()


def test_batch_matches_oracle():
    ws = _uneven(npatch=3, seed=5)
    k, rho, nsteps = 2, 0.5, 5
    pats, states, dts, inits = _setup(ws, tol=1e-12, op_form="assembled", precond="fp64")
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    b.step(states, k, rho, dts, nsteps)
    for w, st, dt, g in zip(ws, states, dts, pats):
        ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
        so = oracle.Stepper(ops, k, rho, tol=1e-12)
        U0, V0 = w.initial()
        X = so.init(U0, V0)
        for _ in range(nsteps):
            X = so.step(X, dt)
        Xg = st.cpu().numpy().reshape(3 * k, g.N)
        for row in (0, 1):
            assert np.linalg.norm(Xg[row] - X[row]) / np.linalg.norm(X[row]) < 1e-9, (w.nel, w.p, row)
    b.close()
    for g in pats:
        g.close()


def test_batch_rebuilds_after_a_workspace_change():
    ws = _uneven(npatch=2, seed=7)
    k, rho = 2, 0.5
    pats, states, dts, inits = _setup(ws, tol=1e-10, op_form="assembled", precond="fp32")
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    b.step(states, k, rho, dts, 2)
    # grow one patch's workspaces (an 8-vector solve): the batch graph must not keep old addresses
    g = pats[0]
    rhs = torch.ones(8 * g.N, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(rhs)
    g.solve_M(rhs, x, nvec=8)
    ref = [s.clone() for s in states]
    b.step(states, k, rho, dts, 3)
    for i, (gg, st, dt) in enumerate(zip(pats, ref, dts)):
        gg.step(st, k, rho, dt, 3)
        assert torch.equal(st, states[i])
    b.close()
    for g in pats:
        g.close()
