"""The general model M U'' + C U' + K U = F on the GPU (Rayleigh damping, harmonic
loads, the device-side time) against the FP64 oracle: initial data, steps, the graph
replay against the host loop, and the batch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TERMS = [(2.0, 0.3), (5.0, -1.0)]  # (omega, phase)
DAMP = (0.4, 1e-4)


def _loads(N, seed=0):
    return np.random.default_rng(seed).standard_normal((len(TERMS), N))


def _forcing(G):
    def F(s, t):
        return sum(G[m] * w ** s * math.sin(w * t + p + s * math.pi / 2) for m, (w, p) in enumerate(TERMS))
    return F


def _dt(ops, rho, frac=0.5):
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    return frac * math.sqrt(oracle.theta_crit(rho) / lmax)


def _gpu(w, G, damping=DAMP, forcing=True, t0=0.0, **kw):
    g = iga.Patch(w.p, w.knots, w.ctrl(), **kw)
    if damping:
        g.set_damping(*damping)
    if forcing:
        g.set_forcing(torch.from_numpy(np.ascontiguousarray(G)).to(DEV), [w_ for w_, _ in TERMS],
                      [p for _, p in TERMS])
    g.set_time(t0)
    return g


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("form", [("matrix_free", "fp64"), ("assembled", "banded"), ("assembled", "banded32"),
                                  ("assembled_df", "banded32")])
@pytest.mark.parametrize("case", ["damped", "forced", "both"])
def test_general_model_steps_match_oracle(k, form, case):
    w = W.small(d=3, nel=(5, 4, 4), p=3, amp=0.1, k=k, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    G = _loads(ops.N)
    damping = DAMP if case in ("damped", "both") else None
    forced = case in ("forced", "both")
    t0 = 0.37
    st = oracle.Stepper(ops, k, w.rho, tol=1e-12, damping=damping, forcing=_forcing(G) if forced else None, t0=t0)
    U0, V0 = w.initial()
    V0 = 0.3 * U0[::-1].copy()
    Xo = st.init(U0, V0)
    X0 = Xo.copy()
    for _ in range(8):
        Xo = st.step(Xo, dt)
    g = _gpu(w, G, damping=damping, forcing=forced, t0=t0, tol=1e-12, op_form=form[0], precond=form[1])
    state = torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(k, torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV), state)
    Xi = state.cpu().numpy().reshape(3 * k, g.N)
    for r in range(3 * k):  # initial data
        assert np.linalg.norm(Xi[r] - X0[r]) <= 1e-9 * max(np.linalg.norm(X0[r]), 1e-300), r
    s = g.step(state, k, w.rho, dt, 8)
    Xg = state.cpu().numpy().reshape(3 * k, g.N)
    for row in (0, 1):
        assert np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row]) < 1e-9, row
    assert s.max_relres <= 1e-12
    tt = t0
    for _ in range(8):
        tt += dt
    assert g.get_time() == tt
    g.close()


@pytest.mark.parametrize("guess", ["zero", "extrap"])
def test_general_model_graph_equals_host_loop(guess):
    w = W.small(d=3, nel=(6, 5, 4), p=3, amp=0.1, k=2, rho=0.5, init="random")
    G = _loads(W.small(d=3, nel=(6, 5, 4), p=3).ndof, seed=1)
    U0, V0 = w.initial()
    out = []
    for graphs in (False, True):
        g = _gpu(w, G, tol=1e-11, op_form="assembled", precond="banded32", guess=guess)
        g.set_graphs(graphs)
        lam, tc = g.cfl(w.rho, iters=20)
        state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
        g.state_init(w.k, torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV), state)
        st = g.step(state, w.k, w.rho, 0.5 * tc, 4)
        st = g.step(state, w.k, w.rho, 0.5 * tc, 5, st)
        out.append((state.cpu().numpy(), st.iters, g.get_time()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_general_model_in_a_batch():
    ws = [W.small(d=3, nel=(4, 5, 3), p=2, amp=0.1, k=2, init="random", seed=1),
          W.small(d=3, nel=(3, 4, 6), p=3, amp=0.12, k=2, init="random", seed=2)]
    pats, states, dts, inits = [], [], [], []
    for i, w in enumerate(ws):
        g = _gpu(w, _loads(w.ndof, seed=10 + i), tol=1e-10, op_form="assembled", precond="fp64")
        lam, tc = g.cfl(0.5, iters=20)
        U0, V0 = w.initial()
        inits.append((torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV)))
        states.append(torch.zeros(6 * g.N, dtype=torch.float64, device=DEV))
        dts.append(0.5 * tc)
        pats.append(g)
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(2, u0, v0, st)
    b = iga.Batch(pats)
    b.step(states, 2, 0.5, dts, 5)
    batched = [s.cpu().numpy().copy() for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.set_time(0.0)
        g.state_init(2, u0, v0, st)
        g.step(st, 2, 0.5, dt, 5)
        assert np.array_equal(st.cpu().numpy(), batched[i]), i
    b.close()
    for g in pats:
        g.close()


def test_general_model_argument_errors():
    w = W.small(d=3, nel=3, p=2)
    g = iga.Patch(w.p, w.knots, w.ctrl())
    with pytest.raises(iga.IgaError):
        g.set_damping(-1.0, 0.0)
    with pytest.raises(iga.IgaError):
        g.set_time(float("nan"))
    G = torch.zeros(9 * g.N, dtype=torch.float64, device=DEV)
    with pytest.raises(iga.IgaError):
        g.set_forcing(G, [1.0] * 9, [0.0] * 9)  # more than 8 terms
    g.set_forcing(None, [], [])  # no loads
    g.close()
