"""GPU parity of the learned warm start against the FP64 oracle (oracle/net.py), and
what the trained network gains over the extrapolated guess.

Tolerances are derived from the arithmetic: the device sums in FP32 (unit
roundoff u = 2^-24) where the oracle sums in FP64, so each checked value may
differ by (number of summed terms) x u x (the same sum taken over absolute
values); a BF16-rounded value may land one BF16 step (2^-7 relative at most)
away where the FP32 and FP64 sums straddle a rounding boundary.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle.net as net
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
U32 = 2.0 ** -24


def _bf16_dev(a):
    """numpy array of BF16-representable values -> device bfloat16 tensor (exact)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).to(torch.bfloat16).to(DEV)


def _f32_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).to(DEV)


def _case(shape, nb, seed):
    n1, n2, n3 = shape
    rng = np.random.default_rng(seed)
    theta = net.bf16_round(rng.uniform(-0.3, 0.3, net.NPARAM))
    xs = np.stack([net.bf16_round(rng.standard_normal((3, n3, n2, n1))) for _ in range(nb)])
    return rng, theta, xs


def _forward(shape, xs, theta):
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    nb = xs.shape[0]
    x = _bf16_dev(xs)
    th = _f32_dev(theta)
    act = torch.empty(nb * 16 * N, dtype=torch.bfloat16, device=DEV)
    y = torch.empty(nb * N, dtype=torch.float32, device=DEV)
    iga.net_forward(shape, x, th, act, y, nb=nb)
    torch.cuda.synchronize()
    A = act.float().cpu().numpy().astype(np.float64).reshape(nb, 16, n3, n2, n1)
    Y = y.cpu().numpy().astype(np.float64).reshape(nb, n3, n2, n1)
    return x, th, act, A, Y


# grids spanning several 16 x 16 x 4 tiles with ragged tails, and smaller than one tile
SHAPES = [(19, 21, 9), (33, 7, 13), (16, 16, 4), (5, 3, 2), (1, 1, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_net_forward_matches_oracle(shape):
    nb = 2
    _, theta, xs = _case(shape, nb, sum(shape))
    _, _, _, A, Y = _forward(shape, xs, theta)
    W1, b1, W2, b2 = net.split_params(theta)
    for s in range(nb):
        h, a, _ = net.forward(xs[s], theta)
        # hidden layer: FP32 sums of 82 terms, then BF16 rounding
        eh = 82 * U32 * net.conv3d(np.abs(xs[s]), np.abs(W1), np.abs(b1))
        diff = np.abs(A[s] - a)
        assert np.all(diff <= 2.0 ** -7 * np.maximum(np.abs(a), np.abs(A[s])) + 2 * eh)
        assert np.mean(diff > 0) < 1e-2
        # output layer on the device's own hidden layer: FP32 sums of 433 terms
        yref = net.conv3d(A[s], W2, b2)[0]
        bound = 433 * U32 * net.conv3d(np.abs(A[s]), np.abs(W2), np.abs(b2))[0]
        assert np.all(np.abs(Y[s] - yref) <= bound + 1e-30)


@pytest.mark.parametrize("shape", [(19, 21, 9), (33, 7, 13), (5, 3, 2)])
def test_net_backward_matches_oracle(shape):
    # gradient check of the device's backward kernels against the CPU oracle; the
    # oracle takes the device's hidden layer, so both make the same ReLU decisions
    nb = 2
    n1, n2, n3 = shape
    N = n1 * n2 * n3
    rng, theta, xs = _case(shape, nb, 100 + sum(shape))
    x, th, act, A, _ = _forward(shape, xs, theta)
    dys = rng.standard_normal((nb, n3, n2, n1)).astype(np.float32).astype(np.float64)
    grad = torch.empty(net.NPARAM, dtype=torch.float32, device=DEV)
    work = torch.empty(iga.net_workspace_bytes(shape, nb), dtype=torch.uint8, device=DEV)
    iga.net_backward(shape, x, th, act, _f32_dev(dys), grad, work, nb=nb)
    g = grad.cpu().numpy().astype(np.float64)
    go = sum(net.backward(xs[s], theta, dys[s], act=A[s]) for s in range(nb))
    gabs = sum(net.backward(np.abs(xs[s]), np.abs(theta), np.abs(dys[s]), act=A[s]) for s in range(nb))
    # per-block FP32 partial sums over <= 1024 points, 27-term FP32 sums inside dh,
    # an FP64 sum over blocks, one rounding to FP32
    bound = (1024 + 28 + 2) * U32 * gabs
    assert np.all(np.abs(g - go) <= bound + 1e-30), np.max(np.abs(g - go) / (bound + 1e-30))
    # the check is not vacuous: the gradient is far above its bound
    assert np.linalg.norm(go) > 100 * np.linalg.norm(bound)


def test_adam_matches_oracle():
    rng = np.random.default_rng(7)
    th0 = rng.uniform(-0.3, 0.3, net.NPARAM).astype(np.float32).astype(np.float64)
    th = _f32_dev(th0)
    m = torch.zeros(net.NPARAM, dtype=torch.float32, device=DEV)
    v = torch.zeros_like(m)
    tho, mo, vo = th0.copy(), np.zeros(net.NPARAM), np.zeros(net.NPARAM)
    lr = 1e-3
    for step in range(1, 6):
        gr = rng.standard_normal(net.NPARAM).astype(np.float32).astype(np.float64)
        gr[:7] = 0.0  # zero gradients leave parameters in place
        iga.net_adam(th, _f32_dev(gr), m, v, step, lr)
        tho, mo, vo = net.adam(tho, gr, mo, vo, step, lr)
    torch.cuda.synchronize()
    got = th.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - tho) <= 5 * (U32 * np.abs(tho) + 1e-5 * lr))
    assert np.array_equal(got[:7], th0[:7])


def _patch_case():
    w = W.small(d=3, nel=(9, 5, 4), p=(3, 2, 3), amp=0.12)
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    g = iga.Patch(w.p, w.knots, w.ctrl())
    return w, P, g


def test_features_match_oracle():
    w, P, g = _patch_case()
    k, N = 2, g.N
    shape = tuple(reversed(P.n))
    assert g.shape == tuple(P.n)
    rng = np.random.default_rng(8)
    vals = {nm: rng.standard_normal(k * N) for nm in ("b", "b1", "b2", "z1", "z2")}
    dev = {nm: torch.from_numpy(v.copy()).to(DEV) for nm, v in vals.items()}
    x = torch.empty(k * 3 * N, dtype=torch.bfloat16, device=DEV)
    E = torch.empty(k * N, dtype=torch.float64, device=DEV)
    sc = torch.empty(2 * k, dtype=torch.float64, device=DEV)
    g.ws_features(k, dev["b"], dev["b1"], dev["b2"], dev["z1"], dev["z2"], x, E, sc)
    D = P.mass_diagonal()
    X = x.float().cpu().numpy().astype(np.float64).reshape(k, 3, N)
    Eg = E.cpu().numpy().reshape(k, N)
    S = sc.cpu().numpy().reshape(k, 2)
    for j in range(k):
        sl = slice(j * N, (j + 1) * N)
        xo, s0, s1, Eo = net.features(vals["b"][sl], vals["b1"][sl], vals["b2"][sl], D, vals["z1"][sl],
                                      vals["z2"][sl], shape)
        assert np.isclose(S[j, 0], s0, rtol=1e-13) and np.isclose(S[j, 1], s1, rtol=1e-13)
        xo = xo.reshape(3, N)
        d = np.abs(X[j] - xo)
        assert np.all(d <= 2.0 ** -7 * np.abs(xo)) and np.mean(d > 0) < 1e-3
        assert np.array_equal(Eg[j], Eo)
    # the histories moved one step
    assert np.array_equal(dev["b1"].cpu().numpy(), vals["b"])
    assert np.array_equal(dev["b2"].cpu().numpy(), vals["b1"])
    assert np.array_equal(dev["z2"].cpu().numpy(), vals["z1"])
    assert np.array_equal(dev["z1"].cpu().numpy(), Eg.ravel())
    g.close()


def _dt(ops, rho, frac=0.5):
    lmax = oracle.lambda_max_dense(ops.patch.band_to_dense(ops.M), ops.patch.band_to_dense(ops.K))
    return frac * math.sqrt(oracle.theta_crit(rho) / lmax)


def test_learned_guess_steps_match_oracle():
    # any parameters: the guess changes where PCG starts, not where it stops
    w = W.small(d=3, nel=(5, 4, 4), p=3, amp=0.1, k=2, rho=0.5, init="random")
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    dt = _dt(ops, w.rho)
    U0, V0 = w.initial()
    st = oracle.Stepper(ops, w.k, w.rho, tol=1e-12)
    Xo = st.init(U0, V0)
    for _ in range(8):
        Xo = st.step(Xo, dt)
    g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-12, guess="learned")
    g.ws_set_params(net.bf16_round(np.random.default_rng(9).uniform(-0.2, 0.2, net.NPARAM)))
    state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(w.k, torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV), state)
    s = g.step(state, w.k, w.rho, dt, 8)
    Xg = state.cpu().numpy().reshape(3 * w.k, g.N)
    for row in (0, 1):
        assert np.linalg.norm(Xg[row] - Xo[row]) / np.linalg.norm(Xo[row]) < 1e-9
    assert s.max_relres <= 1e-12
    g.close()


def test_learned_graph_equals_host_loop():
    w = W.small(d=3, nel=(6, 5, 4), p=3, amp=0.1, k=2, rho=0.5, init="random")
    theta = net.bf16_round(np.random.default_rng(10).uniform(-0.2, 0.2, net.NPARAM))
    U0, V0 = w.initial()
    out = []
    for graphs in (True, False):
        g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-10, guess="learned", op_form="assembled", precond="fp32")
        g.set_graphs(graphs)
        g.ws_set_params(theta)
        lam, tc = g.cfl(w.rho, iters=20)
        state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
        g.state_init(w.k, torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV), state)
        st = g.step(state, w.k, w.rho, 0.5 * tc, 7)
        out.append((state.cpu().numpy(), st.iters, st.init_relres_sum))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert out[0][2] == pytest.approx(out[1][2], rel=1e-12)


def _run(w, guess, n_head, n_eval, record=0, train=None):
    """n_head steps from the initial data (recording samples and training the network
    afterwards when `record` is set), then n_eval steps whose statistics are returned."""
    g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-10, guess=guess, op_form="assembled", precond="fp32")
    lam, tc = g.cfl(w.rho, iters=30)
    dt = 0.5 * tc
    U0, V0 = w.initial()
    state = torch.zeros(3 * w.k * g.N, dtype=torch.float64, device=DEV)
    g.state_init(w.k, torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV), state)
    losses = None
    if record:
        g.ws_collect(record)
    g.step(state, w.k, w.rho, dt, n_head)
    if record:
        assert g.ws_samples() == record
        losses = g.ws_train(*train, seed=1)
        g.ws_collect(0)
    st = g.step(state, w.k, w.rho, dt, n_eval)
    X = state.cpu().numpy().reshape(3 * w.k, g.N)
    g.close()
    return X, st, losses


def test_trained_network_beats_extrapolation():
    # 24^3 deformed cube, p = 3, k = 2, random smooth initial data: 42 steps of which
    # the last 40 record their 80 solves, 30 epochs, then 30 held-out steps per guess
    w = W.small(d=3, nel=24, p=3, amp=0.1, k=2, rho=0.5, init="random")
    n_rec, n_eval = 80, 30
    n_head = n_rec // w.k + 2
    Xl, sl, losses = _run(w, "learned", n_head, n_eval, record=n_rec, train=(30, 2e-3))
    Xe, se, _ = _run(w, "extrap", n_head, n_eval)
    Xz, sz, _ = _run(w, "zero", n_head, n_eval)
    # training reduced the loss
    assert losses[-1] < 0.5 * losses[0], losses
    # same solution, within the solver tolerance carried over the run
    for row in (0, 1):
        for Xo in (Xe, Xz):
            assert np.linalg.norm(Xl[row] - Xo[row]) / np.linalg.norm(Xo[row]) < 1e-8
    # the held-out steps: the learned guess starts closer to the solution than the
    # extrapolated one and needs no more iterations
    init_l = sl.init_relres_sum / sl.solves
    init_e = se.init_relres_sum / se.solves
    print("held-out mean initial residual: learned %.3e extrap %.3e zero 1; iterations/solve: "
          "learned %.3f extrap %.3f zero %.3f" % (init_l, init_e, sl.iters / sl.solves, se.iters / se.solves,
                                                  sz.iters / sz.solves))
    assert init_l < 0.7 * init_e
    assert sl.iters <= se.iters
    assert sz.init_relres_sum == pytest.approx(sz.solves)


def test_ws_argument_errors():
    w, P, g = _patch_case()
    with pytest.raises(iga.IgaError):
        g.ws_train(1)  # no samples recorded
    with pytest.raises(iga.IgaError):
        g.ws_collect(-1)
    with pytest.raises(iga.IgaError):
        g.ws_get_params()  # no parameters yet
    g.ws_init_params(3)
    th = g.ws_get_params()
    assert np.all(np.abs(th[:1296]) <= 1 / 9) and np.all(th[1296:1312] == 0)
    assert np.all(np.abs(th[1312:1744]) <= 1 / math.sqrt(432)) and th[1744] == 0
    assert np.std(th[:1296]) > 0.05
    g.close()
