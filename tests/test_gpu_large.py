"""Full-size check of the largest configuration: 3-D deformed cube, p = 4 (C^3),
128^3 elements, N = 2 197 000 interior dofs, 262 M Gauss points, k = 3 (6th order).

The oracle computes single rows of M and K one by one at this size (the
double-FP32 band products against the bound of their arithmetic); the time
stepping is checked by properties that hold at any size: the mixed and double-FP32
forms stay within 1e-8 of the FP64 form, the graph replay equals the host loop,
and the discrete energy does not grow at rho_inf = 0.5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2102_11536_gb300 as iga
import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def c3():
    w = W.config("cube128_p4")
    g = iga.Patch(w.p, w.knots, w.ctrl(), tol=w.tol)
    yield w, g
    g.close()


def test_cube128_sampled_rows(c3):
    w, g = c3
    P = oracle.Patch(w.p, w.knots, w.ctrl())
    rows = W.sample_indices(P.N, 60, seed=11)
    Mr, Kr = P.assemble(rows)
    X = np.random.default_rng(4).standard_normal(P.N)
    x = torch.from_numpy(X).to(DEV)
    y = torch.empty_like(x)
    for form in ("matrix_free", "assembled"):
        g.set_op_form(form)
        g.apply_M(x, y)
        ym = y.cpu().numpy()[rows]
        ref = P.band_rows_times(rows, Mr, X)
        assert np.abs(ym - ref).max() < 1e-12 * np.abs(ref).max(), form
        g.apply_K(x, y)
        yk = y.cpu().numpy()[rows]
        ref = P.band_rows_times(rows, Kr, X)
        assert np.abs(yk - ref).max() < 1e-11 * np.abs(ref).max(), form
    # double-FP32 band products: each sampled row within 64 2^-48 sum_j |a_ij||x_j|, plus
    # 2^-22 |a_ij x_j| for the terms of tiny slots (every coefficient below 2^-24 of the
    # matrix's largest: one FP32 multiply-add); the mask is a superset of those slots
    g.set_op_form("assembled_df")
    bound = 64 * 2.0 ** -48
    for A, apply in ((Mr, g.apply_M), (Kr, g.apply_K)):
        apply(x, y)
        tiny = (np.abs(A).max(axis=0) < 2.0 ** -20 * np.abs(A).max()).astype(np.float64)
        lim = (bound * P.band_rows_times(rows, np.abs(A), np.abs(X))
               + 2.0 ** -22 * P.band_rows_times(rows, np.abs(A) * tiny[None, :], np.abs(X)))
        assert np.all(np.abs(y.cpu().numpy()[rows] - P.band_rows_times(rows, A, X)) <= lim)
    g.set_op_form("matrix_free")


def _energy(g, X):
    U = torch.from_numpy(X[0]).to(DEV)
    V = torch.from_numpy(X[1]).to(DEV)
    KU = torch.empty_like(U)
    MV = torch.empty_like(V)
    g.apply_K(U, KU)
    g.apply_M(V, MV)
    return 0.5 * float(U @ KU) + 0.5 * float(V @ MV)


def test_cube128_forms_agree(c3):
    w, g = c3
    k, rho = w.k, w.rho
    lam, tc = g.cfl(rho, iters=30)
    dt = 0.5 * tc
    U0, V0 = w.initial()
    u0 = torch.from_numpy(U0).to(DEV)
    v0 = torch.from_numpy(V0).to(DEV)
    state = torch.empty(3 * k * g.N, dtype=torch.float64, device=DEV)
    steps = 6
    finals = {}
    # The BF16 preconditioner stops PCG at points farther apart within the same
    # tolerance; at tol 1e-10 its velocity sits at 1.5e-8 from the FP64 form here, so
    # that form runs at tol 1e-11 to meet 1e-8.
    for name, op, prec, graphs, tol in [("fp64", "assembled", "fp64", True, w.tol),
                                        ("fp32", "assembled", "fp32", True, w.tol),
                                        ("fp32_host", "assembled", "fp32", False, w.tol),
                                        ("bf16", "assembled", "bf16", True, 1e-11),
                                        ("mf", "matrix_free", "fp64", True, w.tol),
                                        ("df", "assembled_df", "banded32", True, w.tol),
                                        ("df_host", "assembled_df", "banded32", False, w.tol)]:
        g.set_op_form(op)
        g.set_precond(prec)
        g.set_graphs(graphs)
        g.set_tol(tol, 500)
        g.state_init(k, u0, v0, state)
        if name == "fp64":
            e0 = _energy(g, state.view(3 * k, g.N)[:2].cpu().numpy())
        st = g.step(state, k, rho, dt, steps)
        assert st.max_relres <= tol
        finals[name] = state.view(3 * k, g.N)[:2].cpu().numpy()
    ref = finals["fp64"]
    for name in ("fp32", "bf16", "mf", "df"):
        for row in (0, 1):
            err = np.linalg.norm(finals[name][row] - ref[row]) / np.linalg.norm(ref[row])
            assert err < 1e-8, (name, row, err)
    assert np.array_equal(finals["fp32"], finals["fp32_host"])
    assert np.array_equal(finals["df"], finals["df_host"])
    g.set_op_form("assembled")
    g.set_precond("fp64")
    g.set_tol(w.tol, 500)
    e1 = _energy(g, ref)
    assert e1 <= e0 * (1 + 1e-4)


def test_cube96_learned_warm_start():
    """96^3 deformed cube, p = 3, k = 2, 16 random modes, 1000 steps: the network is
    trained on the solves of the first 200 steps and then supplies the guesses of the
    remaining 800, compared with the zero and the extrapolated guess on those steps."""
    w = W.config("cube96_p3")
    g = iga.Patch(w.p, w.knots, w.ctrl(), tol=w.tol, op_form="assembled", precond="fp32")
    lam, tc = g.cfl(w.rho, iters=30)
    dt = 0.5 * tc
    k = w.k
    U0, V0 = w.initial()
    u0 = torch.from_numpy(U0).to(DEV)
    v0 = torch.from_numpy(V0).to(DEV)
    state = torch.empty(3 * k * g.N, dtype=torch.float64, device=DEV)
    n_train, n_total = 200, 1000
    res = {}
    for guess in ("learned", "extrap", "zero"):
        g.set_guess(guess)
        g.state_init(k, u0, v0, state)
        if guess == "learned":
            g.ws_collect(k * n_train)
        g.step(state, k, w.rho, dt, n_train + 2)
        if guess == "learned":
            assert g.ws_samples() == k * n_train
            losses = g.ws_train(10, 2e-3, seed=0)
            print("cube96 training: mean loss per epoch", ["%.4g" % v for v in losses])
            g.ws_collect(0)
            assert losses[-1] < 0.5 * losses[0], losses
        st = g.step(state, k, w.rho, dt, n_total - n_train - 2)
        assert st.max_relres <= w.tol
        res[guess] = (st, state.view(3 * k, g.N)[:2].cpu().numpy())
    init = {n: r[0].init_relres_sum / r[0].solves for n, r in res.items()}
    its = {n: r[0].iters / r[0].solves for n, r in res.items()}
    print("cube96 held-out steps: mean initial residual", init, "iterations per solve", its)
    assert init["learned"] < 0.7 * init["extrap"]
    assert its["learned"] <= its["extrap"] <= its["zero"]
    ref = res["zero"][1]
    for n in ("learned", "extrap"):
        for row in (0, 1):
            err = np.linalg.norm(res[n][1][row] - ref[row]) / np.linalg.norm(ref[row])
            print("cube96 %s vs zero guess after %d steps, row %d: %.3e" % (n, n_total, row, err))
            assert err < 1e-7, (n, row, err)
    g.close()


def test_multipatch_batch_48():
    """The 48-patch batch (sizes 16^3..96^3 elements, p in {2, 3, 4}, per-patch
    deformations): FP64 assembled operators, BF16 preconditioner, autotuned band
    launches; the batched graph steps equal every patch stepped alone, and the
    operators of the largest patch and of the 16 smallest match oracle rows."""
    ws = W.multipatch_batch()
    k, rho, nsteps = 2, 0.5, 3
    pats, states, dts, inits = [], [], [], []
    for w in ws:
        g = iga.Patch(w.p, w.knots, w.ctrl(), tol=1e-10, op_form="assembled", precond="bf16")
        lam, tc = g.cfl(rho, iters=20)
        g.autotune(nvec=k, reps=3)
        U0, V0 = w.initial()
        pats.append(g)
        dts.append(0.5 * tc)
        inits.append((torch.from_numpy(U0).to(DEV), torch.from_numpy(V0).to(DEV)))
        states.append(torch.zeros(3 * k * g.N, dtype=torch.float64, device=DEV))
    for g, st, (u0, v0) in zip(pats, states, inits):
        g.state_init(k, u0, v0, st)
    b = iga.Batch(pats)
    stb = b.step(states, k, rho, dts, nsteps)
    assert all(s.max_relres <= 1e-10 for s in stb)
    batched = [s.cpu().numpy() for s in states]
    for i, (g, st, (u0, v0), dt) in enumerate(zip(pats, states, inits, dts)):
        g.state_init(k, u0, v0, st)
        sa = g.step(st, k, rho, dt, nsteps)
        assert np.array_equal(st.cpu().numpy(), batched[i]), i
        assert sa.iters == stb[i].iters
    # operator rows against the oracle: the largest patch (30 rows) and the 16 smallest (6 rows
    # each: every degree, many shapes; the oracle's geometry at every Gauss point bounds the count)
    order = sorted(range(len(pats)), key=lambda i: pats[i].N)
    for i in [order[-1]] + order[:16]:
        w, g = ws[i], pats[i]
        P = oracle.Patch(w.p, w.knots, w.ctrl())
        rows = W.sample_indices(P.N, 30 if i == order[-1] else 6, seed=i)
        Mr, Kr = P.assemble(rows)
        X = np.random.default_rng(i).standard_normal(P.N)
        x = torch.from_numpy(X).to(DEV)
        y = torch.empty_like(x)
        g.apply_M(x, y)
        ref = P.band_rows_times(rows, Mr, X)
        assert np.abs(y.cpu().numpy()[rows] - ref).max() < 1e-12 * np.abs(ref).max()
        g.apply_K(x, y)
        ref = P.band_rows_times(rows, Kr, X)
        assert np.abs(y.cpu().numpy()[rows] - ref).max() < 1e-11 * np.abs(ref).max()
    b.close()
    for g in pats:
        g.close()
