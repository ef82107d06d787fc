"""The tiny-slot cut of the double-FP32 band products, checked on the CPU by an
emulation of their FP32 arithmetic (numpy float32; a fused multiply-add is the exact
product in FP64, which holds 48 bits, plus the addend, rounded to FP32).

The library forms the terms of a slot whose every coefficient lies below 2^-24 of the
matrix's largest (after the power-of-two scaling that puts the largest in [1, 2)) as
one FP32 multiply-add of the high parts instead of the exact product and TwoSum. The
claim checked here: at that cut the products keep the double-FP32 error (a few 2^-48
of sum |a||x|) and PCG with the paper's preconditioner reaches the same true residual
and the same solution as with FP64 products, while a cut far above it (2^-16) visibly
does not -- the cut is where the dropped parts fall below what the form carries.

The emulation follows the kernels' order of operations per row (the diagonal term,
then per run of slots with equal offsets along directions 1 and 2 the upper and the
lower terms, a Fast2Sum renormalisation after each run) but is neither the library's
code nor the oracle's: it is a numerical model of the design choice. The reference
products are the oracle's FP64 band rows."""
import numpy as np
import pytest

import oracle
import workloads as W

F32, F64 = np.float32, np.float64


def _fl(v):
    return np.asarray(v, dtype=F64).astype(F32)


def _fma(a, b, c):
    return _fl(a.astype(F64) * b.astype(F64) + c.astype(F64))


def _add(a, b):
    return _fl(a.astype(F64) + b.astype(F64))


def _sub(a, b):
    return _fl(a.astype(F64) - b.astype(F64))


def _split(v):
    hi = _fl(v)
    return hi, _fl(v - hi.astype(F64))


class Emulated:
    """Double-FP32 band products of one matrix (the oracle's full band rows)."""

    def __init__(self, patch, A, cut):
        self.P, self.A = patch, A
        n = patch.n
        self.N = N = patch.N
        idx = np.arange(N)
        self.i0, self.i1, self.i2 = idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])
        offs = patch.slot_offsets()
        self.slot = {tuple(int(v) for v in o): s for s, o in enumerate(offs)}
        self.EA = np.floor(np.log2(np.abs(A).max()))
        self.As = A / 2.0 ** self.EA
        smax = np.abs(self.As).max(axis=0)
        p = patch.p
        self.runs = [[(o0, 0, 0) for o0 in range(1, p[0] + 1)]]
        self.tiny_ends = [0]
        for o2 in range(0, p[2] + 1):
            for o1 in range(-p[1], p[1] + 1):
                if (o2, o1) <= (0, 0):
                    continue
                run = [(o0, o1, o2) for o0 in range(-p[0], p[0] + 1)]
                m = 0
                while (m < (len(run) + 1) // 2 and smax[self.slot[run[m]]] < cut
                       and smax[self.slot[run[len(run) - 1 - m]]] < cut):
                    m += 1
                self.runs.append(run)
                self.tiny_ends.append(m)

    def _nbr(self, o):
        n = self.P.n
        j0, j1, j2 = self.i0 + o[0], self.i1 + o[1], self.i2 + o[2]
        ok = (j0 >= 0) & (j0 < n[0]) & (j1 >= 0) & (j1 < n[1]) & (j2 >= 0) & (j2 < n[2])
        return ok, np.where(ok, j0 + n[0] * (j1 + n[1] * j2), 0)

    def __call__(self, x):
        xm = np.abs(x).max()
        Ex = np.floor(np.log2(xm)) if xm > 0 else 0.0
        xh, xl = _split(x / 2.0 ** Ex)
        s = np.zeros(self.N, F32)
        c = np.zeros(self.N, F32)

        def term(slot, o, tiny):
            nonlocal s, c
            ok, j = self._nbr(o)
            ah, al = _split(np.where(ok, self.As[:, slot], 0.0))
            xhj = np.where(ok, xh[j], F32(0))
            xlj = np.where(ok, xl[j], F32(0))
            if tiny:
                c = _fma(ah, xhj, c)
                return
            p = _fl(ah.astype(F64) * xhj.astype(F64))
            e = _fma(ah, xhj, -p)
            e = _fma(ah, xlj, e)
            e = _fma(al, xhj, e)
            S = _add(s, p)
            bp = _sub(S, s)
            t = _add(_sub(s, _sub(S, bp)), _sub(p, bp))
            c = _add(c, _add(t, e))
            s = S

        term(self.slot[(0, 0, 0)], (0, 0, 0), False)
        for run, m in zip(self.runs, self.tiny_ends):
            L = len(run)
            for t, o in enumerate(run):  # upper terms: a_i,slot x_{i+o}
                term(self.slot[o], o, t < m or t >= L - m)
            for t, o in enumerate(run):  # lower terms: a_{i-o},slot x_{i-o}, by symmetry the mirrored slot
                mo = (-o[0], -o[1], -o[2])
                term(self.slot[mo], mo, t < m or t >= L - m)
            S = _add(s, c)
            c = _sub(c, _sub(S, s))
            s = S
        return (s.astype(F64) + c.astype(F64)) * 2.0 ** (Ex + self.EA)


def _pcg(apply_M, pre, b, tol=1e-10, maxit=60):
    x = np.zeros_like(b)
    r = b.copy()
    z = pre(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        q = apply_M(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * nb:
            return x, it
        z = pre(r)
        rz2 = r @ z
        p = z + rz2 / rz * p
        rz = rz2
    return x, maxit


@pytest.fixture(scope="module")
def p4():
    w = W.small(d=3, nel=(7, 6, 6), p=4, amp=0.1)
    ops = oracle.Operators(oracle.Patch(w.p, w.knots, w.ctrl()))
    return ops


def test_tiny_terms_keep_the_double_fp32_error(p4):
    """Every row within 64 2^-48 sum|a||x| of the oracle's FP64 product at the 2^-24 cut,
    on M and K, and the cut takes a real share of the terms at p = 4."""
    P = p4.patch
    rows = np.arange(P.N)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(P.N)
    for A in (p4.M, p4.K):
        em = Emulated(P, A, 2.0 ** -24)
        assert sum(2 * min(2 * m, len(r)) for r, m in zip(em.runs, em.tiny_ends)) > 0.1 * A.shape[1]
        y = em(x)
        ref = P.band_rows_times(rows, A, x)
        bound = 64 * 2.0 ** -48 * P.band_rows_times(rows, np.abs(A), np.abs(x))
        assert np.all(np.abs(y - ref) <= bound)


def test_tiny_cut_leaves_pcg_as_fp64_but_a_coarse_cut_does_not(p4):
    """PCG (tol 1e-10) on M with the paper's preconditioner: with the 2^-24 cut the true
    residual and the distance of the solution from FP64-product PCG stay at the exact
    double-FP32 form's level; with a 2^-16 cut the solution drifts two orders further."""
    P = p4.patch
    b = np.random.default_rng(5).uniform(-1.0, 1.0, P.N)
    x64, _ = _pcg(p4.apply_M, p4.apply_Pinv, b)
    out = {}
    for name, cut in (("exact", 0.0), ("cut24", 2.0 ** -24), ("cut16", 2.0 ** -16)):
        em = Emulated(P, p4.M, cut)
        x, _ = _pcg(em, p4.apply_Pinv, b)
        true_res = np.linalg.norm(b - p4.apply_M(x)) / np.linalg.norm(b)
        out[name] = (true_res, np.linalg.norm(x - x64) / np.linalg.norm(x64))
    assert out["cut24"][0] <= 1.5e-10
    assert out["cut24"][1] <= 3 * max(out["exact"][1], 1e-12)
    assert out["cut16"][1] >= 30 * out["cut24"][1]
