"""Plain FP64 CPU oracle of the explicit 2k-order generalized-alpha method with
isogeometric mass/stiffness operators and the diagonal-scaled Kronecker mass
preconditioner (arXiv 2102.11536).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py may import this package. It
shares no code with the CUDA path (paper_2102_11536_gb300) and imports none of
it; both take their inputs from the separate `workloads` module.

Contents and the passage each follows:
  * basis(), gauss_legendre()        -- Cox-de Boor recursion (Sec. 5.1), Gauss rule (C, oracle.c)
  * Patch.assemble()                 -- eq. mass_matrix and the Galerkin stiffness of eq. pde (C)
  * Operators.apply_Pinv()           -- def:single_patch_prec / def:matrices_1, with
                                        (M1 x M2 x M3)^{-1} applied by banded Cholesky
                                        solves along each direction (Sec. 5.5)
  * pcg()                            -- preconditioned conjugate gradients (Sec. 5.5, Sec. 6)
  * galpha_params()                  -- boxed parameter formulas of Sec. 4.1 and eq. HOgamma
  * Stepper.step()                   -- eq. ho1-ho3 (Sec. 4), eq. 4a/4aup for k = 2
  * Stepper.init()                   -- initial high-order data (Sec. 3, after eq. 4aup)
  * theta_crit()                     -- stability limit from eq. charact at lambda = -1
  * modal_response(), spectral_radius() -- the scheme on one mode (Sec. 6.2), stability diagram
Where the paper is silent or garbled, the reading taken is stated beside the code that uses it.

Parity status: every function here is pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import scipy.linalg

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        L.ora_basis.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        L.ora_basis.restype = ctypes.c_int
        L.ora_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.ora_gauss_legendre.restype = None
        L.ora_quad_1d.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp, ip, dp, dp]
        L.ora_quad_1d.restype = ctypes.c_int
        L.ora_geometry.argtypes = [ip, dp, ip, dp, dp, dp, dp, dp, dp]
        L.ora_geometry.restype = ctypes.c_int
        L.ora_assemble_rows.argtypes = [ip, dp, ip, dp, dp, dp, dp, lp, ctypes.c_long, dp, dp]
        L.ora_assemble_rows.restype = ctypes.c_int
        L.ora_band_matvec.argtypes = [ip, ip, dp, dp, dp]
        L.ora_band_matvec.restype = None
        L.ora_mass_diagonal.argtypes = [ip, dp, ip, dp, dp, dp, dp]
        L.ora_mass_diagonal.restype = ctypes.c_int
        L.ora_num_threads.argtypes = []
        L.ora_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def num_threads() -> int:
    return int(lib().ora_num_threads())


# ----------------------------------------------------------------------------
# Spline space (Sec. 5.1)
# ----------------------------------------------------------------------------
def basis(p: int, knots: np.ndarray, x: float):
    """All degree-p B-splines of `knots` and their derivatives at x (Cox-de Boor, Sec. 5.1)."""
    knots = np.ascontiguousarray(knots, dtype=np.float64)
    m = len(knots) - p - 1
    val = np.zeros(m)
    der = np.zeros(m)
    rc = lib().ora_basis(p, len(knots), _d(knots), float(x), _d(val), _d(der))
    if rc != 0:
        raise ValueError("bad basis arguments")
    return val, der


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1]."""
    x = np.zeros(n)
    w = np.zeros(n)
    lib().ora_gauss_legendre(n, _d(x), _d(w))
    return x, w


class Quad1D:
    """Univariate quadrature tables over the elements (non-empty knot spans)."""

    def __init__(self, p: int, knots: np.ndarray, nq: int):
        knots = np.ascontiguousarray(knots, dtype=np.float64)
        self.p, self.knots, self.nq = p, knots, nq
        self.m = len(knots) - p - 1
        cap = (len(knots) - 1) * nq
        self.qx = np.zeros(cap)
        self.qw = np.zeros(cap)
        self.qfirst = np.zeros(cap, dtype=np.int32)
        self.qval = np.zeros(cap * (p + 1))
        self.qder = np.zeros(cap * (p + 1))
        nel = lib().ora_quad_1d(p, len(knots), _d(knots), nq, _d(self.qx), _d(self.qw), _i(self.qfirst),
                                _d(self.qval), _d(self.qder))
        self.nel = nel
        Q = nel * nq
        self.Q = Q
        self.qx, self.qw, self.qfirst = self.qx[:Q].copy(), self.qw[:Q].copy(), self.qfirst[:Q].copy()
        self.qval = self.qval[:Q * (p + 1)].copy()
        self.qder = self.qder[:Q * (p + 1)].copy()

    def dense(self, deriv=False):
        """(Q, m) table of all function values (or derivatives) at the quadrature points."""
        B = np.zeros((self.Q, self.m))
        src = self.qder if deriv else self.qval
        for q in range(self.Q):
            f = self.qfirst[q]
            B[q, f:f + self.p + 1] = src[q * (self.p + 1):(q + 1) * (self.p + 1)]
        return B

    def mass_interior(self):
        """Interior 1-D parametric mass matrix int b_i b_j over [0,1] (def:matrices_1 in one direction)."""
        B = self.dense()[:, 1:-1]
        return B.T @ (self.qw[:, None] * B)

    def stiffness_interior(self):
        """Interior 1-D parametric stiffness int b_i' b_j' over [0,1]."""
        B = self.dense(True)[:, 1:-1]
        return B.T @ (self.qw[:, None] * B)


class Patch:
    """Single-patch tensor-product discretisation (Sec. 5.1-5.2) with Gauss tables
    and the geometric factors W = w|det DF| and G = W DF^-1 DF^-T at every point."""

    def __init__(self, degrees, knots, ctrl, nq=None, geometry=True):
        self.d = d = len(degrees)
        self.p = [int(v) for v in degrees]
        self.nq = nq if nq is not None else max(self.p) + 1
        self.q1 = [Quad1D(self.p[a], knots[a], self.nq) for a in range(d)]
        self.m = [q.m for q in self.q1]
        self.n = [q.m - 2 for q in self.q1]
        self.N = int(np.prod(self.n))
        self.Q = [q.Q for q in self.q1]
        self.ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
        pad = lambda v, fill: list(v) + [fill] * (3 - d)
        self.dims = np.array([d] + pad(self.p, 0) + pad(self.m, 1) + pad(self.Q, 1), dtype=np.int32)
        self.qw_all = np.concatenate([q.qw for q in self.q1])
        self.qfirst_all = np.concatenate([q.qfirst for q in self.q1]).astype(np.int32)
        self.qval_all = np.concatenate([q.qval for q in self.q1])
        self.qder_all = np.concatenate([q.qder for q in self.q1])
        self.W = None
        self.G = None
        self.detmin = None
        if geometry:
            self.compute_geometry()

    def compute_geometry(self):
        Qt = int(np.prod(self.Q))
        ng = 6 if self.d == 3 else 3
        self.W = np.zeros(Qt)
        self.G = np.zeros(Qt * ng)
        dm = np.zeros(1)
        bad = lib().ora_geometry(_i(self.dims), _d(self.qw_all), _i(self.qfirst_all), _d(self.qval_all),
                                 _d(self.qder_all), _d(self.ctrl), _d(self.W), _d(self.G), _d(dm))
        self.detmin = float(dm[0])
        if bad:
            raise ValueError("det DF <= 0 at a quadrature point (min %g)" % self.detmin)

    @property
    def nslots(self):
        return int(np.prod([2 * p + 1 for p in self.p]))

    def assemble(self, rows=None, stiffness=True):
        """Band rows of M and K (see ora_assemble_rows) for `rows` (default: all)."""
        if rows is None:
            nr, rp = self.N, None
        else:
            rows = np.ascontiguousarray(rows, dtype=np.int64)
            nr, rp = len(rows), _l(rows)
        S = self.nslots
        Mr = np.zeros((nr, S))
        Kr = np.zeros((nr, S)) if stiffness else None
        lib().ora_assemble_rows(_i(self.dims), _d(self.qw_all), _i(self.qfirst_all), _d(self.qval_all),
                                _d(self.qder_all), _d(self.W), _d(self.G), rp, nr, _d(Mr),
                                _d(Kr) if stiffness else None)
        return Mr, Kr

    def mass_diagonal(self):
        """diag(M) without assembling M (ora_mass_diagonal)."""
        D = np.zeros(self.N)
        lib().ora_mass_diagonal(_i(self.dims), _d(self.qw_all), _i(self.qfirst_all), _d(self.qval_all),
                                _d(self.qder_all), _d(self.W), _d(D))
        return D

    def band_rows_times(self, rows, A, x):
        """(A x)_i for the given rows, A holding those rows' band slots (sampled checks)."""
        n3 = self.n + [1] * (3 - self.d)
        offs = self.slot_offsets()
        out = np.zeros(len(rows))
        for r, i in enumerate(rows):
            i0, i1, i2 = i % n3[0], (i // n3[0]) % n3[1], i // (n3[0] * n3[1])
            j0, j1, j2 = i0 + offs[:, 0], i1 + offs[:, 1], i2 + offs[:, 2]
            ok = (j0 >= 0) & (j0 < n3[0]) & (j1 >= 0) & (j1 < n3[1]) & (j2 >= 0) & (j2 < n3[2])
            j = j0 + n3[0] * (j1 + n3[1] * j2)
            out[r] = np.sum(A[r][ok] * x[j[ok]])
        return out

    def slot_offsets(self):
        """(S, 3) integer offsets (o0, o1, o2) of the band slots."""
        p3 = self.p + [0] * (3 - self.d)
        offs = []
        for o2 in range(-p3[2], p3[2] + 1):
            for o1 in range(-p3[1], p3[1] + 1):
                for o0 in range(-p3[0], p3[0] + 1):
                    offs.append((o0, o1, o2))
        return np.array(offs)

    def band_to_dense(self, A):
        """Dense (N, N) matrix of full band rows (tests on tiny meshes)."""
        n3 = self.n + [1] * (3 - self.d)
        N = self.N
        D = np.zeros((N, N))
        offs = self.slot_offsets()
        for i in range(N):
            i0, i1, i2 = i % n3[0], (i // n3[0]) % n3[1], i // (n3[0] * n3[1])
            for s, (o0, o1, o2) in enumerate(offs):
                j0, j1, j2 = i0 + o0, i1 + o1, i2 + o2
                if 0 <= j0 < n3[0] and 0 <= j1 < n3[1] and 0 <= j2 < n3[2]:
                    D[i, j0 + n3[0] * (j1 + n3[1] * j2)] = A[i, s]
        return D

    def band_matvec(self, A, x):
        n3 = np.array(self.n + [1] * (3 - self.d), dtype=np.int32)
        p3 = np.array(self.p + [0] * (3 - self.d), dtype=np.int32)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.N)
        lib().ora_band_matvec(_i(n3), _i(p3), _d(np.ascontiguousarray(A)), _d(x), _d(y))
        return y


# ----------------------------------------------------------------------------
# Operators and the preconditioner (Sec. 5.3, 5.5)
# ----------------------------------------------------------------------------
class Preconditioner:
    """The preconditioner P = D^{1/2} Dhat^{-1/2} Mhat Dhat^{-1/2} D^{1/2}
    (def:single_patch_prec), Mhat = Mhat_3 (x) Mhat_2 (x) Mhat_1 the parametric
    (F = identity) mass matrix, Dhat = diag(Mhat), D = diag(M) (def:matrices_1).
    Mhat^{-1} is applied through the Kronecker structure by banded Cholesky solves
    along each direction. D defaults to ora_mass_diagonal."""

    def __init__(self, patch: Patch, D=None):
        self.patch = patch
        self.d = patch.d
        self.n = patch.n
        self.N = patch.N
        self.D = patch.mass_diagonal() if D is None else D
        self.Mhat = [patch.q1[a].mass_interior() for a in range(self.d)]
        self.cho = []
        for a in range(self.d):
            A = self.Mhat[a]
            pa = patch.p[a]
            nb = A.shape[0]
            ab = np.zeros((pa + 1, nb))  # lower banded storage for scipy
            for r in range(pa + 1):
                ab[r, :nb - r] = np.diag(A, -r)
            self.cho.append(scipy.linalg.cholesky_banded(ab, lower=True))
        dh = np.ones(1)
        for a in range(self.d):  # co-lex: direction 0 fastest -> Dhat = diag_{d-1} (x) ... (x) diag_0
            dh = np.kron(np.diag(self.Mhat[a]), dh)
        self.Dhat = dh
        self.scale = np.sqrt(self.Dhat / self.D)  # D^{-1/2} Dhat^{1/2}

    def kron_solve(self, r):
        """Mhat^{-1} r, one banded Cholesky solve along each direction (Kronecker inverse)."""
        shape = tuple(reversed(self.n))  # C-order array (i_{d-1}, ..., i_0)
        t = r.reshape(shape).copy()
        for a in range(self.d):
            ax = self.d - 1 - a
            t = np.moveaxis(t, ax, 0)
            sh = t.shape
            sol = scipy.linalg.cho_solve_banded((self.cho[a], True), t.reshape(sh[0], -1))
            t = np.moveaxis(sol.reshape(sh), 0, ax)
        return np.ascontiguousarray(t).reshape(-1)

    def apply_Pinv(self, r):
        """z = D^{-1/2} Dhat^{1/2} Mhat^{-1} Dhat^{1/2} D^{-1/2} r."""
        return self.scale * self.kron_solve(self.scale * r)


class Operators:
    """Assembled M and K (band rows) with the preconditioner of Sec. 5.3; D is the
    centre slot (the diagonal) of the assembled M."""

    def __init__(self, patch: Patch, stiffness=True):
        self.patch = patch
        self.d = patch.d
        self.n = patch.n
        self.N = patch.N
        self.M, self.K = patch.assemble(stiffness=stiffness)
        self.pre = Preconditioner(patch, D=self.M[:, patch.nslots // 2].copy())
        self.D = self.pre.D
        self.Mhat = self.pre.Mhat

    def apply_M(self, x):
        return self.patch.band_matvec(self.M, x)

    def apply_K(self, x):
        return self.patch.band_matvec(self.K, x)

    def apply_Pinv(self, r):
        return self.pre.apply_Pinv(r)


def pcg(apply_A, apply_Pinv, b, x0=None, tol=1e-10, max_iter=500):
    """Preconditioned conjugate gradients (Sec. 5.5). Stops when ||r||_2 <= tol ||b||_2
    (the paper's relative tolerance; the denominator is ||b||, so that a warm start is
    held to the same target as the null guess). Returns (x, iterations, ||r||/||b||).
    One iteration = one product A p."""
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
    rn = float(np.linalg.norm(r))
    if rn <= tol * bn:
        return x, 0, rn / bn
    z = apply_Pinv(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < max_iter:
        q = apply_A(p)
        pq = float(p @ q)
        if not pq > 0.0:
            raise FloatingPointError("non-positive curvature in PCG")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = float(np.linalg.norm(r))
        if rn <= tol * bn:
            break
        z = apply_Pinv(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rn / bn


# ----------------------------------------------------------------------------
# Time integration (Sec. 3-4)
# ----------------------------------------------------------------------------
def block_params(rho_b: float, rho_s: float, last: bool):
    """alpha, beta of one diagonal block from the boxed formulas of Sec. 4.1.
    last=True: the block j = k; last=False: a block j < k."""
    rb, rs = rho_b, rho_s
    if last:
        alpha = (2 + (1 - rb) * rs) / ((1 + rb) * (1 + rs))
        beta = (-5 - 3 * rb - 4 * rs + 2 * rb * rs + 2 * rb ** 2 * rs - rs ** 2 + rb * rs ** 2) / (
            (1 + rb) ** 2 * (-2 - 3 * rs + rb * rs - rs ** 2 + rb * rs ** 2))
    else:
        alpha = (2 - (1 + rb) * rs) / ((-1 + rb) * (-1 + rs))
        beta = (1 + rb) * (-1 + rb * rs) ** 2 / ((-1 + rb) ** 2 * (-1 + rs) * (-2 + rs + rb * rs))
    return alpha, beta


def galpha_params(k: int, rho: float):
    """Per-block (alpha_j, beta_j, gamma_j, alpha_fj), j = 1..k, for the user parameter
    rho in [0, 1] with rho_b = rho_s (remark after the boxed formulas).
      * j = k: boxed last-block formulas at rho_bk = rho_sk = rho, alpha_fk = 0.
      * j < k: boxed j<k formulas evaluated at rho_bj = rho_sj = -rho, alpha_fj = 1
        (reading: the printed +rho makes the j<k stability limit collapse and contradicts
        the claimed k-independent stability region; -rho maps the j<k bifurcation point
        onto the last block's).
      * gamma_j = 1/2 - alpha_fj + alpha_j (eq. HOgamma)."""
    out = []
    for j in range(1, k + 1):
        last = j == k
        r = rho if last else -rho
        a, b = block_params(r, r, last)
        af = 0.0 if last else 1.0
        out.append((a, b, 0.5 - af + a, af))
    return out


def theta_crit(rho: float) -> float:
    """Stability limit Theta = tau^2 lambda_max of every block: the value at which a root
    of the characteristic polynomial (eq. charact) crosses lambda = -1, with the parameters
    of galpha_params. Substituting lambda = -1 gives Theta = 4(2 alpha - 1)/(4 beta - 2 alpha - 1)
    = 12 (1 + rho)(2 - rho)/(rho^2 - 5 rho + 10)."""
    return 12.0 * (1 + rho) * (2 - rho) / (rho * rho - 5 * rho + 10)


def predictor(X, tau):
    """Taylor predictor T_q = sum_{r >= q} tau^{r-q}/(r-q)! X_r (eq. ho2-ho3), rows q = -2..3k-3."""
    nq = X.shape[0]
    T = np.zeros_like(X)
    for qi in range(nq):
        for r in range(qi, nq):
            T[qi] += tau ** (r - qi) / math.factorial(r - qi) * X[r]
    return T


class Stepper:
    """Explicit 2k-order generalized-alpha stepping (Sec. 4) for M U'' + K U = 0.

    State X: array (3k, N), rows (U, V, A, L^1, ..., L^{3k-3}), i.e. X_q at row q + 2.
    Block j = 1..k solves for s_j = 3j - 3:
        M Z_j = F^{(s_j)}(t_{n + alpha_fj}) - K Y_j - C Y'_j,
        Y_j = T_{s_j - 2}, Y'_j = T_{s_j - 1} (j < k, alpha_f = 1),  Y_k = X_{s_k - 2}, Y'_k = X_{s_k - 1}
        P_j = (Z_j - T_{s_j}) / alpha_j
        X_{s_j} <- T_{s_j} + P_j,  X_{s_j-1} <- T_{s_j-1} + gamma_j tau P_j,
        X_{s_j-2} <- T_{s_j-2} + beta_j tau^2 P_j.
    (Z_j is the paper's L^{s_j}(A_n)^{alpha_j} = T_{s_j} + alpha_j P_{n,j}.) The stiffness
    argument Y_j is the reading that gives order 2k (eq. ho1 taken literally, K U_n for
    every block, gives order 1 and is unstable for k >= 2)."""

    def __init__(self, ops, k: int, rho: float, tol=1e-10, max_iter=500, guess="zero", params=None,
                 damping=None, forcing=None, t0=0.0):
        self.ops, self.k, self.rho = ops, k, rho
        self.tol, self.max_iter, self.guess = tol, max_iter, guess
        self.params = params if params is not None else galpha_params(k, rho)
        self.hist = [[None, None] for _ in range(k)]  # Z_j at the previous two steps
        self.iters = []
        # M U'' + C U' + K U = F (eq. mp): C = a_M M + a_K K (Rayleigh damping) when
        # damping = (a_M, a_K); forcing(s, t) returns F^{(s)}(t), the s-th time derivative
        # of the load vector. None: C = 0, F = 0.
        self.damping = damping
        self.forcing = forcing
        self.t = t0

    def apply_C(self, x):
        aM, aK = self.damping
        return aM * self.ops.apply_M(x) + aK * self.ops.apply_K(x)

    def _load(self, s, t, n):
        return np.zeros(n) if self.forcing is None else np.asarray(self.forcing(s, t), dtype=np.float64)

    def solve(self, b, x0=None):
        x, it, rr = pcg(self.ops.apply_M, self.ops.apply_Pinv, b, x0, self.tol, self.max_iter)
        if rr > self.tol:
            raise RuntimeError("PCG did not converge (rel. residual %g)" % rr)
        return x, it

    def init(self, U0, V0):
        """Initial data (Sec. 3, after eq. 4aup):
        X_a = M^{-1}(F^{(a)}(0) - K X_{a-2} - C X_{a-1}), a = 0..3k-3, with X_{-2} = U0, X_{-1} = V0."""
        nq = 3 * self.k
        n = self.ops.N
        X = np.zeros((nq, n))
        X[0], X[1] = U0, V0
        for a in range(0, 3 * self.k - 2):
            b = self._load(a, self.t, n) - self.ops.apply_K(X[a])
            if self.damping is not None:
                b = b - self.apply_C(X[a + 1])
            X[a + 2], _ = self.solve(b)
        return X

    def _guess(self, j, T, row):
        h1, h2 = self.hist[j]
        if self.guess == "zero" or h1 is None:
            return None
        if self.guess == "prev":
            return h1
        if self.guess == "extrap":
            return h1 if h2 is None else 2 * h1 - h2
        if self.guess == "taylor":
            return T[row]
        raise ValueError(self.guess)

    def step(self, X, tau):
        k = self.k
        T = predictor(X, tau)
        Xn = T.copy()
        its = []
        for j in range(1, k + 1):
            a, b, g, _ = self.params[j - 1]
            row = 3 * j - 3 + 2
            # blocks j < k (alpha_f = 1): the predictors at t_{n+1}; block k (alpha_f = 0): X^n at t_n
            Y = T[row - 2] if j < k else X[row - 2]
            Yv = T[row - 1] if j < k else X[row - 1]
            tj = self.t + tau if j < k else self.t
            rhs = self._load(3 * j - 3, tj, X.shape[1]) - self.ops.apply_K(Y)
            if self.damping is not None:
                rhs = rhs - self.apply_C(Yv)
            Z, it = self.solve(rhs, self._guess(j - 1, T, row))
            its.append(it)
            self.hist[j - 1] = [Z, self.hist[j - 1][0]]
            P = (Z - T[row]) / a
            Xn[row] = T[row] + P
            Xn[row - 1] = T[row - 1] + g * tau * P
            Xn[row - 2] = T[row - 2] + b * tau * tau * P
        self.iters.append(its)
        self.t += tau
        return Xn


class ScalarOps:
    """The modal problem u'' = -lam u (M = 1, K = lam) as an Operators stand-in."""

    def __init__(self, lam):
        self.lam = float(lam)
        self.N = 1

    def apply_M(self, x):
        return x.copy()

    def apply_K(self, x):
        return self.lam * x

    def apply_Pinv(self, r):
        return r.copy()


def scalar_amplification(k, rho, Theta, params=None):
    """Amplification matrix of one step of the scheme on u'' = -lam u with tau = 1 and
    lam = Theta, in the scaled variables (U, tau V, tau^2 A, ...) of Sec. 3.1."""
    st = Stepper(ScalarOps(Theta), k, rho, tol=0.0, params=params)
    nq = 3 * k
    G = np.zeros((nq, nq))
    for c in range(nq):
        X = np.zeros((nq, 1))
        X[c, 0] = 1.0
        G[:, c] = st.step(X, 1.0)[:, 0]
    return G


def spectral_radius(k, rho, Omega):
    """Spectral radius of one step's amplification matrix at Omega = tau sqrt(lam) (the
    stability diagram of Sec. 3.2: below 1 up to the limit sqrt(Theta_crit), rho_inf at
    the bifurcation point)."""
    return float(max(abs(np.linalg.eigvals(scalar_amplification(k, rho, Omega * Omega)))))


def modal_response(k, rho, lam, tau, n, U0=1.0, V0=0.0):
    """The scheme on one mode u'' = -lam u (Sec. 3.1's modal problem): U_s for s = 0..n
    after s steps of length tau from the initial data (U0, V0) (higher derivatives as
    in Stepper.init). The dispersion and dissipation of the discrete scheme on that mode
    (Sec. 6.2) are read off this series against cos(sqrt(lam) t)."""
    st = Stepper(ScalarOps(lam), k, rho, tol=0.0)
    X = st.init(np.array([float(U0)]), np.array([float(V0)]))
    out = [float(X[0, 0])]
    for _ in range(n):
        X = st.step(X, tau)
        out.append(float(X[0, 0]))
    return np.array(out)


def exact_semidiscrete(Md, Kd, U0, V0, t):
    """U(t), V(t) of M U'' + K U = 0 by the generalized eigendecomposition K phi = w^2 M phi."""
    lam, Phi = scipy.linalg.eigh(Kd, Md)
    w = np.sqrt(lam)
    a = Phi.T @ (Md @ U0)
    b = Phi.T @ (Md @ V0)
    U = Phi @ (a * np.cos(w * t) + b * np.sin(w * t) / w)
    V = Phi @ (-a * w * np.sin(w * t) + b * np.cos(w * t))
    return U, V


def lambda_max_dense(Md, Kd):
    return float(scipy.linalg.eigh(Kd, Md, eigvals_only=True)[-1])


def lambda_max_lanczos(ops: Operators, iters=60, seed=0, tol=1e-12, rtol=1e-12):
    """Largest eigenvalue of M^{-1}K by the Lanczos process in the M inner product (M^{-1}K is
    self-adjoint there): v_1 M-normalised, w = M^{-1} K v_j - alpha_j v_j - beta_{j-1} v_{j-1},
    alpha_j = v_j^T K v_j, beta_j = ||w||_M, v_{j+1} = w / beta_j; the estimate is the largest
    eigenvalue of the tridiagonal matrix of the alphas and betas. Stops after `iters` steps,
    or when that estimate changes by less than rtol (relative) from one step to the next."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(ops.N)
    v = v / math.sqrt(v @ ops.apply_M(v))
    vp = np.zeros(ops.N)
    alphas, betas = [], []
    beta = 0.0
    est = None
    for _ in range(iters):
        y = ops.apply_K(v)
        w, _, _ = pcg(ops.apply_M, ops.apply_Pinv, y, None, tol)
        alpha = float(v @ y)
        w = w - alpha * v - beta * vp
        alphas.append(alpha)
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        new = float(np.linalg.eigvalsh(T)[-1])
        if est is not None and abs(new - est) <= rtol * abs(new):
            return new
        est = new
        beta = math.sqrt(max(float(w @ ops.apply_M(w)), 0.0))
        if beta == 0.0:
            return est
        betas.append(beta)
        vp, v = v, w / beta
    return est

