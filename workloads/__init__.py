"""Seeded synthetic inputs for the explicit generalized-alpha IGA workloads.

This module only generates inputs -- knot vectors, control nets and initial
coefficient vectors -- and holds none of the method's arithmetic. Both the CPU
oracle (tests) and the CUDA path (tests, bench) take their inputs from here.

Geometry recipe. The paper's benchmark geometries (blade, donut, fan; Sec. 6)
are not published, so the unit square/cube stands in for them:
  * uniform open knot vectors with maximal regularity C^{p-1};
  * identity map: control points at the Greville abscissae (a spline
    reproduces the linear function with Greville coefficients);
  * deformed map: every Greville point g is moved by
    amp * sin(pi g_1) sin(pi g_2) sin(pi g_3) in each coordinate. Boundary
    Greville points have a zero factor, so the boundary and hence the domain
    stay exactly the unit cube.
Initial data are coefficient vectors on the interior control points, taken as
the value of the continuous field at each control point (Schoenberg's
variation-diminishing quasi-interpolant).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def open_uniform_knots(nel: int, p: int) -> np.ndarray:
    """Open knot vector on [0, 1] with nel equal spans, ends repeated p+1 times."""
    inner = [i / nel for i in range(1, nel)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1), dtype=np.float64)


def greville(knots: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae: mean of the p knots following knot i, one per basis function."""
    m = len(knots) - p - 1
    if p == 0:
        return np.array([(knots[i] + knots[i + 1]) / 2 for i in range(m)])
    return np.array([knots[i + 1:i + p + 1].mean() for i in range(m)])


def control_net(knots: list[np.ndarray], degrees: list[int], amp=0.0) -> np.ndarray:
    """Full control net, co-lexicographic (direction 0 fastest), shape (prod m, d).

    amp: a scalar or a length-d sequence, the deformation amplitude per coordinate.
    """
    d = len(knots)
    gs = [greville(knots[a], degrees[a]) for a in range(d)]
    mesh = np.meshgrid(*gs, indexing="ij")  # mesh[a][i0, i1, ...]
    amps = np.broadcast_to(np.asarray(amp, dtype=np.float64), (d,))
    bump = np.ones_like(mesh[0])
    for a in range(d):
        bump = bump * np.sin(np.pi * mesh[a])
    coords = [mesh[a] + amps[a] * bump for a in range(d)]
    # co-lex: index 0 fastest -> transpose to (i_{d-1}, ..., i_0) before flattening
    out = np.stack([c.transpose(tuple(range(d - 1, -1, -1))).reshape(-1) for c in coords], axis=1)
    return np.ascontiguousarray(out)


def interior_points(ctrl: np.ndarray, m: list[int]) -> np.ndarray:
    """Physical coordinates of the interior control points, co-lex, shape (N, d)."""
    d = len(m)
    grid = ctrl.reshape(tuple(reversed(m)) + (d,))
    sl = tuple(slice(1, -1) for _ in range(d))
    inner = grid[sl]
    return np.ascontiguousarray(inner.reshape(-1, d))


def standing_wave(x: np.ndarray) -> np.ndarray:
    """u0(x) = prod_a sin(pi x_a); with zero velocity the exact solution of
    u_tt = Laplace u on the unit cube is u0(x) cos(sqrt(d) pi t)."""
    return np.prod(np.sin(np.pi * x), axis=1)


def random_modes(x: np.ndarray, nmodes: int = 16, seed: int = 0, maxfreq: int = 8) -> np.ndarray:
    """Sum of nmodes seeded Fourier modes prod_a sin(m_a pi x_a), m in {1..maxfreq}^d,
    amplitudes N(0,1)/|m|^2."""
    rng = np.random.default_rng(seed)
    d = x.shape[1]
    u = np.zeros(x.shape[0])
    for _ in range(nmodes):
        m = rng.integers(1, maxfreq + 1, size=d)
        a = rng.standard_normal() / float(np.dot(m, m))
        u += a * np.prod(np.sin(np.pi * m[None, :] * x), axis=1)
    return u


@dataclasses.dataclass
class Workload:
    """One synthetic single-patch problem: mesh, geometry, initial data, scheme parameters."""
    name: str
    d: int
    nel: tuple
    p: tuple
    amp: float
    k: int
    rho: float
    steps: int
    init: str = "standing"  # 'standing' | 'random'
    seed: int = 0
    tol: float = 1e-10
    cfl_fraction: float = 0.5

    @property
    def knots(self):
        return [open_uniform_knots(self.nel[a], self.p[a]) for a in range(self.d)]

    @property
    def m(self):
        return [self.nel[a] + self.p[a] for a in range(self.d)]

    @property
    def n(self):
        return [self.nel[a] + self.p[a] - 2 for a in range(self.d)]

    @property
    def ndof(self):
        return int(np.prod(self.n))

    def ctrl(self):
        return control_net(self.knots, list(self.p), self.amp)

    def initial(self):
        """(U0, V0) interior coefficient vectors."""
        x = interior_points(self.ctrl(), self.m)
        if self.init == "standing":
            u0 = standing_wave(x)
        else:
            u0 = random_modes(x, seed=self.seed)
        return np.ascontiguousarray(u0), np.zeros_like(u0)


def config(name: str) -> Workload:
    """The five synthetic configurations of the benchmark suite, by name; also
    'cube:<nel>:<p>[:<k>]', the deformed unit cube (amplitude 0.1) with nel^3 elements of
    degree p, k = 3 unless given, 16 seeded random modes (smaller cases of the same kind,
    for profiling and sweeps)."""
    if name.startswith("cube:"):
        f = [int(v) for v in name.split(":")[1:]]
        if len(f) not in (2, 3) or f[0] < 1 or f[1] < 1:
            raise KeyError(name)
        k = f[2] if len(f) == 3 else 3
        return Workload(name, 3, (f[0],) * 3, (f[1],) * 3, 0.1, k, 0.5, 100, init="random")
    if name == "square32_p2":  # 2-D, identity, p=2, 32^2, k=1
        return Workload(name, 2, (32, 32), (2, 2), 0.0, 1, 0.5, 100)
    if name == "cube64_p3":  # 3-D deformed, p=3, 64^3, k=2
        return Workload(name, 3, (64, 64, 64), (3, 3, 3), 0.1, 2, 0.5, 500)
    if name == "cube128_p4":  # 3-D deformed, p=4, 128^3, k=3, random modes
        return Workload(name, 3, (128, 128, 128), (4, 4, 4), 0.1, 3, 0.5, 200, init="random")
    if name == "cube96_p3":  # 3-D deformed, p=3, 96^3, k=2, random modes
        return Workload(name, 3, (96, 96, 96), (3, 3, 3), 0.1, 2, 0.5, 1000, init="random")
    if name == "cube64_p4":  # the 128^3 p=4 discretisation on 64^3 elements (a few GB: profiling captures)
        return Workload(name, 3, (64, 64, 64), (4, 4, 4), 0.1, 3, 0.5, 200, init="random")
    raise KeyError(name)


def small(d=3, nel=4, p=2, amp=0.1, k=2, rho=0.5, steps=10, init="standing", seed=0) -> Workload:
    """A small seeded case for parity tests."""
    nel_t = tuple([nel] * d) if np.isscalar(nel) else tuple(nel)
    p_t = tuple([p] * d) if np.isscalar(p) else tuple(p)
    return Workload("small", d, nel_t, p_t, amp, k, rho, steps, init=init, seed=seed)


def multipatch_batch(npatch: int = 48, seed: int = 0, nel_range=(16, 96), p_choices=(2, 3, 4), amp_max=0.15):
    """Seeded uneven batch of independent 3-D patches (sizes, degrees, deformation amplitudes)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(npatch):
        nel = tuple(int(v) for v in rng.integers(nel_range[0], nel_range[1] + 1, size=3))
        p = int(rng.choice(p_choices))
        amp = tuple(float(v) for v in rng.uniform(0.0, amp_max, size=3))
        w = Workload("patch%d" % r, 3, nel, (p, p, p), 0.0, 2, 0.5, 100)
        w.amp = amp
        out.append(w)
    return out


def sample_indices(N: int, count: int, seed: int = 0) -> np.ndarray:
    """Seeded sorted sample of row indices, always including the first and last row."""
    rng = np.random.default_rng(seed)
    idx = set(int(v) for v in rng.choice(N, size=min(count, N), replace=False))
    idx.update({0, N - 1})
    return np.array(sorted(idx), dtype=np.int64)
