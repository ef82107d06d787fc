// One persistent, cooperative launch per time step of a batch of independent patches:
// every patch's Taylor predictor, batched K product, k mass solves by PCG with the
// diagonal-scaled Kronecker preconditioner (def:single_patch_prec; the Kronecker
// inverse by band Cholesky along each direction, Sec. 5.5) and stage update (Sec. 4,
// eq. ho1-ho3). The work of each phase is a list of (patch, tile) items -- row tiles of
// kPRows rows for the band products and vector updates, tiles of kPLines lines for the
// axis solves -- which the resident blocks take in turn; phases are separated by a grid
// barrier whose wait is bounded (a time-out sets the error word and every block
// returns). The per-system scalars of PCG (one system per patch and stage) are summed from
// per-tile partials in a phase of their own (block b sums systems b, b + G, ... in a fixed
// order), then updated by block 0, so a run is reproducible.
//
// Arithmetic per row and line as in the single-patch kernels: the FP64 band product
// (diagonal, then per stored slot the upper and the lower term), the band-Cholesky
// substitutions with the factor rows scaled by 1 / L_kk (FP32 or FP64), the predictor
// and update of k_predict / k_update. Or the preconditioner by fast diagonalisation
// with 16-bit operands: six mode products whose matrix entries and inputs are rounded
// to BF16 and whose products (exact in FP32) are summed in FP32 -- the arithmetic of
// the tensor-core form, here on the CUDA cores of the persistent blocks (the products
// of one line tile are 32 n^2 multiply-adds, n <= 98 for these patches). PCG:
// Hestenes-Stiefel with the FP64 Kronecker solve, the flexible (Polak-Ribiere) beta
// with the FP32 and BF16 ones; stop at ||r|| <= tol ||b||; x0 = 0.
#include <cuda_bf16.h>

#include "iga_internal.h"

namespace iga {

namespace {

constexpr int kPThreads = 256;     // threads per block
constexpr int kPRows = kPThreads;  // rows per row tile: one per thread
constexpr int kPLines = 32;        // lines per line tile: one warp runs the substitutions
constexpr int kPLS = kPLines + 1;  // shared row stride of a staged tile (odd: no bank conflicts)

// Grid barrier (arrival count bar[0], generation bar[1]). The wait is bounded: after
// `limit` polls, or once another block has reported a time-out, the block records one
// and the caller returns. Every block arrives before it waits, so the count is reset by
// the last one to arrive even when some gave up.
__device__ bool pgrid_sync(unsigned int* bar, long long limit, int* err) {
  __shared__ int gave_up;
  __syncthreads();
  if (threadIdx.x == 0) {
    gave_up = 0;
    __threadfence();
    volatile unsigned int* gen = bar + 1;
    const unsigned int g0 = *gen;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g0) {
        if (++it > limit || *(volatile int*)err) {
          atomicExch(err, 1);
          gave_up = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return gave_up == 0;
}

// fixed-order block sum of one value per thread (valid in thread 0)
__device__ double pblock_sum(double v);

// out[s] = sum over the patch's tiles t of part[(t0 + t) k + j], s = patch k + j: a phase of
// its own, block b summing systems b, b + G, ... (a fixed strided share per thread, then the
// block tree: a fixed order), so that one block does not sum every system's partials
__device__ void psum_phase(const PBatch& B, const double* part, const int* t0, const int* nt, double* out) {
  const int S = B.np * B.k;
  for (int s = blockIdx.x; s < S; s += gridDim.x) {  // uniform over the block
    const int pi = s / B.k, j = s - pi * B.k;
    double a = 0.0;
    for (int t = threadIdx.x; t < nt[pi]; t += kPThreads) a += __ldcg(&part[(long long)(t0[pi] + t) * B.k + j]);
    a = pblock_sum(a);
    if (threadIdx.x == 0) out[s] = a;
  }
}

__device__ double pblock_sum(double v) {
  __shared__ double red[kPThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kPThreads / 32; ++q) s += red[q];
  return s;
}

// ---------------------------------------------------------------- row-tile phases
// Taylor predictor: Y[j] = -Y_j (the argument of K, negated), T[j] = T_{s_j}; x[j] = 0
template <int K>
__device__ void ph_predict(const PBatch& B) {
  constexpr int R = 3 * K;
  for (int it = blockIdx.x; it < B.nrt; it += gridDim.x) {
    const int2 tl = B.rtile[it];
    const PPatch& P = B.pt[tl.x];
    const long long N = P.N, i = (long long)tl.y * kPRows + threadIdx.x;
    if (i >= N) continue;
    double xr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) xr[r] = P.X[r * N + i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int row = 3 * j + 2, ry = row - 2;
      double y;
      if (j < K - 1) {
        y = 0.0;
#pragma unroll
        for (int r = R - 1; r >= ry; --r) y = fma(P.sc.c[r - ry], xr[r], y);
      } else {
        y = xr[ry];
      }
      P.Y[j * N + i] = -y;
      P.z[j * N + i] = 0.0;  // the previous z of the first flexible beta
      double t = 0.0;
#pragma unroll
      for (int r = R - 1; r >= row; --r) t = fma(P.sc.c[r - row], xr[r], t);
      P.T[j * N + i] = t;
      P.x[j * N + i] = 0.0;
    }
  }
}

// y[j] = A x[j] for the patch's active systems (mask act), one row per thread; with
// dot, the per-tile partials of x[j].y[j] (dot = 1) or y[j].y[j] (dot = 2) into part.
// SLOTS slots per pass: their coefficients and x values are all loaded before their
// multiply-adds (SLOTS times the loads in flight; the phase is bound by the FP64 units
// once enough loads are in flight); the terms are added in slot order, the upper term
// before the lower one, as in the single-patch band product, whatever SLOTS is.
template <int K, int SLOTS>
__device__ void ph_band(const PBatch& B, bool stiff, const double* const* xs, double* const* ys, int dot,
                        double* part) {
  for (int it = blockIdx.x; it < B.nrt; it += gridDim.x) {
    const int2 tl = B.rtile[it];
    int on = (1 << K) - 1;  // the systems computed (uniform over the block)
    if (!stiff) {
      on = 0;
#pragma unroll
      for (int v = 0; v < K; ++v)
        if (B.active[tl.x * K + v]) on |= 1 << v;
      if (!on) continue;  // a patch whose systems have all converged
    }
    const PPatch& P = B.pt[tl.x];
    const double* __restrict__ x = xs[tl.x];
    double* y = ys[tl.x];
    const long long N = P.N, i = (long long)tl.y * kPRows + threadIdx.x;
    const int H = P.H, n1 = P.n[1], n2 = P.n[2];
    const bool row = i < N;
    const double* __restrict__ A = stiff ? P.K : P.M;
    const long long* __restrict__ off = P.off;
    const int* __restrict__ o12 = P.o12;
    double acc[K];
    const double a0 = row ? A[i] : 0.0;
#pragma unroll
    for (int v = 0; v < K; ++v) acc[v] = row && (on >> v & 1) ? a0 * x[v * N + i] : 0.0;
    int i1 = 0, i2 = 0;
    if (row) {
      const long long t = i / P.n[0];
      i1 = (int)(t % n1);
      i2 = (int)(t / n1);
    }
    for (int h = 1; h < H; h += SLOTS) {
      bool up[SLOTS], dn[SLOTS];
      double au[SLOTS], ad[SLOTS], xu[SLOTS][K], xd[SLOTS][K];
#pragma unroll
      for (int u = 0; u < SLOTS; ++u) {
        const int hh = h + u;
        up[u] = dn[u] = false;
        long long jp = 0, jm = 0;
        if (hh < H) {
          const long long L = off[hh];
          jp = i + L;
          jm = i - L;
          const int pk = o12[hh];
          const int o1 = (pk & 255) - 64, o2 = ((pk >> 8) & 255) - 64;
          up[u] = row && jp < N && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
          dn[u] = row && jm >= 0 && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
        }
        const double* Ah = A + (long long)hh * N;
        au[u] = up[u] ? Ah[i] : 0.0;
        ad[u] = dn[u] ? Ah[jm] : 0.0;
#pragma unroll
        for (int v = 0; v < K; ++v) {
          xu[u][v] = up[u] && (on >> v & 1) ? x[v * N + jp] : 0.0;
          xd[u][v] = dn[u] && (on >> v & 1) ? x[v * N + jm] : 0.0;
        }
      }
      bool any = false;
#pragma unroll
      for (int u = 0; u < SLOTS; ++u) any = any || up[u] || dn[u];
      if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
      for (int u = 0; u < SLOTS; ++u) {
        if (up[u]) {
#pragma unroll
          for (int v = 0; v < K; ++v)
            if (on >> v & 1) acc[v] = fma(au[u], xu[u][v], acc[v]);
        }
        if (dn[u]) {
#pragma unroll
          for (int v = 0; v < K; ++v)
            if (on >> v & 1) acc[v] = fma(ad[u], xd[u][v], acc[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < K; ++v)
      if (row && (on >> v & 1)) y[v * N + i] = acc[v];
    if (dot) {
#pragma unroll
      for (int v = 0; v < K; ++v) {
        const bool o = row && (on >> v & 1);
        const double t = o ? (dot == 1 ? x[v * N + i] : acc[v]) * acc[v] : 0.0;
        const double s = pblock_sum(t);
        if (threadIdx.x == 0) part[(long long)it * K + v] = s;
      }
    }
  }
}

// p = z (first) or z + beta p; active systems
template <int K>
__device__ void ph_dir(const PBatch& B, bool first) {
  for (int it = blockIdx.x; it < B.nrt; it += gridDim.x) {
    const int2 tl = B.rtile[it];
    bool any = false;
#pragma unroll
    for (int v = 0; v < K; ++v) any = any || B.active[tl.x * K + v];
    if (!any) continue;
    const PPatch& P = B.pt[tl.x];
    const long long N = P.N, i = (long long)tl.y * kPRows + threadIdx.x;
    if (i >= N) continue;
#pragma unroll
    for (int v = 0; v < K; ++v) {
      const int s = tl.x * K + v;
      if (!B.active[s]) continue;
      const double zv = P.z[v * N + i];
      P.p[v * N + i] = first ? zv : fma(B.beta[s], P.p[v * N + i], zv);
    }
  }
}

// x += alpha p, r -= alpha q; partials of r.r
template <int K>
__device__ void ph_xr(const PBatch& B) {
  for (int it = blockIdx.x; it < B.nrt; it += gridDim.x) {
    const int2 tl = B.rtile[it];
    bool any = false;  // a converged patch: its partials are not read (uniform over the block)
#pragma unroll
    for (int v = 0; v < K; ++v) any = any || B.active[tl.x * K + v];
    if (!any) continue;
    const PPatch& P = B.pt[tl.x];
    const long long N = P.N, i = (long long)tl.y * kPRows + threadIdx.x;
    const bool row = i < N;
#pragma unroll
    for (int v = 0; v < K; ++v) {
      const int s = tl.x * K + v;
      double t = 0.0;
      if (row && B.active[s]) {
        const double al = B.alpha[s];
        P.x[v * N + i] = fma(al, P.p[v * N + i], P.x[v * N + i]);
        const double rn = fma(-al, P.q[v * N + i], P.r[v * N + i]);
        P.r[v * N + i] = rn;
        t = rn * rn;
      }
      const double sum = pblock_sum(t);
      if (threadIdx.x == 0) B.part[(long long)it * K + v] = sum;
    }
  }
}

// stage update from the solutions x[j] = Z_j and the predictor
template <int K>
__device__ void ph_update(const PBatch& B) {
  constexpr int R = 3 * K;
  for (int it = blockIdx.x; it < B.nrt; it += gridDim.x) {
    const int2 tl = B.rtile[it];
    const PPatch& P = B.pt[tl.x];
    const long long N = P.N, i = (long long)tl.y * kPRows + threadIdx.x;
    if (i >= N) continue;
    double xr[R], t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) xr[r] = P.X[r * N + i];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      double s = 0.0;
#pragma unroll
      for (int r = R - 1; r >= q; --r) s = fma(P.sc.c[r - q], xr[r], s);
      t[q] = s;
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int row = 3 * j + 2;
      const double Pj = (P.x[j * N + i] - t[row]) * P.sc.ralpha[j];
      P.X[row * N + i] = t[row] + Pj;
      P.X[(row - 1) * N + i] = fma(P.sc.gtau[j], Pj, t[row - 1]);
      P.X[(row - 2) * N + i] = fma(P.sc.btau2[j], Pj, t[row - 2]);
    }
  }
}

// ---------------------------------------------------------------- Kronecker solve
// A line tile of axis a: lines l0 .. l0 + nl - 1 of the patch (line l0 + l = xx + A y, its
// entry k the element xx + A (k + n y)), staged in shared memory for every active system
// of the patch at once (entry k of line l of system v at (v n + k) kPLS + l).
struct LineTile {
  int n, nl, a;
  long long A, N, l0;
  long long base;  // a > 0: the element of entry 0 of this thread's line (lane = line)
};

__device__ __forceinline__ LineTile line_tile(const PPatch& Pp, int a, int tile) {
  LineTile t;
  t.a = a;
  t.n = Pp.n[a];
  t.N = Pp.N;
  t.A = a == 0 ? 1 : (a == 1 ? (long long)Pp.n[0] : (long long)Pp.n[0] * Pp.n[1]);
  t.l0 = (long long)tile * kPLines;
  t.nl = (int)min((long long)kPLines, t.N / t.n - t.l0);
  t.base = 0;
  const int l = threadIdx.x & (kPLines - 1);
  if (a > 0 && l < t.nl) {
    const long long rr = t.l0 + l, y = rr / t.A;
    t.base = (rr - y * t.A) + t.A * (long long)t.n * y;
  }
  return t;
}

// f(k, l, g) over the tile's entries: entry k of line l is element g. Axis 0: the tile
// is one contiguous range, walked by consecutive threads (no division per entry); other
// axes: lane = line (consecutive lines are adjacent elements), warps step over k.
template <typename F>
__device__ __forceinline__ void tile_walk(const LineTile& t, F&& f) {
  if (t.a == 0) {
    const long long g0 = t.l0 * t.n;
    const int cnt = t.nl * t.n;
    const int dl = kPThreads / t.n, dk = kPThreads - dl * t.n;
    int l = threadIdx.x / t.n, k = threadIdx.x - l * t.n;
    for (int e = threadIdx.x; e < cnt; e += kPThreads) {
      f(k, l, g0 + e);
      k += dk;
      l += dl;
      if (k >= t.n) {
        k -= t.n;
        ++l;
      }
    }
  } else {
    const int l = threadIdx.x & (kPLines - 1);
    if (l >= t.nl) return;
    for (int k = threadIdx.x >> 5; k < t.n; k += kPThreads / 32) f(k, l, t.base + t.A * k);
  }
}

// The forward and backward substitutions of line `lane` of one staged system (factor
// rows scaled by 1 / L_kk, recurrence window in registers).
template <int P, typename T>
__device__ void solve_lines(T* sb, const T* sF, const T* sG, int n, int lane) {
  T win[P + 1];
#pragma unroll
  for (int d = 0; d <= P; ++d) win[d] = T(0);
  for (int k = 0; k < n; ++k) {
    const T* F = sF + (size_t)k * (P + 1);
    T acc = F[0] * sb[k * kPLS + lane];
#pragma unroll
    for (int d = P; d >= 2; --d) acc -= F[d] * win[d];
    const T w = acc - F[1] * win[1];
    sb[k * kPLS + lane] = w;
#pragma unroll
    for (int d = P; d >= 2; --d) win[d] = win[d - 1];
    win[1] = w;
  }
#pragma unroll
  for (int d = 0; d <= P; ++d) win[d] = T(0);
  for (int k = n - 1; k >= 0; --k) {
    const T* G = sG + (size_t)k * (P + 1);
    T acc = G[0] * sb[k * kPLS + lane];
#pragma unroll
    for (int d = P; d >= 2; --d) acc -= G[d] * win[d];
    const T z = acc - G[1] * win[1];
    sb[k * kPLS + lane] = z;
#pragma unroll
    for (int d = P; d >= 2; --d) win[d] = win[d - 1];
    win[1] = z;
  }
}

// the active systems of a patch as a bit mask (uniform over the block)
template <int K>
__device__ __forceinline__ int patch_active(const PBatch& B, int patch) {
  int m = 0;
#pragma unroll
  for (int v = 0; v < K; ++v)
    if (B.active[patch * K + v]) m |= 1 << v;
  return m;
}

// Band-Cholesky axis phase: axis 0 reads r scaled by D^-1/2 Dhat^1/2 into t1; axis 1
// t1 -> t2; axis 2 t2 -> z scaled again, with the partials of r.z (new) and r.z (the
// previous z) of each system. Every active system of the tile is staged at once and
// warp v runs the substitutions of system v.
template <int K, typename T>
__device__ void ph_axis(const PBatch& B, int a, unsigned char* smem) {
  for (int it = blockIdx.x; it < B.nlt[a]; it += gridDim.x) {
    const int2 tl = B.ltile[a][it];
    const int act = patch_active<K>(B, tl.x);
    if (!act) {  // a converged patch: only the last phase's partials (zeros)
      if (a == 2 && threadIdx.x < K) {
        B.lpart[(long long)it * K + threadIdx.x] = 0.0;
        B.lpart[(long long)(B.nrzt + it) * K + threadIdx.x] = 0.0;
      }
      continue;
    }
    const PPatch& Pp = B.pt[tl.x];
    const LineTile t = line_tile(Pp, a, tl.y);
    const int n = t.n, p = Pp.deg[a];
    const long long N = t.N;
    T* sF = reinterpret_cast<T*>(smem);
    T* sG = sF + (size_t)n * (p + 1);
    T* sb = sG + (size_t)n * (p + 1);
    const T* L = static_cast<const T*>(Pp.L[a]);
    const T* dinv = static_cast<const T*>(Pp.dinv[a]);
    const T* tin = a == 1 ? static_cast<const T*>(Pp.t1) : static_cast<const T*>(Pp.t2);
    T* tout = a == 0 ? static_cast<T*>(Pp.t1) : static_cast<T*>(Pp.t2);
    __syncthreads();  // the previous item's shared data is consumed
    for (int e = threadIdx.x; e < n * (p + 1); e += kPThreads) {
      const int k = e / (p + 1), d = e - k * (p + 1);
      const T dk = dinv[k];
      sF[e] = d == 0 ? dk : dk * L[e];
      sG[e] = d == 0 ? dk : (k + d < n ? dk * L[(size_t)(k + d) * (p + 1) + d] : T(0));
    }
#pragma unroll
    for (int v = 0; v < K; ++v) {
      if (!(act >> v & 1)) continue;
      T* sv = sb + (size_t)v * n * kPLS;
      const double* rv = Pp.r + v * N;
      const T* iv = tin + v * N;
      if (a == 0) tile_walk(t, [&](int k, int l, long long g) { sv[k * kPLS + l] = (T)(rv[g] * Pp.scale[g]); });
      else tile_walk(t, [&](int k, int l, long long g) { sv[k * kPLS + l] = iv[g]; });
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < K && (act >> w & 1) && lane < t.nl) {
      T* sv = sb + (size_t)w * n * kPLS;
      switch (p) {
        case 2: solve_lines<2, T>(sv, sF, sG, n, lane); break;
        case 3: solve_lines<3, T>(sv, sF, sG, n, lane); break;
        case 4: solve_lines<4, T>(sv, sF, sG, n, lane); break;
        default: solve_lines<1, T>(sv, sF, sG, n, lane); break;
      }
    }
    __syncthreads();
    double snew[K], sold[K];
#pragma unroll
    for (int v = 0; v < K; ++v) {
      snew[v] = sold[v] = 0.0;
      if (!(act >> v & 1)) continue;
      const T* sv = sb + (size_t)v * n * kPLS;
      if (a == 2) {
        double* zv = Pp.z + v * N;
        const double* rv = Pp.r + v * N;
        double s1 = 0.0, s2 = 0.0;
        tile_walk(t, [&](int k, int l, long long g) {
          const double zn = (double)sv[k * kPLS + l] * Pp.scale[g];
          const double rg = rv[g];
          s2 = fma(rg, zv[g], s2);
          s1 = fma(rg, zn, s1);
          zv[g] = zn;
        });
        snew[v] = s1;
        sold[v] = s2;
      } else {
        T* ov = tout + v * N;
        tile_walk(t, [&](int k, int l, long long g) { ov[g] = sv[k * kPLS + l]; });
      }
    }
    if (a == 2) {
#pragma unroll
      for (int v = 0; v < K; ++v) {
        const double s1 = pblock_sum(snew[v]), s2 = pblock_sum(sold[v]);
        if (threadIdx.x == 0) {
          B.lpart[(long long)it * K + v] = s1;
          B.lpart[(long long)(B.nrzt + it) * K + v] = s2;
        }
      }
    }
  }
}

// One mode product of the fast-diagonalisation preconditioner for every active system
// of a line tile of axis a: out_line = Mat bf16(in_line), Mat = U_a^T (tr = 1) or U_a.
// stage 0: in = r D^-1/2 Dhat^1/2 (FP64 scaled, then FP32) -> t1 (axis 0, U^T)
// stage 1: t1 -> t2 (axis 1, U^T); stage 2: t2 -> t1 (axis 2, U^T) times 1 / Lambda
// stage 3: t1 -> t2 (axis 2, U); stage 4: t2 -> t1 (axis 1, U)
// stage 5: t1 -> z (axis 0, U) times D^-1/2 Dhat^1/2, with the partials of r.z (new, old).
// On the tensor cores by warp-level BF16 MMA (m16n8k16, FP32 accumulation): the block's
// product is out (n x 32K) = Mat (n x n) . in (n x 32K), 32K = 32 lines per active-or-not
// system. Shared memory holds Mat as BF16 rows sA[i][j] (copied from its padded image in
// HBM by 16-byte loads) and the inputs as BF16 rows per line sB[line][j], both padded
// with zeros to multiples of 16 and with a row stride of ceil16(n) + 8 elements
// (fragment loads free of bank conflicts), then per line the
// element of entry 0 and (stage 2) 1 / (Lambda_0 Lambda_1). Warp w takes the 16 x 8
// output tiles w, w + 8, ...; fragments are read with 4-byte loads.
constexpr int kFdPad = kPersistFdPad;  // BF16 elements added to each staged row

__host__ __device__ __forceinline__ int fd_round16(int n) { return (n + 15) & ~15; }

__device__ __forceinline__ void mma_bf16_16x8x16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                                 unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int K>
__device__ void ph_fd(const PBatch& B, int stage, unsigned char* smem) {
  const int a = stage < 3 ? stage : 5 - stage;
  const int tr = stage < 3 ? 1 : 0;
  constexpr int NL = 32 * K;  // staged lines: 32 per system
  for (int it = blockIdx.x; it < B.nlt[a]; it += gridDim.x) {
    const int2 tl = B.ltile[a][it];
    const int act = patch_active<K>(B, tl.x);
    if (!act) {
      if (stage == 5 && threadIdx.x < K) {
        B.lpart[(long long)it * K + threadIdx.x] = 0.0;
        B.lpart[(long long)(B.nrzt + it) * K + threadIdx.x] = 0.0;
      }
      continue;
    }
    const PPatch& Pp = B.pt[tl.x];
    const LineTile t = line_tile(Pp, a, tl.y);
    const int n = t.n, n16 = fd_round16(n), ld = n16 + kFdPad;
    const long long N = t.N;
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* sB = sA + (size_t)n16 * ld;
    long long* sbase = reinterpret_cast<long long*>(sB + (size_t)NL * ld);
    float* slam = reinterpret_cast<float*>(sbase + kPLines);
    const uint4* Mat = static_cast<const uint4*>(Pp.Ubf[a][tr]);  // the shared-memory image of sA
    // stages 1, 3, 5 read t1 and 2, 4 read t2; stages 1, 3 write t2 and 0, 2, 4 write t1
    const float* tin = (stage == 2 || stage == 4) ? static_cast<const float*>(Pp.t2) : static_cast<const float*>(Pp.t1);
    float* tout = (stage == 1 || stage == 3) ? static_cast<float*>(Pp.t2) : static_cast<float*>(Pp.t1);
    __syncthreads();  // the previous item's shared data is consumed
    {  // Mat: 16-byte copies of its padded image (n16 ld BF16 = a multiple of 16 bytes)
      uint4* dA = reinterpret_cast<uint4*>(sA);
      const int nq = n16 * ld * (int)sizeof(__nv_bfloat16) / 16;
      for (int e = threadIdx.x; e < nq; e += kPThreads) dA[e] = Mat[e];
    }
    for (int e = threadIdx.x; e < NL * (n16 - n); e += kPThreads) {  // the padding entries j >= n
      const int l = e / (n16 - n), j = n + (e - l * (n16 - n));
      sB[(size_t)l * ld + j] = __float2bfloat16(0.0f);
    }
    if (threadIdx.x < kPLines) {  // per line: the element of entry 0, 1 / (Lambda_0 Lambda_1)
      const int l = threadIdx.x;
      const long long rr = t.l0 + l;
      long long g0 = 0;
      float lam = 1.0f;
      if (l < t.nl) {
        if (a == 0) {
          g0 = rr * n;
        } else {
          const long long y = rr / t.A;
          g0 = (rr - y * t.A) + t.A * (long long)n * y;
        }
        if (stage == 2) lam = Pp.lam[0][(int)(rr % Pp.n[0])] * Pp.lam[1][(int)(rr / Pp.n[0])];
      }
      sbase[l] = g0;
      slam[l] = lam;
    }
#pragma unroll
    for (int v = 0; v < K; ++v) {
      if (!(act >> v & 1)) continue;
      __nv_bfloat16* sv = sB + (size_t)v * kPLines * ld;
      const double* rv = Pp.r + v * N;
      const float* iv = tin + v * N;
      if (stage == 0)
        tile_walk(t, [&](int k, int l, long long g) {
          sv[(size_t)l * ld + k] = __float2bfloat16((float)(rv[g] * Pp.scale[g]));
        });
      else
        tile_walk(t, [&](int k, int l, long long g) { sv[(size_t)l * ld + k] = __float2bfloat16(iv[g]); });
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    double snew[K], sold[K];
#pragma unroll
    for (int v = 0; v < K; ++v) snew[v] = sold[v] = 0.0;
    const int mt = n16 / 16, ntiles = mt * (NL / 8);
    for (int tile = w; tile < ntiles; tile += kPThreads / 32) {
      const int i0 = (tile % mt) * 16, c0 = (tile / mt) * 8;  // output rows i0.., lines c0..
      const int v = c0 / kPLines;
      if (!(act >> v & 1)) continue;  // warp-uniform
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const __nv_bfloat16* ar0 = sA + (size_t)(i0 + gid) * ld + 2 * tig;
      const __nv_bfloat16* ar1 = ar0 + 8 * ld;
      const __nv_bfloat16* br = sB + (size_t)(c0 + gid) * ld + 2 * tig;
      for (int k0 = 0; k0 < n16; k0 += 16) {
        const unsigned a0 = *reinterpret_cast<const unsigned*>(ar0 + k0);
        const unsigned a1 = *reinterpret_cast<const unsigned*>(ar1 + k0);
        const unsigned a2 = *reinterpret_cast<const unsigned*>(ar0 + k0 + 8);
        const unsigned a3 = *reinterpret_cast<const unsigned*>(ar1 + k0 + 8);
        const unsigned b0 = *reinterpret_cast<const unsigned*>(br + k0);
        const unsigned b1 = *reinterpret_cast<const unsigned*>(br + k0 + 8);
        mma_bf16_16x8x16(acc, a0, a1, a2, a3, b0, b1);
      }
      // acc[q]: output row i0 + gid (+ 8 for q >= 2), line c0 + 2 tig (+ 1 for odd q)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + gid + (q >= 2 ? 8 : 0);
        const int l = (c0 + 2 * tig + (q & 1)) - v * kPLines;
        if (i >= n || l >= t.nl) continue;
        const long long g = sbase[l] + (a == 0 ? 1LL : t.A) * i;
        if (stage == 5) {
          const double zn = (double)acc[q] * Pp.scale[g];
          const double rg = Pp.r[v * N + g];
#pragma unroll
          for (int u = 0; u < K; ++u)
            if (u == v) {
              sold[u] = fma(rg, Pp.z[v * N + g], sold[u]);
              snew[u] = fma(rg, zn, snew[u]);
            }
          Pp.z[v * N + g] = zn;
        } else {
          tout[v * N + g] = stage == 2 ? acc[q] * (slam[l] * Pp.lam[2][i]) : acc[q];
        }
      }
    }
    if (stage == 5) {
#pragma unroll
      for (int v = 0; v < K; ++v) {
        const double s1 = pblock_sum(snew[v]), s2 = pblock_sum(sold[v]);
        if (threadIdx.x == 0) {
          B.lpart[(long long)it * K + v] = s1;
          B.lpart[(long long)(B.nrzt + it) * K + v] = s2;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- scalar updates (block 0)
// start: ||b||^2, ||r||^2 = ||b||^2, activity, counters
__device__ void lead_start(const PBatch& B) {
  for (int s = threadIdx.x; s < B.np * B.k; s += kPThreads) {
    B.rr[s] = B.bb[s];
    B.active[s] = B.bb[s] > 0.0 ? 1 : 0;
    B.iters[s] = 0;
  }
}

// after the preconditioner: r.z, and beta for the next direction (plain or flexible)
__device__ void lead_rz(const PBatch& B, bool first) {
  for (int s = threadIdx.x; s < B.np * B.k; s += kPThreads) {
    if (!B.active[s]) continue;
    if (!first) {
      const double num = B.flexible ? B.rznew[s] - B.rzold[s] : B.rznew[s];
      B.beta[s] = num / B.rz[s];
    }
    B.rz[s] = B.rznew[s];
  }
}

// after q = M p: alpha = r.z / p.q (breakdown stops the system)
__device__ void lead_alpha(const PBatch& B) {
  for (int s = threadIdx.x; s < B.np * B.k; s += kPThreads) {
    if (!B.active[s]) continue;
    const double pq = B.pq[s];
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(B.rz[s])) {
      B.active[s] = 0;
      B.status[s] = 1;
      B.alpha[s] = 0.0;
    } else {
      B.alpha[s] = B.rz[s] / pq;
    }
  }
}

// after the x, r update: ||r||^2, iteration count, convergence; flags[0] = any active
__device__ void lead_check(const PBatch& B) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < B.np * B.k; s += kPThreads) {
    if (!B.active[s]) continue;
    const int it = B.iters[s] + 1;
    B.iters[s] = it;
    if (B.rr[s] <= B.tol2 * B.bb[s]) {
      B.active[s] = 0;
    } else if (it >= B.max_iter) {
      B.active[s] = 0;
      B.status[s] = 2;
    } else {
      atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) B.flags[0] = any;
}

// end of a step: iteration statistics
__device__ void lead_stats(const PBatch& B) {
  for (int s = threadIdx.x; s < B.np * B.k; s += kPThreads) {
    B.tot_iters[s] += B.iters[s];
    B.max_iters[s] = max(B.max_iters[s], B.iters[s]);
    const double rel = B.bb[s] > 0.0 ? sqrt(B.rr[s] / B.bb[s]) : 0.0;
    B.last_rel[s] = rel;
    if (B.status[s]) B.flags[1] = B.status[s];
  }
}

// Phase clock: block 0 adds the time since its previous mark to B.ptime[cat] once a
// phase's grid barrier has passed (the barrier passes when the last block arrives, so
// the interval is the phase's duration on the whole grid, barrier included).
enum PhaseCat { kPhPredict, kPhKProduct, kPhScalars, kPhPrecond, kPhDirection, kPhMProduct, kPhXr, kPhUpdate };

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void pmark(const PBatch& B, int cat, unsigned long long& last) {
  if (B.ptime && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long now = gtimer();
    B.ptime[cat] += now - last;
    last = now;
  }
}

// the preconditioner z = P^-1 r (three axis phases) and the r.z scalars
template <int K, typename T>
__device__ bool pprecond(const PBatch& B, unsigned char* smem, bool first, unsigned long long& clk) {
  if (B.fd) {
    for (int st = 0; st < 6; ++st) {
      ph_fd<K>(B, st, smem);
      if (!pgrid_sync(B.bar, B.bar_limit, B.err)) return false;
      pmark(B, kPhPrecond, clk);
    }
  } else {
    for (int a = 0; a < 3; ++a) {
      ph_axis<K, T>(B, a, smem);
      if (!pgrid_sync(B.bar, B.bar_limit, B.err)) return false;
      pmark(B, kPhPrecond, clk);
    }
  }
  psum_phase(B, B.lpart, B.lt2, B.nlt2_p, B.rznew);
  psum_phase(B, B.lpart + (long long)B.nrzt * B.k, B.lt2, B.nlt2_p, B.rzold);
  if (!pgrid_sync(B.bar, B.bar_limit, B.err)) return false;
  if (blockIdx.x == 0) lead_rz(B, first);
  if (!pgrid_sync(B.bar, B.bar_limit, B.err)) return false;
  pmark(B, kPhScalars, clk);
  return true;
}

template <int K, typename T, int SLOTS, int MINB>
__global__ void __launch_bounds__(kPThreads, MINB) k_batch_step(const PBatch B) {
  extern __shared__ __align__(16) unsigned char psmem[];
  unsigned long long clk = (B.ptime && blockIdx.x == 0 && threadIdx.x == 0) ? gtimer() : 0ULL;
#define IGA_PSYNC(cat)                                         \
  do {                                                         \
    if (!pgrid_sync(B.bar, B.bar_limit, B.err)) return;        \
    pmark(B, cat, clk);                                        \
  } while (0)
  ph_predict<K>(B);
  IGA_PSYNC(kPhPredict);
  // b = K (-Y) into r (x0 = 0: r = b), partials of b.b
  ph_band<K, SLOTS>(B, true, B.Yp, B.rp, 2, B.part);
  IGA_PSYNC(kPhKProduct);
  psum_phase(B, B.part, B.rt0, B.nrt_p, B.bb);
  IGA_PSYNC(kPhScalars);
  if (blockIdx.x == 0) lead_start(B);
  IGA_PSYNC(kPhScalars);
  if (!pprecond<K, T>(B, psmem, true, clk)) return;
  bool first = true;
  for (int iter = 0;; ++iter) {
    ph_dir<K>(B, first);
    first = false;
    IGA_PSYNC(kPhDirection);
    ph_band<K, SLOTS>(B, false, B.pp, B.qp, 1, B.part);  // q = M p, partials of p.q
    IGA_PSYNC(kPhMProduct);
    psum_phase(B, B.part, B.rt0, B.nrt_p, B.pq);
    IGA_PSYNC(kPhScalars);
    if (blockIdx.x == 0) lead_alpha(B);
    IGA_PSYNC(kPhScalars);
    ph_xr<K>(B);
    IGA_PSYNC(kPhXr);
    psum_phase(B, B.part, B.rt0, B.nrt_p, B.rr);
    IGA_PSYNC(kPhScalars);
    if (blockIdx.x == 0) lead_check(B);
    IGA_PSYNC(kPhScalars);
    if (*(volatile int*)&B.flags[0] == 0) break;  // the same value in every block
    if (!pprecond<K, T>(B, psmem, false, clk)) return;
  }
#undef IGA_PSYNC
  ph_update<K>(B);
  if (blockIdx.x == 0) lead_stats(B);
  pmark(B, kPhUpdate, clk);  // block 0's own end
}

template <int K, typename T, int SLOTS, int MINB>
cudaError_t batch_go(cudaStream_t s, const PBatch& B, size_t smem, int sms, int* grid_out) {
  auto kern = k_batch_step<K, T, SLOTS, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kPThreads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const int grid = per * sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (grid_out) *grid_out = grid;
  return cudaLaunchKernelEx(&cfg, kern, B);
}

}  // namespace

int batch_row_tiles(long long N) { return (int)((N + kPRows - 1) / kPRows); }
int batch_line_tiles(long long N, int n) { return (int)((N / n + kPLines - 1) / kPLines); }
size_t batch_smem_bytes(int nmax, int pmax, int k, bool f32, bool fd) {
  if (fd)  // Mat and the lines as BF16 rows, then the per-line bases and 1 / Lambda
    return ((size_t)fd_round16(nmax) + 32 * (size_t)k) * (fd_round16(nmax) + kFdPad) * sizeof(__nv_bfloat16) +
           kPLines * (sizeof(long long) + sizeof(float)) + 64;
  return (size_t)nmax * (2 * (pmax + 1) + (size_t)k * kPLS) * (f32 ? sizeof(float) : sizeof(double)) + 64;
}

cudaError_t launch_batch_step(cudaStream_t s, const PBatch& B, bool f32, size_t smem, int variant, int* grid) {
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  // variant 0: three blocks per SM (80 registers), two slots per band pass; variant 1: two
  // blocks per SM (128 registers), four slots per band pass (k <= 2; else as variant 0)
#define IGA_BGV(KK, S, M) \
  return f32 ? batch_go<KK, float, S, M>(s, B, smem, sms, grid) : batch_go<KK, double, S, M>(s, B, smem, sms, grid)
  switch (B.k) {
    case 1:
      if (variant == 1) IGA_BGV(1, 4, 2);
      IGA_BGV(1, 2, 3);
    case 2:
      if (variant == 1) IGA_BGV(2, 4, 2);
      IGA_BGV(2, 2, 3);
    case 3: IGA_BGV(3, 2, 3);
    case 4: IGA_BGV(4, 2, 3);
    default: return cudaErrorInvalidValue;
  }
#undef IGA_BGV
}

}  // namespace iga
