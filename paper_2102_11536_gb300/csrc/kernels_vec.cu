// PCG vector kernels (Sec. 5.5) and the fused generalized-alpha predictor and
// stage update (Sec. 4, eq. ho1-ho3). Reductions use a fixed grid and a fixed
// tree, so every result is bitwise reproducible run to run.
#include "iga_internal.h"

namespace iga {

// block of 256 threads -> one value (valid in thread 0)
__device__ __forceinline__ double block_sum256(double v) {
  __shared__ double sh[8];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < 8 ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_dot(long long N, const double* __restrict__ a, const double* __restrict__ b,
                                             long long vs, double* __restrict__ partial) {
  const int v = blockIdx.y;
  const double* pa = a + v * vs;
  const double* pb = b + v * vs;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    s = fma(pa[i], pb[i], s);
  s = block_sum256(s);
  if (threadIdx.x == 0) partial[v * kRedBlocks + blockIdx.x] = s;
}

cudaError_t launch_dot(cudaStream_t s, long long N, int nvec, const double* a, const double* b, long long vs,
                       double* partial) {
  k_dot<<<dim3(kRedBlocks, nvec), 256, 0, s>>>(N, a, b, vs, partial);
  return cudaGetLastError();
}

constexpr int kEpiThreads = 32 * kMaxVec;

__global__ void __launch_bounds__(kEpiThreads) k_reduce(int nvec, const double* partial, double* result) {
  __shared__ double sa[kMaxVec];
  reduce_partials(nvec, partial, sa, kRedBlocks);
  const int v = threadIdx.x;
  if (v < nvec) result[v] = sa[v];
}

cudaError_t launch_reduce(cudaStream_t s, int nvec, const double* partial, double* result) {
  k_reduce<<<1, kEpiThreads, 0, s>>>(nvec, partial, result);
  return cudaGetLastError();
}

// b.b and r.r at the start; a system is active while ||r|| > tol ||b|| and b != 0.
__global__ void __launch_bounds__(kEpiThreads) k_cg_init(int nvec, const double* pbb, const double* prr, CgScalars c,
                                                         double tol2) {
  __shared__ double sb[kMaxVec], sr[kMaxVec];
  reduce_partials(nvec, pbb, sb, kRedBlocks);
  reduce_partials(nvec, prr, sr, kRedBlocks);
  const int v = threadIdx.x;
  if (v < nvec) {
    const double bb = sb[v], rr = sr[v];
    c.bb[v] = bb;
    c.rr[v] = rr;
    c.rr0[v] = rr;
    c.iters[v] = 0;
    c.status[v] = 0;
    int act = (bb > 0.0) && (rr > tol2 * bb);
    if (!isfinite(bb) || !isfinite(rr)) {
      c.status[v] = IGA_ENUMERIC;
      act = 0;
    }
    c.active[v] = act;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int i = 0; i < nvec; ++i) na += c.active[i];
    *c.nactive = na;
  }
}

cudaError_t launch_cg_init(cudaStream_t s, int nvec, const double* partial_bb, const double* partial_rr,
                           CgScalars c, double tol2) {
  k_cg_init<<<1, kEpiThreads, 0, s>>>(nvec, partial_bb, partial_rr, c, tol2);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kEpiThreads) k_cg_start(int nvec, const double* prz, int np, CgScalars c) {
  __shared__ double sz[kMaxVec];
  reduce_partials(nvec, prz, sz, np);
  const int v = threadIdx.x;
  if (v < nvec) c.rz[v] = sz[v];
}

cudaError_t launch_cg_start(cudaStream_t s, int nvec, const double* partial_rz, int np, CgScalars c) {
  k_cg_start<<<1, kEpiThreads, 0, s>>>(nvec, partial_rz, np, c);
  return cudaGetLastError();
}

// alpha = r.z / p.q; breakdown (p.q <= 0 or not finite) stops the system with IGA_ENUMERIC.
// p.q comes from the band product's per-block partials (N / 128 of them per vector): block
// (b, v) sums the b-th of kAlphaBlocks contiguous chunks of vector v's partials (a fixed
// strided share per thread, then the block tree), and the last block to finish (arrival
// counter c.ticket[1]) adds the chunks' sums in chunk order and sets alpha.
constexpr int kAlphaBlocks = 64;
__global__ void __launch_bounds__(256) k_cg_alpha(int nvec, const double* ppq, int np, CgScalars c) {
  const int v = blockIdx.y, b = blockIdx.x;
  const int chunk = (np + kAlphaBlocks - 1) / kAlphaBlocks;
  const int lo = b * chunk, hi = min(np, lo + chunk);
  double s = 0.0;
#pragma unroll 4
  for (int i = lo + threadIdx.x; i < hi; i += 256) s += __ldcg(&ppq[(long long)v * np + i]);
  s = block_sum256(s);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    c.red[v * kAlphaBlocks + b] = s;
    __threadfence();
    last = atomicAdd(&c.ticket[1], 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int u = threadIdx.x;
  if (u < nvec) {
    double pq = 0.0;
    for (int q = 0; q < kAlphaBlocks; ++q) pq += __ldcg(&c.red[u * kAlphaBlocks + q]);
    if (!c.active[u]) {
      c.alpha[u] = 0.0;
    } else if (!(pq > 0.0) || !isfinite(pq)) {
      c.status[u] = IGA_ENUMERIC;
      c.active[u] = 0;
      c.alpha[u] = 0.0;
    } else {
      c.alpha[u] = c.rz[u] / pq;
    }
  }
  if (threadIdx.x == 0) atomicExch(&c.ticket[1], 0u);  // ready for the next launch
}

cudaError_t launch_cg_alpha(cudaStream_t s, int nvec, const double* partial, int np, CgScalars c) {
  k_cg_alpha<<<dim3(kAlphaBlocks, nvec), 256, 0, s>>>(nvec, partial, np, c);
  return cudaGetLastError();
}

// After x/r update: count the iteration, test ||r||^2 <= tol^2 ||b||^2 (by one block of
// kEpiThreads threads: a kernel of its own, or the last block of the x, r update).
__device__ void cg_check_block(int nvec, const double* prr, CgScalars c, double tol2) {
  __shared__ double sr[kMaxVec];
  reduce_partials(nvec, prr, sr, kRedBlocks);
  const int v = threadIdx.x;
  if (v < nvec && c.active[v]) {
    const double rr = sr[v];
    c.rr[v] = rr;
    c.iters[v] += 1;
    if (!isfinite(rr)) {
      c.status[v] = IGA_ENUMERIC;
      c.active[v] = 0;
    } else if (rr <= tol2 * c.bb[v]) {
      c.active[v] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int i = 0; i < nvec; ++i) na += c.active[i];
    *c.nactive = na;
  }
}

__global__ void __launch_bounds__(kEpiThreads) k_cg_check(int nvec, const double* prr, CgScalars c, double tol2) {
  cg_check_block(nvec, prr, c, tol2);
}

cudaError_t launch_cg_check(cudaStream_t s, int nvec, const double* partial, CgScalars c, double tol2) {
  k_cg_check<<<1, kEpiThreads, 0, s>>>(nvec, partial, c, tol2);
  return cudaGetLastError();
}

// beta = r.z_new / r.z_old (plain CG) or (r.z_new - r.z_prev) / r.z_old (flexible,
// Polak-Ribiere form for a preconditioner that is not exactly linear).
__global__ void __launch_bounds__(kEpiThreads) k_cg_beta(int nvec, const double* prz, const double* prz2, int np,
                                                         CgScalars c, int flexible) {
  __shared__ double sz[kMaxVec], sz2[kMaxVec];
  reduce_partials(nvec, prz, sz, np);
  if (flexible) reduce_partials(nvec, prz2, sz2, np);
  const int v = threadIdx.x;
  if (v >= nvec || !c.active[v]) return;
  const double rz_new = sz[v];
  double num = rz_new;
  if (flexible) num -= sz2[v];
  c.beta[v] = num / c.rz[v];
  c.rz[v] = rz_new;
}

cudaError_t launch_cg_beta(cudaStream_t s, int nvec, const double* partial, const double* partial2, int np,
                           CgScalars c, int flexible) {
  k_cg_beta<<<1, kEpiThreads, 0, s>>>(nvec, partial, partial2, np, c, flexible);
  return cudaGetLastError();
}

// x += alpha p, r -= alpha q (active systems), per-block partials of r.r; with check, the
// last block to finish (arrival counter c.ticket) runs the convergence test on them.
__global__ void __launch_bounds__(256) k_cg_update_xr(long long N, CgScalars c, double* __restrict__ x,
                                                      double* __restrict__ r, const double* __restrict__ p,
                                                      const double* __restrict__ q, long long vs,
                                                      double* __restrict__ partial, int check, double tol2) {
  const int v = blockIdx.y;
  const double a = c.alpha[v];
  const bool act = c.active[v] != 0;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const long long k = v * vs + i;
    double ri = r[k];
    if (act) {
      x[k] = fma(a, p[k], x[k]);
      ri = fma(-a, q[k], ri);
      r[k] = ri;
    }
    s = fma(ri, ri, s);
  }
  s = block_sum256(s);
  if (threadIdx.x == 0) partial[v * kRedBlocks + blockIdx.x] = s;
  if (!check) return;
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // the partial is visible before the arrival
    last = atomicAdd(&c.ticket[0], 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  cg_check_block((int)gridDim.y, partial, c, tol2);
  if (threadIdx.x == 0) atomicExch(&c.ticket[0], 0u);  // ready for the next launch
}

cudaError_t launch_cg_update_xr(cudaStream_t s, long long N, int nvec, CgScalars c, double* x, double* r,
                                const double* p, const double* q, long long vs, double* partial, int check,
                                double tol2) {
  static_assert(kEpiThreads == 256, "the fused convergence test runs in a 256-thread block");
  k_cg_update_xr<<<dim3(kRedBlocks, nvec), 256, 0, s>>>(N, c, x, r, p, q, vs, partial, check, tol2);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_cg_update_p(long long N, CgScalars c, double* __restrict__ p,
                                                     const double* __restrict__ z, long long vs) {
  const int v = blockIdx.y;
  if (!c.active[v]) return;
  const double b = c.beta[v];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const long long k = v * vs + i;
    p[k] = fma(b, p[k], z[k]);
  }
}

cudaError_t launch_cg_update_p(cudaStream_t s, long long N, int nvec, CgScalars c, double* p, const double* z,
                               long long vs) {
  k_cg_update_p<<<dim3(kRedBlocks, nvec), 256, 0, s>>>(N, c, p, z, vs);
  return cudaGetLastError();
}

__global__ void k_sub(long long N, const double* b, const double* q, double* r, long long vs) {
  const int v = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    r[v * vs + i] = b[v * vs + i] - q[v * vs + i];
}

cudaError_t launch_sub(cudaStream_t s, long long N, int nvec, const double* b, const double* q, double* r,
                       long long vs) {
  k_sub<<<dim3(kRedBlocks, nvec), 256, 0, s>>>(N, b, q, r, vs);
  return cudaGetLastError();
}

__global__ void k_copy_active(long long N, const int* active, const double* src, double* dst, long long vs) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    dst[v * vs + i] = src[v * vs + i];
}

cudaError_t launch_copy_active(cudaStream_t s, long long N, int nvec, const int* active, const double* src,
                               double* dst, long long vs) {
  k_copy_active<<<dim3(kRedBlocks, nvec), 256, 0, s>>>(N, active, src, dst, vs);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// generalized-alpha predictor and stage update. Rows of X: q + 2 for
// q = -2..3k-3 (U, V, A, L^1, ...). c[m] = tau^m / m!.
// T_q = sum_{r >= q} c[r-q] X_r (Taylor predictor, eq. ho2-ho3).
// Block j solves for row s_j + 2 = 3j - 1 (0-based j-1: row 3(j-1) + 2).
// ----------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) k_predict(long long N, StepCoefs sc, const double* __restrict__ X,
                                                 double* __restrict__ Yneg, double* __restrict__ T,
                                                 double* __restrict__ Yv) {
  constexpr int R = 3 * K;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = X[r * N + i];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int row = 3 * j + 2;   // solved variable of block j+1
    const int ry = row - 2;      // its "displacement" row
    double y;
    if (j < K - 1) {             // alpha_f = 1: full Taylor predictor T_{s_j - 2}
      y = 0.0;
#pragma unroll
      for (int r = R - 1; r >= ry; --r) y = fma(sc.c[r - ry], x[r], y);
    } else {                     // alpha_f = 0: the current value
      y = x[ry];
    }
    if (sc.damped) {             // the same for the velocity-like row ry + 1
      double yv;
      if (j < K - 1) {
        yv = 0.0;
#pragma unroll
        for (int r = R - 1; r >= ry + 1; --r) yv = fma(sc.c[r - ry - 1], x[r], yv);
      } else {
        yv = x[ry + 1];
      }
      y = fma(sc.aK, yv, y);
      if (Yv) Yv[j * N + i] = -yv;
    }
    Yneg[j * N + i] = -y;
    if (T) {
      double t = 0.0;
#pragma unroll
      for (int r = R - 1; r >= row; --r) t = fma(sc.c[r - row], x[r], t);
      T[j * N + i] = t;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_update(long long N, StepCoefs sc, double* __restrict__ X,
                                                const double* __restrict__ Z) {
  constexpr int R = 3 * K;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[R], t[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = X[r * N + i];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    double s = 0.0;
#pragma unroll
    for (int r = R - 1; r >= q; --r) s = fma(sc.c[r - q], x[r], s);
    t[q] = s;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int row = 3 * j + 2;
    const double P = (Z[j * N + i] - t[row]) * sc.ralpha[j];
    X[row * N + i] = t[row] + P;
    X[(row - 1) * N + i] = fma(sc.gtau[j], P, t[row - 1]);
    X[(row - 2) * N + i] = fma(sc.btau2[j], P, t[row - 2]);
  }
}

cudaError_t launch_predict(cudaStream_t s, long long N, StepCoefs sc, const double* X, double* Yneg, double* T,
                           double* Yv) {
  const unsigned blocks = (unsigned)((N + 255) / 256);
  switch (sc.k) {
    case 1: k_predict<1><<<blocks, 256, 0, s>>>(N, sc, X, Yneg, T, Yv); break;
    case 2: k_predict<2><<<blocks, 256, 0, s>>>(N, sc, X, Yneg, T, Yv); break;
    case 3: k_predict<3><<<blocks, 256, 0, s>>>(N, sc, X, Yneg, T, Yv); break;
    case 4: k_predict<4><<<blocks, 256, 0, s>>>(N, sc, X, Yneg, T, Yv); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_update(cudaStream_t s, long long N, StepCoefs sc, double* X, const double* Z) {
  const unsigned blocks = (unsigned)((N + 255) / 256);
  switch (sc.k) {
    case 1: k_update<1><<<blocks, 256, 0, s>>>(N, sc, X, Z); break;
    case 2: k_update<2><<<blocks, 256, 0, s>>>(N, sc, X, Z); break;
    case 3: k_update<3><<<blocks, 256, 0, s>>>(N, sc, X, Z); break;
    case 4: k_update<4><<<blocks, 256, 0, s>>>(N, sc, X, Z); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Loads of the stage equations: the time derivatives of F(t) = sum_m G_m sin(om_m t + ph_m)
// are closed forms, d^s/dt^s sin(w t + p) = w^s sin(w t + p + s pi/2).
__global__ void __launch_bounds__(256) k_stage_load(long long N, StageLoad a, const double* __restrict__ G,
                                                    const double* __restrict__ time,
                                                    const double* __restrict__ MYv, double* __restrict__ rhs) {
  __shared__ double coef[kMaxK * kMaxForce];
  const int tid = threadIdx.x;
  if (tid < a.nstage * a.nterm) {
    const int j = tid / a.nterm, m = tid - j * a.nterm;
    const int sd = a.sder[j];
    const double t = *time + a.toff[j];
    double w = 1.0;
    for (int q = 0; q < sd; ++q) w *= a.om[m];
    coef[tid] = w * sin(a.om[m] * t + a.ph[m] + sd * 1.5707963267948966);
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + tid; i < N; i += (long long)gridDim.x * blockDim.x)
    for (int j = 0; j < a.nstage; ++j) {
      double r = rhs[j * N + i];
      if (MYv) r = fma(a.aM, MYv[j * N + i], r);
      for (int m = 0; m < a.nterm; ++m) r = fma(coef[j * a.nterm + m], G[m * N + i], r);
      rhs[j * N + i] = r;
    }
}

cudaError_t launch_stage_load(cudaStream_t s, long long N, StageLoad a, const double* G, const double* time,
                              const double* MYv, double* rhs) {
  if (a.nstage < 1 || a.nstage > kMaxK || a.nterm < 0 || a.nterm > kMaxForce) return cudaErrorInvalidValue;
  k_stage_load<<<kRedBlocks, 256, 0, s>>>(N, a, G, time, MYv, rhs);
  return cudaGetLastError();
}

__global__ void k_advance_time(double* time, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *time += dt;
}

cudaError_t launch_advance_time(cudaStream_t s, double* time, double dt) {
  k_advance_time<<<1, 32, 0, s>>>(time, dt);
  return cudaGetLastError();
}

__global__ void k_lincomb(long long n, double ca, const double* __restrict__ a, double cb,
                          const double* __restrict__ b, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = fma(ca, a[i], cb * b[i]);
}

cudaError_t launch_lincomb(cudaStream_t s, long long n, double ca, const double* a, double cb, const double* b,
                           double* out) {
  k_lincomb<<<kRedBlocks, 256, 0, s>>>(n, ca, a, cb, b, out);
  return cudaGetLastError();
}

__global__ void k_extrap(long long n, double* Z, double* Z2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double z = Z[i];
    Z[i] = 2.0 * z - Z2[i];
    Z2[i] = z;
  }
}

cudaError_t launch_extrap(cudaStream_t s, long long n, double* Z, double* Z2) {
  k_extrap<<<kRedBlocks, 256, 0, s>>>(n, Z, Z2);
  return cudaGetLastError();
}

__global__ void k_scale_neg(long long n, double* x) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = -x[i];
}

cudaError_t launch_scale_neg(cudaStream_t s, long long n, double* x) {
  k_scale_neg<<<kRedBlocks, 256, 0, s>>>(n, x);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// device-side PCG loop of the captured step graph
// ----------------------------------------------------------------------------
// loop[0]: iterations of the current solve, loop[1]: body executions summed over
// the solves since the last reset. The while node runs its body as long as the
// value set here is non-zero: some system still active and max_iter not reached.
__global__ void k_set_cond(cudaGraphConditionalHandle hc, const int* nactive, int* loop, int max_iter, int reset) {
  if (reset) {
    loop[0] = 0;
  } else {
    loop[0] += 1;
    loop[1] += 1;
  }
  cudaGraphSetConditional(hc, (*nactive > 0 && loop[0] < max_iter) ? 1u : 0u);
}

cudaError_t launch_set_cond(cudaStream_t s, cudaGraphConditionalHandle hc, const int* nactive, int* loop, int max_iter,
                            int reset) {
  k_set_cond<<<1, 1, 0, s>>>(hc, nactive, loop, max_iter, reset);
  return cudaGetLastError();
}

// After a solve: total and largest iteration counts per system slot, the first
// error status, and whether any system stopped unconverged.
__global__ void k_accum(int nvec, CgScalars c, long long* tot, int* mx, double* init, int* stat) {
  const int v = threadIdx.x;
  if (v < nvec) {
    tot[v] += c.iters[v];
    if (c.bb[v] > 0.0) init[v] += sqrt(c.rr0[v] / c.bb[v]);
    if (c.iters[v] > mx[v]) mx[v] = c.iters[v];
    if (c.status[v] != 0) atomicCAS(stat, 0, c.status[v]);
  }
  if (v == 0 && *c.nactive > 0) stat[1] = 1;
}

cudaError_t launch_accum(cudaStream_t s, int nvec, CgScalars c, long long* tot, int* mx, double* init, int* stat) {
  k_accum<<<1, 32, 0, s>>>(nvec, c, tot, mx, init, stat);
  return cudaGetLastError();
}

}  // namespace iga
