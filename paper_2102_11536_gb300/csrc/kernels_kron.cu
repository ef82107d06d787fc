// Kronecker solve of the preconditioner (Sec. 5.3, def:single_patch_prec) by band
// Cholesky: (Mhat_1 x Mhat_2 x Mhat_3)^{-1} is the product of the univariate
// inverses applied along each direction, and Mhat_a = L_a L_a^T is banded with half
// bandwidth p, so each line along axis a is solved by a forward and a backward
// substitution of p terms per entry (about 4 (p+1) flops per entry and axis, the
// O(N) cost of the paper's Kronecker solvers).
//
// One block of kThreads threads takes kLines lines: all threads stage them in shared
// memory (element (k, line) at k * kLS + line; reads coalesced along the lines
// for axis 0, where a block's lines are one contiguous range, and across the lines
// for the other axes; several loads in flight per thread), the first kLines threads
// run the two substitutions, one line each (with the factor rows pre-scaled by
// 1 / L_kk and the recurrence window in registers), and all threads write the lines
// back the same way. pre multiplies the
// input entries (the first axis: D^{-1/2} Dhat^{1/2}), post the output entries
// (the last axis).
#include "iga_internal.h"


namespace iga {

namespace {

constexpr int kLines = 32;    // lines per block (one warp solves them)
constexpr int kLS = kLines + 1;  // shared row stride: odd, so that both the staging walks
                                 // (consecutive entries of a line) and the solve
                                 // (consecutive lines) are free of bank conflicts
constexpr int kThreads = 256; // threads staging and writing back

// P = p: entries below the diagonal in a row of the factor; T: arithmetic (double, or
// float for the FP32 form); TI / TO: input / output element types. pre / post are
// applied in FP64 before rounding to T / after widening from T.
// rdot (nullable, FP64 output only): also the per-block partials of rdot . out (new) and
// rdot . out (the values out held before: the previous z of flexible PCG) into
// part[v * gridDim.x + b] and part[(gridDim.y + v) * gridDim.x + b].
template <int P, typename T, typename TI, typename TO>
__global__ void __launch_bounds__(kThreads) k_kron_axis(int n, long long A, long long R, const T* __restrict__ L,
                                                      const T* __restrict__ dinv, const int* __restrict__ active,
                                                      const TI* __restrict__ in, TO* __restrict__ out,
                                                      long long vs, const double* __restrict__ pre,
                                                      const double* __restrict__ post,
                                                      const double* __restrict__ rdot, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char kron_smem[];
  // [n][kLS] lines, then the scaled factor rows for the forward [n][P+1] and the
  // backward [n][P+1] substitution
  T* sb = reinterpret_cast<T*>(kron_smem);
  T* sF = sb + (size_t)n * kLS;
  T* sG = sF + (size_t)n * (P + 1);
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const long long l0 = (long long)blockIdx.x * kLines;
  const int nl = (int)min((long long)kLines, R - l0);
  const int t = threadIdx.x;
  const TI* x = in + v * vs;
  TO* o = out + v * vs;
  const int cnt = nl * n;
  // forward  w_k = d_k s_k - sum_d (d_k L_{k,k-d}) w_{k-d},
  // backward z_k = d_k w_k - sum_d (d_k L_{k+d,k}) z_{k+d},   d_k = 1 / L_kk
  for (int e = t; e < n * (P + 1); e += kThreads) {
    const int k = e / (P + 1), d = e - k * (P + 1);
    const T dk = dinv[k];
    sF[e] = d == 0 ? dk : dk * L[e];
    sG[e] = d == 0 ? dk : (k + d < n ? dk * L[(size_t)(k + d) * (P + 1) + d] : T(0));
  }
  // stage (the (entry, line) walks are incremental: no division per element)
  const int dl = kThreads / n, dk = kThreads - dl * n;  // axis 0: e -> e + kThreads
  long long gline = 0;                                  // other axes, full blocks: line t % kLines
  if (A != 1 && nl == kLines) {
    const long long rr = l0 + (t & (kLines - 1));
    const long long y = rr / A;
    gline = (rr - y * A) + A * (long long)n * y;
  }
  if (A == 1) {
    const long long g0 = l0 * n;  // the block's lines are one contiguous range
    int line = t / n, k = t - (t / n) * n;
#pragma unroll 4
    for (int e = t; e < cnt; e += kThreads) {
      double u = (double)x[g0 + e];
      if (pre) u *= pre[g0 + e];
      sb[k * kLS + line] = (T)u;
      k += dk;
      line += dl;
      if (k >= n) {
        k -= n;
        ++line;
      }
    }
  } else if (nl == kLines) {
    const int line = t & (kLines - 1);
#pragma unroll 4
    for (int k = t / kLines; k < n; k += kThreads / kLines) {
      const long long g = gline + A * k;
      double u = (double)x[g];
      if (pre) u *= pre[g];
      sb[k * kLS + line] = (T)u;
    }
  } else {
    for (int e = t; e < cnt; e += kThreads) {
      const int k = e / nl, line = e - k * nl;
      const long long rr = l0 + line;
      const long long y = rr / A, xx = rr - y * A;
      const long long g = xx + A * (k + (long long)n * y);
      double u = (double)x[g];
      if (pre) u *= pre[g];
      sb[k * kLS + line] = (T)u;
    }
  }
  __syncthreads();
  if (t < nl) {
    // The last P values of the recurrence stay in registers (win[d] = value d steps
    // back; zero before the line's start, where the factor entries are zero too), and
    // the terms not involving the previous value are summed first, so one multiply-add
    // per step lies on the dependency chain.
    T win[P + 1];
#pragma unroll
    for (int d = 0; d <= P; ++d) win[d] = T(0);
#pragma unroll 4
    for (int k = 0; k < n; ++k) {
      const T* F = sF + (size_t)k * (P + 1);
      T acc = F[0] * sb[k * kLS + t];
#pragma unroll
      for (int d = P; d >= 2; --d) acc -= F[d] * win[d];
      const T w = acc - F[1] * win[1];
      sb[k * kLS + t] = w;
#pragma unroll
      for (int d = P; d >= 2; --d) win[d] = win[d - 1];
      win[1] = w;
    }
#pragma unroll
    for (int d = 0; d <= P; ++d) win[d] = T(0);
#pragma unroll 4
    for (int k = n - 1; k >= 0; --k) {
      const T* G = sG + (size_t)k * (P + 1);
      T acc = G[0] * sb[k * kLS + t];
#pragma unroll
      for (int d = P; d >= 2; --d) acc -= G[d] * win[d];
      const T z = acc - G[1] * win[1];
      sb[k * kLS + t] = z;
#pragma unroll
      for (int d = P; d >= 2; --d) win[d] = win[d - 1];
      win[1] = z;
    }
  }
  __syncthreads();
  // write back
  const double* rv = rdot ? rdot + v * vs : nullptr;
  double snew = 0.0, sold = 0.0;
  if (A == 1) {
    const long long g0 = l0 * n;
    int line = t / n, k = t - (t / n) * n;
#pragma unroll 4
    for (int e = t; e < cnt; e += kThreads) {
      double u = (double)sb[k * kLS + line];
      if (post) u *= post[g0 + e];
      if (rv) {
        const double rr = rv[g0 + e];
        sold = fma(rr, (double)o[g0 + e], sold);
        snew = fma(rr, u, snew);
      }
      o[g0 + e] = (TO)u;
      k += dk;
      line += dl;
      if (k >= n) {
        k -= n;
        ++line;
      }
    }
  } else if (nl == kLines) {
    const int line = t & (kLines - 1);
#pragma unroll 4
    for (int k = t / kLines; k < n; k += kThreads / kLines) {
      const long long g = gline + A * k;
      double u = (double)sb[k * kLS + line];
      if (post) u *= post[g];
      if (rv) {
        const double rr = rv[g];
        sold = fma(rr, (double)o[g], sold);
        snew = fma(rr, u, snew);
      }
      o[g] = (TO)u;
    }
  } else {
    for (int e = t; e < cnt; e += kThreads) {
      const int k = e / nl, line = e - k * nl;
      const long long rr = l0 + line;
      const long long y = rr / A, xx = rr - y * A;
      const long long g = xx + A * (k + (long long)n * y);
      double u = (double)sb[k * kLS + line];
      if (post) u *= post[g];
      if (rv) {
        const double rr = rv[g];
        sold = fma(rr, (double)o[g], sold);
        snew = fma(rr, u, snew);
      }
      o[g] = (TO)u;
    }
  }
  if (rv) {  // fixed-order block sums
    __shared__ double red[2][kThreads / 32];
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      snew += __shfl_down_sync(0xffffffffu, snew, o2);
      sold += __shfl_down_sync(0xffffffffu, sold, o2);
    }
    if (lane == 0) {
      red[0][w] = snew;
      red[1][w] = sold;
    }
    __syncthreads();
    if (t == 0) {
      double a = 0.0, b = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) {
        a += red[0][q];
        b += red[1][q];
      }
      part[(long long)v * gridDim.x + blockIdx.x] = a;
      part[(long long)(gridDim.y + v) * gridDim.x + blockIdx.x] = b;
    }
  }
}

template <int P, typename T, typename TI, typename TO>
cudaError_t kron_go(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const void* L,
                    const void* dinv, const void* in, void* out, long long vs, const double* pre,
                    const double* post, const double* rdot, double* part, int* npart) {
  const long long R = sh.A * sh.B;
  const size_t smem = (size_t)n * (kLS + 2 * P + 2) * sizeof(T);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_kron_axis<P, T, TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((R + kLines - 1) / kLines), (unsigned)nvec);
  const bool fused = rdot && sizeof(TO) == sizeof(double);
  k_kron_axis<P, T, TI, TO><<<grid, kThreads, smem, s>>>(
      n, sh.A, R, static_cast<const T*>(L), static_cast<const T*>(dinv), active, static_cast<const TI*>(in),
      static_cast<TO*>(out), vs, pre, post, fused ? rdot : nullptr, part);
  if (npart) *npart = fused ? (int)grid.x : 0;
  return cudaGetLastError();
}

template <int P>
cudaError_t kron_types(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, int f32, const void* L,
                       const void* dinv, const void* in, int in_is_double, void* out, int out_is_double, long long vs,
                       const double* pre, const double* post, const double* rdot, double* part, int* npart) {
  if (!f32)
    return kron_go<P, double, double, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                              npart);
  if (in_is_double && !out_is_double)
    return kron_go<P, float, double, float>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                            npart);
  if (!in_is_double && out_is_double)
    return kron_go<P, float, float, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                            npart);
  if (!in_is_double && !out_is_double)
    return kron_go<P, float, float, float>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                           npart);
  return kron_go<P, float, double, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part, npart);
}

}  // namespace

cudaError_t launch_kron_axis(cudaStream_t s, int n, int p, AxisShape sh, int nvec, const int* active, int f32,
                             const void* L, const void* dinv, const void* in, int in_is_double, void* out,
                             int out_is_double, long long vs, const double* pre, const double* post,
                             const double* rdot, double* part, int* npart) {
  if (npart) *npart = 0;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  if (n < 1 || nvec < 1 || (size_t)n * (kLS + 2 * p + 2) * esz > 227 * 1024) return cudaErrorInvalidValue;
  if (!f32 && !(in_is_double && out_is_double)) return cudaErrorInvalidValue;
#define IGA_KRON(PP) \
  return kron_types<PP>(s, n, sh, nvec, active, f32, L, dinv, in, in_is_double, out, out_is_double, vs, pre, post, \
                        rdot, part, npart)
  switch (p) {
    case 1: IGA_KRON(1);
    case 2: IGA_KRON(2);
    case 3: IGA_KRON(3);
    case 4: IGA_KRON(4);
    case 5: IGA_KRON(5);
    case 6: IGA_KRON(6);
    default: return cudaErrorInvalidValue;
  }
#undef IGA_KRON
}

}  // namespace iga
