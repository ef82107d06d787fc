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
#include <type_traits>

#include "iga_internal.h"


namespace iga {

namespace {

constexpr int kLines = 32;    // lines per block (one warp solves them)
constexpr int kLS = kLines + 1;  // shared row stride: odd, so that both the staging walks
                                 // (consecutive entries of a line) and the solve
                                 // (consecutive lines) are free of bank conflicts
constexpr int kThreads = 256; // threads staging and writing back

// Conversions between FP64 and FP32 by integer operations on the bits (GB300 runs the
// hardware conversions on its narrow FP64 units): the same values as the hardware's
// round-to-nearest-even narrowing and exact widening; zero, subnormal, infinite and NaN
// values, and values outside FP32's normal range, take the hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int fe = (int)((b >> 52) & 0x7FF) - 896;  // FP32 biased exponent
  if (fe < 1 || fe > 254) return __double2float_rn(x);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  unsigned q = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFULL);
  if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ++q;  // a carry into the exponent is the rounding up
  return __uint_as_float(((unsigned)(b >> 63) << 31) + ((unsigned)fe << 23) + q);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(double v) { return f64_to_f32_rn(v); }
__device__ __forceinline__ double as_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double as_f64(double v) { return v; }
template <typename T>
__device__ __forceinline__ T narrow(double v);
template <>
__device__ __forceinline__ double narrow<double>(double v) { return v; }
template <>
__device__ __forceinline__ float narrow<float>(double v) { return f64_to_f32_rn(v); }

// one input entry of the tile: x[g] scaled by pre[g] (FP64, or with s32 the FP32 copy of
// the scaling in FP32 arithmetic), in the solve's type T
template <typename T, typename TI>
__device__ __forceinline__ T kron_in(const TI* x, long long g, const double* pre, const float* s32) {
  if constexpr (std::is_same<T, TI>::value) {
    if (!pre) return x[g];
  }
  if constexpr (std::is_same<T, float>::value) {  // the FP32 form scales by s32 (never null with pre)
    if (pre) return as_f32(x[g]) * s32[g];
    return as_f32(x[g]);
  } else {
    if (pre) return as_f64(x[g]) * pre[g];
    return as_f64(x[g]);
  }
}

// one output entry: u scaled by post[g] (FP64, or with s32 in FP32 and widened), the
// partials of rdot . new and rdot . old, stored as TO
template <typename T, typename TO>
__device__ __forceinline__ void kron_out(T u, TO* o, long long g, const double* post, const float* s32,
                                         const double* rv, double& snew, double& sold) {
  if constexpr (std::is_same<T, TO>::value) {
    if (!post && !rv) {
      o[g] = u;
      return;
    }
  }
  double w;
  if constexpr (std::is_same<T, float>::value) w = post ? as_f64(u * s32[g]) : as_f64(u);
  else w = post ? u * post[g] : u;
  if (rv) {
    const double rr = rv[g];
    sold = fma(rr, as_f64(o[g]), sold);
    snew = fma(rr, w, snew);
  }
  o[g] = (TO)narrow<TO>(w);
}

// P = p: entries below the diagonal in a row of the factor; T: arithmetic (double, or
// float for the FP32 form); TI / TO: input / output element types. pre / post are
// applied in FP64 before rounding to T / after widening from T.
// rdot (nullable, FP64 output only): also the per-block partials of rdot . out (new) and
// rdot . out (the values out held before: the previous z of flexible PCG) into
// part[v * gridDim.x + b] and part[(gridDim.y + v) * gridDim.x + b].
template <int P, typename T, typename TI, typename TO, int MODE>
__global__ void __launch_bounds__(kThreads) k_kron_axis(int n, long long A, long long R, const T* __restrict__ L,
                                                      const T* __restrict__ dinv, const int* __restrict__ active,
                                                      const TI* __restrict__ in, TO* __restrict__ out,
                                                      long long vs, const double* __restrict__ pre,
                                                      const double* __restrict__ post,
                                                      const double* __restrict__ rdot, double* __restrict__ part,
                                                      const float* __restrict__ s32) {
  // MODE (bit 0: pre, bit 1: post and rdot) leaves the unused scalings out of the code
  if (!(MODE & 1)) pre = nullptr;
  if (!(MODE & 2)) {
    post = nullptr;
    rdot = nullptr;
  }
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
      sb[k * kLS + line] = kron_in<T>(x, g0 + e, pre, s32);
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
      sb[k * kLS + line] = kron_in<T>(x, g, pre, s32);
    }
  } else {
    for (int e = t; e < cnt; e += kThreads) {
      const int k = e / nl, line = e - k * nl;
      const long long rr = l0 + line;
      const long long y = rr / A, xx = rr - y * A;
      const long long g = xx + A * (k + (long long)n * y);
      sb[k * kLS + line] = kron_in<T>(x, g, pre, s32);
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
      kron_out<T>(sb[k * kLS + line], o, g0 + e, post, s32, rv, snew, sold);
      k += dk;
      line += dl;
      if (k >= n) {
        k -= n;
        ++line;
      }
    }
  } else if (nl == kLines) {
    // four entries at a time: every load of the four (r, the previous output, the scaling)
    // is issued before their stores, which the compiler may not move loads across; the
    // entries are then finished in order (the same order as one at a time)
    const int line = t & (kLines - 1);
    constexpr int KS = kThreads / kLines;
    for (int kb = t / kLines; kb < n; kb += 4 * KS) {
      T u[4], ps[4];  // the entry and its scaling (the FP32 form's s32, or post)
      double rr[4], zo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kb + q * KS;
        rr[q] = zo[q] = 0.0;
        u[q] = ps[q] = T(0);
        if (k < n) {
          const long long g = gline + A * k;
          u[q] = sb[k * kLS + line];
          if (post) {
            if constexpr (std::is_same<T, float>::value) ps[q] = s32[g];
            else ps[q] = post[g];
          }
          if (rv) {
            rr[q] = rv[g];
            zo[q] = as_f64(o[g]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kb + q * KS;
        if (k < n) {
          const long long g = gline + A * k;
          const double w = post ? as_f64(u[q] * ps[q]) : as_f64(u[q]);
          if (rv) {
            sold = fma(rr[q], zo[q], sold);
            snew = fma(rr[q], w, snew);
          }
          o[g] = (TO)narrow<TO>(w);
        }
      }
    }
  } else {
    for (int e = t; e < cnt; e += kThreads) {
      const int k = e / nl, line = e - k * nl;
      const long long rr = l0 + line;
      const long long y = rr / A, xx = rr - y * A;
      const long long g = xx + A * (k + (long long)n * y);
      kron_out<T>(sb[k * kLS + line], o, g, post, s32, rv, snew, sold);
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

template <int P, typename T, typename TI, typename TO, int MODE>
cudaError_t kron_go_m(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const void* L,
                    const void* dinv, const void* in, void* out, long long vs, const double* pre,
                    const double* post, const double* rdot, double* part, int* npart, const float* s32) {
  const long long R = sh.A * sh.B;
  const size_t smem = (size_t)n * (kLS + 2 * P + 2) * sizeof(T);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_kron_axis<P, T, TI, TO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((R + kLines - 1) / kLines), (unsigned)nvec);
  const bool fused = rdot && sizeof(TO) == sizeof(double);
  k_kron_axis<P, T, TI, TO, MODE><<<grid, kThreads, smem, s>>>(
      n, sh.A, R, static_cast<const T*>(L), static_cast<const T*>(dinv), active, static_cast<const TI*>(in),
      static_cast<TO*>(out), vs, pre, post, fused ? rdot : nullptr, part, sizeof(T) == sizeof(float) ? s32 : nullptr);
  if (npart) *npart = fused ? (int)grid.x : 0;
  return cudaGetLastError();
}

// the scalings a launch applies (pre, post) as the kernel's MODE; each type combination
// is compiled for the modes the preconditioner's axes use, and for both (any launch)
template <int P, typename T, typename TI, typename TO>
cudaError_t kron_go(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const void* L,
                    const void* dinv, const void* in, void* out, long long vs, const double* pre,
                    const double* post, const double* rdot, double* part, int* npart, const float* s32) {
  const int mode = (pre ? 1 : 0) | (post ? 2 : 0);
  if (std::is_same<T, float>::value && mode && !s32) return cudaErrorInvalidValue;  // FP32 scaling needs s32
#define IGA_KGO(M) kron_go_m<P, T, TI, TO, M>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part, npart, s32)
  constexpr bool in_d = std::is_same<TI, double>::value, out_d = std::is_same<TO, double>::value;
  constexpr bool fp64 = std::is_same<T, double>::value;  // the FP64 form: every axis in every mode
  if constexpr (fp64 || (!in_d && !out_d)) {  // middle axes
    if (mode == 0) return IGA_KGO(0);
  }
  if constexpr (fp64 || (in_d && !out_d)) {  // first axis
    if (mode == 1) return IGA_KGO(1);
  }
  if constexpr (fp64 || (!in_d && out_d)) {  // last axis
    if (mode == 2) return IGA_KGO(2);
  }
  return IGA_KGO(3);
#undef IGA_KGO
}

template <int P>
cudaError_t kron_types(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, int f32, const void* L,
                       const void* dinv, const void* in, int in_is_double, void* out, int out_is_double, long long vs,
                       const double* pre, const double* post, const double* rdot, double* part, int* npart,
                       const float* s32) {
  if (!f32)
    return kron_go<P, double, double, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                              npart, s32);
  if (in_is_double && !out_is_double)
    return kron_go<P, float, double, float>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                            npart, s32);
  if (!in_is_double && out_is_double)
    return kron_go<P, float, float, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                            npart, s32);
  if (!in_is_double && !out_is_double)
    return kron_go<P, float, float, float>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part,
                                           npart, s32);
  return kron_go<P, float, double, double>(s, n, sh, nvec, active, L, dinv, in, out, vs, pre, post, rdot, part, npart, s32);
}

}  // namespace

cudaError_t launch_kron_axis(cudaStream_t s, int n, int p, AxisShape sh, int nvec, const int* active, int f32,
                             const void* L, const void* dinv, const void* in, int in_is_double, void* out,
                             int out_is_double, long long vs, const double* pre, const double* post,
                             const double* rdot, double* part, int* npart, const float* scale32) {
  if (npart) *npart = 0;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  if (n < 1 || nvec < 1 || (size_t)n * (kLS + 2 * p + 2) * esz > 227 * 1024) return cudaErrorInvalidValue;
  if (!f32 && !(in_is_double && out_is_double)) return cudaErrorInvalidValue;
#define IGA_KRON(PP) \
  return kron_types<PP>(s, n, sh, nvec, active, f32, L, dinv, in, in_is_double, out, out_is_double, vs, pre, post, \
                        rdot, part, npart, scale32)
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
