// Fast-diagonalisation mode products of the preconditioner (Sec. 5.3 and 5.5):
// out[x, i, y] = sum_j Mat(i, j) in[x, j, y] along one axis of the n0 x n1 x n2
// co-lexicographic tensor, Mat = U_a or U_a^T (U_a the orthonormal eigenvectors of
// the univariate parametric mass matrix Mhat_a).
//
// Matrix layout: [U | U^T], each stored as Mat(i, j) at j*np + i, np = n rounded
// up to 8 (zero padding).
//
// One kernel for every axis. A line is the n values along the axis at fixed
// (x, y); a group of G lanes (G = 8, 16 or 32, so 32/G lines per warp) gathers
// its line into shared memory (for axis 0 a contiguous read; otherwise a
// strided gather, served from L2 where the whole tensor of a preconditioner
// application resides) and lane l of the group accumulates the outputs
// i = l, l+G, l+2G, ... with coefficient reads Mat(l + G r, j) that are
// contiguous within the group. Smaller G wastes fewer lanes when n is not a
// multiple of 32 (what matters for FP64, whose pipe is 1/64 of FP32); G = 32
// gives the fewest instructions per output (FP32).
// Epilogue: optional division by Lambda_0(i0) Lambda_1(i1) Lambda_2(i2), optional
// FP64 rescaling, conversion to the output type. An optional FP64 prologue
// scaling multiplies the inputs before they are rounded to the compute type.
#include "iga_internal.h"

namespace iga {

__host__ __device__ inline int fd_np(int n) { return (n + 7) & ~7; }

template <typename TC>
struct FdArgs {
  int n, np;
  const TC* mat;        // the applied matrix, Mat(i, j) at j*np + i
  const double* pre;    // multiply inputs by pre[idx] in FP64 before rounding (nullable)
  const double* post;   // multiply outputs by post[idx] (nullable)
  const TC* lam0;       // divide by lam0[i0] lam1[i1] lam2[i2] (nullable)
  const TC* lam1;
  const TC* lam2;
  int n0, n1;           // tensor sizes for the index decomposition of the epilogue
  long long A;          // stride of the axis (product of the faster sizes)
  long long nlines;     // A * B
};

template <typename TC, typename TO>
__device__ __forceinline__ void fd_store(const FdArgs<TC>& a, TO* out, long long idx, TC acc) {
  if (a.lam0) {
    const int i0 = (int)(idx % a.n0);
    const int i1 = (int)((idx / a.n0) % a.n1);
    const int i2 = (int)(idx / ((long long)a.n0 * a.n1));
    TC l = a.lam0[i0] * a.lam1[i1];
    if (a.lam2) l *= a.lam2[i2];
    acc = acc / l;
  }
  if (a.post) out[idx] = (TO)((double)acc * a.post[idx]);
  else out[idx] = (TO)acc;
}

// G lanes per line, R outputs per lane per output block (G * R outputs per block)
template <typename TI, typename TC, typename TO, int G, int R>
__global__ void __launch_bounds__(256) k_fd_lines(FdArgs<TC> a, const int* __restrict__ active,
                                                  const TI* __restrict__ in, TO* __restrict__ out, long long vs) {
  extern __shared__ unsigned char fd_smem[];
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int lane = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G;  // line slot of this group within the block
  const int ngrp = blockDim.x / G;
  TC* line = reinterpret_cast<TC*>(fd_smem) + grp * a.np;
  const TI* src = in + v * vs;
  TO* dst = out + v * vs;
  const int n = a.n;
  const long long A = a.A;
  for (long long L = (long long)blockIdx.x * ngrp + grp; L < a.nlines; L += (long long)gridDim.x * ngrp) {
    // line L = x + A * y, element j at x + A * (j + n * y)
    const long long y = L / A;
    const long long x = L - y * A;
    const long long base = x + A * n * y;
    for (int j = lane; j < n; j += G) {
      const long long idx = base + (long long)j * A;
      double u = (double)src[idx];
      if (a.pre) u *= a.pre[idx];
      line[j] = (TC)u;
    }
    __syncwarp();
    for (int ib = 0; ib < n; ib += G * R) {
      TC acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = (TC)0;
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const TC u = line[j];
        const TC* mj = a.mat + (long long)j * a.np + ib + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (ib + G * r >= a.np) break;  // uniform across the warp: rounds past the padded row
          if (ib + lane + G * r < a.np) acc[r] = fma(__ldg(mj + G * r), u, acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = ib + lane + G * r;
        if (i < n) fd_store(a, dst, base + (long long)i * A, acc[r]);
      }
    }
    __syncwarp();
  }
}

template <typename TI, typename TC, typename TO, int G, int R>
static cudaError_t fd_run(cudaStream_t s, const FdArgs<TC>& a, int nvec, const int* active, const TI* in, TO* out,
                          long long vs) {
  // lines per block: up to 256 threads, within 48 KB of line buffers (whole warps)
  constexpr int per_warp = 32 / G;
  const size_t line_bytes = sizeof(TC) * (size_t)a.np;
  int groups = 256 / G;
  while (groups > per_warp && groups * line_bytes > 48 * 1024) groups -= per_warp;
  const size_t smem = groups * line_bytes;
  if (smem > 48 * 1024) {  // one warp's lines exceed the default: raise the limit (up to 227 KB)
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_fd_lines<TI, TC, TO, G, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  long long blocks = (a.nlines + groups - 1) / groups;
  const long long cap = 152LL * 16;  // at most 16 resident-size waves of blocks; the rest loop
  if (blocks > cap) blocks = cap;
  k_fd_lines<TI, TC, TO, G, R><<<dim3((unsigned)blocks, nvec), groups * G, smem, s>>>(a, active, in, out, vs);
  return cudaGetLastError();
}

// FP64: the lane group that wastes the fewest FP64 slots on the last output block
template <typename TI, typename TO>
static cudaError_t fd_launch64(cudaStream_t s, const FdArgs<double>& a, int nvec, const int* active, const TI* in,
                               TO* out, long long vs) {
  auto waste = [&](int G) { return (G - a.n % G) % G; };
  int best = 8;
  if (waste(16) < waste(best)) best = 16;
  if (waste(32) < waste(best)) best = 32;
  if (best == 32) return fd_run<TI, double, TO, 32, 4>(s, a, nvec, active, in, out, vs);
  if (best == 16) return fd_run<TI, double, TO, 16, 8>(s, a, nvec, active, in, out, vs);
  return fd_run<TI, double, TO, 8, 16>(s, a, nvec, active, in, out, vs);
}

static FdArgs<double> args64(int n, AxisShape sh, const double* U, int transpose) {
  FdArgs<double> a{};
  a.n = n;
  a.np = fd_np(n);
  a.mat = U + (transpose ? (long long)n * a.np : 0LL);
  a.A = sh.A;
  a.nlines = sh.A * sh.B;
  a.n0 = a.n1 = 1;
  return a;
}

cudaError_t launch_fd_mode64(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const double* U,
                             int transpose, const double* in, double* out, long long vs, const double* pre,
                             FdEpilogue ep) {
  FdArgs<double> a = args64(n, sh, U, transpose);
  a.pre = pre;
  a.post = ep.post;
  a.lam0 = ep.lam[0];
  a.lam1 = ep.lam[1];
  a.lam2 = ep.lam[2];
  a.n0 = ep.n[0] > 0 ? ep.n[0] : 1;
  a.n1 = ep.n[1] > 0 ? ep.n[1] : 1;
  return fd_launch64<double, double>(s, a, nvec, active, in, out, vs);
}

cudaError_t launch_fd_mode32(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const float* U,
                             int transpose, const void* in, int in_is_double, void* out, int out_is_double,
                             long long vs, const double* pre, const double* post, const float* const* lam,
                             const int* nn) {
  FdArgs<float> a{};
  a.n = n;
  a.np = fd_np(n);
  a.mat = U + (transpose ? (long long)n * a.np : 0LL);
  a.pre = pre;
  a.post = post;
  a.lam0 = lam ? lam[0] : nullptr;
  a.lam1 = lam ? lam[1] : nullptr;
  a.lam2 = lam ? lam[2] : nullptr;
  a.n0 = nn ? nn[0] : 1;
  a.n1 = nn ? nn[1] : 1;
  a.A = sh.A;
  a.nlines = sh.A * sh.B;
  if (in_is_double && !out_is_double)
    return fd_run<double, float, float, 32, 4>(s, a, nvec, active, (const double*)in, (float*)out, vs);
  if (!in_is_double && !out_is_double)
    return fd_run<float, float, float, 32, 4>(s, a, nvec, active, (const float*)in, (float*)out, vs);
  if (!in_is_double && out_is_double)
    return fd_run<float, float, double, 32, 4>(s, a, nvec, active, (const float*)in, (double*)out, vs);
  return fd_run<double, float, double, 32, 4>(s, a, nvec, active, (const double*)in, (double*)out, vs);
}

}  // namespace iga
