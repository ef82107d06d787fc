// Fast-diagonalisation mode products of the preconditioner (Sec. 5.3 and 5.5):
// out[x, i, y] = sum_j Mat(i, j) in[x, j, y] along one axis of the n0 x n1 x n2
// co-lexicographic tensor, Mat = U_a or U_a^T (U_a the orthonormal eigenvectors of
// the univariate parametric mass matrix Mhat_a).
//
// Matrix layout: [U | U^T], each stored as Mat(i, j) at j*np + i with the row
// count padded to np = n rounded up to 8, so that the coefficients a thread
// needs for 8 consecutive outputs i form two aligned 16-byte (FP32) or four
// (FP64) vector loads.
//
// Axis 0 (contiguous): one warp per line; the line (optionally multiplied by the
// FP64 diagonal scaling) is staged in shared memory, lane l accumulates outputs
// i = l, l+32, ... with the coefficients Mat(l + 32 r, j) read coalesced.
// Other axes: one thread per (x, y) and 8 consecutive outputs; every input load
// feeds 8 FMAs and the coefficient loads are the same for the whole warp.
// Epilogue: optional division by Lambda_0(i0) Lambda_1(i1) Lambda_2(i2), optional
// FP64 rescaling, conversion to the output type.
#include "iga_internal.h"

namespace iga {

constexpr int kFdR = 8;     // outputs per thread on strided axes
constexpr int kFdRMax = 6;  // outputs per lane per output block on axis 0

__host__ __device__ inline int fd_np(int n) { return (n + 7) & ~7; }

template <typename TC>
struct Vec8 {
  TC v[8];
};

template <typename TC>
__device__ __forceinline__ void load8(const TC* p, TC* o);

template <>
__device__ __forceinline__ void load8<float>(const float* p, float* o) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

template <>
__device__ __forceinline__ void load8<double>(const double* p, double* o) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldg(q + k);
    o[2 * k] = a.x;
    o[2 * k + 1] = a.y;
  }
}

template <typename TC>
struct FdArgs {
  int n, np;
  const TC* mat;        // the applied matrix, Mat(i, j) at j*np + i
  const double* pre;    // multiply inputs by pre[idx] (FP64) before rounding (nullable, axis 0 only)
  const double* post;   // multiply outputs by post[idx] (nullable)
  const TC* lam0;       // divide by lam0[i0] lam1[i1] lam2[i2] (nullable)
  const TC* lam1;
  const TC* lam2;
  int n0, n1;           // tensor sizes for the index decomposition of the epilogue
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

// axis 0: lines of n contiguous values, one warp per line
template <typename TI, typename TC, typename TO>
__global__ void __launch_bounds__(256) k_fd_axis0(FdArgs<TC> a, long long nlines, const int* __restrict__ active,
                                                  const TI* __restrict__ in, TO* __restrict__ out, long long vs) {
  extern __shared__ unsigned char fd_smem[];
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  TC* line = reinterpret_cast<TC*>(fd_smem) + warp * a.np;
  const TI* src = in + v * vs;
  TO* dst = out + v * vs;
  const int n = a.n;
  for (long long y = (long long)blockIdx.x * nw + warp; y < nlines; y += (long long)gridDim.x * nw) {
    const long long base = y * n;
    for (int j = lane; j < n; j += 32) {
      double u = (double)src[base + j];
      if (a.pre) u *= a.pre[base + j];
      line[j] = (TC)u;
    }
    __syncwarp();
    for (int ib = 0; ib < n; ib += 32 * kFdRMax) {  // blocks of 32 * kFdRMax outputs
      TC acc[kFdRMax];
#pragma unroll
      for (int r = 0; r < kFdRMax; ++r) acc[r] = (TC)0;
      for (int j = 0; j < n; ++j) {
        const TC u = line[j];
        const TC* mj = a.mat + (long long)j * a.np + ib;
#pragma unroll
        for (int r = 0; r < kFdRMax; ++r) {
          const int i = lane + 32 * r;
          if (ib + i < n) acc[r] = fma(__ldg(mj + i), u, acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < kFdRMax; ++r) {
        const int i = ib + lane + 32 * r;
        if (i < n) fd_store(a, dst, base + i, acc[r]);
      }
    }
    __syncwarp();
  }
}

// strided axes: thread per (x, output group, y)
template <typename TI, typename TC, typename TO>
__global__ void __launch_bounds__(256) k_fd_axisN(FdArgs<TC> a, int A, const int* __restrict__ active,
                                                  const TI* __restrict__ in, TO* __restrict__ out, long long vs) {
  const int v = blockIdx.z;
  if (active && !active[v]) return;
  const int y = blockIdx.y;
  const int ngroups = a.np / kFdR;
  const int flat = blockIdx.x * blockDim.x + threadIdx.x;
  if (flat >= A * ngroups) return;
  const int g = flat / A;
  const int x = flat - g * A;
  const int n = a.n;
  const long long rowbase = (long long)y * n * A + x;
  const TI* src = in + v * vs + rowbase;
  const int i0 = g * kFdR;
  TC acc[kFdR];
#pragma unroll
  for (int r = 0; r < kFdR; ++r) acc[r] = (TC)0;
  for (int j = 0; j < n; ++j) {
    const TC u = (TC)src[(long long)j * A];
    TC m[kFdR];
    load8<TC>(a.mat + (long long)j * a.np + i0, m);
#pragma unroll
    for (int r = 0; r < kFdR; ++r) acc[r] = fma(m[r], u, acc[r]);
  }
  TO* dst = out + v * vs;
#pragma unroll
  for (int r = 0; r < kFdR; ++r) {
    const int i = i0 + r;
    if (i < n) fd_store(a, dst, rowbase + (long long)i * A, acc[r]);
  }
}

template <typename TI, typename TC, typename TO>
static cudaError_t fd_launch(cudaStream_t s, const FdArgs<TC>& a, AxisShape sh, int nvec, const int* active,
                             const TI* in, TO* out, long long vs) {
  if (sh.A == 1) {
    const long long nlines = sh.B;
    const int warps = 8;
    long long blocks = (nlines + warps - 1) / warps;
    if (blocks > 4 * 152 * 8) blocks = 4 * 152 * 8;
    const size_t smem = sizeof(TC) * (size_t)warps * a.np;
    k_fd_axis0<TI, TC, TO><<<dim3((unsigned)blocks, nvec), 32 * warps, smem, s>>>(a, nlines, active, in, out, vs);
  } else {
    if (a.pre) return cudaErrorInvalidValue;
    const long long plane = sh.A * (a.np / kFdR);
    if (sh.B > 65535 || plane > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((plane + 255) / 256), (unsigned)sh.B, nvec);
    k_fd_axisN<TI, TC, TO><<<grid, 256, 0, s>>>(a, (int)sh.A, active, in, out, vs);
  }
  return cudaGetLastError();
}

cudaError_t launch_fd_mode64(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const double* U,
                             int transpose, const double* in, double* out, long long vs, const double* pre,
                             FdEpilogue ep) {
  FdArgs<double> a{};
  a.n = n;
  a.np = fd_np(n);
  a.mat = U + (transpose ? (long long)n * a.np : 0LL);
  a.pre = pre;
  a.post = ep.post;
  a.lam0 = ep.lam[0];
  a.lam1 = ep.lam[1];
  a.lam2 = ep.lam[2];
  a.n0 = ep.n[0] > 0 ? ep.n[0] : 1;
  a.n1 = ep.n[1] > 0 ? ep.n[1] : 1;
  return fd_launch<double, double, double>(s, a, sh, nvec, active, in, out, vs);
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
  if (in_is_double && !out_is_double)
    return fd_launch<double, float, float>(s, a, sh, nvec, active, (const double*)in, (float*)out, vs);
  if (!in_is_double && !out_is_double)
    return fd_launch<float, float, float>(s, a, sh, nvec, active, (const float*)in, (float*)out, vs);
  if (!in_is_double && out_is_double)
    return fd_launch<float, float, double>(s, a, sh, nvec, active, (const float*)in, (double*)out, vs);
  return fd_launch<double, float, double>(s, a, sh, nvec, active, (const double*)in, (double*)out, vs);
}

}  // namespace iga
