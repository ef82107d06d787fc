// Fast-diagonalisation mode products of the preconditioner (Sec. 5.3 and 5.5):
// out[x, i, y] = sum_j Mat(i, j) in[x, j, y] along one axis of the n0 x n1 x n2
// co-lexicographic tensor, Mat = U_a or U_a^T (U_a the orthonormal eigenvectors of
// the univariate parametric mass matrix Mhat_a).
//
// Each mode product is the small GEMM Y (R x n) = X (R x n) Mat^T over the
// R = N / n lines ("rows") of the tensor along the axis; row r is the line at
// x = r mod A, y = r div A (A = stride of the axis), element j at x + A (j + n y).
//
// Matrix layout: [U | U^T], each stored as Mat(i, j) at j*np + i, np = n rounded
// up to 8 (zero padding).
//
// A block takes a tile of kTileRows consecutive rows: it first stages the whole
// tile in shared memory with one wide, coalesced load (a contiguous block for
// axis 0, and for the strided axes kTileRows consecutive rows of every j, which
// are consecutive addresses), so the load latency is paid once per tile rather
// than once per term; then thread (row t, group g) accumulates the np/8
// consecutive outputs i = g np/8 ... of its row from shared memory, with the
// coefficients Mat(i, j) being the same for the whole warp (broadcast loads).
// Outputs of the strided axes are written directly (consecutive rows are
// consecutive addresses); axis-0 outputs are staged back through shared memory
// and written as one contiguous block. Epilogue: optional division by
// Lambda_0(i0) Lambda_1(i1) Lambda_2(i2) and optional FP64 rescaling; an optional
// FP64 prologue scaling multiplies the inputs before they are rounded.
#include "iga_internal.h"

namespace iga {

constexpr int kTileRows = 16;   // rows per block
constexpr int kGroups = 8;      // output groups per row (128 threads per block)
constexpr int kStage = 8;       // staged loads in flight per thread
// outputs per thread per chunk (template kMaxRI): 9 for np <= 72, else 17 (chunks of 136 outputs)

__host__ __device__ inline int fd_np(int n) { return (n + 7) & ~7; }

template <typename TC>
struct FdArgs {
  int n, np;
  const TC* mat;        // the applied matrix, Mat(i, j) at j*np + i
  const double* pre;    // multiply inputs by pre[idx] in FP64 before rounding (nullable)
  const double* post;   // multiply outputs by post[idx] (nullable)
  const TC* lam0;       // multiply by lam0[i0] lam1[i1] lam2[i2], inverse eigenvalues (nullable)
  const TC* lam1;
  const TC* lam2;
  int n0, n1;           // tensor sizes for the index decomposition of the epilogue
  long long A;          // stride of the axis (product of the faster sizes)
  long long R;          // rows = A * B
};

template <typename TC>
__device__ __forceinline__ TC fd_lambda(const FdArgs<TC>& a, long long idx, TC acc) {
  if (a.lam0) {
    const int i0 = (int)(idx % a.n0);
    const int i1 = (int)((idx / a.n0) % a.n1);
    const int i2 = (int)(idx / ((long long)a.n0 * a.n1));
    TC l = a.lam0[i0] * a.lam1[i1];  // inverse eigenvalues
    if (a.lam2) l *= a.lam2[i2];
    acc = acc * l;
  }
  return acc;
}

template <typename TC, typename TO>
__device__ __forceinline__ void fd_put(const FdArgs<TC>& a, TO* out, long long idx, TC val) {
  if (a.post) out[idx] = (TO)((double)val * a.post[idx]);
  else out[idx] = (TO)val;
}

template <typename TI, typename TC, typename TO, bool AXIS0, int kMaxRI>
__global__ void __launch_bounds__(kTileRows* kGroups) k_fd_tile(FdArgs<TC> a, const int* __restrict__ active,
                                                                const TI* __restrict__ in, TO* __restrict__ out,
                                                                long long vs) {
  extern __shared__ unsigned char fd_smem[];
  TC* Xs = reinterpret_cast<TC*>(fd_smem);  // [kTileRows][ld]
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int n = a.n, np = a.np, ld = np + 1;  // odd row stride: conflict-free column reads
  const long long A = a.A;
  const long long r0 = (long long)blockIdx.x * kTileRows;
  const int rows = (int)min((long long)kTileRows, a.R - r0);
  const TI* src = in + v * vs;
  TO* dst = out + v * vs;
  const int tid = threadIdx.x;
  // ---- stage the tile: kStage independent loads per thread in flight, then the stores
  if (AXIS0) {
    const long long base = r0 * n;
    const int cnt = rows * n;
    for (int f0 = 0; f0 < cnt; f0 += kStage * blockDim.x) {
      double u[kStage];
#pragma unroll
      for (int k = 0; k < kStage; ++k) {
        const int f = f0 + k * blockDim.x + tid;
        u[k] = f < cnt ? (double)src[base + f] : 0.0;
        if (a.pre && f < cnt) u[k] *= a.pre[base + f];
      }
#pragma unroll
      for (int k = 0; k < kStage; ++k) {
        const int f = f0 + k * blockDim.x + tid;
        if (f < cnt) {
          const int rr = f / n, j = f - rr * n;
          Xs[rr * ld + j] = (TC)u[k];
        }
      }
    }
  } else {
    const int cnt = kTileRows * n;
    for (int e0 = 0; e0 < cnt; e0 += kStage * blockDim.x) {
      double u[kStage];
#pragma unroll
      for (int k = 0; k < kStage; ++k) {
        const int e = e0 + k * blockDim.x + tid;
        const int j = e / kTileRows, rr = e - j * kTileRows;
        u[k] = 0.0;
        if (e < cnt && rr < rows) {
          const long long r = r0 + rr;
          const long long y = r / A, x = r - y * A;
          const long long idx = x + A * (j + (long long)n * y);
          u[k] = (double)src[idx];
          if (a.pre) u[k] *= a.pre[idx];
        }
      }
#pragma unroll
      for (int k = 0; k < kStage; ++k) {
        const int e = e0 + k * blockDim.x + tid;
        if (e < cnt) {
          const int j = e / kTileRows, rr = e - j * kTileRows;
          Xs[rr * ld + j] = (TC)u[k];
        }
      }
    }
  }
  __syncthreads();
  // ---- compute: thread (row t, group g)
  const int t = tid % kTileRows;
  const int g = tid / kTileRows;
  const TC* xr = Xs + t * ld;
  TC outv[kMaxRI];
  for (int ic = 0; ic < np; ic += kGroups * kMaxRI) {
    const int span = min(np - ic, kGroups * kMaxRI);  // multiple of 8
    const int RI = span / kGroups;
    const int i0 = ic + g * RI;
    TC acc[kMaxRI];
#pragma unroll
    for (int b = 0; b < kMaxRI; ++b) acc[b] = (TC)0;
#pragma unroll 2
    for (int j = 0; j < n; ++j) {
      const TC u = xr[j];
      const TC* mj = a.mat + (long long)j * np + i0;
#pragma unroll
      for (int b = 0; b < kMaxRI; ++b)
        if (b < RI) acc[b] = fma(__ldg(mj + b), u, acc[b]);
    }
    if (AXIS0) {
      // keep the results (after Lambda) to stage through shared memory
#pragma unroll
      for (int b = 0; b < kMaxRI; ++b)
        if (b < RI) outv[b] = fd_lambda(a, (r0 + t) * n + i0 + b, acc[b]);
      __syncthreads();  // every thread has finished reading Xs
#pragma unroll
      for (int b = 0; b < kMaxRI; ++b)
        if (b < RI && i0 + b < n && t < rows) Xs[t * ld + i0 + b] = outv[b];
      __syncthreads();
      const long long base = r0 * n;
      for (int f = tid; f < rows * n; f += blockDim.x) {
        const int rr = f / n, i = f - rr * n;
        if (i >= ic && i < ic + span) fd_put(a, dst, base + f, Xs[rr * ld + i]);
      }
      __syncthreads();
      if (ic + kGroups * kMaxRI < np) {
        // a further chunk needs the input tile again: restage it
        for (int f = tid; f < rows * n; f += blockDim.x) {
          const int rr = f / n, j = f - rr * n;
          double u = (double)src[base + f];
          if (a.pre) u *= a.pre[base + f];
          Xs[rr * ld + j] = (TC)u;
        }
        __syncthreads();
      }
    } else {
      if (t < rows) {
        const long long r = r0 + t;
        const long long y = r / A, x = r - y * A;
#pragma unroll
        for (int b = 0; b < kMaxRI; ++b) {
          const int i = i0 + b;
          if (b < RI && i < n) {
            const long long idx = x + A * (i + (long long)n * y);
            fd_put(a, dst, idx, fd_lambda(a, idx, acc[b]));
          }
        }
      }
    }
  }
}

// FP32 variant with one output per thread: the whole matrix (n x np floats) and a
// tile of TR = 512 / np rows live in shared memory; thread (t, i) forms
// sum_j X(t, j) Mat(i, j) from a broadcast (X) and a conflict-free (Mat) read.
// Many resident warps hide the latency that limits the register-tiled form when
// there are only a few thousand rows.
template <typename TI, typename TO, bool AXIS0>
__global__ void __launch_bounds__(512) k_fd_smem32(FdArgs<float> a, int TR, const int* __restrict__ active,
                                                   const TI* __restrict__ in, TO* __restrict__ out, long long vs) {
  extern __shared__ __align__(16) float fsm[];
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int n = a.n, np = a.np, ldx = n + 1;
  float* Ms = fsm;             // Mat(i, j) at j*np + i
  float* Xs = fsm + n * np;    // [TR][n+1]
  const long long A = a.A;
  const long long r0 = (long long)blockIdx.x * TR;
  const int rows = (int)min((long long)TR, a.R - r0);
  const TI* src = in + v * vs;
  TO* dst = out + v * vs;
  const int tid = threadIdx.x, nt = blockDim.x;
  {
    const float4* m4 = reinterpret_cast<const float4*>(a.mat);
    float4* s4 = reinterpret_cast<float4*>(Ms);
    for (int e = tid; e < n * np / 4; e += nt) s4[e] = __ldg(m4 + e);
  }
  if (AXIS0) {
    const long long base = r0 * n;
    for (int f = tid; f < rows * n; f += nt) {
      const int rr = f / n, j = f - rr * n;
      double u = (double)src[base + f];
      if (a.pre) u *= a.pre[base + f];
      Xs[rr * ldx + j] = (float)u;
    }
  } else {
    for (int e = tid; e < rows * n; e += nt) {
      const int j = e / rows, rr = e - j * rows;
      const long long r = r0 + rr;
      const long long y = r / A, x = r - y * A;
      const long long idx = x + A * (j + (long long)n * y);
      double u = (double)src[idx];
      if (a.pre) u *= a.pre[idx];
      Xs[rr * ldx + j] = (float)u;
    }
  }
  __syncthreads();
  const int t = tid / np, i = tid - t * np;
  if (t >= rows || i >= n) return;
  const float* xr = Xs + t * ldx;
  float acc = 0.0f;
#pragma unroll 8
  for (int j = 0; j < n; ++j) acc = fmaf(xr[j], Ms[j * np + i], acc);
  const long long r = r0 + t;
  long long idx;
  if (AXIS0) {
    idx = r * n + i;
  } else {
    const long long y = r / A, x = r - y * A;
    idx = x + A * (i + (long long)n * y);
  }
  fd_put(a, dst, idx, fd_lambda(a, idx, acc));
}

template <typename TI, typename TO>
static bool fd_smem32(cudaStream_t s, const FdArgs<float>& a, int nvec, const int* active, const TI* in, TO* out,
                      long long vs, cudaError_t* err) {
  if (a.np > 512) return false;
  const int TR = 512 / a.np;
  const size_t smem = sizeof(float) * ((size_t)a.n * a.np + (size_t)TR * (a.n + 1));
  if (smem > 160 * 1024) return false;
  const long long blocks = (a.R + TR - 1) / TR;
  const dim3 grid((unsigned)blocks, nvec);
  const int threads = ((TR * a.np + 31) / 32) * 32;
  if (a.A == 1) {
    if (smem > 48 * 1024 &&
        (*err = cudaFuncSetAttribute(k_fd_smem32<TI, TO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem)) != cudaSuccess)
      return true;
    k_fd_smem32<TI, TO, true><<<grid, threads, smem, s>>>(a, TR, active, in, out, vs);
  } else {
    if (smem > 48 * 1024 &&
        (*err = cudaFuncSetAttribute(k_fd_smem32<TI, TO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem)) != cudaSuccess)
      return true;
    k_fd_smem32<TI, TO, false><<<grid, threads, smem, s>>>(a, TR, active, in, out, vs);
  }
  *err = cudaGetLastError();
  return true;
}

template <typename TI, typename TC, typename TO, bool AX0, int RI>
static cudaError_t fd_go(cudaStream_t s, const FdArgs<TC>& a, int nvec, const int* active, const TI* in, TO* out,
                         long long vs, size_t smem, dim3 grid) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fd_tile<TI, TC, TO, AX0, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fd_tile<TI, TC, TO, AX0, RI><<<grid, kTileRows * kGroups, smem, s>>>(a, active, in, out, vs);
  return cudaGetLastError();
}

template <typename TI, typename TC, typename TO>
static cudaError_t fd_launch(cudaStream_t s, const FdArgs<TC>& a, int nvec, const int* active, const TI* in, TO* out,
                             long long vs) {
  const size_t smem = sizeof(TC) * (size_t)kTileRows * (a.np + 1);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const long long blocks = (a.R + kTileRows - 1) / kTileRows;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)blocks, nvec);
  const bool small = a.np <= kGroups * 9;
  if (a.A == 1)
    return small ? fd_go<TI, TC, TO, true, 9>(s, a, nvec, active, in, out, vs, smem, grid)
                 : fd_go<TI, TC, TO, true, 17>(s, a, nvec, active, in, out, vs, smem, grid);
  return small ? fd_go<TI, TC, TO, false, 9>(s, a, nvec, active, in, out, vs, smem, grid)
               : fd_go<TI, TC, TO, false, 17>(s, a, nvec, active, in, out, vs, smem, grid);
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
  a.A = sh.A;
  a.R = sh.A * sh.B;
  return fd_launch<double, double, double>(s, a, nvec, active, in, out, vs);
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
  a.R = sh.A * sh.B;
  cudaError_t e = cudaSuccess;
  if (in_is_double && !out_is_double) {
    if (fd_smem32(s, a, nvec, active, (const double*)in, (float*)out, vs, &e)) return e;
  } else if (!in_is_double && !out_is_double) {
    if (fd_smem32(s, a, nvec, active, (const float*)in, (float*)out, vs, &e)) return e;
  } else if (!in_is_double && out_is_double) {
    if (fd_smem32(s, a, nvec, active, (const float*)in, (double*)out, vs, &e)) return e;
  } else {
    if (fd_smem32(s, a, nvec, active, (const double*)in, (double*)out, vs, &e)) return e;
  }
  if (in_is_double && !out_is_double)
    return fd_launch<double, float, float>(s, a, nvec, active, (const double*)in, (float*)out, vs);
  if (!in_is_double && !out_is_double)
    return fd_launch<float, float, float>(s, a, nvec, active, (const float*)in, (float*)out, vs);
  if (!in_is_double && out_is_double)
    return fd_launch<float, float, double>(s, a, nvec, active, (const float*)in, (double*)out, vs);
  return fd_launch<double, float, double>(s, a, nvec, active, (const double*)in, (double*)out, vs);
}

}  // namespace iga
