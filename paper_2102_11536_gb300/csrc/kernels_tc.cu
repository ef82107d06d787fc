// BF16 fast-diagonalisation mode products on the 5th-generation tensor cores
// (tcgen05, sm_103a), FP32 accumulation in tensor memory.
//
// A mode product along one axis is the GEMM D (R x n) = X (R x n) Mat^T, the
// R = N / n rows of the tensor along the axis times the n x n matrix Mat = U_a or
// U_a^T (the preconditioner of Sec. 5.3 applied by fast diagonalisation). One CTA
// of 128 threads takes 128 rows:
//   1. warp 0 allocates 128 or 256 TMEM columns (the 128 x Np FP32 accumulator);
//   2. all threads copy the BF16 matrix (pre-arranged on the host, see below) into
//      shared memory and stage the 128-row tile of X, rounded to BF16 (with the FP64
//      diagonal scaling first for the first mode), both in the canonical K-major,
//      no-swizzle layout: 8-row x 16-byte core matrices, element (r, k) at byte
//      (r/8) SBO + (k/8) LBO + (r%8) 16 + (k%8) 2 with LBO = 128 and SBO = 16 Kp;
//   3. one thread issues Kp/16 MMAs of shape 128 x Np x 16 (kind::f16, BF16 inputs,
//      FP32 accumulator) and commits them to an mbarrier;
//   4. every thread waits on the mbarrier (bounded: on time-out the kernel sets
//      an error word, waits once more, frees its TMEM and returns), then warp w
//      reads TMEM lanes 32w..32w+31 (row = 32w + lane) with tcgen05.ld and writes the
//      outputs with the Lambda^{-1} / FP64 rescaling epilogue.
// n is padded to Kp = Np = n rounded up to 16 (zero rows and columns); Np <= 256.
#include <cuda_bf16.h>

#include <cstring>

#include "iga_internal.h"

namespace iga {

namespace {

constexpr int kTcRows = 128;
constexpr long long kWaitLimit = 1LL << 24;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, no swizzle (layout type 0), version 1
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128
__host__ __device__ constexpr uint32_t make_idesc_bf16(int N) {
  return (1u << 4)                       // D format F32
         | (1u << 7)                     // A format BF16
         | (1u << 10)                    // B format BF16
         | ((uint32_t)(N >> 3) << 17)    // N >> 3
         | ((uint32_t)(kTcRows >> 4) << 24);  // M >> 4
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t core_off(int r, int k, int Kp) {
  // byte offset of element (r, k) in the canonical K-major no-swizzle layout
  return (uint32_t)((r >> 3) * (Kp >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

}  // namespace

template <typename TI, typename TO>
__global__ void __launch_bounds__(kTcRows) k_fd_tc(int n, int Kp, int ncols, long long A, long long R,
                                                   const __nv_bfloat16* __restrict__ Bmat,
                                                   const int* __restrict__ active, const TI* __restrict__ in,
                                                   TO* __restrict__ out, long long vs, const double* __restrict__ pre,
                                                   const double* __restrict__ post, const float* __restrict__ lam0,
                                                   const float* __restrict__ lam1, const float* __restrict__ lam2,
                                                   int n0, int n1, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + 8);
  unsigned char* As = tc_smem + 1024;
  unsigned char* Bs = As + (size_t)kTcRows * Kp * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long r0 = (long long)blockIdx.x * kTcRows;
  const int rows = (int)min((long long)kTcRows, R - r0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B: pre-arranged on the host, a plain 16-byte copy
  {
    const int nvec16 = Kp * Kp * 2 / 16;
    const uint4* src = reinterpret_cast<const uint4*>(Bmat);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int e = tid; e < nvec16; e += kTcRows) dst[e] = __ldg(src + e);
  }
  // A: the 128-row tile, rounded to BF16; zero outside the rows and beyond n
  const TI* x = in + v * vs;
  if (A == 1) {
    for (int e = tid; e < kTcRows * Kp; e += kTcRows) {
      const int r = e / Kp, k = e - r * Kp;
      float val = 0.0f;
      if (r < rows && k < n) {
        const long long idx = (r0 + r) * n + k;
        double u = (double)x[idx];
        if (pre) u *= pre[idx];
        val = (float)u;
      }
      *reinterpret_cast<__nv_bfloat16*>(As + core_off(r, k, Kp)) = __float2bfloat16(val);
    }
  } else {
    for (int e = tid; e < kTcRows * Kp; e += kTcRows) {
      const int k = e / kTcRows, r = e - k * kTcRows;
      float val = 0.0f;
      if (r < rows && k < n) {
        const long long rr = r0 + r;
        const long long y = rr / A, xx = rr - y * A;
        const long long idx = xx + A * (k + (long long)n * y);
        double u = (double)x[idx];
        if (pre) u *= pre[idx];
        val = (float)u;
      }
      *reinterpret_cast<__nv_bfloat16*>(As + core_off(r, k, Kp)) = __float2bfloat16(val);
    }
  }
  // make the generic-proxy shared-memory writes visible to the tensor core
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tslot;
  const uint32_t mb = smem_u32(mbar);
  if (tid == 0) {
    const uint32_t idesc = make_idesc_bf16(Kp);
    const uint32_t sbo = (uint32_t)(Kp >> 3) * 128u;
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    for (int ks = 0; ks < Kp / 16; ++ks) {
      const uint64_t da = make_desc(a0 + ks * 256, 128, sbo);
      const uint64_t db = make_desc(b0 + ks * 256, 128, sbo);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "setp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
          "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                 : "memory");
  }
  bool ok = mbar_wait(mb, 0);
  if (!ok) {
    atomicExch(err, 1);
    mbar_wait(mb, 0);  // one more bounded wait for the MMAs in flight
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = warp * 32 + lane;
    const uint32_t tbase = taddr + ((uint32_t)(warp * 32) << 16);
    TO* o = out + v * vs;
    const long long rr = r0 + row;
    const long long y = rr / A, xx = rr - y * A;
    for (int c0 = 0; c0 < Kp; c0 += 16) {
      uint32_t d[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
            "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
          : "r"(tbase + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < rows) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int i = c0 + c;
          if (i >= n) break;
          float val = __uint_as_float(d[c]);
          const long long idx = (A == 1) ? rr * n + i : xx + A * (i + (long long)n * y);
          if (lam0) {
            const int i0 = (int)(idx % n0), i1 = (int)((idx / n0) % n1), i2 = (int)(idx / ((long long)n0 * n1));
            float l = lam0[i0] * lam1[i1];
            if (lam2) l *= lam2[i2];
            val *= l;
          }
          if (post) o[idx] = (TO)((double)val * post[idx]);
          else o[idx] = (TO)val;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

int tc_pad(int n) { return (n + 15) & ~15; }

size_t tc_smem_bytes(int n) {
  const int Kp = tc_pad(n);
  return 1024 + (size_t)kTcRows * Kp * 2 + (size_t)Kp * Kp * 2;
}

// Host: the applied matrix Mat (i, j) (i output, j summed) in the K-major
// core-matrix layout of the B operand (rows i, K = j), zero-padded to Kp x Kp.
void tc_arrange_bf16(int n, const double* Mat_ij /* row-major n x n: Mat(i,j) at i*n+j */,
                     std::vector<uint16_t>& outbits) {
  const int Kp = tc_pad(n);
  outbits.assign((size_t)Kp * Kp, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const __nv_bfloat16 b = __float2bfloat16((float)Mat_ij[(size_t)i * n + j]);
      uint16_t bits;
      memcpy(&bits, &b, 2);
      const size_t off = ((size_t)(i >> 3) * (Kp >> 3) * 128 + (size_t)(j >> 3) * 128 + (i & 7) * 16 + (j & 7) * 2) / 2;
      outbits[off] = bits;
    }
}

template <typename TI, typename TO>
static cudaError_t tc_go(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active,
                         const __nv_bfloat16* B, const TI* in, TO* out, long long vs, const double* pre,
                         const double* post, const float* const* lam, const int* nn, int* err) {
  const int Kp = tc_pad(n);
  if (Kp > 256) return cudaErrorInvalidValue;
  const int ncols = Kp <= 128 ? 128 : 256;
  const size_t smem = tc_smem_bytes(n);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_fd_tc<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long R = sh.A * sh.B;
  const long long blocks = (R + kTcRows - 1) / kTcRows;
  const float* l0 = lam ? lam[0] : nullptr;
  const float* l1 = lam ? lam[1] : nullptr;
  const float* l2 = lam ? lam[2] : nullptr;
  k_fd_tc<TI, TO><<<dim3((unsigned)blocks, nvec), kTcRows, smem, s>>>(
      n, Kp, ncols, sh.A, R, B, active, in, out, vs, pre, post, l0, l1, l2, nn ? nn[0] : 1, nn ? nn[1] : 1, err);
  return cudaGetLastError();
}

cudaError_t launch_fd_mode_tc(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const void* B,
                              const void* in, int in_is_double, void* out, int out_is_double, long long vs,
                              const double* pre, const double* post, const float* const* lam, const int* nn,
                              int* err) {
  const __nv_bfloat16* Bm = static_cast<const __nv_bfloat16*>(B);
  if (in_is_double && !out_is_double)
    return tc_go<double, float>(s, n, sh, nvec, active, Bm, (const double*)in, (float*)out, vs, pre, post, lam, nn, err);
  if (!in_is_double && !out_is_double)
    return tc_go<float, float>(s, n, sh, nvec, active, Bm, (const float*)in, (float*)out, vs, pre, post, lam, nn, err);
  if (!in_is_double && out_is_double)
    return tc_go<float, double>(s, n, sh, nvec, active, Bm, (const float*)in, (double*)out, vs, pre, post, lam, nn, err);
  return tc_go<double, double>(s, n, sh, nvec, active, Bm, (const double*)in, (double*)out, vs, pre, post, lam, nn, err);
}

}  // namespace iga
