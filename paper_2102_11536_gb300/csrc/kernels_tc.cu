// BF16 and FP16 fast-diagonalisation mode products on the 5th-generation tensor
// cores (tcgen05, sm_103a), FP32 accumulation in tensor memory.
//
// A mode product along one axis is the GEMM D (R x n) = X (R x n) Mat^T, the
// R = N / n lines of the tensor along the axis times the n x n matrix Mat = U_a or
// U_a^T (the preconditioner of Sec. 5.3 applied by fast diagonalisation). Line rr
// = xx + A y holds the elements xx + A (k + n y), k = 0..n-1.
//
// Persistent blocks of 256 threads walk 128-line tiles (tile t of vector t / T):
//   * once per block: warp 0 allocates tensor memory for two 128 x Kp FP32
//     accumulators, the 16-bit matrix (pre-arranged on the host) is copied to
//     shared memory, and the per-column factors (Lambda^{-1} of the axis) too;
//   * per tile: all threads stage the tile, converted to 16 bits (with the FP64
//     diagonal scaling first for the first mode), in the canonical K-major
//     no-swizzle layout (8-row x 16-byte core matrices, element (r, k) at byte
//     (r/8) SBO + (k/8) LBO + (r%8) 16 + (k%8) 2, LBO = 128, SBO = 16 Kp); thread
//     r (mod 128) owns line r and writes whole 16-byte core rows;
//   * one thread issues Kp/16 MMAs 128 x Kp x 16 (kind::f16) and commits them to
//     the buffer's mbarrier; the next tile is staged into the other buffer while
//     they run, and its MMAs are issued before this tile's epilogue;
//   * epilogue: warp w reads lanes 32 (w % 4) .. +31 (line 32 (w%4) + lane) with
//     tcgen05.ld, half the column chunks each for warps 0-3 and 4-7, and writes
//     row factor x column factor x value (x the FP64 scaling for the last mode).
// Every mbarrier wait is bounded; a time-out (made uniform over the block) sets
// the error word, ends the walk, waits once more for the MMAs in flight and frees
// the tensor memory.
//
// FP16 has a 5-bit exponent: each line is scaled by a power of two that puts its
// largest magnitude in [2^13, 2^14) before rounding, and the epilogue multiplies
// by the inverse power. The product is linear in each line, so the scaling is
// exact and the values keep FP16's 11-bit significand.
//
// n is padded to Kp = n rounded up to 16 (zero rows and columns); Kp <= 256.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "iga_internal.h"

namespace iga {

namespace {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 256;
constexpr long long kWaitLimit = 1LL << 24;  // mbarrier polls before giving up
constexpr int kHdr = 5120;  // header: mbarriers, TMEM slot, line maxima and exponents, column factors

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

// instruction descriptor, kind::f16: D = F32, A = B = BF16 (fmt 1) or both F16
// (fmt 0), both K-major, M = 128
__host__ __device__ constexpr uint32_t make_idesc(int N, bool f16) {
  return (1u << 4)                              // D format F32
         | ((f16 ? 0u : 1u) << 7)               // A format
         | ((f16 ? 0u : 1u) << 10)              // B format (same as A)
         | ((uint32_t)(N >> 3) << 17)           // N >> 3
         | ((uint32_t)(kTcRows >> 4) << 24);    // M >> 4
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

__host__ __device__ inline size_t bmat_bytes(int Kp) { return ((size_t)Kp * Kp * 2 + 1023) & ~(size_t)1023; }

struct TcArgs {
  int n, Kp, ncols, nbuf, axis;
  long long A, R, tpv, ntiles, vs;
  const uint16_t* B;
  const int* active;
  const double* pre;
  const double* post;
  const float* lam[3];  // inverse eigenvalues per direction, or all null
  int n0, n1;
  int* err;
};

__device__ __forceinline__ uint16_t to16(float v, bool f16) {
  uint16_t b;
  if (f16) {
    const __half h = __float2half_rn(v);
    memcpy(&b, &h, 2);
  } else {
    const __nv_bfloat16 h = __float2bfloat16(v);
    memcpy(&b, &h, 2);
  }
  return b;
}

__device__ __forceinline__ long long next_tile(const TcArgs& a, long long t) {
  while (t < a.ntiles && a.active && !a.active[t / a.tpv]) t += gridDim.x;
  return t;
}

// Stage tile t into A buffer `buf` (line exponents into rexp for FP16).
template <typename TI, bool F16>
__device__ void stage_tile(const TcArgs& a, const TI* __restrict__ in, long long t, unsigned char* Abuf,
                           double* rowred, int* rexp) {
  const int tid = threadIdx.x;
  const long long v = t / a.tpv;
  const long long r0 = (t - v * a.tpv) * kTcRows;
  const int r = tid & (kTcRows - 1), half = tid >> 7;
  const bool valid = r0 + r < a.R;
  const long long rr = r0 + r;
  const long long y = rr / a.A, xx = rr - y * a.A;
  const long long base = xx + a.A * (long long)a.n * y;
  const TI* x = in + v * a.vs;
  const int nch = a.Kp >> 3;
  double scale = 1.0;
  if (F16) {
    double m = 0.0;
    if (valid)
      for (int c = half; c < nch; c += 2)
        for (int u = 0; u < 8; ++u) {
          const int k = 8 * c + u;
          if (k < a.n) {
            double val = (double)x[base + a.A * k];
            if (a.pre) val *= a.pre[base + a.A * k];
            m = fmax(m, fabs(val));
          }
        }
    rowred[half * kTcRows + r] = m;
    __syncthreads();
    const double M = fmax(rowred[r], rowred[kTcRows + r]);
    int E = 0;
    if (M > 0.0 && isfinite(M)) frexp(M, &E);  // M = f 2^E, f in [0.5, 1)
    scale = ldexp(1.0, 14 - E);
    if (half == 0) rexp[r] = E - 14;
    __syncthreads();  // rowred is reused by the next stage
  }
  for (int c = half; c < nch; c += 2) {
    uint16_t hv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = 8 * c + u;
      double val = 0.0;
      if (valid && k < a.n) {
        val = (double)x[base + a.A * k];
        if (a.pre) val *= a.pre[base + a.A * k];
        if (F16) val *= scale;
      }
      hv[u] = to16((float)val, F16);
    }
    uint4 w;
    w.x = (uint32_t)hv[0] | ((uint32_t)hv[1] << 16);
    w.y = (uint32_t)hv[2] | ((uint32_t)hv[3] << 16);
    w.z = (uint32_t)hv[4] | ((uint32_t)hv[5] << 16);
    w.w = (uint32_t)hv[6] | ((uint32_t)hv[7] << 16);
    *reinterpret_cast<uint4*>(Abuf + core_off(r, 8 * c, a.Kp)) = w;
  }
  // make the generic-proxy shared-memory writes visible to the tensor core
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Axis 0 (A == 1): the tile's lines are one contiguous range of rows x n elements,
// read by all threads in order (coalesced); (r, k) advance incrementally. FP16 line
// maxima are combined with a shared-memory atomic max on the magnitudes' bits.
template <typename TI, bool F16>
__device__ void stage_tile_contig(const TcArgs& a, const TI* __restrict__ in, long long t, unsigned char* Abuf,
                                  unsigned* rmax, float* rscale, int* rexp) {
  const int tid = threadIdx.x;
  const long long v = t / a.tpv;
  const long long r0 = (t - v * a.tpv) * kTcRows;
  const int rows = (int)min((long long)kTcRows, a.R - r0);
  const int n = a.n, Kp = a.Kp;
  const TI* x = in + v * a.vs + r0 * n;
  const double* pr = a.pre ? a.pre + r0 * n : nullptr;
  uint16_t* A16 = reinterpret_cast<uint16_t*>(Abuf);
  const int cnt = rows * n;
  // zeros: padding columns of every line, and the lines past the end (disjoint from the data)
  const int padc = Kp - n;
  for (int e = tid; e < kTcRows * padc; e += kTcThreads) {
    const int r = e / padc, k = n + (e - r * padc);
    A16[core_off(r, k, Kp) >> 1] = 0;
  }
  for (int e = tid; e < (kTcRows - rows) * n; e += kTcThreads) {
    const int r = rows + e / n, k = e - (e / n) * n;
    A16[core_off(r, k, Kp) >> 1] = 0;
  }
  const int sr = kTcThreads / n, sk = kTcThreads - sr * n;  // advance of (r, k) per stride
  if (F16) {
    if (tid < kTcRows) rmax[tid] = 0u;
    __syncthreads();
    int r = tid / n, k = tid - r * n;
    for (int e = tid; e < cnt; e += kTcThreads) {
      double val = (double)x[e];
      if (pr) val *= pr[e];
      atomicMax(&rmax[r], __float_as_uint(fabsf((float)val)));
      r += sr;
      k += sk;
      if (k >= n) { k -= n; ++r; }
    }
    __syncthreads();
    if (tid < kTcRows) {
      const float M = __uint_as_float(rmax[tid]);
      int E = 0;
      if (M > 0.0f && isfinite(M)) frexpf(M, &E);
      rscale[tid] = ldexpf(1.0f, 14 - E);
      rexp[tid] = E - 14;
    }
    __syncthreads();
  }
  int r = tid / n, k = tid - r * n;
  for (int e = tid; e < cnt; e += kTcThreads) {
    double val = (double)x[e];
    if (pr) val *= pr[e];
    if (F16) val *= (double)rscale[r];
    A16[core_off(r, k, Kp) >> 1] = to16((float)val, F16);
    r += sr;
    k += sk;
    if (k >= n) { k -= n; ++r; }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <bool F16>
__device__ __forceinline__ void issue_mma(const TcArgs& a, uint32_t taddr, const unsigned char* Abuf,
                                          const unsigned char* Bs, int buf, uint32_t mbar) {
  const uint32_t idesc = make_idesc(a.Kp, F16);
  const uint32_t sbo = (uint32_t)(a.Kp >> 3) * 128u;
  const uint32_t a0 = smem_u32(Abuf), b0 = smem_u32(Bs);
  const uint32_t d = taddr + (uint32_t)(buf * a.Kp);
  for (int ks = 0; ks < a.Kp / 16; ++ks) {
    const uint64_t da = make_desc(a0 + ks * 256, 128, sbo);
    const uint64_t db = make_desc(b0 + ks * 256, 128, sbo);
    const uint32_t acc = ks > 0 ? 1u : 0u;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

template <typename TO, bool F16>
__device__ void epilogue_tile(const TcArgs& a, TO* __restrict__ out, long long t, uint32_t taddr, int buf,
                              const int* rexp, const float* colf) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, hw = warp >> 2;
  const int row = 32 * q + lane;
  const long long v = t / a.tpv;
  const long long r0 = (t - v * a.tpv) * kTcRows;
  const bool valid = r0 + row < a.R;
  const long long rr = r0 + row;
  const long long y = rr / a.A, xx = rr - y * a.A;
  const long long base = xx + a.A * (long long)a.n * y;
  float rowf = 1.0f;
  if (a.lam[0] && valid) {  // Lambda^{-1} of the directions other than the axis
    const int c0 = (int)(base % a.n0), c1 = (int)((base / a.n0) % a.n1), c2 = (int)(base / ((long long)a.n0 * a.n1));
    const int cc[3] = {c0, c1, c2};
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d != a.axis && a.lam[d]) rowf *= a.lam[d][cc[d]];
  }
  if (F16) rowf *= ldexpf(1.0f, rexp[row]);
  TO* o = out + v * a.vs;
  const uint32_t tbase = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * a.Kp);
  for (int c0 = 16 * hw; c0 < a.Kp; c0 += 32) {
    uint32_t d[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
        : "r"(tbase + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (valid) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int i = c0 + c;
        if (i >= a.n) break;
        const float val = __uint_as_float(d[c]) * rowf * colf[i];
        const long long idx = base + a.A * i;
        if (a.post) o[idx] = (TO)((double)val * a.post[idx]);
        else o[idx] = (TO)val;
      }
    }
  }
}

// Axis 0 epilogue: each warp moves its 32 lines x 16 columns through shared memory
// and writes them as two 16-element line segments per instruction.
template <typename TO, bool F16>
__device__ void epilogue_tile_contig(const TcArgs& a, TO* __restrict__ out, long long t, uint32_t taddr, int buf,
                                     const int* rexp, const float* colf, float* wstage) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, hw = warp >> 2;
  const int row = 32 * q + lane;
  const long long v = t / a.tpv;
  const long long r0 = (t - v * a.tpv) * kTcRows;
  const int rows = (int)min((long long)kTcRows, a.R - r0);
  const int n = a.n;
  float rowf = 1.0f;
  if (a.lam[0] && row < rows) {  // Lambda^{-1} of directions 1 and 2 (the line index)
    const long long line = r0 + row;
    const int c1 = (int)(line % a.n1), c2 = (int)(line / a.n1);
    if (a.lam[1]) rowf *= a.lam[1][c1];
    if (a.lam[2]) rowf *= a.lam[2][c2];
  }
  if (F16) rowf *= ldexpf(1.0f, rexp[row]);
  TO* o = out + v * a.vs + r0 * n;
  const double* po = a.post ? a.post + r0 * n : nullptr;
  float* W = wstage + warp * (32 * 17);
  const uint32_t tbase = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * a.Kp);
  for (int c0 = 16 * hw; c0 < a.Kp; c0 += 32) {
    uint32_t d[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
        : "r"(tbase + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int i = min(c0 + c, a.Kp - 1);
      W[lane * 17 + c] = __uint_as_float(d[c]) * rowf * colf[i];
    }
    __syncwarp();
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
      const int lr = 2 * j + (lane >> 4), c = lane & 15;
      const int rw = 32 * q + lr, i = c0 + c;
      if (rw < rows && i < n) {
        const long long idx = (long long)rw * n + i;
        const float val = W[lr * 17 + c];
        if (po) o[idx] = (TO)((double)val * po[idx]);
        else o[idx] = (TO)val;
      }
    }
    __syncwarp();
  }
}

}  // namespace

template <typename TI, typename TO, bool F16>
__global__ void __launch_bounds__(kTcThreads) k_fd_tc(TcArgs a, const TI* __restrict__ in, TO* __restrict__ out) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem);        // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + 16);
  double* rowred = reinterpret_cast<double*>(tc_smem + 64);      // [2][128]
  int* rexp = reinterpret_cast<int*>(tc_smem + 2112);            // [2][128]
  float* colf = reinterpret_cast<float*>(tc_smem + 3136);        // [256], ends at 4160 <= kHdr
  unsigned* rmax = reinterpret_cast<unsigned*>(tc_smem + 64);    // [128], axis-0 FP16 staging
  float* rscale = reinterpret_cast<float*>(tc_smem + 576);       // [128]
  unsigned char* Bs = tc_smem + kHdr;
  unsigned char* As = Bs + bmat_bytes(a.Kp);
  const uint32_t abytes = (uint32_t)kTcRows * a.Kp * 2;
  float* wstage = reinterpret_cast<float*>(As + a.nbuf * abytes);  // [8 warps][32][17], axis-0 epilogue
  const bool contig = a.A == 1;
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {  // the matrix, pre-arranged on the host: a plain 16-byte copy
    const int nvec16 = a.Kp * a.Kp * 2 / 16;
    const uint4* src = reinterpret_cast<const uint4*>(a.B);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int e = tid; e < nvec16; e += kTcThreads) dst[e] = __ldg(src + e);
  }
  const float* lam_ax = a.lam[0] ? a.lam[a.axis] : nullptr;
  for (int i = tid; i < a.Kp; i += kTcThreads) colf[i] = (lam_ax && i < a.n) ? lam_ax[i] : 1.0f;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tslot;
  const uint32_t mb[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};

  uint32_t phase = 0u, pend = 0u;  // bit b: parity to wait for / MMAs in flight on buffer b
  long long t = next_tile(a, blockIdx.x);
  auto stage = [&](long long tt, int bb) {
    if (contig) stage_tile_contig<TI, F16>(a, in, tt, As + bb * abytes, rmax, rscale, rexp + bb * kTcRows);
    else stage_tile<TI, F16>(a, in, tt, As + bb * abytes, rowred, rexp + bb * kTcRows);
  };
  if (t < a.ntiles) stage(t, 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (t < a.ntiles) {
    if (tid == 0) issue_mma<F16>(a, taddr, As, Bs, 0, mb[0]);
    pend |= 1u;
  }
  int b = 0;
  while (t < a.ntiles) {
    const long long tn = next_tile(a, t + gridDim.x);
    if (a.nbuf == 2) {
      // stage the next tile while this tile's MMAs run, then issue its MMAs
      if (tn < a.ntiles) stage(tn, b ^ 1);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tn < a.ntiles) {
        if (tid == 0) issue_mma<F16>(a, taddr, As + (b ^ 1) * abytes, Bs, b ^ 1, mb[b ^ 1]);
        pend |= 1u << (b ^ 1);
      }
    }
    const bool w = mbar_wait(mb[b], (phase >> b) & 1u);
    const bool all = __syncthreads_and(w) != 0;
    if (!all) {
      if (tid == 0) atomicExch(a.err, 1);
      break;  // buffer b stays marked in flight: waited for once more below
    }
    phase ^= 1u << b;
    pend &= ~(1u << b);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (contig) epilogue_tile_contig<TO, F16>(a, out, t, taddr, b, rexp + b * kTcRows, colf, wstage);
    else epilogue_tile<TO, F16>(a, out, t, taddr, b, rexp + b * kTcRows, colf);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (a.nbuf == 1) {
      __syncthreads();  // accumulator read out and buffer free
      if (tn < a.ntiles) stage(tn, 0);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tn < a.ntiles) {
        if (tid == 0) issue_mma<F16>(a, taddr, As, Bs, 0, mb[0]);
        pend |= 1u;
      }
    } else {
      b ^= 1;
    }
    t = tn;
  }
  for (int bb = 0; bb < 2; ++bb)  // MMAs still in flight (only after a time-out)
    if (pend & (1u << bb)) mbar_wait(mb[bb], (phase >> bb) & 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(a.ncols));
}

int tc_pad(int n) { return (n + 15) & ~15; }

namespace {

constexpr size_t kEpiStage = (size_t)(kTcThreads / 32) * 32 * 17 * sizeof(float);

size_t tc_smem_bytes(int Kp, int nbuf) {
  return kHdr + bmat_bytes(Kp) + (size_t)nbuf * kTcRows * Kp * 2 + kEpiStage;
}

int tc_nbuf(int Kp) { return tc_smem_bytes(Kp, 2) <= 227 * 1024 ? 2 : 1; }

int tc_cols(int Kp, int nbuf) {
  int c = 32;
  while (c < nbuf * Kp) c <<= 1;
  return c;
}

template <typename TI, typename TO, bool F16>
cudaError_t tc_go(cudaStream_t s, TcArgs a, int nvec, const TI* in, TO* out) {
  const size_t smem = tc_smem_bytes(a.Kp, a.nbuf);
  cudaError_t e = cudaFuncSetAttribute(k_fd_tc<TI, TO, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // tensor memory (512 columns per SM) and shared memory bound the blocks per SM
  const int per_sm = (a.ncols <= 256 && 2 * smem <= 228 * 1024) ? 2 : 1;
  a.ntiles = a.tpv * nvec;
  const long long grid = std::min<long long>(a.ntiles, (long long)per_sm * nsm);
  if (grid <= 0) return cudaSuccess;
  k_fd_tc<TI, TO, F16><<<(unsigned)grid, kTcThreads, smem, s>>>(a, in, out);
  return cudaGetLastError();
}

}  // namespace

// Host: the applied matrix Mat (i, j) (i output, j summed) in the K-major
// core-matrix layout of the B operand (rows i, K = j), zero-padded to Kp x Kp,
// as BF16 or FP16 bits.
void tc_arrange(int n, const double* Mat_ij /* row-major n x n: Mat(i,j) at i*n+j */, bool f16,
                std::vector<uint16_t>& outbits) {
  const int Kp = tc_pad(n);
  outbits.assign((size_t)Kp * Kp, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      uint16_t bits;
      if (f16) {
        const __half b = __float2half_rn((float)Mat_ij[(size_t)i * n + j]);
        memcpy(&bits, &b, 2);
      } else {
        const __nv_bfloat16 b = __float2bfloat16((float)Mat_ij[(size_t)i * n + j]);
        memcpy(&bits, &b, 2);
      }
      const size_t off = ((size_t)(i >> 3) * (Kp >> 3) * 128 + (size_t)(j >> 3) * 128 + (i & 7) * 16 + (j & 7) * 2) / 2;
      outbits[off] = bits;
    }
}

cudaError_t launch_fd_mode_tc(cudaStream_t s, int n, int axis, AxisShape sh, int nvec, const int* active,
                              const void* B, int f16, const void* in, int in_is_double, void* out, int out_is_double,
                              long long vs, const double* pre, const double* post, const float* const* lam,
                              const int* nn, int* err) {
  const int Kp = tc_pad(n);
  if (Kp > 256 || n < 1 || nvec < 1) return cudaErrorInvalidValue;
  TcArgs a{};
  a.n = n;
  a.Kp = Kp;
  a.nbuf = tc_nbuf(Kp);
  a.ncols = tc_cols(Kp, a.nbuf);
  a.axis = axis;
  a.A = sh.A;
  a.R = sh.A * sh.B;
  a.tpv = (a.R + kTcRows - 1) / kTcRows;
  a.vs = vs;
  a.B = static_cast<const uint16_t*>(B);
  a.active = active;
  a.pre = pre;
  a.post = post;
  for (int d = 0; d < 3; ++d) a.lam[d] = lam ? lam[d] : nullptr;
  a.n0 = nn ? nn[0] : 1;
  a.n1 = nn ? nn[1] : 1;
  a.err = err;
  if (a.R < 1) return cudaSuccess;
#define IGA_TC(TI, TO)                                                                                  \
  return f16 ? tc_go<TI, TO, true>(s, a, nvec, static_cast<const TI*>(in), static_cast<TO*>(out))     \
             : tc_go<TI, TO, false>(s, a, nvec, static_cast<const TI*>(in), static_cast<TO*>(out))
  if (in_is_double && !out_is_double) IGA_TC(double, float);
  if (!in_is_double && !out_is_double) IGA_TC(float, float);
  if (!in_is_double && out_is_double) IGA_TC(float, double);
  IGA_TC(double, double);
#undef IGA_TC
}

}  // namespace iga
