// Double-FP32 ("double-float") form of the assembled band product.
//
// The band product does one multiply-add per stored coupling, and in FP64 it is
// bound by the FP64 units, which on GB300 run at 1/64 of the FP32 rate. This form
// carries every number as an unevaluated sum of two FP32 numbers instead:
//  * a matrix or a vector is first scaled by a power of two, one per matrix and one
//    per vector, that brings its largest magnitude into [1, 2) (nothing then
//    overflows, and what would underflow lies far below the rounding of the
//    result); each entry v is split into hi = fl32(v) and lo = fl32(v - hi), which
//    keeps 48 significant bits;
//  * each term a x is formed exactly up to the product of the two low parts:
//    p = fl32(ah xh) and e = (ah xh - p) + ah xl + al xh by fused multiply-adds (the
//    first one exact, Dekker's product by FMA);
//  * the p are summed with Knuth's TwoSum, which gives the rounded sum s and the
//    exact error t of every addition; the t and e go into a second FP32 sum c, and
//    after each run of consecutive slots (s, c) is renormalised (Fast2Sum);
//  * y = (fl64(s) + fl64(c)) 2^(E_x + E_A).
// The error of a row is a few 2^-48 of sum_j |a_ij x_j| (FP64: a few 2^-53). The
// per-vector exponent needs the vector's largest magnitude before the split, hence
// three launches per product: block maxima, exponent and split, band product.
//
// Storage: A[h][pad + i] as float2 (hi, lo) with a row stride Np = N + 2 pad and
// zero pads, h the stored slot of the upper half (kernels_band.cu): the pads make
// every neighbour index of a row whose neighbour grid line exists an in-bounds
// read, so the inner loop has no bounds checks. The upper half is walked as runs:
// the slots sharing (o1, o2) have consecutive h and consecutive linear offsets.
// Every launch configuration computes each row with the same operations in the
// same order.
#include <algorithm>

#include "iga_internal.h"

namespace iga {

namespace {

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// exponent E with max|v| 2^-E in [1, 2) from the bit pattern of max|v|; 0 for an
// all-zero vector and for inf / NaN (these then propagate into the result)
__device__ __forceinline__ int df_exponent(unsigned long long mb) {
  const int be = (int)(mb >> 52);
  if (mb == 0 || be == 0x7ff) return 0;
  return be == 0 ? -1022 : be - 1023;
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long m) {
  __shared__ unsigned long long sm[32];
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = m;
  __syncthreads();
  if (w == 0) {
    m = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ULL;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sm[0] = m;
  }
  __syncthreads();
  m = sm[0];
  __syncthreads();
  return m;
}

// part[v][blockIdx.x] = max_i |x[v][i]| over the block's grid-stride share (as bits)
__global__ void k_df_absmax(long long n, const int* __restrict__ active, const double* __restrict__ x, long long vs,
                            unsigned long long* __restrict__ part) {
  const int v = blockIdx.y;
  unsigned long long m = 0;
  if (!active || active[v])
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      m = max(m, abs_bits(x[v * vs + i]));
  m = block_max(m);
  if (threadIdx.x == 0) part[(long long)v * gridDim.x + blockIdx.x] = m;
}

// E_v from the G partial maxima (or Efix[0] for every vector); xs[v][pad + i] =
// split(x[v][i] 2^-E_v). Eout[v] = E_v (written by block 0).
__global__ void k_df_split(long long n, int G, const int* __restrict__ active, const double* __restrict__ x,
                           long long vs, const unsigned long long* __restrict__ part, const int* __restrict__ Efix,
                           float2* __restrict__ xs, long long xvs, int* __restrict__ Eout) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;  // uniform over the block
  int E;
  if (Efix) {
    E = Efix[0];
  } else {
    unsigned long long m = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) m = max(m, part[(long long)v * G + b]);
    E = df_exponent(block_max(m));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && Eout) Eout[v] = E;
  const double sc = ldexp(1.0, -E);
  float2* out = xs + (long long)v * xvs + kDfPad;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = x[v * vs + i] * sc;
    const float hi = __double2float_rn(w);
    out[i] = make_float2(hi, __double2float_rn(w - (double)hi));
  }
}

// s + c += a x (see the file comment); the intrinsics keep every rounding explicit
__device__ __forceinline__ void df_term(float& s, float& c, const float2 a, const float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  float e = __fmaf_rn(a.x, x.x, -p);
  e = __fmaf_rn(a.x, x.y, e);
  e = __fmaf_rn(a.y, x.x, e);
  const float S = __fadd_rn(s, p);
  const float bp = __fsub_rn(S, s);
  const float t = __fadd_rn(__fsub_rn(s, __fsub_rn(S, bp)), __fsub_rn(p, bp));
  c = __fadd_rn(c, __fadd_rn(t, e));
  s = S;
}

template <int NV, int BS>
__global__ void __launch_bounds__(BS) k_band_df(long long N, int nruns, const int4* __restrict__ runs, int n0, int n1,
                                                int n2, const float2* __restrict__ A, long long Np, int EA,
                                                const int* __restrict__ active, int nvec,
                                                const float2* __restrict__ xs, const int* __restrict__ Ex,
                                                const double* __restrict__ x, double* __restrict__ y, long long vs,
                                                double* __restrict__ pq) {
  const long long i = (long long)blockIdx.x * BS + threadIdx.x;
  const bool row = i < N;  // no early return: the run votes need every lane
  const int v0 = blockIdx.y * NV;
  bool on[NV];
  float s[NV], c[NV];
  const float2* xv[NV];  // row pad + i of each vector's split copy
  const float2 a0 = row ? A[kDfPad + i] : make_float2(0.f, 0.f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = min(v0 + v, nvec - 1);
    on[v] = row && v0 + v < nvec && (!active || active[vv]);
    xv[v] = xs + (long long)vv * Np + kDfPad + i;
    s[v] = 0.f;
    c[v] = 0.f;
    if (on[v]) df_term(s[v], c[v], a0, xv[v][0]);
  }
  int i1 = 0, i2 = 0;
  if (row) {
    const long long t = i / n0;
    i1 = (int)(t % n1);
    i2 = (int)(t / n1);
  }
  for (int r = 0; r < nruns; ++r) {
    const int4 R = runs[r];  // first slot, length, packed (o1, o2), linear offset of the first slot
    const int o1 = (R.z & 255) - 64, o2 = ((R.z >> 8) & 255) - 64;
    const bool up = row && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
    const bool dn = row && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
    if (!__any_sync(0xffffffffu, up || dn)) continue;
    // upper term of slot h0 + t: A[h0 + t][i], x[i + L0 + t]; lower term: A[h0 + t][i - L0 - t], x[i - L0 - t]
    const float2* au = A + (long long)R.x * Np + kDfPad + i;
    const float2* ad = au - R.w;
    const int L0 = R.w;
    for (int t = 0; t < R.y; ++t) {
      if (up) {
        const float2 a = au[(long long)t * Np];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (on[v]) df_term(s[v], c[v], a, xv[v][L0 + t]);
      }
      if (dn) {
        const float2 a = ad[(long long)t * (Np - 1)];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (on[v]) df_term(s[v], c[v], a, xv[v][-L0 - t]);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {  // Fast2Sum renormalisation, |c| <= |s| ulp-wise
      const float S = __fadd_rn(s[v], c[v]);
      c[v] = __fsub_rn(c[v], __fsub_rn(S, s[v]));
      s[v] = S;
    }
  }
  double out[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    out[v] = 0.0;
    if (on[v]) {
      const int vv = v0 + v;
      out[v] = ((double)s[v] + (double)c[v]) * ldexp(1.0, Ex[vv] + EA);
      y[vv * vs + i] = out[v];
    }
  }
  if (pq) {  // fixed-order block sums of x_i y_i: warps by shuffles, then the warps in order
    __shared__ double sred[BS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vv = v0 + v;
      if (vv >= nvec) break;
      double t = on[v] ? x[vv * vs + i] * out[v] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) sred[w] = t;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int q = 0; q < BS / 32; ++q) sum += sred[q];
        pq[(long long)vv * gridDim.x + blockIdx.x] = sum;
      }
      __syncthreads();
    }
  }
}

template <int BS>
int band_df_go(cudaStream_t s, int nv, long long N, int nruns, const int4* runs, const int* n, const float2* A,
               long long Np, int EA, const int* active, int nvec, const float2* xs, const int* Ex, const double* x,
               double* y, long long vs, double* pq) {
  const dim3 grid((unsigned)((N + BS - 1) / BS), (unsigned)((nvec + nv - 1) / nv));
  const int n0 = n[0], n1 = n[1], n2 = n[2];
#define IGA_DF_GO(NVV) \
  k_band_df<NVV, BS><<<grid, BS, 0, s>>>(N, nruns, runs, n0, n1, n2, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq)
  switch (nv) {
    case 1: IGA_DF_GO(1); break;
    case 2: IGA_DF_GO(2); break;
    case 3: IGA_DF_GO(3); break;
    default: IGA_DF_GO(4); break;
  }
#undef IGA_DF_GO
  return (int)grid.x;
}

}  // namespace

std::vector<int> band_df_runs(const int* n, const int* p) {
  const int m0 = 2 * p[0] + 1, m1 = 2 * p[1] + 1, m2 = 2 * p[2] + 1;
  const int centre = m0 * m1 * m2 / 2;
  const int qc = centre / m0;  // (o1, o2) = (0, 0)
  std::vector<int> out;
  for (int q = qc; q < m1 * m2; ++q) {
    const int o1 = q % m1 - p[1], o2 = q / m1 - p[2];
    const int first_o0 = q == qc ? 1 : -p[0];
    const int len = q == qc ? p[0] : m0;
    if (len == 0) continue;
    const int h0 = m0 * q + (first_o0 + p[0]) - centre;
    const long long L0 = first_o0 + (long long)n[0] * (o1 + (long long)n[1] * o2);
    out.push_back(h0);
    out.push_back(len);
    out.push_back((o1 + 64) | ((o2 + 64) << 8));
    out.push_back((int)L0);
  }
  return out;
}

cudaError_t launch_df_split_matrix(cudaStream_t s, long long N, int H, const double* A, float2* Adf, long long Np,
                                   unsigned long long* part, int* dE) {
  k_df_absmax<<<dim3(kDfBlocks, 1), 256, 0, s>>>((long long)H * N, nullptr, A, 0, part);
  k_df_split<<<dim3(1, 1), 256, 0, s>>>(0, kDfBlocks, nullptr, A, 0, part, nullptr, Adf, Np, dE);
  const unsigned gx = (unsigned)std::min<long long>((N + 255) / 256, 1024);
  k_df_split<<<dim3(gx, (unsigned)H), 256, 0, s>>>(N, 0, nullptr, A, N, nullptr, dE, Adf, Np, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_df_split(cudaStream_t s, long long N, const int* active, int nvec, const double* x, long long vs,
                            float2* xs, long long Np, int* Ex, unsigned long long* part) {
  k_df_absmax<<<dim3(kDfBlocks, nvec), 256, 0, s>>>(N, active, x, vs, part);
  const unsigned gx = (unsigned)std::min<long long>((N + 255) / 256, 2 * kDfBlocks);
  k_df_split<<<dim3(gx, nvec), 256, 0, s>>>(N, kDfBlocks, active, x, vs, part, nullptr, xs, Np, Ex);
  return cudaGetLastError();
}

cudaError_t launch_band_df(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, const float2* A,
                           long long Np, int EA, const int* active, int nvec, const float2* xs, const int* Ex,
                           const double* x, double* y, long long vs, int threads, int nv, double* pq, int* npq) {
  if (nv <= 0) nv = nvec < 4 ? nvec : 4;
  if (nv < 1) nv = 1;
  if (nv > 4) nv = 4;
  int nb;
  if (threads == 64) nb = band_df_go<64>(s, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else if (threads == 128) nb = band_df_go<128>(s, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else if (threads == 512) nb = band_df_go<512>(s, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else nb = band_df_go<256>(s, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  if (npq) *npq = nb;
  return cudaGetLastError();
}

}  // namespace iga
