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
// same order: the diagonal term, then per run the upper terms and the lower terms
// of the sides whose neighbour line exists, then a renormalisation if the row
// computed any term of the run. Nothing a row computes depends on other rows, so
// all launch shapes (rows per block and per thread, vectors per pass, the order of
// the blocks) give bitwise equal products.
//
// Block order: the lower terms of a row reach up to p2 planes back (the coefficients
// were read as upper terms of those planes' rows). The blocks of the tensor-map
// kernels walk the grid in strips of W1 lines of direction 1, plane after plane
// within a strip, with W1 chosen so that the last p2 planes of a strip (their
// coefficients) fit in a part of L2: the lower terms then come from L2 instead of
// DRAM. A block owns the rows of one strip-plane that fall in its window of R rows
// (window starts even, for the tensor copies' 16-byte alignment).
#include <algorithm>
#include <array>

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

// (hi, lo) of w = x 2^-E by integer operations on x's bits: hi = w rounded to 24
// significant bits (to nearest, ties to even: the 53-bit significand cut after 24 bits),
// lo = the exact remainder w - hi (an integer of at most 29 bits times 2^(e - 52))
// rounded to FP32. The same values as __double2float_rn(w) and __double2float_rn(w - hi),
// without the FP64 conversions, which GB300 runs on its narrow FP64 units. Zero, subnormal,
// infinite and NaN entries, and w outside [2^-74, 4) (hi or the scaled remainder would
// leave FP32's normal range), take that FP64 path (sc = 2^-E).
__device__ __forceinline__ float2 df_split_entry(double x, int E, double sc) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  if (e == 0 && m == 0) return make_float2(__uint_as_float(sign << 31), 0.0f);
  const int ep = e - E;  // biased exponent of w
  if (e == 0 || e == 0x7FF || ep < 949 || ep > 1024) {
    const double w = x * sc;
    const float hi = __double2float_rn(w);
    return make_float2(hi, __double2float_rn(w - (double)hi));
  }
  const unsigned long long M = m | (1ULL << 52);
  unsigned q = (unsigned)(M >> 29);
  const int rem = (int)(M & 0x1FFFFFFFULL);
  int fe = ep - 896;  // FP32 biased exponent
  int r = rem;
  if (rem > (1 << 28) || (rem == (1 << 28) && (q & 1u))) {
    ++q;
    r = rem - (1 << 29);
  }
  if (q == (1u << 24)) {
    q = 1u << 23;
    ++fe;
  }
  const float hi = __uint_as_float((sign << 31) | ((unsigned)fe << 23) | (q & 0x7FFFFFu));
  float lo = 0.0f;
  if (r != 0) {
    lo = __fmul_rn(__int2float_rn(r), __uint_as_float((unsigned)(ep - 948) << 23));  // r 2^(ep - 1075)
    if (sign) lo = -lo;
  }
  return make_float2(hi, lo);
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
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = df_split_entry(x[v * vs + i], E, sc);
}

// The two passes of a vector split in one cooperative launch (two blocks per SM; eight
// entries per thread and pass with their loads issued together):
// block maxima, a grid barrier, then every block reduces the maxima and splits its
// grid-stride share. With z, the first pass also forms the PCG direction x = z + beta x
// (active systems; the same operation as k_cg_update_p; beta given, or computed by every
// block from the r.z partials, BetaArgs) before taking
// the maxima, and the second pass splits what the same thread wrote. bar[0] counts
// arrivals, bar[1] is the barrier's generation; the wait is bounded by `limit` polls of
// at least 64 ns (err = 1 if it runs out; the results are then not to be used). Every
// block arrives whether or not it waited, so the last one always resets the count.
constexpr long long kBarLimit = 1LL << 22;  // default poll limit (about 0.3 s or more)

__global__ void __launch_bounds__(256) k_df_split_coop(long long n, int nvec, const int* __restrict__ active,
                                                       double* __restrict__ x, const double* __restrict__ z,
                                                       const BetaArgs ba, long long vs,
                                                       unsigned long long* __restrict__ part,
                                                       float2* __restrict__ xs, long long xvs, int* __restrict__ Eout,
                                                       unsigned int* bar, int* err, long long limit) {
  const int G = gridDim.x;
  // beta per system: from c, or computed here by every block from the r.z partials
  __shared__ double sbeta[kMaxVec], srz[kMaxVec], srz2[kMaxVec];
  if (z) {
    if (ba.rzp) {
      reduce_partials(nvec, ba.rzp, srz, ba.nrz);
      if (ba.flexible) reduce_partials(nvec, ba.rzp + (long long)nvec * ba.nrz, srz2, ba.nrz);
      const int v = threadIdx.x;
      if (v < nvec) {
        sbeta[v] = 0.0;
        if (!active || active[v]) sbeta[v] = (ba.flexible ? srz[v] - srz2[v] : srz[v]) / ba.c.rz[v];
      }
    } else if ((int)threadIdx.x < nvec) {
      sbeta[threadIdx.x] = ba.c.beta[threadIdx.x];
    }
    __syncthreads();
  }
  const long long stride = (long long)G * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int U = 8;  // entries per thread and pass, their loads issued together
  for (int v = 0; v < nvec; ++v) {
    unsigned long long m = 0;
    if (!active || active[v]) {
      double* xv = x + v * vs;
      if (z) {
        const double b = sbeta[v];
        const double* zv = z + v * vs;
        for (long long i = i0; i < n; i += U * stride) {
          double xa[U], za[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long iu = i + u * stride;
            xa[u] = iu < n ? xv[iu] : 0.0;
            za[u] = iu < n ? zv[iu] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const long long iu = i + u * stride;
            if (iu < n) {
              const double pn = fma(b, xa[u], za[u]);
              xv[iu] = pn;
              m = max(m, abs_bits(pn));
            }
          }
        }
      } else {
        for (long long i = i0; i < n; i += U * stride) {
          double xa[U];
#pragma unroll
          for (int u = 0; u < U; ++u) xa[u] = i + u * stride < n ? xv[i + u * stride] : 0.0;
#pragma unroll
          for (int u = 0; u < U; ++u) m = max(m, abs_bits(xa[u]));
        }
      }
    }
    m = block_max(m);
    if (threadIdx.x == 0) part[(long long)v * G + blockIdx.x] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    volatile unsigned int* gen = bar + 1;
    const unsigned int g0 = *gen;
    if (atomicAdd(bar, 1u) == (unsigned int)G - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g0) {
        if (++it > limit) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  // every block has read c.rz (above): block 0 records beta and the new r.z
  if (z && ba.rzp && blockIdx.x == 0 && (int)threadIdx.x < nvec && (!active || active[threadIdx.x])) {
    ba.c.beta[threadIdx.x] = sbeta[threadIdx.x];
    ba.c.rz[threadIdx.x] = srz[threadIdx.x];
  }
  for (int v = 0; v < nvec; ++v) {
    if (active && !active[v]) continue;  // uniform over the block
    unsigned long long m = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) m = max(m, *(volatile unsigned long long*)&part[(long long)v * G + b]);
    const int E = df_exponent(block_max(m));
    if (blockIdx.x == 0 && threadIdx.x == 0) Eout[v] = E;
    const double sc = ldexp(1.0, -E);
    float2* out = xs + (long long)v * xvs + kDfPad;
    const double* xv = x + v * vs;
    for (long long i = i0; i < n; i += U * stride) {
      double xa[U];
#pragma unroll
      for (int u = 0; u < U; ++u) xa[u] = i + u * stride < n ? xv[i + u * stride] : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (i + u * stride < n) out[i + u * stride] = df_split_entry(xa[u], E, sc);
    }
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

// A term of a tiny slot -- a slot whose coefficients all lie below 2^-24 after the
// matrix's scaling (its largest coefficient in [1, 2)) -- is one FP32 multiply-add of
// the high parts into c. Its error, at most 2^-23 |a x| < 2^-47 max|A| |x|, is of the
// order of the (hi, lo) representation error of the matrix's largest coefficients, so
// the exact product and the low parts would add nothing the result keeps.
__device__ __forceinline__ void df_term_tiny(float& c, const float2 a, const float2 x) {
  c = __fmaf_rn(a.x, x.x, c);
}

// slot t of a run of len slots whose m first and m last slots are tiny
__device__ __forceinline__ bool df_is_tiny(int t, int len, int m) { return t < m || t >= len - m; }

__device__ __forceinline__ void df_term_m(float& s, float& c, const float2 a, const float2 x, bool tiny) {
  if (tiny) df_term_tiny(c, a, x);
  else df_term(s, c, a, x);
}

// the tiny-end count m of a run (bits 16..19 of its packed offsets; 0 for run 0)
__device__ __forceinline__ int df_run_m(const int4& R) { return (R.z >> 16) & 15; }

// Fast2Sum renormalisation of (s, c): |c| is at most a few ulps of s; only for rows
// that computed a term of the run (on)
template <int NV>
__device__ __forceinline__ void df_renorm(float (&s)[NV], float (&c)[NV], bool on) {
  if (!on) return;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float S = __fadd_rn(s[v], c[v]);
    c[v] = __fsub_rn(c[v], __fsub_rn(S, s[v]));
    s[v] = S;
  }
}

// The terms of one run: slot h0 + t contributes A[h0 + t][i] x[i + L0 + t] (upper, when
// the neighbour lines exist: up) and A[h0 + t][i - L0 - t] x[i - L0 - t] (lower: dn).
// au = &A[h0][i], ad = &A[h0][i - L0], xu[v] = &x_v[i + L0], xd[v] = &x_v[i - L0].
// LEN > 0: a compile-time length (the loads of the run can all be issued at once);
// LEN == 0: the runtime length len. m: the run's tiny-end count (df_is_tiny).
template <int LEN, int NV>
__device__ __forceinline__ void df_run(int len, int m, bool up, bool dn, const float2* __restrict__ au,
                                       const float2* __restrict__ ad, long long Np, const float2* const (&xu)[NV],
                                       const float2* const (&xd)[NV], float (&s)[NV], float (&c)[NV]) {
  // the upper terms of the run, then the lower ones
  if constexpr (LEN > 0) {
    if (up) {
#pragma unroll
      for (int t = 0; t < LEN; ++t) {
        const float2 a = au[t * Np];
        const bool tn = df_is_tiny(t, LEN > 0 ? LEN : len, m);
#pragma unroll
        for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xu[v][t], tn);
      }
    }
    if (dn) {
#pragma unroll
      for (int t = 0; t < LEN; ++t) {
        const float2 a = ad[t * (Np - 1)];
        const bool tn = df_is_tiny(t, LEN > 0 ? LEN : len, m);
#pragma unroll
        for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xd[v][-t], tn);
      }
    }
  } else {
    if (up) {
#pragma unroll 1
      for (int t = 0; t < len; ++t) {
        const float2 a = au[t * Np];
        const bool tn = df_is_tiny(t, LEN > 0 ? LEN : len, m);
#pragma unroll
        for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xu[v][t], tn);
      }
    }
    if (dn) {
#pragma unroll 1
      for (int t = 0; t < len; ++t) {
        const float2 a = ad[t * (Np - 1)];
        const bool tn = df_is_tiny(t, LEN > 0 ? LEN : len, m);
#pragma unroll
        for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xd[v][-t], tn);
      }
    }
  }
}

// The rows of block b for blocks of R rows in strip order: the copy window starts at
// *i0c (even), the block's rows are [*lo, *hi) (empty for a block past the strip-plane).
__device__ __forceinline__ void df_block_rows(const DfStrips& g, int R, long long b, long long* i0c, long long* lo,
                                              long long* hi) {
  const long long per0 = (long long)g.n2 * g.nb0;
  long long sg = b / per0, rem;
  int nb;
  if (sg >= g.S - 1) {
    sg = g.S - 1;
    rem = b - (long long)(g.S - 1) * per0;
    nb = g.nbl;
  } else {
    rem = b - sg * per0;
    nb = g.nb0;
  }
  const long long i2 = rem / nb, q = rem - i2 * nb;
  const long long l1 = sg * g.W1;
  const long long w = min((long long)g.W1, (long long)g.n1 - l1);
  const long long a = (long long)g.n0 * (l1 + (long long)g.n1 * i2);
  const long long e = a + w * g.n0;
  const long long c = (a & ~1LL) + q * R;
  *i0c = c;
  *lo = max(a, c);
  *hi = min(e, c + R);
}

// P0: the degree along direction 0 when compiled for it (run lengths P0 and 2 P0 + 1),
// 0 for any degree. A vector slot past nvec repeats the last vector's arithmetic and
// an inactive vector is computed from its stale split copy; neither is stored, so the
// inner loop carries no per-vector conditions.
template <int P0, int NV, int BS>
__global__ void __launch_bounds__(BS) k_band_df(long long N, int nruns, const int4* __restrict__ runs, int n0, int n1,
                                                int n2, const float2* __restrict__ A, long long Np, int EA,
                                                const int* __restrict__ active, int nvec,
                                                const float2* __restrict__ xs, const int* __restrict__ Ex,
                                                const double* __restrict__ x, double* __restrict__ y, long long vs,
                                                double* __restrict__ pq, DfStrips g) {
  long long i0c, lo, hi;
  df_block_rows(g, BS, blockIdx.x, &i0c, &lo, &hi);
  const long long i = i0c + threadIdx.x;
  const bool row = i >= lo && i < hi;  // no early return: the run votes need every lane
  const int v0 = blockIdx.y * NV;
  float s[NV], c[NV];
  const float2* xv[NV];  // row pad + i of each vector's split copy
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    xv[v] = xs + (long long)min(v0 + v, nvec - 1) * Np + kDfPad + i;
    s[v] = 0.f;
    c[v] = 0.f;
  }
  if (row) {
    const float2 a0 = A[kDfPad + i];
#pragma unroll
    for (int v = 0; v < NV; ++v) df_term(s[v], c[v], a0, xv[v][0]);
  }
  int i1 = 0, i2 = 0;
  if (row) {
    const long long t = i / n0;
    i1 = (int)(t % n1);
    i2 = (int)(t / n1);
  }
  for (int r = 0; r < nruns; ++r) {
    const int4 R = runs[r];  // first slot, length, packed (o1, o2), linear offset of the first slot
    bool up = row, dn = row;
    if (r > 0) {  // run 0 is (o1, o2) = (0, 0): both neighbour lines are the row's own
      const int o1 = (R.z & 255) - 64, o2 = ((R.z >> 8) & 255) - 64;
      up = up && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
      dn = dn && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
      if (!__any_sync(0xffffffffu, up || dn)) continue;
    }
    const float2* au = A + (long long)R.x * Np + kDfPad + i;
    const float2* ad = au - R.w;
    const float2* xu[NV];
    const float2* xd[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      xu[v] = xv[v] + R.w;
      xd[v] = xv[v] - R.w;
    }
    const int m = df_run_m(R);
    if (P0 > 0) {
      if (r == 0) df_run<P0, NV>(0, 0, up, dn, au, ad, Np, xu, xd, s, c);
      else df_run<2 * P0 + 1, NV>(0, m, up, dn, au, ad, Np, xu, xd, s, c);
    } else {
      df_run<0, NV>(R.y, m, up, dn, au, ad, Np, xu, xd, s, c);
    }
    df_renorm<NV>(s, c, up || dn);
  }
  bool on[NV];
  double out[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = v0 + v;
    on[v] = row && vv < nvec && (!active || active[vv]);
    out[v] = 0.0;
    if (on[v]) {
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

// ---------------------------------------------------------------------------
// TMA-staged form: a block owns R consecutive rows and walks the runs; a producer
// warp stages each run's operands into a ring of kStages shared-memory buffers with
// bulk copies (cp.async.bulk, completion on an mbarrier) as soon as the consumer
// warps release a buffer, and the consumers (one row per thread) compute from
// shared memory. Per run and buffer:
//   cu[t][j]  = A[h0 + t][i0 + j]                  (upper terms, t < len, j < R)
//   cd[t][.]  = A[h0 + t][i0 - L0 - t + j]         (lower terms; the copy starts at the
//               even index at or below, so the row sits at offset (L0 + t) & 1)
//   xu[v][.]  = x_v[i0 + L0 + j'],  xd[v][.] = x_v[i0 - L0 - (len - 1) + j']  (j' < W,
//               same rounding: offset L0 & 1, resp. (L0 + len - 1) & 1)
// Every index is relative to the padded row layout; the split arrays carry slack
// before and after (kDfSlack) so that every copy lies inside its allocation; rows
// whose neighbour line is outside the grid read slack or other rows but are
// predicated off, exactly as in the register form. The arithmetic, its order and the
// per-warp run votes (which decide the renormalisations) are those of k_band_df.
// buffers in the ring: more for smaller blocks (more blocks per SM share the same
// shared memory, each needs enough runs in flight)
__host__ __device__ constexpr int df_stages(int R) { return R <= 64 ? 4 : (R <= 128 ? 3 : 2); }
constexpr long long kTmaWaitLimit = 1LL << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < kTmaWaitLimit; ++it)
    if (mbar_try(mbar, phase)) return true;
  return false;
}

template <int P0, int NV, int R>
struct DfStage {
  static constexpr int M0 = 2 * P0 + 1;
  static constexpr int W = R + M0 + 1;  // x span length (even)
  static constexpr int CU = 0;
  static constexpr int CD = CU + M0 * R;
  static constexpr int XU = CD + M0 * (R + 2);
  static constexpr int XD = XU + NV * W;
  static constexpr int ELEMS = XD + NV * W;  // float2 per buffer
  static constexpr size_t BYTES = (size_t)ELEMS * 8;
};

// issue the copies of run r (length LEN) into buffer b
template <int P0, int NV, int R, int LEN>
__device__ __forceinline__ void df_issue(const int4 R4, float2* buf, uint32_t mbar, const float2* A, long long Np,
                                         long long i0, const float2* xs, int v0, int nvec) {
  using St = DfStage<P0, NV, R>;
  const long long h0 = R4.x, L0 = R4.w;
  constexpr uint32_t bytes = (uint32_t)((LEN * R + LEN * (R + 2) + 2 * NV * St::W) * 8);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
#pragma unroll
  for (int t = 0; t < LEN; ++t) {
    const long long eu = (h0 + t) * Np + kDfPad + i0;
    bulk_g2s(s_u32(buf + St::CU + t * R), A + eu, R * 8, mbar);
    const long long ed = eu - L0 - t;
    bulk_g2s(s_u32(buf + St::CD + t * (R + 2)), A + (ed & ~1LL), (R + 2) * 8, mbar);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long base = (long long)min(v0 + v, nvec - 1) * Np + kDfPad + i0;
    bulk_g2s(s_u32(buf + St::XU + v * St::W), xs + ((base + L0) & ~1LL), St::W * 8, mbar);
    bulk_g2s(s_u32(buf + St::XD + v * St::W), xs + ((base - L0 - (LEN - 1)) & ~1LL), St::W * 8, mbar);
  }
}

// the terms of run (LEN slots) from buffer buf for row j of the block: the upper
// terms, then the lower ones, as in df_run
template <int P0, int NV, int R, int LEN>
__device__ __forceinline__ void df_run_smem(const float2* buf, int j, int L0, int m, bool up, bool dn, float (&s)[NV],
                                            float (&c)[NV]) {
  using St = DfStage<P0, NV, R>;
  if (up) {
    const float2* xu = buf + St::XU + (L0 & 1) + j;
#pragma unroll
    for (int t = 0; t < LEN; ++t) {
      const float2 a = buf[St::CU + t * R + j];
      const bool tn = df_is_tiny(t, LEN, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xu[v * St::W + t], tn);
    }
  }
  if (dn) {
    const float2* xd = buf + St::XD + ((L0 + LEN - 1) & 1) + j + (LEN - 1);
    const float2* cd0 = buf + St::CD + (L0 & 1) + j;        // even t
    const float2* cd1 = buf + St::CD + ((L0 + 1) & 1) + j;  // odd t
#pragma unroll
    for (int t = 0; t < LEN; ++t) {
      const float2 a = ((t & 1) ? cd1 : cd0)[t * (R + 2)];
      const bool tn = df_is_tiny(t, LEN, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) df_term_m(s[v], c[v], a, xd[v * St::W - t], tn);
    }
  }
}

// Warp-specialised: R / 32 consumer warps (one row per thread) and one producer warp
// whose lane 0 issues the copies. full[b] completes when run r's copies into buffer
// b = r mod kStages have landed; empty[b] when every consumer warp is done with it.
template <int P0, int NV, int R>
__global__ void __launch_bounds__(R + 32) k_band_df_tma(long long N, int nruns, const int4* __restrict__ runs, int n0,
                                                        int n1, int n2, const float2* __restrict__ A, long long Np,
                                                        int EA, const int* __restrict__ active, int nvec,
                                                        const float2* __restrict__ xs, const int* __restrict__ Ex,
                                                        const double* __restrict__ x, double* __restrict__ y,
                                                        long long vs, double* __restrict__ pq, int* __restrict__ err) {
  using St = DfStage<P0, NV, R>;
  constexpr int M0 = St::M0;
  constexpr int NW = R / 32;  // consumer warps
  constexpr int kStages = df_stages(R);
  extern __shared__ __align__(128) float2 dsm[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
  const int j = threadIdx.x;
  const int lane = j & 31;
  const long long i0 = (long long)blockIdx.x * R;
  const int v0 = blockIdx.y * NV;
  if (j == 0) {
    for (int b = 0; b < kStages; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(&empty[b])), "r"(NW));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long i = i0 + j;
  const bool row = j < R && i < N;
  float s[NV], c[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    s[v] = 0.f;
    c[v] = 0.f;
  }
  if (j >= R) {  // producer warp
    if (lane == 0) {
      bool ok = true;
      int last = -1;
      for (int r = 0; r < nruns; ++r) {
        const int b = r % kStages, k = r / kStages;
        if (k > 0 && !mbar_wait_bounded(s_u32(&empty[b]), (uint32_t)((k - 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        float2* buf = dsm + (size_t)b * St::ELEMS;
        if (r == 0) df_issue<P0, NV, R, P0>(runs[0], buf, s_u32(&full[b]), A, Np, i0, xs, v0, nvec);
        else df_issue<P0, NV, R, M0>(runs[r], buf, s_u32(&full[b]), A, Np, i0, xs, v0, nvec);
        last = r;
      }
      if (!ok) atomicExch(err, 1);
      // let every copy in flight land before the block can leave
      for (int q = last - kStages + 1; q <= last; ++q)
        if (q >= 0) mbar_wait_bounded(s_u32(&full[q % kStages]), (uint32_t)((q / kStages) & 1));
    }
  } else {  // consumer warps
    if (row) {
      const float2 a0 = A[kDfPad + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) df_term(s[v], c[v], a0, xs[(long long)min(v0 + v, nvec - 1) * Np + kDfPad + i]);
    }
    int i1 = 0, i2 = 0;
    if (row) {
      const long long t = i / n0;
      i1 = (int)(t % n1);
      i2 = (int)(t / n1);
    }
    bool ok = true;
    for (int r = 0; r < nruns; ++r) {
      const int b = r % kStages;
      const int4 R4 = runs[r];
      bool up = row, dn = row;
      if (r > 0) {
        const int o1 = (R4.z & 255) - 64, o2 = ((R4.z >> 8) & 255) - 64;
        up = up && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
        dn = dn && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
      }
      const bool warp_on = r == 0 || __any_sync(0xffffffffu, up || dn);
      if (ok && !mbar_wait_bounded(s_u32(&full[b]), (uint32_t)((r / kStages) & 1))) {
        ok = false;
        atomicExch(err, 1);
      }
      if (ok && warp_on) {
        const float2* buf = dsm + (size_t)b * St::ELEMS;
        if (r == 0) df_run_smem<P0, NV, R, P0>(buf, j, R4.w, 0, up, dn, s, c);
        else df_run_smem<P0, NV, R, M0>(buf, j, R4.w, df_run_m(R4), up, dn, s, c);
        df_renorm<NV>(s, c, up || dn);
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(&empty[b])) : "memory");
    }
  }
  bool on[NV];
  double out[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = v0 + v;
    on[v] = row && vv < nvec && (!active || active[vv]);
    out[v] = 0.0;
    if (on[v]) {
      out[v] = ((double)s[v] + (double)c[v]) * ldexp(1.0, Ex[vv] + EA);
      y[vv * vs + i] = out[v];
    }
  }
  if (pq) {  // fixed-order block sums of x_i y_i over the consumer warps
    __shared__ double sred[NW];
    const int w = j >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vv = v0 + v;
      if (vv >= nvec) break;
      double t = on[v] ? x[vv * vs + i] * out[v] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0 && w < NW) sred[w] = t;
      __syncthreads();
      if (j == 0) {
        double sum = 0.0;
        for (int q = 0; q < NW; ++q) sum += sred[q];
        pq[(long long)vv * gridDim.x + blockIdx.x] = sum;
      }
      __syncthreads();
    }
  }
}

template <int P0, int NV, int R>
cudaError_t band_df_tma_go(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, const float2* A,
                           long long Np, int EA, const int* active, int nvec, const float2* xs, const int* Ex,
                           const double* x, double* y, long long vs, double* pq, int* err, int* nblocks) {
  using St = DfStage<P0, NV, R>;
  const size_t smem = St::BYTES * df_stages(R);
  static unsigned long long attr = 0;  // devices on which the attribute is set (one bit each)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(attr >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_band_df_tma<P0, NV, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr |= 1ULL << dev;
  }
  const dim3 grid((unsigned)((N + R - 1) / R), (unsigned)((nvec + NV - 1) / NV));
  k_band_df_tma<P0, NV, R><<<grid, R + 32, smem, s>>>(N, nruns, runs, n[0], n[1], n[2], A, Np, EA, active, nvec, xs,
                                                      Ex, x, y, vs, pq, err);
  *nblocks = (int)grid.x;
  return cudaGetLastError();
}

template <int P0>
cudaError_t band_df_tma_p(cudaStream_t s, int R, int nv, long long N, int nruns, const int4* runs, const int* n,
                          const float2* A, long long Np, int EA, const int* active, int nvec, const float2* xs,
                          const int* Ex, const double* x, double* y, long long vs, double* pq, int* err, int* nb) {
  if (R == 64) {
    if (nv == 1) return band_df_tma_go<P0, 1, 64>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
    return band_df_tma_go<P0, 2, 64>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
  }
  if (R == 128) {
    if (nv == 1) return band_df_tma_go<P0, 1, 128>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
    return band_df_tma_go<P0, 2, 128>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
  }
  if (nv == 1) return band_df_tma_go<P0, 1, 256>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
  return band_df_tma_go<P0, 2, 256>(s, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, nb);
}

// ---------------------------------------------------------------------------
// Tensor-map form of the staged kernel (128 rows per block): per run four 2-D TMA
// copies instead of 2 len + 2 NV bulk copies --
//   cu[t][j]  = A[h0 + t][i0 + j]                       box {R, M0} at (i0, h0)
//   cd[t][.]  = A[h0 + t][c0 + .], c0 = i0 - L0 - (M0 - 1) rounded down to even,
//               the bounding box {W, M0} of the lower terms' parallelogram
//   xu[v][.]  = x_{v0 + v}[i0 + L0 rounded down to even + .]   box {W, NV}
//   xd[v][.]  = x_{v0 + v}[c0 + .]                             box {W, NV}
// (indices in the padded row layout). Coordinates outside the tensor read zeros;
// such entries only meet rows whose neighbour line is outside the grid, which are
// predicated off. Row j's lower term of slot h0 + t sits at column
// (L0 & 1) + j + (M0 - 1 - t) of cd and xd, its upper x at (L0 & 1) + j + t of xu.
constexpr int kTmRows = 128;

template <int P0, int NV>
struct DfTmStage {
  static constexpr int R = kTmRows;
  static constexpr int M0 = 2 * P0 + 1;
  static constexpr int W = R + M0 + 1;  // even
  static constexpr int al(int v) { return (v + 15) / 16 * 16; }  // 128-byte sub-buffer starts
  static constexpr int CU = 0;
  static constexpr int CD = al(CU + M0 * R);
  static constexpr int XU = al(CD + M0 * W);
  static constexpr int XD = al(XU + NV * W);
  static constexpr int ELEMS = al(XD + NV * W);
  static constexpr uint32_t TX = (uint32_t)((M0 * R + M0 * W + 2 * NV * W) * 8);
};

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar) : "memory");
}

constexpr int kMaxTmRuns = 128;  // runs staged in shared memory by the tensor-map kernels
constexpr int kTmStages = 1;     // ring buffers of the one-row tensor-map kernel (measured: 1 beats 2)
constexpr int kTm2Stages = 1;    // ring buffers of the two-row tensor-map kernel (measured: 1 beats 2)

// The terms of run (LEN slots) for row j, both sides (the common case), every vector
// (ALL) or the vectors with act[v] (uniform tests over the block). MT >= 0: the run's
// tiny-end count at compile time (the tiny terms' code is then all that is emitted for
// them); MT < 0: the runtime count m.
template <int P0, int NV, int LEN, bool ALL, int MT>
__device__ __forceinline__ void df_run_tm(const float2* buf, int j, int o, int m, const bool (&act)[NV],
                                          float (&s)[NV], float (&c)[NV]) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0, W = St::W;
  const int mm = MT >= 0 ? MT : m;
  const float2* xu = buf + St::XU + o + j;
#pragma unroll
  for (int t = 0; t < LEN; ++t) {
    const float2 a = buf[St::CU + t * R + j];
    const bool tn = df_is_tiny(t, LEN, mm);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (ALL || act[v]) df_term_m(s[v], c[v], a, xu[v * W + t], tn);
  }
  const float2* cd = buf + St::CD + o + j + (M0 - 1);
  const float2* xd = buf + St::XD + o + j + (M0 - 1);
#pragma unroll
  for (int t = 0; t < LEN; ++t) {
    const float2 a = cd[t * W - t];
    const bool tn = df_is_tiny(t, LEN, mm);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (ALL || act[v]) df_term_m(s[v], c[v], a, xd[v * W - t], tn);
  }
}

// a full run (2 P0 + 1 slots) of the common case with every vector: the tiny-end count
// chosen at compile time (m >= P0 + 1: every slot tiny)
template <int P0, int NV>
__device__ __forceinline__ void df_run_tm_full(const float2* buf, int j, int o, int m, const bool (&act)[NV],
                                               float (&s)[NV], float (&c)[NV]) {
  constexpr int M0 = 2 * P0 + 1;
  constexpr int MA = P0 + 1;
  if (m <= 0) df_run_tm<P0, NV, M0, true, 0>(buf, j, o, 0, act, s, c);
  else if (m == 1) df_run_tm<P0, NV, M0, true, 1>(buf, j, o, 1, act, s, c);
  else if (m == 2) df_run_tm<P0, NV, M0, true, 2>(buf, j, o, 2, act, s, c);
  else if (m == 3) df_run_tm<P0, NV, M0, true, (3 < MA ? 3 : MA)>(buf, j, o, 3, act, s, c);
  else if (m == 4) df_run_tm<P0, NV, M0, true, (4 < MA ? 4 : MA)>(buf, j, o, 4, act, s, c);
  else df_run_tm<P0, NV, M0, true, MA>(buf, j, o, m, act, s, c);
}

// the same for any sides and vectors (rows next to the grid's faces, converged systems):
// the same operations per row and vector in the same order, compact code
template <int P0, int NV>
__device__ __forceinline__ void df_run_tm_any(const float2* buf, int j, int o, int len, int m, bool up, bool dn,
                                              const bool (&act)[NV], float (&s)[NV], float (&c)[NV]) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0, W = St::W;
  if (up) {
    const float2* xu = buf + St::XU + o + j;
#pragma unroll 1
    for (int t = 0; t < len; ++t) {
      const float2 a = buf[St::CU + t * R + j];
      const bool tn = df_is_tiny(t, len, m);
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (act[v]) df_term_m(s[v], c[v], a, xu[v * W + t], tn);
    }
  }
  if (dn) {
    const float2* cd = buf + St::CD + o + j + (M0 - 1);
    const float2* xd = buf + St::XD + o + j + (M0 - 1);
#pragma unroll 1
    for (int t = 0; t < len; ++t) {
      const float2 a = cd[t * W - t];
      const bool tn = df_is_tiny(t, len, m);
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (act[v]) df_term_m(s[v], c[v], a, xd[v * W - t], tn);
    }
  }
}

template <int P0, int NV>
__global__ void __launch_bounds__(kTmRows + 32) k_band_df_tm(long long N, int nruns, const int4* __restrict__ runs,
                                                             int n0, int n1, int n2, const float2* __restrict__ A,
                                                             const __grid_constant__ CUtensorMap tmUp,
                                                             const __grid_constant__ CUtensorMap tmDn,
                                                             const __grid_constant__ CUtensorMap tmX, long long Np,
                                                             int EA, const int* __restrict__ active, int nvec,
                                                             const float2* __restrict__ xs, const int* __restrict__ Ex,
                                                             const double* __restrict__ x, double* __restrict__ y,
                                                             long long vs, double* __restrict__ pq,
                                                             int* __restrict__ err, DfStrips g) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0;
  constexpr int NW = R / 32;
  constexpr int S = kTmStages;  // buffers in the ring
  extern __shared__ __align__(128) float2 dsm[];
  __shared__ __align__(8) unsigned long long full[S], empty[S];
  __shared__ int4 sruns[kMaxTmRuns];
  const int j = threadIdx.x;
  const int lane = j & 31;
  const int v0 = blockIdx.y * NV;
  long long i0, lo, hi;
  df_block_rows(g, R, blockIdx.x, &i0, &lo, &hi);
  if (lo >= hi) {  // no rows: only the partials, uniformly over the block
    if (pq && j < NV && v0 + j < nvec) pq[(long long)(v0 + j) * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  for (int r = j; r < nruns; r += blockDim.x) sruns[r] = runs[r];
  if (j == 0) {
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(&empty[b])), "r"(NW));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long i = i0 + j;
  const bool row = j < R && i >= lo && i < hi;
  float s[NV], c[NV];
  bool act[NV];  // the vectors whose products are stored: the others are not computed
  bool all = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    s[v] = 0.f;
    c[v] = 0.f;
    act[v] = v0 + v < nvec && (!active || active[v0 + v]);
    all = all && act[v];
  }
  if (j >= R) {  // producer warp
    if (lane == 0) {
      bool ok = true;
      int last = -1;
      const int xi = (int)(kDfPad + i0);
      for (int r = 0; r < nruns; ++r) {
        const int b = r % S, k = r / S;
        if (k > 0 && !mbar_wait_bounded(s_u32(&empty[b]), (uint32_t)((k - 1) & 1))) {
          ok = false;
          break;
        }
        const int4 R4 = sruns[r];
        const int c0 = (xi - R4.w - (M0 - 1)) & ~1;
        const uint32_t mb = s_u32(&full[b]);
        const uint32_t base = s_u32(dsm + (size_t)b * St::ELEMS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(St::TX) : "memory");
        tma_2d(base + St::CU * 8, &tmUp, xi, R4.x, mb);
        tma_2d(base + St::CD * 8, &tmDn, c0, R4.x, mb);
        tma_2d(base + St::XU * 8, &tmX, (xi + R4.w) & ~1, v0, mb);
        tma_2d(base + St::XD * 8, &tmX, c0, v0, mb);
        last = r;
      }
      if (!ok) atomicExch(err, 1);
      for (int q = last - S + 1; q <= last; ++q)  // let every copy in flight land
        if (q >= 0) mbar_wait_bounded(s_u32(&full[q % S]), (uint32_t)((q / S) & 1));
    }
  } else {  // consumer warps
    if (row) {
      const float2 a0 = A[kDfPad + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) df_term(s[v], c[v], a0, xs[(long long)min(v0 + v, nvec - 1) * Np + kDfPad + i]);
    }
    int i1 = 0, i2 = 0;
    if (row) {
      const long long t = i / n0;
      i1 = (int)(t % n1);
      i2 = (int)(t / n1);
    }
    bool ok = true;
    for (int r = 0; r < nruns; ++r) {
      const int b = r % S;
      const int4 R4 = sruns[r];
      bool up = row, dn = row;
      if (r > 0) {
        const int o1 = (R4.z & 255) - 64, o2 = ((R4.z >> 8) & 255) - 64;
        up = up && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
        dn = dn && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
      }
      const bool warp_on = r == 0 || __any_sync(0xffffffffu, up || dn);
      if (ok && !mbar_wait_bounded(s_u32(&full[b]), (uint32_t)((r / S) & 1))) {
        ok = false;
        atomicExch(err, 1);
      }
      if (ok && warp_on) {
        const float2* buf = dsm + (size_t)b * St::ELEMS;
        const int o = R4.w & 1;
        const int m = r == 0 ? 0 : df_run_m(R4);
        if (up && dn && all) {
          if (r == 0) df_run_tm<P0, NV, P0, true, 0>(buf, j, o, 0, act, s, c);
          else df_run_tm_full<P0, NV>(buf, j, o, m, act, s, c);
        } else if (up && dn) {
          if (r == 0) df_run_tm<P0, NV, P0, false, 0>(buf, j, o, 0, act, s, c);
          else df_run_tm<P0, NV, M0, false, -1>(buf, j, o, m, act, s, c);
        } else {
          df_run_tm_any<P0, NV>(buf, j, o, r == 0 ? P0 : M0, m, up, dn, act, s, c);
        }
        df_renorm<NV>(s, c, up || dn);
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(&empty[b])) : "memory");
    }
  }
  bool on[NV];
  double out[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = v0 + v;
    on[v] = row && vv < nvec && (!active || active[vv]);
    out[v] = 0.0;
    if (on[v]) {
      out[v] = ((double)s[v] + (double)c[v]) * ldexp(1.0, Ex[vv] + EA);
      y[vv * vs + i] = out[v];
    }
  }
  if (pq) {
    __shared__ double sred[NW];
    const int w = j >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vv = v0 + v;
      if (vv >= nvec) break;
      double t = on[v] ? x[vv * vs + i] * out[v] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0 && w < NW) sred[w] = t;
      __syncthreads();
      if (j == 0) {
        double sum = 0.0;
        for (int q = 0; q < NW; ++q) sum += sred[q];
        pq[(long long)vv * gridDim.x + blockIdx.x] = sum;
      }
      __syncthreads();
    }
  }
}

// the tensor map over NV rows of the split vectors
template <int NV>
const CUtensorMap& df_xmap(const DfTmaps& tm) {
  return NV == 1 ? tm.x1 : NV == 2 ? tm.x2 : NV == 3 ? tm.x3 : tm.x4;
}

template <int P0, int NV>
cudaError_t band_df_tm_go(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, const float2* A,
                          const DfTmaps& tm, long long Np, int EA, const int* active, int nvec, const float2* xs,
                          const int* Ex, const double* x, double* y, long long vs, double* pq, int* err,
                          int* nblocks, const DfStrips& g) {
  using St = DfTmStage<P0, NV>;
  const size_t smem = (size_t)St::ELEMS * 8 * kTmStages;
  static unsigned long long attr = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(attr >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_band_df_tm<P0, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr |= 1ULL << dev;
  }
  const dim3 grid((unsigned)df_strip_blocks(g), (unsigned)((nvec + NV - 1) / NV));
  k_band_df_tm<P0, NV><<<grid, kTmRows + 32, smem, s>>>(N, nruns, runs, n[0], n[1], n[2], A, tm.up, tm.dn,
                                                        df_xmap<NV>(tm), Np, EA, active, nvec, xs, Ex, x, y, vs, pq,
                                                        err, g);
  *nblocks = (int)grid.x;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tensor-map form with two rows per consumer thread: the staging (four 2-D copies
// per run, 128 rows per block) is that of k_band_df_tm; thread t computes rows
// 2t and 2t + 1 of the window. The pair's coefficients sit side by side in shared
// memory (one 16-byte load: always for the upper terms, for every other lower term),
// and the two rows' x values overlap: row 2t + 1 needs at term t what row 2t needs at
// term t + 1 (upper) or t - 1 (lower), so each vector costs one 8-byte load per term
// pair. The arithmetic of every row, and its order, are those of the other forms.
// The terms of run (LEN slots) for rows 2t and 2t + 1, every vector, both sides (the
// common case): one coefficient load per term serves both rows (a 16-byte pair for the
// upper terms; for the lower terms on every other term), and the x loads slide
template <int P0, int NV, int LEN, bool ALL>
__device__ __forceinline__ void df_run_tm2(const float2* buf, int jj, int o, int m, const bool (&act)[NV],
                                           float (&s)[2][NV], float (&c)[2][NV]) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0, W = St::W;
  {
    const float2* cu = buf + St::CU + jj;
    const float2* xu = buf + St::XU + o + jj;
    float2 xa[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) xa[v] = xu[v * W];
#pragma unroll
    for (int t = 0; t < LEN; ++t) {
      const float4 a2 = *reinterpret_cast<const float4*>(cu + t * R);
      const bool tn = df_is_tiny(t, LEN, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (!ALL && !act[v]) continue;
        const float2 xb = xu[v * W + t + 1];
        df_term_m(s[0][v], c[0][v], make_float2(a2.x, a2.y), xa[v], tn);
        df_term_m(s[1][v], c[1][v], make_float2(a2.z, a2.w), xb, tn);
        xa[v] = xb;
      }
    }
  }
  {
    // row jj's lower term of slot t at column o + jj + (M0 - 1) - t, row jj + 1's next to it
    const int base = St::CD + o + jj + (M0 - 1);
    const float2* xd = buf + St::XD + o + jj + (M0 - 1);
    float2 xb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) xb[v] = xd[v * W + 1];
#pragma unroll
    for (int t = 0; t < LEN; ++t) {
      const int off = base + t * (W - 1);
      float2 a0, a1;
      if ((off & 1) == 0) {
        const float4 q = *reinterpret_cast<const float4*>(buf + off);
        a0 = make_float2(q.x, q.y);
        a1 = make_float2(q.z, q.w);
      } else {
        a0 = buf[off];
        a1 = buf[off + 1];
      }
      const bool tn = df_is_tiny(t, LEN, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (!ALL && !act[v]) continue;
        const float2 xa = xd[v * W - t];
        df_term_m(s[0][v], c[0][v], a0, xa, tn);
        df_term_m(s[1][v], c[1][v], a1, xb[v], tn);
        xb[v] = xa;
      }
    }
  }
}

// the same for any rows, sides and vectors (rows next to the grid's faces, converged
// systems): per row and vector the same operations in the same order, compact code
template <int P0, int NV>
__device__ __forceinline__ void df_run_tm2_any(const float2* buf, int jj, int o, int len, int m, bool up0, bool up1,
                                               bool dn0, bool dn1, const bool (&act)[NV], float (&s)[2][NV],
                                               float (&c)[2][NV]) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0, W = St::W;
  if (up0 || up1) {
    const float2* cu = buf + St::CU + jj;
    const float2* xu = buf + St::XU + o + jj;
#pragma unroll 1
    for (int t = 0; t < len; ++t) {
      const float2 a0 = cu[t * R], a1 = cu[t * R + 1];
      const bool tn = df_is_tiny(t, len, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (!act[v]) continue;
        if (up0) df_term_m(s[0][v], c[0][v], a0, xu[v * W + t], tn);
        if (up1) df_term_m(s[1][v], c[1][v], a1, xu[v * W + t + 1], tn);
      }
    }
  }
  if (dn0 || dn1) {
    const float2* cd = buf + St::CD + o + jj + (M0 - 1);
    const float2* xd = buf + St::XD + o + jj + (M0 - 1);
#pragma unroll 1
    for (int t = 0; t < len; ++t) {
      const float2 a0 = cd[t * (W - 1)], a1 = cd[t * (W - 1) + 1];
      const bool tn = df_is_tiny(t, len, m);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (!act[v]) continue;
        if (dn0) df_term_m(s[0][v], c[0][v], a0, xd[v * W - t], tn);
        if (dn1) df_term_m(s[1][v], c[1][v], a1, xd[v * W - t + 1], tn);
      }
    }
  }
}

template <int P0, int NV>
__global__ void __launch_bounds__(kTmRows / 2 + 32) k_band_df_tm2(
    long long N, int nruns, const int4* __restrict__ runs, int n0, int n1, int n2, const float2* __restrict__ A,
    const __grid_constant__ CUtensorMap tmUp, const __grid_constant__ CUtensorMap tmDn,
    const __grid_constant__ CUtensorMap tmX, long long Np, int EA, const int* __restrict__ active, int nvec,
    const float2* __restrict__ xs, const int* __restrict__ Ex, const double* __restrict__ x, double* __restrict__ y,
    long long vs, double* __restrict__ pq, int* __restrict__ err, DfStrips g) {
  using St = DfTmStage<P0, NV>;
  constexpr int R = St::R, M0 = St::M0;
  constexpr int NC = R / 2;    // consumer threads
  constexpr int NW = NC / 32;  // consumer warps
  constexpr int S = kTm2Stages;  // buffers in the ring
  extern __shared__ __align__(128) float2 dsm[];
  __shared__ __align__(8) unsigned long long full[S], empty[S];
  __shared__ int4 sruns[kMaxTmRuns];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int v0 = blockIdx.y * NV;
  long long i0, lo, hi;
  df_block_rows(g, R, blockIdx.x, &i0, &lo, &hi);
  if (lo >= hi) {  // no rows: only the partials, uniformly over the block
    if (pq && tid < NV && v0 + tid < nvec) pq[(long long)(v0 + tid) * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  for (int r = tid; r < nruns; r += blockDim.x) sruns[r] = runs[r];
  if (tid == 0) {
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(&empty[b])), "r"(NW));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int jj = 2 * tid;
  const long long i = i0 + jj;  // rows i and i + 1
  const bool row0 = tid < NC && i >= lo && i < hi;
  const bool row1 = tid < NC && i + 1 >= lo && i + 1 < hi;
  float s[2][NV], c[2][NV];
  bool act[NV];  // the vectors whose products are stored: the others are not computed
  bool all = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    s[0][v] = s[1][v] = 0.f;
    c[0][v] = c[1][v] = 0.f;
    act[v] = v0 + v < nvec && (!active || active[v0 + v]);
    all = all && act[v];
  }
  if (tid >= NC) {  // producer warp
    if (lane == 0) {
      bool ok = true;
      int last = -1;
      const int xi = (int)(kDfPad + i0);
      for (int r = 0; r < nruns; ++r) {
        const int b = r % S, k = r / S;
        if (k > 0 && !mbar_wait_bounded(s_u32(&empty[b]), (uint32_t)((k - 1) & 1))) {
          ok = false;
          break;
        }
        const int4 R4 = sruns[r];
        const int c0 = (xi - R4.w - (M0 - 1)) & ~1;
        const uint32_t mb = s_u32(&full[b]);
        const uint32_t base = s_u32(dsm + (size_t)b * St::ELEMS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(St::TX) : "memory");
        tma_2d(base + St::CU * 8, &tmUp, xi, R4.x, mb);
        tma_2d(base + St::CD * 8, &tmDn, c0, R4.x, mb);
        tma_2d(base + St::XU * 8, &tmX, (xi + R4.w) & ~1, v0, mb);
        tma_2d(base + St::XD * 8, &tmX, c0, v0, mb);
        last = r;
      }
      if (!ok) atomicExch(err, 1);
      for (int q = last - S + 1; q <= last; ++q)  // let every copy in flight land
        if (q >= 0) mbar_wait_bounded(s_u32(&full[q % S]), (uint32_t)((q / S) & 1));
    }
  } else {  // consumer warps
    if (row0 || row1) {  // the diagonal: the window start is even, so both rows' pairs are one 16-byte load
      const float4 a2 = *reinterpret_cast<const float4*>(A + kDfPad + i);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (!act[v]) continue;
        const float4 x2 = *reinterpret_cast<const float4*>(xs + (long long)(v0 + v) * Np + kDfPad + i);
        if (row0) df_term(s[0][v], c[0][v], make_float2(a2.x, a2.y), make_float2(x2.x, x2.y));
        if (row1) df_term(s[1][v], c[1][v], make_float2(a2.z, a2.w), make_float2(x2.z, x2.w));
      }
    }
    int i1a = 0, i2a = 0, i1b = 0, i2b = 0;
    if (row0) {
      const long long t = i / n0;
      i1a = (int)(t % n1);
      i2a = (int)(t / n1);
    }
    if (row1) {
      const long long t = (i + 1) / n0;
      i1b = (int)(t % n1);
      i2b = (int)(t / n1);
    }
    bool ok = true;
    for (int r = 0; r < nruns; ++r) {
      const int b = r % S;
      const int4 R4 = sruns[r];
      bool up0 = row0, dn0 = row0, up1 = row1, dn1 = row1;
      if (r > 0) {
        const int o1 = (R4.z & 255) - 64, o2 = ((R4.z >> 8) & 255) - 64;
        up0 = up0 && (unsigned)(i1a + o1) < (unsigned)n1 && (unsigned)(i2a + o2) < (unsigned)n2;
        dn0 = dn0 && (unsigned)(i1a - o1) < (unsigned)n1 && (unsigned)(i2a - o2) < (unsigned)n2;
        up1 = up1 && (unsigned)(i1b + o1) < (unsigned)n1 && (unsigned)(i2b + o2) < (unsigned)n2;
        dn1 = dn1 && (unsigned)(i1b - o1) < (unsigned)n1 && (unsigned)(i2b - o2) < (unsigned)n2;
      }
      const bool warp_on = __any_sync(0xffffffffu, up0 || dn0 || up1 || dn1);
      if (ok && !mbar_wait_bounded(s_u32(&full[b]), (uint32_t)((r / S) & 1))) {
        ok = false;
        atomicExch(err, 1);
      }
      if (ok && warp_on) {
        const float2* buf = dsm + (size_t)b * St::ELEMS;
        const int o = R4.w & 1;
        const int m = r == 0 ? 0 : df_run_m(R4);
        if (up0 && up1 && dn0 && dn1 && all) {
          if (r == 0) df_run_tm2<P0, NV, P0, true>(buf, jj, o, 0, act, s, c);
          else df_run_tm2<P0, NV, M0, true>(buf, jj, o, m, act, s, c);
        } else if (up0 && up1 && dn0 && dn1) {
          if (r == 0) df_run_tm2<P0, NV, P0, false>(buf, jj, o, 0, act, s, c);
          else df_run_tm2<P0, NV, M0, false>(buf, jj, o, m, act, s, c);
        } else {
          df_run_tm2_any<P0, NV>(buf, jj, o, r == 0 ? P0 : M0, m, up0, up1, dn0, dn1, act, s, c);
        }
        df_renorm<NV>(s[0], c[0], up0 || dn0);
        df_renorm<NV>(s[1], c[1], up1 || dn1);
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(&empty[b])) : "memory");
    }
  }
  bool on[2][NV];
  double out[2][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = v0 + v;
    const bool act = vv < nvec && (!active || active[vv]);
    const double sc = act ? ldexp(1.0, Ex[vv] + EA) : 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      on[k][v] = (k ? row1 : row0) && act;
      out[k][v] = 0.0;
      if (on[k][v]) {
        out[k][v] = ((double)s[k][v] + (double)c[k][v]) * sc;
        y[vv * vs + i + k] = out[k][v];
      }
    }
  }
  if (pq) {  // fixed-order block sums of x_i y_i: the thread's two rows, the warp by shuffles, the warps in order
    __shared__ double sred[NW];
    const int w = tid >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vv = v0 + v;
      if (vv >= nvec) break;
      double t = on[0][v] ? x[vv * vs + i] * out[0][v] : 0.0;
      if (on[1][v]) t += x[vv * vs + i + 1] * out[1][v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0 && w < NW) sred[w] = t;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int q = 0; q < NW; ++q) sum += sred[q];
        pq[(long long)vv * gridDim.x + blockIdx.x] = sum;
      }
      __syncthreads();
    }
  }
}

template <int P0, int NV>
cudaError_t band_df_tm2_go(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, const float2* A,
                           const DfTmaps& tm, long long Np, int EA, const int* active, int nvec, const float2* xs,
                           const int* Ex, const double* x, double* y, long long vs, double* pq, int* err,
                           int* nblocks, const DfStrips& g) {
  using St = DfTmStage<P0, NV>;
  const size_t smem = (size_t)St::ELEMS * 8 * kTm2Stages;
  static unsigned long long attr = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(attr >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_band_df_tm2<P0, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr |= 1ULL << dev;
  }
  const dim3 grid((unsigned)df_strip_blocks(g), (unsigned)((nvec + NV - 1) / NV));
  k_band_df_tm2<P0, NV><<<grid, kTmRows / 2 + 32, smem, s>>>(N, nruns, runs, n[0], n[1], n[2], A, tm.up, tm.dn,
                                                             df_xmap<NV>(tm), Np, EA, active, nvec, xs, Ex, x, y, vs,
                                                             pq, err, g);
  *nblocks = (int)grid.x;
  return cudaGetLastError();
}

template <int P0, int BS>
void band_df_nv(cudaStream_t s, int nv, dim3 grid, long long N, int nruns, const int4* runs, const int* n,
                const float2* A, long long Np, int EA, const int* active, int nvec, const float2* xs, const int* Ex,
                const double* x, double* y, long long vs, double* pq, const DfStrips& g) {
#define IGA_DF_GO(NVV)                                                                                          \
  k_band_df<P0, NVV, BS><<<grid, BS, 0, s>>>(N, nruns, runs, n[0], n[1], n[2], A, Np, EA, active, nvec, xs, Ex, \
                                              x, y, vs, pq, g)
  switch (nv) {
    case 1: IGA_DF_GO(1); break;
    case 2: IGA_DF_GO(2); break;
    case 3: IGA_DF_GO(3); break;
    default: IGA_DF_GO(4); break;
  }
#undef IGA_DF_GO
}

template <int BS>
int band_df_go(cudaStream_t s, int nv, int p0, int p2, int H, long long N, int nruns, const int4* runs, const int* n,
               const float2* A, long long Np, int EA, const int* active, int nvec, const float2* xs, const int* Ex,
               const double* x, double* y, long long vs, double* pq) {
  const DfStrips g = df_strips(n, p2, H, BS);
  const dim3 grid((unsigned)df_strip_blocks(g), (unsigned)((nvec + nv - 1) / nv));
  switch (p0) {
    case 2: band_df_nv<2, BS>(s, nv, grid, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, g); break;
    case 3: band_df_nv<3, BS>(s, nv, grid, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, g); break;
    case 4: band_df_nv<4, BS>(s, nv, grid, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, g); break;
    default: band_df_nv<0, BS>(s, nv, grid, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, g); break;
  }
  return (int)grid.x;
}

}  // namespace

DfStrips df_strips(const int* n, int p2, int H, int R) {
  DfStrips g{n[0], n[1], n[2], n[1], 1, 0, 0};
  if (n[2] > 1 && p2 > 0) {
    // lines of direction 1 whose last p2 planes of coefficients fit in ~48 MB
    const double budget = 48e6;
    long long wmax = (long long)(budget / (8.0 * H * p2 * n[0]));
    wmax = std::max(8LL, std::min<long long>(wmax, n[1]));
    const int S = (int)((n[1] + wmax - 1) / wmax);
    g.W1 = (n[1] + S - 1) / S;
    g.S = (n[1] + g.W1 - 1) / g.W1;
  }
  const long long wl = (long long)n[1] - (long long)(g.S - 1) * g.W1;
  g.nb0 = (int)(((long long)g.W1 * n[0] + 1 + R - 1) / R);  // + 1: the window starts at an even row
  g.nbl = (int)((wl * n[0] + 1 + R - 1) / R);
  return g;
}

long long df_strip_blocks(const DfStrips& g) {
  return (long long)(g.S - 1) * g.n2 * g.nb0 + (long long)g.n2 * g.nbl;
}

std::vector<int> band_df_runs(const int* n, const int* p, const unsigned char* tiny) {
  const int m0 = 2 * p[0] + 1, m1 = 2 * p[1] + 1, m2 = 2 * p[2] + 1;
  const int centre = m0 * m1 * m2 / 2;
  const int qc = centre / m0;  // (o1, o2) = (0, 0)
  std::vector<std::array<int, 4>> runs;
  for (int q = qc; q < m1 * m2; ++q) {
    const int o1 = q % m1 - p[1], o2 = q / m1 - p[2];
    const int first_o0 = q == qc ? 1 : -p[0];
    const int len = q == qc ? p[0] : m0;
    if (len == 0) continue;
    const int h0 = m0 * q + (first_o0 + p[0]) - centre;
    const long long L0 = first_o0 + (long long)n[0] * (o1 + (long long)n[1] * o2);
    int m = 0;  // tiny slots at each end of the run (the centre run keeps every slot exact)
    if (tiny && q != qc)
      while (m < (len + 1) / 2 && tiny[h0 + m] && tiny[h0 + len - 1 - m]) ++m;
    runs.push_back({h0, len, (o1 + 64) | ((o2 + 64) << 8) | (m << 16), (int)L0});
  }
  // the centre run first (the kernels take run 0 as the row's own lines), the others by
  // their tiny-end count, so that consecutive runs share one compiled form of the terms
  std::stable_sort(runs.begin() + (runs.empty() ? 0 : 1), runs.end(),
                   [](const std::array<int, 4>& a, const std::array<int, 4>& b) { return (a[2] >> 16) < (b[2] >> 16); });
  std::vector<int> out;
  for (const auto& r : runs) out.insert(out.end(), r.begin(), r.end());
  return out;
}

// per stored slot h, the largest |hi| over the rows of a split band (FP32 bits, which
// order as the magnitudes do): out[h] must be zero on entry
__global__ void k_df_slot_absmax(long long N, const float2* __restrict__ A, long long Np, unsigned* __restrict__ out) {
  const float2* row = A + (long long)blockIdx.y * Np + kDfPad;
  unsigned m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(row[i].x) & 0x7fffffffu);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, m);
}

cudaError_t launch_df_slot_absmax(cudaStream_t s, long long N, int H, const float2* A, long long Np, unsigned* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned) * H, s);
  if (e != cudaSuccess) return e;
  const unsigned gx = (unsigned)std::min<long long>((N + 255) / 256, 64);
  k_df_slot_absmax<<<dim3(gx, (unsigned)H), 256, 0, s>>>(N, A, Np, out);
  return cudaGetLastError();
}

cudaError_t launch_df_split_matrix(cudaStream_t s, long long N, int H, const double* A, float2* Adf, long long Np,
                                   unsigned long long* part, int* dE) {
  k_df_absmax<<<dim3(kDfBlocks, 1), 256, 0, s>>>((long long)H * N, nullptr, A, 0, part);
  k_df_split<<<dim3(1, 1), 256, 0, s>>>(0, kDfBlocks, nullptr, A, 0, part, nullptr, Adf, Np, dE);
  const unsigned gx = (unsigned)std::min<long long>((N + 255) / 256, 1024);
  k_df_split<<<dim3(gx, (unsigned)H), 256, 0, s>>>(N, 0, nullptr, A, N, nullptr, dE, Adf, Np, nullptr);
  return cudaGetLastError();
}

namespace {
// the cooperative split (z: with the direction update x = z + beta x first); returns
// cudaErrorNotSupported when the device has no cooperative launch
cudaError_t df_split_coop(cudaStream_t s, long long N, const int* active, int nvec, double* x, const double* z,
                          const BetaArgs& ba, long long vs, float2* xs, long long Np, int* Ex,
                          unsigned long long* part, unsigned int* bar, int* err, long long limit) {
  static int nsm[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && nsm[dev] == 0) {
    int v = 0, coop = 0;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    nsm[dev] = coop ? v : -1;
  }
  const int sm = dev < 64 ? nsm[dev] : -1;
  if (sm <= 0) return cudaErrorNotSupported;
  // two blocks per SM: co-resident with the kernels of other patches' graph branches
  const long long G = std::min<long long>(std::min<long long>(2LL * sm, kDfBlocks), std::max<long long>(1, (N + 255) / 256));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (limit < 0) limit = kBarLimit;
  return cudaLaunchKernelEx(&cfg, k_df_split_coop, N, nvec, active, x, z, ba, vs, part, xs, Np, Ex, bar, err,
                            limit);
}
}  // namespace

cudaError_t launch_df_split(cudaStream_t s, long long N, const int* active, int nvec, const double* x, long long vs,
                            float2* xs, long long Np, int* Ex, unsigned long long* part, unsigned int* bar, int* err,
                            long long bar_limit) {
  if (bar && err) {  // one cooperative launch, two blocks per SM
    const cudaError_t e = df_split_coop(s, N, active, nvec, const_cast<double*>(x), nullptr, BetaArgs{}, vs, xs,
                                        Np, Ex, part, bar, err, bar_limit);
    if (e != cudaErrorNotSupported) return e;
  }
  k_df_absmax<<<dim3(kDfBlocks, nvec), 256, 0, s>>>(N, active, x, vs, part);
  const unsigned gx = (unsigned)std::min<long long>((N + 255) / 256, 2 * kDfBlocks);
  k_df_split<<<dim3(gx, nvec), 256, 0, s>>>(N, kDfBlocks, active, x, vs, part, nullptr, xs, Np, Ex);
  return cudaGetLastError();
}

cudaError_t launch_df_update_split(cudaStream_t s, long long N, const int* active, int nvec, double* p,
                                   const double* z, const BetaArgs& ba, long long vs, float2* xs, long long Np,
                                   int* Ex, unsigned long long* part, unsigned int* bar, int* err,
                                   long long bar_limit) {
  return df_split_coop(s, N, active, nvec, p, z, ba, vs, xs, Np, Ex, part, bar, err, bar_limit);
}

cudaError_t launch_band_df(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, int p0, int p2,
                           int H, const float2* A, long long Np, int EA, const int* active, int nvec,
                           const float2* xs, const int* Ex, const double* x, double* y, long long vs, int threads,
                           int nv, double* pq, int* npq, int* err, const DfTmaps* tm) {
  if (nv <= 0) nv = nvec < 4 ? nvec : 4;
  if (nv < 1) nv = 1;
  if (nv > 4) nv = 4;
  int nb;
  if ((threads == 96 || threads == 128) && p0 >= 2 && p0 <= 4 && err && tm && tm->ok && nruns <= kMaxTmRuns) {
    const DfStrips g = df_strips(n, p2, H, kTmRows);
    cudaError_t e;
#define IGA_TM_ARGS s, N, nruns, runs, n, A, *tm, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, &nb, g
#define IGA_TM_NV(GO, P) \
  (nv == 1 ? GO<P, 1>(IGA_TM_ARGS) : nv == 2 ? GO<P, 2>(IGA_TM_ARGS) : nv == 3 ? GO<P, 3>(IGA_TM_ARGS) : GO<P, 4>(IGA_TM_ARGS))
    if (threads == 96) {
      if (p0 == 2) e = IGA_TM_NV(band_df_tm2_go, 2);
      else if (p0 == 3) e = IGA_TM_NV(band_df_tm2_go, 3);
      else e = IGA_TM_NV(band_df_tm2_go, 4);
    } else {
      if (p0 == 2) e = IGA_TM_NV(band_df_tm_go, 2);
      else if (p0 == 3) e = IGA_TM_NV(band_df_tm_go, 3);
      else e = IGA_TM_NV(band_df_tm_go, 4);
    }
#undef IGA_TM_NV
#undef IGA_TM_ARGS
    if (npq) *npq = nb;
    return e;
  }
  if ((threads == 64 || threads == 128 || threads == 256) && nv <= 2 && p0 >= 2 && p0 <= 4 && err) {
    cudaError_t e;
    if (p0 == 2) e = band_df_tma_p<2>(s, threads, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, &nb);
    else if (p0 == 3) e = band_df_tma_p<3>(s, threads, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, &nb);
    else e = band_df_tma_p<4>(s, threads, nv, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq, err, &nb);
    if (npq) *npq = nb;
    return e;
  }
  if (threads == 64) nb = band_df_go<64>(s, nv, p0, p2, H, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else if (threads == 128) nb = band_df_go<128>(s, nv, p0, p2, H, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else if (threads == 512) nb = band_df_go<512>(s, nv, p0, p2, H, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  else nb = band_df_go<256>(s, nv, p0, p2, H, N, nruns, runs, n, A, Np, EA, active, nvec, xs, Ex, x, y, vs, pq);
  if (npq) *npq = nb;
  return cudaGetLastError();
}

// The tensor maps of one split band (M or K) and of the split vectors, for the
// 128-row tensor-map kernel: 8-byte elements, rows of stride Np, no swizzle, zero
// fill outside. ok = false (and the bulk-copy kernels serve) if the driver does not
// provide the encoder or refuses a map.
bool df_encode_maps(const float2* A, int H, const float2* xs, int nvmax, long long Np, int p0, DfTmaps* tm) {
  tm->ok = false;
  if (p0 < 2 || p0 > 4) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int M0 = 2 * p0 + 1, W = kTmRows + M0 + 1;
  auto make = [&](CUtensorMap* m, const float2* base, int rows, int bx, int by) {
    const cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Np * 8};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!make(&tm->up, A, H, kTmRows, M0) || !make(&tm->dn, A, H, W, M0) || !make(&tm->x1, xs, nvmax, W, 1) ||
      !make(&tm->x2, xs, nvmax, W, 2) || !make(&tm->x3, xs, nvmax, W, 3) || !make(&tm->x4, xs, nvmax, W, 4))
    return false;
  tm->ok = true;
  return true;
}

}  // namespace iga
