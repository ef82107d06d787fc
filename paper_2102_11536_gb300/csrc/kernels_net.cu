// Learned initial guess of the mass solves: a two-layer 3-D convolutional network
// on the control-point grid (3 -> 16 -> 1 channels, 3x3x3 taps, zero padding,
// ReLU between), its gradients, the Adam update, and the features built from the
// method's own right-hand sides and solutions. The network only supplies the PCG
// starting point of the systems M Z_j = b_j of eq. ho1 (Sec. 4); PCG (Sec. 5.5)
// still iterates to the same residual, so the guess changes cost, not results.
//
// Precision: inputs, activations and parameters are BF16 values (parameters are
// kept in FP32 for Adam and rounded to BF16 when staged); every sum is FP32; the
// features, the extrapolation and the guess are FP64.
//
// Layout: a field is a flat co-lexicographic vector over the n1 x n2 x n3
// interior grid (i1 fastest); channel c of sample s starts at (s * C + c) * N.
// Tap t = e1 + 3 e2 + 9 e3 reads the neighbour at (e1-1, e2-1, e3-1).
// Parameters: W1 [16][3][27], b1 [16], W2 [16][27], b2 [1] (IGA_NET_NPARAM).
//
// Tiling: one block computes a 16 x 16 x 4 tile of outputs, one thread per
// (i1, i2) column and 4 points along i3 held in registers; the input tile with
// its one-point halo (18 x 18 x 6) is staged in shared memory. Every reduction
// over grid points (weight gradients, loss, norms) writes one partial per block
// and is summed in a fixed order, so results do not depend on scheduling.
#include "iga_internal.h"

namespace iga {
namespace {

constexpr int kCin = 3, kChid = 16, kTap = 27;
constexpr int kW1 = kChid * kCin * kTap;  // 1296
constexpr int kB1 = kW1;                  // offset of b1
constexpr int kW2 = kB1 + kChid;          // offset of W2 (1312)
constexpr int kB2 = kW2 + kChid * kTap;   // offset of b2 (1744)
constexpr int kNParam = kB2 + 1;          // 1745
static_assert(kNParam == IGA_NET_NPARAM, "parameter count");
constexpr int kPart1 = kW1 + kChid;       // W1 and b1 partials per block (1312)
constexpr int kPart2 = kChid * kTap + 1;  // W2 and b2 partials per block (433)

constexpr int TX = 16, TY = 16, TZ = 4;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HALO = HX * HY * HZ;  // 1944
constexpr int TILE = TX * TY * TZ;  // 1024
constexpr int NT = TX * TY;         // 256 threads
constexpr int kChunk2 = 8;          // channels staged at once by conv2 / bwd2
constexpr int kChunk1 = 4;          // hidden channels staged at once by bwd1
constexpr int kRed = kRedBlocks;     // fixed grid of the point reductions

struct G3 {
  int n1, n2, n3, t3;
  long long N;
};

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ bool inside(const G3& g, int x, int y, int z) {
  return x >= 0 && x < g.n1 && y >= 0 && y < g.n2 && z >= 0 && z < g.n3;
}

__device__ __forceinline__ long long lin(const G3& g, int x, int y, int z) {
  return x + (long long)g.n1 * (y + (long long)g.n2 * z);
}

// Tile origin and sample of this block.
__device__ __forceinline__ void origin(const G3& g, int& x0, int& y0, int& z0, int& smp) {
  smp = blockIdx.z / g.t3;
  x0 = blockIdx.x * TX;
  y0 = blockIdx.y * TY;
  z0 = (blockIdx.z - smp * g.t3) * TZ;
}

__device__ __forceinline__ void halo_coords(int h, int x0, int y0, int z0, int& gx, int& gy, int& gz) {
  gx = x0 + h % HX - 1;
  gy = y0 + (h / HX) % HY - 1;
  gz = z0 + h / (HX * HY) - 1;
}

// Stage channels [c0, c0 + nc) of a BF16 field (channel stride N) with the halo.
template <typename T>
__device__ void stage_bf16(const G3& g, const __nv_bfloat16* __restrict__ src, int c0, int nc, int x0, int y0,
                           int z0, T* dst) {
  for (int i = threadIdx.x; i < nc * HALO; i += NT) {
    const int c = i / HALO, h = i - c * HALO;
    int gx, gy, gz;
    halo_coords(h, x0, y0, z0, gx, gy, gz);
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (inside(g, gx, gy, gz)) v = src[(long long)(c0 + c) * g.N + lin(g, gx, gy, gz)];
    if constexpr (sizeof(T) == 4) dst[i] = __bfloat162float(v);
    else dst[i] = v;
  }
}

__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_net_conv1(G3 g, const __nv_bfloat16* __restrict__ x,
                                                  const float* __restrict__ theta, __nv_bfloat16* __restrict__ act) {
  __shared__ float xs[kCin * HALO];
  __shared__ __align__(16) float ws[kCin * kTap * kChid];  // [c][t][o]
  __shared__ float bs[kChid];
  int x0, y0, z0, smp;
  origin(g, x0, y0, z0, smp);
  const int tid = threadIdx.x;
  for (int i = tid; i < kCin * kTap * kChid; i += NT) {
    const int o = i % kChid, ct = i / kChid;
    ws[i] = bfr(theta[o * kCin * kTap + ct]);
  }
  if (tid < kChid) bs[tid] = bfr(theta[kB1 + tid]);
  stage_bf16(g, x + (long long)smp * kCin * g.N, 0, kCin, x0, y0, z0, xs);
  __syncthreads();
  const int tx = tid % TX, ty = tid / TX;
  float acc[TZ][kChid];
#pragma unroll
  for (int z = 0; z < TZ; ++z)
#pragma unroll
    for (int o = 0; o < kChid; ++o) acc[z][o] = bs[o];
  for (int c = 0; c < kCin; ++c)
#pragma unroll 1
    for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
      for (int e1 = 0; e1 < 3; ++e1) {
        float col[HZ];
#pragma unroll
        for (int hz = 0; hz < HZ; ++hz) col[hz] = xs[c * HALO + (tx + e1) + HX * ((ty + e2) + HY * hz)];
#pragma unroll
        for (int e3 = 0; e3 < 3; ++e3) {
          const float4* wp = reinterpret_cast<const float4*>(&ws[(c * kTap + e1 + 3 * e2 + 9 * e3) * kChid]);
#pragma unroll
          for (int q = 0; q < kChid / 4; ++q) {
            const float4 w = wp[q];
#pragma unroll
            for (int z = 0; z < TZ; ++z) {
              const float v = col[z + e3];
              acc[z][4 * q + 0] = fmaf(w.x, v, acc[z][4 * q + 0]);
              acc[z][4 * q + 1] = fmaf(w.y, v, acc[z][4 * q + 1]);
              acc[z][4 * q + 2] = fmaf(w.z, v, acc[z][4 * q + 2]);
              acc[z][4 * q + 3] = fmaf(w.w, v, acc[z][4 * q + 3]);
            }
          }
        }
      }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= g.n1 || gy >= g.n2) return;
  __nv_bfloat16* out = act + (long long)smp * kChid * g.N;
#pragma unroll
  for (int z = 0; z < TZ; ++z) {
    const int gz = z0 + z;
    if (gz >= g.n3) break;
    const long long p = lin(g, gx, gy, gz);
#pragma unroll
    for (int o = 0; o < kChid; ++o) out[(long long)o * g.N + p] = __float2bfloat16_rn(fmaxf(acc[z][o], 0.f));
  }
}

// y = W2 * act + b2; with Z != nullptr also Z = E + s0 y (the initial guess, FP64),
// s0 of sample s at s0[2 s].
__global__ void __launch_bounds__(NT) k_net_conv2(G3 g, const __nv_bfloat16* __restrict__ act,
                                                  const float* __restrict__ theta, float* __restrict__ y,
                                                  double* __restrict__ Z, const double* __restrict__ E,
                                                  const double* __restrict__ s0) {
  __shared__ __nv_bfloat16 as[kChunk2 * HALO];
  __shared__ float ws[kChid * kTap];
  int x0, y0, z0, smp;
  origin(g, x0, y0, z0, smp);
  const int tid = threadIdx.x;
  for (int i = tid; i < kChid * kTap; i += NT) ws[i] = bfr(theta[kW2 + i]);
  const int tx = tid % TX, ty = tid / TX;
  const float b2 = bfr(theta[kB2]);
  float acc[TZ];
#pragma unroll
  for (int z = 0; z < TZ; ++z) acc[z] = b2;
  const __nv_bfloat16* src = act + (long long)smp * kChid * g.N;
  for (int c0 = 0; c0 < kChid; c0 += kChunk2) {
    __syncthreads();
    stage_bf16(g, src, c0, kChunk2, x0, y0, z0, as);
    __syncthreads();
#pragma unroll 1
    for (int cc = 0; cc < kChunk2; ++cc)
#pragma unroll
      for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
        for (int e1 = 0; e1 < 3; ++e1) {
          float col[HZ];
#pragma unroll
          for (int hz = 0; hz < HZ; ++hz) col[hz] = ld(&as[cc * HALO + (tx + e1) + HX * ((ty + e2) + HY * hz)]);
#pragma unroll
          for (int e3 = 0; e3 < 3; ++e3) {
            const float w = ws[(c0 + cc) * kTap + e1 + 3 * e2 + 9 * e3];
#pragma unroll
            for (int z = 0; z < TZ; ++z) acc[z] = fmaf(w, col[z + e3], acc[z]);
          }
        }
  }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= g.n1 || gy >= g.n2) return;
#pragma unroll
  for (int z = 0; z < TZ; ++z) {
    const int gz = z0 + z;
    if (gz >= g.n3) break;
    const long long p = (long long)smp * g.N + lin(g, gx, gy, gz);
    if (y) y[p] = acc[z];
    if (Z) Z[p] = E[p] + s0[2 * smp] * (double)acc[z];
  }
}

// ---------------------------------------------------------------------------
// loss and backward
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

// dy = (y - t) / N; part[b] = sum over the block's points of (y - t)^2 (FP64).
__global__ void __launch_bounds__(256) k_net_loss(long long N, const float* __restrict__ y,
                                                  const float* __restrict__ t, float* __restrict__ dy,
                                                  double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  const float inv = 1.0f / (float)N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = d * inv;
    s += (double)d * (double)d;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_net_loss_fin(long long N, const double* __restrict__ part, double* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < kRed; ++b) s += part[b];
  *loss = s / (2.0 * (double)N);
}

// dh = (W2^T * dy) .* [act > 0] for the tile's points; per-block partials of the
// W2 gradient (sum_p dy[p] act[c][p + off]) and of the b2 gradient (sum_p dy[p]).
__global__ void __launch_bounds__(NT) k_net_bwd2(G3 g, const float* __restrict__ dy,
                                                 const __nv_bfloat16* __restrict__ act,
                                                 const float* __restrict__ theta, float* __restrict__ dh,
                                                 float* __restrict__ part) {
  __shared__ float dys[HALO];
  __shared__ __nv_bfloat16 as[kChunk2 * HALO];
  __shared__ float ws[kChid * kTap];
  int x0, y0, z0, smp;
  origin(g, x0, y0, z0, smp);
  const int tid = threadIdx.x;
  const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
  for (int i = tid; i < kChid * kTap; i += NT) ws[i] = bfr(theta[kW2 + i]);
  const float* dys_src = dy + (long long)smp * g.N;
  for (int h = tid; h < HALO; h += NT) {
    int gx, gy, gz;
    halo_coords(h, x0, y0, z0, gx, gy, gz);
    dys[h] = inside(g, gx, gy, gz) ? dys_src[lin(g, gx, gy, gz)] : 0.f;
  }
  const int tx = tid % TX, ty = tid / TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const __nv_bfloat16* asrc = act + (long long)smp * kChid * g.N;
  float* dhs = dh + (long long)smp * kChid * g.N;
  float* pp = part + blk * kPart2;
  for (int c0 = 0; c0 < kChid; c0 += kChunk2) {
    __syncthreads();
    stage_bf16(g, asrc, c0, kChunk2, x0, y0, z0, as);
    __syncthreads();
    // input gradient of the hidden layer, masked by the ReLU
    for (int cc = 0; cc < kChunk2; ++cc) {
      float da[TZ];
#pragma unroll
      for (int z = 0; z < TZ; ++z) da[z] = 0.f;
#pragma unroll
      for (int e2 = 0; e2 < 3; ++e2)
#pragma unroll
        for (int e1 = 0; e1 < 3; ++e1) {
          float col[HZ];
#pragma unroll
          for (int hz = 0; hz < HZ; ++hz) col[hz] = dys[(tx + 2 - e1) + HX * ((ty + 2 - e2) + HY * hz)];
#pragma unroll
          for (int e3 = 0; e3 < 3; ++e3) {
            const float w = ws[(c0 + cc) * kTap + e1 + 3 * e2 + 9 * e3];
#pragma unroll
            for (int z = 0; z < TZ; ++z) da[z] = fmaf(w, col[z + 2 - e3], da[z]);
          }
        }
      if (gx < g.n1 && gy < g.n2) {
#pragma unroll
        for (int z = 0; z < TZ; ++z) {
          const int gz = z0 + z;
          if (gz >= g.n3) break;
          const float a = __bfloat162float(as[cc * HALO + (tx + 1) + HX * ((ty + 1) + HY * (z + 1))]);
          dhs[(long long)(c0 + cc) * g.N + lin(g, gx, gy, gz)] = a > 0.f ? da[z] : 0.f;
        }
      }
    }
    // W2 partials of this chunk: one (channel, tap) per thread
    if (tid < kChunk2 * kTap) {
      const int cc = tid / kTap, t = tid - cc * kTap;
      const int e1 = t % 3, e2 = (t / 3) % 3, e3 = t / 9;
      float s = 0.f;
      for (int z = 0; z < TZ; ++z)
        for (int yy = 0; yy < TY; ++yy)
          for (int xx = 0; xx < TX; ++xx)
            s = fmaf(dys[(xx + 1) + HX * ((yy + 1) + HY * (z + 1))],
                     __bfloat162float(as[cc * HALO + (xx + e1) + HX * ((yy + e2) + HY * (z + e3))]), s);
      pp[(c0 + cc) * kTap + t] = s;
    }
  }
  if (tid == NT - 1) {
    float s = 0.f;
    for (int z = 0; z < TZ; ++z)
      for (int yy = 0; yy < TY; ++yy)
        for (int xx = 0; xx < TX; ++xx) s += dys[(xx + 1) + HX * ((yy + 1) + HY * (z + 1))];
    pp[kChid * kTap] = s;
  }
}

// Per-block partials of the W1 gradient (sum_p dh[o][p] x[c][p + off]) and of the
// b1 gradient (sum_p dh[o][p]).
__global__ void __launch_bounds__(NT) k_net_bwd1(G3 g, const float* __restrict__ dh,
                                                 const __nv_bfloat16* __restrict__ x, float* __restrict__ part) {
  __shared__ float xs[kCin * HALO];
  __shared__ float hs[kChunk1 * TILE];
  int x0, y0, z0, smp;
  origin(g, x0, y0, z0, smp);
  const int tid = threadIdx.x;
  const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
  stage_bf16(g, x + (long long)smp * kCin * g.N, 0, kCin, x0, y0, z0, xs);
  const float* hsrc = dh + (long long)smp * kChid * g.N;
  float* pp = part + blk * kPart1;
  constexpr int kItems = kChunk1 * kCin * kTap + kChunk1;  // 328
  for (int o0 = 0; o0 < kChid; o0 += kChunk1) {
    __syncthreads();
    for (int i = tid; i < kChunk1 * TILE; i += NT) {
      const int oo = i / TILE, r = i - oo * TILE;
      const int xx = r % TX, yy = (r / TX) % TY, z = r / (TX * TY);
      const int gx = x0 + xx, gy = y0 + yy, gz = z0 + z;
      hs[i] = inside(g, gx, gy, gz) ? hsrc[(long long)(o0 + oo) * g.N + lin(g, gx, gy, gz)] : 0.f;
    }
    __syncthreads();
    for (int it = tid; it < kItems; it += NT) {
      float s = 0.f;
      if (it < kChunk1 * kCin * kTap) {
        const int oo = it / (kCin * kTap), ct = it - oo * (kCin * kTap);
        const int c = ct / kTap, t = ct - c * kTap;
        const int e1 = t % 3, e2 = (t / 3) % 3, e3 = t / 9;
        const float* hrow = hs + oo * TILE;
        const float* xrow = xs + c * HALO;
        for (int z = 0; z < TZ; ++z)
          for (int yy = 0; yy < TY; ++yy)
            for (int xx = 0; xx < TX; ++xx)
              s = fmaf(hrow[xx + TX * (yy + TY * z)], xrow[(xx + e1) + HX * ((yy + e2) + HY * (z + e3))], s);
        pp[(o0 + oo) * kCin * kTap + ct] = s;
      } else {
        const int oo = it - kChunk1 * kCin * kTap;
        const float* hrow = hs + oo * TILE;
        for (int i = 0; i < TILE; ++i) s += hrow[i];
        pp[kW1 + o0 + oo] = s;
      }
    }
  }
}

// grad[i] = sum over blocks of the partials, in block order.
__global__ void k_net_reduce(long long nblk, const float* __restrict__ part1, const float* __restrict__ part2,
                             float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  double s = 0.0;
  if (i < kPart1) {
    for (long long b = 0; b < nblk; ++b) s += part1[b * kPart1 + i];
  } else {
    const int j = i - kPart1;
    for (long long b = 0; b < nblk; ++b) s += part2[b * kPart2 + j];
  }
  grad[i] = (float)s;
}

__global__ void k_net_adam(int n, float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = grad[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// part[(2 j + 0) * kRed + b] = sum (D^{-1}(b - 2 b1 + b2))^2, part[(2 j + 1) * kRed + b] = sum z1^2
__global__ void __launch_bounds__(256) k_ws_norm(long long N, const double* __restrict__ b,
                                                 const double* __restrict__ b1, const double* __restrict__ b2,
                                                 const double* __restrict__ D, const double* __restrict__ z1,
                                                 double* __restrict__ part) {
  __shared__ double sh[8];
  const int j = blockIdx.y;
  const long long o = (long long)j * N;
  double s0 = 0.0, s1 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double c0 = (b[o + i] - 2.0 * b1[o + i] + b2[o + i]) / D[i];
    const double z = z1[o + i];
    s0 += c0 * c0;
    s1 += z * z;
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[(2 * j + 0) * kRed + blockIdx.x] = s0;
    part[(2 * j + 1) * kRed + blockIdx.x] = s1;
  }
}

// sc[2 j] = s0, sc[2 j + 1] = s1 (root mean squares, 1 where zero)
__global__ void k_ws_scale(int k, long long N, const double* __restrict__ part, double* __restrict__ sc) {
  const int q = threadIdx.x;
  if (q >= 2 * k) return;
  double s = 0.0;
  for (int b = 0; b < kRed; ++b) s += part[q * kRed + b];
  const double r = sqrt(s / (double)N);
  sc[q] = r > 0.0 ? r : 1.0;
}

// x = BF16 features; E = 2 z1 - z2; then the histories move one step:
// b2 <- b1, b1 <- b, z2 <- z1, z1 <- E (the guess before the network's term).
__global__ void __launch_bounds__(256) k_ws_pack(long long N, const double* __restrict__ b, double* __restrict__ b1,
                                                 double* __restrict__ b2, const double* __restrict__ D,
                                                 double* __restrict__ z1, double* __restrict__ z2,
                                                 const double* __restrict__ sc, __nv_bfloat16* __restrict__ x,
                                                 double* __restrict__ E) {
  const int j = blockIdx.y;
  const long long o = (long long)j * N;
  const double s0 = sc[2 * j], s1 = sc[2 * j + 1];
  __nv_bfloat16* xj = x + (long long)j * kCin * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double bb = b[o + i], bb1 = b1[o + i], bb2 = b2[o + i];
    const double zz1 = z1[o + i], zz2 = z2[o + i];
    const double c0 = (bb - 2.0 * bb1 + bb2) / D[i];
    xj[i] = __float2bfloat16_rn((float)(c0 / s0));
    xj[N + i] = __float2bfloat16_rn((float)(zz1 / s1));
    xj[2 * N + i] = __float2bfloat16_rn((float)(zz2 / s1));
    const double e = 2.0 * zz1 - zz2;
    E[o + i] = e;
    b2[o + i] = bb1;
    b1[o + i] = bb;
    z2[o + i] = zz1;
    z1[o + i] = e;
  }
}

__global__ void __launch_bounds__(256) k_ws_target(long long N, const double* __restrict__ Z,
                                                   const double* __restrict__ E, const double* __restrict__ sc,
                                                   float* __restrict__ t) {
  const int j = blockIdx.y;
  const long long o = (long long)j * N;
  const double s0 = sc[2 * j];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    t[o + i] = (float)((Z[o + i] - E[o + i]) / s0);
}

G3 make_g3(const NetGrid& g, int nb) {
  G3 r;
  r.n1 = g.n1;
  r.n2 = g.n2;
  r.n3 = g.n3;
  r.N = (long long)g.n1 * g.n2 * g.n3;
  r.t3 = (g.n3 + TZ - 1) / TZ;
  (void)nb;
  return r;
}

dim3 net_grid(const NetGrid& g, int nb) {
  return dim3((g.n1 + TX - 1) / TX, (g.n2 + TY - 1) / TY, ((g.n3 + TZ - 1) / TZ) * nb);
}

}  // namespace

long long net_blocks(const NetGrid& g, int nb) {
  const dim3 d = net_grid(g, nb);
  return (long long)d.x * d.y * d.z;
}

size_t net_workspace_bytes(const NetGrid& g, int nb) {
  const long long N = (long long)g.n1 * g.n2 * g.n3;
  const long long nblk = net_blocks(g, nb);
  return sizeof(float) * ((size_t)nb * kChid * N + (size_t)nblk * (kPart1 + kPart2));
}

bool net_grid_ok(const NetGrid& g, int nb) {
  if (g.n1 < 1 || g.n2 < 1 || g.n3 < 1 || nb < 1) return false;
  const dim3 d = net_grid(g, nb);
  return d.y <= 65535u && d.z <= 65535u;
}

cudaError_t launch_net_forward(cudaStream_t s, const NetGrid& g, int nb, const __nv_bfloat16* x, const float* theta,
                               __nv_bfloat16* act, float* y, double* Z, const double* E, const double* s0,
                               long long* nl) {
  const G3 gg = make_g3(g, nb);
  const dim3 grid = net_grid(g, nb);
  k_net_conv1<<<grid, NT, 0, s>>>(gg, x, theta, act);
  k_net_conv2<<<grid, NT, 0, s>>>(gg, act, theta, y, Z, E, s0);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_net_loss(cudaStream_t s, long long N, const float* y, const float* t, float* dy, double* part,
                            double* loss, long long* nl) {
  k_net_loss<<<kRed, 256, 0, s>>>(N, y, t, dy, part);
  k_net_loss_fin<<<1, 32, 0, s>>>(N, part, loss);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_net_backward(cudaStream_t s, const NetGrid& g, int nb, const __nv_bfloat16* x, const float* theta,
                                const __nv_bfloat16* act, const float* dy, float* grad, void* work, long long* nl) {
  const G3 gg = make_g3(g, nb);
  const dim3 grid = net_grid(g, nb);
  const long long nblk = net_blocks(g, nb);
  float* dh = static_cast<float*>(work);
  float* part1 = dh + (size_t)nb * kChid * gg.N;
  float* part2 = part1 + (size_t)nblk * kPart1;
  k_net_bwd2<<<grid, NT, 0, s>>>(gg, dy, act, theta, dh, part2);
  k_net_bwd1<<<grid, NT, 0, s>>>(gg, dh, x, part1);
  k_net_reduce<<<(kNParam + 255) / 256, 256, 0, s>>>(nblk, part1, part2, grad);
  *nl += 3;
  return cudaGetLastError();
}

cudaError_t launch_net_adam(cudaStream_t s, int n, float* theta, const float* grad, float* m, float* v, long long step,
                            double lr, long long* nl) {
  const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)step));
  const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)step));
  k_net_adam<<<(n + 255) / 256, 256, 0, s>>>(n, theta, grad, m, v, (float)lr, (float)c1, (float)c2);
  *nl += 1;
  return cudaGetLastError();
}

cudaError_t launch_ws_features(cudaStream_t s, long long N, int k, const double* b, double* b1, double* b2,
                               const double* D, double* z1, double* z2, __nv_bfloat16* x, double* E, double* part,
                               double* sc, long long* nl) {
  k_ws_norm<<<dim3(kRed, k), 256, 0, s>>>(N, b, b1, b2, D, z1, part);
  k_ws_scale<<<1, 32, 0, s>>>(k, N, part, sc);
  k_ws_pack<<<dim3(kRed, k), 256, 0, s>>>(N, b, b1, b2, D, z1, z2, sc, x, E);
  *nl += 3;
  return cudaGetLastError();
}

cudaError_t launch_ws_target(cudaStream_t s, long long N, int k, const double* Z, const double* E, const double* sc,
                             float* t, long long* nl) {
  k_ws_target<<<dim3(kRed, k), 256, 0, s>>>(N, Z, E, sc, t);
  *nl += 1;
  return cudaGetLastError();
}

}  // namespace iga
