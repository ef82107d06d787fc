// Assembled band form of the isogeometric mass and stiffness matrices.
//
// Storage: the symmetric band is kept as its centre and upper half. With
// S = prod_a (2 p_a + 1) offsets o = (o0, o1, o2), |o_a| <= p_a, in co-lexicographic
// slot order, slot S-1-s holds -o(s); the stored slots are h = 0 (the diagonal,
// slot S/2) and h = 1..H-1 (slots S/2 + h). A[h][i] = A_{i, i+o} (zero where i+o
// leaves the interior), structure of arrays [H][N] so that a warp of consecutive
// rows reads consecutive words.
//
// Product: y_i = A[0][i] x_i + sum_h ( A[h][i] x_{i+L_h} + A[h][i-L_h] x_{i-L_h} ),
// L_h the linear offset of o(h). The second term is the lower half by symmetry.
// Where i +- L_h wraps around an edge of the grid the stored coefficient is zero,
// so only the array bounds are checked.
//
// Assembly by probing: for a colour c in prod_a [0, 2 p_a + 1), the probe vector
// is 1 at the dofs with i_a = c_a (mod 2 p_a + 1) for all a, else 0. Row i of
// A x_c is then the single coefficient A_{i,j} whose column j = i + o has that
// colour (o_a = c_a - i_a mod 2 p_a + 1 folded into [-p_a, p_a]). Every band
// entry is recovered exactly from the operator's own Gauss quadrature.
#include "iga_internal.h"

namespace iga {

// o12 (nullable) packs each stored slot's offsets along directions 1 and 2,
// (o1 + 64) | (o2 + 64) << 8. With it, a slot whose neighbour (i + o for the upper
// term, i - o for the lower) lies outside the grid along direction 1 or 2 for every
// lane of the warp is skipped: its coefficients are zero. Lanes of a warp share
// (i1, i2) except where the warp wraps a grid line, so the vote is almost always
// unanimous; skipped lanes would only have added zeros.
// pq (nullable): per block and vector the partial sum of x_i y_i over the block's rows,
// at pq[v * gridDim.x + blockIdx.x] (0 for inactive vectors) -- the p.q of PCG.
template <int NV, int BS>
__global__ void __launch_bounds__(BS) k_band_spmv(long long N, int H, const long long* __restrict__ off,
                                                  const int* __restrict__ o12, int n0, int n1, int n2,
                                                  const double* __restrict__ A, const int* __restrict__ active,
                                                  int nvec, const double* __restrict__ x, double* __restrict__ y,
                                                  long long vs, double* __restrict__ pq) {
  const long long i = (long long)blockIdx.x * BS + threadIdx.x;
  const bool row = i < N;  // no early return: the slot votes need every lane
  // up to NV vectors per thread share every coefficient load
  const int v0 = blockIdx.y * NV;
  bool on[NV];
  double acc[NV], xi[NV];
  const double a0 = row ? A[i] : 0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int vv = v0 + v;
    on[v] = row && vv < nvec && (!active || active[vv]);
    xi[v] = on[v] ? x[vv * vs + i] : 0.0;
    acc[v] = a0 * xi[v];
  }
  int i1 = 0, i2 = 0;
  if (row && o12) {
    const long long t = i / n0;
    i1 = (int)(t % n1);
    i2 = (int)(t / n1);
  }
  for (int h = 1; h < H; ++h) {
    const long long L = off[h];
    const long long jp = i + L, jm = i - L;
    const double* Ah = A + (long long)h * N;
    bool up = row && jp >= 0 && jp < N;
    bool dn = row && jm >= 0 && jm < N;
    if (o12) {
      const int pk = o12[h];
      const int o1 = (pk & 255) - 64, o2 = ((pk >> 8) & 255) - 64;
      up = up && (unsigned)(i1 + o1) < (unsigned)n1 && (unsigned)(i2 + o2) < (unsigned)n2;
      dn = dn && (unsigned)(i1 - o1) < (unsigned)n1 && (unsigned)(i2 - o2) < (unsigned)n2;
      if (!__any_sync(0xffffffffu, up || dn)) continue;
    }
    if (up) {
      const double a = Ah[i];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (on[v]) acc[v] = fma(a, x[(v0 + v) * vs + jp], acc[v]);
    }
    if (dn) {
      const double a = Ah[jm];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (on[v]) acc[v] = fma(a, x[(v0 + v) * vs + jm], acc[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
    if (on[v]) y[(v0 + v) * vs + i] = acc[v];
  if (pq) {  // fixed-order block sums: warps by shuffles, then the warps in order
    __shared__ double sred[BS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vv = v0 + v;
      if (vv >= nvec) break;
      double t = on[v] ? xi[v] * acc[v] : 0.0;
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

struct BandGeom {
  int n[3];
  int p[3];
  int m[3];     // 2p+1 per direction
  int centre;   // S / 2
};

__device__ __forceinline__ void idx3(long long i, const BandGeom& g, int* ia) {
  ia[0] = (int)(i % g.n[0]);
  ia[1] = (int)((i / g.n[0]) % g.n[1]);
  ia[2] = (int)(i / ((long long)g.n[0] * g.n[1]));
}

// probe vectors for colours first..first+nvec-1 (colour index co-lex over m[0], m[1], m[2])
__global__ void k_probe_gen(long long N, BandGeom g, int first, int ncol, double* __restrict__ x, long long vs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (i >= N) return;
  int ia[3];
  idx3(i, g, ia);
  const int c = first + v;
  const int c0 = c % g.m[0], c1 = (c / g.m[0]) % g.m[1], c2 = c / (g.m[0] * g.m[1]);
  const bool hit = c < ncol && ia[0] % g.m[0] == c0 && ia[1] % g.m[1] == c1 && ia[2] % g.m[2] == c2;
  x[v * vs + i] = hit ? 1.0 : 0.0;
}

__global__ void k_probe_extract(long long N, BandGeom g, int first, int ncol, const double* __restrict__ y,
                                long long vs, double* __restrict__ A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  const int c = first + v;
  if (i >= N || c >= ncol) return;
  int ia[3];
  idx3(i, g, ia);
  const int cc[3] = {c % g.m[0], (c / g.m[0]) % g.m[1], c / (g.m[0] * g.m[1])};
  int o[3];
  for (int a = 0; a < 3; ++a) {
    int r = (cc[a] - ia[a] % g.m[a] + g.m[a]) % g.m[a];  // o_a mod (2p+1)
    if (r > g.p[a]) r -= g.m[a];
    o[a] = r;
    const int j = ia[a] + r;
    if (j < 0 || j >= g.n[a]) return;  // neighbour outside the interior: coefficient stays 0
  }
  const int slot = (o[0] + g.p[0]) + g.m[0] * ((o[1] + g.p[1]) + g.m[1] * (o[2] + g.p[2]));
  if (slot < g.centre) return;  // lower half: taken from the symmetric partner
  A[(long long)(slot - g.centre) * N + i] = y[v * vs + i];
}

static BandGeom make_geom(const int* n, const int* p) {
  BandGeom g;
  int S = 1;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = n[a];
    g.p[a] = p[a];
    g.m[a] = 2 * p[a] + 1;
    S *= g.m[a];
  }
  g.centre = S / 2;
  return g;
}

namespace {
template <int BS>
int band_go(cudaStream_t s, int nv, long long N, int H, const long long* off, const int* o12, const int* n,
            const double* A, const int* active, int nvec, const double* x, double* y, long long vs, double* pq) {
  const dim3 grid((unsigned)((N + BS - 1) / BS), (unsigned)((nvec + nv - 1) / nv));
  const int n0 = n[0], n1 = n[1], n2 = n[2];
  switch (nv) {
    case 1: k_band_spmv<1, BS><<<grid, BS, 0, s>>>(N, H, off, o12, n0, n1, n2, A, active, nvec, x, y, vs, pq); break;
    case 2: k_band_spmv<2, BS><<<grid, BS, 0, s>>>(N, H, off, o12, n0, n1, n2, A, active, nvec, x, y, vs, pq); break;
    case 3: k_band_spmv<3, BS><<<grid, BS, 0, s>>>(N, H, off, o12, n0, n1, n2, A, active, nvec, x, y, vs, pq); break;
    default: k_band_spmv<4, BS><<<grid, BS, 0, s>>>(N, H, off, o12, n0, n1, n2, A, active, nvec, x, y, vs, pq); break;
  }
  return (int)grid.x;
}
}  // namespace

// threads: block size (64, 128, 256 or 512; anything else = 256); nv: vectors per
// thread sharing each coefficient load (1..4; 0 = min(nvec, 4)). Every
// configuration computes each row with the same operations in the same order.
cudaError_t launch_band_spmv(cudaStream_t s, long long N, int H, const long long* off, const int* o12, const int* n,
                             const double* A, const int* active, int nvec, const double* x, double* y, long long vs,
                             int threads, int nv, double* pq, int* npq) {
  if (nv <= 0) nv = nvec < 4 ? nvec : 4;
  if (nv < 1) nv = 1;
  if (nv > 4) nv = 4;
  int nb;
  if (threads == 64) nb = band_go<64>(s, nv, N, H, off, o12, n, A, active, nvec, x, y, vs, pq);
  else if (threads == 128) nb = band_go<128>(s, nv, N, H, off, o12, n, A, active, nvec, x, y, vs, pq);
  else if (threads == 512) nb = band_go<512>(s, nv, N, H, off, o12, n, A, active, nvec, x, y, vs, pq);
  else nb = band_go<256>(s, nv, N, H, off, o12, n, A, active, nvec, x, y, vs, pq);
  if (npq) *npq = nb;
  return cudaGetLastError();
}

cudaError_t launch_probe_gen(cudaStream_t s, long long N, const int* n, const int* p, int first, int ncol, int nvec,
                             double* x, long long vs) {
  k_probe_gen<<<dim3((unsigned)((N + 255) / 256), nvec), 256, 0, s>>>(N, make_geom(n, p), first, ncol, x, vs);
  return cudaGetLastError();
}

cudaError_t launch_probe_extract(cudaStream_t s, long long N, const int* n, const int* p, int first, int ncol,
                                 int nvec, const double* y, long long vs, double* A) {
  k_probe_extract<<<dim3((unsigned)((N + 255) / 256), nvec), 256, 0, s>>>(N, make_geom(n, p), first, ncol, y, vs, A);
  return cudaGetLastError();
}

}  // namespace iga
