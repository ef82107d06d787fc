// Fields at the Gauss points: the physical points x = F(xi) (the geometry map of Sec. 5.1,
// over the full control net) and the pointwise weighting by w |det DF| that turns point
// values into integrals; with the operators' banded passes they give evaluation of a
// spline field and the load vectors int g B_i of the semi-discrete problem (Sec. 2).
#include "iga_internal.h"

namespace iga {
namespace {

struct PtDir {
  const double* val;  // [Q][P]
  const int* qfirst;  // [Q] full index of the point's first function
  int P, Q, m;
};

// x_c(q) = sum over the (p+1)^d functions nonzero at q of C_{i,c} B_i(xi_q)
template <int D>
__global__ void k_points(PtDir g0, PtDir g1, PtDir g2, const double* __restrict__ cx, const double* __restrict__ cy,
                         const double* __restrict__ cz, double* __restrict__ X, long long Qt) {
  const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= Qt) return;
  const int q0 = (int)(qi % g0.Q);
  const int q1 = (int)((qi / g0.Q) % g1.Q);
  const int q2 = D == 3 ? (int)(qi / ((long long)g0.Q * g1.Q)) : 0;
  const int f0 = g0.qfirst[q0], f1 = g1.qfirst[q1], f2 = D == 3 ? g2.qfirst[q2] : 0;
  const int P2 = D == 3 ? g2.P : 1;
  double x[3] = {0.0, 0.0, 0.0};
  for (int l2 = 0; l2 < P2; ++l2) {
    const double v2 = D == 3 ? g2.val[q2 * g2.P + l2] : 1.0;
    for (int l1 = 0; l1 < g1.P; ++l1) {
      const double v12 = g1.val[q1 * g1.P + l1] * v2;
      for (int l0 = 0; l0 < g0.P; ++l0) {
        const double b = g0.val[q0 * g0.P + l0] * v12;
        const long long ci = (f0 + l0) + (long long)g0.m * ((f1 + l1) + (long long)g1.m * (f2 + l2));
        x[0] = fma(cx[ci], b, x[0]);
        x[1] = fma(cy[ci], b, x[1]);
        if (D == 3) x[2] = fma(cz[ci], b, x[2]);
      }
    }
  }
  for (int c = 0; c < D; ++c) X[c * Qt + qi] = x[c];
}

// out[v][q] = W[q] g[v][q]
__global__ void k_weight_points(long long Qt, int nvec, const double* __restrict__ W, const double* __restrict__ g,
                                double* __restrict__ out) {
  const long long n = Qt * nvec;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = W[i % Qt] * g[i];
}

}  // namespace

cudaError_t launch_points(cudaStream_t s, int dim, const DirDev* dirs, const int* m, const double* ctrl_soa,
                          double* X) {
  PtDir g[3];
  long long Qt = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const int* qf = dirs[a].qfirst_geo ? dirs[a].qfirst_geo : dirs[a].qfirst;
      g[a] = PtDir{dirs[a].val, qf, dirs[a].P, dirs[a].Q, m[a]};
      Qt *= dirs[a].Q;
    } else {
      g[a] = PtDir{nullptr, nullptr, 1, 1, 1};
    }
  }
  const long long mt = (long long)m[0] * m[1] * (dim == 3 ? m[2] : 1);
  const unsigned blocks = (unsigned)((Qt + 255) / 256);
  if (dim == 3)
    k_points<3><<<blocks, 256, 0, s>>>(g[0], g[1], g[2], ctrl_soa, ctrl_soa + mt, ctrl_soa + 2 * mt, X, Qt);
  else
    k_points<2><<<blocks, 256, 0, s>>>(g[0], g[1], g[2], ctrl_soa, ctrl_soa + mt, nullptr, X, Qt);
  return cudaGetLastError();
}

cudaError_t launch_weight_points(cudaStream_t s, long long Qt, int nvec, const double* W, const double* g,
                                 double* out) {
  const long long n = Qt * nvec;
  const long long want = (n + 255) / 256;
  const unsigned blocks = (unsigned)std::min<long long>(want, 152LL * 32);
  k_weight_points<<<blocks, 256, 0, s>>>(Qt, nvec, W, g, out);
  return cudaGetLastError();
}

}  // namespace iga
