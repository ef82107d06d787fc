// Matrix-free isogeometric mass and stiffness operators by global sum
// factorisation at the Gauss points, the geometric factors at the Gauss
// points, and the FP64 fast-diagonalisation mode product.
//
// With B_a the (Q_a x n_a) table of the interior univariate B-splines of
// direction a at its Gauss points (p+1 nonzeros per row) and W the diagonal of
// w|det DF| over the Q_0 Q_1 Q_2 tensor points,
//     M x = (B_2 (x) B_1 (x) B_0)^T W (B_2 (x) B_1 (x) B_0) x          (Sec. 5.3, eq. mass_matrix)
//     K x = sum_{a,b} (D_a)^T G_ab (D_b) x,  D_b = tensor table with B'_b in slot b
// (Galerkin stiffness of eq. pde with omega = 1). Each factor is applied as a
// separate pass along one axis of the data, so every pass is a short banded
// contraction with p+1 (forward) or at most (p+1) * nq (transposed) terms:
// the minimum FP64 work of a matrix-free application at these points. All
// passes are gathers -- every output is written once by one thread -- so the
// results are deterministic (no atomics). The last axis is handled by one
// kernel per column that interpolates, applies the point factor and
// integrates back with sliding register windows.
#include "iga_internal.h"

namespace iga {

// ----------------------------------------------------------------------------
// forward pass: coefficients -> points along one axis
// ----------------------------------------------------------------------------
template <int P, bool TWO, bool A1>
__global__ void __launch_bounds__(256) k_fwd(const int* __restrict__ qfirst, const double* __restrict__ T0,
                                             const double* __restrict__ T1, int A, int Lin, int Lout,
                                             const int* __restrict__ active, const double* __restrict__ in,
                                             long long in_vs, double* __restrict__ out0, double* __restrict__ out1,
                                             long long out_vs) {
  const int v = blockIdx.z;
  if (active && !active[v]) return;
  const int y = blockIdx.y;
  const int flat = blockIdx.x * blockDim.x + threadIdx.x;
  if (flat >= A * Lout) return;
  int x, o;
  if (A1) {
    x = 0;
    o = flat;
  } else {
    o = flat / A;
    x = flat - o * A;
  }
  const double* src = in + v * in_vs + (long long)y * Lin * A + x;
  const int j0 = qfirst[o] - 1;
  double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    if (j >= 0 && j < Lin) {
      const double u = src[(long long)j * A];
      acc0 = fma(T0[o * P + l], u, acc0);
      if (TWO) acc1 = fma(T1[o * P + l], u, acc1);
    }
  }
  const long long oi = v * out_vs + ((long long)y * Lout + o) * A + x;
  out0[oi] = acc0;
  if (TWO) out1[oi] = acc1;
}

// ----------------------------------------------------------------------------
// transposed pass: points -> coefficients along one axis (gather form)
// ----------------------------------------------------------------------------
template <int P, bool TWO, bool A1>
__global__ void __launch_bounds__(256) k_tr(const int* __restrict__ qfirst, const int* __restrict__ flo,
                                            const int* __restrict__ fhi, const double* __restrict__ T0,
                                            const double* __restrict__ T1, int A, int Lin, int Lout,
                                            const int* __restrict__ active, const double* __restrict__ in0,
                                            const double* __restrict__ in1, long long in_vs,
                                            double* __restrict__ out, long long out_vs) {
  const int v = blockIdx.z;
  if (active && !active[v]) return;
  const int y = blockIdx.y;
  const int flat = blockIdx.x * blockDim.x + threadIdx.x;
  if (flat >= A * Lout) return;
  int x, i;
  if (A1) {
    x = 0;
    i = flat;
  } else {
    i = flat / A;
    x = flat - i * A;
  }
  const long long base = v * in_vs + (long long)y * Lin * A + x;
  const double* s0 = in0 + base;
  const double* s1 = TWO ? in1 + base : nullptr;
  const int f = i + 1, lo = flo[i], hi = fhi[i];
  double acc = 0.0;
  for (int q = lo; q < hi; ++q) {
    const int l = f - qfirst[q];
    acc = fma(T0[q * P + l], s0[(long long)q * A], acc);
    if (TWO) acc = fma(T1[q * P + l], s1[(long long)q * A], acc);
  }
  out[v * out_vs + ((long long)y * Lout + i) * A + x] = acc;
}

// ----------------------------------------------------------------------------
// last axis of the mass operator: per column, u_q = sum_l B[q][l] in[j0+l],
// s_q = W_q u_q, out[j0+l] += B[q][l] s_q, with the window j0 = qfirst[q]-1
// sliding along the column. Safe in place (a slot is written only after it
// left the window, and read only while inside it).
// ----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_mid_mass(const int* __restrict__ qfirst, const double* __restrict__ Tv,
                                                  int A, int n, int Q, const int* __restrict__ active,
                                                  const double* __restrict__ W, const double* in, double* out,
                                                  long long vs) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A) return;
  const double* src = in + v * vs + x;
  double* dst = out + v * vs + x;
  const double* w = W + x;
  int j0 = qfirst[0] - 1;
  double uin[P], acc[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    uin[l] = (j >= 0 && j < n) ? src[(long long)j * A] : 0.0;
    acc[l] = 0.0;
  }
  for (int q = 0; q < Q; ++q) {
    const int jq = qfirst[q] - 1;
    while (j0 < jq) {
      if (j0 >= 0 && j0 < n) dst[(long long)j0 * A] = acc[0];
#pragma unroll
      for (int l = 0; l < P - 1; ++l) {
        acc[l] = acc[l + 1];
        uin[l] = uin[l + 1];
      }
      const int jn = j0 + P;
      acc[P - 1] = 0.0;
      uin[P - 1] = (jn >= 0 && jn < n) ? src[(long long)jn * A] : 0.0;
      ++j0;
    }
    const double* b = Tv + q * P;
    double u = 0.0;
#pragma unroll
    for (int l = 0; l < P; ++l) u = fma(b[l], uin[l], u);
    const double s = w[(long long)q * A] * u;
#pragma unroll
    for (int l = 0; l < P; ++l) acc[l] = fma(b[l], s, acc[l]);
  }
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    if (j >= 0 && j < n) dst[(long long)j * A] = acc[l];
  }
}

// ----------------------------------------------------------------------------
// last axis of the 3-D stiffness operator. G holds 6 arrays (xx,yy,zz,xy,xz,yz)
// of the symmetric point factor W DF^{-1} DF^{-T}, point index x + A q.
// ----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_mid_stiff3(const int* __restrict__ qfirst, const double* __restrict__ Tv,
                                                    const double* __restrict__ Td, int A, int n, int Q,
                                                    const int* __restrict__ active, const double* __restrict__ G,
                                                    long long gs, double* a, double* b, double* c, long long vs) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A) return;
  double* pa = a + v * vs + x;
  double* pb = b + v * vs + x;
  double* pc = c + v * vs + x;
  int j0 = qfirst[0] - 1;
  double ua[P], ub[P], uc[P], sa[P], sb[P], sc[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    const bool ok = j >= 0 && j < n;
    ua[l] = ok ? pa[(long long)j * A] : 0.0;
    ub[l] = ok ? pb[(long long)j * A] : 0.0;
    uc[l] = ok ? pc[(long long)j * A] : 0.0;
    sa[l] = sb[l] = sc[l] = 0.0;
  }
  for (int q = 0; q < Q; ++q) {
    const int jq = qfirst[q] - 1;
    while (j0 < jq) {
      if (j0 >= 0 && j0 < n) {
        pa[(long long)j0 * A] = sa[0];
        pb[(long long)j0 * A] = sb[0];
        pc[(long long)j0 * A] = sc[0];
      }
#pragma unroll
      for (int l = 0; l < P - 1; ++l) {
        ua[l] = ua[l + 1]; ub[l] = ub[l + 1]; uc[l] = uc[l + 1];
        sa[l] = sa[l + 1]; sb[l] = sb[l + 1]; sc[l] = sc[l + 1];
      }
      const int jn = j0 + P;
      const bool ok = jn >= 0 && jn < n;
      ua[P - 1] = ok ? pa[(long long)jn * A] : 0.0;
      ub[P - 1] = ok ? pb[(long long)jn * A] : 0.0;
      uc[P - 1] = ok ? pc[(long long)jn * A] : 0.0;
      sa[P - 1] = sb[P - 1] = sc[P - 1] = 0.0;
      ++j0;
    }
    const double* bv = Tv + q * P;
    const double* bd = Td + q * P;
    double g2 = 0.0, g1 = 0.0, g0 = 0.0;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      g2 = fma(bd[l], ua[l], g2);
      g1 = fma(bv[l], ub[l], g1);
      g0 = fma(bv[l], uc[l], g0);
    }
    const long long pi = x + (long long)q * A;
    const double gxx = G[pi], gyy = G[gs + pi], gzz = G[2 * gs + pi];
    const double gxy = G[3 * gs + pi], gxz = G[4 * gs + pi], gyz = G[5 * gs + pi];
    const double h0 = gxx * g0 + gxy * g1 + gxz * g2;
    const double h1 = gxy * g0 + gyy * g1 + gyz * g2;
    const double h2 = gxz * g0 + gyz * g1 + gzz * g2;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      sa[l] = fma(bd[l], h2, sa[l]);
      sb[l] = fma(bv[l], h1, sb[l]);
      sc[l] = fma(bv[l], h0, sc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    if (j >= 0 && j < n) {
      pa[(long long)j * A] = sa[l];
      pb[(long long)j * A] = sb[l];
      pc[(long long)j * A] = sc[l];
    }
  }
}

// 2-D: a -> derivative along the last axis (g1), c -> value (g0); G = (xx, yy, xy).
template <int P>
__global__ void __launch_bounds__(128) k_mid_stiff2(const int* __restrict__ qfirst, const double* __restrict__ Tv,
                                                    const double* __restrict__ Td, int A, int n, int Q,
                                                    const int* __restrict__ active, const double* __restrict__ G,
                                                    long long gs, double* a, double* c, long long vs) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A) return;
  double* pa = a + v * vs + x;
  double* pc = c + v * vs + x;
  int j0 = qfirst[0] - 1;
  double ua[P], uc[P], sa[P], sc[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    const bool ok = j >= 0 && j < n;
    ua[l] = ok ? pa[(long long)j * A] : 0.0;
    uc[l] = ok ? pc[(long long)j * A] : 0.0;
    sa[l] = sc[l] = 0.0;
  }
  for (int q = 0; q < Q; ++q) {
    const int jq = qfirst[q] - 1;
    while (j0 < jq) {
      if (j0 >= 0 && j0 < n) {
        pa[(long long)j0 * A] = sa[0];
        pc[(long long)j0 * A] = sc[0];
      }
#pragma unroll
      for (int l = 0; l < P - 1; ++l) {
        ua[l] = ua[l + 1]; uc[l] = uc[l + 1];
        sa[l] = sa[l + 1]; sc[l] = sc[l + 1];
      }
      const int jn = j0 + P;
      const bool ok = jn >= 0 && jn < n;
      ua[P - 1] = ok ? pa[(long long)jn * A] : 0.0;
      uc[P - 1] = ok ? pc[(long long)jn * A] : 0.0;
      sa[P - 1] = sc[P - 1] = 0.0;
      ++j0;
    }
    const double* bv = Tv + q * P;
    const double* bd = Td + q * P;
    double g1 = 0.0, g0 = 0.0;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      g1 = fma(bd[l], ua[l], g1);
      g0 = fma(bv[l], uc[l], g0);
    }
    const long long pi = x + (long long)q * A;
    const double gxx = G[pi], gyy = G[gs + pi], gxy = G[2 * gs + pi];
    const double h0 = gxx * g0 + gxy * g1;
    const double h1 = gxy * g0 + gyy * g1;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      sa[l] = fma(bd[l], h1, sa[l]);
      sc[l] = fma(bv[l], h0, sc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < P; ++l) {
    const int j = j0 + l;
    if (j >= 0 && j < n) {
      pa[(long long)j * A] = sa[l];
      pc[(long long)j * A] = sc[l];
    }
  }
}

// ----------------------------------------------------------------------------
// geometric factors: DF = sum_i C_i (x) grad B_i over the (p+1)^d functions
// nonzero at the point; W = w |det DF|, G = W DF^{-1} DF^{-T}.
// ----------------------------------------------------------------------------
struct GeoDir {
  const double* val;
  const double* der;
  const int* qfirst;
  const double* qw;
  int P, Q, m;
};

template <int D>
__global__ void k_geometry(GeoDir g0, GeoDir g1, GeoDir g2, const double* __restrict__ cx,
                           const double* __restrict__ cy, const double* __restrict__ cz, double* __restrict__ W,
                           double* __restrict__ G, long long gs, int* bad) {
  const long long Qt = (long long)g0.Q * g1.Q * (D == 3 ? g2.Q : 1);
  const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= Qt) return;
  const int q0 = (int)(qi % g0.Q);
  const int q1 = (int)((qi / g0.Q) % g1.Q);
  const int q2 = D == 3 ? (int)(qi / ((long long)g0.Q * g1.Q)) : 0;
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const int f0 = g0.qfirst[q0], f1 = g1.qfirst[q1], f2 = D == 3 ? g2.qfirst[q2] : 0;
  const int P2 = D == 3 ? g2.P : 1;
  for (int l2 = 0; l2 < P2; ++l2) {
    const double v2 = D == 3 ? g2.val[q2 * g2.P + l2] : 1.0;
    const double d2 = D == 3 ? g2.der[q2 * g2.P + l2] : 0.0;
    for (int l1 = 0; l1 < g1.P; ++l1) {
      const double v1 = g1.val[q1 * g1.P + l1], d1 = g1.der[q1 * g1.P + l1];
      for (int l0 = 0; l0 < g0.P; ++l0) {
        const double v0 = g0.val[q0 * g0.P + l0], d0 = g0.der[q0 * g0.P + l0];
        const long long ci = (f0 + l0) + (long long)g0.m * ((f1 + l1) + (long long)g1.m * (f2 + l2));
        const double gr[3] = {d0 * v1 * v2, v0 * d1 * v2, v0 * v1 * d2};
        const double C[3] = {cx[ci], cy[ci], D == 3 ? cz[ci] : 0.0};
        for (int c = 0; c < D; ++c)
          for (int b = 0; b < D; ++b) J[c][b] = fma(C[c], gr[b], J[c][b]);
      }
    }
  }
  const double w = g0.qw[q0] * g1.qw[q1] * (D == 3 ? g2.qw[q2] : 1.0);
  double det, Ji[3][3];
  if (D == 3) {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double r = 1.0 / det;
    Ji[0][0] = c00 * r;
    Ji[1][0] = c01 * r;
    Ji[2][0] = c02 * r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
  } else {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double r = 1.0 / det;
    Ji[0][0] = J[1][1] * r;
    Ji[0][1] = -J[0][1] * r;
    Ji[1][0] = -J[1][0] * r;
    Ji[1][1] = J[0][0] * r;
  }
  if (!(det > 0.0)) atomicExch(bad, 1);
  const double Wq = w * fabs(det);
  W[qi] = Wq;
  double S[3][3];
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      double s = 0.0;
      for (int c = 0; c < D; ++c) s = fma(Ji[a][c], Ji[b][c], s);
      S[a][b] = Wq * s;
    }
  if (D == 3) {
    G[qi] = S[0][0];
    G[gs + qi] = S[1][1];
    G[2 * gs + qi] = S[2][2];
    G[3 * gs + qi] = S[0][1];
    G[4 * gs + qi] = S[0][2];
    G[5 * gs + qi] = S[1][2];
  } else {
    G[qi] = S[0][0];
    G[gs + qi] = S[1][1];
    G[2 * gs + qi] = S[0][1];
  }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
#define IGA_DISPATCH_P(P, ...)                              \
  switch (P) {                                              \
    case 2: { constexpr int PP = 2; __VA_ARGS__; } break;  \
    case 3: { constexpr int PP = 3; __VA_ARGS__; } break;  \
    case 4: { constexpr int PP = 4; __VA_ARGS__; } break;  \
    case 5: { constexpr int PP = 5; __VA_ARGS__; } break;  \
    case 6: { constexpr int PP = 6; __VA_ARGS__; } break;  \
    case 7: { constexpr int PP = 7; __VA_ARGS__; } break;  \
    default: return cudaErrorInvalidValue;                  \
  }

static inline dim3 plane_grid(long long plane, long long B, int nvec, int threads) {
  return dim3((unsigned)((plane + threads - 1) / threads), (unsigned)B, (unsigned)nvec);
}

cudaError_t launch_fwd(cudaStream_t s, const DirDev& d, AxisShape sh, int nvec, const int* active,
                       const double* in, long long in_vs, const double* T0, double* out0, const double* T1,
                       double* out1, long long out_vs) {
  if (sh.B > 65535 || sh.A * sh.Lout > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int A = (int)sh.A;
  dim3 grid = plane_grid(sh.A * sh.Lout, sh.B, nvec, 256);
  const bool two = T1 != nullptr;
  IGA_DISPATCH_P(d.P, {
    if (A == 1) {
      if (two) k_fwd<PP, true, true><<<grid, 256, 0, s>>>(d.qfirst, T0, T1, A, sh.Lin, sh.Lout, active, in, in_vs, out0, out1, out_vs);
      else k_fwd<PP, false, true><<<grid, 256, 0, s>>>(d.qfirst, T0, T1, A, sh.Lin, sh.Lout, active, in, in_vs, out0, out1, out_vs);
    } else {
      if (two) k_fwd<PP, true, false><<<grid, 256, 0, s>>>(d.qfirst, T0, T1, A, sh.Lin, sh.Lout, active, in, in_vs, out0, out1, out_vs);
      else k_fwd<PP, false, false><<<grid, 256, 0, s>>>(d.qfirst, T0, T1, A, sh.Lin, sh.Lout, active, in, in_vs, out0, out1, out_vs);
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_tr(cudaStream_t s, const DirDev& d, AxisShape sh, int nvec, const int* active,
                      const double* in0, const double* T0, const double* in1, const double* T1, long long in_vs,
                      double* out, long long out_vs) {
  if (sh.B > 65535 || sh.A * sh.Lout > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int A = (int)sh.A;
  dim3 grid = plane_grid(sh.A * sh.Lout, sh.B, nvec, 256);
  const bool two = in1 != nullptr;
  IGA_DISPATCH_P(d.P, {
    if (A == 1) {
      if (two) k_tr<PP, true, true><<<grid, 256, 0, s>>>(d.qfirst, d.flo, d.fhi, T0, T1, A, sh.Lin, sh.Lout, active, in0, in1, in_vs, out, out_vs);
      else k_tr<PP, false, true><<<grid, 256, 0, s>>>(d.qfirst, d.flo, d.fhi, T0, T1, A, sh.Lin, sh.Lout, active, in0, in1, in_vs, out, out_vs);
    } else {
      if (two) k_tr<PP, true, false><<<grid, 256, 0, s>>>(d.qfirst, d.flo, d.fhi, T0, T1, A, sh.Lin, sh.Lout, active, in0, in1, in_vs, out, out_vs);
      else k_tr<PP, false, false><<<grid, 256, 0, s>>>(d.qfirst, d.flo, d.fhi, T0, T1, A, sh.Lin, sh.Lout, active, in0, in1, in_vs, out, out_vs);
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_mid_mass(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                            const double* W, const double* in, double* out, long long vs) {
  if (A > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A + 127) / 128), (unsigned)nvec);
  IGA_DISPATCH_P(d.P, { k_mid_mass<PP><<<grid, 128, 0, s>>>(d.qfirst, d.val, (int)A, d.n, d.Q, active, W, in, out, vs); });
  return cudaGetLastError();
}

cudaError_t launch_mid_stiff3(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                              const double* G, long long gstride, double* a, double* b, double* c, long long vs) {
  if (A > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A + 127) / 128), (unsigned)nvec);
  IGA_DISPATCH_P(d.P, { k_mid_stiff3<PP><<<grid, 128, 0, s>>>(d.qfirst, d.val, d.der, (int)A, d.n, d.Q, active, G, gstride, a, b, c, vs); });
  return cudaGetLastError();
}

cudaError_t launch_mid_stiff2(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                              const double* G, long long gstride, double* a, double* c, long long vs) {
  if (A > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A + 127) / 128), (unsigned)nvec);
  IGA_DISPATCH_P(d.P, { k_mid_stiff2<PP><<<grid, 128, 0, s>>>(d.qfirst, d.val, d.der, (int)A, d.n, d.Q, active, G, gstride, a, c, vs); });
  return cudaGetLastError();
}

cudaError_t launch_geometry(cudaStream_t s, int dim, const DirDev* dirs, const int* m, const double* ctrl_soa,
                            double* W, double* G, long long gstride, int* bad) {
  GeoDir g[3];
  long long Qt = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      // the geometry reads the full control net: full function indices
      const int* qf = dirs[a].qfirst_geo ? dirs[a].qfirst_geo : dirs[a].qfirst;
      g[a] = GeoDir{dirs[a].val, dirs[a].der, qf, dirs[a].qw, dirs[a].P, dirs[a].Q, m[a]};
      Qt *= dirs[a].Q;
    } else {
      g[a] = GeoDir{nullptr, nullptr, nullptr, nullptr, 1, 1, 1};
    }
  }
  long long mt = (long long)m[0] * m[1] * (dim == 3 ? m[2] : 1);
  const unsigned blocks = (unsigned)((Qt + 255) / 256);
  if (dim == 3)
    k_geometry<3><<<blocks, 256, 0, s>>>(g[0], g[1], g[2], ctrl_soa, ctrl_soa + mt, ctrl_soa + 2 * mt, W, G, gstride, bad);
  else
    k_geometry<2><<<blocks, 256, 0, s>>>(g[0], g[1], g[2], ctrl_soa, ctrl_soa + mt, nullptr, W, G, gstride, bad);
  return cudaGetLastError();
}

}  // namespace iga
