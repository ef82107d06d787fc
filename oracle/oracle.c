/*
 * oracle.c -- plain FP64 CPU oracle for the isogeometric operators of the
 * explicit high-order generalized-alpha method (arXiv 2102.11536).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.
 * The CUDA product path shares no code with it and never links it.
 *
 * Each routine restates a definition of the paper directly, with no blocking,
 * sum factorisation or reordering beyond what the definition states:
 *   - univariate B-splines by the Cox-de Boor recursion with 0/0 = 0
 *     (Sec. 5.1, "B-splines");
 *   - tensor-product basis and co-lexicographic numbering (Sec. 5.1-5.2,
 *     multivariate B-splines and def:parametric_spline);
 *   - geometry F(xi) = sum_i C_i B_i(xi) (Sec. 5.2);
 *   - mass matrix [M]_ij = int B_i B_j |det DF| (eq. mass_matrix);
 *   - stiffness K_ij = int grad B_i . grad B_j, the Galerkin form of eq. pde
 *     with omega = 1 and c = 0 (Sec. 2.1, Sec. 6), pulled back to the
 *     parametric cube: int gradhat B_i^T DF^-1 DF^-T gradhat B_j |det DF|.
 * The paper does not fix the quadrature; the oracle uses Gauss-Legendre with
 * nq points per element and direction (nq = p+1 by default), the GeoPDEs
 * default that the paper's experiments ran on (Sec. 6).
 *
 * Homogeneous Dirichlet conditions (Sec. 2, remark on homogeneous boundary
 * conditions) drop the first and last univariate function in every direction;
 * "interior" indices below count only the remaining functions.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Cox-de Boor recursion (Sec. 5.1). Evaluates all m = nknots-p-1 degree-p
 * B-splines of the knot vector U at x, and their first derivatives.
 * Degree 0: b_{i,0}(x) = 1 if U_i <= x < U_{i+1}, else 0. At the right end
 * x == U_last the last non-empty span is taken closed on the right (limit
 * from the left), so that the partition of unity also holds at x = 1.
 * Degree r: b_{i,r} = (x-U_i)/(U_{i+r}-U_i) b_{i,r-1}
 *                   + (U_{i+r+1}-x)/(U_{i+r+1}-U_{i+1}) b_{i+1,r-1}, 0/0 = 0.
 * Derivative (de Boor): b'_{i,p} = p b_{i,p-1}/(U_{i+p}-U_i)
 *                                 - p b_{i+1,p-1}/(U_{i+p+1}-U_{i+1}), 0/0 = 0.
 * Returns 0, or -1 on bad arguments.
 * ------------------------------------------------------------------------- */
int ora_basis(int p, int nknots, const double* U, double x, double* val, double* der) {
  int m = nknots - p - 1;
  if (p < 0 || m < 1) return -1;
  int n0 = nknots - 1; /* number of degree-0 functions */
  double* N = (double*)calloc((size_t)n0, sizeof(double));
  double* Nprev = (double*)calloc((size_t)n0, sizeof(double));
  if (!N || !Nprev) { free(N); free(Nprev); return -1; }
  int last = -1;
  for (int i = 0; i < n0; ++i) if (U[i + 1] > U[i]) last = i;
  for (int i = 0; i < n0; ++i) {
    int inside = (U[i] <= x && x < U[i + 1]);
    if (i == last && x == U[i + 1]) inside = 1;
    N[i] = inside ? 1.0 : 0.0;
  }
  for (int r = 1; r <= p; ++r) {
    memcpy(Nprev, N, sizeof(double) * (size_t)n0);
    for (int i = 0; i < n0 - r; ++i) {
      double a = 0.0, b = 0.0;
      double dl = U[i + r] - U[i];
      double dr = U[i + r + 1] - U[i + 1];
      if (dl > 0.0) a = (x - U[i]) / dl * Nprev[i];
      if (dr > 0.0) b = (U[i + r + 1] - x) / dr * Nprev[i + 1];
      N[i] = a + b;
    }
    for (int i = n0 - r; i < n0; ++i) N[i] = 0.0;
  }
  for (int i = 0; i < m; ++i) val[i] = N[i];
  if (der) {
    if (p == 0) {
      for (int i = 0; i < m; ++i) der[i] = 0.0;
    } else {
      /* Nprev holds degree p-1 */
      for (int i = 0; i < m; ++i) {
        double a = 0.0, b = 0.0;
        double dl = U[i + p] - U[i];
        double dr = U[i + p + 1] - U[i + 1];
        if (dl > 0.0) a = p * Nprev[i] / dl;
        if (dr > 0.0) b = p * Nprev[i + 1] / dr;
        der[i] = a - b;
      }
    }
  }
  free(N);
  free(Nprev);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Gauss-Legendre rule with n points on [-1, 1]: nodes are the roots of the
 * Legendre polynomial P_n, found by Newton's method on the three-term
 * recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}; weights
 * w = 2 / ((1 - x^2) P_n'(x)^2). Nodes ascending.
 * ------------------------------------------------------------------------- */
void ora_gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      if (n == 0) p1 = 1.0;
      for (int j = 1; j < n; ++j) {
        double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        /* one more evaluation at the converged node for the weight */
        p0 = 1.0; p1 = z;
        for (int j = 1; j < n; ++j) {
          double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ---------------------------------------------------------------------------
 * Univariate quadrature tables. Every non-empty knot span [U_s, U_{s+1}] is
 * an element; it carries nq Gauss points. For quadrature point q = e*nq + g
 * the tables hold the parametric coordinate qx, the weight qw (Gauss weight
 * times half the span length), the index qfirst of the first of the p+1
 * functions that can be nonzero on that span (s - p, the local support
 * property of Sec. 5.1), and their values qval[q*(p+1)+a] and derivatives
 * qder[q*(p+1)+a]. Returns the number of elements.
 * ------------------------------------------------------------------------- */
int ora_quad_1d(int p, int nknots, const double* U, int nq, double* qx, double* qw, int* qfirst,
                double* qval, double* qder) {
  int m = nknots - p - 1;
  double* gx = (double*)malloc(sizeof(double) * (size_t)nq);
  double* gw = (double*)malloc(sizeof(double) * (size_t)nq);
  double* val = (double*)malloc(sizeof(double) * (size_t)m);
  double* der = (double*)malloc(sizeof(double) * (size_t)m);
  ora_gauss_legendre(nq, gx, gw);
  int e = 0;
  for (int s = p; s < m; ++s) {
    if (!(U[s + 1] > U[s])) continue;
    double h = U[s + 1] - U[s];
    for (int g = 0; g < nq; ++g) {
      int q = e * nq + g;
      double xx = U[s] + 0.5 * h * (gx[g] + 1.0);
      qx[q] = xx;
      qw[q] = 0.5 * h * gw[g];
      qfirst[q] = s - p;
      ora_basis(p, nknots, U, xx, val, der);
      for (int a = 0; a <= p; ++a) {
        qval[q * (p + 1) + a] = val[s - p + a];
        qder[q * (p + 1) + a] = der[s - p + a];
      }
    }
    ++e;
  }
  free(gx); free(gw); free(val); free(der);
  return e;
}

/* Mesh description shared by the routines below (all arrays caller-owned).
 * dims = {d, p0, p1, p2, m0, m1, m2, Q0, Q1, Q2}; the per-direction tables
 * qw/qfirst/qval/qder of ora_quad_1d are concatenated direction after
 * direction. ctrl holds the full control net, co-lexicographic, d coords per
 * point. For d = 2 the third direction is absent (m2 = Q2 = 1 is ignored). */
typedef struct {
  int d, p[3], m[3], Q[3];
  const double* qw[3];
  const int* qfirst[3];
  const double* qval[3];
  const double* qder[3];
} mesh_t;

static void mesh_from(mesh_t* g, const int* dims, const double* qw, const int* qfirst,
                      const double* qval, const double* qder) {
  g->d = dims[0];
  long ow = 0, ov = 0;
  for (int a = 0; a < 3; ++a) {
    g->p[a] = dims[1 + a];
    g->m[a] = dims[4 + a];
    g->Q[a] = dims[7 + a];
    if (a >= g->d) { g->p[a] = 0; g->m[a] = 1; g->Q[a] = 1; }
  }
  for (int a = 0; a < g->d; ++a) {
    g->qw[a] = qw + ow;
    g->qfirst[a] = qfirst + ow;
    g->qval[a] = qval + ov;
    g->qder[a] = qder + ov;
    ow += g->Q[a];
    ov += (long)g->Q[a] * (g->p[a] + 1);
  }
}

/* value / derivative of full univariate function f of direction a at quad point q (0 off support) */
static double bval(const mesh_t* g, int a, int q, int f) {
  if (a >= g->d) return 1.0;
  int l = f - g->qfirst[a][q];
  if (l < 0 || l > g->p[a]) return 0.0;
  return g->qval[a][q * (g->p[a] + 1) + l];
}
static double bder(const mesh_t* g, int a, int q, int f) {
  if (a >= g->d) return 0.0;
  int l = f - g->qfirst[a][q];
  if (l < 0 || l > g->p[a]) return 0.0;
  return g->qder[a][q * (g->p[a] + 1) + l];
}

/* ---------------------------------------------------------------------------
 * Geometric factors at every tensor quadrature point (co-lex over q1,q2,q3):
 *   W = w_q |det DF|,   G = W DF^-1 DF^-T  (symmetric; 3-D order xx,yy,zz,xy,xz,yz,
 *   2-D order xx,yy,xy), with DF_{cb} = sum_i C_{i,c} d B_i / d xi_b
 * summed over the functions whose support contains the point (Sec. 5.2).
 * detmin receives the smallest det DF. Returns 0, or 1 if det DF <= 0 somewhere
 * (Assumption on g_regularity violated).
 * ------------------------------------------------------------------------- */
int ora_geometry(const int* dims, const double* qw, const int* qfirst, const double* qval, const double* qder,
                 const double* ctrl, double* W, double* G, double* detmin) {
  mesh_t g;
  mesh_from(&g, dims, qw, qfirst, qval, qder);
  const int d = g.d;
  const long Qt = (long)g.Q[0] * g.Q[1] * g.Q[2];
  const int ng = d == 3 ? 6 : 3;
  double dmin = 1e300;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(min : dmin) reduction(| : bad)
  for (long qi = 0; qi < Qt; ++qi) {
    int q[3];
    q[0] = (int)(qi % g.Q[0]);
    q[1] = (int)((qi / g.Q[0]) % g.Q[1]);
    q[2] = (int)(qi / ((long)g.Q[0] * g.Q[1]));
    double J[3][3] = {{0}};
    int f0[3], f1[3];
    for (int a = 0; a < 3; ++a) {
      f0[a] = a < d ? g.qfirst[a][q[a]] : 0;
      f1[a] = a < d ? f0[a] + g.p[a] : 0;
    }
    for (int i2 = f0[2]; i2 <= f1[2]; ++i2)
      for (int i1 = f0[1]; i1 <= f1[1]; ++i1)
        for (int i0 = f0[0]; i0 <= f1[0]; ++i0) {
          long idx = i0 + (long)g.m[0] * (i1 + (long)g.m[1] * i2);
          double v0 = bval(&g, 0, q[0], i0), v1 = bval(&g, 1, q[1], i1), v2 = bval(&g, 2, q[2], i2);
          double grad[3];
          grad[0] = bder(&g, 0, q[0], i0) * v1 * v2;
          grad[1] = v0 * bder(&g, 1, q[1], i1) * v2;
          grad[2] = v0 * v1 * bder(&g, 2, q[2], i2);
          for (int c = 0; c < d; ++c)
            for (int b = 0; b < d; ++b) J[c][b] += ctrl[idx * d + c] * grad[b];
        }
    double w = 1.0;
    for (int a = 0; a < d; ++a) w *= g.qw[a][q[a]];
    double det, Ji[3][3];
    if (d == 3) {
      det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      /* inverse by the adjugate */
      Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    } else {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det;
      Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det;
      Ji[1][1] = J[0][0] / det;
    }
    if (det < dmin) dmin = det;
    if (!(det > 0.0)) bad = 1;
    double Wq = w * fabs(det);
    W[qi] = Wq;
    /* (DF^-1 DF^-T)_{ab} = sum_c Ji[a][c] Ji[b][c] */
    double S[3][3];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += Ji[a][c] * Ji[b][c];
        S[a][b] = Wq * s;
      }
    if (d == 3) {
      G[qi * 6 + 0] = S[0][0];
      G[qi * 6 + 1] = S[1][1];
      G[qi * 6 + 2] = S[2][2];
      G[qi * 6 + 3] = S[0][1];
      G[qi * 6 + 4] = S[0][2];
      G[qi * 6 + 5] = S[1][2];
    } else {
      G[qi * 3 + 0] = S[0][0];
      G[qi * 3 + 1] = S[1][1];
      G[qi * 3 + 2] = S[0][1];
    }
    (void)ng;
  }
  *detmin = dmin;
  return bad;
}

/* ---------------------------------------------------------------------------
 * Rows of the interior mass and stiffness matrices by Gauss quadrature.
 * Row i (interior co-lex index, full multi-index f = i + 1 per direction)
 * couples to every interior j with |j_a - f_a| <= p_a; its entries are stored
 * in S = prod_a (2 p_a + 1) "band slots", slot = (o0+p0) + (2p0+1)((o1+p1) +
 * (2p1+1)(o2+p2)) for the offset o = j - f (slots whose j is outside the
 * interior stay zero). For every quadrature point q in the support of B_i
 * and every function B_j nonzero at q:
 *   M_ij += B_i(q) B_j(q) W(q)
 *   K_ij += gradhat B_j(q) . ( G(q) gradhat B_i(q) )
 * which is eq. mass_matrix and the pulled-back stiffness integral summed over
 * the elements of supp B_i. rows == NULL means all rows 0..nrows-1.
 * ------------------------------------------------------------------------- */
int ora_assemble_rows(const int* dims, const double* qw, const int* qfirst, const double* qval,
                      const double* qder, const double* W, const double* G, const long* rows, long nrows,
                      double* Mrows, double* Krows) {
  mesh_t g;
  mesh_from(&g, dims, qw, qfirst, qval, qder);
  const int d = g.d;
  int n[3], S1[3];
  for (int a = 0; a < 3; ++a) {
    n[a] = a < d ? g.m[a] - 2 : 1;
    S1[a] = 2 * g.p[a] + 1;
  }
  const long S = (long)S1[0] * S1[1] * S1[2];
#pragma omp parallel for schedule(dynamic, 16)
  for (long r = 0; r < nrows; ++r) {
    long i = rows ? rows[r] : r;
    double* Mr = Mrows + r * S;
    double* Kr = Krows ? Krows + r * S : NULL;
    for (long s = 0; s < S; ++s) {
      Mr[s] = 0.0;
      if (Kr) Kr[s] = 0.0;
    }
    int f[3];
    f[0] = (int)(i % n[0]) + (d > 0 ? 1 : 0);
    f[1] = (int)((i / n[0]) % n[1]) + (d > 1 ? 1 : 0);
    f[2] = (int)(i / ((long)n[0] * n[1])) + (d > 2 ? 1 : 0);
    /* quadrature points (per direction) in the support of f_a */
    int qlo[3], qhi[3];
    for (int a = 0; a < 3; ++a) {
      if (a >= d) { qlo[a] = 0; qhi[a] = 0; f[a] = 0; continue; }
      qlo[a] = -1; qhi[a] = -2;
      for (int q = 0; q < g.Q[a]; ++q) {
        int l = f[a] - g.qfirst[a][q];
        if (l >= 0 && l <= g.p[a]) {
          if (qlo[a] < 0) qlo[a] = q;
          qhi[a] = q;
        }
      }
    }
    for (int q2 = qlo[2]; q2 <= qhi[2]; ++q2)
      for (int q1 = qlo[1]; q1 <= qhi[1]; ++q1)
        for (int q0 = qlo[0]; q0 <= qhi[0]; ++q0) {
          long qi = q0 + (long)g.Q[0] * (q1 + (long)g.Q[1] * q2);
          double vi0 = bval(&g, 0, q0, f[0]), vi1 = bval(&g, 1, q1, f[1]), vi2 = bval(&g, 2, q2, f[2]);
          double bi = vi0 * vi1 * vi2;
          if (bi == 0.0 && bder(&g, 0, q0, f[0]) == 0.0 && bder(&g, 1, q1, f[1]) == 0.0 &&
              bder(&g, 2, q2, f[2]) == 0.0)
            continue;
          double gi[3] = {bder(&g, 0, q0, f[0]) * vi1 * vi2, vi0 * bder(&g, 1, q1, f[1]) * vi2,
                          vi0 * vi1 * bder(&g, 2, q2, f[2])};
          double h[3] = {0, 0, 0};
          if (Kr) {
            double Gm[3][3] = {{0}};
            if (d == 3) {
              const double* Gq = G + qi * 6;
              Gm[0][0] = Gq[0]; Gm[1][1] = Gq[1]; Gm[2][2] = Gq[2];
              Gm[0][1] = Gm[1][0] = Gq[3];
              Gm[0][2] = Gm[2][0] = Gq[4];
              Gm[1][2] = Gm[2][1] = Gq[5];
            } else {
              const double* Gq = G + qi * 3;
              Gm[0][0] = Gq[0]; Gm[1][1] = Gq[1];
              Gm[0][1] = Gm[1][0] = Gq[2];
            }
            for (int a = 0; a < d; ++a)
              for (int b = 0; b < d; ++b) h[a] += Gm[a][b] * gi[b];
          }
          double wq = W[qi];
          int q[3] = {q0, q1, q2};
          int j0[3], j1[3];
          /* values / derivatives of the functions nonzero at this point, per direction */
          double vj[3][16], dj[3][16];
          for (int a = 0; a < 3; ++a) {
            j0[a] = a < d ? g.qfirst[a][q[a]] : 0;
            j1[a] = a < d ? j0[a] + g.p[a] : 0;
            for (int c = j0[a]; c <= j1[a]; ++c) {
              vj[a][c - j0[a]] = bval(&g, a, q[a], c);
              dj[a][c - j0[a]] = bder(&g, a, q[a], c);
            }
          }
          for (int c2 = j0[2]; c2 <= j1[2]; ++c2) {
            if (d > 2 && (c2 == 0 || c2 == g.m[2] - 1)) continue;
            for (int c1 = j0[1]; c1 <= j1[1]; ++c1) {
              if (d > 1 && (c1 == 0 || c1 == g.m[1] - 1)) continue;
              for (int c0 = j0[0]; c0 <= j1[0]; ++c0) {
                if (c0 == 0 || c0 == g.m[0] - 1) continue;
                int o0 = c0 - f[0], o1 = c1 - f[1], o2 = c2 - f[2];
                if (o0 < -g.p[0] || o0 > g.p[0] || o1 < -g.p[1] || o1 > g.p[1] || o2 < -g.p[2] || o2 > g.p[2])
                  continue;
                long slot = (o0 + g.p[0]) + (long)S1[0] * ((o1 + g.p[1]) + (long)S1[1] * (o2 + g.p[2]));
                double vj0 = vj[0][c0 - j0[0]], vj1 = vj[1][c1 - j0[1]], vj2 = vj[2][c2 - j0[2]];
                Mr[slot] += bi * vj0 * vj1 * vj2 * wq;
                if (Kr) {
                  double gj0 = dj[0][c0 - j0[0]] * vj1 * vj2;
                  double gj1 = vj0 * dj[1][c1 - j0[1]] * vj2;
                  double gj2 = vj0 * vj1 * dj[2][c2 - j0[2]];
                  Kr[slot] += gj0 * h[0] + gj1 * h[1] + gj2 * h[2];
                }
              }
            }
          }
        }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * y = A x for a matrix held as band rows (layout of ora_assemble_rows):
 *   y_i = sum_slot A[i][slot] x_{i + offset(slot)}, offsets inside the interior.
 * n = interior sizes {n0, n1, n2}, p = degrees (p2 = 0 and n2 = 1 for 2-D).
 * ------------------------------------------------------------------------- */
void ora_band_matvec(const int* n, const int* p, const double* A, const double* x, double* y) {
  const long N = (long)n[0] * n[1] * n[2];
  int S1[3] = {2 * p[0] + 1, 2 * p[1] + 1, 2 * p[2] + 1};
  const long S = (long)S1[0] * S1[1] * S1[2];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < N; ++i) {
    int i0 = (int)(i % n[0]), i1 = (int)((i / n[0]) % n[1]), i2 = (int)(i / ((long)n[0] * n[1]));
    const double* Ai = A + i * S;
    double acc = 0.0;
    for (int o2 = -p[2]; o2 <= p[2]; ++o2) {
      int j2 = i2 + o2;
      if (j2 < 0 || j2 >= n[2]) continue;
      for (int o1 = -p[1]; o1 <= p[1]; ++o1) {
        int j1 = i1 + o1;
        if (j1 < 0 || j1 >= n[1]) continue;
        for (int o0 = -p[0]; o0 <= p[0]; ++o0) {
          int j0 = i0 + o0;
          if (j0 < 0 || j0 >= n[0]) continue;
          long slot = (o0 + p[0]) + (long)S1[0] * ((o1 + p[1]) + (long)S1[1] * (o2 + p[2]));
          acc += Ai[slot] * x[j0 + (long)n[0] * (j1 + (long)n[1] * j2)];
        }
      }
    }
    y[i] = acc;
  }
}

/* ---------------------------------------------------------------------------
 * Diagonal of the interior mass matrix, D_i = M_ii = sum_q B_i(q)^2 W(q) over
 * the quadrature points in the support of B_i (def:matrices_1, D = diag(M)).
 * ------------------------------------------------------------------------- */
int ora_mass_diagonal(const int* dims, const double* qw, const int* qfirst, const double* qval, const double* qder,
                      const double* W, double* D) {
  mesh_t g;
  mesh_from(&g, dims, qw, qfirst, qval, qder);
  const int d = g.d;
  int n[3];
  for (int a = 0; a < 3; ++a) n[a] = a < d ? g.m[a] - 2 : 1;
  const long N = (long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < N; ++i) {
    int f[3];
    f[0] = (int)(i % n[0]) + 1;
    f[1] = (int)((i / n[0]) % n[1]) + (d > 1 ? 1 : 0);
    f[2] = (int)(i / ((long)n[0] * n[1])) + (d > 2 ? 1 : 0);
    double acc = 0.0;
    for (int q2 = 0; q2 < g.Q[2]; ++q2) {
      double v2 = bval(&g, 2, q2, f[2]);
      if (v2 == 0.0) continue;
      for (int q1 = 0; q1 < g.Q[1]; ++q1) {
        double v1 = bval(&g, 1, q1, f[1]);
        if (v1 == 0.0) continue;
        for (int q0 = 0; q0 < g.Q[0]; ++q0) {
          double v0 = bval(&g, 0, q0, f[0]);
          if (v0 == 0.0) continue;
          double b = v0 * v1 * v2;
          acc += b * b * W[q0 + (long)g.Q[0] * (q1 + (long)g.Q[1] * q2)];
        }
      }
    }
    D[i] = acc;
  }
  return 0;
}
