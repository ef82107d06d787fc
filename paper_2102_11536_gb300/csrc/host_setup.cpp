// Host-side univariate setup: Gauss rule, B-spline tables, parametric mass
// matrix and its eigen-decomposition for the fast-diagonalisation preconditioner.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "iga_internal.h"

namespace iga {

// Cyclic Jacobi rotations on a symmetric matrix. A = V diag(eval) V^T on exit,
// V stored row-major with eigenvector c in column c. Sweeps until every
// off-diagonal entry is below 1e-300 relative to the Frobenius norm or no
// rotation changes anything.
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& evec, std::vector<double>& eval) {
  evec.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) evec[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    int rotations = 0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        // an entry negligible against the geometric mean of its diagonal is dropped
        if (std::fabs(apq) <= 1e-18 * std::sqrt(std::fabs(app * aqq))) {
          A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
          continue;
        }
        ++rotations;
        // rotation angle that annihilates a_pq: cot(2 phi) = (a_qq - a_pp) / (2 a_pq)
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {  // columns p, q of A
          double arp = A[(size_t)r * n + p], arq = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = c * arp - s * arq;
          A[(size_t)r * n + q] = s * arp + c * arq;
        }
        for (int r = 0; r < n; ++r) {  // rows p, q of A
          double apr = A[(size_t)p * n + r], aqr = A[(size_t)q * n + r];
          A[(size_t)p * n + r] = c * apr - s * aqr;
          A[(size_t)q * n + r] = s * apr + c * aqr;
        }
        A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
        for (int r = 0; r < n; ++r) {  // accumulate V <- V J
          double vrp = evec[(size_t)r * n + p], vrq = evec[(size_t)r * n + q];
          evec[(size_t)r * n + p] = c * vrp - s * vrq;
          evec[(size_t)r * n + q] = s * vrp + c * vrq;
        }
      }
    }
    if (rotations == 0) break;
  }
  eval.resize(n);
  for (int i = 0; i < n; ++i) eval[i] = A[(size_t)i * n + i];
}

// Gauss-Legendre nodes and weights by the Golub-Welsch construction: the nodes
// are the eigenvalues of the symmetric tridiagonal Jacobi matrix of the
// Legendre recurrence (off-diagonal j / sqrt(4 j^2 - 1)), the weights twice the
// squared first components of the normalised eigenvectors.
void gauss_legendre(int n, double* x, double* w) {
  std::vector<double> J((size_t)n * n, 0.0);
  for (int j = 1; j < n; ++j) {
    double b = j / std::sqrt(4.0 * j * j - 1.0);
    J[(size_t)(j - 1) * n + j] = J[(size_t)j * n + (j - 1)] = b;
  }
  std::vector<double> V, lam;
  jacobi_eigen(n, J, V, lam);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  for (int i = 0; i < n; ++i) {
    int c = order[i];
    x[i] = lam[c];
    w[i] = 2.0 * V[c] * V[c];  // row 0, column c
  }
  // one Newton polish of every node on P_n for full double accuracy
  for (int i = 0; i < n; ++i) {
    double z = x[i];
    for (int it = 0; it < 2; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 1; j < n; ++j) {
        double p2 = ((2 * j + 1) * z * p1 - j * p0) / (j + 1);
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      if (n == 1) { p1 = z; dp = 1.0; }
      z -= p1 / dp;
      if (it == 1) w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    x[i] = z;
  }
}

// The p+1 B-splines nonzero on span s (functions s-p..s) and their derivatives at
// x, from the Cox-de Boor recursion written on local indices: at degree r the
// live functions are s-r..s; N_r[t] (function i = s-r+t) gathers
//   (x-U_i)/(U_{i+r}-U_i) N_{r-1}[t-1] + (U_{i+r+1}-x)/(U_{i+r+1}-U_{i+1}) N_{r-1}[t],
// with terms of zero denominators dropped (0/0 = 0).
void bspline_span(int p, const double* U, int s, double x, double* val, double* der) {
  double N[kMaxP + 1] = {1.0}, Nm[kMaxP + 1] = {1.0};
  for (int r = 1; r <= p; ++r) {
    for (int t = 0; t < r; ++t) Nm[t] = N[t];
    for (int t = 0; t <= r; ++t) {
      int i = s - r + t;
      double acc = 0.0;
      if (t >= 1) {
        double den = U[i + r] - U[i];
        if (den > 0) acc += (x - U[i]) / den * Nm[t - 1];
      }
      if (t <= r - 1) {
        double den = U[i + r + 1] - U[i + 1];
        if (den > 0) acc += (U[i + r + 1] - x) / den * Nm[t];
      }
      N[t] = acc;
    }
  }
  for (int t = 0; t <= p; ++t) val[t] = N[t];
  if (der) {
    // Nm holds degree p-1 (live functions s-p+1..s)
    for (int t = 0; t <= p; ++t) {
      if (p == 0) { der[t] = 0.0; continue; }
      int i = s - p + t;
      double acc = 0.0;
      if (t >= 1) {
        double den = U[i + p] - U[i];
        if (den > 0) acc += p * Nm[t - 1] / den;
      }
      if (t <= p - 1) {
        double den = U[i + p + 1] - U[i + 1];
        if (den > 0) acc -= p * Nm[t] / den;
      }
      der[t] = acc;
    }
  }
}

bool build_tables(int p, int nknots, const double* U, int nq, Tables1D& t, std::string& err, int lo, int hi) {
  char buf[256];
  int m = nknots - p - 1;
  if (p < 1 || p > kMaxDeg) { snprintf(buf, sizeof buf, "degree %d outside [1, %d]", p, kMaxDeg); err = buf; return false; }
  if (hi < 0) hi = m - 2;
  if (lo == 1 && hi == m - 2 && m < 3) { err = "fewer than 3 basis functions in a direction"; return false; }
  if (lo < 0 || hi > m - 1 || hi < lo) { err = "function box outside 0 .. m-1 or empty"; return false; }
  if (nq < 1 || nq > 16) { err = "nquad outside [1, 16]"; return false; }
  for (int i = 0; i + 1 < nknots; ++i)
    if (!(U[i + 1] >= U[i])) { err = "knot vector not non-decreasing"; return false; }
  for (int i = 1; i <= p; ++i)
    if (U[i] != U[0] || U[nknots - 1 - i] != U[nknots - 1]) { err = "knot vector not open (ends need multiplicity p+1)"; return false; }
  if (U[0] != 0.0 || U[nknots - 1] != 1.0) { err = "knot vector must span [0, 1]"; return false; }
  for (int i = p + 1; i < m; ++i) {
    int mult = 1;
    while (i + mult < m && U[i + mult] == U[i]) ++mult;
    if (mult > p) { err = "interior knot multiplicity above p"; return false; }
  }
  t.p = p; t.m = m; t.n = hi - lo + 1; t.lo = lo; t.nq = nq;
  std::vector<double> gx(nq), gw(nq);
  gauss_legendre(nq, gx.data(), gw.data());
  std::vector<int> spans;
  for (int s = p; s < m; ++s)
    if (U[s + 1] > U[s]) spans.push_back(s);
  t.nel = (int)spans.size();
  t.Q = t.nel * nq;
  const int P = p + 1;
  t.qx.resize(t.Q); t.qw.resize(t.Q); t.qfirst.resize(t.Q);
  t.val.resize((size_t)t.Q * P); t.der.resize((size_t)t.Q * P);
  for (int e = 0; e < t.nel; ++e) {
    int s = spans[e];
    double a = U[s], h = U[s + 1] - U[s];
    for (int g = 0; g < nq; ++g) {
      int q = e * nq + g;
      double x = a + 0.5 * h * (gx[g] + 1.0);
      t.qx[q] = x;
      t.qw[q] = 0.5 * h * gw[g];
      t.qfirst[q] = s - p;
      bspline_span(p, U, s, x, &t.val[(size_t)q * P], &t.der[(size_t)q * P]);
    }
  }
  // the operators' window start: the box index of the point's first function, plus one
  t.qfirst_op.resize(t.Q);
  for (int q = 0; q < t.Q; ++q) t.qfirst_op[q] = t.qfirst[q] - lo + 1;
  // quadrature ranges of the box's functions (qfirst is non-decreasing in q)
  t.flo.assign(t.n, 0); t.fhi.assign(t.n, 0);
  for (int i = 0; i < t.n; ++i) {
    int f = i + lo, qlo = -1, qhi = -1;
    for (int q = 0; q < t.Q; ++q)
      if (t.qfirst[q] <= f && f <= t.qfirst[q] + p) {
        if (qlo < 0) qlo = q;
        qhi = q + 1;
      }
    if (qlo < 0) { err = "interior function without quadrature support"; return false; }
    t.flo[i] = qlo; t.fhi[i] = qhi;
  }
  // parametric mass matrix over the box (one direction of def:matrices_1)
  t.mhat.assign((size_t)t.n * t.n, 0.0);
  for (int q = 0; q < t.Q; ++q)
    for (int a = 0; a < P; ++a) {
      int i = t.qfirst[q] + a - lo;
      if (i < 0 || i >= t.n) continue;
      for (int b = 0; b < P; ++b) {
        int j = t.qfirst[q] + b - lo;
        if (j < 0 || j >= t.n) continue;
        t.mhat[(size_t)i * t.n + j] += t.qw[q] * t.val[(size_t)q * P + a] * t.val[(size_t)q * P + b];
      }
    }
  jacobi_eigen(t.n, t.mhat, t.evec, t.eval);
  for (double l : t.eval)
    if (!(l > 0)) { err = "parametric mass matrix not positive definite"; return false; }
  if (!band_cholesky(t.n, t.p, t.mhat, t.chol, t.cdinv)) {
    err = "band Cholesky of the parametric mass matrix failed";
    return false;
  }
  return true;
}

// Cholesky factor M = L L^T of a symmetric positive definite matrix with half
// bandwidth p (row-major n x n): L[i*(p+1) + d] = L_{i, i-d} (zero where i-d < 0),
// dinv[i] = 1 / L_ii. Column by column: L_jj = sqrt(M_jj - sum_k L_jk^2) and
// L_ij = (M_ij - sum_k L_ik L_jk) / L_jj for j < i <= j + p, the sums over the
// columns k < j inside both bands.
bool band_cholesky(int n, int p, const std::vector<double>& M, std::vector<double>& L, std::vector<double>& dinv) {
  const int w = p + 1;
  L.assign((size_t)n * w, 0.0);
  dinv.assign((size_t)n, 0.0);
  auto at = [&](int i, int j) -> double& { return L[(size_t)i * w + (i - j)]; };  // needs 0 <= i - j <= p
  for (int j = 0; j < n; ++j) {
    double s = M[(size_t)j * n + j];
    for (int k = std::max(0, j - p); k < j; ++k) s -= at(j, k) * at(j, k);
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    at(j, j) = ljj;
    dinv[j] = 1.0 / ljj;
    for (int i = j + 1; i <= std::min(n - 1, j + p); ++i) {
      double t = M[(size_t)i * n + j];
      for (int k = std::max(0, i - p); k < j; ++k) t -= at(i, k) * at(j, k);
      at(i, j) = t / ljj;
    }
  }
  return true;
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..m) and
// off-diagonal b[0..m-1), by bisection on the Sturm count (the number of negative
// pivots of T - x I = L D L^T is the number of eigenvalues below x), starting from
// the Gershgorin interval.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  if (m == 0) return 0.0;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto below = [&](double x) {
    int cnt = 0;
    double q = a[0] - x;
    for (int i = 0;; ++i) {
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
      if (i + 1 >= m) break;
      q = (a[i + 1] - x) - b[i] * b[i] / q;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 4e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) == m) hi = mid;  // every eigenvalue lies below mid
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace iga
