// Gluing of conforming B-spline patches (Sec. 5.1, Assumption ass:conformity,
// def:mp_basis): interfaces, the global numbering G^(r) and the local index boxes of
// the additive Schwarz preconditioner (Sec. 5.4, def:asp). Host code only.
//
// Interfaces are found face against face: two faces of different patches form an
// interface when, under one of the orientations that map a face's index grid onto the
// other's (a permutation of the tangential directions and a reversal of each), their
// control points coincide one by one. Conformity then asks for equal degrees and knots
// along the matched directions, which is checked. Copies of one function on the two
// faces are merged with a union-find over all functions of all patches (functions at
// edges and vertices are merged across several interfaces that way).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "iga_internal.h"

namespace iga {
namespace {

struct PatchInfo {
  int m[3] = {1, 1, 1};
  long long base = 0;  // first function of the patch in the union-find
  const double* ctrl = nullptr;
  const double* knots[3] = {nullptr, nullptr, nullptr};
  int nknots[3] = {0, 0, 0};
  int p[3] = {0, 0, 0};
};

struct Face {
  int r, a, side;
  int t[2] = {0, 0};  // tangential directions, ascending
  int nt = 0;
  double bmin[3], bmax[3];  // bounding box of the face's control points
};

long long flat(const PatchInfo& P, const int* ix, int dim) {
  long long f = 0;
  for (int a = dim - 1; a >= 0; --a) f = f * P.m[a] + ix[a];
  return f;
}

// Full multi-index of the face point (j0, j1) of face F.
void face_index(const Face& F, const PatchInfo& P, int j0, int j1, int* ix) {
  ix[0] = ix[1] = ix[2] = 0;
  ix[F.a] = F.side == 0 ? 0 : P.m[F.a] - 1;
  if (F.nt > 0) ix[F.t[0]] = j0;
  if (F.nt > 1) ix[F.t[1]] = j1;
}

long long root(std::vector<long long>& par, long long x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return x;
}

}  // namespace

int mp_layout(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
              const double* const* ctrl, double tol, int* lo, int* hi, long long* nglob, int* n_adj, long long* gid,
              long long gid_len, std::string& err) {
  if (npatch < 1 || (dim != 2 && dim != 3) || !degree || !nknots || !knots || !ctrl || !lo || !hi || !nglob ||
      !n_adj) {
    err = "iga_mp_layout: npatch >= 1, dim 2 or 3 and non-null arguments required";
    return IGA_EINVAL;
  }
  if (!(tol >= 0.0) || !std::isfinite(tol)) {
    err = "iga_mp_layout: tol must be finite and >= 0";
    return IGA_EINVAL;
  }
  if (tol == 0.0) tol = 1e-10;
  std::vector<PatchInfo> P(npatch);
  long long total = 0;
  double cmax = 1.0;
  for (int r = 0; r < npatch; ++r) {
    long long cnt = 1;
    for (int a = 0; a < dim; ++a) {
      const int p = degree[r * dim + a], nk = nknots[r * dim + a];
      const double* U = knots[r * dim + a];
      if (p < 1 || p > 6 || !U) {
        err = "iga_mp_layout: patch " + std::to_string(r) + ": degree outside 1..6 or null knots";
        return IGA_EINVAL;
      }
      const int m = nk - p - 1;
      if (m < 2) {
        err = "iga_mp_layout: patch " + std::to_string(r) + ": fewer than 2 functions in a direction";
        return IGA_EINVAL;
      }
      for (int i = 0; i + 1 < nk; ++i)
        if (!(U[i] <= U[i + 1])) {
          err = "iga_mp_layout: patch " + std::to_string(r) + ": knots not non-decreasing";
          return IGA_EINVAL;
        }
      for (int i = 0; i <= p; ++i)
        if (U[i] != U[0] || U[nk - 1 - i] != U[nk - 1]) {
          err = "iga_mp_layout: patch " + std::to_string(r) + ": knot vector not open";
          return IGA_EINVAL;
        }
      P[r].m[a] = m;
      P[r].p[a] = p;
      P[r].knots[a] = U;
      P[r].nknots[a] = nk;
      cnt *= m;
    }
    if (!ctrl[r]) {
      err = "iga_mp_layout: null control net";
      return IGA_EINVAL;
    }
    P[r].ctrl = ctrl[r];
    P[r].base = total;
    total += cnt;
    for (long long i = 0; i < cnt * dim; ++i) {
      if (!std::isfinite(ctrl[r][i])) {
        err = "iga_mp_layout: patch " + std::to_string(r) + ": non-finite control point";
        return IGA_EINVAL;
      }
      cmax = std::max(cmax, std::fabs(ctrl[r][i]));
    }
  }
  const double eps = tol * cmax;

  // faces and their bounding boxes
  std::vector<Face> faces;
  for (int r = 0; r < npatch; ++r)
    for (int a = 0; a < dim; ++a)
      for (int side = 0; side < 2; ++side) {
        Face F;
        F.r = r;
        F.a = a;
        F.side = side;
        for (int b = 0; b < dim; ++b)
          if (b != a) F.t[F.nt++] = b;
        for (int c = 0; c < dim; ++c) {
          F.bmin[c] = INFINITY;
          F.bmax[c] = -INFINITY;
        }
        const int n0 = P[r].m[F.t[0]], n1 = F.nt > 1 ? P[r].m[F.t[1]] : 1;
        for (int j1 = 0; j1 < n1; ++j1)
          for (int j0 = 0; j0 < n0; ++j0) {
            int ix[3];
            face_index(F, P[r], j0, j1, ix);
            const double* x = P[r].ctrl + flat(P[r], ix, dim) * dim;
            for (int c = 0; c < dim; ++c) {
              F.bmin[c] = std::min(F.bmin[c], x[c]);
              F.bmax[c] = std::max(F.bmax[c], x[c]);
            }
          }
        faces.push_back(F);
      }

  // match faces: orientation = permutation of the tangential directions and reversals
  const int nf = (int)faces.size();
  std::vector<int> partner(nf, -1);
  std::vector<long long> par(total);
  std::iota(par.begin(), par.end(), 0LL);
  auto close = [&](const double* x, const double* y) {
    for (int c = 0; c < dim; ++c)
      if (std::fabs(x[c] - y[c]) > eps) return false;
    return true;
  };
  const int nt = dim - 1;
  for (int f = 0; f < nf; ++f)
    for (int g = f + 1; g < nf; ++g) {
      const Face &F = faces[f], &G = faces[g];
      if (F.r == G.r) continue;
      bool boxes = true;
      for (int c = 0; c < dim; ++c)
        if (std::fabs(F.bmin[c] - G.bmin[c]) > eps || std::fabs(F.bmax[c] - G.bmax[c]) > eps) boxes = false;
      if (!boxes) continue;
      const PatchInfo &A = P[F.r], &B = P[G.r];
      const int nperm = nt == 2 ? 2 : 1;
      bool matched = false;
      int best_perm = 0, best_flip = 0;
      for (int perm = 0; perm < nperm && !matched; ++perm)
        for (int flip = 0; flip < (1 << nt) && !matched; ++flip) {
          // F's tangential k maps to G's tangential pk[k]
          const int pk[2] = {perm == 0 ? 0 : 1, perm == 0 ? 1 : 0};
          bool sizes = true;
          for (int k = 0; k < nt; ++k)
            if (A.m[F.t[k]] != B.m[G.t[pk[k]]]) sizes = false;
          if (!sizes) continue;
          const int n0 = A.m[F.t[0]], n1 = nt > 1 ? A.m[F.t[1]] : 1;
          bool all = true;
          for (int j1 = 0; j1 < n1 && all; ++j1)
            for (int j0 = 0; j0 < n0 && all; ++j0) {
              const int jf[2] = {j0, j1};
              int jg[2] = {0, 0};
              for (int k = 0; k < nt; ++k) {
                const int nk = A.m[F.t[k]];
                jg[pk[k]] = (flip >> k & 1) ? nk - 1 - jf[k] : jf[k];
              }
              int ia[3], ib[3];
              face_index(F, A, jf[0], jf[1], ia);
              face_index(G, B, jg[0], jg[1], ib);
              if (!close(A.ctrl + flat(A, ia, dim) * dim, B.ctrl + flat(B, ib, dim) * dim)) all = false;
            }
          if (all) {
            matched = true;
            best_perm = perm;
            best_flip = flip;
          }
        }
      if (!matched) {  // the same extent without matching functions: a non-conforming interface
        err = "iga_mp_layout: a face of patch " + std::to_string(F.r) + " and one of patch " + std::to_string(G.r) +
              " cover the same region with different control points (not conforming)";
        return IGA_EINVAL;
      }
      if (partner[f] >= 0 || partner[g] >= 0) {
        err = "iga_mp_layout: a face of patch " + std::to_string(F.r) +
              " or " + std::to_string(G.r) + " coincides with more than one other face (not conforming)";
        return IGA_EINVAL;
      }
      partner[f] = g;
      partner[g] = f;
      // conformity: equal degrees and knots along matched directions (reversed where flipped)
      const int pk[2] = {best_perm == 0 ? 0 : 1, best_perm == 0 ? 1 : 0};
      for (int k = 0; k < nt; ++k) {
        const int da = F.t[k], db = G.t[pk[k]];
        const bool rev = best_flip >> k & 1;
        bool same = A.p[da] == B.p[db] && A.nknots[da] == B.nknots[db];
        const int nk = A.nknots[da];
        for (int i = 0; same && i < nk; ++i) {
          const double ua = A.knots[da][i];
          const double ub = rev ? (B.knots[db][0] + B.knots[db][nk - 1]) - B.knots[db][nk - 1 - i] : B.knots[db][i];
          if (std::fabs(ua - ub) > 1e-12) same = false;
        }
        if (!same) {
          err = "iga_mp_layout: patches " + std::to_string(F.r) + " and " + std::to_string(G.r) +
                " share a face's control points but not its degrees and knots (not conforming)";
          return IGA_EINVAL;
        }
      }
      // merge the copies
      const int n0 = A.m[F.t[0]], n1 = nt > 1 ? A.m[F.t[1]] : 1;
      for (int j1 = 0; j1 < n1; ++j1)
        for (int j0 = 0; j0 < n0; ++j0) {
          const int jf[2] = {j0, j1};
          int jg[2] = {0, 0};
          for (int k = 0; k < nt; ++k) jg[pk[k]] = (best_flip >> k & 1) ? A.m[F.t[k]] - 1 - jf[k] : jf[k];
          int ia[3], ib[3];
          face_index(F, A, jf[0], jf[1], ia);
          face_index(G, B, jg[0], jg[1], ib);
          const long long x = root(par, A.base + flat(A, ia, dim)), y = root(par, B.base + flat(B, ib, dim));
          if (x != y) par[std::max(x, y)] = std::min(x, y);
        }
    }

  // a class is Dirichlet when one of its copies lies on a face that is not an interface
  std::vector<char> outer(total, 0);
  std::vector<int> copies(total, 0);
  for (int r = 0; r < npatch; ++r) {
    const PatchInfo& A = P[r];
    const long long cnt = (long long)A.m[0] * A.m[1] * (dim == 3 ? A.m[2] : 1);
    for (long long f = 0; f < cnt; ++f) {
      int ix[3] = {(int)(f % A.m[0]), (int)((f / A.m[0]) % A.m[1]), dim == 3 ? (int)(f / ((long long)A.m[0] * A.m[1])) : 0};
      bool on_outer = false;
      for (int a = 0; a < dim; ++a) {
        const int fid = (r * dim + a) * 2;
        if (ix[a] == 0 && partner[fid] < 0) on_outer = true;
        if (ix[a] == A.m[a] - 1 && partner[fid + 1] < 0) on_outer = true;
      }
      const long long c = root(par, A.base + f);
      if (on_outer) outer[c] = 1;
      copies[c] += 1;
    }
  }

  // index boxes, then the numbering walk (patches in order, boxes direction 0 fastest)
  long long need = 0;
  for (int r = 0; r < npatch; ++r) {
    long long cnt = 1;
    for (int a = 0; a < dim; ++a) {
      const int fid = (r * dim + a) * 2;
      lo[r * dim + a] = partner[fid] >= 0 ? 0 : 1;
      hi[r * dim + a] = partner[fid + 1] >= 0 ? P[r].m[a] - 1 : P[r].m[a] - 2;
      cnt *= std::max(0, hi[r * dim + a] - lo[r * dim + a] + 1);
    }
    need += cnt;
  }
  std::vector<long long> id(total, -1);
  long long next = 0;
  int nadj = 0;
  long long w = 0;
  if (gid && gid_len != need) {
    err = "iga_mp_layout: gid_len is " + std::to_string(gid_len) + ", the boxes hold " + std::to_string(need);
    return IGA_EINVAL;
  }
  for (int r = 0; r < npatch; ++r) {
    const int* l = lo + r * dim;
    const int* u = hi + r * dim;
    const int e2 = dim == 3 ? u[2] : 0, s2 = dim == 3 ? l[2] : 0;
    for (int i2 = s2; i2 <= e2; ++i2)
      for (int i1 = l[1]; i1 <= u[1]; ++i1)
        for (int i0 = l[0]; i0 <= u[0]; ++i0) {
          const int ix[3] = {i0, i1, i2};
          const long long c = root(par, P[r].base + flat(P[r], ix, dim));
          long long g = -1;
          if (!outer[c]) {
            if (id[c] < 0) {
              id[c] = next++;
              nadj = std::max(nadj, copies[c]);
            }
            g = id[c];
          }
          if (gid) gid[w] = g;
          ++w;
        }
  }
  *nglob = next;
  *n_adj = nadj;
  return IGA_OK;
}

}  // namespace iga
