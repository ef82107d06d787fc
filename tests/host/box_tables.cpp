// Test driver: prints the library's univariate tables (host_setup.cpp) for one knot
// vector and function box, for tests/test_host_tables.py.
// usage: box_tables p lo hi nq U_0 ... U_{nk-1}   (hi < 0: the interior box)
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "iga_internal.h"

int main(int argc, char** argv) {
  if (argc < 6) return 2;
  const int p = atoi(argv[1]), lo = atoi(argv[2]), hi = atoi(argv[3]), nq = atoi(argv[4]), nk = argc - 5;
  std::vector<double> U(nk);
  for (int i = 0; i < nk; ++i) U[i] = strtod(argv[5 + i], nullptr);
  iga::Tables1D t;
  std::string err;
  if (!iga::build_tables(p, nk, U.data(), nq, t, err, lo, hi)) {
    printf("ERR %s\n", err.c_str());
    return 1;
  }
  printf("%d %d %d %d\n", t.n, t.Q, t.m, t.lo);
  for (double v : t.mhat) printf("%.17g\n", v);
  for (int i = 0; i < t.n; ++i) printf("%d %d\n", t.flo[i], t.fhi[i]);
  for (int q = 0; q < t.Q; ++q) printf("%d %d\n", t.qfirst[q], t.qfirst_op[q]);
  return 0;
}
