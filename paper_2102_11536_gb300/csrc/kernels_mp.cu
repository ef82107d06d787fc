// Gather and scatter between global vectors and the patches' local vectors of a
// multi-patch system (Sec. 5.4: R^(r) and R^(r)T of def:asp, and the global M, K as
// sums of the patches' matrices through G^(r), Sec. 5.1).
#include "iga_internal.h"

namespace iga {
namespace {

// xl (patch r's block at nvec * off[r], vector v at + v * nr[r]) = x at the box entries'
// global functions; entries with no global function (a copy on the Dirichlet boundary)
// get zero, so a patch operator over the whole box acts on the local functions only.
__global__ void k_mp_gather(MpMaps m, int nvec, const int* __restrict__ active, const double* __restrict__ x,
                            double* __restrict__ xl) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.nloc) return;
  const int r = m.epatch[e];
  const long long g = m.gid[e];
  xl[nvec * m.off[r] + v * m.nr[r] + (e - m.off[r])] = g >= 0 ? x[v * m.nglob + g] : 0.0;
}

// y_g = sum of the local results at the entries of global function g, in ascending
// entry order (patch order): deterministic.
__global__ void k_mp_scatter(MpMaps m, int nvec, const int* __restrict__ active, const double* __restrict__ yl,
                             double* __restrict__ y) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m.nglob) return;
  double acc = 0.0;
  for (long long j = m.crow[g]; j < m.crow[g + 1]; ++j) {
    const long long e = m.cent[j];
    const int r = m.epatch[e];
    acc += yl[nvec * m.off[r] + v * m.nr[r] + (e - m.off[r])];
  }
  y[v * m.nglob + g] = acc;
}

// One patch's box <-> the global vector: entries off .. off + nr - 1 of the maps. A patch
// holds at most one copy of each global function, so the scatter-add has no conflicts.
__global__ void k_mp_patch_io(MpMaps m, long long off, long long nr, int nvec, int add, const double* __restrict__ in,
                              double* __restrict__ out) {
  const int v = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  const long long g = m.gid[off + i];
  if (add) {  // in: the box, out: the global vector
    if (g >= 0) out[v * m.nglob + g] += in[v * nr + i];
  } else {    // in: the global vector, out: the box
    out[v * nr + i] = g >= 0 ? in[v * m.nglob + g] : 0.0;
  }
}

}  // namespace

cudaError_t launch_mp_patch_io(cudaStream_t s, const MpMaps& m, long long off, long long nr, int nvec, int add,
                               const double* in, double* out) {
  if (nr <= 0 || nvec <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((nr + 255) / 256), (unsigned)nvec);
  k_mp_patch_io<<<grid, 256, 0, s>>>(m, off, nr, nvec, add, in, out);
  return cudaGetLastError();
}

cudaError_t launch_mp_gather(cudaStream_t s, const MpMaps& m, int nvec, const int* active, const double* x,
                             double* xl) {
  if (m.nloc <= 0 || nvec <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((m.nloc + 255) / 256), (unsigned)nvec);
  k_mp_gather<<<grid, 256, 0, s>>>(m, nvec, active, x, xl);
  return cudaGetLastError();
}

cudaError_t launch_mp_scatter(cudaStream_t s, const MpMaps& m, int nvec, const int* active, const double* yl,
                              double* y) {
  if (m.nglob <= 0 || nvec <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((m.nglob + 255) / 256), (unsigned)nvec);
  k_mp_scatter<<<grid, 256, 0, s>>>(m, nvec, active, yl, y);
  return cudaGetLastError();
}

}  // namespace iga
