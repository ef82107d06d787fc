// Operators of a handle (Sec. 5.2-5.3): K and M matrix-free at the Gauss points (sum
// factorisation) or as assembled bands (FP64 or double-FP32), the preconditioner (fast
// diagonalisation in FP64, FP32 or on the tensor cores, or the band-Cholesky Kronecker
// solve), and the multi-patch system's gather / per-patch operator / scatter-add.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "handle.h"

namespace iga {

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
// Algorithmic work of the last-axis kernels per vector (FMA = 2 flops):
// mass: interpolate (p+1 FMA), scale by W (1 mul), integrate (p+1 FMA) per point;
// stiffness: 3 interpolations, the symmetric 3x3 product (9 mul + 6 add), 3 integrations.
double mass_last_flops(const iga_handle* h) { return (4.0 * h->dd[h->dim - 1].P + 1.0) * (double)h->Qt; }
double stiff_last_flops(const iga_handle* h) {
  const double P = h->dd[h->dim - 1].P;
  return h->dim == 3 ? (12.0 * P + 15.0) * (double)h->Qt : (8.0 * P + 6.0) * (double)h->Qt;
}
// whole mass application: banded passes of every axis, forward and transposed
double mass_apply_flops(const iga_handle* h) {
  const int *n = h->n, *Q = h->Q;
  double f = mass_last_flops(h);
  if (h->dim == 3) {
    f += 2 * 2.0 * h->dd[0].P * (double)Q[0] * n[1] * n[2];
    f += 2 * 2.0 * h->dd[1].P * (double)Q[0] * Q[1] * n[2];
  } else {
    f += 2 * 2.0 * h->dd[0].P * (double)Q[0] * n[1];
  }
  return f;
}

int apply_M_mf(iga_handle* h, int nvec, const int* active, const double* x, double* y) {
  CKS(ensure_op_ws(h, nvec));
  cudaStream_t s = h->stream;
  const int *n = h->n, *Q = h->Q;
  const DirDev* d = h->dd;
  const int nact = active ? h->cur_active : nvec;
  cudaEvent_t ea = nullptr, em = nullptr;
  CKS(prof_begin(h, IGA_PROF_MASS_APPLY, &ea));
  if (h->dim == 3) {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], (long long)n[1] * n[2]}, nvec, active, x, h->N, d[0].val, h->u0, nullptr, nullptr, h->su));
    LK(launch_fwd(s, d[1], {Q[0], n[1], Q[1], n[2]}, nvec, active, h->u0, h->su, d[1].val, h->ta, nullptr, nullptr, h->st));
    CKS(prof_begin(h, IGA_PROF_MASS, &em));
    LK(launch_mid_mass(s, d[2], (long long)Q[0] * Q[1], nvec, active, h->W, h->ta, h->ta, h->st));
    CKS(prof_end(h, em, nact * mass_last_flops(h), 8.0 * (h->Qt + 2.0 * nact * h->st)));
    LK(launch_tr(s, d[1], {Q[0], Q[1], n[1], n[2]}, nvec, active, h->ta, d[1].val, nullptr, nullptr, h->st, h->u0, h->su));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], (long long)n[1] * n[2]}, nvec, active, h->u0, d[0].val, nullptr, nullptr, h->su, y, h->N));
  } else {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], n[1]}, nvec, active, x, h->N, d[0].val, h->u0, nullptr, nullptr, h->su));
    CKS(prof_begin(h, IGA_PROF_MASS, &em));
    LK(launch_mid_mass(s, d[1], Q[0], nvec, active, h->W, h->u0, h->u0, h->su));
    CKS(prof_end(h, em, nact * mass_last_flops(h), 8.0 * (h->Qt + 2.0 * nact * h->su)));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], n[1]}, nvec, active, h->u0, d[0].val, nullptr, nullptr, h->su, y, h->N));
  }
  CKS(prof_end(h, ea, nact * mass_apply_flops(h), 8.0 * (h->Qt + 2.0 * nact * h->N)));
  return IGA_OK;
}

int apply_K_mf(iga_handle* h, int nvec, const int* active, const double* x, double* y) {
  CKS(ensure_op_ws(h, nvec));
  cudaStream_t s = h->stream;
  const int *n = h->n, *Q = h->Q;
  const DirDev* d = h->dd;
  const int nact = active ? h->cur_active : nvec;
  cudaEvent_t ek = nullptr;
  if (h->dim == 3) {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], (long long)n[1] * n[2]}, nvec, active, x, h->N, d[0].val, h->u0, d[0].der, h->u1, h->su));
    LK(launch_fwd(s, d[1], {Q[0], n[1], Q[1], n[2]}, nvec, active, h->u0, h->su, d[1].val, h->ta, d[1].der, h->tb, h->st));
    LK(launch_fwd(s, d[1], {Q[0], n[1], Q[1], n[2]}, nvec, active, h->u1, h->su, d[1].val, h->tc, nullptr, nullptr, h->st));
    CKS(prof_begin(h, IGA_PROF_STIFF, &ek));
    LK(launch_mid_stiff3(s, d[2], (long long)Q[0] * Q[1], nvec, active, h->G, h->gstride, h->ta, h->tb, h->tc, h->st));
    CKS(prof_end(h, ek, nact * stiff_last_flops(h), 8.0 * (6.0 * h->Qt + 6.0 * nact * h->st)));
    LK(launch_tr(s, d[1], {Q[0], Q[1], n[1], n[2]}, nvec, active, h->ta, d[1].val, h->tb, d[1].der, h->st, h->u0, h->su));
    LK(launch_tr(s, d[1], {Q[0], Q[1], n[1], n[2]}, nvec, active, h->tc, d[1].val, nullptr, nullptr, h->st, h->u1, h->su));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], (long long)n[1] * n[2]}, nvec, active, h->u0, d[0].val, h->u1, d[0].der, h->su, y, h->N));
  } else {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], n[1]}, nvec, active, x, h->N, d[0].val, h->u0, d[0].der, h->u1, h->su));
    CKS(prof_begin(h, IGA_PROF_STIFF, &ek));
    LK(launch_mid_stiff2(s, d[1], Q[0], nvec, active, h->G, h->gstride, h->u0, h->u1, h->su));
    CKS(prof_end(h, ek, nact * stiff_last_flops(h), 8.0 * (3.0 * h->Qt + 4.0 * nact * h->su)));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], n[1]}, nvec, active, h->u0, d[0].val, h->u1, d[0].der, h->su, y, h->N));
  }
  return IGA_OK;
}

// The preconditioner of Sec. 5.3 by fast diagonalisation with scratch t1, t2
// (nvec*N doubles each): t = S r (S = D^{-1/2} Dhat^{1/2}), then U^T along each
// axis, division by Lambda_0(i0) Lambda_1(i1) Lambda_2(i2), U along each axis, S.
// FP64 form: all in FP64. FP32 form: the scaled residual is rounded to FP32,
// mode products and Lambda in FP32, final rescale in FP64.
// rzp (nullable): with the band-Cholesky forms, per-block partials of r.z and r.z_old
// (z's previous content) come out of the last axis, [2][nvec][*nrz]; *nrz = 0 otherwise.
int fd_apply(iga_handle* h, int nvec, const int* active, const double* r, double* z, double* t1, double* t2,
             double* rzp, int* nrz) {
  if (nrz) *nrz = 0;
  cudaStream_t s = h->stream;
  const int* n = h->n;
  const DirDev* d = h->dd;
  const long long N = h->N;
  const long long n01 = (long long)n[0] * n[1];
  const long long n12 = (long long)n[1] * n[2];
  const bool d3 = h->dim == 3;
  if (h->opt.precond == IGA_PREC_FP64) {
    FdEpilogue none{}, lam{}, post{};
    lam.lam[0] = d[0].lam64;
    lam.lam[1] = d[1].lam64;
    lam.lam[2] = d3 ? d[2].lam64 : nullptr;
    lam.n[0] = n[0]; lam.n[1] = n[1]; lam.n[2] = n[2];
    post.post = h->scale;
    const double* sc = h->scale;
    if (d3) {
      LK(launch_fd_mode64(s, n[0], {1, n[0], n[0], n12}, nvec, active, d[0].U64, 1, r, t1, N, sc, none));
      LK(launch_fd_mode64(s, n[1], {n[0], n[1], n[1], n[2]}, nvec, active, d[1].U64, 1, t1, t2, N, nullptr, none));
      LK(launch_fd_mode64(s, n[2], {n01, n[2], n[2], 1}, nvec, active, d[2].U64, 1, t2, t1, N, nullptr, lam));
      LK(launch_fd_mode64(s, n[2], {n01, n[2], n[2], 1}, nvec, active, d[2].U64, 0, t1, t2, N, nullptr, none));
      LK(launch_fd_mode64(s, n[1], {n[0], n[1], n[1], n[2]}, nvec, active, d[1].U64, 0, t2, t1, N, nullptr, none));
      LK(launch_fd_mode64(s, n[0], {1, n[0], n[0], n12}, nvec, active, d[0].U64, 0, t1, z, N, nullptr, post));
    } else {
      LK(launch_fd_mode64(s, n[0], {1, n[0], n[0], n[1]}, nvec, active, d[0].U64, 1, r, t1, N, sc, none));
      LK(launch_fd_mode64(s, n[1], {n[0], n[1], n[1], 1}, nvec, active, d[1].U64, 1, t1, t2, N, nullptr, lam));
      LK(launch_fd_mode64(s, n[1], {n[0], n[1], n[1], 1}, nvec, active, d[1].U64, 0, t2, t1, N, nullptr, none));
      LK(launch_fd_mode64(s, n[0], {1, n[0], n[0], n[1]}, nvec, active, d[0].U64, 0, t1, z, N, nullptr, post));
    }
    return IGA_OK;
  }
  if (h->opt.precond == IGA_PREC_BANDED || h->opt.precond == IGA_PREC_BANDED32) {
    // (Mhat_1 x Mhat_2 x Mhat_3)^{-1} by band Cholesky along each axis, FP64 or FP32
    // (FP32 intermediates between the axes)
    const int f32 = h->opt.precond == IGA_PREC_BANDED32;
    const void* L[3] = {f32 ? (const void*)d[0].chol32 : d[0].chol, f32 ? (const void*)d[1].chol32 : d[1].chol,
                        f32 ? (const void*)d[2].chol32 : d[2].chol};
    const void* Di[3] = {f32 ? (const void*)d[0].cdinv32 : d[0].cdinv, f32 ? (const void*)d[1].cdinv32 : d[1].cdinv,
                         f32 ? (const void*)d[2].cdinv32 : d[2].cdinv};
    const int mid = f32 ? 0 : 1;  // intermediates are FP64 only in the FP64 form
    const double* sc = h->scale;
    const float* s32 = f32 ? h->scale32 : nullptr;  // the FP32 form scales in FP32
    if (d3) {
      LK(launch_kron_axis(s, n[0], d[0].p, {1, n[0], n[0], n12}, nvec, active, f32, L[0], Di[0], r, 1, t1, mid, N, sc, nullptr, nullptr, nullptr, nullptr, s32));
      LK(launch_kron_axis(s, n[1], d[1].p, {n[0], n[1], n[1], n[2]}, nvec, active, f32, L[1], Di[1], t1, mid, t2, mid, N, nullptr, nullptr));
      LK(launch_kron_axis(s, n[2], d[2].p, {n01, n[2], n[2], 1}, nvec, active, f32, L[2], Di[2], t2, mid, z, 1, N, nullptr, sc, rzp ? r : nullptr, rzp, nrz, s32));
    } else {
      LK(launch_kron_axis(s, n[0], d[0].p, {1, n[0], n[0], n[1]}, nvec, active, f32, L[0], Di[0], r, 1, t1, mid, N, sc, nullptr, nullptr, nullptr, nullptr, s32));
      LK(launch_kron_axis(s, n[1], d[1].p, {n[0], n[1], n[1], 1}, nvec, active, f32, L[1], Di[1], t1, mid, z, 1, N, nullptr, sc, rzp ? r : nullptr, rzp, nrz, s32));
    }
    return IGA_OK;
  }
  if (h->opt.precond == IGA_PREC_FP32) {
    float* f1 = reinterpret_cast<float*>(t1);
    float* f2 = reinterpret_cast<float*>(t2);
    const float* lam[3] = {d[0].lam32, d[1].lam32, d3 ? d[2].lam32 : nullptr};
    const double* sc = h->scale;
    if (d3) {
      LK(launch_fd_mode32(s, n[0], {1, n[0], n[0], n12}, nvec, active, d[0].U32, 1, r, 1, f1, 0, N, sc, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[1], {n[0], n[1], n[1], n[2]}, nvec, active, d[1].U32, 1, f1, 0, f2, 0, N, nullptr, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[2], {n01, n[2], n[2], 1}, nvec, active, d[2].U32, 1, f2, 0, f1, 0, N, nullptr, nullptr, lam, n));
      LK(launch_fd_mode32(s, n[2], {n01, n[2], n[2], 1}, nvec, active, d[2].U32, 0, f1, 0, f2, 0, N, nullptr, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[1], {n[0], n[1], n[1], n[2]}, nvec, active, d[1].U32, 0, f2, 0, f1, 0, N, nullptr, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[0], {1, n[0], n[0], n12}, nvec, active, d[0].U32, 0, f1, 0, z, 1, N, nullptr, sc, nullptr, n));
    } else {
      LK(launch_fd_mode32(s, n[0], {1, n[0], n[0], n[1]}, nvec, active, d[0].U32, 1, r, 1, f1, 0, N, sc, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[1], {n[0], n[1], n[1], 1}, nvec, active, d[1].U32, 1, f1, 0, f2, 0, N, nullptr, nullptr, lam, n));
      LK(launch_fd_mode32(s, n[1], {n[0], n[1], n[1], 1}, nvec, active, d[1].U32, 0, f2, 0, f1, 0, N, nullptr, nullptr, nullptr, n));
      LK(launch_fd_mode32(s, n[0], {1, n[0], n[0], n[1]}, nvec, active, d[0].U32, 0, f1, 0, z, 1, N, nullptr, sc, nullptr, n));
    }
    return IGA_OK;
  }
  if (h->opt.precond == IGA_PREC_BF16 || h->opt.precond == IGA_PREC_FP16) {
    // the same sequence on the tensor cores: 16-bit operands, FP32 accumulation and intermediates
    const int f16 = h->opt.precond == IGA_PREC_FP16;
    for (int a = 0; a < h->dim; ++a)
      if (!d[a].Btc[0])
        return fail(h, IGA_EINVAL, "tensor-core preconditioner needs at most 256 interior functions per direction");
    void* const* B[3] = {f16 ? d[0].Btc16 : d[0].Btc, f16 ? d[1].Btc16 : d[1].Btc,
                         f16 ? d[2].Btc16 : d[2].Btc};
    float* f1 = reinterpret_cast<float*>(t1);
    float* f2 = reinterpret_cast<float*>(t2);
    const float* lam[3] = {d[0].lam32, d[1].lam32, d3 ? d[2].lam32 : nullptr};
    const double* sc = h->scale;
    int* err = h->dflag + 1;
    if (d3) {
      LK(launch_fd_mode_tc(s, n[0], 0, {1, n[0], n[0], n12}, nvec, active, B[0][1], f16, r, 1, f1, 0, N, sc, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[1], 1, {n[0], n[1], n[1], n[2]}, nvec, active, B[1][1], f16, f1, 0, f2, 0, N, nullptr, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[2], 2, {n01, n[2], n[2], 1}, nvec, active, B[2][1], f16, f2, 0, f1, 0, N, nullptr, nullptr, lam, n, err));
      LK(launch_fd_mode_tc(s, n[2], 2, {n01, n[2], n[2], 1}, nvec, active, B[2][0], f16, f1, 0, f2, 0, N, nullptr, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[1], 1, {n[0], n[1], n[1], n[2]}, nvec, active, B[1][0], f16, f2, 0, f1, 0, N, nullptr, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[0], 0, {1, n[0], n[0], n12}, nvec, active, B[0][0], f16, f1, 0, z, 1, N, nullptr, sc, nullptr, n, err));
    } else {
      LK(launch_fd_mode_tc(s, n[0], 0, {1, n[0], n[0], n[1]}, nvec, active, B[0][1], f16, r, 1, f1, 0, N, sc, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[1], 1, {n[0], n[1], n[1], 1}, nvec, active, B[1][1], f16, f1, 0, f2, 0, N, nullptr, nullptr, lam, n, err));
      LK(launch_fd_mode_tc(s, n[1], 1, {n[0], n[1], n[1], 1}, nvec, active, B[1][0], f16, f2, 0, f1, 0, N, nullptr, nullptr, nullptr, n, err));
      LK(launch_fd_mode_tc(s, n[0], 0, {1, n[0], n[0], n[1]}, nvec, active, B[0][0], f16, f1, 0, z, 1, N, nullptr, sc, nullptr, n, err));
    }
    return IGA_OK;
  }
  return fail(h, IGA_EINVAL, "preconditioner arithmetic not available in this build");
}

// The tensor-core kernels set dflag[1], the TMA-staged band product and the cooperative
// split dflag[2], when an mbarrier or grid-barrier wait runs out.
int check_tc_error(iga_handle* h) {
  if (h->mp) {
    for (size_t r = 0; r < h->mp->patch.size(); ++r) {
      iga_handle* p = h->mp->patch[r];
      p->stream = h->stream;
      const int rc = check_tc_error(p);
      if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
    }
    return IGA_OK;
  }
  const bool tc = h->opt.precond == IGA_PREC_BF16 || h->opt.precond == IGA_PREC_FP16;
  const bool df = h->opt.op_form == IGA_OP_ASSEMBLED_DF;
  if (!tc && !df) return IGA_OK;
  int e[2] = {0, 0};
  CK(cudaMemcpyAsync(e, h->dflag + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e[0] || e[1]) {
    CK(cudaMemsetAsync(h->dflag + 1, 0, 2 * sizeof(int), h->stream));
    // a grid barrier that ran out may have left its arrival count behind: start afresh
    if (e[1] && h->df_bar) CK(cudaMemsetAsync(h->df_bar, 0, 2 * sizeof(unsigned int), h->stream));
    return fail(h, IGA_ECUDA, e[0] ? "tensor-core mode product: mbarrier wait timed out"
                                   : "double-FP32 band product or split: a bounded wait (mbarrier or grid "
                                     "barrier) timed out");
  }
  return IGA_OK;
}

// Assembled band rows of M and K by probing the matrix-free operators with the
// (2p+1)^d colour vectors, 8 colours per application (kernels_band.cu).
int assemble_band64(iga_handle* h) {
  if (h->band_ready) return IGA_OK;
  drop_step_graph(h);  // new addresses
  cudaStream_t s = h->stream;
  int p3[3] = {0, 0, 0};
  for (int a = 0; a < h->dim; ++a) p3[a] = h->dd[a].p;
  int S = 1;
  for (int a = 0; a < 3; ++a) S *= 2 * p3[a] + 1;
  const int centre = S / 2, H = S - centre;
  std::vector<long long> off(H);
  std::vector<int> o12(H);
  for (int hh = 0; hh < H; ++hh) {
    const int sl = centre + hh;
    const int m0 = 2 * p3[0] + 1, m1 = 2 * p3[1] + 1;
    const int o0 = sl % m0 - p3[0], o1 = (sl / m0) % m1 - p3[1], o2 = sl / (m0 * m1) - p3[2];
    off[hh] = o0 + (long long)h->n[0] * (o1 + (long long)h->n[1] * o2);
    o12[hh] = (o1 + 64) | ((o2 + 64) << 8);
  }
  CKS(upload(h, &h->band_o12, o12));
  double nnz = 1.0;
  for (int a = 0; a < 3; ++a) nnz *= (double)h->n[a] * (2 * p3[a] + 1) - (double)p3[a] * (p3[a] + 1);
  CKS(upload(h, &h->band_off, off));
  CKS(dalloc(h, &h->Mband, (size_t)H * h->N));
  CKS(dalloc(h, &h->Kband, (size_t)H * h->N));
  CK(cudaMemsetAsync(h->Mband, 0, sizeof(double) * H * h->N, s));
  CK(cudaMemsetAsync(h->Kband, 0, sizeof(double) * H * h->N, s));
  // Probe vectors in buffers of their own: the assembly may run lazily inside an
  // operator call whose caller holds pointers into the PCG workspace, so it must
  // not resize that workspace.
  constexpr int kBatch = 8;
  struct ProbeBufs {
    double* x = nullptr;
    double* y = nullptr;
    ~ProbeBufs() {
      if (x) cudaFree(x);
      if (y) cudaFree(y);
    }
  } pb;
  CKS(dalloc(h, &pb.x, (size_t)kBatch * h->N));
  CKS(dalloc(h, &pb.y, (size_t)kBatch * h->N));
  for (int first = 0; first < S; first += kBatch) {
    const int nv = std::min(kBatch, S - first);
    LK(launch_probe_gen(s, h->N, h->n, p3, first, S, nv, pb.x, h->N));
    CKS(apply_M_mf(h, nv, nullptr, pb.x, pb.y));
    LK(launch_probe_extract(s, h->N, h->n, p3, first, S, nv, pb.y, h->N, h->Mband));
    CKS(apply_K_mf(h, nv, nullptr, pb.x, pb.y));
    LK(launch_probe_extract(s, h->N, h->n, p3, first, S, nv, pb.y, h->N, h->Kband));
  }
  CK(cudaStreamSynchronize(s));
  h->band_H = H;
  h->band_nnz = nnz;
  h->band_ready = true;
  return IGA_OK;
}

// The double-FP32 copies of the assembled band (kernels_banddf.cu): split once from
// the FP64 band, which is then released.
int assemble_band_df(iga_handle* h) {
  if (h->df_ready) return IGA_OK;
  CKS(assemble_band64(h));
  drop_step_graph(h);
  cudaStream_t s = h->stream;
  const int H = h->band_H;
  const long long N = h->N, Np = df_row_stride(N);
  int p3[3] = {0, 0, 0};
  for (int a = 0; a < h->dim; ++a) p3[a] = h->dd[a].p;
  const std::vector<int> runs = band_df_runs(h->n, p3, nullptr);  // the geometry of the runs
  h->band_nruns = (int)runs.size() / 4;
  long long maxL = 0;  // reach of a run's staged copies beyond its rows
  for (size_t q = 0; q < runs.size(); q += 4) maxL = std::max(maxL, (long long)std::abs(runs[q + 3]) + runs[q + 1]);
  const long long sl = df_slack(maxL);
  h->df_slack = sl;
  const size_t nA = (size_t)H * Np + 2 * sl, nX = (size_t)kMaxVec * Np + 2 * sl;
  CKS(dalloc(h, &h->Mdf, nA));
  CKS(dalloc(h, &h->Kdf, nA));
  CKS(dalloc(h, &h->df_xs, nX));
  CKS(dalloc(h, &h->df_E, (size_t)2 * kMaxVec));
  CKS(dalloc(h, &h->df_part, (size_t)kMaxVec * kDfBlocks));
  CKS(dalloc(h, &h->df_bar, 2));
  CK(cudaMemsetAsync(h->df_bar, 0, 2 * sizeof(unsigned int), s));
  CK(cudaMemsetAsync(h->Mdf, 0, sizeof(float2) * nA, s));
  CK(cudaMemsetAsync(h->Kdf, 0, sizeof(float2) * nA, s));
  CK(cudaMemsetAsync(h->df_xs, 0, sizeof(float2) * nX, s));
  int* dE = h->df_E + kMaxVec;
  int EA[2] = {0, 0};
  LK(launch_df_split_matrix(s, N, H, h->Mband, h->Mdf + sl, Np, h->df_part, dE));
  CK(cudaMemcpyAsync(&EA[0], dE, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  LK(launch_df_split_matrix(s, N, H, h->Kband, h->Kdf + sl, Np, h->df_part, dE));
  CK(cudaMemcpyAsync(&EA[1], dE, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->EAm = EA[0];
  h->EAk = EA[1];
  h->band_Np = Np;
  // each matrix's tiny slots (every coefficient below 2^-24 after the scaling, which puts the
  // largest in [1, 2)): their terms take one FP32 multiply-add (band_df_runs)
  {
    struct Tmp {
      unsigned* p = nullptr;
      ~Tmp() {
        if (p) cudaFree(p);
      }
    } smax;
    CKS(dalloc(h, &smax.p, (size_t)2 * H));
    LK(launch_df_slot_absmax(s, N, H, h->Mdf + sl, Np, smax.p));
    LK(launch_df_slot_absmax(s, N, H, h->Kdf + sl, Np, smax.p + H));
    std::vector<unsigned> hmax((size_t)2 * H);
    CK(cudaMemcpyAsync(hmax.data(), smax.p, sizeof(unsigned) * 2 * H, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    constexpr unsigned kTinyBits = 0x33800000u;  // 2^-24 as FP32 bits
    std::vector<unsigned char> tiny((size_t)2 * H);
    for (size_t q = 0; q < tiny.size(); ++q) tiny[q] = hmax[q] < kTinyBits;
    const std::vector<int> rm = band_df_runs(h->n, p3, tiny.data()), rk = band_df_runs(h->n, p3, tiny.data() + H);
    CKS(upload(h, &h->band_runs, rm));
    CKS(upload(h, &h->band_runs_k, rk));
    // the share of an interior row's terms that are tiny: per run 2 min(2 m, len) of 2 len
    auto share = [](const std::vector<int>& r) {
      long long all = 1, cheap = 0;
      for (size_t q = 0; q < r.size(); q += 4) {
        const int len = r[q + 1], m = (r[q + 2] >> 16) & 15;
        all += 2LL * len;
        cheap += 2LL * std::min(2 * m, len);
      }
      return (double)cheap / (double)all;
    };
    h->df_tiny_m = share(rm);
    h->df_tiny_k = share(rk);
  }
  df_encode_maps(h->Mdf + sl, H, h->df_xs + sl, kMaxVec, Np, p3[0], &h->tmM);
  df_encode_maps(h->Kdf + sl, H, h->df_xs + sl, kMaxVec, Np, p3[0], &h->tmK);
  dfree(h->Mband);
  dfree(h->Kband);
  h->band_ready = false;
  h->df_ready = true;
  return IGA_OK;
}

// the band rows of the handle's assembled form
int assemble_band(iga_handle* h) {
  return h->opt.op_form == IGA_OP_ASSEMBLED_DF ? assemble_band_df(h) : assemble_band64(h);
}

// one band product y = A x in the handle's assembled form (FP64, or double-FP32 with
// the split of x first -- unless presplit: the split copy already holds x, as the PCG
// direction's producers leave it); cls selects the matrix (IGA_PROF_BAND_MASS / _STIFF)
cudaError_t launch_band(iga_handle* h, cudaStream_t s, int cls, int nvec, const int* active, const double* x,
                        double* y, int threads, int nv, double* pq, int* npq, bool presplit) {
  const bool mass = cls == IGA_PROF_BAND_MASS;
  if (h->opt.op_form == IGA_OP_ASSEMBLED_DF) {
    float2* xs = h->df_xs + h->df_slack;
    if (!presplit) {
      const cudaError_t e = launch_df_split(s, h->N, active, nvec, x, h->N, xs, h->band_Np, h->df_E, h->df_part,
                                            h->df_bar, h->dflag + 2, h->bar_limit);
      if (e != cudaSuccess) return e;
    }
    return launch_band_df(s, h->N, h->band_nruns, reinterpret_cast<const int4*>(mass ? h->band_runs : h->band_runs_k),
                          h->n, h->dd[0].p,
                          h->dim == 3 ? h->dd[2].p : 0, h->band_H, (mass ? h->Mdf : h->Kdf) + h->df_slack, h->band_Np, mass ? h->EAm : h->EAk, active, nvec,
                          xs, h->df_E, x, y, h->N, threads, nv, pq, npq, h->dflag + 2, mass ? &h->tmM : &h->tmK);
  }
  return launch_band_spmv(s, h->N, h->band_H, h->band_off, h->band_o12, h->n, mass ? h->Mband : h->Kband, active,
                          nvec, x, y, h->N, threads, nv, pq, npq);
}

int apply_band(iga_handle* h, int cls, int nvec, const int* active, const double* x, double* y,
               double* pq, int* npq, bool presplit) {
  const int nact = active ? h->cur_active : nvec;
  cudaEvent_t e = nullptr;
  CKS(prof_begin(h, cls, &e));
  LK(launch_band(h, h->stream, cls, nvec, active, x, y, h->band_threads, h->band_nv, pq, npq, presplit));
  CKS(prof_end(h, e, 2.0 * h->band_nnz * nact, 8.0 * ((double)h->band_H * h->N + 2.0 * nact * h->N)));
  return IGA_OK;
}

// y = M x; with pq, the assembled form also leaves per-block partials of x . y in pq
// ([nvec][*npq]); *npq = 0 when they were not computed (matrix-free form).
// presplit (double-FP32 form): the split copy of x is already in place
int apply_M(iga_handle* h, int nvec, const int* active, const double* x, double* y, double* pq, int* npq,
            bool presplit) {
  if (npq) *npq = 0;
  if (h->mp) return mp_apply(h, 0, nvec, active, x, y);
  if (is_assembled(h)) {
    CKS(assemble_band(h));
    return apply_band(h, IGA_PROF_BAND_MASS, nvec, active, x, y, pq, npq,
                      presplit && h->opt.op_form == IGA_OP_ASSEMBLED_DF);
  }
  return apply_M_mf(h, nvec, active, x, y);
}
int apply_K(iga_handle* h, int nvec, const int* active, const double* x, double* y) {
  if (h->mp) return mp_apply(h, 1, nvec, active, x, y);
  if (is_assembled(h)) {
    CKS(assemble_band(h));
    return apply_band(h, IGA_PROF_BAND_STIFF, nvec, active, x, y);
  }
  return apply_K_mf(h, nvec, active, x, y);
}
int apply_Pinv(iga_handle* h, int nvec, const int* active, const double* r, double* z, double* rzp, int* nrz) {
  if (h->mp) {
    if (nrz) *nrz = 0;
    return mp_apply(h, 2, nvec, active, r, z);
  }
  const int nact = active ? h->cur_active : nvec;
  double modes = 0.0;  // sum_a n_a: one mode product costs 2 n_a flops per entry, done twice
  for (int a = 0; a < h->dim; ++a) modes += h->n[a];
  cudaEvent_t e = nullptr;
  CKS(prof_begin(h, IGA_PROF_PRECOND, &e));
  CKS(ensure_cg_ws(h, nvec));
  CKS(fd_apply(h, nvec, active, r, z, h->f1, h->f2, rzp, nrz));
  CKS(prof_end(h, e, nact * (4.0 * modes + 3.0) * (double)h->N, 8.0 * (2.0 * nact + 1.0) * (double)h->N));
  return IGA_OK;
}

// Multi-patch operators (Sec. 5.1, 5.4): the global vectors are gathered into every
// patch's box (zero where a box entry is no degree of freedom), the patch's own operator
// acts on its box -- M^(r), K^(r), or the local preconditioner P^(r)^{-1}
// (def:loc_forms2) -- and the local results are summed into the global vector:
// which = 0: M = sum_r R^(r)T M^(r) R^(r); 1: K likewise; 2: P_ad^{-1} (def:asp).
int mp_apply(iga_handle* h, int which, int nvec, const int* active, const double* x, double* y) {
  MpState& mp = *h->mp;
  if (nvec > mp.vec_cap) {
    drop_step_graph(h);
    CKS(dalloc(h, &mp.xl, (size_t)nvec * mp.nloc));
    CKS(dalloc(h, &mp.yl, (size_t)nvec * mp.nloc));
    mp.vec_cap = nvec;
  }
  cudaStream_t s = h->stream;
  // Patches on streams of their own in the host-driven loop only: inside a step capture
  // (s is the capture or loop-body stream) they run in order on s, because the patch
  // streams, once joined to the step's capture, cannot also join the loop body's.
  const bool conc = mp.concurrent && s != h->gs && s != h->gbody;
  LK(launch_mp_gather(s, mp.maps, nvec, active, x, mp.xl));
  if (conc) CK(cudaEventRecord(mp.fork, s));
  for (size_t r = 0; r < mp.patch.size(); ++r) {
    iga_handle* p = mp.patch[r];
    p->stream = s;
    if (conc) {
      CK(cudaStreamWaitEvent(mp.ps[r], mp.fork, 0));
      p->stream = mp.ps[r];
    }
    p->cur_active = h->cur_active;
    const long long l0 = p->nlaunch;
    double* xr = mp.xl + nvec * mp.off[r];
    double* yr = mp.yl + nvec * mp.off[r];
    const int rc = which == 0   ? apply_M(p, nvec, active, xr, yr)
                   : which == 1 ? apply_K(p, nvec, active, xr, yr)
                                : apply_Pinv(p, nvec, active, xr, yr);
    h->nlaunch += p->nlaunch - l0;
    if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
    if (conc) {
      CK(cudaEventRecord(mp.join[r], mp.ps[r]));
      CK(cudaStreamWaitEvent(s, mp.join[r], 0));
      p->stream = s;
    }
  }
  LK(launch_mp_scatter(s, mp.maps, nvec, active, mp.yl, y));
  return IGA_OK;
}

}  // namespace iga
