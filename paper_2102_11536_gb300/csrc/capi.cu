// C ABI of the GB300 explicit generalized-alpha IGA library (include/iga_galpha.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"

using namespace iga;

namespace iga {

thread_local std::string g_create_err;

int fail(iga_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

// Event bracket around the launches of one profiled kernel class.
int prof_begin(iga_handle* h, int cls, cudaEvent_t* e1) {
  *e1 = nullptr;
  if (h->prof_class != cls) return IGA_OK;
  cudaEvent_t a, b;
  if (h->prof_pool.size() >= 2) {
    a = h->prof_pool.back(); h->prof_pool.pop_back();
    b = h->prof_pool.back(); h->prof_pool.pop_back();
  } else {
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
  }
  CK(cudaEventRecord(a, h->stream));
  h->prof_pending.push_back({a, b});
  *e1 = b;
  return IGA_OK;
}

int prof_end(iga_handle* h, cudaEvent_t e1, double flops, double bytes) {
  if (!e1) return IGA_OK;
  CK(cudaEventRecord(e1, h->stream));
  h->prof_flops += flops;
  h->prof_bytes += bytes;
  return IGA_OK;
}


// -- the method's parameters (Sec. 4.1, boxed formulas; eq. HOgamma) ----------
// Block j = k: rho_b = rho_s = rho, alpha_f = 0. Blocks j < k: the boxed j<k
// formulas at rho_b = rho_s = -rho (the reading that keeps the stability limit of
// every block equal to that of the last one), alpha_f = 1.
void galpha_params(int k, double rho, double* alpha, double* beta, double* gamma) {
  for (int j = 1; j <= k; ++j) {
    double a, b, af;
    if (j == k) {
      const double rb = rho, rs = rho;
      a = (2.0 + (1.0 - rb) * rs) / ((1.0 + rb) * (1.0 + rs));
      b = (-5.0 - 3.0 * rb - 4.0 * rs + 2.0 * rb * rs + 2.0 * rb * rb * rs - rs * rs + rb * rs * rs) /
          ((1.0 + rb) * (1.0 + rb) * (-2.0 - 3.0 * rs + rb * rs - rs * rs + rb * rs * rs));
      af = 0.0;
    } else {
      const double rb = -rho, rs = -rho;
      a = (2.0 - (1.0 + rb) * rs) / ((rb - 1.0) * (rs - 1.0));
      b = (1.0 + rb) * (rb * rs - 1.0) * (rb * rs - 1.0) /
          ((rb - 1.0) * (rb - 1.0) * (rs - 1.0) * (rs + rb * rs - 2.0));
      af = 1.0;
    }
    alpha[j - 1] = a;
    beta[j - 1] = b;
    gamma[j - 1] = 0.5 - af + a;
  }
}

// Taylor coefficients tau^m / m! and the block parameters of one step.
StepCoefs step_coefs(int k, double rho, double dt) {
  StepCoefs sc{};
  sc.damped = 0;
  sc.k = k;
  sc.tau = dt;
  double fact = 1.0;
  for (int m = 0; m < 3 * k; ++m) {
    if (m > 0) fact *= m;
    sc.c[m] = std::pow(dt, m) / fact;
  }
  galpha_params(k, rho, sc.alpha, sc.beta, sc.gamma);
  for (int j = 0; j < k; ++j) {  // the update's per-stage factors, once per step instead of per entry
    sc.ralpha[j] = 1.0 / sc.alpha[j];
    sc.gtau[j] = sc.gamma[j] * dt;
    sc.btau2[j] = sc.beta[j] * dt * dt;
  }
  return sc;
}

// The same with the handle's damping (predictor forms Y + aK Y').
StepCoefs handle_coefs(const iga_handle* h, int k, double rho, double dt) {
  StepCoefs sc = step_coefs(k, rho, dt);
  sc.damped = h->damped ? 1 : 0;
  sc.aM = h->aM;
  sc.aK = h->aK;
  return sc;
}

double theta_crit(double rho) { return 12.0 * (1.0 + rho) * (2.0 - rho) / (rho * rho - 5.0 * rho + 10.0); }

// A captured step graph holds workspace addresses: every workspace reallocation
// below drops it, and the next step captures again.
void drop_step_graph(iga_handle* h);
inline bool is_assembled(const iga_handle* h) {
  return h->opt.op_form == IGA_OP_ASSEMBLED || h->opt.op_form == IGA_OP_ASSEMBLED_DF;
}

int ensure_op_ws(iga_handle* h, int nvec) {
  if (h->ws_vec >= nvec) return IGA_OK;
  drop_step_graph(h);
  if (h->dim == 3) {
    h->su = (long long)h->Q[0] * h->n[1] * h->n[2];
    h->st = (long long)h->Q[0] * h->Q[1] * h->n[2];
    CKS(dalloc(h, &h->u0, (size_t)(nvec * h->su)));
    CKS(dalloc(h, &h->u1, (size_t)(nvec * h->su)));
    CKS(dalloc(h, &h->ta, (size_t)(nvec * h->st)));
    CKS(dalloc(h, &h->tb, (size_t)(nvec * h->st)));
    CKS(dalloc(h, &h->tc, (size_t)(nvec * h->st)));
  } else {
    h->su = (long long)h->Q[0] * h->n[1];
    h->st = 0;
    CKS(dalloc(h, &h->u0, (size_t)(nvec * h->su)));
    CKS(dalloc(h, &h->u1, (size_t)(nvec * h->su)));
  }
  h->ws_vec = nvec;
  return IGA_OK;
}

int ensure_cg_ws(iga_handle* h, int nvec) {
  if (h->cg_vec >= nvec) return IGA_OK;
  drop_step_graph(h);
  const size_t sz = (size_t)nvec * h->N;
  CKS(dalloc(h, &h->r, sz));
  CKS(dalloc(h, &h->z, sz));
  CKS(dalloc(h, &h->zold, sz));
  CKS(dalloc(h, &h->p, sz));
  CKS(dalloc(h, &h->q, sz));
  CKS(dalloc(h, &h->f1, sz));
  CKS(dalloc(h, &h->f2, sz));
  CKS(dalloc(h, &h->pq_part, (size_t)nvec * (size_t)df_max_blocks(h->N, h->n)));
  CKS(dalloc(h, &h->rz_part, (size_t)2 * nvec * (size_t)(h->N / 32 + 2)));
  h->cg_vec = nvec;
  return IGA_OK;
}

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
             double* rzp = nullptr, int* nrz = nullptr) {
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
  const std::vector<int> runs = band_df_runs(h->n, p3);
  CKS(upload(h, &h->band_runs, runs));
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
                        double* y, int threads, int nv, double* pq, int* npq, bool presplit = false) {
  const bool mass = cls == IGA_PROF_BAND_MASS;
  if (h->opt.op_form == IGA_OP_ASSEMBLED_DF) {
    float2* xs = h->df_xs + h->df_slack;
    if (!presplit) {
      const cudaError_t e = launch_df_split(s, h->N, active, nvec, x, h->N, xs, h->band_Np, h->df_E, h->df_part,
                                            h->df_bar, h->dflag + 2, h->bar_limit);
      if (e != cudaSuccess) return e;
    }
    return launch_band_df(s, h->N, h->band_nruns, reinterpret_cast<const int4*>(h->band_runs), h->n, h->dd[0].p,
                          h->dim == 3 ? h->dd[2].p : 0, h->band_H, (mass ? h->Mdf : h->Kdf) + h->df_slack, h->band_Np, mass ? h->EAm : h->EAk, active, nvec,
                          xs, h->df_E, x, y, h->N, threads, nv, pq, npq, h->dflag + 2, mass ? &h->tmM : &h->tmK);
  }
  return launch_band_spmv(s, h->N, h->band_H, h->band_off, h->band_o12, h->n, mass ? h->Mband : h->Kband, active,
                          nvec, x, y, h->N, threads, nv, pq, npq);
}

int apply_band(iga_handle* h, int cls, int nvec, const int* active, const double* x, double* y,
               double* pq = nullptr, int* npq = nullptr, bool presplit = false) {
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
int mp_apply(iga_handle* h, int which, int nvec, const int* active, const double* x, double* y);

int apply_M(iga_handle* h, int nvec, const int* active, const double* x, double* y, double* pq = nullptr,
            int* npq = nullptr, bool presplit = false) {
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
int apply_Pinv(iga_handle* h, int nvec, const int* active, const double* r, double* z, double* rzp = nullptr,
               int* nrz = nullptr) {
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

// ---------------------------------------------------------------------------
// batched PCG
// ---------------------------------------------------------------------------
// PCG (Sec. 5.5), split into launch-only pieces so that the same kernels serve the
// host-driven loop and the captured graph (whose loop runs on the device).
// solve_begin: r = b - M x0 (or x = 0, r = b), ||b||^2, ||r||^2, activity flags.
int solve_begin(iga_handle* h, int nvec, const double* b, double* x, bool use_x0) {
  cudaStream_t s = h->stream;
  const long long N = h->N;
  CgScalars& c = h->cs;
  double* pA = h->partial;
  double* pB = h->partial + kMaxVec * kRedBlocks;
  const double tol2 = h->opt.tol * h->opt.tol;
  if (use_x0) {
    CKS(apply_M(h, nvec, nullptr, x, h->q));
    LK(launch_sub(s, N, nvec, b, h->q, h->r, N));
  } else {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * nvec * N, s));
    CK(cudaMemcpyAsync(h->r, b, sizeof(double) * nvec * N, cudaMemcpyDeviceToDevice, s));
  }
  LK(launch_dot(s, N, nvec, b, b, N, pA));
  LK(launch_dot(s, N, nvec, h->r, h->r, N, pB));
  LK(launch_cg_init(s, nvec, pA, pB, c, tol2));
  return IGA_OK;
}

// solve_prime: z = P^{-1} r, r.z, p = z (active systems).
int solve_prime(iga_handle* h, int nvec) {
  cudaStream_t s = h->stream;
  const long long N = h->N;
  CgScalars& c = h->cs;
  int nrz = 0;
  CKS(apply_Pinv(h, nvec, c.active, h->r, h->z, h->rz_part, &nrz));
  if (nrz > 0) {  // r.z came with the preconditioner's last pass
    LK(launch_cg_start(s, nvec, h->rz_part, nrz, c));
  } else {
    LK(launch_dot(s, N, nvec, h->r, h->z, N, h->partial));
    LK(launch_cg_start(s, nvec, h->partial, kRedBlocks, c));
  }
  LK(launch_copy_active(s, N, nvec, c.active, h->z, h->p, N));
  if (h->opt.op_form == IGA_OP_ASSEMBLED_DF) {  // the first product's split, made here (see solve_iter_a)
    CKS(assemble_band(h));
    LK(launch_df_split(s, N, c.active, nvec, h->p, N, h->df_xs + h->df_slack, h->band_Np, h->df_E, h->df_part,
                       h->df_bar, h->dflag + 2, h->bar_limit));
  }
  return IGA_OK;
}

// solve_iter_a: q = M p, alpha = r.z / p.q, x += alpha p, r -= alpha q, convergence test.
int solve_iter_a(iga_handle* h, int nvec, double* x) {
  cudaStream_t s = h->stream;
  const long long N = h->N;
  CgScalars& c = h->cs;
  double* pA = h->partial;
  double* pB = h->partial + kMaxVec * kRedBlocks;
  int npq = 0;
  // double-FP32 form: p's split copy was made where p was (solve_prime, solve_iter_b)
  CKS(apply_M(h, nvec, c.active, h->p, h->q, h->pq_part, &npq, true));
  if (npq > 0) {  // p.q came with the band product
    LK(launch_cg_alpha(s, nvec, h->pq_part, npq, c));
  } else {
    LK(launch_dot(s, N, nvec, h->p, h->q, N, pA));
    LK(launch_cg_alpha(s, nvec, pA, kRedBlocks, c));
  }
  // the convergence test runs in the update's last block
  LK(launch_cg_update_xr(s, N, nvec, c, x, h->r, h->p, h->q, N, pB, 1, h->opt.tol * h->opt.tol));
  return IGA_OK;
}

// solve_iter_b: [flexible: r.z_old] z = P^{-1} r, beta, p = z + beta p.
int solve_iter_b(iga_handle* h, int nvec) {
  cudaStream_t s = h->stream;
  const long long N = h->N;
  CgScalars& c = h->cs;
  double* pA = h->partial;
  double* pC = h->partial + 2 * kMaxVec * kRedBlocks;
  // the FP64 preconditioners are symmetric and linear to rounding: plain CG
  const bool flexible = h->opt.precond != IGA_PREC_FP64 && h->opt.precond != IGA_PREC_BANDED;
  const bool fused = h->opt.precond == IGA_PREC_BANDED || h->opt.precond == IGA_PREC_BANDED32;
  int nrz = 0;
  const double* rzA = pA;  // r.z partials, [nvec][nrzp], and r.z_old for the flexible beta
  const double* rzB = pC;
  int nrzp = kRedBlocks;
  if (fused) {  // r.z and r.z_old come with the preconditioner's last pass
    CKS(apply_Pinv(h, nvec, c.active, h->r, h->z, h->rz_part, &nrz));
    if (nrz <= 0) return fail(h, IGA_ECUDA, "fused inner products missing");
    rzA = h->rz_part;
    rzB = h->rz_part + (size_t)nvec * nrz;
    nrzp = nrz;
  } else {
    if (flexible) LK(launch_dot(s, N, nvec, h->r, h->z, N, pC));  // z still holds the previous z
    CKS(apply_Pinv(h, nvec, c.active, h->r, h->z));
    LK(launch_dot(s, N, nvec, h->r, h->z, N, pA));
  }
  if (h->opt.op_form == IGA_OP_ASSEMBLED_DF) {
    // beta, p = z + beta p and its split for the next product, one launch (the fused r.z
    // partials are laid out [2][nvec][nrz], as BetaArgs reads them)
    float2* xs = h->df_xs + h->df_slack;
    cudaError_t e = cudaErrorNotSupported;
    if (fused) {
      const BetaArgs ba{rzA, nrzp, flexible ? 1 : 0, c};
      e = launch_df_update_split(s, N, c.active, nvec, h->p, h->z, ba, N, xs, h->band_Np, h->df_E, h->df_part,
                                 h->df_bar, h->dflag + 2, h->bar_limit);
    }
    if (e == cudaErrorNotSupported) {
      cudaGetLastError();
      LK(launch_cg_beta(s, nvec, rzA, rzB, nrzp, c, flexible ? 1 : 0));
      LK(launch_cg_update_p(s, N, nvec, c, h->p, h->z, N));
      e = launch_df_split(s, N, c.active, nvec, h->p, N, xs, h->band_Np, h->df_E, h->df_part, h->df_bar,
                          h->dflag + 2, h->bar_limit);
    }
    LK(e);
    return IGA_OK;
  }
  LK(launch_cg_beta(s, nvec, rzA, rzB, nrzp, c, flexible ? 1 : 0));
  LK(launch_cg_update_p(s, N, nvec, c, h->p, h->z, N));
  return IGA_OK;
}

int read_nactive(iga_handle* h, int* nact) {
  CK(cudaMemcpyAsync(h->h_nactive, h->cs.nactive, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *nact = *h->h_nactive;
  h->cur_active = *nact;
  return IGA_OK;
}

// Host-driven batched PCG: one host synchronisation per iteration to test convergence.
int solve(iga_handle* h, int nvec, const double* b, double* x, bool use_x0, int* iters, double* relres) {
  CKS(ensure_cg_ws(h, nvec));
  CKS(ensure_op_ws(h, nvec));
  cudaStream_t s = h->stream;
  CgScalars& c = h->cs;
  CKS(solve_begin(h, nvec, b, x, use_x0));
  int nact = 0;
  CKS(read_nactive(h, &nact));
  if (nact > 0) CKS(solve_prime(h, nvec));
  int it = 0;
  while (nact > 0 && it < h->opt.max_iter) {
    CKS(solve_iter_a(h, nvec, x));
    CKS(read_nactive(h, &nact));
    ++it;
    if (nact == 0) break;
    CKS(solve_iter_b(h, nvec));
  }
  int hit[kMaxVec], hst[kMaxVec];
  double hrr[kMaxVec], hbb[kMaxVec], hr0[kMaxVec];
  CK(cudaMemcpyAsync(hr0, c.rr0, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hit, c.iters, sizeof(int) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hst, c.status, sizeof(int) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hrr, c.rr, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hbb, c.bb, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int status = IGA_OK;
  for (int v = 0; v < nvec; ++v) {
    const double rel = hbb[v] > 0 ? std::sqrt(hrr[v] / hbb[v]) : 0.0;
    h->last_init[v] = hbb[v] > 0 ? std::sqrt(hr0[v] / hbb[v]) : 0.0;
    if (iters) iters[v] = hit[v];
    if (relres) relres[v] = rel;
    if (hst[v] != 0) status = IGA_ENUMERIC;
  }
  CKS(check_tc_error(h));
  if (status != IGA_OK) return fail(h, status, "PCG breakdown (non-positive curvature or non-finite values)");
  if (nact > 0) {
    char buf[160];
    snprintf(buf, sizeof buf, "PCG did not reach tol %.3g in %d iterations", h->opt.tol, h->opt.max_iter);
    return fail(h, IGA_ENOT_CONVERGED, buf);
  }
  return IGA_OK;
}

int check_handle(iga_handle* h) {
  if (!h) return IGA_EINVAL;
  h->err.clear();
  cudaError_t e = cudaSetDevice(h->opt.device);
  if (e != cudaSuccess) return fail(h, IGA_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return IGA_OK;
}

// Entry points that need one patch's grid (the learned guess, profiling, tuning, the
// allocation-free preconditioner, batches) refuse a multi-patch handle.
int single_patch(iga_handle* h, const char* what) {
  if (h && h->mp) return fail(h, IGA_EINVAL, std::string(what) + " is not available on a multi-patch handle");
  return IGA_OK;
}

int ensure_step_ws(iga_handle* h, int k) {
  if (h->step_k >= k) return IGA_OK;
  drop_step_graph(h);
  const size_t sz = (size_t)k * h->N;
  CKS(dalloc(h, &h->Yneg, sz));
  CKS(dalloc(h, &h->rhs, sz));
  CKS(dalloc(h, &h->Z, sz));
  CKS(dalloc(h, &h->Z2, sz));
  h->step_k = k;
  return IGA_OK;
}

// Buffers of the learned guess for k stages: histories, features, hidden layer.
int ensure_ws_step(iga_handle* h, int k) {
  if (!h->ws_theta) {
    CKS(dalloc(h, &h->ws_theta, IGA_NET_NPARAM));
    CKS(dalloc(h, &h->ws_m, IGA_NET_NPARAM));
    CKS(dalloc(h, &h->ws_v, IGA_NET_NPARAM));
    CKS(dalloc(h, &h->ws_grad, IGA_NET_NPARAM));
    CKS(dalloc(h, &h->ws_sc, 2 * kMaxVec));
    CKS(dalloc(h, &h->ws_part, (size_t)2 * kMaxVec * kRedBlocks));
  }
  if (h->ws_k >= k) return IGA_OK;
  drop_step_graph(h);
  const size_t sz = (size_t)k * h->N;
  CKS(dalloc(h, &h->ws_E, sz));
  CKS(dalloc(h, &h->ws_B1, sz));
  CKS(dalloc(h, &h->ws_B2, sz));
  CKS(dalloc(h, &h->ws_x, 3 * sz));
  CKS(dalloc(h, &h->ws_act, 16 * sz));
  h->ws_k = k;
  return IGA_OK;
}

// Buffers of the damping term aM M Y'_j for k stages, and the device time.
int ensure_damp_ws(iga_handle* h, int k) {
  if (!h->d_time) {
    CKS(dalloc(h, &h->d_time, 1));
    CK(cudaMemcpy(h->d_time, &h->time, sizeof(double), cudaMemcpyHostToDevice));
  }
  if (!(h->damped && h->aM != 0.0) || h->yv_k >= k) return IGA_OK;
  drop_step_graph(h);
  CKS(dalloc(h, &h->Yv, (size_t)k * h->N));
  CKS(dalloc(h, &h->MYv, (size_t)k * h->N));
  h->yv_k = k;
  return IGA_OK;
}

bool m_term(const iga_handle* h) { return h->damped && h->aM != 0.0; }

// Loads of the stages after the predictor: rhs_j = F^{(s_j)}(t_{n+alpha_fj}) - K (Y_j + aK Y'_j)
// - aM M Y'_j (eq. ho1 with C = aM M + aK K; Yneg = -(Y_j + aK Y'_j), Yv = -Y'_j).
int stage_rhs(iga_handle* h, cudaStream_t s, int k, const StepCoefs& sc) {
  CKS(apply_K(h, k, nullptr, h->Yneg, h->rhs));
  const bool mt = m_term(h);
  if (mt) CKS(apply_M(h, k, nullptr, h->Yv, h->MYv));
  if (mt || h->nforce > 0) {
    StageLoad a{};
    a.nstage = k;
    for (int j = 0; j < k; ++j) {
      a.sder[j] = 3 * j;
      a.toff[j] = j < k - 1 ? sc.tau : 0.0;  // alpha_f = 1 for the blocks j < k, 0 for the last
    }
    a.nterm = h->nforce;
    for (int m = 0; m < h->nforce; ++m) {
      a.om[m] = h->fom[m];
      a.ph[m] = h->fph[m];
    }
    a.aM = h->aM;
    LK(launch_stage_load(s, h->N, a, h->fG, h->d_time, mt ? h->MYv : nullptr, h->rhs));
  }
  return IGA_OK;
}

NetGrid net_grid_of(const iga_handle* h) { return NetGrid{h->n[0], h->n[1], h->n[2]}; }

// The learned guess of the k solves of a step, two steps of history present:
// features (into x), histories moved, Z = E (+ s0 y once the network is trained).
int learned_guess(iga_handle* h, cudaStream_t s, int k, __nv_bfloat16* x) {
  CK(launch_ws_features(s, h->N, k, h->rhs, h->ws_B1, h->ws_B2, h->Dm, h->Z, h->Z2, x, h->ws_E, h->ws_part,
                        h->ws_sc, &h->nlaunch));
  if (h->ws_trained)
    CK(launch_net_forward(s, net_grid_of(h), k, x, h->ws_theta, h->ws_act, nullptr, h->Z, h->ws_E, h->ws_sc,
                          &h->nlaunch));
  return IGA_OK;
}

// ---------------------------------------------------------------------------
// one time step as a CUDA graph, the PCG loop running on the device
// ---------------------------------------------------------------------------
void drop_step_graph(iga_handle* h) {
  ++h->ws_gen;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  h->gvalid = false;
}

// Everything a step capture uses, allocated beforehand (nothing is allocated while
// capturing); drops the handle's own step graph.
int prepare_capture(iga_handle* h, int k) {
  drop_step_graph(h);
  if (!h->gs) {
    CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->gbody, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  }
  if (!h->d_loop) {
    CKS(dalloc(h, &h->d_loop, 2));
    CKS(dalloc(h, &h->d_tot, kMaxVec));
    CKS(dalloc(h, &h->d_max, kMaxVec));
    CKS(dalloc(h, &h->d_init, kMaxVec));
    CKS(dalloc(h, &h->d_stat, 2));
  }
  CKS(ensure_step_ws(h, k));
  CKS(ensure_cg_ws(h, k));
  CKS(ensure_op_ws(h, k));
  if (h->opt.guess == IGA_GUESS_LEARNED) CKS(ensure_ws_step(h, k));
  CKS(ensure_damp_ws(h, k));
  if (is_assembled(h)) CKS(assemble_band(h));
  if (h->mp) {  // a multi-patch step reaches every patch: their workspaces too, at full size
    MpState& mp = *h->mp;
    if (mp.vec_cap < kMaxVec) {
      CKS(dalloc(h, &mp.xl, (size_t)kMaxVec * mp.nloc));
      CKS(dalloc(h, &mp.yl, (size_t)kMaxVec * mp.nloc));
      mp.vec_cap = kMaxVec;
    }
    for (size_t r = 0; r < mp.patch.size(); ++r) {
      iga_handle* p = mp.patch[r];
      p->stream = h->stream;
      int rc = ensure_op_ws(p, kMaxVec);
      if (rc == IGA_OK) rc = ensure_cg_ws(p, kMaxVec);
      if (rc == IGA_OK && is_assembled(p)) rc = assemble_band(p);
      if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
    }
  }
  return IGA_OK;
}

// Capture one step into the capture that h->gs takes part in: Taylor predictor,
// batched K, the solve's set-up, a conditional while node whose body is one PCG
// iteration followed by the loop test (k_set_cond: some system active and fewer
// than max_iter iterations), the iteration statistics, and the stage update.
int capture_step(iga_handle* h, double* state, int k, const StepCoefs& sc) {
  struct StreamSwap {
    iga_handle* h;
    cudaStream_t user;
    ~StreamSwap() { h->stream = user; }
  } swap{h, h->stream};
  h->stream = h->gs;
  const long long N = h->N;
  const int guess = h->opt.guess;
  const long long l0 = h->nlaunch;
  LK(launch_predict(h->gs, N, sc, state, h->Yneg, guess == IGA_GUESS_TAYLOR ? h->Z : nullptr,
                    m_term(h) ? h->Yv : nullptr));
  CKS(stage_rhs(h, h->gs, k, sc));
  if (guess == IGA_GUESS_EXTRAP) LK(launch_extrap(h->gs, (long long)k * N, h->Z, h->Z2));
  if (guess == IGA_GUESS_LEARNED) CKS(learned_guess(h, h->gs, k, h->ws_x));
  CKS(solve_begin(h, k, h->rhs, h->Z, guess != IGA_GUESS_ZERO));
  CKS(solve_prime(h, k));  // masked: no work for systems that start converged
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->gs, &cst, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, cg, 0, cudaGraphCondAssignDefault));
  LK(launch_set_cond(h->gs, hc, h->cs.nactive, h->d_loop, h->opt.max_iter, 1));
  CK(cudaStreamGetCaptureInfo(h->gs, &cst, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  h->g_pro = h->nlaunch - l0;
  const long long l1 = h->nlaunch;
  h->stream = h->gbody;
  CK(cudaStreamBeginCaptureToGraph(h->gbody, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int brc = solve_iter_a(h, k, h->Z);
  if (brc == IGA_OK) brc = solve_iter_b(h, k);
  if (brc == IGA_OK) {
    const cudaError_t be = launch_set_cond(h->gbody, hc, h->cs.nactive, h->d_loop, h->opt.max_iter, 0);
    if (be != cudaSuccess) brc = fail(h, IGA_ECUDA, std::string("loop test: ") + cudaGetErrorString(be));
    else ++h->nlaunch;
  }
  cudaGraph_t bout = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->gbody, &bout);
  h->stream = h->gs;
  if (brc != IGA_OK) return brc;
  if (ee != cudaSuccess) return fail(h, IGA_ECUDA, std::string("loop body capture: ") + cudaGetErrorString(ee));
  h->g_body = h->nlaunch - l1;
  CK(cudaStreamUpdateCaptureDependencies(h->gs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  const long long l2 = h->nlaunch;
  LK(launch_accum(h->gs, k, h->cs, h->d_tot, h->d_max, h->d_init, h->d_stat));
  LK(launch_update(h->gs, N, sc, state, h->Z));
  LK(launch_advance_time(h->gs, h->d_time, sc.tau));
  h->g_epi = h->nlaunch - l2;
  return IGA_OK;
}

// Instantiate the graph a capture produced (destroyed on failure).
int instantiate(iga_handle* h, int rc, cudaError_t end_err, cudaGraph_t g, cudaGraph_t* graph,
                cudaGraphExec_t* exec) {
  if (rc != IGA_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  }
  if (end_err != cudaSuccess) return fail(h, IGA_ECUDA, std::string("step capture: ") + cudaGetErrorString(end_err));
  cudaGraphExec_t ge = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(h, IGA_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
  }
  *graph = g;
  *exec = ge;
  return IGA_OK;
}

int build_step_graph(iga_handle* h, double* state, int k, const StepCoefs& sc) {
  CKS(prepare_capture(h, k));
  const cudaError_t e0 = cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) return fail(h, IGA_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e0));
  const int rc = capture_step(h, state, k, sc);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->gs, &g);
  CKS(instantiate(h, rc, ee, g, &h->graph, &h->gexec));
  h->gvalid = true;
  return IGA_OK;
}

bool same_key(const iga_handle::GraphKey& a, const iga_handle::GraphKey& b) {
  return a.state == b.state && a.k == b.k && a.op == b.op && a.prec == b.prec && a.guess == b.guess &&
         a.max_iter == b.max_iter && a.dt == b.dt && a.rho == b.rho && a.tol == b.tol;
}

// Zero the device counters that the captured step accumulates into.
int reset_graph_counters(iga_handle* h, cudaStream_t s) {
  CK(cudaMemsetAsync(h->d_tot, 0, sizeof(long long) * kMaxVec, s));
  CK(cudaMemsetAsync(h->d_max, 0, sizeof(int) * kMaxVec, s));
  CK(cudaMemsetAsync(h->d_init, 0, sizeof(double) * kMaxVec, s));
  CK(cudaMemsetAsync(h->d_stat, 0, sizeof(int) * 2, s));
  CK(cudaMemsetAsync(h->d_loop, 0, sizeof(int) * 2, s));
  return IGA_OK;
}

// After nsteps replays (ordered before later work on s): launch count, history,
// statistics and the error status of the solves. Synchronises s.
int collect_graph_run(iga_handle* h, cudaStream_t s, int k, int nsteps, double dt, iga_stats* stats) {
  long long tot[kMaxVec];
  int mx[kMaxVec], st[2], loop[2];
  double rr[kMaxVec], bb[kMaxVec], ini[kMaxVec];
  CK(cudaMemcpyAsync(ini, h->d_init, sizeof(ini), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(tot, h->d_tot, sizeof(tot), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(mx, h->d_max, sizeof(mx), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(st, h->d_stat, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(loop, h->d_loop, sizeof(loop), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rr, h->cs.rr, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(bb, h->cs.bb, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->nlaunch += (long long)nsteps * (h->g_pro + h->g_epi) + (long long)loop[1] * h->g_body;
  h->hist = std::min(h->hist + nsteps, 2);
  for (int i = 0; i < nsteps; ++i) h->time += dt;  // the device adds dt once per step too
  if (stats) {
    stats->steps += nsteps;
    stats->solves += k * nsteps;
    for (int j = 0; j < k; ++j) {
      stats->iters += tot[j];
      stats->init_relres_sum += ini[j];
      stats->max_iters = std::max(stats->max_iters, mx[j]);
      const double rel = bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0;  // last step's solves
      stats->max_relres = std::max(stats->max_relres, rel);
    }
  }
  CKS(check_tc_error(h));
  if (st[0] != 0) return fail(h, IGA_ENUMERIC, "PCG breakdown (non-positive curvature or non-finite values)");
  if (st[1] != 0) {
    char buf[160];
    snprintf(buf, sizeof buf, "PCG did not reach tol %.3g in %d iterations", h->opt.tol, h->opt.max_iter);
    return fail(h, IGA_ENOT_CONVERGED, buf);
  }
  return IGA_OK;
}

iga_handle::GraphKey graph_key(const iga_handle* h, double* state, int k, double rho, double dt) {
  iga_handle::GraphKey key{};
  key.state = state;
  key.k = k;
  key.op = h->opt.op_form;
  key.prec = h->opt.precond;
  key.guess = h->opt.guess;
  key.max_iter = h->opt.max_iter;
  key.dt = dt;
  key.rho = rho;
  key.tol = h->opt.tol;
  return key;
}

// nsteps replays of the captured step on h->gs, ordered after earlier work on the
// caller's stream and before later work on it; one host synchronisation at the end.
int run_step_graph(iga_handle* h, double* state, int k, double rho, const StepCoefs& sc, int nsteps,
                   iga_stats* stats) {
  const iga_handle::GraphKey key = graph_key(h, state, k, rho, sc.tau);
  if (!h->gvalid || !same_key(key, h->gkey)) {
    CKS(build_step_graph(h, state, k, sc));
    h->gkey = key;
  }
  cudaStream_t s = h->stream;
  CKS(reset_graph_counters(h, s));
  CK(cudaEventRecord(h->ev_in, s));
  CK(cudaStreamWaitEvent(h->gs, h->ev_in, 0));
  for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(h->gexec, h->gs));
  CK(cudaEventRecord(h->ev_out, h->gs));
  CK(cudaStreamWaitEvent(s, h->ev_out, 0));
  return collect_graph_run(h, s, k, nsteps, sc.tau, stats);
}

// One patch over the index box lo .. hi per direction (full indices; NULL: the interior
// functions 1 .. m-2, iga_create). The operators see only the box's functions; the
// geometry uses the whole control net.
int create_handle(int dim, const int* degree, const int* nknots, const double* const* knots, const double* ctrl,
                  const int* lo, const int* hi, const iga_options* opt, iga_handle** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, IGA_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(nullptr, IGA_EINVAL, "dim must be 2 or 3");
  if (!degree || !nknots || !knots || !ctrl) return fail(nullptr, IGA_EINVAL, "NULL input array");
  iga_handle* h = new (std::nothrow) iga_handle();
  if (!h) return fail(nullptr, IGA_ENOMEM, "host allocation failed");
  if (opt) h->opt = *opt;
  else iga_options_default(&h->opt);
  if (!(h->opt.tol >= 0.0) || h->opt.max_iter < 1 || h->opt.precond < 0 || h->opt.precond > IGA_PREC_BANDED32 ||
      h->opt.op_form < 0 || h->opt.op_form > IGA_OP_ASSEMBLED_DF || h->opt.guess < 0 || h->opt.guess > IGA_GUESS_LEARNED) {
    delete h;
    return fail(nullptr, IGA_EINVAL, "invalid options");
  }
  h->dim = dim;
  h->stream = (cudaStream_t)h->opt.stream;
  int pmax = 0;
  for (int a = 0; a < dim; ++a) pmax = std::max(pmax, degree[a]);
  const int nq = h->opt.nquad > 0 ? h->opt.nquad : pmax + 1;
  std::string err;
  for (int a = 0; a < dim; ++a) {
    if (!knots[a] || !build_tables(degree[a], nknots[a], knots[a], nq, h->tab[a], err, lo ? lo[a] : 1,
                                   hi ? hi[a] : -1)) {
      delete h;
      return fail(nullptr, IGA_EINVAL, "direction " + std::to_string(a) + ": " + (knots[a] ? err : "NULL knots"));
    }
    h->n[a] = h->tab[a].n;
    h->Q[a] = h->tab[a].Q;
    h->m[a] = h->tab[a].m;
  }
  h->N = (long long)h->n[0] * h->n[1] * h->n[2];
  h->Qt = (long long)h->Q[0] * h->Q[1] * h->Q[2];
  if (cudaSetDevice(h->opt.device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, IGA_ECUDA, "cudaSetDevice failed");
  }
  int rc = IGA_OK;
  auto setup = [&]() -> int {
    for (int a = 0; a < dim; ++a) {
      const Tables1D& t = h->tab[a];
      DirDev& d = h->dd[a];
      d.p = t.p; d.P = t.p + 1; d.n = t.n; d.Q = t.Q;
      std::vector<double> sq(t.val.size());
      for (size_t i = 0; i < sq.size(); ++i) sq[i] = t.val[i] * t.val[i];
      std::vector<float> v32(t.val.begin(), t.val.end()), d32(t.der.begin(), t.der.end());
      // [U | U^T]: element (i, j) of the applied matrix at j*np + i, rows padded to np
      const int np = (t.n + 7) & ~7;
      const size_t blk = (size_t)t.n * np;
      std::vector<double> U(2 * blk, 0.0);
      for (int i = 0; i < t.n; ++i)
        for (int j = 0; j < t.n; ++j) {
          U[(size_t)j * np + i] = t.evec[(size_t)i * t.n + j];        // U(i, j)
          U[blk + (size_t)j * np + i] = t.evec[(size_t)j * t.n + i];  // U^T(i, j) = U(j, i)
        }
      // inverse eigenvalues 1/Lambda_a (the epilogue multiplies)
      std::vector<double> linv(t.n);
      for (int i = 0; i < t.n; ++i) linv[i] = 1.0 / t.eval[i];
      std::vector<float> U32(U.begin(), U.end()), l32(linv.begin(), linv.end());
      CKS(upload(h, &d.val, t.val)); CKS(upload(h, &d.der, t.der)); CKS(upload(h, &d.sq, sq));
      CKS(upload(h, &d.val32, v32)); CKS(upload(h, &d.der32, d32));
      CKS(upload(h, &d.qfirst, t.qfirst_op)); CKS(upload(h, &d.flo, t.flo)); CKS(upload(h, &d.fhi, t.fhi));
      if (t.lo != 1) CKS(upload(h, &d.qfirst_geo, t.qfirst));
      CKS(upload(h, &d.qw, t.qw));
      CKS(upload(h, &d.U64, U)); CKS(upload(h, &d.lam64, linv));
      CKS(upload(h, &d.chol, t.chol)); CKS(upload(h, &d.cdinv, t.cdinv));
      CKS(upload(h, &d.chol32, std::vector<float>(t.chol.begin(), t.chol.end())));
      CKS(upload(h, &d.cdinv32, std::vector<float>(t.cdinv.begin(), t.cdinv.end())));
      if (tc_pad(t.n) <= 256) {  // BF16 tensor-core operands: Mat = U and Mat = U^T, (i, j) row-major
        std::vector<double> Mu((size_t)t.n * t.n), Mt((size_t)t.n * t.n);
        for (int i = 0; i < t.n; ++i)
          for (int j = 0; j < t.n; ++j) {
            Mu[(size_t)i * t.n + j] = t.evec[(size_t)i * t.n + j];
            Mt[(size_t)i * t.n + j] = t.evec[(size_t)j * t.n + i];
          }
        std::vector<uint16_t> bits;
        for (int f16 = 0; f16 < 2; ++f16)
          for (int tr = 0; tr < 2; ++tr) {
            tc_arrange(t.n, tr ? Mt.data() : Mu.data(), f16 != 0, bits);
            uint16_t* pb = nullptr;
            CKS(upload(h, &pb, bits));
            (f16 ? d.Btc16 : d.Btc)[tr] = pb;
          }
      }
      CKS(upload(h, &d.U32, U32)); CKS(upload(h, &d.lam32, l32));
    }
    // control net, point-major -> SoA
    const long long mt = (long long)h->m[0] * h->m[1] * (dim == 3 ? h->m[2] : 1);
    std::vector<double> soa((size_t)(dim * mt));
    for (long long i = 0; i < mt; ++i)
      for (int c = 0; c < dim; ++c) soa[(size_t)(c * mt + i)] = ctrl[i * dim + c];
    CKS(upload(h, &h->ctrl, soa));
    const int ng = dim == 3 ? 6 : 3;
    h->gstride = h->Qt;
    CKS(dalloc(h, &h->W, (size_t)h->Qt));
    CKS(dalloc(h, &h->G, (size_t)(ng * h->Qt)));
    CKS(dalloc(h, &h->dflag, 4));
    CK(cudaMemsetAsync(h->dflag, 0, sizeof(int) * 4, h->stream));
    int mm[3] = {h->m[0], h->m[1], h->m[2]};
    LK(launch_geometry(h->stream, dim, h->dd, mm, h->ctrl, h->W, h->G, h->gstride, h->dflag));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, IGA_EGEOMETRY, "det DF <= 0 at a quadrature point");
    // PCG scalars and reduction scratch
    CKS(dalloc(h, &h->partial, (size_t)3 * kMaxVec * kRedBlocks));
    CKS(dalloc(h, &h->cs.bb, kMaxVec)); CKS(dalloc(h, &h->cs.rz, kMaxVec)); CKS(dalloc(h, &h->cs.rr, kMaxVec)); CKS(dalloc(h, &h->cs.rr0, kMaxVec));
    CKS(dalloc(h, &h->cs.alpha, kMaxVec)); CKS(dalloc(h, &h->cs.beta, kMaxVec));
    CKS(dalloc(h, &h->cs.active, kMaxVec)); CKS(dalloc(h, &h->cs.iters, kMaxVec));
    CKS(dalloc(h, &h->cs.status, kMaxVec)); CKS(dalloc(h, &h->cs.nactive, 1));
    CKS(dalloc(h, &h->cs.ticket, 2));
    CK(cudaMemset(h->cs.ticket, 0, 2 * sizeof(unsigned int)));
    CKS(dalloc(h, &h->cs.red, (size_t)kMaxVec * 64));
    CK(cudaMallocHost((void**)&h->h_nactive, sizeof(int) * 4));
    // diag(M): D = (B_0^2)^T (B_1^2)^T (B_2^2)^T W (transposed passes with squared tables)
    CKS(ensure_op_ws(h, 1));
    CKS(dalloc(h, &h->Dm, (size_t)h->N));
    const int *n = h->n, *Q = h->Q;
    const DirDev* d = h->dd;
    if (dim == 3) {
      LK(launch_tr(h->stream, d[2], {(long long)Q[0] * Q[1], Q[2], n[2], 1}, 1, nullptr, h->W, d[2].sq, nullptr, nullptr, 0, h->ta, 0));
      LK(launch_tr(h->stream, d[1], {Q[0], Q[1], n[1], n[2]}, 1, nullptr, h->ta, d[1].sq, nullptr, nullptr, 0, h->u0, 0));
      LK(launch_tr(h->stream, d[0], {1, Q[0], n[0], (long long)n[1] * n[2]}, 1, nullptr, h->u0, d[0].sq, nullptr, nullptr, 0, h->Dm, 0));
    } else {
      LK(launch_tr(h->stream, d[1], {Q[0], Q[1], n[1], 1}, 1, nullptr, h->W, d[1].sq, nullptr, nullptr, 0, h->u0, 0));
      LK(launch_tr(h->stream, d[0], {1, Q[0], n[0], n[1]}, 1, nullptr, h->u0, d[0].sq, nullptr, nullptr, 0, h->Dm, 0));
    }
    std::vector<double> D((size_t)h->N), sc((size_t)h->N);
    CK(cudaMemcpyAsync(D.data(), h->Dm, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < h->N; ++i) {
      const int i0 = (int)(i % n[0]), i1 = (int)((i / n[0]) % n[1]), i2 = (int)(i / ((long long)n[0] * n[1]));
      double dh = h->tab[0].mhat[(size_t)i0 * n[0] + i0] * h->tab[1].mhat[(size_t)i1 * n[1] + i1];
      if (dim == 3) dh *= h->tab[2].mhat[(size_t)i2 * n[2] + i2];
      if (!(D[i] > 0)) return fail(h, IGA_EGEOMETRY, "non-positive diagonal of M");
      sc[i] = std::sqrt(dh / D[i]);
    }
    CKS(upload(h, &h->scale, sc));
    std::vector<float> sc32(sc.begin(), sc.end());
    CKS(upload(h, &h->scale32, sc32));
    return IGA_OK;
  };
  rc = setup();
  if (rc != IGA_OK) {
    g_create_err = h->err;
    iga_destroy(h);
    return rc;
  }
  *out = h;
  return IGA_OK;
}

}  // namespace iga

namespace iga {

int handle_device(iga_handle* h, int* device) {
  CKS(check_handle(h));
  *device = h->opt.device;
  return IGA_OK;
}

int handle_fail(iga_handle* h, int code, const std::string& msg) { return fail(h, code, msg); }

int pinv_with_scratch(iga_handle* h, int nvec, const double* x, double* y, double* t1, double* t2) {
  CKS(single_patch(h, "iga_apply_Pinv_noalloc"));
  CKS(fd_apply(h, nvec, nullptr, x, y, t1, t2));
  // a tensor-core mode product whose wait ran out is reported here, not by the next call
  return check_tc_error(h);
}

}  // namespace iga

// ===========================================================================
// public API
// ===========================================================================
extern "C" {

void iga_options_default(iga_options* opt) {
  if (!opt) return;
  opt->nquad = 0;
  opt->tol = 1e-10;
  opt->max_iter = 500;
  opt->precond = IGA_PREC_FP64;
  opt->op_form = IGA_OP_MATRIX_FREE;
  opt->guess = IGA_GUESS_ZERO;
  opt->device = 0;
  opt->stream = nullptr;
}

const char* iga_status_string(int status) {
  switch (status) {
    case IGA_OK: return "ok";
    case IGA_EINVAL: return "invalid argument";
    case IGA_ENOMEM: return "out of memory";
    case IGA_ECUDA: return "CUDA error";
    case IGA_ENOT_CONVERGED: return "PCG not converged";
    case IGA_ENUMERIC: return "numerical breakdown";
    case IGA_EUNSTABLE: return "unstable time step";
    case IGA_EGEOMETRY: return "invalid geometry (det DF <= 0)";
    default: return "unknown status";
  }
}

const char* iga_last_error(const iga_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void iga_destroy(iga_handle* h) {
  if (!h) return;
  cudaSetDevice(h->opt.device);
  if (h->mp) {
    MpState* mp = h->mp;
    for (iga_handle* p : mp->patch) iga_destroy(p);
    dfree(mp->d_gid); dfree(mp->d_off); dfree(mp->d_nr); dfree(mp->d_crow); dfree(mp->d_cent); dfree(mp->d_epatch);
    dfree(mp->xl); dfree(mp->yl);
    for (cudaStream_t ps : mp->ps) cudaStreamDestroy(ps);
    for (cudaEvent_t e : mp->join) cudaEventDestroy(e);
    if (mp->fork) cudaEventDestroy(mp->fork);
    delete mp;
    h->mp = nullptr;
  }
  for (int a = 0; a < 3; ++a) {
    DirDev& d = h->dd[a];
    dfree(d.val); dfree(d.der); dfree(d.sq); dfree(d.val32); dfree(d.der32);
    dfree(d.qfirst); dfree(d.qfirst_geo); dfree(d.flo); dfree(d.fhi); dfree(d.qw);
    dfree(d.U64); dfree(d.lam64); dfree(d.U32); dfree(d.lam32); dfree(d.chol); dfree(d.cdinv); dfree(d.chol32); dfree(d.cdinv32);
    for (int t = 0; t < 2; ++t)
      if (d.Btc[t]) { cudaFree(d.Btc[t]); d.Btc[t] = nullptr; }
    for (int t = 0; t < 2; ++t)
      if (d.Btc16[t]) { cudaFree(d.Btc16[t]); d.Btc16[t] = nullptr; }
  }
  dfree(h->ctrl); dfree(h->W); dfree(h->G); dfree(h->Dm); dfree(h->scale); dfree(h->scale32); dfree(h->dflag);
  dfree(h->Mband); dfree(h->Kband); dfree(h->band_off); dfree(h->band_o12);
  dfree(h->Mdf); dfree(h->Kdf); dfree(h->band_runs); dfree(h->df_xs); dfree(h->df_E); dfree(h->df_part); dfree(h->df_bar);
  dfree(h->u0); dfree(h->u1); dfree(h->ta); dfree(h->tb); dfree(h->tc);
  dfree(h->r); dfree(h->z); dfree(h->zold); dfree(h->p); dfree(h->q); dfree(h->f1); dfree(h->f2);
  dfree(h->partial); dfree(h->pq_part); dfree(h->rz_part);
  dfree(h->cs.bb); dfree(h->cs.rz); dfree(h->cs.rr); dfree(h->cs.rr0); dfree(h->cs.alpha); dfree(h->cs.beta);
  dfree(h->cs.active); dfree(h->cs.iters); dfree(h->cs.status); dfree(h->cs.nactive); dfree(h->cs.ticket); dfree(h->cs.red);
  if (h->h_nactive) cudaFreeHost(h->h_nactive);
  for (auto& pr : h->prof_pending) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  dfree(h->Yneg); dfree(h->rhs); dfree(h->Z); dfree(h->Z2); dfree(h->dstate);
  drop_step_graph(h);
  if (h->gs) cudaStreamDestroy(h->gs);
  if (h->gbody) cudaStreamDestroy(h->gbody);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  dfree(h->d_loop); dfree(h->d_tot); dfree(h->d_max); dfree(h->d_init); dfree(h->d_stat);
  dfree(h->fG); dfree(h->Yv); dfree(h->MYv); dfree(h->d_time); dfree(h->pts);
  dfree(h->ws_theta); dfree(h->ws_m); dfree(h->ws_v); dfree(h->ws_grad);
  dfree(h->ws_E); dfree(h->ws_B1); dfree(h->ws_B2); dfree(h->ws_sc); dfree(h->ws_part);
  dfree(h->ws_x); dfree(h->ws_act); dfree(h->ws_sx); dfree(h->ws_st);
  dfree(h->ws_y); dfree(h->ws_dy); dfree(h->ws_loss); dfree(h->ws_lpart);
  if (h->ws_work) cudaFree(h->ws_work);
  delete h;
}

int iga_create(int dim, const int* degree, const int* nknots, const double* const* knots, const double* ctrl,
               const iga_options* opt, iga_handle** out) {
  return create_handle(dim, degree, nknots, knots, ctrl, nullptr, nullptr, opt, out);
}

int iga_ndof(const iga_handle* h, long long* ndof) {
  if (!h || !ndof) return IGA_EINVAL;
  *ndof = h->N;
  return IGA_OK;
}

int iga_set_op_form(iga_handle* h, int op_form) {
  if (!h || op_form < 0 || op_form > IGA_OP_ASSEMBLED_DF) return IGA_EINVAL;
  if (h->mp) {  // the patches' form; the composite dispatches through them
    h->mp->op_form = op_form;
    for (iga_handle* p : h->mp->patch) p->opt.op_form = op_form;
    drop_step_graph(h);
    return IGA_OK;
  }
  h->opt.op_form = op_form;
  return IGA_OK;
}
int iga_set_precond(iga_handle* h, int precond) {
  if (!h || precond < 0 || precond > IGA_PREC_BANDED32) return IGA_EINVAL;
  if (h->mp) {  // the patches' local preconditioners; the composite's PCG follows their class
    h->mp->precond = precond;
    for (iga_handle* p : h->mp->patch) p->opt.precond = precond;
    h->opt.precond = (precond == IGA_PREC_FP64 || precond == IGA_PREC_BANDED) ? IGA_PREC_FP64 : IGA_PREC_FP32;
    drop_step_graph(h);
    return IGA_OK;
  }
  h->opt.precond = precond;
  return IGA_OK;
}
int iga_set_guess(iga_handle* h, int guess) {
  if (!h || guess < 0 || guess > IGA_GUESS_LEARNED) return IGA_EINVAL;
  if (h->mp && guess == IGA_GUESS_LEARNED) return fail(h, IGA_EINVAL, "the learned guess needs a single patch");
  h->opt.guess = guess;
  return IGA_OK;
}
int iga_set_damping(iga_handle* h, double aM, double aK) {
  CKS(check_handle(h));
  if (!(aM >= 0.0 && aK >= 0.0 && std::isfinite(aM) && std::isfinite(aK)))
    return fail(h, IGA_EINVAL, "damping coefficients must be finite and non-negative");
  h->damped = aM != 0.0 || aK != 0.0;
  h->aM = aM;
  h->aK = aK;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_set_forcing(iga_handle* h, int nterm, const double* G, const double* omega, const double* phase) {
  CKS(check_handle(h));
  if (nterm < 0 || nterm > kMaxForce || (nterm > 0 && (!G || !omega || !phase)))
    return fail(h, IGA_EINVAL, "need 0 <= nterm <= 8 and non-NULL arrays");
  for (int m = 0; m < nterm; ++m)
    if (!std::isfinite(omega[m]) || !std::isfinite(phase[m])) return fail(h, IGA_EINVAL, "non-finite frequency");
  CK(cudaStreamSynchronize(h->stream));
  dfree(h->fG);
  h->nforce = 0;
  if (nterm > 0) {
    CKS(dalloc(h, &h->fG, (size_t)nterm * h->N));
    CK(cudaMemcpy(h->fG, G, sizeof(double) * nterm * h->N, cudaMemcpyDeviceToDevice));
    for (int m = 0; m < nterm; ++m) {
      h->fom[m] = omega[m];
      h->fph[m] = phase[m];
    }
    h->nforce = nterm;
  }
  drop_step_graph(h);
  return IGA_OK;
}

int iga_set_time(iga_handle* h, double t) {
  CKS(check_handle(h));
  if (!std::isfinite(t)) return fail(h, IGA_EINVAL, "non-finite time");
  CKS(ensure_damp_ws(h, 0));
  CK(cudaStreamSynchronize(h->stream));
  h->time = t;
  CK(cudaMemcpy(h->d_time, &h->time, sizeof(double), cudaMemcpyHostToDevice));
  return IGA_OK;
}

int iga_get_time(iga_handle* h, double* t) {
  CKS(check_handle(h));
  if (!t) return fail(h, IGA_EINVAL, "t is NULL");
  *t = h->time;
  return IGA_OK;
}

int iga_set_graphs(iga_handle* h, int on) {
  if (!h) return IGA_EINVAL;
  h->use_graphs = on != 0;
  return IGA_OK;
}

int iga_set_barrier_limit(iga_handle* h, long long polls) {
  CKS(check_handle(h));
  if (h->mp) {
    for (iga_handle* p : h->mp->patch) CKS(iga_set_barrier_limit(p, polls));
  }
  h->bar_limit = polls < 0 ? -1 : polls;
  drop_step_graph(h);  // captured launches hold the old limit
  return IGA_OK;
}

int iga_set_tol(iga_handle* h, double tol, int max_iter) {
  if (!h || !(tol >= 0) || max_iter < 1) return IGA_EINVAL;
  h->opt.tol = tol;
  h->opt.max_iter = max_iter;
  return IGA_OK;
}

int iga_assemble(iga_handle* h) {
  CKS(check_handle(h));
  if (h->mp) {
    for (size_t r = 0; r < h->mp->patch.size(); ++r) {
      iga_handle* p = h->mp->patch[r];
      p->stream = h->stream;
      const int rc = assemble_band(p);
      if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
    }
    return IGA_OK;
  }
  return assemble_band(h);
}

int iga_apply_M(iga_handle* h, int nvec, const double* x, double* y) {
  CKS(check_handle(h));
  if (nvec < 1 || nvec > kMaxVec || !x || !y) return fail(h, IGA_EINVAL, "bad arguments");
  return apply_M(h, nvec, nullptr, x, y);
}

int iga_apply_K(iga_handle* h, int nvec, const double* x, double* y) {
  CKS(check_handle(h));
  if (nvec < 1 || nvec > kMaxVec || !x || !y) return fail(h, IGA_EINVAL, "bad arguments");
  return apply_K(h, nvec, nullptr, x, y);
}

int iga_apply_Pinv(iga_handle* h, int nvec, const double* x, double* y) {
  CKS(check_handle(h));
  if (nvec < 1 || nvec > kMaxVec || !x || !y) return fail(h, IGA_EINVAL, "bad arguments");
  CKS(apply_Pinv(h, nvec, nullptr, x, y));
  return check_tc_error(h);
}

int iga_solve_M(iga_handle* h, int nvec, const double* b, double* x, int use_x0, int* iters, double* relres) {
  CKS(check_handle(h));
  if (nvec < 1 || nvec > kMaxVec || !b || !x) return fail(h, IGA_EINVAL, "bad arguments");
  return solve(h, nvec, b, x, use_x0 != 0, iters, relres);
}

int iga_npoints(const iga_handle* h, long long* Qt, int* Q) {
  if (!h || !Qt || h->mp) return IGA_EINVAL;
  *Qt = h->Qt;
  if (Q)
    for (int a = 0; a < h->dim; ++a) Q[a] = h->Q[a];
  return IGA_OK;
}

int iga_gauss_points(iga_handle* h, double* x, double* w) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_gauss_points"));
  if (x) {
    int mm[3] = {h->m[0], h->m[1], h->m[2]};
    LK(launch_points(h->stream, h->dim, h->dd, mm, h->ctrl, x));
  }
  if (w) CK(cudaMemcpyAsync(w, h->W, sizeof(double) * h->Qt, cudaMemcpyDeviceToDevice, h->stream));
  return IGA_OK;
}

// g = B U: the forward banded passes of the mass operator, without the weighting
int iga_evaluate(iga_handle* h, int nvec, const double* U, double* g) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_evaluate"));
  if (nvec < 1 || nvec > kMaxVec || !U || !g) return fail(h, IGA_EINVAL, "bad arguments");
  CKS(ensure_op_ws(h, nvec));
  cudaStream_t s = h->stream;
  const int *n = h->n, *Q = h->Q;
  const DirDev* d = h->dd;
  if (h->dim == 3) {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], (long long)n[1] * n[2]}, nvec, nullptr, U, h->N, d[0].val, h->u0, nullptr, nullptr, h->su));
    LK(launch_fwd(s, d[1], {Q[0], n[1], Q[1], n[2]}, nvec, nullptr, h->u0, h->su, d[1].val, h->ta, nullptr, nullptr, h->st));
    LK(launch_fwd(s, d[2], {(long long)Q[0] * Q[1], n[2], Q[2], 1}, nvec, nullptr, h->ta, h->st, d[2].val, g, nullptr, nullptr, h->Qt));
  } else {
    LK(launch_fwd(s, d[0], {1, n[0], Q[0], n[1]}, nvec, nullptr, U, h->N, d[0].val, h->u0, nullptr, nullptr, h->su));
    LK(launch_fwd(s, d[1], {Q[0], n[1], Q[1], 1}, nvec, nullptr, h->u0, h->su, d[1].val, g, nullptr, nullptr, h->Qt));
  }
  return IGA_OK;
}

// b = B^T (W .* g): the quadrature of int g B_i, by the transposed passes
int iga_integrate(iga_handle* h, int nvec, const double* g, double* b) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_integrate"));
  if (nvec < 1 || nvec > kMaxVec || !g || !b) return fail(h, IGA_EINVAL, "bad arguments");
  CKS(ensure_op_ws(h, nvec));
  if (h->pts_cap < nvec * h->Qt) {
    CK(cudaStreamSynchronize(h->stream));
    CKS(dalloc(h, &h->pts, (size_t)(nvec * h->Qt)));
    h->pts_cap = nvec * h->Qt;
  }
  cudaStream_t s = h->stream;
  const int *n = h->n, *Q = h->Q;
  const DirDev* d = h->dd;
  LK(launch_weight_points(s, h->Qt, nvec, h->W, g, h->pts));
  if (h->dim == 3) {
    LK(launch_tr(s, d[2], {(long long)Q[0] * Q[1], Q[2], n[2], 1}, nvec, nullptr, h->pts, d[2].val, nullptr, nullptr, h->Qt, h->ta, h->st));
    LK(launch_tr(s, d[1], {Q[0], Q[1], n[1], n[2]}, nvec, nullptr, h->ta, d[1].val, nullptr, nullptr, h->st, h->u0, h->su));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], (long long)n[1] * n[2]}, nvec, nullptr, h->u0, d[0].val, nullptr, nullptr, h->su, b, h->N));
  } else {
    LK(launch_tr(s, d[1], {Q[0], Q[1], n[1], 1}, nvec, nullptr, h->pts, d[1].val, nullptr, nullptr, h->Qt, h->u0, h->su));
    LK(launch_tr(s, d[0], {1, Q[0], n[0], n[1]}, nvec, nullptr, h->u0, d[0].val, nullptr, nullptr, h->su, b, h->N));
  }
  return IGA_OK;
}

int iga_galpha_params(int k, double rho_inf, double* alpha, double* beta, double* gamma) {
  if (k < 1 || k > kMaxK || !(rho_inf >= 0.0 && rho_inf <= 1.0) || !alpha || !beta || !gamma) return IGA_EINVAL;
  galpha_params(k, rho_inf, alpha, beta, gamma);
  return IGA_OK;
}

int iga_mp_layout(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
                  const double* const* ctrl, double tol, int* lo, int* hi, long long* nglob, int* n_adj,
                  long long* gid, long long gid_len) {
  std::string msg;
  const int rc = mp_layout(npatch, dim, degree, nknots, knots, ctrl, tol, lo, hi, nglob, n_adj, gid, gid_len, msg);
  return rc == IGA_OK ? IGA_OK : fail(nullptr, rc, msg);
}

int iga_mp_create(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
                  const double* const* ctrl, double tol, const iga_options* opt, iga_handle** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, IGA_EINVAL, "out is NULL");
  *out = nullptr;
  if (npatch < 1 || (dim != 2 && dim != 3) || !degree || !nknots || !knots || !ctrl)
    return fail(nullptr, IGA_EINVAL, "iga_mp_create: npatch >= 1, dim 2 or 3 and non-null arrays required");
  iga_options o;
  if (opt) o = *opt;
  else iga_options_default(&o);
  if (!(o.tol >= 0.0) || o.max_iter < 1 || o.precond < 0 || o.precond > IGA_PREC_BANDED32 || o.op_form < 0 ||
      o.op_form > IGA_OP_ASSEMBLED_DF || o.guess < 0 || o.guess > IGA_GUESS_TAYLOR)
    return fail(nullptr, IGA_EINVAL, "invalid options (the learned guess is not available on a multi-patch handle)");
  // gluing: boxes first, then the global id of every box entry
  std::vector<int> lo((size_t)npatch * dim), hi((size_t)npatch * dim);
  long long nglob = 0;
  int n_adj = 0;
  std::string err;
  int rc = mp_layout(npatch, dim, degree, nknots, knots, ctrl, tol, lo.data(), hi.data(), &nglob, &n_adj, nullptr, 0,
                     err);
  if (rc != IGA_OK) return fail(nullptr, rc, err);
  std::vector<long long> off(npatch), nr(npatch);
  long long nloc = 0;
  for (int r = 0; r < npatch; ++r) {
    long long c = 1;
    for (int a = 0; a < dim; ++a) c *= hi[(size_t)r * dim + a] - lo[(size_t)r * dim + a] + 1;
    off[r] = nloc;
    nr[r] = c;
    nloc += c;
  }
  std::vector<long long> gid((size_t)nloc);
  rc = mp_layout(npatch, dim, degree, nknots, knots, ctrl, tol, lo.data(), hi.data(), &nglob, &n_adj, gid.data(),
                 nloc, err);
  if (rc != IGA_OK) return fail(nullptr, rc, err);
  if (nglob < 1) return fail(nullptr, IGA_EINVAL, "iga_mp_create: no degrees of freedom");
  // global -> entries (CSR, entries ascending) and entry -> patch
  std::vector<long long> crow((size_t)nglob + 1, 0), cent;
  std::vector<int> epatch((size_t)nloc);
  for (int r = 0; r < npatch; ++r)
    for (long long i = 0; i < nr[r]; ++i) epatch[(size_t)(off[r] + i)] = r;
  for (long long e = 0; e < nloc; ++e)
    if (gid[(size_t)e] >= 0) ++crow[(size_t)gid[(size_t)e] + 1];
  for (long long g = 0; g < nglob; ++g) crow[(size_t)g + 1] += crow[(size_t)g];
  cent.assign((size_t)crow[(size_t)nglob], 0);
  {
    std::vector<long long> fill(crow.begin(), crow.end() - 1);
    for (long long e = 0; e < nloc; ++e)
      if (gid[(size_t)e] >= 0) cent[(size_t)fill[(size_t)gid[(size_t)e]]++] = e;
  }
  iga_handle* h = new (std::nothrow) iga_handle();
  if (!h) return fail(nullptr, IGA_ENOMEM, "host allocation failed");
  h->mp = new (std::nothrow) MpState();
  if (!h->mp) {
    delete h;
    return fail(nullptr, IGA_ENOMEM, "host allocation failed");
  }
  MpState& mp = *h->mp;
  h->opt = o;
  h->dim = dim;
  h->stream = (cudaStream_t)o.stream;
  h->N = nglob;
  h->Qt = 1;
  // host-driven loop unless iga_set_graphs(h, 1): a captured step reaches the patches through
  // the stream they are handed on every call, and prepare_capture sizes their workspaces
  h->use_graphs = false;
  // the composite runs the PCG of its preconditioner's class: plain CG for the FP64 forms,
  // flexible CG otherwise; its own operator form is the dispatch through the patches
  mp.op_form = o.op_form;
  mp.precond = o.precond;
  h->opt.op_form = IGA_OP_MATRIX_FREE;
  h->opt.precond = (o.precond == IGA_PREC_FP64 || o.precond == IGA_PREC_BANDED) ? IGA_PREC_FP64 : IGA_PREC_FP32;
  mp.off = off;
  mp.nr = nr;
  mp.nloc = nloc;
  mp.n_adj = n_adj;
  if (cudaSetDevice(o.device) != cudaSuccess) {
    cudaGetLastError();
    iga_destroy(h);
    return fail(nullptr, IGA_ECUDA, "cudaSetDevice failed");
  }
  iga_options po = o;
  po.guess = IGA_GUESS_ZERO;
  for (int r = 0; r < npatch; ++r) {
    iga_handle* p = nullptr;
    rc = create_handle(dim, degree + (size_t)r * dim, nknots + (size_t)r * dim, knots + (size_t)r * dim, ctrl[r],
                       lo.data() + (size_t)r * dim, hi.data() + (size_t)r * dim, &po, &p);
    if (rc != IGA_OK) {
      const std::string msg = "patch " + std::to_string(r) + ": " + g_create_err;
      iga_destroy(h);
      return fail(nullptr, rc, msg);
    }
    mp.patch.push_back(p);
  }
  auto setup = [&]() -> int {
    CKS(upload(h, &mp.d_gid, gid));
    CKS(upload(h, &mp.d_off, off));
    CKS(upload(h, &mp.d_nr, nr));
    CKS(upload(h, &mp.d_crow, crow));
    CKS(upload(h, &mp.d_cent, cent));
    CKS(upload(h, &mp.d_epatch, epatch));
    mp.maps.nloc = nloc;
    mp.maps.nglob = nglob;
    mp.maps.gid = mp.d_gid;
    mp.maps.epatch = mp.d_epatch;
    mp.maps.off = mp.d_off;
    mp.maps.nr = mp.d_nr;
    mp.maps.crow = mp.d_crow;
    mp.maps.cent = mp.d_cent;
    CKS(dalloc(h, &h->dflag, 4));
    CK(cudaMemsetAsync(h->dflag, 0, sizeof(int) * 4, h->stream));
    CKS(dalloc(h, &h->partial, (size_t)3 * kMaxVec * kRedBlocks));
    CKS(dalloc(h, &h->cs.bb, kMaxVec)); CKS(dalloc(h, &h->cs.rz, kMaxVec)); CKS(dalloc(h, &h->cs.rr, kMaxVec)); CKS(dalloc(h, &h->cs.rr0, kMaxVec));
    CKS(dalloc(h, &h->cs.alpha, kMaxVec)); CKS(dalloc(h, &h->cs.beta, kMaxVec));
    CKS(dalloc(h, &h->cs.active, kMaxVec)); CKS(dalloc(h, &h->cs.iters, kMaxVec));
    CKS(dalloc(h, &h->cs.status, kMaxVec)); CKS(dalloc(h, &h->cs.nactive, 1));
    CKS(dalloc(h, &h->cs.ticket, 2));
    CK(cudaMemset(h->cs.ticket, 0, 2 * sizeof(unsigned int)));
    CKS(dalloc(h, &h->cs.red, (size_t)kMaxVec * 64));
    CK(cudaMallocHost((void**)&h->h_nactive, sizeof(int) * 4));
    CK(cudaStreamSynchronize(h->stream));
    return IGA_OK;
  };
  rc = setup();
  if (rc != IGA_OK) {
    const std::string msg = h->err;
    iga_destroy(h);
    return fail(nullptr, rc, msg);
  }
  *out = h;
  return IGA_OK;
}

int iga_mp_set_concurrent(iga_handle* h, int on) {
  CKS(check_handle(h));
  if (!h->mp) return fail(h, IGA_EINVAL, "not a multi-patch handle");
  MpState& mp = *h->mp;
  if (on && mp.ps.empty()) {  // all or nothing: the vectors stay empty if a creation fails
    std::vector<cudaStream_t> ps;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (size_t r = 0; e == cudaSuccess && r < mp.patch.size(); ++r) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) ps.push_back(st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) join.push_back(ev);
    }
    if (e != cudaSuccess) {
      for (cudaStream_t st : ps) cudaStreamDestroy(st);
      for (cudaEvent_t ev : join) cudaEventDestroy(ev);
      if (fork) cudaEventDestroy(fork);
      cudaGetLastError();
      return fail(h, IGA_ECUDA, std::string("iga_mp_set_concurrent: ") + cudaGetErrorString(e));
    }
    mp.ps = ps;
    mp.join = join;
    mp.fork = fork;
  }
  mp.concurrent = on != 0;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_mp_patch(iga_handle* h, int r, iga_handle** patch) {
  if (!h || !h->mp || !patch || r < 0 || r >= (int)h->mp->patch.size()) return IGA_EINVAL;
  *patch = h->mp->patch[(size_t)r];
  (*patch)->stream = h->stream;
  return IGA_OK;
}

int iga_mp_patch_io(iga_handle* h, int r, int nvec, int add, const double* in, double* out) {
  CKS(check_handle(h));
  if (!h->mp || r < 0 || r >= (int)h->mp->patch.size() || nvec < 1 || nvec > kMaxVec || !in || !out)
    return fail(h, IGA_EINVAL, "bad arguments");
  const MpState& mp = *h->mp;
  LK(launch_mp_patch_io(h->stream, mp.maps, mp.off[(size_t)r], mp.nr[(size_t)r], nvec, add != 0, in, out));
  return IGA_OK;
}

int iga_mp_info(const iga_handle* h, int* npatch, int* n_adj, long long* nloc) {
  if (!h || !h->mp) return IGA_EINVAL;
  if (npatch) *npatch = (int)h->mp->patch.size();
  if (n_adj) *n_adj = h->mp->n_adj;
  if (nloc) *nloc = h->mp->nloc;
  return IGA_OK;
}

int iga_state_init(iga_handle* h, int k, const double* U0, const double* V0, double* state) {
  CKS(check_handle(h));
  if (k < 1 || k > kMaxK || !U0 || !V0 || !state) return fail(h, IGA_EINVAL, "bad arguments");
  const long long N = h->N;
  cudaStream_t s = h->stream;
  CKS(ensure_step_ws(h, 2));
  CK(cudaMemcpyAsync(state, U0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(state + N, V0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  CKS(ensure_damp_ws(h, 1));
  const int last = 3 * k - 3;
  if (!h->damped && h->nforce == 0) {
    // X_a = M^{-1}(-K X_{a-2}), a = 0..3k-3: the chains of even and odd a are
    // independent, so consecutive pairs are solved together.
    for (int a = 0; a <= last; a += 2) {
      const int nv = (a + 1 <= last) ? 2 : 1;
      CKS(apply_K(h, nv, nullptr, state + (long long)a * N, h->rhs));
      LK(launch_scale_neg(s, nv * N, h->rhs));
      CKS(solve(h, nv, h->rhs, state + (long long)(a + 2) * N, false, nullptr, nullptr));
    }
  } else {
    // X_a = M^{-1}(F^{(a)}(t) - K X_{a-2} - C X_{a-1}) in order (the damping couples the chains)
    for (int a = 0; a <= last; ++a) {
      const double* xd = state + (long long)a * N;        // X_{a-2}
      const double* xv = state + (long long)(a + 1) * N;  // X_{a-1}
      LK(launch_lincomb(s, N, -1.0, xd, -h->aK, xv, h->Yneg));
      CKS(apply_K(h, 1, nullptr, h->Yneg, h->rhs));
      const bool mt = m_term(h);
      if (mt) {
        LK(launch_lincomb(s, N, -1.0, xv, 0.0, xv, h->Yv));
        CKS(apply_M(h, 1, nullptr, h->Yv, h->MYv));
      }
      StageLoad ld{};
      ld.nstage = 1;
      ld.sder[0] = a;
      ld.toff[0] = 0.0;
      ld.nterm = h->nforce;
      for (int m = 0; m < h->nforce; ++m) {
        ld.om[m] = h->fom[m];
        ld.ph[m] = h->fph[m];
      }
      ld.aM = h->aM;
      LK(launch_stage_load(s, N, ld, h->fG, h->d_time, mt ? h->MYv : nullptr, h->rhs));
      CKS(solve(h, 1, h->rhs, state + (long long)(a + 2) * N, false, nullptr, nullptr));
    }
  }
  h->hist = 0;
  return IGA_OK;
}

int iga_step(iga_handle* h, double* state, int k, double rho_inf, double dt, int nsteps, iga_stats* stats) {
  CKS(check_handle(h));
  if (k < 1 || k > kMaxK || !state || nsteps < 0 || !(dt > 0.0) || !(rho_inf >= 0.0 && rho_inf <= 1.0))
    return fail(h, IGA_EINVAL, "bad arguments");
  const long long N = h->N;
  cudaStream_t s = h->stream;
  CKS(ensure_step_ws(h, k));
  CKS(ensure_damp_ws(h, k));
  const StepCoefs sc = handle_coefs(h, k, rho_inf, dt);
  const long long launches0 = h->nlaunch;
  for (int step = 0; step < nsteps; ++step) {
    const int guess = h->opt.guess;
    // steady state: replay the captured step (device-side PCG loop) for the remaining steps
    const bool recording = guess == IGA_GUESS_LEARNED && h->ws_cap > 0;
    const bool graph_ok = h->use_graphs && h->prof_class == IGA_PROF_OFF && !recording &&
                          (guess == IGA_GUESS_ZERO || guess == IGA_GUESS_TAYLOR || h->hist >= 2);
    if (graph_ok) {
      const iga_handle::GraphKey key = graph_key(h, state, k, rho_inf, dt);
      if (!h->gvalid || !same_key(key, h->gkey)) {
        if (build_step_graph(h, state, k, sc) != IGA_OK) {
          h->use_graphs = false;  // capture refused: keep the host-driven loop for this handle
          h->err.clear();
        } else {
          h->gkey = key;
        }
      }
      if (h->use_graphs) {
        CKS(run_step_graph(h, state, k, rho_inf, sc, nsteps - step, stats));
        if (stats) stats->launches += h->nlaunch - launches0;
        return IGA_OK;
      }
    }
    const bool taylor = guess == IGA_GUESS_TAYLOR;
    LK(launch_predict(s, N, sc, state, h->Yneg, taylor ? h->Z : nullptr, m_term(h) ? h->Yv : nullptr));
    CKS(stage_rhs(h, s, k, sc));
    bool use_x0 = false;
    if (taylor) {
      use_x0 = true;
    } else if (guess == IGA_GUESS_PREV && h->hist >= 1) {
      use_x0 = true;  // Z still holds the previous step's solutions
    } else if (guess == IGA_GUESS_EXTRAP && h->hist >= 1) {
      if (h->hist >= 2) LK(launch_extrap(s, (long long)k * N, h->Z, h->Z2));
      else CK(cudaMemcpyAsync(h->Z2, h->Z, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, s));
      use_x0 = true;
    }
    // learned guess: histories b^{n-1}, b^{n-2} (ws_B1, ws_B2) and Z^{n-1}, Z^{n-2} (Z, Z2)
    const size_t kvec = sizeof(double) * k * N;
    bool record = false;
    if (guess == IGA_GUESS_LEARNED) {
      CKS(ensure_ws_step(h, k));
      if (h->hist >= 2) {
        record = recording && h->ws_count + k <= h->ws_cap;
        __nv_bfloat16* x = record ? h->ws_sx + (size_t)h->ws_count * 3 * N : h->ws_x;
        CKS(learned_guess(h, s, k, x));
        use_x0 = true;
      } else if (h->hist == 1) {  // previous solution as the guess; histories move
        CK(cudaMemcpyAsync(h->Z2, h->Z, kvec, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(h->ws_B2, h->ws_B1, kvec, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(h->ws_B1, h->rhs, kvec, cudaMemcpyDeviceToDevice, s));
        use_x0 = true;
      } else {
        CK(cudaMemcpyAsync(h->ws_B1, h->rhs, kvec, cudaMemcpyDeviceToDevice, s));
      }
    }
    int its[kMaxVec];
    double rel[kMaxVec];
    CKS(solve(h, k, h->rhs, h->Z, use_x0, its, rel));
    if ((guess == IGA_GUESS_EXTRAP || guess == IGA_GUESS_LEARNED) && h->hist == 0)
      CK(cudaMemcpyAsync(h->Z2, h->Z, kvec, cudaMemcpyDeviceToDevice, s));
    if (record) {
      CK(launch_ws_target(s, N, k, h->Z, h->ws_E, h->ws_sc, h->ws_st + (size_t)h->ws_count * N, &h->nlaunch));
      h->ws_count += k;
    }
    LK(launch_update(s, N, sc, state, h->Z));
    LK(launch_advance_time(s, h->d_time, dt));
    h->time += dt;
    h->hist = std::min(h->hist + 1, 2);
    if (stats) {
      stats->steps += 1;
      stats->solves += k;
      for (int j = 0; j < k; ++j) {
        stats->iters += its[j];
        stats->init_relres_sum += h->last_init[j];
        stats->max_iters = std::max(stats->max_iters, its[j]);
        stats->max_relres = std::max(stats->max_relres, rel[j]);
      }
    }
  }
  if (stats) stats->launches += h->nlaunch - launches0;
  CK(cudaStreamSynchronize(s));
  return IGA_OK;
}

int iga_step_host(iga_handle* h, double* state_host, int k, double rho_inf, double dt, int nsteps,
                  iga_stats* stats) {
  CKS(check_handle(h));
  if (k < 1 || k > kMaxK || !state_host) return fail(h, IGA_EINVAL, "bad arguments");
  const long long len = 3LL * k * h->N;
  if (h->dstate_cap < len) {
    CKS(dalloc(h, &h->dstate, (size_t)len));
    h->dstate_cap = len;
  }
  CK(cudaMemcpyAsync(h->dstate, state_host, sizeof(double) * len, cudaMemcpyHostToDevice, h->stream));
  CKS(iga_step(h, h->dstate, k, rho_inf, dt, nsteps, stats));
  CK(cudaMemcpyAsync(state_host, h->dstate, sizeof(double) * len, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return IGA_OK;
}

int iga_profile(iga_handle* h, int kernel_class) {
  CKS(check_handle(h));
  if (kernel_class < IGA_PROF_OFF || kernel_class > IGA_PROF_BAND_STIFF) return fail(h, IGA_EINVAL, "bad kernel class");
  h->prof_class = kernel_class;
  if (h->mp)  // the kernels run in the patches: each brackets its own launches
    for (iga_handle* p : h->mp->patch) p->prof_class = kernel_class;
  return IGA_OK;
}

int iga_profile_read(iga_handle* h, double* total_ms, long long* launches, double* flops, double* bytes) {
  CKS(check_handle(h));
  if (h->mp) {  // the sums over the patches
    double ms = 0.0, fl = 0.0, by = 0.0;
    long long n = 0;
    for (size_t r = 0; r < h->mp->patch.size(); ++r) {
      iga_handle* p = h->mp->patch[r];
      p->stream = h->stream;
      double pm = 0.0, pf = 0.0, pb = 0.0;
      long long pn = 0;
      const int rc = iga_profile_read(p, &pm, &pn, &pf, &pb);
      if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
      ms += pm;
      n += pn;
      fl += pf;
      by += pb;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    if (flops) *flops = fl;
    if (bytes) *bytes = by;
    return IGA_OK;
  }
  CK(cudaStreamSynchronize(h->stream));
  double ms = 0.0;
  for (auto& pr : h->prof_pending) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, pr.first, pr.second));
    ms += t;
    h->prof_pool.push_back(pr.first);
    h->prof_pool.push_back(pr.second);
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = (long long)h->prof_pending.size();
  if (flops) *flops = h->prof_flops;
  if (bytes) *bytes = h->prof_bytes;
  h->prof_pending.clear();
  h->prof_flops = h->prof_bytes = 0.0;
  return IGA_OK;
}

int iga_cfl(iga_handle* h, double rho_inf, int iters, double* lambda_max, double* tau_crit) {
  CKS(check_handle(h));
  if (iters < 1 || !lambda_max || !tau_crit || !(rho_inf >= 0.0 && rho_inf <= 1.0))
    return fail(h, IGA_EINVAL, "bad arguments");
  const long long N = h->N;
  cudaStream_t s = h->stream;
  // Every allocation first: the band assembly grows the operator workspace, and the
  // buffers below are held by pointer.
  if (is_assembled(h)) CKS(assemble_band(h));
  CKS(ensure_step_ws(h, 2));
  CKS(ensure_cg_ws(h, 2));
  CKS(ensure_op_ws(h, 1));
  double* v = h->Z;        // Lanczos vector v_j
  double* vp = h->Z + N;   // v_{j-1}
  double* w = h->Z2;       // M^{-1} K v_j, then the next residual
  double* y = h->rhs;      // K v_j, then M w
  double* pA = h->partial;
  double* res = h->f1;     // reduced scalars
  auto dot = [&](const double* a, const double* b, double* out) -> int {
    LK(launch_dot(s, N, 1, a, b, N, pA));
    LK(launch_reduce(s, 1, pA, res));
    CK(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return IGA_OK;
  };
  // seeded start (splitmix64, uniform in [-1, 1]), M-normalised
  {
    std::vector<double> x0((size_t)N);
    uint64_t st = 0x6A09E667F3BCC909ULL;
    for (auto& xv : x0) {
      st += 0x9E3779B97F4A7C15ULL;
      uint64_t z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
      z ^= z >> 31;
      xv = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    CK(cudaMemcpyAsync(v, x0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CKS(apply_M(h, 1, nullptr, v, y));
  double nv = 0.0;
  CKS(dot(v, y, &nv));
  LK(launch_lincomb(s, N, 1.0 / std::sqrt(nv), v, 0.0, v, v));
  CK(cudaMemsetAsync(vp, 0, sizeof(double) * N, s));
  const double tol_save = h->opt.tol;
  h->opt.tol = std::min(tol_save, 1e-10);
  std::vector<double> al, be;
  double beta = 0.0, est = 0.0;
  int rc = IGA_OK;
  for (int j = 0; j < iters; ++j) {
    // w = M^{-1} K v_j - alpha_j v_j - beta_{j-1} v_{j-1}, alpha_j = v_j^T K v_j
    if ((rc = apply_K(h, 1, nullptr, v, y)) != IGA_OK) break;
    if ((rc = solve(h, 1, y, w, false, nullptr, nullptr)) != IGA_OK) break;
    double alpha = 0.0;
    if ((rc = dot(v, y, &alpha)) != IGA_OK) break;
    LK(launch_lincomb(s, N, 1.0, w, -alpha, v, w));
    LK(launch_lincomb(s, N, 1.0, w, -beta, vp, w));
    al.push_back(alpha);
    const double prev = est;
    est = tridiag_max_eig(al, be);
    if (j > 0 && std::fabs(est - prev) <= 1e-11 * std::fabs(est)) break;
    // beta_j = ||w||_M, v_{j+1} = w / beta_j
    if ((rc = apply_M(h, 1, nullptr, w, y)) != IGA_OK) break;
    double b2 = 0.0;
    if ((rc = dot(w, y, &b2)) != IGA_OK) break;
    beta = std::sqrt(std::max(b2, 0.0));
    if (!(beta > 0.0)) break;
    be.push_back(beta);
    CK(cudaMemcpyAsync(vp, v, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    LK(launch_lincomb(s, N, 1.0 / beta, w, 0.0, w, v));
  }
  h->opt.tol = tol_save;
  CKS(rc);
  if (!(est > 0.0)) return fail(h, IGA_ENUMERIC, "non-positive eigenvalue estimate");
  *lambda_max = est;
  *tau_crit = std::sqrt(theta_crit(rho_inf) / est);
  return IGA_OK;
}


// ---------------------------------------------------------------------------
// learned warm start
// ---------------------------------------------------------------------------
namespace {

uint64_t splitmix64(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& state) { return (double)(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0); }

int ws_upload_params(iga_handle* h, const float* theta) {
  CKS(ensure_ws_step(h, 1));
  CK(cudaMemcpy(h->ws_theta, theta, sizeof(float) * IGA_NET_NPARAM, cudaMemcpyHostToDevice));
  CK(cudaMemset(h->ws_m, 0, sizeof(float) * IGA_NET_NPARAM));
  CK(cudaMemset(h->ws_v, 0, sizeof(float) * IGA_NET_NPARAM));
  h->ws_adam_t = 0;
  h->ws_params = true;
  return IGA_OK;
}

int net_args_ok(int n1, int n2, int n3, int nb) { return net_grid_ok(NetGrid{n1, n2, n3}, nb); }

}  // namespace

int iga_ws_init_params(iga_handle* h, unsigned long long seed) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_init_params"));
  std::vector<float> th(IGA_NET_NPARAM, 0.0f);
  uint64_t st = seed;
  const double b1 = 1.0 / std::sqrt(81.0), b2 = 1.0 / std::sqrt(432.0);
  for (int i = 0; i < 1296; ++i) th[i] = (float)((2.0 * uniform01(st) - 1.0) * b1);
  for (int i = 1312; i < 1744; ++i) th[i] = (float)((2.0 * uniform01(st) - 1.0) * b2);
  CKS(ws_upload_params(h, th.data()));
  h->ws_trained = false;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_ws_set_params(iga_handle* h, const float* theta_host) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_set_params"));
  if (!theta_host) return fail(h, IGA_EINVAL, "theta is NULL");
  CKS(ws_upload_params(h, theta_host));
  h->ws_trained = true;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_ws_get_params(iga_handle* h, float* theta_host) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_get_params"));
  if (!theta_host) return fail(h, IGA_EINVAL, "theta is NULL");
  if (!h->ws_params) return fail(h, IGA_EINVAL, "no parameters yet (iga_ws_init_params, iga_ws_train or iga_ws_set_params)");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(theta_host, h->ws_theta, sizeof(float) * IGA_NET_NPARAM, cudaMemcpyDeviceToHost));
  return IGA_OK;
}

int iga_ws_collect(iga_handle* h, int capacity) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_collect"));
  if (capacity < 0) return fail(h, IGA_EINVAL, "capacity < 0");
  CK(cudaStreamSynchronize(h->stream));
  dfree(h->ws_sx);
  dfree(h->ws_st);
  h->ws_cap = h->ws_count = 0;
  if (capacity == 0) return IGA_OK;
  CKS(dalloc(h, &h->ws_sx, (size_t)capacity * 3 * h->N));
  CKS(dalloc(h, &h->ws_st, (size_t)capacity * h->N));
  h->ws_cap = capacity;
  return IGA_OK;
}

int iga_ws_samples(iga_handle* h, int* count) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_samples"));
  if (!count) return fail(h, IGA_EINVAL, "count is NULL");
  *count = h->ws_count;
  return IGA_OK;
}

int iga_ws_train(iga_handle* h, int epochs, double lr, unsigned long long seed, double* epoch_loss) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_train"));
  if (epochs < 1 || !(lr > 0.0)) return fail(h, IGA_EINVAL, "epochs < 1 or lr <= 0");
  if (h->ws_count < 1) return fail(h, IGA_EINVAL, "no recorded samples (iga_ws_collect, then iga_step)");
  const NetGrid g = net_grid_of(h);
  if (!net_grid_ok(g, 1)) return fail(h, IGA_EINVAL, "grid beyond the network kernels' launch limits");
  if (!h->ws_params) CKS(iga_ws_init_params(h, seed));
  const long long N = h->N;
  const int ns = h->ws_count;
  const long long nupd = (long long)epochs * ns;
  if (!h->ws_y) {
    CKS(dalloc(h, &h->ws_y, (size_t)N));
    CKS(dalloc(h, &h->ws_dy, (size_t)N));
    CKS(dalloc(h, &h->ws_lpart, (size_t)kRedBlocks));
    void* w = nullptr;
    const cudaError_t e = cudaMalloc(&w, net_workspace_bytes(g, 1));
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, IGA_ENOMEM, "network workspace"); }
    h->ws_work = w;
  }
  if (h->ws_loss_cap < nupd) {
    CKS(dalloc(h, &h->ws_loss, (size_t)nupd));
    h->ws_loss_cap = nupd;
  }
  cudaStream_t s = h->stream;
  std::vector<int> order(ns);
  uint64_t st = seed ^ 0xA0761D6478BD642FULL;
  long long u = 0;
  for (int e = 0; e < epochs; ++e) {
    for (int i = 0; i < ns; ++i) order[i] = i;
    for (int i = ns - 1; i > 0; --i) {  // Fisher-Yates
      const int j = (int)(splitmix64(st) % (uint64_t)(i + 1));
      std::swap(order[i], order[j]);
    }
    for (int i = 0; i < ns; ++i, ++u) {
      const __nv_bfloat16* x = h->ws_sx + (size_t)order[i] * 3 * N;
      const float* t = h->ws_st + (size_t)order[i] * N;
      CK(launch_net_forward(s, g, 1, x, h->ws_theta, h->ws_act, h->ws_y, nullptr, nullptr, nullptr, &h->nlaunch));
      CK(launch_net_loss(s, N, h->ws_y, t, h->ws_dy, h->ws_lpart, h->ws_loss + u, &h->nlaunch));
      CK(launch_net_backward(s, g, 1, x, h->ws_theta, h->ws_act, h->ws_dy, h->ws_grad, h->ws_work, &h->nlaunch));
      const double lr_u = lr * 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)u / (double)nupd));
      CK(launch_net_adam(s, IGA_NET_NPARAM, h->ws_theta, h->ws_grad, h->ws_m, h->ws_v, ++h->ws_adam_t, lr_u,
                         &h->nlaunch));
    }
  }
  std::vector<double> L((size_t)nupd);
  CK(cudaMemcpyAsync(L.data(), h->ws_loss, sizeof(double) * nupd, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (epoch_loss)
    for (int e = 0; e < epochs; ++e) {
      double m = 0.0;
      for (int i = 0; i < ns; ++i) m += L[(size_t)e * ns + i];
      epoch_loss[e] = m / ns;
    }
  h->ws_trained = true;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_ws_features(iga_handle* h, int k, const double* b, double* b1, double* b2, double* z1, double* z2,
                    unsigned short* x, double* E, double* scales) {
  CKS(check_handle(h));
  CKS(single_patch(h, "iga_ws_features"));
  if (k < 1 || k > kMaxVec || !b || !b1 || !b2 || !z1 || !z2 || !x || !E || !scales)
    return fail(h, IGA_EINVAL, "bad arguments");
  CKS(ensure_ws_step(h, 1));
  cudaStream_t s = h->stream;
  CK(launch_ws_features(s, h->N, k, b, b1, b2, h->Dm, z1, z2, reinterpret_cast<__nv_bfloat16*>(x), E, h->ws_part,
                        h->ws_sc, &h->nlaunch));
  CK(cudaMemcpyAsync(scales, h->ws_sc, sizeof(double) * 2 * k, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return IGA_OK;
}

int iga_net_forward(int n1, int n2, int n3, int nb, const unsigned short* x, const float* theta,
                    unsigned short* act, float* y, void* stream) {
  if (!net_args_ok(n1, n2, n3, nb) || !x || !theta || !act || !y) return IGA_EINVAL;
  long long nl = 0;
  const cudaError_t e = launch_net_forward((cudaStream_t)stream, NetGrid{n1, n2, n3}, nb,
                                           reinterpret_cast<const __nv_bfloat16*>(x), theta,
                                           reinterpret_cast<__nv_bfloat16*>(act), y, nullptr, nullptr, nullptr, &nl);
  return e == cudaSuccess ? IGA_OK : IGA_ECUDA;
}

unsigned long long iga_net_workspace_bytes(int n1, int n2, int n3, int nb) {
  if (!net_args_ok(n1, n2, n3, nb)) return 0;
  return net_workspace_bytes(NetGrid{n1, n2, n3}, nb);
}

int iga_net_backward(int n1, int n2, int n3, int nb, const unsigned short* x, const float* theta,
                     const unsigned short* act, const float* dy, float* grad, void* work,
                     unsigned long long work_bytes, void* stream) {
  if (!net_args_ok(n1, n2, n3, nb) || !x || !theta || !act || !dy || !grad || !work) return IGA_EINVAL;
  const NetGrid g{n1, n2, n3};
  if (work_bytes < net_workspace_bytes(g, nb)) return IGA_EINVAL;
  long long nl = 0;
  const cudaError_t e = launch_net_backward((cudaStream_t)stream, g, nb, reinterpret_cast<const __nv_bfloat16*>(x),
                                            theta, reinterpret_cast<const __nv_bfloat16*>(act), dy, grad, work, &nl);
  return e == cudaSuccess ? IGA_OK : IGA_ECUDA;
}

int iga_net_adam(int n, float* theta, const float* grad, float* m, float* v, int step, double lr, void* stream) {
  if (n < 1 || step < 1 || !(lr > 0.0) || !theta || !grad || !m || !v) return IGA_EINVAL;
  long long nl = 0;
  const cudaError_t e = launch_net_adam((cudaStream_t)stream, n, theta, grad, m, v, step, lr, &nl);
  return e == cudaSuccess ? IGA_OK : IGA_ECUDA;
}


// ---------------------------------------------------------------------------
// launch tuning and batches of independent patches
// ---------------------------------------------------------------------------
int iga_set_band_config(iga_handle* h, int threads, int nv) {
  CKS(check_handle(h));
  if (!(threads == 0 || threads == 64 || threads == 96 || threads == 128 || threads == 256 || threads == 512) ||
      nv < 0 || nv > 4)
    return fail(h, IGA_EINVAL, "threads must be 0, 64, 96, 128, 256 or 512 and nv 0..4");
  if (h->mp)
    for (iga_handle* p : h->mp->patch) {
      p->band_threads = threads;
      p->band_nv = nv;
    }
  h->band_threads = threads;
  h->band_nv = nv;
  drop_step_graph(h);
  return IGA_OK;
}

int iga_autotune(iga_handle* h, int nvec, int reps, int* threads, int* nv) {
  CKS(check_handle(h));
  if (h->mp) {  // every patch picks its own shape; the outputs are the last patch's
    for (size_t r = 0; r < h->mp->patch.size(); ++r) {
      iga_handle* p = h->mp->patch[r];
      p->stream = h->stream;
      const int rc = iga_autotune(p, nvec, reps, threads, nv);
      if (rc != IGA_OK) return fail(h, rc, "patch " + std::to_string(r) + ": " + p->err);
    }
    drop_step_graph(h);
    return IGA_OK;
  }
  if (nvec < 1 || nvec > kMaxVec || reps < 1) return fail(h, IGA_EINVAL, "need 1 <= nvec <= 8 and reps >= 1");
  CKS(assemble_band(h));
  CKS(ensure_cg_ws(h, nvec));
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->p, 0, sizeof(double) * nvec * h->N, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  const cudaError_t ec = cudaEventCreate(&e1);
  if (ec != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(h, IGA_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ec));
  }
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } ev{e0, e1};
  const int cand_t[5] = {64, 96, 128, 256, 512};
  const int cand_v[4] = {1, 2, 3, 4};
  struct Cand {
    int t, v;
    float ms;
  };
  std::vector<Cand> res;
  for (int ti = 0; ti < 5; ++ti)
    for (int vi = 0; vi < 4; ++vi) {
      if (cand_t[ti] == 96 && h->opt.op_form != IGA_OP_ASSEMBLED_DF) continue;  // a double-FP32 shape only
      const int v = std::min(cand_v[vi], nvec);
      if (vi > 0 && v == std::min(cand_v[vi - 1], nvec)) continue;  // same as the previous candidate
      LK(launch_band(h, s, IGA_PROF_BAND_MASS, nvec, nullptr, h->p, h->q, cand_t[ti], v, nullptr, nullptr));
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r)
        LK(launch_band(h, s, IGA_PROF_BAND_MASS, nvec, nullptr, h->p, h->q, cand_t[ti], v, nullptr, nullptr));
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      res.push_back({cand_t[ti], v, ms});
    }
  // the fastest; among shapes within 3 % of it, the most vectors per thread (each
  // coefficient read once for more vectors: fewer DRAM bytes for the same time)
  float best = 1e30f;
  for (const Cand& c : res) best = std::min(best, c.ms);
  int best_t = 256, best_v = 0;
  float best_ms = 1e30f;
  for (const Cand& c : res)
    if (c.ms <= 1.03f * best && (c.v > best_v || (c.v == best_v && c.ms < best_ms))) {
      best_t = c.t;
      best_v = c.v;
      best_ms = c.ms;
    }
  h->band_threads = best_t;
  h->band_nv = best_v;
  drop_step_graph(h);
  if (threads) *threads = best_t;
  if (nv) *nv = best_v;
  return check_tc_error(h);
}

}  // extern "C"
