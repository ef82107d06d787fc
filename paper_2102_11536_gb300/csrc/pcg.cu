// Batched PCG (Sec. 5.5) over the k stage systems of a step, split into launch-only
// pieces that serve both the host-driven loop and the captured graph, and the host-driven
// loop itself.
#include <cstdio>
#include <string>

#include "handle.h"

namespace iga {

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

}  // namespace iga
