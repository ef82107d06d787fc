// The multi-patch system on the GPU (iga_mp_*, include/iga_multipatch.h): conforming
// patches glued by the host layout (host_multipatch.cpp), one handle per patch over its
// index box, and the system handle whose M, K and additive Schwarz preconditioner act
// through the patches (gather, each patch's own operator, ordered scatter-add:
// kernels_mp.cu); the stepping, solve and CFL calls of the single-patch handle run on it.
#include <string>
#include <vector>

#include "handle.h"

using namespace iga;

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

