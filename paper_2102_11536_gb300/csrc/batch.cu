// Batches of independent patches (iga_batch_*, include/iga_galpha.h): one captured
// graph holding every patch's step, or (iga_batch_set_persistent) one persistent
// cooperative launch per batch step over all patches (kernels_persist.cu).
#include <cuda_bf16.h>

#include <new>
#include <string>
#include <vector>

#include "handle.h"

using namespace iga;

// Device state of the persistent batch step: tables, work vectors, scalars, the graph
// holding its launch, and the key (k, rho, dt, states) they were built for.
struct PersistState {
  int k = 0;
  double rho = -1.0;
  std::vector<double> dt;
  std::vector<double*> states;
  bool f32 = false;
  size_t smem = 0;
  int grid[kPersistVariants] = {};
  PBatch B{};
  std::vector<void*> allocs;  // every device allocation, freed together
  cudaGraph_t graph[kPersistVariants] = {};
  cudaGraphExec_t gexec[kPersistVariants] = {};
  int nvariants = 1;                        // variants built (the second only for k <= 2)
  double phase_ms[kPersistPhases] = {};  // of the last iga_batch_step, summed over its steps
  bool have_phases = false;
};

// Launch variant of the persistent step (kernels_persist.cu: blocks per SM and slots per
// band pass): forced, or chosen by timing the first steps of the batch -- each variant
// twice, alternating -- and taking the faster one. Kept across rebuilds of the state.
struct PersistTuning {
  int force = -1;            // -1: choose by timing
  int chosen = -1;           // the variant in use once chosen
  double ms[kPersistVariants] = {-1.0, -1.0};  // best timed step per variant
  int samples[kPersistVariants] = {0, 0};
  cudaEvent_t ev[2 * kPersistVariants] = {};
};

struct iga_batch {
  std::vector<iga_handle*> p;
  bool persistent = false;
  PersistState* ps = nullptr;
  PersistTuning tune;
  int device = 0;
  cudaStream_t s0 = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool gvalid = false;
  std::vector<iga_handle::GraphKey> keys;
  std::vector<long long> gens;
  std::string err;
};

namespace {

int bfail(iga_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

#define CKB(expr)                \
  do {                           \
    const int s_ = (expr);       \
    if (s_ != IGA_OK) return s_; \
  } while (0)

void drop_batch_graph(iga_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->gvalid = false;
}

void free_persist(PersistState* ps) {
  if (!ps) return;
  for (int v = 0; v < kPersistVariants; ++v) {
    if (ps->gexec[v]) cudaGraphExecDestroy(ps->gexec[v]);
    if (ps->graph[v]) cudaGraphDestroy(ps->graph[v]);
  }
  for (void* a : ps->allocs) cudaFree(a);
  delete ps;
}

// The forms the persistent step computes: 3-D patches, FP64 band operators, the
// band-Cholesky Kronecker preconditioner (all patches FP64 or all FP32) or the BF16 fast
// diagonalisation, zero initial guess, no damping or loads, common tolerance and
// iteration limit, degrees 1..4.
int persist_supported(iga_batch* b) {
  const iga_handle* h0 = b->p[0];
  for (size_t i = 0; i < b->p.size(); ++i) {
    const iga_handle* h = b->p[i];
    const std::string who = "patch " + std::to_string(i) + ": ";
    if (h->dim != 3) return bfail(b, IGA_EINVAL, who + "the persistent batch step needs 3-D patches");
    if (h->opt.op_form != IGA_OP_ASSEMBLED)
      return bfail(b, IGA_EINVAL, who + "the persistent batch step needs the FP64 band operators (IGA_OP_ASSEMBLED)");
    if (h->opt.precond != IGA_PREC_BANDED && h->opt.precond != IGA_PREC_BANDED32 && h->opt.precond != IGA_PREC_BF16)
      return bfail(b, IGA_EINVAL,
                   who + "the persistent batch step needs a band-Cholesky Kronecker or the BF16 preconditioner");
    if (h->opt.precond != h0->opt.precond || h->opt.tol != h0->opt.tol || h->opt.max_iter != h0->opt.max_iter)
      return bfail(b, IGA_EINVAL, who + "preconditioner, tolerance and iteration limit must be those of patch 0");
    if (h->opt.guess != IGA_GUESS_ZERO || h->damped || h->nforce > 0)
      return bfail(b, IGA_EINVAL, who + "the persistent batch step needs the zero guess, no damping and no loads");
    for (int a = 0; a < 3; ++a)
      if (h->dd[a].p < 1 || h->dd[a].p > 4) return bfail(b, IGA_EINVAL, who + "degrees 1..4 only");
  }
  return IGA_OK;
}

template <typename T>
int palloc(iga_batch* b, PersistState* ps, T** out, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, IGA_ENOMEM, "persistent batch: cudaMalloc");
  }
  ps->allocs.push_back(q);
  *out = static_cast<T*>(q);
  return IGA_OK;
}

template <typename T>
int pupload(iga_batch* b, PersistState* ps, T** out, const std::vector<T>& v) {
  CKB(palloc(b, ps, out, v.size()));
  if (cudaMemcpy(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, IGA_ECUDA, "persistent batch: cudaMemcpy");
  return IGA_OK;
}

// Tables, work vectors and scalars of the persistent step for (k, rho, dt, states), and
// the graph holding its one launch.
int build_persist(iga_batch* b, double* const* states, int k, double rho, const double* dt) {
  free_persist(b->ps);
  b->ps = nullptr;
  CKB(persist_supported(b));
  const int np = (int)b->p.size();
  for (int i = 0; i < np; ++i) {
    iga_handle* h = b->p[i];
    h->stream = b->p[i]->stream;
    const int rc = assemble_band(h);
    if (rc != IGA_OK) return bfail(b, rc, "patch " + std::to_string(i) + ": " + h->err);
  }
  PersistState* ps = new (std::nothrow) PersistState;
  if (!ps) return bfail(b, IGA_ENOMEM, "persistent batch: host allocation");
  b->ps = ps;
  ps->k = k;
  ps->rho = rho;
  ps->dt.assign(dt, dt + np);
  ps->states.assign(states, states + np);
  const bool fd = b->p[0]->opt.precond == IGA_PREC_BF16;
  ps->f32 = fd || b->p[0]->opt.precond == IGA_PREC_BANDED32;
  const size_t esz = ps->f32 ? sizeof(float) : sizeof(double);
  std::vector<PPatch> pt(np);
  std::vector<int2> rtile, ltile[3];
  std::vector<int> rt0(np), nrt(np), lt2(np), nlt2(np);
  std::vector<double*> Yp(np), rp(np), pp(np), qp(np);
  int nmax = 1, pmax = 1;
  for (int i = 0; i < np; ++i) {
    iga_handle* h = b->p[i];
    PPatch& P = pt[i];
    P.N = h->N;
    P.H = h->band_H;
    for (int a = 0; a < 3; ++a) {
      P.n[a] = h->n[a];
      P.deg[a] = h->dd[a].p;
      P.L[a] = ps->f32 ? (const void*)h->dd[a].chol32 : (const void*)h->dd[a].chol;
      P.dinv[a] = ps->f32 ? (const void*)h->dd[a].cdinv32 : (const void*)h->dd[a].cdinv;
      nmax = std::max(nmax, h->n[a]);
      pmax = std::max(pmax, h->dd[a].p);
    }
    P.M = h->Mband;
    P.K = h->Kband;
    P.off = h->band_off;
    P.o12 = h->band_o12;
    P.scale = h->scale;
    P.X = states[i];
    const size_t kn = (size_t)k * h->N;
    double** vec[7] = {&P.Y, &P.T, &P.r, &P.x, &P.z, &P.p, &P.q};
    for (double** v : vec) CKB(palloc(b, ps, v, kn));
    char* t = nullptr;
    CKB(palloc(b, ps, &t, 2 * kn * esz));
    P.t1 = t;
    P.t2 = t + kn * esz;
    P.sc = handle_coefs(h, k, rho, dt[i]);
    for (int a = 0; a < 3; ++a) {
      P.lam[a] = h->dd[a].lam32;
      P.Ubf[a][0] = P.Ubf[a][1] = nullptr;
      if (!fd) continue;
      // U_a (column c = eigenvector c of the parametric mass matrix) and U_a^T in BF16, each as
      // the image the mode products copy into shared memory: ceil16(n) rows of ceil16(n) +
      // kPersistFdPad entries, zero beyond n
      const int n = h->tab[a].n, n16 = (n + 15) & ~15, ld = n16 + kPersistFdPad;
      const std::vector<double>& ev = h->tab[a].evec;
      std::vector<__nv_bfloat16> mu((size_t)n16 * ld, __float2bfloat16(0.0f)), mt((size_t)n16 * ld, __float2bfloat16(0.0f));
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          mu[(size_t)r * ld + c] = __float2bfloat16((float)ev[(size_t)r * n + c]);
          mt[(size_t)r * ld + c] = __float2bfloat16((float)ev[(size_t)c * n + r]);
        }
      __nv_bfloat16 *du = nullptr, *dt_ = nullptr;
      CKB(pupload(b, ps, &du, mu));
      CKB(pupload(b, ps, &dt_, mt));
      P.Ubf[a][0] = du;
      P.Ubf[a][1] = dt_;
    }
    rt0[i] = (int)rtile.size();
    nrt[i] = batch_row_tiles(h->N);
    for (int q = 0; q < nrt[i]; ++q) rtile.push_back(make_int2(i, q));
    const int last = fd ? 0 : 2;  // the axis of the preconditioner's last phase (its r.z partials)
    for (int a = 0; a < 3; ++a) {
      if (a == last) lt2[i] = (int)ltile[a].size();
      const int nl = batch_line_tiles(h->N, h->n[a]);
      if (a == last) nlt2[i] = nl;
      for (int q = 0; q < nl; ++q) ltile[a].push_back(make_int2(i, q));
    }
    Yp[i] = P.Y;
    rp[i] = P.r;
    pp[i] = P.p;
    qp[i] = P.q;
  }
  PBatch& B = ps->B;
  B.np = np;
  B.k = k;
  B.max_iter = b->p[0]->opt.max_iter;
  B.flexible = ps->f32 ? 1 : 0;
  B.fd = fd ? 1 : 0;
  B.tol2 = b->p[0]->opt.tol * b->p[0]->opt.tol;
  B.nrt = (int)rtile.size();
  PPatch* dpt = nullptr;
  CKB(pupload(b, ps, &dpt, pt));
  B.pt = dpt;
  int2* drt = nullptr;
  CKB(pupload(b, ps, &drt, rtile));
  B.rtile = drt;
  for (int a = 0; a < 3; ++a) {
    int2* d = nullptr;
    CKB(pupload(b, ps, &d, ltile[a]));
    B.ltile[a] = d;
    B.nlt[a] = (int)ltile[a].size();
  }
  int *d_rt0 = nullptr, *d_nrt = nullptr, *d_lt2 = nullptr, *d_nlt2 = nullptr;
  CKB(pupload(b, ps, &d_rt0, rt0));
  CKB(pupload(b, ps, &d_nrt, nrt));
  CKB(pupload(b, ps, &d_lt2, lt2));
  CKB(pupload(b, ps, &d_nlt2, nlt2));
  B.rt0 = d_rt0;
  B.nrt_p = d_nrt;
  B.lt2 = d_lt2;
  B.nlt2_p = d_nlt2;
  double** dptr[4] = {nullptr, nullptr, nullptr, nullptr};
  const std::vector<double*>* src[4] = {&Yp, &rp, &pp, &qp};
  for (int q = 0; q < 4; ++q) CKB(pupload(b, ps, &dptr[q], *src[q]));
  B.Yp = dptr[0];
  B.rp = dptr[1];
  B.pp = dptr[2];
  B.qp = dptr[3];
  const size_t S = (size_t)np * k;
  CKB(palloc(b, ps, &B.part, (size_t)B.nrt * k));
  B.nrzt = B.nlt[fd ? 0 : 2];
  CKB(palloc(b, ps, &B.lpart, (size_t)2 * B.nrzt * k));
  double** sc[9] = {&B.bb, &B.rr, &B.rz, &B.rznew, &B.rzold, &B.pq, &B.alpha, &B.beta, &B.last_rel};
  for (double** v : sc) CKB(palloc(b, ps, v, S));
  int** si[4] = {&B.active, &B.iters, &B.status, &B.max_iters};
  for (int** v : si) CKB(palloc(b, ps, v, S));
  CKB(palloc(b, ps, &B.tot_iters, S));
  CKB(palloc(b, ps, &B.flags, 2));
  CKB(palloc(b, ps, &B.bar, 2));
  CKB(palloc(b, ps, &B.err, 1));
  CKB(palloc(b, ps, &B.ptime, kPersistPhases));
  // polls of a barrier wait before it gives up (< 0 on the handle: the default, about 0.3 s or
  // more, far beyond the longest phase)
  B.bar_limit = b->p[0]->bar_limit < 0 ? (1LL << 22) : b->p[0]->bar_limit;
  if (cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned int), b->s0) != cudaSuccess ||
      cudaMemsetAsync(B.err, 0, sizeof(int), b->s0) != cudaSuccess ||
      cudaMemsetAsync(B.status, 0, sizeof(int) * S, b->s0) != cudaSuccess ||
      cudaMemsetAsync(B.beta, 0, sizeof(double) * S, b->s0) != cudaSuccess)
    return bfail(b, IGA_ECUDA, "persistent batch: cudaMemsetAsync");
  ps->smem = batch_smem_bytes(nmax, pmax, k, ps->f32, fd);
  // one graph per launch variant, each holding the one cooperative launch of a batch step
  ps->nvariants = k <= 2 ? kPersistVariants : 1;
  for (int v = 0; v < ps->nvariants; ++v) {
    cudaError_t e = cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, IGA_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    const cudaError_t le = launch_batch_step(b->s0, B, ps->f32, ps->smem, v, &ps->grid[v]);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->s0, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return bfail(b, IGA_ECUDA, std::string("persistent batch launch: ") +
                                     cudaGetErrorString(le != cudaSuccess ? le : ee));
    }
    ps->graph[v] = g;
    e = cudaGraphInstantiate(&ps->gexec[v], g, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, IGA_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
  }
  return IGA_OK;
}

bool persist_current(const iga_batch* b, double* const* states, int k, double rho, const double* dt) {
  const PersistState* ps = b->ps;
  if (!ps || !ps->gexec[0] || ps->k != k || ps->rho != rho) return false;
  for (size_t i = 0; i < b->p.size(); ++i)
    if (ps->states[i] != states[i] || ps->dt[i] != dt[i] || b->p[i]->ws_gen < 0) return false;
  return true;
}

// nsteps batch steps, one graph launch (one persistent kernel) each
int persist_steps(iga_batch* b, double* const* states, int k, double rho, const double* dt, int nsteps,
                  iga_stats* stats) {
  if (!persist_current(b, states, k, rho, dt)) CKB(build_persist(b, states, k, rho, dt));
  PersistState* ps = b->ps;
  const PBatch& B = ps->B;
  const int np = (int)b->p.size();
  const size_t S = (size_t)np * k;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < np && e == cudaSuccess; ++i) {  // after earlier work on every patch's stream
    e = cudaEventRecord(b->p[i]->ev_in ? b->p[i]->ev_in : b->join[i], b->p[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s0, b->p[i]->ev_in ? b->p[i]->ev_in : b->join[i], 0);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(B.tot_iters, 0, sizeof(long long) * S, b->s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.max_iters, 0, sizeof(int) * S, b->s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.flags, 0, sizeof(int) * 2, b->s0);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.ptime, 0, sizeof(unsigned long long) * kPersistPhases, b->s0);
  // the variant of every launch; the timed ones (at most one per variant per call) between events
  PersistTuning& tu = b->tune;
  int timed[kPersistVariants] = {0, 0};
  for (int t = 0; t < nsteps && e == cudaSuccess; ++t) {
    int v = tu.force >= 0 ? tu.force : tu.chosen;
    bool time_it = false;
    if (v < 0) {  // still choosing: the variant with the fewest samples (two each), alternating
      v = 0;
      for (int q = 1; q < ps->nvariants; ++q)
        if (tu.samples[q] < tu.samples[v]) v = q;
      time_it = timed[v] == 0;
    }
    if (v >= ps->nvariants) v = 0;
    if (time_it) {
      for (int q = 0; q < 2 && e == cudaSuccess; ++q)
        if (!tu.ev[2 * v + q]) e = cudaEventCreate(&tu.ev[2 * v + q]);
      if (e == cudaSuccess) e = cudaEventRecord(tu.ev[2 * v], b->s0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(ps->gexec[v], b->s0);
    if (time_it && e == cudaSuccess) {
      e = cudaEventRecord(tu.ev[2 * v + 1], b->s0);
      timed[v] = 1;
      ++tu.samples[v];  // counted when launched, read after the synchronisation below
    }
  }
  std::vector<long long> tot(S);
  std::vector<int> mx(S), st(S);
  std::vector<double> rel(S);
  int err = 0, flags[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot.data(), B.tot_iters, sizeof(long long) * S, cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mx.data(), B.max_iters, sizeof(int) * S, cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rel.data(), B.last_rel, sizeof(double) * S, cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st.data(), B.status, sizeof(int) * S, cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, B.err, sizeof(int), cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, B.flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->s0);
  unsigned long long pns[kPersistPhases] = {};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pns, B.ptime, sizeof(unsigned long long) * kPersistPhases, cudaMemcpyDeviceToHost, b->s0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->s0);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, b->s0);
  for (int i = 0; i < np && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->p[i]->stream, b->done, 0);
  if (e != cudaSuccess) return bfail(b, IGA_ECUDA, std::string("persistent batch step: ") + cudaGetErrorString(e));
  for (int c = 0; c < kPersistPhases; ++c) ps->phase_ms[c] = 1e-6 * (double)pns[c];
  ps->have_phases = !err;
  for (int v = 0; v < kPersistVariants && !err; ++v) {
    if (!timed[v]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, tu.ev[2 * v], tu.ev[2 * v + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (tu.ms[v] < 0.0 || ms < tu.ms[v]) tu.ms[v] = ms;
  }
  if (tu.chosen < 0 && tu.force < 0) {  // every variant sampled twice: keep the faster
    bool done = true;
    for (int v = 0; v < ps->nvariants; ++v) done = done && tu.samples[v] >= 2 && tu.ms[v] >= 0.0;
    if (done) {
      tu.chosen = 0;
      for (int v = 1; v < ps->nvariants; ++v)
        if (tu.ms[v] < tu.ms[tu.chosen]) tu.chosen = v;
    }
  }
  if (err) {  // a barrier wait ran out: the step's results are not to be used; start the words afresh
    cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned int), b->s0);
    cudaMemsetAsync(B.err, 0, sizeof(int), b->s0);
    cudaStreamSynchronize(b->s0);
    return bfail(b, IGA_ECUDA, "persistent batch step: a grid barrier wait timed out");
  }
  for (int i = 0; i < np; ++i) {
    iga_handle* h = b->p[i];
    for (int t = 0; t < nsteps; ++t) h->time += dt[i];
    if (!stats) continue;
    iga_stats& s = stats[i];
    s.steps += nsteps;
    s.solves += (long long)k * nsteps;
    for (int j = 0; j < k; ++j) {
      s.iters += tot[(size_t)i * k + j];
      s.max_iters = std::max(s.max_iters, mx[(size_t)i * k + j]);
      s.max_relres = std::max(s.max_relres, rel[(size_t)i * k + j]);
    }
  }
  if (stats) stats[0].launches += nsteps;  // one launch advances the whole batch
  for (size_t q = 0; q < S; ++q) {
    if (st[q] == 1) return bfail(b, IGA_ENUMERIC, "patch " + std::to_string(q / k) + ": PCG breakdown");
    if (st[q] == 2) return bfail(b, IGA_ENOT_CONVERGED, "patch " + std::to_string(q / k) + ": PCG did not converge");
  }
  return IGA_OK;
}

bool needs_host_loop(const iga_handle* h) {
  const int g = h->opt.guess;
  return !h->use_graphs || h->prof_class != IGA_PROF_OFF || (g == IGA_GUESS_LEARNED && h->ws_cap > 0) ||
         !(g == IGA_GUESS_ZERO || g == IGA_GUESS_TAYLOR || h->hist >= 2);
}

// One graph: fork from b->s0 to every patch's capture stream, each patch's step,
// join back on b->s0.
int build_batch_graph(iga_batch* b, double* const* states, int k, double rho, const double* dt) {
  drop_batch_graph(b);
  const int np = (int)b->p.size();
  for (int i = 0; i < np; ++i) {
    const int rc = prepare_capture(b->p[i], k);
    if (rc != IGA_OK) return bfail(b, rc, "patch " + std::to_string(i) + ": " + b->p[i]->err);
  }
  cudaError_t e = cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, IGA_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  int rc = IGA_OK;
  std::string msg;
  e = cudaEventRecord(b->fork, b->s0);
  for (int i = 0; i < np && rc == IGA_OK && e == cudaSuccess; ++i) {
    iga_handle* h = b->p[i];
    e = cudaStreamWaitEvent(h->gs, b->fork, 0);
    if (e != cudaSuccess) break;
    rc = capture_step(h, states[i], k, handle_coefs(h, k, rho, dt[i]));
    if (rc != IGA_OK) {
      msg = "patch " + std::to_string(i) + ": " + h->err;
      break;
    }
    e = cudaEventRecord(b->join[i], h->gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s0, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->s0, &g);
  if (rc != IGA_OK || e != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (rc != IGA_OK) return bfail(b, rc, msg);
    return bfail(b, IGA_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ee));
  }
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return bfail(b, IGA_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  b->graph = g;
  b->gexec = ge;
  b->gvalid = true;
  b->keys.resize(np);
  b->gens.resize(np);
  for (int i = 0; i < np; ++i) {
    b->keys[i] = graph_key(b->p[i], states[i], k, rho, dt[i]);
    b->gens[i] = b->p[i]->ws_gen;
  }
  return IGA_OK;
}

bool batch_graph_current(const iga_batch* b, double* const* states, int k, double rho, const double* dt) {
  if (!b->gvalid) return false;
  for (size_t i = 0; i < b->p.size(); ++i)
    if (!same_key(b->keys[i], graph_key(b->p[i], states[i], k, rho, dt[i])) || b->gens[i] != b->p[i]->ws_gen)
      return false;
  return true;
}

}  // namespace

extern "C" {

int iga_batch_create(int npatch, iga_handle* const* patches, iga_batch** out) {
  if (!out) return IGA_EINVAL;
  *out = nullptr;
  if (npatch < 1 || !patches) return IGA_EINVAL;
  for (int i = 0; i < npatch; ++i)
    if (!patches[i] || patches[i]->mp || patches[i]->opt.device != patches[0]->opt.device) return IGA_EINVAL;
  iga_batch* b = new (std::nothrow) iga_batch;
  if (!b) return IGA_ENOMEM;
  b->p.assign(patches, patches + npatch);
  b->device = patches[0]->opt.device;
  b->join.assign(npatch, nullptr);
  bool ok = cudaSetDevice(b->device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < npatch; ++i)
    ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    iga_batch_destroy(b);
    return IGA_ECUDA;
  }
  *out = b;
  return IGA_OK;
}

void iga_batch_destroy(iga_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->s0) cudaStreamSynchronize(b->s0);
  drop_batch_graph(b);
  free_persist(b->ps);
  for (auto e : b->tune.ev)
    if (e) cudaEventDestroy(e);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

const char* iga_batch_last_error(const iga_batch* b) { return b ? b->err.c_str() : ""; }

int iga_batch_set_persistent(iga_batch* b, int on) {
  if (!b) return IGA_EINVAL;
  b->err.clear();
  if (on) CKB(persist_supported(b));
  b->persistent = on != 0;
  if (!on) {
    free_persist(b->ps);
    b->ps = nullptr;
  }
  return IGA_OK;
}

int iga_batch_set_persistent_variant(iga_batch* b, int variant) {
  if (!b) return IGA_EINVAL;
  b->err.clear();
  if (variant < -1 || variant >= kPersistVariants) return bfail(b, IGA_EINVAL, "variant must be -1, 0 or 1");
  b->tune.force = variant;
  return IGA_OK;
}

int iga_batch_persistent_variant(iga_batch* b, int* variant, double* ms) {
  if (!b) return IGA_EINVAL;
  b->err.clear();
  if (variant) *variant = b->tune.force >= 0 ? b->tune.force : b->tune.chosen;
  if (ms)
    for (int v = 0; v < kPersistVariants; ++v) ms[v] = b->tune.ms[v];
  return IGA_OK;
}

int iga_batch_phase_times(iga_batch* b, double* ms, int n) {
  if (!b) return IGA_EINVAL;
  b->err.clear();
  if (!ms || n < 1) return bfail(b, IGA_EINVAL, "bad arguments");
  if (!b->persistent || !b->ps || !b->ps->have_phases)
    return bfail(b, IGA_EINVAL, "no persistent batch step has completed since the persistent step was set up");
  for (int c = 0; c < n; ++c) ms[c] = c < kPersistPhases ? b->ps->phase_ms[c] : 0.0;
  return IGA_OK;
}

int iga_batch_step(iga_batch* b, double* const* states, int k, double rho_inf, const double* dt, int nsteps,
                   iga_stats* stats) {
  if (!b) return IGA_EINVAL;
  b->err.clear();
  const int np = (int)b->p.size();
  if (!states || !dt || k < 1 || k > kMaxK || nsteps < 0 || !(rho_inf >= 0.0 && rho_inf <= 1.0))
    return bfail(b, IGA_EINVAL, "bad arguments");
  for (int i = 0; i < np; ++i)
    if (!states[i] || !(dt[i] > 0.0)) return bfail(b, IGA_EINVAL, "patch " + std::to_string(i) + ": bad state or dt");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, IGA_ECUDA, "cudaSetDevice");
  if (b->persistent) return nsteps > 0 ? persist_steps(b, states, k, rho_inf, dt, nsteps, stats) : IGA_OK;
  int done = 0;
  auto host_steps = [&](int n) -> int {  // every patch through iga_step, one step at a time
    for (int t = 0; t < n; ++t)
      for (int i = 0; i < np; ++i) {
        const int rc = iga_step(b->p[i], states[i], k, rho_inf, dt[i], 1, stats ? &stats[i] : nullptr);
        if (rc != IGA_OK) return bfail(b, rc, "patch " + std::to_string(i) + ": " + b->p[i]->err);
      }
    return IGA_OK;
  };
  while (done < nsteps) {
    bool any = false;
    for (auto* h : b->p) any = any || needs_host_loop(h);
    if (!any) break;
    const int rc = host_steps(1);
    if (rc != IGA_OK) return rc;
    ++done;
  }
  const int n = nsteps - done;
  if (n == 0) return IGA_OK;
  if (!batch_graph_current(b, states, k, rho_inf, dt)) {
    const int rc = build_batch_graph(b, states, k, rho_inf, dt);
    if (rc != IGA_OK) return rc;
  }
  std::vector<long long> l0(np);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    iga_handle* h = b->p[i];
    l0[i] = h->nlaunch;
    if (reset_graph_counters(h, b->s0) != IGA_OK) return bfail(b, IGA_ECUDA, h->err);
    e = cudaEventRecord(h->ev_in, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s0, h->ev_in, 0);
  }
  for (int t = 0; t < n && e == cudaSuccess; ++t) e = cudaGraphLaunch(b->gexec, b->s0);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, b->s0);
  for (int i = 0; i < np && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->p[i]->stream, b->done, 0);
  if (e != cudaSuccess) return bfail(b, IGA_ECUDA, std::string("batch replay: ") + cudaGetErrorString(e));
  int first = IGA_OK;
  for (int i = 0; i < np; ++i) {
    iga_handle* h = b->p[i];
    const int rc = collect_graph_run(h, b->s0, k, n, dt[i], stats ? &stats[i] : nullptr);
    if (stats) stats[i].launches += h->nlaunch - l0[i];
    if (rc != IGA_OK && first == IGA_OK) {
      first = rc;
      b->err = "patch " + std::to_string(i) + ": " + h->err;
    }
  }
  return first;
}

}  // extern "C"
