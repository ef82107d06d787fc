// C ABI of the GB300 explicit generalized-alpha IGA library (include/iga_galpha.h): handle
// creation and set-up (tables, geometry, diagonal scaling), options, the step-parameter
// helpers, the time step (predictor, stage right-hand sides, the k PCG solves, update) in the
// host-driven loop or as a captured CUDA graph with the PCG loop on the device, initial
// data, fields at the Gauss points, the critical step, profiling and launch tuning. The
// operators are in operators.cu, PCG in pcg.cu, the learned guess in warmstart.cu, the
// multi-patch system in multipatch.cu, batches in batch.cu.
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
  dfree(h->Mdf); dfree(h->Kdf); dfree(h->band_runs); dfree(h->band_runs_k); dfree(h->df_xs); dfree(h->df_E); dfree(h->df_part); dfree(h->df_bar);
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

int iga_band_df_tiny(iga_handle* h, double* frac_m, double* frac_k) {
  CKS(check_handle(h));
  if (h->mp) return fail(h, IGA_EINVAL, "iga_band_df_tiny takes a single patch (iga_mp_patch lends one)");
  if (h->opt.op_form != IGA_OP_ASSEMBLED_DF) return fail(h, IGA_EINVAL, "the handle's form is not IGA_OP_ASSEMBLED_DF");
  CKS(assemble_band(h));
  if (frac_m) *frac_m = h->df_tiny_m;
  if (frac_k) *frac_k = h->df_tiny_k;
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
