// Batches of independent patches (iga_batch_*, include/iga_galpha.h): one captured
// graph holding every patch's step.
#include <new>
#include <string>
#include <vector>

#include "handle.h"

using namespace iga;

struct iga_batch {
  std::vector<iga_handle*> p;
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

void drop_batch_graph(iga_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->gvalid = false;
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
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

const char* iga_batch_last_error(const iga_batch* b) { return b ? b->err.c_str() : ""; }

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
