// The learned initial guess of PCG (iga_ws_*, include/iga_galpha.h): the network's
// parameters, the collection of training samples from the method's own solves, training by
// the library's forward, backward and Adam kernels (kernels_net.cu), and the stand-alone
// network calls (iga_net_*).
#include "handle.h"

using namespace iga;

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


