// Internal definitions shared by the C-ABI translation units of the library: the
// handle of one patch (or of a multi-patch system), the checked-call macros, the
// device allocation helpers and the internal routines that more than one unit uses.
#pragma once
#include <string>
#include <vector>

#include "iga_internal.h"

// the handle types are global (the C ABI's opaque iga_handle) and built from iga's types
using namespace iga;

struct MpState;

struct iga_handle {
  int dim = 0;
  iga_options opt{};
  cudaStream_t stream = nullptr;
  Tables1D tab[3];
  DirDev dd[3]{};
  int n[3] = {1, 1, 1}, Q[3] = {1, 1, 1}, m[3] = {1, 1, 1};
  long long N = 0, Qt = 0;
  double* ctrl = nullptr;   // SoA control net
  double* W = nullptr;      // [Qt]
  double* G = nullptr;      // [ng][Qt]
  long long gstride = 0;
  double* Dm = nullptr;     // diag(M)
  double* scale = nullptr;  // D^{-1/2} Dhat^{1/2}
  float* scale32 = nullptr; // the same rounded to FP32 (the FP32 band-Cholesky solve scales in FP32)
  int* dflag = nullptr;     // device scratch flag
  // assembled form
  double* Mband = nullptr;
  double* Kband = nullptr;
  long long* band_off = nullptr;  // [H] linear offsets of the stored slots
  int* band_o12 = nullptr;        // [H] packed offsets along directions 1, 2
  int band_H = 0;
  bool band_ready = false;
  int band_threads = 0, band_nv = 0;  // launch configuration of the band product (0 = default)
  long long ws_gen = 0;               // bumped whenever an address a captured graph may hold changes
  double band_nnz = 0.0;          // nonzero couplings (for algorithmic flop counts)
  // double-FP32 form of the band (IGA_OP_ASSEMBLED_DF)
  float2* Mdf = nullptr;
  float2* Kdf = nullptr;
  int EAm = 0, EAk = 0;           // power-of-two exponents of the split bands
  int* band_runs = nullptr;       // [nruns][4] runs of the upper half, with M's tiny slots
  int* band_runs_k = nullptr;     // the same runs with K's tiny slots
  double df_tiny_m = 0.0, df_tiny_k = 0.0;  // share of an interior row's terms that are tiny
  int band_nruns = 0;
  long long band_Np = 0;          // row stride of the split bands and vectors
  long long df_slack = 0;         // zeroed elements before and after each split array
  float2* df_xs = nullptr;        // [kMaxVec][Np] split input vectors (zero pads)
  int* df_E = nullptr;            // [kMaxVec] their exponents, [kMaxVec] scratch
  unsigned long long* df_part = nullptr;  // [kMaxVec][kDfBlocks] partial maxima
  unsigned int* df_bar = nullptr;         // grid barrier of the cooperative split (count, generation)
  long long bar_limit = -1;               // polls of that barrier before a time-out (< 0: the default)
  bool df_ready = false;
  DfTmaps tmM, tmK;               // tensor maps of the split bands (and vectors)
  // operator workspace
  int ws_vec = 0;
  double *u0 = nullptr, *u1 = nullptr, *ta = nullptr, *tb = nullptr, *tc = nullptr;
  long long su = 0, st = 0;
  // PCG workspace
  int cg_vec = 0;
  double *r = nullptr, *z = nullptr, *zold = nullptr, *p = nullptr, *q = nullptr, *f1 = nullptr, *f2 = nullptr;
  double* partial = nullptr;  // 3 * kMaxVec * kRedBlocks
  double* pq_part = nullptr;  // per-block partials of p.q from the band product, cg_vec * df_max_blocks
  double* rz_part = nullptr;  // per-block partials of r.z, r.z_old from the preconditioner, 2 cg_vec (N / 32 + 2)
  CgScalars cs{};
  int* h_nactive = nullptr;   // pinned
  // stepping
  int step_k = 0;
  double *Yneg = nullptr, *rhs = nullptr, *Z = nullptr, *Z2 = nullptr;
  int hist = 0;
  double* dstate = nullptr;
  long long dstate_cap = 0;
  // launch counting and profiling of one kernel class
  long long nlaunch = 0;
  int cur_active = 0;  // host-known number of active systems of the running PCG
  int prof_class = IGA_PROF_OFF;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending;
  double prof_flops = 0.0, prof_bytes = 0.0;
  // captured step graph with the PCG loop on the device (conditional while node)
  bool use_graphs = true;
  cudaStream_t gs = nullptr, gbody = nullptr;  // non-default streams for capture and replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool gvalid = false;
  struct GraphKey {
    const double* state;
    int k, op, prec, guess, max_iter;
    double dt, rho, tol;
  } gkey{};
  long long g_pro = 0, g_body = 0, g_epi = 0;  // kernel launches captured before / in / after the loop
  int* d_loop = nullptr;       // [2] iterations of the current solve, body executions since reset
  long long* d_tot = nullptr;  // [kMaxVec] iterations per system slot, summed over solves
  int* d_max = nullptr;        // [kMaxVec] largest count of one solve
  double* d_init = nullptr;    // [kMaxVec] initial relative residuals, summed over solves
  double last_init[kMaxVec] = {};  // initial relative residuals of the last host-driven solve
  int* d_stat = nullptr;       // [2] first error status, any unconverged solve
  // damping C = aM M + aK K and forcing F(t) = sum_m G_m sin(om_m t + ph_m) (eq. mp)
  bool damped = false;
  double aM = 0.0, aK = 0.0;
  int nforce = 0;
  double* fG = nullptr;  // [nforce][N] load vectors
  double fom[kMaxForce] = {}, fph[kMaxForce] = {};
  double *Yv = nullptr, *MYv = nullptr;  // [k][N] when aM != 0
  int yv_k = 0;
  double* d_time = nullptr;  // t_n on the device (advanced inside each step)
  double time = 0.0;         // the same on the host
  // learned initial guess (kernels_net.cu)
  float *ws_theta = nullptr, *ws_m = nullptr, *ws_v = nullptr, *ws_grad = nullptr;
  bool ws_params = false, ws_trained = false;
  long long ws_adam_t = 0;
  int ws_k = 0;                                         // stages the step buffers hold
  double *ws_E = nullptr, *ws_B1 = nullptr, *ws_B2 = nullptr;  // [k][N]
  double *ws_sc = nullptr, *ws_part = nullptr;          // scales [k][2], norm partials
  __nv_bfloat16 *ws_x = nullptr, *ws_act = nullptr;     // [k][3][N], [k][16][N]
  int ws_cap = 0, ws_count = 0;                         // recorded samples
  __nv_bfloat16* ws_sx = nullptr;                       // [cap][3][N]
  float* ws_st = nullptr;                               // [cap][N]
  float *ws_y = nullptr, *ws_dy = nullptr;              // training: [N]
  void* ws_work = nullptr;
  double *ws_loss = nullptr, *ws_lpart = nullptr;
  long long ws_loss_cap = 0;
  double* pts = nullptr;  // [pts_cap] weighted point values (iga_integrate)
  long long pts_cap = 0;
  // multi-patch system (iga_mp_create): M, K and the additive Schwarz preconditioner act
  // through the patches' own handles; null for a single patch
  MpState* mp = nullptr;
  std::string err;
};

// A multi-patch system of conforming patches (Sec. 5.1, 5.4): one handle per patch over
// its index box, and the maps between global and local vectors.
struct MpState {
  std::vector<iga_handle*> patch;
  std::vector<long long> off, nr;  // first entry and size of each patch's box
  long long nloc = 0;              // sum of the box sizes
  int n_adj = 0;
  int op_form = IGA_OP_MATRIX_FREE, precond = IGA_PREC_FP64;  // the patches' forms
  long long *d_gid = nullptr, *d_off = nullptr, *d_nr = nullptr, *d_crow = nullptr, *d_cent = nullptr;
  int* d_epatch = nullptr;
  MpMaps maps;
  double *xl = nullptr, *yl = nullptr;  // [vec_cap][nloc] local inputs and results
  int vec_cap = 0;
  // concurrent patches (iga_mp_set_concurrent): one stream per patch, forked from and
  // joined back into the caller's stream by events around every operator
  bool concurrent = false;
  std::vector<cudaStream_t> ps;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};


namespace iga {

int fail(iga_handle* h, int code, const std::string& msg);

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(h, IGA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

#define CKS(expr)                   \
  do {                              \
    int s_ = (expr);                \
    if (s_ != IGA_OK) return s_;    \
  } while (0)

// a kernel launch: checked and counted
#define LK(call)     \
  do {               \
    CK(call);        \
    ++h->nlaunch;    \
  } while (0)

template <typename T>
int dalloc(iga_handle* h, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(h, IGA_ENOMEM, std::string("cudaMalloc(") + std::to_string(count * sizeof(T)) + " bytes): " +
                                   cudaGetErrorString(e));
  }
  return IGA_OK;
}

template <typename T>
int upload(iga_handle* h, T** p, const std::vector<T>& v) {
  CKS(dalloc(h, p, v.size()));
  CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return IGA_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

inline bool is_assembled(const iga_handle* h) {
  return h->opt.op_form == IGA_OP_ASSEMBLED || h->opt.op_form == IGA_OP_ASSEMBLED_DF;
}

// operators.cu: the handle's operators. pq / npq: the band product's per-block partials of
// x.y ([nvec][*npq]; *npq = 0 when not computed); presplit (double-FP32 form): the split copy
// of x is already in place; rzp / nrz: the preconditioner's last pass's partials of r.z and
// r.z_old ([2][nvec][*nrz]).
double mass_last_flops(const iga_handle* h);
double stiff_last_flops(const iga_handle* h);
double mass_apply_flops(const iga_handle* h);
int fd_apply(iga_handle* h, int nvec, const int* active, const double* r, double* z, double* t1, double* t2,
             double* rzp = nullptr, int* nrz = nullptr);
int assemble_band64(iga_handle* h);
int assemble_band_df(iga_handle* h);
cudaError_t launch_band(iga_handle* h, cudaStream_t s, int cls, int nvec, const int* active, const double* x,
                        double* y, int threads, int nv, double* pq, int* npq, bool presplit = false);
int apply_band(iga_handle* h, int cls, int nvec, const int* active, const double* x, double* y,
               double* pq = nullptr, int* npq = nullptr, bool presplit = false);
int mp_apply(iga_handle* h, int which, int nvec, const int* active, const double* x, double* y);
int apply_M(iga_handle* h, int nvec, const int* active, const double* x, double* y, double* pq = nullptr,
            int* npq = nullptr, bool presplit = false);
int apply_K(iga_handle* h, int nvec, const int* active, const double* x, double* y);
int apply_Pinv(iga_handle* h, int nvec, const int* active, const double* r, double* z, double* rzp = nullptr,
               int* nrz = nullptr);

// pcg.cu: batched PCG (launch-only pieces and the host-driven loop)
int solve_begin(iga_handle* h, int nvec, const double* b, double* x, bool use_x0);
int solve_prime(iga_handle* h, int nvec);
int solve_iter_a(iga_handle* h, int nvec, double* x);
int solve_iter_b(iga_handle* h, int nvec);
int read_nactive(iga_handle* h, int* nact);
int solve(iga_handle* h, int nvec, const double* b, double* x, bool use_x0, int* iters, double* relres);

// internal routines of capi.cu used elsewhere (batch.cu, warmstart.cu, multipatch.cu, operators.cu, pcg.cu)
int fail(iga_handle* h, int code, const std::string& msg);
int prof_begin(iga_handle* h, int cls, cudaEvent_t* e1);
int prof_end(iga_handle* h, cudaEvent_t e1, double flops, double bytes);
int ensure_op_ws(iga_handle* h, int nvec);
double theta_crit(double rho);
extern thread_local std::string g_create_err;  // message of the last failed handle creation
// a handle over the index box lo..hi of a patch (nullptr: the whole patch)
int create_handle(int dim, const int* degree, const int* nknots, const double* const* knots, const double* ctrl,
                  const int* lo, const int* hi, const iga_options* opt, iga_handle** out);
int check_handle(iga_handle* h);
int single_patch(iga_handle* h, const char* what);
int ensure_ws_step(iga_handle* h, int k);
NetGrid net_grid_of(const iga_handle* h);
StepCoefs handle_coefs(const iga_handle* h, int k, double rho, double dt);
void drop_step_graph(iga_handle* h);
int ensure_cg_ws(iga_handle* h, int nvec);
int check_tc_error(iga_handle* h);
int assemble_band(iga_handle* h);
int prepare_capture(iga_handle* h, int k);
int capture_step(iga_handle* h, double* state, int k, const StepCoefs& sc);
bool same_key(const iga_handle::GraphKey& a, const iga_handle::GraphKey& b);
int reset_graph_counters(iga_handle* h, cudaStream_t s);
int collect_graph_run(iga_handle* h, cudaStream_t s, int k, int nsteps, double dt, iga_stats* stats);
iga_handle::GraphKey graph_key(const iga_handle* h, double* state, int k, double rho, double dt);

}  // namespace iga
