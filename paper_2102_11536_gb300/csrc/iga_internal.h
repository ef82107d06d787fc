// Internal declarations of the GB300 generalized-alpha IGA library.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/iga_galpha.h"
#include "../../include/iga_multipatch.h"

namespace iga {

constexpr int kMaxDeg = 6;       // largest supported spline degree
constexpr int kMaxP = kMaxDeg + 1;
constexpr int kMaxVec = 8;       // largest batch of vectors per operator call
constexpr int kMaxK = 4;         // largest order parameter (order 2k)
constexpr int kMaxRows = 3 * kMaxK;

// ---------------------------------------------------------------------------
// Host-side univariate setup (host_setup.cpp)
// ---------------------------------------------------------------------------
struct Tables1D {
  int p = 0, m = 0, n = 0, nel = 0, nq = 0, Q = 0;
  int lo = 1;                       // the box of functions: full indices lo .. lo + n - 1 (1 .. m-2 by default)
  std::vector<double> qx, qw;       // [Q] point, weight (Gauss weight * span/2)
  std::vector<int> qfirst;          // [Q] first full function index nonzero on the span
  std::vector<int> qfirst_op;       // [Q] qfirst - lo + 1: the operators' window starts at box index qfirst_op - 1
  std::vector<double> val, der;     // [Q][p+1]
  std::vector<int> flo, fhi;        // [n] quadrature range [lo, hi) of box function i (full i + lo)
  std::vector<double> mhat;         // [n][n] parametric mass matrix over the box
  std::vector<double> evec;         // [n][n] row-major, column c = eigenvector c
  std::vector<double> eval;         // [n]
  std::vector<double> chol;         // [n][p+1] band Cholesky factor of mhat, chol[i][d] = L_{i,i-d}
  std::vector<double> cdinv;        // [n] 1 / L_ii
};

// Gauss-Legendre rule on [-1, 1].
void gauss_legendre(int n, double* x, double* w);
// Values and derivatives of the degree-p B-splines nonzero at x in span s (s-p..s).
void bspline_span(int p, const double* U, int s, double x, double* val, double* der);
// Build all tables of one direction over the box of functions lo .. hi (full indices;
// hi < 0 means m - 2: the interior functions); returns false on invalid knots or box.
bool build_tables(int p, int nknots, const double* U, int nq, Tables1D& t, std::string& err, int lo = 1,
                  int hi = -1);
// Band Cholesky factor of an SPD matrix with half bandwidth p (row-major n x n):
// L [n][p+1] with L[i][d] = L_{i,i-d}, dinv [n] = 1 / L_ii. False if not positive definite.
bool band_cholesky(int n, int p, const std::vector<double>& M, std::vector<double>& L, std::vector<double>& dinv);
// Largest eigenvalue of the symmetric tridiagonal matrix (diagonal a, off-diagonal b).
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b);
// Multi-patch gather / scatter (kernels_mp.cu). Patch r's local vectors lie at
// xl + nvec * off[r], vector v at + v * nr[r]; entry e of the concatenated boxes belongs to
// patch epatch[e] at box index e - off[r] and to global function gid[e] (-1: none); the
// entries of global function g are cent[crow[g] .. crow[g+1]), ascending. Device arrays.
struct MpMaps {
  long long nloc = 0, nglob = 0;
  const long long* gid = nullptr;   // [nloc]
  const int* epatch = nullptr;      // [nloc]
  const long long* off = nullptr;   // [npatch]
  const long long* nr = nullptr;    // [npatch]
  const long long* crow = nullptr;  // [nglob + 1]
  const long long* cent = nullptr;  // [crow[nglob]]
};
cudaError_t launch_mp_gather(cudaStream_t s, const MpMaps& m, int nvec, const int* active, const double* x,
                             double* xl);
cudaError_t launch_mp_scatter(cudaStream_t s, const MpMaps& m, int nvec, const int* active, const double* yl,
                              double* y);
// One patch's box (entries off .. off + nr - 1): add = 0 gathers the global vector into the
// box (zero where no degree of freedom), add = 1 adds the box into the global vector.
cudaError_t launch_mp_patch_io(cudaStream_t s, const MpMaps& m, long long off, long long nr, int nvec, int add,
                               const double* in, double* out);
// Gluing of conforming patches (host_multipatch.cpp); arguments as iga_mp_layout.
int mp_layout(int npatch, int dim, const int* degree, const int* nknots, const double* const* knots,
              const double* const* ctrl, double tol, int* lo, int* hi, long long* nglob, int* n_adj, long long* gid,
              long long gid_len, std::string& err);
// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major).
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& evec, std::vector<double>& eval);

// ---------------------------------------------------------------------------
// Device-side per-direction tables
// ---------------------------------------------------------------------------
struct DirDev {
  int p, P, n, Q;
  double* val;    // [Q][P]
  double* der;    // [Q][P]
  double* sq;     // [Q][P] squared values (for diag(M))
  float* val32;
  float* der32;
  int* qfirst;    // [Q] the operators' window start + 1 (Tables1D::qfirst_op)
  int* qfirst_geo;  // [Q] full first function index, when it differs from qfirst (a box not starting at 1)
  int* flo;       // [n]
  int* fhi;       // [n]
  double* qw;     // [Q]
  double* U64;    // [2][n][np]: U then U^T, element (i, j) at j*np + i, np = n rounded up to 8
  double* lam64;  // [n] inverse eigenvalues 1 / Lambda_a of Mhat_a
  float* U32;
  float* lam32;
  void* Btc[2];   // BF16 U and U^T in the tensor-core operand layout (kernels_tc.cu)
  void* Btc16[2]; // the same in FP16
  double* chol;   // [n][p+1] band Cholesky factor of the interior parametric mass matrix
  double* cdinv;  // [n] inverse diagonal of the factor
  float* chol32;  // the same in FP32
  float* cdinv32;
};

// ---------------------------------------------------------------------------
// Kernel launchers (kernels_*.cu)
// ---------------------------------------------------------------------------
struct AxisShape {
  long long A;   // product of the sizes of the faster axes
  int Lin;       // length along the axis on input
  int Lout;      // length along the axis on output
  long long B;   // product of the sizes of the slower axes
};

// Interpolation pass along one axis (coefficients -> quadrature points):
// out[x,o,y] = sum_l T[o][l] in[x, qfirst[o]-1+l, y]; up to 2 tables on one input.
cudaError_t launch_fwd(cudaStream_t s, const DirDev& d, AxisShape sh, int nvec, const int* active,
                       const double* in, long long in_vs, const double* T0, double* out0, const double* T1,
                       double* out1, long long out_vs);
// Transposed pass (quadrature points -> coefficients):
// out[x,i,y] = sum_{q in supp i} T0[q][i+1-qfirst[q]] in0[x,q,y] (+ same with T1, in1).
cudaError_t launch_tr(cudaStream_t s, const DirDev& d, AxisShape sh, int nvec, const int* active,
                      const double* in0, const double* T0, const double* in1, const double* T1, long long in_vs,
                      double* out, long long out_vs);
// Fused last-axis kernel of the mass operator: out = B^T (W .* (B in)) along the last axis.
cudaError_t launch_mid_mass(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                            const double* W, const double* in, double* out, long long vs);
// Fused last-axis kernel of the stiffness operator (3-D): inputs a (-> B' a), b (-> B b),
// c (-> B c) are the partial interpolants of the derivative in directions 2, 1, 0; h = G g;
// outputs (in place) a <- B'^T h2, b <- B^T h1, c <- B^T h0.
cudaError_t launch_mid_stiff3(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                              const double* G, long long gstride, double* a, double* b, double* c, long long vs);
// 2-D: inputs a (-> B' a, direction 1), c (-> B c, direction 0); outputs a <- B'^T h1, c <- B^T h0.
cudaError_t launch_mid_stiff2(cudaStream_t s, const DirDev& d, long long A, int nvec, const int* active,
                              const double* G, long long gstride, double* a, double* c, long long vs);
// Geometric factors at the quadrature points; sets *bad = 1 if det DF <= 0 somewhere.
cudaError_t launch_geometry(cudaStream_t s, int dim, const DirDev* dirs, const int* m, const double* ctrl_soa,
                            double* W, double* G, long long gstride, int* bad);
// Fields at the Gauss points (kernels_field.cu): physical points X [dim][Qt] (point
// q = q0 + Q0 (q1 + Q1 q2)) from the SoA control net, and out = W .* g for nvec vectors.
cudaError_t launch_points(cudaStream_t s, int dim, const DirDev* dirs, const int* m, const double* ctrl_soa,
                          double* X);
cudaError_t launch_weight_points(cudaStream_t s, long long Qt, int nvec, const double* W, const double* g,
                                 double* out);

// Fast-diagonalisation mode product along one axis: out[x,i,y] = sum_j Mat(i,j) in[x,j,y]
// with Mat = U (transpose=0) or U^T (transpose=1), U holding [U | U^T] column-major,
// and an optional epilogue (Lambda^{-1} or post scale).
struct FdEpilogue {
  const double* post;            // multiply output by post[idx] (nullable)
  const double* lam[3];          // multiply by lam0[i0] lam1[i1] lam2[i2], the inverse eigenvalues (nullable)
  int n[3];
};
// (kernels_fd.cu) U holds [U | U^T], each Mat(i, j) at j*np + i, np = n rounded up
// to 8; pre (axis 0 only, nullable) multiplies the inputs in FP64 before rounding.
cudaError_t launch_fd_mode64(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const double* U,
                             int transpose, const double* in, double* out, long long vs, const double* pre,
                             FdEpilogue ep);
cudaError_t launch_fd_mode32(cudaStream_t s, int n, AxisShape sh, int nvec, const int* active, const float* U,
                             int transpose, const void* in, int in_is_double, void* out, int out_is_double,
                             long long vs, const double* pre, const double* post, const float* const* lam,
                             const int* nn);

// Vector kernels (kernels_vec.cu)
constexpr int kRedBlocks = 296;  // fixed reduction grid (2 x 148 .. deterministic order)
// partial[v*kRedBlocks + b] = sum over the block's fixed index set of a_v . b_v
cudaError_t launch_dot(cudaStream_t s, long long N, int nvec, const double* a, const double* b, long long vs,
                       double* partial);
// One block per vector: result[v] = sum_b partial[v*kRedBlocks + b] in fixed order.
cudaError_t launch_reduce(cudaStream_t s, int nvec, const double* partial, double* result);

struct CgScalars {  // device arrays, one entry per system
  double* bb;      // ||b||^2
  double* rz;      // r.z (current)
  double* rr;      // ||r||^2
  double* rr0;     // ||r||^2 of the initial guess
  double* alpha;
  double* beta;
  int* active;     // 1 while iterating
  int* iters;
  int* status;     // 0 ok, IGA_ENUMERIC on breakdown
  int* nactive;    // single counter
  unsigned int* ticket;  // [2] arrival counters: the x, r update (its last block tests convergence) and
                         // the alpha reduction (its last block sets alpha); 0 between launches
  double* red;           // [kMaxVec][64] chunk sums of the alpha reduction
};

#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// out[v] = sum of partial[v][0..np) for v < nvec, by the whole block (blockDim.x a
// multiple of 32 with at least nvec warps): each vector gets blockDim.x / 32 / nvec
// warps, which sum fixed strided shares (lane stride 32), then their warp sums are added
// in order -- a fixed order, so the result is reproducible. The partials are read from
// L2 (they may come from other blocks of the same launch).
__device__ __forceinline__ void reduce_partials(int nvec, const double* partial, double* out, int np) {
  __shared__ double wsum[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = (int)(blockDim.x >> 5), per = nw / nvec;  // warps per vector
  const int v = w / per, q = w - v * per;
  if (v < nvec) {
    double s = 0.0;
#pragma unroll 8
    for (int b = q * 32 + lane; b < np; b += per * 32) s += __ldcg(&partial[(long long)v * np + b]);
    s = warp_sum(s);
    if (lane == 0) wsum[w] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < nvec) {
    double s = 0.0;
    for (int i = 0; i < per; ++i) s += wsum[threadIdx.x * per + i];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}
#endif
// Reduction epilogues of PCG (one thread per system, tiny kernels).
// partials [nvec][np]
cudaError_t launch_cg_alpha(cudaStream_t s, int nvec, const double* partial, int np, CgScalars c);
cudaError_t launch_cg_check(cudaStream_t s, int nvec, const double* partial, CgScalars c, double tol2);
cudaError_t launch_cg_beta(cudaStream_t s, int nvec, const double* partial, const double* partial2, int np,
                           CgScalars c, int flexible);
cudaError_t launch_cg_init(cudaStream_t s, int nvec, const double* partial_bb, const double* partial_rr,
                           CgScalars c, double tol2);
cudaError_t launch_cg_start(cudaStream_t s, int nvec, const double* partial_rz, int np, CgScalars c);
// x += alpha p; r -= alpha q; partial ||r||^2; with check != 0 the launch's last block also
// runs the convergence test (launch_cg_check's work) on those partials
cudaError_t launch_cg_update_xr(cudaStream_t s, long long N, int nvec, CgScalars c, double* x, double* r,
                                const double* p, const double* q, long long vs, double* partial, int check,
                                double tol2);
// p = z + beta p
cudaError_t launch_cg_update_p(cudaStream_t s, long long N, int nvec, CgScalars c, double* p, const double* z,
                               long long vs);
// r = b - q (q = M x0)
cudaError_t launch_sub(cudaStream_t s, long long N, int nvec, const double* b, const double* q, double* r,
                       long long vs);
cudaError_t launch_copy_active(cudaStream_t s, long long N, int nvec, const int* active, const double* src,
                               double* dst, long long vs);

struct StepCoefs {
  int k;
  double c[kMaxRows];          // tau^m / m!
  double alpha[kMaxK], beta[kMaxK], gamma[kMaxK];
  double ralpha[kMaxK], gtau[kMaxK], btau2[kMaxK];  // 1 / alpha_j, gamma_j tau, beta_j tau^2
  double tau;
  int damped;                  // Rayleigh damping C = aM M + aK K present
  double aM, aK;
};
// Writes -Y_j (k vectors) and, if T != nullptr, the Taylor predictor T_{s_j} of each
// solved row. With damping: -(Y_j + aK Y'_j) (K acts on it), and -Y'_j into Yv if
// Yv != nullptr (the aM M Y'_j term), Y'_j the predictor of the block's velocity-like row.
cudaError_t launch_predict(cudaStream_t s, long long N, StepCoefs sc, const double* X, double* Yneg, double* T,
                           double* Yv);
// Loads of the stage equations (eq. ho1): rhs[j] += aM * MYv[j] (MYv nullable) +
// sum_m G_m om_m^{s_j} sin(om_m t_j + ph_m + s_j pi/2), t_j = *time + toff[j].
constexpr int kMaxForce = 8;
struct StageLoad {
  int nstage;
  int sder[kMaxK];
  double toff[kMaxK];
  int nterm;
  double om[kMaxForce], ph[kMaxForce];
  double aM;
};
cudaError_t launch_stage_load(cudaStream_t s, long long N, StageLoad a, const double* G, const double* time,
                              const double* MYv, double* rhs);
// *time += dt (one thread)
cudaError_t launch_advance_time(cudaStream_t s, double* time, double dt);
// Fused stage update in place.
cudaError_t launch_update(cudaStream_t s, long long N, StepCoefs sc, double* X, const double* Z);
// Z <- 2 Z - Z2, Z2 <- old Z
cudaError_t launch_extrap(cudaStream_t s, long long n, double* Z, double* Z2);
// device-side loop control of the captured PCG (kernels_vec.cu)
cudaError_t launch_set_cond(cudaStream_t s, cudaGraphConditionalHandle hc, const int* nactive, int* loop, int max_iter,
                            int reset);
// tot += iterations, mx = max iterations, init += ||b - M x0|| / ||b||, stat = first error / unconverged
cudaError_t launch_accum(cudaStream_t s, int nvec, CgScalars c, long long* tot, int* mx, double* init, int* stat);
cudaError_t launch_scale_neg(cudaStream_t s, long long n, double* x);
// out = ca * a + cb * b (n entries)
cudaError_t launch_lincomb(cudaStream_t s, long long n, double ca, const double* a, double cb, const double* b,
                           double* out);

// BF16 / FP16 tensor-core mode product along `axis` (kernels_tc.cu): B is the
// 16-bit matrix arranged by tc_arrange (f16 selects FP16 with per-line power-of-two
// scaling); err (device int) is set to 1 if an mbarrier wait times out.
cudaError_t launch_fd_mode_tc(cudaStream_t s, int n, int axis, AxisShape sh, int nvec, const int* active,
                              const void* B, int f16, const void* in, int in_is_double, void* out, int out_is_double,
                              long long vs, const double* pre, const double* post, const float* const* lam,
                              const int* nn, int* err);
int tc_pad(int n);
// Mat(i, j) row-major n x n (i output, j summed) -> BF16 or FP16 bits in the K-major
// core-matrix layout
void tc_arrange(int n, const double* Mat_ij, bool f16, std::vector<uint16_t>& outbits);

// Assembled band form (kernels_band.cu): H stored slots (centre + upper half),
// off[h] the linear offset of slot h, A [H][N].
// o12 (nullable): packed slot offsets along directions 1, 2 ((o1+64) | (o2+64) << 8) for
// skipping slots outside the grid for a whole warp; n: grid sizes (3 entries).
// threads: block size 64 / 128 / 256 / 512 (other = 256); nv: vectors per thread (0 = min(nvec, 4)).
// pq (nullable): per-block partials of x . y, [nvec][*npq] (the p.q of PCG, fused).
cudaError_t launch_band_spmv(cudaStream_t s, long long N, int H, const long long* off, const int* o12, const int* n,
                             const double* A, const int* active, int nvec, const double* x, double* y, long long vs,
                             int threads, int nv, double* pq = nullptr, int* npq = nullptr);
// Double-FP32 band product (kernels_banddf.cu). Split storage: float2 (hi, lo) rows
// of stride Np (N + 2 kDfPad rounded up to a multiple of 16) with zero pads, and
// df_slack(maxL) zeroed elements before and after every split array (the reach of
// the staged copies); kDfBlocks partial maxima per vector.
constexpr int kDfPad = 16;
constexpr int kDfBlocks = 512;
inline long long df_row_stride(long long N) { return (N + 2 * kDfPad + 15) / 16 * 16; }
inline long long df_slack(long long maxL) { return (maxL + 1024 + 15) / 16 * 16; }
// the runs of the upper half: per run {first slot, length, (o1 + 64) | (o2 + 64) << 8 | m << 16,
// linear offset}, the centre run (o1 = o2 = 0) first and the others ordered by m. m is the
// number of tiny slots at each end of the run (slots t < m and t >= length - m): with
// tiny (nullable, one flag per stored slot) the products form those terms as one FP32
// multiply-add of the high parts; without it m = 0.
std::vector<int> band_df_runs(const int* n, const int* p, const unsigned char* tiny);
// out[h] = largest |hi| of stored slot h over the N rows of a split band, as FP32 bits
cudaError_t launch_df_slot_absmax(cudaStream_t s, long long N, int H, const float2* A, long long Np, unsigned* out);
// Adf = split(A 2^-E) with one exponent E (left in dE[0]) for the whole [H][N] band
cudaError_t launch_df_split_matrix(cudaStream_t s, long long N, int H, const double* A, float2* Adf, long long Np,
                                   unsigned long long* part, int* dE);
// xs[v] = split(x[v] 2^-E_v), E_v (into Ex[v]) from the vector's largest magnitude; with
// bar (2 zeroed device words kept for it) and err, one cooperative launch whose grid
// barrier's wait, bounded by bar_limit polls (< 0: the default), sets *err = 1 if it
// runs out, else two launches
cudaError_t launch_df_split(cudaStream_t s, long long N, const int* active, int nvec, const double* x, long long vs,
                            float2* xs, long long Np, int* Ex, unsigned long long* part, unsigned int* bar, int* err,
                            long long bar_limit = -1);
// The PCG beta of the direction update: rzp == nullptr: c.beta as computed; else every
// block computes it from the preconditioner's per-block partials rzp[0][v][nrz] (r.z) and,
// flexible, rzp[1][v][nrz] (r with the previous z), as launch_cg_beta does, and block 0
// stores beta and r.z into c after the launch's grid barrier (launch_cg_beta's work).
struct BetaArgs {
  const double* rzp;
  int nrz, flexible;
  CgScalars c;
};
// p = z + beta p (active systems, the PCG direction update) and the split of the new p in
// one cooperative launch; cudaErrorNotSupported without cooperative launch (nothing done)
cudaError_t launch_df_update_split(cudaStream_t s, long long N, const int* active, int nvec, double* p,
                                   const double* z, const BetaArgs& ba, long long vs, float2* xs, long long Np,
                                   int* Ex, unsigned long long* part, unsigned int* bar, int* err,
                                   long long bar_limit = -1);
// y = A x from the split copies (xs, Ex from launch_df_split; EA the band's exponent);
// pq / npq as in launch_band_spmv (x is the FP64 input, read only for pq)
// 2-D tensor maps over a split band ([H][Np], boxes for the upper rows and the lower
// parallelogram of a run) and over the split vectors ([kMaxVec][Np], 1 or 2 rows).
struct DfTmaps {
  CUtensorMap up, dn, x1, x2, x3, x4;
  bool ok = false;
};
bool df_encode_maps(const float2* A, int H, const float2* xs, int nvmax, long long Np, int p0, DfTmaps* tm);
// Block order of the band products: windows of R rows over strips of W1 lines of
// direction 1, plane after plane within a strip (S strips, the last one narrower);
// nb0 / nbl windows per strip-plane of a full / the last strip.
struct DfStrips {
  int n0, n1, n2, W1, S, nb0, nbl;
};
// the strips for blocks of R rows: the last p2 planes of a strip hold at most ~48 MB of
// the band's H slots (8 B each), so that the lower terms are read from L2
DfStrips df_strips(const int* n, int p2, int H, int R);
long long df_strip_blocks(const DfStrips& g);
// upper bound on the blocks of any band-product launch shape (per-block partials)
inline long long df_max_blocks(long long N, const int* n) { return N / 64 + (long long)n[1] * n[2] + 2; }
// (p0, p2: the degrees along directions 0 and 2; H the stored slots). threads 96 with
// nv <= 4, p0 in 2..4 and tm->ok selects the tensor-map kernel with two rows per thread;
// threads 128 with nv <= 4, p0 in 2..4 and tm->ok the tensor-map kernel with one row per
// thread; threads 64, 128 or 256 with nv <= 2 and p0 in 2..4 the TMA-staged kernel with
// that many rows per block (err: device int set to 1 if one of its mbarrier waits runs
// out; null: never these kernels); other shapes the register kernel. Every shape gives
// bitwise the same result.
cudaError_t launch_band_df(cudaStream_t s, long long N, int nruns, const int4* runs, const int* n, int p0, int p2,
                           int H, const float2* A, long long Np, int EA, const int* active, int nvec,
                           const float2* xs, const int* Ex, const double* x, double* y, long long vs, int threads,
                           int nv, double* pq, int* npq, int* err, const DfTmaps* tm);
// Persistent batch step (kernels_persist.cu): one cooperative launch advances every
// patch of a batch by one time step with FP64 band operators and the band-Cholesky
// Kronecker preconditioner (FP32 or FP64). Device tables, built by the host.
constexpr int kPersistFdPad = 8;  // BF16 entries added to each staged row of the persistent mode products
struct PPatch {
  long long N;
  int n[3], deg[3], H;
  const double *M, *K;          // [H][N] FP64 bands
  const long long* off;         // [H] linear offsets of the stored slots
  const int* o12;               // [H] packed offsets along directions 1, 2
  const double* scale;          // [N] D^-1/2 Dhat^1/2
  const void *L[3], *dinv[3];   // band Cholesky factors per axis ([n][p+1], [n]), FP32 or FP64
  const void* Ubf[3][2];        // fast diagonalisation: U_a (0) and U_a^T (1) in BF16, row-major, rows of
                                // ceil16(n) + kPersistFdPad entries, ceil16(n) rows, zero beyond n
                                // (Mat(i, j) at i (ceil16(n) + kPersistFdPad) + j, i the output): the
                                // shared-memory image the mode products copy
  const float* lam[3];          // 1 / Lambda_a, FP32
  double* X;                    // state [3k][N] (the caller's)
  double *Y, *T, *r, *x, *z, *p, *q;  // [k][N] work vectors
  void *t1, *t2;                // [k][N] intermediates of the Kronecker solve
  StepCoefs sc;
};
struct PBatch {
  int np, k, max_iter, flexible;
  int fd;                             // 1: BF16 fast diagonalisation, 0: band Cholesky
  double tol2;
  const PPatch* pt;                   // [np]
  const int2* rtile;                  // [nrt] (patch, row tile within the patch)
  const int2* ltile[3];               // [nlt[a]] (patch, line tile within the patch)
  int nrt, nlt[3];
  const int *rt0, *nrt_p;             // [np] first row tile and row tiles per patch
  const int *lt2, *nlt2_p;            // [np] the same for the line tiles of the preconditioner's last
  int nrzt;                           // phase (axis 2: band Cholesky, axis 0: fast diagonalisation)
  double* const* Yp;                  // [np] the patches' Y, r, p, q (band-product operands)
  double* const* rp;
  double* const* pp;
  double* const* qp;
  double* part;                       // [nrt][k] row-tile partials
  double* lpart;                      // [2][nrzt][k] last-phase partials of r.z (new, previous z)
  double *bb, *rr, *rz, *rznew, *rzold, *pq, *alpha, *beta, *last_rel;  // [np k]
  int *active, *iters, *status, *max_iters;                              // [np k]
  long long* tot_iters;                                                  // [np k]
  int* flags;                         // [0] some system active, [1] first failure status
  unsigned int* bar;                  // grid barrier (count, generation)
  long long bar_limit;
  int* err;                           // set when a barrier wait runs out
  unsigned long long* ptime;          // [kPersistPhases] ns per phase kind, added by block 0 (nullable)
};
constexpr int kPersistPhases = 8;     // predictor, K product, PCG scalars, preconditioner, direction,
                                      // M product, x and r update, stage update
int batch_row_tiles(long long N);
int batch_line_tiles(long long N, int n);
size_t batch_smem_bytes(int nmax, int pmax, int k, bool f32, bool fd);
// variant 0: three blocks per SM, two slots per band pass; 1: two blocks per SM, four slots
// (k <= 2); both give bitwise the same results
constexpr int kPersistVariants = 2;
cudaError_t launch_batch_step(cudaStream_t s, const PBatch& B, bool f32, size_t smem, int variant, int* grid);

cudaError_t launch_probe_gen(cudaStream_t s, long long N, const int* n, const int* p, int first, int ncol, int nvec,
                             double* x, long long vs);
cudaError_t launch_probe_extract(cudaStream_t s, long long N, const int* n, const int* p, int first, int ncol,
                                 int nvec, const double* y, long long vs, double* A);

// Learned initial guess (kernels_net.cu). Fields on the n1 x n2 x n3 interior grid;
// x [nb][3][N] BF16 features, act [nb][16][N] BF16 hidden layer, theta the FP32
// parameter vector (IGA_NET_NPARAM). nl counts the kernels launched.
struct NetGrid {
  int n1, n2, n3;
};
long long net_blocks(const NetGrid& g, int nb);
size_t net_workspace_bytes(const NetGrid& g, int nb);  // backward: dh and per-block partials
bool net_grid_ok(const NetGrid& g, int nb);
// act = R(relu(W1 * x + b1)); y = W2 * act + b2 (y nullable); if Z != nullptr also
// Z = E + s0[2 s] y for sample s (the guess).
cudaError_t launch_net_forward(cudaStream_t s, const NetGrid& g, int nb, const __nv_bfloat16* x, const float* theta,
                               __nv_bfloat16* act, float* y, double* Z, const double* E, const double* s0,
                               long long* nl);
// dy = (y - t) / N; *loss = sum (y - t)^2 / (2 N); part: kRedBlocks doubles.
cudaError_t launch_net_loss(cudaStream_t s, long long N, const float* y, const float* t, float* dy, double* part,
                            double* loss, long long* nl);
// grad = d(sum_s sum_p dy y)/d theta over nb samples; work: net_workspace_bytes.
cudaError_t launch_net_backward(cudaStream_t s, const NetGrid& g, int nb, const __nv_bfloat16* x, const float* theta,
                                const __nv_bfloat16* act, const float* dy, float* grad, void* work, long long* nl);
cudaError_t launch_net_adam(cudaStream_t s, int n, float* theta, const float* grad, float* m, float* v, long long step,
                            double lr, long long* nl);
// Features of k solves (x [k][3][N], E, scales sc [k][2] = (s0, s1)); moves the
// histories b2 <- b1 <- b, z2 <- z1 <- E. part: 2 k kRedBlocks doubles.
cudaError_t launch_ws_features(cudaStream_t s, long long N, int k, const double* b, double* b1, double* b2,
                               const double* D, double* z1, double* z2, __nv_bfloat16* x, double* E, double* part,
                               double* sc, long long* nl);
// t [k][N] = (Z - E) / s0, FP32.
cudaError_t launch_ws_target(cudaStream_t s, long long N, int k, const double* Z, const double* E, const double* sc,
                             float* t, long long* nl);

// Kronecker solve along one axis (kernels_kron.cu): every line of the tensor (line
// rr = xx + A y holds elements xx + A (k + n y), k < n) is replaced by Mhat_a^{-1} times
// it, by forward and backward substitution with the band Cholesky factor (half
// bandwidth p); pre / post (nullable, per element) multiply the input / output in
// FP64. f32 selects FP32 arithmetic with the FP32 factor (FP32 or FP64 input / output).
// rdot (nullable; FP64 output only): also per-block partials of rdot . out and of rdot .
// (out before the write), [2][nvec][*npart] in part (*npart = 0 if not computed).
cudaError_t launch_kron_axis(cudaStream_t s, int n, int p, AxisShape sh, int nvec, const int* active, int f32,
                             const void* L, const void* dinv, const void* in, int in_is_double, void* out,
                             int out_is_double, long long vs, const double* pre, const double* post,
                             const double* rdot = nullptr, double* part = nullptr, int* npart = nullptr,
                             const float* scale32 = nullptr);

// Fixed scratch of the allocation-free preconditioner entry point: values per buffer.
constexpr long long kNoAllocMaxElems = 1LL << 20;
// Helpers for entry points defined outside capi.cu.
int handle_device(iga_handle* h, int* device);  // makes h's device current
int handle_fail(iga_handle* h, int code, const std::string& msg);
// The preconditioner in h's arithmetic with caller-provided scratch t1, t2 (each
// nvec * N doubles); allocates nothing.
int pinv_with_scratch(iga_handle* h, int nvec, const double* x, double* y, double* t1, double* t2);

}  // namespace iga
