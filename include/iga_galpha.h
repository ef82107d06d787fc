/*
 * iga_galpha.h -- C ABI of the GB300 implementation of the per-time-step hot
 * path of the explicit 2k-order generalized-alpha method for isogeometric
 * structural dynamics (Behnoudfar, Loli, Reali, Sangalli, Calo; arXiv 2102.11536).
 *
 * The semi-discrete problem is M U'' + K U = F with U(0) = U0, U'(0) = V0
 * (Sec. 2.1, eq. mp / eq. u0), damping C = 0, on one B-spline patch
 * (Sec. 5.1-5.2) with homogeneous Dirichlet conditions. One step of the method
 * (Sec. 4, eq. ho1-ho3) applies the stiffness operator to k predicted vectors,
 * solves k systems with the mass matrix by preconditioned CG (Sec. 5.5) with
 * the preconditioner D^{1/2} Dhat^{-1/2} (Mhat_1 x Mhat_2 x Mhat_3) Dhat^{-1/2} D^{1/2}
 * (Sec. 5.3, def:single_patch_prec), and updates the 3k state variables.
 *
 * Conventions shared by every call:
 *   - All vectors are FP64, length N = prod_a (m_a - 2), the interior control
 *     points (the first and last univariate function of each direction carry
 *     the Dirichlet condition and are dropped). Order is co-lexicographic,
 *     direction 0 fastest (Sec. 5.2, def:parametric_spline). On a handle made by
 *     iga_mp_create (iga_multipatch.h) N is the number of global functions of
 *     the glued patches, in that header's global numbering.
 *   - "device" pointers are CUDA global memory on the handle's device; "host"
 *     pointers are ordinary (preferably pinned) CPU memory.
 *   - Every call returns an IGA_* status; on failure iga_last_error() gives a
 *     message. No C++ exception crosses the ABI.
 *   - Work is issued on the handle's stream (iga_options.stream). Calls that
 *     return results to host memory synchronise that stream; calls that only
 *     write device memory may return before the kernels finish.
 *   - A handle is not thread-safe. The library owns all memory it allocates;
 *     caller buffers are never freed or retained after the call.
 */
#ifndef IGA_GALPHA_H
#define IGA_GALPHA_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define IGA_OK 0
#define IGA_EINVAL 1          /* bad argument (sizes, degrees, pointers, k, rho, dt) */
#define IGA_ENOMEM 2          /* device or host allocation failed */
#define IGA_ECUDA 3           /* a CUDA call failed; the message names it */
#define IGA_ENOT_CONVERGED 4  /* PCG reached max_iter above the tolerance */
#define IGA_ENUMERIC 5        /* NaN/Inf or non-positive curvature p.Mp in PCG */
#define IGA_EUNSTABLE 6       /* energy growth detected (time step above the CFL limit) */
#define IGA_EGEOMETRY 7       /* det DF <= 0 at a quadrature point (Sec. 5.3, Assumption g_regularity) */

/* Form of the K and M operators. */
#define IGA_OP_MATRIX_FREE 0  /* sum-factorised at the Gauss points (default) */
#define IGA_OP_ASSEMBLED 1    /* assembled band rows, (2p+1)^d coefficients per row */
#define IGA_OP_ASSEMBLED_DF 2 /* the same band rows held as pairs of FP32 numbers (hi + lo, 48
                                 significant bits, one power-of-two scale per matrix and per
                                 vector); products in double-FP32 arithmetic: error-free FP32
                                 products and TwoSum accumulation, a few 2^-48 of sum |a||x|,
                                 plus, for entries below about 2^-130 of the vector's largest,
                                 an absolute error of that order; the terms of tiny slots
                                 (every coefficient below 2^-24 of the matrix's largest) are
                                 one FP32 multiply-add each, within 2^-23 |a x| < 2^-47
                                 max|A| |x| (iga_band_df_tiny) */

/* Arithmetic of the preconditioner's fast-diagonalisation mode products. */
#define IGA_PREC_FP64 0       /* FP64 (default); plain CG */
#define IGA_PREC_FP32 1       /* FP32 CUDA cores; flexible CG */
#define IGA_PREC_BF16 2       /* BF16 tensor cores, FP32 accumulation; flexible CG */
#define IGA_PREC_FP16 3       /* FP16 tensor cores, FP32 accumulation; flexible CG */
#define IGA_PREC_BANDED 4     /* FP64 Kronecker solve by band Cholesky along each direction (the O(N)
                                 Kronecker solver of Sec. 5.5) instead of fast diagonalisation; plain CG */
#define IGA_PREC_BANDED32 5   /* the same band Cholesky Kronecker solve in FP32; flexible CG */

/* Initial guess of each mass solve inside a time step. */
#define IGA_GUESS_ZERO 0      /* null vector, as in the paper's experiments (Sec. 6) */
#define IGA_GUESS_PREV 1      /* the same block's solution at the previous step */
#define IGA_GUESS_EXTRAP 2    /* 2 Z^{n-1} - Z^{n-2} */
#define IGA_GUESS_TAYLOR 3    /* the Taylor predictor T_{s_j} of the solved variable */
#define IGA_GUESS_LEARNED 4   /* 2 Z^{n-1} - Z^{n-2} plus the learned network's correction
                                 (iga_ws_*; no counterpart in the paper) */

/* Parameters of the warm-start network: W1 [16][3][27], b1 [16], W2 [16][27], b2 [1]. */
#define IGA_NET_NPARAM 1745

typedef struct iga_options {
  int nquad;        /* Gauss points per element and direction; 0 => max_a(p_a) + 1 */
  double tol;       /* PCG stopping rule ||r||_2 <= tol * ||b||_2; default 1e-10 */
  int max_iter;     /* PCG iteration cap per solve; default 500 */
  int precond;      /* IGA_PREC_*; default IGA_PREC_FP64 */
  int op_form;      /* IGA_OP_*; default IGA_OP_MATRIX_FREE */
  int guess;        /* IGA_GUESS_*; default IGA_GUESS_ZERO */
  int device;       /* CUDA device ordinal; default 0 */
  void* stream;     /* cudaStream_t for all work, NULL = legacy default stream */
} iga_options;

typedef struct iga_stats {
  int steps;            /* time steps taken by the call */
  int solves;           /* mass-matrix solves */
  long long iters;      /* PCG iterations summed over the solves */
  int max_iters;        /* largest iteration count of one solve */
  double max_relres;    /* largest final ||r||/||b|| */
  long long launches;   /* CUDA kernel launches issued by the call */
  double init_relres_sum; /* sum over the solves of ||b - M x0||_2 / ||b||_2 (x0 the initial guess) */
} iga_stats;

/* Kernel classes that iga_profile can time (see iga_profile). */
#define IGA_PROF_OFF 0
#define IGA_PROF_MASS 1       /* the fused last-axis kernel of the matrix-free mass operator */
#define IGA_PROF_STIFF 2      /* the fused last-axis kernel of the matrix-free stiffness operator */
#define IGA_PROF_PRECOND 3    /* one whole preconditioner application (all mode products) */
#define IGA_PROF_MASS_APPLY 4 /* one whole mass-operator application (all passes) */
#define IGA_PROF_BAND_MASS 5  /* the band product of the assembled mass matrix */
#define IGA_PROF_BAND_STIFF 6 /* the band product of the assembled stiffness matrix */

typedef struct iga_handle iga_handle;

/* Fill *opt with the defaults listed above. */
void iga_options_default(iga_options* opt);

/* Static text for a status code. */
const char* iga_status_string(int status);

/* Message of the last failed call on h (empty string if none); valid until the
 * next call on h. h may be NULL for failures of iga_create. */
const char* iga_last_error(const iga_handle* h);

/*
 * iga_create -- set up one patch (Sec. 5.1-5.2).
 *   dim        2 or 3.
 *   degree     [dim] spline degrees p_a >= 1 (at most 6).
 *   nknots     [dim] knot-vector lengths; m_a = nknots[a] - p_a - 1 functions, m_a >= 3.
 *   knots      [dim] host pointers to open knot vectors on [0, 1] (first and last knot
 *              repeated p_a + 1 times, non-decreasing, interior multiplicity <= p_a).
 *   ctrl       host, full control net: prod_a m_a points, co-lexicographic, dim
 *              coordinates per point (point-major). The geometry is
 *              F(xi) = sum_i C_i B_i(xi).
 *   opt        options (NULL => defaults); copied.
 *   out        receives the handle.
 * All inputs are copied; the caller keeps ownership. Builds the univariate
 * Gauss tables, the geometric factors at every quadrature point (W = w|det DF|
 * and G = W DF^{-1} DF^{-T}), diag(M), and the fast-diagonalisation factors
 * Mhat_a = U_a Lambda_a U_a^T of the preconditioner. Returns IGA_EGEOMETRY if
 * det DF <= 0 at some quadrature point.
 */
int iga_create(int dim, const int* degree, const int* nknots, const double* const* knots, const double* ctrl,
               const iga_options* opt, iga_handle** out);

/* Release every resource of h (NULL is allowed). */
void iga_destroy(iga_handle* h);

/* Number of interior degrees of freedom N. */
int iga_ndof(const iga_handle* h, long long* ndof);

/*
 * iga_assemble -- build the assembled band rows of M and K (IGA_OP_ASSEMBLED form).
 * Idempotent. Called implicitly by the first operator use when op_form is
 * IGA_OP_ASSEMBLED. Memory: 2 * N * prod_a (2 p_a + 1) * 8 bytes of device memory.
 */
int iga_assemble(iga_handle* h);

/* Switch the operator form / preconditioner arithmetic / guess / tolerance of an
 * existing handle (same meanings as in iga_options). */
int iga_set_op_form(iga_handle* h, int op_form);
int iga_set_precond(iga_handle* h, int precond);
int iga_set_guess(iga_handle* h, int guess);
int iga_set_tol(iga_handle* h, double tol, int max_iter);

/*
 * iga_set_graphs -- on (default) lets iga_step replay one captured CUDA graph per
 * time step, whose PCG loop runs on the device (a conditional while node tests
 * convergence after every iteration): no host synchronisation inside a step. The
 * graph is captured on the first step of a configuration and re-captured when the
 * state buffer, k, dt, rho_inf, tolerance, max_iter, operator form, preconditioner
 * or guess change. Results are identical to the host-driven loop (off). Steps taken
 * while a kernel class is being profiled, and the first two steps of the PREV and
 * EXTRAP guesses, always use the host-driven loop.
 */
int iga_set_graphs(iga_handle* h, int on);

/*
 * iga_set_barrier_limit -- failure detection on the device (the paper has no
 * counterpart). With IGA_OP_ASSEMBLED_DF every band product first scales and splits
 * its input vectors in one cooperative launch whose blocks meet at a grid barrier;
 * a block waits there by polling a generation word (each poll sleeps at least
 * 64 ns) and gives up after `polls` polls: it then sets the handle's error word and
 * goes on, so the kernel always ends and the context stays usable, but the product
 * that followed is not to be used. The next checked call (iga_solve_M, iga_step,
 * iga_apply_Pinv, iga_autotune) returns IGA_ECUDA with a message, clears the error
 * word and resets the barrier's words; calls after it run normally.
 * polls < 0 restores the default (4,194,304 polls, about 0.3 s or more): a wait
 * that long only runs out if a block of the launch never arrives. Small values
 * exist to exercise this path (a limit of 0 gives up at the first poll). On a
 * multi-patch handle the limit applies to every patch. Drops captured step graphs.
 */
int iga_set_barrier_limit(iga_handle* h, long long polls);

/*
 * Operators (device pointers). x and y hold nvec vectors of N doubles each,
 * vector v at offset v*N; x and y must not overlap.
 *   iga_apply_M:    y = M x, [M]_ij = int B_i B_j |det DF| (Sec. 5.3, eq. mass_matrix).
 *   iga_apply_K:    y = K x, K_ij = int grad B_i . grad B_j (Galerkin form of eq. pde, omega = 1).
 *   iga_apply_Pinv: y = D^{-1/2} Dhat^{1/2} Mhat^{-1} Dhat^{1/2} D^{-1/2} x, the inverse of
 *                   the preconditioner of Sec. 5.3 (def:single_patch_prec, def:matrices_1),
 *                   in the arithmetic chosen by iga_options.precond.
 * 1 <= nvec <= 8.
 */
int iga_apply_M(iga_handle* h, int nvec, const double* x, double* y);
int iga_apply_K(iga_handle* h, int nvec, const double* x, double* y);
int iga_apply_Pinv(iga_handle* h, int nvec, const double* x, double* y);

/*
 * iga_apply_Pinv_noalloc -- the same preconditioner application as
 * iga_apply_Pinv (same arithmetic, same result), for callers that must not
 * allocate device memory at call time. The paper has no counterpart; this is a
 * deployment aid.
 *
 * Who needs it: iga_apply_Pinv keeps its intermediate buffers in the handle and
 * grows them with cudaMalloc the first time a larger nvec is seen. That is not
 * possible for callers whose device memory is already committed to another
 * allocator (a framework's caching pool, so a fresh cudaMalloc fails or
 * fragments), for real-time loops that forbid allocation after start-up, and
 * for code that must stay free of allocation calls while it runs. This entry
 * point instead uses a fixed scratch array built into the library: two buffers
 * of 1,048,576 doubles (16 MiB in total), which every GPU that loads the
 * library holds until the process exits. It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * Arguments as for iga_apply_Pinv (device pointers x, y of nvec*N doubles,
 * 1 <= nvec <= 8). nvec * N must not exceed 1,048,576; larger requests return
 * IGA_EINVAL with a message and do nothing.
 *
 * Set-up: the first call on each device looks up the device address of the
 * scratch array (with that device current) and keeps it together with the id of
 * the device's context. Make that first call before any stream capture. After a
 * cudaDeviceReset the array lives in a new context at a new address: the first
 * call there (again before any capture) looks it up anew; handles created before
 * the reset are void and must be recreated, as for every other call.
 * With the 16-bit tensor-core preconditioners the call waits for its kernels and
 * returns IGA_ECUDA if one of their bounded waits ran out. Every call on a device shares the one array and leaves the
 * last call's values in it (nothing in it needs to start at zero), so calls
 * whose kernels overlap on the GPU -- from different streams, threads or
 * handles on the same device -- race and corrupt each other; serialise them.
 */
int iga_apply_Pinv_noalloc(iga_handle* h, int nvec, const double* x, double* y);

/*
 * iga_solve_M -- solve M x_v = b_v for nvec independent right-hand sides by
 * preconditioned CG (Sec. 5.5), stopping each at ||r||_2 <= tol ||b||_2.
 * b, x: device, nvec*N doubles. use_x0 != 0 takes x as the initial guess, else
 * the null vector. iters (host, [nvec], may be NULL) receives the iteration
 * counts, relres (host, [nvec], may be NULL) the final ||r||/||b||.
 * Synchronises the stream. IGA_ENOT_CONVERGED / IGA_ENUMERIC on failure.
 */
int iga_solve_M(iga_handle* h, int nvec, const double* b, double* x, int use_x0, int* iters, double* relres);

/*
 * Fields at the Gauss points (Sec. 2 and 5.1: the quadrature that defines M, K and the
 * load vectors). The points are the tensor Gauss rule of the handle (nquad per element
 * and direction), point q = q0 + Q0 (q1 + Q1 q2) with q_a running over the Gauss points
 * of direction a element by element; Qt = prod_a Q_a. Single-patch handles only
 * (IGA_EINVAL on a multi-patch handle).
 *
 * iga_npoints -- Qt and, if Q is not NULL, Q_a per direction ([dim], host). Host only.
 */
int iga_npoints(const iga_handle* h, long long* Qt, int* Q);

/*
 * iga_gauss_points -- physical coordinates x = F(xi_q) (device [dim][Qt], coordinate-major)
 * and weights w_q |det DF(xi_q)| (device [Qt]) at the Gauss points; either may be NULL.
 * Asynchronous on the handle's stream.
 */
int iga_gauss_points(iga_handle* h, double* x, double* w);

/*
 * iga_evaluate -- g[v][q] = sum_i U[v][i] B_i(xi_q), the spline fields of nvec coefficient
 * vectors (device [nvec][N]) at the Gauss points (device [nvec][Qt]). 1 <= nvec <= 8.
 */
int iga_evaluate(iga_handle* h, int nvec, const double* U, double* g);

/*
 * iga_integrate -- b[v][i] = sum_q w_q |det DF_q| g[v][q] B_i(xi_q): the load vectors
 * int g B_i of nvec point fields (device [nvec][Qt] -> device [nvec][N]), with the same
 * quadrature as M (so iga_integrate of iga_evaluate(U) is M U). 1 <= nvec <= 8; the first
 * call at a given nvec allocates a [nvec][Qt] scratch that the handle keeps.
 */
int iga_integrate(iga_handle* h, int nvec, const double* g, double* b);

/*
 * iga_galpha_params -- the method's parameters for order 2k and user parameter
 * rho_inf in [0, 1] (Sec. 4.1, boxed formulas with rho_b = rho_s; eq. HOgamma):
 * alpha[k], beta[k], gamma[k] (host arrays, block j at index j-1).
 */
int iga_galpha_params(int k, double rho_inf, double* alpha, double* beta, double* gamma);

/*
 * iga_cfl -- largest eigenvalue of M^{-1} K by the Lanczos process in the M inner
 * product from a seeded start (at most iters steps, each one K product, one PCG
 * solve and one M product; it stops once the largest eigenvalue of the Lanczos
 * tridiagonal matrix changes by less than 1e-11 relative), and the critical step
 * tau_crit = sqrt(Theta_crit(rho_inf) / lambda_max), Theta_crit = 12(1+rho)(2-rho)/(rho^2-5rho+10),
 * the k-independent stability limit of the method (Sec. 3.2 and 4.1).
 * lambda_max and tau_crit are host pointers.
 */
int iga_cfl(iga_handle* h, double rho_inf, int iters, double* lambda_max, double* tau_crit);

/*
 * General model M U'' + C U' + K U = F (Sec. 2.1, eq. mp). Defaults: C = 0, F = 0,
 * t = 0.
 *
 * iga_set_damping -- Rayleigh damping C = aM M + aK K (aM, aK >= 0; both 0 = none).
 *   In block j of a step (eq. ho1) C acts on the predictor of the block's
 *   velocity-like variable, T_{s_j - 1} for j < k and X^n_{s_k - 1} for j = k, as K
 *   acts on T_{s_j - 2} / X^n_{s_k - 2}; aM != 0 costs one more mass product per step.
 * iga_set_forcing -- F(t) = sum_{m < nterm} G_m sin(omega_m t + phase_m), nterm <= 8,
 *   G device [nterm][N] (copied), omega / phase host. Block j uses the derivative
 *   F^{(s_j)} at t_{n+1} for j < k (alpha_f = 1) and at t_n for j = k (alpha_f = 0),
 *   by the closed form d^s/dt^s sin(w t + p) = w^s sin(w t + p + s pi/2).
 * iga_set_time / iga_get_time -- t_n of the handle's state (host double). Each
 *   step advances it by dt on the device and on the host; iga_state_init
 *   evaluates F^{(a)} at the current t and leaves it unchanged.
 * All return IGA_EINVAL for negative or non-finite values; the setters synchronise.
 */
int iga_set_damping(iga_handle* h, double aM, double aK);
int iga_set_forcing(iga_handle* h, int nterm, const double* G, const double* omega, const double* phase);
int iga_set_time(iga_handle* h, double t);
int iga_get_time(iga_handle* h, double* t);

/*
 * iga_state_init -- initial high-order data (Sec. 3, after eq. 4aup):
 * X_a = M^{-1}(F^{(a)}(t) - K X_{a-2} - C X_{a-1}), a = 0..3k-3, with X_{-2} = U0,
 * X_{-1} = V0 (C, F and t as set above; without them the even and odd chains are
 * solved in pairs).
 *   k      order parameter, 1 <= k <= 4 (order 2k).
 *   U0, V0 device, N doubles each.
 *   state  device, 3k*N doubles, caller-owned: rows U, V, A, L^1, ..., L^{3k-3}.
 * Also resets the per-handle history used by the PREV / EXTRAP guesses.
 * Synchronises the stream.
 */
int iga_state_init(iga_handle* h, int k, const double* U0, const double* V0, double* state);

/*
 * iga_step -- advance state (device, 3k*N doubles, layout of iga_state_init) by
 * nsteps explicit steps of size dt (Sec. 4, eq. ho1-ho3). Each step: Taylor
 * predictor, one batched K product over the k predicted vectors, k mass solves
 * by PCG (batched), fused update of the 3k variables. stats (host, may be NULL)
 * accumulates counters. Synchronises the stream.
 */
int iga_step(iga_handle* h, double* state, int k, double rho_inf, double dt, int nsteps, iga_stats* stats);

/*
 * iga_step_host -- iga_step on a HOST state buffer (3k*N doubles): copies the
 * state to the device, steps, and copies it back, inside the call.
 */
int iga_step_host(iga_handle* h, double* state_host, int k, double rho_inf, double dt, int nsteps,
                  iga_stats* stats);

/*
 * Profiling of one kernel class (no counterpart in the paper; measurement aid).
 * iga_profile(h, cls) brackets every later launch of that class on the handle's
 * stream with a pair of CUDA events (IGA_PROF_OFF stops). iga_profile_read
 * synchronises the stream and returns, since the last read: the summed device
 * time in ms, the number of timed launches, and the ALGORITHMIC floating-point
 * operations and DRAM bytes of those launches (the minimum work of the
 * operation, counted by the library from the sizes; not hardware counters).
 * All outputs are host pointers; any may be NULL.
 */
int iga_profile(iga_handle* h, int kernel_class);
int iga_profile_read(iga_handle* h, double* total_ms, long long* launches, double* flops, double* bytes);

/*
 * ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper). A two-layer 3-D convolutional
 * network on the interior control-point grid supplies the initial guess of the
 * k mass solves of each step (Sec. 4, eq. ho1); PCG still stops at the same
 * residual (Sec. 5.5), so the guess changes the iteration count, not the result.
 *
 * Network: y = conv2(R(relu(conv1(x)))), conv1 3 -> 16 and conv2 16 -> 1 channels,
 * 3x3x3 taps (tap t = e1 + 3 e2 + 9 e3 reads the neighbour at offset
 * (e1-1, e2-1, e3-1) along (i1, i2, i3)), zero padding, biases. Inputs,
 * activations and parameters are BF16 values (R rounds to nearest even), sums
 * FP32. Parameter vector: IGA_NET_NPARAM floats, W1 [o][c][t], b1, W2 [c][t], b2.
 *
 * Features of the solve M Z^n = b^n of one stage, from the same stage's right-hand
 * sides b^{n-1}, b^{n-2} and solutions Z^{n-1}, Z^{n-2}, with D = diag(M):
 *   E = 2 Z^{n-1} - Z^{n-2},  c0 = D^{-1}(b^n - 2 b^{n-1} + b^{n-2}),
 *   s0 = rms(c0), s1 = rms(Z^{n-1}) (1 where zero),
 *   x = BF16(FP32(c0/s0, Z^{n-1}/s1, Z^{n-2}/s1)),  guess = E + s0 y.
 * Training target t = (Z^n - E)/s0; loss sum (y - t)^2 / (2N) per sample; Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8), one sample per update.
 * ---------------------------------------------------------------------------
 */

/*
 * iga_ws_collect -- record training samples from later iga_step calls on h:
 * every solve of a step taken with IGA_GUESS_LEARNED and two steps of history
 * stores its features and target (10 bytes per dof on the device). capacity is the
 * number of samples (solves) to keep; recording stops when full. capacity = 0
 * stops recording and frees the samples. Steps taken while recording use the
 * host-driven loop (no step graph). Untrained, the learned guess is E.
 */
int iga_ws_collect(iga_handle* h, int capacity);
/* Number of samples recorded so far (host int). */
int iga_ws_samples(iga_handle* h, int* count);
/*
 * iga_ws_train -- `epochs` passes of Adam over the recorded samples (one sample
 * per update, order a seeded permutation per epoch), on the device with the
 * library's forward and backward kernels. The learning rate of update u of U
 * follows a cosine decay, lr (1 + cos(pi u / U)) / 2. epoch_loss (host, `epochs`
 * doubles, may be NULL) receives the mean loss of each epoch. Parameters not yet
 * set are first drawn by iga_ws_init_params(seed). Afterwards IGA_GUESS_LEARNED
 * uses the trained network. IGA_EINVAL without samples.
 */
int iga_ws_train(iga_handle* h, int epochs, double lr, unsigned long long seed, double* epoch_loss);
/* Draw the parameters: weights uniform in +-1/sqrt(fan_in) (81 for W1, 432 for W2)
 * from a splitmix64 stream seeded by seed, biases zero; resets Adam's moments. */
int iga_ws_init_params(iga_handle* h, unsigned long long seed);
/* Copy the FP32 parameters out (host, IGA_NET_NPARAM floats) / in (the network
 * counts as trained after a set). */
int iga_ws_get_params(iga_handle* h, float* theta_host);
int iga_ws_set_params(iga_handle* h, const float* theta_host);
/*
 * iga_ws_features -- the features of k solves (test hook for the kernels of the
 * learned guess). Device pointers, [k][N] each: b, b1, b2, z1, z2 (b1, b2, z1, z2
 * are overwritten by the moved histories b2 <- b1 <- b, z2 <- z1 <- E); x
 * [k][3][N] BF16 bits; E [k][N]; scales [k][2] = (s0, s1). Synchronises.
 */
int iga_ws_features(iga_handle* h, int k, const double* b, double* b1, double* b2, double* z1, double* z2,
                    unsigned short* x, double* E, double* scales);

/*
 * Handle-free network kernels (building blocks and test hooks). Device pointers;
 * grid n1 x n2 x n3 (N points), nb samples; stream is a cudaStream_t (NULL =
 * legacy default stream). They return IGA_EINVAL for non-positive sizes or a grid
 * beyond the launch limits, IGA_ECUDA if a launch fails; they do not synchronise.
 *   iga_net_forward:  x [nb][3][N] BF16 bits, theta IGA_NET_NPARAM floats ->
 *                     act [nb][16][N] BF16 bits, y [nb][N] floats.
 *   iga_net_backward: gradient of sum_s sum_p dy[s][p] y[s][p] with respect to
 *                     theta (grad, IGA_NET_NPARAM floats) from x, theta, the act of
 *                     iga_net_forward and dy [nb][N]; work: at least
 *                     iga_net_workspace_bytes(n1, n2, n3, nb) bytes.
 *   iga_net_adam:     one Adam update (step counts from 1) of n parameters with
 *                     moments m, v (floats, updated).
 */
int iga_net_forward(int n1, int n2, int n3, int nb, const unsigned short* x, const float* theta,
                    unsigned short* act, float* y, void* stream);
unsigned long long iga_net_workspace_bytes(int n1, int n2, int n3, int nb);
int iga_net_backward(int n1, int n2, int n3, int nb, const unsigned short* x, const float* theta,
                     const unsigned short* act, const float* dy, float* grad, void* work,
                     unsigned long long work_bytes, void* stream);
int iga_net_adam(int n, float* theta, const float* grad, float* m, float* v, int step, double lr, void* stream);

/*
 * ---------------------------------------------------------------------------
 * Launch tuning and batches of independent patches (no counterpart in the paper:
 * its multi-patch spaces are conforming and glued, Sec. 5.4; these patches share
 * nothing).
 * ---------------------------------------------------------------------------
 */

/* Band-product launch configuration of h (assembled operators): threads per block
 * 64, 96, 128, 256 or 512 (0 = 256; 96 counts as 256 outside the double-FP32 form)
 * and vectors per thread 1..4 sharing each coefficient load (0 = all of a call's
 * vectors, at most 4). In the IGA_OP_ASSEMBLED_DF form with a degree 2..4 along the
 * first direction: 96 threads select the tensor-map kernel with 128 rows per block
 * and two rows per thread, 128 threads the tensor-map kernel with one row per
 * thread (both up to 4 vectors per pass; blocks ordered in strips of direction-1
 * lines so that the transposed terms are read from L2), and 64 or 256 threads with
 * at most 2 vectors the bulk-copy staged kernel; one more warp issues the copies
 * (each block's rows, run by run, into a ring of shared-memory buffers ahead of use;
 * its bounded mbarrier waits report IGA_ECUDA on the next checked call if one runs
 * out). Every configuration computes each row with the same operations in the same
 * order, so results are bitwise equal. IGA_EINVAL for other values. */
int iga_set_band_config(iga_handle* h, int threads, int nv);

/*
 * iga_band_df_tiny -- the share of the terms of an interior row that the
 * IGA_OP_ASSEMBLED_DF products form as one FP32 multiply-add (the tiny slots: every
 * coefficient of the slot, after the matrix's power-of-two scaling, below 2^-24 of
 * its largest; taken at the two ends of each run of slots sharing their offsets along
 * directions 1 and 2), for M (frac_m) and K (frac_k); the other terms cost 12 FP32
 * operations. Host outputs, either may be NULL. Assembles the double-FP32 band first
 * if needed. IGA_EINVAL unless h's form is IGA_OP_ASSEMBLED_DF. A numerical choice of
 * this library: the paper has no counterpart.
 */
int iga_band_df_tiny(iga_handle* h, double* frac_m, double* frac_k);

/*
 * iga_autotune -- time every band-product configuration (threads 64/128/256/512 x
 * vectors per thread 1, 2, 4 up to nvec) on nvec vectors with h's assembled mass
 * matrix (assembled first if needed): one warm-up launch, then reps launches
 * between two CUDA events on h's stream. Keeps for h, among the shapes within 3 % of
 * the fastest, the one with the most vectors per thread (each band coefficient read
 * once for more vectors), and returns it in threads / nv (host, may be NULL).
 * 1 <= nvec <= 8, reps >= 1. Synchronises.
 */
int iga_autotune(iga_handle* h, int nvec, int reps, int* threads, int* nv);

typedef struct iga_batch iga_batch;

/* iga_batch_create -- a batch of npatch >= 1 independent patches. The handles stay
 * owned by the caller, must be on one device and must outlive the batch. */
int iga_batch_create(int npatch, iga_handle* const* patches, iga_batch** out);
void iga_batch_destroy(iga_batch* b);
/* Message of the last failed batch call (empty if none). */
const char* iga_batch_last_error(const iga_batch* b);

/*
 * iga_batch_step -- advance patch i (state states[i], device, layout of
 * iga_state_init) by nsteps steps of size dt[i] (host array of npatch), with k
 * and rho_inf common to the batch. One CUDA graph holds the step of every patch
 * (Taylor predictor, batched K, the PCG loop as a device-side conditional node,
 * stage update) as independent branches forked from and joined on one stream, so
 * a single graph launch advances the whole batch by one step; the graph is
 * captured once and replayed until a state pointer, a dt, an option or a
 * workspace of a patch changes. Each patch keeps its own options (operator
 * form, preconditioner, guess, tolerance, band configuration). Steps that need a
 * patch's host-driven loop (a guess still without history, recording samples,
 * profiling, graphs switched off) run through iga_step, one step for all patches
 * at a time. Work is ordered after earlier work on every patch's stream and before
 * later work on it. stats: host array of npatch entries (may be NULL), accumulated
 * per patch. Synchronises. The first failing patch's status is returned and its
 * message is in iga_batch_last_error.
 */
int iga_batch_step(iga_batch* b, double* const* states, int k, double rho_inf, const double* dt, int nsteps,
                   iga_stats* stats);

/*
 * iga_batch_set_persistent -- on != 0: iga_batch_step advances the whole batch with ONE
 * persistent, cooperative kernel launch per step (held in a CUDA graph): the blocks take
 * (patch, tile) work items phase after phase -- Taylor predictor, the batched K product
 * of every patch, PCG (mass products, the three axis phases of the Kronecker solve, the
 * vector updates) until every system of every patch has converged, stage update --
 * with a grid barrier between phases (bounded wait: a time-out returns IGA_ECUDA and the
 * step's results are not to be used; iga_set_barrier_limit of patch 0 sets the limit).
 * The per-system PCG scalars are reduced in a fixed order, so runs are reproducible;
 * they are not bitwise those of the graph path, whose reductions are grouped otherwise.
 * Forms (else IGA_EINVAL with a message, and the batch keeps the graph path): 3-D
 * patches of degree 1..4, FP64 band operators (IGA_OP_ASSEMBLED), on every patch the
 * band-Cholesky Kronecker preconditioner (IGA_PREC_BANDED, plain PCG, or
 * IGA_PREC_BANDED32, flexible PCG) or the BF16 fast diagonalisation (IGA_PREC_BF16,
 * flexible PCG: six mode products with matrix entries and inputs rounded to BF16 and
 * FP32 sums -- the tensor-core form's arithmetic, computed by the persistent blocks on
 * CUDA cores), the zero initial guess, no damping or loads, the same tolerance and
 * iteration limit on every patch. Work vectors (9 k N doubles per patch at most)
 * are allocated on the first step for a (k, rho_inf, dt, states) and kept. stats:
 * steps, solves, iterations, largest relative residual per patch; the launches are
 * counted on patch 0 (one per step). Semantics of the step otherwise as iga_batch_step.
 * The paper has no counterpart (its patches are glued, Sec. 5.4; these share nothing).
 */
int iga_batch_set_persistent(iga_batch* b, int on);

/*
 * iga_batch_phase_times -- where the last persistent iga_batch_step spent its time: ms
 * (host array of n) receives, summed over that call's steps, the milliseconds of each
 * kind of phase, measured on the device by block 0 of the persistent kernel from one
 * passed grid barrier to the next (a phase's time includes its barrier): [0] Taylor
 * predictor, [1] K product with the partials of b.b, [2] PCG scalars (the per-system
 * sums and alpha, beta, convergence, done by one block), [3] preconditioner (axis or
 * mode-product phases), [4] direction update, [5] M product with the partials of p.q,
 * [6] x and r update with the partials of r.r, [7] stage update (block 0's own end).
 * Entries past [7] are set to 0. IGA_EINVAL if the batch is not persistent or no
 * persistent step has completed since it was set up (or the last one timed out).
 * Measurement aid; the paper has no counterpart.
 */
int iga_batch_phase_times(iga_batch* b, double* ms, int n);

/*
 * iga_batch_set_persistent_variant / iga_batch_persistent_variant -- the launch variant
 * of the persistent step: 0 = three blocks of 256 threads per SM (80 registers per
 * thread), the band products loading two stored slots per pass; 1 = two blocks per SM
 * (128 registers), four slots per pass (k <= 2 only; with k > 2 variant 0 runs). Both
 * compute every term, reduction and update in the same order, so they give bitwise the
 * same results; they differ in speed. variant = -1 (the default): the batch times its
 * first persistent steps, each variant twice, alternating, and keeps the faster one for
 * the batch's life (the choice survives changes of k, rho, dt or states); 0 or 1 forces
 * that variant. iga_batch_persistent_variant returns in *variant the variant in use
 * (forced, chosen, or -1 while still timing) and in ms[0..1] (host, may be NULL) the
 * fastest timed step of each variant (-1 if never timed). IGA_EINVAL for another variant
 * number. The paper has no counterpart.
 */
int iga_batch_set_persistent_variant(iga_batch* b, int variant);
int iga_batch_persistent_variant(iga_batch* b, int* variant, double* ms);

/*
 * iga_probe_fp64_fma -- measured FP64 FMA throughput of `device` (no counterpart in
 * the paper; measurement aid): 8 independent FMA chains per thread, 4 blocks of 256
 * threads per SM, 2^14 iterations, averaged over 5 timed launches after 2
 * warm-up launches. tflops (host) receives the rate; sm_clock_ghz (host, may be
 * NULL) the device's nominal maximum SM clock. Allocates and frees a small buffer.
 */
int iga_probe_fp64_fma(int device, double* tflops, double* sm_clock_ghz);

#ifdef __cplusplus
}
#endif
#endif /* IGA_GALPHA_H */
