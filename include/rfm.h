/*
 * rfm.h -- C ABI of the GB300 (sm_103a) library for the random-feature-method
 * nonlinear solvers IPN and AMIPN (arXiv 2510.04170, "Robust and efficient
 * solvers for nonlinear PDEs based on random feature method").
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are device pointers (FP64 unless stated), contiguous,
 *    owned by the caller; the library never frees them.  Pointers named *_host
 *    are host memory.  The library owns every internal workspace of an
 *    rfm_problem and frees it in rfm_problem_destroy.
 *  - All device work is enqueued on the stream given to rfm_problem_create
 *    (NULL = legacy default stream).  Entry points that return host scalars
 *    synchronise that stream before returning.
 *  - Errors are returned as rfm_status; rfm_last_error() gives a thread-local
 *    message.  No entry point falls back to the CPU.
 *  - Layouts: a problem has m collocation rows and n = G * fields * M unknowns,
 *    ordered subdomain-major, then field, then feature.  Rows are ordered:
 *    interior (subdomain, field, grid point), interface (normal axis, left
 *    subdomain, field, derivative order, face point), boundary (axis, side lo/hi,
 *    subdomain, field, face point).
 */
#ifndef RFM_H
#define RFM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RFM_OK = 0,
  RFM_EINVAL = 1,      /* bad argument or size                                  */
  RFM_ENOMEM = 2,      /* device allocation failed                              */
  RFM_ECUDA = 3,       /* a CUDA call failed                                    */
  RFM_ENOCONV = 4,     /* solver hit its iteration cap (iterate still written)  */
  RFM_ERANK = 5,       /* a pivot of R was floored (warning; result written)    */
  RFM_ENONFINITE = 6,  /* a residual norm became NaN/Inf                        */
  RFM_ETIMEOUT = 7     /* a bounded device wait gave up (result invalid)        */
} rfm_status;

typedef struct rfm_problem rfm_problem;

/* Problem description (Sec. 2.2, Sec. 5): domain box [lo, hi], nsub[d]
 * subdomains per axis, M tanh features per subdomain and field with k, b ~
 * U[-feat_range, feat_range] drawn by Philox4x32-10 from `seed`; collocation
 * grids with q_int[b] points per axis on each subdomain (endpoints included),
 * q_bdy[b] / q_iface[b] points per axis on boundary / interface faces;
 * cont_order continuity orders C^0..C^{k-1} across interfaces.
 * pde_kind: 0 -Lap u + p0 u^3 = f; 1 Gray-Scott (2 fields: eps_u, eps_v, F, k);
 *           2 -div(a grad u) + p0 u^3 = f, a = 1 + 0.5 sin(2 pi x);
 *           3 kind 2 with source p1 prod sin(p2 pi x_d) and zero Dirichlet data;
 *           4 Lap u + p0 u + p1 cosh(u) = f (nonlinear Helmholtz, Sec. 6.2:
 *             p0 = -100, p1 = 10), u* = (2 + |x|^2) prod sin(pi x_d);
 *           5 -div((1 + u^2) grad u) = f (Sec. 3.2 benchmark),
 *             u* = (x + y + z) sin(pi x) sin(pi y) cos(pi z);
 *           6 -div((1 + |grad u|^2) grad u) = f (strongly nonlinear, Sec. 6.2),
 *             u* = sin(x(1-x)) sin(y(1-y)) e^(z+1/2).
 *           7 -div((1 + u^2) grad u) + u^3 - u + e^u = f (diffusion-reaction on
 *             the unit ball, Sec. 6.2), u* = |x|^2 prod sin(pi x_d).
 *           Kinds 4-7 are three-dimensional with one field; f and the Dirichlet
 *           data g = u* come from the manufactured u*.
 * geometry 1 (the unit ball, Sec. 6.2): the box [lo, hi] is split into the
 * subdomains as usual, interior and interface grid points with
 * x^2 + y^2 + z^2 < 1 are kept, and the Dirichlet rows sit at n_sphere points
 * of the unit sphere placed by the Fibonacci spiral (z_i = 1 - (2i+1)/N,
 * azimuth i pi (3 - sqrt 5)), each in the subdomain that contains it; rows are
 * interior, interface, then boundary points grouped by subdomain.  dim 3. */
typedef struct {
  int dim;
  double lo[3], hi[3];
  int nsub[3];
  int M;
  int fields;
  int q_int[3];
  int q_bdy[3];
  int q_iface[3];
  int cont_order;
  double feat_range;
  uint64_t seed;
  int pde_kind;
  double pde_params[8];
  int geometry;       /* 0: the box [lo, hi]; 1: the unit ball inside it (below) */
  int64_t n_sphere;   /* geometry 1: Dirichlet points on the unit sphere       */
} rfm_problem_desc;

enum { RFM_SKETCH_COUNT = 0, RFM_SKETCH_GAUSS = 1 };

/* Solver options (Sec. 6 defaults: gamma 3, eta 1e-6, eps 1e-10, tau_rel 1e-3,
 * m_max 3; row scale c 100, Sec. 5).  sketch_rows 0 means ceil(gamma n);
 * lsqr_max_iter 0 means 2n.  precision: 0 FP64 throughout; 1 the Gaussian
 * sketch product S J on the bf16 tensor cores emulated to FP64 accuracy
 * (digit splitting, exact level accumulation); 2 as 1 plus the QR trailing
 * update on the tensor cores the same way.  Residual, line search, LSQR and
 * the QR panels stay in FP64 at every level. */
typedef struct {
  int sketch_kind;
  double gamma;
  int64_t sketch_rows;
  double eta;
  double eps;
  int max_outer;
  int m_max;
  double tau_rel;
  double row_scale_c;
  int precision;
  int64_t lsqr_max_iter;
  double conlim;
} rfm_solve_opts;

/* Per-solve record mirroring the paper's reported columns (IT, NJ, LSQR steps,
 * preconditioning time, final ||F||).  Times in milliseconds (CUDA events). */
typedef struct {
  int status;
  int outer_iters;          /* IT */
  int n_jac;                /* NJ */
  int lsqr_iters_total;
  int lsqr_iters_max;
  int rank_flag;
  double final_resid;       /* ||W F(u)|| at the returned iterate */
  double t_assemble, t_sketch, t_qr, t_lsqr, t_linesearch, t_total;
} rfm_solve_info;

void rfm_default_opts(rfm_solve_opts* opts);
const char* rfm_last_error(void);

/* Builds the problem: uploads the subdomain/row tables, then draws the
 * features (Philox, Sec. 2.2) and the collocation points and right-hand sides
 * (Sec. 5) on the device.  `cuda_stream` is a cudaStream_t or NULL.
 * Errors: RFM_EINVAL for dim not in {2,3}, non-positive counts, fields not 1
 * or 2, cont_order not in {1,2}, pde_kind outside 0..7 or its dimension and
 * field count, geometry outside 0..1 (1 needs dim 3 and n_sphere > 0);
 * RFM_ENOMEM/RFM_ECUDA on device failures. */
rfm_status rfm_problem_create(const rfm_problem_desc* desc, void* cuda_stream, rfm_problem** out);
rfm_status rfm_problem_destroy(rfm_problem* p);

/* Sizes of the least-squares system F: R^n -> R^m of Sec. 3.2 (m = Q_I + Q_b
 * + Q_c rows): m rows, n unknowns, W = fields*M (width of a column block), G
 * subdomains, m_int / m_iface interior and interface row counts, and nnz the
 * stored Jacobian entries ((m + m_iface) * W: one W-wide block per row plus
 * the second block of each interface row).  Null outputs are skipped. */
rfm_status rfm_problem_sizes(const rfm_problem* p, int64_t* m, int64_t* n, int64_t* W,
                             int64_t* G, int64_t* m_int, int64_t* m_iface, int64_t* nnz);

/* Copies the feature table [G*fields*M][4] (k_1..k_d, b, zero padding) and
 * the row points [m][4] (x_1..x_d, padding) to device buffers (Sec. 2.2). */
rfm_status rfm_get_features(const rfm_problem* p, double* feat_dev);
rfm_status rfm_get_points(const rfm_problem* p, double* pts_dev);

/* Assembles F(c) and J(c) (Alg. 3 steps 1-4) and applies the row rescaling
 * lambda_i = c_scale / max_j |J_ij| (Sec. 5) to both; keeps the scaled J and
 * lambda inside the problem.  F_dev [m] (nullable) receives the scaled F,
 * lam_dev [m] (nullable) the row scales. */
rfm_status rfm_assemble(rfm_problem* p, const double* c_dev, double c_scale, double* F_dev, double* lam_dev);

/* Copies the stored scaled Jacobian J = [lambda A_int + mu dg/du; A_con;
 * A_bdy] (Sec. 5, rows scaled by lambda_i): Jp_dev [m][W] holds each row's
 * primary block (columns of subdomain e0), Js_dev [m_iface][W] the secondary
 * block of interface rows (subdomain e1); blk_dev (int32 [m][2], nullable)
 * gets (e0, e1) with e1 = -1 for non-interface rows.  RFM_EINVAL before the
 * first rfm_assemble. */
rfm_status rfm_get_jacobian(const rfm_problem* p, double* Jp_dev, double* Js_dev, int32_t* blk_dev);

/* Scaled residual W F(c) with the stored row scales (no Jacobian).  F_dev [m]
 * nullable; norm_host (nullable) receives ||W F(c)||. */
rfm_status rfm_residual(rfm_problem* p, const double* c_dev, double* F_dev, double* norm_host);

/* Sketch of the stored scaled J for Jacobian evaluation kJ (Sec. 4.1):
 * count sketch (B[h(i),:] += sigma(i) J[i,:]) or Gaussian sketch whose
 * entries are N(0,1) draws rounded to multiples of 2^-4 (each an integer of
 * magnitude <= 137 times 2^-4, exact in bfloat16).  s rows; B kept inside the
 * problem as an s x n column-major matrix.  B_dev (nullable, [n][s]
 * column-major) receives a copy. */
rfm_status rfm_sketch(rfm_problem* p, int kind, int64_t s, int kJ, double* B_dev);

/* Replaces the right-hand sides of the system (Alg. 3: the source f at the
 * interior rows, the Dirichlet data g at the boundary rows) with rhs_dev [m]
 * in row order; interface rows carry no data and stay 0.  By default a
 * problem uses the manufactured data of its pde_kind.  The residual is
 * F_i = (operator row) - rhs_i. */
rfm_status rfm_set_rhs(rfm_problem* p, const double* rhs_dev);

/* Limit on the device-side polls of the bounded flag waits (the grid barriers
 * of the QR panel factorisation and the block flags of the triangular solves)
 * of this problem: 0 restores the default (2^22 polls), a positive count sets
 * that many, a negative value makes every such wait give up at once (for
 * testing the RFM_ETIMEOUT path).  A wait that gives up sets the problem's
 * error word; the call reports RFM_ETIMEOUT and its result is invalid, and
 * the next call starts with a clear error word.  The paper has no
 * counterpart (failure detection of this library). */
rfm_status rfm_set_wait_limit(rfm_problem* p, int64_t polls);

/* Precision level (see rfm_solve_opts.precision) used by rfm_sketch and
 * rfm_qr; the solvers set it from their options.  RFM_EINVAL outside 0..2. */
rfm_status rfm_set_precision(rfm_problem* p, int precision);

/* Householder QR of the stored sketch (Sec. 4.1, thin QR B = QR); keeps R
 * (upper triangular, positive diagonal, pivots below 1e-14 max R_jj floored)
 * as the preconditioner.  R_dev (nullable, [n][n] column-major) receives R. */
rfm_status rfm_qr(rfm_problem* p, double* R_dev);

/* Installs a caller-supplied right preconditioner R (Sec. 4.1: the R factor
 * of the sketch, used as J R^{-1} in Alg. 1 step 3), n x n column-major upper
 * triangular, copied into a buffer the problem owns. */
rfm_status rfm_set_r(rfm_problem* p, const double* R_dev);

/* Standalone Householder R of an s x n column-major matrix (ld = s), the same
 * kernels as rfm_qr.  A_dev is overwritten; R_dev [n][n] column-major. */
rfm_status rfm_householder_r(double* A_dev, int64_t s, int64_t n, void* cuda_stream, double* R_dev,
                             int* rank_flag_host);

/* Householder R of an s x n column-major matrix (ld = s) with the trailing
 * update on the bf16 tensor cores emulated to FP64 accuracy (the precision-2
 * path of rfm_qr): 128-column outer blocks, FP64 panels inside a block, then
 * W = V^T A, W2 = T^T W, A -= V W2 as split products.  A_dev is overwritten;
 * R_dev [n][n] column-major.  Errors as rfm_householder_r. */
rfm_status rfm_householder_r_tc(double* A_dev, int64_t s, int64_t n, void* cuda_stream, double* R_dev,
                                int* rank_flag_host);

/* C (M x N, column-major, ldc) = A (M x K, lda) B (K x N, ldb), all FP64,
 * computed on the bf16 tensor cores by splitting each row of A and column of
 * B into `digits` 7-bit integer digits (exact in bf16) whose level sums are
 * accumulated exactly over 512-deep K chunks and combined in FP64 (1 <=
 * digits <= 8; 8 gives FP64-class error relative to |A||B|).  Allocates its
 * digit buffers; synchronises the stream. */
rfm_status rfm_emulated_dgemm(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                              int64_t M, int64_t N, int64_t K, int digits, void* cuda_stream);

/* Householder R of an s x n column-major matrix exactly like
 * rfm_householder_r, but without allocating device memory: for callers that
 * cannot call cudaMalloc while they run, such as services that reserve all
 * device memory up front in their own pool (where an allocation fails, or
 * implicitly synchronises the device and stalls other streams) and loops with
 * fixed latency budgets.  The paper has no counterpart; this is a deployment
 * variant of the QR step.
 *  - n <= 512 (RFM_EINVAL with a message otherwise); s >= n.
 *  - Scratch is a fixed 17.2 MB file-scope device array (plus 16 KB of barrier
 *    words) present on every GPU that loads the library until process exit.
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.
 *  - All calls share the array, which keeps the last call's contents: calls
 *    that overlap on the GPU (two streams or two host threads) race and must be
 *    serialised by the caller.
 *  - A_dev is overwritten; R_dev [n][n] column-major; the stream is
 *    synchronised before return. */
rfm_status rfm_householder_r_noalloc(double* A_dev, int64_t s, int64_t n, void* cuda_stream, double* R_dev,
                                     int* rank_flag_host);

/* y = J x (trans 0, x [n], y [m]) or y = J^T x (trans 1, x [m], y [n]) with
 * the stored scaled J: the products of the bidiagonalisation that LSQR
 * applies to J R^{-1} (Alg. 1 step 3). */
rfm_status rfm_jmv(rfm_problem* p, int trans, const double* x_dev, double* y_dev);

/* x = R^{-1} b (trans 0) or x = R^{-T} b (trans 1) with the stored R: the
 * preconditioner solves inside LSQR on J R^{-1} and the back-transformation
 * of the Newton direction d = R^{-1} y (Alg. 1 steps 3-4).  RFM_ETIMEOUT if a
 * bounded device wait gave up (x is then invalid). */
rfm_status rfm_trsv(rfm_problem* p, int trans, const double* b_dev, double* x_dev);

/* LSQR (Paige-Saunders) on J R^{-1} y ~ b with atol = btol = eta; returns the
 * Newton direction d = R^{-1} y in d_dev [n] (Alg. 1 steps 3-4).  The scalar
 * recurrences stay on the device; the iterations run in chunks of 16 that the
 * first call on a problem captures into a CUDA graph (on a private stream of
 * the problem) and later calls replay on the problem's stream; the graph is
 * rebuilt when R or the workspace moves.  While per-kernel profiling of the
 * LSQR kernels is on, the same kernels are launched one by one instead. */
rfm_status rfm_lsqr(rfm_problem* p, const double* b_dev, double eta, double conlim, int64_t max_iter,
                    double* d_dev, int* iters_host, int* istop_host);

/* Golden-section line search on phi(alpha) = ||W F(c + alpha d)|| over [0,1]
 * with the stored row scales (Alg. 1 step 5). */
rfm_status rfm_linesearch(rfm_problem* p, const double* c_dev, const double* d_dev, double f0,
                          double* alpha_host, double* fbest_host);

/* IPN (Alg. 1) and AMIPN (Alg. 2) from the initial guess in c_dev [n]
 * (overwritten with the result).  info (nullable) is filled.  AMIPN follows
 * Alg. 2 as printed: an early stop of the inner loop keeps J~ and R for the
 * next outer iteration, so from a poor guess it can stop on a stale Jacobian
 * (a steady Gray-Scott system from u_0 = 0 does); IPN re-linearises at every
 * step. */
rfm_status rfm_ipn_solve(rfm_problem* p, const rfm_solve_opts* opts, double* c_dev, rfm_solve_info* info);
rfm_status rfm_amipn_solve(rfm_problem* p, const rfm_solve_opts* opts, double* c_dev, rfm_solve_info* info);

/* u_n at query points (Sec. 2.2, Eq. 2.7 with the indicator PoU): pts_dev
 * [npts][dim] row-major, u_dev [npts][fields]. */
rfm_status rfm_eval(const rfm_problem* p, const double* c_dev, const double* pts_dev, int64_t npts,
                    double* u_dev);

/* ---- Batched solves (an addition of this library: many independent
 * instances of one PDE family, e.g. different subdomain grids, M and
 * coefficients, solved concurrently on one GPU).
 * rfm_batch_create builds `count` problems from descs[] and `streams` CUDA
 * streams (1..64), each served by one host worker during a solve.
 * rfm_batch_solve runs IPN (solver 0, Alg. 1) or AMIPN (solver 1, Alg. 2) on
 * every instance, largest n^2 s first; c_dev[i] is instance i's coefficient
 * vector (device, n_i doubles, initial guess in, solution out) and infos[i]
 * its record.  opts->precision = -1 lets the autotuner choose each
 * instance's QR configuration (tuned_precision_out[i], nullable, receives the
 * choice); 0..2 fixes it for all.  After its solve an instance frees its
 * sketch and QR buffers.  Returns the first hard error (with the instance in
 * rfm_last_error), else RFM_ENOCONV if any instance hit its iteration cap,
 * else RFM_OK.  Problems of a batch must not be used concurrently with its
 * solve. */
typedef struct rfm_batch rfm_batch;
rfm_status rfm_batch_create(const rfm_problem_desc* descs, int count, int streams, rfm_batch** out);
rfm_status rfm_batch_destroy(rfm_batch* b);
int rfm_batch_size(const rfm_batch* b);
rfm_problem* rfm_batch_problem(rfm_batch* b, int i);
rfm_status rfm_batch_solve(rfm_batch* b, const rfm_solve_opts* opts, int solver, double* const* c_dev,
                           rfm_solve_info* infos, int* tuned_precision_out);
/* QR autotuner: times the first 128 columns of a seeded random s x n
 * factorisation for the FP64 path (precision 0) and the tensor-core path
 * (precision 2), each with the panel factorisation capped at 16, 32, 64 and
 * all SMs' CTAs, and returns the fastest (cached per (s, n) for the process).
 * ms8_out (nullable) receives the eight probe times in ms, FP64 caps first,
 * then tensor-core caps, caps in the order above.  Allocates a probe matrix
 * of s*n doubles plus the QR buffers. */
rfm_status rfm_autotune_qr(int64_t s, int64_t n, void* cuda_stream, int* precision_out, int* panel_cap_out,
                           double* ms8_out);

/* ---- Learned warm start (an addition of this library; the paper starts
 * Newton from a fixed guess): an MLP maps PDE parameters to an initial
 * coefficient vector c_0 for rfm_ipn_solve / rfm_amipn_solve; c_0 = 0 remains
 * the fallback and the final Newton residual judges the result.
 * Network d_in -> H (tanh) -> H (tanh) -> d_out; inputs, weights and hidden
 * activations rounded to bfloat16, products accumulated in FP32, FP32 master
 * weights trained by Adam (beta 0.9/0.999, eps 1e-8).  Parameters are one flat
 * FP32 buffer with blocks W1 [H][d_in], b1, W2 [H][H], b2, W3 [d_out][H], b3
 * at the offsets rfm_mlp_params returns.  All pointers are device pointers
 * unless named *_host; batches are row-major [batch][dim] FP32. */
typedef struct rfm_mlp rfm_mlp;
rfm_status rfm_mlp_create(int d_in, int hidden, int d_out, uint64_t seed, void* cuda_stream, rfm_mlp** out);
rfm_status rfm_mlp_destroy(rfm_mlp* net);
int64_t rfm_mlp_num_params(const rfm_mlp* net);
/* Copies the master parameters out (dst_dev) and/or in (src_dev); offsets_host
 * (6 entries, nullable) receives the block offsets. */
rfm_status rfm_mlp_params(rfm_mlp* net, float* dst_dev, const float* src_dev, int64_t* offsets_host);
rfm_status rfm_mlp_forward(rfm_mlp* net, const float* x_dev, int batch, float* y_dev);
/* Gradient of L = (1/batch) sum_b (y_b - t_b)^T G (y_b - t_b) (G block diagonal
 * with d_out/gblk blocks of gblk x gblk, FP32 [blocks][gblk][gblk]; G_dev NULL
 * means G = I/d_out) into grad_dev [num_params]; loss_host receives L. */
rfm_status rfm_mlp_gradient(rfm_mlp* net, const float* x_dev, const float* t_dev, int batch, const float* G_dev,
                            int gblk, float* grad_dev, double* loss_host);
/* `steps` full-batch Adam steps on the same loss; loss_host gets the last L. */
rfm_status rfm_mlp_train(rfm_mlp* net, const float* x_dev, const float* t_dev, int batch, const float* G_dev, int gblk,
                         int steps, float lr, double* loss_host);
/* Per-subdomain Gram of the features at evaluation points (the metric above):
 * G[e*fields+f] = (1/npts) sum over points of subdomain e of phi_{e,f} phi_{e,f}^T,
 * FP32 [G*fields][M][M].  Points [npts][dim] must be grouped by owning
 * subdomain; owner_start_host (G+1 entries) delimits the groups. */
rfm_status rfm_feature_gram(const rfm_problem* p, const double* pts_dev, int64_t npts,
                            const int64_t* owner_start_host, float* G_dev);

/* Function-space basis for the warm start.  The N snapshot coefficient
 * vectors C [N][n] (converged solutions of one problem geometry) are centred
 * (mean_dev [n] receives cbar) and orthonormalised in the mean-square inner
 * product of u = Phi c over the npts points pts_dev [npts][dim] by modified
 * Gram-Schmidt with column pivoting (largest remaining norm first), stopping
 * when that norm falls to tol times the first.  U_dev [N][n] receives the
 * modes (first *rank_host rows), Z_dev [N][N] the coordinates: snapshot j is
 * cbar + sum_{k<rank} Z[j][k] U[k] up to the truncation.  Scratch is
 * allocated inside; runs on the problem's stream and synchronises. */
rfm_status rfm_function_basis(const rfm_problem* p, const double* C_dev, int N, const double* pts_dev, int64_t npts,
                              double tol, double* mean_dev, double* U_dev, double* Z_dev, int* rank_host);
/* c_dev [batch][n] = mean_dev + scale * y_dev [batch][rank] U_dev [rank][n]
 * (FP64 accumulation); synchronises cuda_stream. */
rfm_status rfm_basis_combine(const double* mean_dev, const double* U_dev, int64_t n, int rank, const float* y_dev,
                             int batch, double scale, double* c_dev, void* cuda_stream);

/* Warm-start object: the function-space basis of N training solutions
 * C_dev [N][n] (rfm_function_basis on the points pts_dev, tolerance tol), their
 * PDE parameters params_dev [N][d_in] (FP64; inputs are standardised per
 * dimension with the training mean and deviation), and a network
 * d_in -> hidden -> hidden -> rank trained on the coordinates divided by their
 * root mean square.  The network's loss is the mean square of the coordinate
 * error, which is the mean square of the error of u_0 over the points since
 * the modes are orthonormal there.  predict writes c_0 [batch][n] (FP64) for
 * params [batch][d_in].  Device pointers; the problem's stream is used. */
typedef struct rfm_warmstart rfm_warmstart;
rfm_status rfm_warmstart_create(const rfm_problem* p, const double* C_dev, const double* params_dev, int N, int d_in,
                                const double* pts_dev, int64_t npts, double tol, int hidden, uint64_t seed,
                                rfm_warmstart** out);
rfm_status rfm_warmstart_destroy(rfm_warmstart* w);
int rfm_warmstart_rank(const rfm_warmstart* w);
rfm_mlp* rfm_warmstart_network(rfm_warmstart* w);
rfm_status rfm_warmstart_train(rfm_warmstart* w, int steps, float lr, double* loss_host);
rfm_status rfm_warmstart_predict(rfm_warmstart* w, const double* params_dev, int batch, double* c_dev);

/* Benchmark instrumentation (not part of the method).  rfm_profile_enable(mask)
 * clears the counters and records a CUDA event pair around every launch of
 * the kernel families whose bit is set in mask (0 disables), on the stream the
 * kernel is launched on; rfm_profile_read synchronises and returns the
 * family's total milliseconds and launch count.  Family names:
 * rfm_profile_name(0 .. rfm_profile_count()-1).  rfm_launch_count() is the
 * number of kernels this library has launched in the process so far. */
rfm_status rfm_profile_enable(int mask);
int64_t rfm_launch_count(void);
/* Algorithmic work recorded for a profiled family since rfm_profile_enable:
 * bf16 tensor flops for oz_gemm, FP64 flops for sketch_gemm, bytes moved for
 * trsv, jmv, jtmv (R or J read once plus vectors) and assemble (J, F, lambda
 * written). */
rfm_status rfm_profile_work(int family, double* units);
int rfm_profile_count(void);
const char* rfm_profile_name(int family);
rfm_status rfm_profile_read(int family, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif
