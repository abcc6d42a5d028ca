/*
 * bta.h -- C ABI of the GB300 (sm_103a) library for the block-tridiagonal-
 * with-arrowhead (BTA) hot path of INLA on spatio-temporal (multivariate)
 * Gaussian processes (arXiv 2507.06938, "DALIA").
 *
 * Each evaluation of the INLA objective f_obj(theta) (Eq. 8) needs the prior
 * precision Q_p (Eq. 1, built from the SPDE / AR(1) / coregional model of
 * Sections II-A, II-B and IV-B) and the conditional precision
 * Q_c = Q_p + A^T D A (Eq. 4).  In the permuted order of Section IV-B.1 both
 * are BTA matrices with n = nt diagonal blocks of size b = nv*ns and an arrow
 * tip of size a = nv*nr, N = n*b + a (Section IV, structured-matrix table).
 * This library assembles them, factors them by block Cholesky, and computes
 * the log-determinant, the conditional-mean solve and the selected inverse
 * (Section III-A), all in CUDA kernels on one GPU.
 *
 * Conventions
 *  - Blocks are stored column-major in FP64, each block contiguous:
 *      D_i = Q[i,i]      (b x b, i = 0..n-1)
 *      B_i = Q[i+1,i]    (b x b, i = 0..n-2)
 *      R_i = Q[tip,i]    (a x b, i = 0..n-1)
 *      T   = Q[tip,tip]  (a x a)
 *    The factor uses the same layout (only the lower triangle of D_i and T is
 *    meaningful); the selected inverse Sigma = Q^{-1} restricted to the BTA
 *    pattern also uses it (D_i and T stored full and symmetric).
 *  - A vector of length N is ordered like the matrix: time block 0..n-1, each
 *    holding variable-major spatial nodes (v*ns + s), then the nv*nr fixed
 *    effects (v*nr + r).
 *  - Every call is asynchronous on the context's stream unless stated.  Device
 *    pointers passed in are borrowed: the caller owns them and keeps them
 *    alive until the stream has passed the call.  Host pointers are read
 *    before the call returns.
 *  - Every function returns BTA_OK or an error code; no error is raised by a
 *    device trap.  Errors found on the device (a non-positive pivot, a
 *    non-finite result) are recorded in a status word of the context and
 *    returned by bta_sync().
 */
#ifndef BTA_H
#define BTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define BTA_OK 0
#define BTA_ERR_ARG 1        /* invalid argument (size, pointer, enum)          */
#define BTA_ERR_OOM 2        /* device allocation failed                        */
#define BTA_ERR_NOT_PD 3     /* non-positive pivot: matrix not positive definite
                                (bta_last_info gives the global row index)      */
#define BTA_ERR_TIMEOUT 4    /* a bounded device wait ran out                    */
#define BTA_ERR_NONFINITE 5  /* NaN or Inf in an input or a result               */
#define BTA_ERR_CUDA 6       /* a CUDA runtime call failed                       */
#define BTA_ERR_STATE 7      /* call out of order (e.g. solve before factor)     */

/* Which matrix of a pair.  A context holds `batch` pairs (parameter slots);
 * the matrix argument `which` of the per-matrix calls is 2 * slot + kind,
 * so for a context of one slot it is BTA_QP or BTA_QC. */
#define BTA_QP 0             /* prior precision Q_p (Eq. 1)                      */
#define BTA_QC 1             /* conditional precision Q_c = Q_p + A^T D A (Eq. 4) */

/* Arithmetic of the factorisation / selected inversion. */
#define BTA_FP64 0           /* every operation in FP64                          */
#define BTA_MIXED 1          /* tensor-core split-precision products, 35-bit
                                digits (5 bf16 slices per FP64 value)           */
#define BTA_MIXED_HI 2       /* the same with 49-bit digits (7 slices), for
                                ill-conditioned models (irregular meshes whose
                                precision has a condition number near 1e10)     */

/* Block kinds for bta_block_ptr. */
#define BTA_BLK_D 0
#define BTA_BLK_B 1
#define BTA_BLK_R 2
#define BTA_BLK_T 3

/* Storage selector for bta_block_ptr. */
#define BTA_STORE_Q 0        /* the assembled matrix                             */
#define BTA_STORE_L 1        /* its Cholesky factor                              */
#define BTA_STORE_SIGMA 2    /* its selected inverse                             */
#define BTA_STORE_LINV 3     /* inverses of the diagonal factor blocks (D, T)    */

typedef struct bta_model_s* bta_model_t;
typedef struct bta_ctx_s* bta_ctx_t;

/*
 * Model description (host arrays, read during bta_model_create only).
 *  nv, ns, nt, nr  response variables, mesh nodes, time steps, fixed effects
 *                  per variable (Section IV-B: N = nv (ns nt + nr)).
 *  nodes           ns x 2 row-major node coordinates.
 *  tri, n_tri      n_tri x 3 row-major node indices of the P1 triangles.
 *  m               number of observations; for each k < m:
 *  obs_var[k]      response variable (0..nv-1), obs_time[k] time step,
 *  obs_xy[2k..]    location, obs_tri[k] triangle containing it,
 *  X[k*nr + r]     covariate r (fixed effect r of variable obs_var[k]),
 *  y[k]            observed value.
 *  beta_prior_prec prior precision of every fixed effect before mixing.
 *  theta0          prior mean of the hyperparameters (length
 *                  4 nv + nv(nv-1)/2), used by the hyperprior of fobj_eval.
 */
typedef struct {
    int nv, ns, nt, nr;
    const double* nodes;
    const int* tri;
    int n_tri;
    int m;
    const int* obs_var;
    const int* obs_time;
    const double* obs_xy;
    const int* obs_tri;
    const double* X;
    const double* y;
    double beta_prior_prec;
    const double* theta0;
} bta_model_desc;

/*
 * bta_model_create -- theta-independent set-up (Sections II-A.1, II-A.2):
 * P1 lumped mass C and stiffness G on the mesh, G C^{-1} G, barycentric
 * interpolation of every observation, the per-(variable, time step) Gram
 * matrices of the observation operator and A^T y, uploaded to the device.
 * Synchronous.  Returns BTA_ERR_ARG for inconsistent sizes or indices.
 * The model is owned by the library until bta_model_destroy.
 */
int bta_model_create(const bta_model_desc* desc, bta_model_t* out);
int bta_model_destroy(bta_model_t model);
/* Sizes of a model: n = nt, b = nv*ns, a = nv*nr, dim(theta). */
int bta_model_dims(bta_model_t model, int* n, int* b, int* a, int* dim_theta);

/*
 * bta_create -- a context for BTA matrices with n diagonal blocks of size b
 * and arrow tip a (n >= 1, b >= 1, a >= 0), the arithmetic `precision`
 * (BTA_FP64, BTA_MIXED or BTA_MIXED_HI) and the CUDA stream `stream` (a cudaStream_t; NULL
 * = legacy default stream).  The context allocates and owns the device
 * storage of Q_p and Q_c, their factors and inverse diagonal factor blocks;
 * selected-inverse storage is allocated on the first bta_selinv of a matrix.
 * Synchronous.  BTA_ERR_OOM if the device memory does not suffice.
 */
int bta_create(int n, int b, int a, int precision, void* stream, bta_ctx_t* out);
/* bta_create_batched -- the same with `batch` parameter slots, i.e. storage
 * for batch pairs (Q_p, Q_c).  fobj_eval runs every slot's pair through the
 * same kernel launches (the 2 dim(theta) + 1 central-difference points of
 * Eq. 10 and the two matrices of each are independent, Sections IV-D.1 and
 * IV-D.2).  bta_create is bta_create_batched with batch = 1. */
int bta_create_batched(int n, int b, int a, int precision, int batch, void* stream, bta_ctx_t* out);
/* bta_create_ex -- bta_create_batched with creation flags: 0, or
 * BTA_CREATE_LOW_MEMORY to allocate the low-memory layout of
 * bta_set_low_memory from the start (the default layout of the same batch
 * may not fit at all).  BTA_ERR_ARG for unknown flags. */
#define BTA_CREATE_LOW_MEMORY 1
int bta_create_ex(int n, int b, int a, int precision, int batch, int flags, void* stream, bta_ctx_t* out);
int bta_batch_size(bta_ctx_t ctx, int* batch);
int bta_destroy(bta_ctx_t ctx);

/*
 * bta_assemble -- write matrix `which` (BTA_QP or BTA_QC) of `model` into
 * the context's Q storage for the model parameters `params_dev` (device
 * array, layout [kappa, tau, rho, sigma, tau_eps] per variable followed by
 * the nv(nv-1)/2 coregionalisation coefficients lambda):
 *   Q_s^u = tau_u^2 (kappa_u^4 C + 2 kappa_u^2 G + G C^{-1} G)   (SPDE, II-A.1)
 *   Q_t^u = stationary AR(1) precision with coefficient rho_u
 *   Q^u   = blockdiag(Q_t^u (x) Q_s^u, beta_prior_prec I_nr)
 *   Q_p   = Lambda^{-T} blockdiag(Q^u) Lambda^{-1}                 (Eq. 11)
 *   Q_c   = Q_p + A^T D A                                         (Eq. 4)
 * permuted to BTA order (Section IV-B.1).  Every entry of every block is
 * written (zeros outside the sparsity pattern).
 */
int bta_assemble(bta_ctx_t ctx, bta_model_t model, const double* params_dev, int which);

/* bta_theta_to_params -- device map theta -> params (layout above) of
 * length 5 nv + nv(nv-1)/2: kappa = sqrt(8)/exp(theta_0), tau^2 =
 * 1/(4 pi kappa^2), rho = exp(-1/exp(theta_1)), sigma = exp(theta_2),
 * tau_eps = exp(theta_3) per variable; lambda copied. */
int bta_theta_to_params(bta_ctx_t ctx, bta_model_t model, const double* theta_dev,
                        double* params_dev);

/*
 * bta_factor -- block Cholesky Q = L L^T of matrix `which` (Section III-A):
 * for i = 0..n-1: L_ii = chol(D_i), L_{i+1,i} = B_i L_ii^{-T},
 * D_{i+1} -= L_{i+1,i} L_{i+1,i}^T, L_{t,i} = R_i L_ii^{-T},
 * R_{i+1} -= L_{t,i} L_{i+1,i}^T, T -= L_{t,i} L_{t,i}^T; L_tt = chol(T).
 * Also keeps L_ii^{-1} and L_tt^{-1}.  The assembled Q is left intact.
 * A non-positive pivot records BTA_ERR_NOT_PD in the status word.
 */
int bta_factor(bta_ctx_t ctx, int which);
/*
 * bta_set_time_partitions -- factor, solve and selectively invert this
 * context's matrices by time-domain partitioning (Sections IV-C, IV-D.3;
 * the nested dissection over time of the distributed solver, run here as one
 * batch on one GPU): P - 1 separator blocks sigma_p = p h - 1, with
 * h = ceil((n + 1) / P), cut the n time blocks into P partitions whose
 * interiors are eliminated together (every (matrix, partition) pair is one
 * instance of the same batched launches), then the separators form a reduced
 * BTA system of P - 1 blocks.  The sequential chain shrinks from n to about
 * n/P + P steps at the price of extra fill products, which pays for small
 * blocks.  P = 1 restores the sequential recurrences.
 * Requires n - (P - 1) h >= 1 (the last partition holds an interior block)
 * and a <= b; otherwise BTA_ERR_ARG and nothing changes.  The block arrays are
 * re-laid out with P h slots per matrix (padding included) and the
 * partitioned path adds two arrays of that size (fill rows of the factor and
 * of the selected inverse) plus per-instance scratch.  Assembled Q matrices
 * are kept; factors, selected inverses and any captured f_obj graph are
 * dropped.  Results agree with the sequential path up to rounding; a
 * non-positive pivot is still reported as BTA_ERR_NOT_PD with the right
 * matrix, but the row given by bta_last_info is then the row inside the
 * failing block's partition.  Synchronises the device.  Errors:
 * BTA_ERR_ARG, BTA_ERR_OOM (the context is then back in the sequential
 * layout, or has no storage left and must be destroyed), BTA_ERR_CUDA.
 */
int bta_set_time_partitions(bta_ctx_t ctx, int P);

/*
 * bta_set_low_memory -- keep this context's matrices in a layout that needs
 * about 0.6 of the default device memory at large n, so that more theta
 * points fit in one batch of the largest models (Section III-A's factor,
 * selected inversion and solve, unchanged in arithmetic):
 *   - the inverse diagonal factor blocks L_ii^{-1} replace L_ii in the
 *     factor's diagonal blocks (the log-determinant is summed while the blocks
 *     are factored), L_tt^{-1} taking a spare block slot;
 *   - the selected inverse overwrites the factor.
 * Per matrix that is Q (n diagonal, n - 1 off-diagonal blocks), the factor
 * (n + 1 and n + 1) and one b x b buffer, against Q, the factor, Sigma and n
 * inverse blocks.  Consequences: after bta_selinv, bta_selinv_batch or
 * bta_fobj_grad the matrix counts as not factored (bta_solve, bta_logdet and
 * bta_selinv return BTA_ERR_STATE until the next factorisation), and the
 * factor's diagonal blocks read through bta_block_ptr hold L_ii^{-1}
 * (BTA_STORE_L, BTA_STORE_LINV and, after the selected inversion,
 * BTA_STORE_SIGMA name the same memory).  enable = 0 restores the default
 * layout (bta_create_ex with BTA_CREATE_LOW_MEMORY starts in the low-memory
 * one).  Assembled Q matrices are kept; factors, selected inverses and a
 * captured f_obj graph are dropped.  BTA_ERR_STATE with time partitions
 * (P > 1); BTA_ERR_OOM if the new layout cannot be allocated (the context
 * then keeps the default one, or has no factor storage and must be
 * destroyed).  Synchronises the device.
 */
int bta_set_low_memory(bta_ctx_t ctx, int enable);

/* bta_factor_batch -- bta_factor of every slot's matrix of kind BTA_QP or
 * BTA_QC in one pass (all matrices in the same launches). */
int bta_factor_batch(bta_ctx_t ctx, int kind);

/* bta_logdet -- log|Q| = 2 sum_k log L_kk of factored matrix `which`
 * (Eq. 1), accumulated in FP64, written to the device scalar *out_dev. */
int bta_logdet(bta_ctx_t ctx, int which, double* out_dev);

/*
 * bta_solve -- x = Q^{-1} rhs for factored matrix `which` by forward and
 * backward block substitution (rhs_dev, x_dev: device vectors of length N;
 * they may alias).  refine_iters >= 0 steps of iterative refinement
 * x += Q^{-1}(rhs - Q x) with an FP64 residual on the assembled blocks.  If
 * resid_dev is not NULL it receives ||rhs - Q x||_2 / ||rhs||_2.
 */
int bta_solve(bta_ctx_t ctx, int which, const double* rhs_dev, double* x_dev,
              int refine_iters, double* resid_dev);

/*
 * bta_selinv -- selected inverse Sigma = Q^{-1} on the BTA pattern of
 * factored matrix `which` (Section III-A, selected inversion):
 * Sigma_tt = L_tt^{-T} L_tt^{-1}; for i = n-1..0 with G_i = L_{i+1,i} L_ii^{-1},
 * F_i = L_{t,i} L_ii^{-1}:
 *   Sigma_{i+1,i} = -Sigma_{i+1,i+1} G_i - Sigma_{t,i+1}^T F_i
 *   Sigma_{t,i}   = -Sigma_{t,i+1} G_i - Sigma_tt F_i
 *   Sigma_ii      = L_ii^{-T} L_ii^{-1} - Sigma_{i+1,i}^T G_i - Sigma_{t,i}^T F_i.
 */
int bta_selinv(bta_ctx_t ctx, int which);
/* bta_selinv_batch -- bta_selinv of every slot's matrix of kind BTA_QP or
 * BTA_QC in one pass; all of them must be factored. */
int bta_selinv_batch(bta_ctx_t ctx, int kind);

/* bta_selinv_diag -- gather the diagonal of the selected inverse of matrix
 * `which` (the marginal variances of Section III, latent marginals) into
 * the device vector out_dev of length N.  BTA_ERR_STATE before bta_selinv. */
int bta_selinv_diag(bta_ctx_t ctx, int which, double* out_dev);

/* bta_block_ptr -- device address of block (kind, i) of storage `store`
 * of matrix `which`; *ld_out receives its leading dimension.  BTA_ERR_STATE
 * if that storage does not exist yet. */
int bta_block_ptr(bta_ctx_t ctx, int which, int store, int kind, int i,
                  double** ptr_out, int* ld_out);

/* bta_matvec -- y = Q x with the assembled blocks of matrix `which`
 * (device vectors of length N, no aliasing). */
int bta_matvec(bta_ctx_t ctx, int which, const double* x_dev, double* y_dev);

/*
 * fobj_eval -- f_obj(theta) of Eq. 8 for n_theta hyperparameter vectors
 * (thetas_dev: device, n_theta x dim(theta) row-major), evaluated at the
 * conditional mean x = mu with the hyperprior log p(theta) = sum_i
 * log N(theta_i; theta0_i, 1):
 *   f = log p(theta) + 1/2 log|Q_p| - 1/2 log|Q_c| - 1/2 (y^T D y - b^T mu)
 *       + 1/2 sum_k log d_k - (m/2) log 2 pi,   b = A^T D y, mu = Q_c^{-1} b,
 * which equals log p(theta) + log l(y|theta,mu) + log p(mu|theta)
 * - log p_G(mu|theta,y) because y^T D y - b^T mu = (y - A mu)^T D (y - A mu)
 * + mu^T Q_p mu.  f_out_dev receives n_theta values.  If mu_out_dev is not
 * NULL it receives the n_theta conditional means (n_theta x N, row j for
 * theta j).  The thetas are evaluated in groups of the context's batch size,
 * each group's 2 x batch matrices going through the same launches (a last,
 * partial group factors its Q_p and Q_c in two passes, as their storage
 * ranges are not adjacent; a context of batch 1 keeps single points in one); in
 * mixed precision the solve takes two refinement steps with an FP64
 * residual.  Afterwards slot j holds the matrices and factors of theta
 * (last group start + j).  From the second full group on, a full group is
 * replayed from a CUDA graph captured on the context's stream (the thetas
 * are first copied into a context buffer), so the stream must not be
 * capturing already; BTA_GRAPH=0 in the environment turns this off.
 */
int fobj_eval(bta_ctx_t ctx, bta_model_t model, const double* thetas_dev, int n_theta,
              double* f_out_dev, double* mu_out_dev);

/*
 * bta_fobj_grad -- f_obj and its gradient with respect to theta for n_theta
 * hyperparameter vectors (device, n_theta x dim(theta)), by the adjoint form
 * of Eq. 8 for a Gaussian likelihood instead of the central differences of
 * Eq. 10 (b = A^T D y, mu = Q_c^{-1} b, Sigma = Q^{-1}):
 *   df/dtheta_k = d log p(theta) + 1/2 tr(Sigma_p dQ_p) - 1/2 tr(Sigma_c dQ_c)
 *                 - 1/2 y^T dD y + db^T mu - 1/2 mu^T dQ_c mu + 1/2 tr(D^{-1} dD).
 * Runs fobj_eval, the selected inversion of every Q_p and Q_c of a group,
 * and the trace kernels; the traces need Sigma only on the BTA pattern.
 * f_out_dev receives n_theta values, grad_out_dev n_theta x dim(theta).
 */
int bta_fobj_grad(bta_ctx_t ctx, bta_model_t model, const double* thetas_dev, int n_theta, double* f_out_dev,
                  double* grad_out_dev);

/*
 * bta_fobj_grad_host -- bta_fobj_grad for a caller whose data lives in host
 * memory: thetas (host, n_theta x dim(theta) row-major) are copied to the
 * device, f_obj and its gradient are computed as by bta_fobj_grad, and
 * f_out (host, n_theta values), grad_out (host, n_theta x dim(theta)) and,
 * if var_out (host, n_theta x N) is not NULL, the marginal variances
 * diag(Sigma_c) of every theta (Section III, latent marginals) are copied
 * back.  Pinned host buffers let the copies run asynchronously.  Returns
 * when the results are in host memory, with the status of bta_sync.  The
 * first call allocates the device staging buffers of the context.
 */
int bta_fobj_grad_host(bta_ctx_t ctx, bta_model_t model, const double* thetas, int n_theta, double* f_out,
                       double* grad_out, double* var_out);

/*
 * bta_fobj_eval_multi -- f_obj (and, where asked, its gradient) for `count`
 * independent problems that may differ in shape, e.g. univariate models of
 * several (ns, nt) evaluated together: the independent function evaluations
 * of Section IV-D.1 without the constraint that they share one model.  One
 * context and one model per problem.  Each problem runs fobj_eval, or
 * bta_fobj_grad when grad_out_dev[i] is not NULL, asynchronously on its own
 * context's stream, so problems whose contexts were created on distinct
 * streams overlap on the GPU; then `join` waits (events) for all of them, so
 * that work queued on `join` afterwards sees every result.
 *   count:        number of problems, >= 1.
 *   ctxs, models: count handles (host arrays); ctxs[i] must have the (n, b, a)
 *                 of models[i].  A context may appear more than once; its
 *                 problems then run one after the other.
 *   thetas_dev:   count device pointers, n_theta[i] x dim(theta of model i).
 *   n_theta:      count host ints >= 1.
 *   f_out_dev:    count device pointers, n_theta[i] values each.
 *   mu_out_dev:   NULL, or count device pointers (entries may be NULL), each
 *                 n_theta[i] x N_i conditional means (fobj_eval problems only).
 *   grad_out_dev: NULL, or count device pointers (entries may be NULL), each
 *                 n_theta[i] x dim(theta of model i).
 *   join:         a cudaStream_t (NULL: the legacy default stream).  Every
 *                 problem's stream first waits for the work queued on `join`
 *                 before the call (so inputs written there are complete),
 *                 and `join` then waits for every problem.
 * Returns BTA_ERR_ARG before launching anything if an argument is invalid,
 * else the first error of a launch; the problems launched until then are
 * still joined.  Device errors are read per context with bta_sync.
 */
int bta_fobj_eval_multi(int count, const bta_ctx_t* ctxs, const bta_model_t* models,
                        const double* const* thetas_dev, const int* n_theta, double* const* f_out_dev,
                        double* const* mu_out_dev, double* const* grad_out_dev, void* join);

/* Likelihoods of bta_fobj_laplace. */
#define BTA_LIK_GAUSSIAN 0   /* y_k ~ N(eta_k, 1/tau_eps of the variable)        */
#define BTA_LIK_POISSON 1    /* y_k ~ Poisson(exp(eta_k)), counts                 */

/*
 * bta_fobj_laplace -- f_obj (Eq. 8) for a non-Gaussian likelihood by the
 * Laplace approximation at the mode x* of the latent field (Section II-A.3:
 * p_G from a second-order Taylor expansion of the log-likelihood ell,
 * Q_c(x) = Q_p + A^T D(x) A with D the negative Hessian of ell in the linear
 * predictor eta = A x, Eq. 4).  x* is found by newton_iters (1..1000) Newton
 * steps from x = 0, each an assembly of Q_c(x_k) with per-observation
 * weights, a block Cholesky and a solve of Q_c(x_k) x_{k+1} = A^T (g + D eta)
 * with g = d ell / d eta (refined with an FP64 residual in mixed precision);
 * then Q_c(x*) is assembled and factored once more and
 *   f = log p(theta) + ell(y | x*) + 1/2 log|Q_p| - 1/2 x*^T Q_p x*
 *       - 1/2 log|Q_c(x*)|.
 * likelihood: BTA_LIK_POISSON (log link; y of the model are counts) or
 * BTA_LIK_GAUSSIAN (the f of fobj_eval, reached in one step).  thetas_dev:
 * device, n_theta x dim(theta) (the noise-precision entries enter only the
 * hyperprior for Poisson data).  f_out_dev: n_theta values; x_out_dev (NULL
 * or n_theta x N): the modes; step_out_dev (NULL or n_theta): max |x_K -
 * x_{K-1}| of the last Newton step, a convergence measure.  Groups of the
 * context's batch run through the same launches.  Afterwards the Q_p and
 * Q_c(x*) storage of slot j hold the last group's matrices and factors.
 */
int bta_fobj_laplace(bta_ctx_t ctx, bta_model_t model, const double* thetas_dev, int n_theta, int likelihood,
                     int newton_iters, double* f_out_dev, double* x_out_dev, double* step_out_dev);

/* bta_fobj_residual -- accuracy of the conditional means of the last
 * fobj_eval / bta_fobj_grad group: out_dev (device, batch values) receives
 * ||b - Q_c mu||_2 / ||b||_2 for every parameter slot (slot j holds theta
 * (last group start + j)), b = A^T D y, computed in FP64 with the assembled
 * blocks of Q_c (the refinement residual of Section III-A's solve stated as
 * an error measure).  BTA_ERR_STATE before the first f_obj evaluation. */
int bta_fobj_residual(bta_ctx_t ctx, double* out_dev);

/* bta_fp64_peak -- measured FP64 throughput of the current GPU (TFLOP/s),
 * the denominator of the FP64 path's roofline: a loop of independent FP64
 * fused multiply-adds (use_dmma = 0) or of FP64 tensor-core MMAs
 * (mma.sync m8n8k4, use_dmma = 1) over every SM, timed with CUDA events
 * after one warm-up launch.  Synchronous; allocates and frees a small
 * device buffer.  Measurement aid, no counterpart in the paper. */
int bta_fp64_peak(int use_dmma, double* tflops_out);

/* bta_sync -- wait for the context's stream; return the first error the
 * device recorded since the last bta_sync (and clear it), else BTA_OK. */
int bta_sync(bta_ctx_t ctx);
/* bta_last_info -- detail of the last device error: for BTA_ERR_NOT_PD the
 * global row index (0..N-1) of the first non-positive pivot, else -1.
 * bta_last_error_matrix -- the matrix (2 * slot + kind) it occurred in, -1
 * if none. */
int bta_last_info(bta_ctx_t ctx, long long* info);
int bta_last_error_matrix(bta_ctx_t ctx, int* which);
/* bta_strerror -- static text of a return code. */
const char* bta_strerror(int code);

/* bta_launch_count -- number of CUDA kernels this library has launched in
 * this process (host-side counter; all contexts). */
long long bta_launch_count(void);

/* bta_profile -- when enable != 0, record CUDA events around the two
 * b x b x b Schur-update GEMM launches of every factorisation step of this
 * context.  bta_profile_read synchronises those events and returns their
 * summed duration (ms), the number of timed launches and their nominal flops
 * (b^3 per matrix each).  When fobj_eval replays its CUDA graph, the events
 * are those of the last replay.  Measurement aid; no effect on results. */
int bta_profile(bta_ctx_t ctx, int enable);
int bta_profile_read(bta_ctx_t ctx, double* ms_total, long long* launches, double* flops_total);

/* bta_profile_phases -- durations (ms, CUDA events) of the phases of the
 * last group of theta points that bta_fobj_grad evaluated while profiling was
 * enabled: [0] theta map and assembly of Q_p and Q_c (Section IV-B),
 * [1] factorisations and log-determinants (Section III-A), [2] right-hand
 * side, solve with refinement and f (Eq. 8), [3] selected inversions,
 * [4] adjoint traces and gradient.  Writes min(count, BTA_PHASES) values to
 * ms_out (host) and synchronises the events.  BTA_ERR_STATE if no such group
 * ran since profiling was enabled; BTA_ERR_ARG for a null pointer or
 * count < 1.  Measurement aid; no effect on results. */
#define BTA_PHASES 5
int bta_profile_phases(bta_ctx_t ctx, double* ms_out, int count);

/* bta_autotune -- choose the launch shapes of the block factorisation and
 * selected inversion for this context's block order, precision and batch by
 * timing candidates on the context's own storage (Section III-A's
 * operations; the sequential diagonal chain and the b x b x b products):
 *   the FP64 leaf order (16, 32, 64), or in mixed precision the
 *   double-float leaf order (32, 64, 128) and the smallest product dimension
 *   sent to the tensor cores (128, 256, 384, 512), timed on the diagonal-block chain;
 *   then, timed on a batched b x b x b lower update, in mixed precision the
 *   split-product tile (35-bit digits: 0 = 128 x 96 tiles with 2 TMA stages,
 *   1 = 128 x 64 with 3; 49-bit digits: 0 = 128 x 64 with 2) and the waves of
 *   the persistent grid below which it splits K (1, 2), in FP64 the CTAs per
 *   SM of the DFMA GEMM's K split (1, 2, 4); then in mixed precision the
 *   tile order of the split product (row tiles per band: 1, 4, 8, 16),
 *   timed separately on a product with a triangular operand (B X^T), on a
 *   general one and on a lower-triangle update.
 * Each candidate runs once untimed and `reps` (>= 1) times timed.  The
 * chosen values are written to chosen[0..8] (host: leaf, double-float leaf,
 * tensor threshold, tile, waves, FP64 CTAs per SM, band of triangular-operand
 * products, band of general products, band of lower-triangle updates) and
 * used by every later call on the context.  The first diagonal block of every matrix is
 * overwritten with a synthetic SPD block: call it before assembling, or
 * assemble again afterwards.  Synchronises the context's stream.  Errors:
 * BTA_ERR_ARG (null pointers, reps < 1), CUDA errors. */
int bta_autotune(bta_ctx_t ctx, int reps, int* chosen);

/*
 * bta_chol_inv_noalloc -- allocation-free Cholesky factor and inverse of one
 * dense symmetric positive definite block.  The paper has no counterpart to
 * this entry point.  It is for callers that may not call cudaMalloc (for
 * example a framework whose own pool already owns the device memory, or a
 * serving loop that cannot take the synchronisation of cudaMalloc/cudaFree):
 * no context is needed and nothing is allocated.
 *   A       device, b x b column-major (leading dimension lda >= b); its
 *           lower triangle is read and overwritten by L with A = L L^T (the
 *           strict upper part of the diagonal 32 x 32 tiles is set to zero,
 *           the rest of the strict upper triangle is left as it was).
 *   X       device, b x b (ldx >= b): receives L^{-1} (lower; strict upper
 *           triangle set to zero).
 *   info_dev device scalar: -1 on success, else the 0-based row of the first
 *           non-positive pivot (the results are then not usable).
 *   stream  the cudaStream_t to run on (NULL = legacy default stream).
 * The workspace is one fixed file-scope device array of 8.5 MiB, held by
 * every GPU that loads the library until the process exits; it limits the
 * block order to b <= 2048 (larger b returns BTA_ERR_ARG, as do bad pointers
 * or leading dimensions).  The first call on a device looks up the device
 * address of that array, so make that first call before any stream
 * capture; the address is kept for the life of the process, so the entry
 * point must not be used on a device after cudaDeviceReset there.  All calls share the one array: calls whose executions overlap
 * on the GPU (other streams, other host threads) race and give wrong
 * results; serialise them.
 */
int bta_chol_inv_noalloc(double* A, int b, int lda, double* X, int ldx, long long* info_dev, void* stream);

/* Nominal flop counts used for throughput figures: block Cholesky
 * n b^3/3 + (n-1) 2 b^3 + n (a b^2 + a^2 b) + (n-1) 2 a b^2 + a^3/3 and
 * selected inversion n 2 b^3/3 + (n-1) 5 b^3 + 6 n a b^2. */
double bta_flops_factor(int n, int b, int a);
double bta_flops_selinv(int n, int b, int a);

#ifdef __cplusplus
}
#endif
#endif /* BTA_H */
