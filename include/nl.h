/*
 * nl.h -- C-ABI of the GB300 nonlocal operator library.
 *
 * Applies the discretised nonlocal operators of Tian & Engquist, "Fast
 * algorithm for computing nonlocal operators with finite interaction
 * distance" (arXiv 1905.08375) on uniform 1-D/2-D/3-D grids:
 *
 *   scalar nonlocal diffusion, Eq. (2.1)-(2.2):
 *       (L u)_i = h^d sum_{j != i, |x_j - x_i| < delta_i} w_ij c_ij (u_j - u_i)
 *       w_ij    = sigma delta_i^{-(d+2)} gamma(|x_j - x_i| / delta_i)
 *   linear bond-based peridynamics, Eq. (1.1)-(1.2):
 *       (L u)_i = h^d sum_{0 < |xi| < delta_i} sigma c_ij (xi xi^T / |xi|^3) (u_j - u_i)
 *   the fast algorithm of Sec. 3 (Algorithm 1 + Steps 1-3, Eq. (3.3)-(3.5))
 *       for polynomial kernels P = sigma C(x) delta(x)^{-(d+2)} p^{2K}(|y-x|/delta(x)),
 *   and conjugate gradients on -L u = f (the Krylov use remarked in Sec. 4).
 *
 * Grid and boundary (Eq. (3.1)): Omega = [0,1]^d, n nodes per dimension,
 * h = 1/n, node i at x_i = (i + 1/2) h, flat index x fastest
 * (i_x + n (i_y + n i_z)).  u = 0 outside Omega (volume constraint).  For a
 * node y outside Omega every coefficient field (a, c, delta) takes the value
 * of the row's own node x.
 *
 * Horizon test: lattice offset o (integer, units of h) lies in the open ball
 * of node i iff (double)|o|^2 < R2_i, R2_i = (delta_i n)^2 in FP64.
 *
 * Conventions for every entry point:
 *   - status codes only (never exceptions); nl_last_error() returns a
 *     thread-local message for the last failure on the calling thread.
 *   - device pointers (u, Lu, f, x) are owned by the caller; the plan owns
 *     its device workspaces and frees them in nl_plan_destroy().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  nl_apply / nl_apply_fast are asynchronous and stream-ordered.
 *   - no entry point calls back into Python or uses any host-side fallback:
 *     every step of an apply runs in this library's CUDA kernels.
 */
#ifndef NL_H
#define NL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NL_OK = 0,
    NL_EINVAL = 1,        /* bad argument (null pointer, size, horizon <= 0, ...) */
    NL_EUNSUPPORTED = 2,  /* valid request this build does not implement */
    NL_ENOMEM = 3,        /* device or host allocation failed */
    NL_ECUDA = 4,         /* a CUDA call failed; message has the CUDA error string */
    NL_ENOTCONV = 5,      /* CG hit maxit before the tolerance */
    NL_ETIMEOUT = 6       /* a bounded device-side wait gave up */
} nl_status;

/* NL_F64_PAIRS (nl_apply only, 2-D symmetric NL_POWER plans with Rmax <= 32): FP64 data in
 * and out, arithmetic on pairs of FP32 numbers (each value hi + lo, 48 significant bits) with
 * error-free sums and products; each term is within a few 2^-46 of its FP64 value relative
 * to |g b_j (u_j - u_i)|.  nl_cg_solve computes its true residual this way on such plans.
 * Other plans: NL_EUNSUPPORTED. */
typedef enum { NL_F32 = 0, NL_F64 = 1, NL_F64_PAIRS = 2 } nl_dtype;

/* Radial profile gamma(s), s = |xi| / delta_i (Eq. (2.2)):
 *   NL_POWER:   gamma(s) = s^{-alpha}, alpha >= 0 (alpha = 0: constant kernel)
 *   NL_POLY:    gamma(s) = p^{2K}(s), the even polynomial of degree 2K that
 *               matches s^{-alpha} and its first K derivatives at s = 1
 *               (the splitting of Sec. 3; K = 0 gives p = 1)
 *   NL_PD_BOND: linear peridynamic bond, micromodulus sigma c_ij / |xi|
 *               (Eq. (1.2)); u and Lu then hold d component planes.  d = 2 (direct
 *               operator, fast path, CG); d = 3 with K = 0 and n = 2^L <= 256 for the
 *               fast path only (nl_apply and nl_cg_solve: NL_EUNSUPPORTED).
 *   NL_KAPPA:   gamma(s) = kappa(s) = s^{-alpha} - p^{2K}(s), the other part of the
 *               splitting of Sec. 3 (s^{-alpha} chi = kappa + p^{2K} chi): singular at
 *               s = 0, C^K at the horizon.  nl_apply only (the direct sum, any d); with the
 *               same sigma, the NL_POWER result is the NL_KAPPA one plus the NL_POLY one. */
typedef enum { NL_POWER = 0, NL_POLY = 1, NL_PD_BOND = 2, NL_KAPPA = 3 } nl_family;

/* Coefficient C(x,y) of Eq. (2.2) built from the node field `a`:
 *   NL_COEF_NONE: C = 1
 *   NL_COEF_X:    C = a(x)            (non-divergence type, Sec. 2 case (a))
 *   NL_COEF_XY:   C = a(x) a(y)
 *   NL_COEF_MEAN: C = (a(x) + a(y))/2 (peridynamic two-phase bond, NL_PD_BOND) */
typedef enum { NL_COEF_NONE = 0, NL_COEF_X = 1, NL_COEF_XY = 2, NL_COEF_MEAN = 3 } nl_coef;

/* Self term of Eq. (3.3) for nl_apply_fast:
 *   NL_SELF_DISCRETE: h^d sum over every lattice cell (inside or outside
 *       Omega) that meets the open ball of p(|x_k - x_i|/delta_i) b_k, with
 *       b = a for NL_COEF_XY (exterior cells take a_i), else 1; then L 1 = 0
 *       wherever the ball stays inside Omega.
 *   NL_SELF_PAPER: the continuous |H_x| form, int_{B_delta} p(|xi|/delta) dxi
 *       (Example 1 of Sec. 4); not defined for NL_COEF_XY. */
typedef enum { NL_SELF_DISCRETE = 0, NL_SELF_PAPER = 1 } nl_self;

/* How nl_apply_fast forms the Step 2/3 sums for K = 0 with FP32 data (FP64 data always use
 * FP64 panel moments summed panel by panel; so does K > 0 except as noted under
 * NL_FAST_LEAFROWS):
 *   NL_FAST_AUTO (0) = NL_FAST_LEAFROWS
 *   NL_FAST_PANELS (1): exact 64-bit fixed-point panel sums (one rounding of each leaf value
 *       to a multiple of 2^-S chosen from max |a u|), added panel by panel (Sec. 3, Steps 1-3);
 *   NL_FAST_ROWPREFIX (2): the same integers kept as prefix sums along each panel row of every
 *       level, so the panels of a run are added as one difference -- bitwise the same result;
 *   NL_FAST_FP64_PANELS (3): FP64 panel sums added panel by panel, as for FP64 data;
 *   NL_FAST_LEAFROWS (4): the panels of Algorithm 1 tile exactly the leaf cells that meet the
 *       ball, so their sum is taken row by row from the leaf-row prefix sums, one difference
 *       per leaf row -- the same integers again, bitwise the same result.  For K >= 1 with
 *       FP32 data and d <= 2 (while (2 Rmax + 3)^d (Rmax + 1)^{2K} <= 2^40) the leaf rows
 *       carry the prefix sums of k^e q (k the column, e <= 2K, modulo 2^64): each row's run
 *       sums of o_x^{2j} q are exact integers, combined once per node with the polynomial's
 *       coefficients in FP64 -- the same leaf-set sum as the moment pyramid's, not bitwise. */
typedef enum { NL_FAST_AUTO = 0, NL_FAST_PANELS = 1, NL_FAST_ROWPREFIX = 2,
               NL_FAST_FP64_PANELS = 3, NL_FAST_LEAFROWS = 4 } nl_fast_variant;

typedef struct {
    int dim;   /* d in {1, 2, 3} */
    int n;     /* nodes per dimension; the fast path needs n = 2^L */
} nl_grid;

typedef struct {
    double delta;               /* constant horizon (used when delta_field is NULL) */
    const double *delta_field;  /* HOST pointer, n^d values, or NULL; copied at plan time */
    int symmetric;              /* 1: divergence-type symmetrised kernel (Sec. 2 case (b)):
                                   w^s_ij = (w_ij + w_ji)/2, each half with its own
                                   node's horizon.  NL_POWER with NL_COEF_NONE/XY (direct
                                   sum), or NL_POLY with K = 0, NL_COEF_NONE/XY and
                                   NL_SELF_DISCRETE on n = 2^L (fast path: nl_apply_fast and
                                   nl_cg_solve only) */
} nl_horizon;

typedef struct {
    int family;        /* nl_family */
    double alpha;      /* exponent of s^{-alpha} (NL_POWER, NL_KAPPA) or of the matched
                          profile (NL_POLY) */
    int K;             /* polynomial order for NL_POLY and NL_KAPPA, 0..3 */
    double scale;      /* multiplies sigma */
    int normalize;     /* 1: sigma = scale 2d(d+2-alpha)/|S^{d-1}| (L -> Laplacian);
                          0: sigma = scale.  Ignored for NL_PD_BOND (sigma = scale). */
    int coef;          /* nl_coef */
    const double *a;   /* HOST pointer, n^d coefficient values (a or c), or NULL */
    int self_term;     /* nl_self, nl_apply_fast only */
    int fast_variant;  /* nl_fast_variant, nl_apply_fast only */
} nl_kernel;

typedef struct nl_plan nl_plan;

/*
 * Build a plan: validates Eq. (2.3) (delta > 0 and finite, coefficient > 0),
 * derives the per-node horizon data, the offset table of the ball, the
 * Hermite-matched polynomial (Sec. 3), the exterior and self terms, and
 * allocates the device workspaces (the Step 2 moment pyramid for the fast
 * path).  Host arrays are read during the call only.  Runs on `stream` and
 * synchronises it before returning.
 * Errors: NL_EINVAL (null, dim, n < 1, delta <= 0, coefficient <= 0, K out of
 * range), NL_EUNSUPPORTED (radius beyond the build's limits), NL_ENOMEM, NL_ECUDA.
 */
nl_status nl_plan_create(nl_plan **out, const nl_grid *grid, const nl_horizon *horizon,
                         const nl_kernel *kernel, void *stream);

/* Free the plan and its device memory (synchronises the device).  NULL is a no-op. */
nl_status nl_plan_destroy(nl_plan *plan);

/*
 * Direct apply (the "Original" matrix-vector product of Sec. 2/4): the plain
 * variable-stencil sum over the open ball of every node, Eq. (2.1)-(2.2) or
 * Eq. (1.2).  u, Lu: DEVICE pointers, nrhs stacked fields, layout
 * [nrhs][n^d] (scalar) or [nrhs][d][n^d] (NL_PD_BOND), element type `dtype`.
 * u and Lu must not overlap.  FP32: FP32 products and sums of differences
 * u_j - u_i; FP64: all FP64; NL_F64_PAIRS: FP64 data, FP32-pair arithmetic (above).
 * Errors: NL_EINVAL (null, nrhs < 1, dtype), NL_ECUDA (launch failure).
 */
nl_status nl_apply(nl_plan *plan, const void *u, void *Lu, int nrhs, int dtype, void *stream);

/*
 * Fast apply (Sec. 3): Step 2 (bottom-up moment pyramid, FP64) and Step 3
 * (per-node sum over the panels of the Step 1 decomposition, Eq. (3.5)),
 * then Eq. (3.3).  The decomposition of Algorithm 1 is not stored: each
 * node enumerates it per level in closed form (the same panel set).  The
 * result equals h^d sum over the leaf cells that meet the ball.
 * Requires family NL_POLY, a non-symmetric horizon, n = 2^L and coefficient
 * NL_COEF_NONE, NL_COEF_X or NL_COEF_XY; else NL_EUNSUPPORTED.
 *
 * On a 2-D NL_PD_BOND plan (n = 2^L <= 8192, FP32 data, K = 0, 1 or 2) it applies the
 * fast-path peridynamic operator (the paper's outlook, Sec. 4): the bond tensor
 * xi xi^T / |xi|^3 replaced by xi xi^T p^{2K}(|xi|/delta_i) / delta_i^3, p^{2K} the Sec. 3
 * polynomial matched to s^{-3} in value and K derivatives at the horizon (K = 0: p = 1),
 * and the sum taken over the same leaf set,
 *     (L u)_i = h^2 sum_{k in LS(i)} sigma c_ik (xi xi^T p^{2K} / delta_i^3) (u_k - u_i),
 * c_ik = (c_i + c_k)/2, u_k = 0 and c_k = c_i outside Omega; a different operator from
 * nl_apply's, computed from exact 64-bit leaf-row moment sums (K = 3: NL_EUNSUPPORTED).
 * On a 3-D NL_PD_BOND plan (K = 0, n = 2^L <= 256, FP32 data) the same operator with
 * xi in R^3 and three component planes (fourteen leaf-row prefix arrays, 112 bytes per node,
 * owned by the plan).
 * On a symmetric NL_POLY plan (K = 0..3) it applies the symmetrised leaf-set operator
 *     (L u)_i = sigma h^d sum_k (w_i(k) + w_k(i))/2 C_ik (u_k - u_i),
 *     w_i(k) = [cell k meets the open ball of node i] delta_i^{-(d+2)} p(|x_k - x_i|/delta_i),
 * k over every lattice cell (u_k = 0, a_k = a_i, delta_k = delta_i outside Omega): the
 * one-sided fast apply for the first half, and for the second its transpose -- each node
 * scatters c_k u_k (c_k = a_k delta_k^{-(d+2)}) into per-leaf-row difference arrays (exact
 * 64-bit integer atomics for FP32 data, FP64 atomics for FP64 data), one prefix sum per row;
 * for K >= 1 the run's weights form a polynomial in the target column, whose 2K + 1
 * coefficients go into difference arrays as two-limb integers (exact for both data types;
 * 16 (2K + 1) bytes per node owned by the plan; NL_EUNSUPPORTED at plan creation when the
 * horizon is too large for the limbs).
 * Symmetric and negative semi-definite, so nl_cg_solve accepts such a plan (Jacobi).
 * Same layouts and ownership as nl_apply.
 */
nl_status nl_apply_fast(nl_plan *plan, const void *u, void *Lu, int nrhs, int dtype, void *stream);

typedef struct {
    int iterations;       /* CG iterations of the slowest right-hand side */
    double rel_residual;  /* max over right-hand sides of ||f + L x|| / ||f|| (FP64, true residual) */
    int converged;        /* 1 if every right-hand side met rtol */
} nl_cg_stats;

/* NL_PRECOND_LEARNED: the network attached with nl_plan_set_net (flexible CG, since the
 * network is nonlinear); it builds on the Jacobi scaling, which stays the fallback. */
typedef enum { NL_PRECOND_NONE = 0, NL_PRECOND_JACOBI = 1, NL_PRECOND_LEARNED = 2 } nl_precond;

/*
 * Preconditioned conjugate gradients for -L x = f with the plan's operator
 * (which must be symmetric: a symmetric NL_POWER plan (direct sum), a symmetric NL_POLY plan
 * (the symmetrised fast operator of nl_apply_fast) or NL_PD_BOND with a constant horizon).
 * f, x: DEVICE pointers, FP64, layout as nl_apply; x0 = 0.  Operator applies in FP32,
 * inner products and vector updates in FP64, with the residual recomputed in FP64 (FP64
 * operator) when the recursive one converges, so that the reported residual is the true FP64
 * one.  Blocks until done; the stats are read back on the host.
 * Errors: NL_EINVAL, NL_EUNSUPPORTED (non-symmetric plan), NL_ENOTCONV, NL_ECUDA.
 */
nl_status nl_cg_solve(nl_plan *plan, const void *f, void *x, int nrhs, double rtol, int maxit,
                      int precond, nl_cg_stats *stats, void *stream);

/*
 * nl_apply_fast_noalloc -- the K = 0 (p = 1), C = 1 fast apply, equal to nl_apply_fast on an
 * NL_POLY, K = 0, NL_COEF_NONE plan with the same horizon, alpha, scale, normalize and self
 * term.  The paper has no counterpart: this entry point only packages that apply for callers
 * that must not allocate device memory -- a host whose device memory is all handed to its own
 * pool allocator (a library cudaMalloc would fail or fragment the pool), or a caller on a
 * latency-critical path that cannot take the implicit device synchronisation that
 * cudaMalloc/cudaFree may cause.  It creates no plan and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * Scratch: a file-scope device array of 32 MiB inside the library, held by every GPU on which
 * the library's module is loaded until the process exits.  It bounds the grid: n = 2^L with
 * at most 8192 (1-D), 1024 (2-D) or 64 (3-D) nodes per dimension; larger grids are rejected
 * with NL_EINVAL and a message giving the bytes needed.  Every call looks up the array's
 * device address (cudaGetSymbolAddress, which allocates nothing) with the caller's device
 * current.  All calls share the array and each call rewrites every part it reads, so no
 * clearing is needed, but calls whose kernels overlap on the GPU (other streams or host
 * threads on the same device) race on it: order them.
 *
 * Arguments: dim 1..3; n nodes per dimension; delta the constant horizon, 0 < delta <= 2
 * (a ball of radius 2 covers Omega), used when delta_field is NULL; delta_field a DEVICE
 * pointer to n^dim FP64 horizons in the same range (caller-owned, read only; values outside
 * it, or NaN, are clamped for the geometry so that the work stays bounded, and the result at
 * such nodes is undefined) or NULL; alpha, scale, normalize as in nl_kernel (sigma);
 * self_term an nl_self; u, Lu DEVICE pointers, nrhs stacked fields [nrhs][n^dim] of `dtype`
 * each (the caller guarantees those sizes).  Stream-ordered and asynchronous.
 * Errors: NL_EINVAL (argument out of range, grid beyond the array), NL_EUNSUPPORTED (n not a
 * power of two), NL_ECUDA.
 */
nl_status nl_apply_fast_noalloc(int dim, int n, double delta, const double *delta_field,
                                double alpha, double scale, int normalize, int self_term,
                                const void *u, void *Lu, int nrhs, int dtype, void *stream);

/*
 * Learned CG preconditioner (a project addition; the paper only remarks, in its conclusion,
 * that the fast product can serve a Krylov method).  For the symmetric 2-D scalar operator:
 *     x = D^{-1} r / s, s = RMS(D^{-1} r) per right-hand side (D = diagonal of -L)
 *     y1 = relu(conv1 x), y2 = relu(conv2 y1), o = conv3 y2, M(r) = s (x + o)
 * with 3x3 convolutions (zero padding, no bias) of 1 -> 32 -> 32 -> 1 channels.  Weights are
 * FP32 masters used as bfloat16; activations and sums are FP32.
 * Weight layout (NL_NET_PARAMS floats): conv1 [32][1][3][3], conv2 [32][32][3][3],
 * conv3 [1][32][3][3], concatenated, each [out][in][ky][kx].
 */
#define NL_NET_PARAMS 9792
typedef struct nl_net nl_net;

/* Create a network from HOST weights (copied).  Synchronises `stream`. */
nl_status nl_net_create(nl_net **out, const float *weights, void *stream);
nl_status nl_net_destroy(nl_net *net);
/* Copy the FP32 master weights to HOST memory (synchronises `stream`). */
nl_status nl_net_get_weights(nl_net *net, float *weights, void *stream);
/* Copy the last training step's gradient (FP32, weight layout) to HOST memory. */
nl_status nl_net_gradient(nl_net *net, float *grad, void *stream);
/* o = conv3(relu(conv2(relu(conv1 x)))) on DEVICE x, o: [batch][H][W] FP32. */
nl_status nl_net_forward(nl_net *net, const float *x, float *o, int batch, int H, int W, void *stream);
/*
 * One Adam step (beta 0.9/0.999, eps 1e-8, learning rate lr) on `batch` crops of S x S
 * gathered from DEVICE fields x, e ([nfields][n][n] FP32) at DEVICE offsets
 * crops[batch][3] = (field, y0, x0) (a crop outside the fields reads zeros).
 * Loss per crop over the interior (margin pixels dropped): sum (x + o - e)^2 / sum e^2,
 * averaged over the batch; written to *loss (HOST, may be NULL: then no synchronisation).
 */
nl_status nl_net_train_step(nl_net *net, const float *x, const float *e, int nfields, int n,
                            const int *crops, int batch, int S, int margin, float lr, float *loss,
                            void *stream);
/*
 * One Adam step on the energy norm of the preconditioned step's error, on whole fields:
 * for each field b in DEVICE fields[batch] of x, e ([nfields][n^2] FP32 from
 * nl_net_prepare_pairs), with r = x / D^{-1} (the scaled residual), z = x + o(x) and
 * A = -L applied by the plan (FP32):
 *     loss_b = (z - e)^T A (z - e) / e^T A e = (z.Az - 2 z.r + e.r) / e.r,
 * averaged over the batch; *loss (HOST, may be NULL).  Needs the symmetric 2-D scalar plan.
 */
nl_status nl_net_train_step_energy(nl_net *net, nl_plan *plan, const float *x, const float *e,
                                   int nfields, const int *fields, int batch, float lr,
                                   float *loss, void *stream);
/* Training pairs from CG iterates: DEVICE r, e [count][n^2] FP64 (residual f + L x_k and
 * error x* - x_k) -> x_out = D^{-1} r / s, e_out = e / s (FP32), s = RMS(D^{-1} r) per field. */
nl_status nl_net_prepare_pairs(nl_plan *plan, const double *r, const double *e, int count,
                               float *x_out, float *e_out, void *stream);
/* z = M(r) on DEVICE FP64 [nrhs][n^2]. */
nl_status nl_net_apply(nl_net *net, nl_plan *plan, const double *r, double *z, int nrhs, void *stream);
/* Training pairs straight from a CG history (nl_cg_history): DEVICE f, x [n^2] (FP64, the
 * right-hand side and the converged solution) and history [count][n^2] (FP64 iterates x_k)
 * -> r_k = f + L x_k (FP64 operator) and e_k = x - x_k, then as nl_net_prepare_pairs into
 * x_out, e_out [count][n^2] (FP32).  Allocates and frees two FP64 work arrays of count n^2
 * values; synchronises `stream`.  Errors: NL_EINVAL, NL_EUNSUPPORTED (not the symmetric 2-D
 * scalar operator), NL_ENOMEM, NL_ECUDA. */
nl_status nl_net_history_pairs(nl_plan *plan, const double *f, const double *x,
                               const double *history, int count, float *x_out, float *e_out,
                               void *stream);
/* Attach (or detach with NULL) the network used by nl_cg_solve with NL_PRECOND_LEARNED. */
nl_status nl_plan_set_net(nl_plan *plan, nl_net *net);
/*
 * Two-level form (block >= 2; block = 0 restores the local form above).  The three layers
 * without activations are one linear map K (1 -> 32 -> 32 -> 1 channels) applied on a coarse
 * grid of ceil(n/block)^2 cells; R sums each block x block block of a field (cells cut by the
 * grid edge sum what they hold), P = R^T copies a cell's value to its block, and
 *     M(r) = D^{-1} r + gamma P K^T K R r,   gamma = 1 / (block^2 mean(diag(-L))),
 * symmetric positive definite for any weights, used by nl_net_apply and by CG with
 * NL_PRECOND_LEARNED.  nl_net_train_step_energy then minimises the same energy-norm loss with
 * z = M r.  Errors: NL_EINVAL (block 1, negative or above 65536).
 */
nl_status nl_net_set_coarse(nl_net *net, int block);

/*
 * nl_cg_solve for one right-hand side that also records the iterate x after every
 * `chunk` iterations (chunk = 16) into DEVICE history[cap][n^d] (FP64); *count receives the
 * number of snapshots written.  Used to build the network's training pairs.
 */
nl_status nl_cg_history(nl_plan *plan, const void *f, void *x, double rtol, int maxit,
                        int precond, double *history, int cap, int *count, nl_cg_stats *stats,
                        void *stream);

/*
 * Per-phase timing of nl_apply_fast (tracing): when enabled, each fast apply records CUDA
 * events on its stream before Step 2, between Step 2 and Step 3, and after Step 3 (up to 64
 * applies between reads).  nl_plan_profile_read synchronises those events, returns the summed
 * Step 2 (partial sums) and Step 3 (gather) milliseconds and the number of applies, and
 * clears the record.  Disabled by default; costs two event records per apply when enabled.
 */
nl_status nl_plan_profile(nl_plan *plan, int enable);
nl_status nl_plan_profile_read(nl_plan *plan, double *step2_ms, double *step3_ms, int *applies);

/*
 * Batches of uneven 2-D instances (each its own n, horizon and coefficient fields; all of one
 * family, NL_POWER or NL_PD_BOND, and one symmetric flag).  A batch owns one plan per
 * instance; its vectors concatenate the instances' fields: instance k occupies elements
 * offsets[k] .. offsets[k+1]-1 (two component planes for NL_PD_BOND).  nl_batch_apply runs
 * the direct apply of every instance in ONE persistent launch whose blocks take
 * (instance, tile) work items from an atomic counter; a tile is 32 x 4, 32 x 8 or 32 x 16
 * output nodes, one per thread.  tile_shape = NL_TILE_AUTO times the three shapes on the
 * batch at creation (the autotuner) and keeps the fastest; 0..2 fixes the shape.
 * nl_batch_cg_solve solves -L_k x_k = f_k for all instances together (each instance one CG
 * segment, one captured graph, Jacobi or no preconditioner); the stats are the worst over
 * instances.  Errors: NL_EINVAL, NL_EUNSUPPORTED, NL_ENOMEM, NL_ECUDA, NL_ENOTCONV.
 */
typedef struct nl_batch nl_batch;
enum { NL_TILE_AUTO = -1, NL_TILE_32x4 = 0, NL_TILE_32x8 = 1, NL_TILE_32x16 = 2 };
nl_status nl_batch_create(nl_batch **out, int count, const nl_grid *grids,
                          const nl_horizon *horizons, const nl_kernel *kernels, int tile_shape,
                          void *stream);
nl_status nl_batch_destroy(nl_batch *batch);
/* offsets: HOST array of count + 1 elements; tile_shape (may be NULL): 0, 1 or 2. */
nl_status nl_batch_layout(const nl_batch *batch, int64_t *offsets, int *tile_shape);
nl_status nl_batch_apply(nl_batch *batch, const void *u, void *Lu, int dtype, void *stream);
nl_status nl_batch_cg_solve(nl_batch *batch, const void *f, void *x, double rtol, int maxit,
                            int precond, nl_cg_stats *stats, void *stream);

/* Plan introspection (host values computed at plan time). */
typedef struct {
    int dim, n, levels;        /* levels = L for n = 2^L, else -1 */
    int max_radius;            /* max_i ceil(delta_i n) */
    int num_offsets;           /* offsets in the largest ball */
    int moments;               /* moments per panel, C(2K+d, d) */
    double sigma;              /* kernel constant */
    double poly[8];            /* p_0 .. p_K of p^{2K} (NL_POLY) */
    size_t device_bytes;       /* device memory owned by the plan */
    size_t step1_bytes;        /* the stored decomposition of the panel route (read by every
                                  panel-route apply), 0 if none */
} nl_plan_info;

nl_status nl_get_plan_info(const nl_plan *plan, nl_plan_info *info);

/*
 * Measured arithmetic peaks of the current device, the denominators of the ALU roofline
 * fractions reported with the direct sums (the paper, which reports MATLAB wall times, has no
 * counterpart).  Eight independent FMA chains per thread on 4 x 256 threads per SM; an FMA is
 * two flops, a paired f32x2 FMA four; best of five launches timed with CUDA events on
 * `stream` (synchronises it).  Outputs in TFLOP/s: scalar FP32 FMA, paired f32x2 FMA, FP64 FMA.
 * Allocates and frees a small sink buffer.  Errors: NL_EINVAL (null output), NL_ECUDA.
 */
nl_status nl_measure_peaks(double *fp32_tflops, double *fp32x2_tflops, double *fp64_tflops,
                           void *stream);

/* Thread-local description of the last error on this thread ("" if none). */
const char *nl_last_error(void);

/*
 * Failure handling on the host (the paper has no counterpart; these serve callers that must
 * bound how long the library may block, and tests of the error paths that need no GPU fault).
 *
 * nl_set_wait_limit: the limit, in seconds (0 < seconds <= 1e6; 600 by default, process-wide),
 * of every bounded host wait of the library -- nl_cg_solve, nl_cg_history and
 * nl_batch_cg_solve wait on each chunk of iterations at most this long and then return
 * NL_ETIMEOUT.  The chunk's kernels are not stopped: they finish on the solver's stream, so a
 * caller that got NL_ETIMEOUT synchronises the device before reusing the plan or its buffers.
 * Errors: NL_EINVAL.
 *
 * nl_wait_poll: the bounded wait itself, exported so that a caller can wait on a condition of
 * its own with the same semantics: calls poll(ctx) about every 50 us until it returns > 0
 * (NL_OK), < 0 (NL_ECUDA) or `seconds` have passed (NL_ETIMEOUT; seconds <= 0 takes the
 * limit of nl_set_wait_limit).  poll runs on the calling thread.
 *
 * nl_debug_fail_host_alloc: failure injection.  With after >= 0 the host allocation that
 * follows `after` successful ones inside nl_plan_create fails once (that call returns
 * NL_ENOMEM and leaves nothing allocated); after < 0 disarms.  Process-wide; for tests.
 */
nl_status nl_set_wait_limit(double seconds);
nl_status nl_wait_poll(int (*poll)(void *ctx), void *ctx, double seconds);
nl_status nl_debug_fail_host_alloc(int after);

#ifdef __cplusplus
}
#endif

#endif /* NL_H */
