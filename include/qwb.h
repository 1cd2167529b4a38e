/*
 * qwb.h -- C ABI of the GB300 library for certified quantization-based bounds
 * on the p-Wasserstein metric between measures on regular N x N grids
 * (Bobrutsky & Moscovich, "Quantization-based Bounds on the Wasserstein
 * Metric").
 *
 * Problem statement (Sec. 2.1, Sec. 2.2, Sec. 5): mu, nu are probability
 * vectors on the grid [N]^2 (row-major, flat index i = row * N + col, unit
 * pixel spacing), rho is the Euclidean distance, C_ij = rho(x_i, y_j)^p,
 * W_p = L_C(mu, nu)^(1/p).  The grid is coarsened by kappa x kappa blocks
 * (N % kappa == 0, n = N / kappa, M = n^2 coarse cells; coarse index
 * k = k1 * n + k2 for the block at block-row k1, block-column k2).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_d are device pointers (cudaMalloc'd or PyTorch tensor
 *     storage on the context's device); *_h are host pointers.  Every buffer
 *     is owned by the caller and must stay valid until the call's work on
 *     `stream` has completed.  The context owns its workspace, cost tables,
 *     launch plans and captured graphs.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it; calls that fill a host result
 *     (*_h outputs, qwb_result) synchronise the stream before returning.
 *   - Every call returns a status (QWB_OK = 0).  No C++ exception crosses the
 *     ABI.  qwb_last_error() gives a thread-local message for the last
 *     failure on the calling thread.
 *   - Input measures must be finite, non-negative and of mass 1 within 1e-12
 *     (QWB_ERR_MASS otherwise).  Validation reads the measures on the device
 *     with a small reduction; it is part of every call that takes measures.
 *   - Certification: every bound is computed with directed rounding (FP32
 *     round-down in the c-transform, round-up in cost reductions, FP64
 *     directed sums) so that lb <= W_p <= ub_primal and W_p <= ub_weighted
 *     hold for the real-number W_p of the given inputs.
 *   - Precision: QWB_PREC_F64 runs every device pass in FP64;
 *     QWB_PREC_MIXED runs the cost reductions, IPF sweeps and c-transforms in
 *     FP32 and every bound sum and certificate in FP64.
 */
#ifndef QWB_H
#define QWB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                              */
/* ------------------------------------------------------------------------ */
enum {
    QWB_OK = 0,
    QWB_ERR_INVALID_ARG = 1,   /* null pointer, N % kappa != 0, p < 1, sizes */
    QWB_ERR_MASS = 2,          /* negative / non-finite entry or |mass - 1| > 1e-12 */
    QWB_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has details) */
    QWB_ERR_NOT_CONVERGED = 4, /* the exact coarse solver hit its pivot cap (or found its tree corrupted) */
    QWB_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
    QWB_ERR_OOM = 6,           /* device or host allocation failed */
    QWB_ERR_UNSUPPORTED = 7,   /* valid problem outside this build's limits */
    QWB_ERR_VERIFY = 8         /* QWB_FLAG_VERIFY found f_i + g_j > c_ij */
};

/* Flags for qwb_batch_create / qwb_bounds: passes a caller does not need.
 * A skipped upper bound is reported as +inf, a skipped lower bound as 0
 * (lb_p = -inf); both remain valid bounds. */
enum {
    QWB_FLAG_NO_WEIGHTED = 1,  /* skip pass (a)'s C-bar and its exact solve */
    QWB_FLAG_NO_PRIMAL = 2,    /* skip pass (b) */
    QWB_FLAG_NO_DUAL = 4,      /* skip pass (c) */
    QWB_FLAG_MINCOST = 8,      /* also compute the min-cost lower bound (Sec. 3.3) */
    QWB_FLAG_SEPARABLE = 16,   /* p = 2 pairs: separable c-transform (see
                                  qwb_ctransform_separable) instead of the
                                  N^4 lazy transform of Sec. 4, and, for
                                  2-D FP32 pairs with kappa 4 or 8, the
                                  separable C-bar (see
                                  qwb_coarse_cost_separable) */
    QWB_FLAG_VERIFY = 64,      /* after each dual pass, check f_i + g_j <= c_ij
                                  on every pair of fine points (2-D; each
                                  sum rounded upward, compared with a lower
                                  bracket of the cost); a failure gives the
                                  pair the status QWB_ERR_VERIFY.  N^4 checks
                                  per pair (FP64 ones for F64 batches: slow);
                                  the environment variable QWB_VERIFY=1
                                  sets it for every batch */
    QWB_FLAG_SYMMETRIC_DUAL = 32 /* also run the dual pass from the coarse
                                  potential g~ (Sec. 3.5 from nu's side) and
                                  report the larger of the two lower bounds */
};

/* Precision of the device passes (see the file comment). */
typedef enum { QWB_PREC_F64 = 0, QWB_PREC_MIXED = 1 } qwb_prec;

/* One problem: grid [N]^d with side N, block side kappa, order p, dimension
 * d = 2 (images; 0 also means 2) or d = 3 (volumes, flattened row-major:
 * index (x1 * N + x2) * N + x3; coarse index (k1 * n + k2) * n + k3).
 * Requirements: 1 <= kappa <= N, N % kappa == 0, p >= 1; d = 2: N <= 1024 and
 * n = N / kappa <= 64; d = 3: N <= 64 and n <= 16. */
typedef struct {
    int32_t N;
    int32_t kappa;
    double p;
    int32_t d;
    int32_t reserved;   /* must be 0 */
} qwb_problem;

/* Results for one pair.  Bounds are in the units of W_p (pixels); the *_p
 * fields are the corresponding certified bounds on W_p^p. */
typedef struct {
    double ub_weighted;    /* Sec. 3.2 / Alg. 3: certified L_Cbar(mu~, nu~)^(1/p) >= W_p */
    double ub_primal;      /* Sec. 3.4 / Alg. 4: W-hat_p + Delta_mu + Delta_nu >= W_p */
    double lb;             /* Sec. 3.5 / Alg. 5: (<f,mu> + <g,nu>)^(1/p) <= W_p, clipped at 0 */
    double lb_p;           /* certified lower bound on W_p^p (may be negative) */
    double ub_weighted_p;  /* certified upper bound on L_Cbar */
    double w_hat_p;        /* certified upper bound on <pi-hat_xi, C> */
    double delta_mu;       /* TV correction of the first marginal (eq. weighted TV) */
    double delta_nu;       /* TV correction of the second marginal */
    double ipf_residual;   /* ||mu-hat - mu||_1 + ||nu - nu-hat||_1 of the final plan */
    double lb_mincost;     /* Sec. 3.3: certified L_Cmin(mu~, nu~)^(1/p) <= W_p (QWB_FLAG_MINCOST; else 0) */
    double t_coarse_cost_ms; /* per-pass device times (batch calls: whole batch) */
    double t_solve_ms;       /* host exact coarse solves */
    double t_primal_ms;
    double t_dual_ms;
    int32_t ipf_sweeps_done;
    int32_t status;          /* per-pair status code */
} qwb_result;

typedef struct qwb_ctx qwb_ctx;
typedef struct qwb_batch qwb_batch;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */
/* Create a context bound to CUDA device `device`.  *out receives the handle.
 * Errors: INVALID_ARG (out == NULL), CUDA (no such device). */
int qwb_ctx_create(qwb_ctx** out, int device);
/* Free the context, its workspace and graphs.  NULL is ignored. */
void qwb_ctx_destroy(qwb_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Pass (a): coarse cost.  Sec. 2.2 (SumPool), Sec. 3.2 (the equation that    */
/* defines the marginally weighted cost C-bar), Alg. 3.                       */
/* ------------------------------------------------------------------------ */
/* Computes mu~ = SumPool(mu), nu~ = SumPool(nu) (FP64, M each) and
 *   C-bar_kl = sum_{x in X_k, y in Y_l} rho(x,y)^p mu(x) nu(y) / (mu~_k nu~_l)
 * reduced over every fine pixel pair of every block pair, as an M x M
 * row-major FP64 matrix rounded upward (each entry >= the real value).
 * Where mu~_k nu~_l = 0 the entry is the unweighted mean of rho^p over the
 * block pair.  mu_d, nu_d: N*N FP64.  cbar_d: M*M FP64 out.  mu_coarse_d,
 * nu_coarse_d: M FP64 out (may be NULL).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, MASS, CUDA, OOM. */
int qwb_coarse_cost(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                    const double* nu_d, double* cbar_d, double* mu_coarse_d,
                    double* nu_coarse_d, qwb_prec prec, void* stream);
/* The same C-bar for p = 2 (d = 2, kappa 4 or 8, FP32 reductions) by
 * separating the squared distance over the two axes (not a step of the
 * paper; an exact regrouping of the sum that defines C-bar in Sec. 3.2):
 * with R, C the row and column sums of a block's masses and
 * D = kappa (k - l) per axis,
 *   sum_{x in X_k, y in Y_l} mu(x) nu(y) rho(x,y)^2
 *     = sum_{a1, b1} R_mu,k[a1] R_nu,l[b1] (D1 + a1 - b1)^2
 *     + sum_{a2, b2} C_mu,k[a2] C_nu,l[b2] (D2 + a2 - b2)^2,
 * 2 kappa^2 + 2 kappa multiply-adds per block pair instead of
 * kappa^4 + kappa^2.  Every operation rounds upward from the rounded-up
 * masses, so each entry is >= the real C-bar, as qwb_coarse_cost's; the two
 * differ by rounding only.  Zero-mass blocks as qwb_coarse_cost.
 * mu_d, nu_d: N*N FP64; cbar_d: M*M FP64 out.  Coarse side n <= 1365
 * (kappa 4) or 722 (kappa 8).  Synchronous with `stream` on return.
 * Errors: INVALID_ARG, UNSUPPORTED (p != 2, d = 3, kappa not 4 or 8, n too
 * large), MASS, CUDA, OOM. */
int qwb_coarse_cost_separable(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                              const double* nu_d, double* cbar_d, void* stream);

/* ------------------------------------------------------------------------ */
/* Host exact coarse solve.  Sec. 2.1 (Kantorovich problem and its dual),     */
/* Sec. 3.2 / Sec. 3.4 / Sec. 3.5 (the coarse problems), Sec. 4 (network      */
/* simplex, at most 2M - 1 positive plan entries).                            */
/* ------------------------------------------------------------------------ */
/* Solves min <pi, C> over couplings of (a, b) and its dual exactly with the
 * library's own network simplex (host, FP64).  C_h: n_src x n_dst row-major,
 * non-negative.  a_h (n_src), b_h (n_dst): non-negative, equal total mass.
 * Outputs (host, caller-allocated): the plan in CSR form with at most
 * n_src + n_dst - 1 entries (rowptr_h: n_src + 1, col_h / val_h: capacity
 * n_src + n_dst), *nnz_out, potentials f_h (n_src) and g_h (n_dst) with
 * f_i + g_j <= C_ij, and *obj_out = <pi, C>.  Any output may be NULL except
 * nnz_out when the plan is requested.  Needs no GPU.
 * Errors: INVALID_ARG, NOT_CONVERGED (pivot cap, or an internal check of the
 * spanning tree failed), OOM. */
int qwb_coarse_solve(int32_t n_src, int32_t n_dst, const double* C_h, const double* a_h,
                     const double* b_h, int32_t* rowptr_h, int32_t* col_h, double* val_h,
                     int32_t* nnz_out, double* f_h, double* g_h, double* obj_out);
/* The same exact solve for a problem on an n_side x n_side grid whose cost
 * depends only on the offset: C_kl = tab_h[|k1 - l1| * n_side + |k2 - l2|]
 * (k = k1 * n_side + k2; the block-centre cost C~ of Sec. 3.4 / 3.5 with
 * tab = rho(kappa d)^p), without an M x M matrix (M = n_side^2).  Solved
 * coarse to fine (the problem on the grid of 2 x 2 cell sums first, its
 * support's children priced first, full scans until no arc has a negative
 * reduced cost).  Outputs and errors as qwb_coarse_solve with n_src = n_dst
 * = M.  Needs no GPU. */
int qwb_coarse_solve_grid(int32_t n_side, const double* tab_h, const double* a_h, const double* b_h,
                          int32_t* rowptr_h, int32_t* col_h, double* val_h, int32_t* nnz_out,
                          double* f_h, double* g_h, double* obj_out);

/* ------------------------------------------------------------------------ */
/* Pass (b): primal upscaling + IPF + upper bound.  Sec. 3.4 (eq. coupling    */
/* tensor upscale, Lemma on the normalised coupling, IPF paragraph, Theorem   */
/* on the upscaling upper bound), Sec. 4 (cost over the support), Alg. 4.     */
/* ------------------------------------------------------------------------ */
/* Upscales the coarse plan pi~ (device CSR: pi_rowptr_d M+1, pi_col_d and
 * pi_val_d nnz) with the uniform kernel K = kappa^-4 (pi-hat = pi~ (x) K,
 * never materialised), fits its marginals to (mu, nu) by IPF sweeps
 * (b <- 1; a <- mu / (pi-hat b); b <- nu / (pi-hat^T a)), then sums the
 * cost of the fitted plan and adds the weighted-TV corrections.
 * MIXED runs `sweeps` FP32 sweeps over the fine vectors followed by one FP64
 * sweep that defines the certified plan; F64 runs them all in FP64.
 * sweeps >= 1.  a_d, b_d (N*N FP64, may be NULL) receive the final scalings.
 * out_h: fills ub_primal, w_hat_p, delta_mu, delta_nu, ipf_residual,
 * ipf_sweeps_done (synchronises `stream`).
 * Errors: INVALID_ARG, MASS, CUDA, OOM. */
int qwb_primal_upscale_ipf(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                           const double* nu_d, const int32_t* pi_rowptr_d,
                           const int32_t* pi_col_d, const double* pi_val_d, int32_t pi_nnz,
                           int32_t sweeps, double* a_d, double* b_d, qwb_result* out_h,
                           qwb_prec prec, void* stream);

/* The same pass with a general normalized positive upscaling kernel (Sec.
 * 3.4, eq. coupling tensor upscale: pi-hat_ij = pi~_{k(i) l(j)} K[u(i), v(j)]
 * with u, v the row-major offsets of i, j inside their kappa x kappa blocks).
 * K_d: kappa^2 x kappa^2 FP64 on the device, row-major K[u * kappa^2 + v],
 * every entry positive and finite (its scale is absorbed by the scalings; the
 * paper's kernels sum to 1); d = 2 and kappa <= 8.  No block-scalar shortcut
 * exists for such K: MIXED and F64 run `sweeps` IPF sweeps on the fine
 * vectors in FP32 / FP64, and the bound is certified for the plan
 * diag(a) pi-hat' diag(b) with those scalings as they are, pi-hat' built with
 * the kernel the sweeps used (K rounded to FP32 for MIXED, K for F64; every
 * positive kernel gives a valid bound): enclosures (FP64 with directed
 * rounding and a-priori error bounds) of its marginals mu-hat, nu-hat and of
 * its total mass s, the cost over its support rounded up and divided by s
 * rounded down, and the weighted-TV corrections between mu-hat / s,
 * nu-hat / s and mu, nu.
 * Other arguments, outputs and errors as qwb_primal_upscale_ipf, plus
 * UNSUPPORTED (d = 3 or kappa > 8) and INVALID_ARG (null or non-positive K). */
int qwb_primal_upscale_ipf_kernel(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                                  const double* nu_d, const int32_t* pi_rowptr_d,
                                  const int32_t* pi_col_d, const double* pi_val_d,
                                  int32_t pi_nnz, const double* K_d, int32_t sweeps,
                                  double* a_d, double* b_d, qwb_result* out_h, qwb_prec prec,
                                  void* stream);

/* ------------------------------------------------------------------------ */
/* Pass (c): dual upscaling + c-transforms + lower bound.  Sec. 3.5 (the     */
/* interpolation R, the c-transform and its double application, the          */
/* proposition on admissible pairs, eq. upscaling lower bound), Sec. 4 (eq.  */
/* lazy c-transform), Alg. 5.                                                 */
/* ------------------------------------------------------------------------ */
/* f_coarse_d (M FP64): a coarse potential f~ (any values; the optimal dual
 * of the C~ problem gives the paper's bound).  The call shifts it so that
 * <f~, mu~> = 0, upsamples it bilinearly at the block centres (linear
 * extrapolation at the border) to f-hat, computes g = f-hat^c and
 * f = g^c with round-down arithmetic (so f_i + g_j <= C_ij exactly), and
 * sums lb_p = <f, mu> + <g, nu> rounded down in FP64.
 * f_d, g_d (N*N FP64, may be NULL) receive the final potentials.
 * out_h: fills lb, lb_p (synchronises `stream`).
 * Errors: INVALID_ARG, MASS, CUDA, OOM. */
int qwb_dual_upscale_ctransform(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                                const double* nu_d, const double* f_coarse_d, double* f_d,
                                double* g_d, qwb_result* out_h, qwb_prec prec, void* stream);

/* One lazy c-transform on the grid (Sec. 4, eq. lazy c-transform):
 *   out_j = min_i rho(x_i, x_j)^p - h_i,  i, j over all N*N pixels,
 * rounded down so that h_i + out_j <= C_ij holds exactly for the given h
 * (MIXED: h is rounded up to FP32 first; the result is FP32 widened to
 * FP64).  h_d, out_d: N*N FP64 device.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA, OOM. */
int qwb_ctransform(qwb_ctx* ctx, int32_t N, double p, const double* h_d, double* out_d,
                   qwb_prec prec, void* stream);

/* qwb_ctransform on [N]^d (d = 2 or 3) with an explicit launch shape instead
 * of the default one, for tuning and for testing every compiled variant
 * (Sec. 4, eq. lazy c-transform; the values do not depend on the shape).
 * The transform runs over the N^d grid points, read as N^(d-1) lines of N:
 *   R        outputs per thread (consecutive along a grid line), must divide N;
 *   TC       input columns per register chunk, must divide N;
 *   packing  0 scalar subtractions; 1 (MIXED only) two columns per packed
 *            f32x2 subtraction; 2 (MIXED only) two input lines per packed
 *            subtraction; 3-6 (MIXED, d = 2 only) packing 2 with the
 *            register budget cut for 3 (packings 3, 4) or 2 (5, 6) resident
 *            CTAs per SM, the p = 2 window costs formed on the fly (3, 6) or
 *            kept in registers (4, 5); 7, 8 (MIXED, d = 2 only) packings 5
 *            and 2 with each candidate pair's subtraction and min fused in
 *            one assembly block; 9, 10 (MIXED, d = 2, p = 2 only) the
 *            shifted form with 2 (9) or 1 (10) resident CTAs per SM: the
 *            line part A of c = A + D is taken off the staged potential
 *            (h - A rounded up) and each candidate is D - (h - A) rounded
 *            down, so the result is still a certified transform
 *            (h_i + out_j <= C_ij) but may lie below the once-rounded one by
 *            the rounding of h - A; 11, 12: 9 and 10 with the chunk's
 *            squared column offsets pinned in registers.
 *   in_rows  input lines per work item (0 = the default split); work items
 *            that see part of the input lines combine by atomic min.
 * Compiled shapes: packing 0: (R, TC) in {1,2,4,8,16} x {same} and (16,8),
 * (8,16); packing 1: (8,8), (16,8), (16,16); packing 2: (8,8), (16,8), (8,16),
 * (16,16); packing 3: (8,8); packing 4: (8,8), (8,16); packing 5: (8,16),
 * (16,8), (16,16); packing 6: (8,16); packing 7: (16,16), (16,8), (8,16);
 * packing 8: (16,16); packing 9: (16,16), (16,8), (8,16); packing 10:
 * (16,16), (32,16), (32,8); packing 11: (16,16), (16,8), (8,16); packing 12:
 * (16,16), (32,8).  Other shapes return QWB_ERR_UNSUPPORTED.
 * h_d, out_d: N^d FP64 device.  Synchronises `stream` before returning.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, OOM. */
int qwb_ctransform_shape(qwb_ctx* ctx, int32_t N, int32_t d, double p, const double* h_d,
                         double* out_d, int32_t R, int32_t TC, int32_t packing, int32_t in_rows,
                         qwb_prec prec, void* stream);

/* The same lazy c-transform (MIXED precision: h rounded up to FP32, result
 * rounded down, widened to FP64) for callers that cannot allocate device
 * memory when they need it -- for instance code running under a frozen or
 * exhausted memory pool, or a plugin whose host process owns every device
 * byte.  This call allocates nothing: its scratch (FP32 copies, cost table,
 * launch plan) lives in one static device array of about 1 MiB that every GPU
 * loading the library holds until the process exits.  The paper has no
 * counterpart; it is a deployment variant of qwb_ctransform.
 *   N <= 256 (QWB_ERR_UNSUPPORTED beyond); h_d, out_d: N*N FP64 device.
 *   Every call shares the static array and rewrites what it reads, so
 *   calls whose GPU work overlaps (other streams, concurrent host threads)
 *   race and corrupt each other: serialise them.
 *   The first call on each device does a one-time set-up: it looks up the
 *   array's device address (cudaGetSymbolAddress) and, under lazy module
 *   loading (the CUDA default), loads the library's kernels, which itself
 *   takes device memory.  Make that first call (a warm-up call will do)
 *   while device memory can still be allocated.  The launch plan reaches
 *   the device as kernel arguments; no call copies host memory.
 *   Asynchronous on `stream`.
 * Errors: INVALID_ARG (null pointer, p < 1), UNSUPPORTED (N > 256), CUDA. */
int qwb_ctransform_noalloc(int32_t N, double p, const double* h_d, double* out_d, void* stream);

/* The same transform for p = 2 by separation of the squared Euclidean cost
 * over the two grid axes (not a step of the paper; an exact reformulation of
 * its lazy c-transform of Sec. 4):
 *   t(i1, j2) = min_i2 (i2 - j2)^2 - h(i1, i2),
 *   out(j1, j2) = min_i1 (i1 - j1)^2 + t(i1, j2),
 * 2 N^3 candidate pairs instead of N^4.  Every candidate is rounded toward
 * -inf, so h_i + out_j <= c_ij holds exactly; out is within two roundings of
 * the exact minimum (MIXED: FP32, h rounded up first; F64: FP64).
 * h_d, out_d: N*N FP64 device.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA, OOM. */
int qwb_ctransform_separable(qwb_ctx* ctx, int32_t N, const double* h_d, double* out_d,
                             qwb_prec prec, void* stream);

/* Gradient of the lower bound with respect to the source measure along the
 * simplex (derived from the proposition of Sec. 3.5: for fixed potentials
 * lb_p = <f, mu> + <g, nu> is linear in mu):
 *   grad_i = (1/p) lb_p^(1/p - 1) (f_i - <f, mu>),  0 when lb_p <= 0.
 * f_d: N*N FP64 (the f from qwb_dual_upscale_ctransform), mu_d: N*N FP64,
 * grad_d: N*N FP64 out.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
int qwb_lb_adjoint(qwb_ctx* ctx, int32_t N, double p, const double* f_d, const double* mu_d,
                   double lb_p, double* grad_d, void* stream);

/* ------------------------------------------------------------------------ */
/* Whole method for many pairs (Sec. 3.2 - 3.5; Alg. 3, 4, 5 together).       */
/* ------------------------------------------------------------------------ */
/* For each pair t: pass (a) on the device, the exact solves of the C~ and
 * C-bar coarse problems on the host (n_threads worker threads, 0 = all
 * cores), then passes (b) and (c) on the device.  mu_d[t], nu_d[t]: device
 * pointers (host arrays of n_pairs pointers).  batched = 0 launches one pair
 * per kernel launch; batched = 1 runs each pass for all pairs in persistent
 * launches replayed from a captured CUDA graph.  ipf_sweeps as in
 * qwb_primal_upscale_ipf.  out_h: n_pairs results (synchronises `stream`).
 * Errors: any of the above; per-pair codes are in out_h[t].status. */
int qwb_bounds(qwb_ctx* ctx, int32_t n_pairs, const qwb_problem* probs_h,
               const double* const* mu_d, const double* const* nu_d, int32_t ipf_sweeps,
               int32_t flags, qwb_result* out_h, qwb_prec prec, int32_t batched,
               int32_t n_threads, void* stream);

/* The same method split into its steps, so that the device passes and the
 * host solves can be timed separately.  A batch owns the workspace and the
 * coarse solutions of n_pairs problems.
 *   qwb_batch_create   -- validate problems, allocate, build launch plans
 *   qwb_batch_coarse   -- pass (a) for every pair (device, asynchronous)
 *   qwb_batch_solve    -- exact C~ and C-bar solves for every pair (host;
 *                         synchronises `stream` to read C-bar)
 *   qwb_batch_fine     -- passes (b) and (c) for every pair (device,
 *                         asynchronous; needs a completed qwb_batch_solve)
 *   qwb_batch_results  -- synchronise and copy the per-pair results out
 *   qwb_batch_potentials -- copy pair t's final dual potentials f, g
 *                         (N*N FP64 each, device, either may be NULL)
 * The pointer arrays must hold the same measures in coarse and fine;
 * qwb_batch_fine uses the coarse solutions of the most recent
 * qwb_batch_solve (re-run solve after the measures change).
 * flags: QWB_FLAG_* bits.  Errors of every step: INVALID_ARG, MASS, CUDA,
 * NOT_CONVERGED, OOM, UNSUPPORTED. */
int qwb_batch_create(qwb_ctx* ctx, int32_t n_pairs, const qwb_problem* probs_h,
                     int32_t ipf_sweeps, int32_t flags, qwb_prec prec, qwb_batch** out);
void qwb_batch_destroy(qwb_batch* batch);
int qwb_batch_coarse(qwb_batch* batch, const double* const* mu_d, const double* const* nu_d,
                     int32_t batched, void* stream);
int qwb_batch_solve(qwb_batch* batch, int32_t n_threads, void* stream);
int qwb_batch_fine(qwb_batch* batch, const double* const* mu_d, const double* const* nu_d,
                   int32_t batched, void* stream);
int qwb_batch_results(qwb_batch* batch, qwb_result* out_h, void* stream);
int qwb_batch_potentials(qwb_batch* batch, int32_t pair, double* f_d, double* g_d, void* stream);
/* Pair t's exact coarse plan pi~ of the C~ problem (Sec. 3.4; the plan the
 * primal pass upscales), from the last qwb_batch_solve, as host CSR:
 * rowptr_h (M + 1), col_h and val_h (cap >= nnz entries each), *nnz_out.  Any
 * of the three arrays may be NULL (a call with all NULL returns the nnz).
 * Errors: INVALID_ARG (bad pair, not solved, cap < nnz). */
int qwb_batch_coarse_plan(qwb_batch* batch, int32_t pair, int32_t* rowptr_h, int32_t* col_h,
                          double* val_h, int32_t cap, int32_t* nnz_out);
/* Pair t's exact coarse dual potentials of the C~ problem (Sec. 2.1 dual,
 * Sec. 3.5: f~ feeds the dual pass, g~ its symmetric form), from the last
 * qwb_batch_solve, before the passes shift them: f_h, g_h (host, M FP64
 * each, either may be NULL) with f~_k + g~_l <= C~_kl.
 * Errors: INVALID_ARG (bad pair, not solved). */
int qwb_batch_coarse_potentials(qwb_batch* batch, int32_t pair, double* f_h, double* g_h);
/* Where the fine FP32 IPF sweeps of the batch's 2-D FP32 pairs with block side
 * 4 or 8 run (Sec. 3.4, IPF paragraph; Alg. 4; the values do not depend on
 * it): C = 0 inside the primal-pass kernel, one CTA per pair; C = 2, 3, 4, 8,
 * 16 on a thread-block cluster of (at most) C CTAs per pair that split the
 * coarse block rows and exchange block sums through distributed shared
 * memory -- the form that keeps HBM busy for large grids.  Each group of
 * pairs with one block side takes, for C = 3, three CTAs if every coarse side
 * is at least 3 (the rows split as ceil(n / 3), the last CTA takes the rest),
 * else the largest power of two <= C dividing all its coarse sides.
 * C | QWB_IPF_WIDE runs that form with CTAs of 512 threads instead of 256
 * (twice the loads in flight per CTA, one CTA per SM).
 * C | QWB_IPF_BULK (C = 2, 4, 8, 16) selects the form that stages the
 * source values by bulk copies (cp.async.bulk into a ring of shared-memory
 * stages, completion on mbarriers, every wait bounded) for groups whose pairs
 * share N; a timed-out wait makes qwb_batch_results return TIMEOUT.
 * Overrides the autotuner's choice, which times both forms;
 * synchronises the device and drops the batch's captured fine-pass graphs.
 * Errors: INVALID_ARG, CUDA. */
#define QWB_IPF_BULK 32
#define QWB_IPF_WIDE 64
int qwb_batch_set_ipf_cluster(qwb_batch* batch, int32_t C);
/* Upscale the coarse plans of the batch's 2-D pairs with block side kappa by
 * the general kernel K_d (Sec. 3.4, eq. coupling tensor upscale; layout,
 * requirements and certification as qwb_primal_upscale_ipf_kernel) instead of
 * the uniform kappa^-4; K_d NULL returns them to the uniform kernel.  K_d is
 * copied (the caller keeps ownership).  Those pairs run the general-kernel
 * primal pass (one CTA or one cluster per pair, qwb_batch_set_upscale_cluster)
 * and leave the cluster IPF groups.  Synchronises the device and drops the batch's captured fine-pass
 * graphs.  Errors: INVALID_ARG (kappa < 1, a non-positive or non-finite
 * entry), UNSUPPORTED (kappa > 8), CUDA, OOM. */
int qwb_batch_set_upscale_kernel(qwb_batch* batch, int32_t kappa, const double* K_d);
/* Where the general-kernel primal pass (the pairs given a kernel K by
 * qwb_batch_set_upscale_kernel) runs: C = 0 one CTA per pair; C = -1 one CTA
 * per pair for the sweeps, then the certified evaluation spread over one CTA
 * per (pair, coarse block row) in four launches; C = 1, 2, 4, 8 the cluster
 * form, one pair on a thread-block cluster of C CTAs of
 * `threads` (256, 128 or 64) threads that split the coarse block rows and
 * read each other's K-product rows through distributed shared memory, which
 * lets a batch of pairs fill every SM at once (Sec. 3.4, eq. coupling tensor
 * upscale; Alg. 4).  The fine sweeps give the same scalings in every form;
 * the certified sums run in another order, so the bounds can differ in
 * their last bits (each is certified).  The cluster form needs FP32 and one
 * block side 2, 4 or 8 for every K pair; otherwise C = 0 runs.  Overrides,
 * for this batch only, the autotuner's choice, which times the forms on the
 * batch's own data; batched and per-pair passes use the same form.  Synchronises the device
 * and drops the batch's captured fine-pass graphs.  Errors: INVALID_ARG (C
 * or threads not listed), UNSUPPORTED (C != 0 while the batch's K pairs
 * cannot take the cluster or spread form), CUDA. */
int qwb_batch_set_upscale_cluster(qwb_batch* batch, int32_t C, int32_t threads);
/* Pair t's scalings after the fine IPF sweeps of the last qwb_batch_fine
 * (Sec. 3.4, IPF paragraph; Alg. 4): the pass-type a, b with
 * a = mu / (pi-hat b), b = nu / (pi-hat^T a) after ipf_sweeps sweeps from
 * b = 1, widened to FP64 (N^d each, device, either may be NULL).  With the
 * uniform kernel the certified bound uses the FP64 block-scalar fit instead
 * (qwb_result fields); with a general kernel it uses these scalings.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
int qwb_batch_fine_scalings(qwb_batch* batch, int32_t pair, double* a_d, double* b_d, void* stream);
/* Device time (ms) of each kernel of the last batched passes, in the order
 * SumPool, C-bar, primal (IPF + upper bound), centre, upsample,
 * c-transform f-hat -> g, c-transform g -> f, lower-bound sum, then the two
 * parts of the primal pass: the cluster IPF sweeps (0 when the sweeps run
 * inside the primal kernel) and the rest (support numerators and the primal
 * kernel); -1 where not measured.
 * Fills min(n, 10) values; call after the stream has completed. */
int qwb_batch_kernel_times(qwb_batch* batch, double* ms_out, int32_t n);
/* Launch configurations the autotuner chose for this batch and the device
 * time of every candidate it measured, as a NUL-terminated JSON object
 * written to json_out (capacity bytes).  The autotuner runs at the first
 * batched coarse / fine pass of a problem signature (set of N, kappa, p,
 * precision and pair count), timing each compiled variant on the batch's own
 * data; results are kept in the context and, when the environment variable
 * QWB_AUTOTUNE_CACHE names a file, stored there and reused by later
 * processes.  QWB_AUTOTUNE=0 keeps the default configuration.
 * Errors: INVALID_ARG (null or too small buffer). */
int qwb_batch_tuning(qwb_batch* batch, char* json_out, int32_t capacity);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */
/* Static name of a status code. */
const char* qwb_status_string(int status);
/* Message of the last failed call on this thread ("" if none). */
const char* qwb_last_error(void);
/* Measured FP32 instruction rate of the current device: the denominator of
 * the rooflines of the passes bound by FP32 arithmetic on the CUDA cores
 * (the c-transform of Sec. 4 and the C-bar reduction of Sec. 3.2; neither is
 * a dense contraction).  The paper has no counterpart.  Every thread runs
 * eight independent dependency chains of one instruction stream, on
 * SMs x ctas_per_sm CTAs of 256 threads (1 <= ctas_per_sm <= 8; one wave),
 * `iters` loop trips of 128 chain steps each, after a shorter warm-up run:
 *   kind 0 fma.rn.f32     1 sub.rm.f32     2 min.f32 (two inputs)
 *        3 min.f32 (three inputs)     4 fma.rn.f32x2     5 sub.rm.f32x2
 *        6 sub.rm.f32x2 then one three-input min.f32 (the line-paired
 *          c-transform's two candidates)
 *        7 two sub.rm.f32 then one three-input min.f32 (two candidates)
 *        8, 9 the shifted c-transform's inner block alone (16 outputs per
 *          thread, 8 columns per chunk, squared offsets in registers, one
 *          rounded-up packed subtraction per column; per candidate pair one
 *          packed round-down subtraction and one three-input min, in one
 *          assembly block (8) or two (9)); 2 CTAs per SM at most
 * ctas_per_sm is lowered to what can be resident at once.
 * out_h (host, 6 doubles): [0] FP32 results (packed: two per instruction;
 * kinds 6, 7: candidates) per cycle per SM, over each SM's span of its cycle
 * counter (first CTA start to last CTA end); [1] the same per second over
 * the whole device, from CUDA events; [2] the cycle counter's rate (MHz)
 * over the timed run; [3] the SM count; [4] the CTAs per SM requested after
 * the occupancy limit; [5] the most CTAs one SM ran.  Allocates a small
 * scratch, uses the current device and the legacy default stream, and
 * synchronises.  Errors: INVALID_ARG, CUDA. */
int qwb_probe_fp32_rate(int32_t kind, int32_t ctas_per_sm, int32_t iters, double* out_h);
/* Number of device kernels this library has launched in this process. */
int64_t qwb_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* QWB_H */
