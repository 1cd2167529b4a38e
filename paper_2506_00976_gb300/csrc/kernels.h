// kernels.h -- device data structures and launchers shared by the entry points.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace qwb {

// Per-pair device descriptor.  Scalar type of the device passes is float
// (MIXED) or double (F64); typed arrays are stored as void* and cast by the
// kernels, which are templated on that type.
struct PairDev {
    int N, kappa, n, M;     // side, block side, coarse side, coarse points n^d
    int d, m, rows;         // dimension (2 or 3), points N^d, lines N^(d-1)
    double p;
    const double* mu;       // N*N fine measures (FP64, caller-owned)
    const double* nu;
    double* mu_c;           // M coarse masses, round-to-nearest sums
    double* nu_c;
    double* mu_c_lo;        // M coarse masses, round-down sums
    double* nu_c_lo;
    double* mu_rinv;        // M upper bounds of 1 / mu~_k (0 where mu~_k = 0)
    double* nu_rinv;
    float* mu_rinv32;       // M FP32 upper bounds of 1 / mu~_k (0: use the FP64 path)
    float* nu_rinv32;
    double* mu_c_hi;        // M coarse masses, round-up sums
    double* nu_c_hi;
    void* mu_t; void* nu_t; // N*N copies of mu, nu in the pass type T (IPF sweeps)
    void* mu_up; void* nu_up; // N*N copies of mu, nu in type T rounded upward (C-bar)
    double* mu_w_hi;        // M upper bounds of sum_{x in X_k} rho(x-bar, x)^p mu(x) (TV weights)
    double* nu_w_hi;
    float* bsum;            // separable p = 2 C-bar (else null): [side][M][2 kappa] FP32 upper
                            // bounds of each block's row sums, then column sums, of mu_up / nu_up
    double* cbar;           // M*M coarse cost out (may be null)
    const void* ctab_lo;    // N*N cost table, lower brackets (T)
    const void* ctab_hi;    // N*N cost table, upper brackets (T)
    const void* ctab_lo_refl;  // lower brackets, rows reflected: [rows][2N], entry c + N - 1 = |c|
    // coarse plan (CSR and CSC) for the primal pass
    const int* rowptr; const int* colidx; const double* val;
    const int* colptr; const int* rowidx; const double* valc;
    const void* val_t; const void* valc_t;   // plan values in the pass type T
    int nnz;
    int sweeps;
    void* supp_num;         // numerators of the support entries (T), from support_num_kernel;
                            // in the plan staging area, one slot per staged entry
    int fine_ext;           // 1: the fine FP32 sweeps run in ipf_fine_kernel, not in primal_kernel
    void* a; void* b;       // N*N fine scalings work (T)
    const double* upK;      // null: the uniform kernel kappa^-2d; else a (kappa^2)^2 kernel K[u, v]
    const void* upK_t;      //   (row-major, offsets row-major in the block) and its copy in type T
    void* kb_t;             // 2 N*N scratch (T) of the general-kernel sweeps, [block][offset]
    double* kscratch;       // 2 N*N scratch (FP64) of its certified evaluation
    double* a_out; double* b_out;   // optional FP64 outputs
    // dual pass
    const double* f_coarse; // M
    const double* g_coarse; // M (the other coarse potential; upscaled when both sides are used)
    void* fhat; void* g; void* f;   // N*N (T)
    double* f_out; double* g_out;   // optional FP64 outputs
    void* tsep;             // N^d (T) scratches of the separable p = 2 c-transform
    void* tsep2;            // (tsep2: second buffer, d = 3 only; may be null)
    int ct_split;           // > 1 when c-transform outputs are combined by atomics
    int out_index;          // index into the results array
};

// Device-side results (one per pair).
struct PairOut {
    double lb, lb_p, w_hat_p, ub_primal, delta_mu, delta_nu, ipf_residual;
    double mass_mu, mass_nu, centre_shift;
    int bad_mu, bad_nu;
    int sweeps_done;
    int verify_bad;         // QWB_FLAG_VERIFY: 1 when some f_i + g_j > c_ij was found
};

struct CbarItem { int pair, w1, seg, pad; };   // wrapped block-row diagonal w1 (seg unused)
struct CtItem { int pair, out0, in_row0, in_rows; };
constexpr int CT_TILE = 4096;   // outputs per c-transform work item (a multiple of every R)
struct PixItem { int pair, start; };
struct SepItem { int pair, line0, lines; };   // separable c-transform: lines [line0, line0 + lines)

// Launch configuration of the c-transform (chosen by the autotuner).
struct CtConfig {
    int R = 8;          // outputs per thread (consecutive in a row)
    int TC = 8;         // input columns per register chunk
    int threads = 256;  // threads per CTA
    int in_rows = 4;    // input rows per work item (split of the min)
    bool p2 = false;    // every pair of the launch has p = 2 (exact integer costs)
    // FP32 packing: 0 none; 1 two columns per packed f32x2 subtraction;
    // 2 two input lines per packed subtraction (row-paired kernel)
    int packed = 0;
    bool has_3d = false;  // some pair of the launch is a volume (selects the 3-D line indexing)
};

// Launchers.  All enqueue on `stream` and return a qwb status.
int launch_cost_tables3(int N, double p, bool f64, void* lo, void* hi, cudaStream_t stream);
int launch_cbar3(const PairDev* pairs_d, const PixItem* items, int n_items, bool f64,
                 cudaStream_t stream);
int launch_cost_tables(int N, double p, bool f64, void* lo, void* hi, cudaStream_t stream);
int launch_reflect_table(int N, int d, bool f64, const void* lo, void* refl, cudaStream_t stream);
int launch_prepare(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items,
                   bool f64, cudaStream_t stream);
constexpr int CBAR_S = 4;   // block rows per C-bar work item
int launch_cbar(const PairDev* pairs_d, const CbarItem* items, int n_items, int kappa_max,
                int n_max, int N_max, bool f64, cudaStream_t stream, int variant = 0);
// C-bar of FP32 2-D p = 2 pairs with kappa (4 or 8) through the separation of
// the squared cost over the two axes (P.bsum set); items (pair, w1 = source
// block row k1); n_max >= every pair's coarse side.
int launch_cbar_sep(const PairDev* pairs_d, const CbarItem* items, int n_items, int kappa, int n_max,
                    cudaStream_t stream);
// support_num_kernel over the pairs of pair_ids, entries [0, nnz_max) of each
// (nnz_max >= every pair's nnz; supp_num has room for the pair's staged plan)
int launch_support_num(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int nnz_max, bool f64,
                       cudaStream_t stream);
int launch_primal(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                  int M_max, int nnz_max, bool f64, cudaStream_t stream);
// The same sweeps with bulk-copy staging (ipf_stream_kernel): every pair of
// the launch has coarse side n and side N (C divides n, N % 4 == 0); err: a
// device int that a timed-out wait sets to nonzero; timeout_ns: the limit of
// every mbarrier wait (global timer); skip_chunk >= 0: every CTA leaves that
// chunk unissued (host-side fault injection for the time-out path), else -1.
int launch_ipf_stream(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int kappa, int C, int n,
                      int N, int* err, unsigned long long timeout_ns, int skip_chunk, cudaStream_t stream);
// The certificate check of the dual potentials (QWB_FLAG_VERIFY): every pair
// (i, j) of fine points of a 2-D pair, f_i + g_j rounded up against a lower
// bracket of c_ij minus `shift` (0; a positive shift is host-side fault
// injection that makes tight pairs fail); sets outs[..].verify_bad.  Items:
// the upsample items (256 output points each).
int launch_verify(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items, bool f64,
                  double shift, cudaStream_t stream);
// primal pass with a general upscaling kernel (P.upK set; d = 2, kappa <= kappa_max <= 8;
// all_kappa4: every pair of the launch has kappa 4, which selects the register-row kernel)
int launch_primalk(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa_max,
                   int M_max, int nnz_max, int m_max, bool all_kappa4, bool f64, cudaStream_t stream,
                   int sweeps_only = 0);
// The certified evaluation of that pass spread over many CTAs, after
// launch_primalk(..., sweeps_only = 1) (FP32 pairs that all have block side
// kappa 2, 4 or 8; n_max >= every pair's coarse side): the K products of
// both sides, the marginal entries, the support cost and the TV terms per
// block row, then one combination per pair and the pixel layout of a, b.
int launch_primalk_eval(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa,
                        int n_max, cudaStream_t stream);
// The same pass for FP32 pairs that all have block side kappa (2, 4 or 8),
// one pair on a cluster of C (1..8) CTAs; variant 0, 1, 2: 256, 128, 64
// threads per CTA; n_max >= every pair's coarse side n.
int launch_primalk_cl(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa,
                      int C, int variant, int n_max, cudaStream_t stream);
// Fine FP32 IPF sweeps on clusters of C (1..16) CTAs of `threads` (256 or
// 512) threads per pair (2-D, kappa 4 or 8, FP32; CTA r owns the block rows
// [r R, (r+1) R), R = ceil(n / C)); the pairs have fine_ext = 1.
int launch_ipf_fine(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int kappa, int C,
                    int M_max, int nnz_max, cudaStream_t stream, int threads = 256);
// side 0 upscales f~ (the dual pass of Alg. 5); side 1 upscales g~ (the
// same pass started from the other coarse potential)
int launch_upsample(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items,
                    bool f64, cudaStream_t stream, int side = 0);
int launch_centre(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                  cudaStream_t stream, int side = 0);
int launch_ctransform(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                      const CtConfig& cfg, int N_max, bool f64, int grid_cap,
                      cudaStream_t stream);
int sep_lines_per_cta(int N);
int launch_sep(const PairDev* pairs_d, const SepItem* items, int n_items, int phase, int stage,
               int N_max, bool f64, int grid_cap, cudaStream_t stream);
int launch_lbsum(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                 bool f64, cudaStream_t stream, int side = 0);
int launch_to_work(const double* h, void* work_in, void* work_out, int m, bool f64,
                   cudaStream_t stream);
int launch_from_work(const void* work, double* out, int m, bool f64, cudaStream_t stream);
int launch_adjoint(int N, double p, const double* f, const double* mu, double lb_p,
                   double* grad, double* scratch, cudaStream_t stream);

// Valid (R, TC) for a grid side N (both must divide N).
int ct_pick_r(int N, int want);

}  // namespace qwb
