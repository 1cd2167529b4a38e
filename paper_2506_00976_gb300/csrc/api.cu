// api.cu -- C ABI entry points (include/qwb.h): context, batches, passes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <fstream>
#include <functional>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "fault.h"
#include "kernels.h"
#include "netsimplex.h"

namespace qwb {

int cuda_fail(cudaError_t e, const char* what) {
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return QWB_ERR_CUDA;
}

static int fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

static int check_problem(const qwb_problem* p) {
    if (!p) return fail(QWB_ERR_INVALID_ARG, "null problem");
    if (p->d != 0 && p->d != 2 && p->d != 3) return fail(QWB_ERR_INVALID_ARG, "d must be 2 or 3");
    if (p->reserved != 0) return fail(QWB_ERR_INVALID_ARG, "qwb_problem.reserved must be 0");
    if (p->N < 1 || p->N > 1024) return fail(QWB_ERR_INVALID_ARG, "N must be in [1, 1024]");
    if (p->kappa < 1 || p->kappa > p->N || p->N % p->kappa != 0)
        return fail(QWB_ERR_INVALID_ARG, "kappa must divide N");
    if (!(p->p >= 1.0) || !std::isfinite(p->p)) return fail(QWB_ERR_INVALID_ARG, "p must be >= 1");
    const int n = p->N / p->kappa;
    if (p->d == 3) {
        if (p->N > 64) return fail(QWB_ERR_UNSUPPORTED, "3-D grids are limited to N <= 64");
        if (n > 16) return fail(QWB_ERR_UNSUPPORTED, "3-D coarse grid larger than 16^3");
        if (p->kappa > 16) return fail(QWB_ERR_UNSUPPORTED, "3-D blocks are limited to kappa <= 16");
        return QWB_OK;
    }
    if (n > 64) return fail(QWB_ERR_UNSUPPORTED, "coarse grid larger than 64 x 64");
    return QWB_OK;
}

static inline int dim_of(const qwb_problem& p) { return p.d == 3 ? 3 : 2; }
static inline int ipow(int x, int d) { int r = 1; while (d-- > 0) r *= x; return r; }

}  // namespace qwb

using namespace qwb;

// --------------------------------------------------------------------------
// Context
// --------------------------------------------------------------------------
struct CostTable {
    int N;
    double p;
    bool f64;
    void* lo;
    void* hi;
    int d;
    void* lo_refl;   // lo with reflected rows (line-paired c-transform)
};

// Launch configuration chosen by the autotuner for one problem signature.
struct TuneEntry {
    std::string key;
    int R = 0, TC = 0, packed = 0, cbar_variant = 2, cbar8_variant = 4, ipf_C = 0;
    int upk_C = 0, upk_var = 0;                       // general-kernel primal pass (cluster form)
    bool ct_done = false, cbar_done = false, ipf_done = false, upk_done = false;
    std::string ct_report, cbar_report, ipf_report, upk_report;   // JSON fragments: candidate -> ms
};

struct qwb_ctx {
    int device = 0;
    int sm_count = 0;
    std::mutex mtx;
    std::vector<CostTable> tables;
    std::vector<qwb_batch*> single_cache;   // single-pair batches for standalone calls
    std::deque<TuneEntry> tunes;            // autotuner results (stable addresses)
    bool autotune = true;                   // QWB_AUTOTUNE=0 keeps the default configuration
    std::string tune_cache;                 // QWB_AUTOTUNE_CACHE: file of tuned configurations
};

static void tune_cache_load(qwb_ctx* c) {
    if (c->tune_cache.empty()) return;
    std::ifstream in(c->tune_cache);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        TuneEntry e;
        std::string r, tc, pk, cv, ipf, upk;
        if (!std::getline(ls, e.key, '|') || !std::getline(ls, r, '|') || !std::getline(ls, tc, '|') ||
            !std::getline(ls, pk, '|') || !std::getline(ls, cv, '|'))
            continue;
        if (std::getline(ls, ipf, '|') && !ipf.empty()) {       // optional: fine-IPF cluster size
            e.ipf_C = std::atoi(ipf.c_str());
            e.ipf_done = true;
            e.ipf_report = "\"cached\"";
        }
        if (std::getline(ls, upk, '|') && !upk.empty()) {       // optional: "C/variant" of the K pass
            e.upk_C = std::atoi(upk.c_str());
            const size_t sl = upk.find('/');
            if (sl != std::string::npos) e.upk_var = std::atoi(upk.c_str() + sl + 1);
            e.upk_done = true;
            e.upk_report = "\"cached\"";
        }
        e.R = std::atoi(r.c_str()); e.TC = std::atoi(tc.c_str());
        e.packed = std::atoi(pk.c_str()); e.cbar_variant = std::atoi(cv.c_str());
        const size_t slash = cv.find('/');                      // "kappa4 variant/kappa8 variant"
        if (slash != std::string::npos) e.cbar8_variant = std::atoi(cv.c_str() + slash + 1);
        e.ct_done = e.R > 0; e.cbar_done = true;
        e.ct_report = "\"cached\""; e.cbar_report = "\"cached\"";
        c->tunes.push_back(e);
    }
}

static void tune_cache_store(qwb_ctx* c) {
    if (c->tune_cache.empty()) return;
    std::ofstream out(c->tune_cache, std::ios::trunc);
    for (auto& e : c->tunes)
        if (e.ct_done && e.cbar_done)
        {
            out << e.key << '|' << e.R << '|' << e.TC << '|' << e.packed << '|' << e.cbar_variant << '/'
                << e.cbar8_variant << '|';
            if (e.ipf_done) out << e.ipf_C;
            out << '|';
            if (e.upk_done) out << e.upk_C << '/' << e.upk_var;
            out << "|\n";
        }
}

static int ctx_table(qwb_ctx* c, int N, double p, bool f64, cudaStream_t s, const void** lo,
                     const void** hi, int d = 2, const void** lo_refl = nullptr) {
    for (auto& t : c->tables)
        if (t.N == N && t.p == p && t.f64 == f64 && t.d == d) {
            *lo = t.lo; *hi = t.hi;
            if (lo_refl) *lo_refl = t.lo_refl;
            return QWB_OK;
        }
    CostTable t{N, p, f64, nullptr, nullptr, d, nullptr};
    const size_t bytes = (size_t)ipow(N, d) * (f64 ? 8 : 4);
    if (cudaMalloc(&t.lo, bytes) != cudaSuccess) return fail(QWB_ERR_OOM, "cost table allocation");
    if (cudaMalloc(&t.hi, bytes) != cudaSuccess) { cudaFree(t.lo); return fail(QWB_ERR_OOM, "cost table allocation"); }
    if (cudaMalloc(&t.lo_refl, 2 * bytes) != cudaSuccess) {
        cudaFree(t.lo); cudaFree(t.hi);
        return fail(QWB_ERR_OOM, "cost table allocation");
    }
    int st = d == 3 ? launch_cost_tables3(N, p, f64, t.lo, t.hi, s) : launch_cost_tables(N, p, f64, t.lo, t.hi, s);
    if (!st) st = launch_reflect_table(N, d, f64, t.lo, t.lo_refl, s);
    if (st) { cudaFree(t.lo); cudaFree(t.hi); cudaFree(t.lo_refl); return st; }
    c->tables.push_back(t);
    *lo = t.lo; *hi = t.hi;
    if (lo_refl) *lo_refl = t.lo_refl;
    return QWB_OK;
}

// --------------------------------------------------------------------------
// Batch: workspace and launch plans for n pairs
// --------------------------------------------------------------------------
struct GraphEntry {
    std::vector<const double*> mu, nu;
    int kind;                 // 0 = coarse pass, 1 = fine passes
    cudaGraphExec_t exec;
    int64_t kernels;          // kernel nodes in the graph
};

struct qwb_batch {
    qwb_ctx* ctx = nullptr;
    int n = 0;
    bool f64 = false;
    int sweeps = 1;
    int flags = 0;
    std::vector<qwb_problem> probs;
    std::vector<PairDev> pairs_h;
    std::vector<int> Ms;
    char* dmem = nullptr;
    PairDev* pairs_d = nullptr;
    PairOut* outs_d = nullptr;
    int* pair_ids_d = nullptr;
    PixItem* prep_items_d = nullptr;
    PixItem* pix_items_d = nullptr;
    CbarItem* cbar_items_d = nullptr;
    CtItem* ct_b_items_d = nullptr;
    CtItem* ct_p_items_d = nullptr;
    SepItem* sep_items_d = nullptr;          // separable p = 2 c-transform items
    std::vector<int> sep_off, sep_cnt;       // per pair (count 0: brute-force transform)
    int n_sep = 0, sep_stages = 0;           // stages: the largest d of a separable pair
    PixItem* cbar3_items_d = nullptr;        // 3-D C-bar items (one per source block)
    std::vector<int> cbar3_off, cbar3_cnt;
    int n_cbar3 = 0;
    bool has_3d = false;
    int n_max2 = 0, N_max2 = 0;              // largest n, N over the other 2-D pairs (generic C-bar kernel)
    // 2-D C-bar items in three groups: FP32 pairs with kappa = 4 and with
    // kappa = 8 whose n is a power of two (cbar4 / cbar8 kernels), then the
    // others (one generic launch, kappa_code)
    int n_cb4 = 0, n_max4 = 0, N_max4 = 0;
    int n_cb8 = 0, n_max8 = 0, N_max8 = 0;
    int cbar8_variant = 4;
    // separable p = 2 C-bar (QWB_FLAG_SEPARABLE, FP32, kappa 4 or 8): groups 12, 16
    int n_cbs4 = 0, n_cbs8 = 0, n_maxs = 0;
    std::vector<char> cbar_group;       // per pair: 4, 8, 12 (separable, kappa 4), 16 (kappa 8) or 0
    // fine IPF sweeps on thread-block clusters (ipf_fine_kernel): 2-D FP32
    // pairs grouped by kappa (4, 8); ipf_C is the requested cluster size
    // (0: every pair sweeps inside primal_kernel), each group runs with the
    // largest power of two <= ipf_C that divides all its coarse sides
    // (stream: the bulk-copy variant ipf_stream_kernel, for groups whose pairs
    // share N; n_same, N_same: that common coarse and fine side, else 0)
    // (wide: CTAs of 512 threads instead of 256, register form only; n_min:
    // the smallest coarse side, which bounds a cluster size that need not
    // divide the sides)
    struct IpfGroup { int kappa, off, cnt, M_max, gcd_n, C, n_same, N_same; bool stream; int n_min; bool wide; };
    std::vector<IpfGroup> ipf_groups;
    std::vector<int> ipf_group_of;      // per pair: its group or -1
    int* ipf_ids_d = nullptr;
    int ipf_C = 0;                      // | QWB_IPF_BULK: the bulk-copy form; | QWB_IPF_WIDE: 512 threads
    int* dev_err = nullptr;             // device error word of bounded waits (0 = none)
    unsigned long long wait_ns = 0;     // limit of every bounded device wait (QWB_WAIT_TIMEOUT_MS)
    int fault_skip_chunk = -1;          // QWB_FAULT ipf_bulk_skip_chunk (tests), else -1
    double verify_shift = 0.0;          // QWB_FAULT verify_shift (tests): tightens the verify check
    // pairs upscaled with a general kernel K (primalk_kernel, 2-D, kappa <= 8):
    // K per kappa, and prim_ids_d = [uniform pairs..., K pairs...]
    std::vector<std::pair<int, std::vector<double>>> upk;   // (kappa, K)
    std::vector<char> upk_on;           // per pair
    char* upk_mem = nullptr;
    int* prim_ids_d = nullptr;
    int n_uni = 0, n_upk = 0, upk_kappa_max = 0, upk_M_max = 0, upk_m_max = 0;
    bool upk_all4 = false;
    // the cluster form of that pass (primalk_cl_kernel): upk_kappa = the
    // common kappa of the K pairs when it is 2, 4 or 8 and the batch is FP32
    // (else 0: the cluster form is not available); upk_C = 0 runs
    // primalk_kernel, else clusters of upk_C CTAs of the thread variant upk_var
    int upk_kappa = 0, upk_n_max = 0, upk_C = 0, upk_var = 0;
    bool upk_req = false;               // qwb_batch_set_upscale_cluster was called:
    int upk_req_C = 0, upk_req_var = 0;     //   its choice
    std::vector<int> prep_off, prep_cnt, pix_off, pix_cnt, cbar_off, cbar_cnt, ct_off, ct_cnt;
    int n_prep = 0, n_pix = 0, n_cbar = 0, n_ct_b = 0;
    int n_ct_b_p2 = 0;   // batched c-transform items: the p = 2 pairs' items come first
    CtConfig ct_cfg_b, ct_cfg_p;
    int kappa_code = 0, n_max = 0, N_max = 0, M_max = 0;
    // coarse-plan staging (pinned host <-> device)
    std::vector<size_t> plan_off;
    size_t plan_bytes = 0;
    char* plan_h = nullptr;
    char* plan_d = nullptr;
    // host copies for the exact solves
    double* cbar_h = nullptr;   // pinned, sum of M^2
    std::vector<size_t> cbar_h_off;
    double* mu_c_h = nullptr;   // pinned: coarse masses of every pair (nu_c_h follows mu_c_h)
    double* nu_c_h = nullptr;
    std::vector<size_t> mc_off;
    // overlap of the exact solves with the C-bar pass: the SumPool results are
    // read on `aux` once the SumPool kernel of a batched coarse pass is done,
    // C-bar comes back in groups of kCbarGroup pairs, each marked by an event
    bool coarse_batched = false;
    cudaStream_t aux = nullptr;
    std::vector<cudaEvent_t> cb_ev;
    std::vector<double> ubw, ubw_p, lbmin;
    std::vector<int> status;
    bool solved = false;
    double t_solve_ms = 0.0;
    cudaEvent_t ev[6] = {};
    cudaEvent_t kev[11] = {};   // per-kernel boundaries of the batched passes
    bool ev_ok = false;
    std::vector<const double*> cur_mu, cur_nu;
    std::vector<GraphEntry> graphs;
    TuneEntry* tune = nullptr;
    int cbar_variant = 0;
    bool cbar_forced = false;   // QWB_CBAR_VARIANT set: the tuner leaves the kappa = 4 choice alone
    int N_gcd = 1;
    bool all_p2 = false;
};

static void batch_free(qwb_batch* b) {
    if (!b) return;
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    if (b->dmem) cudaFree(b->dmem);
    if (b->plan_d) cudaFree(b->plan_d);
    if (b->plan_h) cudaFreeHost(b->plan_h);
    if (b->cbar_h) cudaFreeHost(b->cbar_h);
    if (b->mu_c_h) cudaFreeHost(b->mu_c_h);
    for (auto& e : b->cb_ev) cudaEventDestroy(e);
    if (b->aux) cudaStreamDestroy(b->aux);
    if (b->upk_mem) cudaFree(b->upk_mem);
    if (b->ev_ok) {
        for (auto& e : b->ev) cudaEventDestroy(e);
        for (auto& e : b->kev) cudaEventDestroy(e);
    }
    delete b;
}

struct PlanLayout {   // per-pair coarse plan region
    size_t rowptr, col, val, colptr, rowidx, valc, val_t, valc_t, supp, fco, gco, total;
};
static PlanLayout plan_layout(int M, int cap_nnz = 0) {
    PlanLayout L;
    const int cap = std::max(2 * M, cap_nnz);
    size_t o = 0;
    L.rowptr = o; o = align_up(o + sizeof(int) * (M + 1), 16);
    L.col = o; o = align_up(o + sizeof(int) * cap, 16);
    L.val = o; o = align_up(o + sizeof(double) * cap, 16);
    L.colptr = o; o = align_up(o + sizeof(int) * (M + 1), 16);
    L.rowidx = o; o = align_up(o + sizeof(int) * cap, 16);
    L.valc = o; o = align_up(o + sizeof(double) * cap, 16);
    L.val_t = o; o = align_up(o + sizeof(double) * cap, 16);    // room for either type
    L.valc_t = o; o = align_up(o + sizeof(double) * cap, 16);
    L.supp = o; o = align_up(o + sizeof(double) * cap, 16);      // support numerators (device only)
    L.fco = o; o = align_up(o + sizeof(double) * M, 256);
    L.gco = o; o = align_up(o + sizeof(double) * M, 256);
    L.total = o;
    return L;
}

// Plan values in the pass type, for the fine sweeps.
static void stage_typed_values(char* ph, const PlanLayout& L, int nnz, bool f64) {
    const double* v = (const double*)(ph + L.val);
    const double* vc = (const double*)(ph + L.valc);
    if (f64) {
        std::memcpy(ph + L.val_t, v, sizeof(double) * nnz);
        std::memcpy(ph + L.valc_t, vc, sizeof(double) * nnz);
    } else {
        float* vt = (float*)(ph + L.val_t);
        float* vct = (float*)(ph + L.valc_t);
        for (int e = 0; e < nnz; ++e) { vt[e] = (float)v[e]; vct[e] = (float)vc[e]; }
    }
}

// Cluster size of the fine IPF sweeps: every group takes the largest power of
// two <= C that divides its coarse sides (below 2: sweeps inside
// primal_kernel); the descriptors' fine_ext flags are re-uploaded.
// Group the 2-D FP32 pairs of kappa 4 and 8 that use the uniform kernel for
// the cluster sweeps; returns the pair ids in group order.
static std::vector<int> build_ipf_groups(qwb_batch* b) {
    b->ipf_group_of.assign(b->n, -1);
    b->ipf_groups.clear();
    std::vector<int> ipf_ids;
    if (b->f64) return ipf_ids;
    for (int kap : {4, 8}) {
        qwb_batch::IpfGroup G{kap, (int)ipf_ids.size(), 0, 0, 0, 0, -1, -1, false, 1 << 30, false};
        for (int t = 0; t < b->n; ++t) {
            if (dim_of(b->probs[t]) != 2 || b->probs[t].kappa != kap || b->upk_on[t]) continue;
            const int nn = b->probs[t].N / kap;
            G.n_same = G.n_same < 0 ? nn : (G.n_same == nn ? nn : 0);
            G.N_same = G.N_same < 0 ? b->probs[t].N : (G.N_same == b->probs[t].N ? G.N_same : 0);
            int x = G.gcd_n, y = nn;
            while (y) { const int r = x % y; x = y; y = r; }
            G.gcd_n = x;
            G.M_max = std::max(G.M_max, nn * nn);
            G.n_min = std::min(G.n_min, nn);
            b->ipf_group_of[t] = (int)b->ipf_groups.size();
            ipf_ids.push_back(t);
            ++G.cnt;
        }
        if (G.cnt) b->ipf_groups.push_back(G);
    }
    return ipf_ids;
}

// the fine sweeps of group G (pairs ids[0..cnt)) on clusters
static int launch_ipf_group(qwb_batch* b, const qwb_batch::IpfGroup& G, const int* ids, int cnt, int M,
                            cudaStream_t s) {
    if (G.stream)
        return launch_ipf_stream(b->pairs_d, ids, cnt, G.kappa, G.C, G.n_same, G.N_same, b->dev_err, b->wait_ns,
                                 b->fault_skip_chunk, s);
    return launch_ipf_fine(b->pairs_d, ids, cnt, G.kappa, G.C, M, 0, s, G.wide ? 512 : 256);
}

static int apply_ipf_choice(qwb_batch* b, int C) {
    b->ipf_C = C;
    const int Cs = C & 31;
    for (auto& G : b->ipf_groups) {
        int c = 1;
        if (Cs == 3) {
            c = G.n_min >= 3 ? 3 : 1;        // block rows split unevenly: no divisibility needed
        } else {
            while (c * 2 <= Cs && c * 2 <= 16 && G.gcd_n % (c * 2) == 0) c *= 2;
        }
        G.C = c >= 2 ? c : 0;
        G.stream = (C & QWB_IPF_BULK) && G.C > 0 && G.n_same > 0 && G.N_same > 0;
        G.wide = (C & QWB_IPF_WIDE) && G.C > 0 && !G.stream;
    }
    for (int t = 0; t < b->n; ++t) {
        const int g = b->ipf_group_of[t];
        b->pairs_h[t].fine_ext = (g >= 0 && b->ipf_groups[g].C > 0) ? 1 : 0;
    }
    QWB_CUDA(cudaMemcpy(b->pairs_d, b->pairs_h.data(), sizeof(PairDev) * b->n, cudaMemcpyHostToDevice));
    return QWB_OK;
}

// QWB_CBAR_VARIANT (testing, tuning): force the kappa = 4 C-bar kernel variant
static void apply_cbar_env(qwb_batch* b) {
    if (const char* v = std::getenv("QWB_CBAR_VARIANT")) {
        const int cv = std::atoi(v);
        if (cv == 2 || cv == 3 || (cv >= 6 && cv <= 8)) { b->cbar_variant = cv; b->cbar_forced = true; }
    }
}

static CtConfig pick_ct_config(int N_gcd, bool all_p2) {
    CtConfig c;
    c.R = ct_pick_r(N_gcd, 16);
    c.TC = c.R;
    c.threads = 256;
    c.p2 = all_p2;
    return c;
}

// in_rows so that one pair is split into about `target` items
static int pick_in_rows(int N, int tiles, int target) {
    int splits = std::max(1, target / std::max(1, tiles));
    splits = std::min(splits, N);
    int rows = (N + splits - 1) / splits;
    return std::max(1, rows);
}

static int batch_build(qwb_ctx* ctx, int n, const qwb_problem* probs, int sweeps, int flags,
                       qwb_prec prec, qwb_batch** out) {
    if (n <= 0 || !probs || !out) return fail(QWB_ERR_INVALID_ARG, "batch: bad arguments");
    if (prec != QWB_PREC_F64 && prec != QWB_PREC_MIXED) return fail(QWB_ERR_INVALID_ARG, "bad precision");
    if (sweeps < 1) return fail(QWB_ERR_INVALID_ARG, "ipf sweeps must be >= 1");
    for (int t = 0; t < n; ++t) { int st = check_problem(&probs[t]); if (st) return st; }
    qwb_batch* b = new qwb_batch();
    b->ctx = ctx; b->n = n; b->f64 = (prec == QWB_PREC_F64); b->sweeps = sweeps;
    b->flags = flags;
    b->wait_ns = wait_timeout_ns();
    b->fault_skip_chunk = (int)fault_param("ipf_bulk_skip_chunk", -1);
    b->verify_shift = (double)fault_param("verify_shift", 0);
    b->probs.assign(probs, probs + n);
    const size_t tsz = b->f64 ? 8 : 4;
    // sizes
    size_t off = 0;
    std::vector<size_t> pair_off(n);
    int kap0 = -1;                 // the 2-D C-bar kernel's kappa (over 2-D pairs)
    bool same_kap = true, all_p2 = true;
    int N_gcd = 0;   // the c-transform's outputs per thread must divide every N
    // p = 2 pairs take the separable c-transform when QWB_FLAG_SEPARABLE is set
    auto separable = [&](int t) { return (flags & QWB_FLAG_SEPARABLE) && probs[t].p == 2.0; };
    const bool want_cbar = !(flags & QWB_FLAG_NO_WEIGHTED);
    for (int t = 0; t < n; ++t) {
        const int dd = dim_of(probs[t]);
        const int N = probs[t].N, kap = probs[t].kappa, nn = N / kap, M = ipow(nn, dd), m = ipow(N, dd);
        b->Ms.push_back(M);
        if (dd == 3) b->has_3d = true;
        const bool pow2 = dd == 2 && !(nn & (nn - 1)) && nn <= 64 && !b->f64;
        const bool sepcb = want_cbar && separable(t) && dd == 2 && !b->f64 && (kap == 4 || kap == 8) &&
                           sizeof(float) * ((size_t)nn * 2 * kap + ((nn + 3) & ~3)) <= 48 * 1024;
        const int grp = sepcb ? (kap == 4 ? 12 : 16) : (pow2 && kap == 4) ? 4 : (pow2 && kap == 8) ? 8 : 0;
        b->cbar_group.push_back((char)grp);
        if (grp >= 12) {
            b->n_maxs = std::max(b->n_maxs, nn);
        } else if (grp == 4) {
            b->n_max4 = std::max(b->n_max4, nn);
            b->N_max4 = std::max(b->N_max4, N);
        } else if (grp == 8) {
            b->n_max8 = std::max(b->n_max8, nn);
            b->N_max8 = std::max(b->N_max8, N);
        } else if (dd == 2) {
            if (kap0 < 0) kap0 = kap;
            same_kap &= (kap == kap0);
            b->kappa_code = std::max(b->kappa_code, kap);
            b->n_max2 = std::max(b->n_max2, nn);
            b->N_max2 = std::max(b->N_max2, N);
        }
        if (separable(t)) b->sep_stages = std::max(b->sep_stages, dd);
        if (!separable(t)) {
            all_p2 &= (probs[t].p == 2.0);
            int a = N_gcd, c = N;
            while (c) { const int r = a % c; a = c; c = r; }
            N_gcd = a;
        }
        b->N_max = std::max(b->N_max, N);
        b->n_max = std::max(b->n_max, nn);
        b->M_max = std::max(b->M_max, M);
        pair_off[t] = off;
        off += align_up(12 * sizeof(double) * M);
        if (want_cbar) off += align_up(sizeof(double) * (size_t)M * M);
        if (grp >= 12) off += align_up(sizeof(float) * 4 * (size_t)kap * M);
        off += (separable(t) ? (dd == 3 ? 11 : 10) : 9) * align_up(tsz * m);
        if (flags & QWB_FLAG_SYMMETRIC_DUAL) off += 2 * align_up(sizeof(double) * m);
    }
    if (N_gcd == 0) N_gcd = 8;   // every pair is separable: no brute-force items
    if (kap0 < 0) b->kappa_code = 1;          // no 2-D pair: the 2-D C-bar kernel has no items
    else if (!(same_kap && (kap0 == 1 || kap0 == 2 || kap0 == 4))) b->kappa_code = -b->kappa_code;
    // descriptors and item lists
    const int sm = ctx->sm_count > 0 ? ctx->sm_count : 148;
    std::vector<PixItem> prep, pix;
    std::vector<CbarItem> cb;
    std::vector<CtItem> ctb, ctp;
    std::vector<SepItem> sep;
    b->ct_cfg_b = pick_ct_config(N_gcd, all_p2);
    b->ct_cfg_b.has_3d = b->has_3d;
    b->ct_cfg_p = b->ct_cfg_b;
    b->N_gcd = N_gcd;
    b->all_p2 = all_p2;
    {   // autotuner entry for this problem signature
        std::ostringstream key;
        key << (b->f64 ? "f64" : "mixed") << ":" << n;
        std::vector<std::string> parts;
        for (int t = 0; t < n; ++t) {
            std::ostringstream p1;
            p1 << probs[t].N << "/" << probs[t].kappa << "/" << probs[t].p;
            if (dim_of(probs[t]) == 3) p1 << "/d3";
            parts.push_back(p1.str());
        }
        std::sort(parts.begin(), parts.end());
        parts.erase(std::unique(parts.begin(), parts.end()), parts.end());
        for (auto& p1 : parts) key << ":" << p1;
        TuneEntry* found = nullptr;
        for (auto& e : ctx->tunes) if (e.key == key.str()) found = &e;
        if (!found) { ctx->tunes.push_back(TuneEntry{}); found = &ctx->tunes.back(); found->key = key.str(); }
        b->tune = found;
        if (found->ct_done && found->R > 0 && N_gcd % found->R == 0 && N_gcd % found->TC == 0) {
            b->ct_cfg_b.R = found->R; b->ct_cfg_b.TC = found->TC; b->ct_cfg_b.packed = found->packed;
        }
        // the kappa = 4 row-direct kernel: three (2) or two (3) CTAs per SM, or
        // the variants with first terms as products (6, 7, 8)
        b->cbar_variant = 2;
        if (found->cbar_done && (found->cbar_variant == 2 || found->cbar_variant == 3 ||
                                 (found->cbar_variant >= 6 && found->cbar_variant <= 8)))
            b->cbar_variant = found->cbar_variant;
        if (found->cbar_done && (found->cbar8_variant == 4 || found->cbar8_variant == 5))
            b->cbar8_variant = found->cbar8_variant;
    }
    apply_cbar_env(b);
    const int tile_out = CT_TILE;
    long total_tiles = 0;
    for (int t = 0; t < n; ++t) total_tiles += ((long)ipow(probs[t].N, dim_of(probs[t])) + tile_out - 1) / tile_out;
    // Input-line splits of the batched c-transform items.  The persistent
    // grid (SMs x resident CTAs, 1 to 3 per SM depending on the kernel the
    // autotuner picks) walks the items round-robin, so the last round runs
    // partly empty unless the item count nearly fills a whole number of
    // rounds: take the split, between the one giving about 4 items per SM
    // and 16, whose worst round fill over 1, 2 and 3 CTAs per SM is best
    // (ties to fewer splits, i.e. more input lines per item).
    long splits_fill = 1;
    {
        double best = -1.0;
        const long s_lo = std::max<long>(1, (4L * sm + total_tiles - 1) / std::max<long>(1, total_tiles));
        for (long sp = s_lo; sp <= std::max<long>(s_lo, 16); ++sp) {
            const long items = total_tiles * sp;
            double worst = 1.0;
            for (int occ = 1; occ <= 3; ++occ) {
                const long g = (long)sm * occ;
                const long rounds = (items + g - 1) / g;
                worst = std::min(worst, (double)items / (double)(rounds * g));
            }
            if (worst > best + 1e-3) { best = worst; splits_fill = sp; }
        }
    }
    std::vector<PixItem> cb3;      // 3-D C-bar: one item per source block
    for (int t = 0; t < n; ++t) {
        const int dd = dim_of(probs[t]);
        const int N = probs[t].N, nn = N / probs[t].kappa, M = ipow(nn, dd), m = ipow(N, dd);
        const int rows_all = ipow(N, dd - 1);         // lines of N points
        b->prep_off.push_back((int)prep.size());
        for (int k = 0; k < M; k += 256) prep.push_back({t, k});
        b->prep_cnt.push_back((int)prep.size() - b->prep_off.back());
        b->pix_off.push_back((int)pix.size());
        for (int i = 0; i < m; i += 256) pix.push_back({t, i});
        b->pix_cnt.push_back((int)pix.size() - b->pix_off.back());
        b->cbar3_off.push_back((int)cb3.size());
        if (dd == 3)
            for (int k = 0; k < M; ++k) cb3.push_back({t, k});
        b->cbar3_cnt.push_back((int)cb3.size() - b->cbar3_off.back());
        b->sep_off.push_back((int)sep.size());
        if (separable(t)) {
            const int lines = sep_lines_per_cta(N);
            for (int r0 = 0; r0 < rows_all; r0 += lines) sep.push_back({t, r0, std::min(lines, rows_all - r0)});
            b->sep_cnt.push_back((int)sep.size() - b->sep_off.back());
            b->ct_off.push_back((int)ctp.size());
            b->ct_cnt.push_back(0);
            continue;
        }
        b->sep_cnt.push_back(0);
        const int tiles = (m + tile_out - 1) / tile_out;
        // batched form: each pair's input lines split splits_fill ways (see
        // above; input lines staged per item: at most 32 KB of shared memory)
        const int rows_cap = std::max(1, (int)(32768 / (tsz * (size_t)N)));
        const long splits_b = splits_fill;
        const int rows_b = std::min(rows_cap, pick_in_rows(rows_all, 1, (int)std::min<long>(splits_b, rows_all)));
        for (int o = 0; o < m; o += tile_out)
            for (int r0 = 0; r0 < rows_all; r0 += rows_b) ctb.push_back({t, o, r0, std::min(rows_b, rows_all - r0)});
        // plain form: one pair fills the GPU, about 2 items per SM
        const int rows_p = std::min(rows_cap, pick_in_rows(rows_all, tiles, 2 * sm));
        b->ct_off.push_back((int)ctp.size());
        for (int o = 0; o < m; o += tile_out)
            for (int r0 = 0; r0 < rows_all; r0 += rows_p) ctp.push_back({t, o, r0, std::min(rows_p, rows_all - r0)});
        b->ct_cnt.push_back((int)ctp.size() - b->ct_off.back());
        int maxrows = 0;
        for (auto& it : ctb) maxrows = std::max(maxrows, it.in_rows);
        for (auto& it : ctp) maxrows = std::max(maxrows, it.in_rows);
        b->ct_cfg_b.in_rows = std::max(b->ct_cfg_b.in_rows, maxrows);
        b->ct_cfg_p.in_rows = b->ct_cfg_b.in_rows;
    }
    // 2-D C-bar items: the cbar4 group, the cbar8 group, the separable groups,
    // then the others
    b->cbar_off.assign(n, 0); b->cbar_cnt.assign(n, 0);
    for (int grp : {4, 8, 12, 16, 0}) {
        const int before = (int)cb.size();
        for (int t = 0; t < n; ++t) {
            if (dim_of(probs[t]) != 2 || b->cbar_group[t] != grp) continue;
            b->cbar_off[t] = (int)cb.size();
            for (int w1 = 0; w1 < probs[t].N / probs[t].kappa; ++w1) cb.push_back({t, w1, 0, 0});
            b->cbar_cnt[t] = (int)cb.size() - b->cbar_off[t];
        }
        if (grp == 4) b->n_cb4 = (int)cb.size() - before;
        if (grp == 8) b->n_cb8 = (int)cb.size() - before;
        if (grp == 12) b->n_cbs4 = (int)cb.size() - before;
        if (grp == 16) b->n_cbs8 = (int)cb.size() - before;
    }
    b->n_prep = (int)prep.size(); b->n_pix = (int)pix.size(); b->n_cbar = (int)cb.size();
    b->n_cbar3 = (int)cb3.size();
    // p = 2 pairs first: their items take the exact integer-cost kernels
    std::stable_partition(ctb.begin(), ctb.end(), [&](const CtItem& it) { return probs[it.pair].p == 2.0; });
    b->n_ct_b_p2 = 0;
    for (const auto& it : ctb) b->n_ct_b_p2 += probs[it.pair].p == 2.0 ? 1 : 0;
    b->n_ct_b = (int)ctb.size();
    b->n_sep = (int)sep.size();
    // device allocation
    const size_t o_pairs = align_up(off);
    const size_t o_outs = align_up(o_pairs + sizeof(PairDev) * n);
    const size_t o_ids = align_up(o_outs + sizeof(PairOut) * n);
    const size_t o_prep = align_up(o_ids + sizeof(int) * n);
    const size_t o_pix = align_up(o_prep + sizeof(PixItem) * prep.size());
    const size_t o_cb = align_up(o_pix + sizeof(PixItem) * pix.size());
    const size_t o_ctb = align_up(o_cb + sizeof(CbarItem) * cb.size());
    const size_t o_ctp = align_up(o_ctb + sizeof(CtItem) * ctb.size());
    const size_t o_sep = align_up(o_ctp + sizeof(CtItem) * ctp.size());
    const size_t o_cb3 = align_up(o_sep + sizeof(SepItem) * sep.size());
    b->upk_on.assign(n, 0);
    const std::vector<int> ipf_ids = build_ipf_groups(b);
    const size_t o_ipf = align_up(o_cb3 + sizeof(PixItem) * cb3.size());
    const size_t o_err = align_up(o_ipf + sizeof(int) * std::max<size_t>(1, ipf_ids.size()));
    const size_t total = align_up(o_err + sizeof(int));
    if (cudaMalloc(&b->dmem, total) != cudaSuccess) { batch_free(b); return fail(QWB_ERR_OOM, "batch workspace"); }
    b->pairs_d = (PairDev*)(b->dmem + o_pairs);
    b->outs_d = (PairOut*)(b->dmem + o_outs);
    b->pair_ids_d = (int*)(b->dmem + o_ids);
    b->prep_items_d = (PixItem*)(b->dmem + o_prep);
    b->pix_items_d = (PixItem*)(b->dmem + o_pix);
    b->cbar_items_d = (CbarItem*)(b->dmem + o_cb);
    b->ct_b_items_d = (CtItem*)(b->dmem + o_ctb);
    b->ct_p_items_d = (CtItem*)(b->dmem + o_ctp);
    b->sep_items_d = (SepItem*)(b->dmem + o_sep);
    b->cbar3_items_d = (PixItem*)(b->dmem + o_cb3);
    b->ipf_ids_d = (int*)(b->dmem + o_ipf);
    b->dev_err = (int*)(b->dmem + o_err);
    // coarse-plan staging
    size_t poff = 0;
    for (int t = 0; t < n; ++t) { b->plan_off.push_back(poff); poff += plan_layout(b->Ms[t]).total; }
    b->plan_bytes = poff;
    if (cudaMalloc(&b->plan_d, poff) != cudaSuccess || cudaMallocHost(&b->plan_h, poff) != cudaSuccess) {
        batch_free(b); return fail(QWB_ERR_OOM, "plan staging");
    }
    size_t coff = 0;
    for (int t = 0; t < n; ++t) { b->cbar_h_off.push_back(coff); if (want_cbar) coff += (size_t)b->Ms[t] * b->Ms[t]; }
    if (coff > 0 && cudaMallocHost(&b->cbar_h, sizeof(double) * coff) != cudaSuccess) {
        batch_free(b); return fail(QWB_ERR_OOM, "host C-bar buffer");
    }
    size_t moff = 0;
    for (int t = 0; t < n; ++t) { b->mc_off.push_back(moff); moff += b->Ms[t]; }
    if (cudaMallocHost(&b->mu_c_h, sizeof(double) * 2 * std::max<size_t>(moff, 1)) != cudaSuccess) {
        b->mu_c_h = nullptr; batch_free(b); return fail(QWB_ERR_OOM, "host coarse-mass buffer");
    }
    b->nu_c_h = b->mu_c_h + moff;
    b->ubw.assign(n, 0.0); b->ubw_p.assign(n, 0.0); b->lbmin.assign(n, 0.0); b->status.assign(n, QWB_OK);
    // per-pair descriptors
    cudaStream_t s0 = 0;
    for (int t = 0; t < n; ++t) {
        const int dd = dim_of(probs[t]);
        const int N = probs[t].N, kap = probs[t].kappa, nn = N / kap, M = ipow(nn, dd), m = ipow(N, dd);
        char* base = b->dmem + pair_off[t];
        PairDev P;
        std::memset(&P, 0, sizeof(P));
        P.N = N; P.kappa = kap; P.n = nn; P.M = M; P.p = probs[t].p;
        P.d = dd; P.m = m; P.rows = ipow(N, dd - 1);
        P.mu_c = (double*)base; P.nu_c = P.mu_c + M; P.mu_c_lo = P.nu_c + M; P.nu_c_lo = P.mu_c_lo + M;
        P.mu_rinv = P.nu_c_lo + M; P.nu_rinv = P.mu_rinv + M;
        P.mu_rinv32 = (float*)(P.nu_rinv + M); P.nu_rinv32 = P.mu_rinv32 + M;
        P.mu_c_hi = (double*)(P.nu_rinv32 + M); P.nu_c_hi = P.mu_c_hi + M;
        P.mu_w_hi = P.nu_c_hi + M; P.nu_w_hi = P.mu_w_hi + M;
        base += align_up(12 * sizeof(double) * M);
        if (want_cbar) { P.cbar = (double*)base; base += align_up(sizeof(double) * (size_t)M * M); }
        if (b->cbar_group[t] >= 12) { P.bsum = (float*)base; base += align_up(sizeof(float) * 4 * (size_t)kap * M); }
        P.fhat = base; base += align_up(tsz * m);
        P.g = base; base += align_up(tsz * m);
        P.f = base; base += align_up(tsz * m);
        P.a = base; base += align_up(tsz * m);
        P.b = base; base += align_up(tsz * m);
        P.mu_t = base; base += align_up(tsz * m);
        P.nu_t = base; base += align_up(tsz * m);
        P.mu_up = base; base += align_up(tsz * m);
        P.nu_up = base; base += align_up(tsz * m);
        if (separable(t)) { P.tsep = base; base += align_up(tsz * m); }
        if (separable(t) && dd == 3) { P.tsep2 = base; base += align_up(tsz * m); }
        if (flags & QWB_FLAG_SYMMETRIC_DUAL) {   // the kept side's potentials (FP64)
            P.f_out = (double*)base; base += align_up(sizeof(double) * m);
            P.g_out = (double*)base; base += align_up(sizeof(double) * m);
        }
        const void *lo, *hi;
        const void* lo_refl = nullptr;
        int st = ctx_table(ctx, N, probs[t].p, b->f64, s0, &lo, &hi, dd, &lo_refl);
        if (st) { batch_free(b); return st; }
        P.ctab_lo = lo; P.ctab_hi = hi; P.ctab_lo_refl = lo_refl;
        const PlanLayout L = plan_layout(M);
        char* pd = b->plan_d + b->plan_off[t];
        P.rowptr = (int*)(pd + L.rowptr); P.colidx = (int*)(pd + L.col); P.val = (double*)(pd + L.val);
        P.colptr = (int*)(pd + L.colptr); P.rowidx = (int*)(pd + L.rowidx); P.valc = (double*)(pd + L.valc);
        P.val_t = pd + L.val_t; P.valc_t = pd + L.valc_t;
        P.supp_num = pd + L.supp;
        P.f_coarse = (double*)(pd + L.fco);
        P.g_coarse = (double*)(pd + L.gco);
        P.sweeps = sweeps;
        P.ct_split = 2;
        P.out_index = t;
        b->pairs_h.push_back(P);
    }
    std::vector<int> ids(n);
    for (int t = 0; t < n; ++t) ids[t] = t;
    auto up = [&](void* dst, const void* src, size_t bytes) -> int {
        if (bytes == 0) return QWB_OK;
        QWB_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return QWB_OK;
    };
    int st = up(b->pairs_d, b->pairs_h.data(), sizeof(PairDev) * n);
    if (!st) st = up(b->pair_ids_d, ids.data(), sizeof(int) * n);
    if (!st) st = up(b->prep_items_d, prep.data(), sizeof(PixItem) * prep.size());
    if (!st) st = up(b->pix_items_d, pix.data(), sizeof(PixItem) * pix.size());
    if (!st) st = up(b->cbar_items_d, cb.data(), sizeof(CbarItem) * cb.size());
    if (!st) st = up(b->sep_items_d, sep.data(), sizeof(SepItem) * sep.size());
    if (!st) st = up(b->cbar3_items_d, cb3.data(), sizeof(PixItem) * cb3.size());
    if (!st) st = up(b->ct_b_items_d, ctb.data(), sizeof(CtItem) * ctb.size());
    if (!st) st = up(b->ct_p_items_d, ctp.data(), sizeof(CtItem) * ctp.size());
    if (!st) st = up(b->ipf_ids_d, ipf_ids.data(), sizeof(int) * ipf_ids.size());
    if (!st && cudaMemset(b->dev_err, 0, sizeof(int)) != cudaSuccess) st = fail(QWB_ERR_CUDA, "batch set-up");
    if (!st && b->tune && b->tune->ipf_done) st = apply_ipf_choice(b, b->tune->ipf_C);
    if (!st) {
        b->ev_ok = true;
        for (auto& e : b->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { b->ev_ok = false; }
        for (auto& e : b->kev)
            if (cudaEventCreate(&e) != cudaSuccess) { b->ev_ok = false; }
        if (!b->ev_ok) st = fail(QWB_ERR_CUDA, "event creation");
    }
    if (!st) { cudaError_t e = cudaDeviceSynchronize(); if (e != cudaSuccess) st = cuda_fail(e, "batch set-up"); }
    if (st) { batch_free(b); return st; }
    *out = b;
    return QWB_OK;
}

// Point the descriptors at new measure buffers (host -> device copy when changed).
static int batch_set_measures(qwb_batch* b, const double* const* mu, const double* const* nu) {
    if (!mu || !nu) return fail(QWB_ERR_INVALID_ARG, "null measure pointer array");
    bool changed = b->cur_mu.size() != (size_t)b->n;
    for (int t = 0; t < b->n; ++t) {
        if (!mu[t] || !nu[t]) return fail(QWB_ERR_INVALID_ARG, "null measure pointer");
        if (!changed && (b->cur_mu[t] != mu[t] || b->cur_nu[t] != nu[t])) changed = true;
    }
    if (!changed) return QWB_OK;
    b->cur_mu.assign(mu, mu + b->n);
    b->cur_nu.assign(nu, nu + b->n);
    for (int t = 0; t < b->n; ++t) { b->pairs_h[t].mu = mu[t]; b->pairs_h[t].nu = nu[t]; }
    QWB_CUDA(cudaMemcpy(b->pairs_d, b->pairs_h.data(), sizeof(PairDev) * b->n, cudaMemcpyHostToDevice));
    return QWB_OK;
}

// the generic C-bar kernel's register budget: three CTAs per SM in FP32
static int generic_cbar_variant(bool f64) { return f64 ? 0 : 1; }
// the C-bar variant of pair t when it is launched on its own
static int pair_cbar_variant(const qwb_batch* b, int t) {
    return b->cbar_group[t] == 4 ? b->cbar_variant : b->cbar_group[t] == 8 ? b->cbar8_variant
                                                                           : generic_cbar_variant(b->f64);
}

// An NVTX range over a host call (shown by profilers that record NVTX).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static int mark(qwb_batch* b, int i, cudaStream_t s) {
    // external records become event nodes of a captured graph
    if (b->ev_ok) QWB_CUDA(cudaEventRecordWithFlags(b->kev[i], s, cudaEventRecordExternal));
    return QWB_OK;
}

static int enqueue_coarse(qwb_batch* b, bool batched, cudaStream_t s) {
    int st;
    if (batched) {
        QWB_CUDA(cudaMemsetAsync(b->outs_d, 0, sizeof(PairOut) * b->n, s));
        if ((st = mark(b, 0, s))) return st;
        if ((st = launch_prepare(b->pairs_d, b->outs_d, b->prep_items_d, b->n_prep, b->f64, s))) return st;
        if ((st = mark(b, 1, s))) return st;
        if (!(b->flags & QWB_FLAG_NO_WEIGHTED)) {
            if ((st = launch_cbar(b->pairs_d, b->cbar_items_d, b->n_cb4, 4, b->n_max4, b->N_max4,
                                  b->f64, s, b->cbar_variant)))
                return st;
            if ((st = launch_cbar(b->pairs_d, b->cbar_items_d + b->n_cb4, b->n_cb8, 8, b->n_max8, b->N_max8,
                                  b->f64, s, b->cbar8_variant)))
                return st;
            const int soff = b->n_cb4 + b->n_cb8;
            if ((st = launch_cbar_sep(b->pairs_d, b->cbar_items_d + soff, b->n_cbs4, 4, b->n_maxs, s))) return st;
            if ((st = launch_cbar_sep(b->pairs_d, b->cbar_items_d + soff + b->n_cbs4, b->n_cbs8, 8, b->n_maxs, s)))
                return st;
            const int off = soff + b->n_cbs4 + b->n_cbs8;
            if ((st = launch_cbar(b->pairs_d, b->cbar_items_d + off, b->n_cbar - off, b->kappa_code,
                                  b->n_max2, b->N_max2, b->f64, s, generic_cbar_variant(b->f64))))
                return st;
            if ((st = launch_cbar3(b->pairs_d, b->cbar3_items_d, b->n_cbar3, b->f64, s))) return st;
        }
        return mark(b, 2, s);
    }
    for (int t = 0; t < b->n; ++t) {
        QWB_CUDA(cudaMemsetAsync(b->outs_d + t, 0, sizeof(PairOut), s));
        if ((st = launch_prepare(b->pairs_d, b->outs_d, b->prep_items_d + b->prep_off[t], b->prep_cnt[t], b->f64, s))) return st;
        if (b->flags & QWB_FLAG_NO_WEIGHTED) continue;
        if (dim_of(b->probs[t]) == 3) {
            if ((st = launch_cbar3(b->pairs_d, b->cbar3_items_d + b->cbar3_off[t], b->cbar3_cnt[t], b->f64, s))) return st;
            continue;
        }
        const int nn = b->probs[t].N / b->probs[t].kappa;
        if (b->cbar_group[t] >= 12) {
            if ((st = launch_cbar_sep(b->pairs_d, b->cbar_items_d + b->cbar_off[t], b->cbar_cnt[t],
                                      b->probs[t].kappa, nn, s))) return st;
            continue;
        }
        const int kc = (b->probs[t].kappa == 1 || b->probs[t].kappa == 2 || b->probs[t].kappa == 4 ||
                        b->cbar_group[t] == 8) ? b->probs[t].kappa : -b->probs[t].kappa;
        if ((st = launch_cbar(b->pairs_d, b->cbar_items_d + b->cbar_off[t], b->cbar_cnt[t], kc, nn,
                              b->probs[t].N, b->f64, s, pair_cbar_variant(b, t)))) return st;
    }
    return QWB_OK;
}

// The batched c-transform: one launch over the p = 2 pairs' items (exact
// integer costs), one over the others (cost table).
static int launch_ct_batched(qwb_batch* b, int phase, CtConfig cfg, int cap, cudaStream_t s) {
    int st;
    cfg.p2 = true;
    if ((st = launch_ctransform(b->pairs_d, b->ct_b_items_d, b->n_ct_b_p2, phase, cfg, b->N_max, b->f64, cap, s)))
        return st;
    cfg.p2 = false;
    // the shifted kernels are p = 2 only: the other pairs take the line-paired
    // kernel with per-line costs and the same budget (R capped at 16)
    if (cfg.packed == 9 || cfg.packed == 11) cfg.packed = 5;
    else if (cfg.packed == 10 || cfg.packed == 12) { cfg.packed = 2; cfg.R = std::min(cfg.R, 16); }
    return launch_ctransform(b->pairs_d, b->ct_b_items_d + b->n_ct_b_p2, b->n_ct_b - b->n_ct_b_p2, phase, cfg,
                             b->N_max, b->f64, cap, s);
}

// The general-kernel primal pass over n pairs of ids: primalk_kernel, or the
// cluster form when one was chosen.
static int launch_upk(qwb_batch* b, const int* ids, int n, cudaStream_t s) {
    if (b->upk_C > 0 && b->upk_kappa)
        return launch_primalk_cl(b->pairs_d, b->outs_d, ids, n, b->upk_kappa, b->upk_C, b->upk_var,
                                 b->upk_n_max, s);
    if (b->upk_C < 0 && b->upk_kappa) {        // one-CTA sweeps, evaluation spread over the GPU
        const int st = launch_primalk(b->pairs_d, b->outs_d, ids, n, b->upk_kappa_max, b->upk_M_max, 0,
                                      b->upk_m_max, b->upk_all4, b->f64, s, 1);
        if (st) return st;
        return launch_primalk_eval(b->pairs_d, b->outs_d, ids, n, b->upk_kappa, b->upk_n_max, s);
    }
    return launch_primalk(b->pairs_d, b->outs_d, ids, n, b->upk_kappa_max, b->upk_M_max, 0, b->upk_m_max,
                          b->upk_all4, b->f64, s);
}

static int enqueue_fine(qwb_batch* b, bool batched, cudaStream_t s) {
    int st;
    const int sm = b->ctx->sm_count > 0 ? b->ctx->sm_count : 148;
    const bool do_primal = !(b->flags & QWB_FLAG_NO_PRIMAL), do_dual = !(b->flags & QWB_FLAG_NO_DUAL);
    if (batched) {
        if ((st = mark(b, 3, s))) return st;
        if (do_primal)
            for (const auto& G : b->ipf_groups)
                if (G.C > 0 && (st = launch_ipf_group(b, G, b->ipf_ids_d + G.off, G.cnt, G.M_max, s)))
                    return st;
        if ((st = mark(b, 10, s))) return st;
        if (do_primal) {
            const int* uni = b->n_upk ? b->prim_ids_d : b->pair_ids_d;
            const int n_uni = b->n_upk ? b->n_uni : b->n;
            if ((st = launch_support_num(b->pairs_d, uni, n_uni, 2 * b->M_max, b->f64, s))) return st;
            if ((st = launch_primal(b->pairs_d, b->outs_d, uni, n_uni, b->M_max, 0, b->f64, s))) return st;
            if (b->n_upk && (st = launch_upk(b, b->prim_ids_d + b->n_uni, b->n_upk, s))) return st;
        }
        if ((st = mark(b, 4, s))) return st;
        const int cap = sm;       // persistent grid: all resident CTAs walk the item list
        if (do_dual) {
            if ((st = launch_centre(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, s))) return st;
            if ((st = mark(b, 5, s))) return st;
            if ((st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, s))) return st;
            if ((st = mark(b, 6, s))) return st;
            for (int phase = 0; phase < 2; ++phase) {
                for (int stage = 0; stage < b->sep_stages; ++stage)
                    if ((st = launch_sep(b->pairs_d, b->sep_items_d, b->n_sep, phase, stage, b->N_max, b->f64, cap, s))) return st;
                if ((st = launch_ct_batched(b, phase, b->ct_cfg_b, cap, s))) return st;
                if (phase == 0 && (st = mark(b, 7, s))) return st;
            }
            if ((st = mark(b, 8, s))) return st;
            if ((st = launch_lbsum(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, b->f64, s))) return st;
        } else {
            for (int i = 5; i <= 8; ++i) if ((st = mark(b, i, s))) return st;
        }
        if ((st = mark(b, 9, s))) return st;
        if (do_dual && (b->flags & QWB_FLAG_VERIFY) &&
            (st = launch_verify(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, b->verify_shift, s)))
            return st;
        if (do_dual && (b->flags & QWB_FLAG_SYMMETRIC_DUAL)) {
            // the same pass from g~: g-hat -> f -> g, keep the larger bound
            if ((st = launch_centre(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, s, 1))) return st;
            if ((st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, s, 1))) return st;
            for (int phase = 0; phase < 2; ++phase) {
                for (int stage = 0; stage < b->sep_stages; ++stage)
                    if ((st = launch_sep(b->pairs_d, b->sep_items_d, b->n_sep, phase, stage, b->N_max, b->f64, cap, s))) return st;
                if ((st = launch_ct_batched(b, phase, b->ct_cfg_b, cap, s))) return st;
            }
            if ((st = launch_lbsum(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, b->f64, s, 1))) return st;
            if ((b->flags & QWB_FLAG_VERIFY) &&
                (st = launch_verify(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, b->verify_shift, s)))
                return st;
        }
        return QWB_OK;
    }
    for (int t = 0; t < b->n; ++t) {
        const int* id = b->pair_ids_d + t;
        const int M = b->Ms[t];
        if (do_primal && b->upk_on[t]) {
            if (b->upk_C > 0) {     // the same form and shape as the batched pass
                if ((st = launch_primalk_cl(b->pairs_d, b->outs_d, id, 1, b->upk_kappa, b->upk_C, b->upk_var,
                                            b->probs[t].N / b->upk_kappa, s)))
                    return st;
            } else if (b->upk_C < 0) {
                const int kap = b->probs[t].kappa;
                if ((st = launch_primalk(b->pairs_d, b->outs_d, id, 1, kap, M, 0, b->probs[t].N * b->probs[t].N,
                                         kap == 4, b->f64, s, 1)))
                    return st;
                if ((st = launch_primalk_eval(b->pairs_d, b->outs_d, id, 1, kap, b->probs[t].N / kap, s))) return st;
            } else {
                const int kap = b->probs[t].kappa;
                if ((st = launch_primalk(b->pairs_d, b->outs_d, id, 1, kap, M, 0, b->probs[t].N * b->probs[t].N,
                                         kap == 4, b->f64, s)))
                    return st;
            }
        } else if (do_primal) {
            if ((st = launch_support_num(b->pairs_d, id, 1, 2 * M, b->f64, s))) return st;
            if (b->ipf_group_of[t] >= 0 && b->ipf_groups[b->ipf_group_of[t]].C > 0) {
                const auto& G = b->ipf_groups[b->ipf_group_of[t]];
                if ((st = launch_ipf_group(b, G, id, 1, M, s))) return st;
            }
            if ((st = launch_primal(b->pairs_d, b->outs_d, id, 1, M, 0, b->f64, s))) return st;
        }
        if (!do_dual) continue;
        if ((st = launch_centre(b->pairs_d, b->outs_d, id, 1, s))) return st;
        if ((st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d + b->pix_off[t], b->pix_cnt[t], b->f64, s))) return st;
        CtConfig c = b->ct_cfg_p;
        c.p2 = (b->probs[t].p == 2.0);
        c.has_3d = dim_of(b->probs[t]) == 3;
        const int sides = (b->flags & QWB_FLAG_SYMMETRIC_DUAL) ? 2 : 1;
        for (int side = 0; side < sides; ++side) {
            if (side == 1) {
                if ((st = launch_centre(b->pairs_d, b->outs_d, id, 1, s, 1))) return st;
                if ((st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d + b->pix_off[t], b->pix_cnt[t], b->f64, s, 1))) return st;
            }
            for (int phase = 0; phase < 2; ++phase) {
                const SepItem* si = b->sep_items_d + b->sep_off[t];
                for (int stage = 0; stage < dim_of(b->probs[t]) && b->sep_cnt[t] > 0; ++stage)
                    if ((st = launch_sep(b->pairs_d, si, b->sep_cnt[t], phase, stage, b->probs[t].N, b->f64, 0, s))) return st;
                if ((st = launch_ctransform(b->pairs_d, b->ct_p_items_d + b->ct_off[t], b->ct_cnt[t], phase, c, b->probs[t].N, b->f64, 0, s))) return st;
            }
            if ((st = launch_lbsum(b->pairs_d, b->outs_d, id, 1, b->f64, s, side))) return st;
            if ((b->flags & QWB_FLAG_VERIFY) &&
                (st = launch_verify(b->pairs_d, b->outs_d, b->pix_items_d + b->pix_off[t], b->pix_cnt[t], b->f64,
                                    b->verify_shift, s)))
                return st;
        }
    }
    return QWB_OK;
}

// ---- autotuner -------------------------------------------------------------
// Times each compiled variant of a pass on the batch's own data (CUDA events,
// best of two runs after one warm-up) and keeps the fastest.  Every variant
// computes the same values, so the buffers are simply overwritten.
static int time_variant(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                        const std::function<int()>& launch, double* ms) {
    int st = launch();
    if (st) return st;
    double best = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
        QWB_CUDA(cudaEventRecord(e0, s));
        if ((st = launch())) return st;
        QWB_CUDA(cudaEventRecord(e1, s));
        QWB_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        QWB_CUDA(cudaEventElapsedTime(&t, e0, e1));
        best = std::min(best, (double)t);
    }
    *ms = best;
    return QWB_OK;
}

static const char* cbar_variant_name(int v) {
    switch (v) {
        case 0: return "staged_rows/2_ctas_per_sm";
        case 1: return "staged_rows/3_ctas_per_sm";
        case 2: return "kappa4_direct_rows/3_ctas_per_sm";
        case 3: return "kappa4_direct_rows/2_ctas_per_sm";
        case 4: return "kappa8_direct_rows/2_ctas_per_sm";
        case 5: return "kappa8_direct_rows/1_cta_per_sm";
        case 6: return "kappa4_direct_rows_8staged_firstmul/3_ctas_per_sm";
        case 7: return "kappa4_direct_rows_8staged_firstmul/2_ctas_per_sm";
        default: return "kappa4_direct_rows_firstmul/3_ctas_per_sm";
    }
}

static int tune_cbar(qwb_batch* b, cudaStream_t s) {
    TuneEntry* e = b->tune;
    if (!b->ctx->autotune || !e || e->cbar_done || !b->ev_ok) return QWB_OK;
    if ((b->n_cb4 == 0 && b->n_cb8 == 0) || (b->flags & QWB_FLAG_NO_WEIGHTED)) { e->cbar_done = true; e->cbar_report = "{}"; return QWB_OK; }
    int st = launch_prepare(b->pairs_d, b->outs_d, b->prep_items_d, b->n_prep, b->f64, s);
    if (st) return st;
    std::ostringstream rep;
    double best = 1e30;
    rep << "{";
    bool first = true;
    for (int v : {2, 3, 6, 7, 8}) {
        if (b->n_cb4 == 0) break;
        double ms;
        st = time_variant(s, b->ev[0], b->ev[1], [&] {
            return launch_cbar(b->pairs_d, b->cbar_items_d, b->n_cb4, 4, b->n_max4, b->N_max4, b->f64, s, v);
        }, &ms);
        if (st) return st;
        rep << (first ? "" : ", ") << "\"" << cbar_variant_name(v) << "\": " << ms;
        first = false;
        if (ms < best) { best = ms; e->cbar_variant = v; }
    }
    double best8 = 1e30;
    for (int v = 4; v < 6 && b->n_cb8 > 0; ++v) {
        double ms;
        st = time_variant(s, b->ev[0], b->ev[1], [&] {
            return launch_cbar(b->pairs_d, b->cbar_items_d + b->n_cb4, b->n_cb8, 8, b->n_max8, b->N_max8, b->f64,
                               s, v);
        }, &ms);
        if (st) return st;
        rep << (first ? "" : ", ") << "\"" << cbar_variant_name(v) << "\": " << ms;
        first = false;
        if (ms < best8) { best8 = ms; e->cbar8_variant = v; }
    }
    rep << "}";
    e->cbar_report = rep.str();
    e->cbar_done = true;
    if (!b->cbar_forced) b->cbar_variant = e->cbar_variant;
    b->cbar8_variant = e->cbar8_variant;
    tune_cache_store(b->ctx);
    return QWB_OK;
}

static int tune_ctransform(qwb_batch* b, cudaStream_t s) {
    TuneEntry* e = b->tune;
    if (!b->ctx->autotune || !e || e->ct_done || !b->ev_ok || (b->flags & QWB_FLAG_NO_DUAL)) return QWB_OK;
    int st = launch_centre(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, s);
    if (!st) st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, s);
    if (st) return st;
    const int cand[][3] = {{4, 4, 0}, {8, 8, 0}, {16, 8, 0}, {16, 16, 0}, {8, 16, 0},
                           {8, 8, 1}, {16, 8, 1}, {16, 16, 1},
                           {8, 8, 2}, {16, 8, 2}, {8, 16, 2}, {16, 16, 2},
                           {8, 8, 3}, {8, 8, 4}, {8, 16, 4}, {8, 16, 5}, {16, 8, 5}, {16, 16, 5},
                           {8, 16, 6}, {16, 16, 7}, {16, 8, 7}, {8, 16, 7}, {16, 16, 8},
                           {16, 16, 9}, {16, 8, 9}, {8, 16, 9}, {16, 16, 10}, {32, 16, 10}, {32, 8, 10},
                           {16, 16, 11}, {16, 8, 11}, {8, 16, 11}, {16, 16, 12}, {32, 8, 12}};
    static const char* const kPackName[] = {"", "_packed", "_linepairs", "_linepairs_3cta_fly",
                                            "_linepairs_3cta", "_linepairs_2cta", "_linepairs_2cta_fly",
                                            "_linepairs_2cta_fused", "_linepairs_fused",
                                            "_linepairs_shifted_2cta", "_linepairs_shifted",
                                            "_linepairs_shifted_pinned_2cta", "_linepairs_shifted_pinned"};
    const int sm = b->ctx->sm_count > 0 ? b->ctx->sm_count : 148;
    std::ostringstream rep;
    double best = 1e30;
    bool first = true;
    rep << "{";
    for (auto& c : cand) {
        if (b->N_gcd % c[0] || b->N_gcd % c[1] || (c[2] && b->f64) || (c[2] >= 3 && b->has_3d)) continue;
        if (c[2] >= 9 && b->n_ct_b_p2 == 0) continue;            // p = 2 only
        CtConfig cfg = b->ct_cfg_b;
        cfg.R = c[0]; cfg.TC = c[1]; cfg.packed = c[2];
        double ms;
        st = time_variant(s, b->ev[0], b->ev[1], [&] {
            return launch_ct_batched(b, 0, cfg, sm, s);
        }, &ms);
        if (st) return st;
        rep << (first ? "" : ", ") << "\"R" << c[0] << "xT" << c[1] << kPackName[c[2]] << "\": " << ms;
        first = false;
        if (ms < best) { best = ms; e->R = c[0]; e->TC = c[1]; e->packed = c[2]; }
    }
    rep << "}";
    e->ct_report = rep.str();
    e->ct_done = e->R > 0;
    if (e->ct_done) { b->ct_cfg_b.R = e->R; b->ct_cfg_b.TC = e->TC; b->ct_cfg_b.packed = e->packed; }
    tune_cache_store(b->ctx);
    return QWB_OK;
}

// Fine IPF: sweeps inside primal_kernel (C = 0) or on clusters of 2, 4, 8, 16
// CTAs per pair (256 threads, or 512 for C = 2, 4; or the bulk-copy form),
// timed as the whole primal pass.
static int tune_ipf(qwb_batch* b, cudaStream_t s) {
    TuneEntry* e = b->tune;
    if (!b->ctx->autotune || !e || e->ipf_done || !b->ev_ok || (b->flags & QWB_FLAG_NO_PRIMAL) ||
        b->ipf_groups.empty())
        return QWB_OK;
    {   // the primal kernel reads the support numerators
        const int st0 = launch_support_num(b->pairs_d, b->pair_ids_d, b->n, 2 * b->M_max, b->f64, s);
        if (st0) return st0;
    }
    std::ostringstream rep;
    rep << "{";
    double best = 1e30;
    int bestC = 0;
    // (three CTAs per pair measured slower than four on every workload tried:
    // settable, not timed)
    for (int C : {0, 2, 4, 8, 16, QWB_IPF_WIDE | 2, QWB_IPF_WIDE | 4, QWB_IPF_BULK | 2, QWB_IPF_BULK | 4,
                  QWB_IPF_BULK | 8, QWB_IPF_BULK | 16}) {
        int st = apply_ipf_choice(b, C);
        if (st) return st;
        if (C > 0) {
            bool any = false;
            for (const auto& G : b->ipf_groups)
                any |= G.C == (C & 31) && G.stream == ((C & QWB_IPF_BULK) != 0) &&
                       G.wide == ((C & QWB_IPF_WIDE) != 0);
            if (!any) continue;                  // no group takes this size / form
        }
        double ms;
        st = time_variant(s, b->ev[0], b->ev[1], [&] {
            int st2;
            for (const auto& G : b->ipf_groups)
                if (G.C > 0 && (st2 = launch_ipf_group(b, G, b->ipf_ids_d + G.off, G.cnt, G.M_max, s)))
                    return st2;
            return launch_primal(b->pairs_d, b->outs_d, b->pair_ids_d, b->n, b->M_max, 0, b->f64, s);
        }, &ms);
        if (st) return st;
        rep << (C ? ", " : "") << "\""
            << ((C & QWB_IPF_BULK) ? "bulk" : (C & QWB_IPF_WIDE) ? "wide" : "cluster")
            << (C & 31) << "\": " << ms;
        if (ms < best) { best = ms; bestC = C; }
    }
    rep << "}";
    const int st = apply_ipf_choice(b, bestC);
    if (st) return st;
    e->ipf_C = bestC;
    e->ipf_report = rep.str();
    e->ipf_done = true;
    tune_cache_store(b->ctx);
    return QWB_OK;
}

// General-kernel primal pass: primalk_kernel (one CTA per pair, "single")
// or the cluster form with C CTAs per pair and 256, 128 or 64 threads per
// CTA, timed as the launch over the batch's K pairs.
static int tune_upk(qwb_batch* b, cudaStream_t s) {
    TuneEntry* e = b->tune;
    if (!b->n_upk || !b->upk_kappa || b->upk_req) return QWB_OK;
    if (e && e->upk_done) {                              // timed by another batch of this signature
        b->upk_C = e->upk_C;
        b->upk_var = e->upk_var;
        return QWB_OK;
    }
    if (!b->ctx->autotune || !e || !b->ev_ok || (b->flags & QWB_FLAG_NO_PRIMAL)) return QWB_OK;
    static const int threads_of[3] = {256, 128, 64};
    struct Cand { int C, var; };
    const Cand cands[] = {{0, 0}, {-1, 0}, {1, 0}, {2, 0}, {2, 1}, {4, 1}, {4, 2}, {8, 1}, {8, 2}};
    std::ostringstream rep;
    rep << "{";
    double best = 1e30;
    Cand pick{0, 0};
    bool first = true;
    for (const Cand& c : cands) {
        if (c.C > b->upk_n_max) continue;                    // every CTA owns at least one block row
        b->upk_C = c.C;
        b->upk_var = c.var;
        double ms;
        const int st = time_variant(s, b->ev[0], b->ev[1], [&] {
            return launch_upk(b, b->prim_ids_d + b->n_uni, b->n_upk, s);
        }, &ms);
        if (st == QWB_ERR_UNSUPPORTED) continue;             // shared memory does not fit this size
        if (st) { b->upk_C = 0; return st; }
        rep << (first ? "" : ", ") << "\"";
        if (c.C > 0) rep << "cluster" << c.C << "x" << threads_of[c.var];
        else rep << (c.C < 0 ? "single_sweeps_spread_eval" : "single");
        rep << "\": " << ms;
        first = false;
        if (ms < best) { best = ms; pick = c; }
    }
    rep << "}";
    b->upk_C = pick.C;
    b->upk_var = pick.var;
    e->upk_C = pick.C;
    e->upk_var = pick.var;
    e->upk_report = rep.str();
    e->upk_done = true;
    tune_cache_store(b->ctx);
    return QWB_OK;
}

// Run a pass for the whole batch, through a captured CUDA graph when batched.
static int run_pass(qwb_batch* b, int kind, bool batched, cudaStream_t s) {
    if (!batched) return kind == 0 ? enqueue_coarse(b, false, s) : enqueue_fine(b, false, s);
    for (auto& g : b->graphs)
        if (g.kind == kind && g.mu == b->cur_mu && g.nu == b->cur_nu) {
            QWB_CUDA(cudaGraphLaunch(g.exec, s));
            count_launch(g.kernels);
            return QWB_OK;
        }
    // tune this pass's kernels on the batch's data before the first capture
    {
        int st_t = kind == 0 ? tune_cbar(b, s) : tune_ctransform(b, s);
        if (!st_t && kind == 1) st_t = tune_ipf(b, s);
        if (!st_t && kind == 1) st_t = tune_upk(b, s);
        if (st_t) return st_t;
    }
    // capture on a private stream, then launch on the caller's stream
    cudaStream_t cs;
    QWB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int st = QWB_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(e, "begin capture"); }
    const int64_t before = qwb_kernel_launch_count();
    st = kind == 0 ? enqueue_coarse(b, true, cs) : enqueue_fine(b, true, cs);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    const int64_t captured = qwb_kernel_launch_count() - before;
    count_launch(-captured);                            // captured, not yet launched
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    GraphEntry g{b->cur_mu, b->cur_nu, kind, nullptr, captured};
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graphs.push_back(g);
    QWB_CUDA(cudaGraphLaunch(g.exec, s));
    count_launch(g.kernels);
    return QWB_OK;
}

// ---- host exact solves ---------------------------------------------------
// Coarse-grid costs depend only on the block offset |k - l| per axis; tables
// hold them for every offset, tab[(|dk1| * n + |dk2|) * n + |dk3|] (2-D: no dk3).
static int grid_offset(int d, int nn, int k, int l) {
    if (d == 3) {
        const int a = std::abs(k / (nn * nn) - l / (nn * nn)), b = std::abs((k / nn) % nn - (l / nn) % nn);
        return (a * nn + b) * nn + std::abs(k % nn - l % nn);
    }
    return std::abs(k / nn - l / nn) * nn + std::abs(k % nn - l % nn);
}

// |delta|^p from the exact squared length s, rounded down (round_down) or to
// nearest: the centre cost feeds an exact solve, the minimum cost a bound.
static double cost_of_sq(double s, double p, bool round_down) {
    if (p == 2.0) return s;
    double c = p == 1.0 ? std::sqrt(s) : std::pow(s, 0.5 * p);
    if (round_down) {
        if (p == 1.0) { if (c * c > s) c = std::nextafter(c, 0.0); }
        else c *= 1.0 - std::ldexp(1.0, -49);
    }
    return c;
}

// C^min on the coarse grid (Sec. 3.3): the per-axis gap between two blocks is
// max(0, kappa |dk| - (kappa - 1)) points, C^min = (sum of gap^2)^(p/2),
// rounded down so that the LP value stays a lower bound.
static void mincost_table(const qwb_problem& pr, std::vector<double>& tab) {
    const int nn = pr.N / pr.kappa, d = dim_of(pr), d3 = d == 3 ? nn : 1;
    tab.resize((size_t)ipow(nn, d));
    for (int d1 = 0; d1 < nn; ++d1)
        for (int d2 = 0; d2 < nn; ++d2)
            for (int dz = 0; dz < d3; ++dz) {
                const double g1 = std::max(0, pr.kappa * d1 - (pr.kappa - 1));
                const double g2 = std::max(0, pr.kappa * d2 - (pr.kappa - 1));
                const double g3 = d == 3 ? std::max(0, pr.kappa * dz - (pr.kappa - 1)) : 0.0;
                tab[((size_t)d1 * nn + d2) * d3 + dz] = cost_of_sq(g1 * g1 + g2 * g2 + g3 * g3, pr.p, true);
            }
}

// C~ on the coarse grid as a table over block offsets: (kappa |dk|)^p.
static void centre_cost_table(const qwb_problem& pr, std::vector<double>& tab) {
    const int nn = pr.N / pr.kappa, d = dim_of(pr), d3 = d == 3 ? nn : 1;
    tab.resize((size_t)ipow(nn, d));
    for (int d1 = 0; d1 < nn; ++d1)
        for (int d2 = 0; d2 < nn; ++d2)
            for (int dz = 0; dz < d3; ++dz) {
                const double x = (double)pr.kappa * d1, y = (double)pr.kappa * d2;
                const double z = d == 3 ? (double)pr.kappa * dz : 0.0;
                tab[((size_t)d1 * nn + d2) * d3 + dz] = cost_of_sq(x * x + y * y + z * z, pr.p, false);
            }
}

// Exact solve of a coarse problem whose cost is a block-offset table: the
// grid network simplex (no M x M matrix) in 2-D, the dense one in 3-D.
static int solve_table(const qwb_problem& pr, const std::vector<double>& tab, const double* a,
                       const double* b, NSSolution& out, NSBasis* basis_out, const NSBasis* warm) {
    const int nn = pr.N / pr.kappa, d = dim_of(pr);
    if (d == 2) return network_simplex_grid(nn, tab.data(), a, b, out, -1, basis_out, warm);
    const int M = ipow(nn, d);
    std::vector<double> C((size_t)M * M);
    for (int k = 0; k < M; ++k)
        for (int l = 0; l < M; ++l) C[(size_t)k * M + l] = tab[grid_offset(d, nn, k, l)];
    return network_simplex(M, M, C.data(), a, b, out, -1, warm, basis_out);
}

// wait_cbar (may be empty): blocks until pair t's C-bar is on the host
static int solve_pair(qwb_batch* b, int t, const std::function<int(int)>& wait_cbar) {
    const qwb_problem& pr = b->probs[t];
    const int M = b->Ms[t];
    const double* mc = b->mu_c_h + b->mc_off[t];
    const double* nc = b->nu_c_h + b->mc_off[t];
    // (1) C~ problem: plan and potential for the primal and dual passes
    std::vector<double> Ct;
    centre_cost_table(pr, Ct);
    NSSolution sol;
    NSBasis basis;
    int st = solve_table(pr, Ct, mc, nc, sol, &basis, nullptr);
    if (st) return st;
    const PlanLayout L = plan_layout(M);
    char* ph = b->plan_h + b->plan_off[t];
    const int nnz = (int)sol.col.size();
    std::memcpy(ph + L.rowptr, sol.rowptr.data(), sizeof(int) * (M + 1));
    std::memcpy(ph + L.col, sol.col.data(), sizeof(int) * nnz);
    std::memcpy(ph + L.val, sol.val.data(), sizeof(double) * nnz);
    std::vector<int> cnt(M + 1, 0);
    for (int e = 0; e < nnz; ++e) cnt[sol.col[e] + 1]++;
    for (int l = 0; l < M; ++l) cnt[l + 1] += cnt[l];
    int* colptr = (int*)(ph + L.colptr);
    int* rowidx = (int*)(ph + L.rowidx);
    double* valc = (double*)(ph + L.valc);
    std::memcpy(colptr, cnt.data(), sizeof(int) * (M + 1));
    std::vector<int> cur(cnt.begin(), cnt.end() - 1);
    for (int k = 0; k < M; ++k)                   // rows in order: CSC rows sorted
        for (int e = sol.rowptr[k]; e < sol.rowptr[k + 1]; ++e) {
            const int pos = cur[sol.col[e]]++;
            rowidx[pos] = k; valc[pos] = sol.val[e];
        }
    std::memcpy(ph + L.fco, sol.f.data(), sizeof(double) * M);
    std::memcpy(ph + L.gco, sol.g.data(), sizeof(double) * M);
    stage_typed_values(ph, L, nnz, b->f64);
    b->pairs_h[t].nnz = nnz;
    // (1b) optional min-cost lower bound: a dual-feasible pair of the C^min
    // problem bounds L_Cmin <= W_p^p from below (weak duality); the dual
    // objective is summed with an error margin
    if (b->flags & QWB_FLAG_MINCOST) {
        std::vector<double> Cm;
        mincost_table(pr, Cm);
        NSSolution sm;
        st = solve_table(pr, Cm, mc, nc, sm, nullptr, &basis);
        if (st) return st;
        const int nn = pr.N / pr.kappa, dd = dim_of(pr);
        // g_j = min_i C_ij - f_i rounded down keeps f_i + g_j <= C_ij exactly
        std::vector<double> g(M, HUGE_VAL);
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                const double c = Cm[grid_offset(dd, nn, i, j)];
                double v = c - sm.f[i];
                if (v + sm.f[i] > c) v = std::nextafter(v, -HUGE_VAL);
                g[j] = std::min(g[j], v);
            }
        double s = 0.0, mag = 0.0;
        for (int k = 0; k < M; ++k) {
            s += sm.f[k] * mc[k] + g[k] * nc[k];
            mag += std::fabs(sm.f[k]) * mc[k] + std::fabs(g[k]) * nc[k];
        }
        const double u = std::ldexp(1.0, -53);
        const double s_lo = s - (2.0 * M + 4) * u * mag;
        const double p = pr.p;
        b->lbmin[t] = s_lo > 0.0 ? std::pow(s_lo, 1.0 / p) * (1.0 - 4 * u) : 0.0;
    }
    // (2) C-bar problem: certified weighted-cost upper bound
    if (b->flags & QWB_FLAG_NO_WEIGHTED) {
        b->ubw_p[t] = HUGE_VAL; b->ubw[t] = HUGE_VAL;
        return QWB_OK;
    }
    // same supplies: the C~ optimum is a feasible starting basis, and the
    // arcs from each source to the 3 x 3 (3 x 3 x 3) neighbourhoods of its C~
    // plan targets are priced first (the solve still ends optimal over all arcs)
    if (wait_cbar) {
        const int stw = wait_cbar(t);
        if (stw) return stw;
    }
    NSSolution sb;
    const double* Cb = b->cbar_h + b->cbar_h_off[t];
    std::vector<int64_t> cand;
    {
        const int nn = pr.N / pr.kappa, dd = dim_of(pr);
        cand.reserve((size_t)sol.col.size() * (dd == 3 ? 27 : 9));
        for (int k = 0; k < M; ++k)
            for (int e = sol.rowptr[k]; e < sol.rowptr[k + 1]; ++e) {
                const int l = sol.col[e];
                const int l1 = dd == 3 ? l / (nn * nn) : l / nn, l2 = dd == 3 ? (l / nn) % nn : l % nn;
                const int l3 = dd == 3 ? l % nn : 0;
                for (int d1 = -1; d1 <= 1; ++d1)
                    for (int d2 = -1; d2 <= 1; ++d2)
                        for (int d3 = (dd == 3 ? -1 : 0); d3 <= (dd == 3 ? 1 : 0); ++d3) {
                            const int r1 = l1 + d1, r2 = l2 + d2, r3 = l3 + d3;
                            if (r1 < 0 || r2 < 0 || r3 < 0 || r1 >= nn || r2 >= nn || (dd == 3 && r3 >= nn)) continue;
                            const int r = dd == 3 ? (r1 * nn + r2) * nn + r3 : r1 * nn + r2;
                            cand.push_back((int64_t)k * M + r);
                        }
            }
    }
    // every C-bar entry is a weighted mean of fine costs, all at most the cost
    // of the grid's diagonal; twice that covers the upward rounding, and the
    // solve checks each entry against it in its full scans (no pass of its own)
    const double diag_sq = (double)dim_of(pr) * (double)(pr.N - 1) * (double)(pr.N - 1);
    const double cb_bound = 2.0 * cost_of_sq(diag_sq, pr.p, false) + 1.0;
    st = network_simplex(M, M, Cb, mc, nc, sb, -1, &basis, nullptr, &cand, false, cb_bound);   // the plan only
    if (st) return st;
    double L_sum = 0.0;
    const int nnzb = (int)sb.col.size();
    std::vector<double> rowsum(M, 0.0), colsum(M, 0.0);
    for (int k = 0; k < M; ++k)
        for (int e = sb.rowptr[k]; e < sb.rowptr[k + 1]; ++e) {
            L_sum += sb.val[e] * Cb[(size_t)k * M + sb.col[e]];
            rowsum[k] += sb.val[e];
            colsum[sb.col[e]] += sb.val[e];
        }
    // non-negative terms: |fl(sum) - sum| <= gamma_(nnz+1) * sum; round up
    const double u = std::ldexp(1.0, -53);
    const double L_up = L_sum * (1.0 + 2.0 * (nnzb + 4) * u);
    // TV correction for the plan's marginal rounding errors (tiny)
    // |computed - exact| of each row sum is at most (degree + 2) u times it
    std::vector<int> rdeg(M, 0), cdeg(M, 0);
    for (int k = 0; k < M; ++k)
        for (int e = sb.rowptr[k]; e < sb.rowptr[k + 1]; ++e) { rdeg[k]++; cdeg[sb.col[e]]++; }
    double dm = 0.0, dn = 0.0;
    for (int k = 0; k < M; ++k) {
        dm += std::fabs(rowsum[k] - mc[k]) + (rdeg[k] + 3) * u * (rowsum[k] + mc[k]);
        dn += std::fabs(colsum[k] - nc[k]) + (cdeg[k] + 3) * u * (colsum[k] + nc[k]);
    }
    dm *= 1.0 + 4.0 * M * u;
    dn *= 1.0 + 4.0 * M * u;
    const double r = 0.5 * std::sqrt(2.0) * pr.N;   // radius of the grid (Sec. 3.4 remark)
    const double p = pr.p;
    const double tv = std::pow(2.0, 1.0 - 1.0 / p) * r * (std::pow(dm, 1.0 / p) + std::pow(dn, 1.0 / p));
    b->ubw_p[t] = L_up;
    b->ubw[t] = (std::pow(L_up, 1.0 / p) * (1.0 + 4 * u) + tv) * (1.0 + 4 * u);
    return QWB_OK;
}

constexpr int kCbarGroup = 8;   // pairs per C-bar copy group (one event each)

static int batch_solve(qwb_batch* b, int n_threads, cudaStream_t s) {
    // After a batched coarse pass the SumPool kernel's end is marked by an
    // event inside the captured graph: the coarse masses (all the C~ solves
    // need) are read as soon as it has passed, on a second stream, while the
    // C-bar kernels still run; C-bar comes back on the caller's stream in
    // groups, and a worker waits for its pair's group only before the C-bar
    // solve.  Otherwise everything is read after the whole coarse pass.
    const bool overlap = b->coarse_batched && b->ev_ok && !(b->flags & QWB_FLAG_NO_WEIGHTED);
    const int n_groups = (b->n + kCbarGroup - 1) / kCbarGroup;
    std::vector<PairOut> outs(b->n);
    if (overlap) {
        if (!b->aux) QWB_CUDA(cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking));
        while ((int)b->cb_ev.size() < n_groups) {
            cudaEvent_t e;
            QWB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            b->cb_ev.push_back(e);
        }
        QWB_CUDA(cudaStreamWaitEvent(b->aux, b->kev[1], 0));
        QWB_CUDA(cudaMemcpyAsync(outs.data(), b->outs_d, sizeof(PairOut) * b->n, cudaMemcpyDeviceToHost, b->aux));
        for (int t = 0; t < b->n; ++t) {
            const int M = b->Ms[t];
            const PairDev& P = b->pairs_h[t];
            QWB_CUDA(cudaMemcpyAsync(b->mu_c_h + b->mc_off[t], P.mu_c, sizeof(double) * M, cudaMemcpyDeviceToHost, b->aux));
            QWB_CUDA(cudaMemcpyAsync(b->nu_c_h + b->mc_off[t], P.nu_c, sizeof(double) * M, cudaMemcpyDeviceToHost, b->aux));
        }
        for (int g = 0; g < n_groups; ++g) {
            for (int t = g * kCbarGroup; t < std::min(b->n, (g + 1) * kCbarGroup); ++t) {
                const int M = b->Ms[t];
                QWB_CUDA(cudaMemcpyAsync(b->cbar_h + b->cbar_h_off[t], b->pairs_h[t].cbar,
                                         sizeof(double) * (size_t)M * M, cudaMemcpyDeviceToHost, s));
            }
            QWB_CUDA(cudaEventRecord(b->cb_ev[g], s));
        }
        QWB_CUDA(cudaStreamSynchronize(b->aux));
    } else {
        QWB_CUDA(cudaStreamSynchronize(s));
        QWB_CUDA(cudaMemcpy(outs.data(), b->outs_d, sizeof(PairOut) * b->n, cudaMemcpyDeviceToHost));
        for (int t = 0; t < b->n; ++t) {
            const int M = b->Ms[t];
            const PairDev& P = b->pairs_h[t];
            QWB_CUDA(cudaMemcpyAsync(b->mu_c_h + b->mc_off[t], P.mu_c, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
            QWB_CUDA(cudaMemcpyAsync(b->nu_c_h + b->mc_off[t], P.nu_c, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
            if (!(b->flags & QWB_FLAG_NO_WEIGHTED))
                QWB_CUDA(cudaMemcpyAsync(b->cbar_h + b->cbar_h_off[t], P.cbar, sizeof(double) * (size_t)M * M, cudaMemcpyDeviceToHost, s));
        }
        QWB_CUDA(cudaStreamSynchronize(s));
    }
    int first_bad = QWB_OK;
    for (int t = 0; t < b->n; ++t) {
        const PairOut& O = outs[t];
        b->status[t] = QWB_OK;
        if (O.bad_mu || O.bad_nu || !(std::fabs(O.mass_mu - 1.0) <= 1e-12) || !(std::fabs(O.mass_nu - 1.0) <= 1e-12)) {
            b->status[t] = QWB_ERR_MASS;
            if (!first_bad) first_bad = QWB_ERR_MASS;
        }
    }
    if (first_bad) {
        b->solved = false;
        if (overlap) QWB_CUDA(cudaStreamSynchronize(s));      // no copy left in flight
        return fail(first_bad, "measures must be finite, non-negative and of mass 1 (1e-12)");
    }
    std::function<int(int)> wait_cbar;
    if (overlap)
        wait_cbar = [b](int t) -> int {
            const cudaError_t e = cudaEventSynchronize(b->cb_ev[t / kCbarGroup]);
            return e == cudaSuccess ? QWB_OK : QWB_ERR_CUDA;
        };
    const auto t0 = std::chrono::steady_clock::now();
    int nt = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    nt = std::min(nt, b->n);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (;;) {
            const int t = next.fetch_add(1);
            if (t >= b->n) break;
            int st;
            try { st = solve_pair(b, t, wait_cbar); } catch (...) { st = QWB_ERR_OOM; }
            b->status[t] = st;
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < nt; ++i) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    b->t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (overlap) QWB_CUDA(cudaStreamSynchronize(s));          // every C-bar copy has landed
    for (int t = 0; t < b->n; ++t)
        if (b->status[t]) { b->solved = false; return fail(b->status[t], "exact coarse solve failed"); }
    // upload the plans (and nnz in the descriptors)
    QWB_CUDA(cudaMemcpyAsync(b->plan_d, b->plan_h, b->plan_bytes, cudaMemcpyHostToDevice, s));
    QWB_CUDA(cudaMemcpyAsync(b->pairs_d, b->pairs_h.data(), sizeof(PairDev) * b->n, cudaMemcpyHostToDevice, s));
    QWB_CUDA(cudaStreamSynchronize(s));
    b->solved = true;
    return QWB_OK;
}

static int batch_results(qwb_batch* b, qwb_result* out, cudaStream_t s) {
    if (!out) return fail(QWB_ERR_INVALID_ARG, "null results");
    QWB_CUDA(cudaStreamSynchronize(s));
    std::vector<PairOut> o(b->n);
    QWB_CUDA(cudaMemcpy(o.data(), b->outs_d, sizeof(PairOut) * b->n, cudaMemcpyDeviceToHost));
    int dev_err = 0;
    QWB_CUDA(cudaMemcpy(&dev_err, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    float tc = 0.f, tp = 0.f, td = 0.f;
    if (b->ev_ok) {
        if (cudaEventElapsedTime(&tc, b->ev[0], b->ev[1]) != cudaSuccess) tc = 0.f;
        if (cudaEventElapsedTime(&tp, b->ev[2], b->ev[3]) != cudaSuccess) tp = 0.f;
        if (cudaEventElapsedTime(&td, b->ev[3], b->ev[4]) != cudaSuccess) td = 0.f;
        cudaGetLastError();
    }
    for (int t = 0; t < b->n; ++t) {
        qwb_result& r = out[t];
        std::memset(&r, 0, sizeof(r));
        r.ub_weighted = b->ubw[t];
        r.ub_weighted_p = b->ubw_p[t];
        r.ub_primal = o[t].ub_primal;
        r.lb = o[t].lb;
        r.lb_p = o[t].lb_p;
        r.w_hat_p = o[t].w_hat_p;
        r.delta_mu = o[t].delta_mu;
        r.delta_nu = o[t].delta_nu;
        r.ipf_residual = o[t].ipf_residual;
        r.ipf_sweeps_done = o[t].sweeps_done;
        r.lb_mincost = b->lbmin[t];
        if (b->flags & QWB_FLAG_NO_PRIMAL) { r.ub_primal = HUGE_VAL; r.w_hat_p = HUGE_VAL; }
        if (b->flags & QWB_FLAG_NO_DUAL) { r.lb = 0.0; r.lb_p = -HUGE_VAL; }
        r.t_coarse_cost_ms = tc; r.t_solve_ms = b->t_solve_ms; r.t_primal_ms = tp; r.t_dual_ms = td;
        r.status = dev_err ? QWB_ERR_TIMEOUT : b->status[t];
        if (r.status == QWB_OK && (b->flags & QWB_FLAG_VERIFY) && !(b->flags & QWB_FLAG_NO_DUAL) && o[t].verify_bad)
            r.status = QWB_ERR_VERIFY;
    }
    if (dev_err) return fail(QWB_ERR_TIMEOUT, "a bounded device wait timed out (bulk-copy IPF sweeps)");
    return QWB_OK;
}

// --------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------
extern "C" {

int qwb_ctx_create(qwb_ctx** out, int device) {
    if (!out) return fail(QWB_ERR_INVALID_ARG, "qwb_ctx_create: null out");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(QWB_ERR_CUDA, "no such CUDA device");
    QWB_CUDA(cudaSetDevice(device));
    qwb_ctx* c = new qwb_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (const char* v = std::getenv("QWB_AUTOTUNE")) c->autotune = std::strcmp(v, "0") != 0;
    if (const char* v = std::getenv("QWB_AUTOTUNE_CACHE")) c->tune_cache = v;
    tune_cache_load(c);
    *out = c;
    return QWB_OK;
}

void qwb_ctx_destroy(qwb_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto* b : ctx->single_cache) batch_free(b);
    for (auto& t : ctx->tables) { cudaFree(t.lo); cudaFree(t.hi); cudaFree(t.lo_refl); }
    delete ctx;
}

int qwb_batch_create(qwb_ctx* ctx, int32_t n_pairs, const qwb_problem* probs_h, int32_t ipf_sweeps,
                     int32_t flags, qwb_prec prec, qwb_batch** out) {
    if (!ctx || !out) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_create: null argument");
    if (flags & ~127) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_create: unknown flags");
    if (const char* v = std::getenv("QWB_VERIFY"))          // the verify mode for every batch
        if (std::strcmp(v, "0") != 0) flags |= QWB_FLAG_VERIFY;
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    return batch_build(ctx, n_pairs, probs_h, ipf_sweeps, flags, prec, out);
}

void qwb_batch_destroy(qwb_batch* batch) {
    if (!batch) return;
    cudaSetDevice(batch->ctx->device);
    cudaDeviceSynchronize();
    batch_free(batch);
}

int qwb_batch_coarse(qwb_batch* b, const double* const* mu_d, const double* const* nu_d,
                     int32_t batched, void* stream) {
    if (!b) return fail(QWB_ERR_INVALID_ARG, "null batch");
    const NvtxRange range("qwb coarse pass (SumPool, C-bar)");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    int st = batch_set_measures(b, mu_d, nu_d);
    if (st) return st;
    if (b->ev_ok) QWB_CUDA(cudaEventRecord(b->ev[0], s));
    st = run_pass(b, 0, batched != 0, s);
    if (st) return st;
    b->coarse_batched = batched != 0;
    if (b->ev_ok) QWB_CUDA(cudaEventRecord(b->ev[1], s));
    return QWB_OK;
}

int qwb_batch_solve(qwb_batch* b, int32_t n_threads, void* stream) {
    const NvtxRange range("qwb exact coarse solves");
    if (!b) return fail(QWB_ERR_INVALID_ARG, "null batch");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    return batch_solve(b, n_threads, (cudaStream_t)stream);
}

int qwb_batch_fine(qwb_batch* b, const double* const* mu_d, const double* const* nu_d,
                   int32_t batched, void* stream) {
    const NvtxRange range("qwb fine passes (IPF and upper bound, c-transforms and lower bound)");
    if (!b) return fail(QWB_ERR_INVALID_ARG, "null batch");
    if (!b->solved) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_fine needs a completed qwb_batch_solve");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    int st = batch_set_measures(b, mu_d, nu_d);
    if (st) return st;
    if (b->ev_ok) QWB_CUDA(cudaEventRecord(b->ev[2], s));
    if (batched) {
        st = run_pass(b, 1, true, s);
        if (st) return st;
        if (b->ev_ok) { QWB_CUDA(cudaEventRecord(b->ev[3], s)); QWB_CUDA(cudaEventRecord(b->ev[4], s)); }
        return QWB_OK;
    }
    st = enqueue_fine(b, false, s);
    if (st) return st;
    if (b->ev_ok) { QWB_CUDA(cudaEventRecord(b->ev[3], s)); QWB_CUDA(cudaEventRecord(b->ev[4], s)); }
    return QWB_OK;
}

int qwb_batch_results(qwb_batch* b, qwb_result* out_h, void* stream) {
    if (!b) return fail(QWB_ERR_INVALID_ARG, "null batch");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    return batch_results(b, out_h, (cudaStream_t)stream);
}

int qwb_batch_kernel_times(qwb_batch* b, double* ms_out, int32_t n) {
    if (!b || !ms_out || n < 0) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_kernel_times: bad argument");
    if (!b->ev_ok) return fail(QWB_ERR_CUDA, "no timing events");
    const int pairs[10][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {7, 8}, {8, 9}, {3, 10}, {10, 4}};
    for (int i = 0; i < n && i < 10; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->kev[pairs[i][0]], b->kev[pairs[i][1]]) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.f;
        }
        ms_out[i] = ms;
    }
    return QWB_OK;
}

int qwb_batch_tuning(qwb_batch* b, char* json_out, int32_t capacity) {
    if (!b || !json_out || capacity <= 0) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_tuning: bad argument");
    std::ostringstream o;
    o << "{\"key\": \"" << (b->tune ? b->tune->key : "") << "\", \"ctransform\": {\"R\": " << b->ct_cfg_b.R
      << ", \"TC\": " << b->ct_cfg_b.TC << ", \"packed\": " << b->ct_cfg_b.packed
      << ", \"candidates_ms\": " << (b->tune && !b->tune->ct_report.empty() ? b->tune->ct_report : "{}")
      << "}, \"cbar\": {\"variant\": \"" << cbar_variant_name(b->cbar_variant) << "\""
      << ", \"candidates_ms\": " << (b->tune && !b->tune->cbar_report.empty() ? b->tune->cbar_report : "{}")
      << "}, \"ipf\": {\"cluster\": " << b->ipf_C
      << ", \"candidates_ms\": " << (b->tune && !b->tune->ipf_report.empty() ? b->tune->ipf_report : "{}")
      << "}, \"upscale_kernel\": {\"cluster\": " << b->upk_C << ", \"threads\": "
      << (b->upk_C > 0 ? (b->upk_var == 0 ? 256 : b->upk_var == 1 ? 128 : 64) : (b->f64 ? 512 : 1024))
      << ", \"candidates_ms\": "
      << (b->upk_req ? std::string("\"set\"")
                            : b->tune && !b->tune->upk_report.empty() ? b->tune->upk_report : std::string("{}"))
      << "}, \"enabled\": " << (b->ctx->autotune ? "true" : "false") << "}";
    const std::string str = o.str();
    if ((int)str.size() + 1 > capacity) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_tuning: buffer too small");
    std::memcpy(json_out, str.c_str(), str.size() + 1);
    return QWB_OK;
}

int qwb_batch_potentials(qwb_batch* b, int32_t pair, double* f_d, double* g_d, void* stream) {
    if (!b || pair < 0 || pair >= b->n) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_potentials: bad pair");
    if (b->flags & QWB_FLAG_NO_DUAL) return fail(QWB_ERR_INVALID_ARG, "the batch skipped the dual pass");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int m = ipow(b->probs[pair].N, dim_of(b->probs[pair]));
    int st;
    const PairDev& P = b->pairs_h[pair];
    if (P.f_out) {   // both sides ran: the lower-bound kernel kept the better pair
        if (f_d) QWB_CUDA(cudaMemcpyAsync(f_d, P.f_out, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
        if (g_d) QWB_CUDA(cudaMemcpyAsync(g_d, P.g_out, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
        return QWB_OK;
    }
    if (f_d && (st = launch_from_work(P.f, f_d, m, b->f64, s))) return st;
    if (g_d && (st = launch_from_work(P.g, g_d, m, b->f64, s))) return st;
    return QWB_OK;
}

int qwb_batch_coarse_plan(qwb_batch* b, int32_t pair, int32_t* rowptr_h, int32_t* col_h, double* val_h,
                          int32_t cap, int32_t* nnz_out) {
    if (!b || pair < 0 || pair >= b->n || !nnz_out)
        return fail(QWB_ERR_INVALID_ARG, "qwb_batch_coarse_plan: bad arguments");
    if (!b->solved) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_coarse_plan: the batch has not been solved");
    const int M = b->Ms[pair];
    const int nnz = b->pairs_h[pair].nnz;
    *nnz_out = nnz;
    if ((col_h || val_h) && cap < nnz) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_coarse_plan: cap < nnz");
    const PlanLayout L = plan_layout(M);
    const char* ph = b->plan_h + b->plan_off[pair];
    if (rowptr_h) std::memcpy(rowptr_h, ph + L.rowptr, sizeof(int) * (M + 1));
    if (col_h) std::memcpy(col_h, ph + L.col, sizeof(int) * nnz);
    if (val_h) std::memcpy(val_h, ph + L.val, sizeof(double) * nnz);
    return QWB_OK;
}

int qwb_batch_coarse_potentials(qwb_batch* b, int32_t pair, double* f_h, double* g_h) {
    if (!b || pair < 0 || pair >= b->n)
        return fail(QWB_ERR_INVALID_ARG, "qwb_batch_coarse_potentials: bad pair");
    if (!b->solved) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_coarse_potentials: the batch has not been solved");
    const int M = b->Ms[pair];
    const PlanLayout L = plan_layout(M);
    const char* ph = b->plan_h + b->plan_off[pair];
    if (f_h) std::memcpy(f_h, ph + L.fco, sizeof(double) * M);
    if (g_h) std::memcpy(g_h, ph + L.gco, sizeof(double) * M);
    return QWB_OK;
}

int qwb_batch_set_ipf_cluster(qwb_batch* b, int32_t C) {
    const int Cs = C & 31, form = C & ~31;
    if (!b || (Cs != 0 && Cs != 2 && Cs != 3 && Cs != 4 && Cs != 8 && Cs != 16) ||
        (form != 0 && form != QWB_IPF_BULK && form != QWB_IPF_WIDE) ||
        (form != 0 && Cs == 0) || (form == QWB_IPF_BULK && Cs == 3))
        return fail(QWB_ERR_INVALID_ARG,
                    "qwb_batch_set_ipf_cluster: C must be 0, 2, 3, 4, 8 or 16, the others than 0 optionally with "
                    "QWB_IPF_WIDE, and 2, 4, 8, 16 with QWB_IPF_BULK");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    QWB_CUDA(cudaDeviceSynchronize());
    // captured fine passes hold the previous launch configuration
    std::vector<GraphEntry> keep;
    for (auto& g : b->graphs) {
        if (g.kind == 1) cudaGraphExecDestroy(g.exec);
        else keep.push_back(g);
    }
    b->graphs.swap(keep);
    if (b->tune) { b->tune->ipf_done = true; b->tune->ipf_C = C; b->tune->ipf_report = "\"set\""; }
    return apply_ipf_choice(b, C);
}

int qwb_batch_set_upscale_cluster(qwb_batch* b, int32_t C, int32_t threads) {
    if (!b || (C != -1 && C != 0 && C != 1 && C != 2 && C != 4 && C != 8) ||
        (C > 0 && threads != 256 && threads != 128 && threads != 64))
        return fail(QWB_ERR_INVALID_ARG,
                    "qwb_batch_set_upscale_cluster: C must be -1, 0, 1, 2, 4 or 8 and threads 256, 128 or 64");
    if (C != 0 && b->n_upk && !b->upk_kappa)
        return fail(QWB_ERR_UNSUPPORTED,
                    "the cluster form needs FP32 and one block side (2, 4 or 8) for every pair with a kernel K");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    QWB_CUDA(cudaDeviceSynchronize());
    std::vector<GraphEntry> keep;                // captured fine passes hold the previous form
    for (auto& g : b->graphs) {
        if (g.kind == 1) cudaGraphExecDestroy(g.exec);
        else keep.push_back(g);
    }
    b->graphs.swap(keep);
    const int var = C <= 0 ? 0 : threads == 256 ? 0 : threads == 128 ? 1 : 2;
    b->upk_req = true;
    b->upk_req_C = C;
    b->upk_req_var = var;
    b->upk_C = b->upk_kappa ? C : 0;
    b->upk_var = var;
    return QWB_OK;
}

int qwb_batch_set_upscale_kernel(qwb_batch* b, int32_t kappa, const double* K_d) {
    if (!b || kappa < 1) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_set_upscale_kernel: bad arguments");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    QWB_CUDA(cudaDeviceSynchronize());
    const int kk = kappa * kappa;
    std::vector<double> Kh;
    if (K_d) {
        if (kappa > 8) return fail(QWB_ERR_UNSUPPORTED, "a general upscaling kernel needs kappa <= 8");
        Kh.resize((size_t)kk * kk);
        QWB_CUDA(cudaMemcpy(Kh.data(), K_d, sizeof(double) * kk * kk, cudaMemcpyDeviceToHost));
        for (double v : Kh)
            if (!(v > 0.0) || !std::isfinite(v))
                return fail(QWB_ERR_INVALID_ARG, "upscaling kernel entries must be positive and finite");
    }
    // captured fine passes hold the previous pair lists
    std::vector<GraphEntry> keep;
    for (auto& g : b->graphs) {
        if (g.kind == 1) cudaGraphExecDestroy(g.exec);
        else keep.push_back(g);
    }
    b->graphs.swap(keep);
    auto it = std::find_if(b->upk.begin(), b->upk.end(), [&](const auto& e) { return e.first == kappa; });
    if (it != b->upk.end()) b->upk.erase(it);
    if (K_d) b->upk.emplace_back(kappa, std::move(Kh));
    // lay out: per kernel K (FP64) and K (pass type); per K pair the KB and
    // evaluation scratches; the primal pair lists
    const size_t tsz = b->f64 ? 8 : 4;
    std::vector<size_t> k_off(b->upk.size());
    size_t off = 0;
    for (size_t q = 0; q < b->upk.size(); ++q) {
        const size_t e = b->upk[q].second.size();
        k_off[q] = off;
        off = align_up(off + e * (8 + tsz));
    }
    std::vector<int> which(b->n, -1);
    std::vector<size_t> s_off(b->n, 0);
    for (int t = 0; t < b->n; ++t) {
        if (dim_of(b->probs[t]) != 2) continue;
        for (size_t q = 0; q < b->upk.size(); ++q)
            if (b->upk[q].first == b->probs[t].kappa) which[t] = (int)q;
        if (which[t] < 0) continue;
        const size_t m = (size_t)b->probs[t].N * b->probs[t].N;
        s_off[t] = off;
        off = align_up(off + align_up(2 * m * tsz) + 16 * m);
    }
    const size_t ids_off = off;
    off = align_up(off + sizeof(int) * b->n);
    if (b->upk_mem) { cudaFree(b->upk_mem); b->upk_mem = nullptr; }
    if (cudaMalloc(&b->upk_mem, off) != cudaSuccess) return fail(QWB_ERR_OOM, "upscaling kernel scratch");
    for (size_t q = 0; q < b->upk.size(); ++q) {
        const auto& K = b->upk[q].second;
        std::vector<char> host(K.size() * (8 + tsz));
        std::memcpy(host.data(), K.data(), 8 * K.size());
        for (size_t t = 0; t < K.size(); ++t) {
            if (b->f64) ((double*)(host.data() + 8 * K.size()))[t] = K[t];
            else ((float*)(host.data() + 8 * K.size()))[t] = (float)K[t];
        }
        QWB_CUDA(cudaMemcpy(b->upk_mem + k_off[q], host.data(), host.size(), cudaMemcpyHostToDevice));
    }
    std::vector<int> uni, kp;
    b->upk_kappa_max = 0;
    b->upk_M_max = 0;
    b->upk_m_max = 0;
    b->upk_all4 = true;
    for (int t = 0; t < b->n; ++t) {
        PairDev& P = b->pairs_h[t];
        b->upk_on[t] = which[t] >= 0;
        if (which[t] < 0) {
            P.upK = nullptr; P.upK_t = nullptr; P.kb_t = nullptr; P.kscratch = nullptr;
            uni.push_back(t);
            continue;
        }
        const size_t kbytes = b->upk[which[t]].second.size();
        const size_t m = (size_t)b->probs[t].N * b->probs[t].N;
        P.upK = (const double*)(b->upk_mem + k_off[which[t]]);
        P.upK_t = b->upk_mem + k_off[which[t]] + 8 * kbytes;
        P.kb_t = b->upk_mem + s_off[t];
        P.kscratch = (double*)(b->upk_mem + s_off[t] + align_up(2 * m * tsz));
        kp.push_back(t);
        b->upk_kappa_max = std::max(b->upk_kappa_max, b->probs[t].kappa);
        b->upk_M_max = std::max(b->upk_M_max, b->Ms[t]);
        b->upk_m_max = std::max(b->upk_m_max, b->probs[t].N * b->probs[t].N);
        b->upk_all4 = b->upk_all4 && b->probs[t].kappa == 4;
    }
    b->n_uni = (int)uni.size();
    b->n_upk = (int)kp.size();
    // the cluster form needs FP32 and one kappa in {2, 4, 8} for every K pair
    b->upk_kappa = 0;
    b->upk_n_max = 0;
    if (!b->f64 && !kp.empty()) {
        const int k0 = b->probs[kp[0]].kappa;
        bool same = k0 == 2 || k0 == 4 || k0 == 8;
        for (int t : kp) {
            same = same && b->probs[t].kappa == k0;
            b->upk_n_max = std::max(b->upk_n_max, b->probs[t].N / k0);
        }
        if (same) b->upk_kappa = k0;
    }
    if (b->upk_req) { b->upk_C = b->upk_req_C; b->upk_var = b->upk_req_var; }
    else if (b->tune && b->tune->upk_done) { b->upk_C = b->tune->upk_C; b->upk_var = b->tune->upk_var; }
    if (!b->upk_kappa) b->upk_C = 0;
    uni.insert(uni.end(), kp.begin(), kp.end());
    b->prim_ids_d = (int*)(b->upk_mem + ids_off);
    QWB_CUDA(cudaMemcpy(b->prim_ids_d, uni.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
    // the cluster sweeps keep the uniform pairs only
    const std::vector<int> ipf_ids = build_ipf_groups(b);
    if (!ipf_ids.empty())
        QWB_CUDA(cudaMemcpy(b->ipf_ids_d, ipf_ids.data(), sizeof(int) * ipf_ids.size(), cudaMemcpyHostToDevice));
    return apply_ipf_choice(b, b->ipf_C);
}

int qwb_batch_fine_scalings(qwb_batch* b, int32_t pair, double* a_d, double* b_d, void* stream) {
    if (!b || pair < 0 || pair >= b->n) return fail(QWB_ERR_INVALID_ARG, "qwb_batch_fine_scalings: bad pair");
    if (b->flags & QWB_FLAG_NO_PRIMAL) return fail(QWB_ERR_INVALID_ARG, "the batch skipped the primal pass");
    QWB_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int m = ipow(b->probs[pair].N, dim_of(b->probs[pair]));
    const PairDev& P = b->pairs_h[pair];
    int st;
    if (a_d && (st = launch_from_work(P.a, a_d, m, b->f64, s))) return st;
    if (b_d && (st = launch_from_work(P.b, b_d, m, b->f64, s))) return st;
    return QWB_OK;
}

int qwb_bounds(qwb_ctx* ctx, int32_t n_pairs, const qwb_problem* probs_h, const double* const* mu_d,
               const double* const* nu_d, int32_t ipf_sweeps, int32_t flags, qwb_result* out_h,
               qwb_prec prec, int32_t batched, int32_t n_threads, void* stream) {
    if (!ctx || !out_h) return fail(QWB_ERR_INVALID_ARG, "qwb_bounds: null argument");
    qwb_batch* b = nullptr;
    int st = qwb_batch_create(ctx, n_pairs, probs_h, ipf_sweeps, flags, prec, &b);
    if (st) return st;
    st = qwb_batch_coarse(b, mu_d, nu_d, batched, stream);
    if (!st) st = qwb_batch_solve(b, n_threads, stream);
    if (!st) st = qwb_batch_fine(b, mu_d, nu_d, batched, stream);
    if (!st) st = qwb_batch_results(b, out_h, stream);
    if (st && st != QWB_OK) {
        for (int t = 0; t < n_pairs; ++t) out_h[t].status = b->status.size() > (size_t)t && b->status[t] ? b->status[t] : st;
    }
    qwb_batch_destroy(b);
    return st;
}

}  // extern "C"

// ---- standalone pass entry points ----------------------------------------
static int single_batch(qwb_ctx* ctx, const qwb_problem* prob, int sweeps, qwb_prec prec,
                        qwb_batch** out, int flags = 0) {
    for (auto* b : ctx->single_cache)
        if (b->probs[0].N == prob->N && b->probs[0].kappa == prob->kappa && b->probs[0].p == prob->p &&
            dim_of(b->probs[0]) == dim_of(*prob) && b->f64 == (prec == QWB_PREC_F64) && b->flags == flags) {
            b->sweeps = sweeps;
            b->pairs_h[0].sweeps = sweeps;
            *out = b;
            return QWB_OK;
        }
    qwb_batch* b = nullptr;
    int st = batch_build(ctx, 1, prob, sweeps, flags, prec, &b);
    if (st) return st;
    if (ctx->single_cache.size() >= 8) { batch_free(ctx->single_cache.front()); ctx->single_cache.erase(ctx->single_cache.begin()); }
    ctx->single_cache.push_back(b);
    *out = b;
    return QWB_OK;
}

// Upload the descriptor of a single-pair batch with the given pointers.
static int single_upload(qwb_batch* b, cudaStream_t s) {
    b->cur_mu.clear(); b->cur_nu.clear();
    QWB_CUDA(cudaMemcpyAsync(b->pairs_d, b->pairs_h.data(), sizeof(PairDev), cudaMemcpyHostToDevice, s));
    return QWB_OK;
}

static int single_validate(qwb_batch* b, cudaStream_t s) {
    int st = launch_prepare(b->pairs_d, b->outs_d, b->prep_items_d, b->n_prep, b->f64, s);
    if (st) return st;
    PairOut o;
    QWB_CUDA(cudaMemcpyAsync(&o, b->outs_d, sizeof(PairOut), cudaMemcpyDeviceToHost, s));
    QWB_CUDA(cudaStreamSynchronize(s));
    if (o.bad_mu || o.bad_nu || !(std::fabs(o.mass_mu - 1.0) <= 1e-12) || !(std::fabs(o.mass_nu - 1.0) <= 1e-12))
        return fail(QWB_ERR_MASS, "measures must be finite, non-negative and of mass 1 (1e-12)");
    return QWB_OK;
}

extern "C" {

int qwb_coarse_cost(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d, const double* nu_d,
                    double* cbar_d, double* mu_coarse_d, double* nu_coarse_d, qwb_prec prec,
                    void* stream) {
    if (!ctx || !mu_d || !nu_d || !cbar_d) return fail(QWB_ERR_INVALID_ARG, "qwb_coarse_cost: null argument");
    int st = check_problem(prob);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, prob, 1, prec, &b))) return st;
    apply_cbar_env(b);
    PairDev& P = b->pairs_h[0];
    double* own_cbar = P.cbar;
    P.mu = mu_d; P.nu = nu_d; P.cbar = cbar_d;
    if ((st = single_upload(b, s))) { P.cbar = own_cbar; return st; }
    P.cbar = own_cbar;
    QWB_CUDA(cudaMemsetAsync(b->outs_d, 0, sizeof(PairOut), s));
    if ((st = single_validate(b, s))) return st;
    const int kc = (prob->kappa == 1 || prob->kappa == 2 || prob->kappa == 4 || b->cbar_group[0] == 8)
                       ? prob->kappa : -prob->kappa;
    if (dim_of(*prob) == 3) {
        if ((st = launch_cbar3(b->pairs_d, b->cbar3_items_d, b->n_cbar3, b->f64, s))) return st;
    } else if ((st = launch_cbar(b->pairs_d, b->cbar_items_d, b->n_cbar, kc, prob->N / prob->kappa, prob->N,
                                 b->f64, s, pair_cbar_variant(b, 0)))) {
        return st;
    }
    const size_t M = b->Ms[0];
    if (mu_coarse_d) QWB_CUDA(cudaMemcpyAsync(mu_coarse_d, P.mu_c, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    if (nu_coarse_d) QWB_CUDA(cudaMemcpyAsync(nu_coarse_d, P.nu_c, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    QWB_CUDA(cudaStreamSynchronize(s));   // the cached descriptor is reused by the next call
    return QWB_OK;
}

int qwb_coarse_cost_separable(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d, const double* nu_d,
                              double* cbar_d, void* stream) {
    if (!ctx || !mu_d || !nu_d || !cbar_d)
        return fail(QWB_ERR_INVALID_ARG, "qwb_coarse_cost_separable: null argument");
    int st = check_problem(prob);
    if (st) return st;
    if (prob->p != 2.0 || dim_of(*prob) != 2 || (prob->kappa != 4 && prob->kappa != 8))
        return fail(QWB_ERR_UNSUPPORTED, "qwb_coarse_cost_separable: needs p = 2, d = 2 and kappa 4 or 8");
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, prob, 1, QWB_PREC_MIXED, &b, QWB_FLAG_SEPARABLE))) return st;
    if (b->cbar_group[0] < 12)
        return fail(QWB_ERR_UNSUPPORTED, "qwb_coarse_cost_separable: the coarse side is too large");
    PairDev& P = b->pairs_h[0];
    double* own_cbar = P.cbar;
    P.mu = mu_d; P.nu = nu_d; P.cbar = cbar_d;
    if ((st = single_upload(b, s))) { P.cbar = own_cbar; return st; }
    P.cbar = own_cbar;
    QWB_CUDA(cudaMemsetAsync(b->outs_d, 0, sizeof(PairOut), s));
    if ((st = single_validate(b, s))) return st;
    if ((st = launch_cbar_sep(b->pairs_d, b->cbar_items_d, b->n_cbar, prob->kappa, prob->N / prob->kappa, s)))
        return st;
    QWB_CUDA(cudaStreamSynchronize(s));   // the cached descriptor is reused by the next call
    return QWB_OK;
}

}  // extern "C"

// The primal pass of one pair: the uniform kernel when K_d is null, else the
// general kernel K_d ((kappa^2)^2 FP64 on the device, d = 2, kappa <= 8).
static int primal_single(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d, const double* nu_d,
                         const int32_t* pi_rowptr_d, const int32_t* pi_col_d, const double* pi_val_d,
                         int32_t pi_nnz, int32_t sweeps, const double* K_d, double* a_d, double* b_d,
                         qwb_result* out_h, qwb_prec prec, void* stream) {
    if (!ctx || !mu_d || !nu_d || !pi_rowptr_d || !pi_col_d || !pi_val_d || !out_h)
        return fail(QWB_ERR_INVALID_ARG, "qwb_primal_upscale_ipf: null argument");
    int st = check_problem(prob);
    if (st) return st;
    if (sweeps < 1) return fail(QWB_ERR_INVALID_ARG, "sweeps must be >= 1");
    const int kk = prob->kappa * prob->kappa;
    std::vector<double> Kh;
    if (K_d) {
        if (dim_of(*prob) != 2 || prob->kappa > 8)
            return fail(QWB_ERR_UNSUPPORTED, "a general upscaling kernel needs d = 2 and kappa <= 8");
        Kh.resize((size_t)kk * kk);
        QWB_CUDA(cudaMemcpy(Kh.data(), K_d, sizeof(double) * kk * kk, cudaMemcpyDeviceToHost));
        for (double v : Kh)
            if (!(v > 0.0) || !std::isfinite(v))
                return fail(QWB_ERR_INVALID_ARG, "upscaling kernel entries must be positive and finite");
    }
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, prob, sweeps, prec, &b))) return st;
    const int M = b->Ms[0];
    if (pi_nnz < 0 || (int64_t)pi_nnz > (int64_t)M * M) return fail(QWB_ERR_INVALID_ARG, "plan has more than M^2 entries");
    // the plan: read the CSR, transpose it on the host, stage both forms
    std::vector<int> rowptr(M + 1), col(pi_nnz);
    std::vector<double> val(pi_nnz);
    QWB_CUDA(cudaMemcpy(rowptr.data(), pi_rowptr_d, sizeof(int) * (M + 1), cudaMemcpyDeviceToHost));
    if (rowptr[0] != 0 || rowptr[M] != pi_nnz) return fail(QWB_ERR_INVALID_ARG, "plan rowptr inconsistent with nnz");
    if (pi_nnz) {
        QWB_CUDA(cudaMemcpy(col.data(), pi_col_d, sizeof(int) * pi_nnz, cudaMemcpyDeviceToHost));
        QWB_CUDA(cudaMemcpy(val.data(), pi_val_d, sizeof(double) * pi_nnz, cudaMemcpyDeviceToHost));
    }
    for (int k = 0; k < M; ++k) if (rowptr[k + 1] < rowptr[k]) return fail(QWB_ERR_INVALID_ARG, "plan rowptr not monotone");
    for (int e = 0; e < pi_nnz; ++e)
        if (col[e] < 0 || col[e] >= M || !(val[e] >= 0.0) || !std::isfinite(val[e]))
            return fail(QWB_ERR_INVALID_ARG, "plan entry out of range");
    // the batch's staging holds 2M entries (a basic plan); larger plans (any
    // optimal coupling may be passed) get a temporary staging area
    const PlanLayout L = plan_layout(M, pi_nnz);
    char* ph = b->plan_h;
    char* pd = b->plan_d;
    char* tmp_h = nullptr;
    char* tmp_d = nullptr;
    if (L.total > b->plan_bytes) {
        if (cudaMallocHost(&tmp_h, L.total) != cudaSuccess) return fail(QWB_ERR_OOM, "plan staging");
        if (cudaMalloc(&tmp_d, L.total) != cudaSuccess) { cudaFreeHost(tmp_h); return fail(QWB_ERR_OOM, "plan staging"); }
        ph = tmp_h; pd = tmp_d;
    }
    struct Release {
        char *h, *d;
        ~Release() { if (h) cudaFreeHost(h); if (d) cudaFree(d); }
    } release{tmp_h, tmp_d};
    std::memcpy(ph + L.rowptr, rowptr.data(), sizeof(int) * (M + 1));
    std::memcpy(ph + L.col, col.data(), sizeof(int) * pi_nnz);
    std::memcpy(ph + L.val, val.data(), sizeof(double) * pi_nnz);
    std::vector<int> cnt(M + 1, 0);
    for (int e = 0; e < pi_nnz; ++e) cnt[col[e] + 1]++;
    for (int l = 0; l < M; ++l) cnt[l + 1] += cnt[l];
    std::memcpy(ph + L.colptr, cnt.data(), sizeof(int) * (M + 1));
    std::vector<int> cur(cnt.begin(), cnt.end() - 1);
    for (int k = 0; k < M; ++k)
        for (int e = rowptr[k]; e < rowptr[k + 1]; ++e) {
            const int pos = cur[col[e]]++;
            ((int*)(ph + L.rowidx))[pos] = k;
            ((double*)(ph + L.valc))[pos] = val[e];
        }
    stage_typed_values(ph, L, pi_nnz, b->f64);
    QWB_CUDA(cudaMemcpyAsync(pd, ph, L.total, cudaMemcpyHostToDevice, s));
    // general kernel: K in FP64 and in the pass type, the sweep and evaluation scratches
    char* kbuf = nullptr;
    const size_t m_pts = (size_t)prob->N * prob->N;
    const size_t tsz = b->f64 ? 8 : 4;
    // [K FP64 | K pass type | KB, KA (2 m_pts, pass type) | evaluation scratch (2 m_pts FP64)]
    const size_t k64_off = 0, kt_off = 8 * (size_t)kk * kk, kb_off = kt_off + 8 * (size_t)kk * kk,
                 ks_off = kb_off + 2 * tsz * m_pts, k_total = ks_off + 16 * m_pts;
    struct KRelease {
        char* d;
        ~KRelease() { if (d) cudaFree(d); }
    } krelease{nullptr};
    if (K_d) {
        if (cudaMalloc(&kbuf, k_total) != cudaSuccess) return fail(QWB_ERR_OOM, "kernel scratch");
        krelease.d = kbuf;
        std::vector<char> kt(tsz * kk * kk);
        for (int t = 0; t < kk * kk; ++t) {
            if (b->f64) ((double*)kt.data())[t] = Kh[t];
            else ((float*)kt.data())[t] = (float)Kh[t];
        }
        QWB_CUDA(cudaMemcpyAsync(kbuf + k64_off, K_d, sizeof(double) * kk * kk, cudaMemcpyDeviceToDevice, s));
        QWB_CUDA(cudaMemcpyAsync(kbuf + kt_off, kt.data(), kt.size(), cudaMemcpyHostToDevice, s));
    }
    PairDev& P = b->pairs_h[0];
    const PairDev saved = P;
    P.mu = mu_d; P.nu = nu_d; P.nnz = pi_nnz; P.sweeps = sweeps; P.a_out = a_d; P.b_out = b_d;
    if (K_d) {
        P.upK = (const double*)(kbuf + k64_off); P.upK_t = kbuf + kt_off;
        P.kb_t = kbuf + kb_off; P.kscratch = (double*)(kbuf + ks_off);
    }
    P.rowptr = (int*)(pd + L.rowptr); P.colidx = (int*)(pd + L.col); P.val = (double*)(pd + L.val);
    P.colptr = (int*)(pd + L.colptr); P.rowidx = (int*)(pd + L.rowidx); P.valc = (double*)(pd + L.valc);
    P.val_t = pd + L.val_t; P.valc_t = pd + L.valc_t; P.supp_num = pd + L.supp;
    st = single_upload(b, s);
    {   // the cached descriptor keeps the batch's own buffers
        const PairDev cur = P;
        P = saved;
        P.mu = cur.mu; P.nu = cur.nu; P.sweeps = cur.sweeps;
    }
    if (st) return st;
    QWB_CUDA(cudaMemsetAsync(b->outs_d, 0, sizeof(PairOut), s));
    if ((st = single_validate(b, s))) return st;
    if (K_d) {
        if ((st = launch_primalk(b->pairs_d, b->outs_d, b->pair_ids_d, 1, prob->kappa, M, pi_nnz,
                                      prob->N * prob->N, prob->kappa == 4,
                                      b->f64, s))) return st;
    } else {
        if ((st = launch_support_num(b->pairs_d, b->pair_ids_d, 1, pi_nnz, b->f64, s))) return st;
        if ((st = launch_primal(b->pairs_d, b->outs_d, b->pair_ids_d, 1, M, pi_nnz, b->f64, s))) return st;
    }
    PairOut o;
    QWB_CUDA(cudaMemcpyAsync(&o, b->outs_d, sizeof(PairOut), cudaMemcpyDeviceToHost, s));
    QWB_CUDA(cudaStreamSynchronize(s));
    std::memset(out_h, 0, sizeof(*out_h));
    out_h->ub_primal = o.ub_primal; out_h->w_hat_p = o.w_hat_p; out_h->delta_mu = o.delta_mu;
    out_h->delta_nu = o.delta_nu; out_h->ipf_residual = o.ipf_residual; out_h->ipf_sweeps_done = o.sweeps_done;
    return QWB_OK;
}

extern "C" {

int qwb_primal_upscale_ipf(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                           const double* nu_d, const int32_t* pi_rowptr_d, const int32_t* pi_col_d,
                           const double* pi_val_d, int32_t pi_nnz, int32_t sweeps, double* a_d,
                           double* b_d, qwb_result* out_h, qwb_prec prec, void* stream) {
    return primal_single(ctx, prob, mu_d, nu_d, pi_rowptr_d, pi_col_d, pi_val_d, pi_nnz, sweeps, nullptr,
                         a_d, b_d, out_h, prec, stream);
}

int qwb_primal_upscale_ipf_kernel(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                                  const double* nu_d, const int32_t* pi_rowptr_d, const int32_t* pi_col_d,
                                  const double* pi_val_d, int32_t pi_nnz, const double* K_d, int32_t sweeps,
                                  double* a_d, double* b_d, qwb_result* out_h, qwb_prec prec, void* stream) {
    if (!K_d) return fail(QWB_ERR_INVALID_ARG, "qwb_primal_upscale_ipf_kernel: null kernel");
    return primal_single(ctx, prob, mu_d, nu_d, pi_rowptr_d, pi_col_d, pi_val_d, pi_nnz, sweeps, K_d,
                         a_d, b_d, out_h, prec, stream);
}

int qwb_dual_upscale_ctransform(qwb_ctx* ctx, const qwb_problem* prob, const double* mu_d,
                                const double* nu_d, const double* f_coarse_d, double* f_d,
                                double* g_d, qwb_result* out_h, qwb_prec prec, void* stream) {
    if (!ctx || !mu_d || !nu_d || !f_coarse_d || !out_h)
        return fail(QWB_ERR_INVALID_ARG, "qwb_dual_upscale_ctransform: null argument");
    int st = check_problem(prob);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, prob, 1, prec, &b))) return st;
    PairDev& P = b->pairs_h[0];
    const int M = b->Ms[0];
    QWB_CUDA(cudaMemcpyAsync((void*)P.f_coarse, f_coarse_d, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    P.mu = mu_d; P.nu = nu_d; P.f_out = f_d; P.g_out = g_d;
    st = single_upload(b, s);
    P.f_out = nullptr; P.g_out = nullptr;
    if (st) return st;
    QWB_CUDA(cudaMemsetAsync(b->outs_d, 0, sizeof(PairOut), s));
    if ((st = single_validate(b, s))) return st;
    if ((st = launch_centre(b->pairs_d, b->outs_d, b->pair_ids_d, 1, s))) return st;
    if ((st = launch_upsample(b->pairs_d, b->outs_d, b->pix_items_d, b->n_pix, b->f64, s))) return st;
    CtConfig c = b->ct_cfg_p;
    c.p2 = (prob->p == 2.0);
    if ((st = launch_ctransform(b->pairs_d, b->ct_p_items_d, b->ct_cnt[0], 0, c, prob->N, b->f64, 0, s))) return st;
    if ((st = launch_ctransform(b->pairs_d, b->ct_p_items_d, b->ct_cnt[0], 1, c, prob->N, b->f64, 0, s))) return st;
    if ((st = launch_lbsum(b->pairs_d, b->outs_d, b->pair_ids_d, 1, b->f64, s))) return st;
    PairOut o;
    QWB_CUDA(cudaMemcpyAsync(&o, b->outs_d, sizeof(PairOut), cudaMemcpyDeviceToHost, s));
    QWB_CUDA(cudaStreamSynchronize(s));
    std::memset(out_h, 0, sizeof(*out_h));
    out_h->lb = o.lb; out_h->lb_p = o.lb_p;
    return QWB_OK;
}

// The standalone transform with the default launch shape (shape == nullptr)
// or a given one; in_rows > 0 re-splits the input lines into items of that
// many lines each.
static int ctransform_impl(qwb_ctx* ctx, int32_t N, double p, const double* h_d, double* out_d,
                           qwb_prec prec, void* stream, const CtConfig* shape, int in_rows, int d = 2) {
    if (!ctx || !h_d || !out_d) return fail(QWB_ERR_INVALID_ARG, "qwb_ctransform: null argument");
    if (d != 2 && d != 3) return fail(QWB_ERR_INVALID_ARG, "qwb_ctransform: d must be 2 or 3");
    qwb_problem prob{N, N, p, d, 0};
    if (d == 3)      // the coarse grid is unused here; pick a block side check_problem accepts
        for (int k = 1; k <= 16; ++k)
            if (N % k == 0 && N / k <= 16) { prob.kappa = k; break; }
    int st = check_problem(&prob);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, &prob, 1, prec, &b))) return st;
    PairDev& P = b->pairs_h[0];
    P.f_out = nullptr; P.g_out = nullptr;
    if ((st = single_upload(b, s))) return st;
    CtConfig c = b->ct_cfg_p;
    if (shape) { c.R = shape->R; c.TC = shape->TC; c.packed = shape->packed; }
    c.p2 = (p == 2.0);
    const CtItem* items = b->ct_p_items_d;
    int n_items = b->ct_cnt[0];
    CtItem* own = nullptr;
    const int m = ipow(N, d), lines = ipow(N, d - 1);
    if (in_rows > 0) {           // a one-off item list with the requested split
        std::vector<CtItem> it;
        for (int o = 0; o < m; o += CT_TILE)
            for (int r0 = 0; r0 < lines; r0 += in_rows) it.push_back({0, o, r0, std::min(in_rows, lines - r0)});
        if (cudaMalloc((void**)&own, sizeof(CtItem) * it.size()) != cudaSuccess)
            return fail(QWB_ERR_OOM, "qwb_ctransform_shape: item list");
        QWB_CUDA(cudaMemcpyAsync(own, it.data(), sizeof(CtItem) * it.size(), cudaMemcpyHostToDevice, s));
        items = own; n_items = (int)it.size();
        c.in_rows = in_rows;
    }
    // outputs start at +inf: items that see part of the lines combine by atomic min
    st = launch_to_work(h_d, P.fhat, P.g, m, b->f64, s);
    if (!st) st = launch_ctransform(b->pairs_d, items, n_items, 0, c, N, b->f64, 0, s);
    if (!st) st = launch_from_work(P.g, out_d, m, b->f64, s);
    if (own) {
        const cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(own);
        if (e != cudaSuccess) return cuda_fail(e, "qwb_ctransform_shape");
    }
    if (st) return st;
    QWB_CUDA(cudaStreamSynchronize(s));
    return QWB_OK;
}

int qwb_ctransform(qwb_ctx* ctx, int32_t N, double p, const double* h_d, double* out_d, qwb_prec prec,
                   void* stream) {
    return ctransform_impl(ctx, N, p, h_d, out_d, prec, stream, nullptr, 0);
}

int qwb_ctransform_shape(qwb_ctx* ctx, int32_t N, int32_t d, double p, const double* h_d,
                         double* out_d, int32_t R, int32_t TC, int32_t packing, int32_t in_rows,
                         qwb_prec prec, void* stream) {
    if (R < 1 || TC < 1 || N < 1 || N % R || N % TC || packing < 0 || packing > 12 || in_rows < 0)
        return fail(QWB_ERR_INVALID_ARG, "qwb_ctransform_shape: R and TC must divide N; packing in 0..12");
    if (packing && prec == QWB_PREC_F64)
        return fail(QWB_ERR_INVALID_ARG, "qwb_ctransform_shape: packing needs MIXED precision");
    CtConfig c;
    c.R = R; c.TC = TC; c.packed = packing;
    const int st = ctransform_impl(ctx, N, p, h_d, out_d, prec, stream, &c, in_rows, d);
    if (st == QWB_ERR_UNSUPPORTED) return fail(st, "qwb_ctransform_shape: shape not compiled");
    return st;
}

int qwb_ctransform_separable(qwb_ctx* ctx, int32_t N, const double* h_d, double* out_d,
                             qwb_prec prec, void* stream) {
    if (!ctx || !h_d || !out_d) return fail(QWB_ERR_INVALID_ARG, "qwb_ctransform_separable: null argument");
    qwb_problem prob{N, N, 2.0};
    int st = check_problem(&prob);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_batch* b;
    if ((st = single_batch(ctx, &prob, 1, prec, &b, QWB_FLAG_SEPARABLE))) return st;
    PairDev& P = b->pairs_h[0];
    P.f_out = nullptr; P.g_out = nullptr;
    if ((st = single_upload(b, s))) return st;
    if ((st = launch_to_work(h_d, P.fhat, P.g, N * N, b->f64, s))) return st;
    if ((st = launch_sep(b->pairs_d, b->sep_items_d, b->n_sep, 0, 0, N, b->f64, 0, s))) return st;
    if ((st = launch_sep(b->pairs_d, b->sep_items_d, b->n_sep, 0, 1, N, b->f64, 0, s))) return st;
    if ((st = launch_from_work(P.g, out_d, N * N, b->f64, s))) return st;
    QWB_CUDA(cudaStreamSynchronize(s));
    return QWB_OK;
}

int qwb_lb_adjoint(qwb_ctx* ctx, int32_t N, double p, const double* f_d, const double* mu_d,
                   double lb_p, double* grad_d, void* stream) {
    if (!ctx || !f_d || !mu_d || !grad_d) return fail(QWB_ERR_INVALID_ARG, "qwb_lb_adjoint: null argument");
    if (N < 1 || N > 1024 || !(p >= 1.0)) return fail(QWB_ERR_INVALID_ARG, "qwb_lb_adjoint: bad N or p");
    std::lock_guard<std::mutex> lk(ctx->mtx);
    QWB_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    qwb_problem prob{N, N, p};
    qwb_batch* b;
    int st = single_batch(ctx, &prob, 1, QWB_PREC_F64, &b);
    if (st) return st;
    return launch_adjoint(N, p, f_d, mu_d, lb_p, grad_d, b->pairs_h[0].mu_c, s);
}

}  // extern "C"
