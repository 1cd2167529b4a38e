// api_host.cpp -- host-only parts of the C ABI: status strings, thread-local
// error messages, the launch counter and the exact coarse solve entry point.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <string>

#include "../../include/qwb.h"
#include "fault.h"
#include "netsimplex.h"

namespace qwb {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_last_error(const std::string& msg) { g_last_error = msg; }
void count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int64_t fault_param(const char* site, int64_t def) {
    const char* env = std::getenv("QWB_FAULT");
    if (!env || !*env) return def;
    const std::string all(env), key = std::string(site) + "=";
    size_t pos = 0;
    while (pos <= all.size()) {
        const size_t end = std::min(all.find(',', pos), all.size());
        const std::string item = all.substr(pos, end - pos);
        if (item.compare(0, key.size(), key) == 0) return std::strtoll(item.c_str() + key.size(), nullptr, 10);
        pos = end + 1;
    }
    return def;
}

uint64_t wait_timeout_ns() {
    const char* env = std::getenv("QWB_WAIT_TIMEOUT_MS");
    const double ms = (env && *env) ? std::strtod(env, nullptr) : 2000.0;
    return (uint64_t)((ms > 0.0 ? ms : 2000.0) * 1e6);
}

}  // namespace qwb

extern "C" {

const char* qwb_status_string(int status) {
    switch (status) {
        case QWB_OK: return "QWB_OK";
        case QWB_ERR_INVALID_ARG: return "QWB_ERR_INVALID_ARG";
        case QWB_ERR_MASS: return "QWB_ERR_MASS";
        case QWB_ERR_CUDA: return "QWB_ERR_CUDA";
        case QWB_ERR_NOT_CONVERGED: return "QWB_ERR_NOT_CONVERGED";
        case QWB_ERR_TIMEOUT: return "QWB_ERR_TIMEOUT";
        case QWB_ERR_OOM: return "QWB_ERR_OOM";
        case QWB_ERR_UNSUPPORTED: return "QWB_ERR_UNSUPPORTED";
        case QWB_ERR_VERIFY: return "QWB_ERR_VERIFY";
        default: return "QWB_ERR_UNKNOWN";
    }
}

const char* qwb_last_error(void) { return qwb::g_last_error.c_str(); }

int64_t qwb_kernel_launch_count(void) { return qwb::g_launches.load(); }

}  // extern "C"

// Copies a solution to the caller's buffers (the plan arrays only when given).
static int export_solution(const qwb::NSSolution& sol, int st, const char* who, int32_t n_src, int32_t n_dst,
                           int32_t* rowptr_h, int32_t* col_h, double* val_h, int32_t* nnz_out, double* f_h,
                           double* g_h, double* obj_out) {
    if (st != QWB_OK) {
        qwb::set_last_error(st == QWB_ERR_NOT_CONVERGED
                                ? std::string(who) + ": pivot cap reached or artificial flow left"
                                : std::string(who) + ": invalid costs or masses");
        return st;
    }
    const int32_t nnz = (int32_t)sol.col.size();
    if (nnz_out) *nnz_out = nnz;
    if (rowptr_h) {
        std::memcpy(rowptr_h, sol.rowptr.data(), sizeof(int32_t) * (n_src + 1));
        std::memcpy(col_h, sol.col.data(), sizeof(int32_t) * nnz);
        std::memcpy(val_h, sol.val.data(), sizeof(double) * nnz);
    }
    if (f_h) std::memcpy(f_h, sol.f.data(), sizeof(double) * n_src);
    if (g_h) std::memcpy(g_h, sol.g.data(), sizeof(double) * n_dst);
    if (obj_out) *obj_out = sol.obj;
    return QWB_OK;
}

extern "C" {

int qwb_coarse_solve(int32_t n_src, int32_t n_dst, const double* C_h, const double* a_h,
                     const double* b_h, int32_t* rowptr_h, int32_t* col_h, double* val_h,
                     int32_t* nnz_out, double* f_h, double* g_h, double* obj_out) {
    if (n_src <= 0 || n_dst <= 0 || !C_h || !a_h || !b_h) {
        qwb::set_last_error("qwb_coarse_solve: bad sizes or null input");
        return QWB_ERR_INVALID_ARG;
    }
    if ((rowptr_h || col_h || val_h) && !(rowptr_h && col_h && val_h && nnz_out)) {
        qwb::set_last_error("qwb_coarse_solve: plan outputs need rowptr, col, val and nnz_out");
        return QWB_ERR_INVALID_ARG;
    }
    qwb::NSSolution sol;
    int st;
    try {
        st = qwb::network_simplex(n_src, n_dst, C_h, a_h, b_h, sol);
    } catch (...) {
        qwb::set_last_error("qwb_coarse_solve: host allocation failed");
        return QWB_ERR_OOM;
    }
    return export_solution(sol, st, "qwb_coarse_solve", n_src, n_dst, rowptr_h, col_h, val_h, nnz_out, f_h, g_h,
                           obj_out);
}

int qwb_coarse_solve_grid(int32_t n_side, const double* tab_h, const double* a_h, const double* b_h,
                          int32_t* rowptr_h, int32_t* col_h, double* val_h, int32_t* nnz_out, double* f_h,
                          double* g_h, double* obj_out) {
    if (n_side <= 0 || !tab_h || !a_h || !b_h) {
        qwb::set_last_error("qwb_coarse_solve_grid: bad size or null input");
        return QWB_ERR_INVALID_ARG;
    }
    if ((rowptr_h || col_h || val_h) && !(rowptr_h && col_h && val_h && nnz_out)) {
        qwb::set_last_error("qwb_coarse_solve_grid: plan outputs need rowptr, col, val and nnz_out");
        return QWB_ERR_INVALID_ARG;
    }
    const int32_t M = n_side * n_side;
    qwb::NSSolution sol;
    int st;
    try {
        st = qwb::network_simplex_grid(n_side, tab_h, a_h, b_h, sol);
    } catch (...) {
        qwb::set_last_error("qwb_coarse_solve_grid: host allocation failed");
        return QWB_ERR_OOM;
    }
    return export_solution(sol, st, "qwb_coarse_solve_grid", M, M, rowptr_h, col_h, val_h, nnz_out, f_h, g_h,
                           obj_out);
}

}  // extern "C"
