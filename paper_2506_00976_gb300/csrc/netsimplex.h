// netsimplex.h -- the library's exact solver for the small coarse Kantorovich
// problems (Sec. 2.1; coarse problems of Sec. 3.2, 3.4, 3.5; network simplex
// with at most 2M - 1 positive plan entries, Sec. 4).  Host C++, FP64.
#pragma once
#include <cstdint>
#include <vector>

namespace qwb {

struct NSSolution {
    std::vector<int32_t> rowptr;  // CSR of the plan, n_src + 1
    std::vector<int32_t> col;     // nnz
    std::vector<double> val;      // nnz, > 0
    std::vector<double> f;        // n_src potentials
    std::vector<double> g;        // n_dst potentials, g_j = min_i C_ij - f_i
    double obj = 0.0;             // <plan, C>
    int64_t pivots = 0;
};

// Final spanning tree of a solve (parent, arc to the parent, its direction per
// node, the artificial root excluded).  Any basis of a problem with the same
// supplies is a feasible start for other costs.
struct NSBasis {
    std::vector<int> parent;
    std::vector<int64_t> pred;
    std::vector<signed char> up;
    bool valid = false;
};

// Returns a qwb status code (0 = OK, NOT_CONVERGED when max_pivots is hit).
// C: n_src x n_dst row-major, non-negative and finite.  a, b: non-negative.
// warm: optional starting basis from a solve with the same supplies;
// basis_out: optional final basis; candidates: optional arcs (i * n_dst + j)
// priced first -- when none of them can enter, a scan of all arcs adds those
// that can, so the result is optimal over all arcs either way.
// exact_dual = false skips the final c-transforms: f, g are then the
// optimal tree potentials (f_i + g_j = C_ij on the plan's support and
// <= C_ij up to the pricing tolerance elsewhere), for callers that use only
// the plan.
// cost_bound >= 0 (with candidates): an upper bound on every C_ij known to
// the caller.  It sets the artificial arc cost in place of the maximum, and
// the entries (0 <= C_ij <= cost_bound) are checked by the solve's full scans
// instead of by a pass of their own before it; a failing entry still returns
// QWB_ERR_INVALID_ARG.
int network_simplex(int32_t n_src, int32_t n_dst, const double* C, const double* a,
                    const double* b, NSSolution& out, int64_t max_pivots = -1,
                    const NSBasis* warm = nullptr, NSBasis* basis_out = nullptr,
                    const std::vector<int64_t>* candidates = nullptr, bool exact_dual = true,
                    double cost_bound = -1.0);

// The same for the grid problem with C_kl = tab[|k1 - l1| * n_side + |k2 - l2|]
// on an n_side x n_side coarse grid (k = k1 * n_side + k2): the centre cost
// C~ of Sec. 3.4 / 3.5 without an M x M matrix.
int network_simplex_grid(int32_t n_side, const double* tab, const double* a, const double* b,
                         NSSolution& out, int64_t max_pivots = -1, NSBasis* basis_out = nullptr,
                         const NSBasis* warm = nullptr);

}  // namespace qwb
