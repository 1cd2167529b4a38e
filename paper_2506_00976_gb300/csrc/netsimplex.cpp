// netsimplex.cpp -- primal network simplex for the coarse transport LPs.
//
// Solves min <pi, C> subject to pi 1 = a, pi^T 1 = b, pi >= 0 (Sec. 2.1) and
// returns an optimal basic plan (at most n_src + n_dst - 1 positive entries,
// Sec. 4) with optimal Kantorovich potentials.  The coarse problems of Sec.
// 3.2 (C-bar), 3.4 and 3.5 (C~) are all of this form.
//
// Design (textbook primal network simplex, written for this library):
//   * graph: sources 0..n-1, sinks n..n+m-1, an artificial root n+m;
//     real arc a = i*m + j (source i -> sink j) and one artificial arc per
//     node (source with supply -> root, root -> other nodes) with a cost BIG
//     above any path cost, so that the all-artificial star is a strongly
//     feasible starting tree;
//   * costs come either from a dense matrix (C-bar) or, for the grid centre
//     cost C~, from a table over block offsets (|dk1|, |dk2|), so that pricing
//     does not stream an M x M matrix;
//   * spanning tree stored as parent pointers plus its pre-order as a
//     circular doubly linked thread with the last node of every subtree, so
//     a subtree is one thread segment (the textbook threaded-index form);
//     the flow of each tree arc is kept on its child node;
//   * block-search pricing over the real arcs (block ~ sqrt(#arcs)), each
//     block walked as contiguous runs of one source row (grid costs through
//     a reflected table row, so a run is two unit-stride streams),
//     reduced cost rc(u,w) = c(u,w) - pot[u] + pot[w];
//   * leaving arc by the strongly feasible rule (the last blocking arc met
//     when the pivot cycle is traversed from its apex along the entering
//     arc's direction), which prevents cycling under degeneracy;
//   * the apex of a pivot cycle is found by walking up from both ends of the
//     entering arc in turn, stamping the nodes, until one walk meets the
//     other's trail (no depths are kept); after the pivot the re-hung subtree
//     gets its potentials shifted by one common amount (its internal arcs do
//     not change); every V pivots, and before every full scan of the sparse
//     pricing, all potentials are recomputed from the tree and re-centred, so
//     that neither the shifts' rounding nor the artificial cost eats their
//     precision;
//   * a solve can start from the final tree of another solve with the same
//     supplies (a feasible, strongly feasible basis for any costs): the C-bar
//     problem starts from the C~ optimum;
//   * the grid problem is solved coarse to fine: the same problem on the
//     (n/2) x (n/2) grid of 2 x 2 cell sums (costs at doubled offsets) is
//     solved first; the fine solve starts from a feasible tree built from
//     the coarse plan (its flows split over the children by north-west
//     corner passes) and prices only the arcs between the children of the
//     coarse plan's support (sparse pricing) until none of them has a
//     negative reduced cost; then one scan of all arcs adds every arc that
//     still has one, and pricing resumes, until a full scan finds none (so
//     the result is optimal over all arcs);
//   * at the end the tree flows are recomputed exactly from the supplies
//     (leaf elimination) and the potentials are made exactly dual feasible by
//     one coarse c-transform each way (g = f^c, f = g^c).
#include "netsimplex.h"
#include "fault.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <type_traits>

#include "../../include/qwb.h"

namespace qwb {
namespace {

// Cost of real arc (i, j): dense matrix or grid block-offset table.
struct DenseCost {
    const double* C;
    int m;
    double operator()(int i, int j) const { return C[(int64_t)i * m + j]; }
};
struct GridCost {
    const double* tab;   // ns x ns, tab[|dk1| * ns + |dk2|]
    int ns;
    const double* refl = nullptr;   // ns x (2 ns - 1): refl[d1][ns - 1 + d2] = tab[d1][|d2|]
    bool separable = false;         // tab[d1][d2] == tab[d1][0] + tab[0][d2] exactly (e.g. p = 2)
    double operator()(int i, int j) const {
        const int d1 = std::abs(i / ns - j / ns), d2 = std::abs(i % ns - j % ns);
        return tab[d1 * ns + d2];
    }
};

template <typename Cost>
struct Solver {
    int n = 0, m = 0, V = 0, root = 0;
    int64_t NM = 0;
    Cost cst;
    double BIG = 0.0, eps = 0.0;
    std::vector<double> supply;
    std::vector<signed char> art_up;  // artificial arc of node v: 1 = v -> root
    // the tree: parent pointers, and its pre-order as a circular doubly
    // linked thread through the root with the last node of every subtree
    // (a subtree is the thread segment [v, last[v]])
    std::vector<int> parent, thread, rev, last;
    std::vector<int64_t> mark;        // apex search: 2 * stamp + side of the last walk through a node
    int64_t stamp = 0;
    std::vector<int64_t> pred;        // arc joining v and parent[v]
    std::vector<signed char> up;      // 1 if pred[v] is directed v -> parent[v]
    std::vector<double> flow;         // flow on pred[v]
    std::vector<double> pot;
    std::vector<int> stack, path, walk_k, walk_l, lold, rold, aold;
    std::vector<int64_t> old_pred;
    std::vector<signed char> old_up;
    std::vector<double> old_flow;
    int64_t price_pos = 0, block = 64;
    // sparse pricing over a candidate arc list (coarse-to-fine solves)
    bool sparse = false;
    std::vector<int64_t> cand;
    std::vector<int> cand_i, cand_j;  // endpoints and cost of each candidate
    std::vector<double> cand_c;
    std::vector<uint64_t> in_cand;    // bitset over the real arcs
    std::vector<double> row_buf;
    int64_t cand_pos = 0;
    void push_candidate(int64_t a) {
        in_cand[(size_t)(a >> 6)] |= 1ull << (a & 63);
        cand.push_back(a);
        const int i = (int)(a / m), j = (int)(a % m);
        cand_i.push_back(i);
        cand_j.push_back(j);
        cand_c.push_back(cst(i, j));
    }

    int tail(int64_t a) const {
        if (a < NM) return (int)(a / m);
        int v = (int)(a - NM);
        return art_up[v] ? v : root;
    }
    double cost(int64_t a) const { return a < NM ? cst((int)(a / m), (int)(a % m)) : BIG; }

    void pot_from_parent(int v) {
        const int p = parent[v];
        const double c = cost(pred[v]);
        pot[v] = up[v] ? c + pot[p] : pot[p] - c;   // rc of the tree arc is zero
    }
    // the re-hung subtree keeps its internal arcs: its potentials move by one
    // common amount (one pass along its thread segment)
    void shift_subtree(int r) {
        const double old = pot[r];
        pot_from_parent(r);
        const double d = pot[r] - old;
        const int end = last[r];
        const int* th = thread.data();
        double* pt = pot.data();
        int steps = 0;
        for (int v = r; v != end && ++steps < V;) {
            v = th[v];
            pt[v] += d;
        }
        if (steps >= V) broken = true;
    }
    void recentre() {
        // subtract a common constant (rc is invariant); keep real nodes small
        double s = 0.0;
        for (int v = 0; v < n + m; ++v) s += pot[v];
        s /= (double)(n + m);
        for (int v = 0; v < V; ++v) pot[v] -= s;
        refresh_below_root();
    }
    // every potential from its parent's, in pre-order from the root
    void refresh_below_root() {
        int steps = 0;
        for (int v = root; v != last[root] && ++steps < V;) {
            v = thread[v];
            pot_from_parent(v);
        }
        if (steps >= V) broken = true;
    }
    // set when a walk over the tree runs past V nodes (a corrupted tree, an
    // internal error): the solve then stops with QWB_ERR_NOT_CONVERGED
    // instead of looping
    bool broken = false;
    // thread, rev and last from the parent pointers (children in increasing
    // node order); false when the parent pointers do not form one tree
    bool build_thread() {
        std::vector<int> cnt(V + 1, 0), kids(V);
        for (int v = 0; v < V; ++v)
            if (v != root) {
                if (parent[v] < 0 || parent[v] >= V) return false;
                cnt[parent[v] + 1]++;
            }
        for (int v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
        {
            std::vector<int> cur(cnt.begin(), cnt.end() - 1);
            for (int v = 0; v < V; ++v)
                if (v != root) kids[cur[parent[v]]++] = v;
        }
        std::vector<int> order;
        order.reserve(V);
        if ((int)stack.size() < V) stack.resize(V);
        int* st = stack.data();
        int top = 0;
        st[top++] = root;
        while (top > 0) {
            const int v = st[--top];
            order.push_back(v);
            if ((int)order.size() > V) return false;
            for (int e = cnt[v + 1] - 1; e >= cnt[v]; --e) st[top++] = kids[e];
        }
        if ((int)order.size() != V) return false;
        std::vector<int> size(V, 1), pos(V);
        for (int i = 0; i < V; ++i) {
            const int a = order[i], b = order[(i + 1) % V];
            thread[a] = b;
            rev[b] = a;
            pos[a] = i;
        }
        for (int i = V - 1; i >= 1; --i) size[parent[order[i]]] += size[order[i]];
        for (int v = 0; v < V; ++v) last[v] = order[pos[v] + size[v] - 1];
        return true;
    }

    void init_common(int n_, int m_, const double* a, const double* b, double maxc) {
        n = n_; m = m_; V = n + m + 1; root = n + m; NM = (int64_t)n * m;
        BIG = (double)(V + 1) * (maxc + 1.0);
        eps = 1e-12 * (maxc + 1.0);
        supply.assign(V, 0.0);
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < n; ++i) { supply[i] = a[i]; sa += a[i]; }
        for (int j = 0; j < m; ++j) { supply[n + j] = -b[j]; sb += b[j]; }
        supply[root] = sb - sa;
        art_up.assign(V, 0);
        for (int v = 0; v < n; ++v) art_up[v] = a[v] > 0.0 ? 1 : 0;
        parent.assign(V, -1); mark.assign(V, -1); stamp = 0;
        thread.assign(V, root); rev.assign(V, root); last.assign(V, root);
        pred.assign(V, -1); up.assign(V, 0); flow.assign(V, 0.0); pot.assign(V, 0.0);
        block = std::max<int64_t>(64, (int64_t)std::sqrt((double)NM));
        price_pos = 0;
    }

    // the all-artificial star
    void init_star(const double* a, const double* b) {
        for (int v = 0; v < n + m; ++v) {
            parent[v] = root;
            pred[v] = NM + v;
            up[v] = art_up[v];
            flow[v] = (v < n) ? a[v] : b[v - n];
            pot[v] = art_up[v] ? BIG : -BIG;
        }
        build_thread();
    }

    // a previous final tree (same supplies, any costs); false when its
    // parent pointers do not form one tree
    bool init_basis(const NSBasis& B) {
        for (int v = 0; v < n + m; ++v) {
            parent[v] = B.parent[v];
            pred[v] = B.pred[v];
            up[v] = B.up[v];
        }
        if (!build_thread()) return false;
        refresh_below_root();
        recompute_flows();
        return !broken;
    }

    // A starting tree built by the caller (not a previous final tree): after
    // the flows are recomputed from the supplies, rounding-level negative
    // flows (>= -tol) become zero; the tree is kept only when every flow is
    // then non-negative and every zero-flow arc points away from the root
    // (strongly feasible), else the caller starts from the star.
    bool init_basis_checked(const NSBasis& B, double tol) {
        if (!init_basis(B)) return false;
        for (int v = 0; v < n + m; ++v) {
            if (flow[v] < 0.0) {
                if (flow[v] < -tol) return false;
                flow[v] = 0.0;
            }
            if (flow[v] == 0.0 && up[v]) return false;
        }
        return true;
    }
    void reset_tree() {
        std::fill(parent.begin(), parent.end(), -1);
        broken = false;
    }

    // minimum of c[t] + pg[t] over a contiguous run: four independent chains
    // of two-lane vectors (GCC vector extensions: SSE2 or NEON registers; the
    // compiler keeps a scalar min reduction serial); the minimum of a set
    // does not depend on the order in which it is taken
    typedef double v2d __attribute__((vector_size(16)));
    static v2d load2(const double* p) { v2d v; std::memcpy(&v, p, sizeof v); return v; }
    static v2d vmin(v2d a, v2d b) { return a < b ? a : b; }
    static double run_min(const double* c, const double* pg, int len) {
        const v2d inf = {HUGE_VAL, HUGE_VAL};
        v2d m0 = inf, m1 = inf, m2 = inf, m3 = inf;
        int t = 0;
        for (; t + 8 <= len; t += 8) {
            m0 = vmin(load2(c + t) + load2(pg + t), m0);
            m1 = vmin(load2(c + t + 2) + load2(pg + t + 2), m1);
            m2 = vmin(load2(c + t + 4) + load2(pg + t + 4), m2);
            m3 = vmin(load2(c + t + 6) + load2(pg + t + 6), m3);
        }
        m0 = vmin(vmin(m0, m1), vmin(m2, m3));
        double mn = m0[0] < m0[1] ? m0[0] : m0[1];
        for (; t < len; ++t) { const double r = c[t] + pg[t]; mn = r < mn ? r : mn; }
        return mn;
    }
    // out[t] = min(out[t], row[t] + s), element-wise
    static void min_plus_row(double* out, const double* row, double s, int len) {
        for (int t = 0; t < len; ++t) {
            const double v = row[t] + s;
            out[t] = v < out[t] ? v : out[t];
        }
    }
    // the same minimum, and whether every c[t] lies in [0, hi] (false for NaN)
    static double run_min_checked(const double* c, const double* pg, int len, double hi, bool& ok) {
        typedef long long v2l __attribute__((vector_size(16)));
        const v2d inf = {HUGE_VAL, HUGE_VAL}, zero = {0.0, 0.0}, top = {hi, hi};
        v2d m0 = inf, m1 = inf;
        v2l good = {-1, -1};
        int t = 0;
        for (; t + 4 <= len; t += 4) {
            const v2d c0 = load2(c + t), c1 = load2(c + t + 2);
            good &= (c0 >= zero) & (c0 <= top) & (c1 >= zero) & (c1 <= top);
            m0 = vmin(c0 + load2(pg + t), m0);
            m1 = vmin(c1 + load2(pg + t + 2), m1);
        }
        m0 = vmin(m0, m1);
        double mn = m0[0] < m0[1] ? m0[0] : m0[1];
        bool g = good[0] == -1 && good[1] == -1;
        for (; t < len; ++t) {
            g = g && c[t] >= 0.0 && c[t] <= hi;
            const double r = c[t] + pg[t];
            mn = r < mn ? r : mn;
        }
        ok = g;
        return mn;
    }
    // scan row i, columns [j0, j1): cost run against sink potentials
    void scan_run(int i, int j0, int j1, double& best, int64_t& best_a) {
        const double pi = pot[i];
        const double* pg = pot.data() + n;
        if constexpr (std::is_same<Cost, GridCost>::value) {
            const int ns = cst.ns;
            const int i1 = i / ns, i2 = i % ns;
            int j = j0, jr = j0 / ns, jc0 = j0 % ns;   // grid row and column of j (no division per run)
            while (j < j1) {
                const int len = std::min(ns - jc0, j1 - j);
                // reflected table row: refl[ns - 1 + d] = tab[|i1 - jr|][|d|]
                const double* refl = cst.refl + (size_t)std::abs(i1 - jr) * (2 * ns - 1) + (ns - 1 - i2);
                const double mn = run_min(refl + jc0, pg + j, len) - pi;
                if (mn < best) {
                    for (int t = 0; t < len; ++t) {
                        const double rc = refl[jc0 + t] + pg[j + t] - pi;
                        if (rc < best) { best = rc; best_a = (int64_t)i * m + j + t; }
                    }
                }
                j += len;
                ++jr;
                jc0 = 0;
            }
        } else {
            const double* c = cst.C + (int64_t)i * m;
            const double mn = run_min(c + j0, pg + j0, j1 - j0) - pi;
            if (mn < best)
                for (int j = j0; j < j1; ++j) {
                    const double rc = c[j] + pg[j] - pi;
                    if (rc < best) { best = rc; best_a = (int64_t)i * m + j; }
                }
        }
    }

    // Block-search pricing: the most negative reduced cost in the first block
    // that has one.  Returns -1 at optimality.
    int64_t find_entering(double* rc_out) {
        int64_t scanned = 0;
        int64_t pos = price_pos;
        while (scanned < NM) {
            const int64_t end = std::min<int64_t>(pos + block, NM);
            double best = -eps;
            int64_t best_a = -1;
            for (int64_t a = pos; a < end;) {
                const int i = (int)(a / m), j0 = (int)(a % m);
                const int j1 = (int)std::min<int64_t>(m, j0 + (end - a));
                scan_run(i, j0, j1, best, best_a);
                a += j1 - j0;
            }
            scanned += end - pos;
            pos = (end == NM) ? 0 : end;
            if (best_a >= 0) {
                price_pos = pos;
                *rc_out = best;
                return best_a;
            }
        }
        return -1;
    }

    void set_candidates(const std::vector<int64_t>& arcs) {
        sparse = true;
        in_cand.assign((size_t)((NM + 63) / 64), 0ull);
        cand.clear(); cand_i.clear(); cand_j.clear(); cand_c.clear();
        for (int64_t a : arcs)
            if (!((in_cand[(size_t)(a >> 6)] >> (a & 63)) & 1ull)) push_candidate(a);
        cand_pos = 0;
        qn = 0;
    }
    // Block search over the candidate arcs: the most negative reduced cost in
    // the first block of about sqrt(#candidates) arcs that has one.  The
    // block's next few most negative arcs are queued; the following calls
    // take the best queued arc that is still negative at the current
    // potentials before scanning again (partial pricing with a short
    // candidate list: fewer scans for about as many pivots).
    static constexpr int kQueue = 6;  // arcs kept from a block scan (the best included)
    int qn = 0;                       // queued candidates from the last block scan
    int64_t qt[kQueue];
    int64_t find_entering_sparse(double* rc_out) {
        const int64_t nc = (int64_t)cand.size();
        if (nc == 0) return -1;
        const int* ci = cand_i.data();
        const int* cj = cand_j.data();
        const double* cc = cand_c.data();
        const double* pg = pot.data() + n;
        // first the arcs queued by the last scan, at today's potentials
        if (qn > 0) {
            double best = -eps;
            int bi = -1, keep = 0;
            for (int u = 0; u < qn; ++u) {
                const int64_t t = qt[u];
                const double rc = cc[t] - pot[ci[t]] + pg[cj[t]];
                if (rc < -eps) {
                    qt[keep] = t;
                    if (rc < best) { best = rc; bi = keep; }
                    ++keep;
                }
            }
            qn = keep;
            if (bi >= 0) {
                const int64_t t = qt[bi];
                qt[bi] = qt[--qn];
                *rc_out = best;
                return cand[(size_t)t];
            }
        }
        constexpr int K = kQueue;
        const int64_t blk = std::max<int64_t>(32, (int64_t)std::sqrt((double)nc));
        int64_t scanned = 0, pos = cand_pos;
        while (scanned < nc) {
            const int64_t end = std::min<int64_t>(pos + blk, nc);
            // the K most negative reduced costs of the block, sorted
            double brc[K];
            int64_t bt[K];
            int nb = 0;
            double worst = -eps;
            for (int64_t t = pos; t < end; ++t) {
                const double rc = cc[t] - pot[ci[t]] + pg[cj[t]];
                if (rc < worst) {
                    int u = nb < K ? nb++ : K - 1;
                    while (u > 0 && brc[u - 1] > rc) { brc[u] = brc[u - 1]; bt[u] = bt[u - 1]; --u; }
                    brc[u] = rc; bt[u] = t;
                    if (nb == K) worst = brc[K - 1];
                }
            }
            scanned += end - pos;
            pos = (end == nc) ? 0 : end;
            if (nb > 0) {
                cand_pos = pos;
                qn = 0;
                for (int u = 1; u < nb; ++u) qt[qn++] = bt[u];
                *rc_out = brc[0];
                return cand[(size_t)bt[0]];
            }
        }
        return -1;
    }
    // check_bound >= 0: the costs were not checked before the solve; every
    // full scan checks the entries it reads (0 <= c <= check_bound, which also
    // excludes NaN and infinity) and sets bad_cost when one fails
    double check_bound = -1.0;
    bool bad_cost = false;
    // One scan of every real arc: add the arcs with a negative reduced cost to
    // the candidates.  Returns how many were added.
    int64_t add_violators() {
        int64_t added = 0;
        const double* pg = pot.data() + n;
        std::vector<double>& rcs = row_buf;
        rcs.resize(m);
        // separable grid costs: every row's min_j (c_ij + pot_j) by two 1-D
        // min-plus passes (O(ns^3) for all rows instead of O(ns^4)); a row
        // whose minimum clears -eps by more than the rounding margin has no
        // violator, the others are scanned exactly as before
        bool filter = false;
        if constexpr (std::is_same<Cost, GridCost>::value) filter = cst.separable;
        if (filter) row_minima_separable();
        for (int i = 0; i < n; ++i) {
            if (filter && rowmin[i] - pot[i] >= -eps + rowmin_margin) continue;
            if constexpr (std::is_same<Cost, DenseCost>::value) {
                if (check_bound >= 0.0) {           // row minimum and the entries' check in one pass
                    bool ok = true;
                    const double mn = run_min_checked(cst.C + (int64_t)i * m, pg, m, check_bound, ok);
                    if (!ok) { bad_cost = true; return 0; }
                    if (!(mn - pot[i] < -eps)) continue;
                } else {
                    double best = -eps;
                    int64_t dummy = -1;
                    scan_run(i, 0, m, best, dummy);   // row minimum below -eps?
                    if (dummy < 0) continue;
                }
            } else if (!filter) {                    // (a row the filter kept is scanned directly)
                double best = -eps;
                int64_t dummy = -1;
                scan_run(i, 0, m, best, dummy);       // row minimum below -eps?
                if (dummy < 0) continue;
            }
            const double* crow;
            if constexpr (std::is_same<Cost, DenseCost>::value) {
                crow = cst.C + (int64_t)i * m;
            } else {
                row_costs(i, rcs.data());
                crow = rcs.data();
            }
            const double pi = pot[i];
            auto take = [&](int j) {
                const double rc = crow[j] - pi + pg[j];
                if (rc < -eps) {
                    const int64_t a = (int64_t)i * m + j;
                    if (!((in_cand[(size_t)(a >> 6)] >> (a & 63)) & 1ull)) {
                        push_candidate(a);
                        ++added;
                    }
                }
            };
            // four reduced costs per step on two-lane vectors (the same sums
            // as the scalar test), which looks at a group only when it holds
            // a violator
            const v2d vpi = {pi, pi}, vlim = {-eps, -eps};
            int j = 0;
            for (; j + 4 <= m; j += 4) {
                const v2d r0 = load2(crow + j) - vpi + load2(pg + j);
                const v2d r1 = load2(crow + j + 2) - vpi + load2(pg + j + 2);
                const auto hit = (r0 < vlim) | (r1 < vlim);
                if (hit[0] | hit[1])
                    for (int t = j; t < j + 4; ++t) take(t);
            }
            for (; j < m; ++j) take(j);
        }
        return added;
    }
    // rowmin[i] ~ min_j (c_ij + pot_j) for separable grid costs
    // c_ij = A(|i1 - j1|) + B(|i2 - j2|): H[j1][i2] = min_j2 (B + pot), then
    // rowmin[i1][i2] = min_j1 (A + H).  Each is within a few roundings of the
    // exact minimum; rowmin_margin bounds that gap.
    std::vector<double> rowmin, hbuf;
    double rowmin_margin = 0.0;
    void row_minima_separable() {
        if constexpr (std::is_same<Cost, GridCost>::value) {
            const int ns = cst.ns;
            const double* pg = pot.data() + n;
            rowmin.resize(n);
            hbuf.resize((size_t)ns * ns);
            double pmax = 0.0, cmax = 0.0;
            for (int j = 0; j < m; ++j) pmax = std::max(pmax, std::fabs(pg[j]));
            for (int d = 0; d < ns; ++d) cmax = std::max(cmax, cst.tab[(size_t)(ns - 1) * ns + d]);
            // both passes as element-wise minima over contiguous rows (the
            // reflected table row refl[ns - 1 + x] = B(|x|)); the same sums
            // as the direct loops, and a minimum does not depend on the order
            const double* refl0 = cst.refl + (ns - 1);
            for (int j1 = 0; j1 < ns; ++j1) {
                double* h = hbuf.data() + (size_t)j1 * ns;
                std::fill(h, h + ns, HUGE_VAL);
                for (int j2 = 0; j2 < ns; ++j2)
                    min_plus_row(h, refl0 - j2, pg[j1 * ns + j2], ns);   // B(|i2 - j2|) + pg
            }
            for (int i1 = 0; i1 < ns; ++i1) {
                double* r = rowmin.data() + (size_t)i1 * ns;
                std::fill(r, r + ns, HUGE_VAL);
                for (int j1 = 0; j1 < ns; ++j1)
                    min_plus_row(r, hbuf.data() + (size_t)j1 * ns, cst.tab[(size_t)std::abs(i1 - j1) * ns], ns);
            }
            // three roundings of terms below cmax + pmax each, on both sides of
            // the comparison (with the potential of the row): a wide margin
            double pimax = 0.0;
            for (int i = 0; i < n; ++i) pimax = std::max(pimax, std::fabs(pot[i]));
            rowmin_margin = 16.0 * 0x1p-52 * (cmax + pmax + pimax) + 1e-300;
        }
    }

    // the costs of row i (grid costs through the reflected table rows)
    void row_costs(int i, double* out) const {
        if constexpr (std::is_same<Cost, GridCost>::value) {
            const int ns = cst.ns, i1 = i / ns, i2 = i % ns;
            for (int jr = 0; jr < ns; ++jr) {
                const double* refl = cst.refl + (size_t)std::abs(i1 - jr) * (2 * ns - 1) + (ns - 1 - i2);
                for (int c = 0; c < ns; ++c) out[jr * ns + c] = refl[c];
            }
        } else {
            const double* c = cst.C + (int64_t)i * m;
            for (int j = 0; j < m; ++j) out[j] = c[j];
        }
    }

    void pivot(int64_t e) {
        const int k = tail(e);
        const int l = n + (int)(e % m);   // entering arcs are real arcs
        // apex: alternate single steps up from k and from l, stamping nodes,
        // until a walk reaches a node the other walk has passed (the root
        // ends a walk; both ends lie in the one spanning tree).  The walks
        // are recorded, so the cycle's two sides are arrays afterwards.
        if ((int)walk_k.size() < V + 1) { walk_k.resize(V + 1); walk_l.resize(V + 1); }
        int* wk = walk_k.data();
        int* wl = walk_l.data();
        int nk = 0, nl = 0;
        ++stamp;
        const int64_t sk = 2 * stamp, sl = 2 * stamp + 1;
        int u = k, w = l, apex = -1;
        mark[u] = sk;
        wk[nk++] = u;
        if (mark[w] == sk) apex = w;
        else { mark[w] = sl; wl[nl++] = w; }
        int guard = 0;
        while (apex < 0) {
            if (++guard > 2 * V) { broken = true; return; }
            if (u != root) {
                u = parent[u];
                if (mark[u] == sl) { apex = u; break; }
                mark[u] = sk;
                wk[nk++] = u;
            }
            if (w != root) {
                w = parent[w];
                if (mark[w] == sk) { apex = w; break; }
                mark[w] = sl;
                wl[nl++] = w;
            }
        }
        // the walk that passed the apex first went on above it: cut it there
        for (int i = 0; i < nk; ++i) if (wk[i] == apex) { nk = i; break; }
        for (int i = 0; i < nl; ++i) if (wl[i] == apex) { nl = i; break; }
        // l side (traversed upward): the last arc of least flow against the
        // cycle's direction; k side (traversed downward): the first one.
        // Their minimum is the step delta, and the leaving arc is the l
        // side's candidate when it attains delta (the strongly feasible rule)
        double min_l = std::numeric_limits<double>::infinity(), min_k = min_l;
        int ql = -1, qk = -1;
        for (int i = 0; i < nl; ++i) {
            const int v = wl[i];
            if (!up[v] && flow[v] <= min_l) { min_l = flow[v]; ql = i; }
        }
        for (int i = 0; i < nk; ++i) {
            const int v = wk[i];
            if (up[v] && flow[v] < min_k) { min_k = flow[v]; qk = i; }
        }
        const bool on_l_side = ql >= 0 && min_l <= min_k;
        const double delta = on_l_side ? min_l : min_k;
        const int q = on_l_side ? wl[ql] : wk[qk];
        for (int i = 0; i < nl; ++i) { const int v = wl[i]; flow[v] += up[v] ? delta : -delta; }
        for (int i = 0; i < nk; ++i) { const int v = wk[i]; flow[v] += up[v] ? -delta : delta; }
        const int e1 = on_l_side ? l : k;
        const int e2 = on_l_side ? k : l;
        const int* side = on_l_side ? wl : wk;       // e1 up to q: a prefix of its walk
        const int qi = on_l_side ? ql : qk;
        path.assign(side, side + qi + 1);
        const int t = qi;
        // thread update.  T, the subtree of q, is the segment [q, last[q]];
        // re-rooted at e1 its pre-order is e1's old segment, then for each
        // s = 1..t the segment of path[s] without that of path[s - 1] (two
        // runs around the hole), and it goes in right after e2.
        lold.resize(t + 1); rold.resize(t + 1); aold.resize(t + 1);
        for (int s2 = 0; s2 <= t; ++s2) {
            const int v = path[s2];
            lold[s2] = last[v]; rold[s2] = rev[v]; aold[s2] = thread[last[v]];
        }
        const int q_parent = parent[q];
        thread[rold[t]] = aold[t];                   // cut T out
        rev[aold[t]] = rold[t];
        for (int u = q_parent, k2 = 0; u >= 0 && last[u] == lold[t] && k2 < V; u = parent[u], ++k2) last[u] = rold[t];
        int tl = lold[0];                            // end of the new order so far
        for (int s2 = 1; s2 <= t; ++s2) {
            const int v = path[s2];
            thread[tl] = v; rev[v] = tl;             // path[s2] .. the node before the hole
            tl = rold[s2 - 1];
            if (lold[s2 - 1] != lold[s2]) {          // the run after the hole
                thread[tl] = aold[s2 - 1]; rev[aold[s2 - 1]] = tl;
                tl = lold[s2];
            }
        }
        for (int s2 = 0; s2 <= t; ++s2) last[path[s2]] = tl;
        {
            const int nx = thread[e2];               // splice in after e2
            const bool leaf = last[e2] == e2;
            thread[e2] = e1; rev[e1] = e2;
            thread[tl] = nx; rev[nx] = tl;
            if (leaf)
                for (int u = e2, k2 = 0; u >= 0 && last[u] == e2 && k2 < V; u = parent[u], ++k2) last[u] = tl;
        }
        // parent pointers, arcs and flows along the reversed path
        old_pred.resize(t); old_up.resize(t); old_flow.resize(t);
        for (int s = 0; s < t; ++s) {
            old_pred[s] = pred[path[s]]; old_up[s] = up[path[s]]; old_flow[s] = flow[path[s]];
        }
        for (int s = 0; s < t; ++s) {
            const int child = path[s + 1];
            parent[child] = path[s];
            pred[child] = old_pred[s];
            up[child] = old_up[s] ? 0 : 1;
            flow[child] = old_flow[s];
        }
        parent[e1] = e2;
        pred[e1] = e;
        up[e1] = (tail(e) == e1) ? 1 : 0;
        flow[e1] = delta;
        shift_subtree(e1);
    }

    // Exact tree flows from the supplies (leaf elimination in reverse
    // pre-order: every node after all of its descendants).
    void recompute_flows() {
        std::vector<double> S(supply);
        int steps = 0;
        for (int v = rev[root]; v != root && steps++ < V; v = rev[v]) {
            flow[v] = up[v] ? S[v] : -S[v];
            S[parent[v]] += S[v];
        }
        if (steps >= V) broken = true;
    }
};

template <typename Cost>
int solve(int32_t n_src, int32_t n_dst, Cost cst, double maxc, const double* a, const double* b,
          NSSolution& out, int64_t max_pivots, const NSBasis* warm, NSBasis* basis_out,
          const std::vector<int64_t>* candidates = nullptr, bool exact_dual = true,
          double check_bound = -1.0, bool warm_built = false) {
    const int64_t NM = (int64_t)n_src * n_dst;
    if (max_pivots < 0) max_pivots = 20 * NM + 1000000;
    const int64_t cap = fault_param("ns_pivot_cap", -1);     // host-side fault injection (tests)
    if (cap >= 0) max_pivots = std::min<int64_t>(max_pivots, cap);
    Solver<Cost> S;
    S.cst = cst;
    S.check_bound = check_bound;
    S.init_common(n_src, n_dst, a, b, maxc);
    bool started = false;
    if (warm && warm->valid && (int)warm->parent.size() == n_src + n_dst) {
        if (!warm_built) {
            started = S.init_basis(*warm);
            if (!started) S.reset_tree();
        } else {
            double mass = 0.0;
            for (int i = 0; i < n_src; ++i) mass += a[i];
            started = S.init_basis_checked(*warm, 1e-13 * (mass + 1.0));
            if (!started) S.reset_tree();
        }
    }
    if (!started) S.init_star(a, b);
    if (candidates) S.set_candidates(*candidates);
    int64_t piv = 0;
    const int64_t recentre_every = std::max<int64_t>(256, S.V);
    for (;;) {
        double rc;
        const int64_t e = S.sparse ? S.find_entering_sparse(&rc) : S.find_entering(&rc);
        if (e < 0) {
            // sparse pricing: optimal over the candidates; a full scan decides
            // (on re-centred potentials: the potentials of a tree that still
            // holds artificial arcs sit near the artificial cost, and their
            // rounding would hide every row from the separable row filter)
            if (S.sparse) {
                S.recentre();
                if (S.broken) return QWB_ERR_NOT_CONVERGED;
                const int64_t added = S.add_violators();
                if (S.bad_cost) return QWB_ERR_INVALID_ARG;
                if (added > 0) continue;
            }
            break;
        }
        if (++piv > max_pivots) return QWB_ERR_NOT_CONVERGED;
        S.pivot(e);
        if (S.broken) return QWB_ERR_NOT_CONVERGED;
        if (piv % recentre_every == 0) S.recentre();
        if (S.broken) return QWB_ERR_NOT_CONVERGED;
    }
    S.recompute_flows();
    if (S.broken) return QWB_ERR_NOT_CONVERGED;
    double mass = 0.0;
    for (int i = 0; i < n_src; ++i) mass += a[i];
    for (int v = 0; v < S.n + S.m; ++v)
        if (S.pred[v] >= NM && S.flow[v] > 1e-9 * std::max(1.0, mass)) return QWB_ERR_NOT_CONVERGED;
    if (basis_out) {
        basis_out->parent.assign(S.parent.begin(), S.parent.end() - 1);
        basis_out->pred.assign(S.pred.begin(), S.pred.end() - 1);
        basis_out->up.assign(S.up.begin(), S.up.end() - 1);
        basis_out->valid = true;
    }
    // plan (CSR) from the real tree arcs with positive flow: counted per row,
    // placed, then each row's few entries put in column order
    out.rowptr.assign(n_src + 1, 0);
    for (int v = 0; v < S.n + S.m; ++v)
        if (S.pred[v] < NM && S.flow[v] > 0.0) out.rowptr[S.pred[v] / n_dst + 1]++;
    for (int i = 0; i < n_src; ++i) out.rowptr[i + 1] += out.rowptr[i];
    const int nnz = out.rowptr[n_src];
    out.col.resize(nnz);
    out.val.resize(nnz);
    {
        std::vector<int32_t> cur(out.rowptr.begin(), out.rowptr.end() - 1);
        for (int v = 0; v < S.n + S.m; ++v) {
            const int64_t arc = S.pred[v];
            if (arc < NM && S.flow[v] > 0.0) {
                const int pos = cur[arc / n_dst]++;
                out.col[pos] = (int32_t)(arc % n_dst);
                out.val[pos] = S.flow[v];
            }
        }
    }
    double obj = 0.0;
    for (int i = 0; i < n_src; ++i) {
        const int e0 = out.rowptr[i], e1 = out.rowptr[i + 1];
        for (int e = e0 + 1; e < e1; ++e)             // insertion sort by column (distinct)
            for (int f = e; f > e0 && out.col[f - 1] > out.col[f]; --f) {
                std::swap(out.col[f - 1], out.col[f]);
                std::swap(out.val[f - 1], out.val[f]);
            }
        for (int e = e0; e < e1; ++e) obj += out.val[e] * cst(i, out.col[e]);
    }
    out.obj = obj;
    // potentials: f_i = pot[i] shifted to a zero midrange (a warm start can
    // leave every potential offset by a multiple of the artificial arc cost,
    // and sums of large offset terms would lose the digits that matter; the
    // dual objective does not change, the masses being equal); then exact
    // dual feasibility by c-transforms
    out.f.assign(n_src, 0.0);
    out.g.assign(n_dst, std::numeric_limits<double>::infinity());
    double f_lo = std::numeric_limits<double>::infinity(), f_hi = -f_lo;
    for (int i = 0; i < n_src; ++i) { f_lo = std::min(f_lo, S.pot[i]); f_hi = std::max(f_hi, S.pot[i]); }
    const double shift = n_src > 0 ? 0.5 * (f_lo + f_hi) : 0.0;
    for (int i = 0; i < n_src; ++i) out.f[i] = S.pot[i] - shift;
    double* g = out.g.data();
    if (!exact_dual) {
        // the tree potentials as they are: f_i + g_j = C_ij on the tree arcs,
        // <= C_ij + eps elsewhere (optimality up to the pricing tolerance)
        for (int j = 0; j < n_dst; ++j) g[j] = -S.pot[n_src + j] + shift;
        out.pivots = piv;
        return QWB_OK;
    }
    if constexpr (std::is_same<Cost, GridCost>::value) {
        if (cst.separable) {
            // separable grid costs c = A(|i1 - j1|) + B(|i2 - j2|): each
            // transform by two 1-D min-plus passes, O(ns^3) (the values may
            // differ from the direct minima by rounding only)
            const int ns = cst.ns;
            const double* tb = cst.tab;                   // A(d) = tb[d * ns], B(d) = tb[d]
            const double* refl0 = cst.refl + (ns - 1);   // refl0[x] = B(|x|), |x| < ns
            std::vector<double> T((size_t)ns * ns), src(n_src);
            auto transform = [&](const double* h, double* outv) {
                // outv[j1, j2] = min_{i1, i2} A(|i1 - j1|) + B(|i2 - j2|) - h[i1, i2],
                // each pass as element-wise minima over contiguous rows
                for (int i1 = 0; i1 < ns; ++i1) {
                    double* Ti = T.data() + (size_t)i1 * ns;
                    std::fill(Ti, Ti + ns, HUGE_VAL);
                    for (int i2 = 0; i2 < ns; ++i2)
                        S.min_plus_row(Ti, refl0 - i2, -h[i1 * ns + i2], ns);   // B(|j2 - i2|) - h
                }
                for (int j1 = 0; j1 < ns; ++j1) {
                    double* o = outv + (size_t)j1 * ns;
                    std::fill(o, o + ns, HUGE_VAL);
                    for (int i1 = 0; i1 < ns; ++i1)
                        S.min_plus_row(o, T.data() + (size_t)i1 * ns, tb[(size_t)std::abs(i1 - j1) * ns], ns);
                }
            };
            transform(out.f.data(), g);
            transform(g, src.data());
            out.f.swap(src);
            out.pivots = piv;
            return QWB_OK;
        }
    }
    // g = f^c, then f = g^c, row by row; each row is walked as runs of
    // contiguous costs (one run per grid row for table costs) with four
    // independent min chains in the reduction
    std::vector<double> crow(n_dst);
    for (int i = 0; i < n_src; ++i) {
        S.row_costs(i, crow.data());
        const double fi = out.f[i];
        const double* c = crow.data();
        for (int j = 0; j < n_dst; ++j) {
            const double v = c[j] - fi;
            g[j] = v < g[j] ? v : g[j];
        }
    }
    std::vector<double> mg(n_dst);
    for (int j = 0; j < n_dst; ++j) mg[j] = -g[j];
    for (int i = 0; i < n_src; ++i) {
        S.row_costs(i, crow.data());
        out.f[i] = S.run_min(crow.data(), mg.data(), n_dst);
    }
    out.pivots = piv;
    return QWB_OK;
}

bool check_masses(int32_t n_src, int32_t n_dst, const double* a, const double* b) {
    for (int i = 0; i < n_src; ++i) if (!(a[i] >= 0.0) || !std::isfinite(a[i])) return false;
    for (int j = 0; j < n_dst; ++j) if (!(b[j] >= 0.0) || !std::isfinite(b[j])) return false;
    return true;
}

}  // namespace

int network_simplex(int32_t n_src, int32_t n_dst, const double* C, const double* a,
                    const double* b, NSSolution& out, int64_t max_pivots, const NSBasis* warm,
                    NSBasis* basis_out, const std::vector<int64_t>* candidates, bool exact_dual,
                    double cost_bound) {
    if (n_src <= 0 || n_dst <= 0 || !C || !a || !b) return QWB_ERR_INVALID_ARG;
    const int64_t NM = (int64_t)n_src * n_dst;
    if (!check_masses(n_src, n_dst, a, b)) return QWB_ERR_INVALID_ARG;
    if (candidates)
        for (int64_t a_ : *candidates)
            if (a_ < 0 || a_ >= NM) return QWB_ERR_INVALID_ARG;
    if (candidates && cost_bound >= 0.0 && std::isfinite(cost_bound)) {
        // the entries are checked by the full scans of the sparse pricing
        // (every one is read at least once, by the last scan)
        for (int64_t a_ : *candidates)
            if (!(C[a_] >= 0.0) || !(C[a_] <= cost_bound)) return QWB_ERR_INVALID_ARG;
        if (warm && warm->valid && (int64_t)warm->pred.size() == (int64_t)n_src + n_dst)
            for (int64_t a_ : warm->pred)          // the starting tree's real arcs
                if (a_ >= 0 && a_ < NM && (!(C[a_] >= 0.0) || !(C[a_] <= cost_bound)))
                    return QWB_ERR_INVALID_ARG;
        return solve(n_src, n_dst, DenseCost{C, n_dst}, cost_bound, a, b, out, max_pivots, warm, basis_out,
                     candidates, exact_dual, cost_bound);
    }
    // one pass: the maximum, and whether every entry is finite and non-negative
    double maxc = 0.0;
    bool ok = true;
    for (int64_t k = 0; k < NM; ++k) {
        ok &= (C[k] >= 0.0) & (C[k] <= std::numeric_limits<double>::max());
        maxc = C[k] > maxc ? C[k] : maxc;
    }
    if (!ok) return QWB_ERR_INVALID_ARG;
    return solve(n_src, n_dst, DenseCost{C, n_dst}, maxc, a, b, out, max_pivots, warm, basis_out,
                 candidates, exact_dual);
}

namespace {
constexpr int kMultiscaleMin = 16;   // coarse-to-fine from this grid side up (even sides)
// fine cells added around the children of each coarse target (a wider set
// lets more poor arcs enter early and costs more pivots than it saves)
constexpr int kCandHalo = 0;

int grid_solve(int32_t n_side, const double* tab, const double* a, const double* b, NSSolution& out,
               int64_t max_pivots, NSBasis* basis_out, const NSBasis* warm);

// Candidate arcs from the solution of the half-resolution problem: every
// (fine source, fine sink) pair whose parents are joined by the coarse plan.
// A feasible starting tree for the fine problem from the half-resolution
// plan sh: each coarse arc's flow F_KL is split over the children of L by a
// north-west corner pass per coarse sink (the arcs into L against the
// children's masses), then each coarse source K splits those pieces over its
// own children by a second pass.  Both passes conserve mass, so the fine
// flow has the fine marginals up to rounding; its positive arcs form a
// forest, and each component hangs from the root by the artificial arc of
// one of its sinks (zero flow, pointing away from the root).  start.valid
// stays false when an arc would close a cycle.
void expand_plan(int32_t n_side, const double* a, const double* b, const NSSolution& sh, NSBasis& start) {
    const int h = n_side / 2, Mh = h * h, M = n_side * n_side;
    start.valid = false;
    auto child = [&](int K, int c) { return (2 * (K / h) + c / 2) * n_side + 2 * (K % h) + c % 2; };
    const int nnz = (int)sh.col.size();
    // arcs into each coarse sink (CSC order: sources in increasing order)
    std::vector<int> cptr(Mh + 1, 0), cidx(nnz);
    for (int e = 0; e < nnz; ++e) cptr[sh.col[e] + 1]++;
    for (int L = 0; L < Mh; ++L) cptr[L + 1] += cptr[L];
    {
        std::vector<int> cur(cptr.begin(), cptr.end() - 1);
        for (int K = 0; K < Mh; ++K)
            for (int e = sh.rowptr[K]; e < sh.rowptr[K + 1]; ++e) cidx[cur[sh.col[e]]++] = e;
    }
    // pass 1: piece (fine sink w, amount) lists per coarse arc, at most 4 each
    std::vector<int> pw((size_t)nnz * 4, -1);
    std::vector<double> px((size_t)nnz * 4, 0.0);
    std::vector<int> pn(nnz, 0);
    for (int L = 0; L < Mh; ++L) {
        double rb[4];
        for (int c = 0; c < 4; ++c) rb[c] = b[child(L, c)];
        int c = 0;
        for (int t = cptr[L]; t < cptr[L + 1]; ++t) {
            const int e = cidx[t];
            double rem = sh.val[e];
            while (rem > 0.0 && c < 4) {
                if (rb[c] <= 0.0) { ++c; continue; }
                const double x = rem < rb[c] ? rem : rb[c];
                pw[(size_t)e * 4 + pn[e]] = child(L, c);
                px[(size_t)e * 4 + pn[e]] = x;
                ++pn[e];
                rem -= x;
                rb[c] -= x;
                if (rb[c] <= 0.0) ++c;
            }
        }
    }
    // pass 2: fine arcs (u, w, amount) per coarse source
    std::vector<int> au, aw;
    for (int K = 0; K < Mh; ++K) {
        double ra[4];
        for (int c = 0; c < 4; ++c) ra[c] = a[child(K, c)];
        int c = 0;
        for (int e = sh.rowptr[K]; e < sh.rowptr[K + 1]; ++e)
            for (int q = 0; q < pn[e]; ++q) {
                double rem = px[(size_t)e * 4 + q];
                const int w = pw[(size_t)e * 4 + q];
                while (rem > 0.0 && c < 4) {
                    if (ra[c] <= 0.0) { ++c; continue; }
                    const double x = rem < ra[c] ? rem : ra[c];
                    au.push_back(child(K, c));
                    aw.push_back(w);
                    rem -= x;
                    ra[c] -= x;
                    if (ra[c] <= 0.0) ++c;
                }
            }
    }
    // spanning forest of those arcs (sources 0..M-1, sinks M..2M-1)
    const int Vn = 2 * M;
    std::vector<int> uf(Vn);
    for (int v = 0; v < Vn; ++v) uf[v] = v;
    auto find = [&](int v) { while (uf[v] != v) { uf[v] = uf[uf[v]]; v = uf[v]; } return v; };
    std::vector<int> adj_ptr(Vn + 1, 0), adj((size_t)au.size() * 2);
    for (size_t t = 0; t < au.size(); ++t) {
        const int x = find(au[t]), y = find(M + aw[t]);
        if (x == y) return;                          // a cycle: no starting tree
        uf[x] = y;
        adj_ptr[au[t] + 1]++;
        adj_ptr[M + aw[t] + 1]++;
    }
    for (int v = 0; v < Vn; ++v) adj_ptr[v + 1] += adj_ptr[v];
    {
        std::vector<int> cur(adj_ptr.begin(), adj_ptr.end() - 1);
        for (size_t t = 0; t < au.size(); ++t) {
            adj[cur[au[t]]++] = M + aw[t];
            adj[cur[M + aw[t]]++] = au[t];
        }
    }
    start.parent.assign(Vn, -1);
    start.pred.assign(Vn, -1);
    start.up.assign(Vn, 0);
    const int root = Vn;
    const int64_t NM = (int64_t)M * M;
    std::vector<int> queue;
    queue.reserve(Vn);
    std::vector<char> seen(Vn, 0);
    // components hang from a sink (or, alone, from themselves): sinks first;
    // a component's sink is the one nearest the middle of a longest path
    // (two breadth-first walks), which keeps the tree shallow
    std::vector<int> dist(Vn, -1), from(Vn, -1), comp;
    auto bfs_far = [&](int s0) {
        comp.clear();
        comp.push_back(s0);
        dist[s0] = 0; from[s0] = -1;
        int far = s0;
        for (size_t qi = 0; qi < comp.size(); ++qi) {
            const int v = comp[qi];
            if (dist[v] > dist[far]) far = v;
            for (int t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t)
                if (dist[adj[t]] < 0) { dist[adj[t]] = dist[v] + 1; from[adj[t]] = v; comp.push_back(adj[t]); }
        }
        for (int v : comp) dist[v] = -1;
        return far;
    };
    for (int pass = 0; pass < 2; ++pass)
        for (int r0 = 0; r0 < M; ++r0) {
            int r = pass == 0 ? M + r0 : r0;
            if (seen[r]) continue;
            if (pass == 0 && adj_ptr[r + 1] > adj_ptr[r]) {
                const int f = bfs_far(r);
                const int g = bfs_far(f);               // from[] now leads from g back to f
                int len = 0;
                for (int v = g; v >= 0; v = from[v]) ++len;
                int c = g;
                for (int k = 0; k < len / 2; ++k) c = from[c];
                if (c < M) c = adj[adj_ptr[c]];         // a source: one of its sinks
                r = c;
            }
            seen[r] = 1;
            start.parent[r] = root;
            start.pred[r] = NM + r;
            start.up[r] = (r < M && a[r] > 0.0) ? 1 : 0;   // the artificial arc's direction
            queue.clear();
            queue.push_back(r);
            for (size_t qi = 0; qi < queue.size(); ++qi) {
                const int v = queue[qi];
                for (int t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t) {
                    const int w = adj[t];
                    if (seen[w]) continue;
                    seen[w] = 1;
                    start.parent[w] = v;
                    if (w < M) {                      // source child, sink parent: arc w -> v
                        start.pred[w] = (int64_t)w * M + (v - M);
                        start.up[w] = 1;
                    } else {                          // sink child, source parent: arc v -> w
                        start.pred[w] = (int64_t)v * M + (w - M);
                        start.up[w] = 0;
                    }
                    queue.push_back(w);
                }
            }
        }
    start.valid = true;
}

int grid_candidates(int32_t n_side, const double* tab, const double* a, const double* b,
                    std::vector<int64_t>& cand, NSBasis* start) {
    const int h = n_side / 2, Mh = h * h, M = n_side * n_side;
    std::vector<double> ah(Mh, 0.0), bh(Mh, 0.0), tabh((size_t)Mh);
    for (int r = 0; r < n_side; ++r)
        for (int c = 0; c < n_side; ++c) {
            ah[(r / 2) * h + c / 2] += a[r * n_side + c];
            bh[(r / 2) * h + c / 2] += b[r * n_side + c];
        }
    for (int d1 = 0; d1 < h; ++d1)
        for (int d2 = 0; d2 < h; ++d2) tabh[(size_t)d1 * h + d2] = tab[(size_t)(2 * d1) * n_side + 2 * d2];
    NSSolution sh;
    const int st = grid_solve(h, tabh.data(), ah.data(), bh.data(), sh, -1, nullptr, nullptr);
    if (st) return st;
    if (start) expand_plan(n_side, a, b, sh, *start);
    cand.clear();
    for (int K = 0; K < Mh; ++K)
        for (int e = sh.rowptr[K]; e < sh.rowptr[K + 1]; ++e) {
            const int L = sh.col[e];
            const int K1 = K / h, K2 = K % h, L1 = L / h, L2 = L % h;
            for (int u = 0; u < 4; ++u) {
                const int k = (2 * K1 + u / 2) * n_side + 2 * K2 + u % 2;
                for (int r = 2 * L1 - kCandHalo; r <= 2 * L1 + 1 + kCandHalo; ++r)
                    for (int c = 2 * L2 - kCandHalo; c <= 2 * L2 + 1 + kCandHalo; ++c)
                        if (r >= 0 && c >= 0 && r < n_side && c < n_side)
                            cand.push_back((int64_t)k * M + r * n_side + c);
            }
        }
    return QWB_OK;
}

int grid_solve(int32_t n_side, const double* tab, const double* a, const double* b, NSSolution& out,
               int64_t max_pivots, NSBasis* basis_out, const NSBasis* warm) {
    double maxc = 0.0;
    for (int k = 0; k < n_side * n_side; ++k) maxc = std::max(maxc, tab[k]);
    const int32_t M = n_side * n_side;
    std::vector<double> refl((size_t)n_side * (2 * n_side - 1));
    for (int d1 = 0; d1 < n_side; ++d1)
        for (int d2 = -(n_side - 1); d2 < n_side; ++d2)
            refl[(size_t)d1 * (2 * n_side - 1) + n_side - 1 + d2] = tab[d1 * n_side + std::abs(d2)];
    std::vector<int64_t> cand;
    NSBasis start;
    const bool ms = !(warm && warm->valid) && n_side >= kMultiscaleMin && n_side % 2 == 0;
    if (ms) {
        const int st = grid_candidates(n_side, tab, a, b, cand, &start);
        if (st) return st;
    }
    bool sep = true;
    for (int d1 = 0; d1 < n_side && sep; ++d1)
        for (int d2 = 0; d2 < n_side; ++d2)
            if (tab[(size_t)d1 * n_side + d2] != tab[(size_t)d1 * n_side] + tab[d2]) { sep = false; break; }
    if (ms && start.valid)
        return solve(M, M, GridCost{tab, n_side, refl.data(), sep}, maxc, a, b, out, max_pivots, &start,
                     basis_out, &cand, true, -1.0, true);
    return solve(M, M, GridCost{tab, n_side, refl.data(), sep}, maxc, a, b, out, max_pivots, warm, basis_out,
                 ms ? &cand : nullptr);
}
}  // namespace

int network_simplex_grid(int32_t n_side, const double* tab, const double* a, const double* b,
                         NSSolution& out, int64_t max_pivots, NSBasis* basis_out, const NSBasis* warm) {
    if (n_side <= 0 || !tab || !a || !b) return QWB_ERR_INVALID_ARG;
    double maxc = 0.0;
    for (int k = 0; k < n_side * n_side; ++k) {
        if (!(tab[k] >= 0.0) || !std::isfinite(tab[k])) return QWB_ERR_INVALID_ARG;
        maxc = std::max(maxc, tab[k]);
    }
    const int32_t M = n_side * n_side;
    if (!check_masses(M, M, a, b)) return QWB_ERR_INVALID_ARG;
    (void)maxc;
    return grid_solve(n_side, tab, a, b, out, max_pivots, basis_out, warm);
}

}  // namespace qwb
