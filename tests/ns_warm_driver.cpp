// Test driver of the library's host exact solver (no GPU): the two solves of
// one pair of a batch, in the batch's order.  The grid solve of the centre
// cost C~ (offset table) gives a plan and its final basis; the dense solve of
// the measure-weighted cost C-bar (Sec. 3.2) starts from that basis, prices
// the 3 x 3 block neighbourhoods of the C~ plan's targets first and, when
// bound >= 0, checks the entries of C-bar only in its full scans against that
// bound.  Input (binary, native endianness): int32 n_side; double tab[ns^2],
// a[M], b[M], C[M * M], bound.  Output: "status obj nnz row_err col_err".
#include <cmath>
#include <cstdio>
#include <vector>

#include "../paper_2506_00976_gb300/csrc/netsimplex.h"

namespace qwb {
int64_t fault_param(const char*, int64_t def) { return def; }
}

int main(int argc, char** argv) {
    if (argc != 2) return 2;
    FILE* fh = std::fopen(argv[1], "rb");
    if (!fh) return 2;
    int32_t ns = 0;
    bool ok = std::fread(&ns, 4, 1, fh) == 1 && ns > 0 && ns <= 64;
    const int M = ok ? ns * ns : 0;
    std::vector<double> tab((size_t)ns * ns), a(M), b(M), C((size_t)M * M);
    double bound = -1.0;
    ok = ok && std::fread(tab.data(), 8, tab.size(), fh) == tab.size() &&
         std::fread(a.data(), 8, M, fh) == (size_t)M && std::fread(b.data(), 8, M, fh) == (size_t)M &&
         std::fread(C.data(), 8, C.size(), fh) == C.size() && std::fread(&bound, 8, 1, fh) == 1;
    std::fclose(fh);
    if (!ok) return 2;
    qwb::NSSolution sol;
    qwb::NSBasis basis;
    int st = qwb::network_simplex_grid(ns, tab.data(), a.data(), b.data(), sol, -1, &basis, nullptr);
    if (st) { std::printf("%d nan 0 nan nan\n", st); return 0; }
    std::vector<int64_t> cand;
    for (int k = 0; k < M; ++k)
        for (int e = sol.rowptr[k]; e < sol.rowptr[k + 1]; ++e) {
            const int l1 = sol.col[e] / ns, l2 = sol.col[e] % ns;
            for (int d1 = -1; d1 <= 1; ++d1)
                for (int d2 = -1; d2 <= 1; ++d2) {
                    const int r1 = l1 + d1, r2 = l2 + d2;
                    if (r1 >= 0 && r2 >= 0 && r1 < ns && r2 < ns) cand.push_back((int64_t)k * M + r1 * ns + r2);
                }
        }
    qwb::NSSolution sb;
    st = qwb::network_simplex(M, M, C.data(), a.data(), b.data(), sb, -1, &basis, nullptr, &cand, false, bound);
    if (st) { std::printf("%d nan 0 nan nan\n", st); return 0; }
    std::vector<double> rs(M, 0.0), cs(M, 0.0);
    for (int k = 0; k < M; ++k)
        for (int e = sb.rowptr[k]; e < sb.rowptr[k + 1]; ++e) { rs[k] += sb.val[e]; cs[sb.col[e]] += sb.val[e]; }
    double re = 0.0, ce = 0.0;
    for (int k = 0; k < M; ++k) { re = std::fmax(re, std::fabs(rs[k] - a[k])); ce = std::fmax(ce, std::fabs(cs[k] - b[k])); }
    std::printf("%d %.17g %d %.3g %.3g\n", st, sb.obj, (int)sb.col.size(), re, ce);
    return 0;
}
