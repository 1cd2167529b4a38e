/*
 * oracle/ssp.c -- exact discrete Kantorovich solver for the test oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code with the CUDA library.
 *
 * Solves the Kantorovich problem of Sec. 2.1 (L_C(mu, nu) = min <pi, C> over
 * couplings pi with pi 1 = a, pi^T 1 = b) and its dual (max <f,a> + <g,b>
 * subject to f_i + g_j <= C_ij), in plain FP64, by successive shortest paths:
 * a primal-dual method that is a different algorithm from the network simplex
 * the library ships, so that agreement between the two is a real check.
 *
 * Method (textbook successive shortest paths with node potentials):
 *   residual graph: forward arc i->j for every (source i, sink j), cost C_ij,
 *   unbounded capacity; backward arc j->i while x_ij > 0, cost -C_ij,
 *   capacity x_ij.  Node potentials pot[] keep every residual reduced cost
 *   rc(u,v) = c(u,v) - pot[u] + pot[v] non-negative.  Each round runs a
 *   dense Dijkstra from all sources with remaining excess, stops at the first
 *   sink with remaining deficit, lowers the potentials by the truncated
 *   distances and augments along the path by the largest feasible amount.
 *   At the end f_i = pot[i], g_j = -pot[n + j]:  C_ij - f_i - g_j = rc >= 0,
 *   with equality wherever x_ij > 0 (complementary slackness).
 *
 * Costs must be non-negative (so zero potentials are a valid start).
 * Returns 0 on success, 1 on bad arguments, 2 when the round cap is reached.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

int oracle_ssp(int n, int m, const double *C, const double *a, const double *b,
               double *plan, double *f, double *g, double *obj, int *rounds_out)
{
    if (n <= 0 || m <= 0 || !C || !a || !b || !plan || !f || !g || !obj) return 1;
    for (long k = 0; k < (long)n * m; ++k)
        if (!(C[k] >= 0.0) || !isfinite(C[k])) return 1;

    const int V = n + m;
    double *pot = calloc((size_t)V, sizeof(double));
    double *dist = malloc((size_t)V * sizeof(double));
    double *exc = malloc((size_t)n * sizeof(double));
    double *def = malloc((size_t)m * sizeof(double));
    int *prev = malloc((size_t)V * sizeof(int));
    char *done = malloc((size_t)V);
    if (!pot || !dist || !exc || !def || !prev || !done) {
        free(pot); free(dist); free(exc); free(def); free(prev); free(done);
        return 1;
    }
    memcpy(exc, a, (size_t)n * sizeof(double));
    memcpy(def, b, (size_t)m * sizeof(double));
    memset(plan, 0, (size_t)n * m * sizeof(double));

    const long max_rounds = 200L * V + 1000;
    long rounds = 0;
    int status = 0;
    for (;;) {
        int any_exc = 0, any_def = 0;
        for (int i = 0; i < n; ++i) if (exc[i] > 0.0) { any_exc = 1; break; }
        for (int j = 0; j < m; ++j) if (def[j] > 0.0) { any_def = 1; break; }
        if (!any_exc || !any_def) break;
        if (++rounds > max_rounds) { status = 2; break; }

        /* Dijkstra from every source that still has excess. */
        for (int v = 0; v < V; ++v) { dist[v] = DBL_MAX; prev[v] = -1; done[v] = 0; }
        for (int i = 0; i < n; ++i) if (exc[i] > 0.0) dist[i] = 0.0;
        int target = -1;
        for (;;) {
            int u = -1;
            double du = DBL_MAX;
            for (int v = 0; v < V; ++v)
                if (!done[v] && dist[v] < du) { du = dist[v]; u = v; }
            if (u < 0) break;              /* nothing reachable is left */
            done[u] = 1;
            if (u >= n && def[u - n] > 0.0) { target = u; break; }
            if (u < n) {                   /* source: forward arcs to every sink */
                const double *Ci = C + (long)u * m;
                for (int j = 0; j < m; ++j) {
                    if (done[n + j]) continue;
                    double rc = Ci[j] - pot[u] + pot[n + j];
                    if (rc < 0.0) rc = 0.0;
                    double nd = du + rc;
                    if (nd < dist[n + j]) { dist[n + j] = nd; prev[n + j] = u; }
                }
            } else {                       /* sink: backward arcs along positive flow */
                int j = u - n;
                for (int i = 0; i < n; ++i) {
                    if (done[i] || plan[(long)i * m + j] <= 0.0) continue;
                    double rc = -(C[(long)i * m + j] - pot[i] + pot[u]);
                    if (rc < 0.0) rc = 0.0;
                    double nd = du + rc;
                    if (nd < dist[i]) { dist[i] = nd; prev[i] = u; }
                }
            }
        }
        if (target < 0) break;             /* remaining excess cannot reach any deficit */

        const double D = dist[target];
        for (int v = 0; v < V; ++v) pot[v] -= (dist[v] < D ? dist[v] : D);

        /* Walk the path back to its source and find the bottleneck. */
        double delta = def[target - n];
        int v = target;
        while (prev[v] >= 0) {
            int u = prev[v];
            if (u >= n) {                  /* u sink -> v source is a backward arc */
                double x = plan[(long)v * m + (u - n)];
                if (x < delta) delta = x;
            }
            v = u;
        }
        const int src = v;
        if (exc[src] < delta) delta = exc[src];

        /* Augment.  Quantities equal to delta are set to exactly zero. */
        v = target;
        while (prev[v] >= 0) {
            int u = prev[v];
            if (u < n) {
                plan[(long)u * m + (v - n)] += delta;
            } else {
                double *x = &plan[(long)v * m + (u - n)];
                *x = (*x == delta) ? 0.0 : *x - delta;
                if (*x < 0.0) *x = 0.0;
            }
            v = u;
        }
        exc[src] = (exc[src] == delta) ? 0.0 : exc[src] - delta;
        def[target - n] = (def[target - n] == delta) ? 0.0 : def[target - n] - delta;
        if (exc[src] < 0.0) exc[src] = 0.0;
        if (def[target - n] < 0.0) def[target - n] = 0.0;
    }

    double s = 0.0;
    for (long k = 0; k < (long)n * m; ++k) s += plan[k] * C[k];
    *obj = s;
    for (int i = 0; i < n; ++i) f[i] = pot[i];
    for (int j = 0; j < m; ++j) g[j] = -pot[n + j];
    if (rounds_out) *rounds_out = (int)rounds;
    free(pot); free(dist); free(exc); free(def); free(prev); free(done);
    return status;
}
