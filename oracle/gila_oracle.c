/*
 * FP64 CPU oracle of the GiLA layout step -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct restatement of what the paper (Arleo,
 * Didimo, Liotta, Montecchiani: "A Distributed Force-Directed Algorithm on
 * Giraph: Design and Experiments", arXiv 1606.02162) computes, used only to
 * check the CUDA library. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it; the product library never does, and the two
 * share no code.
 *
 * What it computes, by section of the paper:
 *   Section 4.5  N_v(k) = vertices at graph distance 1..k from v, built here
 *                by a textbook breadth-first search from every v and stored
 *                as ascending vertex ids (v itself excluded).
 *   Section 3.1  F(u) = sum over edges (u,v) of f^a_uv + sum over repelling
 *                vertices v of f^r_uv, with |f^a| = delta^p / d and
 *                |f^r| = d^2 / delta^q, attraction pulling u toward v and
 *                repulsion pushing u away from v. In GiLA the repelling set
 *                of u is N_u(k) (Section 4.5), and adjacent vertices give
 *                both terms (Section 4.5, second superstep).
 *   Section 3.1  The displacement of u is F(u) cut to length t (the
 *                temperature) when longer; t falls over the iterations.
 *   Section 4.5  All vertices move together after every force is known
 *                (positions change only when no message is left).
 *   Section 4.3  Pruning: degree-one vertices are removed before the layout;
 *                each kept vertex remembers how many it lost.
 *   Section 4.6  Reinsertion: the removed vertices are put back on a small
 *                circle around their neighbour; during the layout a vertex
 *                repels with a weight that grows with that number.
 *
 * Readings where the paper is silent (kept identical on the CUDA side):
 *   - a vertex does not repel itself; a pair at distance 0 contributes 0;
 *   - a zero resultant force gives a zero displacement;
 *   - temperature schedules: linear t_i = t0 (iters - i) / iters, or the
 *     geometric form of Section 5.1, t_i = t0 * 0.93^i;
 *   - the attractive and repulsive sums are formed separately in the order
 *     of the CSR rows and then added;
 *   - pruning is one pass (vertices that reach degree one only after it stay);
 *     a single-edge component keeps its smaller id; the repulsion weight of
 *     a kept vertex is 1 + (number of removed neighbours), since a weight
 *     of zero would switch off the repulsion of every vertex without
 *     removed neighbours;
 *   - reinsertion radius 0.2 * shortest incident edge of the pruned drawing
 *     (0.2 * d when there is none); removed neighbours evenly spaced on the
 *     circle, rotated to stay off the vertex's edges (see oracle_reinsert).
 *
 * Every loop over u is independent, so the OpenMP split over vertices does
 * not change any result: the per-vertex summation order is fixed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Breadth-first search from src to depth k (Section 4.5: N_v(k) holds the
 * vertices whose graph-theoretic distance from v is at most k).
 * dist[] must hold -1 for every vertex on entry and is restored on exit.
 * queue[] receives the visited vertices in BFS order, src first.
 * Returns the number of visited vertices, src included.
 */
static int64_t bfs_ball(const int64_t *row, const int32_t *col, int k,
                        int32_t src, int32_t *dist, int32_t *queue)
{
    int64_t head = 0, tail = 0;
    queue[tail++] = src;
    dist[src] = 0;
    while (head < tail) {
        int32_t w = queue[head++];
        if (dist[w] == k) continue; /* do not expand beyond depth k */
        for (int64_t e = row[w]; e < row[w + 1]; ++e) {
            int32_t x = col[e];
            if (dist[x] < 0) {
                dist[x] = dist[w] + 1;
                queue[tail++] = x;
            }
        }
    }
    return tail;
}

static void reset_dist(int32_t *dist, const int32_t *queue, int64_t cnt)
{
    for (int64_t i = 0; i < cnt; ++i) dist[queue[i]] = -1;
}

/* |N_v(k)| for every v; returns the total (nnz of the k-hop lists). */
int64_t oracle_khop_count(int64_t n, const int64_t *row, const int32_t *col,
                          int k, int64_t *counts)
{
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) dist[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t v = 0; v < n; ++v) {
            int64_t cnt = bfs_ball(row, col, k, (int32_t)v, dist, queue);
            counts[v] = cnt - 1;
            total += cnt - 1;
            reset_dist(dist, queue, cnt);
        }
        free(dist);
        free(queue);
    }
    return total;
}

/* Sorted N_v(k) rows into kcol, at offsets krow (krow[v+1]-krow[v] must
 * equal |N_v(k)|). Returns 0, or -1 when a row length disagrees. */
int oracle_khop_fill(int64_t n, const int64_t *row, const int32_t *col, int k,
                     const int64_t *krow, int32_t *kcol)
{
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) dist[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t v = 0; v < n; ++v) {
            int64_t cnt = bfs_ball(row, col, k, (int32_t)v, dist, queue);
            reset_dist(dist, queue, cnt);
            if (krow[v + 1] - krow[v] != cnt - 1) { bad = 1; continue; }
            int32_t *dst = kcol + krow[v];
            memcpy(dst, queue + 1, sizeof(int32_t) * (size_t)(cnt - 1));
            qsort(dst, (size_t)(cnt - 1), sizeof(int32_t), cmp_i32);
        }
        free(dist);
        free(queue);
    }
    return bad ? -1 : 0;
}

/*
 * N_v(k) for a chosen list of sources (for sampled checks of large graphs).
 * counts[i] = |N_{src[i]}(k)|. If out is not NULL the sorted rows are
 * written back to back in the order of src; out_cap bounds the total.
 * Returns the total written (or counted), or -1 if out_cap is too small.
 */
int64_t oracle_khop_rows(int64_t n, const int64_t *row, const int32_t *col, int k,
                         int64_t nsrc, const int64_t *src, int64_t *counts,
                         int32_t *out, int64_t out_cap)
{
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    int64_t off = 0;
    for (int64_t i = 0; i < nsrc; ++i) {
        int64_t cnt = bfs_ball(row, col, k, (int32_t)src[i], dist, queue);
        reset_dist(dist, queue, cnt);
        counts[i] = cnt - 1;
        if (out) {
            if (off + cnt - 1 > out_cap) { off = -1; break; }
            memcpy(out + off, queue + 1, sizeof(int32_t) * (size_t)(cnt - 1));
            qsort(out + off, (size_t)(cnt - 1), sizeof(int32_t), cmp_i32);
        }
        off += cnt - 1;
    }
    free(dist);
    free(queue);
    return off;
}

/* delta^e for a small non-negative integer e (Section 3.1: p and q are
 * integers). */
static double ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/*
 * Resultant force on u (Section 3.1 with the repelling set of Section 4.5):
 *   repulsion: for v in N_u(k): magnitude d^2 / delta^q along (x_u - x_v)/delta,
 *              times wt[v] when repulsion weights are given (wt != NULL)
 *   attraction: for v adjacent to u: magnitude delta^p / d along (x_v - x_u)/delta
 */
static void force_on(int64_t u, const int64_t *row, const int32_t *col,
                     const int64_t *krow, const int32_t *kcol, const double *wt,
                     const double *pos, double d, int p, int q, double *fx, double *fy)
{
    const double xu = pos[2 * u], yu = pos[2 * u + 1];
    double rx = 0.0, ry = 0.0, ax = 0.0, ay = 0.0;
    for (int64_t j = krow[u]; j < krow[u + 1]; ++j) {
        int32_t v = kcol[j];
        if (v == u) continue;
        double dx = xu - pos[2 * (int64_t)v], dy = yu - pos[2 * (int64_t)v + 1];
        double delta = sqrt(dx * dx + dy * dy);
        if (delta == 0.0) continue;
        double mag = d * d / ipow(delta, q);
        if (wt) mag *= wt[v];  /* Section 4.6: v repels with its own weight */
        rx += mag * (dx / delta);
        ry += mag * (dy / delta);
    }
    for (int64_t j = row[u]; j < row[u + 1]; ++j) {
        int32_t v = col[j];
        if (v == u) continue;
        double dx = pos[2 * (int64_t)v] - xu, dy = pos[2 * (int64_t)v + 1] - yu;
        double delta = sqrt(dx * dx + dy * dy);
        if (delta == 0.0) continue;
        double mag = ipow(delta, p) / d;
        ax += mag * (dx / delta);
        ay += mag * (dy / delta);
    }
    *fx = rx + ax;
    *fy = ry + ay;
}

/* F(u) for all u (sel == NULL) or for the nsel listed vertices; F is
 * interleaved (Fx, Fy). */
void oracle_forces_w(int64_t n, const int64_t *row, const int32_t *col,
                     const int64_t *krow, const int32_t *kcol, const double *wt,
                     const double *pos, double d, int p, int q, int64_t nsel,
                     const int64_t *sel, double *F)
{
    int64_t cnt = sel ? nsel : n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < cnt; ++i) {
        int64_t u = sel ? sel[i] : i;
        force_on(u, row, col, krow, kcol, wt, pos, d, p, q, &F[2 * i], &F[2 * i + 1]);
    }
}

void oracle_forces(int64_t n, const int64_t *row, const int32_t *col,
                   const int64_t *krow, const int32_t *kcol, const double *pos,
                   double d, int p, int q, int64_t nsel, const int64_t *sel, double *F)
{
    oracle_forces_w(n, row, col, krow, kcol, NULL, pos, d, p, q, nsel, sel, F);
}

/* Section 3.1: the move is the force, cut to length t when it is longer. */
static void capped(double fx, double fy, double t, double *dx, double *dy)
{
    double norm = sqrt(fx * fx + fy * fy);
    if (norm > t) {
        double s = (norm > 0.0) ? t / norm : 0.0;
        *dx = fx * s;
        *dy = fy * s;
    } else {
        *dx = fx;
        *dy = fy;
    }
}

/*
 * One synchronous iteration (Section 4.5): every F(u) is computed from the
 * positions at the start of the iteration, then all vertices move.
 * pos_out may not alias pos_in. disp (optional) receives the moves.
 */
void oracle_step_w(int64_t n, const int64_t *row, const int32_t *col,
                   const int64_t *krow, const int32_t *kcol, const double *wt,
                   const double *pos_in, double d, int p, int q, double t, double *pos_out,
                   double *disp)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t u = 0; u < n; ++u) {
        double fx, fy, mx, my;
        force_on(u, row, col, krow, kcol, wt, pos_in, d, p, q, &fx, &fy);
        capped(fx, fy, t, &mx, &my);
        pos_out[2 * u] = pos_in[2 * u] + mx;
        pos_out[2 * u + 1] = pos_in[2 * u + 1] + my;
        if (disp) {
            disp[2 * u] = mx;
            disp[2 * u + 1] = my;
        }
    }
}

void oracle_step(int64_t n, const int64_t *row, const int32_t *col,
                 const int64_t *krow, const int32_t *kcol, const double *pos_in,
                 double d, int p, int q, double t, double *pos_out, double *disp)
{
    oracle_step_w(n, row, col, krow, kcol, NULL, pos_in, d, p, q, t, pos_out, disp);
}

/* Temperature of iteration i (0-based) of `iters`.
 * schedule 0: linear from t0 down to 0, t_i = t0 (iters - i) / iters.
 * schedule 1: geometric, t_i = t0 * 0.93^i (Section 5.1). */
double oracle_temperature(int schedule, double t0, int i, int iters)
{
    if (schedule == 1) return t0 * pow(0.93, (double)i);
    return t0 * (double)(iters - i) / (double)iters;
}

/*
 * Default initial temperature when the caller gives none.
 * linear:    0.1 * sqrt(n)
 * geometric: sqrt(n * d / a), a = height / width of the bounding box of the
 *            initial placement (Section 5.1).
 */
double oracle_default_t0(int schedule, int64_t n, double d, const double *pos)
{
    if (schedule != 1) return 0.1 * sqrt((double)n);
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int64_t u = 0; u < n; ++u) {
        double x = pos[2 * u], y = pos[2 * u + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    double w = xmax - xmin, h = ymax - ymin;
    double a = (w > 0.0 && h > 0.0) ? h / w : 1.0;
    return sqrt((double)n * d / a);
}

/*
 * `iters` synchronous iterations from pos0 under the given schedule.
 * t0 <= 0 selects the default above. Writes the final placement to pos_out.
 * Returns 0, or -1 on allocation failure.
 */
int oracle_run_w(int64_t n, const int64_t *row, const int32_t *col,
                 const int64_t *krow, const int32_t *kcol, const double *wt,
                 const double *pos0, double d, int p, int q, int schedule, double t0,
                 int iters, double *pos_out)
{
    double *a = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double *b = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, pos0, sizeof(double) * 2 * (size_t)n);
    if (t0 <= 0.0) t0 = oracle_default_t0(schedule, n, d, pos0);
    for (int i = 0; i < iters; ++i) {
        double t = oracle_temperature(schedule, t0, i, iters);
        oracle_step_w(n, row, col, krow, kcol, wt, a, d, p, q, t, b, NULL);
        double *s = a; a = b; b = s;
    }
    memcpy(pos_out, a, sizeof(double) * 2 * (size_t)n);
    free(a);
    free(b);
    return 0;
}

int oracle_run(int64_t n, const int64_t *row, const int32_t *col,
               const int64_t *krow, const int32_t *kcol, const double *pos0,
               double d, int p, int q, int schedule, double t0, int iters,
               double *pos_out)
{
    return oracle_run_w(n, row, col, krow, kcol, NULL, pos0, d, p, q, schedule, t0, iters,
                        pos_out);
}

/*
 * Layout quality figures of a placement.
 *   out[0] edge-length mean over the undirected edges
 *   out[1] edge-length population standard deviation (two passes)
 *   out[2] coefficient of variation out[1] / out[0]
 *   out[3] repulsive total: sum over unordered pairs {u,v}, v in N_u(k), of d^2/delta^q
 *   out[4] attractive total: sum over undirected edges of delta^p / d
 *   out[5] ratio out[3] / out[4]
 * Pairs at distance 0 are left out of out[3] and out[4], as in the forces.
 */
void oracle_metrics(int64_t n, const int64_t *row, const int32_t *col,
                    const int64_t *krow, const int32_t *kcol, const double *pos,
                    double d, int p, int q, double *out)
{
    double sum = 0.0, att = 0.0, rep = 0.0;
    int64_t m = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t j = row[u]; j < row[u + 1]; ++j) {
            int64_t v = col[j];
            if (v <= u) continue;
            double dx = pos[2 * u] - pos[2 * v], dy = pos[2 * u + 1] - pos[2 * v + 1];
            double delta = sqrt(dx * dx + dy * dy);
            sum += delta;
            if (delta > 0.0) att += ipow(delta, p) / d;
            ++m;
        }
    }
    double mean = m ? sum / (double)m : 0.0;
    double var = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t j = row[u]; j < row[u + 1]; ++j) {
            int64_t v = col[j];
            if (v <= u) continue;
            double dx = pos[2 * u] - pos[2 * v], dy = pos[2 * u + 1] - pos[2 * v + 1];
            double delta = sqrt(dx * dx + dy * dy);
            var += (delta - mean) * (delta - mean);
        }
    }
    var = m ? var / (double)m : 0.0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t j = krow[u]; j < krow[u + 1]; ++j) {
            int64_t v = kcol[j];
            if (v <= u) continue;
            double dx = pos[2 * u] - pos[2 * v], dy = pos[2 * u + 1] - pos[2 * v + 1];
            double delta = sqrt(dx * dx + dy * dy);
            if (delta > 0.0) rep += d * d / ipow(delta, q);
        }
    }
    out[0] = mean;
    out[1] = sqrt(var);
    out[2] = mean > 0.0 ? out[1] / mean : 0.0;
    out[3] = rep;
    out[4] = att;
    out[5] = att > 0.0 ? rep / att : 0.0;
}

/*
 * Pruning (Section 4.3): every vertex with exactly one neighbour is removed
 * before the layout and remembered by the neighbour it hangs on. When both
 * ends of an edge have degree one (a component that is a single edge) only
 * the end with the larger id is removed, so that every removed vertex has a
 * kept anchor. Outputs, per original vertex v:
 *   anchor[v] = the neighbour of v if v is removed, else -1;
 *   w[v]      = number of removed neighbours of v (0 for removed vertices);
 *   newid[v]  = index of v among the kept vertices in ascending id order,
 *               or -1 if v is removed.
 * Returns the number of kept vertices.
 */
int64_t oracle_prune(int64_t n, const int64_t *row, const int32_t *col, int32_t *anchor,
                     int32_t *w, int32_t *newid)
{
    for (int64_t v = 0; v < n; ++v) {
        anchor[v] = -1;
        w[v] = 0;
    }
    for (int64_t v = 0; v < n; ++v) {
        if (row[v + 1] - row[v] != 1) continue;
        int32_t a = col[row[v]];
        int a_is_leaf = (row[(int64_t)a + 1] - row[a] == 1);
        if (a_is_leaf && a > v) continue; /* single edge: the smaller id stays */
        anchor[v] = a;
    }
    for (int64_t v = 0; v < n; ++v)
        if (anchor[v] >= 0) w[anchor[v]] += 1;
    int64_t kept = 0;
    for (int64_t v = 0; v < n; ++v) newid[v] = anchor[v] >= 0 ? -1 : (int32_t)kept++;
    return kept;
}

/*
 * The pruned graph: the subgraph induced by the kept vertices, renumbered by
 * newid (ascending original order, so every row stays sorted). prow has
 * kept + 1 entries; returns the number of stored entries written to pcol.
 */
int64_t oracle_pruned_csr(int64_t n, const int64_t *row, const int32_t *col,
                          const int32_t *newid, int64_t *prow, int32_t *pcol)
{
    int64_t k = 0, e = 0;
    prow[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (newid[v] < 0) continue;
        for (int64_t j = row[v]; j < row[v + 1]; ++j)
            if (newid[col[j]] >= 0) pcol[e++] = newid[col[j]];
        prow[++k] = e;
    }
    return e;
}

/*
 * Reinsertion (Section 4.6). Given the placement ppos of the pruned graph
 * (prow, pcol), every kept vertex keeps its position and its removed
 * neighbours are placed on the circle around it of radius
 *   rho = 0.2 * (length of the shortest pruned-graph edge at v)
 * (0.2 * d when v has no such edge), evenly spaced: with m removed
 * neighbours the i-th (ascending original id) goes to angle theta + i s,
 * s = 2 pi / m, in the order of v's adjacency row (ascending ids for a
 * sorted CSR). The rotation theta keeps them off v's edges: among the
 * REINSERT_CANDIDATES rotations theta_c = s (c + 1/2) / REINSERT_CANDIDATES
 * it is the one whose smallest angular distance (modulo s) to the direction
 * of an edge at v is largest, the smallest c on ties. pos_out holds the
 * full placement (original ids).
 */
#define REINSERT_CANDIDATES 64
#define REINSERT_RHO 0.2

static double angle_mod(double a, double s)
{
    double r = a - s * floor(a / s);
    if (r >= s) r -= s;
    if (r < 0.0) r = 0.0;
    return r;
}

void oracle_reinsert(int64_t n, const int64_t *row, const int32_t *col, const int32_t *newid,
                     const int32_t *anchor, const int32_t *w, const int64_t *prow,
                     const int32_t *pcol, const double *ppos, double d, double *pos_out)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t v = 0; v < n; ++v) {
        if (newid[v] < 0) continue;
        int64_t pv = newid[v];
        double xv = ppos[2 * pv], yv = ppos[2 * pv + 1];
        pos_out[2 * v] = xv;
        pos_out[2 * v + 1] = yv;
        int m = w[v];
        if (m == 0) continue;
        double s = two_pi / (double)m;
        double shortest = INFINITY;
        for (int64_t j = prow[pv]; j < prow[pv + 1]; ++j) {
            double dx = ppos[2 * (int64_t)pcol[j]] - xv, dy = ppos[2 * (int64_t)pcol[j] + 1] - yv;
            double len = sqrt(dx * dx + dy * dy);
            if (len < shortest) shortest = len;
        }
        double rho = REINSERT_RHO * (prow[pv + 1] > prow[pv] ? shortest : d);
        int best = 0;
        double best_score = -1.0;
        for (int c = 0; c < REINSERT_CANDIDATES; ++c) {
            double theta = s * ((double)c + 0.5) / (double)REINSERT_CANDIDATES;
            double score = INFINITY;
            for (int64_t j = prow[pv]; j < prow[pv + 1]; ++j) {
                double dx = ppos[2 * (int64_t)pcol[j]] - xv;
                double dy = ppos[2 * (int64_t)pcol[j] + 1] - yv;
                double diff = fabs(angle_mod(atan2(dy, dx), s) - theta);
                double dist = diff < s - diff ? diff : s - diff;
                if (dist < score) score = dist;
            }
            if (score > best_score) {
                best_score = score;
                best = c;
            }
        }
        double theta = s * ((double)best + 0.5) / (double)REINSERT_CANDIDATES;
        int i = 0;
        for (int64_t j = row[v]; j < row[v + 1]; ++j) {
            int32_t u = col[j];
            if (anchor[u] != v) continue;
            double a = theta + (double)i * s;
            pos_out[2 * (int64_t)u] = xv + rho * cos(a);
            pos_out[2 * (int64_t)u + 1] = yv + rho * sin(a);
            ++i;
        }
    }
}

/*
 * Connected components (Section 4.6: the pipeline runs on every connected
 * component on its own). label[v] = index of v's component, components
 * numbered in the order of their smallest vertex id (a breadth-first search
 * from each vertex not yet reached, in ascending order). Returns the count.
 */
int32_t oracle_components(int64_t n, const int64_t *row, const int32_t *col, int32_t *label)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) label[v] = -1;
    int32_t count = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (label[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        label[s] = count;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t j = row[u]; j < row[u + 1]; ++j) {
                int32_t w = col[j];
                if (label[w] < 0) {
                    label[w] = count;
                    queue[tail++] = w;
                }
            }
        }
        ++count;
    }
    free(queue);
    return count;
}

/*
 * Arrangement of the component drawings "in a matrix" (Section 4.6), read as
 * shelf packing: boxes (bbox[4c..4c+3] = xmin, ymin, xmax, ymax of component
 * c) are taken by decreasing vertex count (size[c]), ties by component index;
 * rows are filled left to right with `gap` between boxes, a new row starting
 * `gap` above the tallest box of the previous one when the next box would
 * pass the row width W = max(widest box, sqrt(sum over boxes of
 * (width + gap)(height + gap))). offset[2c], offset[2c+1] receive the
 * translation that moves box c's lower-left corner to its place; the first
 * box sits at the origin.
 */
static const int64_t *pack_size_key;
static int pack_cmp(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (pack_size_key[i] != pack_size_key[j]) return pack_size_key[i] > pack_size_key[j] ? -1 : 1;
    return (i > j) - (i < j);
}

int oracle_pack(int32_t count, const double *bbox, const int64_t *size, double gap,
                double *offset)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(count > 0 ? count : 1));
    if (!order) return -1;
    double area = 0.0, widest = 0.0;
    for (int32_t c = 0; c < count; ++c) {
        order[c] = c;
        double w = bbox[4 * c + 2] - bbox[4 * c], h = bbox[4 * c + 3] - bbox[4 * c + 1];
        area += (w + gap) * (h + gap);
        if (w > widest) widest = w;
    }
    pack_size_key = size;
    qsort(order, (size_t)count, sizeof(int32_t), pack_cmp);
    double W = sqrt(area);
    if (widest > W) W = widest;
    double x = 0.0, y = 0.0, row_h = 0.0;
    int in_row = 0;
    for (int32_t i = 0; i < count; ++i) {
        int32_t c = order[i];
        double w = bbox[4 * c + 2] - bbox[4 * c], h = bbox[4 * c + 3] - bbox[4 * c + 1];
        if (in_row > 0 && x + w > W) {
            y += row_h + gap;
            x = 0.0;
            row_h = 0.0;
            in_row = 0;
        }
        offset[2 * c] = x - bbox[4 * c];
        offset[2 * c + 1] = y - bbox[4 * c + 1];
        x += w + gap;
        if (h > row_h) row_h = h;
        ++in_row;
    }
    free(order);
    return 0;
}
