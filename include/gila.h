/*
 * gila.h -- C ABI of the GiLA k-hop Fruchterman-Reingold layout library
 * (single GB300 GPU, sm_103a).
 *
 * The method (Arleo, Didimo, Liotta, Montecchiani, "A Distributed
 * Force-Directed Algorithm on Giraph", arXiv 1606.02162):
 *   - Section 3.1: each vertex u feels F(u) = sum over edges (u,v) of an
 *     attraction of length delta^p / d toward v, plus a repulsion of length
 *     d^2 / delta^q away from every repelling vertex v (delta = |x_u - x_v|,
 *     d = ideal edge length, p = 2 and q = 1 in Fruchterman-Reingold). The
 *     move of u is F(u) cut to the temperature t, which falls per iteration.
 *   - Section 4.5: the repelling set of v is its k-neighbourhood N_v(k),
 *     the vertices at graph distance 1..k; all vertices move together once
 *     every force is known.
 *   - Section 5.1: the geometric cooling t_h = sqrt(n d / a) 0.93^h, with n
 *     and a taken per connected component.
 *   - Sections 4.3 and 4.6: degree-one vertices are pruned before the layout
 *     and reinserted around their neighbour after it; meanwhile a vertex
 *     repels with a weight that grows with its pruned neighbours. The
 *     pipeline runs on each connected component, whose drawings are then
 *     arranged without overlap.
 *
 * Conventions for every call:
 *   - Every call returns a gila_status; nothing throws across the ABI. On
 *     failure gila_last_error() returns a message (thread-local, valid until
 *     the next failing call on the same thread).
 *   - Host arrays belong to the caller; the library copies what it keeps.
 *     Device buffers created by the library belong to the graph and are
 *     freed by gila_graph_destroy. Pointers named *_dev are device
 *     pointers owned by the caller (e.g. a torch tensor's data_ptr()).
 *   - A graph is bound to the CUDA device current at creation and issues
 *     its work on the stream set by gila_graph_set_stream (default: the
 *     legacy default stream). Calls on one graph must not run concurrently.
 *   - Placements are arrays of n (x, y) pairs, row-major: element 2u is x_u,
 *     2u+1 is y_u. Host placements are always double. Device placements are
 *     float2 in GILA_FP32 / GILA_FP32_COMPENSATED and double2 in GILA_FP64 /
 *     GILA_FP64_ORDERED.
 */
#ifndef GILA_H
#define GILA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gila_status {
    GILA_OK = 0,
    GILA_EINVAL = 1,    /* bad argument or malformed graph */
    GILA_ENOMEM = 2,    /* device or host allocation failed */
    GILA_EBUDGET = 3,   /* admission refused: over the memory budget */
    GILA_ETIMEDOUT = 4, /* a bounded wait ran out */
    GILA_ECUDA = 5,     /* CUDA runtime or launch error */
    GILA_EBUSY = 6,     /* object still in use */
    GILA_ESTATE = 7     /* call out of order */
} gila_status;

/* Arithmetic of the force step. */
enum {
    GILA_FP32 = 0,             /* float positions and force sums */
    GILA_FP64 = 1,             /* double everywhere (validation mode) */
    GILA_FP32_COMPENSATED = 2, /* float, with compensated (two-sum) force sums */
    GILA_FP64_ORDERED = 3      /* double, validation: each force summed in the order of its
                                  definition (repulsion over N_u(k) by ascending id, then
                                  attraction in CSR order), every operation an individually
                                  rounded IEEE double op; reproduces a sequential FP64
                                  evaluation bit for bit. Slow. */
};

/* Cooling schedules: temperature of iteration i of `iters` (0-based). */
enum {
    GILA_COOL_LINEAR = 0,   /* t_i = t0 (iters - i) / iters; default t0 = 0.1 sqrt(n) */
    GILA_COOL_GEOMETRIC = 1 /* t_i = t0 0.93^i; default t0 = sqrt(n d / a), Section 5.1,
                               a = height / width of the initial bounding box */
};

/* gila_graph_create flags. */
enum {
    GILA_GRAPH_VALIDATE = 1, /* check the CSR is simple and symmetric (else GILA_EINVAL) */
    GILA_GRAPH_SIMPLIFY = 2  /* symmetrise, drop self-loops and repeats before upload */
};

typedef struct gila_params {
    int32_t k;         /* radius of the repelling set N_v(k), 1 <= k <= 64 (Section 4.5) */
    int32_t iters;     /* iterations run by gila_layout_run*, >= 0 */
    double d;          /* ideal edge length, > 0 (Section 3.1) */
    double t0;         /* initial temperature; <= 0 selects the schedule's default */
    int32_t schedule;  /* GILA_COOL_* */
    int32_t p;         /* attraction exponent, 0..8 (2 = Fruchterman-Reingold) */
    int32_t q;         /* repulsion exponent, 0..8 (1 = Fruchterman-Reingold) */
    int32_t precision; /* GILA_FP32 | GILA_FP64 | GILA_FP32_COMPENSATED | GILA_FP64_ORDERED */
} gila_params;

/* Layout quality figures of a placement, all accumulated in FP64 (for
 * FP32 placements each k-hop term d^2 / delta^q is formed in FP32, relative
 * error below 1e-6; the edge figures are FP64 throughout). */
typedef struct gila_metrics {
    double edge_mean;     /* mean edge length over the undirected edges */
    double edge_std;      /* population standard deviation of edge lengths */
    double edge_cv;       /* edge_std / edge_mean */
    double rep_total;     /* sum over unordered k-hop pairs of d^2 / delta^q */
    double att_total;     /* sum over undirected edges of delta^p / d */
    double rep_att_ratio; /* rep_total / att_total */
} gila_metrics;

/* Scheduling knobs of the iteration kernels. Each setting gives
 * deterministic results; different settings may differ in the last bits of
 * FP32 sums (different summation trees). Zero fields keep the defaults. */
typedef struct gila_tuning {
    int32_t tiled;         /* -1 automatic (default), 0 never, 1 always: stage positions in
                              shared memory instead of gathering them through L2. Graphs
                              whose row ranges touch narrow id windows get one window per
                              range, and each range's CTA finishes its rows (automatic mode:
                              where the windows' positions stay below the id stream's
                              bytes); other graphs get tiles of positions and a second
                              kernel that adds each row's tile partials */
    int32_t tile_vertices; /* positions per tile; 0 = as many as fit in 200 KiB */
    int32_t min_segment;   /* automatic mode tiles placements with at least 4 10^6 k-hop
                              entries when nnz_khop / (n * tiles) >= this (0: always) */
    int32_t small_max;     /* untiled kernel: rows of length <= this use 8-lane groups (64) */
    int32_t warp_max;      /* ... rows <= this use one warp (8192) */
    int32_t block_max;     /* ... rows <= this use one block (65536); longer rows are chunked */
    int32_t chunk;         /* entries per chunk of a chunked row (32768) */
    int32_t ctas_per_sm;   /* blocked path: each tile's rows are cut into ranges so that the
                              grid holds at most about this many CTAs per SM, all of about
                              equal cost (tiles: 1 below 10^8 k-hop entries, 3 below 2e9, 6
                              beyond; windows: 2) */
    int32_t bank_spread;   /* blocked path: 0 or 1 (default on) orders each row's entries of
                              a tile so that the lanes of one shared-memory gather read
                              distinct banks where the entries allow; -1 keeps ascending
                              id order */
    int32_t step_schedule; /* blocked path, FP32: 0 or 1 (default) issues each step's eight
                              terms once for the whole warp, only the closing of rows
                              diverging; -1 issues them apart for the lanes that close a
                              row in the step */
} gila_tuning;

typedef struct gila_graph gila_graph;

/* Fills *p with k = 2, iters = 300, d = 1, t0 = 0 (default), linear
 * cooling, p = 2, q = 1, GILA_FP32. */
void gila_params_default(gila_params* p);

/* Host-only check that (row_ptr, col_idx) is a simple undirected graph in
 * symmetric CSR form (Table 1 of the paper: no self-loops, no parallel
 * edges): row_ptr[0] = 0, non-decreasing, ids in [0, n), no self-loop, no
 * repeat within a row, and u in row v whenever v in row u. Returns GILA_OK
 * or GILA_EINVAL with the first violation in gila_last_error(). Touches no
 * GPU. */
gila_status gila_csr_validate(int64_t n, const int64_t* row_ptr, const int32_t* col_idx);

/* Upload a graph. n vertices (0 <= n < 2^31); row_ptr int64[n+1] and
 * col_idx int32[row_ptr[n]] are host arrays in symmetric CSR form (each
 * undirected edge stored in both rows). flags: GILA_GRAPH_VALIDATE rejects a
 * malformed CSR with GILA_EINVAL; GILA_GRAPH_SIMPLIFY repairs it instead.
 * Without either flag only what the kernels need to index safely is checked
 * (row_ptr[0] = 0, non-decreasing, every id in [0, n); GILA_EINVAL
 * otherwise); symmetry and simplicity are then the caller's to guarantee.
 * On success *out owns device copies of the arrays. */
gila_status gila_graph_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                              int32_t flags, gila_graph** out);

/* Free the graph and every device buffer it owns. NULL is ignored. */
void gila_graph_destroy(gila_graph* g);

/* Issue all later work of g on this cudaStream_t (NULL = legacy default
 * stream). The stream stays owned by the caller. */
gila_status gila_graph_set_stream(gila_graph* g, void* cuda_stream);

/* Set the scheduling knobs of g (see gila_tuning). Changing a row-class
 * bound drops the cached k-hop lists (the next call rebuilds them).
 * gila_graph_get_tuning returns the values in force, defaults filled in. */
gila_status gila_graph_tune(gila_graph* g, const gila_tuning* t);
gila_status gila_graph_get_tuning(const gila_graph* g, gila_tuning* out);

/* Sizes: vertices, stored adjacency entries (2E), the k of the built
 * k-hop lists (0 if none) and their total length. Any pointer may be NULL. */
gila_status gila_graph_info(const gila_graph* g, int64_t* n, int64_t* nnz_adj,
                            int32_t* k_built, int64_t* nnz_khop);

/* Build the k-hop lists N_v(k) of every vertex (Section 4.5) on the GPU:
 * breadth-first expansion to depth k, deduplicated, each list sorted by
 * ascending id, v itself excluded. Idempotent for the same k (a second call
 * returns at once); a different k rebuilds. *nnz_out (may be NULL) receives
 * the total list length. Synchronises the graph's stream. Memory: the lists
 * (4 bytes per entry) belong to the graph; on graphs with large balls the
 * build also keeps, for the graph's next build, the balls it stored between
 * counting and filling and (k = 3) one n-bit bitmap per vertex, at most
 * 16 GiB each, all freed with the graph. */
gila_status gila_build_khop(gila_graph* g, int32_t k, int64_t* nnz_out);

/* Drop the cached k-hop lists so the next build recomputes them (buffers
 * are kept for reuse). */
gila_status gila_khop_reset(gila_graph* g);

/* Copy the built lists to host arrays: krow int64[n+1] (offsets) and kcol
 * int32[nnz_khop] (ids, ascending per row). GILA_ESTATE if none are built. */
gila_status gila_khop_export(const gila_graph* g, int64_t* krow_host, int32_t* kcol_host);

/* Copy selected rows only (for lists too large for the host): counts_host
 * int64[nsel] receives |N_v(k)| of each sel_host[i]; when cols_host is not
 * NULL the rows follow back to back (int32, ascending each), at most
 * cols_cap entries (GILA_EINVAL if the total is larger). GILA_ESTATE if no
 * lists are built. Synchronous. */
gila_status gila_khop_export_rows(const gila_graph* g, int64_t nsel, const int64_t* sel_host,
                                  int64_t* counts_host, int32_t* cols_host, int64_t cols_cap);

/* One synchronous iteration at temperature t (Sections 3.1, 4.5): every
 * F(u) is formed from pos_in_dev, then pos_out_dev[u] = pos_in_dev[u] +
 * F(u) min(1, t / |F(u)|). Builds the k-hop lists for prm->k first when
 * needed. pos_in_dev and pos_out_dev are caller device arrays of n
 * float2 (FP32 modes) or double2 (GILA_FP64) and must not overlap.
 * disp_out_dev (may be NULL) receives the moves, same type. Asynchronous
 * on the graph's stream. The iteration kernel bounds its waits for the
 * shared-memory tile copies; a wait that gives up leaves that iteration's
 * forces incomplete and is reported as GILA_ECUDA by the next
 * gila_layout_run or gila_layout_metrics call in the process. */
gila_status gila_layout_step(gila_graph* g, const gila_params* prm, double t,
                             const void* pos_in_dev, void* pos_out_dev, void* disp_out_dev);

/* prm->iters iterations on a device-resident placement (float2 or double2
 * per prm->precision), under prm->schedule. Builds the k-hop lists first
 * when needed. The result is left in pos_dev_inout. Asynchronous on the
 * graph's stream apart from the k-hop build. */
gila_status gila_layout_run_device(gila_graph* g, const gila_params* prm, void* pos_dev_inout);

/* Whole layout from and to host memory: uploads pos_in_host (double[2n];
 * FP32 modes round once on the device), builds the k-hop lists when needed,
 * runs prm->iters iterations and writes the final placement to
 * pos_out_host (double[2n]; may equal pos_in_host). When metrics_out is not
 * NULL it receives the quality figures of the final placement, as
 * gila_layout_metrics computes them. Returns after the result is on the
 * host. */
gila_status gila_layout_run(gila_graph* g, const gila_params* prm,
                            const double* pos_in_host, double* pos_out_host,
                            gila_metrics* metrics_out);

/* Quality figures of a device placement (float2 or double2 per
 * prm->precision) with the k-hop lists of prm->k, in FP64 with a fixed
 * reduction order. Synchronises the graph's stream. */
gila_status gila_layout_metrics(gila_graph* g, const gila_params* prm, const void* pos_dev,
                                gila_metrics* out);

/* ------------------------------------------------------------------------
 * Batches: many independent graphs laid out together (thousands of small
 * graphs of uneven sizes). The batch is the disjoint union of
 * its graphs, so one k-hop build serves all of them; the layouts then run in
 * one persistent kernel launch in which each CTA takes one graph at a time
 * and carries it through all iterations with its placement staged in shared
 * memory. The launch is captured in a CUDA graph and replayed while the
 * arguments stay the same. Every graph follows its own temperature schedule
 * (default t0 from its own n and initial bounding box). A graph's result
 * depends only on the graph, its placement, the parameters and the batch
 * tuning, not on the other graphs of the batch. Precisions: GILA_FP32,
 * GILA_FP32_COMPENSATED, GILA_FP64. Placements are concatenated in graph
 * order: graph i starts at vertex offset n[0] + ... + n[i-1].
 * ------------------------------------------------------------------------ */
typedef struct gila_batch gila_batch;

typedef struct gila_batch_tuning {
    int32_t threads;     /* threads per CTA: 256, 512 or 1024; 0 = 512 */
    int32_t ctas_per_sm; /* CTAs per SM (1..8); 0 = 2 when two graphs fit in shared memory */
    int32_t group4_max;  /* graphs whose mean k-hop row length is <= this use 4 lanes per
                            vertex; 0 = 8 */
    int32_t group8_max;  /* ... 8 lanes; 0 = 24 */
    int32_t group16_max; /* ... 16 lanes; 0 = 64; longer rows use 32 lanes */
} gila_batch_tuning;

/* Pack `count` host CSR graphs (n[i], row_ptr[i], col_idx[i], each as for
 * gila_graph_create) into one device batch (one upload). flags:
 * GILA_GRAPH_VALIDATE checks every graph. */
gila_status gila_batch_create(int32_t count, const int64_t* n, const int64_t* const* row_ptr,
                              const int32_t* const* col_idx, int32_t flags, gila_batch** out);
void gila_batch_destroy(gila_batch* b);
gila_status gila_batch_set_stream(gila_batch* b, void* cuda_stream);
gila_status gila_batch_info(const gila_batch* b, int32_t* count, int64_t* total_n,
                            int64_t* nnz_khop);
/* k-hop lists of every graph of the batch (one build over the union);
 * cached per k like gila_build_khop. gila_batch_khop_reset drops them. */
gila_status gila_batch_build_khop(gila_batch* b, int32_t k, int64_t* nnz_out);
gila_status gila_batch_khop_reset(gila_batch* b);
/* Copy the built k-hop lists N_v(k) of the whole batch (Section 4.5) to
 * host memory, as for gila_khop_export: krow_host int64[total_n + 1],
 * kcol_host int32[nnz_khop], rows sorted ascending. Vertex v of graph i is
 * row voff_i + v, where voff_i is the vertex count of graphs 0..i-1, and
 * its entries are numbered the same way (a graph's lists stay inside its
 * own id range). GILA_ESTATE when no lists are built. */
gila_status gila_batch_khop_export(const gila_batch* b, int64_t* krow_host, int32_t* kcol_host);
/* Set (or read back, defaults filled in for a precision) the launch shape
 * and lanes-per-vertex thresholds of the batched kernel. */
gila_status gila_batch_tune(gila_batch* b, const gila_batch_tuning* t);
gila_status gila_batch_get_tuning(const gila_batch* b, int32_t precision, gila_batch_tuning* out);
/* Time candidate tunings on this batch (probe_iters iterations each, from
 * the placement pos_dev, which is not modified), keep the fastest and
 * return it in *chosen. */
gila_status gila_batch_autotune(gila_batch* b, const gila_params* prm, const void* pos_dev,
                                int32_t probe_iters, gila_batch_tuning* chosen);
/* prm->iters iterations of every graph on a device placement (float2 or
 * double2 per precision, concatenated), in one persistent launch; builds the
 * k-hop lists first when needed. Asynchronous on the batch's stream. */
gila_status gila_layout_batch_device(gila_batch* b, const gila_params* prm, void* pos_dev_inout);
/* The same from and to host memory (double[2 * total_n]); returns when the
 * result is on the host. */
gila_status gila_layout_batch_run(gila_batch* b, const gila_params* prm,
                                  const double* pos_in_host, double* pos_out_host);
/* Lay out `count` already-created graphs together: their device CSRs are
 * packed into a temporary batch; pos_in[i] / pos_out[i] are host
 * double[2 n_i] placements. Runs on the stream of gs[0]. */
gila_status gila_layout_batch(gila_graph* const* gs, int32_t count, const gila_params* prm,
                              const double* const* pos_in, double* const* pos_out);

/* ------------------------------------------------------------------------
 * Serving: a request loop for layout jobs of mixed sizes. Jobs are admitted
 * in arrival order by the device memory they need (the exact size of their
 * k-hop lists is counted before any list memory is taken) and by a slot
 * limit; admitted jobs keep placement and temperature on the device and
 * advance together, a chunk of iterations per job per round, each job on
 * its own CUDA stream, so their kernels overlap. Jobs arriving while others
 * run are admitted as soon as memory and a slot free up. A job runs the same
 * kernels as alone, so its result does not depend on the other jobs.
 * Precisions: GILA_FP32, GILA_FP32_COMPENSATED, GILA_FP64. Concurrency
 * between streams is limited by the CUDA_DEVICE_MAX_CONNECTIONS environment
 * variable (default 8) of the process.
 * ------------------------------------------------------------------------ */
typedef struct gila_server gila_server;

typedef struct gila_job_info {
    int32_t status;    /* GILA_OK or the job's failure (e.g. GILA_EBUDGET) */
    int64_t nnz_khop;  /* total k-hop list length of the job's graph */
    double queue_ms;   /* submit -> admitted (lists built, placement on the device) */
    double run_ms;     /* admitted -> result on the host */
    double latency_ms; /* submit -> result on the host */
} gila_job_info;

typedef struct gila_server_stats {
    int64_t completed, failed, pending, running;
    size_t bytes_in_use, bytes_peak, budget;
} gila_server_stats;

/* Start a server on the current device: mem_budget_bytes bounds the device
 * memory of admitted jobs, max_slots the number of jobs on the GPU at once.
 * Two host threads serve it until gila_server_destroy. */
gila_status gila_server_create(size_t mem_budget_bytes, int32_t max_slots, gila_server** out);
/* Stop the threads, fail unfinished jobs, free everything. Must not run
 * concurrently with other calls on the same server. */
void gila_server_destroy(gila_server* s);
/* Queue a job: graph (host CSR, as for gila_graph_create without flags:
 * offsets and ids are checked, symmetry is the caller's), 
 * parameters (prm->iters iterations), initial placement (host double[2n]).
 * The arrays are copied before the call returns. *ticket identifies it. */
gila_status gila_server_submit(gila_server* s, int64_t n, const int64_t* row_ptr,
                               const int32_t* col_idx, const gila_params* prm,
                               const double* pos_in, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a job; on success its final
 * placement goes to pos_out (host double[2n], may be NULL) and the ticket is
 * released. GILA_ETIMEDOUT leaves the job running and the ticket valid. A
 * failed job returns its status (info->status too). */
gila_status gila_server_wait(gila_server* s, uint64_t ticket, int32_t timeout_ms,
                             double* pos_out, gila_job_info* info);
/* *done = 1 when the job has finished (without releasing the ticket). */
gila_status gila_server_poll(gila_server* s, uint64_t ticket, int32_t* done);
/* Counters: jobs completed / failed / queued / on the GPU, device bytes
 * reserved now and at most, and the budget. */
gila_status gila_server_get_stats(gila_server* s, gila_server_stats* out);

/* ------------------------------------------------------------------------
 * Degree-one pruning and reinsertion (Sections 4.3 and 4.6).
 *
 * Pruning removes, in one pass, every vertex with exactly one neighbour (of
 * the two ends of a single-edge component only the larger id) and remembers
 * the neighbour it hangs on. The kept vertices, in ascending id order, form
 * the pruned graph (the subgraph they induce), a gila_graph whose vertices
 * repel with weight 1 + (number of removed neighbours) (Section 4.6: the
 * repulsion of a vertex grows with the vertices that will be put back
 * around it). Reinsertion puts the removed neighbours of a kept vertex v on
 * the circle around v of radius 0.2 x (shortest pruned-graph edge at v, or
 * 0.2 d when v has none), evenly spaced in the order of v's adjacency row,
 * at the one of 64 rotations s (c + 1/2) / 64 (s = 2 pi / count) whose
 * smallest angular distance, modulo s, to the direction of an edge at v is
 * largest (the smallest c on ties). The paper fixes the radius factor 0.2;
 * the candidate rotations are this library's reading of "avoiding edge
 * overlap".
 * ------------------------------------------------------------------------ */
typedef struct gila_pruned gila_pruned;

/* Repulsion weights: the repulsion that vertex v exerts is multiplied by
 * weight_host[v] (double[n], finite, >= 0; copied). NULL removes them.
 * Applied by the plain iteration kernel (automatic tiling then stays off);
 * GILA_FP64_ORDERED rejects weighted graphs with GILA_EINVAL. The quality
 * figures of gila_layout_metrics stay unweighted. */
gila_status gila_graph_set_repulsion_weights(gila_graph* g, const double* weight_host);

/* Prune g on its device and stream. *out owns the pruned graph (with its
 * weights set); g must outlive *out. Synchronises g's stream. */
gila_status gila_prune_degree_one(gila_graph* g, gila_pruned** out);
void gila_pruned_destroy(gila_pruned* p);
/* The pruned graph, owned by p: usable with every gila_graph call (k-hop
 * build, tuning, steps, runs, metrics); ids are 0..kept-1. */
gila_graph* gila_pruned_graph(gila_pruned* p);
/* Kept and removed vertex counts (either pointer may be NULL). */
gila_status gila_pruned_info(const gila_pruned* p, int64_t* kept, int64_t* removed);
/* Host copies over the original ids (each may be NULL): anchor int32[n]
 * (neighbour of a removed vertex, else -1), w int32[n] (removed neighbours
 * of a kept vertex, else 0), newid int32[n] (index in the pruned graph of a
 * kept vertex, else -1). Synchronous. */
gila_status gila_pruned_export(const gila_pruned* p, int32_t* anchor, int32_t* w, int32_t* newid);
/* Gather the kept vertices' rows of a full device placement (n float2 or
 * double2 per precision) into a pruned placement (kept of the same type).
 * Asynchronous on g's stream. */
gila_status gila_pruned_gather(gila_pruned* p, int32_t precision, const void* pos_full_dev,
                               void* pos_pruned_dev);
/* Reinsertion: write the full placement (n float2 or double2 per
 * prm->precision; prm->d gives the radius of vertices without edges) from a
 * pruned placement. Asynchronous on g's stream. */
gila_status gila_reinsert_degree_one(gila_pruned* p, const gila_params* prm,
                                     const void* pos_pruned_dev, void* pos_full_dev);
/* The whole pipeline on a full device placement (n float2 or double2):
 * gather the kept vertices, lay out the pruned graph with prm (default t0
 * from the pruned graph's n), reinsert. The result replaces the input.
 * GILA_FP64_ORDERED is rejected (weighted repulsion). */
gila_status gila_layout_pruned_run_device(gila_pruned* p, const gila_params* prm,
                                          void* pos_full_dev_inout);
/* The same from and to host memory (double[2n] of the original graph);
 * returns when the result is on the host. */
gila_status gila_layout_pruned_run(gila_pruned* p, const gila_params* prm,
                                   const double* pos_in_host, double* pos_out_host);

/* ------------------------------------------------------------------------
 * Per-component layout (Section 4.6: the pipeline is applied to every
 * connected component on its own and the drawings are arranged without
 * overlap; Section 5.1: a component's maximum displacement follows its own
 * n and initial frame).
 * ------------------------------------------------------------------------ */

/* Connected components on the device: label_host int32[n] receives the
 * index of each vertex's component, components numbered in the order of
 * their smallest vertex id; *count (may be NULL) their number. Synchronous. */
gila_status gila_graph_components(gila_graph* g, int32_t* label_host, int32_t* count);

/* Lay out every connected component on its own with prm (with prm->t0 <= 0
 * each component takes its own default initial temperature: 0.1 sqrt(n_c)
 * linear, sqrt(n_c d / a_c) geometric with a_c the height/width of its own
 * initial frame): components of up to 4096 vertices together in one
 * persistent batch launch, larger ones one by one on the single-graph
 * kernels, isolated vertices unchanged. The drawings are then packed into
 * rows: boxes by decreasing vertex count (ties by component index), left to
 * right with `gap` between boxes (gap <= 0: prm->d), a new row `gap` above
 * the tallest box of the last one when the next box would pass the width
 * W = max(widest box, sqrt(sum over boxes of (width + gap)(height + gap)));
 * the first box's lower-left corner sits at the origin. The paper says only
 * that the drawings are "arranged in a matrix" to avoid overlap; the row
 * packing is this library's reading. Host placements double[2n];
 * *count_out (may be NULL) receives the number of components. */
gila_status gila_layout_components_run(gila_graph* g, const gila_params* prm, double gap,
                                       const double* pos_in_host, double* pos_out_host,
                                       int32_t* count_out);

/* Test hook for failure detection: while on (1), the blocked path's CTAs
 * announce their shared-memory tile on its mbarrier but issue no copy, so
 * every tile wait runs out after 1 ms instead of the normal 1 s bound; the
 * CTAs then return without computing, and the next synchronising call
 * (gila_layout_run, gila_layout_metrics) reports GILA_ECUDA. Nothing is left
 * in flight and the CUDA context stays usable; turn it off (0) to resume
 * normal iterations. For tests only. */
gila_status gila_graph_set_wait_test(gila_graph* g, int32_t on);

/* Temperature of iteration i under prm (t0 = resolved initial temperature). */
double gila_temperature(const gila_params* prm, double t0, int32_t i);

/* Per-graph timing by CUDA events recorded on the graph's stream while
 * enabled (on = 1 or 2; 0 turns it off; other values give GILA_EINVAL):
 * k-hop builds (count, ms; the one-time blocked-path plan of the lists is
 * added to build_ms, not counted as a build) and iteration sequences
 * (launches, ms of the launch sequence). gila_profile_read returns the
 * totals since the previous read, then clears them; it waits for the last
 * recorded event. */
gila_status gila_profile_enable(gila_graph* g, int32_t on);
gila_status gila_profile_read(gila_graph* g, int64_t* builds, double* build_ms,
                              int64_t* iter_launches, double* iter_ms);

/* With on = 2 each iteration's repulsion kernel (the one that streams the
 * k-hop lists of Section 4.5: "blocked_kernel", "blocked_kernel (window)",
 * "iteration_kernel" or "ordered_kernel") is also timed on its own, between
 * events recorded directly before and after its launch. Returns the number
 * of such launches since the previous call and their total ms, and copies
 * the name of the last kernel timed into name (NUL-terminated, at most
 * name_cap - 1 characters; name may be NULL); then clears those totals.
 * Waits for the recorded events. Call gila_profile_read first when both are
 * wanted (it folds pending records of every kind). */
gila_status gila_profile_read_kernel(gila_graph* g, int64_t* launches, double* ms, char* name,
                                     int32_t name_cap);

/* Message of the last failing call on this thread ("" if none). */
const char* gila_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * graphs, all threads), for accounting of device work. */
int64_t gila_kernel_launches(void);

/* Sizes |N_v(k)| of every k-hop list, computed without allocating any
 * memory. The paper has no counterpart: this is a service for callers that
 * must not allocate device memory themselves or have it allocated for them,
 * for example a serving process whose memory manager owns the whole device
 * and decides admission by the bytes a graph's k-hop lists would need
 * (it must learn that size before it may reserve anything), or a caller
 * that cannot afford the device-wide synchronisation that cudaMalloc and
 * cudaFree may imply while other streams are busy.
 *
 * Inputs are caller-owned device arrays: row_ptr_dev int64[n+1] and
 * col_idx_dev int32[row_ptr[n]] in symmetric CSR form (as for
 * gila_graph_create, unchecked). Output: counts_dev int64[n] (device, caller
 * owned) receives |N_v(k)| for every v; *total_host (may be NULL) receives
 * their sum. Work runs on cuda_stream (NULL = legacy default stream) and the
 * call returns after it has finished.
 *
 * Scratch lives in one fixed device array inside the library (about 5.1 MiB)
 * which bounds n to at most 262,144 vertices: larger n returns GILA_EINVAL
 * with a message. The call makes no cudaMalloc or cudaFree call and uses no
 * allocating library routine. The array is reserved when the library's
 * k-hop module is loaded on a device: with CUDA's default lazy module
 * loading that happens at the first k-hop call on that device (this one or
 * gila_build_khop), and it then stays until the process exits. A caller
 * whose memory manager reserves most of the device should therefore make
 * one call at startup, before it reserves memory; that first call also
 * looks up the array's address for the device (cudaGetSymbolAddress with
 * the device current). Every call synchronises cuda_stream and copies the
 * total to the host, so it cannot be recorded into a CUDA graph (calling it
 * while the stream is being captured is an error). Every call reuses the
 * same scratch: calls that overlap on the GPU (other threads, other
 * streams) race and must be serialised by the caller. */
gila_status gila_khop_count_noalloc(int64_t n, const int64_t* row_ptr_dev,
                                    const int32_t* col_idx_dev, int32_t k, int64_t* counts_dev,
                                    int64_t* total_host, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GILA_H */
