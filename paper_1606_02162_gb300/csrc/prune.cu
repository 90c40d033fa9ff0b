// Degree-one pruning before the layout and reinsertion after it (Sections
// 4.3 and 4.6), on the device.
//
// Pruning removes every vertex of degree one in one pass (of the two ends
// of a single-edge component the larger id goes), remembers for each
// removed vertex the neighbour it hangs on (its anchor) and for each kept
// vertex how many removed neighbours it has (w). The kept vertices, in
// ascending id order, form the pruned graph (the induced subgraph), whose
// vertices repel with weight 1 + w during the layout (Section 4.6).
//
// Reinsertion puts the removed neighbours of a kept vertex v back on the
// circle around v of radius 0.2 x (shortest pruned-graph edge at v; 0.2 d if
// there is none), evenly spaced in the order of v's adjacency row, at the
// rotation that keeps them farthest from v's pruned-graph edges: among 64
// candidate rotations, the one whose smallest angular distance (modulo the
// spacing) to an edge direction is largest, the first on ties.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "force.cuh"
#include "gila_impl.h"

struct gila_pruned {
    gila_graph* full = nullptr;   // the caller's graph (borrowed)
    gila_graph* g = nullptr;      // the pruned graph (owned)
    int64_t n = 0, kept = 0;
    int32_t* anchor = nullptr;    // n: neighbour of a removed vertex, else -1
    int32_t* w = nullptr;         // n: removed neighbours of a kept vertex
    int32_t* newid = nullptr;     // n: index in the pruned graph, else -1
    int32_t* kept_ids = nullptr;  // kept: original id of each pruned-graph vertex
    double* stage = nullptr;      // 2 n doubles: host transfers
    void* ppos = nullptr;         // pruned placement (double2 capacity)
    void* fpos = nullptr;         // full placement in the layout's type
};

namespace gila {

namespace {

constexpr int kPThreads = 256;
constexpr int kCandidates = 64;
constexpr double kRho = 0.2;

unsigned blocks_for(int64_t n, int per_block = kPThreads)
{
    return (unsigned)std::max<int64_t>(1, (n + per_block - 1) / per_block);
}

__global__ void prune_mark_kernel(int64_t n, const int64_t* __restrict__ row,
                                  const int32_t* __restrict__ col, int32_t* __restrict__ anchor,
                                  int64_t* __restrict__ keep)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t a = -1;
    if (row[v + 1] - row[v] == 1) {
        const int32_t nb = col[row[v]];
        const bool nb_leaf = row[(int64_t)nb + 1] - row[nb] == 1;
        if (!(nb_leaf && nb > v)) a = nb;  // single edge: the smaller id stays
    }
    anchor[v] = a;
    keep[v] = a < 0 ? 1 : 0;
}

__global__ void prune_count_kernel(int64_t n, const int32_t* __restrict__ anchor,
                                   int32_t* __restrict__ w)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && anchor[v] >= 0) atomicAdd(&w[anchor[v]], 1);
}

// newid from the exclusive scan of the keep flags; kept vertices' ids and
// the pruned graph's row lengths.
__global__ void prune_ids_kernel(int64_t n, const int64_t* __restrict__ row,
                                 const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ anchor,
                                 const int64_t* __restrict__ scan, int32_t* __restrict__ newid,
                                 int32_t* __restrict__ kept_ids, int64_t* __restrict__ plen)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (anchor[v] >= 0) {
        newid[v] = -1;
        return;
    }
    const int64_t id = scan[v];
    newid[v] = (int32_t)id;
    kept_ids[id] = (int32_t)v;
    int64_t c = 0;
    for (int64_t j = row[v]; j < row[v + 1]; ++j) c += anchor[col[j]] < 0 ? 1 : 0;
    plen[id] = c;
}

// The induced subgraph's rows (ascending renumbered ids, since renumbering
// keeps the order) and the repulsion weights 1 + w.
__global__ void prune_fill_kernel(int64_t kept, const int64_t* __restrict__ row,
                                  const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ newid,
                                  const int32_t* __restrict__ kept_ids,
                                  const int32_t* __restrict__ w, const int64_t* __restrict__ prow,
                                  int32_t* __restrict__ pcol, double* __restrict__ wt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kept) return;
    const int64_t v = kept_ids[i];
    int64_t o = prow[i];
    for (int64_t j = row[v]; j < row[v + 1]; ++j) {
        const int32_t u = newid[col[j]];
        if (u >= 0) pcol[o++] = u;
    }
    wt[i] = 1.0 + (double)w[v];
}

template <class T>
__global__ void gather_kept_kernel(int64_t kept, const int32_t* __restrict__ kept_ids,
                                   const typename V2<T>::type* __restrict__ full,
                                   typename V2<T>::type* __restrict__ pruned)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kept) pruned[i] = full[kept_ids[i]];
}

// a - s floor(a / s) in [0, s), every operation rounded on its own
__device__ __forceinline__ double angle_mod(double a, double s)
{
    double r = __dsub_rn(a, __dmul_rn(s, floor(__ddiv_rn(a, s))));
    if (r >= s) r = __dsub_rn(r, s);
    if (r < 0.0) r = 0.0;
    return r;
}

template <class T>
__device__ __forceinline__ double2 ld_pos(const void* p, int64_t i)
{
    const typename V2<T>::type q = reinterpret_cast<const typename V2<T>::type*>(p)[i];
    return make_double2((double)q.x, (double)q.y);
}

template <class T>
__device__ __forceinline__ void st_pos(void* p, int64_t i, double x, double y)
{
    typename V2<T>::type q;
    q.x = (T)x;
    q.y = (T)y;
    reinterpret_cast<typename V2<T>::type*>(p)[i] = q;
}

// One warp per original vertex: kept vertices copy their position; the
// removed neighbours of a kept vertex are placed on its circle.
template <class T>
__global__ void __launch_bounds__(kPThreads)
reinsert_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col,
                const int32_t* __restrict__ newid, const int32_t* __restrict__ anchor,
                const int32_t* __restrict__ w, const int64_t* __restrict__ prow,
                const int32_t* __restrict__ pcol, const void* ppos, double d, void* fpos)
{
    const int lane = threadIdx.x & 31;
    const int64_t v = ((int64_t)blockIdx.x * kPThreads + threadIdx.x) >> 5;
    if (v >= n || newid[v] < 0) return;  // whole warp
    const int64_t pv = newid[v];
    const double2 xv = ld_pos<T>(ppos, pv);
    if (lane == 0) st_pos<T>(fpos, v, xv.x, xv.y);
    const int m = w[v];
    if (m == 0) return;
    const double two_pi = 6.283185307179586476925286766559;
    const double s = two_pi / (double)m;
    const int64_t e0 = prow[pv], e1 = prow[pv + 1];
    // shortest pruned-graph edge at v
    double shortest = INFINITY;
    for (int64_t j = e0 + lane; j < e1; j += 32) {
        const double2 xu = ld_pos<T>(ppos, pcol[j]);
        const double dx = __dsub_rn(xu.x, xv.x), dy = __dsub_rn(xu.y, xv.y);
        const double len = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        shortest = fmin(shortest, len);
    }
    for (int o = 16; o > 0; o >>= 1) shortest = fmin(shortest, __shfl_xor_sync(kFull, shortest, o));
    const double rho = __dmul_rn(kRho, e1 > e0 ? shortest : d);
    // scores of candidates lane and lane + 32
    double score[2] = {INFINITY, INFINITY};
    double theta[2];
    for (int h = 0; h < 2; ++h)
        theta[h] = __ddiv_rn(__dmul_rn(s, (double)(lane + 32 * h) + 0.5), (double)kCandidates);
    for (int64_t j = e0; j < e1; ++j) {
        const double2 xu = ld_pos<T>(ppos, pcol[j]);
        const double a = angle_mod(atan2(__dsub_rn(xu.y, xv.y), __dsub_rn(xu.x, xv.x)), s);
        for (int h = 0; h < 2; ++h) {
            const double diff = fabs(__dsub_rn(a, theta[h]));
            const double sd = __dsub_rn(s, diff);
            score[h] = fmin(score[h], diff < sd ? diff : sd);
        }
    }
    // best candidate: largest score, smallest index on ties
    double bs = score[0];
    int bc = lane;
    if (score[1] > bs) {
        bs = score[1];
        bc = lane + 32;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double os = __shfl_xor_sync(kFull, bs, o);
        const int oc = __shfl_xor_sync(kFull, bc, o);
        if (os > bs || (os == bs && oc < bc)) {
            bs = os;
            bc = oc;
        }
    }
    const double th = __ddiv_rn(__dmul_rn(s, (double)bc + 0.5), (double)kCandidates);
    // the removed neighbours in the order of v's adjacency row
    int base = 0;
    for (int64_t j0 = row[v]; j0 < row[v + 1]; j0 += 32) {
        const int64_t j = j0 + lane;
        int32_t u = -1;
        if (j < row[v + 1]) u = col[j];
        const bool leaf = u >= 0 && anchor[u] == (int32_t)v;
        const unsigned mask = __ballot_sync(kFull, leaf);
        if (leaf) {
            const int i = base + __popc(mask & lanemask_lt());
            const double a = __dadd_rn(th, __dmul_rn((double)i, s));
            st_pos<T>(fpos, u, __dadd_rn(xv.x, __dmul_rn(rho, cos(a))),
                      __dadd_rn(xv.y, __dmul_rn(rho, sin(a))));
        }
        base += __popc(mask);
    }
}

__global__ void f64_to_type_kernel(int64_t n2, const double* __restrict__ src, float* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2) dst[i] = (float)src[i];
}

__global__ void type_to_f64_kernel(int64_t n2, const float* __restrict__ src, double* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2) dst[i] = (double)src[i];
}

gila_status check_launch(const char* what)
{
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GILA_OK : cuda_fail(e, what);
}

gila_status gather(gila_pruned* p, bool f64, const void* full, void* pruned, cudaStream_t st)
{
    if (p->kept == 0) return GILA_OK;
    if (f64)
        gather_kept_kernel<double><<<blocks_for(p->kept), kPThreads, 0, st>>>(
            p->kept, p->kept_ids, (const double2*)full, (double2*)pruned);
    else
        gather_kept_kernel<float><<<blocks_for(p->kept), kPThreads, 0, st>>>(
            p->kept, p->kept_ids, (const float2*)full, (float2*)pruned);
    return check_launch("gather_kept_kernel");
}

gila_status reinsert(gila_pruned* p, bool f64, double d, const void* pruned, void* full,
                     cudaStream_t st)
{
    if (p->n == 0) return GILA_OK;
    const unsigned grid = blocks_for(p->n * 32);
    if (f64)
        reinsert_kernel<double><<<grid, kPThreads, 0, st>>>(
            p->n, p->full->row, p->full->col, p->newid, p->anchor, p->w, p->g->row, p->g->col,
            pruned, d, full);
    else
        reinsert_kernel<float><<<grid, kPThreads, 0, st>>>(
            p->n, p->full->row, p->full->col, p->newid, p->anchor, p->w, p->g->row, p->g->col,
            pruned, d, full);
    return check_launch("reinsert_kernel");
}

}  // namespace

}  // namespace gila

using namespace gila;

gila_status gila_prune_degree_one(gila_graph* g, gila_pruned** out)
{
    if (!g || !out) return fail(GILA_EINVAL, "graph or out is NULL");
    *out = nullptr;
    GILA_CUDA(cudaSetDevice(g->device));
    gila_pruned* p = new (std::nothrow) gila_pruned();
    if (!p) return fail(GILA_ENOMEM, "host allocation");
    p->full = g;
    p->n = g->n;
    const int64_t n = g->n;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    cudaStream_t st = g->stream;
    int64_t* keep = nullptr;
    int64_t* scan = nullptr;
    int64_t* plen = nullptr;
    int64_t* prow = nullptr;
    int32_t* pcol = nullptr;
    double* wt = nullptr;
    auto cleanup = [&]() {
        cudaFree(keep);
        cudaFree(scan);
        cudaFree(plen);
        cudaFree(prow);
        cudaFree(pcol);
        cudaFree(wt);
    };
    auto bail = [&](gila_status s) {
        cleanup();
        gila_pruned_destroy(p);
        return s;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&p->anchor, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&p->w, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&p->newid, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&p->kept_ids, sizeof(int32_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&keep, sizeof(int64_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&scan, sizeof(int64_t) * (nn + 1));
    if (e == cudaSuccess) e = cudaMalloc(&plen, sizeof(int64_t) * nn);
    if (e == cudaSuccess) e = cudaMalloc(&prow, sizeof(int64_t) * (nn + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->w, 0, sizeof(int32_t) * nn, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pruning buffers"));
    gila_status s = GILA_OK;
    if (n > 0) {
        prune_mark_kernel<<<blocks_for(n), kPThreads, 0, st>>>(n, g->row, g->col, p->anchor, keep);
        if ((s = check_launch("prune_mark_kernel")) != GILA_OK) return bail(s);
        prune_count_kernel<<<blocks_for(n), kPThreads, 0, st>>>(n, p->anchor, p->w);
        if ((s = check_launch("prune_count_kernel")) != GILA_OK) return bail(s);
        if ((s = scan_exclusive_i64(keep, n, scan, st)) != GILA_OK) return bail(s);
        prune_ids_kernel<<<blocks_for(n), kPThreads, 0, st>>>(n, g->row, g->col, p->anchor, scan,
                                                             p->newid, p->kept_ids, plen);
        if ((s = check_launch("prune_ids_kernel")) != GILA_OK) return bail(s);
        e = cudaMemcpyAsync(&p->kept, scan + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "kept count"));
    }
    const int64_t kept = p->kept;
    int64_t pnnz = 0;
    if (kept > 0) {
        if ((s = scan_exclusive_i64(plen, kept, prow, st)) != GILA_OK) return bail(s);
        e = cudaMemcpyAsync(&pnnz, prow + kept, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "pruned size"));
    } else {
        e = cudaMemsetAsync(prow, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "pruned rows"));
    }
    e = cudaMalloc(&pcol, sizeof(int32_t) * (size_t)std::max<int64_t>(pnnz, 1));
    if (e == cudaSuccess) e = cudaMalloc(&wt, sizeof(double) * (size_t)std::max<int64_t>(kept, 1));
    if (e != cudaSuccess) return bail(cuda_fail(e, "pruned graph"));
    if (kept > 0) {
        prune_fill_kernel<<<blocks_for(kept), kPThreads, 0, st>>>(
            kept, g->row, g->col, p->newid, p->kept_ids, p->w, prow, pcol, wt);
        if ((s = check_launch("prune_fill_kernel")) != GILA_OK) return bail(s);
    }
    if ((s = graph_create_from_device(kept, prow, pcol, pnnz, st, &p->g)) != GILA_OK) return bail(s);
    // with nothing removed every weight is 1, the unweighted force: the
    // pruned graph then runs exactly the kernels of the plain graph
    if (kept > 0 && kept < n && (s = set_repulsion_weights(p->g, wt, true)) != GILA_OK)
        return bail(s);
    cleanup();
    *out = p;
    return GILA_OK;
}

void gila_pruned_destroy(gila_pruned* p)
{
    if (!p) return;
    if (p->g) gila_graph_destroy(p->g);
    cudaFree(p->anchor);
    cudaFree(p->w);
    cudaFree(p->newid);
    cudaFree(p->kept_ids);
    cudaFree(p->stage);
    cudaFree(p->ppos);
    cudaFree(p->fpos);
    delete p;
}

gila_graph* gila_pruned_graph(gila_pruned* p)
{
    return p ? p->g : nullptr;
}

gila_status gila_pruned_info(const gila_pruned* p, int64_t* kept, int64_t* removed)
{
    if (!p) return fail(GILA_EINVAL, "pruned handle is NULL");
    if (kept) *kept = p->kept;
    if (removed) *removed = p->n - p->kept;
    return GILA_OK;
}

gila_status gila_pruned_export(const gila_pruned* p, int32_t* anchor, int32_t* w, int32_t* newid)
{
    if (!p) return fail(GILA_EINVAL, "pruned handle is NULL");
    GILA_CUDA(cudaSetDevice(p->full->device));
    const size_t b = sizeof(int32_t) * (size_t)p->n;
    if (p->n == 0) return GILA_OK;
    if (anchor) GILA_CUDA(cudaMemcpy(anchor, p->anchor, b, cudaMemcpyDeviceToHost));
    if (w) GILA_CUDA(cudaMemcpy(w, p->w, b, cudaMemcpyDeviceToHost));
    if (newid) GILA_CUDA(cudaMemcpy(newid, p->newid, b, cudaMemcpyDeviceToHost));
    return GILA_OK;
}

gila_status gila_pruned_gather(gila_pruned* p, int32_t precision, const void* pos_full_dev,
                               void* pos_pruned_dev)
{
    if (!p) return fail(GILA_EINVAL, "pruned handle is NULL");
    if (p->kept > 0 && (!pos_full_dev || !pos_pruned_dev))
        return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(p->full->device));
    return gather(p, is_f64(precision), pos_full_dev, pos_pruned_dev, p->full->stream);
}

gila_status gila_reinsert_degree_one(gila_pruned* p, const gila_params* prm,
                                     const void* pos_pruned_dev, void* pos_full_dev)
{
    if (!p || !prm) return fail(GILA_EINVAL, "pruned handle or params is NULL");
    if (p->n > 0 && (!pos_full_dev || (p->kept > 0 && !pos_pruned_dev)))
        return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(p->full->device));
    return reinsert(p, is_f64(prm->precision), prm->d, pos_pruned_dev, pos_full_dev,
                    p->full->stream);
}

gila_status gila_layout_pruned_run_device(gila_pruned* p, const gila_params* prm,
                                          void* pos_full_dev_inout)
{
    if (!p || !prm) return fail(GILA_EINVAL, "pruned handle or params is NULL");
    if (prm->precision == GILA_FP64_ORDERED)
        return fail(GILA_EINVAL, "GILA_FP64_ORDERED takes no repulsion weights");
    if (p->n > 0 && !pos_full_dev_inout) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(p->full->device));
    if (p->n == 0) return GILA_OK;
    const bool f64 = is_f64(prm->precision);
    cudaStream_t st = p->full->stream;
    p->g->stream = st;
    if (!p->ppos) GILA_CUDA(cudaMalloc(&p->ppos, 16 * (size_t)std::max<int64_t>(p->kept, 1)));
    gila_status s = gather(p, f64, pos_full_dev_inout, p->ppos, st);
    if (s != GILA_OK) return s;
    if (p->kept > 0 && (s = gila_layout_run_device(p->g, prm, p->ppos)) != GILA_OK) return s;
    return reinsert(p, f64, prm->d, p->ppos, pos_full_dev_inout, st);
}

gila_status gila_layout_pruned_run(gila_pruned* p, const gila_params* prm,
                                   const double* pos_in_host, double* pos_out_host)
{
    if (!p || !prm) return fail(GILA_EINVAL, "pruned handle or params is NULL");
    if (p->n > 0 && (!pos_in_host || !pos_out_host)) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(p->full->device));
    if (p->n == 0) return GILA_OK;
    const bool f64 = is_f64(prm->precision);
    const int64_t n2 = 2 * p->n;
    cudaStream_t st = p->full->stream;
    if (!p->stage) GILA_CUDA(cudaMalloc(&p->stage, sizeof(double) * (size_t)n2));
    if (!p->fpos) GILA_CUDA(cudaMalloc(&p->fpos, sizeof(double) * (size_t)n2));
    GILA_CUDA(cudaMemcpyAsync(p->stage, pos_in_host, sizeof(double) * (size_t)n2,
                              cudaMemcpyHostToDevice, st));
    void* work = p->stage;
    if (!f64) {
        f64_to_type_kernel<<<blocks_for(n2), kPThreads, 0, st>>>(n2, p->stage, (float*)p->fpos);
        gila_status s = check_launch("f64_to_type_kernel");
        if (s != GILA_OK) return s;
        work = p->fpos;
    }
    gila_status s = gila_layout_pruned_run_device(p, prm, work);
    if (s != GILA_OK) return s;
    if (!f64) {
        type_to_f64_kernel<<<blocks_for(n2), kPThreads, 0, st>>>(n2, (const float*)p->fpos,
                                                                 p->stage);
        if ((s = check_launch("type_to_f64_kernel")) != GILA_OK) return s;
    }
    GILA_CUDA(cudaMemcpyAsync(pos_out_host, p->stage, sizeof(double) * (size_t)n2,
                              cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    return blocked_tile_wait_failed(st);
}
