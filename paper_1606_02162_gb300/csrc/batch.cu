// Batched layouts: many graphs in one persistent launch.
//
// A batch is the disjoint union of its graphs (ids offset per graph), so one
// k-hop build serves all of them. The layout of every graph then runs inside
// a single CTA from its first to its last iteration: the CTA stages the
// graph's placement in shared memory (two buffers, Jacobi), streams the
// graph's k-hop rows (small enough to stay in L2 across iterations) and
// separates iterations with __syncthreads, so no grid-wide barrier and no
// per-iteration launch exists. CTAs take graphs from a global counter,
// largest first. Graphs too large for shared memory iterate on two global
// buffers in the same way.
//
// Lanes per vertex (4, 8, 16 or 32) follow the graph's own mean k-hop row
// length; a graph's result therefore does not depend on the other graphs of
// the batch. The temperature of each graph follows its own schedule: the
// default t0 uses that graph's n (and, for geometric cooling, the aspect of
// its own initial bounding box).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "force.cuh"
#include "gila_impl.h"

struct gila_batch {
    gila_graph* g = nullptr;  // disjoint union of the graphs
    int32_t count = 0;
    std::vector<int64_t> voff_h;  // vertex offsets, count + 1
    int64_t* voff = nullptr;
    int32_t* order = nullptr;     // graphs in processing order
    int* work = nullptr;          // next position in `order`
    double* geo = nullptr;        // 0.93^i table
    size_t geo_cap = 0;
    void* tmp = nullptr;          // second global placement for graphs beyond shared memory
    size_t tmp_cap = 0;
    void* pos[2] = {nullptr, nullptr};  // placement buffers of the host-memory calls
    size_t pos_cap[2] = {0, 0};
    double* stage = nullptr;
    size_t stage_cap = 0;
    int64_t max_n = 0;
    cudaStream_t user = nullptr;   // caller's stream
    cudaStream_t own = nullptr;    // capture stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> exec_key;  // arguments the captured graph was made with
    gila_batch_tuning tune = {0, 0, 0, 0, 0};
};

namespace gila {

namespace {

struct BatchArgs {
    const int64_t* voff;
    const int32_t* order;
    int32_t count;
    const int64_t* row;
    const int32_t* col;
    const int64_t* krow;
    const uint32_t* kcol;
    int* work;
    const double* geo;
    int iters, schedule;
    double d, t0;
    int p, q;
    void* pos;
    void* tmp;
    int smem_verts;
    int g4_max, g8_max, g16_max;
};

template <class T>
__device__ __forceinline__ void capped(T t, T fx, T fy, T& mx, T& my)
{
    const T fn = sqrt(fx * fx + fy * fy);
    mx = fx;
    my = fy;
    if (fn > t) {
        const T sc = t / fn;
        mx = fx * sc;
        my = fy * sc;
    }
}

// One CTA lays out one graph at a time; see the file comment.
template <class T, int MODEL, bool COMP>
__global__ void __launch_bounds__(1024) batch_kernel(const BatchArgs A)
{
    using P2 = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_g;
    __shared__ double s_box[32][4];
    P2* sbuf0 = reinterpret_cast<P2*>(smem_raw);
    P2* sbuf1 = sbuf0 + A.smem_verts;
    P2* gpos = reinterpret_cast<P2*>(A.pos);
    P2* gtmp = reinterpret_cast<P2*>(A.tmp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_g = atomicAdd(A.work, 1);
        __syncthreads();
        const int gi = s_g;
        __syncthreads();
        if (gi >= A.count) break;
        const int gid = A.order[gi];
        const int64_t v0 = A.voff[gid];
        const int64_t n = A.voff[gid + 1] - v0;
        if (n == 0) continue;
        const int64_t nnz = A.krow[v0 + n] - A.krow[v0];
        const int64_t avg = nnz / n;
        const int G = avg <= A.g4_max ? 4 : avg <= A.g8_max ? 8 : avg <= A.g16_max ? 16 : 32;
        const bool in_smem = n <= A.smem_verts;
        P2* cur = in_smem ? sbuf0 : gpos + v0;
        P2* nxt = in_smem ? sbuf1 : gtmp + v0;
        if (in_smem)
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) cur[i] = gpos[v0 + i];
        __syncthreads();
        // initial temperature of this graph
        double t0 = A.t0;
        if (!(t0 > 0.0)) {
            if (A.schedule != GILA_COOL_GEOMETRIC) {
                t0 = 0.1 * sqrt((double)n);
            } else {
                double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const P2 p = cur[i];
                    x0 = fmin(x0, (double)p.x);
                    x1 = fmax(x1, (double)p.x);
                    y0 = fmin(y0, (double)p.y);
                    y1 = fmax(y1, (double)p.y);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    x0 = fmin(x0, __shfl_xor_sync(kFull, x0, o));
                    x1 = fmax(x1, __shfl_xor_sync(kFull, x1, o));
                    y0 = fmin(y0, __shfl_xor_sync(kFull, y0, o));
                    y1 = fmax(y1, __shfl_xor_sync(kFull, y1, o));
                }
                if (lane == 0) {
                    s_box[warp][0] = x0;
                    s_box[warp][1] = x1;
                    s_box[warp][2] = y0;
                    s_box[warp][3] = y1;
                }
                __syncthreads();
                x0 = s_box[0][0];
                x1 = s_box[0][1];
                y0 = s_box[0][2];
                y1 = s_box[0][3];
                for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                    x0 = fmin(x0, s_box[w][0]);
                    x1 = fmax(x1, s_box[w][1]);
                    y0 = fmin(y0, s_box[w][2]);
                    y1 = fmax(y1, s_box[w][3]);
                }
                __syncthreads();
                const double w = x1 - x0, h = y1 - y0;
                const double a = (w > 0.0 && h > 0.0) ? h / w : 1.0;
                t0 = sqrt((double)n * A.d / a);
            }
        }
        Rep<T, MODEL, COMP, kSrcGeneric> f;
        f.src.base = (uint32_t)v0;
        f.d2 = (T)(A.d * A.d);
        f.q = A.q;
        Att<T, MODEL, COMP, kSrcGeneric> att;
        att.src.base = (uint32_t)v0;
        att.inv_d = (T)(1.0 / A.d);
        att.p = A.p;
        const int groups = blockDim.x / G;
        const int grp = threadIdx.x / G, gl = threadIdx.x % G;
        for (int it = 0; it < A.iters; ++it) {
            const double td = A.schedule == GILA_COOL_GEOMETRIC
                                  ? t0 * A.geo[it]
                                  : t0 * (double)(A.iters - it) / (double)A.iters;
            const T t = (T)td;
            // ids are global; the buffer holds this graph's vertices from 0
            f.src.pos = cur;
            att.src.pos = cur;
            for (int64_t vb = 0; vb < n; vb += groups) {
                const int64_t v = vb + grp;
                const bool live = v < n;
                Acc<T, COMP> a;
                P2 pu;
                pu.x = T(0);
                pu.y = T(0);
                if (live) {
                    pu = cur[v];
                    f.xu = pu.x;
                    f.yu = pu.y;
                    att.xu = pu.x;
                    att.yu = pu.y;
                    // lanes take entries by their place in the row, so the
                    // order does not depend on where the row sits in the batch
                    row_sum_rel(A.kcol, A.krow[v0 + v], A.krow[v0 + v + 1], gl, G, f, a);
                    row_sum_rel(reinterpret_cast<const uint32_t*>(A.col), A.row[v0 + v],
                                A.row[v0 + v + 1], gl, G, att, a);
                }
                a.group_reduce(G);
                if (live && gl == 0) {
                    T mx, my;
                    capped<T>(t, a.fx(), a.fy(), mx, my);
                    P2 o;
                    o.x = pu.x + mx;
                    o.y = pu.y + my;
                    nxt[v] = o;
                }
            }
            __syncthreads();
            P2* s = cur;
            cur = nxt;
            nxt = s;
        }
        // the result goes to the caller's buffer
        if (in_smem || cur != gpos + v0)
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) gpos[v0 + i] = cur[i];
        __syncthreads();
    }
}

// Pack graphs given as device CSRs into the union CSR (one block per graph).
struct PackSrc {
    const int64_t* row;
    const int32_t* col;
    int64_t n, voff, eoff;
};

__global__ void pack_kernel(const PackSrc* __restrict__ src, int64_t* __restrict__ row,
                            int32_t* __restrict__ col)
{
    const PackSrc s = src[blockIdx.x];
    for (int64_t i = threadIdx.x; i < s.n; i += blockDim.x) row[s.voff + i] = s.eoff + s.row[i];
    const int64_t nnz = s.row[s.n] - s.row[0];
    for (int64_t i = threadIdx.x; i < nnz; i += blockDim.x)
        col[s.eoff + i] = (int32_t)(s.voff + s.col[s.row[0] + i]);
}

gila_batch_tuning resolved(const gila_batch* b, size_t esz, int sms)
{
    gila_batch_tuning t = b->tune;
    if (t.threads != 256 && t.threads != 512 && t.threads != 1024) t.threads = 512;
    if (t.group4_max <= 0) t.group4_max = 8;
    if (t.group8_max <= 0) t.group8_max = 24;
    if (t.group16_max <= 0) t.group16_max = 64;
    const int64_t smem_cap = 227 * 1024 - 2048;  // opt-in limit less the static arrays
    if (t.ctas_per_sm <= 0) {
        // two CTAs per SM unless a graph then no longer fits
        const int64_t need = 2 * b->max_n * (int64_t)esz;
        t.ctas_per_sm = (need * 2 <= smem_cap) ? 2 : 1;
    }
    t.ctas_per_sm = std::max(1, std::min(t.ctas_per_sm, 2048 / t.threads));
    (void)sms;
    return t;
}

template <class T, int MODEL, bool COMP>
cudaError_t launch_batch(const BatchArgs& A, int grid, int threads, size_t smem, cudaStream_t st)
{
    batch_kernel<T, MODEL, COMP><<<grid, threads, smem, st>>>(A);
    count_launch();
    return cudaGetLastError();
}

// Shared-memory opt-in for every instantiation on the current device
// (outside any stream capture); once per device, callers may race.
cudaError_t configure_batch_kernels()
{
    static std::atomic<uint64_t> done{0};
    int device = 0;
    cudaError_t de = cudaGetDevice(&device);
    if (de != cudaSuccess) return de;
    const uint64_t bit = 1ull << (device & 63);
    if (done.load() & bit) return cudaSuccess;
    const int lim = 227 * 1024;
    cudaError_t e = cudaSuccess;
#define GILA_OPT_IN(T, M, C)                                                                 \
    if (e == cudaSuccess)                                                                    \
        e = cudaFuncSetAttribute(batch_kernel<T, M, C>,                                      \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, lim - 2048);
    GILA_OPT_IN(float, kFR, false)
    GILA_OPT_IN(float, kGeneric, false)
    GILA_OPT_IN(float, kFR, true)
    GILA_OPT_IN(float, kGeneric, true)
    GILA_OPT_IN(double, kFR, false)
    GILA_OPT_IN(double, kGeneric, false)
#undef GILA_OPT_IN
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

gila_status batch_finish_create(gila_batch* b)
{
    const int32_t count = b->count;
    // processing order: largest graphs first
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
        return b->voff_h[a + 1] - b->voff_h[a] > b->voff_h[c + 1] - b->voff_h[c];
    });
    b->max_n = 0;
    for (int32_t i = 0; i < count; ++i)
        b->max_n = std::max<int64_t>(b->max_n, b->voff_h[i + 1] - b->voff_h[i]);
    GILA_CUDA(cudaMalloc(&b->voff, sizeof(int64_t) * (count + 1)));
    GILA_CUDA(cudaMalloc(&b->order, sizeof(int32_t) * std::max(count, 1)));
    GILA_CUDA(cudaMalloc(&b->work, sizeof(int)));
    GILA_CUDA(cudaMemcpy(b->voff, b->voff_h.data(), sizeof(int64_t) * (count + 1),
                         cudaMemcpyHostToDevice));
    if (count > 0)
        GILA_CUDA(cudaMemcpy(b->order, order.data(), sizeof(int32_t) * count,
                             cudaMemcpyHostToDevice));
    GILA_CUDA(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
    GILA_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    GILA_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    return GILA_OK;
}

gila_status check_batch_params(const gila_params* p)
{
    if (!p) return fail(GILA_EINVAL, "params is NULL");
    if (p->k < 1 || p->k > 64) return fail(GILA_EINVAL, "k must be in [1, 64]");
    if (p->iters < 0) return fail(GILA_EINVAL, "iters must be >= 0");
    if (!(p->d > 0.0) || !std::isfinite(p->d)) return fail(GILA_EINVAL, "d must be finite and > 0");
    if (!std::isfinite(p->t0)) return fail(GILA_EINVAL, "t0 must be finite");
    if (p->schedule != GILA_COOL_LINEAR && p->schedule != GILA_COOL_GEOMETRIC)
        return fail(GILA_EINVAL, "unknown cooling schedule");
    if (p->p < 0 || p->p > 8 || p->q < 0 || p->q > 8)
        return fail(GILA_EINVAL, "p and q must be in [0, 8]");
    if (p->precision != GILA_FP32 && p->precision != GILA_FP64 &&
        p->precision != GILA_FP32_COMPENSATED)
        return fail(GILA_EINVAL, "batched layouts support GILA_FP32, GILA_FP32_COMPENSATED and "
                                 "GILA_FP64");
    return GILA_OK;
}

// Launch (or replay) the persistent kernel on the batch's capture stream,
// ordered after and before the caller's stream.
gila_status batch_run(gila_batch* b, const gila_params* prm, void* pos)
{
    gila_graph* g = b->g;
    const size_t esz = is_f64(prm->precision) ? 16 : 8;
    if (b->count == 0 || g->n == 0 || prm->iters == 0) return GILA_OK;
    gila_status s;
    if (prm->schedule == GILA_COOL_GEOMETRIC) {
        s = ensure((void**)&b->geo, &b->geo_cap, sizeof(double) * (size_t)prm->iters);
        if (s != GILA_OK) return s;
        std::vector<double> geo((size_t)prm->iters);
        for (int i = 0; i < prm->iters; ++i) geo[i] = std::pow(0.93, (double)i);
        GILA_CUDA(cudaMemcpy(b->geo, geo.data(), sizeof(double) * geo.size(),
                             cudaMemcpyHostToDevice));
    }
    const int sms = sm_count(g->device);
    const gila_batch_tuning tu = resolved(b, esz, sms);
    const int64_t smem_cap = 227 * 1024 - 2048;
    int64_t per_cta = smem_cap / tu.ctas_per_sm;
    int64_t smem_verts = std::min<int64_t>(b->max_n, per_cta / (2 * (int64_t)esz));
    if (smem_verts < 2) smem_verts = 2;
    const size_t smem = (size_t)smem_verts * 2 * esz;
    if (b->max_n > smem_verts) {
        s = ensure(&b->tmp, &b->tmp_cap, esz * (size_t)g->n);
        if (s != GILA_OK) return s;
    }
    BatchArgs A;
    A.voff = b->voff;
    A.order = b->order;
    A.count = b->count;
    A.row = g->row;
    A.col = g->col;
    A.krow = g->krow;
    A.kcol = g->kcol;
    A.work = b->work;
    A.geo = b->geo;
    A.iters = prm->iters;
    A.schedule = prm->schedule;
    A.d = prm->d;
    A.t0 = prm->t0;
    A.p = prm->p;
    A.q = prm->q;
    A.pos = pos;
    A.tmp = b->tmp;
    A.smem_verts = (int)smem_verts;
    A.g4_max = tu.group4_max;
    A.g8_max = tu.group8_max;
    A.g16_max = tu.group16_max;
    const int grid = std::max(1, std::min<int>(sms * tu.ctas_per_sm, b->count));
    // the captured graph is reused while every argument is the same
    std::vector<unsigned char> key(sizeof(A) + sizeof(int) * 3);
    memcpy(key.data(), &A, sizeof(A));
    const int extra[3] = {grid, tu.threads, prm->precision};
    memcpy(key.data() + sizeof(A), extra, sizeof(extra));
    GILA_CUDA(configure_batch_kernels());
    GILA_CUDA(cudaEventRecord(b->ev_in, b->user));
    GILA_CUDA(cudaStreamWaitEvent(b->own, b->ev_in, 0));
    if (!b->exec || key != b->exec_key) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        GILA_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(b->work, 0, sizeof(int), b->own);
        const bool fr = (prm->p == 2 && prm->q == 1);
        cudaError_t e;
        switch (prm->precision) {
        case GILA_FP64:
            e = fr ? launch_batch<double, kFR, false>(A, grid, tu.threads, smem, b->own)
                   : launch_batch<double, kGeneric, false>(A, grid, tu.threads, smem, b->own);
            break;
        case GILA_FP32_COMPENSATED:
            e = fr ? launch_batch<float, kFR, true>(A, grid, tu.threads, smem, b->own)
                   : launch_batch<float, kGeneric, true>(A, grid, tu.threads, smem, b->own);
            break;
        default:
            e = fr ? launch_batch<float, kFR, false>(A, grid, tu.threads, smem, b->own)
                   : launch_batch<float, kGeneric, false>(A, grid, tu.threads, smem, b->own);
            break;
        }
        cudaError_t e2 = cudaStreamEndCapture(b->own, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "batch_kernel");
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        cudaError_t e3 = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e3, "cudaGraphInstantiate");
        }
        b->exec_key = key;
    }
    GILA_CUDA(cudaGraphLaunch(b->exec, b->own));
    GILA_CUDA(cudaEventRecord(b->ev_out, b->own));
    GILA_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return GILA_OK;
}

}  // namespace
}  // namespace gila

using namespace gila;

extern "C" {

gila_status gila_batch_create(int32_t count, const int64_t* n, const int64_t* const* row_ptr,
                              const int32_t* const* col_idx, int32_t flags, gila_batch** out)
{
    if (!out) return fail(GILA_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 0) return fail(GILA_EINVAL, "count must be >= 0");
    if (count > 0 && (!n || !row_ptr || !col_idx)) return fail(GILA_EINVAL, "array is NULL");
    std::vector<int64_t> voff(count + 1, 0), eoff(count + 1, 0);
    for (int32_t i = 0; i < count; ++i) {
        if (n[i] < 0 || !row_ptr[i]) return fail(GILA_EINVAL, "graph " + std::to_string(i) + ": bad n or row_ptr");
        if (flags & GILA_GRAPH_VALIDATE) {
            gila_status s = gila_csr_validate(n[i], row_ptr[i], col_idx[i]);
            if (s != GILA_OK) return fail(s, "graph " + std::to_string(i) + ": " + gila_last_error());
        } else {
            gila_status s = check_csr_bounds(n[i], row_ptr[i], col_idx[i]);
            if (s != GILA_OK) return fail(s, "graph " + std::to_string(i) + ": " + gila_last_error());
        }
        voff[i + 1] = voff[i] + n[i];
        eoff[i + 1] = eoff[i] + (row_ptr[i][n[i]] - row_ptr[i][0]);
    }
    if (voff[count] >= ((int64_t)1 << 31)) return fail(GILA_EINVAL, "batch has too many vertices");
    // union CSR on the host, uploaded once
    std::vector<int64_t> row((size_t)voff[count] + 1);
    std::vector<int32_t> col((size_t)eoff[count]);
    for (int32_t i = 0; i < count; ++i) {
        const int64_t b0 = row_ptr[i][0];
        for (int64_t u = 0; u < n[i]; ++u) row[voff[i] + u] = eoff[i] + (row_ptr[i][u] - b0);
        for (int64_t j = 0; j < eoff[i + 1] - eoff[i]; ++j)
            col[eoff[i] + j] = (int32_t)(voff[i] + col_idx[i][b0 + j]);
    }
    row[voff[count]] = eoff[count];
    gila_batch* b = new (std::nothrow) gila_batch();
    if (!b) return fail(GILA_ENOMEM, "host allocation");
    gila_status s = gila_graph_create(voff[count], row.data(), col.data(), 0, &b->g);
    if (s != GILA_OK) {
        delete b;
        return s;
    }
    b->count = count;
    b->voff_h = voff;
    s = batch_finish_create(b);
    if (s != GILA_OK) {
        gila_batch_destroy(b);
        return s;
    }
    *out = b;
    return GILA_OK;
}

void gila_batch_destroy(gila_batch* b)
{
    if (!b) return;
    if (b->g) cudaSetDevice(b->g->device);
    if (b->own) cudaStreamSynchronize(b->own);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->own) cudaStreamDestroy(b->own);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    cudaFree(b->voff);
    cudaFree(b->order);
    cudaFree(b->work);
    cudaFree(b->geo);
    cudaFree(b->tmp);
    cudaFree(b->pos[0]);
    cudaFree(b->pos[1]);
    cudaFree(b->stage);
    gila_graph_destroy(b->g);
    delete b;
}

gila_status gila_batch_set_stream(gila_batch* b, void* cuda_stream)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    b->user = (cudaStream_t)cuda_stream;
    return gila_graph_set_stream(b->g, cuda_stream);
}

gila_status gila_batch_info(const gila_batch* b, int32_t* count, int64_t* total_n,
                            int64_t* nnz_khop)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    if (count) *count = b->count;
    if (total_n) *total_n = b->g->n;
    if (nnz_khop) *nnz_khop = b->g->k_built ? b->g->nnz_khop : 0;
    return GILA_OK;
}

gila_status gila_batch_build_khop(gila_batch* b, int32_t k, int64_t* nnz_out)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    return gila_build_khop(b->g, k, nnz_out);
}

gila_status gila_batch_khop_reset(gila_batch* b)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    return gila_khop_reset(b->g);
}

gila_status gila_batch_khop_export(const gila_batch* b, int64_t* krow_host, int32_t* kcol_host)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    return gila_khop_export(b->g, krow_host, kcol_host);
}

gila_status gila_batch_tune(gila_batch* b, const gila_batch_tuning* t)
{
    if (!b || !t) return fail(GILA_EINVAL, "batch or tuning is NULL");
    if (t->threads != 0 && t->threads != 256 && t->threads != 512 && t->threads != 1024)
        return fail(GILA_EINVAL, "threads must be 256, 512 or 1024");
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 8) return fail(GILA_EINVAL, "ctas_per_sm in [0, 8]");
    b->tune = *t;
    return GILA_OK;
}

gila_status gila_batch_get_tuning(const gila_batch* b, int32_t precision, gila_batch_tuning* out)
{
    if (!b || !out) return fail(GILA_EINVAL, "batch or out is NULL");
    *out = resolved(b, is_f64(precision) ? 16 : 8, sm_count(b->g->device));
    return GILA_OK;
}

gila_status gila_batch_autotune(gila_batch* b, const gila_params* prm, const void* pos_dev,
                                int32_t probe_iters, gila_batch_tuning* chosen)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    gila_status s = check_batch_params(prm);
    if (s != GILA_OK) return s;
    if (probe_iters < 1) return fail(GILA_EINVAL, "probe_iters must be >= 1");
    gila_graph* g = b->g;
    if (g->n > 0 && !pos_dev) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(g->device));
    s = gila_build_khop(g, prm->k, nullptr);
    if (s != GILA_OK) return s;
    const size_t esz = is_f64(prm->precision) ? 16 : 8;
    const size_t bytes = esz * (size_t)g->n;
    if ((s = ensure(&b->pos[1], &b->pos_cap[1], bytes)) != GILA_OK) return s;
    gila_params q = *prm;
    q.iters = probe_iters;
    static const int kThreadsSet[3] = {256, 512, 1024};
    static const int kCtasSet[4] = {1, 2, 4, 8};
    static const int kGroups[3][3] = {{8, 24, 64}, {4, 12, 32}, {16, 48, 128}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GILA_CUDA(cudaEventCreate(&e0));
    GILA_CUDA(cudaEventCreate(&e1));
    const gila_batch_tuning saved = b->tune;
    gila_batch_tuning best = saved;
    float best_ms = INFINITY;
    s = GILA_OK;
    for (int ti = 0; ti < 3 && s == GILA_OK; ++ti)
        for (int ci = 0; ci < 4 && s == GILA_OK; ++ci) {
            if (kCtasSet[ci] * kThreadsSet[ti] > 2048) continue;
            for (int gi = 0; gi < 3 && s == GILA_OK; ++gi) {
                gila_batch_tuning c = {kThreadsSet[ti], kCtasSet[ci], kGroups[gi][0],
                                       kGroups[gi][1], kGroups[gi][2]};
                b->tune = c;
                float ms = 0.0f;
                for (int rep = 0; rep < 2 && s == GILA_OK; ++rep) {  // first run captures
                    if (bytes)
                        cudaMemcpyAsync(b->pos[1], pos_dev, bytes, cudaMemcpyDeviceToDevice,
                                        b->user);
                    cudaEventRecord(e0, b->user);
                    s = batch_run(b, &q, b->pos[1]);
                    cudaEventRecord(e1, b->user);
                }
                if (s != GILA_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    s = cuda_fail(e, "autotune timing");
                    break;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tune = (s == GILA_OK) ? best : saved;
    if (s != GILA_OK) return s;
    if (chosen) *chosen = resolved(b, esz, sm_count(g->device));
    return GILA_OK;
}

gila_status gila_layout_batch_device(gila_batch* b, const gila_params* prm, void* pos_dev_inout)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    gila_status s = check_batch_params(prm);
    if (s != GILA_OK) return s;
    if (b->g->n > 0 && !pos_dev_inout) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(b->g->device));
    s = gila_build_khop(b->g, prm->k, nullptr);
    if (s != GILA_OK) return s;
    return batch_run(b, prm, pos_dev_inout);
}

gila_status gila_layout_batch_run(gila_batch* b, const gila_params* prm, const double* pos_in_host,
                                  double* pos_out_host)
{
    if (!b) return fail(GILA_EINVAL, "batch is NULL");
    gila_status s = check_batch_params(prm);
    if (s != GILA_OK) return s;
    gila_graph* g = b->g;
    if (g->n > 0 && (!pos_in_host || !pos_out_host)) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(g->device));
    s = gila_build_khop(g, prm->k, nullptr);
    if (s != GILA_OK) return s;
    if (g->n == 0) return GILA_OK;
    const size_t n = (size_t)g->n;
    const bool f64 = is_f64(prm->precision);
    const size_t esz = f64 ? 16 : 8;
    if ((s = ensure(&b->pos[0], &b->pos_cap[0], esz * n)) != GILA_OK) return s;
    if (!f64 && (s = ensure((void**)&b->stage, &b->stage_cap, 16 * n)) != GILA_OK) return s;
    if (f64) {
        GILA_CUDA(cudaMemcpyAsync(b->pos[0], pos_in_host, 16 * n, cudaMemcpyHostToDevice, b->user));
    } else {
        GILA_CUDA(cudaMemcpyAsync(b->stage, pos_in_host, 16 * n, cudaMemcpyHostToDevice, b->user));
        if ((s = convert_positions(g, prm->precision, b->stage, b->pos[0], true)) != GILA_OK)
            return s;
    }
    if ((s = batch_run(b, prm, b->pos[0])) != GILA_OK) return s;
    if (f64) {
        GILA_CUDA(cudaMemcpyAsync(pos_out_host, b->pos[0], 16 * n, cudaMemcpyDeviceToHost, b->user));
    } else {
        if ((s = convert_positions(g, prm->precision, b->stage, b->pos[0], false)) != GILA_OK)
            return s;
        GILA_CUDA(cudaMemcpyAsync(pos_out_host, b->stage, 16 * n, cudaMemcpyDeviceToHost, b->user));
    }
    GILA_CUDA(cudaStreamSynchronize(b->user));
    return GILA_OK;
}

gila_status gila_layout_batch(gila_graph* const* gs, int32_t count, const gila_params* prm,
                              const double* const* pos_in, double* const* pos_out)
{
    if (count < 0) return fail(GILA_EINVAL, "count must be >= 0");
    if (count > 0 && (!gs || !pos_in || !pos_out)) return fail(GILA_EINVAL, "array is NULL");
    gila_status s = check_batch_params(prm);
    if (s != GILA_OK) return s;
    if (count == 0) return GILA_OK;
    for (int32_t i = 0; i < count; ++i)
        if (!gs[i] || gs[i]->device != gs[0]->device)
            return fail(GILA_EINVAL, "graphs must be non-NULL and on one device");
    GILA_CUDA(cudaSetDevice(gs[0]->device));
    cudaStream_t st = gs[0]->stream;
    // pack the graphs' device CSRs into one union graph
    std::vector<int64_t> voff(count + 1, 0), eoff(count + 1, 0);
    std::vector<PackSrc> src(count);
    for (int32_t i = 0; i < count; ++i) {
        voff[i + 1] = voff[i] + gs[i]->n;
        eoff[i + 1] = eoff[i] + gs[i]->nnz_adj;
        src[i] = PackSrc{gs[i]->row, gs[i]->col, gs[i]->n, voff[i], eoff[i]};
    }
    if (voff[count] >= ((int64_t)1 << 31)) return fail(GILA_EINVAL, "batch has too many vertices");
    gila_batch* b = new (std::nothrow) gila_batch();
    if (!b) return fail(GILA_ENOMEM, "host allocation");
    b->g = new (std::nothrow) gila_graph();
    if (!b->g) {
        delete b;
        return fail(GILA_ENOMEM, "host allocation");
    }
    gila_graph* g = b->g;
    g->device = gs[0]->device;
    g->n = voff[count];
    g->nnz_adj = eoff[count];
    g->stream = st;
    b->user = st;
    b->count = count;
    b->voff_h = voff;
    PackSrc* dsrc = nullptr;
    cudaError_t e = cudaMalloc(&g->row, sizeof(int64_t) * (size_t)(g->n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int32_t) * (size_t)std::max<int64_t>(g->nnz_adj, 1));
    if (e == cudaSuccess) e = cudaMalloc(&dsrc, sizeof(PackSrc) * count);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsrc, src.data(), sizeof(PackSrc) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        pack_kernel<<<count, 256, 0, st>>>(dsrc, g->row, g->col);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->row + g->n, &eoff[count], sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dsrc);
    if (e != cudaSuccess) {
        gila_batch_destroy(b);
        return cuda_fail(e, "batch pack");
    }
    s = batch_finish_create(b);
    std::vector<double> in, outv;
    if (s == GILA_OK) {
        in.resize(2 * (size_t)g->n);
        outv.resize(2 * (size_t)g->n);
        for (int32_t i = 0; i < count; ++i)
            if (gs[i]->n > 0)
                memcpy(in.data() + 2 * voff[i], pos_in[i], sizeof(double) * 2 * gs[i]->n);
        s = gila_layout_batch_run(b, prm, in.data(), outv.data());
    }
    if (s == GILA_OK)
        for (int32_t i = 0; i < count; ++i)
            if (gs[i]->n > 0)
                memcpy(pos_out[i], outv.data() + 2 * voff[i], sizeof(double) * 2 * gs[i]->n);
    gila_batch_destroy(b);
    return s;
}

}  // extern "C"
