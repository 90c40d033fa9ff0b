// One layout iteration as a single kernel launch, plus FP64 quality
// reductions and placement conversions.
//
// Iteration (Sections 3.1 and 4.5 of the paper): for every vertex u
//   F(u) = sum over v in N_u(k) of d^2/delta^q along (x_u - x_v)/delta
//        + sum over edges (u,v)  of delta^p/d along (x_v - x_u)/delta
//   x_u <- x_u + F(u) min(1, t/|F(u)|), all vertices at once.
// Per entry of a k-hop row the kernels compute Delta = x_u - x_v and add
// d^2/delta^(q+1) Delta (for q = 1 in FP32: d^2 rcp(r^2) Delta, one MUFU and
// no divide); a short second pass over u's adjacency row adds the
// attraction -delta^(p-1)/d Delta. The k-hop stream is the only large read.
//
// Work is split by row length into four classes, each a range of blocks
// of the same launch (heaviest first): rows split into chunks summed by the
// last chunk to finish, one block per row, one warp per row, and groups of
// 8 lanes per row. A row's reduction order depends only on its length and
// its position in the k-hop list, so results are reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "ff.cuh"
#include "force.cuh"
#include "gila_impl.h"

namespace gila {

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

struct IterArgs {
    const int64_t* row;
    const int32_t* col;
    const int64_t* krow;
    const uint32_t* kcol;
    const int32_t* list0;
    const int32_t* list1;
    const int32_t* list2;
    const Chunk* chunks;
    int32_t* giant_counter;
    double* partials;
    int32_t n0, n1, n2, nchunks;
    int32_t b3, b2, b1, b0;  // blocks per class, launched in the order 3, 2, 1, 0
    double d, t;
    int p, q;
    const void* pos_in;
    void* pos_out;
    void* disp_out;
    const void* wt;  // repulsion weights (T[n]) or null
};

template <class T>
__device__ __forceinline__ void apply_move_it(const IterArgs& A, int64_t u, T xu, T yu, T fx,
                                              T fy)
{
    apply_move<T>(A.t, A.pos_out, A.disp_out, u, xu, yu, fx, fy);
}

// Block-wide sum of an accumulator in a fixed order (warps, then warp 0).
template <class T, bool COMP>
__device__ __forceinline__ void block_reduce(Acc<T, COMP>& a, T* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a.group_reduce(32);
    if (lane == 0) {
        sh[warp * 4 + 0] = a.sx;
        sh[warp * 4 + 1] = a.sy;
        sh[warp * 4 + 2] = a.cx;
        sh[warp * 4 + 3] = a.cy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc<T, COMP> r;
        r.sx = sh[0];
        r.sy = sh[1];
        r.cx = sh[2];
        r.cy = sh[3];
        for (int w = 1; w < kWarpsPerBlock; ++w)
            r.merge(sh[w * 4 + 0], sh[w * 4 + 1], sh[w * 4 + 2], sh[w * 4 + 3]);
        a = r;
    }
}

// Repulsion over k-hop entries [ks, ke) of u and, when with_att, attraction
// over u's adjacency row, by lanes gl = 0..G-1 of a group.
template <class T, int MODEL, bool COMP, class R, class P2>
__device__ __forceinline__ void vertex_sum(const IterArgs& A, R rep,
                                           Att<T, MODEL, COMP> att, int64_t u, P2 pu, int64_t ks,
                                           int64_t ke, bool with_att, int gl, int G,
                                           Acc<T, COMP>& a)
{
    rep.xu = pu.x;
    rep.yu = pu.y;
    row_sum(A.kcol, ks, ke, gl, G, rep, a);
    if (with_att) {
        att.xu = pu.x;
        att.yu = pu.y;
        row_sum_rel(reinterpret_cast<const uint32_t*>(A.col), A.row[u], A.row[u + 1], gl, G, att,
                    a);
    }
}

// FP32 variants are held to 32 registers so that eight 256-thread blocks
// (all 64 warps) fit an SM: the short-row classes are latency-bound and gain
// from the warps (mesh k = 3 compensated: 0.162 -> 0.145 ms per iteration);
// FP64 needs its registers.
template <class T>
constexpr int plain_min_blocks()
{
    return sizeof(T) == 4 ? 8 : 1;
}

template <class T, int MODEL, bool COMP, bool W>
__global__ void __launch_bounds__(kThreads, plain_min_blocks<T>())
iteration_kernel(const IterArgs A)
{
    using P2 = typename V2<T>::type;
    __shared__ T sh[kWarpsPerBlock * 4];
    __shared__ int s_last;
    const P2* __restrict__ pos = reinterpret_cast<const P2*>(A.pos_in);
    Rep<T, MODEL, COMP, kSrcGlobal, false, W> rep;
    rep.src.pos = pos;
    rep.d2 = (T)(A.d * A.d);
    rep.q = A.q;
    rep.wt = reinterpret_cast<const T*>(A.wt);
    Att<T, MODEL, COMP> att;
    att.src.pos = pos;
    att.inv_d = (T)(1.0 / A.d);
    att.p = A.p;
    int b = blockIdx.x;
    if (b < A.b3) {
        // a chunk of a giant row: block sum, then the last chunk finishes u;
        // the row's first chunk also carries the attraction terms
        const Chunk ch = A.chunks[b];
        const int64_t u = ch.vertex;
        const P2 pu = pos[u];
        Acc<T, COMP> a;
        vertex_sum<T, MODEL, COMP>(A, rep, att, u, pu, ch.begin, ch.end, b == ch.first, threadIdx.x, kThreads, a);
        block_reduce<T, COMP>(a, sh);
        if (threadIdx.x == 0) {
            double* part = A.partials + (int64_t)b * 4;
            part[0] = (double)a.sx;
            part[1] = (double)a.sy;
            part[2] = (double)a.cx;
            part[3] = (double)a.cy;
            __threadfence();
            const int prev = atomicAdd(&A.giant_counter[ch.giant], 1);
            s_last = (prev == ch.count - 1);
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();
            double fx = 0.0, fy = 0.0;
            for (int i = 0; i < ch.count; ++i) {
                const double* q = A.partials + (int64_t)(ch.first + i) * 4;
                fx += __ldcg(q + 0) + __ldcg(q + 2);
                fy += __ldcg(q + 1) + __ldcg(q + 3);
            }
            A.giant_counter[ch.giant] = 0;
            apply_move_it<T>(A, u, pu.x, pu.y, (T)fx, (T)fy);
        }
        return;
    }
    b -= A.b3;
    if (b < A.b2) {
        const int64_t u = A.list2[b];
        const P2 pu = pos[u];
        Acc<T, COMP> a;
        vertex_sum<T, MODEL, COMP>(A, rep, att, u, pu, A.krow[u], A.krow[u + 1], true, threadIdx.x, kThreads, a);
        block_reduce<T, COMP>(a, sh);
        if (threadIdx.x == 0) apply_move_it<T>(A, u, pu.x, pu.y, a.fx(), a.fy());
        return;
    }
    b -= A.b2;
    if (b < A.b1) {
        const int i = b * kWarpsPerBlock + (threadIdx.x >> 5);
        if (i >= A.n1) return;  // whole warp leaves together
        const int lane = threadIdx.x & 31;
        const int64_t u = A.list1[i];
        const P2 pu = pos[u];
        Acc<T, COMP> a;
        vertex_sum<T, MODEL, COMP>(A, rep, att, u, pu, A.krow[u], A.krow[u + 1], true, lane, 32, a);
        a.group_reduce(32);
        if (lane == 0) apply_move_it<T>(A, u, pu.x, pu.y, a.fx(), a.fy());
        return;
    }
    b -= A.b1;
    {
        constexpr int G = 8;
        const int gl = threadIdx.x & (G - 1);
        const int i = b * (kThreads / G) + (threadIdx.x / G);
        const bool live = i < A.n0;
        // lanes of a group stay together through the shuffles below
        const int64_t u = live ? A.list0[i] : 0;
        Acc<T, COMP> a;
        P2 pu;
        pu.x = T(0);
        pu.y = T(0);
        if (live) {
            pu = pos[u];
            vertex_sum<T, MODEL, COMP>(A, rep, att, u, pu, A.krow[u], A.krow[u + 1], true, gl, G, a);
        }
        a.group_reduce(G);
        if (live && gl == 0) apply_move_it<T>(A, u, pu.x, pu.y, a.fx(), a.fy());
    }
}

// FP64 validation mode that sums every force in the order of the definition:
// repulsion over N_u(k) by ascending id, attraction over the adjacency row in
// CSR order, each term rounded as magnitude * (component / delta), the two
// sums added last; every operation is an explicitly rounded IEEE double op
// (no fused multiply-add), so the result depends on nothing but the inputs.
// One warp per vertex: lanes form 32 consecutive terms, then every lane
// folds them in order.
__device__ __forceinline__ double ordered_pow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r = __dmul_rn(r, x);
    return r;
}

__global__ void __launch_bounds__(kThreads)
ordered_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col,
               const int64_t* __restrict__ krow, const uint32_t* __restrict__ kcol, double d,
               int p, int q, double t, const double2* __restrict__ pos_in,
               double2* __restrict__ pos_out, double2* __restrict__ disp_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t u = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    if (u >= n) return;  // whole warp
    const double2 pu = pos_in[u];
    const double dd = __dmul_rn(d, d);
    double s[2][2] = {{0.0, 0.0}, {0.0, 0.0}};  // [repulsion|attraction][x|y]
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t b = pass == 0 ? krow[u] : row[u];
        const int64_t e = pass == 0 ? krow[u + 1] : row[u + 1];
        for (int64_t j0 = b; j0 < e; j0 += 32) {
            const int64_t j = j0 + lane;
            double tx = 0.0, ty = 0.0;
            if (j < e) {
                const int64_t v = pass == 0 ? (int64_t)kcol[j] : (int64_t)col[j];
                const double2 pv = pos_in[v];
                // repulsion along x_u - x_v, attraction along x_v - x_u
                const double dx = pass == 0 ? __dsub_rn(pu.x, pv.x) : __dsub_rn(pv.x, pu.x);
                const double dy = pass == 0 ? __dsub_rn(pu.y, pv.y) : __dsub_rn(pv.y, pu.y);
                const double dl = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
                if (dl != 0.0 && v != u) {
                    const double mag = pass == 0 ? __ddiv_rn(dd, ordered_pow(dl, q))
                                                 : __ddiv_rn(ordered_pow(dl, p), d);
                    tx = __dmul_rn(mag, __ddiv_rn(dx, dl));
                    ty = __dmul_rn(mag, __ddiv_rn(dy, dl));
                } else {
                    tx = ty = -0.0;  // identity of the sum: the term is skipped
                }
            }
            const int cnt = (e - j0) < 32 ? (int)(e - j0) : 32;
            for (int i = 0; i < cnt; ++i) {
                s[pass][0] = __dadd_rn(s[pass][0], __shfl_sync(kFull, tx, i));
                s[pass][1] = __dadd_rn(s[pass][1], __shfl_sync(kFull, ty, i));
            }
        }
    }
    if (lane != 0) return;
    const double fx = __dadd_rn(s[0][0], s[1][0]);
    const double fy = __dadd_rn(s[0][1], s[1][1]);
    const double norm = __dsqrt_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)));
    double mx = fx, my = fy;
    if (norm > t) {
        const double sc = norm > 0.0 ? __ddiv_rn(t, norm) : 0.0;
        mx = __dmul_rn(fx, sc);
        my = __dmul_rn(fy, sc);
    }
    pos_out[u] = make_double2(__dadd_rn(pu.x, mx), __dadd_rn(pu.y, my));
    if (disp_out) disp_out[u] = make_double2(mx, my);
}

template <class T, int MODEL, bool COMP>
cudaError_t launch_typed(const IterArgs& A, unsigned grid, cudaStream_t st)
{
    if (A.wt)
        iteration_kernel<T, MODEL, COMP, true><<<grid, kThreads, 0, st>>>(A);
    else
        iteration_kernel<T, MODEL, COMP, false><<<grid, kThreads, 0, st>>>(A);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------- metrics

constexpr int kRedBlocks = 1216;  // a full wave of 256-thread blocks on 152 SMs
constexpr int kRedThreads = 256;

template <class T>
__device__ __forceinline__ double2 load_pos(const void* pos, int64_t u)
{
    using P2 = typename V2<T>::type;
    const P2 p = reinterpret_cast<const P2*>(pos)[u];
    return make_double2((double)p.x, (double)p.y);
}

__device__ __forceinline__ double dipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// pass 0: [sum delta, count, sum delta^p/d, sum over k-hop pairs d^2/delta^q]
// pass 1: [sum (delta - mean)^2, 0, 0, 0]
// Each warp owns a fixed set of vertices; partial sums are combined in a
// fixed order, so the result does not depend on timing.
template <class T>
__global__ void __launch_bounds__(kRedThreads)
metrics_kernel(int pass, int64_t n, const int64_t* __restrict__ row,
               const int32_t* __restrict__ col, const int64_t* __restrict__ krow,
               const uint32_t* __restrict__ kcol, const void* pos, double d, int p, int q,
               double mean, double* __restrict__ partials, int skip_khop)
{
    __shared__ double sh[kRedThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * (kRedThreads / 32);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int64_t u = (int64_t)blockIdx.x * (kRedThreads / 32) + warp; u < n; u += nw) {
        const double2 pu = load_pos<T>(pos, u);
        for (int64_t e = row[u] + lane; e < row[u + 1]; e += 32) {
            const int64_t v = col[e];
            if (v <= u) continue;
            const double2 pv = load_pos<T>(pos, v);
            const double dx = pu.x - pv.x, dy = pu.y - pv.y;
            const double dl = sqrt(dx * dx + dy * dy);
            if (pass == 0) {
                a0 += dl;
                a1 += 1.0;
                if (dl > 0.0) a2 += dipow(dl, p) / d;
            } else {
                a0 += (dl - mean) * (dl - mean);
            }
        }
        if (pass == 0 && sizeof(T) == 4 && !skip_khop) {
            // FP32 placements: each pair's term d^2 / delta^q in double-float
            // arithmetic (pairs of FP32 numbers, relative error about 1e-14,
            // far below FP32's 6e-8), eight terms per lane summed as a
            // double-float, then added in FP64. The FP64 pipe of GB300 is a
            // small fraction of its FP32 rate, and a per-pair FP64 sqrt and
            // divide made this pass ALU-bound; the pair form keeps FP64
            // accuracy at FP32 throughput.
            const float2* pf = reinterpret_cast<const float2*>(pos);
            const float2 qu = pf[u];
            const Ff d2f = ff_from_double(d * d);
            const int64_t e1 = krow[u + 1];
            for (int64_t e0 = krow[u]; e0 < e1; e0 += 256) {
                Ff s = {0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int64_t e = e0 + j * 32 + lane;
                    if (e >= e1) continue;
                    const int64_t v = kcol[e];
                    if (v <= u) continue;
                    const float2 pv = pf[v];
                    const Ff r2 = ff_dist2(qu.x, qu.y, pv.x, pv.y);
                    if (r2.hi >= 1e-30f && r2.hi <= 1e30f) {
                        s = ff_add(s, ff_mul(d2f, ff_rsqrt_pow(r2, q)));
                    } else {
                        // distances outside the pair form's safe range (or
                        // coincident vertices): the FP64 term from the exact
                        // FP64 differences, none at distance 0
                        const double dx = (double)qu.x - (double)pv.x;
                        const double dy = (double)qu.y - (double)pv.y;
                        const double dl = sqrt(dx * dx + dy * dy);
                        if (dl > 0.0) a3 += d * d / dipow(dl, q);
                    }
                }
                a3 += (double)s.hi + (double)s.lo;
            }
        } else if (pass == 0 && !skip_khop) {
            for (int64_t e = krow[u] + lane; e < krow[u + 1]; e += 32) {
                const int64_t v = kcol[e];
                if (v <= u) continue;
                const double2 pv = load_pos<T>(pos, v);
                const double dx = pu.x - pv.x, dy = pu.y - pv.y;
                const double dl = sqrt(dx * dx + dy * dy);
                if (dl > 0.0) a3 += d * d / dipow(dl, q);
            }
        }
    }
    a0 = group_sum(a0, 32);
    a1 = group_sum(a1, 32);
    a2 = group_sum(a2, 32);
    a3 = group_sum(a3, 32);
    if (lane == 0) {
        sh[warp][0] = a0;
        sh[warp][1] = a1;
        sh[warp][2] = a2;
        sh[warp][3] = a3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// Sum the per-block partials in block order (one thread per component).
__global__ void reduce_partials_kernel(const double* __restrict__ partials, int nblocks,
                                       double* __restrict__ out)
{
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * 4 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <class T>
__global__ void bbox_kernel(int64_t n, const void* pos, double* __restrict__ partials)
{
    __shared__ double sh[kRedThreads][4];
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = load_pos<T>(pos, u);
        x0 = fmin(x0, p.x);
        x1 = fmax(x1, p.x);
        y0 = fmin(y0, p.y);
        y1 = fmax(y1, p.y);
    }
    sh[threadIdx.x][0] = x0;
    sh[threadIdx.x][1] = x1;
    sh[threadIdx.x][2] = y0;
    sh[threadIdx.x][3] = y1;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < blockDim.x; ++i) {
            x0 = fmin(x0, sh[i][0]);
            x1 = fmax(x1, sh[i][1]);
            y0 = fmin(y0, sh[i][2]);
            y1 = fmax(y1, sh[i][3]);
        }
        partials[blockIdx.x * 4 + 0] = x0;
        partials[blockIdx.x * 4 + 1] = x1;
        partials[blockIdx.x * 4 + 2] = y0;
        partials[blockIdx.x * 4 + 3] = y1;
    }
}

__global__ void to_float2_kernel(int64_t n, const double* __restrict__ src, float2* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
}

__global__ void from_float2_kernel(int64_t n, const float2* __restrict__ src, double* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 p = src[i];
        dst[2 * i] = (double)p.x;
        dst[2 * i + 1] = (double)p.y;
    }
}

gila_status ensure_red(gila_graph* g, size_t doubles)
{
    return ensure((void**)&g->red, &g->red_cap, doubles * sizeof(double));
}

}  // namespace

gila_status launch_iteration(gila_graph* g, const gila_params* prm, double t, const void* pos_in,
                             void* pos_out, void* disp_out)
{
    {
        bool handled = false;
        gila_status s = launch_blocked(g, prm, t, pos_in, pos_out, disp_out, &handled);
        if (s != GILA_OK || handled) return s;
    }
    if (prm->precision == GILA_FP64_ORDERED) {
        if (g->wt64) return fail(GILA_EINVAL, "GILA_FP64_ORDERED takes no repulsion weights");
        if (g->n == 0) return GILA_OK;
        const unsigned grid = (unsigned)((g->n * 32 + kThreads - 1) / kThreads);
        cudaEvent_t pa = prof_kernel_begin(g);
        ordered_kernel<<<grid, kThreads, 0, g->stream>>>(
            g->n, g->row, g->col, g->krow, g->kcol, prm->d, prm->p, prm->q, t,
            (const double2*)pos_in, (double2*)pos_out, (double2*)disp_out);
        count_launch();
        cudaError_t e = cudaGetLastError();
        prof_kernel_end(g, pa, "ordered_kernel");
        if (e != cudaSuccess) return cuda_fail(e, "ordered_kernel");
        return GILA_OK;
    }
    const Bins& B = g->bins;
    IterArgs A;
    A.row = g->row;
    A.col = g->col;
    A.krow = g->krow;
    A.kcol = g->kcol;
    A.list0 = B.lists;
    A.list1 = B.lists + B.n0;
    A.list2 = B.lists + B.n0 + B.n1;
    A.chunks = B.chunks;
    A.giant_counter = B.giant_counter;
    A.partials = (double*)B.partials;
    A.n0 = B.n0;
    A.n1 = B.n1;
    A.n2 = B.n2;
    A.nchunks = B.nchunks;
    A.b3 = B.nchunks;
    A.b2 = B.n2;
    A.b1 = (B.n1 + kWarpsPerBlock - 1) / kWarpsPerBlock;
    A.b0 = (B.n0 + (kThreads / 8) - 1) / (kThreads / 8);
    A.d = prm->d;
    A.t = t;
    A.p = prm->p;
    A.q = prm->q;
    A.pos_in = pos_in;
    A.pos_out = pos_out;
    A.disp_out = disp_out;
    A.wt = is_f64(prm->precision) ? (const void*)g->wt64 : (const void*)g->wt32;
    const int64_t grid = (int64_t)A.b3 + A.b2 + A.b1 + A.b0;
    if (grid == 0) return GILA_OK;
    const bool fr = (prm->p == 2 && prm->q == 1);
    cudaError_t e;
    cudaEvent_t pa = prof_kernel_begin(g);
    switch (prm->precision) {
    case GILA_FP64:
        e = fr ? launch_typed<double, kFR, false>(A, (unsigned)grid, g->stream)
               : launch_typed<double, kGeneric, false>(A, (unsigned)grid, g->stream);
        break;
    case GILA_FP32_COMPENSATED:
        e = fr ? launch_typed<float, kFR, true>(A, (unsigned)grid, g->stream)
               : launch_typed<float, kGeneric, true>(A, (unsigned)grid, g->stream);
        break;
    default:
        e = fr ? launch_typed<float, kFR, false>(A, (unsigned)grid, g->stream)
               : launch_typed<float, kGeneric, false>(A, (unsigned)grid, g->stream);
        break;
    }
    prof_kernel_end(g, pa, "iteration_kernel");
    if (e != cudaSuccess) return cuda_fail(e, "iteration_kernel");
    return GILA_OK;
}

gila_status compute_metrics(gila_graph* g, const gila_params* prm, const void* pos,
                            gila_metrics* out)
{
    gila_status s = ensure_red(g, (size_t)kRedBlocks * 4 + 8);
    if (s != GILA_OK) return s;
    double* part = g->red;
    double* res = g->red + (size_t)kRedBlocks * 4;
    double h[4];
    const bool f64 = is_f64(prm->precision);
    // FP32 placements with a blocked plan take the k-hop term over the
    // plan's shared-memory position tiles (the pairs' positions are
    // otherwise random gathers through L2); the edge terms stay here
    bool tiled = false;
    double rep_tiled = 0.0;
    {
        gila_status bs = blocked_khop_metric(g, prm, pos, &tiled, &rep_tiled);
        if (bs != GILA_OK) return bs;
    }
    auto run = [&](int pass, double mean) -> cudaError_t {
        if (f64)
            metrics_kernel<double><<<kRedBlocks, kRedThreads, 0, g->stream>>>(
                pass, g->n, g->row, g->col, g->krow, g->kcol, pos, prm->d, prm->p, prm->q, mean,
                part, 0);
        else
            metrics_kernel<float><<<kRedBlocks, kRedThreads, 0, g->stream>>>(
                pass, g->n, g->row, g->col, g->krow, g->kcol, pos, prm->d, prm->p, prm->q, mean,
                part, tiled ? 1 : 0);
        count_launch();
        reduce_partials_kernel<<<1, 32, 0, g->stream>>>(part, kRedBlocks, res);
        count_launch();
        cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
        return cudaStreamSynchronize(g->stream);
    };
    cudaError_t e = run(0, 0.0);
    if (e != cudaSuccess) return cuda_fail(e, "metrics pass 0");
    const double m = h[1];
    const double mean = m > 0 ? h[0] / m : 0.0;
    const double att = h[2], rep = tiled ? rep_tiled : h[3];
    e = run(1, mean);
    if (e != cudaSuccess) return cuda_fail(e, "metrics pass 1");
    const double var = m > 0 ? h[0] / m : 0.0;
    out->edge_mean = mean;
    out->edge_std = sqrt(var);
    out->edge_cv = mean > 0 ? out->edge_std / mean : 0.0;
    out->rep_total = rep;
    out->att_total = att;
    out->rep_att_ratio = att > 0 ? rep / att : 0.0;
    return GILA_OK;
}

gila_status bbox_aspect(gila_graph* g, int precision, const void* pos, double* aspect)
{
    gila_status s = ensure_red(g, (size_t)kRedBlocks * 4 + 8);
    if (s != GILA_OK) return s;
    const int blocks = 64;
    if (is_f64(precision))
        bbox_kernel<double><<<blocks, kRedThreads, 0, g->stream>>>(g->n, pos, g->red);
    else
        bbox_kernel<float><<<blocks, kRedThreads, 0, g->stream>>>(g->n, pos, g->red);
    count_launch();
    std::vector<double> h(blocks * 4);
    GILA_CUDA(cudaMemcpyAsync(h.data(), g->red, sizeof(double) * blocks * 4,
                              cudaMemcpyDeviceToHost, g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int b = 0; b < blocks; ++b) {
        x0 = std::min(x0, h[b * 4 + 0]);
        x1 = std::max(x1, h[b * 4 + 1]);
        y0 = std::min(y0, h[b * 4 + 2]);
        y1 = std::max(y1, h[b * 4 + 3]);
    }
    const double w = x1 - x0, hh = y1 - y0;
    *aspect = (w > 0 && hh > 0) ? hh / w : 1.0;
    return GILA_OK;
}

gila_status convert_positions(gila_graph* g, int precision, const double* src, void* dst,
                              bool to_device_type)
{
    // FP64 placements need no conversion; callers copy them directly.
    if (is_f64(precision)) return GILA_OK;
    const int64_t n = g->n;
    if (n == 0) return GILA_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (to_device_type)
        to_float2_kernel<<<grid, 256, 0, g->stream>>>(n, src, (float2*)dst);
    else
        from_float2_kernel<<<grid, 256, 0, g->stream>>>(n, (const float2*)dst, (double*)src);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    return GILA_OK;
}

__global__ void weights_to_f32_kernel(int64_t n, const double* __restrict__ w,
                                      float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)w[i];
}

gila_status set_repulsion_weights(gila_graph* g, const double* w, bool w_on_device)
{
    if (!w) {
        cudaFree(g->wt64);
        cudaFree(g->wt32);
        g->wt64 = nullptr;
        g->wt32 = nullptr;
        return GILA_OK;
    }
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    if (!g->wt64) GILA_CUDA(cudaMalloc(&g->wt64, sizeof(double) * n));
    if (!g->wt32) GILA_CUDA(cudaMalloc(&g->wt32, sizeof(float) * n));
    if (g->n == 0) return GILA_OK;
    GILA_CUDA(cudaMemcpyAsync(g->wt64, w, sizeof(double) * (size_t)g->n,
                              w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              g->stream));
    weights_to_f32_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, g->stream>>>(g->n, g->wt64,
                                                                              g->wt32);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    return GILA_OK;
}

void free_layout(gila_graph* g)
{
    cudaFree(g->pos[0]);
    cudaFree(g->pos[1]);
    cudaFree(g->stage);
    cudaFree(g->red);
    cudaFree(g->wt64);
    cudaFree(g->wt32);
    g->wt64 = nullptr;
    g->wt32 = nullptr;
    free_tile_plans(g);
    g->pos[0] = g->pos[1] = nullptr;
    g->stage = nullptr;
    g->red = nullptr;
    g->pos_cap[0] = g->pos_cap[1] = 0;
    g->stage_cap = 0;
    g->red_cap = 0;
}

}  // namespace gila
