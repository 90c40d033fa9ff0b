// Per-component layout (Section 4.6: the pipeline runs on every connected
// component, and the component drawings are arranged without overlap;
// Section 5.1: each component's maximum displacement follows its own n and
// initial frame).
//
// Components are found on the device by hooking and pointer jumping: every
// vertex starts as its own parent; a round lowers the parent of a vertex's
// root to the smallest parent seen across its edges (atomicMin, so values
// only fall and stay inside the component) and then points every vertex at
// its root. The unique fixed point labels every vertex with the smallest id
// of its component, so the result does not depend on scheduling. A scan of
// the roots numbers the components in that order.
//
// The layout then runs each component on its own: components of up to
// kBatchMaxN vertices together in one persistent batch launch (each graph of
// a batch follows its own temperature schedule), larger ones as ordinary
// graphs (blocked or plain kernels), isolated vertices stay where they are.
// Finally the drawings are packed into rows ("arranged in a matrix"): boxes
// by decreasing vertex count (ties by component index), left to right with a
// gap, a new row when the next box would pass the width
// W = max(widest box, sqrt(sum of (width + gap)(height + gap))).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "gila_impl.h"

namespace gila {

namespace {

constexpr int kCThreads = 256;
constexpr int64_t kBatchMaxN = 4096;  // largest component laid out in the batch launch

unsigned cblocks(int64_t n)
{
    return (unsigned)std::max<int64_t>(1, (n + kCThreads - 1) / kCThreads);
}

__global__ void cc_init_kernel(int64_t n, int32_t* __restrict__ comp)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) comp[v] = (int32_t)v;
}

__global__ void cc_hook_kernel(int64_t n, const int64_t* __restrict__ row,
                               const int32_t* __restrict__ col, int32_t* comp, int* changed)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t cv = comp[v];
    int32_t low = cv;
    for (int64_t e = row[v]; e < row[v + 1]; ++e) low = min(low, comp[col[e]]);
    if (low < cv) {
        atomicMin(&comp[cv], low);
        *changed = 1;
    }
}

__global__ void cc_jump_kernel(int64_t n, int32_t* comp)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t c = comp[v];
    for (;;) {
        const int32_t cc = comp[c];
        if (cc == c) break;
        c = cc;
    }
    comp[v] = c;
}

__global__ void cc_roots_kernel(int64_t n, const int32_t* __restrict__ comp,
                                int64_t* __restrict__ is_root)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) is_root[v] = comp[v] == (int32_t)v ? 1 : 0;
}

__global__ void cc_label_kernel(int64_t n, const int32_t* __restrict__ comp,
                                const int64_t* __restrict__ scan, int32_t* __restrict__ label)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) label[v] = (int32_t)scan[comp[v]];
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

// Labels of the connected components into label_host (int32[n]); *count.
gila_status components_labels(gila_graph* g, int32_t* label_host, int32_t* count)
{
    const int64_t n = g->n;
    *count = 0;
    if (n == 0) return GILA_OK;
    cudaStream_t st = g->stream;
    DevBuf comp, flag, roots, scan, label;
    GILA_CUDA(cudaMalloc(&comp.p, sizeof(int32_t) * (size_t)n));
    GILA_CUDA(cudaMalloc(&flag.p, sizeof(int)));
    GILA_CUDA(cudaMalloc(&roots.p, sizeof(int64_t) * (size_t)n));
    GILA_CUDA(cudaMalloc(&scan.p, sizeof(int64_t) * (size_t)(n + 1)));
    GILA_CUDA(cudaMalloc(&label.p, sizeof(int32_t) * (size_t)n));
    int32_t* c = (int32_t*)comp.p;
    cc_init_kernel<<<cblocks(n), kCThreads, 0, st>>>(n, c);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    // each round at least halves the depth of the forest; a path of n
    // vertices needs about log2(n) rounds, so 64 rounds bound any graph here
    for (int round = 0;; ++round) {
        if (round >= 64) return fail(GILA_ECUDA, "components did not converge");
        int changed = 0;
        GILA_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
        cc_hook_kernel<<<cblocks(n), kCThreads, 0, st>>>(n, g->row, g->col, c, (int*)flag.p);
        count_launch();
        cc_jump_kernel<<<cblocks(n), kCThreads, 0, st>>>(n, c);
        count_launch();
        GILA_CUDA(cudaGetLastError());
        GILA_CUDA(cudaMemcpyAsync(&changed, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        GILA_CUDA(cudaStreamSynchronize(st));
        if (!changed) break;
    }
    cc_roots_kernel<<<cblocks(n), kCThreads, 0, st>>>(n, c, (int64_t*)roots.p);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    gila_status s = scan_exclusive_i64((const int64_t*)roots.p, n, (int64_t*)scan.p, st);
    if (s != GILA_OK) return s;
    cc_label_kernel<<<cblocks(n), kCThreads, 0, st>>>(n, c, (const int64_t*)scan.p,
                                                      (int32_t*)label.p);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    int64_t total = 0;
    GILA_CUDA(cudaMemcpyAsync(&total, (int64_t*)scan.p + n, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaMemcpyAsync(label_host, label.p, sizeof(int32_t) * (size_t)n,
                              cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    *count = (int32_t)total;
    return GILA_OK;
}

}  // namespace gila

using namespace gila;

extern "C" {

gila_status gila_graph_components(gila_graph* g, int32_t* label_host, int32_t* count)
{
    if (!g || (g->n > 0 && !label_host)) return fail(GILA_EINVAL, "graph or labels is NULL");
    GILA_CUDA(cudaSetDevice(g->device));
    int32_t c = 0;
    gila_status s = components_labels(g, label_host, &c);
    if (s == GILA_OK && count) *count = c;
    return s;
}

gila_status gila_layout_components_run(gila_graph* g, const gila_params* prm, double gap,
                                       const double* pos_in_host, double* pos_out_host,
                                       int32_t* count_out)
{
    if (!g || !prm) return fail(GILA_EINVAL, "graph or params is NULL");
    if (g->n > 0 && (!pos_in_host || !pos_out_host)) return fail(GILA_EINVAL, "placement is NULL");
    GILA_CUDA(cudaSetDevice(g->device));
    const int64_t n = g->n;
    if (count_out) *count_out = 0;
    if (n == 0) return GILA_OK;
    if (!(gap > 0.0)) gap = prm->d;
    std::vector<int32_t> label((size_t)n);
    int32_t count = 0;
    gila_status s = components_labels(g, label.data(), &count);
    if (s != GILA_OK) return s;
    if (count_out) *count_out = count;
    // host copy of the adjacency, vertices grouped by component (ascending ids)
    std::vector<int64_t> row((size_t)n + 1);
    std::vector<int32_t> col((size_t)std::max<int64_t>(g->nnz_adj, 1));
    GILA_CUDA(cudaMemcpy(row.data(), g->row, sizeof(int64_t) * (size_t)(n + 1),
                         cudaMemcpyDeviceToHost));
    if (g->nnz_adj > 0)
        GILA_CUDA(cudaMemcpy(col.data(), g->col, sizeof(int32_t) * (size_t)g->nnz_adj,
                             cudaMemcpyDeviceToHost));
    std::vector<int64_t> size((size_t)count, 0), start((size_t)count + 1, 0);
    for (int64_t v = 0; v < n; ++v) ++size[(size_t)label[(size_t)v]];
    for (int32_t c = 0; c < count; ++c) start[(size_t)c + 1] = start[(size_t)c] + size[(size_t)c];
    std::vector<int32_t> order((size_t)n), local((size_t)n);
    {
        std::vector<int64_t> cur(start.begin(), start.end() - 1);
        for (int64_t v = 0; v < n; ++v) {
            const int32_t c = label[(size_t)v];
            local[(size_t)v] = (int32_t)(cur[(size_t)c] - start[(size_t)c]);
            order[(size_t)cur[(size_t)c]++] = (int32_t)v;
        }
    }
    // per-component CSR (local ids) and initial placement
    struct Comp {
        std::vector<int64_t> row;
        std::vector<int32_t> col;
        std::vector<double> pos;
    };
    std::vector<Comp> comps((size_t)count);
    std::vector<int32_t> small, large;
    for (int32_t c = 0; c < count; ++c) {
        const int64_t nc = size[(size_t)c];
        Comp& C = comps[(size_t)c];
        C.row.assign((size_t)nc + 1, 0);
        C.pos.resize(2 * (size_t)nc);
        for (int64_t i = 0; i < nc; ++i) {
            const int32_t v = order[(size_t)(start[(size_t)c] + i)];
            C.row[(size_t)i + 1] = C.row[(size_t)i] + (row[(size_t)v + 1] - row[(size_t)v]);
            C.pos[2 * (size_t)i] = pos_in_host[2 * (size_t)v];
            C.pos[2 * (size_t)i + 1] = pos_in_host[2 * (size_t)v + 1];
        }
        C.col.resize((size_t)std::max<int64_t>(C.row[(size_t)nc], 1));
        for (int64_t i = 0, o = 0; i < nc; ++i) {
            const int32_t v = order[(size_t)(start[(size_t)c] + i)];
            for (int64_t e = row[(size_t)v]; e < row[(size_t)v + 1]; ++e)
                C.col[(size_t)o++] = local[(size_t)col[(size_t)e]];
        }
        if (nc == 1) continue;  // an isolated vertex feels no force
        if (nc <= kBatchMaxN && prm->precision != GILA_FP64_ORDERED) small.push_back(c);
        else large.push_back(c);
    }
    std::vector<std::vector<double>> result((size_t)count);
    for (int32_t c = 0; c < count; ++c) result[(size_t)c] = comps[(size_t)c].pos;
    // small components: one persistent batch launch
    if (!small.empty()) {
        std::vector<int64_t> bn;
        std::vector<const int64_t*> brow;
        std::vector<const int32_t*> bcol;
        std::vector<double> bin, bout;
        for (int32_t c : small) {
            bn.push_back(size[(size_t)c]);
            brow.push_back(comps[(size_t)c].row.data());
            bcol.push_back(comps[(size_t)c].col.data());
            bin.insert(bin.end(), comps[(size_t)c].pos.begin(), comps[(size_t)c].pos.end());
        }
        bout.resize(bin.size());
        gila_batch* b = nullptr;
        s = gila_batch_create((int32_t)small.size(), bn.data(), brow.data(), bcol.data(), 0, &b);
        if (s != GILA_OK) return s;
        if ((s = gila_batch_set_stream(b, g->stream)) == GILA_OK)
            s = gila_layout_batch_run(b, prm, bin.data(), bout.data());
        gila_batch_destroy(b);
        if (s != GILA_OK) return s;
        size_t o = 0;
        for (int32_t c : small) {
            const size_t m = 2 * (size_t)size[(size_t)c];
            result[(size_t)c].assign(bout.begin() + (std::ptrdiff_t)o,
                                     bout.begin() + (std::ptrdiff_t)(o + m));
            o += m;
        }
    }
    // large components: one ordinary layout each
    for (int32_t c : large) {
        gila_graph* h = nullptr;
        const Comp& C = comps[(size_t)c];
        s = gila_graph_create(size[(size_t)c], C.row.data(), C.col.data(), 0, &h);
        if (s != GILA_OK) return s;
        h->stream = g->stream;
        h->tune = g->tune;
        s = gila_layout_run(h, prm, C.pos.data(), result[(size_t)c].data(), nullptr);
        gila_graph_destroy(h);
        if (s != GILA_OK) return s;
    }
    // pack the drawings into rows
    std::vector<double> box(4 * (size_t)count);
    double area = 0.0, widest = 0.0;
    for (int32_t c = 0; c < count; ++c) {
        const std::vector<double>& r = result[(size_t)c];
        double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
        for (size_t i = 0; i < r.size(); i += 2) {
            x0 = std::min(x0, r[i]);
            x1 = std::max(x1, r[i]);
            y0 = std::min(y0, r[i + 1]);
            y1 = std::max(y1, r[i + 1]);
        }
        box[4 * (size_t)c] = x0;
        box[4 * (size_t)c + 1] = y0;
        box[4 * (size_t)c + 2] = x1;
        box[4 * (size_t)c + 3] = y1;
        area += (x1 - x0 + gap) * (y1 - y0 + gap);
        widest = std::max(widest, x1 - x0);
    }
    std::vector<int32_t> by_size((size_t)count);
    std::iota(by_size.begin(), by_size.end(), 0);
    std::stable_sort(by_size.begin(), by_size.end(), [&](int32_t a, int32_t b) {
        return size[(size_t)a] > size[(size_t)b];
    });
    const double W = std::max(widest, std::sqrt(area));
    double x = 0.0, y = 0.0, row_h = 0.0;
    bool row_empty = true;
    std::vector<double> shift(2 * (size_t)count);
    for (int32_t c : by_size) {
        const double w = box[4 * (size_t)c + 2] - box[4 * (size_t)c];
        const double h = box[4 * (size_t)c + 3] - box[4 * (size_t)c + 1];
        if (!row_empty && x + w > W) {
            y += row_h + gap;
            x = 0.0;
            row_h = 0.0;
            row_empty = true;
        }
        shift[2 * (size_t)c] = x - box[4 * (size_t)c];
        shift[2 * (size_t)c + 1] = y - box[4 * (size_t)c + 1];
        x += w + gap;
        row_h = std::max(row_h, h);
        row_empty = false;
    }
    for (int32_t c = 0; c < count; ++c) {
        const std::vector<double>& r = result[(size_t)c];
        for (int64_t i = 0; i < size[(size_t)c]; ++i) {
            const int32_t v = order[(size_t)(start[(size_t)c] + i)];
            pos_out_host[2 * (size_t)v] = r[2 * (size_t)i] + shift[2 * (size_t)c];
            pos_out_host[2 * (size_t)v + 1] = r[2 * (size_t)i + 1] + shift[2 * (size_t)c + 1];
        }
    }
    return GILA_OK;
}

}  // extern "C"
