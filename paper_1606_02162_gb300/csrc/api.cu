// C ABI of libgila: argument checks, host-side CSR validation, buffer
// management, cooling schedules and the iteration loops. The compute runs
// in the kernels of khop.cu and layout.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gila_impl.h"

namespace gila {

static thread_local std::string t_err;
static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaEvent_t prof_kernel_begin(gila_graph* g)
{
    if (g->prof_on < 2) return nullptr;
    cudaEvent_t a = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaEventRecord(a, g->stream);
    return a;
}

void prof_kernel_end(gila_graph* g, cudaEvent_t a, const char* name)
{
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(a);
        return;
    }
    cudaEventRecord(b, g->stream);
    g->prof.push_back(ProfileRec{a, b, 2, 1});
    g->prof_kernel_name = name;
}

void set_error(const std::string& msg) { t_err = msg; }

gila_status fail(gila_status s, const std::string& msg)
{
    t_err = msg;
    return s;
}

gila_status cuda_fail(cudaError_t e, const char* what)
{
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error so later calls can report their own
    return e == cudaErrorMemoryAllocation ? GILA_ENOMEM : GILA_ECUDA;
}

gila_status ensure(void** p, size_t* cap, size_t bytes)
{
    if (*p && *cap >= bytes) return GILA_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(GILA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    *cap = bytes;
    return GILA_OK;
}

namespace {

gila_status check_params(const gila_params* p)
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
        p->precision != GILA_FP32_COMPENSATED && p->precision != GILA_FP64_ORDERED)
        return fail(GILA_EINVAL, "unknown precision");
    return GILA_OK;
}

size_t pos_elem(int precision) { return is_f64(precision) ? 16 : 8; }

gila_status use_device(const gila_graph* g)
{
    GILA_CUDA(cudaSetDevice(g->device));
    return GILA_OK;
}

gila_status ensure_khop(gila_graph* g, int k)
{
    if (g->k_built == k) return GILA_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    if (g->prof_on) {
        GILA_CUDA(cudaEventCreate(&a));
        GILA_CUDA(cudaEventCreate(&b));
        GILA_CUDA(cudaEventRecord(a, g->stream));
    }
    g->k_built = 0;
    invalidate_tile_plans(g);
    gila_status s = build_khop(g, k);
    if (g->prof_on) {
        cudaEventRecord(b, g->stream);
        g->prof.push_back(ProfileRec{a, b, 0, 1});
    }
    return s;
}

// prepare_iteration (the blocked-path plan, once per k-hop build) inside a
// build-kind profile record, so that iteration timings hold iterations only.
gila_status timed_prepare(gila_graph* g, const gila_params* prm)
{
    const int w = is_f64(prm->precision) ? 1 : 0;
    if (prm->precision == GILA_FP64_ORDERED || g->n == 0 || g->tplan[w].ready)
        return GILA_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    if (g->prof_on) {
        GILA_CUDA(cudaEventCreate(&a));
        GILA_CUDA(cudaEventCreate(&b));
        GILA_CUDA(cudaEventRecord(a, g->stream));
    }
    gila_status s = prepare_iteration(g, prm);
    if (a) {
        cudaEventRecord(b, g->stream);
        g->prof.push_back(ProfileRec{a, b, 0, 0});
    }
    return s;
}

// Temperature of iteration i (0-based) of prm->iters.
double temperature(const gila_params* prm, double t0, int i)
{
    if (prm->schedule == GILA_COOL_GEOMETRIC) return t0 * std::pow(0.93, (double)i);
    return t0 * (double)(prm->iters - i) / (double)prm->iters;
}

gila_status resolve_t0(gila_graph* g, const gila_params* prm, const void* pos_dev, double* t0)
{
    if (prm->t0 > 0.0) {
        *t0 = prm->t0;
        return GILA_OK;
    }
    if (prm->schedule != GILA_COOL_GEOMETRIC) {
        *t0 = 0.1 * std::sqrt((double)g->n);
        return GILA_OK;
    }
    double a = 1.0;
    gila_status s = bbox_aspect(g, prm->precision, pos_dev, &a);
    if (s != GILA_OK) return s;
    *t0 = std::sqrt((double)g->n * prm->d / a);
    return GILA_OK;
}

gila_status run_loop(gila_graph* g, const gila_params* prm, void* pos, void* tmp)
{
    double t0 = 0.0;
    gila_status s = resolve_t0(g, prm, pos, &t0);
    if (s != GILA_OK) return s;
    // the one-time blocked-path plan of the current k-hop lists, timed with
    // the build when profiling
    if ((s = timed_prepare(g, prm)) != GILA_OK) return s;
    cudaEvent_t a = nullptr, b = nullptr;
    if (g->prof_on && prm->iters > 0) {
        GILA_CUDA(cudaEventCreate(&a));
        GILA_CUDA(cudaEventCreate(&b));
        GILA_CUDA(cudaEventRecord(a, g->stream));
    }
    void* buf[2] = {pos, tmp};
    for (int i = 0; i < prm->iters; ++i) {
        s = launch_iteration(g, prm, temperature(prm, t0, i), buf[i & 1], buf[(i + 1) & 1], nullptr);
        if (s != GILA_OK) return s;
    }
    if (a) {
        GILA_CUDA(cudaEventRecord(b, g->stream));
        g->prof.push_back(ProfileRec{a, b, 1, prm->iters});
    }
    if (prm->iters & 1)
        GILA_CUDA(cudaMemcpyAsync(pos, tmp, pos_elem(prm->precision) * (size_t)g->n,
                                  cudaMemcpyDeviceToDevice, g->stream));
    return GILA_OK;
}

// Simple symmetric CSR from an arbitrary one: drop self-loops and repeats,
// add missing reverse entries.
void simplify_csr(int64_t n, const int64_t* row, const int32_t* col, std::vector<int64_t>& orow,
                  std::vector<int32_t>& ocol)
{
    std::vector<std::pair<int32_t, int32_t>> e;
    e.reserve((size_t)row[n] * 2);
    for (int64_t u = 0; u < n; ++u)
        for (int64_t j = row[u]; j < row[u + 1]; ++j) {
            const int32_t v = col[j];
            if (v == u || v < 0 || v >= n) continue;
            e.emplace_back((int32_t)u, v);
            e.emplace_back(v, (int32_t)u);
        }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    orow.assign((size_t)n + 1, 0);
    ocol.resize(e.size());
    for (size_t i = 0; i < e.size(); ++i) {
        orow[(size_t)e[i].first + 1]++;
        ocol[i] = e[i].second;
    }
    for (int64_t u = 0; u < n; ++u) orow[(size_t)u + 1] += orow[(size_t)u];
}

}  // namespace
gila_status graph_create_from_device(int64_t n, const int64_t* row_dev, const int32_t* col_dev,
                                     int64_t nnz, cudaStream_t st, gila_graph** out)
{
    *out = nullptr;
    gila_graph* g = new (std::nothrow) gila_graph();
    if (!g) return fail(GILA_ENOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&g->device);
    g->n = n;
    g->nnz_adj = nnz;
    g->stream = st;
    if (e == cudaSuccess) e = cudaMalloc(&g->row, sizeof(int64_t) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->row, row_dev, sizeof(int64_t) * (size_t)(n + 1),
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(g->col, col_dev, sizeof(int32_t) * (size_t)nnz,
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        gila_status s = cuda_fail(e, "graph copy");
        gila_graph_destroy(g);
        return s;
    }
    *out = g;
    return GILA_OK;
}


gila_status check_csr_bounds(int64_t n, const int64_t* row_ptr, const int32_t* col_idx)
{
    if (row_ptr[0] != 0) return fail(GILA_EINVAL, "row_ptr[0] != 0");
    for (int64_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u])
            return fail(GILA_EINVAL, "row_ptr decreases at row " + std::to_string(u));
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return fail(GILA_EINVAL, "col_idx is NULL");
    for (int64_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= n)
            return fail(GILA_EINVAL, "id " + std::to_string(col_idx[e]) + " out of range at entry " +
                                         std::to_string(e));
    return GILA_OK;
}


}  // namespace gila

using namespace gila;

extern "C" {

void gila_params_default(gila_params* p)
{
    if (!p) return;
    p->k = 2;
    p->iters = 300;
    p->d = 1.0;
    p->t0 = 0.0;
    p->schedule = GILA_COOL_LINEAR;
    p->p = 2;
    p->q = 1;
    p->precision = GILA_FP32;
}


gila_status gila_csr_validate(int64_t n, const int64_t* row_ptr, const int32_t* col_idx)
{
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(GILA_EINVAL, "n out of range");
    if (!row_ptr) return fail(GILA_EINVAL, "row_ptr is NULL");
    if (row_ptr[0] != 0) return fail(GILA_EINVAL, "row_ptr[0] != 0");
    for (int64_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u])
            return fail(GILA_EINVAL, "row_ptr decreases at row " + std::to_string(u));
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return fail(GILA_EINVAL, "col_idx is NULL");
    std::vector<int32_t> sorted(col_idx, col_idx + nnz);
    for (int64_t u = 0; u < n; ++u) {
        int32_t* b = sorted.data() + row_ptr[u];
        int32_t* e = sorted.data() + row_ptr[u + 1];
        for (int32_t* x = b; x < e; ++x) {
            if (*x < 0 || *x >= n)
                return fail(GILA_EINVAL, "id out of range in row " + std::to_string(u));
            if (*x == u) return fail(GILA_EINVAL, "self-loop at vertex " + std::to_string(u));
        }
        std::sort(b, e);
        for (int32_t* x = b; x + 1 < e; ++x)
            if (x[0] == x[1])
                return fail(GILA_EINVAL, "repeated edge " + std::to_string(u) + "-" +
                                             std::to_string(x[0]));
    }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            const int32_t v = sorted[j];
            if (!std::binary_search(sorted.data() + row_ptr[v], sorted.data() + row_ptr[v + 1],
                                    (int32_t)u))
                return fail(GILA_EINVAL, "edge " + std::to_string(u) + "-" + std::to_string(v) +
                                             " has no reverse entry");
        }
    return GILA_OK;
}

gila_status gila_graph_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                              int32_t flags, gila_graph** out)
{
    if (!out) return fail(GILA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(GILA_EINVAL, "n out of range");
    if (!row_ptr) return fail(GILA_EINVAL, "row_ptr is NULL");
    std::vector<int64_t> srow;
    std::vector<int32_t> scol;
    if (flags & GILA_GRAPH_SIMPLIFY) {
        if (row_ptr[0] != 0) return fail(GILA_EINVAL, "row_ptr[0] != 0");
        for (int64_t u = 0; u < n; ++u)
            if (row_ptr[u + 1] < row_ptr[u]) return fail(GILA_EINVAL, "row_ptr decreases");
        simplify_csr(n, row_ptr, col_idx, srow, scol);
        row_ptr = srow.data();
        col_idx = scol.data();
    } else if (flags & GILA_GRAPH_VALIDATE) {
        gila_status s = gila_csr_validate(n, row_ptr, col_idx);
        if (s != GILA_OK) return s;
    } else {
        // always: offsets and ids the kernels can index safely
        gila_status s = check_csr_bounds(n, row_ptr, col_idx);
        if (s != GILA_OK) return s;
    }
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return fail(GILA_EINVAL, "col_idx is NULL");
    gila_graph* g = new (std::nothrow) gila_graph();
    if (!g) return fail(GILA_ENOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaGetDevice");
    }
    g->n = n;
    g->nnz_adj = nnz;
    e = cudaMalloc(&g->row, sizeof(int64_t) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->row, row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpy(g->col, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gila_status s = cuda_fail(e, "graph upload");
        gila_graph_destroy(g);
        return s;
    }
    *out = g;
    return GILA_OK;
}


gila_status gila_graph_set_wait_test(gila_graph* g, int32_t on)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    g->wait_test = on ? 1 : 0;
    return GILA_OK;
}

gila_status gila_graph_set_repulsion_weights(gila_graph* g, const double* weight_host)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    gila_status s = use_device(g);
    if (s != GILA_OK) return s;
    if (weight_host)
        for (int64_t i = 0; i < g->n; ++i)
            if (!(weight_host[i] >= 0.0) || !std::isfinite(weight_host[i]))
                return fail(GILA_EINVAL, "repulsion weights must be finite and >= 0");
    return set_repulsion_weights(g, weight_host, false);
}

void gila_graph_destroy(gila_graph* g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    for (auto& r : g->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    free_khop(g);
    free_layout(g);
    cudaFree(g->row);
    cudaFree(g->col);
    delete g;
}

gila_status gila_graph_set_stream(gila_graph* g, void* cuda_stream)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    g->stream = (cudaStream_t)cuda_stream;
    return GILA_OK;
}

gila_status gila_graph_tune(gila_graph* g, const gila_tuning* t)
{
    if (!g || !t) return fail(GILA_EINVAL, "graph or tuning is NULL");
    if (t->tiled < -1 || t->tiled > 1) return fail(GILA_EINVAL, "tiled must be -1, 0 or 1");
    if (t->tile_vertices < 0 || t->min_segment < 0 || t->small_max < 0 || t->warp_max < 0 ||
        t->block_max < 0 || t->chunk < 0 || t->ctas_per_sm < 0)
        return fail(GILA_EINVAL, "tuning values must be >= 0");
    if (t->bank_spread < -1 || t->bank_spread > 1)
        return fail(GILA_EINVAL, "bank_spread must be -1, 0 or 1");
    if (t->step_schedule < -1 || t->step_schedule > 1)
        return fail(GILA_EINVAL, "step_schedule must be -1, 0 or 1");
    BinConfig c;  // defaults
    if (t->small_max) c.small_max = t->small_max;
    if (t->warp_max) c.warp_max = t->warp_max;
    if (t->block_max) c.block_max = t->block_max;
    if (t->chunk) c.chunk = t->chunk;
    if (!(c.small_max <= c.warp_max && c.warp_max <= c.block_max))
        return fail(GILA_EINVAL, "row-class bounds must satisfy small_max <= warp_max <= block_max");
    BinConfig& old = g->bins.cfg;
    if (old.small_max != c.small_max || old.warp_max != c.warp_max ||
        old.block_max != c.block_max || old.chunk != c.chunk) {
        old = c;
        g->k_built = 0;  // classes are assigned at build time
    }
    g->tune = *t;
    invalidate_tile_plans(g);
    return GILA_OK;
}

gila_status gila_graph_get_tuning(const gila_graph* g, gila_tuning* out)
{
    if (!g || !out) return fail(GILA_EINVAL, "graph or out is NULL");
    *out = g->tune;
    out->min_segment = g->tune.min_segment;
    out->ctas_per_sm = g->tune.ctas_per_sm > 0
                           ? g->tune.ctas_per_sm
                           : (int32_t)default_ctas_per_sm(g->nnz_khop, g->tplan[0].window);
    out->bank_spread = g->tune.bank_spread >= 0 ? 1 : -1;
    out->step_schedule = g->tune.step_schedule >= 0 ? 1 : -1;
    out->small_max = g->bins.cfg.small_max;
    out->warp_max = g->bins.cfg.warp_max;
    out->block_max = g->bins.cfg.block_max;
    out->chunk = g->bins.cfg.chunk;
    return GILA_OK;
}

gila_status gila_graph_info(const gila_graph* g, int64_t* n, int64_t* nnz_adj, int32_t* k_built,
                            int64_t* nnz_khop)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (nnz_adj) *nnz_adj = g->nnz_adj;
    if (k_built) *k_built = g->k_built;
    if (nnz_khop) *nnz_khop = g->k_built ? g->nnz_khop : 0;
    return GILA_OK;
}

gila_status gila_build_khop(gila_graph* g, int32_t k, int64_t* nnz_out)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    if (k < 1 || k > 64) return fail(GILA_EINVAL, "k must be in [1, 64]");
    gila_status s = use_device(g);
    if (s != GILA_OK) return s;
    s = ensure_khop(g, k);
    if (s != GILA_OK) return s;
    if (nnz_out) *nnz_out = g->nnz_khop;
    return GILA_OK;
}

gila_status gila_khop_reset(gila_graph* g)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    g->k_built = 0;
    return GILA_OK;
}

gila_status gila_khop_export(const gila_graph* g, int64_t* krow_host, int32_t* kcol_host)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    if (!g->k_built) return fail(GILA_ESTATE, "no k-hop lists built");
    if (!krow_host || (g->nnz_khop > 0 && !kcol_host))
        return fail(GILA_EINVAL, "output array is NULL");
    gila_status s = use_device(g);
    if (s != GILA_OK) return s;
    GILA_CUDA(cudaMemcpyAsync(krow_host, g->krow, sizeof(int64_t) * (size_t)(g->n + 1),
                              cudaMemcpyDeviceToHost, g->stream));
    if (g->nnz_khop > 0)
        GILA_CUDA(cudaMemcpyAsync(kcol_host, g->kcol, sizeof(int32_t) * (size_t)g->nnz_khop,
                                  cudaMemcpyDeviceToHost, g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    return GILA_OK;
}

gila_status gila_khop_export_rows(const gila_graph* g, int64_t nsel, const int64_t* sel_host,
                                  int64_t* counts_host, int32_t* cols_host, int64_t cols_cap)
{
    if (!g || nsel < 0 || (nsel > 0 && (!sel_host || !counts_host)))
        return fail(GILA_EINVAL, "graph, selection or counts is NULL");
    if (!g->krow || g->k_built == 0) return fail(GILA_ESTATE, "no k-hop lists are built");
    GILA_CUDA(cudaSetDevice(g->device));
    std::vector<int64_t> b((size_t)nsel), e((size_t)nsel);
    for (int64_t i = 0; i < nsel; ++i) {
        if (sel_host[i] < 0 || sel_host[i] >= g->n) return fail(GILA_EINVAL, "vertex out of range");
        GILA_CUDA(cudaMemcpy(&b[(size_t)i], g->krow + sel_host[i], sizeof(int64_t),
                             cudaMemcpyDeviceToHost));
        GILA_CUDA(cudaMemcpy(&e[(size_t)i], g->krow + sel_host[i] + 1, sizeof(int64_t),
                             cudaMemcpyDeviceToHost));
    }
    int64_t total = 0;
    for (int64_t i = 0; i < nsel; ++i) {
        counts_host[i] = e[(size_t)i] - b[(size_t)i];
        total += counts_host[i];
    }
    if (!cols_host) return GILA_OK;
    if (total > cols_cap) return fail(GILA_EINVAL, "cols_cap is smaller than the rows' total");
    int64_t o = 0;
    for (int64_t i = 0; i < nsel; ++i) {
        if (counts_host[i] > 0)
            GILA_CUDA(cudaMemcpy(cols_host + o, g->kcol + b[(size_t)i],
                                 sizeof(int32_t) * (size_t)counts_host[i], cudaMemcpyDeviceToHost));
        o += counts_host[i];
    }
    return GILA_OK;
}

gila_status gila_layout_step(gila_graph* g, const gila_params* prm, double t,
                             const void* pos_in_dev, void* pos_out_dev, void* disp_out_dev)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    gila_status s = check_params(prm);
    if (s != GILA_OK) return s;
    if (!(t >= 0.0) || !std::isfinite(t)) return fail(GILA_EINVAL, "t must be finite and >= 0");
    if (g->n > 0 && (!pos_in_dev || !pos_out_dev)) return fail(GILA_EINVAL, "placement is NULL");
    if (pos_in_dev == pos_out_dev && g->n > 0)
        return fail(GILA_EINVAL, "pos_in_dev and pos_out_dev must not overlap");
    if ((s = use_device(g)) != GILA_OK) return s;
    if ((s = ensure_khop(g, prm->k)) != GILA_OK) return s;
    if ((s = timed_prepare(g, prm)) != GILA_OK) return s;
    cudaEvent_t a = nullptr, b = nullptr;
    if (g->prof_on) {
        GILA_CUDA(cudaEventCreate(&a));
        GILA_CUDA(cudaEventCreate(&b));
        GILA_CUDA(cudaEventRecord(a, g->stream));
    }
    s = launch_iteration(g, prm, t, pos_in_dev, pos_out_dev, disp_out_dev);
    if (a) {
        cudaEventRecord(b, g->stream);
        g->prof.push_back(ProfileRec{a, b, 1, 1});
    }
    return s;
}

gila_status gila_layout_run_device(gila_graph* g, const gila_params* prm, void* pos_dev_inout)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    gila_status s = check_params(prm);
    if (s != GILA_OK) return s;
    if (g->n > 0 && !pos_dev_inout) return fail(GILA_EINVAL, "placement is NULL");
    if ((s = use_device(g)) != GILA_OK) return s;
    if ((s = ensure_khop(g, prm->k)) != GILA_OK) return s;
    if (g->n == 0 || prm->iters == 0) return GILA_OK;
    const size_t bytes = pos_elem(prm->precision) * (size_t)g->n;
    if ((s = ensure(&g->pos[1], &g->pos_cap[1], bytes)) != GILA_OK) return s;
    return run_loop(g, prm, pos_dev_inout, g->pos[1]);
}

gila_status gila_layout_run(gila_graph* g, const gila_params* prm, const double* pos_in_host,
                            double* pos_out_host, gila_metrics* metrics_out)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    gila_status s = check_params(prm);
    if (s != GILA_OK) return s;
    if (g->n > 0 && (!pos_in_host || !pos_out_host)) return fail(GILA_EINVAL, "placement is NULL");
    if ((s = use_device(g)) != GILA_OK) return s;
    if ((s = ensure_khop(g, prm->k)) != GILA_OK) return s;
    if (g->n == 0) {
        if (metrics_out) *metrics_out = gila_metrics{};
        return GILA_OK;
    }
    const size_t n = (size_t)g->n;
    const size_t bytes = pos_elem(prm->precision) * n;
    if ((s = ensure(&g->pos[0], &g->pos_cap[0], bytes)) != GILA_OK) return s;
    if ((s = ensure(&g->pos[1], &g->pos_cap[1], bytes)) != GILA_OK) return s;
    const bool f64 = is_f64(prm->precision);
    if (!f64 && (s = ensure((void**)&g->stage, &g->stage_cap, 16 * n)) != GILA_OK) return s;
    if (f64) {
        GILA_CUDA(cudaMemcpyAsync(g->pos[0], pos_in_host, 16 * n, cudaMemcpyHostToDevice, g->stream));
    } else {
        GILA_CUDA(cudaMemcpyAsync(g->stage, pos_in_host, 16 * n, cudaMemcpyHostToDevice, g->stream));
        if ((s = convert_positions(g, prm->precision, g->stage, g->pos[0], true)) != GILA_OK)
            return s;
    }
    if ((s = run_loop(g, prm, g->pos[0], g->pos[1])) != GILA_OK) return s;
    if (metrics_out && (s = compute_metrics(g, prm, g->pos[0], metrics_out)) != GILA_OK) return s;
    if (f64) {
        GILA_CUDA(cudaMemcpyAsync(pos_out_host, g->pos[0], 16 * n, cudaMemcpyDeviceToHost,
                                  g->stream));
    } else {
        if ((s = convert_positions(g, prm->precision, g->stage, g->pos[0], false)) != GILA_OK)
            return s;
        GILA_CUDA(cudaMemcpyAsync(pos_out_host, g->stage, 16 * n, cudaMemcpyDeviceToHost,
                                  g->stream));
    }
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    return blocked_tile_wait_failed(g->stream);
}

gila_status gila_layout_metrics(gila_graph* g, const gila_params* prm, const void* pos_dev,
                                gila_metrics* out)
{
    if (!g || !out) return fail(GILA_EINVAL, "graph or out is NULL");
    gila_status s = check_params(prm);
    if (s != GILA_OK) return s;
    if (g->n > 0 && !pos_dev) return fail(GILA_EINVAL, "placement is NULL");
    if ((s = use_device(g)) != GILA_OK) return s;
    if ((s = ensure_khop(g, prm->k)) != GILA_OK) return s;
    if ((s = compute_metrics(g, prm, pos_dev, out)) != GILA_OK) return s;
    return blocked_tile_wait_failed(g->stream);
}

double gila_temperature(const gila_params* prm, double t0, int32_t i)
{
    if (!prm || prm->iters <= 0) return 0.0;
    return temperature(prm, t0, i);
}

gila_status gila_profile_enable(gila_graph* g, int32_t on)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    if (on < 0 || on > 2) return fail(GILA_EINVAL, "on must be 0, 1 or 2");
    g->prof_on = on;
    return GILA_OK;
}

gila_status gila_profile_read(gila_graph* g, int64_t* builds, double* build_ms,
                              int64_t* iter_launches, double* iter_ms)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    gila_status s = use_device(g);
    if (s != GILA_OK) return s;
    for (auto& r : g->prof) {
        float ms = 0.0f;
        GILA_CUDA(cudaEventSynchronize(r.b));
        GILA_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.kind == 0) {
            g->prof_builds += r.launches;
            g->prof_build_ms += ms;
        } else if (r.kind == 2) {
            g->prof_kernel_launches += r.launches;
            g->prof_kernel_ms += ms;
        } else {
            g->prof_launches += r.launches;
            g->prof_iter_ms += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g->prof.clear();
    if (builds) *builds = g->prof_builds;
    if (build_ms) *build_ms = g->prof_build_ms;
    if (iter_launches) *iter_launches = g->prof_launches;
    if (iter_ms) *iter_ms = g->prof_iter_ms;
    g->prof_builds = 0;
    g->prof_launches = 0;
    g->prof_build_ms = 0.0;
    g->prof_iter_ms = 0.0;
    return GILA_OK;
}

gila_status gila_profile_read_kernel(gila_graph* g, int64_t* launches, double* ms, char* name,
                                     int32_t name_cap)
{
    if (!g) return fail(GILA_EINVAL, "graph is NULL");
    // folds the pending repulsion-kernel records into the totals; records of
    // the other kinds stay for gila_profile_read
    int64_t kl = 0;
    double kms = 0.0;
    {
        gila_status s = use_device(g);
        if (s != GILA_OK) return s;
        for (auto& r : g->prof) {
            if (r.kind != 2) continue;
            float m = 0.0f;
            GILA_CUDA(cudaEventSynchronize(r.b));
            GILA_CUDA(cudaEventElapsedTime(&m, r.a, r.b));
            kl += r.launches;
            kms += m;
        }
        std::vector<ProfileRec> rest;
        for (auto& r : g->prof) {
            if (r.kind == 2) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            } else {
                rest.push_back(r);
            }
        }
        g->prof.swap(rest);
    }
    kl += g->prof_kernel_launches;
    kms += g->prof_kernel_ms;
    g->prof_kernel_launches = 0;
    g->prof_kernel_ms = 0.0;
    if (launches) *launches = kl;
    if (ms) *ms = kms;
    if (name && name_cap > 0) {
        std::strncpy(name, g->prof_kernel_name, (size_t)name_cap - 1);
        name[name_cap - 1] = '\0';
    }
    return GILA_OK;
}

const char* gila_last_error(void) { return t_err.c_str(); }

int64_t gila_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
