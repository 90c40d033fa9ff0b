// Internal declarations shared by the translation units of libgila.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gila.h"

namespace gila {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);
gila_status fail(gila_status s, const std::string& msg);
gila_status cuda_fail(cudaError_t e, const char* what);

#define GILA_CUDA(call)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::gila::cuda_fail(e_, #call); \
    } while (0)

inline bool is_f64(int precision)
{
    return precision == GILA_FP64 || precision == GILA_FP64_ORDERED;
}

// ---------------------------------------------------------------- binning

// Row-length classes of the iteration kernel.
//   class 0: len <= kSmallMax, kGroupSmall lanes per vertex
//   class 1: len <= kWarpMax, one warp per vertex
//   class 2: len <= kBlockMax, one block per vertex
//   class 3: longer, split into chunks of kChunk entries, one block each,
//            summed in chunk order by the last block to finish
struct BinConfig {
    int small_max = 64;  // rows of 33..64 entries on a whole warp left most lanes idle (mesh: 4x)
    int group_small = 8;
    int warp_max = 8192;
    int block_max = 65536;
    int chunk = 32768;
};

struct Chunk {
    int64_t begin;   // first entry (absolute index into kcol)
    int64_t end;     // one past the last entry
    int32_t vertex;  // owner
    int32_t giant;   // index of the owner in the giant list
    int32_t first;   // index of the owner's first chunk
    int32_t count;   // number of chunks of the owner
};

// Scratch that a single k-hop build needs (reused across builds).
struct KhopScratch {
    int64_t* counts = nullptr;  // n
    int32_t* queue = nullptr;   // n: sources whose ball overflowed tier 1
    int* qn = nullptr;          // 1
    uint32_t* bitmaps = nullptr;
    int32_t* lists = nullptr;
    uint32_t* store = nullptr;  // tier-2 balls kept from count to fill (capacity kept
    size_t store_cap = 0;       // across builds)
    bool stored = false;        // the last count pass stored its balls
    uint32_t* b2 = nullptr;     // radius-2 bitmaps of the k = 3 count (capacity kept)
    size_t b2_cap = 0;
    bool keep_balls = true;     // allow the store (the server turns it off: it may wait
                                // between count and fill, outside its memory accounting)
    int64_t bitmap_words = 0;   // per block
    int t2_blocks = 0;
    size_t cap_n = 0;
    size_t scratch_cap = 0;     // tier-2 scratch limit in bytes (0 = 2 GiB)
    // state between the count and the fill phase
    int counted_k = 0;
    int64_t nnz = 0;
    int nq = 0, t2_used = 0;
    int64_t t1_blocks = 0, nwords = 0;
};

struct Bins {
    int32_t* lists = nullptr;   // all classes back to back: class 0, 1, 2
    int32_t n0 = 0, n1 = 0, n2 = 0;
    Chunk* chunks = nullptr;
    int32_t nchunks = 0;
    int32_t ngiant = 0;
    int32_t* giant_counter = nullptr;  // ngiant, zero between launches
    void* partials = nullptr;          // nchunks x 4 doubles
    size_t cap_lists = 0, cap_chunks = 0, cap_giant = 0;
    BinConfig cfg;
};

// Blocked-path plan of the iteration for one position width (index 0:
// float2, 1: double2): tiles of positions, row ranges and the k-hop ids
// rearranged block by block. Rebuilt after every k-hop build.
struct TilePlan {
    bool ready = false;  // decided for the current k-hop lists
    bool use = false;    // the blocked path serves this graph
    int32_t nt = 0, tv = 0, nb = 0;  // tiles, tile (or largest window) size, blocks (CTAs)
    int32_t rmax = 0;                // most rows of a range (window mode: cells per CTA)
    int32_t* bdesc = nullptr;        // 4 nb: first row, end row and tile of block b, 0
    size_t bdesc_cap = 0;
    int32_t* rdir = nullptr;         // per tile its row ranges and their blocks (layout scratch)
    size_t rdir_cap = 0;
    int64_t* blk = nullptr;          // 2 nb: start in tk and entry count of block b
    size_t blk_cap = 0;
    int64_t* toff = nullptr;         // nt n: start of (tile j, row u) in tk
    size_t toff_cap = 0;
    uint16_t* tk = nullptr;          // tile-relative 16-bit ids in block order
    size_t tk_cap = 0;
    void* part = nullptr;            // nt n x 4 T partial forces
    size_t part_cap = 0;
    int32_t* hubs = nullptr;         // vertices of adjacency degree > 64 (combine kernel)
    size_t hubs_cap = 0;
    int32_t nhub = 0;
    int64_t* len = nullptr;          // nt n segment lengths (plan scratch)
    size_t len_cap = 0;
    // window mode: one window of positions per row range, covering every id
    // its rows touch; rows are finished by their range's CTA
    bool window = false;
    int64_t* wtile = nullptr;        // 2 nb: first id and length of block b's window
    size_t wtile_cap = 0;
    int32_t* rowspan = nullptr;      // 2 n: first and last id of each row (plan scratch)
    size_t rowspan_cap = 0;
};

struct ProfileRec {
    cudaEvent_t a, b;
    int kind;  // 0 build (or blocked plan), 1 iterations, 2 one repulsion kernel
    int64_t launches;
};

}  // namespace gila

struct gila_graph {
    int64_t n = 0;
    int64_t nnz_adj = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t* row = nullptr;
    int32_t* col = nullptr;
    // k-hop lists
    int32_t k_built = 0;
    int64_t nnz_khop = 0;
    int64_t* krow = nullptr;
    uint32_t* kcol = nullptr;
    size_t cap_kcol = 0;
    gila::KhopScratch ks;
    gila::Bins bins;
    gila::TilePlan tplan[2];
    gila_tuning tune = {-1, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // placement buffers for the run calls
    void* pos[2] = {nullptr, nullptr};
    size_t pos_cap[2] = {0, 0};
    double* stage = nullptr;  // double[2n] upload/download staging
    size_t stage_cap = 0;
    // FP64 reduction scratch
    double* red = nullptr;
    size_t red_cap = 0;
    // repulsion weights (Section 4.6), both widths; null when unset
    double* wt64 = nullptr;
    float* wt32 = nullptr;
    // test hook: blocked-path tiles are announced but not copied, so their
    // bounded waits run out (failure-detection test)
    int wait_test = 0;
    // profiling: 0 off, 1 builds and iteration sequences, 2 also the
    // repulsion kernel of every iteration on its own
    int prof_on = 0;
    std::vector<gila::ProfileRec> prof;
    int64_t prof_builds = 0, prof_launches = 0, prof_kernel_launches = 0;
    double prof_build_ms = 0.0, prof_iter_ms = 0.0, prof_kernel_ms = 0.0;
    const char* prof_kernel_name = "";
};

namespace gila {

// k-hop build (khop.cu): count (sizes, offsets, total) then fill (ids,
// row classes); build_khop does both.
gila_status build_khop(gila_graph* g, int k);
gila_status build_khop_count(gila_graph* g, int k, int64_t* nnz_out);
gila_status build_khop_count_impl(gila_graph* g, int k);
gila_status build_khop_fill(gila_graph* g, int k);
void release_khop_scratch(gila_graph* g);  // frees the build-only buffers
void free_khop(gila_graph* g);

// iteration + metrics (layout.cu)
gila_status launch_iteration(gila_graph* g, const gila_params* prm, double t,
                             const void* pos_in, void* pos_out, void* disp_out);
gila_status compute_metrics(gila_graph* g, const gila_params* prm, const void* pos,
                            gila_metrics* out);
gila_status bbox_aspect(gila_graph* g, int precision, const void* pos, double* aspect);
void invalidate_tile_plans(gila_graph* g);
void free_tile_plans(gila_graph* g);
// blocked path (blocked.cu): *handled = false when the plain kernel must run
gila_status launch_blocked(gila_graph* g, const gila_params* prm, double t, const void* pos_in,
                           void* pos_out, void* disp_out, bool* handled);
// Whether automatic mode (or the tuning) puts a graph of these sizes on the
// blocked path; and building its plan ahead of the first iteration.
bool blocked_auto_applies(int64_t n, int64_t nnz_khop, size_t esz, const gila_tuning& tune);
// CTAs per SM the blocked grid aims at unless the tuning sets it.
int64_t default_ctas_per_sm(int64_t nnz_khop, bool window);
gila_status prepare_iteration(gila_graph* g, const gila_params* prm);
// The repulsive total of the quality reductions over the blocked plan's
// position tiles (FP32 placements with a plan only; *done = false otherwise).
gila_status blocked_khop_metric(gila_graph* g, const gila_params* prm, const void* pos,
                                bool* done, double* rep_total);
// GILA_ECUDA (and clears the flag) when a blocked-path CTA gave up waiting
// for its tile copy since the last call; synchronises st.
gila_status blocked_tile_wait_failed(cudaStream_t st);
gila_status convert_positions(gila_graph* g, int precision, const double* src, void* dst,
                              bool to_device_type);
// Offsets non-decreasing from 0 and every id in [0, n): what the kernels need
// to index safely (GILA_EINVAL otherwise). Host arrays.
gila_status check_csr_bounds(int64_t n, const int64_t* row_ptr, const int32_t* col_idx);
// Repulsion weights from host or device doubles (null clears); synchronises.
gila_status set_repulsion_weights(gila_graph* g, const double* w, bool w_on_device);
// Upload a graph from device CSR arrays (copied; ids trusted).
gila_status graph_create_from_device(int64_t n, const int64_t* row_dev, const int32_t* col_dev,
                                     int64_t nnz, cudaStream_t st, gila_graph** out);
void free_layout(gila_graph* g);

// memory helper: grow a device buffer to at least `bytes`
gila_status ensure(void** p, size_t* cap, size_t bytes);

int sm_count(int device);

// out[0] = 0, out[i + 1] = in[0] + ... + in[i]; synchronises st.
gila_status scan_exclusive_i64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st);

// Count one kernel launch issued by the library (all launch sites call it).
void count_launch();

// Profiling mode 2: an event recorded on g's stream before the repulsion
// kernel of an iteration (null when the mode is off), and the matching end
// record after it, kept with the kernel's name.
cudaEvent_t prof_kernel_begin(gila_graph* g);
void prof_kernel_end(gila_graph* g, cudaEvent_t a, const char* name);

}  // namespace gila
