// Blocked iteration path: positions staged in shared memory by tiles, the
// k-hop ids rearranged once so that every CTA streams one contiguous block.
//
// Tiles: tile j holds the positions of ids [j tv, (j+1) tv). Ranges: each
// tile's rows are cut into contiguous ranges on their own, so that the
// blocks (j, r) cost about the same whichever tile holds the most entries
// (on a power-law graph the hubs' tile holds twice the mean). Block (j, r)
// holds, for every row u of range r in order, the entries of u's k-hop row
// that fall in tile j, in an order chosen so that the lanes of one gather
// read distinct shared-memory banks; block starts are 16-byte aligned. An
// entry is stored as a 16-bit id relative to the tile's first id (a tile
// holds at most 65,534 positions), so the id stream, the only compulsory
// DRAM traffic of an iteration, is 2 bytes per entry instead of 4. One
// CTA per block loads tile j and the block's row directory into shared
// memory; each thread takes an equal, 8-aligned share of the block's
// entries (stored so that a warp's 16-byte id loads of one step, eight ids
// per lane, are contiguous), gathers positions from the tile and sums them
// row by row on its own. A row wholly inside a share is stored by its
// thread; the parts of rows cut by share bounds are added by a segmented
// scan across the warp, and rows cut by warp bounds by a second segmented
// scan in warp order, then stored as the row's partial for tile j. A
// second kernel adds each row's tile partials in tile order, adds its
// attraction terms and applies the capped move. (Window mode, for banded
// graphs: one window of positions per range instead of tiles, and the CTA
// finishes its rows itself.) Every partial has a fixed place and a fixed
// order of additions, so results do not depend on scheduling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "ff.cuh"
#include "force.cuh"
#include "gila_impl.h"

namespace gila {

namespace {

constexpr int kBThreads = 1024;
constexpr int kBWarps = kBThreads / 32;
static_assert(kBWarps == 32, "the slot flush gives lane w of warp 0 the slots of warp w");
constexpr int kSmemCap = 227 * 1024;
constexpr int kMaxRows = 4096;  // rows per range (directory in shared memory)
constexpr int kMaxRowsTiles = 8192;  // tile mode: the directory may grow to this where the
                                     // 4096-row limit alone would exceed the CTA target
constexpr int kTileBudget = kSmemCap - (kMaxRows + 1) * 4 - 4096;
constexpr int64_t kMaxTile = 65534;  // tile-relative ids and the far slot's id fit 16 bits
constexpr uint32_t kBulkChunk = 32768;      // bytes per bulk copy instruction
constexpr int64_t kBlockedMinNnz = 4000000;  // automatic mode: k-hop entries needed (tiles)
constexpr uint64_t kWaitNs = 1000000000ull;  // bound on a tile wait (1 s, far above any copy)
constexpr uint64_t kTestWaitNs = 1000000ull;   // the bound while the wait test hook is on
// Every (tile j, row) segment is padded to a multiple of 8 entries with the
// relative id tv, whose tile slot (one past the tile) holds a position so far
// away that its term is exactly zero: in FP32 the factor rcp(r^2 + 2^-100)
// of r^2 = 2e38 is below the smallest normal and flushes to 0; in FP64 r^2
// = 1.48e308 flushes rcp to 0 the same way; the generic model cuts terms
// beyond r^2 = 1e38 (FP32) or 1e300 (FP64). 0 * Delta then adds nothing.
template <class T> struct FarSlot;
template <> struct FarSlot<float> { static constexpr float v = 1.0e19f; };
template <> struct FarSlot<double> { static constexpr double v = 8.6e153; };

constexpr int kPrefetch = 4;  // steps between an L2 prefetch of ids and their ring load (4, 12, 24
                               // measured: 4 best; longer distances crowd L2)

// Set when a CTA gave up waiting for its tile copy (the launch's partials
// are then incomplete); read and cleared by blocked_tile_wait_failed().
__device__ int g_tile_wait_failed = 0;

struct BlockedArgs {
    const uint16_t* tk;        // tile-relative ids, block by block, in share storage order
    const int64_t* toff;       // nt n: start of segment (tile j, row u) within its block
    const int64_t* blk;        // 2 nb: first slot in tk and entry count of block b
    const int4* bdesc;         // nb: first row, end row and tile of block b
    int64_t n;
    int32_t nt, tv;
    int q;
    const void* pos;
    void* part;                // nt n cells of 4 T: (sx, sy, cx, cy) without the factor d^2
    uint64_t wait_ns;          // bound on the tile wait
    int skip_copy;             // test hook: announce the tile but copy nothing
    // window mode (one window of positions per row range, rows finished in
    // the CTA): first id and length of block b's window, the largest window
    // and range, and what the finish needs
    const int64_t* wbase;      // 2 nb
    int32_t wmax, rmax;
    const int64_t* row;
    const int32_t* col;
    double d, t;
    int p;
    void* pos_out;
    void* disp_out;
    int uniform;               // FP32 steps taken warp-uniformly (tuning step_schedule >= 0)
};

template <class T, bool COMP>
struct Slot {
    int32_t row;
    T v[4];
};

// Cell (tile j, row u) of the partials: the sum as one position-type pair,
// followed by its compensation pair in the compensated mode (8 bytes a cell
// for plain FP32, so that the partials of short-row graphs with many tiles
// do not outweigh their id stream).
template <class T, bool COMP>
__device__ __forceinline__ typename V2<T>::type* cell_ptr(void* part, int64_t n, int j, int64_t u)
{
    using P2 = typename V2<T>::type;
    return reinterpret_cast<P2*>(part) + ((int64_t)j * n + u) * (COMP ? 2 : 1);
}

template <class T, bool COMP>
__device__ __forceinline__ void store_cell(typename V2<T>::type* c, const Acc<T, COMP>& a)
{
    using P2 = typename V2<T>::type;
    P2 s;
    s.x = a.sx;
    s.y = a.sy;
    c[0] = s;
    if (COMP) {
        P2 k;
        k.x = a.cx;
        k.y = a.cy;
        c[1] = k;
    }
}

// Entries per step: one 16-byte load of eight 16-bit ids.
constexpr int kStep = 8;

// Entries of block (j, r) per thread: thread t takes [lane_start(L, t),
// lane_start(L, t + 1)), 8-aligned; in storage every thread has lane_len(L)
// slots (a multiple of 8, at least its share), laid out per warp step-major:
// the k-th group of eight slots of lane l of warp w is at
// (w 32 lane_len + 256 k + 8 l) from the block's start, so that a warp's
// 16-byte loads of one step are one contiguous 512-byte run.
__host__ __device__ __forceinline__ int32_t lane_start(int32_t L, int t)
{
    return (t >= kBThreads) ? L : (int32_t)(((int64_t)L * t / kBThreads) & ~int64_t(kStep - 1));
}
__host__ __device__ __forceinline__ int32_t lane_len(int32_t L)
{
    // a share is at most L / kBThreads + 8 entries (8-aligned cuts)
    return (L == 0) ? 0 : ((L / kBThreads + 2 * kStep - 1) & ~(kStep - 1));
}

// acc += (x, y) with a two-sum error term per component; in FP32 both
// components go through packed two-lane operations (six instead of twelve).
template <class T, bool COMP>
__device__ __forceinline__ void add_compensated(Acc<T, COMP>& acc, T x, T y)
{
    if constexpr (sizeof(T) == 4 && COMP) {
        uint64_t s, c, v, t, bp, e1, e2;
        asm("mov.b64 %0, {%1, %2};" : "=l"(s) : "f"(acc.sx), "f"(acc.sy));
        asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(acc.cx), "f"(acc.cy));
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x), "f"(y));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(s), "l"(v));    // t = s + v
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bp) : "l"(t), "l"(s));   // bp = t - s
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(e1) : "l"(t), "l"(bp));  // t - bp
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(e1) : "l"(s), "l"(e1));  // s - (t - bp)
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(e2) : "l"(v), "l"(bp));  // v - bp
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e1) : "l"(e1), "l"(e2));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(c) : "l"(c), "l"(e1));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc.sx), "=f"(acc.sy) : "l"(t));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc.cx), "=f"(acc.cy) : "l"(c));
    } else {
        acc.merge(x, y, T(0), T(0));
    }
}

// Window mode's finish of the rows [u0, u0 + nrows) of a range, after their
// cells (sum of the unscaled repulsion terms, with compensation) are
// complete in shared memory: F = d^2 cell + attraction, then the capped move.
// Rows with at most kFinishDeg neighbours take one thread each; longer ones
// are taken by the whole warp their row falls to, lanes striding the
// adjacency row. Every row's order of additions is fixed.
template <class T, int MODEL, bool COMP>
__device__ __forceinline__ void window_finish(const struct BlockedArgs& A,
                                              const typename V2<T>::type* tile, int64_t tb,
                                              const typename V2<T>::type* cells, int64_t u0,
                                              int nrows);

// Window mode's finish: rows whose adjacency row is longer than this are
// finished by a whole warp (a few per range), the others by one thread.
constexpr int kFinishDeg = 32;

template <class T, int MODEL, bool COMP, bool WIN>
__global__ void __launch_bounds__(kBThreads, 1) blocked_kernel(const BlockedArgs A)
{
    using P2 = typename V2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // shared memory: the tile (or the range's window) with one more slot for
    // the padding's far position, the row directory, and in window mode the
    // rows' force cells
    const int tcap = WIN ? A.wmax : A.tv;
    P2* tile = reinterpret_cast<P2*>(smem_raw);
    int32_t* D = reinterpret_cast<int32_t*>(smem_raw + (size_t)(tcap + 1) * sizeof(P2));
    P2* cells = reinterpret_cast<P2*>(
        smem_raw + (((size_t)(tcap + 1) * sizeof(P2) + (size_t)(A.rmax + 1) * 4 + 15) & ~size_t(15)));
    __shared__ Slot<T, COMP> head[kBWarps], tail[kBWarps];
    __shared__ __align__(8) uint64_t tile_bar;
    __shared__ int tile_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 bd = A.bdesc[blockIdx.x];  // rows [bd.x, bd.y) of tile bd.z (0 in window mode)
    const int j = WIN ? 0 : bd.z;
    const int64_t u0 = bd.x, u1 = bd.y;
    const int nrows = (int)(u1 - u0);
    const int64_t bsp = A.blk[2 * (int64_t)blockIdx.x];  // the block's first slot in tk
    // a block holds at most kMaxRows segments of at most tv entries: < 2^31
    const int32_t L = (int32_t)A.blk[2 * (int64_t)blockIdx.x + 1];
    const P2* __restrict__ pos = reinterpret_cast<const P2*>(A.pos);
    const int64_t tb = WIN ? A.wbase[2 * blockIdx.x] : (int64_t)j * A.tv;
    const int64_t tn = WIN ? A.wbase[2 * blockIdx.x + 1]
                           : ((A.n - tb < A.tv) ? A.n - tb : (int64_t)A.tv);
    // the cell of row i of the range: in shared memory (window mode) or the
    // global partial of (tile j, row u0 + i)
    auto cellp = [&](int64_t i) -> P2* {
        return WIN ? cells + 2 * i : cell_ptr<T, COMP>(A.part, A.n, j, u0 + i);
    };
    if (threadIdx.x == 0) {
        // tile j by the bulk-copy engine (tv is even and the placement is
        // 16-byte aligned, so the source is too); an odd float2 tail by hand
        const uint32_t bytes = (uint32_t)(((size_t)tn * sizeof(P2)) & ~size_t(15));
        mbar_init(&tile_bar, 1);
        mbar_arrive_expect_tx(&tile_bar, bytes);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(pos + tb);
        for (uint32_t o = 0; o < bytes && !A.skip_copy; o += kBulkChunk)
            bulk_g2s(smem_raw + o, src + o, (bytes - o < kBulkChunk) ? bytes - o : kBulkChunk,
                     &tile_bar);
        if ((size_t)tn * sizeof(P2) != bytes) tile[tn - 1] = pos[tb + tn - 1];
        P2 far;  // the padding's slot, outside the copied range
        far.x = FarSlot<T>::v;
        far.y = FarSlot<T>::v;
        tile[WIN ? tn : (int64_t)A.tv] = far;
    }
    if (WIN && threadIdx.x == 32) {
        // the finish's adjacency (row offsets, neighbour ids) and the rows'
        // own positions, pulled into L2 while the window loads and the
        // entries stream
        const int64_t ab = A.row[u0], ae = A.row[u1];
        prefetch_l2_range(A.row + u0, sizeof(int64_t) * (size_t)(u1 - u0 + 1));
        prefetch_l2_range(A.col + ab, sizeof(int32_t) * (size_t)(ae - ab));
        prefetch_l2_range(pos + u0, sizeof(P2) * (size_t)(u1 - u0));
    }
    // meanwhile: the row directory (segment starts within the block) and
    // zero partials for rows with no entries in this tile
    for (int i = threadIdx.x; i < nrows; i += kBThreads) {
        D[i] = (int32_t)A.toff[(int64_t)j * A.n + u0 + i];
        P2* c = cellp(i);
        P2 z;
        z.x = T(0);
        z.y = T(0);
        c[0] = z;
        if (COMP) c[1] = z;
    }
    if (threadIdx.x == 0) D[nrows] = L;
    if (threadIdx.x < kBWarps) {
        head[threadIdx.x].row = -1;
        tail[threadIdx.x].row = -1;
    }
    if (threadIdx.x == 0) {
        bool ok = mbar_wait(&tile_bar, 0, A.wait_ns);
        if (!ok) {
            atomicExch(&g_tile_wait_failed, 1);
            mbar_wait(&tile_bar, 0, A.wait_ns);  // let the copy land before the CTA ends
        }
        tile_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!tile_ok) return;  // uniform across the CTA
    mbar_wait(&tile_bar, 0, A.wait_ns);  // completed: acquires the tile for this thread

    if (L > 0) {
        Rep<T, MODEL, COMP, kSrcShared, true> f;  // d^2 is applied when the partials are added
        f.src.set_shared(tile, 0u);  // ids are relative to the tile
        f.d2 = T(1);
        f.q = A.q;
        // this thread's entries [a, b) (a < L), their storage, and the row of a
        const int32_t a = lane_start(L, threadIdx.x), b = lane_start(L, threadIdx.x + 1);
        const int32_t m8 = lane_len(L);
        const uint4* ids4 =
            reinterpret_cast<const uint4*>(A.tk + bsp + (int64_t)warp * 32 * m8) + lane;
        int lo = 0, hi = nrows;
        while (lo < hi) {  // the last i with D[i] <= a
            const int mid = (lo + hi + 1) >> 1;
            if (D[mid] <= a) lo = mid; else hi = mid - 1;
        }
        int ri = lo;
        while (D[ri + 1] <= a) ++ri;  // skip empty rows at a (a < L = D[nrows])
        const int ra = ri;  // the first row
        // it continues the previous share's last row (that share holds its
        // earlier entries, or is empty and ends in the row that holds a)
        const bool open_left =
            D[ra] < a || (threadIdx.x > 0 && lane_start(L, threadIdx.x - 1) == a);
        int32_t re = D[ri + 1];
        // the next nonempty row and its own position, fetched one row ahead
        auto next_row = [&](int i) {
            int x = i + 1;
            while (x < nrows && D[x + 1] == D[x]) ++x;
            return x < nrows ? x : i;
        };
        int nx = next_row(ri);
        P2 xr = pos[u0 + ri];
        P2 xn = pos[u0 + nx];
        f.xu = xr.x;
        f.yu = xr.y;
        Acc<T, COMP> acc, first;
        // compensated mode: the terms of the steps since the last merge,
        // summed plainly; added to acc with its error term at the end of
        // each ring of steps and before a row closes
        Acc<T, false> pend;
        auto merge_pending = [&]() {
            if (COMP) {
                add_compensated(acc, pend.sx, pend.sy);
                pend = Acc<T, false>();
            }
        };
        bool in_first = true;
        // the current row is complete: the first row's sum is kept for the
        // warp's scan; a later row lies wholly in [a, b) and is stored
        auto close_row = [&]() {
            merge_pending();
            if (in_first) {
                first = acc;
                in_first = false;
            } else {
                store_cell<T, COMP>(cellp(ri), acc);
            }
            acc = Acc<T, COMP>();
            ri = nx;
            re = D[ri + 1];
            xr = xn;
            f.xu = xr.x;
            f.yu = xr.y;
            nx = next_row(ri);
            xn = pos[u0 + nx];
        };
        // 16-byte id loads run kRing steps ahead (four, three with the
        // compensated sums, which need the registers); each unrolled step
        // consumes its own ring register and refills it: no register moves
        constexpr int kRing = COMP ? 3 : 4;
        const int nsteps = m8 / kStep;  // the same for every thread of the block
        uint4 ring[kRing];
#pragma unroll
        for (int st = 0; st < kRing; ++st) ring[st] = ld_ids4(ids4 + 32 * st);
        // the warp's ids kPrefetch steps ahead of the ring are pulled into L2
        // by one lane, kRing steps (kRing x 512 bytes) at a time
        const uint4* warp_ids = ids4 - lane;
        if (lane == 0)
            for (int k = kRing; k < kPrefetch + kRing && k < nsteps; k += kRing)
                bulk_prefetch_l2(warp_ids + 32 * k,
                                 (uint32_t)(512 * ((nsteps - k < kRing) ? nsteps - k : kRing)));
        // segments and shares are multiples of 8 entries: every step lies in
        // one row, and rows change only between steps. A step before the
        // current row's end (and the share's) goes straight to its eight
        // terms; a step where a row begins first closes the rows before it
        int32_t lim = (re < b) ? re : b;
        int32_t p = a;
        auto eight = [&](const uint4 c) {
            if (COMP) {
                // compensated mode: into the plain pending sum
                f(c.x & 0xffffu, pend);
                f(c.x >> 16, pend);
                f(c.y & 0xffffu, pend);
                f(c.y >> 16, pend);
                f(c.z & 0xffffu, pend);
                f(c.z >> 16, pend);
                f(c.w & 0xffffu, pend);
                f(c.w >> 16, pend);
            } else {
                f(c.x & 0xffffu, acc);
                f(c.x >> 16, acc);
                f(c.y & 0xffffu, acc);
                f(c.y >> 16, acc);
                f(c.z & 0xffffu, acc);
                f(c.z >> 16, acc);
                f(c.w & 0xffffu, acc);
                f(c.w >> 16, acc);
            }
        };
        // one step: its eight terms, after closing the rows that end before
        // it; the ring register refilled kRing steps ahead (the id array has
        // kRing steps of slack at its end, so the refill needs no test)
        auto step = [&](uint4& r, int k) {
            const uint4 c = r;
            r = ld_ids4(ids4 + 32 * (k + kRing));
            if (sizeof(T) == 8) {
                // FP64 (costly terms): the warp takes every step together
                // and only the closing of rows diverges, so no term is
                // issued twice (BA k = 3: 5.15 ms; 7.08 ms as for FP32)
                if (p < b) {
                    while (p >= re) close_row();
                    eight(c);
                }
            } else if (A.uniform) {
                // FP32, default: only the closing of rows diverges, the
                // step's terms are issued once for the warp; steps past the
                // share hold the far slot's id and add zeros
                if (p >= lim) {
                    if (p < b) {
                        while (p >= re) close_row();
                        lim = (re < b) ? re : b;
                    } else {
                        lim = INT32_MAX;
                    }
                }
                eight(c);
            } else if (p < lim) {
                // FP32, tuning step_schedule = -1: lanes that close a row
                // in this step issue its terms apart from the others
                eight(c);
            } else if (p < b) {
                while (p >= re) close_row();
                lim = (re < b) ? re : b;
                eight(c);
            }
            p += kStep;
        };
        int k0 = 0;
        for (; k0 + kRing <= nsteps; k0 += kRing) {
            const int kp = k0 + kPrefetch + kRing;
            if (lane == 0 && kp < nsteps)
                bulk_prefetch_l2(warp_ids + 32 * kp,
                                 (uint32_t)(512 * ((nsteps - kp < kRing) ? nsteps - kp : kRing)));
#pragma unroll
            for (int st = 0; st < kRing; ++st) step(ring[st], k0 + st);
            merge_pending();
        }
#pragma unroll
        for (int st = 0; st < kRing - 1; ++st)
            if (k0 + st < nsteps) step(ring[st], k0 + st);
        merge_pending();
        const bool has_b = !in_first;  // the share ends in a later row than it began
        if (in_first) first = acc;
        const int orow = has_b ? ri : ra;  // the row the share ends in
        const bool open_right = re > b;

        // Rows cut by share bounds, in lane order: element A (row ra, sum
        // first) and, with has_b, element B (row ri, sum acc). A segmented
        // scan of the warp's elements (A continues the previous lane's last
        // row, B always starts a run) gives each run's sum where it ends.
        Acc<T, COMP> x = has_b ? acc : first;
        const int prev_orow = __shfl_up_sync(kFull, orow, 1);
        const bool cont = lane > 0 && prev_orow == ra;
        const bool start = has_b || !cont;
        const unsigned starts = __ballot_sync(kFull, start);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            // the run of lane - o reaches this lane when no run starts in
            // lanes (lane - o, lane]
            const unsigned span = (lane >= o) ? (((1u << o) - 1u) << (lane - o + 1)) : 0u;
            const T sx = __shfl_up_sync(kFull, x.sx, o);
            const T sy = __shfl_up_sync(kFull, x.sy, o);
            const T cx = COMP ? __shfl_up_sync(kFull, x.cx, o) : T(0);
            const T cy = COMP ? __shfl_up_sync(kFull, x.cy, o) : T(0);
            if (lane >= o && (starts & span) == 0) {
                Acc<T, COMP> y;
                y.sx = sx;
                y.sy = sy;
                y.cx = cx;
                y.cy = cy;
                y.merge(x.sx, x.sy, x.cx, x.cy);
                x = y;
            }
        }
        // the sum of the run that reaches into A of a lane with B
        Acc<T, COMP> carry;
        {
            const T sx = __shfl_up_sync(kFull, x.sx, 1);
            const T sy = __shfl_up_sync(kFull, x.sy, 1);
            const T cx = COMP ? __shfl_up_sync(kFull, x.cx, 1) : T(0);
            const T cy = COMP ? __shfl_up_sync(kFull, x.cy, 1) : T(0);
            if (cont) {
                carry.sx = sx;
                carry.sy = sy;
                carry.cx = cx;
                carry.cy = cy;
            }
        }
        // runs that include lane 0's A belong to a row begun before the
        // warp's entries when lane 0's first row is open on the left; such a
        // run, and one running past the warp's last entry, goes to the
        // warp's slots, every other run to its cell
        const bool lane0_open = __shfl_sync(kFull, open_left, 0);
        const bool lane0_has_b = __shfl_sync(kFull, has_b, 0);
        const bool last_open = __shfl_sync(kFull, open_right, 31);
        const unsigned below = starts & ((2u << lane) - 1u) & ~1u;  // starts in lanes 1..lane
        auto put = [&](int row, const Acc<T, COMP>& v, bool from_lane0, bool past_end) {
            if (from_lane0 && lane0_open) {
                Slot<T, COMP>& sl = head[warp];
                sl.row = row;
                sl.v[0] = v.sx;
                sl.v[1] = v.sy;
                sl.v[2] = v.cx;
                sl.v[3] = v.cy;
            } else if (past_end) {
                Slot<T, COMP>& sl = tail[warp];
                sl.row = row;
                sl.v[0] = v.sx;
                sl.v[1] = v.sy;
                sl.v[2] = v.cx;
                sl.v[3] = v.cy;
            } else {
                store_cell<T, COMP>(cellp(row), v);
            }
        };
        if (has_b) {
            // A's run ends here: the carry plus this lane's first row
            carry.merge(first.sx, first.sy, first.cx, first.cy);
            const bool a_from0 =
                (lane == 0) || (cont && !lane0_has_b && (below & ~(1u << lane)) == 0);
            put(ra, carry, a_from0, false);
        }
        const int next_ra = __shfl_down_sync(kFull, ra, 1);
        const bool ends_here = (lane == 31) || next_ra != orow;
        if (ends_here) {
            const bool o_from0 = !has_b && !lane0_has_b && below == 0;
            put(orow, x, o_from0, lane == 31 && last_open);
        }
    }
    __syncthreads();
    if (warp == 0) {
        // rows cut by warp bounds: warp w's slots (a row begun before the
        // warp, a row running past its end) go to lane w of warp 0, and a
        // segmented scan across the lanes adds each row's slots in warp
        // order (a row's slots lie in consecutive warps; a warp without
        // slots lies between no two slots of one row)
        const Slot<T, COMP>& hs = head[lane];
        const Slot<T, COMP>& ts = tail[lane];
        auto acc_of = [](const Slot<T, COMP>& sl) {
            Acc<T, COMP> v;
            v.sx = sl.v[0];
            v.sy = sl.v[1];
            v.cx = sl.v[2];
            v.cy = sl.v[3];
            return v;
        };
        // the lane's elements: A (its first row) and, with has_b, B (a
        // second row); a lane without slots takes a row no lane has
        const bool hh = hs.row >= 0, ht = ts.row >= 0;
        const int ra = hh ? hs.row : (ht ? ts.row : -2 - lane);
        Acc<T, COMP> ea = hh ? acc_of(hs) : (ht ? acc_of(ts) : Acc<T, COMP>());
        bool has_b = false;
        Acc<T, COMP> eb;
        if (hh && ht) {
            if (ts.row == hs.row) {
                ea.merge(ts.v[0], ts.v[1], ts.v[2], ts.v[3]);
            } else {
                has_b = true;
                eb = acc_of(ts);
            }
        }
        const int orow = has_b ? ts.row : ra;
        Acc<T, COMP> x = has_b ? eb : ea;
        const int prev_orow = __shfl_up_sync(kFull, orow, 1);
        const bool cont = lane > 0 && prev_orow == ra;
        const unsigned starts = __ballot_sync(kFull, has_b || !cont);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned span = (lane >= o) ? (((1u << o) - 1u) << (lane - o + 1)) : 0u;
            const T sx = __shfl_up_sync(kFull, x.sx, o);
            const T sy = __shfl_up_sync(kFull, x.sy, o);
            const T cx = COMP ? __shfl_up_sync(kFull, x.cx, o) : T(0);
            const T cy = COMP ? __shfl_up_sync(kFull, x.cy, o) : T(0);
            if (lane >= o && (starts & span) == 0) {
                Acc<T, COMP> y;
                y.sx = sx;
                y.sy = sy;
                y.cx = cx;
                y.cy = cy;
                y.merge(x.sx, x.sy, x.cx, x.cy);
                x = y;
            }
        }
        const T px = __shfl_up_sync(kFull, x.sx, 1);
        const T py = __shfl_up_sync(kFull, x.sy, 1);
        const T pcx = COMP ? __shfl_up_sync(kFull, x.cx, 1) : T(0);
        const T pcy = COMP ? __shfl_up_sync(kFull, x.cy, 1) : T(0);
        if (has_b) {
            // A's run ends here: the run reaching into A, then A
            Acc<T, COMP> carry;
            if (cont) {
                carry.sx = px;
                carry.sy = py;
                carry.cx = pcx;
                carry.cy = pcy;
            }
            carry.merge(ea.sx, ea.sy, ea.cx, ea.cy);
            store_cell<T, COMP>(cellp(ra), carry);
        }
        const int next_ra = __shfl_down_sync(kFull, ra, 1);
        if (orow >= 0 && (lane == 31 || next_ra != orow)) store_cell<T, COMP>(cellp(orow), x);
    }
    if constexpr (WIN) {
        // every row of the range is complete here: F = d^2 (its cell) + the
        // attraction over its adjacency row (whose neighbours lie in the
        // window, as A is part of N(k)), then the capped move
        __syncthreads();
        window_finish<T, MODEL, COMP>(A, tile, tb, cells, u0, nrows);
    }
}


template <class T, int MODEL, bool COMP>
__device__ __forceinline__ void finish_row(const BlockedArgs& A, const Att<T, MODEL, COMP, kSrcShared>& att0,
                                           const typename V2<T>::type* cells, int64_t u0, int i,
                                           const Acc<T, COMP>& at)
{
    using P2 = typename V2<T>::type;
    const P2 pu = reinterpret_cast<const P2*>(A.pos)[u0 + i];
    const T d2 = (T)(A.d * A.d);
    Acc<T, COMP> rep;
    const P2 c0 = cells[2 * i];
    rep.sx = c0.x * d2;
    rep.sy = c0.y * d2;
    if (COMP) {
        const P2 c1 = cells[2 * i + 1];
        rep.cx = c1.x * d2;
        rep.cy = c1.y * d2;
    }
    rep.merge(at.sx, at.sy, at.cx, at.cy);
    apply_move<T>(A.t, A.pos_out, A.disp_out, u0 + i, pu.x, pu.y, rep.fx(), rep.fy());
}

template <class T, int MODEL, bool COMP>
__device__ __forceinline__ void window_finish(const BlockedArgs& A,
                                              const typename V2<T>::type* tile, int64_t tb,
                                              const typename V2<T>::type* cells, int64_t u0,
                                              int nrows)
{
    using P2 = typename V2<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const P2* __restrict__ pos = reinterpret_cast<const P2*>(A.pos);
    Att<T, MODEL, COMP, kSrcShared> att;
    att.src.set_shared(tile, (uint32_t)tb);
    att.inv_d = (T)(1.0 / A.d);
    att.p = A.p;
    const uint32_t* col = reinterpret_cast<const uint32_t*>(A.col);
    // warp w takes rows [32 w, 32 w + 32), then 1024 further on: each lane
    // one row; rows with more than kFinishDeg neighbours are then taken by
    // the whole warp, one after the other, lanes striding the adjacency row
    // (no barrier; a row's order of additions depends only on its length)
    for (int base = warp * 32; base < nrows; base += kBThreads) {
        const int i = base + lane;
        const bool live = i < nrows;
        int64_t rb = 0, re = 0;
        if (live) {
            rb = A.row[u0 + i];
            re = A.row[u0 + i + 1];
        }
        const bool hub = live && re - rb > kFinishDeg;
        if (live && !hub) {
            Att<T, MODEL, COMP, kSrcShared> a1 = att;
            const P2 pu = pos[u0 + i];
            a1.xu = pu.x;
            a1.yu = pu.y;
            Acc<T, COMP> at;
            row_sum_rel(col, rb, re, 0, 1, a1, at);
            finish_row<T, MODEL, COMP>(A, att, cells, u0, i, at);
        }
        unsigned hubs = __ballot_sync(kFull, hub);
        while (hubs) {
            const int l = __ffs(hubs) - 1;
            hubs &= hubs - 1;
            const int ih = base + l;
            const int64_t hb = __shfl_sync(kFull, rb, l), he = __shfl_sync(kFull, re, l);
            const P2 pu = pos[u0 + ih];
            Att<T, MODEL, COMP, kSrcShared> a1 = att;
            a1.xu = pu.x;
            a1.yu = pu.y;
            Acc<T, COMP> at;
            row_sum_rel(col, hb, he, lane, 32, a1, at);
            at.group_reduce(32);
            if (lane == 0) finish_row<T, MODEL, COMP>(A, att, cells, u0, ih, at);
        }
    }
}

struct CombineArgs {
    const int64_t* row;
    const int32_t* col;
    int64_t n;
    int32_t nt;
    double d, t;
    int p;
    const void* pos_in;
    const void* part;
    void* pos_out;
    void* disp_out;
    const int32_t* hubs;  // rows with more than kHubDeg neighbours, one block each
    int32_t nhub;         // hub blocks, first in the grid
    int32_t nreg;         // blocks of the regular part of the grid, after the hubs
};

// Regular rows: four lanes per vertex (more vertices in flight; measured
// 1.8% faster per iteration than eight on the Barabasi-Albert workload).
// Hubs (adjacency rows longer than kHubDeg) take a block of kCombineThreads
// each, at the start of the grid, so no vertex walks a long row on a few
// lanes while the rest of the GPU waits and the hubs do not form a tail.
constexpr int kCombineLanes = 4;
constexpr int kCombineThreads = 256;
constexpr int kHubDeg = 64;

// Entries [s, e) of ids, lane gl of a group of G taking s + gl, s + gl + G,
// ... as row_sum_rel does (same terms, same order of additions), with the
// ids of U consecutive turns loaded before their terms, so that a lane has U
// id loads and then U position gathers in flight instead of one of each.
template <int U, class F, class A>
__device__ __forceinline__ void row_sum_batched(const uint32_t* __restrict__ ids, int64_t s,
                                                int64_t e, int gl, int G, const F& f, A& a)
{
    const uint32_t* p = ids + s;
    const int len = (int)(e - s);
    int j = gl;
    for (; j + (U - 1) * G < len; j += U * G) {
        uint32_t v[U];
#pragma unroll
        for (int k = 0; k < U; ++k) v[k] = ld_id(p + j + k * G);
#pragma unroll
        for (int k = 0; k < U; ++k) f(v[k], a);
    }
    for (; j < len; j += G) f(ld_id(p + j), a);
}

template <class T, bool COMP>
__device__ __forceinline__ void add_cell(const void* part, int64_t n, int j, int64_t u,
                                         Acc<T, COMP>& s)
{
    using P2 = typename V2<T>::type;
    const P2* c = cell_ptr<T, COMP>(const_cast<void*>(part), n, j, u);
    const P2 v = c[0];
    if (COMP) {
        const P2 k = c[1];
        s.merge(v.x, v.y, k.x, k.y);
    } else {
        s.merge(v.x, v.y, T(0), T(0));
    }
}

// F = d^2 (sum of the tile partials) + attraction; then the capped move.
template <class T, bool COMP>
__device__ __forceinline__ void finish_vertex(const CombineArgs& A, int64_t u, T xu, T yu,
                                              Acc<T, COMP> rep, const Acc<T, COMP>& att)
{
    const T d2 = (T)(A.d * A.d);
    rep.sx *= d2;
    rep.sy *= d2;
    rep.cx *= d2;
    rep.cy *= d2;
    rep.merge(att.sx, att.sy, att.cx, att.cy);
    apply_move<T>(A.t, A.pos_out, A.disp_out, u, xu, yu, rep.fx(), rep.fy());
}

template <class T, int MODEL, bool COMP>
__global__ void __launch_bounds__(kCombineThreads) combine_kernel(const CombineArgs A)
{
    using P2 = typename V2<T>::type;
    const P2* __restrict__ pos = reinterpret_cast<const P2*>(A.pos_in);
    Att<T, MODEL, COMP> att;
    att.src.pos = pos;
    att.inv_d = (T)(1.0 / A.d);
    att.p = A.p;
    Acc<T, COMP> rep, at;
    if ((int)blockIdx.x < A.nhub) {
        // one hub per block
        __shared__ T sh[kCombineThreads / 32][8];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int64_t u = A.hubs[blockIdx.x];
        const P2 pu = pos[u];
        for (int jj = threadIdx.x; jj < A.nt; jj += kCombineThreads)
            add_cell<T, COMP>(A.part, A.n, jj, u, rep);
        att.xu = pu.x;
        att.yu = pu.y;
        row_sum_batched<4>(reinterpret_cast<const uint32_t*>(A.col), A.row[u], A.row[u + 1],
                           (int)threadIdx.x, kCombineThreads, att, at);
        rep.group_reduce(32);
        at.group_reduce(32);
        if (lane == 0) {
            sh[warp][0] = rep.sx;
            sh[warp][1] = rep.sy;
            sh[warp][2] = rep.cx;
            sh[warp][3] = rep.cy;
            sh[warp][4] = at.sx;
            sh[warp][5] = at.sy;
            sh[warp][6] = at.cx;
            sh[warp][7] = at.cy;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Acc<T, COMP> r2, a2;
            for (int w = 0; w < kCombineThreads / 32; ++w) {
                r2.merge(sh[w][0], sh[w][1], sh[w][2], sh[w][3]);
                a2.merge(sh[w][4], sh[w][5], sh[w][6], sh[w][7]);
            }
            finish_vertex<T, COMP>(A, u, pu.x, pu.y, r2, a2);
        }
        return;
    }
    const int gl = threadIdx.x & (kCombineLanes - 1);
    const int64_t u = ((int64_t)(blockIdx.x - A.nhub) * kCombineThreads + threadIdx.x) / kCombineLanes;
    bool live = u < A.n;
    int64_t rb = 0, re = 0;
    if (live) {
        rb = A.row[u];
        re = A.row[u + 1];
        live = re - rb <= kHubDeg;  // hubs are done by their own blocks
    }
    P2 pu;
    pu.x = T(0);
    pu.y = T(0);
    if (live) {
        // tile partials first (independent loads), lane gl takes tiles gl, gl + 8, ...
        for (int jj = gl; jj < A.nt; jj += kCombineLanes) add_cell<T, COMP>(A.part, A.n, jj, u, rep);
        pu = pos[u];
        att.xu = pu.x;
        att.yu = pu.y;
        row_sum_batched<2>(reinterpret_cast<const uint32_t*>(A.col), rb, re, gl, kCombineLanes, att,
                           at);
    }
    rep.group_reduce(kCombineLanes);
    at.group_reduce(kCombineLanes);
    if (live && gl == 0) finish_vertex<T, COMP>(A, u, pu.x, pu.y, rep, at);
}

// Length of row u's segment in tile j (binary search on the sorted row).
__device__ __forceinline__ void seg_bounds(const int64_t* __restrict__ krow,
                                           const uint32_t* __restrict__ kcol, int64_t u, int j,
                                           int nt, int tv, int64_t* lo, int64_t* hi)
{
    const int64_t kb = krow[u], ke = krow[u + 1];
    auto lower = [&](uint32_t key) {
        int64_t x = kb, y = ke;
        while (x < y) {
            const int64_t mid = (x + y) >> 1;
            if (kcol[mid] < key) x = mid + 1; else y = mid;
        }
        return x;
    };
    *lo = (j == 0) ? kb : lower((uint32_t)j * (uint32_t)tv);
    *hi = (j == nt - 1) ? ke : lower((uint32_t)(j + 1) * (uint32_t)tv);
}

__global__ void seglen_kernel(int64_t n, const int64_t* __restrict__ krow,
                              const uint32_t* __restrict__ kcol, int nt, int tv,
                              int64_t* __restrict__ len)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nt) return;
    int64_t lo, hi;
    seg_bounds(krow, kcol, i % n, (int)(i / n), nt, tv, &lo, &hi);
    len[i] = hi - lo;
}

// Copy every (tile, row) segment into its block's share storage as 16-bit
// ids relative to the tile: entry p of the block, held by the share of
// thread t (s = p - lane_start(L, t)), goes to slot
// (t / 32) 32 lane_len(L) + 256 (s / 8) + 8 (t % 32) + s % 8.
//
// With SPREAD each segment's ids are also ordered for blocked_kernel's
// shared-memory gathers. A warp's gather is served in groups of G lanes
// (G = 128 bytes / position size: 16 for float2, 8 for double2), one
// wavefront per group when the group's tile offsets are distinct modulo G
// (distinct banks), one more per repeat; in ascending id order the residues
// fall at random and a 16-lane group takes about three. In one gather the
// lanes of a group read entry s of their own shares, so entry s of thread t
// aims at residue (t + s) mod G, distinct across the group for every s. A
// row's sum does not depend on the order of its entries (up to rounding)
// and a segment is one row, so its ids are dealt to its entries: each entry
// takes an id of its target residue while one is left (lanes in order),
// else one of the nearest residue above it (cyclically) that has ids left.
// One warp per segment, through shared memory by chunks of at most
// kSpreadChunk entries: count the chunk's residues, group its ids by residue
// (stable), deal them 32 entries at a time.
// A larger chunk leaves fewer entries without their target residue (each
// such entry costs its half-warp one more gather wavefront): 2048 entries
// held as 16-bit relative ids (4 KB a warp) against 1024 as 32-bit ids took
// Chung-Lu n = 250,000, k = 3 from 4.27 to 4.18 ms per launch, the plan
// from 174 to 170 ms; 4096 gave 4.15 ms but a 229 ms plan (half the
// occupancy).
constexpr int kSpreadWarps = 4;
constexpr int kSpreadChunk = 2048;

// Every slot of block b's share storage set to the block's padding id (its
// far slot) before the layout kernel writes the entries: the slots past
// each thread's share keep it, so that the FP32 kernel takes a thread's
// last steps like any other (their terms are exact zeros). Block starts are
// multiples of 8 slots: whole 16-byte stores.
__global__ void pad_fill_kernel(uint16_t* __restrict__ tk, const int64_t* __restrict__ blk,
                                const int64_t* __restrict__ wbase, int tv, int64_t nb)
{
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t bsp = blk[2 * b];
        const int64_t words = (int64_t)kBThreads * lane_len((int32_t)blk[2 * b + 1]) / 8;
        const uint32_t pad = wbase ? (uint32_t)wbase[2 * b + 1] : (uint32_t)tv;
        const uint32_t pp = pad | (pad << 16);
        const uint4 v = make_uint4(pp, pp, pp, pp);
        uint4* dst = reinterpret_cast<uint4*>(tk + bsp);
        for (int64_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = v;
    }
}

template <int G, bool SPREAD>
__global__ void __launch_bounds__(kSpreadWarps * 32) block_layout_kernel(
    int64_t n, const int64_t* __restrict__ krow, const uint32_t* __restrict__ kcol, int nt,
    int tv, const int64_t* __restrict__ wbase, const int64_t* __restrict__ toff,
    const int64_t* __restrict__ blk, const int32_t* __restrict__ tfirst,
    const int32_t* __restrict__ rstart, const int32_t* __restrict__ rblock,
    uint16_t* __restrict__ tk)
{
    __shared__ uint16_t s_in[kSpreadWarps][kSpreadChunk];  // the chunk's relative ids by residue
    __shared__ int s_run[kSpreadWarps][G];
    __shared__ int s_ask[kSpreadWarps][G];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n * nt) return;  // warp-uniform
    const int j = (int)(i / n);
    const int64_t u = i % n;
    int64_t lo, hi;
    seg_bounds(krow, kcol, u, j, nt, tv, &lo, &hi);
    if (hi == lo) return;
    // the range of tile j that holds row u (tile j's ranges: blocks
    // tfirst[j] .. tfirst[j + 1] - 1 in tile order, their row bounds at
    // rstart + tfirst[j] + j), and that range's block
    const int32_t f0 = tfirst[j];
    const int32_t* st = rstart + f0 + j;
    int ra = 0, rb = tfirst[j + 1] - f0 - 1;
    while (ra < rb) {
        const int mid = (ra + rb + 1) >> 1;
        if (st[mid] <= u) ra = mid; else rb = mid - 1;
    }
    const int64_t b = rblock[f0 + ra];
    // ids are relative to tile j, or in window mode to block b's window;
    // the padding takes the far slot one past the tile or window
    const uint32_t tb = wbase ? (uint32_t)wbase[2 * b] : (uint32_t)j * (uint32_t)tv;
    const uint16_t pad = wbase ? (uint16_t)wbase[2 * b + 1] : (uint16_t)tv;
    const int64_t bsp = blk[2 * b];
    const int32_t L = (int32_t)blk[2 * b + 1];
    const int32_t m8 = lane_len(L);
    const int32_t S0 = (int32_t)toff[i], S1 = S0 + (int32_t)(hi - lo);
    const int32_t S8 = S0 + (int32_t)((hi - lo + kStep - 1) & ~int64_t(kStep - 1));  // padded end
    // the share holding entry p (t follows p, which only grows) and the slot
    int t = (int)((int64_t)S0 * kBThreads / L);
    int32_t sidx = 0;  // p's index in its share, set by place
    auto place = [&](int32_t p) -> int64_t {
        while (t > 0 && lane_start(L, t) > p) --t;
        while (t < kBThreads - 1 && lane_start(L, t + 1) <= p) ++t;
        sidx = p - lane_start(L, t);
        return bsp + (int64_t)(t >> 5) * 32 * m8 + 256 * (sidx >> 3) + 8 * (t & 31) + (sidx & 7);
    };
    if (!SPREAD) {
        for (int32_t p = S0 + lane; p < S8; p += 32)
            tk[place(p)] = (p < S1) ? (uint16_t)(kcol[lo + (p - S0)] - tb) : pad;
        return;
    }
    uint16_t* in = s_in[wl];
    int* run = s_run[wl];
    int* ask = s_ask[wl];
    for (int32_t c0 = S0; c0 < S1; c0 += kSpreadChunk) {
        const int len = (S1 - c0 < kSpreadChunk) ? S1 - c0 : kSpreadChunk;
        const uint32_t* src = kcol + lo + (c0 - S0);
        // residue counts of the chunk and their exclusive prefix (lane c: residue c)
        if (lane < G) run[lane] = 0;
        __syncwarp();
        for (int e = lane; e < len; e += 32) atomicAdd(&run[(src[e] - tb) % G], 1);
        __syncwarp();
        const int cnt = (lane < G) ? run[lane] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int cstart = incl - cnt;
        __syncwarp();
        if (lane < G) run[lane] = cstart;
        __syncwarp();
        // stable grouping by residue
        for (int e0 = 0; e0 < len; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < len;
            const uint32_t id = act ? src[e] : 0u;
            const int c = act ? (int)((id - tb) % G) : G + lane;
            const unsigned m = __match_any_sync(kFull, c);
            const int o = act ? run[c] + __popc(m & ((1u << lane) - 1u)) : 0;
            __syncwarp();
            if (act && lane == 31 - __clz(m)) run[c] += __popc(m);
            __syncwarp();
            if (act) in[o] = (uint16_t)(id - tb);
        }
        __syncwarp();  // the grouped ids are visible to the whole warp

        // deal: lane c < G keeps residue c's ids left and taken
        int rem = cnt, used = 0;
        for (int e0 = 0; e0 < len; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < len;
            const int64_t d = act ? place(c0 + e) : 0;
            const int want = act ? (int)(((t % G) + sidx) % G) : 0;
            // the target residue for as many lanes as it has ids left, in lane order
            const unsigned m = __match_any_sync(kFull, act ? want : G + lane);
            const int rank = __popc(m & ((1u << lane) - 1u));
            const int left = __shfl_sync(kFull, rem, want);
            const int base = __shfl_sync(kFull, cstart + used, want);
            const bool got = act && rank < left;
            uint16_t id = got ? in[base + rank] : (uint16_t)0;
            // residue c's lane takes off the lanes that asked for c (at most rem)
            if (lane < G) ask[lane] = 0;
            __syncwarp();
            if (act && rank == 0) ask[want] = __popc(m);
            __syncwarp();
            if (lane < G) {
                const int give = (ask[lane] < rem) ? ask[lane] : rem;
                rem -= give;
                used += give;
            }
            // the others in lane order: the nearest residue at or above the
            // target (cyclically) that has ids left
            unsigned pend = __ballot_sync(kFull, act && !got);
            while (pend) {
                const int l = __ffs(pend) - 1;
                const int wt = __shfl_sync(kFull, want, l);
                const unsigned av = __ballot_sync(kFull, lane < G && rem > 0) & ((1u << G) - 1u);
                if (av == 0) break;  // cannot happen: ids left equal entries left
                const unsigned rot = ((av >> wt) | (av << (G - wt))) & ((1u << G) - 1u);
                const int c = (wt + __ffs(rot) - 1) % G;
                const int at = __shfl_sync(kFull, cstart + used, c);
                if (lane == c) {
                    --rem;
                    ++used;
                }
                if (lane == l) id = in[at];
                pend &= pend - 1;
            }
            if (act) tk[d] = id;
        }
        __syncwarp();  // the next chunk reuses the buffers
    }
    // the padding (at most 7 entries, lanes 0-6)
    if (S1 + lane < S8) tk[place(S1 + lane)] = pad;
}

template <class T, int MODEL, bool COMP, bool WIN>
cudaError_t launch_blocked_typed(gila_graph* g, const BlockedArgs& B, const CombineArgs& C,
                                 int grid, size_t smem, cudaStream_t st, int device)
{
    static std::atomic<uint64_t> configured{0};  // one bit per device; callers may race
    const uint64_t bit = 1ull << (device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(blocked_kernel<T, MODEL, COMP, WIN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemCap - 4096);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    cudaEvent_t pa = prof_kernel_begin(g);
    blocked_kernel<T, MODEL, COMP, WIN><<<grid, kBThreads, smem, st>>>(B);
    count_launch();
    cudaError_t e = cudaGetLastError();
    prof_kernel_end(g, pa, WIN ? "blocked_kernel (window)" : "blocked_kernel");
    if (e != cudaSuccess || WIN) return e;
    combine_kernel<T, MODEL, COMP><<<(unsigned)(C.nreg + C.nhub), kCombineThreads, 0, st>>>(C);
    count_launch();
    return cudaGetLastError();
}

template <class T, int MODEL, bool COMP>
cudaError_t launch_pair(gila_graph* g, const BlockedArgs& B, const CombineArgs& C, int grid,
                        size_t smem, cudaStream_t st, int device, bool win)
{
    return win ? launch_blocked_typed<T, MODEL, COMP, true>(g, B, C, grid, smem, st, device)
               : launch_blocked_typed<T, MODEL, COMP, false>(g, B, C, grid, smem, st, device);
}

// The k-hop term of the quality reductions, sum over unordered k-hop pairs
// {u, v} of d^2 / delta^q, for FP32 placements that have a blocked plan:
// one CTA per (tile or window, row range), positions from the shared-memory
// tile, each pair counted once from its smaller end. Every row is sorted,
// so the entries of row u in the tile are one contiguous run that starts
// after the row's runs in earlier tiles (the plan's segment lengths), and
// only the tile that holds u itself needs a binary search to drop the ids
// up to u. The CTA takes its rows by batches: their runs are numbered by a
// block scan and each warp takes an equal slice of the batch's entries (a
// warp per row left the CTA's warps waiting on the one with a hub's row:
// barrier stalls 5.1 per issue, 38% issue active on Chung-Lu n = 40,000).
// Each term is in double-float arithmetic (ff.cuh), sixteen terms per lane
// summed as a double-float, then added in FP64; the CTA's FP64 partial goes
// to its own slot, and the partials are added in CTA order.
constexpr int kMetThreads = 1024;
constexpr int kMetWarps = kMetThreads / 32;
constexpr int kMetBatch = 512;  // rows per batch (10.5 KB of shared memory beside the tile)
constexpr int kMetSmemMax = kSmemCap - 12 * 1024;  // the tile's share of shared memory

struct MetricArgs {
    const int64_t* krow;
    const int64_t* len;    // tile mode: nt n segment lengths (row u's entries in tile j)
    const uint32_t* kcol;
    const int4* bdesc;     // nb: first row, end row and tile of block b
    const int64_t* wbase;  // window mode: 2 nb (first id, length), else null
    int64_t n;
    int32_t nt, tv, tcap;
    double d;
    int q;
    const float2* pos;
    double* partial;       // one per CTA
    uint64_t wait_ns;
};

__global__ void __launch_bounds__(kMetThreads, 1) khop_metric_kernel(const MetricArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* tile = reinterpret_cast<float2*>(smem_raw);
    __shared__ __align__(8) uint64_t tile_bar;
    __shared__ int tile_ok;
    __shared__ double s_part[kMetWarps];
    __shared__ int s_wsum[kMetWarps];
    __shared__ int s_pre[kMetBatch + 1];
    __shared__ int64_t s_lo[kMetBatch];
    __shared__ float2 s_q[kMetBatch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 bd = A.bdesc[blockIdx.x];
    const int j = bd.z;
    const int64_t u0 = bd.x, u1 = bd.y;
    const int64_t tb = A.wbase ? A.wbase[2 * blockIdx.x] : (int64_t)j * A.tv;
    const int64_t tn = A.wbase ? A.wbase[2 * blockIdx.x + 1]
                               : ((A.n - tb < A.tv) ? A.n - tb : (int64_t)A.tv);
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(((size_t)tn * sizeof(float2)) & ~size_t(15));
        mbar_init(&tile_bar, 1);
        mbar_arrive_expect_tx(&tile_bar, bytes);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(A.pos + tb);
        for (uint32_t o = 0; o < bytes; o += kBulkChunk)
            bulk_g2s(smem_raw + o, src + o, (bytes - o < kBulkChunk) ? bytes - o : kBulkChunk,
                     &tile_bar);
        if ((size_t)tn * sizeof(float2) != bytes) tile[tn - 1] = A.pos[tb + tn - 1];
        bool ok = mbar_wait(&tile_bar, 0, A.wait_ns);
        if (!ok) {
            atomicExch(&g_tile_wait_failed, 1);
            mbar_wait(&tile_bar, 0, A.wait_ns);
        }
        tile_ok = ok ? 1 : 0;
    }
    __syncthreads();
    double part = 0.0;
    if (tile_ok) {
        mbar_wait(&tile_bar, 0, A.wait_ns);
        const Ff d2f = ff_from_double(A.d * A.d);
        const bool unit = A.d == 1.0 && A.q == 1;
        Ff s = {0.f, 0.f};
        int cnt = 0;
        // one pair {u, v}: d^2 / delta^q in double-float, sixteen terms of a
        // lane summed as a double-float, then added to its FP64 sum
        auto term = [&](float2 qu, uint32_t v) {
            const float2 pv = tile[v - tb];
            const Ff r2 = ff_dist2(qu.x, qu.y, pv.x, pv.y);
            if (r2.hi >= 1e-30f && r2.hi <= 1e30f) {
                // d = 1, q = 1 (the defaults): the products by 1 are exact
                // and left out
                s = ff_add(s, unit ? ff_rsqrt(r2) : ff_mul(d2f, ff_rsqrt_pow(r2, A.q)));
            } else {
                const double dx = (double)qu.x - (double)pv.x;
                const double dy = (double)qu.y - (double)pv.y;
                const double dl = sqrt(dx * dx + dy * dy);
                if (dl > 0.0) {
                    double w = 1.0;
                    for (int i = 0; i < A.q; ++i) w *= dl;
                    part += A.d * A.d / w;
                }
            }
            if (++cnt == 16) {
                part += (double)s.hi + (double)s.lo;
                s = {0.f, 0.f};
                cnt = 0;
            }
        };
        // rows by batches of kMetBatch: thread t finds row r0 + t's run of
        // ids above u in this tile; a block scan numbers the batch's entries;
        // each warp then takes an equal slice of them (whatever the rows'
        // lengths), lanes striding it and following the row boundaries
        for (int64_t r0 = u0; r0 < u1; r0 += kMetBatch) {
            const int64_t u = r0 + threadIdx.x;
            int64_t lo = 0, hi = 0;
            if (threadIdx.x < kMetBatch && u < u1 && tb + tn > u + 1) {
                // the row's entries in this tile: the whole row in window
                // mode; in tile mode the segment after the row's segments in
                // earlier tiles (their lengths, summed in order)
                lo = A.krow[u];
                if (A.wbase) {
                    hi = A.krow[u + 1];
                } else {
                    for (int jj = 0; jj < j; ++jj) lo += A.len[(int64_t)jj * A.n + u];
                    hi = lo + A.len[(int64_t)j * A.n + u];
                }
                if (tb <= u) {
                    // the tile holds u: keep the ids above it (binary search)
                    int64_t x = lo, y = hi;
                    while (x < y) {
                        const int64_t mid = (x + y) >> 1;
                        if (A.kcol[mid] <= (uint32_t)u) x = mid + 1; else y = mid;
                    }
                    lo = x;
                }
                if (lo > hi) lo = hi;
            }
            const int len = (int)(hi - lo);
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += x;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const int x0 = s_wsum[lane];
                int x = x0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, x, o);
                    if (lane >= o) x += y;
                }
                s_wsum[lane] = x - x0;  // warps before this one
                if (lane == 31) s_pre[kMetBatch] = x;
            }
            __syncthreads();
            if (threadIdx.x < kMetBatch) {
                s_pre[threadIdx.x] = s_wsum[warp] + incl - len;
                s_lo[threadIdx.x] = lo;
                float2 q = make_float2(0.f, 0.f);
                if (u < u1) q = A.pos[u];
                s_q[threadIdx.x] = q;
            }
            __syncthreads();
            const int total = s_pre[kMetBatch];
            const int beg = (int)((int64_t)total * warp / kMetWarps);
            const int end = (int)((int64_t)total * (warp + 1) / kMetWarps);
            if (beg + lane < end) {
                // the row holding entry beg + lane: the last with s_pre <= it
                int r = 0, hr = kMetBatch - 1;
                while (r < hr) {
                    const int mid = (r + hr + 1) >> 1;
                    if (s_pre[mid] <= beg + lane) r = mid; else hr = mid - 1;
                }
                for (int i = beg + lane; i < end; i += 32) {
                    while (s_pre[r + 1] <= i) ++r;
                    term(s_q[r], A.kcol[s_lo[r] + (i - s_pre[r])]);
                }
            }
            __syncthreads();  // the next batch reuses the arrays
        }
        part += (double)s.hi + (double)s.lo;
    }
    // fixed-order block sum: lanes, then warps in order
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) s_part[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMetWarps; ++w) t += s_part[w];
        A.partial[blockIdx.x] = t;
    }
}

__global__ void sum_in_order_kernel(const double* __restrict__ v, int count, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < count; ++i) t += v[i];
        *out = t;
    }
}

}  // namespace

void invalidate_tile_plans(gila_graph* g)
{
    g->tplan[0].ready = false;
    g->tplan[1].ready = false;
}

gila_status blocked_tile_wait_failed(cudaStream_t st)
{
    int h = 0;
    const int zero = 0;
    GILA_CUDA(cudaMemcpyFromSymbolAsync(&h, g_tile_wait_failed, sizeof(int), 0,
                                        cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    if (h) {
        GILA_CUDA(cudaMemcpyToSymbolAsync(g_tile_wait_failed, &zero, sizeof(int), 0,
                                          cudaMemcpyHostToDevice, st));
        GILA_CUDA(cudaStreamSynchronize(st));
        return fail(GILA_ECUDA, "a tile copy of the iteration kernel did not complete in time");
    }
    return GILA_OK;
}

void free_tile_plans(gila_graph* g)
{
    for (TilePlan& P : g->tplan) {
        cudaFree(P.hubs);
        cudaFree(P.wtile);
        cudaFree(P.rowspan);
        cudaFree(P.bdesc);
        cudaFree(P.rdir);
        cudaFree(P.blk);
        cudaFree(P.toff);
        cudaFree(P.tk);
        cudaFree(P.part);
        cudaFree(P.len);
        P = TilePlan();
    }
}

// First and last id of every k-hop row (rows are sorted); INT32_MAX and -1
// for empty rows.
__global__ void rowspan_kernel(int64_t n, const int64_t* __restrict__ krow,
                               const uint32_t* __restrict__ kcol, int32_t* __restrict__ span)
{
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int64_t b = krow[u], e = krow[u + 1];
    span[2 * u] = b < e ? (int32_t)kcol[b] : INT32_MAX;
    span[2 * u + 1] = b < e ? (int32_t)kcol[e - 1] : -1;
}

// Cost of a row in one tile's (or window's) block: its padded entries and a
// per-row term where it has entries (directory, row change, cell store),
// else only the zeroed cell.
inline int64_t row_cost(int64_t len)
{
    return len > 0 ? 8 + ((len + kStep - 1) & ~int64_t(kStep - 1)) : 1;
}

// Greedy cut of one tile's rows into ranges of cost at most cap (a range
// takes at least one row) and at most max_rows rows; pre holds the prefix
// sums of the rows' costs (n + 1 values). Returns the number of ranges,
// stopping once it exceeds limit; fills cuts (the range bounds) if given.
int64_t cut_rows(const int64_t* pre, int64_t n, int64_t cap, int64_t limit, int64_t max_rows,
                 std::vector<int32_t>* cuts)
{
    int64_t s = 0, count = 0;
    if (cuts) cuts->assign(1, 0);
    while (s < n) {
        // the last e with pre[e] - pre[s] <= cap, at least s + 1
        int64_t e = (int64_t)(std::upper_bound(pre + s + 1, pre + n + 1, pre[s] + cap) - pre) - 1;
        e = std::min<int64_t>(std::max<int64_t>(e, s + 1), s + max_rows);
        if (cuts) cuts->push_back((int32_t)e);
        if (++count > limit) return count;
        s = e;
    }
    return count;
}

// Row ranges of every tile (window mode: one), all blocks with at most the
// same cost, the smallest for which the blocks number at most `target` (or
// the fewest the row limit allows). pre: nt prefix-sum arrays of n + 1
// costs, tile after tile. A grid of about target equal CTAs then ends
// together, where equal row ranges for all tiles left the hubs' tile with
// CTAs twice the mean and one more range than the target sent a few CTAs
// into a second wave (Barabasi-Albert n = 100,000, k = 2: 156 CTAs on 152
// SMs, the SMs busy 54% of the kernel's time).
std::vector<std::vector<int32_t>> partition_blocks(const std::vector<int64_t>& pre, int64_t n,
                                                   int64_t nt, int64_t target, int64_t max_rows)
{
    auto count = [&](int64_t cap, int64_t limit) {
        int64_t c = 0;
        for (int64_t j = 0; j < nt && c <= limit; ++j)
            c += cut_rows(pre.data() + j * (n + 1), n, cap, limit - c, max_rows, nullptr);
        return c;
    };
    int64_t hi = 0;  // a cap every tile fits in whole: the fewest ranges
    for (int64_t j = 0; j < nt; ++j) hi = std::max<int64_t>(hi, pre[(size_t)(j * (n + 1) + n)]);
    target = std::max<int64_t>(target, count(hi, INT64_MAX));
    int64_t lo = 0;  // count(lo) > target unless single rows already fit
    if (count(lo, target) <= target) hi = lo;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (count(mid, target) <= target) hi = mid; else lo = mid;
    }
    std::vector<std::vector<int32_t>> rs((size_t)nt);
    for (int64_t j = 0; j < nt; ++j)
        cut_rows(pre.data() + j * (n + 1), n, hi, INT64_MAX, max_rows, &rs[(size_t)j]);
    return rs;
}

// CTAs per SM the blocked grid aims at by default (blocks of equal cost,
// costliest first). Tiles: one wave below 10^8 k-hop entries, where loading
// a tile per CTA is a large part of an iteration (BA n = 100,000, k = 2:
// 0.0374 ms per iteration at 1, 0.0419 at 2); 3 up to 2e9 entries (BA
// n = 100,000, k = 3: 0.140, 0.138, 0.148, 0.157 ms per launch at 2, 3, 4,
// 6); 6 beyond, where a CTA streams tens of MB and the end of the grid
// waits on the slowest (Chung-Lu 1.1e10: 4.38, 4.15, 4.19, 4.19, 4.26 ms
// at 4, 6, 8, 12, 16). Windows: 2 (the mesh, k = 3: 0.0698, 0.0680, 0.0742
// ms at 1, 2, 3).
int64_t default_ctas_per_sm(int64_t nnz_khop, bool window)
{
    if (window) return 2;
    return nnz_khop < 100000000LL ? 1 : nnz_khop < 2000000000LL ? 3 : 6;
}

// CTAs (blocks) the grid aims at: about ctas_per_sm per SM.
int64_t blocks_target(const gila_graph* g, bool window)
{
    const int64_t per_sm = g->tune.ctas_per_sm > 0 ? g->tune.ctas_per_sm
                                                   : default_ctas_per_sm(g->nnz_khop, window);
    return std::max<int64_t>(1, per_sm * (int64_t)sm_count(g->device));
}

// The adjacency rows longer than kHubDeg, which the combine kernel gives a
// block each.
gila_status plan_hubs(gila_graph* g, TilePlan& P)
{
    const int64_t n = g->n;
    std::vector<int64_t> arow((size_t)n + 1);
    GILA_CUDA(cudaMemcpyAsync(arow.data(), g->row, sizeof(int64_t) * (n + 1),
                              cudaMemcpyDeviceToHost, g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int32_t> hubs;
    for (int64_t u = 0; u < n; ++u)
        if (arow[(size_t)u + 1] - arow[(size_t)u] > kHubDeg) hubs.push_back((int32_t)u);
    if (!hubs.empty()) {
        gila_status s = ensure((void**)&P.hubs, &P.hubs_cap, sizeof(int32_t) * hubs.size());
        if (s != GILA_OK) return s;
        GILA_CUDA(cudaMemcpyAsync(P.hubs, hubs.data(), sizeof(int32_t) * hubs.size(),
                                  cudaMemcpyHostToDevice, g->stream));
    }
    GILA_CUDA(cudaStreamSynchronize(g->stream));  // the host vector goes out of scope
    P.nhub = (int32_t)hubs.size();
    return GILA_OK;
}

// Shared memory a window-mode CTA needs: the window with the far slot, the
// row directory, and two position-type cells per row.
size_t window_smem(int64_t wmax, int64_t rmax, size_t esz)
{
    return (((size_t)(wmax + 1) * esz + (size_t)(rmax + 1) * 4 + 15) & ~size_t(15)) +
           (size_t)rmax * 2 * esz;
}

// Window mode: rows are cut into ranges, and each range's rows, whose k-hop
// ids span a window [b, b + len) of consecutive ids narrow enough for
// shared memory (meshes, grids, locality-preserving orders, and every graph
// small enough to fit whole), read their positions from that window. Each
// row then lies wholly in its range's block, so the CTA finishes its rows
// itself (no partials, no second kernel). *fits tells whether every range's
// window fits; `len` receives the row lengths, `rs` the ranges, `wb` the
// windows (2 nr: first id, length).
gila_status plan_window(gila_graph* g, size_t esz, TilePlan& P, bool* fits,
                        std::vector<int64_t>& len, std::vector<int32_t>& rs,
                        std::vector<int64_t>& wb, int64_t* wmax_out, int64_t* rmax_out)
{
    *fits = false;
    const int64_t n = g->n;
    std::vector<int64_t> krow((size_t)n + 1);
    GILA_CUDA(cudaMemcpyAsync(krow.data(), g->krow, sizeof(int64_t) * (n + 1),
                              cudaMemcpyDeviceToHost, g->stream));
    gila_status s = ensure((void**)&P.rowspan, &P.rowspan_cap, sizeof(int32_t) * 2 * (size_t)n);
    if (s != GILA_OK) return s;
    rowspan_kernel<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(n, g->krow, g->kcol,
                                                                      P.rowspan);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    std::vector<int32_t> span(2 * (size_t)n);
    GILA_CUDA(cudaMemcpyAsync(span.data(), P.rowspan, sizeof(int32_t) * 2 * n,
                              cudaMemcpyDeviceToHost, g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    len.assign((size_t)n, 0);
    std::vector<int64_t> pre((size_t)n + 1, 0);
    for (int64_t u = 0; u < n; ++u) {
        len[(size_t)u] = krow[(size_t)u + 1] - krow[(size_t)u];
        pre[(size_t)u + 1] = pre[(size_t)u] + row_cost(len[(size_t)u]);
    }
    // enough ranges for several CTAs per SM, but at least about 16 entries
    // per thread of a CTA (a small graph is one or a few ranges)
    const int64_t by_work = std::max<int64_t>(1, pre[(size_t)n] / ((int64_t)kBThreads * 16));
    rs = partition_blocks(pre, n, 1, std::min<int64_t>(blocks_target(g, true), by_work),
                          kMaxRows)[0];
    const int64_t nr = (int64_t)rs.size() - 1;
    wb.assign(2 * (size_t)nr, 0);
    int64_t wmax = 0, rmax = 0;
    for (int64_t r = 0; r < nr; ++r) {
        int64_t lo = INT64_MAX, hi = -1;
        for (int64_t u = rs[(size_t)r]; u < rs[(size_t)r + 1]; ++u) {
            lo = std::min<int64_t>(lo, span[2 * (size_t)u]);
            hi = std::max<int64_t>(hi, span[2 * (size_t)u + 1]);
        }
        if (hi < 0) lo = hi = rs[(size_t)r];  // no entries: a one-id window
        const int64_t base = lo & ~int64_t(1);  // even first id: a 16-byte aligned float2 window
        wb[2 * (size_t)r] = base;
        wb[2 * (size_t)r + 1] = hi - base + 1;
        wmax = std::max<int64_t>(wmax, hi - base + 1);
        rmax = std::max<int64_t>(rmax, (int64_t)(rs[(size_t)r + 1] - rs[(size_t)r]));
        if (wmax > kMaxTile) return GILA_OK;  // 16-bit relative ids
    }
    if (window_smem(wmax, rmax, esz) > (size_t)(kSmemCap - 4096)) return GILA_OK;
    // windows pay where they are narrow: the positions all CTAs load stay
    // below half the bytes of the 16-bit id stream (the mesh: 22 MB of
    // windows for 75 MB of ids, 0.086 ms per iteration against 0.150 plain;
    // a Barabasi-Albert graph of 10,000 vertices at k = 3, whose every range
    // needs the whole graph, about as many window bytes as id bytes: 0.039
    // against 0.030 plain)
    int64_t wsum = 0;
    for (int64_t r = 0; r < nr; ++r) wsum += wb[2 * (size_t)r + 1];
    if (g->tune.tiled < 0 && wsum * (int64_t)esz > g->nnz_khop) return GILA_OK;
    *wmax_out = wmax;
    *rmax_out = rmax;
    *fits = true;
    return GILA_OK;
}

// The block layout shared by tiles and windows: blocks (j, r) for each
// tile j's ranges rs[j], each in share storage (lane_len(L) slots per
// thread; block starts are multiples of 8 slots, 16 bytes); segments padded
// to multiples of 8 entries; segment starts within their block; ids
// rearranged into 16-bit relative ids. wb (window mode, one tile) gives each
// range's window; tiles are [j tv, (j + 1) tv). Blocks are numbered (and
// launched) costliest first, so that in a grid of several waves the CTAs
// that start last are short ones.
gila_status build_layout(gila_graph* g, size_t esz, TilePlan& P, int64_t nt, int64_t tv,
                         const std::vector<int64_t>& len,
                         const std::vector<std::vector<int32_t>>& rs,
                         const std::vector<int64_t>* wb)
{
    const int64_t n = g->n;
    const int64_t cells = n * nt;
    struct Blk {
        int32_t j, r, u0, u1;
        int64_t L, cost;
    };
    std::vector<Blk> bl;
    std::vector<int64_t> toff((size_t)cells);
    // directory for the layout kernel: tfirst (nt + 1), then each tile's
    // range bounds (nb + nt), then the block of each (tile, range) (nb)
    std::vector<int32_t> tfirst((size_t)nt + 1, 0), rstart;
    for (int64_t j = 0; j < nt; ++j) {
        tfirst[(size_t)j] = (int32_t)bl.size();
        const std::vector<int32_t>& c = rs[(size_t)j];
        rstart.insert(rstart.end(), c.begin(), c.end());
        for (size_t r = 0; r + 1 < c.size(); ++r) {
            int64_t off = 0, cost = 0;
            for (int64_t u = c[r]; u < c[r + 1]; ++u) {
                const int64_t l = len[(size_t)(j * n + u)];
                toff[(size_t)(j * n + u)] = off;
                off += (l + kStep - 1) & ~int64_t(kStep - 1);  // padded
                cost += row_cost(l);
            }
            bl.push_back({(int32_t)j, (int32_t)r, c[r], c[r + 1], off, cost});
        }
    }
    tfirst[(size_t)nt] = (int32_t)bl.size();
    const int64_t nb = (int64_t)bl.size();
    std::vector<int32_t> order((size_t)nb);
    for (int64_t b = 0; b < nb; ++b) order[(size_t)b] = (int32_t)b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return bl[(size_t)x].cost > bl[(size_t)y].cost; });
    std::vector<int64_t> blk(2 * (size_t)nb), wbb(wb ? 2 * (size_t)nb : 0);
    std::vector<int32_t> bdesc(4 * (size_t)nb), rblock((size_t)nb);
    int64_t slots = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const Blk& x = bl[(size_t)order[(size_t)b]];
        blk[2 * (size_t)b] = slots;
        blk[2 * (size_t)b + 1] = x.L;
        slots += (int64_t)kBThreads * lane_len((int32_t)x.L);
        bdesc[4 * (size_t)b] = x.u0;
        bdesc[4 * (size_t)b + 1] = x.u1;
        bdesc[4 * (size_t)b + 2] = x.j;
        bdesc[4 * (size_t)b + 3] = 0;
        rblock[(size_t)(tfirst[(size_t)x.j] + x.r)] = (int32_t)b;
        if (wb) {
            wbb[2 * (size_t)b] = (*wb)[2 * (size_t)x.r];
            wbb[2 * (size_t)b + 1] = (*wb)[2 * (size_t)x.r + 1];
        }
    }
    std::vector<int32_t> dir(tfirst);
    dir.insert(dir.end(), rstart.begin(), rstart.end());
    dir.insert(dir.end(), rblock.begin(), rblock.end());
    const int64_t tk_len = slots + kStep + 256 * 4;  // slack: the kernel's ring reads ahead
    gila_status s;
    if ((s = ensure((void**)&P.toff, &P.toff_cap, sizeof(int64_t) * (size_t)cells)) != GILA_OK)
        return s;
    if ((s = ensure((void**)&P.blk, &P.blk_cap, sizeof(int64_t) * blk.size())) != GILA_OK) return s;
    if ((s = ensure((void**)&P.bdesc, &P.bdesc_cap, sizeof(int32_t) * bdesc.size())) != GILA_OK)
        return s;
    if ((s = ensure((void**)&P.rdir, &P.rdir_cap, sizeof(int32_t) * dir.size())) != GILA_OK)
        return s;
    if ((s = ensure((void**)&P.tk, &P.tk_cap, sizeof(uint16_t) * (size_t)tk_len)) != GILA_OK)
        return s;
    if (wb) {
        if ((s = ensure((void**)&P.wtile, &P.wtile_cap, sizeof(int64_t) * wbb.size())) != GILA_OK)
            return s;
        GILA_CUDA(cudaMemcpyAsync(P.wtile, wbb.data(), sizeof(int64_t) * wbb.size(),
                                  cudaMemcpyHostToDevice, g->stream));
    } else if ((s = ensure(&P.part, &P.part_cap, 2 * esz * (size_t)cells)) != GILA_OK) {
        return s;
    }
    GILA_CUDA(cudaMemcpyAsync(P.toff, toff.data(), sizeof(int64_t) * cells, cudaMemcpyHostToDevice,
                              g->stream));
    GILA_CUDA(cudaMemcpyAsync(P.blk, blk.data(), sizeof(int64_t) * blk.size(),
                              cudaMemcpyHostToDevice, g->stream));
    GILA_CUDA(cudaMemcpyAsync(P.bdesc, bdesc.data(), sizeof(int32_t) * bdesc.size(),
                              cudaMemcpyHostToDevice, g->stream));
    GILA_CUDA(cudaMemcpyAsync(P.rdir, dir.data(), sizeof(int32_t) * dir.size(),
                              cudaMemcpyHostToDevice, g->stream));
    // every block's slots set to its padding id, then the ids ordered for
    // conflict-free gathers, or in ascending order; the slack after the
    // last block (read ahead by the kernel's ring, never used) is zeroed
    const int64_t* wdev = wb ? P.wtile : nullptr;
    GILA_CUDA(cudaMemsetAsync(P.tk + slots, 0, sizeof(uint16_t) * (size_t)(tk_len - slots),
                              g->stream));
    if (nb > 0) {
        pad_fill_kernel<<<(unsigned)std::min<int64_t>(nb, 4096), 256, 0, g->stream>>>(
            P.tk, P.blk, wdev, (int)tv, nb);
        count_launch();
        GILA_CUDA(cudaGetLastError());
    }
    const int32_t* d_tfirst = P.rdir;
    const int32_t* d_rstart = P.rdir + nt + 1;
    const int32_t* d_rblock = P.rdir + nt + 1 + nb + nt;
    const unsigned lay_blocks = (unsigned)((cells + kSpreadWarps - 1) / kSpreadWarps);
    if (g->tune.bank_spread >= 0 && esz == 8)
        block_layout_kernel<16, true><<<lay_blocks, kSpreadWarps * 32, 0, g->stream>>>(
            n, g->krow, g->kcol, (int)nt, (int)tv, wdev, P.toff, P.blk, d_tfirst, d_rstart,
            d_rblock, P.tk);
    else if (g->tune.bank_spread >= 0)
        block_layout_kernel<8, true><<<lay_blocks, kSpreadWarps * 32, 0, g->stream>>>(
            n, g->krow, g->kcol, (int)nt, (int)tv, wdev, P.toff, P.blk, d_tfirst, d_rstart,
            d_rblock, P.tk);
    else
        block_layout_kernel<16, false><<<lay_blocks, kSpreadWarps * 32, 0, g->stream>>>(
            n, g->krow, g->kcol, (int)nt, (int)tv, wdev, P.toff, P.blk, d_tfirst, d_rstart,
            d_rblock, P.tk);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    if (!wb) {
        // hubs of the adjacency for the combine kernel (synchronises)
        if ((s = plan_hubs(g, P)) != GILA_OK) return s;
    }
    // the host vectors above go out of scope
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    P.nt = (int32_t)nt;
    P.nb = (int32_t)nb;
    P.use = true;
    return GILA_OK;
}

// Decide whether the blocked path serves g for positions of `esz` bytes and
// build its layout: a window per row range (window mode), or tiles, row
// ranges, block offsets and rearranged ids.
gila_status plan_tiles(gila_graph* g, size_t esz, TilePlan& P)
{
    P.ready = true;
    P.use = false;
    P.window = false;
    const int64_t n = g->n;
    if (n == 0 || g->nnz_khop == 0 || g->tune.tiled == 0) return GILA_OK;
    // tiles for a row directory of rmax entries: positions per tile (one
    // slot for the padding's position) and the number of tiles
    int64_t tv = 0, nt = 0;
    auto geometry = [&](int64_t rmax) {
        int64_t tv_max = (kSmemCap - (rmax + 1) * 4 - 4096) / (int64_t)esz - 1;
        if (g->tune.tile_vertices > 0) tv_max = std::min<int64_t>(tv_max, g->tune.tile_vertices);
        tv_max = std::max<int64_t>(2, std::min<int64_t>(tv_max, kMaxTile) & ~int64_t(1));
        nt = (n + tv_max - 1) / tv_max;
        tv = std::min<int64_t>(tv_max, (((n + nt - 1) / nt) + 1) & ~int64_t(1));
    };
    geometry(kMaxRows);
    const int min_seg = g->tune.min_segment;  // 0: no limit
    const double avg_seg = (double)g->nnz_khop / ((double)n * (double)nt);
    {
        // window mode wherever every range's window fits shared memory (a
        // tile size set by the tuning asks for tiles instead); automatic mode
        // leaves lists below 4 10^6 entries to the plain kernel, which
        // spreads small graphs over more SMs (32 x 32 grid, FP64: 0.017 ms
        // plain, 0.105 ms in one window; triangulated 200 x 200 mesh, k = 3:
        // 0.015 against 0.021)
        if (g->tune.tile_vertices <= 0 && (g->tune.tiled > 0 || g->nnz_khop >= kBlockedMinNnz)) {
            bool fits = false;
            std::vector<int64_t> len, wb;
            std::vector<int32_t> rs;
            int64_t wmax = 0, rmax = 0;
            gila_status s = plan_window(g, esz, P, &fits, len, rs, wb, &wmax, &rmax);
            if (s != GILA_OK) return s;
            if (fits) {
                if ((s = build_layout(g, esz, P, 1, 0, len, {rs}, &wb)) != GILA_OK) return s;
                P.window = true;
                P.tv = (int32_t)wmax;
                P.rmax = (int32_t)rmax;
                return GILA_OK;
            }
        }
    }
    // automatic mode: tiles from 4 10^6 k-hop entries on (BA n = 100,000,
    // k = 2, 1.4e7 entries in segments of 36: 0.0493 ms per iteration
    // against 0.0609 plain; BA n = 333,334, k = 2, segments of 12: 0.183
    // against 0.209). FP64 follows the same rule (its tiles hold half as
    // many positions): on BA k = 3 blocked 5.14 ms vs plain 6.03 ms
    const bool tiles_pay = !(g->tune.tiled < 0 && avg_seg < min_seg);
    if (!tiles_pay || (g->tune.tiled < 0 && g->nnz_khop < kBlockedMinNnz)) return GILA_OK;
    // many rows: where 4096-row ranges alone make more blocks than the CTA
    // target, a larger directory (smaller tiles) gives fewer blocks, each
    // loading its tile once; but only for segments long enough that the
    // extra tiles add little padding (BA n = 333,334, k = 3, 323 entries a
    // segment: 0.702 -> 0.588 ms per iteration with 8192-row ranges; k = 2,
    // 12 entries: 0.148 -> 0.170 ms, so it keeps 4096)
    int64_t rmax = kMaxRows;
    const int64_t target = blocks_target(g, false);
    while (rmax < kMaxRowsTiles && (n + rmax - 1) / rmax * nt > target &&
           (double)g->nnz_khop >= 64.0 * (double)n * (double)nt) {
        rmax *= 2;
        geometry(rmax);
    }
    const int64_t cells = n * nt;
    gila_status s = ensure((void**)&P.len, &P.len_cap, sizeof(int64_t) * (size_t)cells);
    if (s != GILA_OK) return s;
    seglen_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, g->stream>>>(n, g->krow, g->kcol,
                                                                        (int)nt, (int)tv, P.len);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    std::vector<int64_t> len((size_t)cells);
    GILA_CUDA(cudaMemcpyAsync(len.data(), P.len, sizeof(int64_t) * cells, cudaMemcpyDeviceToHost,
                              g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    // each tile's row ranges: blocks of about equal cost (padded entries +
    // a per-row term), at most rmax rows each, about ctas_per_sm per SM
    std::vector<int64_t> pre((size_t)(nt * (n + 1)), 0);
    for (int64_t j = 0; j < nt; ++j) {
        int64_t* pj = pre.data() + j * (n + 1);
        for (int64_t u = 0; u < n; ++u) pj[u + 1] = pj[u] + row_cost(len[(size_t)(j * n + u)]);
    }
    // the block count: at least 5% above what the row limit alone makes,
    // so that a tile with more entries than the others (the hubs' ids) can
    // still be cut finer, and whole waves of one CTA per SM, since blocks of
    // equal cost end together (BA n = 333,334, k = 3: 574 row-limited blocks
    // against a target of 456: 1.27 ms per iteration with no room, 0.63 with
    // 631 blocks, 0.59 with 608)
    const int64_t sms = sm_count(g->device);
    const int64_t floor_blocks = (n + rmax - 1) / rmax * nt;
    const int64_t want = std::max<int64_t>(target, (floor_blocks * 21 + 19) / 20);
    const int64_t tgt = (want + sms - 1) / sms * sms;
    const std::vector<std::vector<int32_t>> rs = partition_blocks(pre, n, nt, tgt, rmax);
    if ((s = build_layout(g, esz, P, nt, tv, len, rs, nullptr)) != GILA_OK) return s;
    P.tv = (int32_t)tv;
    P.rmax = (int32_t)rmax;
    return GILA_OK;
}

bool blocked_auto_applies(int64_t n, int64_t nnz_khop, size_t esz, const gila_tuning& tune)
{
    if (n == 0 || nnz_khop == 0 || tune.tiled == 0) return tune.tiled == 1 && n > 0;
    if (tune.tiled == 1) return true;
    int64_t tv_max = kTileBudget / (int64_t)esz - 1;  // one slot for the padding's position
    if (tune.tile_vertices > 0) tv_max = std::min<int64_t>(tv_max, tune.tile_vertices);
    tv_max = std::max<int64_t>(2, std::min<int64_t>(tv_max, kMaxTile) & ~int64_t(1));
    const int64_t nt = (n + tv_max - 1) / tv_max;
    return nnz_khop >= kBlockedMinNnz &&
           (double)nnz_khop / ((double)n * (double)nt) >= (double)tune.min_segment;
}

gila_status prepare_iteration(gila_graph* g, const gila_params* prm)
{
    if (prm->precision == GILA_FP64_ORDERED || g->n == 0 || g->wt64) return GILA_OK;
    TilePlan& P = g->tplan[is_f64(prm->precision) ? 1 : 0];
    return P.ready ? GILA_OK : plan_tiles(g, is_f64(prm->precision) ? 16 : 8, P);
}

gila_status launch_blocked(gila_graph* g, const gila_params* prm, double t, const void* pos_in,
                           void* pos_out, void* disp_out, bool* handled)
{
    *handled = false;
    // repulsion weights are applied by the plain kernel only
    if (prm->precision == GILA_FP64_ORDERED || g->n == 0 || g->wt64) return GILA_OK;
    const size_t esz = is_f64(prm->precision) ? 16 : 8;
    TilePlan& P = g->tplan[esz == 16 ? 1 : 0];
    if (!P.ready) {
        gila_status s = plan_tiles(g, esz, P);
        if (s != GILA_OK) return s;
    }
    if (!P.use || ((uintptr_t)pos_in & 15) != 0) return GILA_OK;
    BlockedArgs B;
    B.tk = P.tk;
    B.toff = P.toff;
    B.blk = P.blk;
    B.bdesc = reinterpret_cast<const int4*>(P.bdesc);
    B.n = g->n;
    B.nt = P.nt;
    B.tv = P.tv;
    B.q = prm->q;
    B.pos = pos_in;
    B.part = P.part;
    B.wait_ns = g->wait_test ? kTestWaitNs : kWaitNs;
    B.skip_copy = g->wait_test ? 1 : 0;
    B.wbase = P.window ? P.wtile : nullptr;
    B.wmax = P.window ? P.tv : 0;
    B.rmax = P.rmax;
    B.row = g->row;
    B.col = g->col;
    B.d = prm->d;
    B.t = t;
    B.p = prm->p;
    B.pos_out = pos_out;
    B.disp_out = disp_out;
    // FP32 steps warp-uniform by default (measured against the divergent
    // schedule: Chung-Lu n = 250,000, k = 3, 4.88 vs 4.96 ms per launch;
    // Barabasi-Albert n = 100,000, k = 3, 0.172 vs 0.186 ms). The kernel
    // keeps both schedules: with the divergent one compiled beside it the
    // uniform schedule itself measured faster (4.88 vs 5.08 ms on Chung-Lu)
    B.uniform = g->tune.step_schedule >= 0 ? 1 : 0;
    CombineArgs C;
    C.row = g->row;
    C.col = g->col;
    C.n = g->n;
    C.nt = P.nt;
    C.d = prm->d;
    C.t = t;
    C.p = prm->p;
    C.pos_in = pos_in;
    C.part = P.part;
    C.pos_out = pos_out;
    C.disp_out = disp_out;
    C.hubs = P.hubs;
    C.nhub = P.nhub;
    C.nreg = (int32_t)((g->n * kCombineLanes + kCombineThreads - 1) / kCombineThreads);
    const int grid = P.nb;
    const size_t smem = P.window ? window_smem(P.tv, P.rmax, esz)
                                 : (size_t)(P.tv + 1) * esz + (size_t)(P.rmax + 1) * 4;
    const bool fr = (prm->p == 2 && prm->q == 1);
    const bool w = P.window;
    cudaError_t e;
    switch (prm->precision) {
    case GILA_FP64:
        e = fr ? launch_pair<double, kFR, false>(g, B, C, grid, smem, g->stream, g->device, w)
               : launch_pair<double, kGeneric, false>(g, B, C, grid, smem, g->stream, g->device, w);
        break;
    case GILA_FP32_COMPENSATED:
        e = fr ? launch_pair<float, kFR, true>(g, B, C, grid, smem, g->stream, g->device, w)
               : launch_pair<float, kGeneric, true>(g, B, C, grid, smem, g->stream, g->device, w);
        break;
    default:
        e = fr ? launch_pair<float, kFR, false>(g, B, C, grid, smem, g->stream, g->device, w)
               : launch_pair<float, kGeneric, false>(g, B, C, grid, smem, g->stream, g->device, w);
        break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "blocked_kernel");
    *handled = true;
    return GILA_OK;
}

gila_status blocked_khop_metric(gila_graph* g, const gila_params* prm, const void* pos,
                                bool* done, double* rep_total)
{
    *done = false;
    const TilePlan& P = g->tplan[0];
    if (is_f64(prm->precision) || !P.ready || !P.use || g->n == 0 || g->wt64) return GILA_OK;
    if (((uintptr_t)pos & 15) != 0) return GILA_OK;
    // the tile (or window) beside the kernel's own shared arrays; a larger
    // window leaves the term to the generic reduction
    const size_t smem = ((size_t)P.tv + 1) * sizeof(float2);
    if (smem > (size_t)kMetSmemMax) return GILA_OK;
    const int grid = P.nb;
    gila_status s = ensure((void**)&g->red, &g->red_cap, sizeof(double) * ((size_t)grid + 8));
    if (s != GILA_OK) return s;
    MetricArgs M;
    M.krow = g->krow;
    M.len = P.window ? nullptr : P.len;
    M.kcol = g->kcol;
    M.bdesc = reinterpret_cast<const int4*>(P.bdesc);
    M.wbase = P.window ? P.wtile : nullptr;
    M.n = g->n;
    M.nt = P.nt;
    M.tv = P.tv;
    M.tcap = P.tv;
    M.d = prm->d;
    M.q = prm->q;
    M.pos = reinterpret_cast<const float2*>(pos);
    M.partial = g->red;
    M.wait_ns = kWaitNs;
    static std::atomic<uint64_t> configured{0};
    const uint64_t bit = 1ull << (g->device & 63);
    if (!(configured.load() & bit)) {
        GILA_CUDA(cudaFuncSetAttribute(khop_metric_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMetSmemMax));
        configured.fetch_or(bit);
    }
    khop_metric_kernel<<<grid, kMetThreads, smem, g->stream>>>(M);
    count_launch();
    sum_in_order_kernel<<<1, 32, 0, g->stream>>>(g->red, grid, g->red + grid);
    count_launch();
    GILA_CUDA(cudaGetLastError());
    double h = 0.0;
    GILA_CUDA(cudaMemcpyAsync(&h, g->red + grid, sizeof(double), cudaMemcpyDeviceToHost,
                              g->stream));
    GILA_CUDA(cudaStreamSynchronize(g->stream));
    *rep_total = h;
    *done = true;
    return GILA_OK;
}

}  // namespace gila
