// k-hop list build (Section 4.5 of the paper: the repelling set of v is
// N_v(k), the vertices at graph distance 1..k from v).
//
// The paper rebuilds these sets every iteration by TTL-limited flooding of
// messages through Giraph supersteps. The topology never changes during a
// layout, so here they are built once, on the GPU, as a CSR of sorted ids:
//
//   tier 1  one warp per source: breadth-first expansion level by level,
//           with a shared-memory open-addressing set for de-duplication
//           and warp-aggregated appends; balls of up to kT1Cap vertices.
//   tier 2  one block per remaining source: the same expansion with a
//           global-memory bitmap per block; the sorted row comes out of a
//           scan over the bitmap.
//   Both tiers run twice (count, then fill) around an exclusive scan of
//   the counts, so the output needs no atomics and is the same every run.
//   Afterwards rows are classed by length for scheduling.
#include <algorithm>
#include <climits>
#include <mutex>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "gila_impl.h"

namespace gila {

namespace {

constexpr int kT1Cap = 512;          // ball size limit of tier 1 (source included)
constexpr int kT1HashBits = 10;
constexpr int kT1Hash = 1 << kT1HashBits;  // open-addressing slots
constexpr int kT1Warps = 8;          // warps per block
constexpr int kT2Threads = 256;

struct T1Smem {
    int32_t table[kT1Hash];
    int32_t list[kT1Cap];
};

__device__ __forceinline__ unsigned t1_hash(unsigned x)
{
    return (x * 2654435761u) >> (32 - kT1HashBits);
}

// Insert x; true if it was not present. The table holds at most
// kT1Cap + 31 < kT1Hash keys, so a free slot always exists.
__device__ __forceinline__ bool t1_insert(int32_t* table, int32_t x)
{
    unsigned h = t1_hash((unsigned)x);
    for (int probe = 0; probe < kT1Hash; ++probe) {
        int old = atomicCAS(&table[h], -1, x);
        if (old == -1) return true;
        if (old == x) return false;
        h = (h + 1) & (kT1Hash - 1);
    }
    return false;
}

// Ball of radius k around src in warp-private shared memory. Returns its
// size (src included), or -1 once it exceeds kT1Cap. Warp-uniform result.
__device__ int t1_ball(const int64_t* __restrict__ row, const int32_t* __restrict__ col, int k,
                       int32_t src, T1Smem& S, int lane)
{
    for (int i = lane; i < kT1Hash; i += 32) S.table[i] = -1;
    __syncwarp();
    if (lane == 0) {
        S.table[t1_hash((unsigned)src)] = src;
        S.list[0] = src;
    }
    __syncwarp();
    int cnt = 1, lb = 0, le = 1;
    const unsigned lt = lanemask_lt();
    for (int depth = 1; depth <= k && lb < le; ++depth) {
        for (int fb = lb; fb < le; fb += 32) {
            const int f = fb + lane;
            int64_t start = 0;
            int deg = 0;
            if (f < le) {
                const int32_t w = S.list[f];
                start = row[w];
                deg = (int)(row[w + 1] - start);
            }
            const int incl = warp_inclusive_scan(deg, lane);
            const int total = __shfl_sync(kFull, incl, 31);
            const int excl = incl - deg;
            for (int base = 0; base < total; base += 32) {
                const int e = base + lane;
                // owner lane: the number of lanes whose inclusive prefix is <= e
                int j = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    int v = __shfl_sync(kFull, incl, j + s - 1);
                    if (v <= e) j += s;
                }
                const int64_t st = __shfl_sync(kFull, start, j);
                const int ex = __shfl_sync(kFull, excl, j);
                bool ins = false;
                int32_t x = 0;
                if (e < total) {
                    x = col[st + (e - ex)];
                    ins = t1_insert(S.table, x);
                }
                const unsigned m = __ballot_sync(kFull, ins);
                const int p = cnt + __popc(m & lt);
                if (ins && p < kT1Cap) S.list[p] = x;
                cnt += __popc(m);
                if (cnt > kT1Cap) return -1;
            }
            __syncwarp();
        }
        lb = le;
        le = cnt;
    }
    return cnt;
}

__device__ void warp_bitonic_sort(int32_t* a, int P, int lane)
{
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < (P >> 1); i += 32) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const int32_t x = a[lo], y = a[hi];
                if ((x > y) == up) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kT1Warps * 32)
t1_count_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col, int k,
                int64_t* __restrict__ counts, int32_t* __restrict__ queue, int* __restrict__ qn)
{
    __shared__ T1Smem sm[kT1Warps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t v = (int64_t)blockIdx.x * kT1Warps + warp; v < n;
         v += (int64_t)gridDim.x * kT1Warps) {
        const int c = t1_ball(row, col, k, (int32_t)v, sm[warp], lane);
        if (lane == 0) {
            if (c < 0) {
                counts[v] = -1;
                queue[atomicAdd(qn, 1)] = (int32_t)v;
            } else {
                counts[v] = c - 1;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kT1Warps * 32)
t1_fill_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col, int k,
               const int64_t* __restrict__ counts, const int64_t* __restrict__ krow,
               uint32_t* __restrict__ kcol)
{
    __shared__ T1Smem sm[kT1Warps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t v = (int64_t)blockIdx.x * kT1Warps + warp; v < n;
         v += (int64_t)gridDim.x * kT1Warps) {
        if (counts[v] + 1 > kT1Cap) continue;  // warp-uniform: tier 2 owns this source
        T1Smem& S = sm[warp];
        const int c = t1_ball(row, col, k, (int32_t)v, S, lane);
        const int m = c - 1;
        int P = 1;
        while (P < m) P <<= 1;
        // the table is no longer needed: sort the ball (source excluded) in it
        for (int i = lane; i < P; i += 32) S.table[i] = (i < m) ? S.list[1 + i] : INT_MAX;
        __syncwarp();
        warp_bitonic_sort(S.table, P, lane);
        uint32_t* out = kcol + krow[v];
        for (int i = lane; i < m; i += 32) out[i] = (uint32_t)S.table[i];
        __syncwarp();
    }
}

// Tier 2: one block per source with a global bitmap and visit list.
// fill == false: counts[src] = |N_src(k)|; fill == true: sorted row at krow[src].
__global__ void __launch_bounds__(kT2Threads)
t2_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col, int k,
          const int32_t* __restrict__ queue, int nq, uint32_t* __restrict__ bitmaps,
          int32_t* __restrict__ lists, int64_t nwords, int64_t* __restrict__ counts,
          const int64_t* __restrict__ krow, uint32_t* __restrict__ kcol, int fill)
{
    __shared__ int64_t s_incl[kT2Threads];
    __shared__ int64_t s_start[kT2Threads];
    __shared__ int64_t s_deg[kT2Threads];
    __shared__ int64_t s_wt[kT2Threads / 32 + 1];
    __shared__ int s_cnt;
    const int tid = threadIdx.x;
    uint32_t* B = bitmaps + (int64_t)blockIdx.x * nwords;
    int32_t* V = lists + (int64_t)blockIdx.x * n;
    for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t src = queue[qi];
        if (tid == 0) {
            B[src >> 5] |= 1u << (src & 31);
            V[0] = src;
            s_cnt = 1;
        }
        __syncthreads();
        int64_t lb = 0, le = 1;
        for (int depth = 1; depth <= k && lb < le; ++depth) {
            for (int64_t fb = lb; fb < le; fb += kT2Threads) {
                const int64_t f = fb + tid;
                int64_t start = 0, deg = 0;
                if (f < le) {
                    const int32_t w = V[f];
                    start = row[w];
                    deg = row[w + 1] - start;
                }
                int64_t total;
                const int64_t incl = block_inclusive_scan<int64_t, kT2Threads>(deg, s_wt, &total);
                s_incl[tid] = incl;
                s_start[tid] = start;
                s_deg[tid] = deg;
                __syncthreads();
                for (int64_t base = 0; base < total; base += kT2Threads) {
                    const int64_t e = base + tid;
                    if (e < total) {
                        int lo = 0, hi = kT2Threads - 1;  // first j with incl[j] > e
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (s_incl[mid] > e) hi = mid; else lo = mid + 1;
                        }
                        const int64_t off = e - (s_incl[lo] - s_deg[lo]);
                        const int32_t x = col[s_start[lo] + off];
                        const uint32_t bit = 1u << (x & 31);
                        const uint32_t old = atomicOr(&B[x >> 5], bit);
                        if (!(old & bit)) V[atomicAdd(&s_cnt, 1)] = x;
                    }
                }
                __syncthreads();
            }
            lb = le;
            le = s_cnt;
            __syncthreads();
        }
        const int cnt = s_cnt;
        if (!fill) {
            if (tid == 0) counts[src] = cnt - 1;
        } else {
            uint32_t* out = kcol + krow[src];
            int64_t base = 0;
            for (int64_t w0 = 0; w0 < nwords; w0 += kT2Threads) {
                const int64_t wi = w0 + tid;
                uint32_t w = (wi < nwords) ? B[wi] : 0u;
                if (wi == (src >> 5)) w &= ~(1u << (src & 31));
                int64_t total;
                const int64_t incl =
                    block_inclusive_scan<int64_t, kT2Threads>((int64_t)__popc(w), s_wt, &total);
                int64_t o = base + incl - __popc(w);
                while (w) {
                    const int b = __ffs(w) - 1;
                    out[o++] = (uint32_t)(wi * 32 + b);
                    w &= w - 1;
                }
                base += total;
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += kT2Threads) B[V[i] >> 5] = 0u;
        __syncthreads();
    }
}

// Tier 2 with the visited bitmap in shared memory (graphs of up to
// kT2SmemWords * 32 vertices): the same breadth-first search as t2_kernel,
// but every visit is a shared-memory atomicOr, and the frontier slot that
// owns an edge is found without a search: each slot marks where its edges
// start in the current chunk of kT2Threads edges and an inclusive max-scan
// over the marks gives every edge its slot.
constexpr int64_t kT2SmemWords = (160 * 1024) / 4;
constexpr size_t kStoreCap = (size_t)16 << 30;  // device bytes for the stored tier-2 balls
constexpr size_t kB2Cap = (size_t)16 << 30;     // device bytes for the radius-2 balls (k = 3)

template <bool FILL>
__global__ void __launch_bounds__(kT2Threads)
t2s_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col, int k,
           const int32_t* __restrict__ queue, int nq, int32_t* __restrict__ lists,
           int64_t nwords, int64_t* __restrict__ counts, const int64_t* __restrict__ krow,
           uint32_t* __restrict__ kcol, uint32_t* __restrict__ store)
{
    extern __shared__ uint32_t B[];  // visited bitmap of the current source
    __shared__ int64_t s_first[kT2Threads];
    __shared__ int64_t s_start[kT2Threads];
    __shared__ int32_t s_mark[kT2Threads];
    __shared__ int32_t s_wmax[kT2Threads / 32];
    __shared__ int64_t s_wt[kT2Threads / 32 + 1];
    __shared__ int s_cnt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t* V = lists + (int64_t)blockIdx.x * n;
    for (int64_t i = tid; i < nwords; i += kT2Threads) B[i] = 0u;
    __syncthreads();
    for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t src = queue[qi];
        if (tid == 0) {
            B[src >> 5] |= 1u << (src & 31);
            V[0] = src;
            s_cnt = 1;
        }
        __syncthreads();
        int64_t lb = 0, le = 1;
        for (int depth = 1; depth <= k && lb < le; ++depth) {
            for (int64_t fb = lb; fb < le; fb += kT2Threads) {
                const int64_t f = fb + tid;
                int64_t start = 0, deg = 0;
                if (f < le) {
                    const int32_t w = V[f];
                    start = row[w];
                    deg = row[w + 1] - start;
                }
                int64_t total;
                const int64_t incl = block_inclusive_scan<int64_t, kT2Threads>(deg, s_wt, &total);
                const int64_t first = incl - deg;
                s_first[tid] = first;
                s_start[tid] = start;
                for (int64_t base = 0; base < total; base += kT2Threads) {
                    s_mark[tid] = -1;
                    __syncthreads();
                    // a slot marks the first position of its edges in this chunk
                    if (deg > 0) {
                        if (first >= base && first < base + kT2Threads)
                            s_mark[first - base] = tid;
                        else if (first < base && incl > base)
                            s_mark[0] = tid;  // its edges run into this chunk
                    }
                    __syncthreads();
                    // inclusive max-scan: the owner of edge base + tid
                    int32_t o = s_mark[tid];
                    for (int d = 1; d < 32; d <<= 1) {
                        const int32_t y = __shfl_up_sync(kFull, o, d);
                        if (lane >= d) o = max(o, y);
                    }
                    if (lane == 31) s_wmax[warp] = o;
                    __syncthreads();
                    for (int w = 0; w < warp; ++w) o = max(o, s_wmax[w]);
                    const int64_t e = base + tid;
                    if (e < total) {
                        const int32_t x = col[s_start[o] + (e - s_first[o])];
                        const uint32_t bit = 1u << (x & 31);
                        const uint32_t old = atomicOr(&B[x >> 5], bit);
                        if (!(old & bit)) V[atomicAdd(&s_cnt, 1)] = x;
                    }
                    __syncthreads();
                }
            }
            lb = le;
            le = s_cnt;
            __syncthreads();
        }
        const int cnt = s_cnt;
        if (!FILL) {
            if (tid == 0) counts[src] = cnt - 1;
            if (store) {  // keep the ball for the fill pass (nwords is a multiple of 4)
                uint4* dst = reinterpret_cast<uint4*>(store + (int64_t)qi * nwords);
                const uint4* b4 = reinterpret_cast<const uint4*>(B);
                for (int64_t i = tid; i < nwords / 4; i += kT2Threads) dst[i] = b4[i];
            }
        } else {
            uint32_t* out = kcol + krow[src];
            int64_t base = 0;
            for (int64_t w0 = 0; w0 < nwords; w0 += kT2Threads) {
                const int64_t wi = w0 + tid;
                uint32_t w = (wi < nwords) ? B[wi] : 0u;
                if (wi == (src >> 5)) w &= ~(1u << (src & 31));
                int64_t total;
                const int64_t incl =
                    block_inclusive_scan<int64_t, kT2Threads>((int64_t)__popc(w), s_wt, &total);
                int64_t o = base + incl - __popc(w);
                while (w) {
                    const int b = __ffs(w) - 1;
                    out[o++] = (uint32_t)(wi * 32 + b);
                    w &= w - 1;
                }
                base += total;
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt; i += kT2Threads) B[V[i] >> 5] = 0u;
        __syncthreads();
    }
}

// Radius-3 balls as unions of radius-2 balls (the count pass of k = 3 when
// most balls are large, as on power-law graphs): a vertex w is within 3 hops
// of s exactly when it is within 2 hops of s or of a neighbour of s, so
//   B3(s) = B2(s) | OR over v in N(s) of B2(v).
// ball2_kernel writes B2(v) of every vertex as a bitmap of n bits (one block
// per vertex: its own bit, its neighbours', their neighbours', by
// shared-memory atomics); ball3_or_kernel then forms B3 of each tier-2
// source by OR-ing the (deg + 1) bitmaps, kept in registers, the block's
// threads each owning a fixed slice of the words; the popcount gives the
// count, and the ball is stored for the fill (t2_fill_stored_kernel). The
// work is (2E + n) bitmaps read, n / 8 bytes each, instead of a
// breadth-first search per source whose cost grows with the edges of every
// ball of radius 2.
__global__ void __launch_bounds__(kT2Threads)
ball2_kernel(int64_t n, const int64_t* __restrict__ row, const int32_t* __restrict__ col,
             int64_t nwords, uint32_t* __restrict__ b2)
{
    extern __shared__ uint32_t B[];
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < nwords; i += kT2Threads) B[i] = 0u;
    __syncthreads();
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        if (tid == 0) atomicOr(&B[v >> 5], 1u << (v & 31));
        const int64_t vb = row[v], ve = row[v + 1];
        for (int64_t e = vb + tid; e < ve; e += kT2Threads) {
            const int32_t u = col[e];
            atomicOr(&B[u >> 5], 1u << (u & 31));
        }
        for (int64_t e = vb; e < ve; ++e) {
            const int32_t u = col[e];
            const int64_t ub = row[u], ue = row[u + 1];
            for (int64_t f = ub + tid; f < ue; f += kT2Threads) {
                const int32_t x = col[f];
                atomicOr(&B[x >> 5], 1u << (x & 31));
            }
        }
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(b2 + v * nwords);
        uint4* b4 = reinterpret_cast<uint4*>(B);
        for (int64_t i = tid; i < nwords / 4; i += kT2Threads) {
            dst[i] = b4[i];
            b4[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
    }
}

constexpr int kOrRegs = 8;  // uint4 words of the ball each thread keeps per pass

__global__ void __launch_bounds__(kT2Threads)
ball3_or_kernel(const int32_t* __restrict__ queue, int nq, const int64_t* __restrict__ row,
                const int32_t* __restrict__ col, int64_t nwords, const uint32_t* __restrict__ b2,
                int64_t* __restrict__ counts, uint32_t* __restrict__ store)
{
    __shared__ int64_t s_wt[kT2Threads / 32 + 1];
    const int tid = threadIdx.x;
    const int64_t n4 = nwords / 4;  // nwords is a multiple of 4
    for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t src = queue[qi];
        const int64_t sb = row[src], se = row[src + 1];
        int64_t cnt = 0;
        uint4* dst = reinterpret_cast<uint4*>(store + (int64_t)qi * nwords);
        for (int64_t c0 = 0; c0 < n4; c0 += (int64_t)kT2Threads * kOrRegs) {
            uint4 acc[kOrRegs];
            const uint4* own = reinterpret_cast<const uint4*>(b2 + (int64_t)src * nwords);
#pragma unroll
            for (int r = 0; r < kOrRegs; ++r) {
                const int64_t i = c0 + (int64_t)r * kT2Threads + tid;
                acc[r] = i < n4 ? own[i] : make_uint4(0u, 0u, 0u, 0u);
            }
            for (int64_t e = sb; e < se; ++e) {
                const uint4* nb = reinterpret_cast<const uint4*>(b2 + (int64_t)col[e] * nwords);
#pragma unroll
                for (int r = 0; r < kOrRegs; ++r) {
                    const int64_t i = c0 + (int64_t)r * kT2Threads + tid;
                    if (i < n4) {
                        const uint4 w = __ldg(nb + i);
                        acc[r].x |= w.x;
                        acc[r].y |= w.y;
                        acc[r].z |= w.z;
                        acc[r].w |= w.w;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kOrRegs; ++r) {
                const int64_t i = c0 + (int64_t)r * kT2Threads + tid;
                if (i < n4) {
                    dst[i] = acc[r];
                    cnt += __popc(acc[r].x) + __popc(acc[r].y) + __popc(acc[r].z) +
                           __popc(acc[r].w);
                }
            }
        }
        int64_t total;
        block_inclusive_scan<int64_t, kT2Threads>(cnt, s_wt, &total);
        if (tid == 0) counts[src] = total - 1;  // the source itself is not in its list
        __syncthreads();
    }
}

// Fill from the balls the count pass stored: each block writes the sorted
// rows of its sources straight from their bitmaps (no second search). A
// chunk of 256 words is expanded into shared memory at the offsets a block
// scan of their popcounts gives, then copied out with coalesced stores.
constexpr int kFillStage = kT2Threads * 32;  // ids a chunk of 256 words can hold

__global__ void __launch_bounds__(kT2Threads)
t2_fill_stored_kernel(const int32_t* __restrict__ queue, int nq, int64_t nwords,
                      const uint32_t* __restrict__ store, const int64_t* __restrict__ krow,
                      uint32_t* __restrict__ kcol)
{
    __shared__ int64_t s_wt[kT2Threads / 32 + 1];
    __shared__ uint32_t s_ids[kFillStage];
    const int tid = threadIdx.x;
    for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
        const int32_t src = queue[qi];
        const uint32_t* B = store + (int64_t)qi * nwords;
        uint32_t* out = kcol + krow[src];
        int64_t base = 0;
        for (int64_t w0 = 0; w0 < nwords; w0 += kT2Threads) {
            const int64_t wi = w0 + tid;
            uint32_t w = (wi < nwords) ? B[wi] : 0u;
            if (wi == (src >> 5)) w &= ~(1u << (src & 31));
            int64_t total;
            const int64_t incl =
                block_inclusive_scan<int64_t, kT2Threads>((int64_t)__popc(w), s_wt, &total);
            int o = (int)(incl - __popc(w));
            while (w) {
                const int b = __ffs(w) - 1;
                s_ids[o++] = (uint32_t)(wi * 32 + b);
                w &= w - 1;
            }
            __syncthreads();
            for (int i = tid; i < (int)total; i += kT2Threads) out[base + i] = s_ids[i];
            __syncthreads();
            base += total;
        }
    }
}

// --------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// out[i + 1] = in[0] + ... + in[i] within each tile; tile totals to bsum.
__global__ void __launch_bounds__(kScanThreads)
scan_tiles_kernel(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out,
                  int64_t* __restrict__ bsum)
{
    __shared__ int64_t wt[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int64_t total;
    const int64_t incl = block_inclusive_scan<int64_t, kScanThreads>(s, wt, &total);
    int64_t run = incl - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        run += v[i];
        if (base + i < n) out[base + i + 1] = run;
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the tile totals, in place, by one block.
__global__ void __launch_bounds__(kScanThreads)
scan_bsum_kernel(int64_t* __restrict__ bsum, int64_t nb)
{
    __shared__ int64_t wt[kScanThreads / 32 + 1];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = (i < nb) ? bsum[i] : 0;
        int64_t total;
        const int64_t incl = block_inclusive_scan<int64_t, kScanThreads>(v, wt, &total);
        if (i < nb) bsum[i] = carry + incl - v;
        carry += total;
    }
}

__global__ void scan_add_kernel(int64_t* __restrict__ out, int64_t n,
                                const int64_t* __restrict__ bsum)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) out[0] = 0;
    if (i < n) out[i + 1] += bsum[i / kScanTile];
}

// --------------------------------------------------------------- binning

constexpr int kBinThreads = 1024;

__device__ __forceinline__ int row_class(int64_t len, BinConfig c)
{
    if (len <= c.small_max) return 0;
    if (len <= c.warp_max) return 1;
    if (len <= c.block_max) return 2;
    return 3;
}

// Per-block class counts (block b covers vertices [b*1024, (b+1)*1024)).
__global__ void __launch_bounds__(kBinThreads)
bin_count_kernel(int64_t n, const int64_t* __restrict__ krow, BinConfig cfg,
                 int* __restrict__ bcount)
{
    __shared__ int cnt[4];
    if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    if (v < n) atomicAdd(&cnt[row_class(krow[v + 1] - krow[v], cfg)], 1);
    __syncthreads();
    if (threadIdx.x < 4) bcount[blockIdx.x * 4 + threadIdx.x] = cnt[threadIdx.x];
}

// Scatter vertex ids to their class lists in ascending id order.
__global__ void __launch_bounds__(kBinThreads)
bin_scatter_kernel(int64_t n, const int64_t* __restrict__ krow, BinConfig cfg,
                   const int* __restrict__ boff, int32_t* __restrict__ lists,
                   int32_t* __restrict__ giants)
{
    __shared__ int wcnt[kBinThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t v = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    const int c = (v < n) ? row_class(krow[v + 1] - krow[v], cfg) : -1;
    int rank = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned m = __ballot_sync(kFull, c == q);
        if (c == q) rank = __popc(m & lanemask_lt());
        if (lane == 0) wcnt[warp][q] = __popc(m);
    }
    __syncthreads();
    if (c >= 0) {
        int pre = 0;
        for (int w = 0; w < warp; ++w) pre += wcnt[w][c];
        const int pos = boff[blockIdx.x * 4 + c] + pre + rank;
        if (c < 3) lists[pos] = (int32_t)v; else giants[pos] = (int32_t)v;
    }
}

template <class T>
gila_status dev_alloc(T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GILA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    *p = (T*)q;
    return GILA_OK;
}

gila_status exclusive_scan(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t* bsum = nullptr;
    gila_status s = dev_alloc(&bsum, (size_t)std::max<int64_t>(nb, 1));
    if (s != GILA_OK) return s;
    if (n > 0) {
        scan_tiles_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, bsum);
        count_launch();
        scan_bsum_kernel<<<1, kScanThreads, 0, st>>>(bsum, nb);
        count_launch();
        scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, bsum);
        count_launch();
    } else {
        cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(bsum);
    if (e != cudaSuccess) return cuda_fail(e, "exclusive_scan");
    return GILA_OK;
}

// Offsets (begin, end) of the giant rows, gathered for the host.
__global__ void giant_bounds_kernel(int64_t ng, const int32_t* __restrict__ giants,
                                    const int64_t* __restrict__ krow, int64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    out[2 * i] = krow[giants[i]];
    out[2 * i + 1] = krow[giants[i] + 1];
}

gila_status build_bins(gila_graph* g)
{
    Bins& B = g->bins;
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    const int64_t nb = (n + kBinThreads - 1) / kBinThreads;
    std::vector<int> bc((size_t)nb * 4), boff((size_t)nb * 4);
    int* d_bc = nullptr;
    gila_status s = dev_alloc(&d_bc, (size_t)std::max<int64_t>(nb * 4, 4));
    if (s != GILA_OK) return s;
    if (nb > 0) {
        bin_count_kernel<<<(unsigned)nb, kBinThreads, 0, st>>>(n, g->krow, B.cfg, d_bc);
        count_launch();
        cudaMemcpyAsync(bc.data(), d_bc, sizeof(int) * nb * 4, cudaMemcpyDeviceToHost, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(d_bc); return cuda_fail(e, "bin_count"); }
    int64_t tot[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < nb; ++b)
        for (int c = 0; c < 4; ++c) tot[c] += bc[b * 4 + c];
    int64_t base[4] = {0, tot[0], tot[0] + tot[1], 0};
    for (int c = 0; c < 4; ++c) {
        int64_t run = base[c];
        for (int64_t b = 0; b < nb; ++b) {
            boff[b * 4 + c] = (int)run;
            run += bc[b * 4 + c];
        }
    }
    B.n0 = (int32_t)tot[0];
    B.n1 = (int32_t)tot[1];
    B.n2 = (int32_t)tot[2];
    B.ngiant = (int32_t)tot[3];
    const size_t nlist = (size_t)(tot[0] + tot[1] + tot[2]);
    if (nlist > B.cap_lists || !B.lists) {
        if (B.lists) cudaFree(B.lists);
        B.lists = nullptr;
        s = dev_alloc(&B.lists, std::max<size_t>(nlist, 1));
        if (s != GILA_OK) { cudaFree(d_bc); return s; }
        B.cap_lists = std::max<size_t>(nlist, 1);
    }
    int32_t* d_giants = nullptr;
    int64_t* d_gk = nullptr;
    s = dev_alloc(&d_giants, (size_t)std::max<int64_t>(tot[3], 1));
    if (s != GILA_OK) { cudaFree(d_bc); return s; }
    s = dev_alloc(&d_gk, (size_t)std::max<int64_t>(2 * tot[3], 2));
    if (s != GILA_OK) { cudaFree(d_bc); cudaFree(d_giants); return s; }
    if (nb > 0) {
        cudaMemcpyAsync(d_bc, boff.data(), sizeof(int) * nb * 4, cudaMemcpyHostToDevice, st);
        bin_scatter_kernel<<<(unsigned)nb, kBinThreads, 0, st>>>(n, g->krow, B.cfg, d_bc, B.lists,
                                                                 d_giants);
        count_launch();
    }
    // chunk table of the giant rows, built on the host
    std::vector<int32_t> giants((size_t)tot[3]);
    std::vector<int64_t> gk((size_t)tot[3] * 2);
    if (tot[3] > 0) {
        giant_bounds_kernel<<<(unsigned)((tot[3] + 255) / 256), 256, 0, st>>>(tot[3], d_giants,
                                                                             g->krow, d_gk);
        count_launch();
        cudaMemcpyAsync(giants.data(), d_giants, sizeof(int32_t) * tot[3], cudaMemcpyDeviceToHost,
                        st);
        cudaMemcpyAsync(gk.data(), d_gk, sizeof(int64_t) * 2 * tot[3], cudaMemcpyDeviceToHost, st);
    }
    e = cudaStreamSynchronize(st);
    cudaFree(d_bc);
    cudaFree(d_giants);
    cudaFree(d_gk);
    if (e != cudaSuccess) return cuda_fail(e, "giant rows");
    std::vector<Chunk> chunks;
    for (int64_t i = 0; i < tot[3]; ++i) {
        const int64_t b = gk[2 * i], en = gk[2 * i + 1];
        const int32_t first = (int32_t)chunks.size();
        const int32_t count = (int32_t)((en - b + B.cfg.chunk - 1) / B.cfg.chunk);
        for (int32_t c = 0; c < count; ++c) {
            Chunk ch;
            ch.begin = b + (int64_t)c * B.cfg.chunk;
            ch.end = std::min<int64_t>(en, ch.begin + B.cfg.chunk);
            ch.vertex = giants[i];
            ch.giant = (int32_t)i;
            ch.first = first;
            ch.count = count;
            chunks.push_back(ch);
        }
    }
    B.nchunks = (int32_t)chunks.size();
    if (chunks.size() > B.cap_chunks || !B.chunks) {
        if (B.chunks) cudaFree(B.chunks);
        if (B.partials) cudaFree(B.partials);
        B.chunks = nullptr;
        B.partials = nullptr;
        size_t cap = std::max<size_t>(chunks.size(), 1);
        s = dev_alloc(&B.chunks, cap);
        if (s != GILA_OK) return s;
        double* part = nullptr;
        s = dev_alloc(&part, cap * 4);
        if (s != GILA_OK) return s;
        B.partials = part;
        B.cap_chunks = cap;
    }
    if ((size_t)tot[3] > B.cap_giant || !B.giant_counter) {
        if (B.giant_counter) cudaFree(B.giant_counter);
        B.giant_counter = nullptr;
        size_t cap = std::max<size_t>((size_t)tot[3], 1);
        s = dev_alloc(&B.giant_counter, cap);
        if (s != GILA_OK) return s;
        B.cap_giant = cap;
    }
    if (!chunks.empty())
        GILA_CUDA(cudaMemcpyAsync(B.chunks, chunks.data(), sizeof(Chunk) * chunks.size(),
                                  cudaMemcpyHostToDevice, st));
    GILA_CUDA(cudaMemsetAsync(B.giant_counter, 0, sizeof(int32_t) * B.cap_giant, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    return GILA_OK;
}

}  // namespace

gila_status scan_exclusive_i64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st)
{
    return exclusive_scan(in, n, out, st);
}

int sm_count(int device)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
        v = 1;
    return v;
}

void free_khop(gila_graph* g)
{
    KhopScratch& s = g->ks;
    cudaFree(s.counts);
    cudaFree(s.queue);
    cudaFree(s.qn);
    cudaFree(s.bitmaps);
    cudaFree(s.lists);
    cudaFree(s.store);
    cudaFree(s.b2);
    s = KhopScratch();
    cudaFree(g->krow);
    cudaFree(g->kcol);
    g->krow = nullptr;
    g->kcol = nullptr;
    g->cap_kcol = 0;
    Bins& B = g->bins;
    cudaFree(B.lists);
    cudaFree(B.chunks);
    cudaFree(B.giant_counter);
    cudaFree(B.partials);
    BinConfig cfg = B.cfg;
    B = Bins();
    B.cfg = cfg;
    g->k_built = 0;
    g->nnz_khop = 0;
}

void release_khop_scratch(gila_graph* g)
{
    KhopScratch& s = g->ks;
    cudaFree(s.counts);
    cudaFree(s.queue);
    cudaFree(s.qn);
    cudaFree(s.bitmaps);
    cudaFree(s.lists);
    cudaFree(s.store);
    cudaFree(s.b2);
    const size_t cap = s.scratch_cap;
    const bool keep = s.keep_balls;
    s = KhopScratch();
    s.scratch_cap = cap;
    s.keep_balls = keep;
}

gila_status build_khop(gila_graph* g, int k)
{
    gila_status s = build_khop_count(g, k, nullptr);
    if (s != GILA_OK) return s;
    return build_khop_fill(g, k);
}

gila_status build_khop_count(gila_graph* g, int k, int64_t* nnz_out)
{
    gila_status s = build_khop_count_impl(g, k);
    if (s == GILA_OK && nnz_out) *nnz_out = g->ks.nnz;
    return s;
}

// Whether radius-3 balls are expected to cover a tenth of the graph or
// more, from the degree moments: a ball of radius 3 holds about
// mean(deg) kappa^2 vertices, kappa = E[deg^2] / E[deg] the mean excess
// degree (the 1M-edge Chung-Lu graph: 0.67 by this estimate, 0.18 measured;
// Barabasi-Albert n = 100,000: 0.034 and 0.024). Above that, unions of
// radius-2 bitmaps build the balls faster than a breadth-first search per
// source (Chung-Lu: 137 ms less per build); below it they do not (BA
// n = 100,000: 1.4 ms more).
bool dense_balls(const int64_t* row_dev, int64_t n, cudaStream_t st)
{
    std::vector<int64_t> row((size_t)n + 1);
    if (cudaMemcpyAsync(row.data(), row_dev, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    double s1 = 0.0, s2 = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        const double d = (double)(row[(size_t)u + 1] - row[(size_t)u]);
        s1 += d;
        s2 += d * d;
    }
    if (s1 <= 0.0) return false;
    const double kappa = s2 / s1;
    return (s1 / (double)n) * kappa * kappa >= 0.1 * (double)n;
}

gila_status build_khop_count_impl(gila_graph* g, int k)
{
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    KhopScratch& S = g->ks;
    gila_status s;
    if (!g->krow) {
        s = dev_alloc(&g->krow, (size_t)n + 1);
        if (s != GILA_OK) return s;
    }
    if (S.cap_n < (size_t)n || !S.counts) {
        cudaFree(S.counts);
        cudaFree(S.queue);
        cudaFree(S.qn);
        S.counts = nullptr; S.queue = nullptr; S.qn = nullptr;
        if ((s = dev_alloc(&S.counts, (size_t)std::max<int64_t>(n, 1))) != GILA_OK) return s;
        if ((s = dev_alloc(&S.queue, (size_t)std::max<int64_t>(n, 1))) != GILA_OK) return s;
        if ((s = dev_alloc(&S.qn, 1)) != GILA_OK) return s;
        S.cap_n = (size_t)n;
    }
    GILA_CUDA(cudaMemsetAsync(S.qn, 0, sizeof(int), st));
    const int sms = sm_count(g->device);
    const int64_t t1_blocks = std::max<int64_t>(
        1, std::min<int64_t>((n + kT1Warps - 1) / kT1Warps, (int64_t)sms * 8));
    if (n > 0) {
        t1_count_kernel<<<(unsigned)t1_blocks, kT1Warps * 32, 0, st>>>(n, g->row, g->col, k,
                                                                       S.counts, S.queue, S.qn);
        count_launch();
    }
    int nq = 0;
    GILA_CUDA(cudaMemcpyAsync(&nq, S.qn, sizeof(int), cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    // tier 2 scratch: one bitmap and one visit list per block
    const int64_t nwords = ((n + 31) / 32 + 3) & ~int64_t(3);
    int t2_blocks = 0;
    if (nq > 0) {
        const size_t per_block = (size_t)nwords * 4 + (size_t)n * 4;
        // at most 2 GiB (or the graph's own cap) of tier-2 scratch
        const size_t budget = S.scratch_cap ? S.scratch_cap : ((size_t)2 << 30);
        int64_t want = std::min<int64_t>(nq, (int64_t)sms * 4);
        want = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)(budget / per_block)));
        t2_blocks = (int)want;
        if (nwords <= kT2SmemWords) {
            // bitmaps in shared memory: only the visit lists are global scratch
            const int64_t lw = std::max<int64_t>(1, std::min<int64_t>(
                std::min<int64_t>(nq, (int64_t)sms * 4), (int64_t)(budget / ((size_t)n * 4))));
            t2_blocks = (int)lw;
            if (S.t2_blocks < t2_blocks || !S.lists) {
                cudaFree(S.lists);
                S.lists = nullptr;
                if ((s = dev_alloc(&S.lists, (size_t)n * t2_blocks)) != GILA_OK) return s;
                S.t2_blocks = t2_blocks;
            }
            const size_t smem = (size_t)nwords * 4;
            // keep every tier-2 ball for the fill pass when they fit in
            // kStoreCap bytes of device memory (else the fill searches again)
            // (the store and the radius-2 bitmaps below keep their capacity
            // across builds: freeing 8 GB took 3-5 ms, and a layout loop
            // rebuilds the lists every time)
            const size_t store_bytes = (size_t)nq * (size_t)nwords * 4;
            S.stored = false;
            if (S.keep_balls && store_bytes <= kStoreCap) {
                if (S.store_cap < store_bytes) {
                    cudaFree(S.store);
                    S.store = nullptr;
                    S.store_cap = 0;
                    void* p = nullptr;
                    if (cudaMalloc(&p, store_bytes) == cudaSuccess) {
                        S.store = (uint32_t*)p;
                        S.store_cap = store_bytes;
                    } else {
                        cudaGetLastError();
                    }
                }
                S.stored = S.store != nullptr;
            }
            uint32_t* const store = S.stored ? S.store : nullptr;
            // k = 3 with the balls stored and most sources in tier 2: the
            // balls as unions of the radius-2 balls (one n-bit bitmap per
            // vertex, at most kB2Cap bytes; given back if the fill cannot
            // allocate its lists)
            uint32_t* b2 = nullptr;
            const size_t b2_bytes = (size_t)n * (size_t)nwords * 4;
            if (k == 3 && store && nq >= n / 4 && b2_bytes <= kB2Cap &&
                dense_balls(g->row, n, st)) {
                if (S.b2_cap < b2_bytes) {
                    cudaFree(S.b2);
                    S.b2 = nullptr;
                    S.b2_cap = 0;
                    void* p = nullptr;
                    if (cudaMalloc(&p, b2_bytes) == cudaSuccess) {
                        S.b2 = (uint32_t*)p;
                        S.b2_cap = b2_bytes;
                    } else {
                        cudaGetLastError();
                    }
                }
                b2 = S.b2;
            }
            if (b2) {
                GILA_CUDA(cudaFuncSetAttribute(ball2_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
                ball2_kernel<<<(unsigned)std::min<int64_t>(n, (int64_t)sms * 8), kT2Threads, smem,
                               st>>>(n, g->row, g->col, nwords, b2);
                count_launch();
                ball3_or_kernel<<<(unsigned)std::min<int64_t>(nq, (int64_t)sms * 8), kT2Threads, 0,
                                  st>>>(S.queue, nq, g->row, g->col, nwords, b2, S.counts,
                                        store);
                count_launch();
                cudaError_t e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return cuda_fail(e, "radius-3 balls");
            } else {
                GILA_CUDA(cudaFuncSetAttribute(t2s_kernel<false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));
                t2s_kernel<false><<<t2_blocks, kT2Threads, smem, st>>>(
                    n, g->row, g->col, k, S.queue, nq, S.lists, nwords, S.counts, nullptr,
                    nullptr, store);
                count_launch();
            }
        } else if (S.t2_blocks < t2_blocks || S.bitmap_words != nwords || !S.bitmaps) {
            cudaFree(S.bitmaps);
            cudaFree(S.lists);
            S.bitmaps = nullptr; S.lists = nullptr;
            if ((s = dev_alloc(&S.bitmaps, (size_t)nwords * t2_blocks)) != GILA_OK) return s;
            if ((s = dev_alloc(&S.lists, (size_t)n * t2_blocks)) != GILA_OK) return s;
            GILA_CUDA(cudaMemsetAsync(S.bitmaps, 0, sizeof(uint32_t) * nwords * t2_blocks, st));
            S.t2_blocks = t2_blocks;
            S.bitmap_words = nwords;
        }
        if (nwords > kT2SmemWords) {
            t2_kernel<<<t2_blocks, kT2Threads, 0, st>>>(n, g->row, g->col, k, S.queue, nq,
                                                        S.bitmaps, S.lists, nwords, S.counts,
                                                        nullptr, nullptr, 0);
            count_launch();
        }
    }
    s = exclusive_scan(S.counts, n, g->krow, st);
    if (s != GILA_OK) return s;
    int64_t nnz = 0;
    GILA_CUDA(cudaMemcpyAsync(&nnz, g->krow + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    S.counted_k = k;
    S.nnz = nnz;
    S.nq = nq;
    S.t2_used = t2_blocks;
    S.t1_blocks = t1_blocks;
    S.nwords = nwords;
    return GILA_OK;
}

gila_status build_khop_fill(gila_graph* g, int k)
{
    const int64_t n = g->n;
    cudaStream_t st = g->stream;
    KhopScratch& S = g->ks;
    if (S.counted_k != k) return fail(GILA_ESTATE, "k-hop lists not counted for this k");
    gila_status s;
    const int64_t nnz = S.nnz, t1_blocks = S.t1_blocks, nwords = S.nwords;
    const int nq = S.nq, t2_blocks = S.t2_used;
    const int sms = sm_count(g->device);
    S.counted_k = 0;
    if ((size_t)nnz > g->cap_kcol || !g->kcol) {
        cudaFree(g->kcol);
        g->kcol = nullptr;
        g->cap_kcol = 0;
        // 4 spare entries: the blocked path's window mode reads kcol in
        // 16-byte steps that may end up to 12 bytes past the last row
        s = dev_alloc(&g->kcol, (size_t)nnz + 4);
        if (s != GILA_OK && S.b2) {
            // the radius-2 bitmaps held for the next build give way to the lists
            cudaFree(S.b2);
            S.b2 = nullptr;
            S.b2_cap = 0;
            cudaGetLastError();
            s = dev_alloc(&g->kcol, (size_t)nnz + 4);
        }
        if (s != GILA_OK) return s;
        g->cap_kcol = (size_t)nnz;
    }
    if (n > 0) {
        t1_fill_kernel<<<(unsigned)t1_blocks, kT1Warps * 32, 0, st>>>(n, g->row, g->col, k,
                                                                      S.counts, g->krow, g->kcol);
        count_launch();
    }
    if (nq > 0 && nwords <= kT2SmemWords && S.stored) {
        t2_fill_stored_kernel<<<(unsigned)std::min<int64_t>(nq, (int64_t)sms * 8), kT2Threads, 0,
                                st>>>(S.queue, nq, nwords, S.store, g->krow, g->kcol);
        count_launch();
    } else if (nq > 0 && nwords <= kT2SmemWords) {
        const size_t smem = (size_t)nwords * 4;
        GILA_CUDA(cudaFuncSetAttribute(t2s_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        t2s_kernel<true><<<t2_blocks, kT2Threads, smem, st>>>(
            n, g->row, g->col, k, S.queue, nq, S.lists, nwords, S.counts, g->krow, g->kcol,
            nullptr);
        count_launch();
    } else if (nq > 0) {
        t2_kernel<<<t2_blocks, kT2Threads, 0, st>>>(n, g->row, g->col, k, S.queue, nq, S.bitmaps,
                                                    S.lists, nwords, S.counts, g->krow, g->kcol, 1);
        count_launch();
    }
    (void)sms;
    GILA_CUDA(cudaGetLastError());
    GILA_CUDA(cudaStreamSynchronize(st));
    S.stored = false;  // the stored balls served their one fill (the capacity stays)
    s = build_bins(g);
    if (s != GILA_OK) return s;
    g->nnz_khop = nnz;
    g->k_built = k;
    return GILA_OK;
}

// ------------------------------------------------------------------------
// k-hop list sizes without any allocation (gila_khop_count_noalloc).
//
// The same two counting kernels as above, with their scratch (overflow
// queue, tier-2 bitmaps and visit lists, counters) in one file-scope device
// array instead of cudaMalloc'd buffers. The array exists on every device
// that loads the library, from load until exit.

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 18;           // 262,144 vertices
constexpr int kNoAllocT2Blocks = 4;                           // tier-2 blocks
constexpr int64_t kNoAllocWords = kNoAllocMaxN / 32;          // bitmap words per block

struct NoAllocScratch {
    int32_t queue[kNoAllocMaxN];                        // 1 MiB
    uint32_t bitmaps[kNoAllocT2Blocks * kNoAllocWords]; // 128 KiB, all zero between sources
    int32_t lists[kNoAllocT2Blocks * kNoAllocMaxN];     // 4 MiB
    int64_t total;
    int qn;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

__global__ void __launch_bounds__(1024)
sum_counts_kernel(const int64_t* __restrict__ counts, int64_t n, int64_t* __restrict__ out)
{
    __shared__ int64_t wt[1024 / 32 + 1];
    int64_t s = 0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s += counts[i];
    int64_t total;
    block_inclusive_scan<int64_t, 1024>(s, wt, &total);
    if (threadIdx.x == 0) *out = total;
}

// Device address of the scratch array, looked up once per device with that
// device current (host code cannot use the array's name as an address).
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_ptr[kMaxDevices] = {};

gila_status noalloc_scratch(int device, NoAllocScratch** out)
{
    if (device < 0 || device >= kMaxDevices) return fail(GILA_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[device] = (NoAllocScratch*)p;
    }
    *out = g_noalloc_ptr[device];
    return GILA_OK;
}

}  // namespace
}  // namespace gila

extern "C" gila_status gila_khop_count_noalloc(int64_t n, const int64_t* row_ptr_dev,
                                               const int32_t* col_idx_dev, int32_t k,
                                               int64_t* counts_dev, int64_t* total_host,
                                               void* cuda_stream)
{
    using namespace gila;
    if (n < 0) return fail(GILA_EINVAL, "n must be >= 0");
    if (n > kNoAllocMaxN)
        return fail(GILA_EINVAL, "gila_khop_count_noalloc: n = " + std::to_string(n) +
                                     " exceeds the fixed scratch limit of " +
                                     std::to_string(kNoAllocMaxN) + " vertices");
    if (k < 1 || k > 64) return fail(GILA_EINVAL, "k must be in [1, 64]");
    if (n > 0 && (!row_ptr_dev || !col_idx_dev || !counts_dev))
        return fail(GILA_EINVAL, "device array is NULL");
    int device = 0;
    GILA_CUDA(cudaGetDevice(&device));
    NoAllocScratch* S = nullptr;
    gila_status s = noalloc_scratch(device, &S);
    if (s != GILA_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the queue counter and the bitmaps must start at zero; the rest is
    // written before it is read
    GILA_CUDA(cudaMemsetAsync(&S->qn, 0, sizeof(int), st));
    GILA_CUDA(cudaMemsetAsync(S->bitmaps, 0, sizeof(S->bitmaps), st));
    GILA_CUDA(cudaMemsetAsync(&S->total, 0, sizeof(int64_t), st));
    int nq = 0;
    if (n > 0) {
        const int sms = sm_count(device);
        const int64_t t1_blocks = std::max<int64_t>(
            1, std::min<int64_t>((n + kT1Warps - 1) / kT1Warps, (int64_t)sms * 8));
        t1_count_kernel<<<(unsigned)t1_blocks, kT1Warps * 32, 0, st>>>(
            n, row_ptr_dev, col_idx_dev, k, counts_dev, S->queue, &S->qn);
        count_launch();
        GILA_CUDA(cudaGetLastError());
        GILA_CUDA(cudaMemcpyAsync(&nq, &S->qn, sizeof(int), cudaMemcpyDeviceToHost, st));
        GILA_CUDA(cudaStreamSynchronize(st));
    }
    if (nq > 0) {
        const int64_t nwords = ((n + 31) / 32 + 3) & ~int64_t(3);
        const int blocks = std::min(nq, kNoAllocT2Blocks);
        t2_kernel<<<blocks, kT2Threads, 0, st>>>(n, row_ptr_dev, col_idx_dev, k, S->queue, nq,
                                                 S->bitmaps, S->lists, nwords, counts_dev, nullptr,
                                                 nullptr, 0);
        count_launch();
        GILA_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        sum_counts_kernel<<<1, 1024, 0, st>>>(counts_dev, n, &S->total);
        count_launch();
        GILA_CUDA(cudaGetLastError());
    }
    int64_t total = 0;
    GILA_CUDA(cudaMemcpyAsync(&total, &S->total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GILA_CUDA(cudaStreamSynchronize(st));
    if (total_host) *total_host = total;
    return GILA_OK;
}
