// k_batched.cu -- many independent streams (each B1 or Polar, each with its
// own mu, sigma, key, counter and length) in one persistent launch.
//
// The paper amortises the cost of a call by returning whole arrays (Sec. 3)
// and buffers the variable output of its vector Polar kernel (Sec. 4,
// RANN3/RANN3B).  Here thousands of uneven streams share one grid:
//   k_batched_prep (one CTA) validates the descriptors, turns each stream into
//     work items and scans them, together with the Polar streams' tile status
//     slots, into the workspace.  A B1 stream's items are its tiles; a Polar
//     stream's are its expected number of tiles (primary items) plus one
//     overflow item, placed after every stream's primary items, that runs
//     whatever tiles the stream still needs, one after another;
//   k_batched (persistent, one global work counter) pulls items in order,
//     finds the stream in the item table the prep kernel wrote (one load) and
//     runs a B1 tile or Polar tiles (look-back within the stream's own status
//     words).
// Items are handed out in increasing order, a CTA starts an item as soon as
// it has claimed it, and a stream's tiles are claimed in increasing tile
// order, so a Polar tile only waits on tiles already owned by running CTAs.
// (Claiming the next item while the current one runs was measured: it lets
// a claimed tile start up to a tile later than its successors, which then
// wait in their look-back, and the whole batch ran twice as long.)  A Polar tile taken after its stream is
// complete publishes a prefix of nitems and returns, so that any later tile's
// look-back still ends.
#include <algorithm>
#include <climits>

#include "tiles.cuh"

namespace nrng {

// ------------------------------------------------------------ configs -----
// (threads per CTA, Philox blocks per thread per tile).  A Polar tile stages
// at most 64 accepted points per warp and row, 8 bytes each, in shared
// memory, plus 8 bytes of accept ballots per (row, warp): 33.6 KB for 128 x 16
// or 256 x 8.  Long tiles of 128 threads are the default: the per-item claim
// and the per-tile scan and look-back are spread over more candidates, which
// measured 9% faster on the 4096-stream workload than 128 x 8 although shared
// memory then holds six CTAs per SM (512-thread tiles were never faster).
static const BatchedConfig kConfigs[] = {
    {128, 16}, {128, 12}, {128, 8}, {256, 8}, {128, 4}, {256, 4},
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

int batched_config_count() { return kNumConfigs; }
BatchedConfig batched_config(int id) { return kConfigs[id]; }
int batched_default_config() { return 0; }

// B1 tiles per B1 work item: a claim (an atomic and three dependent loads
// while the CTA waits) is amortised over two tiles.  Measured on the
// 4096-stream workload: 2 is 3.5% faster than 1 on all-B1 batches; 4 loses
// on mixed batches to the longer tail of the last items.
constexpr int kB1TilesPerItem = 2;

__host__ __device__ inline int64_t b1_items(int64_t n, int64_t tile_blocks)
{
    const int64_t nblocks = (n + 3) / 4;
    return (nblocks + tile_blocks - 1) / tile_blocks;
}

// A Polar stream's primary tiles: the expected number of tiles its pairs
// need at acceptance pi/4, ceil(nitems / (cand 0.7854)), at least one and at
// most the tile budget.  They are its work items in the stream-ordered part
// of the item space; whatever the stream still needs after them (a fraction
// of a tile, at most a few) its overflow item takes, in the part of the item
// space claimed after every primary tile.  Items for the whole tile budget
// would spend the budget's margin (the 12-sigma excess and the extra tile)
// on fully drawn tiles that are not needed, most of the work of a short
// stream.
__host__ __device__ inline int64_t polar_primary_tiles(int64_t n, int64_t cand)
{
    const int64_t nitems = (n + 1) / 2;
    const int64_t t = (nitems * 10000 + cand * 7854 - 1) / (cand * 7854);
    const int64_t budget = polar_tiles_for(n, cand);
    return t < 1 ? 1 : (t > budget ? budget : t);
}

// Items and status slots of one stream; -1 items marks an invalid descriptor,
// -2 a counter that would pass 2^64.
__host__ __device__ inline void stream_items(const nrng_stream_desc_t &d, int threads, int bpt,
                                             int64_t &items, int64_t &slots)
{
    items = 0;
    slots = 0;
    const bool finite = (d.mu - d.mu == 0.0f) && (d.sigma - d.sigma == 0.0f);
    if (d.n < 0 || d.offset < 0 || !finite || !(d.sigma >= 0.0f) || d.reserved != 0 ||
        (d.method != NRNG_B1 && d.method != NRNG_POLAR) || (d.method == NRNG_POLAR && d.n > kPolarMaxN)) {
        items = -1;
        return;
    }
    if (d.n == 0) return;
    const int64_t tile_blocks = (int64_t)threads * bpt;
    if (d.method == NRNG_B1) {
        items = b1_items(d.n, tile_blocks * kB1TilesPerItem);
        const uint64_t blocks = (uint64_t)((d.n + 3) / 4);
        if (d.counter > ULLONG_MAX - (blocks - 1)) items = -2;
    } else {
        slots = polar_tiles_for(d.n, 2 * tile_blocks);
        items = polar_primary_tiles(d.n, 2 * tile_blocks);
        const uint64_t blocks = (uint64_t)(slots * tile_blocks);
        if (d.counter > ULLONG_MAX - (blocks - 1)) items = -2;
    }
    // the item table keeps a stream's item index in 32 bits
    if (items > INT_MAX) {
        items = -1;
        slots = 0;
    }
}

size_t batched_workspace_bytes(const nrng_stream_desc_t *h_desc, int32_t k)
{
    // Sized for the configuration with the most status slots, so that any
    // configuration (autotuned or pinned) fits the same workspace.
    // Each configuration needs its tile status words and its item table
    // (one 8-byte entry per primary item).
    size_t best = 0;
    for (int c = 0; c < kNumConfigs; ++c) {
        int64_t slots = 0, items = 0;
        for (int32_t j = 0; j < k; ++j) {
            int64_t it, sl;
            stream_items(h_desc[j], kConfigs[c].threads, kConfigs[c].blocks_per_thread, it, sl);
            if (it > 0) {
                slots += sl;
                items += it;
            }
        }
        best = std::max(best, (size_t)(slots + items));
    }
    return batched_layout(k).tile_status + best * 8;
}

// ------------------------------------------------------------ prep --------
// One CTA: every thread takes a contiguous run of descriptors, sums their
// items and status slots, and one block-wide exclusive scan places them.
// Then every thread writes the item table entries of its streams: entry i
// of the table is (stream, item of the stream) for primary item i, so that a
// claim finds its stream with one load.  The table follows the tile status
// words; its byte offset goes to the header (aux[2]).
constexpr int kPrepThreads = 1024;

__global__ void __launch_bounds__(kPrepThreads)
k_batched_prep(BatchedParams bp, int threads, int bpt)
{
    __shared__ long long s_wi[kPrepThreads / 32], s_ws[kPrepThreads / 32];
    __shared__ long long s_tot_items, s_tot_slots;
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const int32_t per = (bp.k + kPrepThreads - 1) / kPrepThreads;
    const int32_t j0 = tid * per;
    const int32_t j1 = (j0 + per < bp.k) ? j0 + per : bp.k;
    // Each descriptor's items and slots are computed once (64-bit divisions
    // and a square root) and kept for the second pass when they fit here.
    constexpr int kKeep = 4;
    int64_t keep_items[kKeep], keep_slots[kKeep];
    long long mi = 0, ms = 0;
#pragma unroll
    for (int q = 0; q < kKeep; ++q) {   // unrolled: the kept values stay in registers
        keep_items[q] = keep_slots[q] = 0;
        const int32_t j = j0 + q;
        if (j >= j1) continue;
        int64_t items, slots;
        stream_items(bp.desc[j], threads, bpt, items, slots);
        if (items < 0) {
            atomicMax(&s_bad, items == -2 ? kStatusOverflow : kStatusInvalid);
            items = 0;
            slots = 0;
        }
        keep_items[q] = items;
        keep_slots[q] = slots;
        mi += items;
        ms += slots;
    }
    for (int32_t j = j0 + kKeep; j < j1; ++j) {   // more than 4 descriptors a thread
        int64_t items, slots;
        stream_items(bp.desc[j], threads, bpt, items, slots);
        if (items < 0) {
            atomicMax(&s_bad, items == -2 ? kStatusOverflow : kStatusInvalid);
            items = 0;
            slots = 0;
        }
        mi += items;
        ms += slots;
    }
    long long ii = mi, is = ms;   // inclusive within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(0xFFFFFFFFu, ii, o);
        const long long b = __shfl_up_sync(0xFFFFFFFFu, is, o);
        if (lane >= o) { ii += a; is += b; }
    }
    if (lane == 31) { s_wi[warp] = ii; s_ws[warp] = is; }
    __syncthreads();
    if (warp == 0) {
        long long wi = s_wi[lane], ws = s_ws[lane];
        const long long wi0 = wi, ws0 = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long a = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            const long long b = __shfl_up_sync(0xFFFFFFFFu, ws, o);
            if (lane >= o) { wi += a; ws += b; }
        }
        s_wi[lane] = wi - wi0;   // exclusive warp offsets
        s_ws[lane] = ws - ws0;
        if (lane == 31) {
            s_tot_items = wi;
            s_tot_slots = ws;
        }
    }
    __syncthreads();
    // the item table after the status words of every Polar stream; written
    // only when the workspace holds it (else the status word reports it)
    const size_t table_off = batched_layout(bp.k).tile_status + (size_t)s_tot_slots * 8;
    const bool table_fits = table_off + (size_t)s_tot_items * 8 <= bp.ws_bytes;
    int2 *table = reinterpret_cast<int2 *>(reinterpret_cast<char *>(bp.hdr) + table_off);
    long long ci = s_wi[warp] + ii - mi, cs = s_ws[warp] + is - ms;   // exclusive for this thread
#pragma unroll
    for (int q = 0; q < kKeep; ++q) {
        const int32_t j = j0 + q;
        if (j >= j1) continue;
        bp.item_prefix[j] = ci;
        bp.slot_base[j] = cs;
        if (table_fits)
            for (int64_t it = 0; it < keep_items[q]; ++it) table[ci + it] = make_int2(j, (int)it);
        ci += keep_items[q];
        cs += keep_slots[q];
    }
    for (int32_t j = j0 + kKeep; j < j1; ++j) {
        int64_t items, slots;
        stream_items(bp.desc[j], threads, bpt, items, slots);
        if (items < 0) { items = 0; slots = 0; }
        bp.item_prefix[j] = ci;
        bp.slot_base[j] = cs;
        if (table_fits)
            for (int64_t it = 0; it < items; ++it) table[ci + it] = make_int2(j, (int)it);
        ci += items;
        cs += slots;
    }
    if (tid == kPrepThreads - 1) {
        bp.item_prefix[bp.k] = ci;
        int bad = s_bad;
        if (!bad && !table_fits) bad = kStatusWorkspace;
        if (bad) {
            bp.hdr->status = bad;
            bp.hdr->done = 1;
            bp.hdr->aux[0] = 0;
            bp.hdr->aux[1] = 0;
        } else {
            // primary items, then one overflow item per stream
            bp.hdr->aux[0] = (unsigned long long)ci + (unsigned long long)bp.k;
            bp.hdr->aux[1] = (unsigned long long)ci;
            bp.hdr->aux[2] = (unsigned long long)table_off;
        }
    }
}

// ------------------------------------------------------------ main --------
// The batched kernel carries both tile bodies (B1 and Polar) and per-stream
// round keys, so it is compiled for at most 1024 resident threads per SM, and
// for fewer where its tile's shared memory (with the 1 KB the runtime keeps
// per CTA) admits fewer CTAs: the register budget follows from the smaller
// count (128 x 16: six CTAs, up to 80 registers a thread; 128 x 12: eight, 64).
template <int THREADS, int BPT, int MODE>
struct BatchedOccupancy {
    static constexpr int kSmemBlocks = (228 * 1024) / ((int)sizeof(RejSmem<THREADS / 32, BPT>) + 1024 + 256);
    static constexpr int kThreadBlocks = 1024 / THREADS;
    static constexpr int kMin = kSmemBlocks < kThreadBlocks ? kSmemBlocks : kThreadBlocks;
    static constexpr int kMinBlocks = kMin > 0 ? kMin : 1;
};

// One unit of work of a CTA: tiles [t0, t1) of stream `stream` (-1: none left).
struct BatchedWork {
    nrng_stream_desc_t d;
    long long t0, t1;
    int stream;
    int skip;       // Polar stream complete when claimed
    int overflow;   // the stream's overflow item
};

// Claims the next item and resolves it to a stream and tile range (one
// thread).  Items [0, primary) are the streams' primary items in stream
// order, found in the item table with one load; item primary + j is stream
// j's overflow item.
__device__ __forceinline__ void batched_claim(const BatchedParams &bp, const int2 *table,
                                              unsigned long long total_items, unsigned long long primary, int cand,
                                              BatchedWork &w)
{
    // The error flag and the claim are issued together (one round trip, not
    // two); an item claimed after an error is dropped unprocessed.  This flag
    // is set only on an error, and every look-back gives up as soon as the
    // status word is set, so a dropped item never holds up a successor.
    // (Stream completion is the per-stream flag, read after the claim.)
    const int failed = ld_relaxed_s32(&bp.hdr->done);
    const unsigned long long it = atomicAdd(&bp.hdr->tile_counter, 1ull);
    const long long item = (failed == 0 && it < total_items) ? (long long)it : -1;
    if (item < 0) {
        w.stream = -1;
        return;
    }
    int j;
    if ((unsigned long long)item < primary) {
        const int2 e = table[item];
        j = e.x;
        w.t0 = e.y;
        w.t1 = w.t0 + 1;
        w.overflow = 0;
    } else {
        j = (int)(item - (long long)primary);
        w.t0 = bp.item_prefix[j + 1] - bp.item_prefix[j];   // the stream's primary tiles
        w.overflow = 1;
    }
    // The descriptor and the stream's completion flag are loaded together
    // (B1 streams' flags stay 0).
    const int stream_done = ld_relaxed_s32(bp.stream_done + j);
    w.d = bp.desc[j];
    const bool polar = (w.d.method == NRNG_POLAR);
    if (w.overflow) w.t1 = polar ? polar_tiles_for(w.d.n, cand) : w.t0;   // B1 has no overflow
    w.skip = polar ? stream_done : 0;
    w.stream = j;
}

template <int THREADS, int BPT, int MODE, typename T>
__global__ void __launch_bounds__(THREADS, (BatchedOccupancy<THREADS, BPT, MODE>::kMinBlocks))
k_batched(BatchedParams bp)
{
    constexpr int kCand = 2 * THREADS * BPT;
    __shared__ RejSmem<THREADS / 32, BPT> sm;
    __shared__ BatchedWork s_work;
    __shared__ int s_done;

    const unsigned long long total_items = bp.hdr->aux[0];
    const unsigned long long primary = bp.hdr->aux[1];
    const int2 *table = reinterpret_cast<const int2 *>(reinterpret_cast<const char *>(bp.hdr) + bp.hdr->aux[2]);
    char *out_base = static_cast<char *>(bp.out);
    for (;;) {
        if (threadIdx.x == 0) batched_claim(bp, table, total_items, primary, kCand, s_work);
        __syncthreads();
        const int j = s_work.stream;
        if (j < 0) break;
        const nrng_stream_desc_t d = s_work.d;
        const long long t0 = s_work.t0, t1 = s_work.t1;
        const bool overflow = s_work.overflow != 0;
        int skip = s_work.skip;
        RoundKeys rk;
        make_round_keys(d.key, rk);
        T *out = reinterpret_cast<T *>(out_base) + d.offset;
        bool ok = true;
        if (d.method == NRNG_B1) {
            const RadiusCoef cf = radius_coef(d.mu, d.sigma);
            // the item's blocks [first, first + span): carry-free when the low
            // counter word does not wrap over them
            constexpr int64_t kSpan = (int64_t)THREADS * BPT * kB1TilesPerItem;
            const uint64_t first = d.counter + (uint64_t)(t0 * kSpan);
            const bool carry_free = (uint64_t)(uint32_t)first + (uint64_t)kSpan <= (uint64_t(1) << 32);
            if (overflow) {
                // B1 streams have no overflow tiles
            } else if (((uintptr_t)out % (4 * sizeof(T))) == 0) {
                if (carry_free)
                    for (int q = 0; q < kB1TilesPerItem; ++q)
                        b1_tile<THREADS, BPT, MODE, T, true, false>(out, d.n, cf, kSinCos1024, rk, d.counter,
                                                                    t0 * kB1TilesPerItem + q);
                else
                    for (int q = 0; q < kB1TilesPerItem; ++q)
                        b1_tile<THREADS, BPT, MODE, T, true, true>(out, d.n, cf, kSinCos1024, rk, d.counter,
                                                                   t0 * kB1TilesPerItem + q);
            } else {
                for (int q = 0; q < kB1TilesPerItem; ++q)
                    b1_tile<THREADS, BPT, MODE, T, false, true>(out, d.n, cf, kSinCos1024, rk, d.counter,
                                                                t0 * kB1TilesPerItem + q);
            }
        } else if (!(overflow && skip)) {
            const RadiusCoef cf = radius_coef(d.mu, d.sigma);
            PolarStream ps;
            ps.n = d.n;
            ps.nitems = (d.n + 1) / 2;
            ps.counter = d.counter;
            ps.status = bp.tile_status + bp.slot_base[j];
            ps.tiles_max = polar_tiles_for(d.n, kCand);
            ps.done = bp.stream_done + j;
            ps.next_counter = nullptr;
            ps.pair_cand = nullptr;
            ps.silent_tile = -1;
            const bool aligned = ((uintptr_t)out % (2 * sizeof(T))) == 0;
            for (long long t = t0; t < t1; ++t) {
                if (t > t0) {
                    // overflow item: stop once the stream is complete
                    if (threadIdx.x == 0) s_done = ld_relaxed_s32(ps.done);
                    __syncthreads();
                    skip = s_done;
                    __syncthreads();
                    if (skip) break;
                }
                if (skip) {
                    // Stream complete: every later tile's prefix is >= nitems.
                    if (threadIdx.x == 0) st_relaxed(ps.status + t, kFlagPrefix | (unsigned long long)ps.nitems);
                } else if (aligned) {
                    ok = reject_tile<PolarPolicy<MODE>, THREADS / 32, BPT, T, true, true>(sm, out, ps, rk, cf, t, bp.hdr,
                                                                                         bp.spin_limit_ns);
                } else {
                    ok = reject_tile<PolarPolicy<MODE>, THREADS / 32, BPT, T, false, true>(sm, out, ps, rk, cf, t, bp.hdr,
                                                                                          bp.spin_limit_ns);
                }
                __syncthreads();
                if (!ok) break;
            }
        }
        __syncthreads();
        if (!ok) break;
    }
}

template <int THREADS, int BPT, int MODE, typename T>
static cudaError_t batched_main(const BatchedParams &bp, cudaStream_t s)
{
    static std::atomic<int> slot{0};
    int occ = 0;
    const cudaError_t e = cached_occupancy(slot, k_batched<THREADS, BPT, MODE, T>, THREADS, occ);
    if (e != cudaSuccess) return e;
    k_batched<THREADS, BPT, MODE, T><<<sm_count() * occ, THREADS, 0, s>>>(bp);
    return cudaGetLastError();
}

template <int MODE, typename T>
static cudaError_t batched_config_dispatch(const BatchedParams &bp, int config, cudaStream_t s)
{
    switch (config) {
    case 0: return batched_main<128, 16, MODE, T>(bp, s);
    case 1: return batched_main<128, 12, MODE, T>(bp, s);
    case 2: return batched_main<128, 8, MODE, T>(bp, s);
    case 3: return batched_main<256, 8, MODE, T>(bp, s);
    case 4: return batched_main<128, 4, MODE, T>(bp, s);
    default: return batched_main<256, 4, MODE, T>(bp, s);
    }
}

template <int MODE>
static cudaError_t batched_dtype_dispatch(const BatchedParams &bp, int dtype, int config, cudaStream_t s)
{
    switch (dtype) {
    case NRNG_F32: return batched_config_dispatch<MODE, float>(bp, config, s);
    case NRNG_BF16: return batched_config_dispatch<MODE, __nv_bfloat16>(bp, config, s);
    default: return batched_config_dispatch<MODE, __half>(bp, config, s);
    }
}

cudaError_t launch_batched(void *out, const nrng_stream_desc_t *desc, int32_t k, int dtype, int mode,
                           void *ws, size_t ws_bytes, int config, cudaStream_t s)
{
    const BatchedLayout L = batched_layout(k);
    char *w = static_cast<char *>(ws);
    BatchedParams bp;
    bp.out = out;
    bp.desc = desc;
    bp.k = k;
    bp.hdr = reinterpret_cast<WsHeader *>(w);
    bp.item_prefix = reinterpret_cast<int64_t *>(w + L.item_prefix);
    bp.slot_base = reinterpret_cast<int64_t *>(w + L.slot_base);
    bp.stream_done = reinterpret_cast<int *>(w + L.stream_done);
    bp.tile_status = reinterpret_cast<unsigned long long *>(w + L.tile_status);
    bp.ws_bytes = ws_bytes;
    bp.spin_limit_ns = spin_limit_ns();
    cudaError_t e = cudaMemsetAsync(ws, 0, ws_bytes, s);
    if (e != cudaSuccess) return e;
    const BatchedConfig c = kConfigs[config];
    k_batched_prep<<<1, kPrepThreads, 0, s>>>(bp, c.threads, c.blocks_per_thread);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode == kModeFast) return batched_dtype_dispatch<kModeFast>(bp, dtype, config, s);
    return batched_dtype_dispatch<kModeAccurate>(bp, dtype, config, s);
}

}  // namespace nrng
