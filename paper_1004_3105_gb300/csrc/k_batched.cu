// k_batched.cu -- many independent streams (each B1 or Polar, each with its
// own mu, sigma, key, counter and length) in one persistent launch.
//
// The paper amortises the cost of a call by returning whole arrays (Sec. 3)
// and buffers the variable output of its vector Polar kernel (Sec. 4,
// RANN3/RANN3B).  Here thousands of uneven streams share one grid:
//   k_batched_count, k_batched_scan and k_batched_fill validate the
//     descriptors, turn each stream into work items and write the item table
//     (a thread, one CTA and a warp per stream): first every B1 stream's items
//     (runs of its tiles), then every Polar stream's primary items (its
//     expected number of tiles, one item each), then one overflow item per
//     Polar stream that runs whatever tiles the stream still needs, one after
//     another.  Entry i of the table names the stream and the tile of item i.
//   k_batched (persistent, one global work counter) claims items in order,
//     finds the stream in the item table (one load) and runs B1 tiles or
//     Polar tiles (look-back within the stream's own status words).
// The B1 items come first so that a CTA stages the sine/cosine table of the
// accurate B1 path in shared memory once, in the space its Polar tiles use
// later, and the batch ends on short Polar tiles rather than long B1 items.
// The order of the items changes no output: every stream's values depend on
// its own key, counter and length alone.
// Items are handed out in increasing order and a stream's tiles are claimed
// in increasing tile order.  A CTA claims its next item ahead only while the
// rest of its current item waits on nothing (a B1 item, or a Polar tile's
// copy-out once its prefix is known), so a Polar tile only waits on tiles
// owned by CTAs that are running them or about to start them.  (Claiming
// ahead at the start of a Polar tile was measured: it lets a claimed tile
// start up to a tile later than its successors, which then wait in their
// look-back, and the whole batch ran twice as long.)  A Polar tile taken
// after its stream is complete publishes a prefix of nitems and returns, so
// that any later tile's look-back still ends.
#include <algorithm>
#include <climits>

#include "tiles.cuh"

namespace nrng {

// ------------------------------------------------------------ configs -----
// (threads per CTA, Philox blocks per thread per tile).  A Polar tile stages
// at most 64 accepted points per warp and row, 8 bytes each, in shared
// memory, plus 8 bytes of accept ballots per (row, warp): 37.5 KB for 128 x 18,
// 33.6 KB for 128 x 16 or 256 x 8.  Long tiles of 128 threads are the default:
// the per-item claim and the per-tile scan and look-back are spread over more
// candidates (128 x 16 measured 9% faster on the 4096-stream workload than
// 128 x 8, and 128 x 18, the longest tile at which six CTAs still fit per SM,
// 1.4% faster than 128 x 16; 512-thread tiles were never faster).
static const BatchedConfig kConfigs[] = {
    {128, 18}, {128, 16}, {128, 12}, {128, 8}, {256, 8}, {128, 4}, {256, 4},
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

int batched_config_count() { return kNumConfigs; }
BatchedConfig batched_config(int id) { return kConfigs[id]; }
int batched_default_config() { return 0; }

// B1 tiles per B1 work item: a claim (an atomic and two dependent loads while
// the CTA waits) is amortised over four tiles.  The B1 items all precede the
// Polar items, so their length does not lengthen the tail of the batch.
constexpr int kB1TilesPerItem = 4;

__host__ __device__ inline int64_t b1_items(int64_t n, int64_t tile_blocks)
{
    const int64_t nblocks = (n + 3) / 4;
    return (nblocks + tile_blocks - 1) / tile_blocks;
}

// A Polar stream's primary tiles: the expected number of tiles its pairs
// need at acceptance pi/4, ceil(nitems / (cand 0.7854)), at least one and at
// most the tile budget, one work item each; whatever the stream still needs
// after them (a fraction of a tile, at most a few) its overflow item takes,
// in the part of the item space claimed after every primary item.  Items for the whole tile budget
// would spend the budget's margin (the 12-sigma excess and the extra tile)
// on fully drawn tiles that are not needed, most of the work of a short
// stream.
__host__ __device__ inline int64_t polar_primary_tiles(int64_t n, int64_t cand, int64_t budget)
{
    const int64_t nitems = (n + 1) / 2;
    const int64_t t = (nitems * 10000 + cand * 7854 - 1) / (cand * 7854);
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
        items = polar_primary_tiles(d.n, 2 * tile_blocks, slots);
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
    // Sized for the configuration with the most status slots and items, so
    // that any configuration (autotuned or pinned) fits the same workspace.
    // Each configuration needs its tile status words and its item table: one
    // 8-byte entry per item, a Polar stream's overflow item included.
    size_t best = 0;
    for (int c = 0; c < kNumConfigs; ++c) {
        int64_t slots = 0, items = 0;
        for (int32_t j = 0; j < k; ++j) {
            int64_t it, sl;
            stream_items(h_desc[j], kConfigs[c].threads, kConfigs[c].blocks_per_thread, it, sl);
            if (it > 0) {
                slots += sl;
                items += it + (h_desc[j].method == NRNG_POLAR ? 1 : 0);
            }
        }
        best = std::max(best, (size_t)(slots + items));
    }
    return batched_layout(k).tile_status + best * 8;
}

// ------------------------------------------------------------ prep --------
// Three small kernels turn the descriptors into the item table:
//   k_batched_count (a thread per stream) validates each descriptor and
//     records its items and status slots (the 64-bit divisions and square
//     roots, spread over the grid);
//   k_batched_scan (one CTA) scans the four counts (B1 items, Polar primary
//     items, Polar overflow items, slots) in stream order and places every
//     stream: its status words, its first table entry, its overflow entry;
//   k_batched_fill (a warp per stream) writes the stream's table entries:
//     (stream, tile) for a B1 or primary item, (stream, -1 - primary tiles)
//     for an overflow item.
// The table follows the tile status words; its byte offset goes to the
// header (aux[2]).  aux[3] collects the worst descriptor error.
constexpr int kCountThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kFillThreads = 256;
constexpr int kScanSums = 4;   // B1 items, Polar primary items, overflow items, slots

__global__ void __launch_bounds__(kCountThreads)
k_batched_count(BatchedParams bp, int threads, int bpt)
{
    const int32_t j = blockIdx.x * kCountThreads + threadIdx.x;
    if (j >= bp.k) return;
    const nrng_stream_desc_t d = bp.desc[j];
    int64_t items, slots;
    stream_items(d, threads, bpt, items, slots);
    BatchedCount c{0, 0, 0};
    if (items < 0) {
        atomicMax(&bp.hdr->aux[3], (unsigned long long)(items == -2 ? kStatusOverflow : kStatusInvalid));
    } else if (items > 0) {
        c.items = (int32_t)items;
        c.polar = d.method == NRNG_POLAR ? 1 : 0;
        c.slots = slots;
    }
    bp.counts[j] = c;
}

// One 16-byte load of a stream's record.
__device__ __forceinline__ BatchedCount load_count(const BatchedCount *p)
{
    const int4 r = *reinterpret_cast<const int4 *>(p);
    return BatchedCount{r.x, r.y, (int64_t)(((uint64_t)(uint32_t)r.w << 32) | (uint32_t)r.z)};
}

__device__ __forceinline__ void scan_terms(const BatchedCount &c, long long (&v)[kScanSums])
{
    v[0] = c.polar ? 0 : c.items;
    v[1] = c.polar ? c.items : 0;
    v[2] = c.polar;
    v[3] = c.slots;
}

__global__ void __launch_bounds__(kScanThreads)
k_batched_scan(BatchedParams bp)
{
    __shared__ long long s_w[kScanSums][kScanThreads / 32];
    __shared__ long long s_tot[kScanSums];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t per = (bp.k + kScanThreads - 1) / kScanThreads;
    const int32_t j0 = tid * per;
    const int32_t j1 = (j0 + per < bp.k) ? j0 + per : bp.k;
    // The thread's first kKeep records are loaded at once and kept in
    // registers for the second pass.
    constexpr int kKeep = 4;
    BatchedCount keep[kKeep];
#pragma unroll
    for (int r = 0; r < kKeep; ++r) keep[r] = (j0 + r < j1) ? load_count(bp.counts + j0 + r) : BatchedCount{0, 0, 0};
    long long m[kScanSums] = {0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < kKeep; ++r) {
        long long v[kScanSums];
        scan_terms(keep[r], v);
#pragma unroll
        for (int q = 0; q < kScanSums; ++q) m[q] += v[q];
    }
    for (int32_t j = j0 + kKeep; j < j1; ++j) {
        long long v[kScanSums];
        scan_terms(load_count(bp.counts + j), v);
#pragma unroll
        for (int q = 0; q < kScanSums; ++q) m[q] += v[q];
    }
    long long inc[kScanSums];   // inclusive within the warp
#pragma unroll
    for (int q = 0; q < kScanSums; ++q) inc[q] = m[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < kScanSums; ++q) {
            const long long a = __shfl_up_sync(0xFFFFFFFFu, inc[q], o);
            if (lane >= o) inc[q] += a;
        }
    }
    if (lane == 31)
#pragma unroll
        for (int q = 0; q < kScanSums; ++q) s_w[q][warp] = inc[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kScanSums; ++q) {
            long long v = s_w[q][lane];
            const long long v0 = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long a = __shfl_up_sync(0xFFFFFFFFu, v, o);
                if (lane >= o) v += a;
            }
            s_w[q][lane] = v - v0;   // exclusive warp offsets
            if (lane == 31) s_tot[q] = v;
        }
    }
    __syncthreads();
    const long long n_b1 = s_tot[0], n_pp = s_tot[1], n_po = s_tot[2], n_slots = s_tot[3];
    long long x[kScanSums];   // exclusive for this thread
#pragma unroll
    for (int q = 0; q < kScanSums; ++q) x[q] = s_w[q][warp] + inc[q] - m[q];
    long long ib = x[0], ip = n_b1 + x[1], io = n_b1 + n_pp + x[2], cs = x[3];
    auto place = [&](int32_t j, const BatchedCount &c) {
        bp.slot_base[j] = cs;
        *reinterpret_cast<longlong2 *>(bp.item_base + 2 * j) = make_longlong2(c.polar ? ip : ib, c.polar ? io : -1);
        if (c.polar) {
            ip += c.items;
            io += 1;
        } else {
            ib += c.items;
        }
        cs += c.slots;
    };
#pragma unroll
    for (int r = 0; r < kKeep; ++r)
        if (j0 + r < j1) place(j0 + r, keep[r]);
    for (int32_t j = j0 + kKeep; j < j1; ++j) place(j, load_count(bp.counts + j));
    if (tid == kScanThreads - 1) {
        bp.slot_base[bp.k] = cs;
        // the item table after the status words of every Polar stream,
        // written only when the workspace holds it
        const long long n_items = n_b1 + n_pp + n_po;
        const size_t table_off = batched_layout(bp.k).tile_status + (size_t)n_slots * 8;
        const bool table_fits = table_off + (size_t)n_items * 8 <= bp.ws_bytes;
        int bad = (int)bp.hdr->aux[3];
        if (!bad && !table_fits) bad = kStatusWorkspace;
        if (bad) {
            bp.hdr->status = bad;
            bp.hdr->done = 1;
            bp.hdr->aux[0] = 0;
            bp.hdr->aux[1] = 0;
        } else {
            bp.hdr->aux[0] = (unsigned long long)n_items;
            bp.hdr->aux[1] = (unsigned long long)n_b1;
            bp.hdr->aux[2] = (unsigned long long)table_off;
        }
    }
}

__global__ void __launch_bounds__(kFillThreads)
k_batched_fill(BatchedParams bp)
{
    const int32_t j = blockIdx.x * (kFillThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= bp.k || bp.hdr->done) return;   // done: a descriptor or workspace error
    int2 *table = reinterpret_cast<int2 *>(reinterpret_cast<char *>(bp.hdr) + bp.hdr->aux[2]);
    const BatchedCount c = load_count(bp.counts + j);
    const longlong2 base = *reinterpret_cast<const longlong2 *>(bp.item_base + 2 * j);
    for (int32_t it = lane; it < c.items; it += 32) table[base.x + it] = make_int2(j, it);
    if (c.polar && lane == 0) table[base.y] = make_int2(j, -1 - c.items);
}

// ------------------------------------------------------------ main --------
// The batched kernel carries both tile bodies (B1 and Polar) and per-stream
// round keys, so it is compiled for at most 1024 resident threads per SM, and
// for fewer where its tile's shared memory (with the 1 KB the runtime keeps
// per CTA) admits fewer CTAs: the register budget follows from the smaller
// count (128 x 16: six CTAs, up to 80 registers a thread; 128 x 12: eight, 64).
// Shared memory of a batched CTA: a Polar tile's staging, or the sine/cosine
// table of the accurate B1 path (16 KB) while the CTA runs B1 items.
template <int THREADS, int BPT>
union BatchedSmem {
    RejSmem<THREADS / 32, BPT> rej;
    float4 tab[1024];
};

template <int THREADS, int BPT, int MODE>
struct BatchedOccupancy {
    static constexpr int kSmemBlocks = (228 * 1024) / ((int)sizeof(BatchedSmem<THREADS, BPT>) + 1024 + 256);
    static constexpr int kThreadBlocks = 1024 / THREADS;
    static constexpr int kMin = kSmemBlocks < kThreadBlocks ? kSmemBlocks : kThreadBlocks;
    static constexpr int kMinBlocks = kMin > 0 ? kMin : 1;
};

// One unit of work of a CTA: tiles [t0, t1) of stream `stream` (-1: none left).
struct BatchedWork {
    nrng_stream_desc_t d;
    long long t0, t1;
    long long slot0, tiles_max;   // a Polar stream's first status word and tile budget
    int stream;
    int skip;       // Polar stream complete when claimed
    int overflow;   // the stream's overflow item
};

// Resolves claimed item `it` to a stream and tile range (one thread): one
// load of the item table names the stream and the tile, or, for an overflow
// item, the stream's primary tiles (the first tile it may need); an overflow
// item runs up to the stream's tile budget.
__device__ __forceinline__ void batched_resolve(const BatchedParams &bp, const int2 *table, unsigned long long it,
                                                unsigned long long total_items, BatchedWork &w)
{
    // An item claimed after an error is dropped unprocessed.  The error flag
    // is set only on an error, and every look-back gives up as soon as the
    // status word is set, so a dropped item never holds up a successor.
    // (Stream completion is the per-stream flag, read below.)
    const int failed = ld_relaxed_s32(&bp.hdr->done);
    if (failed != 0 || it >= total_items) {
        w.stream = -1;
        return;
    }
    const int2 e = table[it];
    const int j = e.x;
    // The descriptor, the stream's status words and its completion flag are
    // loaded together (B1 streams have no status words, their flags stay 0).
    const int stream_done = ld_relaxed_s32(bp.stream_done + j);
    w.d = bp.desc[j];
    w.slot0 = bp.slot_base[j];
    w.tiles_max = bp.slot_base[j + 1] - w.slot0;
    w.overflow = e.y < 0;
    w.t0 = w.overflow ? -1 - (long long)e.y : e.y;
    w.t1 = w.overflow ? w.tiles_max : w.t0 + 1;
    w.skip = (w.d.method == NRNG_POLAR) ? stream_done : 0;
    w.stream = j;
}

// A Polar primary item claims the next item once its tile's prefix is known:
// only the copy-out is left, so the claimed item starts a copy-out later than
// a claim made after the item (an overflow item, which may run more tiles,
// does not claim ahead).
struct ClaimAhead {
    unsigned long long *counter;
    unsigned long long *ahead;
    bool on;
    __device__ __forceinline__ void operator()() const
    {
        if (on) *ahead = atomicAdd(counter, 1ull);
    }
};

template <int THREADS, int BPT, int MODE, typename T>
__global__ void __launch_bounds__(THREADS, (BatchedOccupancy<THREADS, BPT, MODE>::kMinBlocks))
k_batched(BatchedParams bp)
{
    constexpr int kCand = 2 * THREADS * BPT;
    __shared__ BatchedSmem<THREADS, BPT> sm;
    __shared__ BatchedWork s_work;
    __shared__ int s_done;

    const unsigned long long total_items = bp.hdr->aux[0];
    const unsigned long long b1_items_end = bp.hdr->aux[1];
    const int2 *table = reinterpret_cast<const int2 *>(reinterpret_cast<const char *>(bp.hdr) + bp.hdr->aux[2]);
    char *out_base = static_cast<char *>(bp.out);
    bool tab_staged = false;   // sm.tab holds the sine/cosine table
    // Thread 0's claims: the current item, and the next one when it was
    // claimed ahead (kNone: not yet).  A CTA claims ahead while it runs a B1
    // item, which waits on nothing, or once its Polar tile has its prefix
    // (only the copy-out left, which waits on nothing), so a claimed-ahead
    // Polar tile is started after a bounded time and its successors'
    // look-backs still end.  During a B1 item it claims ahead only far from
    // the end of the B1 items, so that hardly any Polar tile waits a whole B1
    // item (a late tile holds up its stream's later tiles).
    constexpr unsigned long long kNone = ~0ull;
    unsigned long long cur = kNone, ahead = kNone;
    for (;;) {
        if (threadIdx.x == 0) {
            cur = (ahead != kNone) ? ahead : atomicAdd(&bp.hdr->tile_counter, 1ull);
            ahead = kNone;
            batched_resolve(bp, table, cur, total_items, s_work);
        }
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
            if (threadIdx.x == 0 && cur + 2 * (unsigned long long)gridDim.x < b1_items_end)
                ahead = atomicAdd(&bp.hdr->tile_counter, 1ull);   // read at the next claim
            const float4 *tab = kSinCos1024;
            if (MODE == kModeAccurate) {
                if (!tab_staged) {   // the CTA's first B1 item (the items before were none or Polar)
                    for (int i = threadIdx.x; i < 1024; i += THREADS) sm.tab[i] = kSinCos1024[i];
                    __syncthreads();
                    tab_staged = true;
                }
                tab = sm.tab;
            }
            if (((uintptr_t)out % (4 * sizeof(T))) == 0) {
                if (carry_free)
                    for (int q = 0; q < kB1TilesPerItem; ++q)
                        b1_tile<THREADS, BPT, MODE, T, true, false>(out, d.n, cf, tab, rk, d.counter,
                                                                    t0 * kB1TilesPerItem + q);
                else
                    for (int q = 0; q < kB1TilesPerItem; ++q)
                        b1_tile<THREADS, BPT, MODE, T, true, true>(out, d.n, cf, tab, rk, d.counter,
                                                                   t0 * kB1TilesPerItem + q);
            } else {
                for (int q = 0; q < kB1TilesPerItem; ++q)
                    b1_tile<THREADS, BPT, MODE, T, false, true>(out, d.n, cf, tab, rk, d.counter,
                                                                t0 * kB1TilesPerItem + q);
            }
        } else if (!(overflow && skip)) {
            tab_staged = false;   // the Polar tile's staging overwrites the table
            const RadiusCoef cf = radius_coef(d.mu, d.sigma);
            PolarStream ps;
            ps.n = d.n;
            ps.nitems = (d.n + 1) / 2;
            ps.counter = d.counter;
            ps.status = bp.tile_status + s_work.slot0;
            ps.tiles_max = s_work.tiles_max;
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
                    ok = reject_tile<PolarPolicy<MODE>, THREADS / 32, BPT, T, true, true, RoundKeys, false>(
                        sm.rej, out, ps, rk, cf, t, bp.hdr, bp.spin_limit_ns, 0, ClaimAhead{&bp.hdr->tile_counter, &ahead, !overflow});
                } else {
                    ok = reject_tile<PolarPolicy<MODE>, THREADS / 32, BPT, T, false, true, RoundKeys, false>(
                        sm.rej, out, ps, rk, cf, t, bp.hdr, bp.spin_limit_ns, 0, ClaimAhead{&bp.hdr->tile_counter, &ahead, !overflow});
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
    case 0: return batched_main<128, 18, MODE, T>(bp, s);
    case 1: return batched_main<128, 16, MODE, T>(bp, s);
    case 2: return batched_main<128, 12, MODE, T>(bp, s);
    case 3: return batched_main<128, 8, MODE, T>(bp, s);
    case 4: return batched_main<256, 8, MODE, T>(bp, s);
    case 5: return batched_main<128, 4, MODE, T>(bp, s);
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
    bp.slot_base = reinterpret_cast<int64_t *>(w + L.slot_base);
    bp.stream_done = reinterpret_cast<int *>(w + L.stream_done);
    bp.counts = reinterpret_cast<BatchedCount *>(w + L.counts);
    bp.item_base = reinterpret_cast<int64_t *>(w + L.item_base);
    bp.tile_status = reinterpret_cast<unsigned long long *>(w + L.tile_status);
    bp.ws_bytes = ws_bytes;
    bp.spin_limit_ns = spin_limit_ns();
    cudaError_t e = cudaMemsetAsync(ws, 0, ws_bytes, s);
    if (e != cudaSuccess) return e;
    const BatchedConfig c = kConfigs[config];
    if (k > 0) {
        k_batched_count<<<(k + kCountThreads - 1) / kCountThreads, kCountThreads, 0, s>>>(bp, c.threads,
                                                                                        c.blocks_per_thread);
        k_batched_scan<<<1, kScanThreads, 0, s>>>(bp);
        k_batched_fill<<<(k + kFillThreads / 32 - 1) / (kFillThreads / 32), kFillThreads, 0, s>>>(bp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode == kModeFast) return batched_dtype_dispatch<kModeFast>(bp, dtype, config, s);
    return batched_dtype_dispatch<kModeAccurate>(bp, dtype, config, s);
}

}  // namespace nrng
