// k_batched.cu -- many independent streams (each B1 or Polar, each with its
// own mu, sigma, key, counter and length) in one persistent launch.
//
// The paper amortises the cost of a call by returning whole arrays (Sec. 3)
// and buffers the variable output of its vector Polar kernel (Sec. 4,
// RANN3/RANN3B).  Here thousands of uneven streams share one grid:
//   k_batched_count and k_batched_fill validate the descriptors, turn each
//     stream into work items (a thread per stream, one scan across the grid)
//     and write the item table (a warp per stream): first every B1 stream's items
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
// Two small kernels turn the descriptors into the item table:
//   k_batched_count (a thread per stream, kSetupThreads streams a CTA)
//     validates each descriptor, counts its B1 items, Polar primary items,
//     Polar overflow items (one per Polar stream with work) and status slots,
//     and places the stream with one scan over all streams: a block scan, then
//     a decoupled look-back across CTAs (taken in ticket order, so a CTA only
//     waits on CTAs that have started) for each of the four counts and for a
//     fifth, the descriptor errors.  The CTA with the last ticket has the
//     totals and writes them to the header;
//   k_batched_fill (a warp per stream) writes the stream's table entries:
//     (stream, tile) for a B1 or primary item, (stream, -1 - primary tiles)
//     for an overflow item.  The table follows the tile status words: B1
//     items, then Polar primary items, then overflow items.
// Header: aux[0] items, aux[1] B1 items, aux[2] the table's byte offset,
// aux[3] the first overflow item, aux[4] the setup's CTA tickets.
constexpr int kFillThreads = 256;

// One 16-byte load of a stream's record.
__device__ __forceinline__ BatchedCount load_count(const BatchedCount *p)
{
    const int4 r = *reinterpret_cast<const int4 *>(p);
    return BatchedCount{r.x, r.y, (int64_t)(((uint64_t)(uint32_t)r.w << 32) | (uint32_t)r.z)};
}

// Decoupled look-back of warp 0 over NQ quantities at once: status word
// status[q stride + c] holds CTA c's quantity q (aggregate or inclusive
// prefix flag, as the tiles' status words).  Each poll reads 32 predecessors'
// NQ words (one per lane and quantity) and each quantity sums back to its own
// nearest prefix, so one round trip serves all NQ.  Returns false when the
// wait ran out (the error is recorded); every wait is bounded as in
// lookback_warp.
template <int NQ>
__device__ __forceinline__ bool lookback_multi(unsigned long long *status, long long stride, long long c,
                                               const long long (&agg)[NQ], long long (&excl)[NQ], WsHeader *hdr,
                                               unsigned long long limit_ns)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q) excl[q] = 0;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            st_relaxed(status + q * stride + c, (c == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)agg[q]);
    if (c == 0) return true;
    bool found[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) found[q] = false;
    long long base = c - 1;
    unsigned long long t0 = 0;
    unsigned polls = 0;
    for (;;) {
        const long long idx = base - lane;
        unsigned long long w[NQ];
        unsigned pre[NQ], nr[NQ], win[NQ];
        bool wait = false;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            w[q] = (idx >= 0 && !found[q]) ? ld_relaxed(status + q * stride + idx) : kFlagPrefix;
            pre[q] = __ballot_sync(0xFFFFFFFFu, (unsigned)(w[q] >> 62) == 2u);
            nr[q] = __ballot_sync(0xFFFFFFFFu, (unsigned)(w[q] >> 62) == 0u);
            const unsigned lm = pre[q] & (0u - pre[q]);   // the nearest prefix (pre[q] != 0 once found)
            win[q] = pre[q] ? (lm | (lm - 1u)) : 0xFFFFFFFFu;
            wait |= (nr[q] & win[q]) != 0u;
        }
        if (wait) {
            if (polls == 0) t0 = global_timer_ns();
            ++polls;
            bool give_up = (polls >= (1u << 24)) || (global_timer_ns() - t0 > limit_ns) ||
                           (ld_relaxed_s32(&hdr->status) != 0);
            give_up = __shfl_sync(0xFFFFFFFFu, give_up, 0);
            if (give_up) {
                if (lane == 0 && ld_relaxed_s32(&hdr->status) == 0) raise_error(hdr, kStatusTimeout);
                return false;
            }
            __nanosleep(polls < 4 ? 64u : 256u);
            continue;
        }
        bool all = true;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (found[q]) continue;
            long long v = ((win[q] >> lane) & 1u) ? (long long)(w[q] & kValueMask) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            excl[q] += v;
            found[q] = pre[q] != 0u;
            all = all && found[q];
        }
        if (all) break;
        base -= 32;
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) st_relaxed(status + q * stride + c, kFlagPrefix | (unsigned long long)(excl[q] + agg[q]));
    return true;
}

// Errors, summed over the streams without carrying between the two kinds:
// counter overflows in the high half, invalid descriptors in the low half.
constexpr int kErrShift = 31;

__global__ void __launch_bounds__(kSetupThreads)
k_batched_count(BatchedParams bp, int threads, int bpt)
{
    __shared__ long long s_w[kSetupSums][kSetupThreads / 32];
    __shared__ long long s_x[kSetupSums];
    __shared__ long long s_ticket;
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_ticket = (long long)atomicAdd(&bp.hdr->aux[4], 1ull);
    __syncthreads();
    const long long c = s_ticket;
    const long long nctas = ((long long)bp.k + kSetupThreads - 1) / kSetupThreads;
    const long long jl = c * kSetupThreads + tid;
    const int32_t j = (int32_t)jl;
    long long v[kSetupSums] = {0, 0, 0, 0, 0};
    BatchedCount rec{0, 0, 0};
    if (jl < bp.k) {
        const nrng_stream_desc_t d = bp.desc[j];
        int64_t items, slots;
        stream_items(d, threads, bpt, items, slots);
        if (items < 0) {
            v[4] = (items == -2) ? (1ll << kErrShift) : 1ll;
        } else if (items > 0) {
            rec.items = (int32_t)items;
            rec.polar = d.method == NRNG_POLAR ? 1 : 0;
            rec.slots = slots;
            v[rec.polar ? 1 : 0] = items;
            v[2] = rec.polar;
            v[3] = slots;
        }
        bp.counts[j] = rec;
    }
    // block scan of the five quantities
    long long inc[kSetupSums];
#pragma unroll
    for (int q = 0; q < kSetupSums; ++q) inc[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < kSetupSums; ++q) {
            const long long y = __shfl_up_sync(0xFFFFFFFFu, inc[q], o);
            if (lane >= o) inc[q] += y;
        }
    }
    if (lane == 31)
#pragma unroll
        for (int q = 0; q < kSetupSums; ++q) s_w[q][warp] = inc[q];
    __syncthreads();
    if (warp == 0) {
        long long agg[kSetupSums];
#pragma unroll
        for (int q = 0; q < kSetupSums; ++q) {
            long long y = lane < kSetupThreads / 32 ? s_w[q][lane] : 0;
            const long long y0 = y;
#pragma unroll
            for (int o = 1; o < kSetupThreads / 32; o <<= 1) {
                const long long z = __shfl_up_sync(0xFFFFFFFFu, y, o);
                if (lane >= o) y += z;
            }
            if (lane < kSetupThreads / 32) s_w[q][lane] = y - y0;   // exclusive warp offsets
            agg[q] = __shfl_sync(0xFFFFFFFFu, y, kSetupThreads / 32 - 1);
        }
        // the CTA's place among all streams: one look-back for the five
        long long P[kSetupSums];
        const bool ok = lookback_multi<kSetupSums>(bp.setup_status, nctas, c, agg, P, bp.hdr, bp.spin_limit_ns);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < kSetupSums; ++q) s_x[q] = P[q];
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    if (!s_ok) return;   // a look-back gave up: the error is recorded
    long long x[kSetupSums];   // exclusive prefixes of this thread's stream
#pragma unroll
    for (int q = 0; q < kSetupSums; ++q) x[q] = s_x[q] + s_w[q][warp] + inc[q] - v[q];
    if (jl < bp.k) {
        bp.slot_base[j] = x[3];
        *reinterpret_cast<longlong2 *>(bp.item_base + 2 * jl) =
            make_longlong2(rec.polar ? x[1] : x[0], rec.polar ? x[2] : -1);
    }
    if (c == nctas - 1 && tid == kSetupThreads - 1) {
        // the last CTA's last thread: the totals
        const long long n_b1 = x[0] + v[0], n_pp = x[1] + v[1], n_po = x[2] + v[2], n_slots = x[3] + v[3];
        const long long errs = x[4] + v[4];
        const long long n_items = n_b1 + n_pp + n_po;
        bp.slot_base[bp.k] = n_slots;
        // the item table after the status words of every Polar stream,
        // written only when the workspace holds it
        const size_t table_off = batched_layout(bp.k).tile_status + (size_t)n_slots * 8;
        const bool table_fits = table_off + (size_t)n_items * 8 <= bp.ws_bytes;
        int bad = (errs >> kErrShift) ? kStatusOverflow : (errs ? kStatusInvalid : 0);
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
            bp.hdr->aux[3] = (unsigned long long)(n_b1 + n_pp);
        }
    }
}

__global__ void __launch_bounds__(kFillThreads)
k_batched_fill(BatchedParams bp)
{
    const int32_t j = blockIdx.x * (kFillThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= bp.k || bp.hdr->done) return;   // done: a descriptor, workspace or setup error
    int2 *table = reinterpret_cast<int2 *>(reinterpret_cast<char *>(bp.hdr) + bp.hdr->aux[2]);
    const BatchedCount c = load_count(bp.counts + j);
    const longlong2 base = *reinterpret_cast<const longlong2 *>(bp.item_base + 2 * j);
    // B1 items first, then the Polar primary items, then the overflow items
    const long long first = c.polar ? (long long)bp.hdr->aux[1] + base.x : base.x;
    for (int32_t it = lane; it < c.items; it += 32) table[first + it] = make_int2(j, it);
    if (c.polar && lane == 0) table[(long long)bp.hdr->aux[3] + base.y] = make_int2(j, -1 - c.items);
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
            // candidates a short stream's tile 0 is expected to need,
            // nitems / (pi/4): its first draw takes the warps that reach into
            // them (whole warps, so mostly with room to spare), and a second
            // draw the rest when they fall short
            const int limit0 = (ps.nitems < kCand) ? (int)((float)ps.nitems * 1.2732395f) : kCand;
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
                        sm.rej, out, ps, rk, cf, t, bp.hdr, bp.spin_limit_ns, 0,
                        ClaimAhead{&bp.hdr->tile_counter, &ahead, !overflow}, t == 0 ? limit0 : kCand);
                } else {
                    ok = reject_tile<PolarPolicy<MODE>, THREADS / 32, BPT, T, false, true, RoundKeys, false>(
                        sm.rej, out, ps, rk, cf, t, bp.hdr, bp.spin_limit_ns, 0,
                        ClaimAhead{&bp.hdr->tile_counter, &ahead, !overflow}, t == 0 ? limit0 : kCand);
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
    bp.setup_status = reinterpret_cast<unsigned long long *>(w + L.setup_status);
    bp.tile_status = reinterpret_cast<unsigned long long *>(w + L.tile_status);
    bp.ws_bytes = ws_bytes;
    bp.spin_limit_ns = spin_limit_ns();
    cudaError_t e = cudaMemsetAsync(ws, 0, ws_bytes, s);
    if (e != cudaSuccess) return e;
    const BatchedConfig c = kConfigs[config];
    if (k > 0) {
        k_batched_count<<<(k + kSetupThreads - 1) / kSetupThreads, kSetupThreads, 0, s>>>(bp, c.threads,
                                                                                        c.blocks_per_thread);
        k_batched_fill<<<(k + kFillThreads / 32 - 1) / (kFillThreads / 32), kFillThreads, 0, s>>>(bp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode == kModeFast) return batched_dtype_dispatch<kModeFast>(bp, dtype, config, s);
    return batched_dtype_dispatch<kModeAccurate>(bp, dtype, config, s);
}

}  // namespace nrng
