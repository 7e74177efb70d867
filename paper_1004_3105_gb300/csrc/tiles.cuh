// tiles.cuh -- one tile of a B1 stream and one tile of a Polar stream, as
// device functions shared by the single-stream and the batched kernels.
#pragma once

#include "nrng_device.cuh"

namespace nrng {

// ----------------------------------------------------------- B1 tile ------
// Blocks [t*TB, (t+1)*TB) of a stream, TB = THREADS * BPT; block b writes
// out[4b .. 4b+3] (Algorithm B1, two pairs per block).
template <int THREADS, int BPT, int MODE, typename T, bool ALIGNED, typename Key>
__device__ __forceinline__ void b1_tile(T *__restrict__ out, int64_t n, const B1Coef &cf, const float4 *tab,
                                        const Key &rk, uint64_t counter, int64_t t)
{
    const int64_t nblocks = (n + 3) / 4;
    // Two rows per step when both are in range: the two Philox chains are
    // independent and fill each other's multiply stalls.
    for (int r = 0; r < BPT; r += 2) {
        const int64_t b = t * (THREADS * BPT) + r * THREADS + threadIdx.x;
        const int64_t b2 = b + THREADS;
        if (b2 < nblocks && ALIGNED && 4 * b2 + 4 <= n) {
            const float4 o = b1_block<MODE>(philox_block(counter + (uint64_t)b, rk), cf, tab);
            const float4 o2 = b1_block<MODE>(philox_block(counter + (uint64_t)b2, rk), cf, tab);
            store4_aligned(out + 4 * b, o.x, o.y, o.z, o.w);
            store4_aligned(out + 4 * b2, o2.x, o2.y, o2.z, o2.w);
            continue;
        }
        for (int q = 0; q < 2; ++q) {
            const int64_t bq = b + q * THREADS;
            if (bq >= nblocks) return;
            const float4 o = b1_block<MODE>(philox_block(counter + (uint64_t)bq, rk), cf, tab);
            const int64_t i = 4 * bq;
            if (ALIGNED && i + 4 <= n) {
                store4_aligned(out + i, o.x, o.y, o.z, o.w);
            } else {
                if (i < n) store1(out + i, o.x);
                if (i + 1 < n) store1(out + i + 1, o.y);
                if (i + 2 < n) store1(out + i + 2, o.z);
                if (i + 3 < n) store1(out + i + 3, o.w);
            }
        }
    }
}

// Resident threads per SM the Polar tile kernels are compiled for (sets the
// register budget through __launch_bounds__: 40 registers a thread, without
// spills).  With the 33.6 KB tile, six 256-thread CTAs fit per SM.
template <int THREADS, int MODE>
struct PolarOccupancy {
    static constexpr int kThreads = 1536;
    static constexpr int kMinBlocks = (kThreads / THREADS) > 0 ? (kThreads / THREADS) : 1;
};

// --------------------------------------------------------- Polar tile -----
template <int THREADS, int ROWS>
struct PolarSmem {
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kEntries = ROWS * kWarps;   // (row, warp) segments
    static constexpr int kSeg = 64 * ROWS;           // most accepted points a warp holds
    int2 seg[kWarps][kSeg];      // each warp's accepted points in candidate order; step-4 results in place
    uint2 mask[kEntries];        // (row, warp) accept ballots of the two candidate halves
    int off[kEntries];           // (row, warp) counts, then exclusive offsets
    int total;                   // accepted points of the tile
    long long prefix;
};

template <int THREADS, int ROWS>
__device__ __forceinline__ int total_of(const PolarSmem<THREADS, ROWS> &sm, int)
{
    return sm.total;
}

// Where a rejection stream's tile publishes and what it reports.  nitems is
// the number of accepted candidates the stream needs: ceil(n/2) pairs for
// P and P2, n values for R.
struct PolarStream {
    int64_t n, nitems;
    float mu, sigma;
    uint64_t counter;
    unsigned long long *status;   // this stream's tile status words
    int64_t tiles_max;
    int *done;                    // set when the last pair is placed
    uint64_t *next_counter;       // nullable
    int64_t *pair_cand;           // nullable
    long long silent_tile;        // test hook: never publishes (-1: none)
};

template <typename T>
__device__ __forceinline__ int2 pair_bits(float zx, float zy)
{
    if constexpr (sizeof(T) == 4) return make_int2(__float_as_int(zx), __float_as_int(zy));
    else return make_int2((int)pack2<T>(zx, zy), 0);
}

template <typename T>
__device__ __forceinline__ void store_pair_bits(T *p, int2 v, bool both)
{
    if constexpr (sizeof(T) == 4) {
        if (both) {
            __stcs(reinterpret_cast<int2 *>(p), v);
        } else {
            *reinterpret_cast<int *>(p) = v.x;
        }
    } else {
        if (both) {
            __stcs(reinterpret_cast<unsigned int *>(p), (unsigned int)v.x);
        } else {
            *reinterpret_cast<uint16_t *>(p) = (uint16_t)((unsigned)v.x & 0xFFFFu);
        }
    }
}

// One output value (the Ratio method): bits of a float or a 16-bit value.
template <typename T>
__device__ __forceinline__ int2 item_bits(float z)
{
    if constexpr (sizeof(T) == 4) return make_int2(__float_as_int(z), 0);
    else {
        const T tz = OutTraits<T>::cvt(z);
        uint16_t u;
        memcpy(&u, &tz, 2);
        return make_int2((int)u, 0);
    }
}

template <typename T>
__device__ __forceinline__ void store_item_bits(T *p, int2 v)
{
    if constexpr (sizeof(T) == 4) *reinterpret_cast<int *>(p) = v.x;
    else *reinterpret_cast<uint16_t *>(p) = (uint16_t)((unsigned)v.x & 0xFFFFu);
}

// ------------------------------------------------------------ policies ----
// Local candidate index (within the tile) of the j-th accepted candidate of
// row r, warp w, from the row's accept ballots m = (half 0, half 1): the
// candidates of a row run lane by lane, half 0 before half 1.  Only the
// careful copy-out (candidate indices requested, or the stream's last tile)
// needs it, so a binary search over the lanes replaces a stored index per
// accepted point.
template <int THREADS>
__device__ __forceinline__ int accepted_candidate(uint2 m, int j, int r, int w)
{
    int L = 0;   // the lane holding item j: most accepted points below it <= j
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const unsigned lt = (1u << (L + step)) - 1u;
        if (__popc(m.x & lt) + __popc(m.y & lt) <= j) L += step;
    }
    const unsigned lt = (1u << L) - 1u;
    const int before = __popc(m.x & lt) + __popc(m.y & lt);
    const int h = (((m.x >> L) & 1u) && before == j) ? 0 : 1;
    return 2 * (r * THREADS + w * 32 + L) + h;
}

// A rejection method on the candidate stream: each candidate is the two words
// 2h, 2h+1 of a Philox block (h = 0, 1); accept() decides it and keeps a
// payload, transform() turns an accepted payload into kOut output values.

// Algorithm P (Sec. 2): payload (kx', ky'); steps 2-3 exact; step 4.
template <int MODE>
struct PolarPolicy {
    static constexpr int kOut = 2;
    __device__ static bool accept(uint32_t wa, uint32_t wb, int2 &pay)
    {
        const int32_t x = k24(wa), y = k24(wb);
        pay = make_int2(x, y);
        int64_t S;
        return polar_accept(x, y, S);
    }
    __device__ static void transform(int2 p, float mu, float sigma, float &a, float &b)
    {
        polar_pair<MODE>(p.x, p.y, mu, sigma, a, b);
    }
};

// Method P2 (Sec. 4): Algorithm P's steps 1-3, step 4a.
struct P2Policy {
    static constexpr int kOut = 2;
    __device__ static bool accept(uint32_t wa, uint32_t wb, int2 &pay)
    {
        return PolarPolicy<kModeAccurate>::accept(wa, wb, pay);
    }
    __device__ static void transform(int2 p, float mu, float sigma, float &a, float &b)
    {
        p2_pair(p.x, p.y, mu, sigma, a, b);
    }
};

// Algorithm R (Sec. 5): payload (a, b) of the lattice, one value per accept.
template <int MODE>
struct RatioPolicy {
    static constexpr int kOut = 1;
    __device__ static bool accept(uint32_t wu, uint32_t wv, int2 &pay) { return ratio_accept(wu, wv, pay); }
    __device__ static void transform(int2 p, float mu, float sigma, float &a, float &b)
    {
        a = ratio_value<MODE>(p, mu, sigma);
        b = 0.0f;
    }
};

// Tile t of a rejection stream: the method's steps on candidates
// [t*kCand, (t+1)*kCand) (Algorithm P, P2 or R by Policy), in candidate order
// (row, warp, lane, half), with the compress done per warp and a decoupled
// look-back across tiles.
//   A  each warp draws its rows, runs the accept test, and appends the
//      accepted payloads to its own shared-memory segment in candidate order
//      (rank by ballot/popc); lane 0 records each (row, warp) count;
//   B  warp 0 scans the counts and publishes the tile aggregate at once;
//   C  each warp runs the transform densely over its own segment, in place;
//   D  warp 0 looks back for the tile's exclusive prefix P;
//   E  each warp copies its (row) runs to items P + offset(row, warp) + j
//      (elements kOut (P + ...)), coalesced.
// Only A->B and D->E need the whole CTA; the rest is warp-synchronous.
// Returns false when the look-back gave up (error recorded in hdr).
// With KNOWN_PREFIX the tile's exclusive prefix is given (known_prefix, from
// a count pass and a scan): nothing is published and nothing is awaited.
template <class Policy, int THREADS, int ROWS, typename T, bool ALIGNED, typename Key, bool KNOWN_PREFIX = false>
__device__ __forceinline__ bool reject_tile(PolarSmem<THREADS, ROWS> &sm, T *__restrict__ out,
                                            const PolarStream &ps, const Key &rk, int64_t t, WsHeader *hdr,
                                            unsigned long long limit_ns, long long known_prefix = 0)
{
    constexpr int kWarps = THREADS / 32;
    constexpr int kEntries = ROWS * kWarps;
    constexpr int kCand = 2 * THREADS * ROWS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool silent = (t == ps.silent_tile);
    const unsigned lt = (1u << lane) - 1u;
    int2 *seg = sm.seg[warp];

    // A: steps 1-3, compacted per warp.
    int rowbase[ROWS + 1];   // warp-uniform: start of each row's run in the segment
    int base = 0;
    const uint64_t b0 = ps.counter + (uint64_t)t * (THREADS * ROWS) + (uint64_t)tid;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint4 w = philox_block(b0 + (uint64_t)(r * THREADS), rk);
        int2 p0, p1;
        const bool a0 = Policy::accept(w.x, w.y, p0);
        const bool a1 = Policy::accept(w.z, w.w, p1);
        const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0);
        const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1);
        const int pos = base + __popc(m0 & lt) + __popc(m1 & lt);
        if (a0) seg[pos] = p0;
        if (a1) seg[pos + (a0 ? 1 : 0)] = p1;
        const int cnt = __popc(m0) + __popc(m1);
        if (lane == 0) {
            sm.off[r * kWarps + warp] = cnt;
            sm.mask[r * kWarps + warp] = make_uint2(m0, m1);
        }
        rowbase[r] = base;
        base += cnt;
    }
    rowbase[ROWS] = base;
    __syncthreads();

    // B: warp 0 scans the counts (row-major over warps) and publishes.
    int total = 0;
    if (warp == 0) {
#pragma unroll
        for (int c0 = 0; c0 < kEntries; c0 += 32) {
            const int v = (c0 + lane < kEntries) ? sm.off[c0 + lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (c0 + lane < kEntries) sm.off[c0 + lane] = total + incl - v;
            total += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (lane == 0) {
            sm.total = total;
            if (!KNOWN_PREFIX && !silent)
                st_relaxed(ps.status + t, (t == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
        }
    }

    // C: the transform over this warp's segment, dense, results in place.
#pragma unroll 2
    for (int j = lane; j < base; j += 32) {
        float za, zb;
        Policy::transform(seg[j], ps.mu, ps.sigma, za, zb);
        seg[j] = (Policy::kOut == 2) ? pair_bits<T>(za, zb) : item_bits<T>(za);
    }

    // D: warp 0 looks back for the exclusive prefix.
    if (KNOWN_PREFIX) {
        if (tid == 0) sm.prefix = known_prefix;
    } else if (warp == 0) {
        const long long P = silent ? lookback_warp(ps.status, t, total, hdr, limit_ns, false, false)
                                   : lookback_warp(ps.status, t, total, hdr, limit_ns, false, true);
        if (lane == 0) {
            sm.prefix = P;
            if (P >= 0 && t == ps.tiles_max - 1 && P + total < ps.nitems) raise_error(hdr, kStatusExhausted);
        }
    }
    __syncthreads();

    // E: run r of this warp -> items P + off(r, warp) + j.
    constexpr int K = Policy::kOut;
    const long long P = sm.prefix;
    if (P < 0) return false;
    if (P >= ps.nitems) return true;
    const int total_t = sm.total;
    if (ALIGNED && P + total_t < ps.nitems && (K == 1 || P + total_t <= ps.n / 2) && ps.pair_cand == nullptr) {
        // Every item of the tile is placed whole and nothing else is recorded.
        T *tile_out = out + K * P;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int o = sm.off[r * kWarps + warp];
            const int rb = rowbase[r];
            const int cnt = rowbase[r + 1] - rb;   // at most 64: two steps of 32 lanes
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j < cnt) {
                    if (K == 2) store_pair_bits<T>(tile_out + 2 * (o + j), seg[rb + j], true);
                    else store_item_bits<T>(tile_out + (o + j), seg[rb + j]);
                }
            }
        }
        return true;
    }
    const long long rem = ps.nitems - P;                  // items this tile may still place
    const long long rem_full = (K == 2) ? ps.n / 2 - P : rem;   // of which with every element
    const int lim = (int)(rem < kCand ? rem : kCand);
    const int lim_full = (int)(rem_full < kCand ? (rem_full > 0 ? rem_full : 0) : kCand);
    T *tile_out = out + K * P;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int o = sm.off[r * kWarps + warp];
        const int cnt = rowbase[r + 1] - rowbase[r];
        for (int j = lane; j < cnt; j += 32) {
            const int gl = o + j;   // item index within the tile's output
            if (gl >= lim) break;
            const int2 v = seg[rowbase[r] + j];
            if (K == 1) {
                store_item_bits<T>(tile_out + gl, v);
            } else if (ALIGNED) {
                store_pair_bits<T>(tile_out + 2 * gl, v, gl < lim_full);
            } else if constexpr (sizeof(T) == 4) {
                tile_out[2 * gl] = __int_as_float(v.x);
                if (gl < lim_full) tile_out[2 * gl + 1] = __int_as_float(v.y);
            } else {
                const uint16_t lo = (uint16_t)((unsigned)v.x & 0xFFFFu), hi = (uint16_t)((unsigned)v.x >> 16);
                memcpy(&tile_out[2 * gl], &lo, 2);
                if (gl < lim_full) memcpy(&tile_out[2 * gl + 1], &hi, 2);
            }
            if (ps.pair_cand || gl == lim - 1) {
                const long long c = t * kCand + accepted_candidate<THREADS>(sm.mask[r * kWarps + warp], j, r, warp);
                if (ps.pair_cand) ps.pair_cand[P + gl] = c;
                if (P + gl == ps.nitems - 1) {
                    if (ps.next_counter) *ps.next_counter = ps.counter + (uint64_t)(c / 2) + 1u;
                    st_relaxed_s32(ps.done, 1);
                }
            }
        }
    }
    return true;
}

// Algorithm P's tile (the common case, for the single-stream and batched kernels).
template <int THREADS, int ROWS, int MODE, typename T, bool ALIGNED, typename Key, bool KNOWN_PREFIX = false>
__device__ __forceinline__ bool polar_tile(PolarSmem<THREADS, ROWS> &sm, T *__restrict__ out,
                                           const PolarStream &ps, const Key &rk, int64_t t, WsHeader *hdr,
                                           unsigned long long limit_ns, long long known_prefix = 0)
{
    return reject_tile<PolarPolicy<MODE>, THREADS, ROWS, T, ALIGNED, Key, KNOWN_PREFIX>(sm, out, ps, rk, t, hdr,
                                                                                        limit_ns, known_prefix);
}

// Next tile id of a single rejection stream, or -1 once the stream is
// complete or the tile budget is spent.
// The completion flag is read before the claim, never alongside it: a tile
// claimed and then dropped would never publish, and a later tile's look-back
// would wait on it until its limit.  (Issuing the two together was measured:
// an occasional call ran into that wait.)
__device__ __forceinline__ long long claim_tile(const PolarParams &p)
{
    if (ld_relaxed_s32(&p.hdr->done) != 0) return -1;
    const long long t = (long long)atomicAdd(&p.hdr->tile_counter, 1ull);
    return t < p.tiles_max ? t : -1;
}

// One rejection stream over the whole grid: persistent CTAs take tile ids
// from the workspace counter until the stream is complete (done) or the tile
// budget is spent.
// OCC_THREADS: resident threads per SM the kernel is compiled for (its
// register budget): 1536 (40 registers) for Algorithm P, 1280 (48) for the
// P2 and R transforms, measured faster at those budgets.
template <class Policy, int OCC_THREADS, typename T, bool ALIGNED>
__global__ void __launch_bounds__(kPolarThreads, OCC_THREADS / kPolarThreads)
k_reject(const PolarParams p)
{
    __shared__ PolarSmem<kPolarThreads, kPolarRows> sm;
    __shared__ long long s_tile;

    PolarStream ps;
    ps.n = p.n;
    ps.nitems = p.nitems;
    ps.mu = p.mu;
    ps.sigma = p.sigma;
    ps.counter = p.counter;
    ps.status = p.tile_status;
    ps.tiles_max = p.tiles_max;
    ps.done = &p.hdr->done;
    ps.next_counter = p.next_counter;
    ps.pair_cand = p.pair_cand;
    ps.silent_tile = p.debug_silent_tile;
    T *out = static_cast<T *>(p.out);

    for (;;) {
        if (threadIdx.x == 0) s_tile = claim_tile(p);
        __syncthreads();
        const long long t = s_tile;
        if (t < 0) break;
        const bool ok = reject_tile<Policy, kPolarThreads, kPolarRows, T, ALIGNED>(sm, out, ps, p.rk, t, p.hdr,
                                                                                 p.spin_limit_ns);
        __syncthreads();
        if (!ok) break;
    }
}

}  // namespace nrng
