// tiles.cuh -- one tile of a B1 stream and one tile of a Polar stream, as
// device functions shared by the single-stream and the batched kernels.
#pragma once

#include "nrng_device.cuh"

namespace nrng {

// ----------------------------------------------------------- B1 tile ------
// Blocks [t*TB, (t+1)*TB) of a stream, TB = THREADS * BPT; block b writes
// out[4b .. 4b+3] (Algorithm B1, two pairs per block).  With CARRY false the
// low counter word of the tile's blocks does not wrap (the caller checks), so
// the block index and the counter stay 32-bit.
template <int THREADS, int BPT, int MODE, typename T, bool ALIGNED, bool CARRY, typename Key>
__device__ __forceinline__ void b1_tile(T *__restrict__ out, int64_t n, const RadiusCoef &cf, const float4 *tab,
                                        const Key &rk, uint64_t counter, int64_t t)
{
    static_assert(BPT % 2 == 0, "rows are taken in pairs");
    const int64_t nblocks = (n + 3) / 4;
    const int64_t b00 = t * (THREADS * BPT) + threadIdx.x;
    const uint64_t c00 = counter + (uint64_t)b00;
    const uint32_t lo00 = (uint32_t)c00, hi00 = (uint32_t)(c00 >> 32);
    if (ALIGNED && !CARRY && 4 * (t + 1) * (THREADS * BPT) <= n) {
        // The whole tile in range: no bounds checks, a 32-bit counter word
        // and one output pointer stepped per pair of rows.
        T *o = out + 4 * b00;
        uint32_t lo = lo00;
        for (int r = 0; r < BPT; r += 2, lo += 2 * THREADS, o += 8 * THREADS) {
            float4 v, v2;
            b1_block2<MODE>(philox4x32_10(lo, hi00, rk), philox4x32_10(lo + THREADS, hi00, rk), cf, tab, v, v2);
            store4_aligned(o, v.x, v.y, v.z, v.w);
            store4_aligned(o + 4 * THREADS, v2.x, v2.y, v2.z, v2.w);
        }
        return;
    }
    // Two rows per step when both are in range: the two Philox chains are
    // independent and fill each other's multiply stalls.
    for (int r = 0; r < BPT; r += 2) {
        const int64_t b = b00 + r * THREADS;
        const int64_t b2 = b + THREADS;
        if (b2 < nblocks && ALIGNED && 4 * b2 + 4 <= n) {
            uint4 w, w2;
            if (CARRY) {
                w = philox_block(counter + (uint64_t)b, rk);
                w2 = philox_block(counter + (uint64_t)b2, rk);
            } else {
                w = philox4x32_10(lo00 + (uint32_t)(r * THREADS), hi00, rk);
                w2 = philox4x32_10(lo00 + (uint32_t)((r + 1) * THREADS), hi00, rk);
            }
            float4 o, o2;
            b1_block2<MODE>(w, w2, cf, tab, o, o2);
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

// --------------------------------------------------------- rejection tile --
// A tile of a rejection stream (Algorithm P, Method P2, Algorithm R) is NW
// warps x R rows x 32 lanes x 2 candidates.  Candidates are warp-major: warp
// w of tile t draws the Philox blocks t NW R 32 + w R 32 + r 32 + lane (row r,
// r = 0 .. R-1), and block b holds the candidates 2b (words 0, 1) and 2b + 1
// (words 2, 3).  A warp's accepted candidates are then one contiguous run of
// the stream's accepted candidates, in candidate order: the warp compacts them
// into its own shared-memory segment, transforms the segment densely, and once
// the tile's place in the output is known copies it out as one dense run.
template <int NW, int R>
struct RejSmem {
    static constexpr int kSeg = 64 * R;   // most accepted candidates a warp holds
    int2 seg[NW][kSeg];     // payloads after phase A, output bits after phase C
    uint2 mask[NW][R];      // accept ballots of (warp, row): half 0, half 1
    int cnt[NW];            // accepted candidates of each warp
    int off[NW];            // exclusive offsets of the warps within the tile
    int total;              // accepted candidates of the tile
    int drawn;              // accepted candidates of a limited tile 0's first draw
    long long prefix;       // the tile's exclusive prefix (-1 after an error)
    long long tile;         // the claimed tile id (single-stream kernels)
};

// Where a rejection stream's tile publishes and what it reports.  nitems is
// the number of accepted candidates the stream needs: ceil(n/2) pairs for
// P and P2, n values for R.
struct PolarStream {
    int64_t n, nitems;
    uint64_t counter;
    unsigned long long *status;   // this stream's tile status words
    int64_t tiles_max;
    int *done;                    // set once the tile holding the last item is known
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
// A rejection method on the candidate stream: each candidate is the two words
// 2h, 2h+1 of a Philox block (h = 0, 1); accept() decides it exactly and keeps
// a payload, transform() turns an accepted payload into kOut output values.

// Algorithm P (Sec. 2): steps 2-3 exact on the lattice scaled by 2^8, payload
// (kx' 2^8, ky' 2^8); step 4 (polar_pair).
template <int MODE>
struct PolarPolicy {
    static constexpr int kOut = 2;
    static constexpr int kRows = kPolarRows;   // rows of the single-stream tile
    __device__ static bool accept(uint32_t wa, uint32_t wb, int2 &pay) { return polar_accept_scaled(wa, wb, pay); }
    __device__ static void transform(int2 p, const RadiusCoef &c, float &a, float &b)
    {
        polar_pair<MODE>(p.x, p.y, c, a, b);
    }
    __device__ static void transform2(int2 p, int2 q, const RadiusCoef &c, float &a, float &b, float &d, float &e)
    {
        polar_pair2<MODE>(p, q, c, a, b, d, e);
    }
};

// Method P2 (Sec. 4): Algorithm P's steps 1-3, step 4a.
struct P2Policy {
    static constexpr int kOut = 2;
    static constexpr int kRows = kPolarRows;
    __device__ static bool accept(uint32_t wa, uint32_t wb, int2 &pay) { return polar_accept_scaled(wa, wb, pay); }
    __device__ static void transform(int2 p, const RadiusCoef &c, float &a, float &b)
    {
        p2_pair(p.x >> 8, p.y >> 8, c.mu, c.sigma, a, b);   // exact: multiples of 2^8
    }
    __device__ static void transform2(int2 p, int2 q, const RadiusCoef &c, float &a, float &b, float &d, float &e)
    {
        transform(p, c, a, b);
        transform(q, c, d, e);
    }
};

// Algorithm R (Sec. 5): payload (a, b) of the lattice, one value per accept.
template <int MODE>
struct RatioPolicy {
    static constexpr int kOut = 1;
    static constexpr int kRows = kRatioRows;
    __device__ static bool accept(uint32_t wu, uint32_t wv, int2 &pay) { return ratio_accept(wu, wv, pay); }
    __device__ static void transform(int2 p, const RadiusCoef &c, float &a, float &b)
    {
        a = ratio_value<MODE>(p, c.mu, c.sigma);
        b = 0.0f;
    }
    __device__ static void transform2(int2 p, int2 q, const RadiusCoef &c, float &a, float &b, float &d, float &e)
    {
        transform(p, c, a, b);
        transform(q, c, d, e);
    }
};

// Candidate index within the tile of entry e of warp `warp`'s segment, from
// the (warp, row) accept ballots: the row whose run holds e, then the lane by
// a binary search over the row's ballots (its candidates run lane by lane,
// half 0 before half 1).  Only the careful copy-out needs it (candidate
// indices requested, or the stream's last item).
template <int NW, int R>
__device__ __forceinline__ int tile_candidate(const RejSmem<NW, R> &sm, int warp, int e)
{
    int rb = 0, r = 0;
    for (; r < R - 1; ++r) {
        const uint2 m = sm.mask[warp][r];
        const int cr = __popc(m.x) + __popc(m.y);
        if (e < rb + cr) break;
        rb += cr;
    }
    const uint2 m = sm.mask[warp][r];
    const int j = e - rb;
    int L = 0;   // the lane holding item j: most accepted points below it <= j
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const unsigned lt = (1u << (L + step)) - 1u;
        if (__popc(m.x & lt) + __popc(m.y & lt) <= j) L += step;
    }
    const unsigned lt = (1u << L) - 1u;
    const int before = __popc(m.x & lt) + __popc(m.y & lt);
    const int h = (((m.x >> L) & 1u) && before == j) ? 0 : 1;
    return 2 * (warp * R * 32 + r * 32 + L) + h;
}

// Tile t of a rejection stream: the method's steps on candidates
// [t kCand, (t+1) kCand) in candidate order, the compress done per warp and a
// decoupled look-back across tiles.
//   A  each warp draws its R rows, decides each candidate, and appends the
//      accepted payloads to its segment in candidate order (rank by
//      ballot/popc); lane 0 keeps each row's ballots and the warp's count;
//   B  warp 0 scans the warp counts and publishes the tile aggregate at once;
//   C  each warp transforms its segment densely, in place;
//   D  warp 0 looks back for the tile's exclusive prefix P;
//   E  each warp copies its segment to items P + off(warp) + j, coalesced.
// Returns false when the look-back gave up (error recorded in hdr).  With
// KNOWN_PREFIX the tile's exclusive prefix is given (from a count pass and a
// scan): nothing is published and nothing is awaited.  With CARRY false the
// low counter word of the tile's blocks does not wrap (the caller checks).
// on_prefix() runs on thread 0 once the tile's prefix is known (after the
// look-back, before the copy-out), when the look-back succeeded.  cand_limit,
// for tile 0 only (its prefix is 0), is the number of candidates the stream
// is expected to need: a tile 0 that holds more draws only the warps that
// reach into the limit, and the others only if those fall short.
struct NoPrefixHook {
    __device__ void operator()() const {}
};

template <class Policy, int NW, int R, typename T, bool ALIGNED, bool CARRY, typename Key, bool KNOWN_PREFIX = false,
          class OnPrefix = NoPrefixHook>
__device__ __forceinline__ bool reject_tile(RejSmem<NW, R> &sm, T *__restrict__ out, const PolarStream &ps,
                                            const Key &rk, const RadiusCoef &cf, int64_t t, WsHeader *hdr,
                                            unsigned long long limit_ns, long long known_prefix = 0,
                                            OnPrefix on_prefix = OnPrefix(), int cand_limit = 1 << 30)
{
    constexpr int kBPT = NW * R * 32;   // Philox blocks of a tile
    constexpr int kCand = 2 * kBPT;
    constexpr int K = Policy::kOut;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool silent = (t == ps.silent_tile);
    const unsigned lt = (1u << lane) - 1u;

    // A: steps 1-3, compacted per warp.
    auto draw = [&]() {
        const uint64_t c0 = ps.counter + (uint64_t)t * kBPT + (uint64_t)(warp * R * 32 + lane);
        const uint32_t lo0 = (uint32_t)c0, hi0 = (uint32_t)(c0 >> 32);
        int2 *seg = sm.seg[warp];
        int base = 0;
        // Two rows per step: their Philox chains are independent and fill each
        // other's multiply latencies.
        static_assert(R % 2 == 0, "rows are drawn in pairs");
        auto row = [&](int r, const uint4 &w) {
            int2 p0, p1;
            const bool a0 = Policy::accept(w.x, w.y, p0);
            const bool a1 = Policy::accept(w.z, w.w, p1);
            const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0);
            const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1);
            const int pos = base + __popc(m0 & lt) + __popc(m1 & lt);
            if (a0) seg[pos] = p0;
            if (a1) seg[pos + (a0 ? 1 : 0)] = p1;
            if (lane == 0) sm.mask[warp][r] = make_uint2(m0, m1);
            base += __popc(m0) + __popc(m1);
        };
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            const uint32_t lo = lo0 + (uint32_t)(r * 32), lo2 = lo + 32u;
            const uint32_t hi = CARRY ? hi0 + (lo < lo0 ? 1u : 0u) : hi0;
            const uint32_t hi2 = CARRY ? hi0 + (lo2 < lo0 ? 1u : 0u) : hi0;
            const uint4 w = philox4x32_10(lo, hi, rk);
            const uint4 w2 = philox4x32_10(lo2, hi2, rk);
            row(r, w);
            row(r + 1, w2);
        }
        if (lane == 0) sm.cnt[warp] = base;
    };
    if (cand_limit >= kCand) {
        draw();
        __syncthreads();
    } else {
        // Tile 0 of a stream that is expected to need fewer candidates than a
        // tile holds (cand_limit): the warps whose candidates all lie beyond
        // the limit draw nothing at first.  The drawn warps are a prefix
        // of the tile's candidates, so if they hold the stream's nitems accepted
        // candidates the tile's output is the full tile's; otherwise the other
        // warps draw theirs too.  (CTA-uniform: every thread sees the same t
        // and limit.)
        const bool first = warp * R * 64 < cand_limit;
        if (first) draw();
        else if (lane == 0) sm.cnt[warp] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int drawn = 0;
            for (int q = 0; q < NW; ++q) drawn += sm.cnt[q];
            sm.drawn = drawn;
        }
        __syncthreads();
        if (sm.drawn < ps.nitems) {
            if (!first) draw();
            __syncthreads();
        }
    }

    // B: warp 0 scans the warp counts and publishes the aggregate.
    int total = 0;
    if (warp == 0) {
        const int v = lane < NW ? sm.cnt[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < NW) sm.off[lane] = incl - v;
        total = __shfl_sync(0xFFFFFFFFu, incl, NW - 1);
        if (lane == 0) {
            sm.total = total;
            if (!KNOWN_PREFIX && !silent)
                st_relaxed(ps.status + t, (t == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
        }
    }

    // C: the transform over this warp's segment, dense, results in place
    // (two entries a lane per step while both are in range).
    {
        int2 *q = sm.seg[warp] + lane;
        int2 *const end = sm.seg[warp] + sm.cnt[warp];
        for (; q + 32 < end; q += 64) {
            float za, zb, zc, zd;
            Policy::transform2(q[0], q[32], cf, za, zb, zc, zd);
            q[0] = (K == 2) ? pair_bits<T>(za, zb) : item_bits<T>(za);
            q[32] = (K == 2) ? pair_bits<T>(zc, zd) : item_bits<T>(zc);
        }
        if (q < end) {
            float za, zb;
            Policy::transform(q[0], cf, za, zb);
            q[0] = (K == 2) ? pair_bits<T>(za, zb) : item_bits<T>(za);
        }
    }

    // D: warp 0 looks back for the exclusive prefix.
    if (warp == 0) {
        long long P = known_prefix;
        if (!KNOWN_PREFIX)
            P = lookback_warp(ps.status, t, total, hdr, limit_ns, false, !silent);
        if (lane == 0) {
            sm.prefix = P;
            if (P >= 0 && !KNOWN_PREFIX) {
                if (P < ps.nitems && P + total >= ps.nitems) st_relaxed_s32(ps.done, 1);
                if (t == ps.tiles_max - 1 && P + total < ps.nitems) raise_error(hdr, kStatusExhausted);
            }
            if (P >= 0) on_prefix();
        }
    }
    __syncthreads();

    // E: this warp's segment -> items P + off(warp) + j.
    const long long P = sm.prefix;
    if (P < 0) return false;
    if (P >= ps.nitems) return true;
    const long long base = P + sm.off[warp];
    const int c = sm.cnt[warp];
    const int2 *seg = sm.seg[warp];
    if (ALIGNED && base + c <= ps.nitems && (K == 1 || base + c <= ps.n / 2) && ps.pair_cand == nullptr) {
        // every item of the warp placed whole and nothing else recorded
        T *o = out + K * (base + lane);
        const int2 *q = seg + lane;
        const int2 *const end = seg + c;
        for (; q + 32 < end; q += 64, o += 64 * K) {
            const int2 v0 = q[0], v1 = q[32];
            if (K == 2) {
                store_pair_bits<T>(o, v0, true);
                store_pair_bits<T>(o + 64, v1, true);
            } else {
                store_item_bits<T>(o, v0);
                store_item_bits<T>(o + 32, v1);
            }
        }
        if (q < end) {
            if (K == 2) store_pair_bits<T>(o, q[0], true);
            else store_item_bits<T>(o, q[0]);
        }
        return true;
    }
    const long long rem_full = (K == 2) ? ps.n / 2 : ps.nitems;   // items with every element
    for (int e = lane; e < c; e += 32) {
        const long long g = base + e;
        if (g >= ps.nitems) break;
        const int2 v = seg[e];
        if (K == 1) {
            store_item_bits<T>(out + g, v);
        } else if (ALIGNED) {
            store_pair_bits<T>(out + 2 * g, v, g < rem_full);
        } else if constexpr (sizeof(T) == 4) {
            out[2 * g] = __int_as_float(v.x);
            if (g < rem_full) out[2 * g + 1] = __int_as_float(v.y);
        } else {
            const uint16_t lo = (uint16_t)((unsigned)v.x & 0xFFFFu), hi = (uint16_t)((unsigned)v.x >> 16);
            memcpy(&out[2 * g], &lo, 2);
            if (g < rem_full) memcpy(&out[2 * g + 1], &hi, 2);
        }
        if (ps.pair_cand || g == ps.nitems - 1) {
            const long long cand = t * kCand + tile_candidate<NW, R>(sm, warp, e);
            if (ps.pair_cand) ps.pair_cand[g] = cand;
            if (g == ps.nitems - 1 && ps.next_counter) *ps.next_counter = ps.counter + (uint64_t)(cand / 2) + 1u;
        }
    }
    return true;
}

// Next tile id of a single rejection stream, or -1 once the tile budget is
// spent; *late is set when the stream was already complete.  The completion
// flag and the claim are issued together (one round trip).  A tile claimed
// after completion is never dropped unpublished (a later tile's look-back
// would wait on it until its limit): the caller publishes it as complete.
// That is exact: a claim that sees the flag set comes after the tile holding
// the last item, whose look-back had to see every earlier tile published, so
// the claimed tile's prefix is at least nitems.
__device__ __forceinline__ long long claim_tile(const PolarParams &p, int &late)
{
    late = ld_relaxed_s32(&p.hdr->done);
    const long long t = (long long)atomicAdd(&p.hdr->tile_counter, 1ull);
    return t < p.tiles_max ? t : -1;
}

// Resident CTAs per SM a rejection kernel is compiled for: as many as the
// tile's shared memory admits (with the 1 KB the runtime keeps per CTA), so
// that the register budget follows from that count.
template <int NW, int R>
struct RejOccupancy {
    static constexpr int kSmem = (228 * 1024) / ((int)sizeof(RejSmem<NW, R>) + 1024);
    static constexpr int kThreads = 2048 / (NW * 32);
    static constexpr int kMin0 = kSmem < kThreads ? kSmem : kThreads;
    static constexpr int kMinBlocks = kMin0 > 0 ? kMin0 : 1;
};

// One rejection stream over the whole grid: persistent CTAs take tile ids
// from the workspace counter until the stream is complete (done) or the tile
// budget is spent.
template <class Policy, typename T, bool ALIGNED, bool CARRY>
__global__ void __launch_bounds__(kRejWarps * 32, (RejOccupancy<kRejWarps, Policy::kRows>::kMinBlocks))
k_reject(const PolarParams p)
{
    __shared__ RejSmem<kRejWarps, Policy::kRows> sm;
    PolarStream ps;
    ps.n = p.n;
    ps.nitems = p.nitems;
    ps.counter = p.counter;
    ps.status = p.tile_status;
    ps.tiles_max = p.tiles_max;
    ps.done = &p.hdr->done;
    ps.next_counter = p.next_counter;
    ps.pair_cand = p.pair_cand;
    ps.silent_tile = p.debug_silent_tile;
    const RadiusCoef cf = radius_coef(p.mu, p.sigma);
    T *out = static_cast<T *>(p.out);
    for (;;) {
        if (threadIdx.x == 0) {
            int late;
            long long t = claim_tile(p, late);
            if (t >= 0 && late) {
                // the stream is complete: every later tile's prefix is >= nitems
                if (t != ps.silent_tile) st_relaxed(ps.status + t, kFlagPrefix | (unsigned long long)ps.nitems);
                t = -1;
            }
            sm.tile = t;
        }
        __syncthreads();
        const long long t = sm.tile;
        if (t < 0) break;
        const bool ok = reject_tile<Policy, kRejWarps, Policy::kRows, T, ALIGNED, CARRY>(sm, out, ps, p.rk, cf, t,
                                                                                      p.hdr, p.spin_limit_ns);
        __syncthreads();
        if (!ok) break;
    }
}

// Whether the low counter word of every Philox block of a rejection stream's
// tile budget stays below 2^32 (the kernels' carry-free form).
__host__ __device__ inline bool reject_carry_free(uint64_t counter, int64_t tiles_max, int blocks_per_tile)
{
    return (uint64_t)(uint32_t)counter + (uint64_t)tiles_max * (uint64_t)blocks_per_tile <= (uint64_t(1) << 32);
}

}  // namespace nrng
