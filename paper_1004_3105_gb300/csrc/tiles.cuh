// tiles.cuh -- one tile of a B1 stream and one tile of a Polar stream, as
// device functions shared by the single-stream and the batched kernels.
#pragma once

#include "nrng_device.cuh"

namespace nrng {

// ----------------------------------------------------------- B1 tile ------
// Blocks [t*TB, (t+1)*TB) of a stream, TB = THREADS * BPT; block b writes
// out[4b .. 4b+3] (Algorithm B1, two pairs per block).
template <int THREADS, int BPT, int MODE, typename T, bool ALIGNED, typename Key>
__device__ __forceinline__ void b1_tile(T *__restrict__ out, int64_t n, float mu, float sigma,
                                        const Key &rk, uint64_t counter, int64_t t)
{
    const int64_t nblocks = (n + 3) / 4;
#pragma unroll 2
    for (int r = 0; r < BPT; ++r) {
        const int64_t b = t * (THREADS * BPT) + r * THREADS + threadIdx.x;
        if (b >= nblocks) break;
        const uint4 w = philox_block(counter + (uint64_t)b, rk);
        float x0, y0, x1, y1;
        b1_pair<MODE>(w.x, w.y, mu, sigma, x0, y0);
        b1_pair<MODE>(w.z, w.w, mu, sigma, x1, y1);
        const int64_t i = 4 * b;
        if (ALIGNED && i + 4 <= n) {
            store4_aligned(out + i, x0, y0, x1, y1);
        } else {
            if (i < n) store1(out + i, x0);
            if (i + 1 < n) store1(out + i + 1, y0);
            if (i + 2 < n) store1(out + i + 2, x1);
            if (i + 3 < n) store1(out + i + 3, y1);
        }
    }
}

// Resident threads per SM the Polar tile kernels are compiled for (sets the
// register budget through __launch_bounds__: 51 registers a thread).
template <int THREADS, int MODE>
struct PolarOccupancy {
    static constexpr int kThreads = 1280;
    static constexpr int kMinBlocks = (kThreads / THREADS) > 0 ? (kThreads / THREADS) : 1;
};

// --------------------------------------------------------- Polar tile -----
template <int THREADS, int ROWS>
struct PolarSmem {
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kEntries = ROWS * kWarps;   // (row, warp) segments
    static constexpr int kSeg = 64 * ROWS;           // most accepted points a warp holds
    int2 seg[kWarps][kSeg];      // each warp's accepted points in candidate order; step-4 results in place
    uint16_t cl[kWarps][kSeg];   // local candidate index of each entry
    int off[kEntries];           // (row, warp) counts, then exclusive offsets
    int total;                   // accepted points of the tile
    long long prefix;
};

template <int THREADS, int ROWS>
__device__ __forceinline__ int total_of(const PolarSmem<THREADS, ROWS> &sm, int)
{
    return sm.total;
}

// Where a Polar stream's tile publishes and what it reports.
struct PolarStream {
    int64_t n, npairs;
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

// Tile t of a Polar stream: Algorithm P (Sec. 2, steps 1-4) on candidates
// [t*kCand, (t+1)*kCand), in candidate order (row, warp, lane, half), with the
// compress done per warp and a decoupled look-back across tiles.
//   A  each warp draws its rows, tests 0 < S < 2^46 exactly, and appends its
//      accepted points to its own shared-memory segment in candidate order
//      (rank by ballot/popc); lane 0 records each (row, warp) count;
//   B  warp 0 scans the counts and publishes the tile aggregate at once;
//   C  each warp runs step 4 densely over its own segment, in place;
//   D  warp 0 looks back for the tile's exclusive prefix P;
//   E  each warp copies its (row) runs to pairs P + offset(row, warp) + j,
//      coalesced.
// Only A->B and D->E need the whole CTA; the rest is warp-synchronous.
// Returns false when the look-back gave up (error recorded in hdr).
template <int THREADS, int ROWS, int MODE, typename T, bool ALIGNED, typename Key>
__device__ __forceinline__ bool polar_tile(PolarSmem<THREADS, ROWS> &sm, T *__restrict__ out,
                                           const PolarStream &ps, const Key &rk, int64_t t, WsHeader *hdr,
                                           unsigned long long limit_ns)
{
    constexpr int kWarps = THREADS / 32;
    constexpr int kEntries = ROWS * kWarps;
    constexpr int kCand = 2 * THREADS * ROWS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool silent = (t == ps.silent_tile);
    const unsigned lt = (1u << lane) - 1u;
    int2 *seg = sm.seg[warp];
    uint16_t *cl = sm.cl[warp];

    // A: steps 1-3, compacted per warp.
    int rowbase[ROWS + 1];   // warp-uniform: start of each row's run in the segment
    int base = 0;
    const uint64_t b0 = ps.counter + (uint64_t)t * (THREADS * ROWS) + (uint64_t)tid;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint4 w = philox_block(b0 + (uint64_t)(r * THREADS), rk);
        const int32_t x0 = k24(w.x), y0 = k24(w.y), x1 = k24(w.z), y1 = k24(w.w);
        int64_t S0, S1;
        const bool a0 = polar_accept(x0, y0, S0);
        const bool a1 = polar_accept(x1, y1, S1);
        const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0);
        const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1);
        const int pos = base + __popc(m0 & lt) + __popc(m1 & lt);
        const uint16_t c = (uint16_t)(2 * (r * THREADS + tid));
        if (a0) {
            seg[pos] = make_int2(x0, y0);
            cl[pos] = c;
        }
        if (a1) {
            seg[pos + (a0 ? 1 : 0)] = make_int2(x1, y1);
            cl[pos + (a0 ? 1 : 0)] = (uint16_t)(c + 1);
        }
        const int cnt = __popc(m0) + __popc(m1);
        if (lane == 0) sm.off[r * kWarps + warp] = cnt;
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
            if (!silent)
                st_relaxed(ps.status + t, (t == 0 ? kFlagPrefix : kFlagAggregate) | (unsigned long long)total);
        }
    }

    // C: step 4 over this warp's segment, dense, results in place.
#pragma unroll 1
    for (int j = lane; j < base; j += 32) {
        const int2 k = seg[j];
        float zx, zy;
        polar_pair<MODE>(k.x, k.y, ps.mu, ps.sigma, zx, zy);
        seg[j] = pair_bits<T>(zx, zy);
    }

    // D: warp 0 looks back for the exclusive prefix.
    if (warp == 0) {
        const long long P = silent ? lookback_warp(ps.status, t, total, hdr, limit_ns, false, false)
                                   : lookback_warp(ps.status, t, total, hdr, limit_ns, false, true);
        if (lane == 0) {
            sm.prefix = P;
            if (P >= 0 && t == ps.tiles_max - 1 && P + total < ps.npairs) raise_error(hdr, kStatusExhausted);
        }
    }
    __syncthreads();

    // E: run r of this warp -> pairs P + off(r, warp) + j.
    const long long P = sm.prefix;
    if (P < 0) return false;
    if (P >= ps.npairs) return true;
    if (ALIGNED && P + total_of(sm, kEntries) < ps.npairs && P + total_of(sm, kEntries) <= ps.n / 2 &&
        ps.pair_cand == nullptr) {
        // Every pair of the tile is placed whole and nothing else is recorded.
        T *tile_out = out + 2 * P;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int o = sm.off[r * kWarps + warp];
            const int rb = rowbase[r];
            const int cnt = rowbase[r + 1] - rb;
            for (int j = lane; j < cnt; j += 32) store_pair_bits<T>(tile_out + 2 * (o + j), seg[rb + j], true);
        }
        return true;
    }
    const long long rem = ps.npairs - P;                 // pairs this tile may still place
    const long long rem_full = ps.n / 2 - P;             // of which with both x and y
    const int lim = (int)(rem < kCand ? rem : kCand);
    const int lim_full = (int)(rem_full < kCand ? (rem_full > 0 ? rem_full : 0) : kCand);
    T *tile_out = out + 2 * P;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int o = sm.off[r * kWarps + warp];
        const int cnt = rowbase[r + 1] - rowbase[r];
        for (int j = lane; j < cnt; j += 32) {
            const int gl = o + j;   // pair index within the tile's output
            if (gl >= lim) break;
            const int2 v = seg[rowbase[r] + j];
            if (ALIGNED) {
                store_pair_bits<T>(tile_out + 2 * gl, v, gl < lim_full);
            } else {
                float zx, zy;
                if constexpr (sizeof(T) == 4) {
                    zx = __int_as_float(v.x);
                    zy = __int_as_float(v.y);
                    tile_out[2 * gl] = zx;
                    if (gl < lim_full) tile_out[2 * gl + 1] = zy;
                } else {
                    const uint16_t lo = (uint16_t)((unsigned)v.x & 0xFFFFu), hi = (uint16_t)((unsigned)v.x >> 16);
                    memcpy(&tile_out[2 * gl], &lo, 2);
                    if (gl < lim_full) memcpy(&tile_out[2 * gl + 1], &hi, 2);
                }
            }
            if (ps.pair_cand || gl == lim - 1) {
                const long long c = t * kCand + cl[rowbase[r] + j];
                if (ps.pair_cand) ps.pair_cand[P + gl] = c;
                if (P + gl == ps.npairs - 1) {
                    if (ps.next_counter) *ps.next_counter = ps.counter + (uint64_t)(c / 2) + 1u;
                    st_relaxed_s32(ps.done, 1);
                }
            }
        }
    }
    return true;
}

}  // namespace nrng
