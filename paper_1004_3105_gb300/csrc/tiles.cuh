// tiles.cuh -- one tile of a B1 stream and one tile of a Polar stream, as
// device functions shared by the single-stream and the batched kernels.
#pragma once

#include "nrng_device.cuh"

namespace nrng {

// ----------------------------------------------------------- B1 tile ------
// Blocks [t*TB, (t+1)*TB) of a stream, TB = THREADS * BPT; block b writes
// out[4b .. 4b+3] (Algorithm B1, two pairs per block).
template <int THREADS, int BPT, int MODE, typename T, bool ALIGNED>
__device__ __forceinline__ void b1_tile(T *__restrict__ out, int64_t n, float mu, float sigma,
                                        const RoundKeys &rk, uint64_t counter, int64_t t)
{
    const int64_t nblocks = (n + 3) / 4;
#pragma unroll
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

// --------------------------------------------------------- Polar tile -----
template <int THREADS, int ROWS>
struct PolarSmem {
    static constexpr int kCand = 2 * THREADS * ROWS;
    static constexpr int kEntries = ROWS * (THREADS / 32);   // (row, warp) counts
    int2 pts[kCand];
    uint16_t cl[kCand];
    int off[kEntries];
    long long prefix;
    int total;
};

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

// Tile t of a Polar stream (Algorithm P, steps 1-4, with the compress done as
// a decoupled look-back scan; see k_polar.cu).  Returns false when the
// look-back gave up (error recorded in hdr), true otherwise.
template <int THREADS, int ROWS, int MODE, typename T, bool ALIGNED>
__device__ __forceinline__ bool polar_tile(PolarSmem<THREADS, ROWS> &sm, T *__restrict__ out,
                                           const PolarStream &ps, const RoundKeys &rk, int64_t t,
                                           WsHeader *hdr, unsigned long long limit_ns)
{
    constexpr int kWarps = THREADS / 32;
    constexpr int kEntries = PolarSmem<THREADS, ROWS>::kEntries;
    constexpr int kCand = PolarSmem<THREADS, ROWS>::kCand;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Steps 1-3: draw, test exactly, rank accepted candidates in the warp.
    int32_t kx[ROWS][2], ky[ROWS][2];
    bool acc[ROWS][2];
    int rank[ROWS];
    const uint64_t b0 = ps.counter + (uint64_t)t * (THREADS * ROWS) + (uint64_t)tid;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint4 w = philox_block(b0 + (uint64_t)(r * THREADS), rk);
        kx[r][0] = k24(w.x);
        ky[r][0] = k24(w.y);
        kx[r][1] = k24(w.z);
        ky[r][1] = k24(w.w);
        int64_t S;
        acc[r][0] = polar_accept(kx[r][0], ky[r][0], S);
        acc[r][1] = polar_accept(kx[r][1], ky[r][1], S);
        const unsigned m0 = __ballot_sync(0xFFFFFFFFu, acc[r][0]);
        const unsigned m1 = __ballot_sync(0xFFFFFFFFu, acc[r][1]);
        rank[r] = __popc(m0 & lt) + __popc(m1 & lt);
        if (lane == 0) sm.off[r * kWarps + warp] = __popc(m0) + __popc(m1);
    }
    __syncthreads();

    // Exclusive scan of the (row, warp) counts and the look-back, by warp 0.
    if (warp == 0) {
        int carry = 0;
#pragma unroll
        for (int c0 = 0; c0 < kEntries; c0 += 32) {
            const int v = (c0 + lane < kEntries) ? sm.off[c0 + lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (c0 + lane < kEntries) sm.off[c0 + lane] = carry + incl - v;
            carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        const long long P = (t == ps.silent_tile)
                                ? lookback_warp(ps.status, t, carry, hdr, limit_ns, false, false)
                                : lookback_warp(ps.status, t, carry, hdr, limit_ns);
        if (lane == 0) {
            sm.prefix = P;
            sm.total = carry;
            if (P >= 0 && t == ps.tiles_max - 1 && P + carry < ps.npairs)
                raise_error(hdr, kStatusExhausted);
        }
    }
    __syncthreads();
    const long long P = sm.prefix;
    if (P < 0) return false;
    if (P >= ps.npairs) return true;

    // Stage accepted points in candidate order (row, warp, lane, half).
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int base = sm.off[r * kWarps + warp] + rank[r];
        const uint16_t cl = (uint16_t)(2 * (r * THREADS + tid));
        if (acc[r][0]) {
            sm.pts[base] = make_int2(kx[r][0], ky[r][0]);
            sm.cl[base] = cl;
        }
        if (acc[r][1]) {
            const int q = base + (acc[r][0] ? 1 : 0);
            sm.pts[q] = make_int2(kx[r][1], ky[r][1]);
            sm.cl[q] = (uint16_t)(cl + 1);
        }
    }
    __syncthreads();

    // Step 4 on a dense run of accepted points; pair g goes to 2g, 2g + 1.
    const long long remaining = ps.npairs - P;
    const int cnt = (remaining < (long long)sm.total) ? (int)remaining : sm.total;
    for (int j = tid; j < cnt; j += THREADS) {
        const int2 k = sm.pts[j];
        float zx, zy;
        polar_pair<MODE>(k.x, k.y, ps.mu, ps.sigma, zx, zy);
        const long long g = P + j;
        const long long e = 2 * g;
        if (ALIGNED && e + 1 < ps.n) {
            store2_aligned(out + e, zx, zy);
        } else {
            store1(out + e, zx);
            if (e + 1 < ps.n) store1(out + e + 1, zy);
        }
        if (ps.pair_cand || g == ps.npairs - 1) {
            const long long c = t * kCand + sm.cl[j];
            if (ps.pair_cand) ps.pair_cand[g] = c;
            if (g == ps.npairs - 1) {
                if (ps.next_counter) *ps.next_counter = ps.counter + (uint64_t)(c / 2) + 1u;
                st_relaxed_s32(ps.done, 1);
            }
        }
    }
    return true;
}

}  // namespace nrng
