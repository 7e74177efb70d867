// k_polar.cu -- the Polar method, Algorithm P (paper Sec. 2, steps 1-4),
// with rejection done as a single-pass, order-preserving stream compaction.
//
// The paper vectorises P by generating vectors of (x, y, s), compressing out
// the rejected triples and buffering the variable-length result (Sec. 2's
// vector gather; Sec. 4, RANN3B/RANN3).  Here the compress is a decoupled
// look-back scan over tiles of kPolarCandPerTile candidates (k_reject and
// reject_tile in tiles.cuh, with Algorithm P's policy): a persistent CTA takes the next tile id from a global counter
// (dynamic ids, so a tile only ever waits on tiles already owned by running
// CTAs); each warp draws its contiguous run of candidates, tests
// 0 < kx'^2 + ky'^2 < 2^46 exactly in 64-bit integers, compacts the accepted
// ones into its own shared-memory segment by ballot/popc rank, runs step 4
// densely over it and, once warp 0 has looked back for the tile's prefix,
// copies the segment to its place in the output as one dense run.  The tile holding the ceil(n/2)-th accepted pair writes
// next_counter and raises `done`, after which CTAs stop taking tiles.
#include <algorithm>

#include "tiles.cuh"

namespace nrng {

int64_t polar_tiles_max(int64_t n)
{
    return polar_tiles_for(n, kPolarCandPerTile);
}

size_t polar_workspace_bytes(int64_t n)
{
    const size_t bytes = sizeof(WsHeader) + (size_t)polar_tiles_max(n) * sizeof(unsigned long long);
    return (bytes + 255) / 256 * 256;
}

template <int MODE, typename T>
static cudaError_t polar_launch_t(const PolarParams &p, bool aligned, cudaStream_t s)
{
    static std::atomic<int> occ_aligned{0}, occ_plain{0};
    const bool cf = reject_carry_free(p.counter, p.tiles_max, kPolarBlocksPerTile);
    auto kern = aligned ? (cf ? k_reject<PolarPolicy<MODE>, T, true, false> : k_reject<PolarPolicy<MODE>, T, true, true>)
                        : (cf ? k_reject<PolarPolicy<MODE>, T, false, false> : k_reject<PolarPolicy<MODE>, T, false, true>);
    int occ = 0;
    const cudaError_t e = cached_occupancy(aligned ? occ_aligned : occ_plain, kern, kPolarThreads, occ);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>((int64_t)sm_count() * occ, p.tiles_max);
    kern<<<(int)grid, kPolarThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t polar_launch_dtype(const PolarParams &p, int dtype, bool aligned, cudaStream_t s)
{
    switch (dtype) {
    case NRNG_F32: return polar_launch_t<MODE, float>(p, aligned, s);
    case NRNG_BF16: return polar_launch_t<MODE, __nv_bfloat16>(p, aligned, s);
    default: return polar_launch_t<MODE, __half>(p, aligned, s);
    }
}

// ------------------------------------------------------------ two-pass ----
// The same compaction without a look-back: a count pass draws every tile's
// candidates and counts the accepted ones, a one-CTA scan turns the counts
// into exclusive prefixes, and a write pass draws each tile again and places
// its pairs at the known prefix.  Its output equals the single-pass output
// bit for bit; it trades a second Philox evaluation of every candidate for
// the look-back's waits (an ablation of the single-pass design).
constexpr int kCountThreads = kPolarThreads;

__global__ void __launch_bounds__(kCountThreads)
k_polar_count(uint64_t counter, const RoundKeys rk, int64_t tiles, int *__restrict__ counts)
{
    __shared__ int s_warp[kCountThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t b0 = counter + (uint64_t)t * kPolarBlocksPerTile + threadIdx.x;
        int c = 0;
#pragma unroll 4
        for (int r = 0; r < kPolarRows; ++r) {
            const uint4 w = philox_block(b0 + (uint64_t)(r * kPolarThreads), rk);
            int64_t S0, S1;
            c += polar_accept(k24(w.x), k24(w.y), S0) ? 1 : 0;
            c += polar_accept(k24(w.z), k24(w.w), S1) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) s_warp[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int sum = 0;
            for (int q = 0; q < kCountThreads / 32; ++q) sum += s_warp[q];
            counts[t] = sum;
        }
        __syncthreads();
    }
}

// Exclusive scan of the tile counts (one CTA); prefix[tiles] is the total.
// A total short of nitems means the tile budget ran out: NRNG_ERR_EXHAUSTED.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
k_polar_scan(const int *__restrict__ counts, long long *__restrict__ prefix, int64_t tiles, int64_t nitems,
             WsHeader *hdr)
{
    __shared__ long long s_warp[kScanThreads / 32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < tiles; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const long long v = (i < tiles) ? counts[i] : 0;
        long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const long long wv = s_warp[lane];
            long long wi = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            s_warp[lane] = wi - wv;
        }
        __syncthreads();
        const long long carry = s_carry;
        if (i < tiles) prefix[i] = carry + s_warp[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + s_warp[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[tiles] = s_carry;
        if (s_carry < nitems) raise_error(hdr, kStatusExhausted);
    }
}

template <int MODE, typename T, bool ALIGNED>
__global__ void __launch_bounds__(kPolarThreads, (RejOccupancy<kRejWarps, kPolarRows>::kMinBlocks))
k_polar_write(const PolarParams p, const long long *__restrict__ prefix)
{
    __shared__ RejSmem<kRejWarps, kPolarRows> sm;
    const RadiusCoef cf = radius_coef(p.mu, p.sigma);
    PolarStream ps;
    ps.n = p.n;
    ps.nitems = p.nitems;
    ps.counter = p.counter;
    ps.status = nullptr;
    ps.tiles_max = p.tiles_max;
    ps.done = &p.hdr->done;
    ps.next_counter = p.next_counter;
    ps.pair_cand = p.pair_cand;
    ps.silent_tile = -1;
    T *out = static_cast<T *>(p.out);
    if (prefix[p.tiles_max] < p.nitems) return;   // the scan recorded NRNG_ERR_EXHAUSTED
    for (int64_t t = blockIdx.x; t < p.tiles_max; t += gridDim.x) {
        const long long P = prefix[t];   // same value for every thread of the CTA
        if (P >= p.nitems) break;        // prefixes only grow with t
        reject_tile<PolarPolicy<MODE>, kRejWarps, kPolarRows, T, ALIGNED, true, RoundKeys, true>(sm, out, ps, p.rk, cf, t,
                                                                                            p.hdr, p.spin_limit_ns, P);
        __syncthreads();
    }
}

size_t polar_twopass_workspace_bytes(int64_t n)
{
    const int64_t tiles = polar_tiles_max(n);
    const size_t counts = ((size_t)tiles * 4 + 255) / 256 * 256;
    return sizeof(WsHeader) + 192 + counts + (size_t)(tiles + 1) * 8;
}

template <int MODE, typename T>
static cudaError_t polar_twopass_t(const PolarParams &p, bool aligned, cudaStream_t s)
{
    char *w = reinterpret_cast<char *>(p.hdr);
    int *counts = reinterpret_cast<int *>(w + sizeof(WsHeader) + 192);
    long long *prefix = reinterpret_cast<long long *>(
        w + sizeof(WsHeader) + 192 + ((size_t)p.tiles_max * 4 + 255) / 256 * 256);
    const int64_t grid_c = std::min<int64_t>((int64_t)sm_count() * 8, p.tiles_max);
    k_polar_count<<<(int)grid_c, kCountThreads, 0, s>>>(p.counter, p.rk, p.tiles_max, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_polar_scan<<<1, kScanThreads, 0, s>>>(counts, prefix, p.tiles_max, p.nitems, p.hdr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static std::atomic<int> occ_a{0}, occ_p{0};
    auto kern = aligned ? k_polar_write<MODE, T, true> : k_polar_write<MODE, T, false>;
    int occ = 0;
    e = cached_occupancy(aligned ? occ_a : occ_p, kern, kPolarThreads, occ);
    if (e != cudaSuccess) return e;
    // tiles beyond the crossing one are skipped, so size the grid to the
    // expected number of tiles, not the budget
    const int64_t expect = (p.nitems * 100) / ((int64_t)kPolarCandPerTile * 78) + 2;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * occ, expect));
    kern<<<(int)grid, kPolarThreads, 0, s>>>(p, prefix);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t polar_twopass_dtype(const PolarParams &p, int dtype, bool aligned, cudaStream_t s)
{
    switch (dtype) {
    case NRNG_F32: return polar_twopass_t<MODE, float>(p, aligned, s);
    case NRNG_BF16: return polar_twopass_t<MODE, __nv_bfloat16>(p, aligned, s);
    default: return polar_twopass_t<MODE, __half>(p, aligned, s);
    }
}

cudaError_t launch_polar_twopass(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.hdr, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) return e;
    if (mode == kModeFast) return polar_twopass_dtype<kModeFast>(p, dtype, aligned, s);
    return polar_twopass_dtype<kModeAccurate>(p, dtype, aligned, s);
}

__global__ void k_set_u64(uint64_t *p, uint64_t v) { *p = v; }

cudaError_t launch_set_u64(uint64_t *p, uint64_t v, cudaStream_t s)
{
    k_set_u64<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_polar(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.hdr, 0, polar_workspace_bytes(p.n), s);
    if (e != cudaSuccess) return e;
    if (mode == kModeFast) return polar_launch_dtype<kModeFast>(p, dtype, aligned, s);
    return polar_launch_dtype<kModeAccurate>(p, dtype, aligned, s);
}

}  // namespace nrng
