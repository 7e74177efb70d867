// k_polar.cu -- the Polar method, Algorithm P (paper Sec. 2, steps 1-4),
// with rejection done as a single-pass, order-preserving stream compaction.
//
// The paper vectorises P by generating vectors of (x, y, s), compressing out
// the rejected triples and buffering the variable-length result (Sec. 2's
// vector gather; Sec. 4, RANN3B/RANN3).  Here the compress is a decoupled
// look-back scan over tiles of kPolarCandPerTile candidates (polar_tile in
// tiles.cuh): a persistent CTA takes the next tile id from a global counter
// (dynamic ids, so a tile only ever waits on tiles already owned by running
// CTAs); each warp draws its candidates, tests 0 < kx'^2 + ky'^2 < 2^46
// exactly in 64-bit integers, compacts the accepted ones into its own
// shared-memory segment by ballot/popc rank, runs step 4 densely over it and,
// once warp 0 has looked back for the tile's prefix, copies its runs to their
// global positions.  The tile holding the ceil(n/2)-th accepted pair writes
// next_counter and raises `done`, after which CTAs stop taking tiles.
#include <algorithm>

#include "tiles.cuh"

namespace nrng {

template <int MODE, typename T, bool ALIGNED>
__global__ void __launch_bounds__(kPolarThreads, (PolarOccupancy<kPolarThreads, MODE>::kMinBlocks))
k_polar(const PolarParams p)
{
    __shared__ PolarSmem<kPolarThreads, kPolarRows> sm;
    __shared__ long long s_tile;

    PolarStream ps;
    ps.n = p.n;
    ps.npairs = p.npairs;
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
        if (threadIdx.x == 0) {
            long long t = -1;
            if (ld_relaxed_s32(&p.hdr->done) == 0) {
                t = (long long)atomicAdd(&p.hdr->tile_counter, 1ull);
                if (t >= p.tiles_max) t = -1;
            }
            s_tile = t;
        }
        __syncthreads();
        const long long t = s_tile;
        if (t < 0) break;
        const bool ok = polar_tile<kPolarThreads, kPolarRows, MODE, T, ALIGNED>(
            sm, out, ps, p.rk, t, p.hdr, p.spin_limit_ns);
        __syncthreads();
        if (!ok) break;
    }
}

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
    static int occ_aligned = 0, occ_plain = 0;
    int &occ = aligned ? occ_aligned : occ_plain;
    auto kern = aligned ? k_polar<MODE, T, true> : k_polar<MODE, T, false>;
    if (occ == 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kPolarThreads, 0);
        if (e != cudaSuccess) return e;
        occ = std::max(o, 1);
    }
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
