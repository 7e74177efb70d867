// k_paper.cu -- the paper's further methods: Method B3 (Sec. 3), Method P2
// (Sec. 4) and the Ratio method, Algorithm R (Sec. 5).
//
// B3 draws three uniforms per pair (u1, u2, u3), takes u = max(u1, u2)^2 so
// that sqrt(u) = max(u1, u2) needs no square root, evaluates
// sqrt(-ln(1 - u) / u) by the polynomial h(v) for u <= 8/9 (the hardware
// log2 and square root above), and the sine and cosine of 2 pi u3 - pi by Method B2's polynomials
// and double-angle steps.  One thread takes four pairs: twelve words, three
// Philox blocks, eight outputs.  The paper gathers the u > 8/9 cases into a
// list vector; here they are a divergent branch within the warp.
//
// P2 and R run on the rejection tile of tiles.cuh (per-warp compaction and a
// decoupled look-back), with P2's step 4a and R's accept test and step 4.
#include <algorithm>

#include "b3_pair.cuh"
#include "tiles.cuh"

namespace nrng {

constexpr int kB3Threads = 256;

template <typename T, bool ALIGNED>
__global__ void __launch_bounds__(kB3Threads)
k_b3(T *__restrict__ out, int64_t n, int64_t ngroups, float mu, float sigma, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kB3Threads;
    for (int64_t g = (int64_t)blockIdx.x * kB3Threads + threadIdx.x; g < ngroups; g += stride) {
        const uint64_t b = counter + 3 * (uint64_t)g;
        const uint4 A = philox_block(b, rk), B = philox_block(b + 1, rk), C = philox_block(b + 2, rk);
        float v[8];
        b3_pair(A.x, A.y, A.z, mu, sigma, v[0], v[1]);
        b3_pair(A.w, B.x, B.y, mu, sigma, v[2], v[3]);
        b3_pair(B.z, B.w, C.x, mu, sigma, v[4], v[5]);
        b3_pair(C.y, C.z, C.w, mu, sigma, v[6], v[7]);
        const int64_t i = 8 * g;
        if (ALIGNED && i + 8 <= n) {
            store4_aligned(out + i, v[0], v[1], v[2], v[3]);
            store4_aligned(out + i + 4, v[4], v[5], v[6], v[7]);
        } else {
            for (int q = 0; q < 8 && i + q < n; ++q) store1(out + i + q, v[q]);
        }
    }
}

cudaError_t launch_b3(void *out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter, int dtype,
                      bool aligned, cudaStream_t s)
{
    const int64_t ngroups = (n + 7) / 8;
    const RoundKeys rk = round_keys(key);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ngroups + kB3Threads - 1) / kB3Threads,
                                                                 (int64_t)sm_count() * (2048 / kB3Threads)));
#define NRNG_B3_LAUNCH(TYPE)                                                                                      \
    (aligned ? (k_b3<TYPE, true><<<grid, kB3Threads, 0, s>>>((TYPE *)out, n, ngroups, mu, sigma, counter, rk)) \
             : (k_b3<TYPE, false><<<grid, kB3Threads, 0, s>>>((TYPE *)out, n, ngroups, mu, sigma, counter, rk)))
    switch (dtype) {
    case NRNG_F32: NRNG_B3_LAUNCH(float); break;
    case NRNG_BF16: NRNG_B3_LAUNCH(__nv_bfloat16); break;
    default: NRNG_B3_LAUNCH(__half); break;
    }
#undef NRNG_B3_LAUNCH
    return cudaGetLastError();
}

// --------------------------------------------------------------- P2 and R --
template <class Policy, typename T>
static cudaError_t reject_launch_t(const PolarParams &p, bool aligned, cudaStream_t s)
{
    static std::atomic<int> occ_a{0}, occ_p{0};
    const bool cf = reject_carry_free(p.counter, p.tiles_max, kPolarThreads * Policy::kRows);
    auto kern = aligned ? (cf ? k_reject<Policy, T, true, false> : k_reject<Policy, T, true, true>)
                        : (cf ? k_reject<Policy, T, false, false> : k_reject<Policy, T, false, true>);
    int occ = 0;
    const cudaError_t e = cached_occupancy(aligned ? occ_a : occ_p, kern, kPolarThreads, occ);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>((int64_t)sm_count() * occ, p.tiles_max);
    kern<<<(int)grid, kPolarThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <class Policy>
static cudaError_t reject_launch(const PolarParams &p, int dtype, bool aligned, size_t ws_used, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.hdr, 0, ws_used, s);
    if (e != cudaSuccess) return e;
    switch (dtype) {
    case NRNG_F32: return reject_launch_t<Policy, float>(p, aligned, s);
    case NRNG_BF16: return reject_launch_t<Policy, __nv_bfloat16>(p, aligned, s);
    default: return reject_launch_t<Policy, __half>(p, aligned, s);
    }
}

cudaError_t launch_polar_p2(const PolarParams &p, int dtype, bool aligned, cudaStream_t s)
{
    return reject_launch<P2Policy>(p, dtype, aligned, polar_workspace_bytes(p.n), s);
}

int64_t ratio_tiles_max(int64_t n)
{
    return ratio_tiles_for(n, kRatioCandPerTile);
}

size_t ratio_workspace_bytes(int64_t n)
{
    const size_t bytes = sizeof(WsHeader) + (size_t)ratio_tiles_max(n) * sizeof(unsigned long long);
    return (bytes + 255) / 256 * 256;
}

cudaError_t launch_ratio(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s)
{
    if (mode == kModeFast)
        return reject_launch<RatioPolicy<kModeFast>>(p, dtype, aligned, ratio_workspace_bytes(p.n), s);
    return reject_launch<RatioPolicy<kModeAccurate>>(p, dtype, aligned, ratio_workspace_bytes(p.n), s);
}

}  // namespace nrng
