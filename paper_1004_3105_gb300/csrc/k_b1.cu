// k_b1.cu -- uniforms and Box-Muller Algorithm B1 (paper Sec. 2, steps 1-3).
//
// One thread takes one Philox block at a time (grid-stride): four 32-bit
// words give two (u, v) pairs and four outputs, stored with one 16-byte
// (fp32) or 8-byte (bf16/fp16) streaming store.  The only loads are the
// accurate path's 16 KB sin/cos table, copied to shared memory once per CTA.
// The kernel is bound by the HBM write stream or by instruction dispatch
// (Philox's 32x32->64 products and the transform), whichever is tighter.
#include <algorithm>
#include <atomic>

#include "nrng_device.cuh"

namespace nrng {

constexpr int kB1Threads = 512;

template <bool ALIGNED>
__global__ void __launch_bounds__(kB1Threads)
k_uniform(float *__restrict__ out, int64_t n, int64_t nblocks, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kB1Threads;
    for (int64_t b = (int64_t)blockIdx.x * kB1Threads + threadIdx.x; b < nblocks; b += stride) {
        const uint4 w = philox_block(counter + (uint64_t)b, rk);
        const float a = u24(w.x), c = u24(w.y), d = u24(w.z), e = u24(w.w);
        const int64_t i = 4 * b;
        if (ALIGNED && i + 4 <= n) {
            store4_aligned(out + i, a, c, d, e);
        } else {
            if (i < n) out[i] = a;
            if (i + 1 < n) out[i + 1] = c;
            if (i + 2 < n) out[i + 2] = d;
            if (i + 3 < n) out[i + 3] = e;
        }
    }
}

// Any n, any element alignment: the general kernel.
template <int MODE, typename T, bool ALIGNED>
__global__ void __launch_bounds__(kB1Threads)
k_b1(T *__restrict__ out, int64_t n, int64_t nblocks, float mu, float sigma, uint64_t counter,
     const RoundKeys rk)
{
    __shared__ float4 s_tab[MODE == kModeAccurate ? 1024 : 1];
    const float4 *tab = b1_table_to_shared<MODE>(s_tab);
    const RadiusCoef cf = radius_coef(mu, sigma);
    const int64_t stride = (int64_t)gridDim.x * kB1Threads;
    for (int64_t b = (int64_t)blockIdx.x * kB1Threads + threadIdx.x; b < nblocks; b += stride) {
        const float4 o = b1_block<MODE>(philox_block(counter + (uint64_t)b, rk), cf, tab);
        const int64_t i = 4 * b;
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

// The common case: output aligned to 4 elements and fewer than 2^32 blocks.
// The loop runs over whole blocks only, with 32-bit indices; the last,
// partial block (n mod 4 outputs) is done by one thread after it.  With
// CARRY false the low counter word does not wrap over the launch (c_lo plus
// the blocks stays below 2^32), so the high word is the launch constant c_hi:
// the first two Philox rounds then partly fold into launch constants.
template <int MODE, typename T, bool CARRY>
__global__ void __launch_bounds__(kB1Threads)
k_b1_whole(T *__restrict__ out, int64_t n, uint32_t nwhole, float mu, float sigma, uint32_t c_lo,
           uint32_t c_hi, const RoundKeys rk)
{
    __shared__ float4 s_tab[MODE == kModeAccurate ? 1024 : 1];
    const float4 *tab = b1_table_to_shared<MODE>(s_tab);
    const RadiusCoef cf = radius_coef(mu, sigma);
    const uint32_t stride = gridDim.x * kB1Threads;
    // Two blocks per iteration (b and b + stride): their Philox chains are
    // independent, so one fills the other's dependency stalls.
    uint32_t b = blockIdx.x * kB1Threads + threadIdx.x;
    for (; b + stride < nwhole; b += 2 * stride) {
        const uint32_t b2 = b + stride;
        const uint32_t lo = c_lo + b, lo2 = c_lo + b2;
        const uint32_t hi = CARRY ? c_hi + (lo < b ? 1u : 0u) : c_hi;
        const uint32_t hi2 = CARRY ? c_hi + (lo2 < b2 ? 1u : 0u) : c_hi;
        float4 o, o2;
        b1_block2<MODE>(philox4x32_10(lo, hi, rk), philox4x32_10(lo2, hi2, rk), cf, tab, o, o2);
        store4_aligned(out + 4 * (size_t)b, o.x, o.y, o.z, o.w);
        store4_aligned(out + 4 * (size_t)b2, o2.x, o2.y, o2.z, o2.w);
    }
    if (b < nwhole) {
        const uint32_t lo = c_lo + b;
        const uint32_t hi = CARRY ? c_hi + (lo < b ? 1u : 0u) : c_hi;
        const float4 o = b1_block<MODE>(philox4x32_10(lo, hi, rk), cf, tab);
        store4_aligned(out + 4 * (size_t)b, o.x, o.y, o.z, o.w);
    }
    if ((n & 3) && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t c = ((uint64_t)c_hi << 32 | c_lo) + nwhole;
        const float4 o = b1_block<MODE>(philox_block(c, rk), cf, tab);
        const float v[4] = {o.x, o.y, o.z, o.w};
        const int64_t i = 4 * (int64_t)nwhole;
        for (int q = 0; q < 4 && i + q < n; ++q) store1(out + i + q, v[q]);
    }
}

// Philox4x32-10 alone: every block of [counter, counter + nblocks) drawn and
// folded into one word by xor, with no stores but one atomic per warp.  Its
// time is the rate at which this GPU draws Philox blocks, the instruction
// ceiling of every generator here (Philox's twenty 32x32->64 products and
// twenty three-input xors a block).  Two independent blocks per iteration, as
// in the B1 kernel; the low counter word must not wrap over the launch.
__global__ void __launch_bounds__(kB1Threads)
k_philox_ceiling(uint32_t *__restrict__ out, uint32_t nblocks, uint32_t c_lo, uint32_t c_hi, const RoundKeys rk)
{
    const uint32_t stride = gridDim.x * kB1Threads;
    uint32_t acc = 0;
    uint32_t b = blockIdx.x * kB1Threads + threadIdx.x;
    for (; b + stride < nblocks; b += 2 * stride) {
        const uint4 w = philox4x32_10(c_lo + b, c_hi, rk);
        const uint4 w2 = philox4x32_10(c_lo + b + stride, c_hi, rk);
        acc ^= w.x ^ w.y ^ w.z ^ w.w ^ w2.x ^ w2.y ^ w2.z ^ w2.w;
    }
    if (b < nblocks) {
        const uint4 w = philox4x32_10(c_lo + b, c_hi, rk);
        acc ^= w.x ^ w.y ^ w.z ^ w.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(out, acc);
}

// Grid: enough CTAs to fill every SM at full occupancy, grid-striding over
// the blocks beyond that (the kernel holds no state between blocks).
static int b1_grid(int64_t nblocks)
{
    const int64_t ctas = (nblocks + kB1Threads - 1) / kB1Threads;
    const int64_t resident = (int64_t)sm_count() * (2048 / kB1Threads);
    return (int)std::max<int64_t>(1, std::min(ctas, resident));
}

cudaError_t launch_philox_ceiling(uint32_t *out, int64_t nblocks, uint64_t key, uint64_t counter, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_philox_ceiling<<<b1_grid(nblocks), kB1Threads, 0, s>>>(out, (uint32_t)nblocks, (uint32_t)counter,
                                                            (uint32_t)(counter >> 32), round_keys(key));
    return cudaGetLastError();
}

cudaError_t launch_uniform(float *out, int64_t n, uint64_t key, uint64_t counter, cudaStream_t s)
{
    const int64_t nblocks = (n + 3) / 4;
    const RoundKeys rk = round_keys(key);
    const bool aligned = ((uintptr_t)out % 16) == 0;
    if (aligned)
        k_uniform<true><<<b1_grid(nblocks), kB1Threads, 0, s>>>(out, n, nblocks, counter, rk);
    else
        k_uniform<false><<<b1_grid(nblocks), kB1Threads, 0, s>>>(out, n, nblocks, counter, rk);
    return cudaGetLastError();
}

template <int MODE, typename T>
static cudaError_t b1_dispatch_aligned(void *out, int64_t n, int64_t nblocks, float mu, float sigma,
                                uint64_t counter, const RoundKeys &rk, bool aligned, cudaStream_t s)
{
    // the whole-block kernel's grid: its resident CTAs on every SM (no
    // partial second wave), grid-striding beyond
    static std::atomic<int> occ_slot{0};
    int occ = 0;
    const cudaError_t e = cached_occupancy(occ_slot, k_b1_whole<MODE, T, false>, kB1Threads, occ);
    if (e != cudaSuccess) return e;
    const int grid_whole = (int)std::max<int64_t>(
        1, std::min<int64_t>((nblocks + kB1Threads - 1) / kB1Threads, (int64_t)sm_count() * occ));
    const int grid = b1_grid(nblocks);
    const int64_t nwhole = n / 4;
    // the carry-free form when the low counter word does not wrap over the
    // launch (the whole blocks and the partial one)
    const bool carry_free = (uint64_t)(uint32_t)counter + (uint64_t)nblocks <= (uint64_t(1) << 32);
    if (aligned && nwhole < (int64_t(1) << 32) - 2 * (int64_t)grid_whole * kB1Threads && carry_free)
        k_b1_whole<MODE, T, false><<<grid_whole, kB1Threads, 0, s>>>((T *)out, n, (uint32_t)nwhole, mu, sigma,
                                                                     (uint32_t)counter, (uint32_t)(counter >> 32), rk);
    else if (aligned && nwhole < (int64_t(1) << 32) - 2 * (int64_t)grid_whole * kB1Threads)
        k_b1_whole<MODE, T, true><<<grid_whole, kB1Threads, 0, s>>>((T *)out, n, (uint32_t)nwhole, mu, sigma,
                                                                    (uint32_t)counter, (uint32_t)(counter >> 32), rk);
    else if (aligned)
        k_b1<MODE, T, true><<<grid, kB1Threads, 0, s>>>((T *)out, n, nblocks, mu, sigma, counter, rk);
    else
        k_b1<MODE, T, false><<<grid, kB1Threads, 0, s>>>((T *)out, n, nblocks, mu, sigma, counter, rk);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t b1_dispatch_dtype(void *out, int64_t n, int64_t nblocks, float mu, float sigma,
                                     uint64_t counter, const RoundKeys &rk, int dtype, bool aligned,
                                     cudaStream_t s)
{
    switch (dtype) {
    case NRNG_F32: return b1_dispatch_aligned<MODE, float>(out, n, nblocks, mu, sigma, counter, rk, aligned, s);
    case NRNG_BF16:
        return b1_dispatch_aligned<MODE, __nv_bfloat16>(out, n, nblocks, mu, sigma, counter, rk, aligned, s);
    default: return b1_dispatch_aligned<MODE, __half>(out, n, nblocks, mu, sigma, counter, rk, aligned, s);
    }
}

cudaError_t launch_b1(void *out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                      int dtype, int mode, bool aligned, cudaStream_t s)
{
    const int64_t nblocks = (n + 3) / 4;
    const RoundKeys rk = round_keys(key);
    if (mode == kModeFast) return b1_dispatch_dtype<kModeFast>(out, n, nblocks, mu, sigma, counter, rk, dtype, aligned, s);
    if (mode == kModeB2) return b1_dispatch_dtype<kModeB2>(out, n, nblocks, mu, sigma, counter, rk, dtype, aligned, s);
    return b1_dispatch_dtype<kModeAccurate>(out, n, nblocks, mu, sigma, counter, rk, dtype, aligned, s);
}

}  // namespace nrng
