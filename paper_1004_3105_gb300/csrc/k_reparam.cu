// k_reparam.cu -- the reparameterised sample x = mu + sigma z and its
// gradients (an add-on with no counterpart in the paper).  z is element i of
// the B1 stream (paper Sec. 2, Algorithm B1, with mu = 0 and sigma = 1) drawn
// from (key, counter); the backward pass regenerates z from the same counter
// instead of reading a saved tensor, so forward and backward see bitwise
// identical z.
//
// Element i uses parameter p(i) = (i / inner) mod m.  The elementwise case
// (m = n) streams 12 bytes per element forward (read mu, sigma, write x) and
// 8-12 backward (read g, write dsigma and optionally dmu = g); the broadcast
// cases reduce with float atomics after a per-thread pre-sum.
#include <algorithm>

#include "nrng_device.cuh"

namespace nrng {

constexpr int kRepThreads = 256;

static int rep_grid(int64_t nblocks)
{
    const int64_t ctas = (nblocks + kRepThreads - 1) / kRepThreads;
    const int64_t resident = (int64_t)sm_count() * (2048 / kRepThreads);
    return (int)std::max<int64_t>(1, std::min(ctas, resident));
}

// Four standard normals z[4b .. 4b+3] of block b (B1 with mu = 0, sigma = 1).
template <int MODE>
__device__ __forceinline__ float4 b1_block_z(uint64_t counter_plus_b, const RoundKeys &rk)
{
    return b1_block<MODE>(philox_block(counter_plus_b, rk), radius_coef(0.0f, 1.0f), kSinCos1024);
}

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Elementwise forward, all of x, mu, sigma 16-byte aligned.
template <int MODE>
__global__ void __launch_bounds__(kRepThreads)
k_reparam_fwd_elem(float *__restrict__ x, const float *__restrict__ mu, const float *__restrict__ sigma,
                   int64_t n, int64_t nblocks, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kRepThreads;
    for (int64_t b = (int64_t)blockIdx.x * kRepThreads + threadIdx.x; b < nblocks; b += stride) {
        const float4 z = b1_block_z<MODE>(counter + (uint64_t)b, rk);
        const int64_t i = 4 * b;
        if (i + 4 <= n) {
            const float4 m = __ldcs(reinterpret_cast<const float4 *>(mu + i));
            const float4 s = __ldcs(reinterpret_cast<const float4 *>(sigma + i));
            __stcs(reinterpret_cast<float4 *>(x + i),
                   make_float4(fmaf(s.x, z.x, m.x), fmaf(s.y, z.y, m.y), fmaf(s.z, z.z, m.z),
                               fmaf(s.w, z.w, m.w)));
        } else {
            for (int j = 0; j < 4 && i + j < n; ++j) x[i + j] = fmaf(sigma[i + j], comp(z, j), mu[i + j]);
        }
    }
}

// Any (m, inner), any 4-byte alignment.
template <int MODE>
__global__ void __launch_bounds__(kRepThreads)
k_reparam_fwd_bcast(float *__restrict__ x, const float *__restrict__ mu, const float *__restrict__ sigma,
                    int64_t n, int64_t nblocks, int64_t m, int64_t inner, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kRepThreads;
    for (int64_t b = (int64_t)blockIdx.x * kRepThreads + threadIdx.x; b < nblocks; b += stride) {
        const float4 z = b1_block_z<MODE>(counter + (uint64_t)b, rk);
        const int64_t i = 4 * b;
        for (int j = 0; j < 4 && i + j < n; ++j) {
            const int64_t q = ((i + j) / inner) % m;
            x[i + j] = fmaf(sigma[q], comp(z, j), mu[q]);
        }
    }
}

// Elementwise backward: dsigma = g z, dmu = g (when requested).
template <int MODE>
__global__ void __launch_bounds__(kRepThreads)
k_reparam_bwd_elem(float *__restrict__ dmu, float *__restrict__ dsigma, const float *__restrict__ g,
                   int64_t n, int64_t nblocks, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kRepThreads;
    for (int64_t b = (int64_t)blockIdx.x * kRepThreads + threadIdx.x; b < nblocks; b += stride) {
        const float4 z = b1_block_z<MODE>(counter + (uint64_t)b, rk);
        const int64_t i = 4 * b;
        if (i + 4 <= n) {
            const float4 gv = __ldcs(reinterpret_cast<const float4 *>(g + i));
            __stcs(reinterpret_cast<float4 *>(dsigma + i),
                   make_float4(gv.x * z.x, gv.y * z.y, gv.z * z.z, gv.w * z.w));
            if (dmu) __stcs(reinterpret_cast<float4 *>(dmu + i), gv);
        } else {
            for (int j = 0; j < 4 && i + j < n; ++j) {
                dsigma[i + j] = g[i + j] * comp(z, j);
                if (dmu) dmu[i + j] = g[i + j];
            }
        }
    }
}

// Broadcast backward: per-thread sums over runs of equal p, then one atomic
// per run.  dmu/dsigma are zeroed by the launcher first.
template <int MODE>
__global__ void __launch_bounds__(kRepThreads)
k_reparam_bwd_bcast(float *__restrict__ dmu, float *__restrict__ dsigma, const float *__restrict__ g,
                    int64_t n, int64_t nblocks, int64_t m, int64_t inner, uint64_t counter, const RoundKeys rk)
{
    const int64_t stride = (int64_t)gridDim.x * kRepThreads;
    int64_t cur = -1;
    float acc_s = 0.0f, acc_m = 0.0f;
    for (int64_t b = (int64_t)blockIdx.x * kRepThreads + threadIdx.x; b < nblocks; b += stride) {
        const float4 z = b1_block_z<MODE>(counter + (uint64_t)b, rk);
        const int64_t i = 4 * b;
        for (int j = 0; j < 4 && i + j < n; ++j) {
            const int64_t q = ((i + j) / inner) % m;
            if (q != cur) {
                if (cur >= 0) {
                    atomicAdd(dsigma + cur, acc_s);
                    if (dmu) atomicAdd(dmu + cur, acc_m);
                }
                cur = q;
                acc_s = 0.0f;
                acc_m = 0.0f;
            }
            const float gv = g[i + j];
            acc_s = fmaf(gv, comp(z, j), acc_s);
            acc_m += gv;
        }
    }
    // Final flush: when every lane of the warp holds the same parameter (the
    // scalar case, or a broadcast axis longer than the warp's span), reduce in
    // registers and issue one atomic per warp.
    const long long c0 = __shfl_sync(0xFFFFFFFFu, (long long)cur, 0);
    if (__all_sync(0xFFFFFFFFu, cur == c0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_s += __shfl_xor_sync(0xFFFFFFFFu, acc_s, o);
            acc_m += __shfl_xor_sync(0xFFFFFFFFu, acc_m, o);
        }
        if ((threadIdx.x & 31) == 0 && cur >= 0) {
            atomicAdd(dsigma + cur, acc_s);
            if (dmu) atomicAdd(dmu + cur, acc_m);
        }
    } else if (cur >= 0) {
        atomicAdd(dsigma + cur, acc_s);
        if (dmu) atomicAdd(dmu + cur, acc_m);
    }
}

static bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

cudaError_t launch_reparam_fwd(float *x, const float *mu, const float *sigma, int64_t n, int64_t m,
                               int64_t inner, uint64_t key, uint64_t counter, int mode, cudaStream_t s)
{
    const int64_t nblocks = (n + 3) / 4;
    const RoundKeys rk = round_keys(key);
    const int grid = rep_grid(nblocks);
    const bool elem = (m == n) && aligned16(x) && aligned16(mu) && aligned16(sigma);
    if (mode == kModeFast) {
        if (elem) k_reparam_fwd_elem<kModeFast><<<grid, kRepThreads, 0, s>>>(x, mu, sigma, n, nblocks, counter, rk);
        else k_reparam_fwd_bcast<kModeFast><<<grid, kRepThreads, 0, s>>>(x, mu, sigma, n, nblocks, m, inner, counter, rk);
    } else {
        if (elem) k_reparam_fwd_elem<kModeAccurate><<<grid, kRepThreads, 0, s>>>(x, mu, sigma, n, nblocks, counter, rk);
        else k_reparam_fwd_bcast<kModeAccurate><<<grid, kRepThreads, 0, s>>>(x, mu, sigma, n, nblocks, m, inner, counter, rk);
    }
    return cudaGetLastError();
}

cudaError_t launch_reparam_bwd(float *dmu, float *dsigma, const float *g, int64_t n, int64_t m,
                               int64_t inner, uint64_t key, uint64_t counter, int mode, cudaStream_t s)
{
    const int64_t nblocks = (n + 3) / 4;
    const RoundKeys rk = round_keys(key);
    const bool elem = (m == n) && aligned16(g) && aligned16(dsigma) && (dmu == nullptr || aligned16(dmu));
    if (elem) {
        const int grid = rep_grid(nblocks);
        if (mode == kModeFast) k_reparam_bwd_elem<kModeFast><<<grid, kRepThreads, 0, s>>>(dmu, dsigma, g, n, nblocks, counter, rk);
        else k_reparam_bwd_elem<kModeAccurate><<<grid, kRepThreads, 0, s>>>(dmu, dsigma, g, n, nblocks, counter, rk);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(dsigma, 0, (size_t)m * sizeof(float), s);
    if (e == cudaSuccess && dmu) e = cudaMemsetAsync(dmu, 0, (size_t)m * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const int grid = rep_grid(nblocks);
    if (mode == kModeFast) k_reparam_bwd_bcast<kModeFast><<<grid, kRepThreads, 0, s>>>(dmu, dsigma, g, n, nblocks, m, inner, counter, rk);
    else k_reparam_bwd_bcast<kModeAccurate><<<grid, kRepThreads, 0, s>>>(dmu, dsigma, g, n, nblocks, m, inner, counter, rk);
    return cudaGetLastError();
}

}  // namespace nrng
