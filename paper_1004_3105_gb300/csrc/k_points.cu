// k_points.cu -- the per-pair transforms at caller-given lattice points
// (nrng_eval_points), so that tests can reach the special points of the
// lattice (s -> 1, S = 1, u = 0, u = 1 - 2^-24, the quadrant angles) that a
// stream reaches too rarely to test.  The kernels call the same device
// functions as the generators: b1_pair (Algorithm B1, Sec. 2, steps 2-3)
// and polar_accept / polar_pair (Algorithm P, steps 3-4).
#include <algorithm>

#include "nrng_device.cuh"

namespace nrng {

constexpr int kPointThreads = 256;

// kind 0: in[2i], in[2i+1] are the words (wu, wv) of a B1 pair.
// kind 1: in[2i], in[2i+1] are the lattice coordinates (kx', ky') of a Polar
//         candidate; accept[i] is step 3's decision, out holds step 4's values
//         (meaningless where the candidate is rejected).
template <int MODE>
__global__ void __launch_bounds__(kPointThreads)
k_eval_points(int kind, const uint32_t *__restrict__ in, int64_t n, float mu, float sigma,
              float *__restrict__ out, int32_t *__restrict__ accept)
{
    const int64_t stride = (int64_t)gridDim.x * kPointThreads;
    for (int64_t i = (int64_t)blockIdx.x * kPointThreads + threadIdx.x; i < n; i += stride) {
        const uint32_t a = in[2 * i], b = in[2 * i + 1];
        float x, y;
        if (kind == 0) {
            b1_pair<MODE>(a, b, mu, sigma, x, y);
            if (accept) accept[i] = 1;
        } else {
            const int32_t kx = (int32_t)a, ky = (int32_t)b;
            int64_t S;
            const bool ok = polar_accept(kx, ky, S);
            if (MODE == kModeB2) {
                x = y = 0.0f;   // B2 is a B1 mode only
            } else {
                polar_pair<MODE == kModeFast ? kModeFast : kModeAccurate>(kx, ky, mu, sigma, x, y);
            }
            if (accept) accept[i] = ok ? 1 : 0;
        }
        out[2 * i] = x;
        out[2 * i + 1] = y;
    }
}

cudaError_t launch_eval_points(int kind, int mode, const uint32_t *in, int64_t n, float mu, float sigma,
                               float *out, int32_t *accept, cudaStream_t s)
{
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + kPointThreads - 1) / kPointThreads, (int64_t)sm_count() * 8));
    if (mode == kModeFast)
        k_eval_points<kModeFast><<<grid, kPointThreads, 0, s>>>(kind, in, n, mu, sigma, out, accept);
    else if (mode == kModeB2)
        k_eval_points<kModeB2><<<grid, kPointThreads, 0, s>>>(kind, in, n, mu, sigma, out, accept);
    else
        k_eval_points<kModeAccurate><<<grid, kPointThreads, 0, s>>>(kind, in, n, mu, sigma, out, accept);
    return cudaGetLastError();
}

}  // namespace nrng
