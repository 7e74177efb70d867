// k_points.cu -- the per-pair transforms at caller-given inputs
// (nrng_eval_points), so that tests can reach the special points of the
// lattice (s -> 1, S = 1, u = 0, u = 1 - 2^-24, the quadrant angles, the
// switch to the upper branch at 8/9, the accept boundary of R) that a stream
// reaches too rarely to test.  The kernels call the same device functions as
// the generators: b1_pair (Algorithm B1, Sec. 2, steps 2-3), polar_accept /
// polar_pair (Algorithm P, steps 3-4), p2_pair (Method P2, step 4a),
// ratio_accept / ratio_value (Algorithm R, Sec. 5, steps 2-4) and b3_pair
// (Method B3, Sec. 3).
#include <algorithm>

#include "b3_pair.cuh"
#include "nrng_device.cuh"

namespace nrng {

constexpr int kPointThreads = 256;

enum PointKind { kPointsB1 = 0, kPointsPolar = 1, kPointsP2 = 2, kPointsRatio = 3, kPointsB3 = 4 };

// kind 0 (B1):    in[2i], in[2i+1] are the words (wu, wv) of a B1 pair.
// kind 1 (Polar): in[2i], in[2i+1] are the lattice coordinates (kx', ky') of a
//                 candidate; accept[i] is step 3's decision, out holds step 4's
//                 values (meaningless where the candidate is rejected).
// kind 2 (P2):    as kind 1 with step 4a's values.
// kind 3 (R):     in[2i], in[2i+1] are the words (wu, wv) of a candidate;
//                 accept[i] is step 3's decision, out[2i] step 4's value
//                 (meaningless where rejected), out[2i+1] = 0.
// kind 4 (B3):    in[3i], in[3i+1], in[3i+2] are the words (w1, w2, w3).
template <int MODE>
__global__ void __launch_bounds__(kPointThreads)
k_eval_points(int kind, const uint32_t *__restrict__ in, int64_t n, float mu, float sigma,
              float *__restrict__ out, int32_t *__restrict__ accept)
{
    const int64_t stride = (int64_t)gridDim.x * kPointThreads;
    for (int64_t i = (int64_t)blockIdx.x * kPointThreads + threadIdx.x; i < n; i += stride) {
        float x = 0.0f, y = 0.0f;
        int ok = 1;
        if (kind == kPointsB3) {
            b3_pair(in[3 * i], in[3 * i + 1], in[3 * i + 2], mu, sigma, x, y);
        } else {
            const uint32_t a = in[2 * i], b = in[2 * i + 1];
            if (kind == kPointsB1) {
                b1_pair<MODE>(a, b, radius_coef(mu, sigma), kSinCos1024, x, y);
            } else if (kind == kPointsRatio) {
                int2 ab;
                ok = ratio_accept(a, b, ab) ? 1 : 0;
                x = ratio_value<MODE == kModeFast ? kModeFast : kModeAccurate>(ab, mu, sigma);
            } else {
                const int32_t kx = (int32_t)a, ky = (int32_t)b;
                int64_t S;
                ok = polar_accept(kx, ky, S) ? 1 : 0;
                if (kind == kPointsP2)
                    p2_pair(kx, ky, mu, sigma, x, y);
                else if (MODE != kModeB2)   // B2 is a B1 mode only
                    polar_pair<MODE == kModeFast ? kModeFast : kModeAccurate>(kx * 256, ky * 256, radius_coef(mu, sigma), x, y);
            }
        }
        if (accept) accept[i] = ok;
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
