// b3_pair.cuh -- one pair of Method B3 (Sec. 3) from three Philox words,
// shared by the B3 generator (k_paper.cu) and the point evaluator
// (k_points.cu).
#pragma once

#include "nrng_device.cuh"

namespace nrng {

// One B3 pair from words (w1, w2, w3): outputs mu + c r sqrt2, mu + s r sqrt2.
__device__ __forceinline__ void b3_pair(uint32_t w1, uint32_t w2, uint32_t w3, float mu, float sigma,
                                        float &x, float &y)
{
    const float u1 = (float)(w1 >> 8) * 0x1p-24f;
    const float u2 = (float)(w2 >> 8) * 0x1p-24f;
    const float m = fmaxf(u1, u2);
    const float u = m * m;
    float rs;   // r sqrt2 = sigma sqrt(-2 ln(1 - u))
    if (u > 0.888888888f) {
        // 1 - m^2 with one rounding; |log2| > 3.1 there, so the hardware log2
        // and square root keep their relative accuracy (near 2^-22)
        rs = sigma * sqrt_approx(__log2f(fmaf(-m, m, 1.0f)) * -1.38629436f);
    } else {
        rs = sigma * 1.41421356f * m * h_of_u(u);
    }
    float s, c;
    b2_sincos((float)((int32_t)(w3 ^ 0x80000000u) >> 8), s, c);   // angle 2 pi u3 - pi
    x = fmaf(c, rs, mu);
    y = fmaf(s, rs, mu);
}

}  // namespace nrng
