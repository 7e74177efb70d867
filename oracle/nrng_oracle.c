/*
 * nrng_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the normal
 * generators of Brent, "Fast Normal Random Number Generators for Vector
 * Processors" (TR-CS-93-04, 1993).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; every constant below is written out here
 * from its published definition.
 *
 * Every function follows the definition it cites, step by step, in double
 * precision, with no blocking, fusion or reordering:
 *   - Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *     easy as 1, 2, 3", SC'11, the Philox-4x32 round with R = 10.
 *   - uniforms on [0,1) that may be 0 but never 1: paper Sec. 2 (the uniform
 *     generator assumption and note a).
 *   - Algorithm B1 (Box-Muller): paper Sec. 2, steps 1-3 and notes a, b.
 *   - Algorithm P (Polar): paper Sec. 2, steps 1-4; rejected pairs are
 *     compressed away in candidate order (the vector gather of Sec. 2 and the
 *     compress of Sec. 4, RANN3B).
 *   - Method B3 (Sec. 3), Method P2 (Sec. 4, step 4a) and Algorithm R
 *     (Sec. 5), each with the exact function where the paper fits a
 *     polynomial;
 *   - the reparameterised sample x = mu + sigma*z and its gradients (an
 *     add-on: the paper has no autograd; z is B1's output).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): 24-bit dyadic uniforms from the top bits of each Philox word; B1's
 * angle taken as 2*pi*t with t = v - [v >= 1/2] so it lies in [-pi, pi) as
 * note b says while sin/cos equal those of 2*pi*v; Polar rejects s = 0 as
 * well as s >= 1 (the division-by-zero remark of Sec. 2); accepted Polar
 * pairs are emitted in increasing candidate order, x then y, and an odd n
 * drops the last y.
 *
 * Parity pins (tests, not this file): Philox known-answer vectors and cuRAND's
 * host Philox; closed forms and special cases of B1 and P; the exact lattice
 * acceptance count; moments and Kolmogorov-Smirnov against the normal CDF;
 * finite differences for the reparameterised gradients.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* ---------------------------------------------------------------- Philox -- */

/* Philox-4x32 multipliers and Weyl key increments (Salmon et al., SC'11). */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

/* One Philox-4x32 round: two 32x32->64 products, the high halves xored with
 * the other two counter words and the round key, the words permuted. */
static void orc_philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Philox4x32-10: ten rounds, the key bumped by the Weyl increments between
 * rounds (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += ORC_PHILOX_W0;
            k[1] += ORC_PHILOX_W1;
        }
        orc_philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* The generator's block b: counter word (counter + b) split into its low and
 * high 32 bits, the two upper counter words zero; key split the same way. */
static void orc_block(uint64_t key, uint64_t counter, uint64_t b, uint32_t w[4])
{
    uint64_t c = counter + b;
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0u};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    orc_philox4x32_10(ctr, k, w);
}

void orc_philox_blocks(uint32_t *out, int64_t nblocks, uint64_t key, uint64_t counter)
{
    for (int64_t b = 0; b < nblocks; ++b)
        orc_block(key, counter, (uint64_t)b, out + 4 * b);
}

/* ------------------------------------------------------- uniform lattice -- */

/* Uniform on [0,1), may be 0, never 1 (paper Sec. 2, note a): the top 24
 * bits of a word, k = w >> 8, scaled by 2^-24.  Exact in float and double. */
static double orc_u24(uint32_t w)
{
    return (double)(w >> 8) * 0x1p-24;
}

void orc_uniform(double *out, int64_t n, uint64_t key, uint64_t counter)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        orc_block(key, counter, (uint64_t)(i / 4), w);
        out[i] = orc_u24(w[i % 4]);
    }
}

/* ---------------------------------------------------- Algorithm B1 (Sec 2) */

/* One Box-Muller pair from independent uniforms u, v:
 *   step 2: r = sigma * sqrt(-2 ln(1 - u))      (1 - u is exact here)
 *   step 3: x = r sin(2 pi v) + mu,  y = r cos(2 pi v) + mu
 * with the angle written as 2 pi t, t = v - [v >= 1/2] in [-1/2, 1/2), so it
 * lies in [-pi, pi) as note b states; sin and cos are unchanged by the shift. */
static void orc_b1_pair(double u, double v, double mu, double sigma, double *x, double *y)
{
    double r = sigma * sqrt(-2.0 * log(1.0 - u));
    double t = (v >= 0.5) ? v - 1.0 : v;
    double theta = 2.0 * M_PI * t;
    *x = r * sin(theta) + mu;
    *y = r * cos(theta) + mu;
}

/* Element i of the B1 stream: block i/4; pair p = (i%4)/2 takes u from word
 * 2p and v from word 2p+1; even i is x, odd i is y. */
static double orc_b1_element(int64_t i, double mu, double sigma, uint64_t key, uint64_t counter)
{
    uint32_t w[4];
    orc_block(key, counter, (uint64_t)(i / 4), w);
    int p = (int)((i % 4) / 2);
    double x, y;
    orc_b1_pair(orc_u24(w[2 * p]), orc_u24(w[2 * p + 1]), mu, sigma, &x, &y);
    return (i % 2 == 0) ? x : y;
}

void orc_boxmuller(double *out, int64_t n, double mu, double sigma, uint64_t key, uint64_t counter)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_b1_element(i, mu, sigma, key, counter);
}

/* Steps 2-3 at given (u, v) (for hand-picked special cases), shape [m, 2]. */
void orc_b1_points(double *out2, const double *u, const double *v, int64_t m, double mu,
                   double sigma)
{
    for (int64_t j = 0; j < m; ++j)
        orc_b1_pair(u[j], v[j], mu, sigma, &out2[2 * j], &out2[2 * j + 1]);
}

/* The same stream at chosen indices only (for sampled checks at full size). */
void orc_boxmuller_at(double *out, const int64_t *idx, int64_t m, double mu, double sigma,
                      uint64_t key, uint64_t counter)
{
    for (int64_t j = 0; j < m; ++j)
        out[j] = orc_b1_element(idx[j], mu, sigma, key, counter);
}

/* ----------------------------------------------------- Algorithm P (Sec 2) */

/* Candidate c (counted from the first block at `counter`) lives in block c/2
 * and uses words 2(c%2), 2(c%2)+1.  Step 1 draws x, y uniform on [-1, 1): the
 * 24-bit lattice k' = (w >> 8) - 2^23, x = k' * 2^-23 (exact). */
static void orc_polar_candidate(int64_t c, uint64_t key, uint64_t counter, int32_t *kx, int32_t *ky)
{
    uint32_t w[4];
    orc_block(key, counter, (uint64_t)(c / 2), w);
    int h = (int)(c % 2);
    *kx = (int32_t)(w[2 * h] >> 8) - (1 << 23);
    *ky = (int32_t)(w[2 * h + 1] >> 8) - (1 << 23);
}

/* Steps 2-3: s = x^2 + y^2 (exact in FP64: kx'^2 + ky'^2 < 2^47, scaled by
 * 2^-46); reject if s >= 1, and also if s = 0 (the division at step 4). */
static int orc_polar_accept(int32_t kx, int32_t ky)
{
    double x = (double)kx * 0x1p-23;
    double y = (double)ky * 0x1p-23;
    double s = x * x + y * y;
    return s < 1.0 && s > 0.0;
}

/* Step 4: r = sigma sqrt(-2 ln(s)/s); return r x + mu, r y + mu. */
static void orc_polar_step4(int32_t kx, int32_t ky, double mu, double sigma, double *ox, double *oy)
{
    double x = (double)kx * 0x1p-23;
    double y = (double)ky * 0x1p-23;
    double s = x * x + y * y;
    double r = sigma * sqrt(-2.0 * log(s) / s);
    *ox = r * x + mu;
    *oy = r * y + mu;
}

/* Algorithm P over the candidate stream: the i-th accepted candidate (in
 * increasing candidate index) gives out[2i] = x, out[2i+1] = y, until n values
 * are written (ceil(n/2) pairs; odd n drops the last y).
 * pair_cand (nullable, ceil(n/2) entries): candidate index of each pair.
 * next_counter (nullable): the first block with no consumed candidate,
 * i.e. counter + c_last/2 + 1.  Returns the number of candidates examined. */
int64_t orc_polar(double *out, int64_t n, double mu, double sigma, uint64_t key, uint64_t counter,
                  int64_t *pair_cand, uint64_t *next_counter)
{
    int64_t npairs = (n + 1) / 2;
    int64_t i = 0, c = 0, c_last = -1;
    while (i < npairs) {
        int32_t kx, ky;
        orc_polar_candidate(c, key, counter, &kx, &ky);
        if (orc_polar_accept(kx, ky)) {
            double x, y;
            orc_polar_step4(kx, ky, mu, sigma, &x, &y);
            out[2 * i] = x;
            if (2 * i + 1 < n) out[2 * i + 1] = y;
            if (pair_cand) pair_cand[i] = c;
            c_last = c;
            ++i;
        }
        ++c;
    }
    if (next_counter)
        *next_counter = (c_last < 0) ? counter : counter + (uint64_t)(c_last / 2) + 1u;
    return c;
}

/* Raw candidates c in [0, ncand): lattice coordinates and the accept bit. */
void orc_polar_candidates(uint8_t *accept, int32_t *kx, int32_t *ky, int64_t ncand,
                          uint64_t key, uint64_t counter)
{
    for (int64_t c = 0; c < ncand; ++c) {
        int32_t a, b;
        orc_polar_candidate(c, key, counter, &a, &b);
        if (accept) accept[c] = (uint8_t)orc_polar_accept(a, b);
        if (kx) kx[c] = a;
        if (ky) ky[c] = b;
    }
}

/* Step 4 evaluated at given lattice points (for hand-picked cases) and at
 * given candidate indices of a stream (for sampled checks at full size).
 * Writes NaN for a point that step 3 would reject. */
void orc_polar_points(double *out2, const int32_t *kx, const int32_t *ky, int64_t m,
                      double mu, double sigma)
{
    for (int64_t j = 0; j < m; ++j) {
        if (orc_polar_accept(kx[j], ky[j])) {
            orc_polar_step4(kx[j], ky[j], mu, sigma, &out2[2 * j], &out2[2 * j + 1]);
        } else {
            out2[2 * j] = NAN;
            out2[2 * j + 1] = NAN;
        }
    }
}

/* Step 3's accept bit at given lattice points. */
void orc_polar_accept_points(uint8_t *accept, const int32_t *kx, const int32_t *ky, int64_t m)
{
    for (int64_t j = 0; j < m; ++j)
        accept[j] = (uint8_t)orc_polar_accept(kx[j], ky[j]);
}

void orc_polar_at(double *out2, const int64_t *cand, int64_t m, double mu, double sigma,
                  uint64_t key, uint64_t counter)
{
    for (int64_t j = 0; j < m; ++j) {
        int32_t kx, ky;
        orc_polar_candidate(cand[j], key, counter, &kx, &ky);
        orc_polar_points(out2 + 2 * j, &kx, &ky, 1, mu, sigma);
    }
}

/* Exact number of accepted lattice points of half-width H,
 *   A(H) = #{(a, b) in [-H, H)^2 : 0 < a^2 + b^2 < H^2},
 * by brute force over a with an exact integer square root for the range of
 * b.  The generator's lattice has H = 2^23 (x = a 2^-23 in [-1, 1)), and the
 * acceptance probability of step 3 is A(2^23) / 2^48; smaller H give the same
 * count on coarser lattices, so that it can be checked by enumeration. */
static int64_t orc_isqrt(int64_t v) /* largest t >= 0 with t*t <= v, v >= 0 */
{
    int64_t t = (int64_t)sqrt((double)v);
    while (t * t > v) --t;
    while ((t + 1) * (t + 1) <= v) ++t;
    return t;
}

int64_t orc_lattice_accept_count_h(int64_t H)
{
    const int64_t R = H * H;
    int64_t total = 0;
    for (int64_t a = -H; a < H; ++a) {
        int64_t rem = R - a * a; /* need b^2 < rem, i.e. b^2 <= rem - 1 */
        if (rem <= 0) continue;
        int64_t t = orc_isqrt(rem - 1);
        int64_t lo = (-t < -H) ? -H : -t;
        int64_t hi = (t > H - 1) ? H - 1 : t;
        if (hi >= lo) total += hi - lo + 1;
    }
    return total - 1; /* the origin has s = 0 and is rejected */
}

int64_t orc_lattice_accept_count(void)
{
    return orc_lattice_accept_count_h((int64_t)1 << 23);
}

/* ------------------------------------------------------- Method B3 (Sec 3) */

/* Word i of the stream (block i/4, word i mod 4). */
static uint32_t orc_word(int64_t i, uint64_t key, uint64_t counter)
{
    uint32_t w[4];
    orc_block(key, counter, (uint64_t)(i / 4), w);
    return w[i % 4];
}

/* Method B3, with the exact function in place of the paper's polynomial h:
 *   step 1: u1, u2, u3 uniform (words 3p, 3p+1, 3p+2 of the stream for pair p);
 *   step 2: m = max(u1, u2), u = m^2 (uniform on [0, 1));
 *   step 3: r = sigma sqrt(-ln(1 - u));
 *   step 4: s = sin(2 pi u3 - pi), c = cos(2 pi u3 - pi);
 *   step 5: return mu + c r sqrt2 and mu + s r sqrt2 (out[2p], out[2p+1]). */
static void orc_b3_pair(double u1, double u2, double u3, double mu, double sigma, double *x, double *y)
{
    double m = (u1 > u2) ? u1 : u2;
    double u = m * m;                       /* exact: m has 24 bits */
    double r = sigma * sqrt(-log(1.0 - u));
    double a = 2.0 * M_PI * u3 - M_PI;
    *x = mu + cos(a) * r * sqrt(2.0);
    *y = mu + sin(a) * r * sqrt(2.0);
}

void orc_b3(double *out, int64_t n, double mu, double sigma, uint64_t key, uint64_t counter)
{
    for (int64_t p = 0; 2 * p < n; ++p) {
        double x, y;
        orc_b3_pair(orc_u24(orc_word(3 * p, key, counter)), orc_u24(orc_word(3 * p + 1, key, counter)),
                    orc_u24(orc_word(3 * p + 2, key, counter)), mu, sigma, &x, &y);
        out[2 * p] = x;
        if (2 * p + 1 < n) out[2 * p + 1] = y;
    }
}

/* Steps 2-5 at given uniforms (for hand-picked cases). */
void orc_b3_points(double *out2, const double *u1, const double *u2, const double *u3, int64_t m, double mu,
                   double sigma)
{
    for (int64_t j = 0; j < m; ++j)
        orc_b3_pair(u1[j], u2[j], u3[j], mu, sigma, &out2[2 * j], &out2[2 * j + 1]);
}

/* ------------------------------------------------- Method P2 (Sec 4, 4a) */

/* Step 4a with u = 1 - s (independent of the angle): r = sigma sqrt(-ln(1-s)/s),
 * returning x r sqrt2 + mu, y r sqrt2 + mu.  The paper approximates
 * sqrt(-ln(1-s)/s) by the polynomial h for s <= 8/9; the oracle evaluates it. */
static void orc_p2_step4(int32_t kx, int32_t ky, double mu, double sigma, double *ox, double *oy)
{
    double x = (double)kx * 0x1p-23;
    double y = (double)ky * 0x1p-23;
    double s = x * x + y * y;
    double r = sigma * sqrt(-log(1.0 - s) / s);
    *ox = x * r * sqrt(2.0) + mu;
    *oy = y * r * sqrt(2.0) + mu;
}

/* Step 4a at given lattice points (for hand-picked cases); the caller keeps
 * to accepted points (0 < S < 2^46). */
void orc_p2_points(double *out2, const int32_t *kx, const int32_t *ky, int64_t m, double mu, double sigma)
{
    for (int64_t j = 0; j < m; ++j)
        orc_p2_step4(kx[j], ky[j], mu, sigma, &out2[2 * j], &out2[2 * j + 1]);
}

/* Method P2: the candidate stream, acceptance and compaction of Algorithm P,
 * step 4 replaced by step 4a. */
int64_t orc_polar_p2(double *out, int64_t n, double mu, double sigma, uint64_t key, uint64_t counter,
                     int64_t *pair_cand, uint64_t *next_counter)
{
    int64_t npairs = (n + 1) / 2;
    int64_t i = 0, c = 0, c_last = -1;
    while (i < npairs) {
        int32_t kx, ky;
        orc_polar_candidate(c, key, counter, &kx, &ky);
        if (orc_polar_accept(kx, ky)) {
            double x, y;
            orc_p2_step4(kx, ky, mu, sigma, &x, &y);
            out[2 * i] = x;
            if (2 * i + 1 < n) out[2 * i + 1] = y;
            if (pair_cand) pair_cand[i] = c;
            c_last = c;
            ++i;
        }
        ++c;
    }
    if (next_counter)
        *next_counter = (c_last < 0) ? counter : counter + (uint64_t)(c_last / 2) + 1u;
    return c;
}

/* ------------------------------------------------ Algorithm R (Sec 5) ---- */

/* Candidate c: u from word 2(c mod 2), v from word 2(c mod 2) + 1 of block c/2.
 *   step 2: x = sqrt(8/e) (v - 1/2) / (1 - u);
 *   step 3: reject unless x^2 <= -4 ln(1 - u) (the ratio-of-uniforms region;
 *           see the reading of the printed condition in the design notes);
 *   step 4: return sigma x + mu.
 * All in double precision, the paper's. */
static void orc_ratio_candidate(int64_t c, uint64_t key, uint64_t counter, double *u, double *v)
{
    uint32_t w[4];
    orc_block(key, counter, (uint64_t)(c / 2), w);
    int h = (int)(c % 2);
    *u = orc_u24(w[2 * h]);
    *v = orc_u24(w[2 * h + 1]);
}

static int orc_ratio_accept(double u, double v, double *x)
{
    *x = sqrt(8.0 / M_E) * (v - 0.5) / (1.0 - u);
    return (*x) * (*x) <= -4.0 * log(1.0 - u);
}

int64_t orc_ratio(double *out, int64_t n, double mu, double sigma, uint64_t key, uint64_t counter,
                  int64_t *cand_out, uint64_t *next_counter)
{
    int64_t i = 0, c = 0, c_last = -1;
    while (i < n) {
        double u, v, x;
        orc_ratio_candidate(c, key, counter, &u, &v);
        if (orc_ratio_accept(u, v, &x)) {
            out[i] = sigma * x + mu;
            if (cand_out) cand_out[i] = c;
            c_last = c;
            ++i;
        }
        ++c;
    }
    if (next_counter)
        *next_counter = (c_last < 0) ? counter : counter + (uint64_t)(c_last / 2) + 1u;
    return c;
}

void orc_ratio_candidates(uint8_t *accept, int64_t ncand, uint64_t key, uint64_t counter)
{
    for (int64_t c = 0; c < ncand; ++c) {
        double u, v, x;
        orc_ratio_candidate(c, key, counter, &u, &v);
        accept[c] = (uint8_t)orc_ratio_accept(u, v, &x);
    }
}

/* Step 2 and 4 of R at a chosen candidate (sampled checks). */
void orc_ratio_at(double *out, const int64_t *cand, int64_t m, double mu, double sigma, uint64_t key,
                  uint64_t counter)
{
    for (int64_t j = 0; j < m; ++j) {
        double u, v, x;
        orc_ratio_candidate(cand[j], key, counter, &u, &v);
        orc_ratio_accept(u, v, &x);
        out[j] = sigma * x + mu;
    }
}

/* Steps 2-4 of R at given uniforms (for hand-picked cases): accept[j] is
 * step 3's decision, out[j] = sigma x + mu (meaningful where accepted). */
void orc_ratio_points(double *out, uint8_t *accept, const double *u, const double *v, int64_t m, double mu,
                      double sigma)
{
    for (int64_t j = 0; j < m; ++j) {
        double x;
        accept[j] = (uint8_t)orc_ratio_accept(u[j], v[j], &x);
        out[j] = sigma * x + mu;
    }
}

/* ------------------------------------------------------ batched streams -- */

/* Each stream j is an independent B1 (method 0) or Polar (method 1) stream
 * written at out + offset[j]. */
void orc_batched(double *out, int32_t k, const int64_t *offset, const int64_t *n,
                 const float *mu, const float *sigma, const uint64_t *key,
                 const uint64_t *counter, const int32_t *method)
{
    for (int32_t j = 0; j < k; ++j) {
        if (method[j] == 0)
            orc_boxmuller(out + offset[j], n[j], mu[j], sigma[j], key[j], counter[j]);
        else
            orc_polar(out + offset[j], n[j], mu[j], sigma[j], key[j], counter[j], NULL, NULL);
    }
}

/* ------------------------------------------------ reparameterised sample -- */

/* Element i uses parameter index p(i) = (i / inner) mod m: m = n is
 * elementwise, m = 1 a scalar, other (m, inner) one broadcast axis.
 * z_i is element i of the B1 stream with mu = 0, sigma = 1. */
static int64_t orc_param_index(int64_t i, int64_t m, int64_t inner)
{
    return (i / inner) % m;
}

void orc_reparam_fwd(double *x, const float *mu, const float *sigma, int64_t n, int64_t m,
                     int64_t inner, uint64_t key, uint64_t counter)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = orc_param_index(i, m, inner);
        double z = orc_b1_element(i, 0.0, 1.0, key, counter);
        x[i] = (double)mu[p] + (double)sigma[p] * z;
    }
}

/* d x_i / d mu_p = 1 and d x_i / d sigma_p = z_i where p = p(i), so
 * dmu_p = sum g_i and dsigma_p = sum g_i z_i over the i with p(i) = p. */
void orc_reparam_bwd(double *dmu, double *dsigma, const float *g, int64_t n, int64_t m,
                     int64_t inner, uint64_t key, uint64_t counter)
{
    for (int64_t p = 0; p < m; ++p) {
        if (dmu) dmu[p] = 0.0;
        dsigma[p] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = orc_param_index(i, m, inner);
        double z = orc_b1_element(i, 0.0, 1.0, key, counter);
        if (dmu) dmu[p] += (double)g[i];
        dsigma[p] += (double)g[i] * z;
    }
}
