/*
 * nrng.h -- C ABI of the GB300 (sm_103a) normal-variate library.
 *
 * Implements the bulk transformation of uniform variates into N(mu, sigma^2)
 * variates of R. P. Brent, "Fast Normal Random Number Generators for Vector
 * Processors" (TR-CS-93-04, 1993): Box-Muller Algorithm B1 and the Polar
 * Algorithm P of Sec. 2, with P's rejection done as an order-preserving stream
 * compaction (the vector compress/gather of Sec. 2 and Sec. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 * Uniform source.  The paper assumes a good generator of uniforms on [0, 1)
 * that may return 0 but never 1 (Sec. 2, note a).  This library uses
 * Philox4x32-10 (Salmon et al., SC'11).  Block b of a stream (key, counter)
 * is Philox(ctr = (lo32(counter + b), hi32(counter + b), 0, 0),
 * key = (lo32(key), hi32(key))) and yields four 32-bit words w0..w3.  A
 * uniform is u = (w >> 8) * 2^-24, a point of the 24-bit dyadic lattice.
 * The counter unit of every call is one Philox block (four words).
 *
 * Memory.  Every pointer named d_* is device memory owned by the caller; h_*
 * is host memory.  The library never allocates device memory on these paths
 * and keeps no pointer after a call returns.  Outputs need the natural
 * alignment of their element type; wider alignment (16 bytes) selects the
 * vector-store kernels, narrower alignment the element-store kernels.
 *
 * Streams.  Calls are asynchronous and stream-ordered on `stream` (a
 * cudaStream_t; 0 is the legacy default stream).  A call returns after
 * enqueueing its work.  Calls that take a workspace may not overlap on the
 * GPU with another call using the same workspace.
 *
 * Threads.  Every call may be made from several host threads at once, each
 * with its own buffers and workspaces (on its own streams, or ordered on a
 * shared one).  The process-wide state (cached occupancies and SM counts,
 * the batched configuration table and its autotune cache file, the
 * no-workspace Polar call's address lookup) is guarded by atomics or a
 * mutex.  nrng_polar_noalloc's device array itself is shared by every call
 * on a device: such calls must be ordered on the GPU (see that call).
 *
 * Errors.  Every call returns an nrng_status_t.  Errors the host can detect
 * (a null pointer with n > 0, n < 0, n above 2^60, or above 2^48 for the
 * rejection methods, sigma < 0 or not finite, mu not finite,
 * an unknown enum, a misaligned pointer, a workspace that is too small, a
 * Philox counter that would pass 2^64) return at once and enqueue nothing.
 * A failed launch returns NRNG_ERR_CUDA.  Errors only the device can see
 * (a look-back wait that ran out, a Polar stream that ran out of workspace
 * tiles, a bad batched descriptor) are written to the workspace status word;
 * read it with nrng_get_status.  n = 0 is a no-op that returns NRNG_OK.
 */
#ifndef NRNG_H
#define NRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Layout-compatible with cudaStream_t, so this header needs no CUDA header. */
typedef struct CUstream_st *nrng_stream_t;

typedef enum {
    NRNG_OK = 0,
    NRNG_ERR_INVALID_VALUE = 1,   /* bad size, pointer, parameter or enum */
    NRNG_ERR_MISALIGNED = 2,      /* pointer not aligned to its element type */
    NRNG_ERR_WORKSPACE = 3,       /* workspace missing or smaller than required */
    NRNG_ERR_COUNTER_OVERFLOW = 4,/* counter + blocks used would pass 2^64 */
    NRNG_ERR_CUDA = 5,            /* a CUDA runtime call or launch failed */
    NRNG_ERR_TIMEOUT = 6,         /* device: a look-back wait ran out */
    NRNG_ERR_EXHAUSTED = 7,       /* device: Polar needed more tiles than sized */
    NRNG_ERR_NOT_SUPPORTED = 8    /* a valid request this library version does not handle */
} nrng_status_t;

typedef enum { NRNG_F32 = 0, NRNG_BF16 = 1, NRNG_F16 = 2 } nrng_dtype_t;

/* NRNG_ACCURATE: for B1, ln(1 - u) and sin/cos(2 pi v) from the exact
 *   24-bit lattice integers (an exact split of 1 - u into 2^e f with the
 *   atanh series for ln f; angle addition from a table of 256 angles with
 *   short Taylor polynomials of the exact remainder), within 3e-7 relative
 *   and 1e-7 absolute over the whole lattice; for P, CUDA's logf of s held as an exact
 *   double-float.  Square roots and reciprocals by the hardware
 *   approximations, whose relative error (below 2^-22) moves a result by
 *   under 2e-7 of itself.  Error within 4e-6 max(1, |z|) of the FP64
 *   definition.
 * NRNG_FAST: the hardware approximations (log2, sqrt, rsqrt, sin, cos) with a
 *   short series for ln(1 - d) at small d, where the approximate log loses
 *   relative accuracy.  Error within 2e-5 max(1, |z|).
 * NRNG_B2 (nrng_boxmuller only): the paper's Method B2 (Sec. 3), B1 with the
 *   library ln and sqrt and an inline sine and cosine: polynomials at a
 *   sixteenth of the angle and four double-angle steps.  Error within
 *   2e-5 max(1, |z|). */
typedef enum { NRNG_ACCURATE = 0, NRNG_FAST = 1, NRNG_B2 = 2 } nrng_mode_t;

typedef enum { NRNG_B1 = 0, NRNG_POLAR = 1 } nrng_method_t;

/* One stream of a batched call: n normals of N(mu, sigma^2) drawn with
 * `method` from (key, counter), written at element `offset` of the output. */
typedef struct {
    int64_t offset;
    int64_t n;
    float mu;
    float sigma;
    uint64_t key;
    uint64_t counter;
    int32_t method;     /* nrng_method_t */
    int32_t reserved;   /* must be 0 */
} nrng_stream_desc_t;

/* Human-readable name of a status code (static storage). */
const char *nrng_status_string(int32_t status);

/* ABI version; bumps when any declaration in this header changes. */
int32_t nrng_abi_version(void);

/* Uniforms (paper Sec. 2: uniforms on [0, 1) that may be 0, never 1).
 * d_out[i] = (w_{i mod 4} of block i/4) >> 8) * 2^-24 as float, exact.
 * d_out: n floats, 4-byte aligned.  Uses ceil(n/4) blocks from `counter`. */
int32_t nrng_uniform(float *d_out, int64_t n, uint64_t key, uint64_t counter,
                     nrng_stream_t stream);

/* Measurement aid: the uniform generator alone.  Draws the Philox blocks
 * [counter, counter + nblocks) of `key` and stores the xor of all their words
 * in *d_out (one uint32, device memory, 4-byte aligned), with no other
 * stores, so that its time is this GPU's rate of drawing blocks: the
 * instruction ceiling shared by every generator here.  The paper's Table 1
 * counts uniform generation inside the "other" cycles of each method (Sec. 3);
 * this call measures that share on its own.  nblocks <= 2^31 with a low
 * counter word that does not wrap (counter mod 2^32 + nblocks <= 2^32),
 * else NRNG_ERR_NOT_SUPPORTED. */
int32_t nrng_philox_ceiling(uint32_t *d_out, int64_t nblocks, uint64_t key, uint64_t counter,
                            nrng_stream_t stream);

/* Box-Muller, Algorithm B1 (paper Sec. 2, steps 1-3, notes a and b).
 * Block b gives two pairs: (u, v) from words (w0, w1) and from (w2, w3).
 * For each, r = sigma sqrt(-2 ln(1 - u)), x = r sin(2 pi v) + mu,
 * y = r cos(2 pi v) + mu, stored at d_out[4b + 2p] (x) and [4b + 2p + 1] (y).
 * d_out: n elements of `dtype` (fp32, or bf16/fp16 rounded to nearest even
 * from the fp32 result).  Uses ceil(n/4) blocks from `counter`. */
int32_t nrng_boxmuller(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                       uint64_t counter, int32_t dtype, int32_t mode,
                       nrng_stream_t stream);

/* Workspace bytes nrng_polar needs for n outputs (tile status words, the
 * tile counter and the status word).  Pure host computation. */
int32_t nrng_polar_workspace_size(int64_t n, size_t *h_bytes);

/* Largest number of Philox blocks nrng_polar may consume for n outputs
 * (the workspace's tile budget); counter + this must not pass 2^64. */
int32_t nrng_polar_max_blocks(int64_t n, uint64_t *h_blocks);

/* Polar, Algorithm P (paper Sec. 2, steps 1-4), rejection as an
 * order-preserving compaction (Sec. 2's vector gather, Sec. 4's compress).
 * Candidate c (c = 0, 1, ...) is block counter + c/2, words 2(c mod 2) and
 * 2(c mod 2) + 1: kx = (w >> 8) - 2^23, x = kx 2^-23 in [-1, 1), same for y.
 * It is accepted iff 0 < S < 2^46 with S = kx^2 + ky^2 exact in 64-bit
 * integers (s = S 2^-46 < 1, and s = 0 rejected).  The i-th accepted
 * candidate gives d_out[2i] = r x + mu and d_out[2i + 1] = r y + mu with
 * r = sigma sqrt(-2 ln(s) / s), for the first ceil(n/2) accepted candidates;
 * an odd n drops the last y.
 * d_ws/ws_bytes: workspace of at least nrng_polar_workspace_size(n) bytes,
 *   cleared by this call; it holds the status word afterwards.
 * d_next_counter (nullable): receives counter + c_last/2 + 1, the first block
 *   with no consumed candidate, to continue the stream.
 * d_pair_candidate (nullable): ceil(n/2) int64, the candidate index of each
 *   output pair (for verification of the accept order).
 * Device errors (NRNG_ERR_TIMEOUT, NRNG_ERR_EXHAUSTED) go to the status word. */
int32_t nrng_polar(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                   uint64_t counter, int32_t dtype, int32_t mode, void *d_ws,
                   size_t ws_bytes, uint64_t *d_next_counter, int64_t *d_pair_candidate,
                   nrng_stream_t stream);

/* Workspace bytes nrng_polar_twopass needs for n outputs. */
int32_t nrng_polar_twopass_workspace_size(int64_t n, size_t *h_bytes);

/* Polar, Algorithm P, with the compress done in two passes instead of one:
 * a count pass draws every tile of candidates and counts the accepted ones,
 * a scan turns the counts into each tile's first output pair, and a write
 * pass draws each tile again and places its pairs there.  Arguments and
 * outputs are those of nrng_polar, bit for bit (the same candidates, accept
 * order and step-4 arithmetic); only the workspace size differs.  It is the
 * two-pass alternative to nrng_polar's single-pass look-back (paper Sec. 4:
 * the vector compress of RANN3B and the buffering of RANN3), kept for
 * comparison.  Device errors (NRNG_ERR_EXHAUSTED) go to the status word. */
int32_t nrng_polar_twopass(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                           uint64_t counter, int32_t dtype, int32_t mode, void *d_ws,
                           size_t ws_bytes, uint64_t *d_next_counter, int64_t *d_pair_candidate,
                           nrng_stream_t stream);

/* Box-Muller, Method B3 (paper Sec. 3): three uniforms per pair instead of
 * two, so that no square root and, for most pairs, no logarithm is needed.
 * Pair p takes words 3p, 3p + 1, 3p + 2 of the stream (word j is word
 * j mod 4 of block counter + j/4), u_i = (w >> 8) 2^-24.  With
 * m = max(u1, u2) and u = m^2 (uniform on [0, 1)), r = sigma sqrt(-ln(1 - u))
 * is computed as sigma m h(v) by a fitted polynomial h of
 * v = (6u - 4)/(4 - 3u) for u <= 8/9 and by the hardware log2 and square
 * root above (the library step of the paper), and theta =
 * 2 pi u3 - pi by Method B2's sine and cosine polynomials with double-angle
 * steps.  d_out[2p] = sqrt(2) r cos(theta) + mu, d_out[2p + 1] =
 * sqrt(2) r sin(theta) + mu.  Uses 3 ceil(n/8) blocks from `counter` (eight
 * outputs per three blocks).  Single precision throughout; error within
 * 2e-5 max(1, |z|) of the FP64 definition. */
int32_t nrng_boxmuller_b3(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                          uint64_t counter, int32_t dtype, nrng_stream_t stream);

/* Polar, Method P2 (paper Sec. 4): Algorithm P's steps 1-3 (the same
 * candidates, accept test and accept order as nrng_polar) and step 4a,
 * r = sigma sqrt(-2 ln(1 - s) / s): the i-th accepted candidate gives
 * d_out[2i] = r x + mu, d_out[2i + 1] = r y + mu.  1 - s is uniform and
 * independent of the angle, so this is also a normal pair, different from
 * nrng_polar's.  ln(1 - s)/s comes from the polynomial h of Method B3 for
 * s <= 8/9 (no logarithm, no division) and from the hardware log2,
 * reciprocal and square root of the exact 1 - s above.  Workspace,
 * counter use, d_next_counter and d_pair_candidate: as nrng_polar (size it
 * with nrng_polar_workspace_size).  Error within 2e-5 max(1, |z|). */
int32_t nrng_polar_p2(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                      uint64_t counter, int32_t dtype, void *d_ws, size_t ws_bytes,
                      uint64_t *d_next_counter, int64_t *d_pair_candidate,
                      nrng_stream_t stream);

/* Workspace bytes nrng_ratio needs for n outputs.  Pure host computation. */
int32_t nrng_ratio_workspace_size(int64_t n, size_t *h_bytes);

/* The Ratio method, Algorithm R (paper Sec. 5; Kinderman and Monahan), one
 * normal per accepted candidate, in candidate order.  Candidate c is block
 * counter + c/2, words (u, v) = (w_{2h}, w_{2h+1}), h = c mod 2, on the
 * 24-bit lattice.  x = sqrt(8/e) (v - 1/2) / (1 - u); accept iff
 * x^2 <= -4 ln(1 - u) (the reading of the paper's step 3 under which the
 * method yields N(0, 1); acceptance sqrt(pi e)/4 ~ 0.73).  The test is taken
 * on the lattice as 2 a^2 <= e b^2 (-log1p(-u)) (a = v - 1/2, b = 1 - u in
 * units of 2^-24): a float screen settles the clear cases and the rest is
 * decided in double precision.  The i-th accepted candidate gives
 * d_out[i] = sigma x + mu.
 * d_ws/ws_bytes: at least nrng_ratio_workspace_size(n) bytes, cleared by this
 *   call; it holds the status word afterwards.
 * d_next_counter (nullable): counter + c_last/2 + 1.
 * d_candidate (nullable): n int64, the candidate index of each output.
 * mode: NRNG_ACCURATE (IEEE division) or NRNG_FAST (approximate division).
 * Device errors (NRNG_ERR_TIMEOUT, NRNG_ERR_EXHAUSTED) go to the status word. */
int32_t nrng_ratio(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                   uint64_t counter, int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes,
                   uint64_t *d_next_counter, int64_t *d_candidate, nrng_stream_t stream);

/* Diagnostics (no counterpart in the paper): the per-pair transforms at
 * caller-given inputs, so that tests reach points a stream reaches too
 * rarely (s -> 1, S = 1, u = 0, u = 1 - 2^-24, the quadrant angles, the
 * switch to the upper branch at 8/9, the accept boundary of R).  Each kind
 * computes exactly what its generator computes for that input:
 * kind NRNG_POINTS_B1: d_in holds n pairs of 32-bit Philox words (wu, wv);
 *   d_out[2i], d_out[2i + 1] receive B1's x, y (nrng_boxmuller; mode
 *   NRNG_ACCURATE, NRNG_FAST or NRNG_B2).
 * kind NRNG_POINTS_POLAR: d_in holds n pairs of int32 lattice coordinates
 *   (kx', ky') in [-2^23, 2^23); d_accept[i] receives Algorithm P's step-3
 *   decision (1 iff 0 < S < 2^46) and d_out[2i], d_out[2i + 1] step 4's
 *   values (nrng_polar; mode NRNG_ACCURATE or NRNG_FAST), meaningful only
 *   where accepted.
 * kind NRNG_POINTS_P2: as NRNG_POINTS_POLAR with Method P2's step 4a
 *   (nrng_polar_p2; mode NRNG_ACCURATE or NRNG_FAST, which give the same
 *   values).
 * kind NRNG_POINTS_RATIO: d_in holds n pairs of Philox words (wu, wv);
 *   d_accept[i] receives Algorithm R's step-3 decision, d_out[2i] step 4's
 *   value (nrng_ratio; mode NRNG_ACCURATE or NRNG_FAST), meaningful only
 *   where accepted, and d_out[2i + 1] = 0.
 * kind NRNG_POINTS_B3: d_in holds n triples of Philox words (w1, w2, w3);
 *   d_out[2i], d_out[2i + 1] receive Method B3's pair (nrng_boxmuller_b3;
 *   mode NRNG_ACCURATE or NRNG_FAST, which give the same values).
 * d_accept (nullable) receives 1 for every point of kinds B1 and B3.
 * d_in: 2n x 4 bytes (3n x 4 bytes for B3), 4-byte aligned; d_out: 2n
 * floats; d_accept: n int32.  Returns NRNG_ERR_INVALID_VALUE for an unknown
 * kind or a mode the kind does not take. */
typedef enum {
    NRNG_POINTS_B1 = 0, NRNG_POINTS_POLAR = 1, NRNG_POINTS_P2 = 2, NRNG_POINTS_RATIO = 3, NRNG_POINTS_B3 = 4
} nrng_points_kind_t;
int32_t nrng_eval_points(int32_t kind, int32_t mode, const void *d_in, int64_t n, float mu, float sigma,
                         float *d_out, int32_t *d_accept, nrng_stream_t stream);

/* Polar without a workspace, for callers that cannot allocate device memory
 * (no counterpart in the paper).  Some callers cannot obtain the workspace
 * nrng_polar needs: code running inside a host application that owns the
 * device memory budget and forbids allocations of its own, or a
 * latency-critical loop that avoids cudaMalloc because it can synchronise the
 * device.  This call computes exactly what nrng_polar computes (same kernel,
 * same outputs) but keeps its scratch in a fixed 1 MiB device array inside the
 * library, so it allocates nothing; the caller passes only outputs.
 *   n: at most 2^28 (268435456); a larger n returns NRNG_ERR_WORKSPACE and
 *     enqueues nothing.
 *   d_next_counter, d_pair_candidate: as nrng_polar (nullable).
 *   d_status (nullable): one int32 that receives the call's device status
 *     word (NRNG_OK, NRNG_ERR_TIMEOUT, NRNG_ERR_EXHAUSTED) once the kernel is
 *     done, in stream order.
 * The array is held by every GPU that loads the library until the process
 * exits and is shared by every call on that device: each call clears what it
 * uses first, so calls ordered on the GPU are independent, but calls that
 * overlap on the GPU (unordered streams) race on it.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * address is kept for the life of the process, which assumes one CUDA
 * context per device: after cudaDeviceReset the call must not be used again
 * in that process. */
int32_t nrng_polar_noalloc(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                           uint64_t counter, int32_t dtype, int32_t mode,
                           uint64_t *d_next_counter, int64_t *d_pair_candidate,
                           int32_t *d_status, nrng_stream_t stream);

/* Workspace bytes nrng_batched needs for the k streams described in h_desc
 * (host copy of the descriptors).  Pure host computation.  A descriptor with
 * n above 2^60 returns NRNG_ERR_INVALID_VALUE. */
int32_t nrng_batched_workspace_size(const nrng_stream_desc_t *h_desc, int32_t k,
                                    size_t *h_bytes);

/* k independent streams in one persistent launch (B1 or Polar per stream, as
 * nrng_boxmuller / nrng_polar define them, each at d_out + offset in elements
 * of `dtype`).  d_desc: k descriptors in device memory.  Streams may not
 * overlap in the output.  The per-stream work is scheduled as tiles pulled
 * from one global work counter; Polar tiles look back within their stream.
 * Descriptor errors found on the device (n < 0, sigma < 0, bad method, a
 * stream of more than 2^31 work items, i.e. above about 3.5e13 normals, a
 * workspace smaller than the descriptors need) set the status word and the
 * launch writes nothing.  Capturable in a CUDA graph. */
int32_t nrng_batched(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k,
                     int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes,
                     nrng_stream_t stream);

/* Reparameterised sample x = mu + sigma z (an add-on with no counterpart in
 * the paper; z is the B1 stream of nrng_boxmuller with mu = 0, sigma = 1).
 * Element i of x uses parameter p(i) = (i / inner) mod m of d_mu and
 * d_sigma (m floats each): m = n is elementwise, m = 1 a scalar, any other
 * m with inner a single broadcast axis; m * inner must divide n. */
int32_t nrng_reparam_fwd(float *d_x, const float *d_mu, const float *d_sigma, int64_t n,
                         int64_t m, int64_t inner, uint64_t key, uint64_t counter,
                         int32_t mode, nrng_stream_t stream);

/* Gradients of the reparameterised sample for upstream gradient d_g (n
 * floats): d_dmu[p] = sum of g_i and d_dsigma[p] = sum of g_i z_i over the i
 * with p(i) = p, z regenerated from (key, counter) instead of stored.
 * d_dmu is nullable (skip it).  When m < n the sums use float atomics: their
 * rounding order, not their terms, varies between runs. */
int32_t nrng_reparam_bwd(float *d_dmu, float *d_dsigma, const float *d_g, int64_t n,
                         int64_t m, int64_t inner, uint64_t key, uint64_t counter,
                         int32_t mode, nrng_stream_t stream);

/* Reads the status word a workspace call left behind (synchronises stream).
 * Returns NRNG_OK on success of the read itself; *h_status is the word. */
int32_t nrng_get_status(const void *d_ws, nrng_stream_t stream, int32_t *h_status);

/* --------------------------------------------------------------------------
 * Autotuning and graphs for the batched launch.
 * -------------------------------------------------------------------------- */

/* Number of compiled batched launch configurations and the shape of one:
 * threads per CTA and Philox blocks each thread takes per tile. */
int32_t nrng_batched_config_count(void);
int32_t nrng_batched_config_info(int32_t config, int32_t *h_threads, int32_t *h_blocks_per_thread);

/* Pins the configuration nrng_batched uses for (dtype, mode); -1 restores
 * the default (the built-in one, or configuration NRNG_FORCE_CONFIG=<id> from
 * the environment when set to a valid id).  Thread-safe. */
int32_t nrng_batched_set_config(int32_t dtype, int32_t mode, int32_t config);
int32_t nrng_batched_get_config(int32_t dtype, int32_t mode, int32_t *h_config);

/* Times every batched configuration on this workload (reps launches each,
 * CUDA events on `stream`), pins the fastest for (dtype, mode) and returns it
 * with its time in milliseconds per launch.  The workspace must be sized for
 * the largest tile count of any configuration (nrng_batched_workspace_size
 * already is).  If the environment variable NRNG_AUTOTUNE_CACHE names a file,
 * it is a cache of earlier choices, one JSON line each, keyed by dtype, mode,
 * the number of streams and a fingerprint of every stream's length and method:
 * a matching line is used without timing anything (its time is returned),
 * and a new choice is appended.  Synchronises `stream`. */
int32_t nrng_batched_autotune(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k,
                              int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes,
                              int32_t reps, nrng_stream_t stream, int32_t *h_config,
                              float *h_ms);

/* Captures one nrng_batched call on `stream` (not the legacy default stream)
 * into an instantiated CUDA graph; *h_graph receives an opaque handle. */
int32_t nrng_batched_graph_create(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k,
                                  int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes,
                                  nrng_stream_t stream, void **h_graph);
int32_t nrng_graph_launch(void *h_graph, nrng_stream_t stream);
int32_t nrng_graph_destroy(void *h_graph);

#ifdef __cplusplus
}
#endif

#endif /* NRNG_H */
