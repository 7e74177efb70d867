// nrng_internal.h -- declarations shared by the host C-ABI layer and the
// kernels: launch parameter blocks, workspace layouts and launchers.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "nrng.h"

namespace nrng {

constexpr int kModeAccurate = NRNG_ACCURATE;
constexpr int kModeFast = NRNG_FAST;
constexpr int kModeB2 = NRNG_B2;
constexpr int kStatusTimeout = NRNG_ERR_TIMEOUT;
constexpr int kStatusExhausted = NRNG_ERR_EXHAUSTED;
constexpr int kStatusInvalid = NRNG_ERR_INVALID_VALUE;
constexpr int kStatusWorkspace = NRNG_ERR_WORKSPACE;
constexpr int kStatusOverflow = NRNG_ERR_COUNTER_OVERFLOW;

// Philox round keys (key + r * Weyl increment, r = 0..9), computed once on
// the host so that every round's key xor reads a constant-bank operand.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};
RoundKeys round_keys(uint64_t key);

// Header at the start of every workspace.  `status` is the word
// nrng_get_status reads; `done` stops CTAs from taking further tiles.
struct WsHeader {
    int status;
    int done;
    unsigned long long tile_counter;
    unsigned long long aux[6];
};
static_assert(sizeof(WsHeader) == 64, "workspace header is 64 bytes");

// ---------------------------------------------------------------- Polar --
// Tiles of the single-stream rejection kernels: kRejWarps warps x rows x 32
// lanes x 2 candidates, 18 rows for Algorithm P and Method P2 and 14 for
// Algorithm R (measured best for each; at 18 rows six CTAs still fit per SM).
constexpr int kRejWarps = 4;
constexpr int kPolarThreads = kRejWarps * 32;                   // 128
constexpr int kPolarRows = 18;                                  // Philox blocks per thread per tile
constexpr int kRatioRows = 14;
constexpr int kPolarBlocksPerTile = kPolarThreads * kPolarRows; // 2304
constexpr int kPolarCandPerTile = 2 * kPolarBlocksPerTile;      // 4608
constexpr int kRatioBlocksPerTile = kPolarThreads * kRatioRows; // 1792
constexpr int kRatioCandPerTile = 2 * kRatioBlocksPerTile;      // 3584

struct PolarParams {
    void *out;
    int64_t n;
    int64_t nitems;
    float mu, sigma;
    RoundKeys rk;
    uint64_t counter;
    WsHeader *hdr;
    unsigned long long *tile_status;
    int64_t tiles_max;
    uint64_t *next_counter;
    int64_t *pair_cand;
    unsigned long long spin_limit_ns;
    long long debug_silent_tile;   // test hook: this tile never publishes (-1: none)
};

// Largest n a Polar stream accepts (keeps the tile budget arithmetic exact).
constexpr int64_t kPolarMaxN = int64_t(1) << 48;

// floor(sqrt(v)) for 0 <= v < 2^62, exact: a float root (relative error
// below 2^-22), one integer Newton step (then within one of the answer) and
// integer steps that settle it.  No double arithmetic: the device's FP64
// rate is a small fraction of its FP32 rate.
__host__ __device__ inline int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)sqrtf((float)v);
    if (r > 0) r = (r + v / r) / 2;
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Tile budget of a rejection stream that needs `items` accepted candidates,
// in tiles of `cand` candidates accepted with probability at least pct/100:
// enough candidates that running out is a > 12-sigma binomial event, plus one
// spare tile.  Integer-only, so host sizing and device checks agree.
__host__ __device__ inline int64_t reject_tiles_for(int64_t items, int64_t cand, int64_t pct)
{
    const int64_t need = items + 12 * (isqrt64(items) + 1) + 16;
    return (need * 100 + cand * pct - 1) / (cand * pct) + 1;
}

// Polar (and P2): ceil(n/2) pairs, acceptance pi/4 = 0.7854, budgeted at 0.78.
__host__ __device__ inline int64_t polar_tiles_for(int64_t n, int64_t cand)
{
    return reject_tiles_for((n + 1) / 2, cand, 78);
}

// Ratio method: n values, acceptance sqrt(pi e)/4 = 0.7306, budgeted at 0.72.
__host__ __device__ inline int64_t ratio_tiles_for(int64_t n, int64_t cand)
{
    return reject_tiles_for(n, cand, 72);
}

int64_t polar_tiles_max(int64_t n);
size_t polar_workspace_bytes(int64_t n);

// Two-pass Polar (count pass, scan, write pass): header, int32 count and
// int64 prefix per tile (prefix has tiles_max + 1 entries).
size_t polar_twopass_workspace_bytes(int64_t n);

// ------------------------------------------------------------- launchers --
cudaError_t launch_uniform(float *out, int64_t n, uint64_t key, uint64_t counter, cudaStream_t s);
cudaError_t launch_philox_ceiling(uint32_t *out, int64_t nblocks, uint64_t key, uint64_t counter, cudaStream_t s);
cudaError_t launch_b1(void *out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                      int dtype, int mode, bool aligned, cudaStream_t s);
cudaError_t launch_polar(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s);
cudaError_t launch_set_u64(uint64_t *p, uint64_t v, cudaStream_t s);
cudaError_t launch_polar_twopass(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s);

// The paper's further methods (Sec. 3-5): B3, P2 and the Ratio method R.
cudaError_t launch_b3(void *out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter, int dtype,
                      bool aligned, cudaStream_t s);
cudaError_t launch_eval_points(int kind, int mode, const uint32_t *in, int64_t n, float mu, float sigma,
                               float *out, int32_t *accept, cudaStream_t s);
cudaError_t launch_polar_p2(const PolarParams &p, int dtype, bool aligned, cudaStream_t s);
cudaError_t launch_ratio(const PolarParams &p, int dtype, int mode, bool aligned, cudaStream_t s);
int64_t ratio_tiles_max(int64_t n);
size_t ratio_workspace_bytes(int64_t n);

// ---------------------------------------------------------------- reparam
cudaError_t launch_reparam_fwd(float *x, const float *mu, const float *sigma, int64_t n, int64_t m,
                               int64_t inner, uint64_t key, uint64_t counter, int mode, cudaStream_t s);
cudaError_t launch_reparam_bwd(float *dmu, float *dsigma, const float *g, int64_t n, int64_t m,
                               int64_t inner, uint64_t key, uint64_t counter, int mode, cudaStream_t s);

// ---------------------------------------------------------------- batched
struct BatchedConfig {
    int threads;
    int blocks_per_thread;
};

// Workspace of a batched call: header, then per-stream tables, then one tile
// status word per Polar tile of every Polar stream, then the item table.
struct BatchedCount {    // one stream's work, from its descriptor
    int32_t items;       // B1 items, or Polar primary items
    int32_t polar;       // 1 for a Polar stream with work (one overflow item)
    int64_t slots;       // tile status words (a Polar stream's tile budget)
};
static_assert(sizeof(BatchedCount) == 16, "a stream's record is one 16-byte load");
constexpr int kSetupThreads = 256;   // streams per CTA of the batched setup
constexpr int kSetupSums = 5;        // its look-back quantities (see k_batched.cu)
struct BatchedLayout {
    size_t slot_base;     // int64[k + 1]: first tile status word of each stream (the
                          // difference of neighbours: a Polar stream's tile budget)
    size_t stream_done;   // int32[k]: set once a Polar stream has all its pairs
    size_t counts;        // BatchedCount[k]
    size_t item_base;     // int64[2k]: a stream's first item-table entry, its overflow
                          // entry, each counted within its part of the table
    size_t setup_status;  // uint64[kSetupSums x setup CTAs]: the setup's look-back words
    size_t tile_status;   // uint64[slots]
};
__host__ __device__ inline BatchedLayout batched_layout(int32_t k)
{
    BatchedLayout L;
    const size_t ctas = ((size_t)k + kSetupThreads - 1) / kSetupThreads;
    L.slot_base = sizeof(WsHeader);
    L.stream_done = L.slot_base + (size_t)(k + 1) * 8;
    L.counts = (L.stream_done + (size_t)k * 4 + 15) / 16 * 16;
    L.item_base = L.counts + (size_t)k * sizeof(BatchedCount);
    L.setup_status = L.item_base + (size_t)k * 16;
    L.tile_status = (L.setup_status + ctas * kSetupSums * 8 + 255) / 256 * 256;
    return L;
}

struct BatchedParams {
    void *out;
    const nrng_stream_desc_t *desc;
    int32_t k;
    WsHeader *hdr;
    int64_t *slot_base;
    int *stream_done;
    BatchedCount *counts;
    int64_t *item_base;
    unsigned long long *setup_status;
    unsigned long long *tile_status;
    size_t ws_bytes;
    unsigned long long spin_limit_ns;
};
int batched_config_count();
BatchedConfig batched_config(int id);
int batched_default_config();
size_t batched_workspace_bytes(const nrng_stream_desc_t *h_desc, int32_t k);
cudaError_t launch_batched(void *out, const nrng_stream_desc_t *desc, int32_t k, int dtype, int mode,
                           void *ws, size_t ws_bytes, int config, cudaStream_t s);

// Test hooks read from the environment at each call (both off by default):
// NRNG_DEBUG_SILENT_TILE=t makes Polar tile t skip publishing its status, so
// that its successors' bounded look-back waits run out (NRNG_ERR_TIMEOUT);
// NRNG_DEBUG_POLAR_TILES=k caps a Polar call's tile budget at k tiles, so
// that a large n runs out of tiles (NRNG_ERR_EXHAUSTED).
long long debug_silent_tile();
int64_t debug_polar_tiles();

// Device properties cached per device.
int sm_count();
unsigned long long spin_limit_ns();

// Resident CTAs per SM of kernel `kern` at `threads` threads, computed on the
// first call and kept in `slot` (one per kernel instantiation and process).
// Host threads may call concurrently: the slot is a relaxed atomic, and
// concurrent first calls store the same value.
template <typename Kernel>
cudaError_t cached_occupancy(std::atomic<int> &slot, Kernel kern, int threads, int &occ)
{
    int o = slot.load(std::memory_order_relaxed);
    if (o == 0) {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, 0);
        if (e != cudaSuccess) return e;
        o = std::max(o, 1);
        slot.store(o, std::memory_order_relaxed);
    }
    occ = o;
    return cudaSuccess;
}

}  // namespace nrng
