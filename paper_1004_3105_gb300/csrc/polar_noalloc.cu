// polar_noalloc.cu -- nrng_polar_noalloc: the Polar generator of nrng_polar,
// for callers that cannot allocate device memory.
//
// Some callers of this library have no way to obtain the workspace nrng_polar
// asks for: code that is handed a fixed device-memory budget by the
// application that hosts it and may not call cudaMalloc behind its back, and
// latency-critical loops that avoid cudaMalloc because it can synchronise the
// device.  This entry point keeps its scratch (the look-back status words and
// the status header) in one file-scope device array of fixed size instead, so
// it allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine.  The caller still passes the output (and the optional outputs).
//
// Limits and sharing:
//   * the array holds kNoAllocScratchBytes = 1 MiB, enough for the tile words
//     of n <= kNoAllocMaxN normals; larger n is rejected with
//     NRNG_ERR_WORKSPACE before anything is enqueued;
//   * every GPU that loads the library holds this 1 MiB until the process
//     exits;
//   * every call on a device shares the one array, and it keeps the last
//     call's contents; each call clears the part it uses on its stream before
//     its kernel runs, so calls that are ordered on the GPU are independent,
//     but calls that overlap on the GPU (different streams, no ordering) race
//     on the array and give wrong results;
//   * the array's host-side name is only a stand-in for the device symbol: the
//     device address is obtained once per device with cudaGetSymbolAddress,
//     with that device current, by the first call on that device.  Make that
//     first call before any stream capture that would include it.  The cached
//     address assumes one CUDA context per device for the life of the
//     process: after cudaDeviceReset (or any teardown of the primary context)
//     the cached address is stale, so do not call this entry point again in
//     that process.
#include <mutex>

#include "nrng_internal.h"

namespace nrng {

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_polar_scratch[kNoAllocScratchBytes];

// Largest n whose workspace fits the array: the tile budget of n must satisfy
// sizeof(WsHeader) + 8 * tiles <= kNoAllocScratchBytes (checked per call).
constexpr int64_t kNoAllocMaxN = int64_t(1) << 28;

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mutex;
static void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device, with that device current).
static cudaError_t scratch_address(void **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_polar_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void k_copy_status(const WsHeader *h, int32_t *out) { *out = h->status; }

}  // namespace nrng

using namespace nrng;

extern "C" int32_t nrng_polar_noalloc(void *d_out, int64_t n, float mu, float sigma, uint64_t key,
                                      uint64_t counter, int32_t dtype, int32_t mode,
                                      uint64_t *d_next_counter, int64_t *d_pair_candidate,
                                      int32_t *d_status, nrng_stream_t stream)
{
    if (n < 0 || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (dtype != NRNG_F32 && dtype != NRNG_BF16 && dtype != NRNG_F16) return NRNG_ERR_INVALID_VALUE;
    if (mode != NRNG_ACCURATE && mode != NRNG_FAST) return NRNG_ERR_INVALID_VALUE;
    if (!(mu - mu == 0.0f) || !(sigma - sigma == 0.0f) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    const size_t esize = (dtype == NRNG_F32) ? 4 : 2;
    if ((uintptr_t)d_out % esize || (uintptr_t)d_next_counter % 8 || (uintptr_t)d_pair_candidate % 8 ||
        (uintptr_t)d_status % 4)
        return NRNG_ERR_MISALIGNED;
    // the fixed array bounds n; reject before touching the device
    if (n > kNoAllocMaxN || polar_workspace_bytes(n) > kNoAllocScratchBytes) return NRNG_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return NRNG_ERR_CUDA;
    if (n == 0) {
        if (d_next_counter && launch_set_u64(d_next_counter, counter, s) != cudaSuccess) return NRNG_ERR_CUDA;
        if (d_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NRNG_ERR_CUDA;
        return NRNG_OK;
    }
    const uint64_t max_blocks = (uint64_t)polar_tiles_max(n) * kPolarBlocksPerTile;
    if (counter > ~0ull - (max_blocks - 1)) return NRNG_ERR_COUNTER_OVERFLOW;
    PolarParams p;
    p.out = d_out;
    p.n = n;
    p.nitems = (n + 1) / 2;
    p.mu = mu;
    p.sigma = sigma;
    p.rk = round_keys(key);
    p.counter = counter;
    p.hdr = static_cast<WsHeader *>(scratch);
    p.tile_status = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + sizeof(WsHeader));
    p.tiles_max = polar_tiles_max(n);
    p.next_counter = d_next_counter;
    p.pair_cand = d_pair_candidate;
    p.spin_limit_ns = spin_limit_ns();
    p.debug_silent_tile = -1;
    const bool aligned = ((uintptr_t)d_out % (2 * esize)) == 0;
    // launch_polar clears the header and tile words it uses (cudaMemsetAsync on
    // the stream, no allocation) and then runs the look-back kernel.
    if (launch_polar(p, dtype, mode, aligned, s) != cudaSuccess) return NRNG_ERR_CUDA;
    if (d_status) {
        k_copy_status<<<1, 1, 0, s>>>(p.hdr, d_status);
        if (cudaGetLastError() != cudaSuccess) return NRNG_ERR_CUDA;
    }
    return NRNG_OK;
}
