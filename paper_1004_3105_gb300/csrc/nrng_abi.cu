// nrng_abi.cu -- the extern "C" entry points declared in include/nrng.h:
// argument validation (nothing is enqueued on a host-detectable error),
// workspace sizing, kernel dispatch, the device status word, the batched
// autotuner and CUDA graph capture.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <climits>
#include <atomic>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nrng_internal.h"

namespace nrng {

// An NVTX range around each entry point that enqueues GPU work, so that a
// timeline tool shows every call by name (a no-op without a tool attached).
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};

// ------------------------------------------------------------- helpers ----
static int log_level()
{
    static int level = [] {
        const char *e = std::getenv("NRNG_LOG");
        return e ? std::atoi(e) : 0;
    }();
    return level;
}

static void log_msg(const char *fmt, ...)
{
    if (log_level() <= 0) return;
    va_list ap;
    va_start(ap, fmt);
    std::fprintf(stderr, "[nrng] ");
    std::vfprintf(stderr, fmt, ap);
    std::fprintf(stderr, "\n");
    va_end(ap);
}

static int32_t cuda_status(cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return NRNG_OK;
    log_msg("%s: %s", where, cudaGetErrorString(e));
    return NRNG_ERR_CUDA;
}

RoundKeys round_keys(uint64_t key)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)key, k1 = (uint32_t)(key >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += 0x9E3779B9u;   // Philox-4x32 Weyl key increments (Salmon et al., SC'11)
        k1 += 0xBB67AE85u;
    }
    return rk;
}

int sm_count()
{
    // per device; relaxed atomics, since concurrent first calls store the same value
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        v = v > 0 ? v : 148;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

unsigned long long spin_limit_ns()
{
    static unsigned long long v = [] {
        const char *e = std::getenv("NRNG_LOOKBACK_SPIN_LIMIT_MS");
        const double ms = e ? std::atof(e) : 500.0;
        return (unsigned long long)((ms > 0 ? ms : 500.0) * 1e6);
    }();
    return v;
}

long long debug_silent_tile()
{
    const char *e = std::getenv("NRNG_DEBUG_SILENT_TILE");
    return e ? std::atoll(e) : -1;
}

int64_t debug_polar_tiles()
{
    const char *e = std::getenv("NRNG_DEBUG_POLAR_TILES");
    return e ? std::atoll(e) : 0;
}

static bool finite_f(float v) { return std::isfinite(v); }
// Largest element (or point) count a call takes: far above any device
// memory, and low enough that no size arithmetic on it can overflow int64.
constexpr int64_t kMaxElements = int64_t(1) << 60;

static bool valid_dtype(int32_t d) { return d == NRNG_F32 || d == NRNG_BF16 || d == NRNG_F16; }
static bool valid_mode(int32_t m) { return m == NRNG_ACCURATE || m == NRNG_FAST; }
static size_t dtype_size(int32_t d) { return d == NRNG_F32 ? 4 : 2; }

// counter + blocks - 1 must not pass 2^64 - 1.
static bool counter_fits(uint64_t counter, uint64_t blocks)
{
    return blocks == 0 || counter <= ULLONG_MAX - (blocks - 1);
}

// Batched configuration pinned per (dtype, mode); -1 = default.
static std::mutex g_cfg_mutex;
static int g_cfg[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};

// NRNG_FORCE_CONFIG=<id> replaces the built-in default configuration (a
// configuration pinned with nrng_batched_set_config still wins); an id out
// of range is ignored.
static int env_default_config()
{
    static int v = [] {
        const char *e = std::getenv("NRNG_FORCE_CONFIG");
        if (e == nullptr || *e < '0' || *e > '9') return -1;   // unset, empty or not a number
        const int c = std::atoi(e);
        return c < batched_config_count() ? c : -1;
    }();
    return v;
}

static int batched_config_for(int32_t dtype, int32_t mode)
{
    std::lock_guard<std::mutex> lock(g_cfg_mutex);
    const int c = g_cfg[dtype][mode];
    if (c >= 0) return c;
    const int forced = env_default_config();
    return forced >= 0 ? forced : batched_default_config();
}

// ---------------------------------------------------------- autotune cache
// One JSON line per tuned workload in the file named by NRNG_AUTOTUNE_CACHE.
// The fingerprint covers what the timing depends on: every stream's length
// and method (not its key, counter, mu or sigma).
static uint64_t workload_fingerprint(const nrng_stream_desc_t *h, int32_t k)
{
    uint64_t x = 1469598103934665603ull;   // FNV-1a, 64-bit
    auto mix = [&x](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            x ^= (v >> (8 * b)) & 0xFFu;
            x *= 1099511628211ull;
        }
    };
    for (int32_t j = 0; j < k; ++j) {
        mix((uint64_t)h[j].n);
        mix((uint64_t)(uint32_t)h[j].method);
    }
    return x;
}

static const char *kCacheLine =
    "{\"kernel\": \"batched\", \"dtype\": %d, \"mode\": %d, \"streams\": %d, \"fingerprint\": \"%016llx\", "
    "\"config\": %d, \"threads\": %d, \"blocks_per_thread\": %d, \"ms\": %f}";

static bool cache_lookup(const char *path, int32_t dtype, int32_t mode, int32_t k, uint64_t fp, int &cfg, float &ms)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        int d = -1, m = -1, kk = -1, c = -1, th = 0, bpt = 0;
        unsigned long long g = 0;
        float t = 0.0f;
        if (std::sscanf(line, kCacheLine, &d, &m, &kk, &g, &c, &th, &bpt, &t) == 8 && d == dtype && m == mode &&
            kk == k && g == fp && c >= 0 && c < batched_config_count()) {
            cfg = c;   // the last matching line wins
            ms = t;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void cache_store(const char *path, int32_t dtype, int32_t mode, int32_t k, uint64_t fp, int cfg, float ms)
{
    if (FILE *f = std::fopen(path, "a")) {
        const BatchedConfig c = batched_config(cfg);
        std::fprintf(f, kCacheLine, dtype, mode, k, (unsigned long long)fp, cfg, c.threads, c.blocks_per_thread,
                     (double)ms);
        std::fputc('\n', f);
        std::fclose(f);
    }
}

}  // namespace nrng

using namespace nrng;

extern "C" {

const char *nrng_status_string(int32_t status)
{
    switch (status) {
    case NRNG_OK: return "NRNG_OK";
    case NRNG_ERR_INVALID_VALUE: return "NRNG_ERR_INVALID_VALUE: bad size, pointer, parameter or enum";
    case NRNG_ERR_MISALIGNED: return "NRNG_ERR_MISALIGNED: pointer not aligned to its element type";
    case NRNG_ERR_WORKSPACE: return "NRNG_ERR_WORKSPACE: workspace missing or too small";
    case NRNG_ERR_COUNTER_OVERFLOW: return "NRNG_ERR_COUNTER_OVERFLOW: Philox counter would pass 2^64";
    case NRNG_ERR_CUDA: return "NRNG_ERR_CUDA: a CUDA call or launch failed";
    case NRNG_ERR_TIMEOUT: return "NRNG_ERR_TIMEOUT: a look-back wait ran out";
    case NRNG_ERR_EXHAUSTED: return "NRNG_ERR_EXHAUSTED: Polar stream ran out of workspace tiles";
    case NRNG_ERR_NOT_SUPPORTED: return "NRNG_ERR_NOT_SUPPORTED";
    default: return "NRNG_ERR_UNKNOWN";
    }
}

int32_t nrng_abi_version(void) { return 1; }

int32_t nrng_uniform(float *d_out, int64_t n, uint64_t key, uint64_t counter, nrng_stream_t stream)
{
    const CallRange range("nrng_uniform");
    if (n < 0 || n > kMaxElements || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % 4) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    if (!counter_fits(counter, (uint64_t)((n + 3) / 4))) return NRNG_ERR_COUNTER_OVERFLOW;
    return cuda_status(launch_uniform(d_out, n, key, counter, (cudaStream_t)stream), "nrng_uniform");
}

int32_t nrng_philox_ceiling(uint32_t *d_out, int64_t nblocks, uint64_t key, uint64_t counter, nrng_stream_t stream)
{
    const CallRange range("nrng_philox_ceiling");
    if (nblocks < 0 || (nblocks > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % 4) return NRNG_ERR_MISALIGNED;
    if (nblocks == 0) return NRNG_OK;
    // 32-bit block indices and a low counter word that does not wrap
    if (nblocks > (int64_t(1) << 31) || (uint64_t)(uint32_t)counter + (uint64_t)nblocks > (uint64_t(1) << 32))
        return NRNG_ERR_NOT_SUPPORTED;
    return cuda_status(launch_philox_ceiling(d_out, nblocks, key, counter, (cudaStream_t)stream),
                       "nrng_philox_ceiling");
}

int32_t nrng_boxmuller(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                       int32_t dtype, int32_t mode, nrng_stream_t stream)
{
    const CallRange range("nrng_boxmuller");
    if (n < 0 || n > kMaxElements || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype) || !(valid_mode(mode) || mode == NRNG_B2)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % dtype_size(dtype)) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    if (!counter_fits(counter, (uint64_t)((n + 3) / 4))) return NRNG_ERR_COUNTER_OVERFLOW;
    const bool aligned = ((uintptr_t)d_out % (4 * dtype_size(dtype))) == 0;
    return cuda_status(launch_b1(d_out, n, mu, sigma, key, counter, dtype, mode, aligned, (cudaStream_t)stream),
                       "nrng_boxmuller");
}

int32_t nrng_polar_workspace_size(int64_t n, size_t *h_bytes)
{
    if (h_bytes == nullptr || n < 0 || n > kPolarMaxN) return NRNG_ERR_INVALID_VALUE;
    *h_bytes = polar_workspace_bytes(n);
    return NRNG_OK;
}

int32_t nrng_polar_max_blocks(int64_t n, uint64_t *h_blocks)
{
    if (h_blocks == nullptr || n < 0 || n > kPolarMaxN) return NRNG_ERR_INVALID_VALUE;
    *h_blocks = (n == 0) ? 0 : (uint64_t)polar_tiles_max(n) * kPolarBlocksPerTile;
    return NRNG_OK;
}

int32_t nrng_polar(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                   int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes, uint64_t *d_next_counter,
                   int64_t *d_pair_candidate, nrng_stream_t stream)
{
    const CallRange range("nrng_polar");
    if (n < 0 || n > kPolarMaxN || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype) || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % dtype_size(dtype) || (uintptr_t)d_ws % 8 || (uintptr_t)d_next_counter % 8 ||
        (uintptr_t)d_pair_candidate % 8)
        return NRNG_ERR_MISALIGNED;
    if (n == 0) {
        // nothing drawn: the continuation counter is the starting counter
        if (d_next_counter)
            return cuda_status(launch_set_u64(d_next_counter, counter, (cudaStream_t)stream), "nrng_polar");
        return NRNG_OK;
    }
    if (d_ws == nullptr || ws_bytes < polar_workspace_bytes(n)) return NRNG_ERR_WORKSPACE;
    const uint64_t max_blocks = (uint64_t)polar_tiles_max(n) * kPolarBlocksPerTile;
    if (!counter_fits(counter, max_blocks)) return NRNG_ERR_COUNTER_OVERFLOW;
    PolarParams p;
    p.out = d_out;
    p.n = n;
    p.nitems = (n + 1) / 2;
    p.mu = mu;
    p.sigma = sigma;
    p.rk = round_keys(key);
    p.counter = counter;
    p.hdr = static_cast<WsHeader *>(d_ws);
    p.tile_status = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ws) + sizeof(WsHeader));
    p.tiles_max = polar_tiles_max(n);
    if (debug_polar_tiles() > 0 && debug_polar_tiles() < p.tiles_max) p.tiles_max = debug_polar_tiles();
    p.debug_silent_tile = debug_silent_tile();
    p.next_counter = d_next_counter;
    p.pair_cand = d_pair_candidate;
    p.spin_limit_ns = spin_limit_ns();
    const bool aligned = ((uintptr_t)d_out % (2 * dtype_size(dtype))) == 0;
    return cuda_status(launch_polar(p, dtype, mode, aligned, (cudaStream_t)stream), "nrng_polar");
}

int32_t nrng_polar_twopass_workspace_size(int64_t n, size_t *h_bytes)
{
    if (h_bytes == nullptr || n < 0 || n > kPolarMaxN) return NRNG_ERR_INVALID_VALUE;
    *h_bytes = polar_twopass_workspace_bytes(n);
    return NRNG_OK;
}

int32_t nrng_polar_twopass(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                           int32_t dtype, int32_t mode, void *d_ws, size_t ws_bytes, uint64_t *d_next_counter,
                           int64_t *d_pair_candidate, nrng_stream_t stream)
{
    const CallRange range("nrng_polar_twopass");
    if (n < 0 || n > kPolarMaxN || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype) || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % dtype_size(dtype) || (uintptr_t)d_ws % 256 || (uintptr_t)d_next_counter % 8 ||
        (uintptr_t)d_pair_candidate % 8)
        return NRNG_ERR_MISALIGNED;
    if (n == 0) {
        if (d_next_counter)
            return cuda_status(launch_set_u64(d_next_counter, counter, (cudaStream_t)stream), "nrng_polar_twopass");
        return NRNG_OK;
    }
    if (d_ws == nullptr || ws_bytes < polar_twopass_workspace_bytes(n)) return NRNG_ERR_WORKSPACE;
    const uint64_t max_blocks = (uint64_t)polar_tiles_max(n) * kPolarBlocksPerTile;
    if (!counter_fits(counter, max_blocks)) return NRNG_ERR_COUNTER_OVERFLOW;
    PolarParams p;
    p.out = d_out;
    p.n = n;
    p.nitems = (n + 1) / 2;
    p.mu = mu;
    p.sigma = sigma;
    p.rk = round_keys(key);
    p.counter = counter;
    p.hdr = static_cast<WsHeader *>(d_ws);
    p.tile_status = nullptr;
    p.tiles_max = polar_tiles_max(n);
    if (debug_polar_tiles() > 0 && debug_polar_tiles() < p.tiles_max) p.tiles_max = debug_polar_tiles();
    p.next_counter = d_next_counter;
    p.pair_cand = d_pair_candidate;
    p.spin_limit_ns = spin_limit_ns();
    p.debug_silent_tile = -1;
    const bool aligned = ((uintptr_t)d_out % (2 * dtype_size(dtype))) == 0;
    return cuda_status(launch_polar_twopass(p, dtype, mode, aligned, (cudaStream_t)stream), "nrng_polar_twopass");
}

int32_t nrng_boxmuller_b3(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                          int32_t dtype, nrng_stream_t stream)
{
    const CallRange range("nrng_boxmuller_b3");
    if (n < 0 || n > kMaxElements || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % dtype_size(dtype)) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    if (n > (INT64_MAX / 3) || !counter_fits(counter, 3 * (uint64_t)((n + 7) / 8)))
        return NRNG_ERR_COUNTER_OVERFLOW;
    const bool aligned = ((uintptr_t)d_out % (4 * dtype_size(dtype))) == 0;
    return cuda_status(launch_b3(d_out, n, mu, sigma, key, counter, dtype, aligned, (cudaStream_t)stream),
                       "nrng_boxmuller_b3");
}

// Shared checks and parameters of the single-stream rejection calls (P2, R).
static int32_t reject_params(PolarParams &p, void *d_out, int64_t n, int64_t nitems, float mu, float sigma,
                             uint64_t key, uint64_t counter, int32_t dtype, void *d_ws, size_t ws_bytes,
                             size_t ws_need, int64_t tiles, int blocks_per_tile, uint64_t *d_next_counter,
                             int64_t *d_cand)
{
    if ((uintptr_t)d_out % dtype_size(dtype) || (uintptr_t)d_ws % 8 || (uintptr_t)d_next_counter % 8 ||
        (uintptr_t)d_cand % 8)
        return NRNG_ERR_MISALIGNED;
    if (d_ws == nullptr || ws_bytes < ws_need) return NRNG_ERR_WORKSPACE;
    if (!counter_fits(counter, (uint64_t)tiles * blocks_per_tile)) return NRNG_ERR_COUNTER_OVERFLOW;
    p.out = d_out;
    p.n = n;
    p.nitems = nitems;
    p.mu = mu;
    p.sigma = sigma;
    p.rk = round_keys(key);
    p.counter = counter;
    p.hdr = static_cast<WsHeader *>(d_ws);
    p.tile_status = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_ws) + sizeof(WsHeader));
    p.tiles_max = tiles;
    if (debug_polar_tiles() > 0 && debug_polar_tiles() < p.tiles_max) p.tiles_max = debug_polar_tiles();
    p.debug_silent_tile = debug_silent_tile();
    p.next_counter = d_next_counter;
    p.pair_cand = d_cand;
    p.spin_limit_ns = spin_limit_ns();
    return NRNG_OK;
}

int32_t nrng_polar_p2(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter,
                      int32_t dtype, void *d_ws, size_t ws_bytes, uint64_t *d_next_counter,
                      int64_t *d_pair_candidate, nrng_stream_t stream)
{
    const CallRange range("nrng_polar_p2");
    if (n < 0 || n > kPolarMaxN || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if (n == 0) {
        if ((uintptr_t)d_next_counter % 8) return NRNG_ERR_MISALIGNED;
        if (d_next_counter)
            return cuda_status(launch_set_u64(d_next_counter, counter, (cudaStream_t)stream), "nrng_polar_p2");
        return NRNG_OK;
    }
    PolarParams p;
    const int32_t st = reject_params(p, d_out, n, (n + 1) / 2, mu, sigma, key, counter, dtype, d_ws, ws_bytes,
                                     polar_workspace_bytes(n), polar_tiles_max(n), kPolarBlocksPerTile,
                                     d_next_counter, d_pair_candidate);
    if (st != NRNG_OK) return st;
    const bool aligned = ((uintptr_t)d_out % (2 * dtype_size(dtype))) == 0;
    return cuda_status(launch_polar_p2(p, dtype, aligned, (cudaStream_t)stream), "nrng_polar_p2");
}

int32_t nrng_ratio_workspace_size(int64_t n, size_t *h_bytes)
{
    if (h_bytes == nullptr || n < 0 || n > kPolarMaxN) return NRNG_ERR_INVALID_VALUE;
    *h_bytes = ratio_workspace_bytes(n);
    return NRNG_OK;
}

int32_t nrng_ratio(void *d_out, int64_t n, float mu, float sigma, uint64_t key, uint64_t counter, int32_t dtype,
                   int32_t mode, void *d_ws, size_t ws_bytes, uint64_t *d_next_counter, int64_t *d_candidate,
                   nrng_stream_t stream)
{
    const CallRange range("nrng_ratio");
    if (n < 0 || n > kPolarMaxN || (n > 0 && d_out == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype) || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if (n == 0) {
        if ((uintptr_t)d_next_counter % 8) return NRNG_ERR_MISALIGNED;
        if (d_next_counter)
            return cuda_status(launch_set_u64(d_next_counter, counter, (cudaStream_t)stream), "nrng_ratio");
        return NRNG_OK;
    }
    PolarParams p;
    const int32_t st = reject_params(p, d_out, n, n, mu, sigma, key, counter, dtype, d_ws, ws_bytes,
                                     ratio_workspace_bytes(n), ratio_tiles_max(n), kRatioBlocksPerTile,
                                     d_next_counter, d_candidate);
    if (st != NRNG_OK) return st;
    const bool aligned = ((uintptr_t)d_out % (2 * dtype_size(dtype))) == 0;
    return cuda_status(launch_ratio(p, dtype, mode, aligned, (cudaStream_t)stream), "nrng_ratio");
}

int32_t nrng_eval_points(int32_t kind, int32_t mode, const void *d_in, int64_t n, float mu, float sigma,
                         float *d_out, int32_t *d_accept, nrng_stream_t stream)
{
    const CallRange range("nrng_eval_points");
    if (kind < NRNG_POINTS_B1 || kind > NRNG_POINTS_B3) return NRNG_ERR_INVALID_VALUE;
    if (!(valid_mode(mode) || (mode == NRNG_B2 && kind == NRNG_POINTS_B1))) return NRNG_ERR_INVALID_VALUE;
    if (n < 0 || n > kMaxElements || (n > 0 && (d_in == nullptr || d_out == nullptr))) return NRNG_ERR_INVALID_VALUE;
    if (!finite_f(mu) || !finite_f(sigma) || sigma < 0.0f) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_in % 4 || (uintptr_t)d_out % 4 || (uintptr_t)d_accept % 4) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    return cuda_status(launch_eval_points(kind, mode, static_cast<const uint32_t *>(d_in), n, mu, sigma, d_out,
                                          d_accept, (cudaStream_t)stream),
                       "nrng_eval_points");
}

int32_t nrng_batched_workspace_size(const nrng_stream_desc_t *h_desc, int32_t k, size_t *h_bytes)
{
    if (h_bytes == nullptr || k < 0 || (k > 0 && h_desc == nullptr)) return NRNG_ERR_INVALID_VALUE;
    for (int32_t j = 0; j < k; ++j)
        if (h_desc[j].n > kMaxElements) return NRNG_ERR_INVALID_VALUE;
    *h_bytes = batched_workspace_bytes(h_desc, k);
    return NRNG_OK;
}

static int32_t batched_check(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k, int32_t dtype,
                             int32_t mode, void *d_ws, size_t ws_bytes)
{
    if (k < 0 || (k > 0 && (d_out == nullptr || d_desc == nullptr))) return NRNG_ERR_INVALID_VALUE;
    if (!valid_dtype(dtype) || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_out % dtype_size(dtype) || (uintptr_t)d_desc % 8 || (uintptr_t)d_ws % 256)
        return NRNG_ERR_MISALIGNED;
    if (k > 0 && (d_ws == nullptr || ws_bytes < batched_layout(k).tile_status)) return NRNG_ERR_WORKSPACE;
    return NRNG_OK;
}

int32_t nrng_batched(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k, int32_t dtype, int32_t mode,
                     void *d_ws, size_t ws_bytes, nrng_stream_t stream)
{
    const CallRange range("nrng_batched");
    const int32_t st = batched_check(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes);
    if (st != NRNG_OK || k == 0) return st;
    return cuda_status(launch_batched(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes,
                                      batched_config_for(dtype, mode), (cudaStream_t)stream),
                       "nrng_batched");
}

int32_t nrng_reparam_fwd(float *d_x, const float *d_mu, const float *d_sigma, int64_t n, int64_t m,
                         int64_t inner, uint64_t key, uint64_t counter, int32_t mode, nrng_stream_t stream)
{
    const CallRange range("nrng_reparam_fwd");
    if (n < 0 || n > kMaxElements || m < 1 || inner < 1 || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if (n > 0 && (d_x == nullptr || d_mu == nullptr || d_sigma == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (m > INT64_MAX / inner || n % (m * inner) != 0) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_x % 4 || (uintptr_t)d_mu % 4 || (uintptr_t)d_sigma % 4) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    if (!counter_fits(counter, (uint64_t)((n + 3) / 4))) return NRNG_ERR_COUNTER_OVERFLOW;
    return cuda_status(launch_reparam_fwd(d_x, d_mu, d_sigma, n, m, inner, key, counter, mode,
                                          (cudaStream_t)stream), "nrng_reparam_fwd");
}

int32_t nrng_reparam_bwd(float *d_dmu, float *d_dsigma, const float *d_g, int64_t n, int64_t m, int64_t inner,
                         uint64_t key, uint64_t counter, int32_t mode, nrng_stream_t stream)
{
    const CallRange range("nrng_reparam_bwd");
    if (n < 0 || n > kMaxElements || m < 1 || inner < 1 || !valid_mode(mode)) return NRNG_ERR_INVALID_VALUE;
    if (n > 0 && (d_dsigma == nullptr || d_g == nullptr)) return NRNG_ERR_INVALID_VALUE;
    if (m > INT64_MAX / inner || n % (m * inner) != 0) return NRNG_ERR_INVALID_VALUE;
    if ((uintptr_t)d_dmu % 4 || (uintptr_t)d_dsigma % 4 || (uintptr_t)d_g % 4) return NRNG_ERR_MISALIGNED;
    if (n == 0) return NRNG_OK;
    if (!counter_fits(counter, (uint64_t)((n + 3) / 4))) return NRNG_ERR_COUNTER_OVERFLOW;
    return cuda_status(launch_reparam_bwd(d_dmu, d_dsigma, d_g, n, m, inner, key, counter, mode,
                                          (cudaStream_t)stream), "nrng_reparam_bwd");
}

int32_t nrng_get_status(const void *d_ws, nrng_stream_t stream, int32_t *h_status)
{
    const CallRange range("nrng_get_status");
    if (d_ws == nullptr || h_status == nullptr) return NRNG_ERR_INVALID_VALUE;
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, d_ws, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e, "nrng_get_status");
    *h_status = v;
    return NRNG_OK;
}

// ------------------------------------------------------ autotune/graphs ---
int32_t nrng_batched_config_count(void) { return batched_config_count(); }

int32_t nrng_batched_config_info(int32_t config, int32_t *h_threads, int32_t *h_blocks_per_thread)
{
    if (config < 0 || config >= batched_config_count() || !h_threads || !h_blocks_per_thread)
        return NRNG_ERR_INVALID_VALUE;
    const BatchedConfig c = batched_config(config);
    *h_threads = c.threads;
    *h_blocks_per_thread = c.blocks_per_thread;
    return NRNG_OK;
}

int32_t nrng_batched_set_config(int32_t dtype, int32_t mode, int32_t config)
{
    if (!valid_dtype(dtype) || !valid_mode(mode) || config < -1 || config >= batched_config_count())
        return NRNG_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_cfg_mutex);
    g_cfg[dtype][mode] = config;
    return NRNG_OK;
}

int32_t nrng_batched_get_config(int32_t dtype, int32_t mode, int32_t *h_config)
{
    if (!valid_dtype(dtype) || !valid_mode(mode) || h_config == nullptr) return NRNG_ERR_INVALID_VALUE;
    *h_config = batched_config_for(dtype, mode);
    return NRNG_OK;
}

int32_t nrng_batched_autotune(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k, int32_t dtype,
                              int32_t mode, void *d_ws, size_t ws_bytes, int32_t reps, nrng_stream_t stream,
                              int32_t *h_config, float *h_ms)
{
    const CallRange range("nrng_batched_autotune");
    int32_t st = batched_check(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes);
    if (st != NRNG_OK) return st;
    if (k == 0 || reps < 1) return NRNG_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;

    // A cached choice for the same workload shape is reused without timing.
    const char *cache = std::getenv("NRNG_AUTOTUNE_CACHE");
    uint64_t fp = 0;
    if (cache) {
        std::vector<nrng_stream_desc_t> h((size_t)k);
        if (cudaMemcpyAsync(h.data(), d_desc, sizeof(nrng_stream_desc_t) * (size_t)k, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return NRNG_ERR_CUDA;
        fp = workload_fingerprint(h.data(), k);
        int cfg = -1;
        float ms = 0.0f;
        if (cache_lookup(cache, dtype, mode, k, fp, cfg, ms)) {
            nrng_batched_set_config(dtype, mode, cfg);
            if (h_config) *h_config = cfg;
            if (h_ms) *h_ms = ms;
            log_msg("autotune: cached config %d for %d streams (%016llx)", cfg, k, (unsigned long long)fp);
            return NRNG_OK;
        }
    }

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return NRNG_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return NRNG_ERR_CUDA; }
    int best = -1;
    float best_ms = 0.0f;
    st = NRNG_OK;
    for (int c = 0; c < batched_config_count() && st == NRNG_OK; ++c) {
        // one untimed launch (warm-up, and its status must be clean)
        st = cuda_status(launch_batched(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes, c, s), "autotune");
        if (st != NRNG_OK) break;
        int32_t dev_status = 0;
        st = nrng_get_status(d_ws, stream, &dev_status);
        if (st != NRNG_OK) break;
        if (dev_status != NRNG_OK) { st = dev_status; break; }
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == NRNG_OK; ++r)
            st = cuda_status(launch_batched(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes, c, s), "autotune");
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = NRNG_ERR_CUDA;
        if (st != NRNG_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        log_msg("autotune config %d (%d threads x %d blocks): %.4f ms", c, batched_config(c).threads,
                batched_config(c).blocks_per_thread, ms);
        if (best < 0 || ms < best_ms) { best = c; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NRNG_OK) return st;
    nrng_batched_set_config(dtype, mode, best);
    if (h_config) *h_config = best;
    if (h_ms) *h_ms = best_ms;
    if (cache) cache_store(cache, dtype, mode, k, fp, best, best_ms);
    return NRNG_OK;
}

struct NrngGraph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

int32_t nrng_batched_graph_create(void *d_out, const nrng_stream_desc_t *d_desc, int32_t k, int32_t dtype,
                                  int32_t mode, void *d_ws, size_t ws_bytes, nrng_stream_t stream,
                                  void **h_graph)
{
    const CallRange range("nrng_batched_graph_create");
    if (h_graph == nullptr || stream == nullptr) return NRNG_ERR_INVALID_VALUE;
    int32_t st = batched_check(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes);
    if (st != NRNG_OK) return st;
    if (k == 0) return NRNG_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e, "graph capture begin");
    const cudaError_t le = launch_batched(d_out, d_desc, k, dtype, mode, d_ws, ws_bytes,
                                          batched_config_for(dtype, mode), s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(le != cudaSuccess ? le : e, "graph capture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_status(e, "graph instantiate");
    }
    *h_graph = new NrngGraph{g, ex};
    return NRNG_OK;
}

int32_t nrng_graph_launch(void *h_graph, nrng_stream_t stream)
{
    const CallRange range("nrng_graph_launch");
    if (h_graph == nullptr) return NRNG_ERR_INVALID_VALUE;
    return cuda_status(cudaGraphLaunch(static_cast<NrngGraph *>(h_graph)->exec, (cudaStream_t)stream),
                       "graph launch");
}

int32_t nrng_graph_destroy(void *h_graph)
{
    if (h_graph == nullptr) return NRNG_ERR_INVALID_VALUE;
    NrngGraph *g = static_cast<NrngGraph *>(h_graph);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return NRNG_OK;
}

}  // extern "C"
