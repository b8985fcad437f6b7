// splash_sort_pairs_u32_noalloc: the onesweep pair sort for callers that
// cannot allocate device memory. Its scratch (ping-pong pair buffers, digit
// histograms, partition tickets, look-back flags and a status word) lives in
// one file-scope static __device__ array, so the call itself never allocates.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace {

using namespace splash;

constexpr int64_t kMaxPairs = 1 << 20;  // largest n this entry point accepts
constexpr int64_t kPartsMax = (kMaxPairs + kSortTile - 1) / kSortTile + 1;
constexpr size_t kPairWords = 2 * (size_t)kMaxPairs;                       // temp keys + temp values
constexpr size_t kScratchWords = 4 * kRadixMax + 64 + (size_t)kLookbackPerPart * kPartsMax;  // sort_scratch_carve layout
constexpr size_t kStatusWord = kPairWords + kScratchWords;
constexpr size_t kTotalWords = kStatusWord + 64;  // ~10 MB

// Resident in every device context that loads the library, until exit.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kTotalWords];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {};

// Device address of the static array on the current device. The first call
// on a device looks it up (cudaGetSymbolAddress, with that device current).
splash_status scratch_on_current_device(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        splash_set_error(std::string("splash_sort_pairs_u32_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SPLASH_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        splash_set_error("splash_sort_pairs_u32_noalloc: device index out of range");
        return SPLASH_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            splash_set_error(std::string("splash_sort_pairs_u32_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SPLASH_ERR_CUDA;
        }
        g_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_addr[dev];
    return SPLASH_OK;
}

}  // namespace

extern "C" splash_status splash_sort_pairs_u32_noalloc(const uint32_t *keys_in, const uint32_t *vals_in,
                                                       uint32_t *keys_out, uint32_t *vals_out, int64_t n,
                                                       int32_t key_bits, uint32_t *status_out, void *stream)
{
    if (n < 0 || n > kMaxPairs) {
        splash_set_error("splash_sort_pairs_u32_noalloc: n = " + std::to_string(n) + " is outside [0, " +
                         std::to_string(kMaxPairs) + "], the size of its static scratch");
        return SPLASH_ERR_INVALID_ARG;
    }
    if (key_bits < 0 || key_bits > 32) {
        splash_set_error("splash_sort_pairs_u32_noalloc: key_bits must be in 0..32");
        return SPLASH_ERR_INVALID_ARG;
    }
    if (n > 0 && (!keys_in || !keys_out || !vals_out)) {
        splash_set_error("splash_sort_pairs_u32_noalloc: null buffer");
        return SPLASH_ERR_INVALID_ARG;
    }
    if (n > 0 && (reinterpret_cast<uintptr_t>(keys_in) & 15)) {
        splash_set_error("splash_sort_pairs_u32_noalloc: keys_in must be 16-byte aligned");
        return SPLASH_ERR_INVALID_ARG;
    }
    uint32_t *base = nullptr;
    splash_status rc = scratch_on_current_device(&base);
    if (rc != SPLASH_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *status = base + kStatusWord;
    SPLASH_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    if (n > 0) {
        uint32_t *tk = base, *tv = base + kMaxPairs;
        SortScratch ss;
        sort_scratch_carve(base + kPairWords, kMaxPairs, &ss);  // histograms, tickets, look-back
        // sort_pairs clears the histograms, tickets and look-back flags it uses
        const int which = sort_pairs(keys_in, vals_in, keys_out, vals_out, tk, tv, n, nullptr, key_bits, ss, status,
                                     1 << 22, 0, s);
        if (which) {
            SPLASH_CUDA_TRY(cudaMemcpyAsync(keys_out, tk, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
            SPLASH_CUDA_TRY(cudaMemcpyAsync(vals_out, tv, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
        }
    }
    if (status_out) SPLASH_CUDA_TRY(cudaMemcpyAsync(status_out, status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
