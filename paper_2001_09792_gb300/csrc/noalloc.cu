// rg_radix_sort_pairs_noalloc: the radix sort of rg_radix_sort_pairs for
// callers that must not allocate device memory themselves or through us --
// for example code that runs while a stream is being captured into a CUDA
// graph (a plain cudaMalloc is refused during capture), code whose device
// memory is owned by a caching allocator that has already reserved what the
// GPU has free, or a frame loop that may not stall on an allocation.
//
// The sort's temporaries (ping-pong keys and values, per-tile digit counts)
// live in one fixed array in this file's device memory.  Host code only sees a
// host-side stand-in for that array's name, so the device address is looked
// up once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.  Every byte the sort reads from the array is written
// earlier in the same call, so nothing has to be cleared between calls; but
// all calls share the array, so calls whose GPU work overlaps race.
#include <cuda_runtime.h>

#include <mutex>

#include "rg_internal.cuh"

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kMaxPairs = RG_NOALLOC_SORT_MAX_PAIRS;
constexpr size_t kTilePairs = 2048;  // pairs per sort tile (one count block)
constexpr size_t kScratchBytes =
    align256(kMaxPairs * 8) + align256(kMaxPairs * 4) + align256(256 * ((kMaxPairs + kTilePairs - 1) / kTilePairs) * 4);

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" rg_status rg_radix_sort_pairs_noalloc(const void* d_keys, const uint32_t* d_vals, uint32_t n,
                                                 uint32_t key_bits, void* d_keys_out, uint32_t* d_vals_out,
                                                 void* stream) {
    if (key_bits != 32 && key_bits != 64) return rg::report_error(RG_ERR_INVALID_ARG, "key_bits must be 32 or 64");
    if (n > RG_NOALLOC_SORT_MAX_PAIRS)
        return rg::report_error(RG_ERR_INVALID_ARG,
                                "rg_radix_sort_pairs_noalloc: n exceeds RG_NOALLOC_SORT_MAX_PAIRS (262144)");
    if (n == 0) return RG_OK;
    if (!d_keys || !d_vals || !d_keys_out || !d_vals_out) return rg::report_error(RG_ERR_INVALID_ARG, "bad arguments");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rg::report_error(RG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rg::report_error(RG_ERR_INVALID_ARG, "device index out of range");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return rg::report_error(RG_ERR_CUDA, "cudaGetSymbolAddress of the sort scratch array failed");
            }
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    if (rg::radix_sort_scratch_bytes(n, (int)key_bits) > kScratchBytes)
        return rg::report_error(RG_ERR_INVALID_ARG, "sort scratch larger than the fixed array");
    e = rg::radix_sort_pairs(d_keys, d_vals, n, (int)key_bits, d_keys_out, d_vals_out, scratch,
                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rg::report_error(RG_ERR_CUDA, cudaGetErrorString(e));
    }
    return RG_OK;
}
