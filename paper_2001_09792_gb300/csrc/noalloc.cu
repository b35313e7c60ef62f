// rg_radix_sort_pairs_noalloc: the radix sort of rg_radix_sort_pairs for
// callers that cannot allocate device memory themselves or through us -- for
// example code whose device memory is owned by a caching allocator that has
// already reserved what the GPU has free (a cudaMalloc behind its back fails or
// fragments its pool), or a frame loop that may not stall on an allocation.
//
// The sort's temporaries (ping-pong keys and values, per-tile digit counts)
// live in one fixed array in this file's device memory.  Host code only sees a
// host-side stand-in for that array's name, so the device address is looked
// up once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.  That cached address belongs to the device's current
// context: it does not survive cudaDeviceReset.  Every byte the sort reads
// from the array is written earlier in the same call, so nothing has to be
// cleared between calls; but all calls share the array, so calls whose GPU
// work overlaps race.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "rg_internal.cuh"

namespace {

// sized for the largest call: RG_NOALLOC_SORT_MAX_PAIRS pairs of 64-bit keys
constexpr size_t kScratchBytes = rg::radix_sort_scratch_bytes(RG_NOALLOC_SORT_MAX_PAIRS, 64);
static_assert(kScratchBytes >= rg::radix_sort_scratch_bytes(RG_NOALLOC_SORT_MAX_PAIRS, 32),
              "32-bit keys need no more scratch than 64-bit keys");

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" rg_status rg_radix_sort_pairs_noalloc(const void* d_keys, const uint32_t* d_vals, uint32_t n,
                                                 uint32_t key_bits, void* d_keys_out, uint32_t* d_vals_out,
                                                 void* stream) {
    if (key_bits != 32 && key_bits != 64) return rg::report_error(RG_ERR_INVALID_ARG, "key_bits must be 32 or 64");
    if (n > RG_NOALLOC_SORT_MAX_PAIRS) {
        char msg[128];
        snprintf(msg, sizeof msg, "rg_radix_sort_pairs_noalloc: n = %u exceeds RG_NOALLOC_SORT_MAX_PAIRS (%u)", n,
                 (unsigned)RG_NOALLOC_SORT_MAX_PAIRS);
        return rg::report_error(RG_ERR_INVALID_ARG, msg);
    }
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
    e = rg::radix_sort_pairs(d_keys, d_vals, n, (int)key_bits, d_keys_out, d_vals_out, scratch,
                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rg::report_error(RG_ERR_CUDA, cudaGetErrorString(e));
    }
    return RG_OK;
}
