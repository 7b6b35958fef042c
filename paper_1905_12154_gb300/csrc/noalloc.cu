// noalloc.cu -- bfm_poisson_noalloc: the Neumann Poisson solve with no
// workspace argument, for callers that cannot allocate device memory.
//
// Some callers have no way to hand the library a workspace: code whose device
// memory is owned and fully reserved by another memory manager, services that
// forbid allocation after start-up because cudaMalloc/cudaFree synchronise the
// device and stall other work, or thin foreign-language bindings with no
// device allocator at all.  For them this entry point keeps its scratch (the
// FFT twiddle / digit-reversal / eigenvalue tables, the FP64 partial sums and
// the reduction state of bfm_poisson) in one file-scope device array of
// kScratchBytes.  The array exists once per device in every process that loads
// the library and stays resident until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; later calls on that device reuse it.
//
// Nothing in the array needs to start at zero: every call rewrites the tables,
// every partial sum it reads and the reduction state before reading them.
// All calls on one device share the array, so calls whose GPU work overlaps
// (on different streams, or from different host threads) race on it.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(1) << 20;   // 1 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_poisson_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
bfm_status scratch_on_current_device(unsigned char** out)
{
    int dev = -1;
    BFM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        bfm::set_last_error("bfm_poisson_noalloc: device index out of range");
        return BFM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_poisson_scratch);
        if (e != cudaSuccess) return bfm::cuda_status(e, "cudaGetSymbolAddress(g_poisson_scratch)");
        if (!p || (reinterpret_cast<uintptr_t>(p) & 255u)) {
            bfm::set_last_error("bfm_poisson_noalloc: scratch array is not 256-byte aligned");
            return BFM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return BFM_OK;
}

}  // namespace

extern "C" bfm_status bfm_poisson_noalloc(const void* f, void* g_out, const bfm_grid* grid,
                                          bfm_precision prec, double* G_out, void* stream)
{
    bfm::Grid g;
    if (prec != BFM_FP32 && prec != BFM_FP64) return BFM_ERR_INVALID_ARG;
    if (!bfm::make_grid(grid, &g)) {
        bfm::set_last_error("grid must have ndim 2 or 3 and 2 <= n <= 8192 per axis");
        return BFM_ERR_INVALID_ARG;
    }
    bfm::FftRadices rs;
    for (int a = 0; a < g.ndim; ++a)
        if (!bfm::fft_radices(g.n[a], &rs)) {
            bfm::set_last_error("every n[a] must be 2^p 3^q");
            return BFM_ERR_UNSUPPORTED;
        }
    if (!f || !g_out) return BFM_ERR_INVALID_ARG;
    const size_t need = bfm::poisson_scratch_bytes(g, prec == BFM_FP64 ? 8 : 4);
    if (need > kScratchBytes) {
        bfm::set_last_error("bfm_poisson_noalloc: this grid needs more than the 1 MiB of "
                            "built-in scratch; use bfm_poisson with a workspace");
        return BFM_ERR_UNSUPPORTED;
    }
    unsigned char* scratch = nullptr;
    bfm_status s = scratch_on_current_device(&scratch);
    if (s != BFM_OK) return s;
    return bfm::poisson_on_scratch(f, g_out, g, prec, G_out, scratch, (cudaStream_t)stream);
}
