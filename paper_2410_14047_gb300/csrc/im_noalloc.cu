// Estimate + argmax for callers that cannot allocate device memory.
//
// The allocating path (im_sketch_pick, im_select_seeds) keeps the kernel's
// scratch (one partial minimum per block and a completion ticket) in memory
// the context allocates.  This file holds the same scratch in one file-scope
// device array instead, so the entry point below never allocates: every GPU
// that loads the library holds the array (about 15 KB) until the process
// exits.  Host code may not use the array's name as a device address; the
// address is looked up with cudaGetSymbolAddress once per device.
#include <cstdint>
#include <mutex>

#include "../../include/difuser_im.h"
#include "im_launch.h"

namespace {

constexpr int kNoAllocMaxBlocks = 152 * 8;  // the largest grid pick_grid() returns

struct NoAllocScratch {
    unsigned long long part_S[kNoAllocMaxBlocks];
    int32_t part_u[kNoAllocMaxBlocks];
    unsigned int ticket;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_address(int dev, NoAllocScratch** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" im_status im_argmax_noalloc(const uint8_t* M, int32_t n, int32_t J, uint32_t* picked,
                                       void* cuda_stream, int32_t* s_out, uint64_t* S_out,
                                       double* est_out) {
    if (!M || !picked || !s_out || !S_out || !est_out) return IM_E_INVAL;
    // the kernel reads register rows as 16-byte vectors and the outputs as
    // naturally aligned words: a misaligned buffer (say, a slice of a larger
    // tensor at an odd offset) is refused here, before anything reaches the GPU
    if ((reinterpret_cast<uintptr_t>(M) & 15u) || (reinterpret_cast<uintptr_t>(picked) & 3u) ||
        (reinterpret_cast<uintptr_t>(s_out) & 3u) || (reinterpret_cast<uintptr_t>(S_out) & 7u) ||
        (reinterpret_cast<uintptr_t>(est_out) & 7u))
        return IM_E_INVAL;
    if (n < 1 || n >= (1 << 26)) return IM_E_RANGE;
    if (J < 16 || J > im::kMaxJ || (J & (J - 1)) != 0) return IM_E_INVAL;
    if (im::pick_grid(n, J) > kNoAllocMaxBlocks) return IM_E_RANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IM_E_CUDA;
    NoAllocScratch* sc = nullptr;
    if (scratch_address(dev, &sc) != cudaSuccess) return IM_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the ticket must start at zero; a previous call normally leaves it there
    if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return IM_E_CUDA;
    im::PickArgs a{};
    a.M = const_cast<uint8_t*>(M);  // read only: mark = 0 writes no register
    a.J = J;
    a.n = n;
    a.seed_bits = picked;
    a.part_S = sc->part_S;
    a.part_u = sc->part_u;
    a.ticket = &sc->ticket;
    a.out_seed = s_out;
    a.out_S = reinterpret_cast<unsigned long long*>(S_out);
    a.out_est = est_out;
    a.k = 0;
    a.mark = 0;
    a.tile = 4;  // the grid pick_grid(n, J) sized above
    if (im::launch_pick(a, st) != cudaSuccess) return IM_E_CUDA;
    return IM_OK;
}
