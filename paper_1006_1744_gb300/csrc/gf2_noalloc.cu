// gf2_noalloc.cu -- rank with no device allocation at all.
//
// Some callers may not call cudaMalloc: code that runs while a CUDA graph is
// being captured (a plain allocation there breaks the capture), latency-bound
// loops where an allocation would stall the device, and plug-ins whose host
// application owns all device memory and hands out no allocator. For them,
// gf2_rank_noalloc takes its workspace from one fixed array compiled into the
// library instead of asking for memory.
//
// The array lives in device memory of every GPU that loads the library and
// stays allocated until the process exits. Host code cannot use its name as an
// address (on the host it only names a stand-in object), so the device address
// is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "gf2_common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_scratch[GF2_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_addr[64] = {};

// Device address of g_scratch on the current device (looked up on first use).
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return gf2::note_cuda(e);
    if (dev < 0 || dev >= 64)
        return GF2_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return gf2::note_cuda(e);
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GF2_OK;
}

}  // namespace

extern "C" int gf2_rank_noalloc(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank,
                                void *stream)
{
    if (m < 0 || n < 0 || m > INT32_MAX - 64 || n > INT32_MAX - 64)
        return GF2_EINVAL;
    // everything the elimination writes (row order, panel words, state, the copy of A)
    // must fit in the fixed array; k_init resets the state and row order on every call
    const size_t need = gf2::elim_layout(GF2_OP_RANK, m, n).total;
    if (need > (size_t)GF2_NOALLOC_SCRATCH_BYTES)
        return GF2_ETOOBIG;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc)
        return rc;
    return gf2_rank(A, m, n, stride, rank, scratch, (size_t)GF2_NOALLOC_SCRATCH_BYTES, nullptr, stream);
}
