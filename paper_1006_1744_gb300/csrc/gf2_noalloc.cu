// gf2_noalloc.cu -- rank with no device allocation at all.
//
// Some callers cannot call cudaMalloc. A plug-in embedded in a host application
// that owns the whole device-memory budget (and hands out no allocator) is not
// allowed to; a latency-bound loop cannot take the device-wide synchronisation
// and the milliseconds that cudaMalloc and cudaFree may cost; a process whose
// device memory is already reserved by another framework's caching allocator
// may find that an allocation fails. For them, gf2_rank_noalloc takes its
// workspace from one fixed array compiled into the library.
//
// The array lives in device memory of every GPU that loads the library and
// stays allocated until the process exits. Host code cannot use its name as an
// address (on the host it only names a stand-in object), so the device address
// is looked up once per device with cudaGetSymbolAddress, with that device
// current, and cached. The same one-time set-up creates the side stream and the
// three events the elimination orders its two streams with, so that a call
// creates nothing. Each call runs the elimination directly: it is never
// recorded into or replayed from a library-owned CUDA graph.
#include <mutex>

#include "gf2_common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_scratch[GF2_NOALLOC_SCRATCH_BYTES];

struct DeviceSetup {
    void *scratch = nullptr;  // device address of g_scratch on this device
    gf2::ElimAux aux{};       // side stream and ordering events, kept until exit
    bool ready = false;
};

std::mutex g_mu;  // held for the whole call: set-up and enqueueing of concurrent host calls are serialised
DeviceSetup g_dev[64];

// One-time set-up of the current device (dev): symbol address, side stream, events.
int setup_device(int dev)
{
    DeviceSetup &d = g_dev[dev];
    if (d.ready)
        return GF2_OK;
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
        return gf2::note_cuda(e);
    gf2::ElimAux aux{};
    e = cudaStreamCreateWithFlags(&aux.side, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&aux.ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : aux.ev)
            if (x)
                cudaEventDestroy(x);
        if (aux.side)
            cudaStreamDestroy(aux.side);
        return gf2::note_cuda(e);
    }
    d.scratch = p;
    d.aux = aux;
    d.ready = true;
    return GF2_OK;
}

}  // namespace

extern "C" int gf2_rank_noalloc(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank,
                                void *stream)
{
    int rc = gf2::check_mat(A, m, n, stride);
    if (rc)
        return rc;
    if (!rank)
        return GF2_EINVAL;
    // everything the elimination writes (row order, panel words, state, the copy of A)
    // must fit in the fixed array; k_init resets the state and row order on every call
    const size_t need = gf2::elim_layout(GF2_OP_RANK, m, n).total;
    if (need > (size_t)GF2_NOALLOC_SCRATCH_BYTES)
        return GF2_ETOOBIG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return gf2::note_cuda(e);
    if (dev < 0 || dev >= 64)
        return GF2_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if ((rc = setup_device(dev)))
        return rc;
    const DeviceSetup &d = g_dev[dev];
    return gf2::rank_direct(A, m, n, stride, rank, static_cast<char *>(d.scratch), d.aux, (cudaStream_t)stream);
}
