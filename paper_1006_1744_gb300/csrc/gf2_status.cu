// gf2_status.cu -- the per-device status word that bounded waits report into.
//
// A kernel whose wait gives up cannot return an error code to the host call
// that launched it (the call has long returned), so it records the code in a
// word of device memory compiled into the library; gf2_sync_status reads and
// clears it.
#include <mutex>

#include "gf2_common.cuh"

namespace {

static __device__ int g_status;
static __device__ int g_never_set;  // the flag gf2_diag_wait_timeout waits on

std::mutex g_mu;
int *g_addr[64] = {};
int *g_never_addr[64] = {};

int lookup(int **status, int **never)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return GF2_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *a = nullptr, *b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_status);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress(&b, g_never_set);
        if (e != cudaSuccess)
            return gf2::note_cuda(e);
        g_addr[dev] = (int *)a;
        g_never_addr[dev] = (int *)b;
    }
    *status = g_addr[dev];
    if (never)
        *never = g_never_addr[dev];
    return GF2_OK;
}

// Spins on *flag (never set) until limit_ns have passed, then records GF2_ETIMEOUT.
__global__ void k_wait_flag(const volatile int *flag, u64 limit_ns, int *status)
{
    if (threadIdx.x != 0)
        return;
    const u64 t0 = globaltimer_ns();
    for (;;) {
        if (*flag != 0)
            return;
        if (globaltimer_ns() - t0 > limit_ns) {
            record_status(status, GF2_ETIMEOUT);
            return;
        }
        __nanosleep(1000);
    }
}

}  // namespace

namespace gf2 {

int *status_word()
{
    int *st = nullptr;
    return lookup(&st, nullptr) == GF2_OK ? st : nullptr;
}

}  // namespace gf2

extern "C" {

int gf2_sync_status(void *stream)
{
    int *st = nullptr;
    int rc = lookup(&st, nullptr);
    if (rc)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int value = 0;
    cudaError_t e = cudaMemcpyAsync(&value, st, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return gf2::note_cuda(e);
    if (value != 0) {
        e = cudaMemsetAsync(st, 0, sizeof(int), s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return gf2::note_cuda(e);
    }
    return value;
}

int gf2_diag_wait_timeout(uint64_t limit_ns, void *stream)
{
    int *st = nullptr, *never = nullptr;
    int rc = lookup(&st, &never);
    if (rc)
        return rc;
    if (limit_ns > GF2_WAIT_LIMIT_NS)
        limit_ns = GF2_WAIT_LIMIT_NS;
    k_wait_flag<<<1, 32, 0, (cudaStream_t)stream>>>(never, (u64)limit_ns, st);
    gf2::prof_launched(1);
    return gf2::note_cuda(cudaGetLastError());
}

}  // extern "C"
