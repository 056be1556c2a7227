// gf2_prof.cu -- optional launch counting and per-kernel CUDA-event timing.
//
// Off by default. When enabled, every kernel launch of the library is
// counted, and (flag 2) each launch of a timed kernel class is bracketed by a
// pair of CUDA events recorded on the launching stream; gf2_prof_collect()
// waits for those events and accumulates the elapsed times per class.
#include <atomic>
#include <mutex>
#include <vector>

#include "gf2_common.cuh"

namespace gf2 {

namespace {
struct Prof {
    std::mutex mu;
    std::atomic<int> flags{0};
    std::atomic<long long> launches{0};
    std::vector<cudaEvent_t> pool;
    struct Pair {
        int cls, a, b;
    };
    std::vector<Pair> pending;
    size_t next = 0;
    double ms[GF2_PROF_CLASSES] = {};
    long long n[GF2_PROF_CLASSES] = {};
};
Prof &prof()
{
    static Prof p;
    return p;
}

int take_event(Prof &p)
{
    if (p.next == p.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess)
            return -1;
        p.pool.push_back(e);
    }
    return (int)p.next++;
}
}  // namespace

bool prof_timing_on() { return prof().flags.load(std::memory_order_relaxed) & 2; }

// every launch of this thread, counted or not (lets a replayed graph report its launches)
static thread_local long long t_all_launches = 0;
long long launches_by_thread() { return t_all_launches; }

void prof_launched(int count)
{
    t_all_launches += count;
    Prof &p = prof();
    if ((p.flags.load(std::memory_order_relaxed) & 1) && !capturing_on_this_thread())  // a capture runs nothing
        p.launches.fetch_add(count, std::memory_order_relaxed);
}

int prof_begin(cudaStream_t s)
{
    Prof &p = prof();
    if (!(p.flags.load(std::memory_order_relaxed) & 2))
        return -1;
    std::lock_guard<std::mutex> lock(p.mu);
    int a = take_event(p);
    if (a >= 0)
        cudaEventRecord(p.pool[a], s);
    return a;
}

void prof_end(cudaStream_t s, int cls, int a)
{
    if (a < 0)
        return;
    Prof &p = prof();
    std::lock_guard<std::mutex> lock(p.mu);
    int b = take_event(p);
    if (b < 0)
        return;
    cudaEventRecord(p.pool[b], s);
    p.pending.push_back({cls, a, b});
}

}  // namespace gf2

using namespace gf2;

extern "C" {

void gf2_prof_enable(int flags)
{
    prof().flags.store(flags);
}

void gf2_prof_reset(void)
{
    Prof &p = prof();
    std::lock_guard<std::mutex> lock(p.mu);
    p.launches.store(0);
    p.pending.clear();
    p.next = 0;
    for (int c = 0; c < GF2_PROF_CLASSES; ++c) {
        p.ms[c] = 0;
        p.n[c] = 0;
    }
}

long long gf2_prof_launches(void) { return prof().launches.load(); }

int gf2_prof_collect(int cls, double *ms_total, long long *launches)
{
    Prof &p = prof();
    std::lock_guard<std::mutex> lock(p.mu);
    for (const auto &pr : p.pending) {
        cudaError_t e = cudaEventSynchronize(p.pool[pr.b]);
        if (e != cudaSuccess)
            return note_cuda(e);
        float ms = 0;
        e = cudaEventElapsedTime(&ms, p.pool[pr.a], p.pool[pr.b]);
        if (e != cudaSuccess)
            return note_cuda(e);
        p.ms[pr.cls] += ms;
        p.n[pr.cls] += 1;
    }
    p.pending.clear();
    p.next = 0;
    if (cls < 0 || cls >= GF2_PROF_CLASSES)
        return GF2_EINVAL;
    if (ms_total)
        *ms_total = p.ms[cls];
    if (launches)
        *launches = p.n[cls];
    return GF2_OK;
}

}  // extern "C"
