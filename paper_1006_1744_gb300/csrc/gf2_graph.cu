// gf2_graph.cu -- replay of repeated calls from CUDA graphs.
//
// One elimination is a few hundred dependent launches on two streams. A call
// whose arguments (pointers, sizes, options, device) equal an earlier call's is
// captured into a CUDA graph on its second occurrence and replayed from then
// on, which removes most of the launch gaps. The capture runs on a private
// origin stream (with a private side stream), so any caller stream, the legacy
// default stream included, can launch the graph. Replays see the current
// contents of the same buffers, so results are those of an eager call.
// Calls are not captured while launch timing is on, while the caller's stream
// is itself being captured, or when a capture fails (they then run eagerly); at
// most MAX_GRAPHS are kept, the least recently used is dropped.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "gf2_common.cuh"

namespace {

constexpr size_t MAX_GRAPHS = 32;

struct Entry {
    gf2::CallKey key;
    std::vector<char> extra;
    int state = 0;  // 1: seen once (ran eagerly), 2: replayable, -1: capture failed
    cudaGraphExec_t exec = nullptr;
    void *stage = nullptr;  // pinned host buffer read by the graph's host-to-device copies
    int launches = 0;       // kernel launches in the graph
    unsigned long long used = 0;
};

std::mutex g_mu;
std::vector<Entry> g_entries;
unsigned long long g_clock = 0;
std::atomic<int> g_on{1};
std::atomic<long long> g_captured{0}, g_replayed{0};
std::mutex g_capture_mu;  // one capture at a time (they share the private streams)
thread_local bool t_capturing = false;
thread_local void *t_stage = nullptr;

bool same(const Entry &e, const gf2::CallKey &k, const void *extra, size_t extra_bytes)
{
    return std::memcmp(&e.key, &k, sizeof(k)) == 0 && e.extra.size() == extra_bytes &&
           (extra_bytes == 0 || std::memcmp(e.extra.data(), extra, extra_bytes) == 0);
}

// a dropped graph may still be running (or about to read its staging buffer): wait
// for its own device first
void release(Entry &e)
{
    if (e.exec || e.stage) {
        int cur = 0;
        const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != e.key.device &&
                              cudaSetDevice(e.key.device) == cudaSuccess;
        cudaDeviceSynchronize();
        if (e.exec)
            cudaGraphExecDestroy(e.exec);
        if (e.stage)
            cudaFreeHost(e.stage);
        if (switched)
            cudaSetDevice(cur);
        cudaGetLastError();
    }
    e.exec = nullptr;
    e.stage = nullptr;
}

}  // namespace

namespace gf2 {

bool capturing_on_this_thread() { return t_capturing; }

void *capture_stage() { return t_capturing ? t_stage : nullptr; }

int run_replayed(const CallKey &key, cudaStream_t s, const std::function<int(cudaStream_t)> &body,
                 const void *extra, size_t extra_bytes, size_t stage_bytes)
{
    if (!g_on.load(std::memory_order_relaxed) || prof_timing_on())
        return body(s);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return body(s);
    }
    if (cs != cudaStreamCaptureStatusNone)
        return body(s);  // the caller is capturing: the launches go into its graph
    int state = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = std::find_if(g_entries.begin(), g_entries.end(),
                               [&](const Entry &e) { return same(e, key, extra, extra_bytes); });
        if (it == g_entries.end()) {
            if (g_entries.size() >= MAX_GRAPHS) {
                auto old = std::min_element(g_entries.begin(), g_entries.end(),
                                            [](const Entry &a, const Entry &b) { return a.used < b.used; });
                release(*old);
                g_entries.erase(old);
            }
            Entry e;
            e.key = key;
            if (extra_bytes)
                e.extra.assign((const char *)extra, (const char *)extra + extra_bytes);
            e.state = 1;
            e.used = ++g_clock;
            g_entries.push_back(e);
            state = 0;
        } else {
            it->used = ++g_clock;
            state = it->state;
            if (state == 2) {  // launched under the lock: no other thread can drop the graph meanwhile
                prof_launched(it->launches);
                g_replayed.fetch_add(1, std::memory_order_relaxed);
                return note_cuda(cudaGraphLaunch(it->exec, s));
            }
        }
    }
    if (state == 0 || state == -1)
        return body(s);  // first occurrence, or capture not possible: eagerly
    // second occurrence: capture on the private origin stream, instantiate, launch on s
    cudaGraphExec_t made = nullptr;
    void *stage = nullptr;
    int made_launches = 0;
    {
        std::lock_guard<std::mutex> lock(g_capture_mu);
        cudaStream_t origin = nullptr, side = nullptr;
        if (stage_bytes && cudaHostAlloc(&stage, stage_bytes, cudaHostAllocDefault) != cudaSuccess)
            stage = nullptr;
        if ((!stage_bytes || stage) && capture_streams(&origin, &side) == GF2_OK &&
            cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            t_capturing = true;
            t_stage = stage;
            const long long l0 = launches_by_thread();
            const int rc = body(origin);
            made_launches = (int)(launches_by_thread() - l0);
            t_capturing = false;
            t_stage = nullptr;
            cudaGraph_t graph = nullptr;
            cudaError_t err = cudaStreamEndCapture(origin, &graph);
            if (rc == GF2_OK && err == cudaSuccess && graph)
                err = cudaGraphInstantiate(&made, graph, 0);
            if (graph)
                cudaGraphDestroy(graph);
            if (err != cudaSuccess && made) {
                cudaGraphExecDestroy(made);
                made = nullptr;
            }
        }
        cudaGetLastError();  // a failed capture leaves nothing enqueued
        if (!made && stage) {
            cudaFreeHost(stage);
            stage = nullptr;
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = std::find_if(g_entries.begin(), g_entries.end(),
                               [&](const Entry &e) { return same(e, key, extra, extra_bytes); });
        if (it != g_entries.end() && it->state == 1) {
            it->state = made ? 2 : -1;
            it->exec = made;
            it->stage = stage;
            it->launches = made_launches;
            if (made) {
                g_captured.fetch_add(1, std::memory_order_relaxed);
                prof_launched(made_launches);
                return note_cuda(cudaGraphLaunch(made, s));
            }
        } else if (made) {  // dropped, or captured by another thread meanwhile (never launched)
            cudaGraphExecDestroy(made);
            if (stage)
                cudaFreeHost(stage);
        }
    }
    return body(s);  // nothing of the capture ran
}

}  // namespace gf2

extern "C" void gf2_replay_enable(int on) { g_on.store(on ? 1 : 0, std::memory_order_relaxed); }

extern "C" void gf2_replay_stats(long long *captured, long long *replayed)
{
    if (captured)
        *captured = g_captured.load(std::memory_order_relaxed);
    if (replayed)
        *replayed = g_replayed.load(std::memory_order_relaxed);
}
