// gf2_common.cuh -- shared internals of the GF(2) CUDA library (sm_103a).
//
// Bit layout (see include/gf2.h): column j of a row is bit (j & 63) of word
// j >> 6, least significant bit = leftmost column.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>

#include "../../include/gf2.h"

typedef unsigned long long u64;

#define GF2_FULL 0xffffffffu

// ---------------------------------------------------------------------------
// Per-call device state of the panel elimination (lives in the workspace).
// The pivot kernel of panel b writes it, the table sweep of panel b reads it.
// ---------------------------------------------------------------------------
struct PanelState {
    int r_cur;      // rank before the current panel
    int r_next;     // rank after the current panel
    int kbar;       // pivots found in the current panel (0..64)
    int status;     // sticky device-side error code (0 = ok)
    int zero_tail;  // 1 once every remaining row is zero in every remaining column
    int nz;         // set by this panel's sweep when it found no pivot but a nonzero word right of
                    // the panel in a trailing row (checked only then)
    int mode;       // form of this panel's sweep: 0 = PLS (trailing rows), 1 = reduced form (every row)
    int r_switch;   // hybrid: rank before the first panel swept in PLS form (INT_MAX while none)
    u64 J;          // pivot columns of the panel, as a bit mask of the panel word
    unsigned long long pop;  // hybrid: set bits of the trailing rows' next panel word, counted by this sweep
    int prow[64];   // physical row of pivot t (rows are never moved during elimination)
    int pcol[64];   // panel-relative column of pivot t
    u64 newblk[64]; // pivot t -> its final panel word (U_t plus its own multipliers)
    u64 zpiv[64];   // pivot t -> row t of L^-1: U_t as a sum of the ORIGINAL pivot rows O
    u64 zmap[64];   // column c -> row of (O_J)^-1 = U_J^-1 L^-1 for the pivot at c (0 elsewhere)
    u64 xmap[64];   // column c -> row of U_J^-1 for the pivot at c, scattered to the pivot columns
    // Row-order changes of this panel, applied to the position -> row map by the
    // next panel's pivot search (a sweep running meanwhile reads them from here):
    int nwin;        // window positions r_cur .. r_cur + nwin - 1 ...
    int nx;          // ... and nx positions past the window
    int wperm[128];  // window position - r_cur -> physical row
    int xpos[64];    // position past the window -> physical row xval
    int xval[64];
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 lowmask(int k)  // bits [0, k), k in [0, 64]
{
    return k >= 64 ? ~0ull : ((1ull << k) - 1ull);
}

__device__ __forceinline__ int ctz64(u64 x) { return __ffsll((long long)x) - 1; }

// Software parallel bit extract: the bits of x at the set positions of m,
// packed towards bit 0 (walks the runs of consecutive ones in m).
__device__ __forceinline__ u64 pext64(u64 x, u64 m)
{
    u64 r = 0;
    int k = 0;
    while (m) {
        int lo = ctz64(m);
        u64 s = m >> lo;
        int len = (~s == 0ull) ? 64 - lo : ctz64(~s);
        u64 run = lowmask(len);
        r |= ((x >> lo) & run) << k;
        k += len;
        m &= ~(run << lo);
    }
    return r;
}

// Software parallel bit deposit: the low bits of x placed at the set positions of m.
__device__ __forceinline__ u64 pdep64(u64 x, u64 m)
{
    u64 r = 0;
    int k = 0;
    while (m) {
        int lo = ctz64(m);
        u64 s = m >> lo;
        int len = (~s == 0ull) ? 64 - lo : ctz64(~s);
        u64 run = lowmask(len);
        r |= ((x >> k) & run) << lo;
        k += len;
        m &= ~(run << lo);
    }
    return r;
}

// MakeTable's Gray-code enumeration (Sec. 3.1) of the 16 sums base + {subsets
// of rows r0..r3}: entry gray(i) is entry gray(i - 1) plus one row, stored at
// T[gray(i) * ts]. The four rows come in registers, so the chain of stores
// never waits on a load that might alias them.
__device__ __forceinline__ void gray16(u64 base, u64 r0, u64 r1, u64 r2, u64 r3, u64 *__restrict__ T, int ts)
{
    u64 cur = base;
    T[0] = cur;
#pragma unroll
    for (int i = 1; i < 16; ++i) {
        const int k = __ffs(i) - 1;  // the row that changes between gray(i - 1) and gray(i)
        cur ^= k == 0 ? r0 : k == 1 ? r1 : k == 2 ? r2 : r3;
        T[(i ^ (i >> 1)) * ts] = cur;
    }
}

// Physical row at trailing position p >= r of the panel that st describes: its
// window order, its swaps past the window, else perm (which the next panel's
// pivot search may be rewriting meanwhile, at exactly those positions).
__device__ __forceinline__ int trailing_row(const int *__restrict__ perm, const PanelState *__restrict__ st, int r,
                                            int nwin, int nx, int p)
{
    if (p < r + nwin)
        return st->wperm[p - r];
    for (int x = 0; x < nx; ++x)
        if (st->xpos[x] == p)
            return st->xval[x];
    return perm[p];
}

// ---------------------------------------------------------------------------
// bounded waits and the device status word
// ---------------------------------------------------------------------------
// Every spin-wait in the library gives up after this long, records
// GF2_ETIMEOUT in the status word and lets its kernel finish.
#define GF2_WAIT_LIMIT_NS 2000000000ull

__device__ __forceinline__ u64 globaltimer_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// first error wins; later ones leave it in place until gf2_sync_status clears it
__device__ __forceinline__ void record_status(int *status, int code)
{
    if (status)
        atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
namespace gf2 {

int *status_word();  // device address of this device's status word (nullptr on failure)
int note_cuda(cudaError_t e);  // records e for gf2_last_cuda_error, returns GF2_ECUDA or GF2_OK

// a side stream of the current device for overlapped work (gf2_pls.cu)
int side_stream(cudaStream_t *out);

// events that order two streams within one call, released when the call returns
struct EventSet {
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    EventSet() = default;
    EventSet(const EventSet &) = delete;
    EventSet &operator=(const EventSet &) = delete;
    ~EventSet()
    {
        for (cudaEvent_t x : ev)
            if (x)
                cudaEventDestroy(x);  // released once the recorded work completes
    }
    int create()
    {
        for (cudaEvent_t &x : ev) {
            cudaError_t err = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
            if (err != cudaSuccess)
                return note_cuda(err);
        }
        return GF2_OK;
    }
};

// Replay of repeated calls from CUDA graphs (gf2_graph.cu): the key holds every
// argument that the launches depend on; body enqueues the call on its stream.
// Graph replay of repeated calls (gf2_graph.cu). The key is everything a call's
// launches depend on; the stream is not part of it (graphs are captured on a
// private stream and launched on the caller's). body(st) enqueues the call's
// work on st.
struct CallKey {
    int op, device, tile_words, grid;
    const void *A;
    int64_t m, n, stride;
    const void *P, *Q, *rank, *pivots, *work;
    size_t work_bytes;
};
// extra (nullable): further bytes the launches depend on (compared bytewise, e.g.
// a batch's item list); stage_bytes: size of a pinned host buffer the graph owns,
// which body reaches through capture_stage() while it is being captured (host
// data that the graph copies to the device, unchanged for every replay).
int run_replayed(const CallKey &key, cudaStream_t s, const std::function<int(cudaStream_t)> &body,
                 const void *extra = nullptr, size_t extra_bytes = 0, size_t stage_bytes = 0);
bool capturing_on_this_thread();  // side_stream() then hands out the private capture side stream
void *capture_stage();            // the capture's pinned buffer (nullptr outside a capture)
// private streams of the current device for captures: origin and side (gf2_pls.cu)
int capture_streams(cudaStream_t *origin, cudaStream_t *side);
// Function attributes (the dynamic shared-memory limit) are per device: a launch site
// keeps a mask of the devices it has set them on (setting twice is harmless).
inline bool attr_needed(const std::atomic<unsigned long long> &devs)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return true;
    return !((devs.load(std::memory_order_relaxed) >> dev) & 1ull);
}
inline void attr_done(std::atomic<unsigned long long> &devs)
{
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64)
        devs.fetch_or(1ull << dev, std::memory_order_relaxed);
}
bool prof_timing_on();  // launch timing (events around launches) is enabled
long long launches_by_thread();  // all launches this thread has made (profiling on or off)

// argument checks and the internal per-device workspace (gf2_api.cu)
int get_work(void *&work, size_t &work_bytes, size_t need);  // caller's work if given, else the internal one
int check_mat(const void *A, int64_t m, int64_t n, int64_t stride);
int check_opts(const gf2_opts *o);

void prof_launched(int count);              // counts kernel launches when profiling is on
int prof_begin(cudaStream_t s);             // event before a timed launch (-1: profiling off)
void prof_end(cudaStream_t s, int cls, int token);
int sm_count();                // streaming multiprocessors of the current device
size_t align_up(size_t x, size_t a);

// Workspace carve-up of the panel elimination for an m x n matrix.
struct ElimLayout {
    size_t state;   // PanelState[2]: panel b writes state b & 1 and reads the other
    size_t perm;    // int32[m]: position -> physical row
    size_t side;    // u64[2][m]: panel word of each physical row (double buffered)
    size_t pmask;   // u64[W]: pivot-column mask
    size_t out;     // u64[m * stride]: rows in final order (pls / rref), or the copy (rank)
    size_t rref_b;  // rref: non-pivot part of S, compacted
    size_t rref_x;  // rref: solved non-pivot part
    size_t rref_d;  // rref: inverses of the 64x64 diagonal blocks
    size_t ups;     // rref: u64[2][m]: panel word of each row above the panel, by position (double buffered)
    size_t total;
};
int64_t min_stride(int64_t n);
ElimLayout elim_layout(int op, int64_t m, int64_t n, int pps = 1);  // pps: panels per sweep (1 or 2)
int pps_choice(const gf2_opts *o, int64_t m, int64_t n);           // panels per sweep of a PLS-form elimination

// The state a finished elimination leaves its rank in: the one of its last panel.
__host__ __device__ inline PanelState *final_state(PanelState *st, int64_t W) { return st + ((W + 1) & 1); }

struct Elim {
    uint64_t *A;      // matrix being eliminated (caller's A, or the copy for rank)
    int64_t m, n, stride, W;
    PanelState *st;   // the two panel states
    PanelState *stf;  // final_state(st, W): rank and pivots after elim_run
    int *perm;
    u64 *side;
    u64 *pmask;
    uint64_t *out;    // final-order rows (nullptr for rank)
    int64_t ostride;  // row pitch of out, words (minimal: ceil(n/64) rounded up to 16)
    u64 *ups;         // reduced form: panel word of the rows above, by position, double buffered (2 x m)
    int64_t *P, *Q;   // nullable for rank
    cudaStream_t s;
    int tile_words, grid;
    int mode;         // table sweeps: 0 = PLS (trailing rows), 1 = reduced echelon form (every row),
                      // 2 = hybrid (reduced form until the density reaches hybrid_permille, then PLS)
    int hybrid_permille;
    int k;            // bits per Gray-code table of the 16-word PLS-form sweep: 8 or 4
    int pps;          // panels per table sweep (PLS form): 1, or 2 (gf2_pair.cu: state slots b & 3)
};

// One matrix of a batched elimination (device-resident array, one per matrix).
struct ElimDesc {
    uint64_t *A;
    int64_t stride;
    PanelState *st;
    int *perm;
    u64 *side;
    u64 *pmask;
    uint64_t *out;
    int64_t ostride;
    int64_t *P, *Q, *rank;
    int m, n, W, pad;
};

// Batched panel elimination (gf2_pls.cu). Step b runs panel b of the nact
// matrices idx[0..nact) in two launches; the sweep's CTAs are split among them
// by the prefix pre[0..nact] (matrix idx[j] gets CTAs pre[j]..pre[j+1]-1).
int batch_init(const ElimDesc *D, int count, int max_m, cudaStream_t s);
int batch_pivot(const ElimDesc *D, const int *idx, int nact, int b, cudaStream_t s);
int batch_sweep(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b, int tile_words,
                cudaStream_t s);
int batch_finish(const ElimDesc *D, int count, int max_m, cudaStream_t s);
// The whole batch in one persistent cooperative launch (one CTA per SM): team t < nteams (CTAs
// team_start[t] .. + team_size[t]; team_of[cta] = its team or -1) takes the matrices
// big[team_first[t] .. team_first[t + 1]), then every CTA takes the matrices small[0 .. nsmall)
// from a work queue. All arrays are device memory; counters: nteams + 2 ints.
struct PersistArrays {
    const int *team_of, *team_start, *team_size, *team_first, *big, *small;
};
int batch_persistent(const ElimDesc *D, int nteams, const PersistArrays &a, int nsmall, int *counters,
                     cudaStream_t s);
int batch_persistent_grid();  // CTAs of that launch
int sweep_rows_per_pass(int tile_words);
// table sweep of panel b over 16-word tiles (gf2_sweep.cu), in the form e.mode selects
int launch_sweep16(const Elim &e, int b, cudaStream_t s);
// the same for panel b of a batch (PLS form), CTAs shared out as for batch_sweep
int batch_sweep16(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b, int k, cudaStream_t s);
constexpr int SWEEP16_ROWS = 128;  // rows per block of work of the 16-word sweep
int sweep_ctas_per_sm(int tile_words);

// panel elimination: runs every panel; afterwards st->r_next is the rank.
int elim_run(const Elim &e);
// The same, with the side stream and the three ordering events supplied by the caller
// (elim_run(e) takes a side stream of the device and creates and releases its own events).
struct ElimAux {
    cudaStream_t side;
    cudaEvent_t ev[3];
};
int elim_run(const Elim &e, const ElimAux &aux);
// two panels per sweep (gf2_pair.cu), and the pieces of gf2_pls.cu it uses
int elim_run_pair(const Elim &e, const ElimAux &aux);
int apply_final_order(const Elim &e);
// rank of A (unchanged) by a direct elimination of a copy in work (gf2_api.cu): never replayed
// from a graph, allocates nothing
int rank_direct(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, char *work,
                const ElimAux &aux, cudaStream_t s);
// writes P/Q identity fill, rank, gathers rows into e.out in final order
int elim_gather(const Elim &e, int64_t *rank);
// compress L in e.out and copy e.out back into e.A
int pls_finish(const Elim &e);
// RREF from the eliminated rows in e.out, written into e.A
int rref_finish(const Elim &e, const ElimLayout &L, char *work, int64_t *rank, int64_t *pivots);
// RREF of an elimination in reduced form (e.mode 1): gather, copy back, pivots
int m4ri_finish(const Elim &e, int64_t *rank, int64_t *pivots);
// product
int mul_xor(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb,
            int64_t m, int64_t k, int64_t n, int acc, int tile_words, int grid, cudaStream_t s);
int mul_tensor(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb,
               int64_t m, int64_t k, int64_t n, int acc, void *work, size_t work_bytes, cudaStream_t s);
size_t mul_tensor_workspace(int64_t m, int64_t k, int64_t n);
// Strassen-Winograd product (gf2_strassen.cu): leaf = smallest dimension recursed on,
// leaf_kind = GF2_PRODUCT_XOR or GF2_PRODUCT_TENSOR
constexpr int64_t STRASSEN_LEAF_DEFAULT = 8192;
size_t mul_strassen_workspace(int64_t m, int64_t k, int64_t n, int64_t leaf, int leaf_kind);
int mul_strassen(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
                 int64_t k, int64_t n, int accumulate, void *work, size_t work_bytes, int64_t leaf, int leaf_kind,
                 cudaStream_t s);
// recursive PLS (gf2_rec.cu)
size_t rec_workspace_bytes(int64_t m, int64_t n, int64_t cutoff);
int pls_recursive(uint64_t *A, int64_t stride, int64_t m, int64_t n, int64_t *P, int64_t *Q, int64_t *rank,
                  char *work, const gf2_opts *opts, cudaStream_t s);

}  // namespace gf2
