// gf2_batch.cu -- gf2_pls_batched: MMPF block elimination of many independent
// matrices, one launch per panel step over all matrices that have that panel.
//
// The host plans the schedule from the sizes alone: step b runs the pivot
// search of panel b on every matrix with W > b (one warp each) and one table
// sweep whose CTAs are shared out in proportion to an upper bound of each
// matrix's trailing work, m x (W - b) words. The plan, the per-matrix
// descriptors and the per-matrix elimination workspaces live in the caller's
// (or the internal) workspace; the plan goes up in one copy from a pinned
// staging buffer.
#include <mutex>
#include <vector>
#include <cstring>

#include "gf2_common.cuh"

namespace {

using gf2::align_up;

struct BatchLayout {
    size_t descs, idx, pre, mats, total;
    int64_t n_idx, n_pre;
    int Wmax, max_m;
};

BatchLayout batch_layout(const gf2_batch_item *items, int64_t count)
{
    BatchLayout L{};
    int64_t sumW = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t W = (items[i].n + 63) / 64;
        if (items[i].m > 0 && W > 0)
            sumW += W;
        if (W > L.Wmax)
            L.Wmax = (int)W;
        if (items[i].m > L.max_m)
            L.max_m = (int)items[i].m;
    }
    L.n_idx = sumW;
    L.n_pre = sumW + L.Wmax;
    size_t off = 0;
    L.descs = off;
    off = align_up(off + (size_t)count * sizeof(gf2::ElimDesc), 256);
    L.idx = off;
    off = align_up(off + (size_t)L.n_idx * sizeof(int), 256);
    L.pre = off;
    off = align_up(off + (size_t)(L.n_pre + 1) * sizeof(int), 256);
    L.mats = off;
    for (int64_t i = 0; i < count; ++i)
        off = align_up(off + gf2::elim_layout(GF2_OP_PLS, items[i].m, items[i].n).total, 256);
    L.total = off;
    return L;
}

// pinned staging for the plan upload, one per device; the event marks when the
// previous upload has left the buffer
struct Staging {
    std::mutex mu;
    void *host = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
};
Staging g_stage[64];

int upload(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return gf2::note_cuda(e);
    if (dev < 0 || dev >= 64)
        return GF2_EINVAL;
    Staging &S = g_stage[dev];
    std::lock_guard<std::mutex> lock(S.mu);
    if (!S.ev && (e = cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming)) != cudaSuccess)
        return gf2::note_cuda(e);
    if ((e = cudaEventSynchronize(S.ev)) != cudaSuccess)
        return gf2::note_cuda(e);
    if (S.bytes < bytes) {
        if (S.host)
            cudaFreeHost(S.host);
        S.host = nullptr;
        S.bytes = 0;
        if (cudaHostAlloc(&S.host, bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return GF2_ENOMEM;
        }
        S.bytes = bytes;
    }
    memcpy(S.host, src, bytes);
    if ((e = cudaMemcpyAsync(dst, S.host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return gf2::note_cuda(e);
    return gf2::note_cuda(cudaEventRecord(S.ev, s));
}

int check_sizes(const gf2_batch_item *items, int64_t count)
{
    if (count < 0 || count > INT32_MAX / 2 || (count > 0 && !items))
        return GF2_EINVAL;
    for (int64_t i = 0; i < count; ++i) {
        const gf2_batch_item &it = items[i];
        if (it.m < 0 || it.n < 0 || it.m > INT32_MAX - 64 || it.n > INT32_MAX - 64 || it.stride < (it.n + 63) / 64)
            return GF2_EINVAL;
    }
    return GF2_OK;
}

int check_items(const gf2_batch_item *items, int64_t count)
{
    if (count < 0 || count > INT32_MAX / 2 || (count > 0 && !items))
        return GF2_EINVAL;
    for (int64_t i = 0; i < count; ++i) {
        const gf2_batch_item &it = items[i];
        int rc = gf2::check_mat(it.A, it.m, it.n, it.stride);
        if (rc)
            return rc;
        if ((it.m > 0 && !it.P) || (it.n > 0 && !it.Q))
            return GF2_EINVAL;
    }
    return GF2_OK;
}

int batched_run(const gf2_batch_item *items, int64_t count, int64_t *ranks, char *w, const BatchLayout &L, int tw,
                cudaStream_t s);

}  // namespace

extern "C" {

size_t gf2_pls_batched_workspace_bytes(const gf2_batch_item *items, int64_t count, const gf2_opts *opts)
{
    if (gf2::check_opts(opts) || check_sizes(items, count))
        return 0;
    return batch_layout(items, count).total;
}

int gf2_pls_batched(const gf2_batch_item *items, int64_t count, int64_t *ranks, void *work, size_t work_bytes,
                    const gf2_opts *opts, void *stream)
{
    int rc = gf2::check_opts(opts);
    if (rc || (rc = check_items(items, count)))
        return rc;
    if (count == 0)
        return GF2_OK;
    if (!ranks)
        return GF2_EINVAL;
    const BatchLayout L = batch_layout(items, count);
    if ((rc = gf2::get_work(work, work_bytes, L.total)))
        return rc;
    const int tw = (opts && opts->tile_words) ? opts->tile_words : 16;
    // a repeated call (same items, ranks, workspace, options) replays a captured graph
    gf2::CallKey key;
    std::memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.op = -GF2_OP_PLS;
    key.tile_words = tw;
    key.m = count;
    key.rank = ranks;
    key.work = work;
    key.work_bytes = work_bytes;
    return gf2::run_replayed(
        key, (cudaStream_t)stream,
        [&](cudaStream_t s) { return batched_run(items, count, ranks, (char *)work, L, tw, s); }, items,
        (size_t)count * sizeof(gf2_batch_item), L.mats);
}

}  // extern "C"

namespace {

int batched_run(const gf2_batch_item *items, int64_t count, int64_t *ranks, char *w, const BatchLayout &L, int tw,
                cudaStream_t s)
{
    int rc = GF2_OK;

    // host image of descriptors + plan, uploaded in one copy
    std::vector<char> img(L.mats);
    gf2::ElimDesc *D = reinterpret_cast<gf2::ElimDesc *>(img.data() + L.descs);
    size_t off = L.mats;
    for (int64_t i = 0; i < count; ++i) {
        const gf2_batch_item &it = items[i];
        const gf2::ElimLayout E = gf2::elim_layout(GF2_OP_PLS, it.m, it.n);
        char *base = w + off;
        gf2::ElimDesc d{};
        d.A = it.A;
        d.stride = it.stride;
        d.st = reinterpret_cast<PanelState *>(base + E.state);
        d.perm = reinterpret_cast<int *>(base + E.perm);
        d.side = reinterpret_cast<u64 *>(base + E.side);
        d.pmask = reinterpret_cast<u64 *>(base + E.pmask);
        d.out = reinterpret_cast<uint64_t *>(base + E.out);
        d.ostride = gf2::min_stride(it.n);
        d.P = it.P;
        d.Q = it.Q;
        d.rank = ranks + i;
        d.m = (int)it.m;
        d.n = (int)it.n;
        d.W = (int)((it.n + 63) / 64);
        D[i] = d;
        off = align_up(off + E.total, 256);
    }
    int *idx = reinterpret_cast<int *>(img.data() + L.idx);
    int *pre = reinterpret_cast<int *>(img.data() + L.pre);
    std::vector<int> step_idx_off(L.Wmax), step_pre_off(L.Wmax), step_nact(L.Wmax), step_total(L.Wmax);
    const int target = 2 * gf2::sm_count() * gf2::sweep_ctas_per_sm(tw);
    const int pass = gf2::sweep_rows_per_pass(tw);
    int64_t io = 0, po = 0;
    std::vector<double> work_est;
    for (int b = 0; b < L.Wmax; ++b) {
        step_idx_off[b] = (int)io;
        step_pre_off[b] = (int)po;
        const int wstart = b & ~(tw - 1);  // the sweep's first tile
        double total_work = 0;
        int nact = 0;
        work_est.clear();
        for (int64_t i = 0; i < count; ++i)
            if (D[i].m > 0 && D[i].W > b) {
                idx[io + nact++] = (int)i;
                const double wk = (double)D[i].m * (double)(D[i].W - wstart);
                work_est.push_back(wk);
                total_work += wk;
            }
        const int T = nact > target ? nact : target;
        int acc = 0;
        for (int j = 0; j < nact; ++j) {
            const gf2::ElimDesc &d = D[idx[io + j]];
            const int tiles = (d.W - wstart + tw - 1) / tw;
            const int64_t cap = (int64_t)tiles * ((d.m + pass - 1) / pass);
            int64_t c = (int64_t)((double)T * work_est[j] / total_work);
            if (c > cap)
                c = cap;
            if (c < 1)
                c = 1;
            pre[po + j] = acc;
            acc += (int)c;
        }
        pre[po + nact] = acc;
        step_nact[b] = nact;
        step_total[b] = acc;
        io += nact;
        po += nact + 1;
    }
    if (void *stage = gf2::capture_stage()) {  // captured: the graph's own buffer, read on every replay
        std::memcpy(stage, img.data(), L.mats);
        if ((rc = gf2::note_cuda(cudaMemcpyAsync(w, stage, L.mats, cudaMemcpyHostToDevice, s))))
            return rc;
    } else if ((rc = upload(w, img.data(), L.mats, s))) {
        return rc;
    }
    const gf2::ElimDesc *dD = reinterpret_cast<const gf2::ElimDesc *>(w + L.descs);
    const int *dIdx = reinterpret_cast<const int *>(w + L.idx);
    const int *dPre = reinterpret_cast<const int *>(w + L.pre);
    // grid.y of the per-matrix kernels is limited to 65535 matrices per launch
    for (int64_t c0 = 0; c0 < count; c0 += 65535) {
        const int cn = (int)(count - c0 < 65535 ? count - c0 : 65535);
        if ((rc = gf2::batch_init(dD + c0, cn, L.max_m, s)))
            return rc;
    }
    // Pivot searches on s, sweeps on a side stream t: the sweeps of step b overlap the
    // pivot searches of step b + 1, which wait for the sweeps of step b - 1 (the same
    // ordering as the single-matrix elimination, for every matrix at once).
    cudaStream_t t = nullptr;
    gf2::EventSet E;
    if ((rc = gf2::side_stream(&t)) || (rc = E.create()))
        return rc;
    cudaEvent_t ev_piv = E.ev[0], ev_rest[2] = {E.ev[1], E.ev[2]};
    for (int b = 0; b < L.Wmax; ++b) {
        if (b >= 2 && (rc = gf2::note_cuda(cudaStreamWaitEvent(s, ev_rest[b & 1], 0))))
            return rc;
        if ((rc = gf2::batch_pivot(dD, dIdx + step_idx_off[b], step_nact[b], b, s)))
            return rc;
        if ((rc = gf2::note_cuda(cudaEventRecord(ev_piv, s))) || (rc = gf2::note_cuda(cudaStreamWaitEvent(t, ev_piv, 0))))
            return rc;
        if ((rc = gf2::batch_sweep(dD, dIdx + step_idx_off[b], dPre + step_pre_off[b], step_nact[b], step_total[b], b,
                                   tw, t)))
            return rc;
        if ((rc = gf2::note_cuda(cudaEventRecord(ev_rest[b & 1], t))))
            return rc;
    }
    if (L.Wmax > 0 && (rc = gf2::note_cuda(cudaStreamWaitEvent(s, ev_rest[(L.Wmax - 1) & 1], 0))))
        return rc;
    for (int64_t c0 = 0; c0 < count; c0 += 65535) {
        const int cn = (int)(count - c0 < 65535 ? count - c0 : 65535);
        if ((rc = gf2::batch_finish(dD + c0, cn, L.max_m, s)))
            return rc;
    }
    return GF2_OK;
}

}  // namespace
