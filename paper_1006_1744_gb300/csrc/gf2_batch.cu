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
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "gf2_common.cuh"

namespace {

using gf2::align_up;

struct BatchLayout {
    size_t descs, idx, pre, pplan, mats, total;
    int64_t n_idx, n_pre;
    int Wmax, max_m;
};

// ints of the persistent launch's plan: team_of (one per CTA, <= MAX_CTAS), team_start,
// team_size, team_first (<= MAX_CTAS + 1 each), big, small (count each), counters (next_small,
// abort, one barrier per team)
constexpr int MAX_CTAS = 1024;
constexpr int64_t PP_TEAM_OF = 0, PP_START = MAX_CTAS, PP_SIZE = 2 * MAX_CTAS, PP_FIRST = 3 * MAX_CTAS,
                  PP_BIG = 4 * MAX_CTAS + 1;
int64_t pplan_ints(int64_t count) { return PP_BIG + 2 * count + (MAX_CTAS + 2); }

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
    L.pplan = off;
    off = align_up(off + (size_t)pplan_ints(count) * sizeof(int), 256);
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
                int mode, int kbits, cudaStream_t s);
bool persistent_suits(const gf2_batch_item *items, int64_t count);

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
    const int kbits = (opts && opts->k) ? opts->k : 8;
    int mode = opts ? opts->batch_mode : GF2_BATCH_AUTO;
    if (mode == GF2_BATCH_AUTO)
        mode = tw == 16 && kbits == 8 && persistent_suits(items, count) ? GF2_BATCH_PERSISTENT : GF2_BATCH_STEPS;
    if (mode == GF2_BATCH_PERSISTENT && tw != 16)
        return GF2_EINVAL;  // the persistent schedule runs the 16-word sweep
    // a repeated call (same items, ranks, workspace, options) replays a captured graph
    gf2::CallKey key;
    std::memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.op = -GF2_OP_PLS;
    key.tile_words = tw;
    key.grid = mode + (kbits << 8);
    key.m = count;
    key.rank = ranks;
    key.work = work;
    key.work_bytes = work_bytes;
    return gf2::run_replayed(
        key, (cudaStream_t)stream,
        [&](cudaStream_t s) { return batched_run(items, count, ranks, (char *)work, L, tw, mode, kbits, s); }, items,
        (size_t)count * sizeof(gf2_batch_item), L.mats);
}

}  // extern "C"

namespace {

// Plan of the persistent launch: the cost of a matrix on G CTAs (microseconds) is its W pivot
// searches and team barriers plus its sweep bytes (full-rank bound) at a per-CTA rate. The
// target makespan T is the larger of the average load per CTA and the longest single matrix on
// its best team. A matrix whose one-CTA cost exceeds T gets a team: the smallest power-of-two G
// (up to the CTA count) that brings it under T, as long as its sweeps still outweigh its pivot
// chain. Teams are contiguous CTA ranges, largest matrices first; a matrix joins an existing
// team of its size while that team's load stays under T, else opens a new one while CTAs remain,
// else goes to the least loaded team of at least its size. Every other matrix goes, largest
// first, to the device work queue.
struct PersistHostPlan {
    int nteams = 0;
    std::vector<int> team_of;                     // per CTA: its team, or -1
    std::vector<int> team_start, team_size;       // per team
    std::vector<int> team_first, big, small;      // team t: big[team_first[t] .. team_first[t + 1])
};

PersistHostPlan plan_persistent(const gf2::ElimDesc *D, int64_t count, int N)
{
    const double T_PIV = 22.0, T_BAR1 = 1.0, T_BARG = 4.0, B1 = 30000.0;  // us, us, us, bytes per us per CTA
    std::vector<double> bytes((size_t)count, 0.0), c1((size_t)count, 0.0);
    double total = 0;
    for (int64_t i = 0; i < count; ++i) {
        const int W = D[i].W, m = D[i].m;
        double by = 0;
        for (int b = 0; b < W; ++b) {
            const double rows = m - 64.0 * b > 0 ? m - 64.0 * b : 0.0;
            by += rows * (double)(W - (b & ~15)) * 16.0;
        }
        bytes[i] = by;
        c1[i] = W * (T_PIV + T_BAR1) + by / B1;
        total += c1[i];
    }
    auto cost = [&](int64_t i, int G) {
        return D[i].W * (T_PIV + (G > 1 ? T_BARG : T_BAR1)) + bytes[i] / ((double)G * B1);
    };
    int Gmax = 1;
    while (Gmax * 2 <= N)
        Gmax *= 2;
    double T = total / (N > 0 ? N : 1);
    for (int64_t i = 0; i < count; ++i)
        T = std::max(T, cost(i, Gmax));
    PersistHostPlan P;
    P.team_of.assign((size_t)N, -1);
    std::vector<int> gi((size_t)count, 1), bigs;
    for (int64_t i = 0; i < count; ++i) {
        while (gi[i] < Gmax && cost(i, gi[i]) > T && bytes[i] / ((double)gi[i] * B1) > D[i].W * T_PIV)
            gi[i] *= 2;
        (gi[i] > 1 ? bigs : P.small).push_back((int)i);
    }
    std::sort(P.small.begin(), P.small.end(), [&](int a, int b) { return c1[a] > c1[b]; });
    std::sort(bigs.begin(), bigs.end(), [&](int a, int b) { return cost(a, gi[a]) > cost(b, gi[b]); });
    std::vector<std::vector<int>> lists;
    std::vector<double> load;
    int next_cta = 0;
    for (int i : bigs) {
        const int G = gi[i];
        const double c = cost(i, G);
        int pick = -1;
        for (size_t t = 0; t < lists.size(); ++t)
            if (P.team_size[t] == G && load[t] + c <= T && (pick < 0 || load[t] < load[pick]))
                pick = (int)t;
        if (pick < 0 && next_cta + G <= N) {
            pick = (int)lists.size();
            lists.emplace_back();
            load.push_back(0.0);
            P.team_start.push_back(next_cta);
            P.team_size.push_back(G);
            for (int k = 0; k < G; ++k)
                P.team_of[next_cta + k] = pick;
            next_cta += G;
        }
        if (pick < 0)
            for (size_t t = 0; t < lists.size(); ++t)
                if (P.team_size[t] >= G && (pick < 0 || load[t] < load[pick]))
                    pick = (int)t;
        if (pick < 0) {  // no team can take it (cannot happen: the first big matrix opens one)
            P.small.insert(P.small.begin(), i);
            continue;
        }
        lists[pick].push_back(i);
        load[pick] += cost(i, P.team_size[pick]);
    }
    P.nteams = (int)lists.size();
    P.team_first.push_back(0);
    for (auto &l : lists) {
        P.big.insert(P.big.end(), l.begin(), l.end());
        P.team_first.push_back((int)P.big.size());
    }
    return P;
}

// The automatic choice of schedule: the persistent launch, unless a member is so large that its
// plan would give it a team of more than 16 CTAs. A team runs each panel's pivot search and sweep
// one after the other, while the per-step schedule overlaps the pivot search of panel b + 1 with
// the sweep of panel b on every SM; for the largest members that overlap wins.
bool persistent_suits(const gf2_batch_item *items, int64_t count)
{
    std::vector<gf2::ElimDesc> D((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        D[i] = gf2::ElimDesc{};
        D[i].m = (int)items[i].m;
        D[i].n = (int)items[i].n;
        D[i].W = (int)((items[i].n + 63) / 64);
    }
    const PersistHostPlan P = plan_persistent(D.data(), count, gf2::batch_persistent_grid());
    for (int g : P.team_size)
        if (g > 16)
            return false;
    return true;
}

int batched_run(const gf2_batch_item *items, int64_t count, int64_t *ranks, char *w, const BatchLayout &L, int tw,
                int mode, int kbits, cudaStream_t s)
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
    if (mode == GF2_BATCH_PERSISTENT) {
        const int N = gf2::batch_persistent_grid();
        if (N > MAX_CTAS)
            return GF2_EINVAL;
        const PersistHostPlan P = plan_persistent(D, count, N);
        int *pp = reinterpret_cast<int *>(img.data() + L.pplan);
        const int64_t nsmall = (int64_t)P.small.size();
        std::memcpy(pp + PP_TEAM_OF, P.team_of.data(), P.team_of.size() * sizeof(int));
        std::memcpy(pp + PP_START, P.team_start.data(), P.team_start.size() * sizeof(int));
        std::memcpy(pp + PP_SIZE, P.team_size.data(), P.team_size.size() * sizeof(int));
        std::memcpy(pp + PP_FIRST, P.team_first.data(), P.team_first.size() * sizeof(int));
        std::memcpy(pp + PP_BIG, P.big.data(), P.big.size() * sizeof(int));
        std::memcpy(pp + PP_BIG + count, P.small.data(), (size_t)nsmall * sizeof(int));
        if (void *stage = gf2::capture_stage()) {
            std::memcpy(stage, img.data(), L.mats);
            if ((rc = gf2::note_cuda(cudaMemcpyAsync(w, stage, L.mats, cudaMemcpyHostToDevice, s))))
                return rc;
        } else if ((rc = upload(w, img.data(), L.mats, s))) {
            return rc;
        }
        const int *dpp = reinterpret_cast<const int *>(w + L.pplan);
        int *counters = reinterpret_cast<int *>(w + L.pplan) + PP_BIG + 2 * count;
        gf2::PersistArrays a{dpp + PP_TEAM_OF, dpp + PP_START, dpp + PP_SIZE, dpp + PP_FIRST, dpp + PP_BIG,
                             dpp + PP_BIG + count};
        return gf2::batch_persistent(reinterpret_cast<const gf2::ElimDesc *>(w + L.descs), P.nteams, a, (int)nsmall,
                                     counters, s);
    }
    int *idx = reinterpret_cast<int *>(img.data() + L.idx);
    int *pre = reinterpret_cast<int *>(img.data() + L.pre);
    std::vector<int> step_idx_off(L.Wmax), step_pre_off(L.Wmax), step_nact(L.Wmax), step_total(L.Wmax);
    // 16-word tiles (the default) run the 16-word sweep of the single-matrix path
    const bool sweep16 = tw == 16;
    const int target = 2 * gf2::sm_count() * (sweep16 ? 1 : gf2::sweep_ctas_per_sm(tw));
    const int pass = sweep16 ? gf2::SWEEP16_ROWS : gf2::sweep_rows_per_pass(tw);
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
        rc = sweep16 ? gf2::batch_sweep16(dD, dIdx + step_idx_off[b], dPre + step_pre_off[b], step_nact[b],
                                          step_total[b], b, kbits, t)
                     : gf2::batch_sweep(dD, dIdx + step_idx_off[b], dPre + step_pre_off[b], step_nact[b],
                                        step_total[b], b, tw, t);
        if (rc)
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

/*
 * Diagnostic (host only): the persistent schedule's plan for these shapes on `ctas` CTAs.
 * team_of (length ctas): each CTA's team or -1; team_size (length >= teams); member_team
 * (length count): each matrix's team, or -1 for the work queue. Returns the team count, or -1
 * for invalid arguments.
 */
extern "C" int gf2_batch_plan(const gf2_batch_item *items, int64_t count, int ctas, int *team_of, int *team_size,
                              int *member_team)
{
    if (check_sizes(items, count) || ctas <= 0 || ctas > MAX_CTAS || !team_of || !team_size || !member_team)
        return -1;
    std::vector<gf2::ElimDesc> D((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        D[i] = gf2::ElimDesc{};
        D[i].m = (int)items[i].m;
        D[i].n = (int)items[i].n;
        D[i].W = (int)((items[i].n + 63) / 64);
    }
    const PersistHostPlan P = plan_persistent(D.data(), count, ctas);
    for (int c = 0; c < ctas; ++c)
        team_of[c] = P.team_of[c];
    for (int t = 0; t < P.nteams; ++t)
        team_size[t] = P.team_size[t];
    for (int64_t i = 0; i < count; ++i)
        member_team[i] = -1;
    for (int t = 0; t < P.nteams; ++t)
        for (int k = P.team_first[t]; k < P.team_first[t + 1]; ++k)
            member_team[P.big[k]] = t;
    return P.nteams;
}
