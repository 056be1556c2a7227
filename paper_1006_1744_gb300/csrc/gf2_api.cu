// gf2_api.cu -- C ABI entry points: argument checks, workspace, dispatch.
#include <cstring>
#include <mutex>
#include <stdint.h>
#include <stdio.h>

#include "gf2_common.cuh"

namespace gf2 {

static thread_local int g_last_cuda = 0;

int note_cuda(cudaError_t e)
{
    if (e == cudaSuccess)
        return GF2_OK;
    g_last_cuda = (int)e;
    return GF2_ECUDA;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return 148;
    return n;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int64_t min_stride(int64_t n)
{
    int64_t s = ((n + 63) / 64 + 15) / 16 * 16;
    return s < 16 ? 16 : s;
}

// Two panels per sweep once the trailing block's sweeps outweigh the serial pivot searches: a
// panel's sweep grows with rows x words, the pivot search does not (measured on GB300, one panel
// per sweep against two: 20480^2 6.79 / 6.94 ms, 24576^2 9.33 / 9.09, 16384 x 65536 12.10 / 11.58,
// 65536 x 16384 10.37 / 8.73, 65536^2 92 / 74; 16384^2 4.9 / 6.1, where the pivot chain sets the time)
int pps_choice(const gf2_opts *o, int64_t m, int64_t n)
{
    if (o && o->panels_per_sweep)
        return o->panels_per_sweep;
    const int64_t W = (n + 63) / 64;
    return m >= 16384 && m * W >= (int64_t)8 << 20 ? 2 : 1;
}

// gf2_rref: the PLS route takes the panels per sweep of the PLS form; the reduced-form routes
// sweep one panel at a time
static int rref_pps(const gf2_opts *o, int64_t m, int64_t n)
{
    const int method = (o && o->rref_method) ? o->rref_method : GF2_RREF_PLS;
    return method == GF2_RREF_PLS ? pps_choice(o, m, n) : 1;
}

ElimLayout elim_layout(int op, int64_t m, int64_t n, int pps)
{
    ElimLayout L{};
    const int64_t W = (n + 63) / 64;
    const int64_t stride = min_stride(n);
    size_t off = 0;
    L.state = off;
    off = align_up(off + 4 * sizeof(PanelState), 256);  // two slots, or four for two panels per sweep
    L.perm = off;
    off = align_up(off + (size_t)m * sizeof(int), 256);
    L.side = off;
    // two panel words of every row (double buffered); two panels per sweep: the coordinates of
    // every row over both panels' pivot rows, and words b .. b + 3 of every row (double buffered)
    off = align_up(off + (size_t)(pps == 2 ? 10 : 2) * m * sizeof(u64), 256);
    L.pmask = off;
    off = align_up(off + (size_t)(W + 1) * sizeof(u64), 256);
    L.out = off;
    off = align_up(off + (size_t)m * stride * sizeof(u64), 256);
    // Q (rref) or P,Q scratch (rank) share one area after `out`
    L.rref_b = L.rref_x = L.rref_d = off;
    if (op == GF2_OP_RREF) {
        L.rref_b = off;
        off = align_up(off + (size_t)m * W * sizeof(u64), 256);
        L.rref_x = off;
        off = align_up(off + (size_t)m * W * sizeof(u64), 256);
        L.rref_d = off;
        off = align_up(off + (size_t)((m + 63) / 64 + 1) * 64 * sizeof(u64), 256);
    }
    L.ups = off;
    if (op == GF2_OP_RREF)
        off = align_up(off + (size_t)2 * m * sizeof(u64), 256);
    // int64 Q scratch for rref (length n)
    off = align_up(off + (size_t)(n + 1) * sizeof(int64_t), 256);
    L.total = off;
    return L;
}

static size_t q_scratch_offset(const ElimLayout &L, int64_t n)
{
    return L.total - align_up((size_t)(n + 1) * sizeof(int64_t), 256);
}

int identity_fill(int64_t *P, int64_t m, int64_t *Q, int64_t n, int64_t *rank, cudaStream_t s);
int identity_perm(int *perm, int64_t m, cudaStream_t s);

// internal workspace, one per device, grown on demand
struct InternalWork {
    std::mutex mu;
    void *ptr[64] = {};
    size_t bytes[64] = {};
};
static InternalWork g_work;

int get_work(void *&work, size_t &work_bytes, size_t need)
{
    if (work) {
        if ((uintptr_t)work % 256)
            return GF2_EALIGN;
        if (work_bytes < need)
            return GF2_ENOSPACE;
        return GF2_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return note_cuda(e);
    if (dev < 0 || dev >= 64)
        return GF2_EINVAL;
    std::lock_guard<std::mutex> lock(g_work.mu);
    if (g_work.bytes[dev] < need) {
        if (g_work.ptr[dev]) {
            cudaDeviceSynchronize();
            cudaFree(g_work.ptr[dev]);
            g_work.ptr[dev] = nullptr;
            g_work.bytes[dev] = 0;
        }
        void *p = nullptr;
        e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return GF2_ENOMEM;
        }
        g_work.ptr[dev] = p;
        g_work.bytes[dev] = need;
    }
    work = g_work.ptr[dev];
    work_bytes = g_work.bytes[dev];
    return GF2_OK;
}

int check_mat(const void *A, int64_t m, int64_t n, int64_t stride)
{
    if (m < 0 || n < 0 || m > INT32_MAX - 64 || n > INT32_MAX - 64)
        return GF2_EINVAL;
    const int64_t W = (n + 63) / 64;
    if (stride < W || stride < 0)
        return GF2_EINVAL;
    if (m > 0 && n > 0) {
        if (!A)
            return GF2_EINVAL;
        if ((uintptr_t)A % 128)
            return GF2_EALIGN;
        if (stride % 16)
            return GF2_EALIGN;
    }
    return GF2_OK;
}

int check_opts(const gf2_opts *o)
{
    if (!o)
        return GF2_OK;
    if (o->k != 0 && o->k != 4 && o->k != 8)
        return GF2_EINVAL;
    if (o->k == 4 && ((o->tile_words != 0 && o->tile_words != 16) || o->rref_method == GF2_RREF_M4RI ||
                      o->rref_method == GF2_RREF_HYBRID || o->batch_mode == GF2_BATCH_PERSISTENT))
        return GF2_EINVAL;  // k = 4 is built into the 16-word PLS-form sweep only
    if (o->tile_words != 0 && o->tile_words != 4 && o->tile_words != 8 && o->tile_words != 16)
        return GF2_EINVAL;
    if (o->grid_ctas < 0 || o->product < 0 || o->product > GF2_PRODUCT_STRASSEN_TENSOR || o->cutoff_cols < 0)
        return GF2_EINVAL;
    if (o->cutoff_cols != 0 && o->cutoff_cols < 128)
        return GF2_EINVAL;
    if (o->rref_method < 0 || o->rref_method > GF2_RREF_HYBRID || o->hybrid_permille < 0 || o->hybrid_permille > 1000)
        return GF2_EINVAL;
    if (o->batch_mode < 0 || o->batch_mode > GF2_BATCH_PERSISTENT)
        return GF2_EINVAL;
    if (o->panels_per_sweep < 0 || o->panels_per_sweep > 2)
        return GF2_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (o->reserved[i])
            return GF2_EINVAL;
    return GF2_OK;
}

static Elim make_elim(uint64_t *A, int64_t m, int64_t n, int64_t stride, char *work, const ElimLayout &L,
                      int64_t *P, int64_t *Q, bool with_out, const gf2_opts *o, cudaStream_t s, int pps = 1)
{
    Elim e{};
    e.A = A;
    e.m = m;
    e.n = n;
    e.stride = stride;
    e.W = (n + 63) / 64;
    e.st = reinterpret_cast<PanelState *>(work + L.state);
    e.stf = final_state(e.st, e.W);
    e.perm = reinterpret_cast<int *>(work + L.perm);
    e.side = reinterpret_cast<u64 *>(work + L.side);
    e.pmask = reinterpret_cast<u64 *>(work + L.pmask);
    e.out = with_out ? reinterpret_cast<uint64_t *>(work + L.out) : nullptr;
    e.ups = nullptr;  // set by gf2_rref for the reduced form
    e.ostride = min_stride(n);
    e.P = P;
    e.Q = Q;
    e.s = s;
    e.tile_words = (o && o->tile_words) ? o->tile_words : 16;
    e.mode = 0;
    e.hybrid_permille = o ? o->hybrid_permille : 0;
    e.k = (o && o->k) ? o->k : 8;
    e.pps = pps;
    if (e.pps == 2)
        e.stf = e.W > 0 ? e.st + ((e.W - 1) & 3) : e.st;  // panel b's state lives in slot b & 3
    // default: one CTA per SM but one, so the look-ahead pivot search (which cannot share an
    // SM with a 1024-thread sweep CTA) never holds back a CTA of the sweep it overlaps
    const int nsm = sm_count();
    e.grid = (o && o->grid_ctas) ? o->grid_ctas : (nsm > 1 ? nsm - 1 : 1);
    return e;
}

// Panel elimination (MMPF) of one view: the base case of the recursive PLS.
// perm_out receives the position -> view row map of the result.
int pls_base(uint64_t *A, int64_t stride, int64_t m, int64_t n, int64_t *P, int64_t *Q, int *perm_out, int64_t *rank,
             char *work, const gf2_opts *opts, cudaStream_t s)
{
    if (m == 0 || n == 0)  // empty view: rank 0, identity P and Q, rows in place
        return identity_fill(P, m, Q, n, rank, s) || identity_perm(perm_out, m, s) ? GF2_ECUDA : GF2_OK;
    const ElimLayout L = elim_layout(GF2_OP_PLS, m, n);
    Elim e = make_elim(A, m, n, stride, work, L, P, Q, true, opts, s);
    int rc;
    if ((rc = elim_run(e)) || (rc = elim_gather(e, rank)) || (rc = pls_finish(e)))
        return rc;
    return note_cuda(cudaMemcpyAsync(perm_out, e.perm, (size_t)m * sizeof(int), cudaMemcpyDeviceToDevice, s));
}

// Rank of A (left unchanged) by one direct elimination of a copy held in `work`: no graph
// replay and no allocation; the side stream and events come from the caller.
int rank_direct(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, char *work,
                const ElimAux &aux, cudaStream_t s)
{
    if (m == 0 || n == 0)
        return identity_fill(nullptr, 0, nullptr, 0, rank, s);
    const ElimLayout L = elim_layout(GF2_OP_RANK, m, n);
    uint64_t *copy = reinterpret_cast<uint64_t *>(work + L.out);
    const int64_t cs = min_stride(n);
    const Elim e = make_elim(copy, m, n, cs, work, L, nullptr, nullptr, false, nullptr, s);
    const cudaError_t err = cudaMemcpy2DAsync(copy, (size_t)cs * 8, A, (size_t)stride * 8,
                                              (size_t)((n + 63) / 64) * 8, (size_t)m, cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess)
        return note_cuda(err);
    const int rc = elim_run(e, aux);
    return rc ? rc : elim_gather(e, rank);
}

static CallKey call_key(int op, const void *A, int64_t m, int64_t n, int64_t stride, const void *P, const void *Q,
                        const void *rank, const void *pivots, const void *work, size_t work_bytes, const Elim &e)
{
    CallKey k;
    std::memset(&k, 0, sizeof(k));  // padding too: keys are compared bytewise
    cudaGetDevice(&k.device);
    k.op = op;
    k.tile_words = e.tile_words;
    k.grid = e.grid + (e.k << 27) + (e.pps << 24);  // the table width and panels per sweep change the launches too
    k.A = A;
    k.m = m;
    k.n = n;
    k.stride = stride;
    k.P = P;
    k.Q = Q;
    k.rank = rank;
    k.pivots = pivots;
    k.work = work;
    k.work_bytes = work_bytes;
    return k;
}

}  // namespace gf2

using namespace gf2;

extern "C" {

size_t gf2_workspace_bytes(int op, int64_t m, int64_t n, const gf2_opts *opts)
{
    if (check_opts(opts) || m < 0 || n < 0 || m > INT32_MAX - 64 || n > INT32_MAX - 64)
        return 0;
    switch (op) {
    case GF2_OP_PLS:
        if (opts && opts->cutoff_cols > 0 && n > opts->cutoff_cols)
            return rec_workspace_bytes(m, n, opts->cutoff_cols);
        return elim_layout(op, m, n, pps_choice(opts, m, n)).total;
    case GF2_OP_RREF:
        return elim_layout(op, m, n, rref_pps(opts, m, n)).total;
    case GF2_OP_RANK:
        return elim_layout(op, m, n, pps_choice(opts, m, n)).total;
    case GF2_OP_MUL:  // (m, n) = (inner dimension k, columns n); Strassen forms: a k x k A assumed
        if (opts && (opts->product == GF2_PRODUCT_STRASSEN || opts->product == GF2_PRODUCT_STRASSEN_TENSOR))
            return gf2_mul_workspace_bytes(m, m, n, opts);
        return align_up(mul_tensor_workspace(0, m, n), 256);
    default:
        return 0;
    }
}

int gf2_pls(uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *P, int64_t *Q, int64_t *rank,
            void *work, size_t work_bytes, const gf2_opts *opts, void *stream)
{
    int rc = check_mat(A, m, n, stride);
    if (rc)
        return rc;
    if ((rc = check_opts(opts)))
        return rc;
    if (!rank || (m > 0 && !P) || (n > 0 && !Q))
        return GF2_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0 || n == 0)
        return identity_fill(P, m, Q, n, rank, s);
    if (opts && opts->cutoff_cols > 0 && n > opts->cutoff_cols) {
        // recursive PLS (Sec. 5) down to the MMPF base case at the cutoff (Sec. 6)
        if ((rc = get_work(work, work_bytes, rec_workspace_bytes(m, n, opts->cutoff_cols))))
            return rc;
        return pls_recursive(A, stride, m, n, P, Q, rank, (char *)work, opts, s);
    }
    const int pps = pps_choice(opts, m, n);
    const ElimLayout L = elim_layout(GF2_OP_PLS, m, n, pps);
    if ((rc = get_work(work, work_bytes, L.total)))
        return rc;
    const Elim e = make_elim(A, m, n, stride, (char *)work, L, P, Q, true, opts, s, pps);
    return run_replayed(call_key(GF2_OP_PLS, A, m, n, stride, P, Q, rank, nullptr, work, work_bytes, e), s,
                        [&](cudaStream_t st) {
                            Elim es = e;
                            es.s = st;
                            int r2 = elim_run(es);
                            if (!r2)
                                r2 = elim_gather(es, rank);
                            return r2 ? r2 : pls_finish(es);
                        });
}

int gf2_rref(uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, int64_t *pivots, void *work,
             size_t work_bytes, const gf2_opts *opts, void *stream)
{
    int rc = check_mat(A, m, n, stride);
    if (rc)
        return rc;
    if ((rc = check_opts(opts)))
        return rc;
    if (!rank)
        return GF2_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0 || n == 0)
        return identity_fill(nullptr, 0, pivots, pivots ? n : 0, rank, s);
    const int pps = rref_pps(opts, m, n);
    const ElimLayout L = elim_layout(GF2_OP_RREF, m, n, pps);
    if ((rc = get_work(work, work_bytes, L.total)))
        return rc;
    char *w = (char *)work;
    int64_t *Qs = reinterpret_cast<int64_t *>(w + q_scratch_offset(L, n));
    Elim e = make_elim(A, m, n, stride, w, L, nullptr, Qs, true, opts, s, pps);
    const int method = (opts && opts->rref_method) ? opts->rref_method : GF2_RREF_PLS;
    // the sweep form: PLS panels (then the upper solve), reduced-form panels (M4RI), or the hybrid
    e.mode = method == GF2_RREF_M4RI ? 1 : method == GF2_RREF_HYBRID ? 2 : 0;
    e.ups = reinterpret_cast<u64 *>(w + L.ups);
    if (e.mode && e.tile_words != 16)
        return GF2_EINVAL;  // the reduced form is built on the 16-word sweep only
    CallKey key = call_key(GF2_OP_RREF + 16 * e.mode, A, m, n, stride, nullptr, nullptr, rank, pivots, work,
                           work_bytes, e);
    key.grid += e.hybrid_permille << 16;  // the threshold changes the launches' behaviour
    return run_replayed(key, s, [&](cudaStream_t st) {
        Elim es = e;
        es.s = st;
        const int r2 = elim_run(es);
        if (r2)
            return r2;
        return es.mode == 1 ? m4ri_finish(es, rank, pivots) : rref_finish(es, L, w, rank, pivots);
    });
}

int gf2_rank(const uint64_t *A, int64_t m, int64_t n, int64_t stride, int64_t *rank, void *work,
             size_t work_bytes, const gf2_opts *opts, void *stream)
{
    int rc = check_mat(A, m, n, stride);
    if (rc)
        return rc;
    if ((rc = check_opts(opts)))
        return rc;
    if (!rank)
        return GF2_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0 || n == 0)
        return identity_fill(nullptr, 0, nullptr, 0, rank, s);
    const int pps = pps_choice(opts, m, n);
    const ElimLayout L = elim_layout(GF2_OP_RANK, m, n, pps);
    if ((rc = get_work(work, work_bytes, L.total)))
        return rc;
    char *w = (char *)work;
    uint64_t *copy = reinterpret_cast<uint64_t *>(w + L.out);
    const int64_t cs = min_stride(n);
    const Elim e = make_elim(copy, m, n, cs, w, L, nullptr, nullptr, false, opts, s, pps);
    return run_replayed(call_key(GF2_OP_RANK, A, m, n, stride, nullptr, nullptr, rank, nullptr, work, work_bytes, e),
                        s, [&](cudaStream_t st) {
                            cudaError_t err = cudaMemcpy2DAsync(copy, (size_t)cs * 8, A, (size_t)stride * 8,
                                                                (size_t)((n + 63) / 64) * 8, (size_t)m,
                                                                cudaMemcpyDeviceToDevice, st);
                            if (err != cudaSuccess)
                                return note_cuda(err);
                            Elim es = e;
                            es.s = st;
                            const int r2 = elim_run(es);
                            return r2 ? r2 : elim_gather(es, rank);
                        });
}

int gf2_mul(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
            int64_t k, int64_t n, int accumulate, void *work, size_t work_bytes, const gf2_opts *opts, void *stream)
{
    int rc;
    if ((rc = check_mat(C, m, n, sc)) || (rc = check_mat(A, m, k, sa)) || (rc = check_mat(B, k, n, sb)))
        return rc;
    if ((rc = check_opts(opts)))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0 || n == 0)
        return GF2_OK;
    if (!C)
        return GF2_EINVAL;
    const int product = opts ? opts->product : GF2_PRODUCT_AUTO;
    if (product == GF2_PRODUCT_STRASSEN || product == GF2_PRODUCT_STRASSEN_TENSOR) {
        const int kind = product == GF2_PRODUCT_STRASSEN ? GF2_PRODUCT_XOR : GF2_PRODUCT_TENSOR;
        const int64_t leaf = (opts && opts->cutoff_cols) ? opts->cutoff_cols : STRASSEN_LEAF_DEFAULT;
        const size_t need = mul_strassen_workspace(m, k, n, leaf, kind);
        if (need && (rc = get_work(work, work_bytes, need)))
            return rc;
        if (kind == GF2_PRODUCT_XOR && k == 0 && !accumulate)
            return note_cuda(cudaMemset2DAsync(C, (size_t)sc * 8, 0, (size_t)((n + 63) / 64) * 8, (size_t)m, s));
        if (kind == GF2_PRODUCT_XOR && k == 0)
            return GF2_OK;
        return mul_strassen(C, sc, A, sa, B, sb, m, k, n, accumulate, work, work_bytes, leaf, kind, s);
    }
    if (product == GF2_PRODUCT_TENSOR) {
        const size_t need = mul_tensor_workspace(m, k, n);
        if ((rc = get_work(work, work_bytes, need)))
            return rc;
        return mul_tensor(C, sc, A, sa, B, sb, m, k, n, accumulate, work, work_bytes, s);
    }
    if (k == 0) {
        if (!accumulate) {
            cudaError_t err = cudaMemset2DAsync(C, (size_t)sc * 8, 0, (size_t)((n + 63) / 64) * 8, (size_t)m, s);
            return note_cuda(err);
        }
        return GF2_OK;
    }
    return mul_xor(C, sc, A, sa, B, sb, m, k, n, accumulate, opts ? opts->tile_words : 0,
                   opts ? opts->grid_ctas : 0, s);
}

size_t gf2_mul_workspace_bytes(int64_t m, int64_t k, int64_t n, const gf2_opts *opts)
{
    if (check_opts(opts) || m < 0 || k < 0 || n < 0 || m > INT32_MAX - 64 || k > INT32_MAX - 64 ||
        n > INT32_MAX - 64)
        return 0;
    const int product = opts ? opts->product : GF2_PRODUCT_AUTO;
    if (product == GF2_PRODUCT_STRASSEN || product == GF2_PRODUCT_STRASSEN_TENSOR) {
        const int kind = product == GF2_PRODUCT_STRASSEN ? GF2_PRODUCT_XOR : GF2_PRODUCT_TENSOR;
        const int64_t leaf = (opts && opts->cutoff_cols) ? opts->cutoff_cols : STRASSEN_LEAF_DEFAULT;
        return align_up(mul_strassen_workspace(m, k, n, leaf, kind), 256);
    }
    if (product == GF2_PRODUCT_TENSOR)
        return align_up(mul_tensor_workspace(m, k, n), 256);
    return 0;
}

const char *gf2_strerror(int code)
{
    switch (code) {
    case GF2_OK:
        return "ok";
    case GF2_EINVAL:
        return "invalid argument (null pointer, size, stride or option)";
    case GF2_EALIGN:
        return "misaligned data (128 bytes), stride (16 words) or workspace (256 bytes)";
    case GF2_ENOMEM:
        return "device memory allocation for the internal workspace failed";
    case GF2_ECUDA:
        return "CUDA runtime error (see gf2_last_cuda_error)";
    case GF2_ENOSPACE:
        return "workspace smaller than gf2_workspace_bytes()";
    case GF2_EDIM:
        return "mismatched dimensions";
    case GF2_ETOOBIG:
        return "matrix too large for the fixed scratch of gf2_rank_noalloc (GF2_NOALLOC_SCRATCH_BYTES)";
    case GF2_ETIMEOUT:
        return "a device-side wait gave up (bounded wait expired)";
    default:
        return "unknown error";
    }
}

int gf2_last_cuda_error(void) { return g_last_cuda; }

int gf2_version(void) { return 100; }

}  // extern "C"
