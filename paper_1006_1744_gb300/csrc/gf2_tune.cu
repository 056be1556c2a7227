// gf2_tune.cu -- autotuner for the performance knobs of gf2_opts.
//
// None of these knobs changes a result (the sweep's tile width, the recursive
// split's cutoff, the XOR-table or tensor-core product, the route to the
// reduced echelon form); they only change the time. gf2_autotune times the candidates on a synthetic matrix of the
// requested size and density on the current device and returns the fastest,
// caching the answer per size and density bucket.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gf2_common.cuh"

namespace {

// seeded fill for timing only: bit (i, j) is 1 with probability p (threshold on a
// 64-bit hash of (seed, i, j)); padding bits and words stay zero
__global__ void k_tune_fill(uint64_t *A, int64_t m, int64_t n, int64_t stride, double p, u64 seed)
{
    const int64_t W = (n + 63) / 64;
    const u64 thr = p >= 1.0 ? ~0ull : (u64)(p * 18446744073709551616.0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * stride;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / stride, w = e % stride;
        u64 word = 0;
        if (w < W) {
            for (int b = 0; b < 64; ++b) {
                u64 z = seed ^ ((u64)i * 0x9E3779B97F4A7C15ull) ^ ((u64)(64 * w + b) * 0xC2B2AE3D27D4EB4Full);
                z ^= z >> 31;
                z *= 0xBF58476D1CE4E5B9ull;
                z ^= z >> 29;
                z *= 0x94D049BB133111EBull;
                z ^= z >> 32;
                word |= (z < thr ? 1ull : 0ull) << b;
            }
            if (w == W - 1 && (n & 63))
                word &= lowmask((int)(n & 63));
        }
        A[e] = word;
    }
}

using Key = std::tuple<int, int, int, int, int>;  // device, op, log2 m, log2 n, density bucket
std::mutex g_mu;
std::map<Key, std::pair<gf2_opts, double>> g_cache;

int bucket(int64_t x) { return x <= 1 ? 0 : (int)std::ceil(std::log2((double)x)); }
int dbucket(double p) { return p >= 0.3 ? 0 : p >= 0.03 ? 1 : 2; }

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p)
            cudaFree(p);
    }
};

}  // namespace

extern "C" int gf2_autotune(int op, int64_t m, int64_t n, double density, gf2_opts *best, double *ms_out,
                            void *stream)
{
    if (!best || m <= 0 || n <= 0 || m > INT32_MAX - 64 || n > INT32_MAX - 64 || !(density > 0.0) ||
        density > 1.0 || (op != GF2_OP_PLS && op != GF2_OP_RREF && op != GF2_OP_RANK && op != GF2_OP_MUL))
        return GF2_EINVAL;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess)
        return gf2::note_cuda(err);
    const Key key{dev, op, bucket(m), bucket(n), dbucket(density)};
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *best = it->second.first;
            if (ms_out)
                *ms_out = it->second.second;
            return GF2_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<gf2_opts> cands;
    auto opt = [](int tw, int64_t cutoff, int product) {
        gf2_opts o{};
        o.tile_words = tw;
        o.cutoff_cols = cutoff;
        o.product = product;
        return o;
    };
    if (op == GF2_OP_MUL) {
        cands.push_back(opt(0, 0, GF2_PRODUCT_XOR));
        cands.push_back(opt(0, 0, GF2_PRODUCT_TENSOR));
        // Strassen-Winograd over either leaf, where at least one level applies
        const int64_t leaf = gf2::STRASSEN_LEAF_DEFAULT;
        if (m % 2 == 0 && n % 2048 == 0 && m >= 2 * leaf && n >= 2 * leaf) {
            cands.push_back(opt(0, 0, GF2_PRODUCT_STRASSEN));
            cands.push_back(opt(0, 0, GF2_PRODUCT_STRASSEN_TENSOR));
        }
    } else {
        for (int tw : {4, 8, 16}) {
            gf2_opts o = opt(tw, 0, 0);
            o.panels_per_sweep = 1;  // the tile width is the one-panel sweep's
            cands.push_back(o);
        }
        {
            gf2_opts o = opt(16, 0, 0);  // 4-bit tables (Sec. 3.1's k) on the 16-word sweep
            o.k = 4;
            o.panels_per_sweep = 1;
            cands.push_back(o);
        }
        for (int pps : {1, 2}) {
            gf2_opts o = opt(0, 0, 0);  // one panel per sweep, or two (gf2_pair.cu)
            o.panels_per_sweep = pps;
            cands.push_back(o);
        }
        if (op == GF2_OP_RREF) {
            // the direct reduced form (M4RI, Sec. 3.1) and the hybrid at the paper's two thresholds
            for (int meth : {GF2_RREF_M4RI, GF2_RREF_HYBRID}) {
                gf2_opts o = opt(16, 0, 0);
                o.rref_method = meth;
                if (meth == GF2_RREF_HYBRID)
                    for (int pm : {150, 200}) {
                        o.hybrid_permille = pm;
                        cands.push_back(o);
                    }
                else
                    cands.push_back(o);
            }
        }
        if (op == GF2_OP_PLS && n > 2 * 4096) {
            cands.push_back(opt(16, 4096, GF2_PRODUCT_XOR));
            cands.push_back(opt(16, 4096, GF2_PRODUCT_TENSOR));
        }
    }
    const int64_t stride = gf2::min_stride(n);
    const size_t mat = (size_t)m * stride * 8;
    DevBuf A0, A, C, B, ws, aux;
    if (cudaMalloc(&A0.p, mat) != cudaSuccess || cudaMalloc(&A.p, mat) != cudaSuccess ||
        cudaMalloc(&aux.p, (size_t)(m + n + 2) * 8) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ENOMEM;
    }
    const int64_t mb = op == GF2_OP_MUL ? n : 0;  // MUL: A is m x n, B is n x n, C is m x n
    if (op == GF2_OP_MUL && (cudaMalloc(&B.p, (size_t)n * stride * 8) != cudaSuccess ||
                             cudaMalloc(&C.p, mat) != cudaSuccess)) {
        cudaGetLastError();
        return GF2_ENOMEM;
    }
    k_tune_fill<<<2 * gf2::sm_count(), 256, 0, s>>>((uint64_t *)A0.p, m, n, stride, density, 0x10061744ull);
    if (op == GF2_OP_MUL)
        k_tune_fill<<<2 * gf2::sm_count(), 256, 0, s>>>((uint64_t *)B.p, mb, n, stride, density, 0x2001ull);
    if ((err = cudaGetLastError()) != cudaSuccess)
        return gf2::note_cuda(err);
    int64_t *P = (int64_t *)aux.p, *Q = P + m, *rank = Q + n;
    cudaEvent_t e0, e1;
    if ((err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess)
        return gf2::note_cuda(err);
    double best_ms = 1e300;
    gf2_opts best_opts{};
    int rc = GF2_OK;
    for (const gf2_opts &o : cands) {
        // a product's workspace depends on its form (none for the XOR-table form)
        const size_t need = op == GF2_OP_MUL ? gf2_mul_workspace_bytes(m, n, n, &o) : gf2_workspace_bytes(op, m, n, &o);
        if (!need && op != GF2_OP_MUL) {
            rc = GF2_EINVAL;
            break;
        }
        if (ws.p)
            cudaFree(ws.p);
        ws.p = nullptr;
        if (need && cudaMalloc(&ws.p, need) != cudaSuccess) {
            cudaGetLastError();
            continue;  // this candidate does not fit next to the test matrices
        }
        double total = 0.0;
        const int reps = 3;
        for (int it = 0; it <= reps && rc == GF2_OK; ++it) {
            if ((err = cudaMemcpyAsync(A.p, A0.p, mat, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
                rc = gf2::note_cuda(err);
                break;
            }
            cudaEventRecord(e0, s);
            switch (op) {
            case GF2_OP_PLS:
                rc = gf2_pls((uint64_t *)A.p, m, n, stride, P, Q, rank, ws.p, need, &o, s);
                break;
            case GF2_OP_RREF:
                rc = gf2_rref((uint64_t *)A.p, m, n, stride, rank, Q, ws.p, need, &o, s);
                break;
            case GF2_OP_RANK:
                rc = gf2_rank((const uint64_t *)A.p, m, n, stride, rank, ws.p, need, &o, s);
                break;
            default:
                rc = gf2_mul((uint64_t *)C.p, stride, (const uint64_t *)A.p, stride, (const uint64_t *)B.p, stride,
                             m, n, n, 0, ws.p, need, &o, s);
            }
            cudaEventRecord(e1, s);
            if ((err = cudaEventSynchronize(e1)) != cudaSuccess) {
                rc = gf2::note_cuda(err);
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0)  // the first run warms up
                total += ms;
        }
        if (rc)
            break;
        const double mean = total / reps;
        if (mean < best_ms) {
            best_ms = mean;
            best_opts = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc)
        return rc;
    if (best_ms >= 1e299)
        return GF2_ENOMEM;
    const int status = gf2_sync_status(stream);  // a wait that gave up disqualifies nothing silently
    if (status)
        return status;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = {best_opts, best_ms};
    }
    *best = best_opts;
    if (ms_out)
        *ms_out = best_ms;
    return GF2_OK;
}
