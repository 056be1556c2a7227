// gf2_mul.cu -- GF(2) product C = (C +) A.B, XOR-table form.
//
// The trailing update A_SE <- A_SE + A_SW.A_NE of Algorithm PLS (Sec. 5) is a
// GF(2) matrix product; the paper cites the Method of the Four Russians for it
// (Sec. 3.1 explains the table idea). For every block of 64 rows of B, a CTA
// builds eight Gray-code tables (k = 8: all 256 sums of 8 rows of B over its
// column tile) in shared memory; each row of C then adds eight table rows,
// indexed by the 8-bit pieces of its word of A. Partial sums stay in registers
// over the whole inner dimension, so C is read and written once.
#include "gf2_common.cuh"

namespace {

template <int TW, int RPT>
__global__ void __launch_bounds__(256, 1)
k_mul_xor(uint64_t *__restrict__ C, int64_t sc, const uint64_t *__restrict__ A, int64_t sa,
          const uint64_t *__restrict__ B, int64_t sb, int m, int k, int n, int acc)
{
    constexpr int TPR = TW / 2;
    constexpr int RPP = 256 / TPR;
    constexpr int ROWS = RPP * RPT;
    extern __shared__ __align__(16) u64 sm[];
    u64 *sT = sm;                 // [8][256][TW]
    u64 *sO = sT + 8 * 256 * TW;  // [64][TW]
    const int W = (n + 63) >> 6, KW = (k + 63) >> 6;
    const int tiles = (W + TW - 1) / TW;
    const int rblocks = (m + ROWS - 1) / ROWS;
    const int items = tiles * rblocks;
    const int tid = threadIdx.x, sub = tid % TPR, rg = tid / TPR;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item % tiles, rb = item / tiles;
        const int wbase = tile * TW;
        const int w0 = wbase + 2 * sub;
        u64 a0[RPT], a1[RPT], av[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            a0[j] = 0;
            a1[j] = 0;
            const int i = rb * ROWS + j * RPP + rg;
            av[j] = (i < m && KW > 0) ? A[(int64_t)i * sa] : 0ull;
        }
        for (int q = 0; q < KW; ++q) {
            __syncthreads();
            for (int e = tid; e < 64 * TW; e += 256) {
                const int s = e / TW, wi = e % TW;
                const int row = 64 * q + s;
                sO[e] = (row < k && wbase + wi < W) ? B[(int64_t)row * sb + wbase + wi] : 0ull;
            }
            __syncthreads();
            const int kk = min(64, k - 64 * q);
            const int ng = (kk + 7) >> 3;
            for (int e = tid; e < ng * TW * 16; e += 256) {
                const int wi = e % TW, rest = e / TW, vh = rest & 15, g = rest >> 4;
                const u64 *Og = sO + (8 * g) * TW + wi;
                u64 cur = 0;
#pragma unroll
                for (int bit = 0; bit < 4; ++bit)
                    if ((vh >> bit) & 1)
                        cur ^= Og[(4 + bit) * TW];
                gray16(cur, Og[0], Og[TW], Og[2 * TW], Og[3 * TW], sT + (g * 256 + (vh << 4)) * TW + wi, TW);
            }
            __syncthreads();
            u64 cur_a[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                cur_a[j] = av[j];
                const int i = rb * ROWS + j * RPP + rg;
                av[j] = (i < m && q + 1 < KW) ? A[(int64_t)i * sa + q + 1] : 0ull;
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const u64 u = cur_a[j];
                for (int g = 0; g < ng; ++g) {
                    const ulonglong2 e2 = *reinterpret_cast<const ulonglong2 *>(
                        sT + (g * 256 + (int)((u >> (8 * g)) & 255ull)) * TW + 2 * sub);
                    a0[j] ^= e2.x;
                    a1[j] ^= e2.y;
                }
            }
        }
        if (w0 < W) {
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int i = rb * ROWS + j * RPP + rg;
                if (i >= m)
                    continue;
                uint64_t *c = C + (int64_t)i * sc + w0;
                if (acc) {
                    c[0] ^= a0[j];
                    if (w0 + 1 < W)
                        c[1] ^= a1[j];
                } else {
                    c[0] = a0[j];
                    if (w0 + 1 < W)
                        c[1] = a1[j];
                }
            }
        }
    }
}

}  // namespace

namespace gf2 {

int mul_xor(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
            int64_t k, int64_t n, int acc, int tile_words, int grid, cudaStream_t s)
{
    constexpr int TW = 8, RPT = 8;
    const size_t smem = (size_t)(8 * 256 * TW + 64 * TW) * sizeof(u64);
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        int rc = note_cuda(
            cudaFuncSetAttribute(k_mul_xor<TW, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (rc)
            return rc;
        attr_done(attr_devs);
    }
    (void)tile_words;
    const int W = (int)((n + 63) >> 6);
    const int tiles = (W + TW - 1) / TW;
    const int rows = (256 / (TW / 2)) * RPT;
    const int64_t items = (int64_t)tiles * ((m + rows - 1) / rows);
    int g = grid > 0 ? grid : sm_count();
    if (items < g)
        g = (int)items;
    if (g < 1)
        g = 1;
    const int tok = prof_begin(s);
    k_mul_xor<TW, RPT><<<g, 256, smem, s>>>(C, sc, A, sa, B, sb, (int)m, (int)k, (int)n, acc);
    prof_end(s, GF2_PROF_MUL, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

}  // namespace gf2
