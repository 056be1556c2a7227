// gf2_mul_tc.cu -- GF(2) product C = (C +) A.B on the tensor cores (sm_103a).
//
// The trailing update A_SE <- A_SE + A_SW.A_NE of Algorithm PLS (Sec. 5) is a
// matrix product over GF(2). Here every bit becomes an FP8 (e4m3) 0.0 or 1.0,
// the product runs as tcgen05.mma kind::f8f6f4 with FP32 accumulators in
// tensor memory, and the low bit of each sum is kept: the sum of the 0/1
// products is an integer and its parity is the GF(2) dot product. (sm_103a has
// no 8-bit integer MMA.) To keep every sum far inside the range the
// accumulator holds exactly, the inner dimension is cut into segments of at
// most `seg` chunks; after each segment the parities are folded into registers
// and the accumulator restarts from zero.
//
// Per CTA: a 128 x 256 tile of C, accumulated in 256 TMEM columns. For every
// 128-bit chunk of the inner dimension, eight warps expand the A tile
// (128 rows x 128 bits) and the B tile (128 x 256 bits, transposed by warp
// butterflies into 256 rows x 128 bits) to bytes in shared memory, in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes); one thread then issues four MMAs of K = 32 and commits them to the
// stage's mbarrier. Two stages: expanding chunk c + 1 overlaps the MMAs of
// chunk c. Every wait is bounded: one that gives up records GF2_ETIMEOUT in the
// status word and the CTA returns without writing C.
#include "gf2_common.cuh"

namespace {

constexpr int TM = 128;                  // rows of C per CTA (MMA M)
constexpr int TN = 256;                  // columns of C per CTA (MMA N)
constexpr int KC = 128;                  // inner-dimension bits per chunk (= bytes per expanded row)
constexpr int NTHR = 256;                // eight warps
constexpr int A_BYTES = TM * KC;         // 16 KB
constexpr int B_BYTES = TN * KC;         // 32 KB
constexpr int STAGE = A_BYTES + B_BYTES; // 48 KB
constexpr int SMEM = 2 * STAGE + 1024 + 4096;  // two stages, alignment and tail slack
constexpr int DEFAULT_SEG = 64;          // chunks per accumulation segment: sums stay <= 8192

// four bits -> four bytes of 0x00 / 0x38 (e4m3 1.0); bit i -> byte i
__device__ __forceinline__ unsigned expand4(unsigned nib)
{
    return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
}

// 16 bits -> one 16-byte core-matrix row
__device__ __forceinline__ void store16(unsigned char *p, unsigned b)
{
    uint4 v;
    v.x = expand4(b & 15u);
    v.y = expand4((b >> 4) & 15u);
    v.z = expand4((b >> 8) & 15u);
    v.w = expand4((b >> 12) & 15u);
    *reinterpret_cast<uint4 *>(p) = v;
}

// byte offset of (row, 16-byte column group cg) in the K-major no-swizzle layout:
// core matrix (row / 8, cg) at (row / 8) * SBO + cg * LBO, row inside it at (row % 8) * 16
constexpr int LBO = 128;             // next core matrix along K
constexpr int SBO = (KC / 16) * 128; // next group of 8 rows
__device__ __forceinline__ int core_off(int row, int cg) { return (row >> 3) * SBO + cg * LBO + (row & 7) * 16; }

// shared-memory matrix descriptor: start, LBO, SBO (16-byte units), version 1, no swizzle
__device__ __forceinline__ u64 smem_desc(uint32_t saddr)
{
    return (u64)((saddr & 0x3FFFFu) >> 4) | ((u64)(LBO >> 4) << 16) | ((u64)(SBO >> 4) << 32) | (1ull << 46);
}

// instruction descriptor: D = F32, A = B = E4M3, both K-major, N = TN, M = TM
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity)
{
    const u64 t0 = globaltimer_ns();
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(mb), "r"(parity)
                     : "memory");
        if (done)
            return true;
        if ((it & 63u) == 63u && globaltimer_ns() - t0 > GF2_WAIT_LIMIT_NS)
            return false;
    }
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit c = column c);
// afterwards lane c holds column c (bit l = row l).
__device__ __forceinline__ unsigned transpose32(unsigned x, int lane)
{
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const unsigned y = __shfl_xor_sync(GF2_FULL, x, j);
        x = (lane & j) ? ((x & ~masks[s]) | ((y >> j) & masks[s])) : ((x & masks[s]) | ((y & masks[s]) << j));
    }
    return x;
}

__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// parities of this thread's 4 x 32 accumulator columns, XORed into par[]
__device__ __forceinline__ void fold_parity(uint32_t taddr, int warp, unsigned (&par)[4])
{
    const uint32_t base = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t v[32];
        tmem_ld32(base + 32 * c, v);
        unsigned bits = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            bits |= ((unsigned)__float2int_rn(__uint_as_float(v[j])) & 1u) << j;
        par[c] ^= bits;
    }
}

__global__ void __launch_bounds__(NTHR, 2)
k_mul_tc(uint64_t *__restrict__ C, int64_t sc, const uint64_t *__restrict__ A, int64_t sa,
         const uint64_t *__restrict__ B, int64_t sb, int m, int k, int n, int acc, int seg, int *__restrict__ status)
{
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned stage base
    unsigned char *sm = smraw + ((1024u - ((uint32_t)__cvta_generic_to_shared(smraw) & 1023u)) & 1023u);
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) u64 s_mbar[2];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const int KW = (k + 63) >> 6, NW = (n + 63) >> 6;
    const int nchunks = (k + KC - 1) / KC;
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&s_mbar[0]);
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb0), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb0 + 8), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t sm_addr = (uint32_t)__cvta_generic_to_shared(sm);
    unsigned par[4] = {0u, 0u, 0u, 0u};
    int issued = 0;  // chunks whose MMAs have been issued (and committed)
    for (int ch = 0; ch < nchunks; ++ch) {
        const int st = ch & 1;
        unsigned char *sA = sm + st * STAGE;
        unsigned char *sB = sA + A_BYTES;
        // stage st was last read by chunk ch - 2: wait for its commit
        if (ch >= 2 && !mbar_wait(mb0 + 8 * st, (uint32_t)(((ch >> 1) - 1) & 1)))
            s_fail = 1;
        const int w0 = ch * (KC / 64);
        // A tile: thread -> (row, half): one word of one row, four core rows
        {
            const int r = tid & (TM - 1), half = tid >> 7, gr = row0 + r, w = w0 + half;
            const u64 a = (gr < m && w < KW) ? A[(int64_t)gr * sa + w] : 0ull;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                store16(sA + core_off(r, 4 * half + j), (unsigned)(a >> (16 * j)) & 0xFFFFu);
        }
        // B tile: 128 rows (inner dimension) x 4 words; warp -> two (row block, word) units
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int unit = warp * 2 + u;  // 0..15
            const int kb = unit >> 2, wi = unit & 3;
            const int krow = ch * KC + 32 * kb + lane;
            const int wcol = (col0 >> 6) + wi;
            const u64 b = (krow < k && wcol < NW) ? B[(int64_t)krow * sb + wcol] : 0ull;
            const unsigned lo = transpose32((unsigned)b, lane);          // column 64 wi + lane
            const unsigned hi = transpose32((unsigned)(b >> 32), lane);  // column 64 wi + 32 + lane
            const int r_lo = 64 * wi + lane, r_hi = r_lo + 32;
            store16(sB + core_off(r_lo, 2 * kb), lo & 0xFFFFu);
            store16(sB + core_off(r_lo, 2 * kb + 1), lo >> 16);
            store16(sB + core_off(r_hi, 2 * kb), hi & 0xFFFFu);
            store16(sB + core_off(r_hi, 2 * kb + 1), hi >> 16);
        }
        // generic-proxy writes must be visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail)
            break;
        const bool restart = (ch % seg) == 0;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_addr = sm_addr + st * STAGE, b_addr = a_addr + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < KC / 32; ++kk) {
                // K = 32 bytes = two core matrices along K
                const u64 ad = smem_desc(a_addr + kk * 2 * LBO);
                const u64 bd = smem_desc(b_addr + kk * 2 * LBO);
                const uint32_t en = (restart && kk == 0) ? 0u : 1u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                             "l"(ad), "l"(bd), "r"(IDESC), "r"(en)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb0 + 8 * st)
                         : "memory");
        }
        issued = ch + 1;
        // end of a segment: wait for its MMAs, fold the parities, restart the accumulator
        if ((ch + 1) % seg == 0 && ch + 1 < nchunks) {
            if (!mbar_wait(mb0 + 8 * st, (uint32_t)((ch >> 1) & 1)))
                s_fail = 1;
            __syncthreads();
            if (s_fail)
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            fold_parity(taddr, warp, par);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    // the last commit covers every MMA issued before it; the other stage's last
    // arrival is awaited too, so that no arrival is still on its way at exit
    if (issued > 0 && !mbar_wait(mb0 + 8 * ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1)))
        s_fail = 1;
    if (issued > 1 && !mbar_wait(mb0 + 8 * ((issued - 2) & 1), (uint32_t)(((issued - 2) >> 1) & 1)))
        s_fail = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        if (issued > 0)
            fold_parity(taddr, warp, par);
        // warp -> TMEM lane quarter (rows) and column half
        const int r = row0 + 32 * (warp & 3) + lane;
        if (r < m) {
            unsigned *crow = reinterpret_cast<unsigned *>(C + (int64_t)r * sc);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = col0 + 128 * (warp >> 2) + 32 * c;
                if (col >= 64 * NW)
                    continue;
                unsigned bits = par[c];
                if (col >= n)
                    bits = 0;
                else if (col + 32 > n)
                    bits &= (1u << (n - col)) - 1u;
                if (acc)
                    crow[col >> 5] ^= bits;
                else
                    crow[col >> 5] = bits;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_fail && tid == 0) {
        record_status(status, GF2_ETIMEOUT);
        // give the MMAs in flight one more bounded chance to finish before TMEM is freed
        if (issued > 0)
            (void)mbar_wait(mb0 + 8 * ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1));
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TN));
}

}  // namespace

namespace gf2 {

size_t mul_tensor_workspace(int64_t m, int64_t k, int64_t n)
{
    (void)m;
    (void)k;
    (void)n;
    return 0;  // B is transposed tile by tile inside the kernel
}

int mul_tensor(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
               int64_t k, int64_t n, int acc, void *work, size_t work_bytes, cudaStream_t s)
{
    (void)work;
    (void)work_bytes;
    if (m == 0 || n == 0)
        return GF2_OK;
    if (k == 0) {
        if (!acc)
            return note_cuda(cudaMemset2DAsync(C, (size_t)sc * 8, 0, (size_t)((n + 63) / 64) * 8, (size_t)m, s));
        return GF2_OK;
    }
    static bool attr = false;
    if (!attr) {
        int rc = note_cuda(cudaFuncSetAttribute(k_mul_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        if (rc)
            return rc;
        attr = true;
    }
    int *status = status_word();
    if (!status)
        return GF2_ECUDA;
    // grid.y is limited to 65535 row tiles: larger products go in slabs of rows
    constexpr int64_t SLAB = (int64_t)65535 * TM;
    for (int64_t r0 = 0; r0 < m; r0 += SLAB) {
        const int64_t mr = m - r0 < SLAB ? m - r0 : SLAB;
        const dim3 grid((unsigned)((n + TN - 1) / TN), (unsigned)((mr + TM - 1) / TM));
        const int tok = prof_begin(s);
        k_mul_tc<<<grid, NTHR, SMEM, s>>>(C + r0 * sc, sc, A + r0 * sa, sa, B, sb, (int)mr, (int)k, (int)n, acc,
                                          DEFAULT_SEG, status);
        prof_end(s, GF2_PROF_MUL, tok);
        prof_launched(1);
        const int rc = note_cuda(cudaGetLastError());
        if (rc)
            return rc;
    }
    return GF2_OK;
}

}  // namespace gf2
