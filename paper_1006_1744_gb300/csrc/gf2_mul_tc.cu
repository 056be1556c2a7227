// gf2_mul_tc.cu -- GF(2) product C = (C +) A.B on the tensor cores (sm_103a).
//
// The trailing update A_SE <- A_SE + A_SW.A_NE of Algorithm PLS (Sec. 5) is a
// matrix product over GF(2). Here every bit becomes an FP8 (e4m3) 0.0 or 1.0,
// the product runs as tcgen05.mma kind::f8f6f4 with FP32 accumulators in
// tensor memory, and the low bit of each sum is kept: the sum of the 0/1
// products is an integer and its parity is the GF(2) dot product. (sm_103a has
// no 8-bit integer MMA.) To keep every sum far inside the range the
// accumulator holds exactly, the inner dimension is cut into segments of at
// most `seg` chunks whose parities are folded into registers.
//
// Per CTA: a 128 x 256 tile of C, warp-specialised:
//   warps 0-7   expand 128-bit chunks of A (128 rows) and of B^T (256 rows; B
//               is transposed once per product into the workspace) to e4m3
//               bytes in shared memory, in the K-major layout with the 128-byte
//               swizzle, into a ring of STAGES buffers;
//   warp 8      (one thread) issues four MMAs of K = 32 per chunk into one of
//               two TMEM accumulators (256 columns each) -- one per segment,
//               alternating -- and commits them to the stage's "empty" barrier
//               and, at a segment's end, to that accumulator's "full" barrier;
//   warps 9-12  fold a finished segment's parities into registers (their TMEM
//               lane quarter each) while the next segment accumulates, then
//               write C.
// Every wait is bounded: one that gives up records GF2_ETIMEOUT in the status
// word and the CTA returns without writing C.
#include "gf2_common.cuh"

namespace {

constexpr int TM = 128;                   // rows of C per CTA (MMA M)
constexpr int TN = 256;                   // columns of C per CTA (MMA N)
constexpr int KC = 128;                   // inner-dimension bits per chunk (= bytes per expanded row)
constexpr int STAGES = 4;                 // shared-memory ring
constexpr int NPROD = 8;                  // producer warps
constexpr int MMA_WARP = NPROD;           // warp 8
constexpr int NTHR = (NPROD + 1 + 4) * 32;
constexpr int A_BYTES = TM * KC;          // 16 KB
constexpr int B_BYTES = TN * KC;          // 32 KB
constexpr int STAGE = A_BYTES + B_BYTES;  // 48 KB
constexpr int SMEM = STAGES * STAGE + 1024 + 4096;  // ring, alignment and tail slack
constexpr int DEFAULT_SEG = 64;           // chunks per accumulation segment: sums stay <= 8192

// A 1 bit becomes the e4m3 byte 0x08 (2^-6), a 0 bit 0x00; a product of two
// ones is 2^-12 and a sum of c of them is c * 2^-12, exact in FP32.
constexpr float ONE_SQ_INV = 4096.0f;  // 1 / (2^-6)^2

// four bits -> four bytes (bit i -> byte i): one multiply spreads bit i to bit
// 8 i + 3 (the shifted copies do not overlap), one mask keeps those bits
__device__ __forceinline__ unsigned expand4(unsigned nib) { return (nib * 0x01020408u) & 0x08080808u; }

// 16 bits -> one 16-byte row chunk
__device__ __forceinline__ void store16(unsigned char *p, unsigned b)
{
    uint4 v;
    v.x = expand4(b & 15u);
    v.y = expand4((b >> 4) & 15u);
    v.z = expand4((b >> 8) & 15u);
    v.w = expand4((b >> 12) & 15u);
    *reinterpret_cast<uint4 *>(p) = v;
}

// byte offset of (row, 16-byte column group cg) in the K-major layout with the
// 128-byte swizzle: each expanded row is one 128-byte swizzle row; rows come in
// atoms of 8 rows (1024 bytes), and chunk cg of row r sits at chunk cg ^ (r % 8)
// (the hardware applies the same XOR to the address bits, so stages are
// 1024-byte aligned)
constexpr int SBO = 1024;  // next group of 8 rows
__device__ __forceinline__ int core_off(int row, int cg)
{
    return (row >> 3) * SBO + (row & 7) * 128 + ((cg ^ (row & 7)) << 4);
}

// shared-memory matrix descriptor: start, LBO (unused with this swizzle), SBO (16-byte
// units), version 1, layout 128-byte swizzle
__device__ __forceinline__ u64 smem_desc(uint32_t saddr)
{
    return (u64)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((u64)(SBO >> 4) << 32) | (1ull << 46) | (2ull << 61);
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

// B (k x n bits, pitch sb) -> BT (n x k bits, pitch sbt words): 32 x 32 blocks,
// butterfly transpose across a warp; BT's padding words are zero
__global__ void k_transpose_bits(const uint64_t *__restrict__ B, int64_t sb, uint64_t *__restrict__ BT,
                                 int64_t sbt, int k, int n)
{
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int kslots = (int)(sbt * 2);  // 32-bit slots per BT row
    const int kb = (k + 31) / 32, nb = (n + 31) / 32;
    for (int blk = warp; blk < kslots * nb; blk += nwarps) {
        const int bk = blk % kslots, bn = blk / kslots;
        const int row = 32 * bk + lane;  // row of B
        unsigned x = 0;
        if (bk < kb && row < k) {
            const int col = 32 * bn;
            x = (unsigned)(B[(int64_t)row * sb + (col >> 6)] >> (col & 63));
        }
        x = transpose32(x, lane);  // lane c: column 32 bn + c over rows 32 bk .. 32 bk + 31
        const int ocol = 32 * bn + lane;
        if (ocol < n)
            reinterpret_cast<unsigned *>(BT + (int64_t)ocol * sbt)[bk] = x;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mb)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(mb) : "memory");
}

__global__ void __launch_bounds__(NTHR, 1)
k_mul_tc(uint64_t *__restrict__ C, int64_t sc, const uint64_t *__restrict__ A, int64_t sa,
         const uint64_t *__restrict__ B /* B transposed: n x k bits */, int64_t sb, int m, int k, int n, int acc,
         int seg, int *__restrict__ status)
{
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned ring
    unsigned char *sm = smraw + ((1024u - ((uint32_t)__cvta_generic_to_shared(smraw) & 1023u)) & 1023u);
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) u64 s_full[STAGES], s_empty[STAGES], s_sfull[2], s_sempty[2];
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
    const int KW = (k + 63) >> 6, NW = (n + 63) >> 6;
    const int nchunks = (k + KC - 1) / KC;
    const int nseg = (nchunks + seg - 1) / seg;
    const uint32_t full0 = (uint32_t)__cvta_generic_to_shared(&s_full[0]);
    const uint32_t empty0 = (uint32_t)__cvta_generic_to_shared(&s_empty[0]);
    const uint32_t sfull0 = (uint32_t)__cvta_generic_to_shared(&s_sfull[0]);
    const uint32_t sempty0 = (uint32_t)__cvta_generic_to_shared(&s_sempty[0]);
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(2 * TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * i), "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty0 + 8 * i), "r"(1));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sfull0 + 8 * i), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sempty0 + 8 * i), "r"(4));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t sm_addr = (uint32_t)__cvta_generic_to_shared(sm);
    unsigned par[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};

    if (warp < NPROD) {
        // ---------------- producers: expand chunk c into stage c % STAGES ----------------
        // The packed words of the next PD chunks are in flight in registers, so a chunk
        // never waits for its own global loads.
        constexpr int PD = 4;
        const int ar = tid & (TM - 1), ahalf = tid >> 7, agr = row0 + ar;
        const int bgr = col0 + tid;  // row of BT (= column of B) this thread expands
        u64 qa[PD], qb0[PD], qb1[PD];
        auto load = [&](int c, u64 &a, u64 &b0, u64 &b1) {
            const int w = c * (KC / 64);
            a = (c < nchunks && agr < m && w + ahalf < KW) ? A[(int64_t)agr * sa + w + ahalf] : 0ull;
            b0 = 0;
            b1 = 0;
            if (c < nchunks && bgr < n) {  // BT's pitch is even: both words of a chunk exist
                const ulonglong2 v2 = *reinterpret_cast<const ulonglong2 *>(B + (int64_t)bgr * sb + w);
                b0 = v2.x;
                b1 = v2.y;
            }
        };
#pragma unroll
        for (int i = 0; i < PD; ++i)
            load(i, qa[i], qb0[i], qb1[i]);
        for (int c = 0; c < nchunks && !s_fail; ++c) {
            const int st = c % STAGES;
            if (!mbar_wait(empty0 + 8 * st, (uint32_t)(((c / STAGES) & 1) ^ 1))) {
                s_fail = 1;
                break;
            }
            unsigned char *sA = sm + st * STAGE;
            unsigned char *sB = sA + A_BYTES;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                store16(sA + core_off(ar, 4 * ahalf + j), (unsigned)(qa[0] >> (16 * j)) & 0xFFFFu);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                store16(sB + core_off(tid, j), (unsigned)(qb0[0] >> (16 * j)) & 0xFFFFu);
                store16(sB + core_off(tid, 4 + j), (unsigned)(qb1[0] >> (16 * j)) & 0xFFFFu);
            }
            // generic-proxy writes must be visible to the tensor cores (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                mbar_arrive(full0 + 8 * st);
#pragma unroll
            for (int i = 0; i < PD - 1; ++i) {
                qa[i] = qa[i + 1];
                qb0[i] = qb0[i + 1];
                qb1[i] = qb1[i + 1];
            }
            load(c + PD, qa[PD - 1], qb0[PD - 1], qb1[PD - 1]);
        }
        // the last stages' release arrivals, so that none lands after the CTA exits
        for (int c = max(0, nchunks - STAGES); c < nchunks && !s_fail; ++c)
            if (!mbar_wait(empty0 + 8 * (c % STAGES), (uint32_t)((c / STAGES) & 1)))
                s_fail = 1;
    } else if (warp == MMA_WARP) {
        // ---------------- one thread issues the MMAs ----------------
        if (lane == 0) {
            for (int c = 0; c < nchunks && !s_fail; ++c) {
                const int st = c % STAGES, sg = c / seg, a = sg & 1;
                const bool first = c % seg == 0;
                const bool last = c % seg == seg - 1 || c == nchunks - 1;
                if (first && !mbar_wait(sempty0 + 8 * a, (uint32_t)(((sg >> 1) & 1) ^ 1))) {
                    s_fail = 1;
                    break;
                }
                if (!mbar_wait(full0 + 8 * st, (uint32_t)((c / STAGES) & 1))) {
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a_addr = sm_addr + st * STAGE, b_addr = a_addr + A_BYTES;
                const uint32_t dst = taddr + (uint32_t)(a * TN);
#pragma unroll
                for (int kk = 0; kk < KC / 32; ++kk) {
                    // K = 32 bytes: the next 32 bytes of every 128-byte row
                    const u64 ad = smem_desc(a_addr + kk * 32);
                    const u64 bd = smem_desc(b_addr + kk * 32);
                    const uint32_t en = (first && kk == 0) ? 0u : 1u;
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(dst),
                                 "l"(ad), "l"(bd), "r"(IDESC), "r"(en)
                                 : "memory");
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * st)
                    : "memory");
                if (last)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     sfull0 + 8 * a)
                                 : "memory");
            }
        }
    } else {
        // ---------------- epilogue: fold every segment, then write C ----------------
        const int q = warp & 3;  // TMEM lane quarter = rows 32 q .. 32 q + 31
        for (int sg = 0; sg < nseg && !s_fail; ++sg) {
            const int a = sg & 1;
            if (!mbar_wait(sfull0 + 8 * a, (uint32_t)((sg >> 1) & 1))) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * TN);
#pragma unroll
            for (int c32 = 0; c32 < TN / 32; ++c32) {
                uint32_t v[32];
                tmem_ld32(base + 32 * c32, v);
                unsigned bits = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    bits |= ((unsigned)__float2int_rn(__uint_as_float(v[j]) * ONE_SQ_INV) & 1u) << j;
                par[c32] ^= bits;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                mbar_arrive(sempty0 + 8 * a);
        }
        if (!s_fail && nchunks > 0) {
            const int r = row0 + 32 * q + lane;
            if (r < m) {
                unsigned *crow = reinterpret_cast<unsigned *>(C + (int64_t)r * sc);
#pragma unroll
                for (int c32 = 0; c32 < TN / 32; ++c32) {
                    const int col = col0 + 32 * c32;
                    if (col >= 64 * NW)
                        continue;
                    unsigned bits = par[c32];
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_fail && tid == 0)
        record_status(status, GF2_ETIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * TN));
}

}  // namespace

namespace gf2 {

// row pitch (words) of B^T: whole 128-bit chunks
static int64_t bt_pitch(int64_t k)
{
    const int64_t w = (k + 63) / 64;
    return w < 2 ? 2 : (w + 1) / 2 * 2;
}

size_t mul_tensor_workspace(int64_t m, int64_t k, int64_t n)
{
    (void)m;
    return align_up((size_t)n * (size_t)bt_pitch(k) * 8, 256);  // B^T
}

int mul_tensor(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
               int64_t k, int64_t n, int acc, void *work, size_t work_bytes, cudaStream_t s)
{
    if (m == 0 || n == 0)
        return GF2_OK;
    if (k > 0 && (!work || work_bytes < mul_tensor_workspace(m, k, n)))
        return GF2_ENOSPACE;
    if (k == 0) {
        if (!acc)
            return note_cuda(cudaMemset2DAsync(C, (size_t)sc * 8, 0, (size_t)((n + 63) / 64) * 8, (size_t)m, s));
        return GF2_OK;
    }
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        int rc = note_cuda(cudaFuncSetAttribute(k_mul_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        if (rc)
            return rc;
        attr_done(attr_devs);
    }
    int *status = status_word();
    if (!status)
        return GF2_ECUDA;
    uint64_t *BT = reinterpret_cast<uint64_t *>(work);
    const int64_t sbt = bt_pitch(k);
    k_transpose_bits<<<2 * sm_count(), 256, 0, s>>>(B, sb, BT, sbt, (int)k, (int)n);
    prof_launched(1);
    int rc0 = note_cuda(cudaGetLastError());
    if (rc0)
        return rc0;
    // grid.y is limited to 65535 row tiles: larger products go in slabs of rows
    constexpr int64_t SLAB = (int64_t)65535 * TM;
    for (int64_t r0 = 0; r0 < m; r0 += SLAB) {
        const int64_t mr = m - r0 < SLAB ? m - r0 : SLAB;
        const dim3 grid((unsigned)((n + TN - 1) / TN), (unsigned)((mr + TM - 1) / TM));
        const int tok = prof_begin(s);
        k_mul_tc<<<grid, NTHR, SMEM, s>>>(C + r0 * sc, sc, A + r0 * sa, sa, BT, sbt, (int)mr, (int)k, (int)n, acc,
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
