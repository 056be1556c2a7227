// gf2_rref.cu -- reduced row echelon form from the PLS elimination.
//
// The "PLS" column of Table 1 (Sec. 7) times a PLS decomposition followed by
// the RREF computed from it; the paper does not spell out the second step. Here
// it is the upper-triangular solve R = (S_J)^-1 . S, where S is the echelon
// part of the pivot rows and S_J its columns at the pivot positions Q[0..r)
// (unit upper triangular). With the columns split into pivot and non-pivot
// ones, S = [U1 | B] and R = [I | U1^-1 B]; only X = U1^-1 B is computed
// (back substitution over 64-pivot blocks, from the last block up), then R is
// scattered back to the original column order. The RREF is unique
// (Definition "Reduced Row Echelon Form"), so this matches any other route.
#include "gf2_common.cuh"

namespace {

// Per pivot row i (< r): drop everything left of its pivot Q[i], split the
// remaining bits into pivot columns (-> U1 row i, positions i.., stored in the
// caller's matrix which is overwritten by the result anyway) and non-pivot
// columns (-> B row i, positions Q[i]-i .., the positions before are zero).
__global__ void k_rref_compact(const uint64_t *__restrict__ S, int64_t stride, const int64_t *__restrict__ Q,
                               const u64 *__restrict__ pmask, const PanelState *__restrict__ st,
                               uint64_t *__restrict__ U1, int64_t ustride, u64 *__restrict__ Bc, int64_t sb, int n,
                               int W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = st->r_next;
    if (i >= r)
        return;
    const int nn = n - r;
    const int64_t q = Q[i];
    const uint64_t *row = S + (int64_t)i * stride;
    uint64_t *urow = U1 + (int64_t)i * ustride;
    u64 *brow = Bc + (int64_t)i * sb;
    // U1 stream from position i, B stream from position q - i
    int64_t up = i, bp = q - i;
    int64_t uw = up >> 6, bw = bp >> 6;
    u64 ucur = 0, bcur = 0;
    const int NBw = (nn + 63) >> 6;
    for (int64_t w = 0; w < bw && w < NBw; ++w)
        brow[w] = 0;
    for (int64_t w = q >> 6; w < W; ++w) {
        u64 word = row[w];
        u64 valid = (w == W - 1 && (n & 63)) ? lowmask(n & 63) : ~0ull;
        if (w == (q >> 6))
            valid &= ~lowmask((int)(q & 63));
        word &= valid;
        const u64 pm = pmask[w] & valid, nm = ~pmask[w] & valid;
        const u64 ub = pext64(word, pm), bb = pext64(word, nm);
        const int uk = __popcll(pm), bk = __popcll(nm);
        int off = (int)(up & 63);
        ucur |= ub << off;
        if (off + uk >= 64) {
            urow[uw++] = ucur;
            ucur = off == 0 ? 0ull : (ub >> (64 - off));
        }
        up += uk;
        off = (int)(bp & 63);
        bcur |= bb << off;
        if (off + bk >= 64) {
            brow[bw++] = bcur;
            bcur = off == 0 ? 0ull : (bb >> (64 - off));
        }
        bp += bk;
    }
    if (up & 63)
        urow[uw] = ucur;
    if ((bp & 63) && bw < NBw)
        brow[bw] = bcur;
}

// Inverses of the 64x64 unit upper-triangular diagonal blocks of U1 (one warp
// per block; rows past the rank are identity). Back substitution by columns:
// X = I; for h = 63 .. 0, every row i < h with D[i][h] = 1 gets X[h] added.
__global__ void k_diag_inv(const uint64_t *__restrict__ U1, int64_t stride, const PanelState *__restrict__ st,
                           u64 *__restrict__ Dinv, int nblk)
{
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int r = st->r_next;
    if (q >= nblk || 64 * q >= r)
        return;
    const int base = 64 * q;
    u64 d0 = 1ull << lane, d1 = 1ull << (lane + 32);
    if (base + lane < r)
        d0 |= U1[(int64_t)(base + lane) * stride + q] & ~lowmask(lane + 1);
    if (base + lane + 32 < r)
        d1 |= U1[(int64_t)(base + lane + 32) * stride + q] & ~lowmask(lane + 33);
    u64 x0 = 1ull << lane, x1 = 1ull << (lane + 32);
    for (int h = 63; h >= 1; --h) {
        const u64 xh = __shfl_sync(GF2_FULL, h < 32 ? x0 : x1, h & 31);
        if (lane < h && ((d0 >> h) & 1ull))
            x0 ^= xh;
        if (lane + 32 < h && ((d1 >> h) & 1ull))
            x1 ^= xh;
    }
    Dinv[(int64_t)q * 64 + lane] = x0;
    Dinv[(int64_t)q * 64 + lane + 32] = x1;
}

// Back substitution X = U1^-1 B over groups of G blocks of 64 pivots, from the
// last group up. Within a group (k_rref_group, one CTA per tile of TW1 words of
// B): for each block q from the group's last to its first,
//   X_q = Dinv_q . B_q              (B_q holds every update from below),
//   B_i += U1[i, block q] . X_q     for the group's rows i above block q.
// Then (k_rref_bulk) every row above the group takes the whole group at once:
//   B_i += sum over the group's blocks q of U1[i, block q] . X_q,
// with one Gray-code table per 8 pivots (G x 8 tables).
constexpr int G = 8;     // blocks per group
constexpr int TW1 = 1;   // words of B per CTA in the group solve (a near-full-rank matrix has one)
constexpr int TWG = 1;   // words of B per CTA in the bulk update
static_assert(TWG == 1, "the bulk update's lookups assume one word per tile");

// Gray-code tables of 64 rows x TW words: T[g][v][w] = sum of the rows 8 g + e
// for the set bits e of v (MakeTable: each entry one row away from the last)
template <int TW>
__device__ __forceinline__ void gray_tables(const u64 *__restrict__ rows, u64 *__restrict__ T, int tid)
{
    for (int e = tid; e < 8 * TW * 16; e += blockDim.x) {
        const int w = e % TW, rest = e / TW, vh = rest & 15, g = rest >> 4;
        const u64 *Og = rows + (8 * g) * TW + w;
        u64 cur = 0;
#pragma unroll
        for (int bit = 0; bit < 4; ++bit)
            if ((vh >> bit) & 1)
                cur ^= Og[(4 + bit) * TW];
        gray16(cur, Og[0], Og[TW], Og[2 * TW], Og[3 * TW], T + (g * 256 + (vh << 4)) * TW + w, TW);
    }
}

__global__ void __launch_bounds__(256, 1)
k_rref_group(u64 *__restrict__ Bc, u64 *__restrict__ Xc, int64_t sb, const uint64_t *__restrict__ U1,
             int64_t stride, const u64 *__restrict__ Dinv, const PanelState *__restrict__ st, int n, int q0)
{
    extern __shared__ __align__(16) u64 smg[];
    u64 *sB = smg;                   // [G * 64][TW1]  the group's rows of B
    u64 *sU = sB + G * 64 * TW1;     // [G * 64][G]    the group's rows of U1 at the group's blocks
    u64 *sT = sU + G * 64 * G;       // [8][256][TW1]  tables of X_q
    u64 *sX = sT + 8 * 256 * TW1;    // [64][TW1]
    u64 *sD = sX + 64 * TW1;         // [G][64] inverses of the group's diagonal blocks
    const int r = st->r_next;
    const int NB = (n - r + 63) >> 6;
    const int base = 64 * q0;
    if (base >= r || NB == 0)
        return;
    const int tid = threadIdx.x;
    const int wb = blockIdx.x * TW1;
    if (wb >= NB)
        return;
    const int rows = min(G * 64, r - base);
    const int qend = q0 + (rows + 63) / 64;  // one past the group's last block
    if (64 * qend <= st->r_switch) {
        // every row of the group was reduced by the hybrid's reduced-form panels: its diagonal
        // blocks are the identity and it has no entries in its own blocks, so X = B
        for (int e = tid; e < rows * TW1; e += blockDim.x) {
            const int i = e / TW1, w = e % TW1;
            if (wb + w < NB)
                Xc[(int64_t)(base + i) * sb + wb + w] = Bc[(int64_t)(base + i) * sb + wb + w];
        }
        return;
    }
    for (int e = tid; e < G * 64 * TW1; e += blockDim.x) {
        const int i = e / TW1, w = e % TW1;
        sB[e] = (i < rows && wb + w < NB) ? Bc[(int64_t)(base + i) * sb + wb + w] : 0ull;
    }
    for (int e = tid; e < G * 64 * G; e += blockDim.x) {
        const int i = e / G, qq = e % G;
        sU[e] = (i < rows && q0 + qq < qend) ? U1[(int64_t)(base + i) * stride + q0 + qq] : 0ull;
    }
    for (int e = tid; e < (qend - q0) * 64; e += blockDim.x)
        sD[e] = Dinv[(int64_t)q0 * 64 + e];
    for (int q = qend - 1; q >= q0; --q) {
        const int lq = q - q0;
        const int nrow = min(64, r - 64 * q);
        __syncthreads();
        // X_q = Dinv_q B_q: tables of B_q's rows, eight lookups per row of X_q
        gray_tables<TW1>(sB + lq * 64 * TW1, sT, tid);
        __syncthreads();
        for (int e = tid; e < 64 * TW1; e += blockDim.x) {
            const int s2 = e / TW1, w = e % TW1;
            const u64 d = sD[lq * 64 + s2];
            u64 x = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g)
                x ^= sT[(g * 256 + (int)((d >> (8 * g)) & 255ull)) * TW1 + w];
            sX[e] = x;
            if (s2 < nrow && wb + w < NB)
                Xc[(int64_t)(64 * q + s2) * sb + wb + w] = x;
        }
        if (lq == 0)
            break;  // no group rows above the first block
        __syncthreads();
        gray_tables<TW1>(sX, sT, tid);  // tables of X_q's rows
        __syncthreads();
        // the group's rows above block q
        for (int e = tid; e < lq * 64 * TW1; e += blockDim.x) {
            const int i = e / TW1, w = e % TW1;
            const u64 u = sU[i * G + lq];
            u64 acc = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g)
                acc ^= sT[(g * 256 + (int)((u >> (8 * g)) & 255ull)) * TW1 + w];
            sB[e] ^= acc;
        }
    }
}

__global__ void __launch_bounds__(256, 1)
k_rref_bulk(u64 *__restrict__ Bc, const u64 *__restrict__ Xc, int64_t sb, const uint64_t *__restrict__ U1,
            int64_t stride, const PanelState *__restrict__ st, int n, int q0)
{
    extern __shared__ __align__(16) u64 smk[];
    u64 *sT = smk;                      // [G][8][256][TWG]
    u64 *sXg = sT + G * 8 * 256 * TWG;  // [G * 64][TWG]
    const int r = st->r_next;
    const int NB = (n - r + 63) >> 6;
    const int above = 64 * q0;
    if (above == 0 || above >= r || NB == 0)
        return;
    const int tid = threadIdx.x;
    const int nblk = min(G, (r - above + 63) / 64);
    if (64 * (q0 + nblk) <= st->r_switch)
        return;  // the group and every row above it were reduced by the hybrid's reduced-form panels
    const int tiles = (NB + TWG - 1) / TWG;
    int chunks = gridDim.x / tiles;
    if (chunks < 1)
        chunks = 1;
    const int R = (above + chunks - 1) / chunks;
    const int items = tiles * chunks;
    int cur_tile = -1;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item / chunks, chunk = item % chunks;
        const int wb = tile * TWG;
        const int i0 = chunk * R, i1 = min(above, i0 + R);
        // this thread's first row of U1, in flight while the tables are built
        u64 upre[G];
#pragma unroll
        for (int qq = 0; qq < G; ++qq)
            upre[qq] = (i0 + tid < i1 && qq < nblk) ? U1[(int64_t)(i0 + tid) * stride + q0 + qq] : 0ull;
        if (tile != cur_tile) {
            __syncthreads();
            for (int e = tid; e < G * 64 * TWG; e += blockDim.x) {
                const int i = e / TWG, w = e % TWG;
                sXg[e] = (i < min(G * 64, r - above) && wb + w < NB) ? Xc[(int64_t)(above + i) * sb + wb + w] : 0ull;
            }
            __syncthreads();
            for (int e = tid; e < nblk * 8 * TWG * 16; e += blockDim.x) {
                const int w = e % TWG, rest = e / TWG, vh = rest & 15, g = (rest >> 4) & 7, qq = rest >> 7;
                const u64 *Xg = sXg + (64 * qq + 8 * g) * TWG + w;
                u64 cur = 0;
#pragma unroll
                for (int bit = 0; bit < 4; ++bit)
                    if ((vh >> bit) & 1)
                        cur ^= Xg[(4 + bit) * TWG];
                gray16(cur, Xg[0], Xg[TWG], Xg[2 * TWG], Xg[3 * TWG], sT + ((qq * 8 + g) * 256 + (vh << 4)) * TWG + w,
                       TWG);
            }
            __syncthreads();
            cur_tile = tile;
        }
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
            const uint64_t *urow = U1 + (int64_t)i * stride + q0;
            u64 acc = 0;
#pragma unroll
            for (int qq = 0; qq < G; ++qq) {
                if (qq < nblk) {
                    const u64 u = i == i0 + tid ? upre[qq] : urow[qq];
#pragma unroll
                    for (int g = 0; g < 8; ++g)
                        acc ^= sT[((qq * 8 + g) * 256 + (int)((u >> (8 * g)) & 255ull)) * TWG];
                }
            }
            Bc[(int64_t)i * sb + wb] ^= acc;
        }
    }
}

// R row i < r: 1 at Q[i], X row i deposited into the non-pivot columns.
// Rows >= r: zero.
__global__ void k_rref_scatter(uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ Xc, int64_t sb,
                               const int64_t *__restrict__ Q, const u64 *__restrict__ pmask,
                               const PanelState *__restrict__ st, int m, int n, int W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m)
        return;
    const int r = st->r_next;
    uint64_t *row = A + (int64_t)i * stride;
    if (i >= r) {
        for (int w = 0; w < W; ++w)
            row[w] = 0;
        return;
    }
    const u64 *xr = Xc + (int64_t)i * sb;
    const int64_t q = Q[i];
    int64_t xp = 0;
    for (int w = 0; w < W; ++w) {
        const u64 valid = (w == W - 1 && (n & 63)) ? lowmask(n & 63) : ~0ull;
        const u64 nm = ~pmask[w] & valid;
        const int k = __popcll(nm);
        u64 v = 0;
        if (k) {
            const int off = (int)(xp & 63);
            u64 bits = xr[xp >> 6] >> off;
            if (off + k > 64)
                bits |= xr[(xp >> 6) + 1] << (64 - off);
            v = pdep64(bits & lowmask(k), nm);
            xp += k;
        }
        if ((q >> 6) == w)
            v |= 1ull << (q & 63);
        row[w] = v;
    }
}

__global__ void k_rref_outputs(const int64_t *__restrict__ Q, const PanelState *__restrict__ st, int n,
                               int64_t *__restrict__ pivots, int64_t *__restrict__ rank)
{
    const int r = st->r_next;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (pivots)
        for (int i = g; i < n; i += gridDim.x * blockDim.x)
            pivots[i] = i < r ? Q[i] : i;
    if (g == 0 && rank)
        *rank = r;
}

__global__ void k_pmask2(const int64_t *__restrict__ Q, const PanelState *__restrict__ st, u64 *__restrict__ pmask)
{
    const int r = st->r_next;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < r; s += gridDim.x * blockDim.x) {
        const int64_t c = Q[s];
        atomicOr(&pmask[c >> 6], 1ull << (c & 63));
    }
}

}  // namespace

namespace gf2 {

// Algorithm M4RI's result: the pivot rows are already reduced (in `out`, final positions, words
// from their panel on); the gather adds their zero words left of the panel and the zero rows
// past the rank, then `out` is copied back. pivots = Q.
int m4ri_finish(const Elim &e, int64_t *rank, int64_t *pivots)
{
    int rc = elim_gather(e, rank);
    if (rc)
        return rc;
    cudaError_t err = cudaMemcpy2DAsync(e.A, (size_t)e.stride * 8, e.out, (size_t)e.ostride * 8, (size_t)e.W * 8,
                                        (size_t)e.m, cudaMemcpyDeviceToDevice, e.s);
    if (err == cudaSuccess && pivots)
        err = cudaMemcpyAsync(pivots, e.Q, (size_t)e.n * sizeof(int64_t), cudaMemcpyDeviceToDevice, e.s);
    return note_cuda(err);
}

int rref_finish(const Elim &e, const ElimLayout &L, char *work, int64_t *rank, int64_t *pivots)
{
    const int m = (int)e.m, n = (int)e.n, W = (int)e.W;
    const int64_t sb = e.W;  // row pitch of B and X in words
    u64 *Bc = reinterpret_cast<u64 *>(work + L.rref_b);
    u64 *Xc = reinterpret_cast<u64 *>(work + L.rref_x);
    u64 *Dinv = reinterpret_cast<u64 *>(work + L.rref_d);
    cudaError_t err = cudaMemsetAsync(e.pmask, 0, (size_t)W * sizeof(u64), e.s);
    if (err != cudaSuccess)
        return note_cuda(err);
    k_pmask2<<<64, 256, 0, e.s>>>(e.Q, e.stf, e.pmask);
    const int rmax = m < n ? m : n;
    k_rref_compact<<<(rmax + 127) / 128, 128, 0, e.s>>>(e.out, e.ostride, e.Q, e.pmask, e.stf, e.A, e.stride, Bc, sb, n,
                                                          W);
    const int nblk = (rmax + 63) / 64;
    k_diag_inv<<<(nblk + 3) / 4, 128, 0, e.s>>>(e.A, e.stride, e.stf, Dinv, nblk);
    prof_launched(3);
    int rc = note_cuda(cudaGetLastError());
    if (rc)
        return rc;
    const int grid = sm_count();
    const size_t smem_g = (size_t)(G * 64 * TW1 + G * 64 * G + 8 * 256 * TW1 + 64 * TW1 + G * 64) * sizeof(u64);
    const size_t smem_b = (size_t)(G * 8 * 256 * TWG + G * 64 * TWG) * sizeof(u64);
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        rc = note_cuda(cudaFuncSetAttribute(k_rref_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g));
        if (!rc)
            rc = note_cuda(
                cudaFuncSetAttribute(k_rref_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
        if (rc)
            return rc;
        attr_done(attr_devs);
    }
    // B tiles of the group solve: ceil(NB / TW1) CTAs, NB <= W
    const int gtiles = (W + TW1 - 1) / TW1;
    for (int q0 = (nblk - 1) / G * G; q0 >= 0; q0 -= G) {
        int tok = prof_begin(e.s);
        k_rref_group<<<gtiles, 256, smem_g, e.s>>>(Bc, Xc, sb, e.A, e.stride, Dinv, e.stf, n, q0);
        prof_end(e.s, GF2_PROF_RREF, tok);
        if (q0 > 0) {
            tok = prof_begin(e.s);
            k_rref_bulk<<<grid, 256, smem_b, e.s>>>(Bc, Xc, sb, e.A, e.stride, e.stf, n, q0);
            prof_end(e.s, GF2_PROF_RREF, tok);
        }
        prof_launched(q0 > 0 ? 2 : 1);
        rc = note_cuda(cudaGetLastError());
        if (rc)
            return rc;
    }
    k_rref_scatter<<<(m + 127) / 128, 128, 0, e.s>>>(e.A, e.stride, Xc, sb, e.Q, e.pmask, e.stf, m, n, W);
    k_rref_outputs<<<32, 256, 0, e.s>>>(e.Q, e.stf, n, pivots, rank);
    prof_launched(2);
    return note_cuda(cudaGetLastError());
}

}  // namespace gf2
