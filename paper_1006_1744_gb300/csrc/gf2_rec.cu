// gf2_rec.cu -- recursive PLS decomposition (Algorithm PLS, Sec. 5) with the
// panel elimination (MMPF, Sec. 4.1) as the base case below a column cutoff
// (Sec. 6).
//
// PLS(A) on an m x n view whose columns start on a word boundary:
//   n0  = a word boundary near n/2 (Sec. 6: cut along word boundaries; here a
//         1024- or 128-column boundary so that every view stays aligned);
//   r0  = PLS(A0 = columns [0, n0));                     first recursive call
//   A1 <- P.A1                                           row gather, k_row_gather
//   A_NE <- L_NW^-1 A_NE                                 lower solve over 64-row blocks
//   A_SE <- A_SE + A_SW.A_NE                             product (gf2_mul kernels)
//   r1  = PLS(A_SE);                                     second recursive call
//   A_SW <- P1.A_SW                                      row gather
//   P, Q merged; the second call's L columns move next to the first call's
//   (k_colshift: the swaps of columns i and n0+i-r0 from row i on).
// Rows are permuted with explicit position -> row maps (each call also
// returns the map of its own row order), so "P.A1" is one gather.
//
// The host reads r0 of every recursion node (one stream synchronisation per
// node) to size the views of the next steps.
#include <algorithm>
#include <vector>

#include "gf2_common.cuh"

namespace {

// dst rows p <- src rows perm[p], words [0, W)
__global__ void k_row_gather(const uint64_t *__restrict__ src, int64_t ss, uint64_t *__restrict__ dst, int64_t ds,
                             const int *__restrict__ perm, int m, int W)
{
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int p = wid; p < m; p += warps) {
        const uint64_t *s = src + (int64_t)perm[p] * ss;
        uint64_t *d = dst + (int64_t)p * ds;
        for (int w = lane; w < W; w += 32)
            d[w] = s[w];
    }
}

// out[i] = perm0[i] (i < r0), perm0[r0 + perm1[i - r0]] (i >= r0)
__global__ void k_perm_compose(const int *__restrict__ perm0, const int *__restrict__ perm1, int *__restrict__ out,
                               int r0, int m)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[i] = i < r0 ? perm0[i] : perm0[r0 + perm1[i - r0]];
}

// P[r0 + i] += r0 (the second call's local swaps), Q[n0 + i] += n0 into tmp
__global__ void k_pq_shift(int64_t *__restrict__ P, int r0, int m, const int64_t *__restrict__ Q, int n0, int n,
                           int64_t *__restrict__ tmp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = g; i < m - r0; i += nt)
        P[r0 + i] += r0;
    for (int i = g; i < n - n0; i += nt)
        tmp[i] = Q[n0 + i] + n0;
}

// Q[r0 + i] = second call's pivot columns (i < r1), identity beyond the rank
__global__ void k_q_merge(int64_t *__restrict__ Q, const int64_t *__restrict__ tmp, int r0, int r1, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = r0 + g; i < n; i += nt)
        Q[i] = (i < r0 + r1) ? tmp[i - r0] : i;
}

__global__ void k_set_rank(int64_t *rank, int64_t v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *rank = v;
}

// Compression of the second call's L columns: for every row i >= r0 (view
// rows), with u = min(i - r0, r1 - 1): bits [r0, r0+u] <- bits [n0, n0+u] and
// bits (r0+u, n0+u] <- 0. This is the effect of swapping columns j and
// n0 + j - r0 from row j on, for j = r0 .. r0+r1-1, given that rows >= r0 are
// zero in columns [r0, n0) after the first call. One warp per row, words in
// increasing order (each output word reads only words at or right of it).
__global__ void k_colshift(uint64_t *__restrict__ A, int64_t stride, int m, int r0, int n0, int r1)
{
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t d = (int64_t)n0 - r0;
    if (r1 <= 0 || d <= 0)
        return;
    for (int i = r0 + wid; i < m; i += warps) {
        const int u = min(i - r0, r1 - 1);
        const int64_t lo = r0, hi = (int64_t)n0 + u;  // modified bit range [lo, hi]
        const int64_t cend = (int64_t)r0 + u;          // last copied destination bit
        uint64_t *row = A + (int64_t)i * stride;
        const int64_t w0 = lo >> 6, w1 = hi >> 6;
        for (int64_t base = w0; base <= w1; base += 32) {
            const int64_t ow = base + lane;
            u64 nv = 0;
            bool act = ow <= w1;
            if (act) {
                const u64 old = row[ow];
                // masks within this word: bits modified, bits copied
                const int64_t wlo = 64 * ow, whi = wlo + 63;
                const int64_t ml = lo > wlo ? lo - wlo : 0, mh = hi < whi ? hi - wlo : 63;
                const int64_t cl = lo > wlo ? lo - wlo : 0, ch = cend < whi ? cend - wlo : 63;
                u64 mod = 0, cop = 0;
                if (ml <= mh)
                    mod = lowmask((int)(mh + 1)) & ~lowmask((int)ml);
                if (cend >= wlo && cl <= ch)
                    cop = lowmask((int)(ch + 1)) & ~lowmask((int)cl);
                u64 shifted = 0;
                if (cop) {
                    // source of destination bit x is bit x + d <= hi: words at or before hi >> 6
                    const int64_t sb = 64 * ow + d;
                    const int64_t sw = sb >> 6;
                    const int sh = (int)(sb & 63);
                    const u64 s0 = row[sw];
                    const u64 s1 = (sh && (sw + 1) * 64 <= hi) ? row[sw + 1] : 0ull;
                    shifted = sh ? ((s0 >> sh) | (s1 << (64 - sh))) : s0;
                }
                nv = (old & ~mod) | (shifted & cop);
            }
            __syncwarp();
            if (act)
                row[ow] = nv;
            __syncwarp();
        }
    }
}

// inverses of the 64x64 unit lower-triangular diagonal blocks of L (rows
// 64q+s, word q, bits < s); rows past r are identity
__global__ void k_diag_inv_lower(const uint64_t *__restrict__ L, int64_t stride, int r, u64 *__restrict__ Dinv,
                                 int nblk)
{
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nblk)
        return;
    const int base = 64 * q;
    u64 d0 = 1ull << lane, d1 = 1ull << (lane + 32);
    if (base + lane < r)
        d0 |= L[(int64_t)(base + lane) * stride + q] & lowmask(lane);
    if (base + lane + 32 < r)
        d1 |= L[(int64_t)(base + lane + 32) * stride + q] & lowmask(lane + 32);
    // forward substitution by columns: X = I; for h = 0 .. 63, every row i > h with
    // D[i][h] = 1 gets X[h] added (X[h] is final once the columns left of it are done)
    u64 x0 = 1ull << lane, x1 = 1ull << (lane + 32);
    for (int h = 0; h < 63; ++h) {
        const u64 xh = __shfl_sync(GF2_FULL, h < 32 ? x0 : x1, h & 31);
        if (lane > h && ((d0 >> h) & 1ull))
            x0 ^= xh;
        if (lane + 32 > h && ((d1 >> h) & 1ull))
            x1 ^= xh;
    }
    Dinv[(int64_t)q * 64 + lane] = x0;
    Dinv[(int64_t)q * 64 + lane + 32] = x1;
}

template <int TWB>
__device__ __forceinline__ void rec_tables(const u64 *__restrict__ rows, u64 *__restrict__ T, int tid)
{
    for (int e = tid; e < 8 * TWB * 16; e += blockDim.x) {
        const int wi = e % TWB, rest = e / TWB, vh = rest & 15, g = rest >> 4;
        const u64 *Og = rows + (8 * g) * TWB + wi;
        u64 cur = 0;
#pragma unroll
        for (int bit = 0; bit < 4; ++bit)
            if ((vh >> bit) & 1)
                cur ^= Og[(4 + bit) * TWB];
        gray16(cur, Og[0], Og[TWB], Og[2 * TWB], Og[3 * TWB], T + (g * 256 + (vh << 4)) * TWB + wi, TWB);
    }
}

// One 64-row block q of the lower solve X = L^-1 B (B: r rows of NB words):
//   X_q = Dinv_q . B_q       (B_q holds every update from the blocks above)
//   B_i += L[i, block q] . X_q for every row i in [64q+64, r).
// X_q goes to X (a separate buffer: B_q is read by every CTA).
constexpr int TWR = 2;
__global__ void __launch_bounds__(256, 1)
k_trsm_step(uint64_t *__restrict__ B, int64_t sb, uint64_t *__restrict__ X, int64_t sx, const uint64_t *__restrict__ L,
            int64_t sl, const u64 *__restrict__ Dinv, int r, int NB, int q)
{
    extern __shared__ __align__(16) u64 smt[];
    u64 *sTB = smt;
    u64 *sTX = sTB + 8 * 256 * TWR;
    u64 *sB = sTX + 8 * 256 * TWR;
    u64 *sX = sB + 64 * TWR;
    u64 *sD = sX + 64 * TWR;
    const int base = 64 * q;
    if (base >= r || NB == 0)
        return;
    const int tid = threadIdx.x;
    const int nrow = min(64, r - base);
    const int tiles = (NB + TWR - 1) / TWR;
    const int below = max(0, r - base - 64);
    int chunks = gridDim.x / tiles;
    if (chunks < 1)
        chunks = 1;
    int R = (below + chunks - 1) / chunks;
    R = (R + 255) / 256 * 256;
    if (R == 0)
        R = 256;
    chunks = below > 0 ? (below + R - 1) / R : 1;
    const int items = tiles * chunks;
    if (tid < 64)
        sD[tid] = Dinv[(int64_t)q * 64 + tid];
    int cur_tile = -1;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item / chunks, chunk = item % chunks;
        const int wb = tile * TWR;
        if (tile != cur_tile) {
            __syncthreads();
            for (int e = tid; e < 64 * TWR; e += blockDim.x) {
                const int s = e / TWR, wi = e % TWR;
                sB[e] = (s < nrow && wb + wi < NB) ? B[(int64_t)(base + s) * sb + wb + wi] : 0ull;
            }
            __syncthreads();
            rec_tables<TWR>(sB, sTB, tid);
            __syncthreads();
            for (int e = tid; e < 64 * TWR; e += blockDim.x) {
                const int s = e / TWR, wi = e % TWR;
                const u64 d = sD[s];
                u64 acc = 0;
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    acc ^= sTB[(g * 256 + (int)((d >> (8 * g)) & 255ull)) * TWR + wi];
                sX[e] = acc;
                if (chunk == 0 && s < nrow && wb + wi < NB)
                    X[(int64_t)(base + s) * sx + wb + wi] = acc;
            }
            __syncthreads();
            rec_tables<TWR>(sX, sTX, tid);
            __syncthreads();
            cur_tile = tile;
        }
        const int i0 = base + 64 + chunk * R, i1 = min(r, i0 + R);
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
            const u64 u = L[(int64_t)i * sl + q];
            u64 a0 = 0, a1 = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const ulonglong2 e2 =
                    *reinterpret_cast<const ulonglong2 *>(sTX + (g * 256 + (int)((u >> (8 * g)) & 255ull)) * TWR);
                a0 ^= e2.x;
                a1 ^= e2.y;
            }
            uint64_t *brow = B + (int64_t)i * sb + wb;
            brow[0] ^= a0;
            if (wb + 1 < NB)
                brow[1] ^= a1;
        }
    }
}

}  // namespace

namespace gf2 {

// Column split of a view of n columns: a 1024-column boundary (128-byte aligned
// views) when there is one below n/2, else a 128-column boundary (16-byte
// aligned, as the 128-bit accesses of the kernels need); 0 = no split.
static int64_t split_cols(int64_t n)
{
    int64_t n0 = ((n / 2) / 1024) * 1024;
    if (n0 == 0)
        n0 = ((n / 2) / 128) * 128;
    return n0;
}

// Depth and widest base case of the recursion tree for n columns.
static void rec_tree(int64_t n, int64_t cutoff, int d, int &maxd, int64_t &maxw)
{
    const int64_t n0 = split_cols(n);
    if (n <= cutoff || n0 == 0) {
        maxd = std::max(maxd, d);
        maxw = std::max(maxw, n);
        return;
    }
    rec_tree(n0, cutoff, d + 1, maxd, maxw);
    rec_tree(n - n0, cutoff, d + 1, maxd, maxw);
}

int pls_base(uint64_t *A, int64_t stride, int64_t m, int64_t n, int64_t *P, int64_t *Q, int *perm_out, int64_t *rank,
             char *work, const gf2_opts *opts, cudaStream_t s);

struct RecWork {
    char *elim;           // workspace of the base case
    uint64_t *scratch;    // m x W words (gathers, lower-solve output)
    int64_t scratch_stride;
    u64 *dinv;            // ((m + 63) / 64 + 1) x 64 words
    int *perms;           // (depth + 2) x m ints
    int64_t *qtmp;        // n + 1 int64
    int64_t *rank1;       // one int64 on the device
    uint64_t *bt;         // the tensor-core product's B^T (n x (W + 2) words)
    size_t bt_bytes;
    int64_t m_full;
    int depth_max;
};

static int launch_ok() { return note_cuda(cudaGetLastError()); }

// lower solve in place: B (r x nbits, pitch sb) <- L^-1 B, L = the first r rows of L (unit lower)
static int trsm_lower(const uint64_t *L, int64_t sl, uint64_t *B, int64_t sb, int r, int64_t nbits, RecWork &w,
                      cudaStream_t s)
{
    if (r <= 0 || nbits <= 0)
        return GF2_OK;
    const int NB = (int)((nbits + 63) / 64);
    const int nblk = (r + 63) / 64;
    k_diag_inv_lower<<<(nblk + 3) / 4, 128, 0, s>>>(L, sl, r, w.dinv, nblk);
    prof_launched(1);
    int rc = launch_ok();
    if (rc)
        return rc;
    const size_t smem = (size_t)(2 * 8 * 256 * TWR + 2 * 64 * TWR + 64) * sizeof(u64);
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        if ((rc = note_cuda(cudaFuncSetAttribute(k_trsm_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))))
            return rc;
        attr_done(attr_devs);
    }
    uint64_t *X = w.scratch;
    const int64_t sx = w.scratch_stride;
    for (int q = 0; q < nblk; ++q) {
        k_trsm_step<<<sm_count(), 256, smem, s>>>(B, sb, X, sx, L, sl, w.dinv, r, NB, q);
        prof_launched(1);
        if ((rc = launch_ok()))
            return rc;
    }
    return note_cuda(cudaMemcpy2DAsync(B, (size_t)sb * 8, X, (size_t)sx * 8, (size_t)NB * 8, (size_t)r,
                                       cudaMemcpyDeviceToDevice, s));
}

static int gather_rows(uint64_t *A, int64_t stride, int m, int W, const int *perm, RecWork &w, cudaStream_t s)
{
    if (m <= 0 || W <= 0)
        return GF2_OK;
    k_row_gather<<<2 * sm_count(), 256, 0, s>>>(A, stride, w.scratch, w.scratch_stride, perm, m, W);
    prof_launched(1);
    int rc = launch_ok();
    if (rc)
        return rc;
    return note_cuda(cudaMemcpy2DAsync(A, (size_t)stride * 8, w.scratch, (size_t)w.scratch_stride * 8, (size_t)W * 8,
                                       (size_t)m, cudaMemcpyDeviceToDevice, s));
}

// Recursive PLS of the view A (m x n, first column on a word boundary). P (m)
// and Q (n) are local to the view; perm_out[p] = view row now at position p.
static int pls_rec(uint64_t *A, int64_t stride, int64_t m, int64_t n, int64_t *P, int64_t *Q, int *perm_out,
                   int64_t &r_out, RecWork &w, int depth, const gf2_opts *opts, cudaStream_t s)
{
    const int64_t cutoff = opts->cutoff_cols;
    const int64_t n0 = split_cols(n);
    if (n <= cutoff || n0 == 0 || m == 0) {
        int rc = pls_base(A, stride, m, n, P, Q, perm_out, w.rank1, w.elim, opts, s);
        if (rc)
            return rc;
        int64_t rr = 0;
        if ((rc = note_cuda(cudaMemcpyAsync(&rr, w.rank1, sizeof(int64_t), cudaMemcpyDeviceToHost, s))))
            return rc;
        if ((rc = note_cuda(cudaStreamSynchronize(s))))
            return rc;
        r_out = rr;
        return GF2_OK;
    }
    int rc;
    int *perm0 = w.perms + (size_t)(2 * depth + 2) * w.m_full;
    int *perm1 = w.perms + (size_t)(2 * depth + 3) * w.m_full;
    // first recursive call on the left columns
    int64_t r0 = 0;
    if ((rc = pls_rec(A, stride, m, n0, P, Q, perm0, r0, w, depth + 1, opts, s)))
        return rc;
    uint64_t *A1 = A + n0 / 64;
    const int W1 = (int)((n - n0 + 63) / 64);
    // A1 <- P.A1
    if ((rc = gather_rows(A1, stride, (int)m, W1, perm0, w, s)))
        return rc;
    if (r0 > 0) {
        // A_NE <- L_NW^-1 A_NE
        if ((rc = trsm_lower(A, stride, A1, stride, (int)r0, n - n0, w, s)))
            return rc;
        // A_SE <- A_SE + A_SW . A_NE
        if (m > r0) {
            const int product = (opts->product == GF2_PRODUCT_TENSOR || opts->product == GF2_PRODUCT_STRASSEN_TENSOR)
                                    ? GF2_PRODUCT_TENSOR
                                    : GF2_PRODUCT_XOR;
            if (product == GF2_PRODUCT_TENSOR)
                rc = mul_tensor(A1 + r0 * stride, stride, A + r0 * stride, stride, A1, stride, m - r0, r0, n - n0, 1,
                                w.bt, w.bt_bytes, s);
            else
                rc = mul_xor(A1 + r0 * stride, stride, A + r0 * stride, stride, A1, stride, m - r0, r0, n - n0, 1,
                             opts->tile_words, opts->grid_ctas, s);
            if (rc)
                return rc;
        }
    }
    // second recursive call on A_SE
    int64_t r1 = 0;
    if ((rc = pls_rec(A1 + r0 * stride, stride, m - r0, n - n0, P + r0, Q + n0, perm1, r1, w, depth + 1, opts, s)))
        return rc;
    // A_SW <- P1.A_SW (rows r0.., columns [0, r0))
    if (r0 > 0 && r1 > 0) {
        if ((rc = gather_rows(A + r0 * stride, stride, (int)(m - r0), (int)((r0 + 63) / 64), perm1, w, s)))
            return rc;
    }
    // row order of this call, P and Q
    k_perm_compose<<<64, 256, 0, s>>>(perm0, perm1, perm_out, (int)r0, (int)m);
    k_pq_shift<<<64, 256, 0, s>>>(P, (int)r0, (int)m, Q, (int)n0, (int)n, w.qtmp);
    k_q_merge<<<64, 256, 0, s>>>(Q, w.qtmp, (int)r0, (int)r1, (int)n);
    // second call's L columns next to the first call's
    k_colshift<<<2 * sm_count(), 256, 0, s>>>(A, stride, (int)m, (int)r0, (int)n0, (int)r1);
    prof_launched(4);
    if ((rc = launch_ok()))
        return rc;
    r_out = r0 + r1;
    return GF2_OK;
}

size_t rec_workspace_bytes(int64_t m, int64_t n, int64_t cutoff)
{
    const int64_t W = (n + 63) / 64;
    const int64_t ss = ((W + 15) / 16) * 16;
    int depth = 0;
    int64_t bw = 0;
    rec_tree(n, cutoff, 0, depth, bw);
    size_t off = align_up(elim_layout(GF2_OP_PLS, m, bw).total, 256);
    off += align_up((size_t)m * ss * 8, 256);
    off += align_up((size_t)((m + 63) / 64 + 1) * 64 * 8, 256);
    off += align_up((size_t)(2 * depth + 4) * (size_t)std::max<int64_t>(m, 1) * 4, 256);
    off += align_up((size_t)(n + 1) * 8, 256);
    off += 256;
    off += align_up((size_t)std::max<int64_t>(n, 1) * (size_t)(W + 2) * 8, 256);
    return off;
}

int pls_recursive(uint64_t *A, int64_t stride, int64_t m, int64_t n, int64_t *P, int64_t *Q, int64_t *rank,
                  char *work, const gf2_opts *opts, cudaStream_t s)
{
    const int64_t cutoff = opts->cutoff_cols;
    const int64_t W = (n + 63) / 64;
    const int64_t ss = ((W + 15) / 16) * 16;
    int depth = 0;
    int64_t bw = 0;
    rec_tree(n, cutoff, 0, depth, bw);
    RecWork w{};
    size_t off = 0;
    w.elim = work + off;
    off += align_up(elim_layout(GF2_OP_PLS, m, bw).total, 256);
    w.scratch = reinterpret_cast<uint64_t *>(work + off);
    w.scratch_stride = ss;
    off += align_up((size_t)m * ss * 8, 256);
    w.dinv = reinterpret_cast<u64 *>(work + off);
    off += align_up((size_t)((m + 63) / 64 + 1) * 64 * 8, 256);
    w.perms = reinterpret_cast<int *>(work + off);
    off += align_up((size_t)(2 * depth + 4) * (size_t)std::max<int64_t>(m, 1) * 4, 256);
    w.qtmp = reinterpret_cast<int64_t *>(work + off);
    off += align_up((size_t)(n + 1) * 8, 256);
    w.rank1 = reinterpret_cast<int64_t *>(work + off);
    off += 256;
    w.bt = reinterpret_cast<uint64_t *>(work + off);
    w.bt_bytes = align_up((size_t)std::max<int64_t>(n, 1) * (size_t)(W + 2) * 8, 256);
    w.m_full = m;
    w.depth_max = depth;
    int64_t r = 0;
    int rc = pls_rec(A, stride, m, n, P, Q, w.perms, r, w, 0, opts, s);
    if (rc)
        return rc;
    k_set_rank<<<1, 32, 0, s>>>(rank, r);
    prof_launched(1);
    return launch_ok();
}

}  // namespace gf2
