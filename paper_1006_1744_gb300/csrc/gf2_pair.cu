// gf2_pair.cu -- MMPF elimination with two panels per table sweep.
//
// The one-panel pipeline (gf2_pls.cu, gf2_sweep.cu) reads and writes the whole
// trailing block once per 64-column panel. Here the pivots of panels b and
// b + 1 (b even) are found first and the trailing block is then swept once for
// both (AddRowsFromTable of Sec. 3.1 / 4.1 over 128 pivot columns), which halves
// the DRAM traffic of the sweeps and keeps their shared-memory lookups per panel
// the same:
//   * k_pivot_pair (gf2_pls.cu): the pivots of panel b, then of panel c = b + 1
//     (word b + 1 plus panel b's contribution, the look-ahead of the one-panel
//     pipeline), reading the rows' words from F, a contiguous buffer of words
//     b .. b + 3 of every row; panel b's row order is left out of perm while
//     the previous sweep still reads it;
//   * k_pair_front: the coordinates z_b of every row below panel b's pivots over
//     panel b's pivot rows O_b, and z_c of every row below both panels' pivots
//     over O_c (panel c's pivot rows after panel b), from its words b and b + 1;
//     it writes the multipliers of L into words b and b + 1, both panels'
//     updates into words b + 2 and b + 3 (the next pair's panel words), the
//     pivot rows' final words b .. b + 3 into `out`, and panel b's row order into
//     perm. 4-bit tables of the linear maps involved do all of it;
//   * k_pair_sweep: MakeTable1 for both panels on 8-word column tiles, O_c formed
//     from O_b's tables, and row ^= z_b.O_b ^ z_c.O_c on every trailing row from
//     word b + 4 on. One 128-byte line of shared memory holds entry v of both
//     panels' tables; the two rows of a quarter-warp read opposite halves of
//     their lines, so every lookup instruction is free of bank conflicts. The two
//     CTAs of a pair take the two halves of the same 128-byte lines of the same
//     rows, so each line is fetched from DRAM once.
// The next pair's pivot searches need only words b + 2 and b + 3, so they run
// while the sweep of the rest goes on.
// Every result equals the one-panel pipeline's, hence the Gaussian PLS's.
#include <climits>

#include "gf2_common.cuh"

namespace {

constexpr int NT = 512;          // threads per CTA
constexpr int TPR = 4;           // threads per row, two words each
constexpr int RPU = NT / TPR;    // rows per block (128)
constexpr int LW = 16;           // words per table line: 8 of panel b's entry, 8 of panel c's
constexpr int NLINE = 8 * 128 + 256;  // 8 half tables of 128 entries, one table of the groups' top rows

struct PairSmem {
    u64 T[NLINE * LW];
    u64 Ob[64 * 8], Oc[64 * 8];  // pivot rows of the current tile (Oc: after panel b)
    u64 zpb[64], zpc[64];        // pivot t -> its final row's coordinates (row t of L^-1)
    int prb[64], prc[64];        // physical rows of the pivots
    int xblk[64];                // blocks holding the positions panel c's search swapped from past its window
};

struct PairArgs {
    uint64_t *A;
    int64_t stride;
    const int *perm;
    const PanelState *sb, *sc;
    const u64 *zb, *zc;  // per physical row: coordinates over O_b, over O_c
    u64 *F;              // next pair's panel words: words b + 4, b + 5 of every row go to F[4 ph + 2, 3]
    uint64_t *out;
    int64_t ostride;
    int m, W, b, wlo, whi, paired;
};

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// bits 7, 15, ..., 63 of z gathered into one byte
__device__ __forceinline__ unsigned top8(u64 z)
{
    const unsigned lo = (unsigned)z, hi = (unsigned)(z >> 32);
    return ((((lo >> 7) & 0x01010101u) * 0x01020408u) >> 24) | (((((hi >> 7) & 0x01010101u) * 0x01020408u) >> 24) << 4);
}

// (z_b.O_b ^ z_c.O_c) at this thread's two words. Even rows read their panel-b half first,
// odd rows their panel-c half: in each instruction the two rows of a quarter-warp touch
// opposite halves of their lines.
__device__ __forceinline__ void lookup2(const u64 *__restrict__ T, int sub, int odd, u64 zb, u64 zc, u64 &x0, u64 &x1)
{
    const int ob = 2 * sub, oc = 8 + 2 * sub;
    u64 a0 = 0, a1 = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const int vb = (int)((zb >> (8 * g)) & 127u), vc = (int)((zc >> (8 * g)) & 127u);
        const int lb = (g * 128 + vb) * LW + ob, lc = (g * 128 + vc) * LW + oc;
        const ulonglong2 p = *reinterpret_cast<const ulonglong2 *>(T + (odd ? lc : lb));
        const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(T + (odd ? lb : lc));
        a0 ^= p.x ^ q.x;
        a1 ^= p.y ^ q.y;
    }
    {
        const int lb = (1024 + (int)top8(zb)) * LW + ob, lc = (1024 + (int)top8(zc)) * LW + oc;
        const ulonglong2 p = *reinterpret_cast<const ulonglong2 *>(T + (odd ? lc : lb));
        const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(T + (odd ? lb : lc));
        a0 ^= p.x ^ q.x;
        a1 ^= p.y ^ q.y;
    }
    x0 = a0;
    x1 = a1;
}

// word wi of z.O_b, from panel b's tables (one word, for forming O_c)
__device__ __forceinline__ u64 lookup_b1(const u64 *__restrict__ T, u64 z, int wi)
{
    u64 a = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g)
        a ^= T[(g * 128 + (int)((z >> (8 * g)) & 127u)) * LW + wi];
    return a ^ T[(1024 + (int)top8(z)) * LW + wi];
}

// MakeTable1 of one panel's 64 pivot rows O (8 words each) into half h of every line, words
// [va, vb) of the tile: group g's entry v < 128 sums rows 8 g + bit of v; the top table's
// entry v sums rows 8 g + 7 for the set bits g of v. Gray-code order, one XOR per entry.
__device__ __forceinline__ void build_tables(u64 *__restrict__ T, const u64 *__restrict__ O, int h, int va, int vb)
{
    const int tid = threadIdx.x, nw = vb - va;
    if (nw <= 0)
        return;
    for (int e = tid; e < 8 * 8 * nw; e += NT) {
        const int wi = va + e % nw, vh = (e / nw) & 7, g = e / (8 * nw);
        const u64 *Og = O + (8 * g) * 8 + wi;
        u64 base = 0;
#pragma unroll
        for (int bit = 0; bit < 3; ++bit)
            base ^= ((vh >> bit) & 1) ? Og[(4 + bit) * 8] : 0ull;
        gray16(base, Og[0], Og[8], Og[16], Og[24], T + (g * 128 + (vh << 4)) * LW + 8 * h + wi, LW);
    }
    for (int e = tid; e < 16 * nw; e += NT) {
        const int wi = va + e % nw, vh = e / nw;
        const u64 *O7 = O + 7 * 8 + wi;  // row 8 g + 7 at O7[64 g]
        u64 base = 0;
#pragma unroll
        for (int bit = 0; bit < 4; ++bit)
            base ^= ((vh >> bit) & 1) ? O7[64 * (4 + bit)] : 0ull;
        gray16(base, O7[0], O7[64], O7[128], O7[192], T + (1024 + (vh << 4)) * LW + 8 * h + wi, LW);
    }
}

struct PairRows {
    int R0, R1, R2;      // panel b's pivots at [R0, R1), panel c's at [R1, R2), trailing rows from R2
    int nwin, nx;        // panel c's window and swaps past it
    int plain_from;      // positions from here on are perm[p], except panel c's nx swapped ones
};

// Pipelined sweep of blocks [ja, jb) of trailing rows given by perm alone. Per thread: the
// physical row 5 blocks ahead, an L2 prefetch of its tile 4 ahead, its coordinates 3 ahead,
// its two words 2 ahead.
__device__ __forceinline__ void pair_plain(const PairArgs &a, const PairSmem &S, const PairRows &R, int sub, int rg,
                                           int odd, int w0, bool v0, bool v1, int ja, int jb, bool check, bool &nzw)
{
    const bool cz = check;  // the zero-tail test proper
    const int pbase = R.R0 + rg, plast = a.m - 1;
    const bool idle = !v0 && !v1, both = v0 && v1;
    // words b + 4 and b + 5 also go to the next pair's contiguous buffer (its front and pivot
    // searches read them there), so that thread reads and writes every row
    const bool fw = v0 && w0 == a.b + 4;
    check = check || fw;
    auto pos = [&](int jj) { return min(max(pbase + jj * RPU, 0), plast); };
    int ph0 = 0, ph1 = 0, ph2 = 0, ph3 = 0, ph4 = 0, ph5 = 0;
    u64 zb0 = 0, zb1 = 0, zb2 = 0, zb3 = 0, zc0 = 0, zc1 = 0, zc2 = 0, zc3 = 0;
    u64 d00 = 0, d01 = 0, d10 = 0, d11 = 0, d20 = 0, d21 = 0;
    for (int j = ja - 5; j < jb; ++j) {
        ph5 = a.perm[pos(j + 5)];
        if (!idle)
            prefetch_l2(a.A + (int64_t)ph4 * a.stride + w0);
        zb3 = a.zb[ph3];
        zc3 = a.zc[ph3];
        if (!idle && ((zb2 | zc2) != 0 || check)) {
            const uint64_t *src = a.A + (int64_t)ph2 * a.stride + w0;
            if (both) {
                const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(src));
                d20 = v.x;
                d21 = v.y;
            } else {
                d20 = v0 ? src[0] : 0ull;
                d21 = v1 ? src[1] : 0ull;
            }
        } else {
            d20 = d21 = 0;
        }
        if (j >= ja) {
            u64 x0, x1;
            lookup2(S.T, sub, odd, zb0, zc0, x0, x1);
            const int p = pbase + j * RPU;
            if (p < a.m && !idle && ((zb0 | zc0) != 0 || check)) {
                const u64 n0 = d00 ^ x0, n1 = d01 ^ x1;
                if (cz)
                    nzw = nzw || (v0 && n0 != 0) || (v1 && n1 != 0);
                if (fw) {
                    a.F[4 * (int64_t)ph0 + 2] = n0;
                    if (v1)
                        a.F[4 * (int64_t)ph0 + 3] = n1;
                }
                if ((zb0 | zc0) != 0) {
                    uint64_t *dst = a.A + (int64_t)ph0 * a.stride + w0;
                    if (both) {
                        ulonglong2 v;
                        v.x = n0;
                        v.y = n1;
                        __stcs(reinterpret_cast<ulonglong2 *>(dst), v);
                    } else {
                        if (v0)
                            dst[0] = n0;
                        if (v1)
                            dst[1] = n1;
                    }
                }
            }
        }
        ph0 = ph1;
        ph1 = ph2;
        ph2 = ph3;
        ph3 = ph4;
        ph4 = ph5;
        zb0 = zb1;
        zb1 = zb2;
        zb2 = zb3;
        zc0 = zc1;
        zc1 = zc2;
        zc2 = zc3;
        d00 = d10;
        d01 = d11;
        d10 = d20;
        d11 = d21;
    }
}

// One block of any rows: the pivot rows of both panels (their final rows go to `out`), the
// window rows of panel c and rows it swapped from past its window.
__device__ __forceinline__ void pair_general(const PairArgs &a, const PairSmem &S, const PairRows &R, int sub, int rg,
                                             int odd, int w0, bool v0, bool v1, int j, bool check, bool &nzw)
{
    const int p = R.R0 + j * RPU + rg;
    int kind = 0, ph = 0;  // 0 none, 1 pivot of b, 2 pivot of c, 3 trailing
    u64 zb = 0, zc = 0;
    if (p < a.m) {
        if (p < R.R1) {
            kind = 1;
            zb = S.zpb[p - R.R0];
        } else if (p < R.R2) {
            kind = 2;
            zc = S.zpc[p - R.R1];
        } else {
            kind = 3;
            ph = trailing_row(a.perm, a.sc, R.R1, R.nwin, R.nx, p);
            zb = a.zb[ph];
            zc = a.zc[ph];
        }
    }
    u64 x0, x1;
    lookup2(S.T, sub, odd, zb, zc, x0, x1);
    if (kind == 3) {
        uint64_t *row = a.A + (int64_t)ph * a.stride + w0;
        const u64 n0 = v0 ? row[0] ^ x0 : 0ull, n1 = v1 ? row[1] ^ x1 : 0ull;
        if (check)
            nzw = nzw || n0 != 0 || n1 != 0;
        if (v0)
            row[0] = n0;
        if (v1)
            row[1] = n1;
        if (v0 && w0 == a.b + 4) {
            a.F[4 * (int64_t)ph + 2] = n0;
            if (v1)
                a.F[4 * (int64_t)ph + 3] = n1;
        }
    } else if (kind && a.out) {
        uint64_t *row = a.out + (int64_t)p * a.ostride + w0;
        if (v0)
            row[0] = x0;
        if (v1)
            row[1] = x1;
    }
}

__global__ void __launch_bounds__(NT, 1) k_pair_sweep(PairArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    PairSmem &S = *reinterpret_cast<PairSmem *>(smraw);
    const int tid = threadIdx.x;
    const PanelState *__restrict__ sb = a.sb, *__restrict__ sc = a.sc;
    PairRows R;
    R.R0 = sb->r_cur;
    R.R1 = R.R0 + sb->kbar;
    R.R2 = R.R1 + sc->kbar;
    R.nwin = sc->nwin;
    R.nx = sc->nx;
    R.plain_from = R.R1 + max(sc->kbar, R.nwin);
    const int kb = sb->kbar, kc = sc->kbar;
    // no pivot in panel c: look for a nonzero word right of it in any trailing row (none means
    // no later panel has a pivot), unless that is known already
    const bool check = kc == 0 && !sc->zero_tail;
    bool nzw = false;
    const int lo = max(a.wlo, a.b + 2), hi = min(a.whi, a.W);
    const int M = a.m - R.R0;
    if ((kb || kc || check) && M > 0 && lo < hi) {
        if (tid < 64) {
            S.prb[tid] = tid < kb ? sb->prow[tid] : 0;
            S.prc[tid] = tid < kc ? sc->prow[tid] : 0;
            S.zpb[tid] = tid < kb ? sb->zpiv[tid] : 0ull;
            S.zpc[tid] = tid < kc ? sc->zpiv[tid] : 0ull;
            S.xblk[tid] = tid < R.nx ? (sc->xpos[tid] - R.R0) / RPU : INT_MAX;
        }
        const int nblk = (M + RPU - 1) / RPU;
        const int plain_blk = min(nblk, (R.plain_from - R.R0 + RPU - 1) / RPU);
        // units: (tile, block) in tile-major order; paired: (128-byte line, block), the two CTAs of
        // a pair taking the line's two tiles
        const int half = a.paired ? (int)(blockIdx.x & 1) : 0;
        const int team = a.paired ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
        const int nteam = a.paired ? (int)(gridDim.x >> 1) : (int)gridDim.x;
        const int c0 = a.paired ? (lo >> 4) : (lo >> 3), c1 = a.paired ? ((hi + 15) >> 4) : ((hi + 7) >> 3);
        const long long total = (long long)(c1 - c0) * nblk;
        const long long q_lo = total * team / nteam, q_hi = total * (team + 1) / nteam;
        const int sub = tid & (TPR - 1), rg = tid / TPR, odd = (tid >> 2) & 1;
        for (long long q = q_lo; q < q_hi;) {
            const int col = (int)(q / nblk);
            const long long q_end = min(q_hi, (long long)(col + 1) * nblk);
            const int blk0 = (int)(q - (long long)col * nblk), blk1 = (int)(q_end - (long long)col * nblk);
            q = q_end;
            const int tile = a.paired ? 2 * (c0 + col) + half : c0 + col;
            const int tb = 8 * tile;
            const int va = max(lo, tb) - tb, vb = min(hi, tb + 8) - tb;
            if (va >= vb)
                continue;  // CTA-uniform: this half of the line holds no word to sweep
            // ---- tables of this tile: panel b's, O_c from them, panel c's ----
            __syncthreads();
            for (int e = tid; e < 64 * 8; e += NT) {
                const int t = e >> 3, wi = e & 7;
                const bool in = wi >= va && wi < vb;
                S.Ob[e] = in && t < kb ? a.A[(int64_t)S.prb[t] * a.stride + tb + wi] : 0ull;
                S.Oc[e] = in && t < kc ? a.A[(int64_t)S.prc[t] * a.stride + tb + wi] : 0ull;
            }
            __syncthreads();
            build_tables(S.T, S.Ob, 0, va, vb);
            __syncthreads();
            for (int e = tid; e < 64 * 8; e += NT) {
                const int t = e >> 3, wi = e & 7;
                if (t < kc && wi >= va && wi < vb)
                    S.Oc[e] ^= lookup_b1(S.T, a.zb[S.prc[t]], wi);
            }
            __syncthreads();
            build_tables(S.T, S.Oc, 1, va, vb);
            __syncthreads();
            const int w0 = tb + 2 * sub;
            const bool v0 = w0 >= lo && w0 < hi, v1 = w0 + 1 >= lo && w0 + 1 < hi;
            for (int j = blk0; j < min(blk1, plain_blk); ++j)
                pair_general(a, S, R, sub, rg, odd, w0, v0, v1, j, check, nzw);
            // runs of plain blocks through the pipeline, each block holding a swapped position alone
            for (int ja = max(blk0, plain_blk); ja < blk1;) {
                int jx = blk1;
                for (int x = 0; x < R.nx; ++x)
                    jx = S.xblk[x] >= ja && S.xblk[x] < jx ? S.xblk[x] : jx;
                if (ja < jx)
                    pair_plain(a, S, R, sub, rg, odd, w0, v0, v1, ja, jx, check, nzw);
                if (jx < blk1)
                    pair_general(a, S, R, sub, rg, odd, w0, v0, v1, jx, check, nzw);
                ja = jx + 1;
            }
        }
    }
    if (check && __syncthreads_or(nzw) && tid == 0) {
        atomicExch(const_cast<int *>(&sb->nz), 1);
        atomicExch(const_cast<int *>(&sc->nz), 1);
    }
}

// ---------------------------------------------------------------------------
// The front of a pair: every row's coordinates, the multipliers of L in words b and b + 1, and
// both panels' updates of words b + 2 and b + 3 (the next pair's panel words), all from 4-bit
// tables (16 positions x 16 values) of linear maps of a row's panel words:
//   from word b:                   Zb -> z_b, Xb -> panel b's multipliers (z_b.X_b, X_t = pivot
//                                  t's multipliers plus its own bit), Cb, E2b, E3b -> z_b.O_b at
//                                  words b + 1, b + 2, b + 3;
//   from word b + 1 after panel b: Zc -> z_c, Xc -> panel c's multipliers, E2c, E3c -> z_c.O_c at
//                                  words b + 2, b + 3.
// ---------------------------------------------------------------------------
constexpr int NMAP = 9;
enum { M_ZB, M_XB, M_CB, M_E2B, M_E3B, M_ZC, M_XC, M_E2C, M_E3C };

struct FrontSmem {
    u64 tab[NMAP][256];  // 4-bit tables of the maps (16 positions x 16 values): one 128-byte bank row per position
    u64 img[NMAP][64];   // image of each bit of the panel word
    u64 Xb[64], Xc[64];
    u64 Ob[3][64];       // panel b's pivot rows at words b + 1, b + 2, b + 3
    u64 Oc[3][64];       // panel c's pivot rows: word b (raw), then words b + 2, b + 3 after panel b
    u64 zmb[64], zmc[64];  // the panels' zmaps
    u64 ztc[64];           // panel c's pivot rows: coordinates over panel b's pivot rows
    int prb[64], prc[64];  // physical rows of the pivots
    // 4-bit tables (16 positions x 16 values) of the sums of rows of Xb, Ob[0..2], zmb, Xc, Oc[1..2]
    u64 nib[8][256];
    int sc_[6];          // r_cur, kbar of panel b, kbar of panel c, window and swaps of b and c
};
enum { N_XB, N_OB0, N_OB1, N_OB2, N_ZMB, N_XC, N_OC1, N_OC2 };


// sum of the 64 rows src[0..63] selected by the set bits of z, through its 4-bit table (sixteen
// lookups, two XOR chains)
__device__ __forceinline__ u64 select_sum(u64 z, const u64 *__restrict__ nib)
{
    u64 a0 = 0, a1 = 0;
#pragma unroll
    for (int q = 0; q < 16; q += 2) {
        a0 ^= nib[q * 16 + (int)((z >> (4 * q)) & 15u)];
        a1 ^= nib[(q + 1) * 16 + (int)((z >> (4 * q + 4)) & 15u)];
    }
    return a0 ^ a1;
}

// the image of a panel word w under a linear map, through the map's 4-bit table: the sixteen
// entries of a position fill one 128-byte row of banks, so every lookup is free of bank conflicts
__device__ __forceinline__ u64 select_sum_w(const u64 *__restrict__ nib, u64 w) { return select_sum(w, nib); }

// 4-bit tables of 64 rows: entry (q, v) = the sum of rows 4 q + j for the set bits j of v. Lane l
// of a warp writes entries l and l + 32 of a table (consecutive lanes, consecutive entries).
__device__ __forceinline__ void build_nib(u64 *__restrict__ nib, const u64 *__restrict__ src, int e)
{
    const int q = e >> 4, v = e & 15;
    u64 a = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        a ^= ((v >> j) & 1) ? src[4 * q + j] : 0ull;
    nib[e] = a;
}

// 4-bit tables of the maps [m0, m1), from their images of the 64 bits
__device__ __forceinline__ void build_bytetabs(FrontSmem &S, int m0, int m1)
{
    for (int e = threadIdx.x; e < (m1 - m0) * 256; e += NT)
        build_nib(S.tab[m0 + (e >> 8)], S.img[m0 + (e >> 8)], e & 255);
}

// Physical row at trailing position p >= R2 of a pair: panel c's order, else panel b's, else perm
// (the positions panel b changed are read through sb: this kernel writes them into perm).
__device__ __forceinline__ int pair_row(const int *__restrict__ perm, const PanelState *__restrict__ sb,
                                        const PanelState *__restrict__ sc, int R0, int R1, int nwb, int nxb, int nwc,
                                        int nxc, int p)
{
    if (sc) {
        if (p < R1 + nwc)
            return sc->wperm[p - R1];
        for (int x = 0; x < nxc; ++x)
            if (sc->xpos[x] == p)
                return sc->xval[x];
    }
    if (p < R0 + nwb)
        return sb->wperm[p - R0];
    for (int x = 0; x < nxb; ++x)
        if (sb->xpos[x] == p)
            return sb->xval[x];
    return perm[p];
}

__global__ void __launch_bounds__(NT, 1)
k_pair_front(uint64_t *__restrict__ A, int64_t stride, int *__restrict__ perm, const PanelState *__restrict__ sb,
             const PanelState *__restrict__ sc, u64 *__restrict__ zb, u64 *__restrict__ zc,
             const u64 *__restrict__ Fc, u64 *__restrict__ Fn, uint64_t *__restrict__ out, int64_t ostride, int m,
             int W, int b)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    FrontSmem &S = *reinterpret_cast<FrontSmem *>(smraw);
    const int tid = threadIdx.x;
    if (tid < 6)
        S.sc_[tid] = tid == 0 ? sb->r_cur : tid == 1 ? sb->kbar : tid == 2 ? (sc ? sc->kbar : 0)
                   : tid == 3 ? sb->nwin : tid == 4 ? sb->nx : (sc ? sc->nwin * 256 + sc->nx : 0);
    if (tid >= 64 && tid < 128)
        S.zmb[tid - 64] = sb->zmap[tid - 64];
    if (tid >= 128 && tid < 192)
        S.zmc[tid - 128] = sc ? sc->zmap[tid - 128] : 0ull;
    __syncthreads();
    const int kb = S.sc_[1], kc = S.sc_[2];
    const int R0 = S.sc_[0], R1 = R0 + kb, R2 = R1 + kc;
    const int nwb = S.sc_[3], nxb = S.sc_[4], nwc = S.sc_[5] >> 8, nxc = S.sc_[5] & 255;
    const bool has1 = b + 1 < W, has2 = b + 2 < W, has3 = b + 3 < W;
    // consecutive positions go to different CTAs, so the pivot rows (the first positions, whose
    // rows cost most here) spread over the grid
    const int g = tid * gridDim.x + blockIdx.x, gs = gridDim.x * NT;
    // a CTA past the last row only takes its share of the row-order update below
    const bool rows = R0 + (int)blockIdx.x < m;
    const bool pivots = rows && (kb > 0 || kc > 0);
    // every word this launch reads was written before it started (the previous pair's front
    // and sweep precede it on the stream): one round of loads, then the tables in six phases
    int p = R0 + g, ph = -1;
    u64 w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    if (pivots && p >= R1 && p < m) {
        ph = p < R2 ? sc->prow[p - R1] : pair_row(perm, sb, sc, R0, R1, nwb, nxb, nwc, nxc, p);
        const ulonglong2 lo = *reinterpret_cast<const ulonglong2 *>(Fc + 4 * (int64_t)ph);
        w0 = lo.x;
        w1 = lo.y;
        if (p >= R2) {
            const ulonglong2 hi = *reinterpret_cast<const ulonglong2 *>(Fc + 4 * (int64_t)ph + 2);
            w2 = hi.x;
            w3 = hi.y;
        }
    }
    if (pivots) {
        if (tid < 64) {
            // the pivot rows' words b .. b + 3 (panel c's as they were before panel b)
            const int t = tid;
            S.prb[t] = t < kb ? sb->prow[t] : 0;
            S.prc[t] = t < kc ? sc->prow[t] : 0;
            S.Xb[t] = t < kb ? sb->newblk[t] & sb->J & lowmask(sb->pcol[t] + 1) : 0ull;
            S.Xc[t] = t < kc ? sc->newblk[t] & sc->J & lowmask(sc->pcol[t] + 1) : 0ull;
            const u64 *fb = Fc + 4 * (int64_t)S.prb[t], *fc = Fc + 4 * (int64_t)S.prc[t];
            S.Ob[0][t] = t < kb && has1 ? fb[1] : 0ull;
            S.Ob[1][t] = t < kb && has2 ? fb[2] : 0ull;
            S.Ob[2][t] = t < kb && has3 ? fb[3] : 0ull;
            S.Oc[0][t] = t < kc ? fc[0] : 0ull;
            S.Oc[1][t] = t < kc && has2 ? fc[2] : 0ull;
            S.Oc[2][t] = t < kc && has3 ? fc[3] : 0ull;
        }
        __syncthreads();
        for (int e = tid; e < 6 * 256; e += NT) {
            const int k = e >> 8;  // Xb, Ob0, zmb, Xc, Ob1, Ob2
            const int slot = k == 0 ? N_XB : k == 1 ? N_OB0 : k == 2 ? N_ZMB : k == 3 ? N_XC : k == 4 ? N_OB1 : N_OB2;
            const u64 *src = k == 0 ? S.Xb : k == 1 ? S.Ob[0] : k == 2 ? S.zmb : k == 3 ? S.Xc : S.Ob[k - 3];
            build_nib(S.nib[slot], src, e & 255);
        }
        __syncthreads();
        if (tid < 3 * 64) {
            // panel b's maps of word b: z_b, multipliers, contribution to word b + 1
            const int mp = tid >> 6, i = tid & 63;
            const u64 zm = S.zmb[i];
            S.img[mp][i] = mp == 0 ? zm : select_sum(zm, S.nib[mp == 1 ? N_XB : N_OB0]);
        } else if (tid < 5 * 64) {
            // panel c's maps of word b + 1 after panel b: z_c, multipliers
            const int mp = (tid >> 6) - 3, i = tid & 63;
            const u64 zm = S.zmc[i];
            S.img[M_ZC + mp][i] = mp == 0 ? zm : select_sum(zm, S.nib[N_XC]);
        } else if (tid < 6 * 64) {
            // panel c's pivot rows: their coordinates over panel b's pivot rows, and their words
            // b + 2, b + 3 after panel b
            const int t = tid - 5 * 64;
            const u64 z = t < kc ? select_sum(S.Oc[0][t], S.nib[N_ZMB]) : 0ull;
            S.ztc[t] = z;
            if (t < kc) {
                S.Oc[1][t] ^= select_sum(z, S.nib[N_OB1]);
                S.Oc[2][t] ^= select_sum(z, S.nib[N_OB2]);
            }
        } else {
            // panel b's contributions to words b + 2, b + 3
            const int mp = (tid >> 6) - 6, i = tid & 63;
            S.img[M_E2B + mp][i] = select_sum(S.zmb[i], S.nib[N_OB1 + mp]);
        }
        __syncthreads();
        build_bytetabs(S, M_ZB, M_E3B + 1);
        build_bytetabs(S, M_ZC, M_XC + 1);
        for (int e = tid; e < 2 * 256; e += NT)
            build_nib(S.nib[N_OC1 + (e >> 8)], S.Oc[1 + (e >> 8)], e & 255);
        __syncthreads();
        if (tid < 2 * 64) {
            // panel c's contributions to words b + 2, b + 3
            const int mp = tid >> 6, i = tid & 63;
            S.img[M_E2C + mp][i] = select_sum(S.zmc[i], S.nib[N_OC1 + mp]);
        }
        __syncthreads();
        build_bytetabs(S, M_E2C, M_E3C + 1);
        __syncthreads();
    }
    // panel b's row order into perm (the rows below read it through sb)
    if (sc) {
        for (int i = g; i < nwb; i += gs)
            perm[R0 + i] = sb->wperm[i];
        for (int x = g; x < nxb; x += gs)
            perm[sb->xpos[x]] = sb->xval[x];
    }
    if (!rows)
        return;
    if (!pivots) {
        // no pivot: words b, b + 1 of every row below are zero; words b + 2, b + 3 pass to the next
        // pair unchanged (zero too once the tail is known to be zero)
        const bool zt = sb->zero_tail;
        for (int q = R0 + g; q < m; q += gs) {
            const int r = pair_row(perm, sb, sc, R0, R1, nwb, nxb, nwc, nxc, q);
            uint64_t *row = A + (int64_t)r * stride + b;
            row[0] = 0ull;
            if (sc)
                row[1] = 0ull;
            if (sc && has2) {
                Fn[4 * (int64_t)r] = zt ? 0ull : Fc[4 * (int64_t)r + 2];
                if (has3)
                    Fn[4 * (int64_t)r + 1] = zt ? 0ull : Fc[4 * (int64_t)r + 3];
            }
        }
        return;
    }
    for (; p < m; p += gs) {
        if (ph < 0 && p >= R1) {
            // a later row of this thread (more rows than threads)
            ph = p < R2 ? sc->prow[p - R1] : pair_row(perm, sb, sc, R0, R1, nwb, nxb, nwc, nxc, p);
            const u64 *f = Fc + 4 * (int64_t)ph;
            w0 = f[0];
            w1 = f[1];
            w2 = f[2];
            w3 = f[3];
        }
        if (p < R1) {
            // pivot of panel b: its final words b .. b + 3
            const int t = p - R0;
            if (out) {
                uint64_t *o = out + (int64_t)p * ostride + b;
                const u64 zt = sb->zpiv[t];
                o[0] = sb->newblk[t];
                if (has1)
                    o[1] = select_sum(zt, S.nib[N_OB0]);
                if (has2)
                    o[2] = select_sum(zt, S.nib[N_OB1]);
                if (has3)
                    o[3] = select_sum(zt, S.nib[N_OB2]);
            }
        } else if (p < R2) {
            // pivot of panel c: panel b's multipliers in A, its final words b + 1 .. b + 3
            const int t = p - R1;
            uint64_t *row = A + (int64_t)ph * stride + b;
            zb[ph] = select_sum_w(S.tab[M_ZB], w0);
            row[0] = select_sum_w(S.tab[M_XB], w0);
            if (out) {
                uint64_t *o = out + (int64_t)p * ostride + b;
                const u64 zt = sc->zpiv[t];
                o[1] = sc->newblk[t];
                if (has2)
                    o[2] = select_sum(zt, S.nib[N_OC1]);
                if (has3)
                    o[3] = select_sum(zt, S.nib[N_OC2]);
            }
        } else {
            uint64_t *row = A + (int64_t)ph * stride + b;
            const u64 zbv = select_sum_w(S.tab[M_ZB], w0);
            u64 n2 = w2 ^ select_sum_w(S.tab[M_E2B], w0), n3 = w3 ^ select_sum_w(S.tab[M_E3B], w0);
            row[0] = select_sum_w(S.tab[M_XB], w0);
            zb[ph] = zbv;
            if (sc) {
                const u64 v1 = w1 ^ select_sum_w(S.tab[M_CB], w0);
                zc[ph] = select_sum_w(S.tab[M_ZC], v1);
                row[1] = select_sum_w(S.tab[M_XC], v1);
                n2 ^= select_sum_w(S.tab[M_E2C], v1);
                n3 ^= select_sum_w(S.tab[M_E3C], v1);
            }
            // words b + 2, b + 3 after both panels: the next pair's panel words, read by its pivot
            // searches and its front from here (A gets them as multipliers then)
            if (has2)
                Fn[4 * (int64_t)ph] = n2;
            if (has3)
                Fn[4 * (int64_t)ph + 1] = n3;
        }
        ph = -1;
    }
}

// words 0 .. 3 of every row into the first pair's buffer
__global__ void k_pair_init(const uint64_t *__restrict__ A, int64_t stride, u64 *__restrict__ F, int m, int W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m)
        for (int k = 0; k < 4; ++k)
            F[4 * (int64_t)i + k] = k < W ? A[(int64_t)i * stride + k] : 0ull;
}

constexpr size_t PAIR_SMEM = sizeof(PairSmem);
constexpr size_t FRONT_SMEM = sizeof(FrontSmem);

}  // namespace

namespace gf2 {

int launch_pivot_pair(const Elim &e, int b, const u64 *wsrc, int64_t wstride, const u64 *side_prev,
                      int64_t side_stride, const PanelState *st_prev, PanelState *st, bool defer, bool programmatic,
                      cudaStream_t s);

// the side region of the workspace: coordinates over panel b's and panel c's pivot rows (m each),
// then two buffers of words b .. b + 3 of every row (4 m each), alternating with the pair
static u64 *pair_zb(const Elim &e) { return e.side; }
static u64 *pair_zc(const Elim &e) { return e.side + e.m; }
static u64 *pair_F(const Elim &e, int b) { return e.side + 2 * e.m + (size_t)(((b >> 1) & 1) * 4) * e.m; }
int init_states(const Elim &e, int nstates);

static int sweep_pair(const Elim &e, int b, int wlo, int whi, bool paired, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        cudaError_t err = cudaFuncSetAttribute(k_pair_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PAIR_SMEM);
        if (err != cudaSuccess)
            return note_cuda(err);
        attr_done(attr_devs);
    }
    PairArgs a{};
    a.A = e.A;
    a.stride = e.stride;
    a.perm = e.perm;
    a.sb = e.st + (b & 3);
    a.sc = e.st + ((b + 1) & 3);
    a.zb = pair_zb(e);
    a.zc = pair_zc(e);
    a.F = pair_F(e, b + 2);
    a.out = e.out;
    a.ostride = e.ostride;
    a.m = (int)e.m;
    a.W = (int)e.W;
    a.b = b;
    a.wlo = wlo;
    a.whi = whi;
    a.paired = paired ? 1 : 0;
    const int nsm = sm_count();
    // one SM left to the pivot search that runs meanwhile; an even count for pairs
    int grid = e.grid > 0 ? e.grid : (nsm > 1 ? nsm - 1 : 1);
    if (paired)
        grid = grid >= 2 ? grid & ~1 : 2;
    const int tok = prof_begin(s);
    k_pair_sweep<<<grid, NT, PAIR_SMEM, s>>>(a);
    prof_end(s, GF2_PROF_SWEEP, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

static int pair_front(const Elim &e, int b, bool has_c, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        cudaError_t err =
            cudaFuncSetAttribute(k_pair_front, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FRONT_SMEM);
        if (err != cudaSuccess)
            return note_cuda(err);
        attr_done(attr_devs);
    }
    const int nsm = sm_count();
    const int64_t need = (e.m + NT - 1) / NT;
    const int grid = (int)(need < nsm ? (need > 0 ? need : 1) : nsm);
    const int tok = prof_begin(s);
    k_pair_front<<<grid, NT, FRONT_SMEM, s>>>(e.A, e.stride, e.perm, e.st + (b & 3),
                                              has_c ? e.st + ((b + 1) & 3) : nullptr, pair_zb(e), pair_zc(e),
                                              pair_F(e, b), pair_F(e, b + 2), e.out, e.ostride, (int)e.m, (int)e.W, b);
    prof_end(s, GF2_PROF_COORDS, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

// Two panels per sweep (see the top of this file). Streams: pivot searches on e.s, the
// coordinates and sweeps on aux.side. Panel b uses state slot b & 3: the pivot search of
// panel b + 2 runs while the sweep of panels b, b + 1 still reads their slots.
int elim_run_pair(const Elim &e, const ElimAux &aux)
{
    int rc;
    if ((rc = init_states(e, 4)))
        return rc;
    const int W = (int)e.W;
    if (W == 0)
        return GF2_OK;
    k_pair_init<<<(int)((e.m + 255) / 256), 256, 0, e.s>>>(e.A, e.stride, pair_F(e, 0), (int)e.m, W);
    prof_launched(1);
    if ((rc = note_cuda(cudaGetLastError())))
        return rc;
    cudaStream_t s = e.s, t = aux.side;
    cudaEvent_t ev_piv = aux.ev[0], ev_edge = aux.ev[1], ev_done = aux.ev[2];
    for (int b = 0; b < W; b += 2) {
        const bool has_c = b + 1 < W;
        PanelState *sb = e.st + (b & 3), *sc = e.st + ((b + 1) & 3);
        const PanelState *sp = e.st + ((b + 3) & 3);  // panel b - 1 (slot 3, initialised, for b = 0)
        if (b >= 2 && (rc = note_cuda(cudaStreamWaitEvent(s, ev_edge, 0))))
            return rc;
        const u64 *F = pair_F(e, b);  // words b .. b + 3 of every row
        if ((rc = launch_pivot_pair(e, b, F, 4, nullptr, 0, sp, sb, false, false, s)))
            return rc;
        if (has_c && (rc = launch_pivot_pair(e, b + 1, F + 1, 4, F, 4, sb, sc, true, true, s)))
            return rc;
        if ((rc = note_cuda(cudaEventRecord(ev_piv, s))) || (rc = note_cuda(cudaStreamWaitEvent(t, ev_piv, 0))))
            return rc;
        // the front: coordinates, multipliers, words b + 2 and b + 3 (what the next pair's
        // pivot searches read), then the rest of the trailing block
        if ((rc = pair_front(e, b, has_c, t)) || (rc = note_cuda(cudaEventRecord(ev_edge, t))))
            return rc;
        if (has_c && b + 4 < W && (rc = sweep_pair(e, b, b + 4, W, true, t)))
            return rc;
    }
    // the last panel's row order once every sweep and coordinate step is done
    if ((rc = note_cuda(cudaEventRecord(ev_done, t))) || (rc = note_cuda(cudaStreamWaitEvent(s, ev_done, 0))))
        return rc;
    return apply_final_order(e);
}

}  // namespace gf2
