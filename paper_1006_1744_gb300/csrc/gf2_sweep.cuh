// gf2_sweep.cuh -- device code of the 16-word table sweep (see gf2_sweep.cu), shared by the
// sweep kernels and the persistent batched elimination (gf2_pls.cu). Everything here has
// internal linkage: each translation unit that includes it gets its own copy.
#pragma once
#include <climits>

#include "gf2_common.cuh"

namespace {

constexpr int TW = 16;         // words per column tile (one 128-byte line of a row)
constexpr int NT = 512;        // threads per CTA
constexpr int TPR = 4;         // threads per row, four words each
constexpr int RPU = NT / TPR;  // rows per block (128)

// The sweep runs on NTH threads starting at thread TOFF of the CTA: the whole CTA (NTH = NT,
// TOFF = 0, CTA barriers) or, in the persistent batched elimination, the warps after the pivot
// search's, which synchronise on named barrier 2 of their own.
template <int NTH, int TOFF>
__device__ __forceinline__ void sweep_sync()
{
    if (NTH == NT && TOFF == 0)
        __syncthreads();
    else
        asm volatile("bar.sync 2, %0;" ::"n"(NTH) : "memory");
}

template <int NTH, int TOFF>
__device__ __forceinline__ bool sweep_sync_or(bool v)
{
    if (NTH == NT && TOFF == 0)
        return __syncthreads_or(v) != 0;
    unsigned r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((unsigned)v), "n"(NTH)
                 : "memory");
    return r != 0;
}

struct SweepSmem {
    u64 T[8 * 128 * TW];  // half tables: group g, entry v < 128 at (g * 128 + v) * TW
    u64 U[256 * TW];      // sums of the rows 8 g + 7 selected by the 8 top bits
    u64 Z[256 * 16];      // panel byte v at byte position q -> coordinates over O, two copies: v * 16 + copy * 8 + q
    u64 O[64 * TW];       // rows of the tables for the current tile
    u64 map[64];          // zmap of the panel
    int prow[64];         // physical rows of the pivots
    int xblk[64];         // blocks holding the positions the pivot search swapped from past its window
};

// row codes: >= 0 trailing row (physical index), -1 none, -2 row above (MODE 1, kept in
// `out` at its position), <= -3 pivot row -3 - code
constexpr int CODE_NONE = -1;
constexpr int CODE_UP = -2;

struct Cfg {
    uint64_t *A;
    int64_t stride;
    const u64 *side_cur;
    u64 *side_nxt;
    const int *perm;
    const PanelState *st;
    uint64_t *out;
    int64_t ostride;
    const u64 *ups_cur;  // reduced form: panel word b of the rows above, by position (read only here)
    u64 *ups_nxt;        // reduced form: their word b + 1 after this panel, for the next sweep
    int m, W, b, r, kbar, nwin, nx, row0;
};

struct Lanes {
    int sub;       // which 4 words of the tile row
    int rg;        // row of the block
    int odd;       // second row of its quarter-warp: reads its halves in the other order
    int zcopy;     // copy of Z this row's lanes read (rows of a half-warp alternate)
    const u64 *Tb; // S.T + 4 * sub
    const u64 *Ub; // S.U + 4 * sub
};

// Coordinates over O of a row with panel word wv: this thread's two bytes, then the sum over
// the row's four threads. The rows of a half-warp use two copies of Z and take their two bytes
// in opposite order, so that the 16 lanes of each lookup hit 16 different bank pairs.
__device__ __forceinline__ u64 coords(const SweepSmem &S, const Lanes &L, u64 wv)
{
    const int q1 = 2 * L.sub + L.odd, q2 = 2 * L.sub + 1 - L.odd;
    const unsigned v1 = (unsigned)(wv >> (8 * q1)) & 255u, v2 = (unsigned)(wv >> (8 * q2)) & 255u;
    const int zb = L.zcopy * 8;
    u64 z = S.Z[v1 * 16 + zb + q1] ^ S.Z[v2 * 16 + zb + q2];
    z ^= __shfl_xor_sync(GF2_FULL, z, 1);
    z ^= __shfl_xor_sync(GF2_FULL, z, 2);
    return z;
}

// x[0..3] = (z.O) at this thread's 4 words of the tile. KB = 8: 8 half-table rows and 1 top-bit
// row; KB = 4: 16 rows of 16-entry tables.
template <int KB>
__device__ __forceinline__ void lookup(const Lanes &L, u64 z, u64 (&x)[4])
{
    const int h1 = L.odd ? 2 : 0, h2 = 2 - h1;
    const unsigned zl = (unsigned)z, zh = (unsigned)(z >> 32);
    u64 p0 = 0, p1 = 0, q0 = 0, q1 = 0;
    if (KB == 4) {
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            const unsigned v = ((g < 8 ? zl : zh) >> (4 * (g & 7))) & 15u;
            const u64 *e = L.Tb + (g * 16 + (int)v) * TW;
            const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(e + h1);
            const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(e + h2);
            p0 ^= a.x;
            p1 ^= a.y;
            q0 ^= c.x;
            q1 ^= c.y;
        }
        x[0] = L.odd ? q0 : p0;
        x[1] = L.odd ? q1 : p1;
        x[2] = L.odd ? p0 : q0;
        x[3] = L.odd ? p1 : q1;
        return;
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const unsigned v = ((g < 4 ? zl : zh) >> (8 * (g & 3))) & 127u;
        const u64 *e = L.Tb + (g * 128 + (int)v) * TW;
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(e + h1);
        const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(e + h2);
        p0 ^= a.x;
        p1 ^= a.y;
        q0 ^= c.x;
        q1 ^= c.y;
    }
    {
        // bits 7, 15, ..., 63 of z gathered into one byte
        const unsigned top = ((((zl >> 7) & 0x01010101u) * 0x01020408u) >> 24) |
                             (((((zh >> 7) & 0x01010101u) * 0x01020408u) >> 24) << 4);
        const u64 *e = L.Ub + (int)top * TW;
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(e + h1);
        const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(e + h2);
        p0 ^= a.x;
        p1 ^= a.y;
        q0 ^= c.x;
        q1 ^= c.y;
    }
    x[0] = L.odd ? q0 : p0;
    x[1] = L.odd ? q1 : p1;
    x[2] = L.odd ? p0 : q0;
    x[3] = L.odd ? p1 : q1;
}

__device__ __forceinline__ void load4(const uint64_t *src, u64 (&d)[4])
{
    const ulonglong2 a = reinterpret_cast<const ulonglong2 *>(src)[0];
    const ulonglong2 c = reinterpret_cast<const ulonglong2 *>(src)[1];
    d[0] = a.x;
    d[1] = a.y;
    d[2] = c.x;
    d[3] = c.y;
}

__device__ __forceinline__ void store4(uint64_t *dst, const u64 (&d)[4])
{
    ulonglong2 a, c;
    a.x = d[0];
    a.y = d[1];
    c.x = d[2];
    c.y = d[3];
    reinterpret_cast<ulonglong2 *>(dst)[0] = a;
    reinterpret_cast<ulonglong2 *>(dst)[1] = c;
}

// Pipelined sweep of blocks [ja, jb) of one tile whose rows are all plain: trailing rows found
// through perm (UP false) or rows above the panel kept in `out` (UP true, MODE 1). EDGE: the tile
// holds the panel word b, word b + 1 or words past W, so stores are per word.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Pipelined sweep of blocks [ja, jb) of one tile whose rows are all plain: trailing rows found
// through perm (UP false) or rows above the panel kept in `out` (UP true, MODE 1). EDGE: the tile
// holds the panel word b, word b + 1 or words past W, so threads with such words store per word.
// Pipeline: physical row 5 blocks ahead, an L2 prefetch of the row's 128-byte line 4 ahead, the
// panel word 3 ahead, the row data 2 ahead (registers), then the block itself.
template <int MODE, bool UP, bool EDGE, bool COUNT, int KB, int RP = RPU>
__device__ __forceinline__ void lean_blocks(const Cfg &c, const SweepSmem &S, const Lanes &L, int w0, int ja, int jb,
                                            unsigned long long &cnt)
{
    const int pbase = c.row0 + L.rg;
    const int plast = c.m - 1;
    // In an edge tile, a thread whose four words are all left of the panel word has nothing to
    // do; the others read and write their 32 bytes whole (words left of b and word b + 1, which
    // goes to the side buffer, are written back unchanged) unless the row ends inside them.
    const bool idle = EDGE && w0 + 3 < c.b;
    const bool full4 = !EDGE || w0 + 3 < c.W;
    int ph0 = 0, ph1 = 0, ph2 = 0, ph3 = 0, ph4 = 0, ph5 = 0;
    u64 wv0 = 0, wv1 = 0, wv2 = 0, wv3 = 0;
    u64 d0[4] = {0, 0, 0, 0}, d1[4] = {0, 0, 0, 0}, d2[4] = {0, 0, 0, 0};
    // positions clamped into [0, m): the loads of the pipeline's first and last iterations (blocks
    // before ja or past the range or the matrix) read valid rows and are never used
    auto pos = [&](int jj) { return min(max(pbase + jj * RP, 0), plast); };
    for (int j = ja - 5; j < jb; ++j) {
        if (!UP) {
            ph5 = c.perm[pos(j + 5)];
            if (L.sub == 0)
                prefetch_l2(c.A + (int64_t)ph4 * c.stride + (w0 & ~(TW - 1)));
            wv3 = c.side_cur[ph3];
        } else {
            if (L.sub == 0)
                prefetch_l2(c.out + (int64_t)pos(j + 4) * c.ostride + (w0 & ~(TW - 1)));
            wv3 = c.ups_cur[pos(j + 3)];
        }
        {
            const int p2 = pos(j + 2);
            const uint64_t *src = UP ? c.out + (int64_t)p2 * c.ostride + w0 : c.A + (int64_t)ph2 * c.stride + w0;
            // in an edge tile every row is read: its word b + 1 goes to the side buffer (trailing rows)
            // or to the next panel-word buffer of the rows above
            if (!idle && (wv2 != 0 || EDGE)) {
                if (full4) {
                    load4(src, d2);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        d2[k] = w0 + k < c.W ? src[k] : 0ull;
                }
            } else {
                d2[0] = d2[1] = d2[2] = d2[3] = 0;
            }
        }
        if (j >= ja) {
            const int p = pbase + j * RP;
            const u64 z = coords(S, L, wv0);
            u64 x[4];
            lookup<KB>(L, z, x);
            if (p < c.m && !idle && (wv0 != 0 || EDGE)) {
                uint64_t *row = UP ? c.out + (int64_t)p * c.ostride : c.A + (int64_t)ph0 * c.stride;
                u64 nw[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int w = w0 + k;
                    if (EDGE && UP && w == c.b + 1)
                        c.ups_nxt[p] = d0[k] ^ x[k];  // (x = 0 when the row's panel word is zero)
                    if (!EDGE || UP)
                        nw[k] = (!EDGE || w >= c.b) ? d0[k] ^ x[k] : d0[k];
                    else if (w < c.b || w == c.b + 1)
                        nw[k] = d0[k];  // left of the panel, or word b + 1 (kept in A, sent to the side buffer)
                    else if (w == c.b)
                        nw[k] = MODE ? 0ull : x[k];  // multipliers (PLS), nothing left (reduced form)
                    else
                        nw[k] = d0[k] ^ x[k];
                    if (EDGE && !UP && w == c.b + 1) {
                        const u64 nv = d0[k] ^ x[k];
                        c.side_nxt[ph0] = nv;  // A's word b + 1 is read by the next pivot search
                        if (COUNT)
                            cnt += __popcll(nv);
                    }
                }
                if (UP && wv0 == 0) {
                    // unchanged row above (only word b + 1 was passed on)
                } else if (full4) {
                    store4(row + w0, nw);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w0 + k < c.W && w0 + k >= c.b)
                            row[w0 + k] = nw[k];
                }
            }
        }
        ph0 = ph1;
        ph1 = ph2;
        ph2 = ph3;
        ph3 = ph4;
        ph4 = ph5;
        wv0 = wv1;
        wv1 = wv2;
        wv2 = wv3;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            d0[k] = d1[k];
            d1[k] = d2[k];
        }
    }
}

__device__ __forceinline__ int row_code(const Cfg &c, int p)
{
    if (p >= c.m)
        return CODE_NONE;
    if (p < c.r)
        return CODE_UP;
    if (p < c.r + c.kbar)
        return -3 - (p - c.r);
    return trailing_row(c.perm, c.st, c.r, c.nwin, c.nx, p);
}

// One block of any tile, any rows (pivot rows, window rows, the panel word's tile).
template <int MODE, bool COUNT, int KB, int RP = RPU>
__device__ __forceinline__ void general_block(const Cfg &c, const SweepSmem &S, const Lanes &L, int w0, int j,
                                              unsigned long long &cnt)
{
    const int p = c.row0 + j * RP + L.rg;
    const int code = row_code(c, p);
    u64 wv = 0;
    if (code >= 0)
        wv = c.side_cur[code];
    else if (code == CODE_UP)
        wv = c.ups_cur[p];
    u64 d[4] = {0, 0, 0, 0};
    if (code >= 0 || code == CODE_UP) {
        const uint64_t *src = code >= 0 ? c.A + (int64_t)code * c.stride : c.out + (int64_t)p * c.ostride;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            d[k] = w0 + k < c.W ? src[w0 + k] : 0ull;
    }
    u64 z = coords(S, L, wv);
    if (code <= -3)
        z = MODE ? c.st->zmap[c.st->pcol[-3 - code]] : c.st->zpiv[-3 - code];
    u64 x[4];
    lookup<KB>(L, z, x);
    if (code == CODE_NONE)
        return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int w = w0 + k;
        if (w >= c.W || w < c.b)
            continue;
        if (code >= 0) {
            uint64_t *row = c.A + (int64_t)code * c.stride;
            if (w == c.b)
                row[w] = MODE ? 0ull : x[k];  // multipliers (PLS), nothing left (reduced form)
            else if (w == c.b + 1) {
                const u64 nv = d[k] ^ x[k];
                c.side_nxt[code] = nv;  // A's word b + 1 is read by the next pivot search
                if (COUNT)
                    cnt += __popcll(nv);
            } else
                row[w] = d[k] ^ x[k];
        } else if (code == CODE_UP) {
            if (w == c.b + 1)
                c.ups_nxt[p] = d[k] ^ x[k];
            if (wv != 0)
                c.out[(int64_t)p * c.ostride + w] = d[k] ^ x[k];
        } else if (c.out) {  // pivot row, at its final position (no pivot rows are kept for the rank alone)
            c.out[(int64_t)p * c.ostride + w] = (!MODE && w == c.b) ? c.st->newblk[-3 - code] : x[k];
            if (MODE && w == c.b + 1)
                c.ups_nxt[p] = x[k];  // a row above from the next panel on
        }
    }
}

// The sweep proper (the panel has pivots): tables per tile, then the blocks of each tile.
template <int MODE, bool COUNT, int KB, int NTH = NT, int TOFF = 0>
__device__ __forceinline__ void sweep_body(Cfg &c, SweepSmem &S, unsigned long long &cnt, int cta, int ncta)
{
    constexpr int RP = NTH / TPR;  // rows per block
    c.row0 = MODE ? 0 : c.r;
    const int tid = (int)threadIdx.x - TOFF;
    const int m = c.m, W = c.W, b = c.b;
    const int64_t stride = c.stride;
    const uint64_t *__restrict__ A = c.A;
    const PanelState *__restrict__ st = c.st;
    const u64 *__restrict__ side_cur = c.side_cur;
    const int M = m - c.row0;
    if (M <= 0)
        return;
    const int wstart = b & ~(TW - 1);
    const int tiles = (W - wstart + TW - 1) / TW;
    const int nblk = (M + RP - 1) / RP;
    const long long total = (long long)tiles * nblk;
    const long long q_lo = total * cta / ncta, q_hi = total * (cta + 1) / ncta;
    if (q_lo >= q_hi)
        return;
    // blocks [0, up_end) hold only rows above the panel (MODE 1); blocks from plain_blk on hold
    // trailing rows that perm alone gives, except the blocks holding a position the pivot search
    // swapped from past its window (xblk); those and the blocks between take the general path
    const int up_end = MODE ? (c.r - c.row0) / RP : 0;
    const int plain_from = c.r + max(c.kbar, c.nwin);
    const int plain_blk = min(nblk, (plain_from - c.row0 + RP - 1) / RP);

    if (tid < 64) {
        S.map[tid] = st->zmap[tid];
        S.prow[tid] = tid < c.kbar ? st->prow[tid] : 0;
        S.xblk[tid] = tid < c.nx ? (st->xpos[tid] - c.row0) / RP : INT_MAX;
    }
    sweep_sync<NTH, TOFF>();
    if (tid < 8 * 16) {
        // coordinate table of byte position q, entries (vh << 4) | low in Gray-code order of the
        // low nibble (one XOR per entry), both copies
        const int q = tid >> 4, vh = tid & 15;
        const u64 *mq = S.map + 8 * q;
        u64 cur = 0;
#pragma unroll
        for (int bit = 0; bit < 4; ++bit)
            cur ^= ((vh >> bit) & 1) ? mq[4 + bit] : 0ull;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i)
                cur ^= mq[__ffs(i) - 1];
            const int v = (vh << 4) | (i ^ (i >> 1));
            S.Z[v * 16 + q] = cur;
            S.Z[v * 16 + 8 + q] = cur;
        }
    }
    Lanes L;
    L.sub = tid & (TPR - 1);
    L.rg = tid / TPR;
    L.odd = (tid >> 2) & 1;
    L.zcopy = (tid >> 3) & 1;  // rows 2, 3 of each half-warp
    L.Tb = S.T + 4 * L.sub;
    L.Ub = S.U + 4 * L.sub;

    for (long long q = q_lo; q < q_hi;) {
        const int tile = (int)(q / nblk);
        const long long q_end = min(q_hi, (long long)(tile + 1) * nblk);
        const int blk0 = (int)(q - (long long)tile * nblk), blk1 = (int)(q_end - (long long)tile * nblk);
        q = q_end;
        const int wbase = wstart + tile * TW;
        // ---- tables of this tile (MakeTable over the rows of O, Gray-code order) ----
        sweep_sync<NTH, TOFF>();
        for (int e = tid; e < 64 * TW; e += NTH) {
            const int t = e / TW, w = wbase + e % TW;
            u64 v = 0;
            if (t < c.kbar && w < W && w >= b) {
                const int pr = S.prow[t];
                if (w > b)
                    v = A[(int64_t)pr * stride + w];
                else if (MODE)
                    v = side_cur[pr];  // the pivot row's current panel word
                else
                    v = st->newblk[t] & st->J & lowmask(st->pcol[t] + 1);  // X_t: multipliers and own bit
            }
            S.O[e] = v;
        }
        sweep_sync<NTH, TOFF>();
        if (KB == 4) {
            // 16 tables of the 16 sums of 4 pivot rows each
            for (int e = tid; e < 16 * TW; e += NTH) {
                const int wi = e % TW, g = e / TW;
                const u64 *Og = S.O + (4 * g) * TW + wi;
                gray16(0ull, Og[0], Og[TW], Og[2 * TW], Og[3 * TW], S.T + (g * 16) * TW + wi, TW);
            }
            sweep_sync<NTH, TOFF>();
        } else {
            for (int e = tid; e < 8 * 8 * TW; e += NTH) {
                // group g, high bits vh (rows 8 g + 4 .. 8 g + 6), word wi: 16 entries by Gray code
                const int wi = e % TW, vh = (e / TW) & 7, g = e / (8 * TW);
                const u64 *Og = S.O + (8 * g) * TW + wi;
                u64 base = 0;
    #pragma unroll
                for (int bit = 0; bit < 3; ++bit)
                    base ^= ((vh >> bit) & 1) ? Og[(4 + bit) * TW] : 0ull;
                gray16(base, Og[0], Og[TW], Og[2 * TW], Og[3 * TW], S.T + (g * 128 + (vh << 4)) * TW + wi, TW);
            }
            if (tid < 16 * TW) {
                const int wi = tid % TW, vh = tid / TW;
                const u64 *O7 = S.O + 7 * TW + wi;  // row 8 g + 7 at O7[8 g TW]
                u64 base = 0;
    #pragma unroll
                for (int bit = 0; bit < 4; ++bit)
                    base ^= ((vh >> bit) & 1) ? O7[8 * (4 + bit) * TW] : 0ull;
                gray16(base, O7[0], O7[8 * TW], O7[16 * TW], O7[24 * TW], S.U + (vh << 4) * TW + wi, TW);
            }
            sweep_sync<NTH, TOFF>();
        }
        const int w0 = wbase + 4 * L.sub;
        const bool interior = wbase >= b + 2 && wbase + TW <= W;
        const int ua = blk0, ub = min(blk1, up_end);
        if (MODE && ua < ub) {
            if (interior)
                lean_blocks<MODE, true, false, COUNT, KB, RP>(c, S, L, w0, ua, ub, cnt);
            else
                lean_blocks<MODE, true, true, COUNT, KB, RP>(c, S, L, w0, ua, ub, cnt);
        }
        for (int j = max(blk0, up_end); j < min(blk1, plain_blk); ++j)
            general_block<MODE, COUNT, KB, RP>(c, S, L, w0, j, cnt);
        // runs of plain blocks through the pipeline, each block holding a swapped position alone
        for (int ja = max(blk0, plain_blk); ja < blk1;) {
            int jx = blk1;
            for (int x = 0; x < c.nx; ++x)
                jx = S.xblk[x] >= ja && S.xblk[x] < jx ? S.xblk[x] : jx;
            if (ja < jx) {
                if (interior)
                    lean_blocks<MODE, false, false, COUNT, KB, RP>(c, S, L, w0, ja, jx, cnt);
                else
                    lean_blocks<MODE, false, true, COUNT, KB, RP>(c, S, L, w0, ja, jx, cnt);
            }
            if (jx < blk1)
                general_block<MODE, COUNT, KB, RP>(c, S, L, w0, jx, cnt);
            ja = jx + 1;
        }
    }
}


// One panel's sweep by CTAs cta of ncta. FORM 0: PLS; 1: reduced echelon form; 2: hybrid, the
// form the pivot search chose for this panel (st->mode), and the set bits of the trailing rows'
// next panel word are counted into st->pop.
template <int FORM, int KB, int NTH = NT, int TOFF = 0>
__device__ __forceinline__ void sweep_panel16(SweepSmem &S, uint64_t *__restrict__ A, int64_t stride,
                                              const u64 *__restrict__ side_cur, u64 *__restrict__ side_nxt,
                                              const int *__restrict__ perm, const PanelState *__restrict__ st,
                                              uint64_t *__restrict__ out, int64_t ostride, u64 *__restrict__ ups,
                                              int m, int W, int b, int cta, int ncta)
{
    const int tid = (int)threadIdx.x - TOFF;
    Cfg c;
    c.A = A;
    c.stride = stride;
    c.side_cur = side_cur;
    c.side_nxt = side_nxt;
    c.perm = perm;
    c.st = st;
    c.out = out;
    c.ostride = ostride;
    c.m = m;
    c.W = W;
    c.b = b;
    c.r = st->r_cur;
    c.kbar = st->kbar;
    c.nwin = st->nwin;
    c.nx = st->nx;
    c.ups_cur = ups ? ups + (size_t)(b & 1) * m : nullptr;
    c.ups_nxt = ups ? ups + (size_t)((b + 1) & 1) * m : nullptr;
    unsigned long long cnt = 0;
    const bool reduced = FORM == 1 || (FORM == 2 && st->mode == 1);
    if (c.kbar == 0 && reduced && b + 1 < W) {
        // the rows above keep their rows; pass their word b + 1 on
        for (int p = cta * NTH + tid; p < c.r; p += ncta * NTH)
            c.ups_nxt[p] = out[(int64_t)p * ostride + b + 1];
    }
    if (c.kbar == 0) {
        // no pivot: every trailing row's panel word is zero; word b + 1 is unchanged. Unless
        // the tail is already known to be zero, look for a nonzero word right of the panel in
        // any trailing row (none means no later panel has a pivot). Rows above stay as they are.
        const bool check = !st->zero_tail;
        bool nzw = false;
        for (int p = c.r + cta * NTH + tid; p < m; p += ncta * NTH) {
            const int ph = trailing_row(perm, st, c.r, c.nwin, c.nx, p);
            const uint64_t *row = A + (int64_t)ph * stride;
            A[(int64_t)ph * stride + b] = side_cur[ph];
            if (b + 1 < W) {
                const u64 v = row[b + 1];
                side_nxt[ph] = v;
                if (FORM == 2)
                    cnt += __popcll(v);
                if (check) {
                    nzw = nzw || v != 0;
                    for (int w = b + 2; w < W && !nzw; ++w)
                        nzw = row[w] != 0;
                }
            }
        }
        if (sweep_sync_or<NTH, TOFF>(nzw) && tid == 0)
            atomicExch(const_cast<int *>(&st->nz), 1);
    } else if (!reduced) {
        sweep_body<0, FORM == 2, KB, NTH, TOFF>(c, S, cnt, cta, ncta);
    } else {
        sweep_body<1, FORM == 2, 8, NTH, TOFF>(c, S, cnt, cta, ncta);  // the reduced form is built for k = 8
    }
    if (FORM == 2) {
        // the density count for the hybrid's switch
        for (int o = 16; o > 0; o >>= 1)
            cnt += __shfl_xor_sync(GF2_FULL, cnt, o);
        if ((tid & 31) == 0 && cnt)
            atomicAdd(const_cast<unsigned long long *>(&st->pop), cnt);
    }
}

}  // namespace
