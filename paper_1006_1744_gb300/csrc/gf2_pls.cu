// gf2_pls.cu -- panel elimination for PLS decomposition and rank over GF(2).
//
// The method is MMPF (Sec. 4.1) with 64-column panels aligned to words:
//   * k_pivot      PlsSubmatrix's job (appendix): the pivots of one panel word
//                  by the Gaussian PLS rule (leftmost column with a 1 in a row
//                  >= r, first such row in the current row order), rows swapped
//                  only logically through a position -> row map;
//   * k_sweep      MakeTable1 + AddRowsFromTable (Sec. 3.1, 4.1): Gray-code
//                  tables of the pivot rows in shared memory, one table per 8
//                  pivots (k = 8), and a 128-bit XOR sweep over the trailing
//                  rows that also writes the multipliers of L into the panel;
//   * k_gather     applies the row order once at the end;
//   * k_compress   "compress L" (swap columns j and Q[j] from row j on).
// The result is the Gaussian PLS result bit for bit (Sec. 4: the table lookup
// writes exactly the forward-substitution multipliers).
#include <climits>

#include <algorithm>
#include <mutex>

#include "gf2_common.cuh"
#include "gf2_sweep.cuh"

namespace {

constexpr int WIN = 96;    // rows held by the pivot warp (3 per lane)
constexpr int NSLOT = WIN / 32;

// ---------------------------------------------------------------------------
// initialisation: identity row order, panel word 0 of every row, state reset
// ---------------------------------------------------------------------------
__global__ void k_init(const uint64_t *__restrict__ A, int64_t stride, int *__restrict__ perm,
                       u64 *__restrict__ side0, PanelState *st, int m, int nst = 2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        perm[i] = i;
        if (side0)
            side0[i] = A[(int64_t)i * stride];
    }
    if (i < nst && st) {  // every panel state slot
        st[i].nwin = 0;
        st[i].nx = 0;
        st[i].r_cur = 0;
        st[i].r_next = 0;
        st[i].kbar = 0;
        st[i].status = 0;
        st[i].zero_tail = 0;
        st[i].nz = 0;
        st[i].J = 0;
        st[i].mode = 0;
        st[i].r_switch = INT_MAX;
        st[i].pop = 0;
    }
}

// ---------------------------------------------------------------------------
// Pivot search of panel b (one warp).
//
// Rows at positions >= r are candidates. Pivot t is the smallest column
// j > j_{t-1} with a 1 in some candidate (reduced by the pivots found so far in
// this panel), and among those the candidate with the smallest position:
// exactly the rule of the Gaussian PLS algorithm restricted to this panel.
//
// Outputs per pivot t: its physical row, position (P) and column (Q), its
// final panel word (the Gaussian PLS row: multipliers of L left of its pivot,
// the reduced bits right of it) and its multipliers as a bit vector over the
// earlier pivots; per pivot column: the row of U_J^-1 (U_J = the pivots'
// reduced rows at the pivot columns), which turns the raw panel word of any
// later row into its multipliers.
//
// Fast path (pivot_fast): the first WIN = 96 positions. Lane l holds the rows at
// initial positions l, l + 32, l + 64 and their current positions; a pivot costs
// one warp min-reduction of (position, slot, lane) over the candidates, one
// shuffle of the pivot row, a relabel of two positions (the swap) and a masked
// XOR per row. L^-1 and U_J^-1 follow from the pivot rows after the loop. A
// dense panel needs about 66 rows; if a column has no candidate in the window
// while rows exist past it, the panel is redone by the row-form path
// (pivot_rows), which also scans past the window.
// ---------------------------------------------------------------------------
constexpr int GROUP = 8;  // columns per group step of the row-form path
constexpr int SW = 16;    // rows of the prefix eliminated per group step

// 32 x 32 bit transpose across a warp: lane i holds row i on input, lane c
// holds column c on output (five butterfly exchanges).
__device__ __forceinline__ unsigned bt32(unsigned x, int lane)
{
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const unsigned m = masks[k];
        const unsigned y = __shfl_xor_sync(GF2_FULL, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

struct PivotShared {
    // window, indexed by position - r (row form)
    u64 Ww[WIN], Wx[WIN];
    int Wph[WIN];
    // Gauss-Jordan basis of the pivots so far (row form): word, U-coordinates, column
    u64 sVw[64], sVx[64];
    int sVc[64], sC2P[64];
    // results: final panel word, multipliers, rows of U_J^-1 and L^-1, position, column of each pivot
    u64 sNew[64], sXl[64], sUi[64], sLi[64];
    int sPpos[64], sPcol[64];
    // group scratch of the row-form path
    u64 TVw[256], TVx[256];
    u64 gVw[GROUP], gVx[GROUP];
    int gIpos[GROUP], gX8[GROUP], gLinv[GROUP], gMm[GROUP], gUinv[GROUP];
    // previous panel: its maps (raw panel bits -> coordinates) and its pivot rows' word b,
    // as 4-bit tables: pNZ[q][v] = sum of the maps of the set bits of v at bits 4q..4q+3,
    // pNO[q][v] likewise over the pivot rows
    u64 pZ[64], pO[64];
    u64 pNZ[16][16], pNO[16][16];
    // positions past the window swapped in this panel (position -> physical row)
    int nx;
    int xpos[64], xval[64];
    // the previous panel's swaps past its window, while perm does not hold them yet
    int pnx;
    int pxpos[64], pxval[64];
};

// Context for the panel word b of a row: the previous panel's sweep updates
// word b only in its side buffer, so the pivot search derives it from A
// (current up to panel b - 2) plus panel b - 1's contribution.
struct WordCtx {
    const uint64_t *wsrc;  // word b of row 0 (A + b, or a buffer of the rows' panel words) ...
    int64_t wstride;       // ... and the words between consecutive rows there
    const u64 *side_prev;  // panel word b - 1 of every row (nullptr: wsrc's word b is already current)
    int64_t side_stride;   // words between consecutive rows of side_prev
};

// word b of a row from its value in A and its panel word b - 1 (v)
__device__ __forceinline__ u64 word_after(const PivotShared &S, u64 w, u64 v)
{
    u64 z = 0, acc = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        z ^= S.pNZ[q][(int)((v >> (4 * q)) & 15ull)];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        acc ^= S.pNO[q][(int)((z >> (4 * q)) & 15ull)];
    return w ^ acc;
}

__device__ __forceinline__ u64 panel_word(const WordCtx &c, const PivotShared &S, int ph)
{
    const u64 w = c.wsrc[(int64_t)ph * c.wstride];
    return c.side_prev ? word_after(S, w, c.side_prev[(int64_t)ph * c.side_stride]) : w;
}

// position -> physical row during the pivot search (perm plus this panel's swaps past the window)
__device__ __forceinline__ int perm_at(const int *__restrict__ perm, const PivotShared &S, int p)
{
    for (int x = 0; x < S.nx; ++x)
        if (S.xpos[x] == p)
            return S.xval[x];
    for (int x = 0; x < S.pnx; ++x)
        if (S.pxpos[x] == p)
            return S.pxval[x];
    return perm[p];
}

__device__ bool pivot_fast(int r, int m, int nwin, int nbits, int &t_out, u64 &J_out, PivotShared &S)
{
    const int lane = threadIdx.x;
    // lane l holds the window rows at initial positions l + 32 k; a swap of positions
    // only relabels two rows, no row moves
    u64 row[NSLOT];
    int pos[NSLOT], phys[NSLOT];
    bool act[NSLOT];
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) {
        const int i = lane + 32 * k;
        act[k] = i < nwin;
        phys[k] = act[k] ? S.Wph[i] : 0;
        row[k] = act[k] ? S.Ww[i] : 0ull;
        pos[k] = i;
    }
    __syncwarp();
    // pivot s: lane s & 31 keeps its panel word, position (at the time of the step) and column
    u64 nw0 = 0, nw1 = 0;
    int recp0 = 0, recp1 = 0, recj0 = 0, recj1 = 0;
    const bool all_rows = (m - r) <= WIN;
    int t = 0, j = 0;
    u64 J = 0;
    // bit j of each row, kept one step ahead: after a pivot it follows from the row's old
    // bit j + 1 and one bit of the pivot row, so the 64-bit XOR stays off the chain
    bool cb[NSLOT];
#pragma unroll
    for (int k = 0; k < NSLOT; ++k)
        cb[k] = row[k] & 1ull;
    while (t < 64 && j < nbits && t < nwin) {
        bool cand[NSLOT];
        int key = INT_MAX;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            cand[k] = act[k] && cb[k];
            key = cand[k] ? min(key, (pos[k] << 7) | (k << 5) | lane) : key;
        }
        // first candidate in the current row order
        const int best = __reduce_min_sync(GF2_FULL, key);
        if (best == INT_MAX) {
            if (!all_rows)
                return false;  // a candidate may sit past the window
            ++j;               // zero column among all remaining rows
#pragma unroll
            for (int k = 0; k < NSLOT; ++k)
                cb[k] = (row[k] >> (j & 63)) & 1ull;
            continue;
        }
        const int p = best >> 7, slot = (best >> 5) & 3, plane = best & 31;
        u64 mine = row[0];
#pragma unroll
        for (int k = 1; k < NSLOT; ++k)
            mine = slot == k ? row[k] : mine;
        const u64 prow = __shfl_sync(GF2_FULL, mine, plane);
        if (t < 32) {
            nw0 = lane == t ? prow : nw0;
            recp0 = lane == t ? p : recp0;
            recj0 = lane == t ? j : recj0;
        } else {
            nw1 = lane == t - 32 ? prow : nw1;
            recp1 = lane == t - 32 ? p : recp1;
            recj1 = lane == t - 32 ? j : recj1;
        }
        // swap positions t and p: the pivot takes t (and leaves the candidates), the row
        // at t takes p; rows below with a 1 in column j get the pivot row right of j
        const u64 pm = prow & (~1ull << j);
        const int j1 = (j + 1) & 63;
        const bool pb1 = (prow >> j1) & 1ull;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            const bool isp = lane == plane && k == slot;
            const bool x = cand[k] && !isp;
            const bool ob1 = (row[k] >> j1) & 1ull;
            row[k] ^= x ? pm : 0ull;
            cb[k] = ob1 ^ (x && pb1);
            pos[k] = isp ? t : (pos[k] == t ? p : pos[k]);
            act[k] = act[k] && !isp;
        }
        J |= 1ull << j;
        ++j;
        ++t;
    }
#pragma unroll
    for (int k = 0; k < NSLOT; ++k)
        if (lane + 32 * k < nwin)
            S.Wph[pos[k]] = phys[k];
    // pivot rows: the Gaussian-PLS panel word -- multipliers of L at the earlier pivot
    // columns, 1 at its own, reduced bits right of it
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s2 = lane + 32 * k;
        if (s2 < t) {
            const u64 rw = k ? nw1 : nw0;
            const int js = k ? recj1 : recj0;
            S.sNew[s2] = rw;
            S.sPpos[s2] = r + (k ? recp1 : recp0);
            S.sPcol[s2] = js;
            // multipliers over the earlier pivots, and the U_J row (pivot columns >= js)
            S.sXl[s2] = pext64(rw & lowmask(js), J);
            S.sVw[s2] = pext64(rw & ~lowmask(js), J);
        }
    }
    __syncwarp();
    t_out = t;
    J_out = J;
    return true;
}

// Row-form path: window rows in shared memory indexed by position, pivots taken
// GROUP columns at a time when the first SW candidate rows hold a 1 in each of
// them (a contiguous prefix of the row order, so a 1 found there is the first
// one in its column), one at a time otherwise, with rows past the window
// reduced from scratch by the Gauss-Jordan basis.
__device__ void pivot_rows(const WordCtx &wc, const int *__restrict__ perm, int r, int m, int nwin, int nbits,
                           int &t_out, u64 &J_out, PivotShared &S)
{
    const int lane = threadIdx.x;
    int t = 0;
    u64 J = 0;
    for (int i = lane; i < nwin; i += 32)
        S.Wx[i] = 0;
    __syncwarp();
    int jlow = 0;
    while (nwin > 0 && t < 64 && jlow < nbits && r + t < m) {
        const int kbmax = min(GROUP, nbits - jlow);
        // ---------------- group step: the first SW candidate rows, GROUP columns ----------------
        {
            const bool rv = lane < SW && t + lane < nwin;
            int sl = rv ? (int)((S.Ww[t + lane] >> jlow) & (u64)((1u << kbmax) - 1u)) : 0;
            int pos = lane;   // position in the prefix (current order)
            int comb = 0;     // raw pivot rows in this row's reduced slice
            int mul = 0;      // multipliers for the group's pivots
            int pidx = -1;    // pivot index within the group, once chosen
            int gjb = 0, gjc = 0, gju = 0;  // Gauss-Jordan row: slice, raw-row combination, U-coordinates
            int lcomb = 0, lmul = 0, lpos = 0;
            int kb = 0;
            for (int c = 0; c < kbmax; ++c) {
                const bool cand = rv && pidx < 0 && ((sl >> c) & 1);
                const int kmin = __reduce_min_sync(GF2_FULL, cand ? pos : 1 << 20);
                if (kmin >= (1 << 20))
                    break;
                const int owner = __ffs(__ballot_sync(GF2_FULL, cand && pos == kmin)) - 1;
                const int pv = __shfl_sync(GF2_FULL, sl, owner);
                const int lc = __shfl_sync(GF2_FULL, comb, owner) | (1 << c);
                if (lane == owner) {
                    lpos = kmin;
                    lcomb = lc;
                    lmul = mul;
                    pidx = c;
                    gjb = pv;
                    gjc = lc;
                    gju = 1 << c;
                } else if (pidx < 0 && pos == c) {
                    pos = kmin;  // the head row takes the pivot's old position
                }
                if (lane == owner)
                    pos = c;
                if (pidx < 0 && rv && pos > c && ((sl >> c) & 1)) {
                    sl ^= pv;
                    comb ^= lc;
                    mul |= 1 << c;
                }
                if (pidx >= 0 && pidx < c && ((gjb >> c) & 1)) {
                    gjb ^= pv;
                    gjc ^= lc;
                    gju ^= 1 << c;
                }
                kb = c + 1;
            }
            if (kb > 0) {
                u64 mw = 0, mx = 0;
                int mph = 0;
                if (rv) {
                    mw = S.Ww[t + lane];
                    mx = S.Wx[t + lane];
                    mph = S.Wph[t + lane];
                }
                __syncwarp();
                if (rv) {
                    S.Ww[t + pos] = mw;
                    S.Wx[t + pos] = mx;
                    S.Wph[t + pos] = mph;
                }
                if (pidx >= 0) {
                    S.gIpos[pidx] = lpos;
                    S.gX8[pidx] = lmul;
                    S.gLinv[pidx] = lcomb;
                    S.gMm[pidx] = gjc;
                    S.gUinv[pidx] = gju;
                }
                __syncwarp();
                u64 rw8[GROUP];
#pragma unroll
                for (int c2 = 0; c2 < GROUP; ++c2)
                    rw8[c2] = c2 < kb ? S.Ww[t + c2] : 0ull;
                if (lane < kb) {
                    const int c = lane;
                    const int li = S.gLinv[c], mi = S.gMm[c];
                    u64 uw = 0, vw = 0;
#pragma unroll
                    for (int c2 = 0; c2 < GROUP; ++c2) {
                        if ((li >> c2) & 1)
                            uw ^= rw8[c2];
                        if ((mi >> c2) & 1)
                            vw ^= rw8[c2];
                    }
                    const u64 xl = S.Wx[t + c] | ((u64)S.gX8[c] << t);
                    // scatter the multipliers over the pivot columns so far, this group's included
                    S.sNew[t + c] = uw | pdep64(xl, J | ((((u64)1 << kb) - 1ull) << jlow));
                    S.sXl[t + c] = xl;
                    S.sPpos[t + c] = r + t + S.gIpos[c];
                    S.sPcol[t + c] = jlow + c;
                    S.gVw[c] = vw;
                    S.gVx[c] = (u64)S.gUinv[c] << t;
                }
                __syncwarp();
                u64 vw8[GROUP], vx8[GROUP];
#pragma unroll
                for (int c = 0; c < GROUP; ++c) {
                    vw8[c] = c < kb ? S.gVw[c] : 0ull;
                    vx8[c] = c < kb ? S.gVx[c] : 0ull;
                }
                const int nt = 1 << kb;
                if (8 * lane < nt || lane == 0) {
                    u64 aw = 0, ax = 0;
#pragma unroll
                    for (int c = 3; c < GROUP; ++c)
                        if ((lane >> (c - 3)) & 1) {
                            aw ^= vw8[c];
                            ax ^= vx8[c];
                        }
                    const int base = 8 * lane;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (i) {
                            const int f = (i & 1) ? 0 : ((i & 2) ? 1 : 2);  // lowest set bit of i
                            aw ^= vw8[f];
                            ax ^= vx8[f];
                        }
                        const int v = base + (i ^ (i >> 1));
                        if (v < nt) {
                            S.TVw[v] = aw;
                            S.TVx[v] = ax;
                        }
                    }
                }
                __syncwarp();
                const u64 msk = (u64)(nt - 1);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int s2 = lane + 32 * k;
                    if (s2 < t) {
                        const int bb = (int)((S.sVw[s2] >> jlow) & msk);
                        S.sVw[s2] ^= S.TVw[bb];
                        S.sVx[s2] ^= S.TVx[bb];
                    }
                }
                if (lane < kb) {
                    S.sVw[t + lane] = S.gVw[lane];
                    S.sVx[t + lane] = S.gVx[lane];
                    S.sVc[t + lane] = jlow + lane;
                    S.sC2P[jlow + lane] = t + lane;
                }
                u64 ww[NSLOT];
                int bbk[NSLOT];
#pragma unroll
                for (int k = 0; k < NSLOT; ++k) {
                    const int i = t + kb + lane + 32 * k;
                    ww[k] = i < nwin ? S.Ww[i] : 0ull;
                    bbk[k] = (int)((ww[k] >> jlow) & msk);
                }
#pragma unroll
                for (int k = 0; k < NSLOT; ++k) {
                    const int i = t + kb + lane + 32 * k;
                    if (i < nwin) {
                        S.Ww[i] = ww[k] ^ S.TVw[bbk[k]];
                        S.Wx[i] ^= S.TVx[bbk[k]];
                    }
                }
                __syncwarp();
                t += kb;
                J |= msk << jlow;
                jlow += kb;
            }
            if (kb == kbmax)
                continue;
            if (!(t < 64 && jlow < nbits && r + t < m))
                break;
        }
        // ---------------- general step: one pivot, any column >= jlow ----------------
        int key = INT_MAX;
        for (int i = t + lane; i < nwin; i += 32)
            if ((S.Ww[i] >> jlow) & 1ull) {
                key = i;
                break;
            }
        const int best = __reduce_min_sync(GF2_FULL, key);
        int pc, pos;
        bool from_out = false;
        u64 ow = 0, ox = 0;
        int oph = -1;
        if (best != INT_MAX) {
            pc = jlow;
            pos = r + best;
        } else {
            int myc = 64, myi = INT_MAX;
            for (int i = t + lane; i < nwin; i += 32) {
                const u64 mk = S.Ww[i] & ~lowmask(jlow);
                const int c = mk ? ctz64(mk) : 64;
                if (c < myc) {
                    myc = c;
                    myi = i;
                }
            }
            const int cw = __reduce_min_sync(GF2_FULL, myc);
            const int iw = __reduce_min_sync(GF2_FULL, myc == cw ? myi : INT_MAX);
            int bc = cw, bl = cw < 64 ? r + iw : INT_MAX;
            for (int p0 = r + WIN; p0 < m && !(bc == jlow && p0 >= bl); p0 += 32) {
                const int p = p0 + lane;
                int c = 64, phh = -1;
                u64 ww = 0, xx = 0;
                if (p < m) {
                    phh = perm_at(perm, S, p);
                    ww = panel_word(wc, S, phh);
                    u64 pm = ww & J;
                    while (pm) {
                        const int cc = ctz64(pm);
                        pm &= pm - 1;
                        const int sidx = S.sC2P[cc];
                        ww ^= S.sVw[sidx];
                        xx ^= S.sVx[sidx];
                    }
                    const u64 mk = ww & ~lowmask(jlow);
                    c = mk ? ctz64(mk) : 64;
                }
                const int cc = __reduce_min_sync(GF2_FULL, c);
                if (cc < 64) {
                    const int cp = __reduce_min_sync(GF2_FULL, c == cc ? p : INT_MAX);
                    if (cc < bc || (cc == bc && cp < bl)) {
                        const int src = cp - p0;
                        bc = cc;
                        bl = cp;
                        from_out = true;
                        ow = __shfl_sync(GF2_FULL, ww, src);
                        ox = __shfl_sync(GF2_FULL, xx, src);
                        oph = __shfl_sync(GF2_FULL, phh, src);
                    }
                }
            }
            if (bc == 64)
                break;  // no further pivot in this panel
            pc = bc;
            pos = bl;
        }
        if (lane == 0) {
            if (from_out) {
                // the head row takes the pivot's old position (recorded, applied later)
                int x = 0;
                while (x < S.nx && S.xpos[x] != pos)
                    ++x;
                S.xpos[x] = pos;
                S.xval[x] = S.Wph[t];
                if (x == S.nx)
                    ++S.nx;
                S.Ww[t] = ow;
                S.Wx[t] = ox;
                S.Wph[t] = oph;
            } else if (pos != r + t) {
                const int i = pos - r;
                u64 a = S.Ww[t];
                S.Ww[t] = S.Ww[i];
                S.Ww[i] = a;
                a = S.Wx[t];
                S.Wx[t] = S.Wx[i];
                S.Wx[i] = a;
                const int q = S.Wph[t];
                S.Wph[t] = S.Wph[i];
                S.Wph[i] = q;
            }
        }
        __syncwarp();
        const u64 pw = S.Ww[t], tb = 1ull << t;
        if (lane == 0) {
            S.sNew[t] = pw | pdep64(S.Wx[t], J);
            S.sXl[t] = S.Wx[t];
            S.sPpos[t] = pos;
            S.sPcol[t] = pc;
        }
        for (int s2 = lane; s2 < t; s2 += 32)
            if ((S.sVw[s2] >> pc) & 1ull) {
                S.sVw[s2] ^= pw;
                S.sVx[s2] ^= tb;
            }
        if (lane == 0) {
            S.sVw[t] = pw;
            S.sVx[t] = tb;
            S.sVc[t] = pc;
            S.sC2P[pc] = t;
        }
        for (int i = t + 1 + lane; i < nwin; i += 32)
            if ((S.Ww[i] >> pc) & 1ull) {
                S.Ww[i] ^= pw;
                S.Wx[i] |= tb;
            }
        __syncwarp();
        J |= 1ull << pc;
        jlow = pc + 1;
        ++t;
    }
    __syncwarp();
    // rows of U_J^-1 are the U-coordinates of the Gauss-Jordan rows
    for (int s2 = lane; s2 < t; s2 += 32)
        S.sUi[s2] = S.sVx[s2];
    t_out = t;
    J_out = J;
}

constexpr int PIVOT_THREADS = 128;  // warp 0 runs the elimination chain; all four share the rest

// The pivot search's threads (the first PIVOT_THREADS of the CTA) synchronise on a named barrier of
// their own, so that a larger CTA can run it while its other warps do something else.
__device__ __forceinline__ void pivot_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(PIVOT_THREADS) : "memory"); }
static_assert(WIN <= PIVOT_THREADS, "one window row per thread when the window is formed");

// Pivot search of panel b. It first applies panel b - 1's row-order changes to
// perm (no sweep reads those positions from perm), then forms the window: the
// panel word b of the rows at positions r .. r + nwin - 1, from A plus panel
// b - 1's contribution (side_prev = panel word b - 1 of every row, side_stride
// words apart; nullptr when A's word b already holds it, as for b = 0). This
// panel's own row-order changes go to st (nwin, wperm, nx, xpos, xval) for the
// sweep of this panel and the pivot search of the next one. st holds the state
// of panel b - zt_lag on entry (the states rotate through zt_lag slots), whose
// sweep has completed: the zero-tail test reads it. defer_prev: panel b - 1's
// row order is left out of perm (a sweep still running reads those positions
// there; the step after this search applies it) and taken from st_prev here.
__device__ __forceinline__ void pivot_panel(const uint64_t *__restrict__ wsrc, int64_t wstride,
                                            const u64 *__restrict__ side_prev, int64_t side_stride,
                                            int *__restrict__ perm, const PanelState *__restrict__ st_prev,
                                            PanelState *st, int64_t *P, int64_t *Q, int m, int b, int nbits,
                                            int form, int thr_permille, int zt_lag = 2, bool defer_prev = false)
{
    __shared__ PivotShared S;
    __shared__ u64 sXp[64], sXm[64];
    __shared__ u64 sJ;
    __shared__ int sT, sFast;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = st_prev->r_next;
    // Zero tail: the sweep of panel b - 2 (complete: this search waits for it) found no
    // pivot and no nonzero word right of it in any trailing row, so no later panel has a
    // pivot. st still holds panel b - 2's state here (this search overwrites it below).
    const int zt = st_prev->zero_tail || (b >= zt_lag && st->kbar == 0 && st->nz == 0 && st->r_next == r);
    const int nwin = (r < m && !zt) ? min(WIN, m - r) : 0;
    // panel b - 1's contribution to word b is added here unless A holds it already
    const bool contrib = b > 0 && side_prev != nullptr;
    const WordCtx wc{wsrc, wstride, contrib ? side_prev : nullptr, side_stride};
    // window rows: the previous panel's order where it changed it, perm elsewhere
    // (one row per thread; nwin <= PIVOT_THREADS)
    int ph = 0;
    u64 w = 0, v = 0;
    {
        const int pr = b > 0 ? st_prev->r_cur : 0, pn = b > 0 ? st_prev->nwin : 0, px = b > 0 ? st_prev->nx : 0;
        if (tid < nwin) {
            const int p = r + tid;
            if (p < pr + pn) {
                ph = st_prev->wperm[p - pr];
            } else {
                ph = -1;
                for (int x = 0; x < px; ++x)
                    if (st_prev->xpos[x] == p)
                        ph = st_prev->xval[x];
                if (ph < 0)
                    ph = perm[p];
            }
            w = wsrc[(int64_t)ph * wstride];
            if (contrib)
                v = side_prev[(int64_t)ph * side_stride];
        }
        // apply the previous panel's order to perm (no sweep reads these positions from perm)
        if (!defer_prev) {
            for (int i = tid; i < pn; i += PIVOT_THREADS)
                perm[pr + i] = st_prev->wperm[i];
            for (int x = tid; x < px; x += PIVOT_THREADS)
                perm[st_prev->xpos[x]] = st_prev->xval[x];
        }
        // with the order deferred, the previous panel's window lies inside this one's (it
        // starts at most 64 positions earlier and is no longer), so only its swaps past
        // that window stay to be looked up
        for (int x = tid; x < (defer_prev ? px : 0); x += PIVOT_THREADS) {
            S.pxpos[x] = st_prev->xpos[x];
            S.pxval[x] = st_prev->xval[x];
        }
    }
    if (contrib && tid < 64) {
        S.pZ[tid] = st_prev->zmap[tid];
        S.pO[tid] = tid < st_prev->kbar ? wsrc[(int64_t)st_prev->prow[tid] * wstride] : 0ull;
    }
    if (tid == 0) {
        S.nx = 0;
        S.pnx = defer_prev && b > 0 ? st_prev->nx : 0;
    }
    pivot_barrier();
    if (contrib)
        for (int e = tid; e < 2 * 256; e += PIVOT_THREADS) {
            const int which = e >> 8, q = (e >> 4) & 15, vv = e & 15;
            const u64 *src = which ? S.pO : S.pZ;
            u64 x = 0;
#pragma unroll
            for (int bit = 0; bit < 4; ++bit)
                x ^= ((vv >> bit) & 1) ? src[4 * q + bit] : 0ull;
            (which ? S.pNO : S.pNZ)[q][vv] = x;
        }
    pivot_barrier();
    if (tid < nwin) {
        S.Wph[tid] = ph;
        S.Ww[tid] = contrib ? word_after(S, w, v) : w;
    }
    pivot_barrier();
    if (warp == 0) {
        int t = 0, fast = 1;
        u64 J = 0;
        if (nwin > 0) {
            fast = pivot_fast(r, m, nwin, nbits, t, J, S) ? 1 : 0;
            __syncwarp();
            if (!fast)
                pivot_rows(wc, perm, r, m, nwin, nbits, t, J, S);
        }
        if (lane == 0) {
            sT = t;
            sJ = J;
            sFast = fast;
        }
    } else if (tid < 96) {
        sXp[tid - 32] = 0;
        sXm[tid - 32] = 0;
    }
    pivot_barrier();
    const int t = sT;
    const u64 J = sJ;
    // Inverses, one column per lane: warps 2, 3 -> L^-1 (rows top-down: row s = e_s +
    // the rows k < s that pivot s's multipliers select); warps 0, 1 -> U_J^-1 (rows
    // bottom-up: row s = e_s + the rows k > s that U_J's row s selects; the row-form
    // path has it already). Bit s of a column = parity of (selector & column).
    {
        const bool isU = warp < 2;
        if (!isU || sFast) {
            const int col = lane + 32 * (warp & 1);
            // four rows per step: their parities against the bits found so far are
            // independent; a row selecting an earlier row of the same step is resolved after
            const u64 *sel = isU ? S.sVw : S.sXl;
            u64 X = 0;
            for (int i0 = 0; i0 < t; i0 += 4) {
                int rr[4], bb[4];
                u64 sv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = i0 + u < t;
                    rr[u] = ok ? (isU ? t - 1 - i0 - u : i0 + u) : 0;
                    sv[u] = ok ? sel[rr[u]] : 0ull;
                    const u64 a = sv[u] & X;
                    bb[u] = ok ? ((__popc((unsigned)a ^ (unsigned)(a >> 32)) & 1) ^ (int)(col == rr[u])) : 0;
                }
                // the step's rows sit at base .. base + 3 (base < 0 only in U's last, partial
                // step, whose missing rows select nothing): one shift per selector, then the
                // in-step entries are constant-position bits
                const int base = isU ? t - 4 - i0 : i0;
                unsigned sl[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    sl[u] = base >= 0 ? (unsigned)(sv[u] >> base) : (unsigned)(sv[u] << -base);
#pragma unroll
                for (int u = 1; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < u; ++v)
                        bb[u] ^= (int)((sl[u] >> (isU ? 3 - v : v)) & 1u) & bb[v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    X |= (u64)bb[u] << rr[u];
            }
            // 32 columns x 64 rows -> the warp's 32-bit half of every row
            unsigned *dst = reinterpret_cast<unsigned *>(isU ? S.sUi : S.sLi);
            const unsigned lo = bt32((unsigned)X, lane), hi = bt32((unsigned)(X >> 32), lane);
            if (lane < t)
                dst[2 * lane + (warp & 1)] = lo;
            if (lane + 32 < t)
                dst[2 * (lane + 32) + (warp & 1)] = hi;
        }
    }
    pivot_barrier();
    // maps for the sweep, by pivot column: row of M = U_J^-1 L^-1 (= (O_J)^-1: raw panel bits ->
    // coordinates over the original pivot rows) and the row of U_J^-1 scattered to the pivot
    // columns. Two threads per row of M, each over half of the inner index.
    {
        const int row = tid >> 1, half = tid & 1;
        const u64 ua = row < t ? S.sUi[row] : 0ull;  // no bits at t and above
        u64 acc[4] = {0ull, 0ull, 0ull, 0ull};        // four independent XOR chains
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 32 * half + k0 + u;
                acc[u] ^= ((ua >> k) & 1ull) ? S.sLi[k] : 0ull;
            }
        u64 ma = (acc[0] ^ acc[1]) ^ (acc[2] ^ acc[3]);
        ma ^= __shfl_xor_sync(GF2_FULL, ma, 1);
        if (half == 0 && row < t) {
            sXp[S.sPcol[row]] = ma;
            sXm[S.sPcol[row]] = pdep64(ua, J);
        }
    }
    pivot_barrier();
    // row order of the window (applied to perm by the next panel), P and Q, the panel state
    for (int i = tid; i < nwin; i += PIVOT_THREADS)
        st->wperm[i] = S.Wph[i];
    for (int x = tid; x < S.nx; x += PIVOT_THREADS) {
        st->xpos[x] = S.xpos[x];
        st->xval[x] = S.xval[x];
    }
    for (int s2 = tid; s2 < t; s2 += PIVOT_THREADS) {
        if (P)
            P[r + s2] = S.sPpos[s2];
        if (Q)
            Q[r + s2] = 64ll * b + S.sPcol[s2];
        st->prow[s2] = S.Wph[s2];
        st->pcol[s2] = S.sPcol[s2];
        st->newblk[s2] = S.sNew[s2];
        st->zpiv[s2] = S.sLi[s2];
    }
    if (tid < 64) {
        st->zmap[tid] = sXp[tid];
        st->xmap[tid] = sXm[tid];
    }
    if (tid == 0) {
        // form of this panel's sweep. Hybrid ("M+P", Sec. 6): the reduced form while the
        // density of the remaining rows -- the set bits of word b - 1 that the sweep of panel
        // b - 2 counted over its trailing rows -- stays below the threshold, PLS from then on.
        // st still holds panel b - 2's state here.
        int mode = form < 2 ? form : 1;
        if (form == 2) {
            const int prev = b > 0 ? st_prev->mode : 1;
            const long long rows = (long long)m - st->r_next;
            if (prev == 0)
                mode = 0;
            else if (b >= 2 && rows > 0 && (long long)st->pop * 1000 >= (long long)thr_permille * rows * 64)
                mode = 0;
        }
        const int rsw_prev = b > 0 ? st_prev->r_switch : INT_MAX;
        st->mode = mode;
        st->r_switch = (mode == 0 && rsw_prev == INT_MAX) ? r : rsw_prev;
        st->pop = 0;
        st->r_cur = r;
        st->kbar = t;
        st->r_next = r + t;
        st->J = J;
        st->nwin = nwin;
        st->nx = S.nx;
        st->zero_tail = zt;
        st->nz = 0;
    }
}

// The last panel's row-order changes (before the final gather).
__device__ __forceinline__ void apply_order(int *__restrict__ perm, const PanelState *__restrict__ st)
{
    for (int i = threadIdx.x; i < st->nwin; i += blockDim.x)
        perm[st->r_cur + i] = st->wperm[i];
    for (int x = threadIdx.x; x < st->nx; x += blockDim.x)
        perm[st->xpos[x]] = st->xval[x];
}

__global__ void k_apply_order(int *__restrict__ perm, const PanelState *__restrict__ st) { apply_order(perm, st); }

// Launched as a programmatic dependent of the previous panel's search (same stream):
// it may be scheduled while that search still runs, lets the next one be scheduled in
// turn, and waits on the device until its predecessor has completed and its writes
// are visible. Without the launch attribute both instructions are no-ops.
__global__ void __launch_bounds__(PIVOT_THREADS, 1)
k_pivot(const uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ side_prev, int *__restrict__ perm,
        const PanelState *__restrict__ st_prev, PanelState *st, int64_t *P, int64_t *Q, int m, int b, int nbits,
        int form, int thr_permille)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    pivot_panel(A + b, stride, side_prev, 1, perm, st_prev, st, P, Q, m, b, nbits, form, thr_permille);
}

// Pivot search of one panel of a two-panel sweep step (gf2_pair.cu): states in four slots,
// the previous panel's word from side_prev with any row pitch, its row order optionally
// deferred. Programmatic dependent of the preceding search, as k_pivot.
__global__ void __launch_bounds__(PIVOT_THREADS, 1)
k_pivot_pair(const uint64_t *__restrict__ wsrc, int64_t wstride, const u64 *__restrict__ side_prev,
             int64_t side_stride, int *__restrict__ perm, const PanelState *__restrict__ st_prev, PanelState *st,
             int64_t *P, int64_t *Q, int m, int b, int nbits, int defer)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    pivot_panel(wsrc, wstride, side_prev, side_stride, perm, st_prev, st, P, Q, m, b, nbits, 0, 0, 4, defer != 0);
}

// ---------------------------------------------------------------------------
// Table sweep of panel b (MakeTable1 + AddRowsFromTable).
//
// For a row at position p >= r+kbar with raw panel word w:
//   z       = its coordinates over the original pivot rows O (eight byte
//             lookups into tables built from zmap),
//   panel   <- its multipliers scattered to the pivot columns (tables from xmap),
//   trailing words ^= z.O (eight 128-bit lookups, one Gray-code table of 256
//             sums per 8 pivots: MakeTable over the rows of O).
// Pivot row t gets its final row U_t = zpiv[t].O, written to `out` at its
// final position; pivot rows are never written in A, so the tables can be built
// from A while the sweep runs. The CTA holding word b+1 also stores it in the
// next panel's side buffer.
//
// Work: column tiles of TW words (from the even word <= b) x blocks of rows; each
// CTA takes an equal contiguous run of that tile-major sequence, builds a tile's
// tables once per tile it meets, and keeps RPT rows per thread in flight.
// ---------------------------------------------------------------------------
// rows of one pass of the sweep: position -> physical row, pivot row or not, in range
template <int RPT, int RPP>
__device__ __forceinline__ void pass_rows(int pb, int rg, int p_end, int r, int kbar, int nwin, int nx,
                                          const PanelState *__restrict__ st, const int *__restrict__ perm,
                                          int (&ph)[RPT], bool (&valid)[RPT], bool (&isp)[RPT])
{
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int p = pb + j * RPP + rg;
        valid[j] = p < p_end;
        isp[j] = valid[j] && p < r + kbar;
        ph[j] = !valid[j] ? 0 : (isp[j] ? st->prow[p - r] : trailing_row(perm, st, r, nwin, nx, p));
    }
}

// their panel words and their current words of the tile (not needed for pivot rows)
template <int RPT>
__device__ __forceinline__ void pass_loads(const uint64_t *__restrict__ A, int64_t stride,
                                           const u64 *__restrict__ side_cur, int w0, bool two, bool wact,
                                           const int (&ph)[RPT], const bool (&valid)[RPT], const bool (&isp)[RPT],
                                           u64 (&wv)[RPT], u64 (&o0)[RPT], u64 (&o1)[RPT])
{
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const bool live = valid[j] && !isp[j];
        wv[j] = live ? side_cur[ph[j]] : 0ull;
        o0[j] = 0;
        o1[j] = 0;
        if (live && wact) {
            const uint64_t *a = A + (int64_t)ph[j] * stride + w0;
            if (two) {
                const ulonglong2 v2 = *reinterpret_cast<const ulonglong2 *>(a);
                o0[j] = v2.x;
                o1[j] = v2.y;
            } else {
                o0[j] = a[0];
            }
        }
    }
}

template <int TW, int RPT, int NT>
__device__ __forceinline__ void sweep_panel(uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ side_cur,
                                            u64 *__restrict__ side_nxt, const int *__restrict__ perm,
                                            const PanelState *__restrict__ st, uint64_t *__restrict__ out,
                                            int64_t ostride, int m, int W, int b, int cta, int ncta)
{
    constexpr int TPR = TW / 2;     // threads per row, two words each
    constexpr int RPP = NT / TPR;   // rows per thread slot and pass
    constexpr int BPL = 8 / TPR;    // z-table bytes per thread
    // HALF (16-word tiles, 128-byte table rows: a quarter-warp reads one whole
    // row, so lookups never hit the same bank twice): each 8-bit table keeps only
    // the sums of its first 7 rows, and one more table holds the sums of the 8
    // tables' last rows, indexed by bit 7 of every byte of z.
    constexpr bool HALF = TW == 16;
    constexpr int TE = HALF ? 128 : 256;  // entries per 8-bit table
    extern __shared__ __align__(16) u64 sm[];
    u64 *sT = sm;                          // [8][TE][TW] Gray-code tables of the pivot rows O
    u64 *sU = sT + 8 * TE * TW;            // [256][TW]   (HALF) sums of the rows 8 g + 7
    u64 *sZ = sU + (HALF ? 256 * TW : 0);  // [8][256]    raw panel byte -> coordinates z
    u64 *sX = sZ + 8 * 256;                // [8][256]    raw panel byte -> new panel word
    u64 *sO = sX + 8 * 256;                // [64][TW]    pivot rows, current tile
    u64 *sMap = sO + 64 * TW;              // [128]       zmap, xmap

    const int r = st->r_cur, kbar = st->kbar, nwin = st->nwin, nx = st->nx;
    const int M = m - r;
    if (M <= 0)
        return;
    const int tid = threadIdx.x;
    if (kbar == 0) {
        // no pivot: every trailing row's panel word is zero; word b + 1 is unchanged. Unless
        // the tail is already known to be zero, look for a nonzero word right of the panel
        // in any trailing row (none means no later panel has a pivot).
        const bool check = !st->zero_tail;
        bool nzw = false;
        for (int p = r + cta * NT + tid; p < m; p += ncta * NT) {
            const int ph = trailing_row(perm, st, r, nwin, nx, p);
            const uint64_t *row = A + (int64_t)ph * stride;
            A[(int64_t)ph * stride + b] = side_cur[ph];
            if (b + 1 < W) {
                const u64 v = row[b + 1];
                side_nxt[ph] = v;
                if (check) {
                    nzw = nzw || v != 0;
                    for (int w = b + 2; w < W && !nzw; ++w)
                        nzw = row[w] != 0;
                }
            }
        }
        if (__syncthreads_or(nzw) && tid == 0)
            atomicExch(const_cast<int *>(&st->nz), 1);
        return;
    }
    // tiles start on a 64-byte boundary (32 bytes for 4-word tiles), so a row-tile's
    // store covers whole DRAM atoms; words left of b - 1 in the first tile are skipped
    constexpr int WAL = TW;
    const int wstart = b & ~(WAL - 1);
    const int tiles = (W - wstart + TW - 1) / TW;
    constexpr int PASS = RPP * RPT;  // rows per pass of the CTA
    // Work: the tiles x (blocks of PASS rows) in tile-major order, cut into ncta
    // contiguous runs of equal length (to one block): every CTA is busy and a run
    // spans at most a few tiles, so the tables are rebuilt at most that often
    const int nblk = (M + PASS - 1) / PASS;
    const long long T = (long long)tiles * nblk;
    const long long q_lo = T * cta / ncta, q_hi = T * (cta + 1) / ncta;
    const int ng = (kbar + 7) >> 3;

    if (tid < 64)
        sMap[tid] = st->zmap[tid];
    else if (tid < 128)
        sMap[tid] = st->xmap[tid - 64];
    __syncthreads();
    for (int e = tid; e < 8 * 256; e += NT) {
        const int q = e >> 8, v = e & 255;
        u64 zz = 0, xx = 0;
#pragma unroll
        for (int bit = 0; bit < 8; ++bit)
            if ((v >> bit) & 1) {
                zz ^= sMap[8 * q + bit];
                xx ^= sMap[64 + 8 * q + bit];
            }
        sZ[e] = zz;
        sX[e] = xx;
    }
    const int sub = tid % TPR, rg = tid / TPR;
    const int lane = tid & 31;
    // lanes of one row form an aligned group of TPR lanes
    const unsigned gmask = (TPR == 32 ? GF2_FULL : ((1u << TPR) - 1u) << (lane & ~(TPR - 1)));
    int cur_tile = -1;
    for (long long q = q_lo; q < q_hi;) {
        const int tile = (int)(q / nblk);
        const long long q_end = min(q_hi, (long long)(tile + 1) * nblk);
        const int blk0 = (int)(q - (long long)tile * nblk), blk1 = (int)(q_end - (long long)tile * nblk);
        q = q_end;
        const int wbase = wstart + tile * TW;
        if (tile != cur_tile) {
            __syncthreads();
            for (int e = tid; e < 64 * TW; e += NT) {
                const int s2 = e / TW, wi = e % TW;
                u64 v = 0;
                if (s2 < kbar && wbase + wi < W)
                    v = A[(int64_t)st->prow[s2] * stride + wbase + wi];
                sO[e] = v;
            }
            __syncthreads();
            // MakeTable: entry hi << 4 | gray(i) from entry hi << 4 | gray(i - 1) by one row
            constexpr int HIB = HALF ? 3 : 4;  // high bits enumerated directly
            for (int e = tid; e < ng * TW * (1 << HIB); e += NT) {
                // word index fastest: the lanes of a warp store to consecutive words
                const int wi = e % TW, rest = e / TW, vh = rest & ((1 << HIB) - 1), g = rest >> HIB;
                const u64 *Og = sO + (8 * g) * TW + wi;
                u64 cur = 0;
#pragma unroll
                for (int bit = 0; bit < HIB; ++bit)
                    if ((vh >> bit) & 1)
                        cur ^= Og[(4 + bit) * TW];
                gray16(cur, Og[0], Og[TW], Og[2 * TW], Og[3 * TW], sT + (g * TE + (vh << 4)) * TW + wi, TW);
            }
            if (HALF)
                for (int e = tid; e < TW * 16; e += NT) {
                    const int wi = e % TW, vh = e / TW;
                    const u64 *O7 = sO + 7 * TW + wi;  // row 8 g + 7 at O7[8 g TW]
                    u64 cur = 0;
#pragma unroll
                    for (int bit = 0; bit < 4; ++bit)
                        if ((vh >> bit) & 1)
                            cur ^= O7[8 * (4 + bit) * TW];
                    gray16(cur, O7[0], O7[8 * TW], O7[16 * TW], O7[24 * TW], sU + (vh << 4) * TW + wi, TW);
                }
            __syncthreads();
            cur_tile = tile;
        }
        const int p_begin = r + blk0 * PASS;
        const int p_end = min(m, r + blk1 * PASS);
        const int w0 = wbase + 2 * sub;
        const bool two = w0 + 1 < W;
        const bool wact = w0 < W && w0 + 1 >= b;  // both words left of the panel: untouched
        // software pipeline over passes: the physical rows of the pass after next and
        // the words of the next pass are in flight while this pass is computed
        int ph[RPT], phB[RPT], phC[RPT];
        bool valid[RPT], validB[RPT], validC[RPT], isp[RPT], ispB[RPT], ispC[RPT];
        u64 wv[RPT], o0[RPT], o1[RPT], wvB[RPT], o0B[RPT], o1B[RPT];
        pass_rows<RPT, RPP>(p_begin, rg, p_end, r, kbar, nwin, nx, st, perm, ph, valid, isp);
        pass_loads<RPT>(A, stride, side_cur, w0, two, wact, ph, valid, isp, wv, o0, o1);
        pass_rows<RPT, RPP>(p_begin + PASS, rg, p_end, r, kbar, nwin, nx, st, perm, phB, validB, ispB);
        for (int pb = p_begin; pb < p_end; pb += PASS) {
            pass_rows<RPT, RPP>(pb + 2 * PASS, rg, p_end, r, kbar, nwin, nx, st, perm, phC, validC, ispC);
            pass_loads<RPT>(A, stride, side_cur, w0, two, wact, phB, validB, ispB, wvB, o0B, o1B);
            // (c) coordinates, table lookups, stores
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int p = pb + j * RPP + rg;
                u64 zz = 0;
                {
                    // this thread's BPL bytes of the panel word
                    const unsigned mine = (unsigned)(wv[j] >> (8 * BPL * sub));
#pragma unroll
                    for (int q = 0; q < BPL; ++q)
                        zz ^= sZ[((sub * BPL + q) << 8) | (int)((mine >> (8 * q)) & 255u)];
                }
#pragma unroll
                for (int o = 1; o < TPR; o <<= 1)
                    zz ^= __shfl_xor_sync(gmask, zz, o);
                const u64 z = isp[j] ? st->zpiv[p - r] : zz;
                const unsigned zw[2] = {(unsigned)z, (unsigned)(z >> 32)};
                u64 acc0 = 0, acc1 = 0;
                const u64 *tb0 = sT + 2 * sub;
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    if (g < ng) {
                        const int v = (int)((zw[g >> 2] >> (8 * (g & 3))) & (TE - 1u));
                        const ulonglong2 e2 = *reinterpret_cast<const ulonglong2 *>(tb0 + (g * TE + v) * TW);
                        acc0 ^= e2.x;
                        acc1 ^= e2.y;
                    }
                }
                if (HALF) {
                    // bits 7, 15, ..., 63 of z gathered into one byte
                    const unsigned top = ((((zw[0] >> 7) & 0x01010101u) * 0x01020408u) >> 24) |
                                         (((((zw[1] >> 7) & 0x01010101u) * 0x01020408u) >> 24) << 4);
                    const ulonglong2 e2 =
                        *reinterpret_cast<const ulonglong2 *>(sU + (int)(top & 255u) * TW + 2 * sub);
                    acc0 ^= e2.x;
                    acc1 ^= e2.y;
                }
                if (!valid[j] || !wact)
                    continue;
                if (isp[j]) {
                    // pivot row t = p - r: final row U_t, written in final position
                    if (out) {
                        uint64_t *o = out + (int64_t)p * ostride;
                        if (w0 >= b)
                            o[w0] = (w0 == b) ? st->newblk[p - r] : acc0;
                        if (two)
                            o[w0 + 1] = (w0 + 1 == b) ? st->newblk[p - r] : acc1;
                    }
                    continue;
                }
                u64 n0 = o0[j], n1 = o1[j];
                if (w0 == b || w0 + 1 == b) {
                    u64 nb = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        nb ^= sX[(q << 8) | (int)((wv[j] >> (8 * q)) & 255ull)];
                    if (w0 == b) {
                        n0 = nb;
                        n1 ^= acc1;
                    } else {
                        n1 = nb;  // word w0 = b-1 belongs to earlier panels
                    }
                } else {
                    n0 ^= acc0;
                    n1 ^= acc1;
                }
                // word b + 1 goes only to the next side buffer: the next pivot search reads
                // it in A (as it was before this panel) while this sweep runs, and the next
                // panel's sweep writes that word's final value
                uint64_t *a = A + (int64_t)ph[j] * stride + w0;
                if (w0 == b + 1) {
                    if (two)
                        a[1] = n1;
                } else if (w0 + 1 == b + 1) {
                    a[0] = n0;
                } else if (two) {
                    ulonglong2 v2;
                    v2.x = n0;
                    v2.y = n1;
                    *reinterpret_cast<ulonglong2 *>(a) = v2;
                } else {
                    a[0] = n0;
                }
                if (b + 1 < W) {
                    if (w0 == b + 1)
                        side_nxt[ph[j]] = n0;
                    else if (two && w0 + 1 == b + 1)
                        side_nxt[ph[j]] = n1;
                }
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                ph[j] = phB[j];
                valid[j] = validB[j];
                isp[j] = ispB[j];
                wv[j] = wvB[j];
                o0[j] = o0B[j];
                o1[j] = o1B[j];
                phB[j] = phC[j];
                validB[j] = validC[j];
                ispB[j] = ispC[j];
            }
        }
    }
}

template <int TW, int RPT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_sweep(uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ side_cur, u64 *__restrict__ side_nxt,
        const int *__restrict__ perm, const PanelState *__restrict__ st, uint64_t *__restrict__ out, int64_t ostride,
        int m, int W, int b)
{
    sweep_panel<TW, RPT, NT>(A, stride, side_cur, side_nxt, perm, st, out, ostride, m, W, b, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// final row order: out[p] <- A[perm[p]] for the words the sweep did not write
// (all words for p >= r, the words left of the pivot's panel for p < r),
// identity fill of P and Q beyond the rank, rank.
// ---------------------------------------------------------------------------
// Words [0, nw) of one row from src to dst by the 32 lanes of a warp, 16 bytes per access and up
// to four accesses of a lane in flight. Both rows start on a 16-byte boundary: matrices and the
// workspace are 128-byte aligned with strides of whole 128-byte lines, and the recursive PLS's
// column views start on an even word (its splits fall on multiples of 128 columns).
__device__ __forceinline__ void copy_words(uint64_t *__restrict__ dst, const uint64_t *__restrict__ src, int nw,
                                           int lane)
{
    const int n2 = nw >> 1;  // whole 16-byte pairs
    const ulonglong2 *__restrict__ s2 = reinterpret_cast<const ulonglong2 *>(src);
    ulonglong2 *__restrict__ d2 = reinterpret_cast<ulonglong2 *>(dst);
    int i = lane;
    for (; i + 96 < n2; i += 128) {
        const ulonglong2 a = s2[i], b = s2[i + 32], c = s2[i + 64], e = s2[i + 96];
        d2[i] = a;
        d2[i + 32] = b;
        d2[i + 64] = c;
        d2[i + 96] = e;
    }
    for (; i < n2; i += 32)
        d2[i] = s2[i];
    if ((nw & 1) && lane == 0)
        dst[nw - 1] = src[nw - 1];
}

__device__ __forceinline__ void gather_rows(const uint64_t *__restrict__ A, int64_t stride,
                                            const int *__restrict__ perm, const PanelState *__restrict__ st,
                                            int64_t *__restrict__ P, int64_t *__restrict__ Q,
                                            uint64_t *__restrict__ out, int64_t ostride, int m, int n, int W,
                                            int64_t *rank, int cta, int ncta)
{
    const int r = st->r_next;
    const int warps = ncta * (blockDim.x >> 5);
    const int wid = cta * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (out) {
        for (int p = wid; p < m; p += warps) {
            const int ph = perm[p];
            const int wend = p < r ? (int)(Q[p] >> 6) : W;
            copy_words(out + (int64_t)p * ostride, A + (int64_t)ph * stride, wend, lane);
        }
    }
    const int g = cta * blockDim.x + threadIdx.x;
    const int nt = ncta * blockDim.x;
    if (P)
        for (int i = r + g; i < m; i += nt)
            P[i] = i;
    if (Q)
        for (int i = r + g; i < n; i += nt)
            Q[i] = i;
    if (g == 0 && rank)
        *rank = r;
}

__global__ void k_gather(const uint64_t *__restrict__ A, int64_t stride, const int *__restrict__ perm,
                         const PanelState *__restrict__ st, int64_t *__restrict__ P, int64_t *__restrict__ Q,
                         uint64_t *__restrict__ out, int64_t ostride, int m, int n, int W, int64_t *rank)
{
    gather_rows(A, stride, perm, st, P, Q, out, ostride, m, n, W, rank, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void pivot_mask(const int64_t *__restrict__ Q, const PanelState *__restrict__ st,
                                           u64 *__restrict__ pmask, int cta, int ncta)
{
    const int r = st->r_next;
    for (int s = cta * blockDim.x + threadIdx.x; s < r; s += ncta * blockDim.x) {
        const int64_t c = Q[s];
        atomicOr(&pmask[c >> 6], 1ull << (c & 63));
    }
}

__global__ void k_pmask(const int64_t *__restrict__ Q, const PanelState *__restrict__ st, u64 *__restrict__ pmask)
{
    pivot_mask(Q, st, pmask, blockIdx.x, gridDim.x);
}

// Compress L: row i (t = min(i, r-1)) gets the bits of columns Q[c0..t] at
// positions c0..t, zeros up to Q[t], the rest unchanged (c0 = first s with
// Q[s] != s). This is the effect of swapping columns j and Q[j] from row j on
// for j = 0..r-1, done as one ordered bit extraction per row.
__device__ __forceinline__ void compress_row(uint64_t *__restrict__ out, int64_t stride,
                                             const int64_t *__restrict__ Q, const u64 *__restrict__ pmask,
                                             const PanelState *__restrict__ st, int m, int i)
{
    const int r = st->r_next;
    if (i >= m || r == 0)
        return;
    const int t = min(i, r - 1);
    const int64_t qt = Q[t];
    if (qt == t)
        return;
    int lo = 0, hi = t;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (Q[mid] != mid)
            hi = mid;
        else
            lo = mid + 1;
    }
    const int64_t c0 = lo;
    uint64_t *row = out + (int64_t)i * stride;
    int64_t pos = c0;
    int64_t cw = c0 >> 6;
    u64 cur = row[cw] & lowmask((int)(c0 & 63));
    const int64_t ew = qt >> 6;
    for (int64_t w = c0 >> 6; w <= ew; ++w) {
        const u64 word = row[w];
        u64 msk = pmask[w];
        if (w == (c0 >> 6))
            msk &= ~lowmask((int)(c0 & 63));
        if (w == ew)
            msk &= lowmask((int)(qt & 63) + 1);
        const u64 bits = pext64(word, msk);
        const int k = __popcll(msk);
        const int off = (int)(pos & 63);
        cur |= bits << off;
        if (off + k >= 64) {
            row[cw] = cur;
            ++cw;
            cur = off == 0 ? 0ull : (bits >> (64 - off));
        }
        pos += k;
    }
    while (cw <= ew) {
        if (cw == ew)
            row[cw] = cur | (row[cw] & ~lowmask((int)(qt & 63) + 1));
        else
            row[cw] = cur;
        cur = 0;
        ++cw;
    }
}

__global__ void k_compress(uint64_t *__restrict__ out, int64_t stride, const int64_t *__restrict__ Q,
                           const u64 *__restrict__ pmask, const PanelState *__restrict__ st, int m)
{
    compress_row(out, stride, Q, pmask, st, m, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_identity(int64_t *P, int64_t m, int64_t *Q, int64_t n, int64_t *rank)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    if (P)
        for (int64_t i = g; i < m; i += nt)
            P[i] = i;
    if (Q)
        for (int64_t i = g; i < n; i += nt)
            Q[i] = i;
    if (g == 0 && rank)
        *rank = 0;
}

template <int TW>
constexpr size_t sweep_smem()
{
    return (TW == 16 ? (size_t)(8 * 128 * TW + 256 * TW) : (size_t)(8 * 256 * TW)) * sizeof(u64) +
           (size_t)(2 * 8 * 256 + 64 * TW + 128) * sizeof(u64);
}

template <int TW, int RPT, int NT, int MINB>
int launch_sweep(const gf2::Elim &e, int b, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    constexpr size_t smem = sweep_smem<TW>();
    if (gf2::attr_needed(attr_devs)) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sweep<TW, RPT, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return gf2::note_cuda(err);
        gf2::attr_done(attr_devs);
    }
    const u64 *cur = e.side + (size_t)(b & 1) * e.m;
    u64 *nxt = e.side + (size_t)((b + 1) & 1) * e.m;
    const int tok = gf2::prof_begin(s);
    k_sweep<TW, RPT, NT, MINB><<<e.grid * MINB, NT, smem, s>>>(e.A, e.stride, cur, nxt, e.perm, e.st + (b & 1), e.out,
                                                               e.ostride, (int)e.m, (int)e.W, b);
    gf2::prof_end(s, GF2_PROF_SWEEP, tok);
    gf2::prof_launched(1);
    return gf2::note_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// batched elimination: the same panel steps over many matrices per launch
// ---------------------------------------------------------------------------
__global__ void k_init_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc d = D[blockIdx.y];
    const int g = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = g; i < d.m; i += nt) {
        d.perm[i] = i;
        if (d.W > 0)
            d.side[i] = d.A[(int64_t)i * d.stride];
    }
    for (int w = g; w < d.W + 1; w += nt)
        d.pmask[w] = 0;
    if (g < 2) {
        d.st[g].nwin = 0;
        d.st[g].nx = 0;
        d.st[g].r_cur = 0;
        d.st[g].r_next = 0;
        d.st[g].kbar = 0;
        d.st[g].status = 0;
        d.st[g].zero_tail = 0;
        d.st[g].nz = 0;
        d.st[g].J = 0;
        d.st[g].mode = 0;
        d.st[g].r_switch = 0;
        d.st[g].pop = 0;
    }
}

__global__ void __launch_bounds__(PIVOT_THREADS, 1) k_pivot_b(const gf2::ElimDesc *__restrict__ D, const int *__restrict__ idx, int b)
{
    const gf2::ElimDesc &d = D[idx[blockIdx.x]];
    const int nbits = min(64, d.n - 64 * b);
    pivot_panel(d.A + b, d.stride, d.side + (size_t)((b + 1) & 1) * d.m, 1, d.perm, d.st + ((b + 1) & 1), d.st + (b & 1),
                d.P, d.Q, d.m, b, nbits, 0, 0);
}

template <int TW, int RPT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_sweep_b(const gf2::ElimDesc *__restrict__ D, const int *__restrict__ idx, const int *__restrict__ pre, int nact, int b)
{
    // matrix j with pre[j] <= blockIdx.x < pre[j + 1]
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const gf2::ElimDesc &d = D[idx[lo]];
    sweep_panel<TW, RPT, NT>(d.A, d.stride, d.side + (size_t)(b & 1) * d.m, d.side + (size_t)((b + 1) & 1) * d.m,
                              d.perm, d.st + (b & 1), d.out, d.ostride, d.m, d.W, b, (int)blockIdx.x - pre[lo],
                              pre[lo + 1] - pre[lo]);
}

__global__ void k_apply_order_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc &d = D[blockIdx.y];
    apply_order(d.perm, gf2::final_state(d.st, d.W));
}

__global__ void k_gather_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc &d = D[blockIdx.y];
    gather_rows(d.A, d.stride, d.perm, gf2::final_state(d.st, d.W), d.P, d.Q, d.out, d.ostride, d.m, d.n, d.W, d.rank,
                blockIdx.x, gridDim.x);
}

__global__ void k_pmask_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc &d = D[blockIdx.y];
    pivot_mask(d.Q, gf2::final_state(d.st, d.W), d.pmask, blockIdx.x, gridDim.x);
}

__global__ void k_compress_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc &d = D[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.m)
        compress_row(d.out, d.ostride, d.Q, d.pmask, gf2::final_state(d.st, d.W), d.m, i);
}

// out -> A, one warp per row
__global__ void k_copyback_b(const gf2::ElimDesc *__restrict__ D)
{
    const gf2::ElimDesc &d = D[blockIdx.y];
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < d.m; i += warps)
        copy_words(d.A + (int64_t)i * d.stride, d.out + (int64_t)i * d.ostride, d.W, lane);
}

// ---------------------------------------------------------------------------
// Batched elimination in one persistent launch (cooperative: every CTA is
// resident). Teams of G CTAs eliminate one matrix at a time, panel by panel:
// the pivot search of panel b + 1 (the first PIVOT_THREADS threads of the
// team's first CTA) beside the table sweep of panel b (the other threads of all
// of the team's CTAs), with a team barrier after each step, then the finishing
// steps (row order, gather, compression of L, copy back). The large matrices go to teams of CTAs (a
// contiguous CTA range and a list of matrices per team, planned on the host);
// every CTA then takes small matrices one at a time from a device work queue,
// as a team of one.
// ---------------------------------------------------------------------------
struct PersistPlan {
    int nteams;
    const int *team_of;       // per CTA: its large-matrix team, or -1
    const int *team_start;    // per team: its first CTA ...
    const int *team_size;     // ... and its CTA count
    const int *team_first;    // team t's matrices: big[team_first[t] .. team_first[t + 1])
    const int *big;
    const int *small;         // matrices for single CTAs, largest first
    int nsmall;
    int *next_small;          // work-queue cursor into small (zero at launch)
    unsigned *bars;           // barrier counter of each team (zero at launch)
    int *abort;               // set when a barrier wait gave up (zero at launch)
    int *status;              // device status word
};

__device__ __forceinline__ unsigned ld_volatile(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Barrier of the G CTAs of a team (a plain CTA barrier for G = 1). The wait is bounded: one that
// gives up records GF2_ETIMEOUT and sets the abort flag, and every CTA then leaves.
__device__ __forceinline__ bool team_barrier(unsigned *bar, unsigned &target, int G, const PersistPlan &pl)
{
    __shared__ int s_ok;
    __syncthreads();
    if (G == 1)
        return true;
    if (threadIdx.x == 0) {
        target += (unsigned)G;
        __threadfence();
        atomicAdd(bar, 1u);
        const u64 t0 = globaltimer_ns();
        int ok = 1;
        while (ld_volatile(bar) < target) {
            if (*(volatile int *)pl.abort || globaltimer_ns() - t0 > GF2_WAIT_LIMIT_NS) {
                if (!*(volatile int *)pl.abort)
                    record_status(pl.status, GF2_ETIMEOUT);
                atomicExch(pl.abort, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole MMPF elimination of one matrix by CTA tr of a team of G.
__device__ bool team_eliminate(SweepSmem &S, const gf2::ElimDesc &d, int tr, int G, unsigned *bar, unsigned &target,
                               const PersistPlan &pl)
{
    const int tid = threadIdx.x;
    const int m = d.m, W = d.W;
    const int g0 = tr * NT + tid, gs = G * NT;
    for (int i = g0; i < m; i += gs) {
        d.perm[i] = i;
        if (W > 0)
            d.side[i] = d.A[(int64_t)i * d.stride];
    }
    for (int w = g0; w < W + 1; w += gs)
        d.pmask[w] = 0;
    if (tr == 0 && tid < 2) {
        PanelState &q = d.st[tid];
        q.nwin = q.nx = q.r_cur = q.r_next = q.kbar = q.status = q.zero_tail = q.nz = q.mode = 0;
        q.r_switch = 0;
        q.J = 0;
        q.pop = 0;
    }
    if (!team_barrier(bar, target, G, pl))
        return false;
    // pivot search of panel c by the first PIVOT_THREADS threads of the team's first CTA
    auto search = [&](int c) {
        pivot_panel(d.A + c, d.stride, d.side + (size_t)((c + 1) & 1) * m, 1, d.perm, d.st + ((c + 1) & 1),
                    d.st + (c & 1), d.P, d.Q, m, c, min(64, d.n - 64 * c), 0, 0);
    };
    if (W > 0 && tr == 0 && tid < PIVOT_THREADS)
        search(0);
    if (!team_barrier(bar, target, G, pl))
        return false;
    for (int b = 0; b < W; ++b) {
        // The search of panel b + 1 runs beside the sweep of panel b (the other warps of every CTA
        // of the team), as the two kernels do in the one-matrix elimination: it forms its window's
        // words from A's word b + 1, which this sweep leaves as it is, and panel b's coordinates
        // in the side buffer, which this sweep only reads; the rows whose order panel b changed
        // are read by the sweep from panel b's state, not from perm.
        if (tid < PIVOT_THREADS) {
            if (tr == 0 && b + 1 < W)
                search(b + 1);
        } else {
            sweep_panel16<0, 8, NT - PIVOT_THREADS, PIVOT_THREADS>(
                S, d.A, d.stride, d.side + (size_t)(b & 1) * m, d.side + (size_t)((b + 1) & 1) * m, d.perm,
                d.st + (b & 1), d.out, d.ostride, nullptr, m, W, b, tr, G);
        }
        if (!team_barrier(bar, target, G, pl))
            return false;
    }
    const PanelState *stf = gf2::final_state(d.st, W);
    if (tr == 0)
        apply_order(d.perm, stf);
    if (!team_barrier(bar, target, G, pl))
        return false;
    gather_rows(d.A, d.stride, d.perm, stf, d.P, d.Q, d.out, d.ostride, m, d.n, W, d.rank, tr, G);
    if (!team_barrier(bar, target, G, pl))
        return false;
    pivot_mask(d.Q, stf, d.pmask, tr, G);
    if (!team_barrier(bar, target, G, pl))
        return false;
    for (int i = g0; i < m; i += gs)
        compress_row(d.out, d.ostride, d.Q, d.pmask, stf, m, i);
    if (!team_barrier(bar, target, G, pl))
        return false;
    const int lane = tid & 31;
    for (int i = (tr * NT + tid) >> 5; i < m; i += gs >> 5)
        copy_words(d.A + (int64_t)i * d.stride, d.out + (int64_t)i * d.ostride, W, lane);
    return team_barrier(bar, target, G, pl);
}

__global__ void __launch_bounds__(NT, 1) k_batch_persist(const gf2::ElimDesc *__restrict__ D, PersistPlan pl)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SweepSmem &S = *reinterpret_cast<SweepSmem *>(smraw);
    __shared__ int s_item;
    const int cta = blockIdx.x;
    const int t = pl.team_of[cta];
    if (t >= 0) {
        const int G = pl.team_size[t], tr = cta - pl.team_start[t];
        unsigned target = 0;
        for (int k = pl.team_first[t]; k < pl.team_first[t + 1]; ++k)
            if (!team_eliminate(S, D[pl.big[k]], tr, G, pl.bars + t, target, pl))
                return;
    }
    for (;;) {
        if (threadIdx.x == 0)
            s_item = *(volatile int *)pl.abort ? pl.nsmall : atomicAdd(pl.next_small, 1);
        __syncthreads();
        const int k = s_item;
        __syncthreads();
        if (k >= pl.nsmall)
            return;
        unsigned target = 0;
        team_eliminate(S, D[pl.small[k]], 0, 1, nullptr, target, pl);
    }
}

}  // namespace

namespace gf2 {

// rows per pass of the batched sweep variants below (threads / threads per row)
int sweep_rows_per_pass(int tile_words) { return tile_words == 4 ? 512 / 2 : tile_words == 16 ? 1024 / 8 : 1024 / 4; }
int sweep_ctas_per_sm(int tile_words) { return tile_words == 4 ? 2 : 1; }

int batch_init(const ElimDesc *D, int count, int max_m, cudaStream_t s)
{
    if (count <= 0)
        return GF2_OK;
    const dim3 grid((unsigned)((max_m + 255) / 256 > 0 ? (max_m + 255) / 256 : 1), (unsigned)count);
    k_init_b<<<grid, 256, 0, s>>>(D);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int batch_pivot(const ElimDesc *D, const int *idx, int nact, int b, cudaStream_t s)
{
    if (nact <= 0)
        return GF2_OK;
    const int tok = prof_begin(s);
    k_pivot_b<<<nact, PIVOT_THREADS, 0, s>>>(D, idx, b);
    prof_end(s, GF2_PROF_PIVOT, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

template <int TW, int RPT, int NT, int MINB>
static int launch_sweep_b(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b,
                          cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    constexpr size_t smem = sweep_smem<TW>();
    if (attr_needed(attr_devs)) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sweep_b<TW, RPT, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return note_cuda(err);
        attr_done(attr_devs);
    }
    const int tok = prof_begin(s);
    k_sweep_b<TW, RPT, NT, MINB><<<total, NT, smem, s>>>(D, idx, pre, nact, b);
    prof_end(s, GF2_PROF_SWEEP, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int batch_sweep(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b, int tile_words,
                cudaStream_t s)
{
    if (nact <= 0 || total <= 0)
        return GF2_OK;
    return tile_words == 4    ? launch_sweep_b<4, 1, 512, 2>(D, idx, pre, nact, total, b, s)
           : tile_words == 16 ? launch_sweep_b<16, 1, 1024, 1>(D, idx, pre, nact, total, b, s)
                              : launch_sweep_b<8, 1, 1024, 1>(D, idx, pre, nact, total, b, s);
}

int batch_finish(const ElimDesc *D, int count, int max_m, cudaStream_t s)
{
    if (count <= 0)
        return GF2_OK;
    const unsigned gx = (unsigned)((max_m + 127) / 128 > 0 ? (max_m + 127) / 128 : 1);
    k_apply_order_b<<<dim3(1, (unsigned)count), 128, 0, s>>>(D);
    k_gather_b<<<dim3(gx < 8 ? gx : 8, (unsigned)count), 256, 0, s>>>(D);
    k_pmask_b<<<dim3(1, (unsigned)count), 256, 0, s>>>(D);
    k_compress_b<<<dim3(gx, (unsigned)count), 128, 0, s>>>(D);
    k_copyback_b<<<dim3(gx < 16 ? gx : 16, (unsigned)count), 256, 0, s>>>(D);
    prof_launched(5);
    return note_cuda(cudaGetLastError());
}

// One persistent, cooperative launch of the whole batch (k_batch_persist). The plan arrays are
// device memory: team_first (nteams + 1), big, small; the counters (next_small, bars[nteams],
// abort) are zeroed here before the launch.
int batch_persistent(const ElimDesc *D, int nteams, const PersistArrays &a, int nsmall, int *counters,
                     cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    const size_t smem = sizeof(SweepSmem);
    if (attr_needed(attr_devs)) {
        cudaError_t err = cudaFuncSetAttribute(k_batch_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return note_cuda(err);
        attr_done(attr_devs);
    }
    cudaError_t err = cudaMemsetAsync(counters, 0, (size_t)(nteams + 2) * sizeof(int), s);
    if (err != cudaSuccess)
        return note_cuda(err);
    PersistPlan pl{};
    pl.nteams = nteams;
    pl.team_of = a.team_of;
    pl.team_start = a.team_start;
    pl.team_size = a.team_size;
    pl.team_first = a.team_first;
    pl.big = a.big;
    pl.small = a.small;
    pl.nsmall = nsmall;
    pl.next_small = counters;
    pl.abort = counters + 1;
    pl.bars = reinterpret_cast<unsigned *>(counters + 2);
    pl.status = status_word();
    int dev = 0, nsm = 0, per_sm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess ||
        (err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persist, NT, smem)) != cudaSuccess)
        return note_cuda(err);
    if (per_sm < 1)
        return GF2_ENOMEM;  // the kernel does not fit on an SM
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nsm);  // one CTA per SM, all resident
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int tok = prof_begin(s);
    err = cudaLaunchKernelEx(&cfg, k_batch_persist, D, pl);
    prof_end(s, GF2_PROF_SWEEP, tok);
    prof_launched(1);
    return note_cuda(err);
}

int batch_persistent_grid()
{
    return sm_count();
}

int identity_perm(int *perm, int64_t m, cudaStream_t s)
{
    if (m <= 0)
        return GF2_OK;
    k_init<<<(int)((m + 255) / 256), 256, 0, s>>>(nullptr, 0, perm, nullptr, nullptr, (int)m);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int identity_fill(int64_t *P, int64_t m, int64_t *Q, int64_t n, int64_t *rank, cudaStream_t s)
{
    k_identity<<<64, 256, 0, s>>>(P, m, Q, n, rank);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

// Side streams for the look-ahead, created on first use. Per device: four
// handed out round robin, plus the origin and side stream of graph captures
// (used by one capture at a time).
struct SideStreams {
    std::mutex mu;
    cudaStream_t s[64][6] = {};
    unsigned next[64] = {};
};
static SideStreams g_side;

static int device_streams(cudaStream_t **out)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess)
        return note_cuda(err);
    if (dev < 0 || dev >= 64)
        return GF2_EINVAL;
    if (!g_side.s[dev][0])  // all at once, so that no later call creates one
        for (int k = 0; k < 6; ++k)
            if ((err = cudaStreamCreateWithFlags(&g_side.s[dev][k], cudaStreamNonBlocking)) != cudaSuccess)
                return note_cuda(err);
    *out = g_side.s[dev];
    return GF2_OK;
}

int side_stream(cudaStream_t *out)
{
    std::lock_guard<std::mutex> lock(g_side.mu);
    cudaStream_t *ds = nullptr;
    if (const int rc = device_streams(&ds))
        return rc;
    if (capturing_on_this_thread()) {
        *out = ds[5];
        return GF2_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    *out = ds[g_side.next[dev]++ & 3u];
    return GF2_OK;
}

int capture_streams(cudaStream_t *origin, cudaStream_t *side)
{
    std::lock_guard<std::mutex> lock(g_side.mu);
    cudaStream_t *ds = nullptr;
    if (const int rc = device_streams(&ds))
        return rc;
    *origin = ds[4];
    *side = ds[5];
    return GF2_OK;
}

// Panel elimination with a look-ahead of one panel. The pivot searches run on
// stream s, the table sweeps on the side stream t: the sweep of panel b starts
// when the pivot search of panel b is done and overlaps the pivot search of
// panel b + 1, which derives its window from A (current up to panel b - 1, so
// it waits for the sweep of panel b - 1) plus panel b's contribution. Panel
// states and side buffers alternate with the parity of b.
int elim_run(const Elim &e)
{
    ElimAux aux{};
    EventSet E;
    int rc;
    if ((rc = side_stream(&aux.side)) || (rc = E.create()))
        return rc;
    for (int i = 0; i < 3; ++i)
        aux.ev[i] = E.ev[i];
    return elim_run(e, aux);
}

int launch_pivot_pair(const Elim &e, int b, const u64 *wsrc, int64_t wstride, const u64 *side_prev,
                      int64_t side_stride, const PanelState *st_prev, PanelState *st, bool defer, bool programmatic,
                      cudaStream_t s)
{
    const int nbits = (int)((e.n - 64ll * b) < 64 ? (e.n - 64ll * b) : 64);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(PIVOT_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = programmatic ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int tok = prof_begin(s);
    int rc = note_cuda(cudaLaunchKernelEx(&cfg, k_pivot_pair, (const uint64_t *)wsrc, wstride, side_prev, side_stride,
                                          e.perm, st_prev, st, e.P, e.Q, (int)e.m, b, nbits, defer ? 1 : 0));
    prof_end(s, GF2_PROF_PIVOT, tok);
    prof_launched(1);
    return rc ? rc : note_cuda(cudaGetLastError());
}

int init_states(const Elim &e, int nstates)
{
    const int m = (int)e.m;
    k_init<<<(m + 255) / 256 > 0 ? (m + 255) / 256 : 1, 256, 0, e.s>>>(e.A, e.stride, e.perm, nullptr, e.st, m,
                                                                       nstates);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int apply_final_order(const Elim &e)
{
    k_apply_order<<<1, 128, 0, e.s>>>(e.perm, e.stf);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int elim_run(const Elim &e, const ElimAux &aux)
{
    if (e.pps == 2 && e.mode == 0)
        return elim_run_pair(e, aux);
    const int m = (int)e.m;
    k_init<<<(m + 255) / 256, 256, 0, e.s>>>(e.A, e.stride, e.perm, e.side, e.st, m);
    prof_launched(1);
    int rc = note_cuda(cudaGetLastError());
    if (rc || e.W == 0)
        return rc;
    cudaStream_t t = aux.side;
    cudaEvent_t ev_piv = aux.ev[0], ev_rest[2] = {aux.ev[1], aux.ev[2]};
    for (int b = 0; b < (int)e.W; ++b) {
        const int nbits = (int)((e.n - 64ll * b) < 64 ? (e.n - 64ll * b) : 64);
        const u64 *prev = e.side + (size_t)((b + 1) & 1) * e.m;  // panel word b - 1 of every row
        PanelState *stb = e.st + (b & 1);
        if (b >= 2 && (rc = note_cuda(cudaStreamWaitEvent(e.s, ev_rest[b & 1], 0))))
            return rc;
        const int tok = prof_begin(e.s);
        {
            // the previous panel's search is the preceding kernel on s: a programmatic
            // dependency lets this launch be scheduled before it completes (k_pivot waits)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1);
            cfg.blockDim = dim3(PIVOT_THREADS);
            cfg.stream = e.s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = b > 0 ? 1 : 0;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const PanelState *stp = e.st + ((b + 1) & 1);
            const int thr = e.hybrid_permille > 0 ? e.hybrid_permille : 150;
            rc = note_cuda(cudaLaunchKernelEx(&cfg, k_pivot, (const uint64_t *)e.A, e.stride, prev, e.perm, stp, stb,
                                              e.P, e.Q, m, b, nbits, e.mode, thr));
        }
        prof_end(e.s, GF2_PROF_PIVOT, tok);
        prof_launched(1);
        if (rc || (rc = note_cuda(cudaGetLastError())) || (rc = note_cuda(cudaEventRecord(ev_piv, e.s))) ||
            (rc = note_cuda(cudaStreamWaitEvent(t, ev_piv, 0))))
            return rc;
        rc = e.tile_words == 4   ? launch_sweep<4, 1, 512, 2>(e, b, t)
             : e.tile_words == 8 ? launch_sweep<8, 1, 1024, 1>(e, b, t)
                                 : launch_sweep16(e, b, t);
        if (rc || (rc = note_cuda(cudaEventRecord(ev_rest[b & 1], t))))
            return rc;
    }
    // the last panel's row order, then wait for the last sweep
    k_apply_order<<<1, 128, 0, e.s>>>(e.perm, e.stf);
    prof_launched(1);
    if ((rc = note_cuda(cudaGetLastError())))
        return rc;
    return note_cuda(cudaStreamWaitEvent(e.s, ev_rest[(e.W - 1) & 1], 0));
}

int elim_gather(const Elim &e, int64_t *rank)
{
    k_gather<<<2 * sm_count(), 256, 0, e.s>>>(e.A, e.stride, e.perm, e.stf, e.P, e.Q, e.out, e.ostride,
                                              (int)e.m, (int)e.n, (int)e.W, rank);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int pls_finish(const Elim &e)
{
    cudaError_t err = cudaMemsetAsync(e.pmask, 0, (size_t)e.W * sizeof(u64), e.s);
    if (err != cudaSuccess)
        return note_cuda(err);
    k_pmask<<<64, 256, 0, e.s>>>(e.Q, e.stf, e.pmask);
    k_compress<<<(int)((e.m + 127) / 128), 128, 0, e.s>>>(e.out, e.ostride, e.Q, e.pmask, e.stf, (int)e.m);
    prof_launched(2);
    int rc = note_cuda(cudaGetLastError());
    if (rc)
        return rc;
    err = cudaMemcpy2DAsync(e.A, (size_t)e.stride * 8, e.out, (size_t)e.ostride * 8, (size_t)e.W * 8,
                            (size_t)e.m, cudaMemcpyDeviceToDevice, e.s);
    return note_cuda(err);
}

}  // namespace gf2
