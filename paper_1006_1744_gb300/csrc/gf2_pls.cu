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

#include "gf2_common.cuh"

namespace {

constexpr int WIN = 128;   // rows held by the pivot warp (4 per lane)
constexpr int NSLOT = WIN / 32;

// ---------------------------------------------------------------------------
// initialisation: identity row order, panel word 0 of every row, state reset
// ---------------------------------------------------------------------------
__global__ void k_init(const uint64_t *__restrict__ A, int64_t stride, int *__restrict__ perm,
                       u64 *__restrict__ side0, PanelState *st, int m)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        perm[i] = i;
        side0[i] = A[(int64_t)i * stride];
    }
    if (i == 0) {
        st->r_cur = 0;
        st->r_next = 0;
        st->kbar = 0;
        st->status = 0;
        st->zero_tail = 0;
        st->J = 0;
    }
}

// ---------------------------------------------------------------------------
// Pivot search of panel b (one warp).
//
// Rows at positions >= r are candidates. Each holds its panel word w (as left
// by the previous panels), reduced by the pivots found so far in this panel.
// Pivot t is the smallest column j > j_{t-1} with a 1 in some candidate, and
// among those the candidate with the smallest position: exactly the rule of
// the Gaussian PLS algorithm restricted to this panel. The first WIN positions
// live in registers and are reduced incrementally; positions beyond are only
// scanned (reduced from scratch) when no windowed row has a 1 in the next
// column, which is rare for dense inputs.
//
// Bookkeeping per row: x = its multipliers (bit s: pivot s was added, i.e. the
// entry of L), z = its coordinates over the ORIGINAL panel words O of the
// pivot rows (reduced word = w + z.O). The pivots are also kept in
// Gauss-Jordan form V (1 at their own column, 0 at the other pivot columns),
// which gives, for any later row, its multipliers and coordinates straight
// from the bits of its raw panel word (zmap, xmap) -- the table sweep needs
// nothing else.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32, 1)
k_pivot(const u64 *__restrict__ side, int *__restrict__ perm, PanelState *st, int64_t *P,
        int64_t *Q, int m, int b, int nbits)
{
    // pivot records, written by the lane that held the pivot row
    __shared__ u64 sUw[64], sXp[64], sZp[64];
    __shared__ int sProw[64];
    // basis and column map, materialised only for scans past the window and at the end
    __shared__ u64 sVw[64], sVz[64], sVx[64];
    __shared__ int sC2P[64];
    __shared__ u64 sZm[64], sXm[64];

    const int lane = threadIdx.x;
    const int r = st->r_next;
    int t = 0;
    u64 J = 0;
    // basis rows s = lane (j = 0) and s = lane + 32 (j = 1), Gauss-Jordan form
    u64 vw[2] = {0, 0}, vz[2] = {0, 0}, vx[2] = {0, 0};
    int vc[2] = {0, 0};
    int pp[2] = {0, 0};  // P entries of pivots lane and lane + 32: position the row came from

    if (r < m && !st->zero_tail) {
        u64 w[NSLOT], z[NSLOT], x[NSLOT];
        int lab[NSLOT], ph[NSLOT], pt[NSLOT];  // pt: pivot index a slot became (-1: none)
        bool act[NSLOT];
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            int p = r + lane + 32 * k;
            pt[k] = -1;
            act[k] = p < m;
            lab[k] = p;
            ph[k] = act[k] ? perm[p] : -1;
            w[k] = act[k] ? side[ph[k]] : 0ull;
            z[k] = 0ull;
            x[k] = 0ull;
        }
        int jlow = 0;
        while (t < 64 && jlow < nbits && r + t < m) {
            // (1) windowed candidate with a 1 at column jlow and the smallest position;
            // key = (position - r) * 32 + lane, positions past the window collapse to WIN
            int key = INT_MAX, myk = 0;
            u64 tw = 0, tz = 0;
#pragma unroll
            for (int k = 0; k < NSLOT; ++k)
                if (act[k] && ((w[k] >> jlow) & 1ull)) {
                    const int rel = lab[k] - r;
                    const int kk = rel < WIN ? ((rel << 5) | lane) : (WIN << 5);
                    if (kk < key) {
                        key = kk;
                        myk = k;
                        tw = w[k];
                        tz = z[k];
                    }
                }
            const int best = __reduce_min_sync(GF2_FULL, key);
            int pc, plab, owner = -1;
            bool from_out = false;
            u64 pw = 0, ut = 0;
            if (best < (WIN << 5)) {
                // every position past the window is larger than one inside it
                pc = jlow;
                plab = r + (best >> 5);
                owner = best & 31;
            } else {
                // (2) slow path: materialise the basis for from-scratch reductions
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int sidx = lane + 32 * j;
                    if (sidx < t) {
                        sVw[sidx] = vw[j];
                        sVz[sidx] = vz[j];
                        sVx[sidx] = vx[j];
                        sC2P[vc[j]] = sidx;
                    }
                }
                __syncwarp();
                // (2a) smallest (column, position) among windowed rows (a windowed row
                // may carry a label past the window after an earlier swap)
                int myc = 64, mylab = INT_MAX, myk2 = 0;
#pragma unroll
                for (int k = 0; k < NSLOT; ++k) {
                    if (!act[k])
                        continue;
                    u64 mk = w[k] & ~lowmask(jlow);
                    int c = mk ? ctz64(mk) : 64;
                    if (c < myc || (c == myc && lab[k] < mylab)) {
                        myc = c;
                        mylab = lab[k];
                        myk2 = k;
                    }
                }
                const int cw = __reduce_min_sync(GF2_FULL, myc);
                int lw = __reduce_min_sync(GF2_FULL, myc == cw ? mylab : INT_MAX);
                if (cw == 64)
                    lw = INT_MAX;
                // (2b) rows past the window, reduced from scratch by the basis
                int bc = cw, bl = lw;
                u64 ow = 0, oz = 0, ox = 0;
                int oph = -1;
                for (int p0 = r + WIN; p0 < m && !(bc == jlow && p0 >= bl); p0 += 32) {
                    const int p = p0 + lane;
                    int c = 64, phh = -1;
                    u64 ww = 0, zz = 0, xx = 0;
                    if (p < m) {
                        phh = perm[p];
                        ww = side[phh];
                        u64 pm = ww & J;
                        while (pm) {
                            int cc = ctz64(pm);
                            pm &= pm - 1;
                            int sidx = sC2P[cc];
                            ww ^= sVw[sidx];
                            zz ^= sVz[sidx];
                            xx ^= sVx[sidx];
                        }
                        u64 mk = ww & ~lowmask(jlow);
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
                            oz = __shfl_sync(GF2_FULL, zz, src);
                            ox = __shfl_sync(GF2_FULL, xx, src);
                            oph = __shfl_sync(GF2_FULL, phh, src);
                        }
                    }
                }
                if (bc == 64)
                    break;  // no further pivot in this panel
                pc = bc;
                plab = bl;
                if (from_out) {
                    pw = ow;
                    ut = oz ^ (1ull << t);
                    if (lane == 0) {
                        sUw[t] = ow;
                        sXp[t] = ox;
                        sZp[t] = oz;
                        sProw[t] = oph;
                    }
                } else {
                    owner = __ffs(__ballot_sync(GF2_FULL, myc == cw && mylab == bl)) - 1;
                    myk = myk2;
#pragma unroll
                    for (int k = 0; k < NSLOT; ++k)
                        if (k == myk2) {
                            tw = w[k];
                            tz = z[k];
                        }
                }
            }
            if (!from_out) {
                // the owner's slot becomes pivot t; its registers stay frozen from now on and
                // its records are written after the loop
                pw = __shfl_sync(GF2_FULL, tw, owner);
                ut = __shfl_sync(GF2_FULL, tz, owner) ^ (1ull << t);
                const bool mine = lane == owner;
#pragma unroll
                for (int k = 0; k < NSLOT; ++k) {
                    const bool sel = mine && k == myk;
                    pt[k] = sel ? t : pt[k];
                    act[k] = act[k] && !sel;
                }
            }
            // (3) swap positions r+t and plab (logically)
            const int h = r + t;
            if (plab != h) {
#pragma unroll
                for (int k = 0; k < NSLOT; ++k)
                    if (act[k] && lab[k] == h) {
                        lab[k] = plab;
                        if (plab >= r + WIN)  // keep perm exact for later scans past the window
                            perm[plab] = ph[k];
                    }
            }
            // (4) Gauss-Jordan: clear column pc from the earlier basis rows, add row t
            const u64 tb = 1ull << t;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int sidx = lane + 32 * j;
                if (sidx < t && ((vw[j] >> pc) & 1ull)) {
                    vw[j] ^= pw;
                    vz[j] ^= ut;
                    vx[j] ^= tb;
                }
                if (sidx == t) {
                    vw[j] = pw;
                    vz[j] = ut;
                    vx[j] = tb;
                    vc[j] = pc;
                    pp[j] = plab;
                }
            }
            // (5) reduce the windowed candidates
#pragma unroll
            for (int k = 0; k < NSLOT; ++k)
                if (act[k] && ((w[k] >> pc) & 1ull)) {
                    w[k] ^= pw;
                    z[k] ^= ut;
                    x[k] |= tb;
                }
            J |= 1ull << pc;
            jlow = pc + 1;
            ++t;
        }
        // records of the pivots taken from the window (pivots from past the window were
        // recorded by lane 0 when they were found); the row of pivot t sits at position r+t
#pragma unroll
        for (int k = 0; k < NSLOT; ++k)
            if (pt[k] >= 0) {
                sUw[pt[k]] = w[k];
                sXp[pt[k]] = x[k];
                sZp[pt[k]] = z[k];
                sProw[pt[k]] = ph[k];
            }
        __syncwarp();
        // row order of the window back to memory
#pragma unroll
        for (int k = 0; k < NSLOT; ++k)
            if (act[k])
                perm[lab[k]] = ph[k];
        for (int s = lane; s < t; s += 32)
            perm[r + s] = sProw[s];
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (P && lane + 32 * j < t)
                P[r + lane + 32 * j] = pp[j];
    }
    // maps for the sweep: column c -> coordinates / multipliers of the basis row with its 1 at c
    sZm[lane] = 0;
    sZm[lane + 32] = 0;
    sXm[lane] = 0;
    sXm[lane + 32] = 0;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int sidx = lane + 32 * j;
        if (sidx < t) {
            sZm[vc[j]] = vz[j];
            sXm[vc[j]] = pdep64(vx[j], J);
            st->pcol[sidx] = vc[j];
            if (Q)
                Q[r + sidx] = 64ll * b + vc[j];
        }
    }
    __syncwarp();
    for (int c = lane; c < 64; c += 32) {
        st->zmap[c] = sZm[c];
        st->xmap[c] = sXm[c];
    }
    for (int s = lane; s < t; s += 32) {
        st->prow[s] = sProw[s];
        st->zpiv[s] = sZp[s] ^ (1ull << s);
        st->newblk[s] = sUw[s] | pdep64(sXp[s], J);
    }
    if (lane == 0) {
        st->r_cur = r;
        st->kbar = t;
        st->r_next = r + t;
        st->J = J;
    }
}

// ---------------------------------------------------------------------------
// Table sweep of panel b (MakeTable1 + AddRowsFromTable).
//
// For a row at position p >= r+kbar with raw panel word w:
//   z       = coordinates of w over the original pivot words O (8 lookups in
//             the byte tables ZT built from zmap),
//   panel   = its multipliers scattered to the pivot columns (byte tables XT),
//   trailing words ^= z.O (8 lookups, one Gray-code table per 8 pivots).
// Pivot row t gets its final row U_t = zpiv[t].O, written to `out` at its
// final position (pivot rows are never modified in A, so the tables can be
// built from A while the sweep runs). The CTA holding word b+1 also stores it
// in the next panel's side buffer.
//
// Work: column tiles of TW words (from the even word <= b) x row chunks; a
// CTA keeps its tables while consecutive work items share a tile.
// ---------------------------------------------------------------------------
template <int TW, int RPT, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_sweep(uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ side_cur,
        u64 *__restrict__ side_nxt, const int *__restrict__ perm, const PanelState *__restrict__ st,
        uint64_t *__restrict__ out, int64_t ostride, int m, int W, int b)
{
    constexpr int TPR = TW / 2;     // threads per row, two words each
    constexpr int RPP = 256 / TPR;  // rows per thread slot and pass
    constexpr int BPL = 8 / TPR;    // z-table bytes per thread
    extern __shared__ __align__(16) u64 sm[];
    u64 *sT = sm;                 // [8][256][TW]  Gray-code tables of the pivot rows
    u64 *sZ = sT + 8 * 256 * TW;  // [8][256]      raw panel byte -> coordinates z
    u64 *sX = sZ + 8 * 256;       // [8][256]      raw panel byte -> new panel word
    u64 *sO = sX + 8 * 256;       // [64][TW]      pivot rows, current tile
    u64 *sMap = sO + 64 * TW;     // [128]         zmap, xmap

    const int r = st->r_cur, kbar = st->kbar;
    const int M = m - r;
    if (M <= 0)
        return;
    const int tid = threadIdx.x;
    if (kbar == 0) {
        if (b + 1 < W)
            for (int p = r + blockIdx.x * 256 + tid; p < m; p += gridDim.x * 256) {
                int ph = perm[p];
                side_nxt[ph] = A[(int64_t)ph * stride + b + 1];
            }
        return;
    }
    const int wstart = b & ~1;
    const int tiles = (W - wstart + TW - 1) / TW;
    constexpr int PASS = RPP * RPT;  // rows per pass of the CTA
    int chunks = gridDim.x / tiles;
    if (chunks < 1)
        chunks = 1;
    int R = (M + chunks - 1) / chunks;
    R = (R + PASS - 1) / PASS * PASS;
    chunks = (M + R - 1) / R;
    const int items = tiles * chunks;
    const int ng = (kbar + 7) >> 3;

    if (tid < 64)
        sMap[tid] = st->zmap[tid];
    else if (tid < 128)
        sMap[tid] = st->xmap[tid - 64];
    __syncthreads();
    for (int e = tid; e < 8 * 256; e += 256) {
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
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item / chunks, chunk = item % chunks;
        const int wbase = wstart + tile * TW;
        if (tile != cur_tile) {
            __syncthreads();
            for (int e = tid; e < 64 * TW; e += 256) {
                const int s = e / TW, wi = e % TW;
                u64 v = 0;
                if (s < kbar && wbase + wi < W)
                    v = A[(int64_t)st->prow[s] * stride + wbase + wi];
                sO[e] = v;
            }
            __syncthreads();
            for (int e = tid; e < ng * TW * 16; e += 256) {
                const int vh = e & 15, gw = e >> 4, wi = gw % TW, g = gw / TW;
                const u64 *Og = sO + (8 * g) * TW + wi;
                u64 cur = 0;
#pragma unroll
                for (int bit = 0; bit < 4; ++bit)
                    if ((vh >> bit) & 1)
                        cur ^= Og[(4 + bit) * TW];
                u64 *Tg = sT + (g * 256 + (vh << 4)) * TW + wi;
                Tg[0] = cur;
#pragma unroll
                for (int i = 1; i < 16; ++i) {
                    cur ^= Og[(__ffs(i) - 1) * TW];
                    Tg[(i ^ (i >> 1)) * TW] = cur;
                }
            }
            __syncthreads();
            cur_tile = tile;
        }
        const int p_begin = r + chunk * R;
        const int p_end = min(m, p_begin + R);
        const int w0 = wbase + 2 * sub;
        const bool two = w0 + 1 < W;
        const bool wact = w0 < W;
        for (int pb = p_begin; pb < p_end; pb += PASS) {
            int ph[RPT];
            bool valid[RPT], isp[RPT];
            u64 wv[RPT], o0[RPT], o1[RPT];
            // (a) rows of this pass: position -> physical row
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int p = pb + j * RPP + rg;
                valid[j] = p < p_end;
                isp[j] = valid[j] && p < r + kbar;
                ph[j] = !valid[j] ? 0 : (isp[j] ? st->prow[p - r] : perm[p]);
            }
            // (b) their panel words and current words of the tile, all in flight
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
            // (c) coordinates, table lookups, stores
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int p = pb + j * RPP + rg;
                u64 zz = 0;
#pragma unroll
                for (int q = sub * BPL; q < (sub + 1) * BPL; ++q)
                    zz ^= sZ[(q << 8) | (int)((wv[j] >> (8 * q)) & 255ull)];
#pragma unroll
                for (int o = 1; o < TPR; o <<= 1)
                    zz ^= __shfl_xor_sync(gmask, zz, o);
                const u64 z = isp[j] ? st->zpiv[p - r] : zz;
                u64 acc0 = 0, acc1 = 0;
                for (int g = 0; g < ng; ++g) {
                    const int v = (int)((z >> (8 * g)) & 255ull);
                    const ulonglong2 e2 = *reinterpret_cast<const ulonglong2 *>(sT + (g * 256 + v) * TW + 2 * sub);
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
                uint64_t *a = A + (int64_t)ph[j] * stride + w0;
                if (two) {
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
        }
    }
}

// ---------------------------------------------------------------------------
// final row order: out[p] <- A[perm[p]] for the words the sweep did not write
// (all words for p >= r, the words left of the pivot's panel for p < r),
// identity fill of P and Q beyond the rank, rank.
// ---------------------------------------------------------------------------
__global__ void k_gather(const uint64_t *__restrict__ A, int64_t stride, const int *__restrict__ perm,
                         const PanelState *__restrict__ st, int64_t *__restrict__ P,
                         int64_t *__restrict__ Q, uint64_t *__restrict__ out, int64_t ostride, int m,
                         int n, int W, int64_t *rank)
{
    const int r = st->r_next;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (out) {
        for (int p = wid; p < m; p += warps) {
            const int ph = perm[p];
            const int wend = p < r ? (int)(Q[p] >> 6) : W;
            const uint64_t *src = A + (int64_t)ph * stride;
            uint64_t *dst = out + (int64_t)p * ostride;
            for (int w = lane; w < wend; w += 32)
                dst[w] = src[w];
        }
    }
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = gridDim.x * blockDim.x;
    if (P)
        for (int i = r + g; i < m; i += nt)
            P[i] = i;
    if (Q)
        for (int i = r + g; i < n; i += nt)
            Q[i] = i;
    if (g == 0 && rank)
        *rank = r;
}

__global__ void k_pmask(const int64_t *__restrict__ Q, const PanelState *__restrict__ st,
                        u64 *__restrict__ pmask)
{
    const int r = st->r_next;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < r; s += gridDim.x * blockDim.x) {
        const int64_t c = Q[s];
        atomicOr(&pmask[c >> 6], 1ull << (c & 63));
    }
}

// Compress L: row i (t = min(i, r-1)) gets the bits of columns Q[c0..t] at
// positions c0..t, zeros up to Q[t], the rest unchanged (c0 = first s with
// Q[s] != s). This is the effect of swapping columns j and Q[j] from row j on
// for j = 0..r-1, done as one ordered bit extraction per row.
__global__ void k_compress(uint64_t *__restrict__ out, int64_t stride, const int64_t *__restrict__ Q,
                           const u64 *__restrict__ pmask, const PanelState *__restrict__ st, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
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
    return (size_t)(8 * 256 * TW + 2 * 8 * 256 + 64 * TW + 128) * sizeof(u64);
}

template <int TW, int RPT, int MINB>
int launch_sweep(const gf2::Elim &e, int b)
{
    static bool attr_set = false;  // per process; the attribute is per function
    constexpr size_t smem = sweep_smem<TW>();
    if (!attr_set) {
        cudaError_t err = cudaFuncSetAttribute(k_sweep<TW, RPT, MINB>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return gf2::note_cuda(err);
        attr_set = true;
    }
    const u64 *cur = e.side + (size_t)(b & 1) * e.m;
    u64 *nxt = e.side + (size_t)((b + 1) & 1) * e.m;
    const int tok = gf2::prof_begin(e.s);
    k_sweep<TW, RPT, MINB><<<e.grid * MINB, 256, smem, e.s>>>(e.A, e.stride, cur, nxt, e.perm, e.st, e.out,
                                                              e.ostride, (int)e.m, (int)e.W, b);
    gf2::prof_end(e.s, GF2_PROF_SWEEP, tok);
    gf2::prof_launched(1);
    return gf2::note_cuda(cudaGetLastError());
}

}  // namespace

namespace gf2 {

int identity_fill(int64_t *P, int64_t m, int64_t *Q, int64_t n, int64_t *rank, cudaStream_t s)
{
    k_identity<<<64, 256, 0, s>>>(P, m, Q, n, rank);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int elim_run(const Elim &e)
{
    const int m = (int)e.m;
    k_init<<<(m + 255) / 256, 256, 0, e.s>>>(e.A, e.stride, e.perm, e.side, e.st, m);
    prof_launched(1);
    int rc = note_cuda(cudaGetLastError());
    if (rc)
        return rc;
    for (int b = 0; b < (int)e.W; ++b) {
        const int nbits = (int)((e.n - 64ll * b) < 64 ? (e.n - 64ll * b) : 64);
        const int tok = prof_begin(e.s);
        k_pivot<<<1, 32, 0, e.s>>>(e.side + (size_t)(b & 1) * e.m, e.perm, e.st, e.P, e.Q, m, b, nbits);
        prof_end(e.s, GF2_PROF_PIVOT, tok);
        prof_launched(1);
        rc = note_cuda(cudaGetLastError());
        if (rc)
            return rc;
        rc = e.tile_words == 4 ? launch_sweep<4, 4, 2>(e, b) : launch_sweep<8, 4, 1>(e, b);
        if (rc)
            return rc;
    }
    return GF2_OK;
}

int elim_gather(const Elim &e, int64_t *rank)
{
    k_gather<<<2 * sm_count(), 256, 0, e.s>>>(e.A, e.stride, e.perm, e.st, e.P, e.Q, e.out, e.ostride,
                                              (int)e.m, (int)e.n, (int)e.W, rank);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int pls_finish(const Elim &e)
{
    cudaError_t err = cudaMemsetAsync(e.pmask, 0, (size_t)e.W * sizeof(u64), e.s);
    if (err != cudaSuccess)
        return note_cuda(err);
    k_pmask<<<64, 256, 0, e.s>>>(e.Q, e.st, e.pmask);
    k_compress<<<(int)((e.m + 127) / 128), 128, 0, e.s>>>(e.out, e.ostride, e.Q, e.pmask, e.st, (int)e.m);
    prof_launched(2);
    int rc = note_cuda(cudaGetLastError());
    if (rc)
        return rc;
    err = cudaMemcpy2DAsync(e.A, (size_t)e.stride * 8, e.out, (size_t)e.ostride * 8, (size_t)e.W * 8,
                            (size_t)e.m, cudaMemcpyDeviceToDevice, e.s);
    return note_cuda(err);
}

}  // namespace gf2
