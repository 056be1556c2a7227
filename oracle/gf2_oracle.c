/*
 * gf2_oracle.c -- plain, slow CPU reference for the GF(2) decompositions of
 * Albrecht & Pernet, "Efficient Decomposition of Dense Matrices over GF(2)".
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or constant with the CUDA library, and neither includes the other.
 *
 * Matrix layout: row-major uint64 words; column j of row i is bit (j & 63) of
 * word A[i*stride + (j >> 6)] (least significant bit = leftmost column).
 * Bits at columns >= n are zero on input and stay zero.
 *
 * Entry points and the passage each one follows:
 *   gf2o_pls      -- Gaussian PLS decomposition (appendix algorithm "Gaussian
 *                    PLS Decomposition", Sec. 4 intro): the definition the
 *                    other methods must reproduce exactly.
 *   gf2o_rref     -- classical Gauss-Jordan elimination to reduced row echelon
 *                    form (Sec. 3, Definition "Reduced Row Echelon Form").
 *   gf2o_mul      -- C (+)= A.B by the definition of the matrix product.
 *   gf2o_make_table / gf2o_add_rows_from_table -- Algorithms MakeTable,
 *                    MakeTable1 and AddRowsFromTable (Sec. 3.1, Sec. 4.1).
 *   gf2o_pls_mmpf -- Algorithm MMPF with PlsSubmatrix (Sec. 4.1, appendix).
 *   gf2o_pls_rec  -- Algorithm "PLS Decomposition" (Sec. 5), recursive, with
 *                    MMPF as the base case below a column cutoff (Sec. 6).
 *   gf2o_m4ri     -- Algorithm M4RI with GaussSubmatrix (Sec. 3.1, appendix):
 *                    the reduced row echelon form without PLS.
 *
 * Readings of the paper where it is garbled or silent (each listed in the
 * design notes): swap vectors P, Q (transpositions i <-> P[i] applied in
 * increasing i); identity fill of P and Q beyond the rank; MakeTable enumerates
 * T[i] = T[i-1] + (one row) in Gray-code order; table ids are read big-endian
 * over the k columns; the recursive algorithm's typos are read as
 * "if r0 > 0", "P[r0+i]", "0 <= i < n0" and "j <- j+1".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* word-level helpers (Gaussian PLS, Gauss-Jordan, product)                */
/* ---------------------------------------------------------------------- */

static int getb(const uint64_t *A, int64_t s, int64_t i, int64_t j)
{
    return (int)((A[i * s + (j >> 6)] >> (j & 63)) & 1u);
}

static void setb(uint64_t *A, int64_t s, int64_t i, int64_t j, int v)
{
    uint64_t bit = (uint64_t)1 << (j & 63);
    if (v)
        A[i * s + (j >> 6)] |= bit;
    else
        A[i * s + (j >> 6)] &= ~bit;
}

/* row dst ^= row src, on columns c .. n-1 only */
static void add_row_from(uint64_t *A, int64_t s, int64_t n, int64_t dst, int64_t src, int64_t c)
{
    if (c >= n)
        return;
    int64_t W = (n + 63) >> 6, w0 = c >> 6;
    uint64_t *d = A + dst * s;
    const uint64_t *p = A + src * s;
    d[w0] ^= p[w0] & (~(uint64_t)0 << (c & 63));
    for (int64_t w = w0 + 1; w < W; ++w)
        d[w] ^= p[w];
}

static void swap_rows(uint64_t *A, int64_t s, int64_t n, int64_t a, int64_t b)
{
    if (a == b)
        return;
    int64_t W = (n + 63) >> 6;
    for (int64_t w = 0; w < W; ++w) {
        uint64_t t = A[a * s + w];
        A[a * s + w] = A[b * s + w];
        A[b * s + w] = t;
    }
}

/* swap columns a and b in rows row0 .. m-1 */
static void swap_cols_from(uint64_t *A, int64_t s, int64_t m, int64_t a, int64_t b, int64_t row0)
{
    if (a == b)
        return;
    for (int64_t i = row0; i < m; ++i) {
        int va = getb(A, s, i, a), vb = getb(A, s, i, b);
        setb(A, s, i, a, vb);
        setb(A, s, i, b, va);
    }
}

/*
 * Gaussian PLS decomposition, in place. Pivot search: the leftmost column
 * j >= c holding a 1 in some row i >= r, and the first such row. Swap it to
 * row r, then add row r to every later row with a 1 in column j, starting at
 * column j+1 so that the 1 (the entry of L) stays. At the end P and Q are
 * identity-filled beyond the rank and L is compressed by swapping columns j
 * and Q[j] in rows >= j. Returns the rank r.
 */
int64_t gf2o_pls(uint64_t *A, int64_t m, int64_t n, int64_t s, int64_t *P, int64_t *Q)
{
    int64_t r = 0, c = 0;
    while (r < m && c < n) {
        int64_t pi = -1, pj = -1;
        for (int64_t j = c; j < n && pi < 0; ++j) {
            for (int64_t i = r; i < m; ++i) {
                if (getb(A, s, i, j)) {
                    pi = i;
                    pj = j;
                    break;
                }
            }
        }
        if (pi < 0)
            break;
        P[r] = pi;
        Q[r] = pj;
        swap_rows(A, s, n, r, pi);
        if (pj + 1 < n) {
            for (int64_t l = r + 1; l < m; ++l)
                if (getb(A, s, l, pj))
                    add_row_from(A, s, n, l, r, pj + 1);
        }
        r += 1;
        c = pj + 1;
    }
    for (int64_t i = r; i < m; ++i)
        P[i] = i;
    for (int64_t i = r; i < n; ++i)
        Q[i] = i;
    for (int64_t j = 0; j < r; ++j)
        swap_cols_from(A, s, m, j, Q[j], j);
    return r;
}

/*
 * The same Gaussian PLS, timed as the all-cores CPU baseline: within each
 * pivot step the rows below the pivot are independent, and so are the rows
 * during the final column swaps, so those two loops are spread over threads
 * when the file is compiled with OpenMP (liboracle_gf2_omp.so). The result is
 * gf2o_pls's, bit for bit; compiled without OpenMP it is gf2o_pls.
 */
int64_t gf2o_pls_omp(uint64_t *A, int64_t m, int64_t n, int64_t s, int64_t *P, int64_t *Q)
{
    int64_t r = 0, c = 0;
    while (r < m && c < n) {
        int64_t pi = -1, pj = -1;
        for (int64_t j = c; j < n && pi < 0; ++j) {
            for (int64_t i = r; i < m; ++i) {
                if (getb(A, s, i, j)) {
                    pi = i;
                    pj = j;
                    break;
                }
            }
        }
        if (pi < 0)
            break;
        P[r] = pi;
        Q[r] = pj;
        swap_rows(A, s, n, r, pi);
        if (pj + 1 < n) {
#pragma omp parallel for schedule(static)
            for (int64_t l = r + 1; l < m; ++l)
                if (getb(A, s, l, pj))
                    add_row_from(A, s, n, l, r, pj + 1);
        }
        r += 1;
        c = pj + 1;
    }
    for (int64_t i = r; i < m; ++i)
        P[i] = i;
    for (int64_t i = r; i < n; ++i)
        Q[i] = i;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < r && j <= i; ++j)
            if (Q[j] != j) {
                int va = getb(A, s, i, j), vb = getb(A, s, i, Q[j]);
                setb(A, s, i, j, vb);
                setb(A, s, i, Q[j], va);
            }
    return r;
}

/*
 * Gauss-Jordan elimination to reduced row echelon form, in place. For each
 * column left to right: take the first row >= r with a 1, swap it to row r,
 * and clear the column in every other row. Row r is zero left of column j at
 * that point, so the addition may start at column j. Rows >= rank end zero.
 * pivots (nullable, length >= rank) receives the pivot columns.
 */
int64_t gf2o_rref(uint64_t *A, int64_t m, int64_t n, int64_t s, int64_t *pivots)
{
    int64_t r = 0;
    for (int64_t j = 0; j < n && r < m; ++j) {
        int64_t pi = -1;
        for (int64_t i = r; i < m; ++i) {
            if (getb(A, s, i, j)) {
                pi = i;
                break;
            }
        }
        if (pi < 0)
            continue;
        swap_rows(A, s, n, r, pi);
        for (int64_t l = 0; l < m; ++l)
            if (l != r && getb(A, s, l, j))
                add_row_from(A, s, n, l, r, j);
        if (pivots)
            pivots[r] = j;
        r += 1;
    }
    return r;
}

/*
 * C = A.B (acc == 0) or C = C + A.B (acc != 0), A m x k, B k x n, C m x n:
 * row i of the product is the sum of the rows l of B with A[i,l] = 1.
 */
void gf2o_mul(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B,
              int64_t sb, int64_t m, int64_t k, int64_t n, int acc)
{
    int64_t W = (n + 63) >> 6;
    for (int64_t i = 0; i < m; ++i) {
        uint64_t *ci = C + i * sc;
        if (!acc)
            memset(ci, 0, (size_t)W * sizeof(uint64_t));
        for (int64_t l = 0; l < k; ++l) {
            if (getb(A, sa, i, l)) {
                const uint64_t *bl = B + l * sb;
                for (int64_t w = 0; w < W; ++w)
                    ci[w] ^= bl[w];
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* bit-level views (SubMatrix of Sec. 5) for the literal MMPF and PLS      */
/* ---------------------------------------------------------------------- */

typedef struct {
    uint64_t *base;
    int64_t s;      /* stride of the underlying matrix, words */
    int64_t r0, c0; /* offset of the view */
    int64_t m, n;   /* size of the view */
} view_t;

static view_t sub(view_t v, int64_t rs, int64_t cs, int64_t m, int64_t n)
{
    view_t w = v;
    w.r0 = v.r0 + rs;
    w.c0 = v.c0 + cs;
    w.m = m;
    w.n = n;
    return w;
}

static int vget(view_t v, int64_t i, int64_t j)
{
    return getb(v.base, v.s, v.r0 + i, v.c0 + j);
}

static void vset(view_t v, int64_t i, int64_t j, int b)
{
    setb(v.base, v.s, v.r0 + i, v.c0 + j, b);
}

/* view row dst += view row src on view columns from .. n-1 */
static void vadd_row(view_t v, int64_t dst, int64_t src, int64_t from)
{
    for (int64_t j = from; j < v.n; ++j)
        if (vget(v, src, j))
            vset(v, dst, j, !vget(v, dst, j));
}

/* row dst of view d += row src of view e, columns from .. n-1 (same n) */
static void vadd_row2(view_t d, int64_t dst, view_t e, int64_t src, int64_t from)
{
    for (int64_t j = from; j < d.n; ++j)
        if (vget(e, src, j))
            vset(d, dst, j, !vget(d, dst, j));
}

static void vswap_rows(view_t v, int64_t a, int64_t b)
{
    if (a == b)
        return;
    for (int64_t j = 0; j < v.n; ++j) {
        int x = vget(v, a, j), y = vget(v, b, j);
        vset(v, a, j, y);
        vset(v, b, j, x);
    }
}

static void vswap_cols_from(view_t v, int64_t a, int64_t b, int64_t row0)
{
    if (a == b)
        return;
    for (int64_t i = row0; i < v.m; ++i) {
        int x = vget(v, i, a), y = vget(v, i, b);
        vset(v, i, a, y);
        vset(v, i, b, x);
    }
}

/* k bits of view row i at columns c .. c+k-1, read big-endian */
static int64_t vid(view_t v, int64_t i, int64_t c, int k)
{
    int64_t id = 0;
    for (int t = 0; t < k; ++t)
        id |= (int64_t)vget(v, i, c + t) << (k - 1 - t);
    return id;
}

/*
 * MakeTable / MakeTable1. U holds k rows (rows 0..k-1 of the view). T (a
 * 2^k x U.n view) receives, in Gray-code order, T[0] = 0 and
 * T[i] = T[i-1] + U[k-1-b] from column c on, where b is the bit that flips
 * between the Gray codes of i-1 and i; L[id] = i for the id (big-endian k
 * bits at column c) of T[i]. With fix (MakeTable1) the a-priori id of T[i],
 * i.e. which rows of U it sums (row t <-> Gray bit k-1-t), is then added onto
 * its first k bits, so that AddRowsFromTable writes the multipliers.
 */
static void vmake_table(view_t U, int k, int64_t c, int fix, view_t T, int64_t *L)
{
    int64_t N = (int64_t)1 << k;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < T.n; ++j)
            vset(T, i, j, 0);
    for (int64_t i = 1; i < N; ++i) {
        int b = __builtin_ctzll((unsigned long long)i);
        int64_t row = k - 1 - b;
        for (int64_t j = c; j < T.n; ++j)
            vset(T, i, j, vget(T, i - 1, j) ^ vget(U, row, j));
    }
    for (int64_t i = 0; i < N; ++i)
        L[vid(T, i, c, k)] = i;
    if (fix) {
        for (int64_t i = 1; i < N; ++i) {
            int64_t g = i ^ (i >> 1);
            for (int t = 0; t < k; ++t) {
                int bt = (int)((g >> (k - 1 - t)) & 1);
                vset(T, i, c + t, vget(T, i, c + t) ^ bt);
            }
        }
    }
}

/* AddRowsFromTable: rows rs .. re-1 of A get T[L[id]] added from column c. */
static void vadd_rows_from_table(view_t A, int64_t rs, int64_t re, int64_t c, int k, view_t T,
                                 const int64_t *L)
{
    for (int64_t i = rs; i < re; ++i) {
        int64_t j = L[vid(A, i, c, k)];
        vadd_row2(A, i, T, j, c);
    }
}

static view_t whole(uint64_t *A, int64_t m, int64_t n, int64_t s)
{
    view_t v = {A, s, 0, 0, m, n};
    return v;
}

void gf2o_make_table(const uint64_t *A, int64_t s, int64_t n, int64_t r, int k, int64_t c, int fix,
                     uint64_t *T, int64_t ts, int64_t *L)
{
    view_t U = sub(whole((uint64_t *)A, r + k, n, s), r, 0, k, n);
    vmake_table(U, k, c, fix, whole(T, (int64_t)1 << k, n, ts), L);
}

void gf2o_add_rows_from_table(uint64_t *A, int64_t s, int64_t n, int64_t rs, int64_t re, int64_t c,
                              int k, const uint64_t *T, int64_t ts, const int64_t *L)
{
    vadd_rows_from_table(whole(A, re, n, s), rs, re, c, k, whole((uint64_t *)T, (int64_t)1 << k, n, ts),
                         L);
}

/*
 * PlsSubmatrix: up to k pivots in the consecutive columns sc, sc+1, ... of
 * the rows from sr on. Rows are cleared lazily ("clear before", tracked per
 * pivot in done[]); the rows between a pivot's "done" mark and d_r are
 * finished at the end. Returns kbar, writes d_r (the last row touched).
 * The finishing loop reads "row sr+c2", "column sc+c2" and "sc+c2 < n-1".
 */
static int pls_submatrix(view_t A, int64_t sr, int64_t sc, int k, int64_t *P, int64_t *Q,
                         int64_t *d_r)
{
    int64_t done[64];
    int kbar = 0;
    for (int l = 0; l < 64; ++l)
        done[l] = 0;
    for (int r = 0; r < k; ++r) {
        int found = 0;
        int64_t i;
        for (i = sr + r; i < A.m; ++i) {
            for (int l = 0; l < r; ++l) {
                if (done[l] < i) {
                    if (vget(A, i, sc + l))
                        vadd_row(A, i, sr + l, sc + l + 1);
                    done[l] = i;
                }
            }
            if (vget(A, i, sc + r)) {
                found = 1;
                break;
            }
        }
        if (!found)
            break;
        P[sr + r] = i;
        Q[sr + r] = sc + r;
        vswap_rows(A, sr + r, i);
        done[r] = i;
        kbar = r + 1;
    }
    int64_t dr = 0;
    for (int l = 0; l < kbar; ++l)
        if (done[l] > dr)
            dr = done[l];
    for (int c2 = 0; c2 < kbar && sc + c2 < A.n - 1; ++c2) {
        for (int64_t r2 = done[c2] + 1; r2 <= dr; ++r2)
            if (vget(A, r2, sc + c2))
                vadd_row(A, r2, sr + c2, sc + c2 + 1);
    }
    *d_r = dr;
    return kbar;
}

/* Algorithm MMPF on a view; P (length m) and Q (length n) are local. */
static int64_t mmpf_view(view_t A, int64_t *P, int64_t *Q, int k)
{
    int64_t r = 0, c = 0;
    for (int64_t i = 0; i < A.n; ++i)
        Q[i] = i;
    for (int64_t i = 0; i < A.m; ++i)
        P[i] = i;
    int64_t N = (int64_t)1 << k;
    int64_t ts = (A.n + 63) / 64 + 1;
    uint64_t *Tbuf = (uint64_t *)calloc((size_t)(N * ts), sizeof(uint64_t));
    uint64_t *Ubuf = (uint64_t *)calloc((size_t)(k * ts), sizeof(uint64_t));
    int64_t *L = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    while (r < A.m && c < A.n) {
        if (c + k > A.n)
            k = (int)(A.n - c);
        int64_t dr = 0;
        int kbar = pls_submatrix(A, r, c, k, P, Q, &dr);
        if (kbar > 0) {
            /* U: the kbar pivot rows with every entry left of the upper
               triangle that starts at (r, c) zeroed out */
            view_t U = whole(Ubuf, kbar, A.n, ts);
            for (int t = 0; t < kbar; ++t)
                for (int64_t j = 0; j < A.n; ++j)
                    vset(U, t, j, j < c + t ? 0 : vget(A, r + t, j));
            view_t T = whole(Tbuf, (int64_t)1 << kbar, A.n, ts);
            vmake_table(U, kbar, c, 1, T, L);
            vadd_rows_from_table(A, dr + 1, A.m, c, kbar, T, L);
            r += kbar;
            c += kbar;
        } else {
            c += 1; /* skip zero column */
        }
    }
    for (int64_t j = 0; j < r; ++j)
        vswap_cols_from(A, j, Q[j], j);
    free(Tbuf);
    free(Ubuf);
    free(L);
    return r;
}

int64_t gf2o_pls_mmpf(uint64_t *A, int64_t m, int64_t n, int64_t s, int64_t *P, int64_t *Q, int k)
{
    if (k < 1 || k > 16)
        return -1;
    return mmpf_view(whole(A, m, n, s), P, Q, k);
}

/*
 * GaussSubmatrix (appendix; used by Algorithm M4RI, Sec. 3.1): Gauss-Jordan
 * elimination of the k columns c .. c+k-1 over the rows r .. r_end-1. For
 * column j, each candidate row i (from the next free row r_s on) first has
 * its bits at the block's earlier columns cleared by the block's pivot rows
 * (pivot row r+l clears column c+l, added from that column on); the first
 * candidate left with a 1 at column j is swapped to row r_s and added (from
 * column j on) to the block's earlier pivot rows that have a 1 at column j.
 * Returns the number of consecutive columns from c that got a pivot (it stops
 * at the first column without one).
 */
static int gauss_submatrix(view_t A, int64_t r, int64_t c, int k, int64_t r_end)
{
    int64_t rs = r;
    for (int64_t j = c; j < c + k; ++j) {
        int found = 0;
        for (int64_t i = rs; i < r_end; ++i) {
            for (int64_t l = 0; l < j - c; ++l)
                if (vget(A, i, c + l))
                    vadd_row(A, i, r + l, c + l);
            if (vget(A, i, j)) {
                vswap_rows(A, i, rs);
                for (int64_t l = r; l < rs; ++l)
                    if (vget(A, l, j))
                        vadd_row(A, l, rs, j);
                rs += 1;
                found = 1;
                break;
            }
        }
        if (!found)
            return (int)(j - c);
    }
    return k;
}

/*
 * Algorithm M4RI (Sec. 3.1): reduced row echelon form, in place. Per step,
 * GaussSubmatrix finds kbar <= k pivots in consecutive columns from c (the
 * block becomes the identity there), MakeTable enumerates the 2^kbar sums of
 * those rows from column c on, and AddRowsFromTable clears the kbar columns
 * in every other row, above (rows 0 .. r-1) and below (rows r+kbar .. m-1).
 * A column without a pivot is skipped. k shrinks to n - c near the right end.
 * pivots (nullable, length >= rank) receives the pivot columns. Returns the
 * rank, or -1 for k outside 1 .. 16.
 */
int64_t gf2o_m4ri(uint64_t *A, int64_t m, int64_t n, int64_t s, int k, int64_t *pivots)
{
    if (k < 1 || k > 16)
        return -1;
    view_t V = whole(A, m, n, s);
    int64_t ts = (n + 63) / 64 + 1;
    uint64_t *Tbuf = (uint64_t *)calloc((size_t)(((int64_t)1 << k) * ts), sizeof(uint64_t));
    int64_t *L = (int64_t *)calloc((size_t)1 << k, sizeof(int64_t));
    int64_t r = 0, c = 0;
    while (c < n) {
        if (c + k > n)
            k = (int)(n - c);
        int kbar = gauss_submatrix(V, r, c, k, m);
        if (kbar > 0) {
            view_t T = whole(Tbuf, (int64_t)1 << kbar, n, ts);
            vmake_table(sub(V, r, 0, kbar, n), kbar, c, 0, T, L);
            vadd_rows_from_table(V, 0, r, c, kbar, T, L);
            vadd_rows_from_table(V, r + kbar, m, c, kbar, T, L);
            if (pivots)
                for (int t = 0; t < kbar; ++t)
                    pivots[r + t] = c + t;
        }
        r += kbar;
        c += kbar;
        if (k != kbar)
            c += 1;
    }
    free(Tbuf);
    free(L);
    return r;
}

/*
 * Algorithm "PLS Decomposition" (recursive). Split the columns at n0, recurse
 * on the left block, permute the right block, A_NE <- L_NW^-1 A_NE,
 * A_SE <- A_SE + A_SW A_NE, recurse on A_SE, permute A_SW, merge P and Q and
 * move the second call's L columns next to the first call's. Below the column
 * cutoff the base case is MMPF. split_words != 0 cuts on a 64-column word
 * boundary (Sec. 6); otherwise n0 = n/2.
 */
static int64_t pls_rec(view_t A, int64_t *P, int64_t *Q, int64_t cutoff, int k, int split_words)
{
    if (A.m == 0 || A.n == 0) {
        for (int64_t i = 0; i < A.m; ++i)
            P[i] = i;
        for (int64_t i = 0; i < A.n; ++i)
            Q[i] = i;
        return 0;
    }
    int64_t n0 = A.n / 2;
    if (split_words)
        n0 = (A.n / 2) & ~(int64_t)63;
    if (A.n <= cutoff || n0 == 0)
        return mmpf_view(A, P, Q, k);

    view_t A0 = sub(A, 0, 0, A.m, n0);
    int64_t r0 = pls_rec(A0, P, Q, cutoff, k, split_words); /* Q0 = Q[0..n0) in place */

    view_t A1 = sub(A, 0, n0, A.m, A.n - n0);
    view_t ANE = sub(A, 0, n0, r0, A.n - n0);
    view_t ANW = sub(A, 0, 0, r0, r0);
    view_t ASW = sub(A, r0, 0, A.m - r0, r0);
    view_t ASE = sub(A, r0, n0, A.m - r0, A.n - n0);
    if (r0 > 0) {
        for (int64_t i = 0; i < r0; ++i) /* A1 <- P x A1 */
            vswap_rows(A1, i, P[i]);
        for (int64_t i = 0; i < r0; ++i) /* A_NE <- L_NW^-1 A_NE (unit lower) */
            for (int64_t l = 0; l < i; ++l)
                if (vget(ANW, i, l))
                    vadd_row(ANE, i, l, 0);
        for (int64_t i = 0; i < ASE.m; ++i) /* A_SE <- A_SE + A_SW A_NE */
            for (int64_t l = 0; l < r0; ++l)
                if (vget(ASW, i, l))
                    vadd_row2(ASE, i, ANE, l, 0);
    }
    int64_t *P1 = P + r0, *Q1 = Q + n0;
    int64_t r1 = pls_rec(ASE, P1, Q1, cutoff, k, split_words);
    for (int64_t i = 0; i < r1; ++i) /* A_SW <- P1 x A_SW */
        vswap_rows(ASW, i, P1[i]);
    for (int64_t i = 0; i < A.m - r0; ++i)
        P[r0 + i] = P1[i] + r0;
    for (int64_t i = 0; i < A.n - n0; ++i)
        Q[n0 + i] = Q1[i] + n0;
    int64_t j = r0;
    for (int64_t i = n0; i < n0 + r1; ++i) {
        Q[j] = Q[i];
        j += 1;
    }
    for (int64_t i = r0 + r1; i < A.n; ++i) /* identity beyond the rank */
        Q[i] = i;
    j = n0;
    for (int64_t i = r0; i < r0 + r1; ++i) { /* compress L */
        vswap_cols_from(A, i, j, i);
        j += 1;
    }
    return r0 + r1;
}

int64_t gf2o_pls_rec(uint64_t *A, int64_t m, int64_t n, int64_t s, int64_t *P, int64_t *Q,
                     int64_t cutoff, int k, int split_words)
{
    if (k < 1 || k > 16)
        return -1;
    return pls_rec(whole(A, m, n, s), P, Q, cutoff, k, split_words);
}
