// gf2_strassen.cu -- the Strassen-Winograd product over GF(2).
//
// The paper's trailing update A_SE <- A_SE + A_SW.A_NE (Algorithm PLS, Sec. 5)
// is a matrix product, and the paper reduces its PLS to a product done "as in"
// its cited multiplication library: Strassen-Winograd recursion down to a
// Method-of-the-Four-Russians base case. One level splits A (m x k), B (k x n)
// and C into 2 x 2 blocks and forms C from 7 half-size products and 15 block
// additions (Winograd's form; over GF(2) every subtraction is an addition, an
// XOR). The leaves are this library's exact products: the XOR-table form or the
// tensor-core form. Results are bit-identical to the plain product.
//
// A level is taken while m, k and n are at least twice the leaf size and k and n
// are multiples of 2048 bits (m even), so that every block is a view starting on
// a 128-byte boundary; otherwise the leaf product runs on the whole.
#include "gf2_common.cuh"

namespace {

// D = X ^ Y, or D ^= X when Y is null; rows x words, words even, views 16-byte aligned
__global__ void k_xor_views(uint64_t *__restrict__ D, int64_t sd, const uint64_t *__restrict__ X, int64_t sx,
                            const uint64_t *__restrict__ Y, int64_t sy, int rows, int pairs)
{
    const int total = rows * pairs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = e / pairs, p = e - i * pairs;
        uint64_t *d = D + (int64_t)i * sd + 2 * p;
        ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(X + (int64_t)i * sx + 2 * p);
        const ulonglong2 y = Y ? *reinterpret_cast<const ulonglong2 *>(Y + (int64_t)i * sy + 2 * p)
                               : *reinterpret_cast<const ulonglong2 *>(d);
        x.x ^= y.x;
        x.y ^= y.y;
        *reinterpret_cast<ulonglong2 *>(d) = x;
    }
}

int xor_views(uint64_t *D, int64_t sd, const uint64_t *X, int64_t sx, const uint64_t *Y, int64_t sy, int64_t rows,
              int64_t words, cudaStream_t s)
{
    const int64_t total = rows * (words / 2);
    if (total <= 0)
        return GF2_OK;
    const int64_t cap = 8ll * gf2::sm_count();
    const int grid = (int)((total + 255) / 256 < cap ? (total + 255) / 256 : cap);
    k_xor_views<<<grid, 256, 0, s>>>(D, sd, X, sx, Y, sy, (int)rows, (int)(words / 2));
    gf2::prof_launched(1);
    return gf2::note_cuda(cudaGetLastError());
}

bool splits(int64_t m, int64_t k, int64_t n, int64_t leaf)
{
    return m % 2 == 0 && k % 2048 == 0 && n % 2048 == 0 && m >= 2 * leaf && k >= 2 * leaf && n >= 2 * leaf;
}

struct Leaf {
    int kind;  // GF2_PRODUCT_XOR or GF2_PRODUCT_TENSOR
    void *work;
    size_t bytes;
};

int leaf_product(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
                 int64_t k, int64_t n, const Leaf &lf, cudaStream_t s)
{
    if (lf.kind == GF2_PRODUCT_TENSOR)
        return gf2::mul_tensor(C, sc, A, sa, B, sb, m, k, n, 0, lf.work, lf.bytes, s);
    return gf2::mul_xor(C, sc, A, sa, B, sb, m, k, n, 0, 0, 0, s);
}

// temporaries of one level and everything below it (bytes)
size_t level_bytes(int64_t m, int64_t k, int64_t n, int64_t leaf)
{
    if (!splits(m, k, n, leaf))
        return 0;
    const int64_t m2 = m / 2, kw = k / 128, nw = n / 128;
    return (size_t)(m2 * kw + (k / 2) * nw + m2 * nw) * 8 + level_bytes(m2, k / 2, n / 2, leaf);
}

// the largest leaf product's tensor-core workspace (leaves all have the same shape)
size_t leaf_bytes(int64_t m, int64_t k, int64_t n, int64_t leaf, int kind)
{
    while (splits(m, k, n, leaf)) {
        m /= 2;
        k /= 2;
        n /= 2;
    }
    return kind == GF2_PRODUCT_TENSOR ? gf2::mul_tensor_workspace(m, k, n) : 0;
}

// C = A.B (overwrite), Winograd's schedule with three temporaries per level:
// X (m/2 x k/2), Y (k/2 x n/2), Z (m/2 x n/2); C's blocks hold the partial sums
int strassen(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
             int64_t k, int64_t n, int64_t leaf, char *tmp, const Leaf &lf, cudaStream_t s)
{
    if (!splits(m, k, n, leaf))
        return leaf_product(C, sc, A, sa, B, sb, m, k, n, lf, s);
    const int64_t m2 = m / 2, k2 = k / 2, n2 = n / 2;
    const int64_t kw = k2 / 64, nw = n2 / 64;  // words per half row (multiples of 16)
    const uint64_t *A11 = A, *A12 = A + kw, *A21 = A + m2 * sa, *A22 = A + m2 * sa + kw;
    const uint64_t *B11 = B, *B12 = B + nw, *B21 = B + k2 * sb, *B22 = B + k2 * sb + nw;
    uint64_t *C11 = C, *C12 = C + nw, *C21 = C + m2 * sc, *C22 = C + m2 * sc + nw;
    uint64_t *X = reinterpret_cast<uint64_t *>(tmp);
    uint64_t *Y = X + m2 * kw;
    uint64_t *Z = Y + k2 * nw;
    char *below = reinterpret_cast<char *>(Z + m2 * nw);
    int rc;
#define GF2_TRY(call)                                                                                              \
    if ((rc = (call)))                                                                                             \
    return rc
    // S3 = A11 + A21, T3 = B22 + B12, P7 = S3.T3 -> C21
    GF2_TRY(xor_views(X, kw, A11, sa, A21, sa, m2, kw, s));
    GF2_TRY(xor_views(Y, nw, B22, sb, B12, sb, k2, nw, s));
    GF2_TRY(strassen(C21, sc, X, kw, Y, nw, m2, k2, n2, leaf, below, lf, s));
    // S1 = A21 + A22, T1 = B12 + B11, P5 = S1.T1 -> C22
    GF2_TRY(xor_views(X, kw, A21, sa, A22, sa, m2, kw, s));
    GF2_TRY(xor_views(Y, nw, B12, sb, B11, sb, k2, nw, s));
    GF2_TRY(strassen(C22, sc, X, kw, Y, nw, m2, k2, n2, leaf, below, lf, s));
    // S2 = S1 + A11, T2 = B22 + T1, P6 = S2.T2 -> C12
    GF2_TRY(xor_views(X, kw, A11, sa, nullptr, 0, m2, kw, s));
    GF2_TRY(xor_views(Y, nw, B22, sb, nullptr, 0, k2, nw, s));
    GF2_TRY(strassen(C12, sc, X, kw, Y, nw, m2, k2, n2, leaf, below, lf, s));
    // S4 = A12 + S2, P3 = S4.B22 -> C11
    GF2_TRY(xor_views(X, kw, A12, sa, nullptr, 0, m2, kw, s));
    GF2_TRY(strassen(C11, sc, X, kw, B22, sb, m2, k2, n2, leaf, below, lf, s));
    // P1 = A11.B11 -> Z
    GF2_TRY(strassen(Z, nw, A11, sa, B11, sb, m2, k2, n2, leaf, below, lf, s));
    // U2 = P1 + P6 (C12), U3 = U2 + P7 (C21), U4 = U2 + P5 (C12), U7 = U3 + P5 (C22), U5 = U4 + P3 (C12)
    GF2_TRY(xor_views(C12, sc, Z, nw, nullptr, 0, m2, nw, s));
    GF2_TRY(xor_views(C21, sc, C12, sc, nullptr, 0, m2, nw, s));
    GF2_TRY(xor_views(C12, sc, C22, sc, nullptr, 0, m2, nw, s));
    GF2_TRY(xor_views(C22, sc, C21, sc, nullptr, 0, m2, nw, s));
    GF2_TRY(xor_views(C12, sc, C11, sc, nullptr, 0, m2, nw, s));
    // T4 = T2 + B21, P4 = A22.T4 -> C11, U6 = U3 + P4 (C21)
    GF2_TRY(xor_views(Y, nw, B21, sb, nullptr, 0, k2, nw, s));
    GF2_TRY(strassen(C11, sc, A22, sa, Y, nw, m2, k2, n2, leaf, below, lf, s));
    GF2_TRY(xor_views(C21, sc, C11, sc, nullptr, 0, m2, nw, s));
    // P2 = A12.B21 -> C11, U1 = P1 + P2 (C11)
    GF2_TRY(strassen(C11, sc, A12, sa, B21, sb, m2, k2, n2, leaf, below, lf, s));
    GF2_TRY(xor_views(C11, sc, Z, nw, nullptr, 0, m2, nw, s));
#undef GF2_TRY
    return GF2_OK;
}

}  // namespace

namespace gf2 {

size_t mul_strassen_workspace(int64_t m, int64_t k, int64_t n, int64_t leaf, int leaf_kind)
{
    if (!splits(m, k, n, leaf))
        return leaf_kind == GF2_PRODUCT_TENSOR ? mul_tensor_workspace(m, k, n) : 0;
    // the product for an accumulating call (m x n), the levels' temporaries, the leaf's
    const size_t acc = align_up((size_t)m * (size_t)(n / 64) * 8, 256);
    const size_t lv = align_up(level_bytes(m, k, n, leaf), 256);
    return acc + lv + leaf_bytes(m, k, n, leaf, leaf_kind);
}

int mul_strassen(uint64_t *C, int64_t sc, const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb, int64_t m,
                 int64_t k, int64_t n, int accumulate, void *work, size_t work_bytes, int64_t leaf, int leaf_kind,
                 cudaStream_t s)
{
    if (!splits(m, k, n, leaf)) {
        if (leaf_kind == GF2_PRODUCT_TENSOR)
            return mul_tensor(C, sc, A, sa, B, sb, m, k, n, accumulate, work, work_bytes, s);
        return mul_xor(C, sc, A, sa, B, sb, m, k, n, accumulate, 0, 0, s);
    }
    if (work_bytes < mul_strassen_workspace(m, k, n, leaf, leaf_kind))
        return GF2_ENOSPACE;
    char *w = static_cast<char *>(work);
    const size_t acc = align_up((size_t)m * (size_t)(n / 64) * 8, 256);
    const size_t lv = align_up(level_bytes(m, k, n, leaf), 256);
    Leaf lf{leaf_kind, w + acc + lv, work_bytes - acc - lv};
    if (!accumulate)
        return strassen(C, sc, A, sa, B, sb, m, k, n, leaf, w + acc, lf, s);
    uint64_t *D = reinterpret_cast<uint64_t *>(w);  // A.B, then added into C
    const int64_t sd = n / 64;
    int rc = strassen(D, sd, A, sa, B, sb, m, k, n, leaf, w + acc, lf, s);
    return rc ? rc : xor_views(C, sc, D, sd, nullptr, 0, m, sd, s);
}

}  // namespace gf2
