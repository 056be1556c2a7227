// gf2_sweep.cu -- the table sweep of one panel over 16-word column tiles.
//
// One launch per panel does MakeTable1 and AddRowsFromTable (Sec. 3.1, 4.1)
// for the panel's (up to) 64 pivots: Gray-code tables of the pivot rows per
// column tile, and table rows added to every swept row. Two forms:
//   * PLS (MODE 0): the rows below the pivots (trailing rows); the panel word
//     becomes the row's multipliers (the entries of L), as in MMPF (Sec. 4.1);
//   * reduced echelon form (MODE 1): every row but the panel's pivot rows, the
//     rows above included, as in Algorithm M4RI (Sec. 3.1); the panel word of
//     a trailing row becomes zero and the pivot rows become the rows of the
//     panel's reduced echelon block.
//
// For a swept row with current panel word w, z = its coordinates over the
// panel's original pivot rows O (two byte lookups per thread, summed over the
// row's four threads), and row ^= z.O over the tile. In PLS form the tables'
// entries at the panel word hold X_t = pivot t's multipliers plus its own bit,
// so the same lookups produce the row's multipliers there. Pivot rows never
// change in A during the sweep; their new rows go to `out` at their final
// positions.
//
// Tables (k = 8 pivots per table, stored as halves): for each group g of 8
// pivots, the sums of its first 7 rows (128 entries of 128 bytes), and one
// more table of the sums of the groups' last rows, indexed by bit 7 of every
// byte of z: nine 128-byte lookups per row and tile. A thread holds 4 words
// of a row; the two rows one quarter-warp serves read the two 16-byte halves
// of their 32 bytes in opposite order, so each lookup instruction is one bank
// wavefront.
//
// Work: (column tile, block of 128 rows) units in tile-major order, cut into
// equal contiguous runs, one per CTA. Blocks of plain rows (rows found from
// `perm` alone, or the rows above in MODE 1) run a pipelined loop: the
// physical row 5 blocks ahead, an L2 prefetch of its 128-byte line 4 ahead,
// the panel word 3 ahead and the row data 2 ahead; in interior tiles a row
// whose panel word is zero is neither loaded nor stored. In edge tiles (the
// panel word and the next one, a partial last tile) the threads holding those
// words store word by word. The one or two blocks holding pivot and window
// rows take a plain per-block path.
#include "gf2_sweep.cuh"

namespace {

template <int FORM, int KB>
__global__ void __launch_bounds__(NT, 1)
k_sweep16(uint64_t *__restrict__ A, int64_t stride, const u64 *__restrict__ side_cur, u64 *__restrict__ side_nxt,
          const int *__restrict__ perm, const PanelState *__restrict__ st, uint64_t *__restrict__ out,
          int64_t ostride, u64 *__restrict__ ups, int m, int W, int b)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    sweep_panel16<FORM, KB>(*reinterpret_cast<SweepSmem *>(smraw), A, stride, side_cur, side_nxt, perm, st, out, ostride,
                        ups, m, W, b, blockIdx.x, gridDim.x);
}

// Batched: panel b of the nact matrices idx[0..nact), matrix idx[j] swept by CTAs pre[j] .. pre[j+1]-1.
template <int KB>
__global__ void __launch_bounds__(NT, 1)
k_sweep16_b(const gf2::ElimDesc *__restrict__ D, const int *__restrict__ idx, const int *__restrict__ pre, int nact,
            int b)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int lo = 0, hi = nact - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const gf2::ElimDesc &d = D[idx[lo]];
    sweep_panel16<0, KB>(*reinterpret_cast<SweepSmem *>(smraw), d.A, d.stride, d.side + (size_t)(b & 1) * d.m,
                     d.side + (size_t)((b + 1) & 1) * d.m, d.perm, d.st + (b & 1), d.out, d.ostride, nullptr, d.m, d.W,
                     b, (int)blockIdx.x - pre[lo], pre[lo + 1] - pre[lo]);
}

constexpr size_t SWEEP_SMEM = sizeof(SweepSmem);

template <int FORM, int KB>
int launch(const gf2::Elim &e, int b, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    if (gf2::attr_needed(attr_devs)) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sweep16<FORM, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
        if (err != cudaSuccess)
            return gf2::note_cuda(err);
        gf2::attr_done(attr_devs);
    }
    const u64 *cur = e.side + (size_t)(b & 1) * e.m;
    u64 *nxt = e.side + (size_t)((b + 1) & 1) * e.m;
    const int tok = gf2::prof_begin(s);
    k_sweep16<FORM, KB><<<e.grid, NT, SWEEP_SMEM, s>>>(e.A, e.stride, cur, nxt, e.perm, e.st + (b & 1), e.out, e.ostride,
                                                   e.ups, (int)e.m, (int)e.W, b);
    gf2::prof_end(s, GF2_PROF_SWEEP, tok);
    gf2::prof_launched(1);
    return gf2::note_cuda(cudaGetLastError());
}

}  // namespace

namespace gf2 {

template <int KB>
static int batch_sweep16_k(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b,
                           cudaStream_t s)
{
    static std::atomic<unsigned long long> attr_devs{0};
    if (attr_needed(attr_devs)) {
        cudaError_t err =
            cudaFuncSetAttribute(k_sweep16_b<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
        if (err != cudaSuccess)
            return note_cuda(err);
        attr_done(attr_devs);
    }
    const int tok = prof_begin(s);
    k_sweep16_b<KB><<<total, NT, SWEEP_SMEM, s>>>(D, idx, pre, nact, b);
    prof_end(s, GF2_PROF_SWEEP, tok);
    prof_launched(1);
    return note_cuda(cudaGetLastError());
}

int batch_sweep16(const ElimDesc *D, const int *idx, const int *pre, int nact, int total, int b, int k, cudaStream_t s)
{
    if (nact <= 0 || total <= 0)
        return GF2_OK;
    return k == 4 ? batch_sweep16_k<4>(D, idx, pre, nact, total, b, s) : batch_sweep16_k<8>(D, idx, pre, nact, total, b, s);
}

int launch_sweep16(const Elim &e, int b, cudaStream_t s)
{
    if (e.mode && !e.ups)
        return GF2_EINVAL;
    if (e.mode == 2)
        return launch<2, 8>(e, b, s);
    if (e.mode == 1)
        return launch<1, 8>(e, b, s);
    return e.k == 4 ? launch<0, 4>(e, b, s) : launch<0, 8>(e, b, s);
}

}  // namespace gf2
