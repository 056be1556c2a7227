// gf2_synth.cu -- device twin of the seeded input generators (synth.py).
//
// Holds none of the elimination, table or product arithmetic: it only fills
// packed matrices from the SplitMix64 output function (Steele, Lea, Flood,
// OOPSLA 2014), with the same counters as the host module, so that large
// inputs can be produced on the device. Tests check both sides bit for bit.
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/gf2_synth.h"

namespace {

__device__ __forceinline__ unsigned long long mix(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr unsigned long long TAG_P = 0xD1B54A32D192ED03ull;

__global__ void k_fill(uint64_t *A, int64_t m, int64_t n, int64_t stride, uint64_t seed, uint64_t thresh,
                       int dense, double frac)
{
    const int64_t W = (n + 63) / 64;
    const int64_t total = m * stride;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / stride, w = e % stride;
        uint64_t v = 0;
        if (w < W) {
            if (dense) {
                v = mix(seed ^ mix(((unsigned long long)i << 32) | (unsigned long long)w));
            } else {
                const int64_t start = frac > 0.0 ? (int64_t)floor(frac * (double)i * (double)n / (double)m) : 0;
                for (int bit = 0; bit < 64; ++bit) {
                    const int64_t j = 64 * w + bit;
                    if (j >= n)
                        break;
                    const unsigned long long h =
                        mix(seed ^ TAG_P ^ mix(((unsigned long long)i << 32) | (unsigned long long)j));
                    if ((h >> 11) < thresh && j >= start)
                        v |= 1ull << bit;
                }
            }
            if (w == W - 1 && (n & 63))
                v &= (1ull << (n & 63)) - 1ull;
        }
        A[e] = v;
    }
}

}  // namespace

extern "C" int gf2_synth_fill(uint64_t *A, int64_t m, int64_t n, int64_t stride, uint64_t seed, double p,
                              double echelon_frac, void *stream)
{
    if (m < 0 || n < 0 || stride < (n + 63) / 64 || (m > 0 && n > 0 && !A))
        return 1;
    if (p < 0.0 || p > 1.0 || echelon_frac < 0.0)
        return 1;
    if (m == 0 || stride == 0)
        return 0;
    const int dense = (p == 0.5 && echelon_frac == 0.0);
    const uint64_t thresh = (uint64_t)(p * 9007199254740992.0);
    k_fill<<<1024, 256, 0, (cudaStream_t)stream>>>(A, m, n, stride, seed, thresh, dense, echelon_frac);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
