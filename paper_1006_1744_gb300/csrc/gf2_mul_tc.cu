// gf2_mul_tc.cu -- GF(2) product on the tensor cores (not built yet).
#include "gf2_common.cuh"

namespace gf2 {

size_t mul_tensor_workspace(int64_t, int64_t, int64_t) { return 0; }

int mul_tensor(uint64_t *, int64_t, const uint64_t *, int64_t, const uint64_t *, int64_t, int64_t, int64_t,
               int64_t, int, void *, size_t, cudaStream_t)
{
    return GF2_EINVAL;
}

}  // namespace gf2
