// M2L on the tensor cores (tcgen05, sm_103a). Same-level M2L is a dense
// contraction: for a tile of 128 target cells and one translation vector v,
// L~[128 x p^2] += gather(M~)[128 x p^2] * T_v^T, T_v the level-independent
// p^2 x p^2 operator of Sec. 2.1's M2L in the scaled real layout.
#include "fmm_internal.cuh"

namespace fmm {

bool tensor_m2l_supported(fmm_ctx *) { return false; }

void tensor_tables_init(fmm_ctx *) {}

void m2l_tensor(fmm_ctx *, float *, const float *)
{
    throw Error{FMM_ECUDA, "tensor-core M2L is not available in this build"};
}

}  // namespace fmm
