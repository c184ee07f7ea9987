// One operator application in the requested precision: FP32 CUDA cores or BF16 tcgen05.
#include "aexp_internal.cuh"

namespace aexp {

cudaError_t op_apply_forward(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st) {
    if (L.precision == AEXP_FP32) {
        cudaError_t e = op_coil_weight(L, x, ws, st);
        return e == cudaSuccess ? op_forward_core(L, ws, st) : e;
    }
    return op_forward_tc(L, x, ws, st);
}

cudaError_t op_reduce_forward_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st) {
    return L.precision == AEXP_FP32 ? op_forward_reduce_public(L, ws, y, st)
                                    : op_forward_reduce_planar_public(L, ws, y, st);
}

cudaError_t op_reduce_forward_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                       cudaStream_t st) {
    return L.precision == AEXP_FP32 ? op_forward_reduce_residual(L, ws, ymeas_t, rt, st)
                                    : op_forward_reduce_planar_residual(L, ws, ymeas_t, rt, st);
}

cudaError_t op_apply_adjoint(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    return L.precision == AEXP_FP32 ? op_adjoint_core(L, yt, ws, st) : op_adjoint_tc(L, yt, ws, st);
}

cudaError_t op_residual_adjoint(const OpLayout &L, char *ws, const float2 *ymeas_t, cudaStream_t st) {
    if (L.precision == AEXP_BF16_TC) return op_residual_adjoint_tc(L, ws, ymeas_t, st);
    float2 *rt = (float2 *)(ws + L.off_yt);
    cudaError_t e = op_reduce_forward_residual(L, ws, ymeas_t, rt, st);
    return e == cudaSuccess ? op_apply_adjoint(L, rt, ws, st) : e;
}

}  // namespace aexp
