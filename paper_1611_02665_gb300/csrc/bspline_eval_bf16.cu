// Evaluation kernels instantiated for __nv_bfloat16 coefficient tables.
#include "bspline_eval_kernels.cuh"

namespace bsg {
bspline_status launch_eval_bf16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                               int num_sms, cudaStream_t s) {
    return launch_eval_typed<__nv_bfloat16>(kind, tu, A, map, num_sms, s);
}
bspline_status launch_ratio_bf16(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                cudaStream_t s) {
    return launch_ratio_typed<__nv_bfloat16>(kind, A, uinv, ldu, ratio, s);
}
bspline_status launch_ratio_mma_bf16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                                    int num_sms, const float *uinv, int ldu, float *ratio, cudaStream_t s) {
    return launch_ratio_mma_typed<__nv_bfloat16>(kind, tu, A, map, num_sms, uinv, ldu, ratio, s);
}
}  // namespace bsg
