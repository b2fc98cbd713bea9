// Evaluation kernels instantiated for __half coefficient tables.
#include "bspline_eval_kernels.cuh"

namespace bsg {
bspline_status launch_eval_f16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                               int num_sms, cudaStream_t s) {
    return launch_eval_typed<__half>(kind, tu, A, map, num_sms, s);
}
bspline_status launch_ratio_f16(int kind, const EvalArgs &A, const float *uinv, int ldu, float *ratio,
                                cudaStream_t s) {
    return launch_ratio_typed<__half>(kind, A, uinv, ldu, ratio, s);
}
bspline_status launch_ratio_mma_f16(int kind, const bspline_tuning &tu, const EvalArgs &A, const CUtensorMap *map,
                                    int num_sms, const float *uinv, int ldu, float *ratio, cudaStream_t s) {
    return launch_ratio_mma_typed<__half>(kind, tu, A, map, num_sms, uinv, ldu, ratio, s);
}
}  // namespace bsg
