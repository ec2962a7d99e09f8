// tblock5_bf16.cu -- BF16-storage instances of the D2Q5 wavefront temporal blocking
// (tblock5.cuh), compiled apart from the FP32 ones.  The rho tape of adjoint replays is
// recorded by FP32 contexts only, so there is no recording instance here.
#include <cuda_runtime.h>

#include "lb_runtime.h"
#include "tblock5.cuh"

namespace lbtb5 {
Tb5Fn pick_bf16(int K, bool mrt, bool rec) {
    if (rec) return nullptr;
    switch (K) {
        case 2: return pick_k<2, __nv_bfloat16, false>(mrt, false);
        case 4: return pick_k<4, __nv_bfloat16, false>(mrt, false);
        case 6: return pick_k<6, __nv_bfloat16, false>(mrt, false);
        case 8: return pick_k<8, __nv_bfloat16, false>(mrt, false);
        case 16: return pick_k<16, __nv_bfloat16, false>(mrt, false);
        default: return nullptr;
    }
}
Tb5BatchFn pick_batch_bf16(int K, bool mrt) {
    if (K != kServeTb) return nullptr;
    return mrt ? tb5_batch_kernel<true, kServeTb, __nv_bfloat16>
               : tb5_batch_kernel<false, kServeTb, __nv_bfloat16>;
}
}  // namespace lbtb5
