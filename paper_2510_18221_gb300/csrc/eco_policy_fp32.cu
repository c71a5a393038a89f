// eco_policy_fp32.cu -- the FP32 instances of the policy kernel (compiled in
// a translation unit of their own so that the three precisions build in
// parallel).
#include "eco_policy_kernel.cuh"

namespace eco {

PolicyFn policy_pick_fp32(int H, int variant) { return policy_pick_width<PREC_FP32>(H, variant); }

}  // namespace eco
