// eco_policy_fp8.cu -- the FP8 instances of the policy kernel (compiled in
// a translation unit of their own so that the three precisions build in
// parallel).
#include "eco_policy_kernel.cuh"

namespace eco {

PolicyFn policy_pick_fp8(int H, int variant) { return policy_pick_width<PREC_FP8>(H, variant); }

}  // namespace eco
