// eco_policy_bf16.cu -- the BF16 instances of the policy kernel (compiled in
// a translation unit of their own so that the three precisions build in
// parallel).
#include "eco_policy_kernel.cuh"

namespace eco {

PolicyFn policy_pick_bf16(int H, int variant) { return policy_pick_width<PREC_BF16>(H, variant); }

}  // namespace eco
