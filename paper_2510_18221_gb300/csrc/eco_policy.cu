// eco_policy.cu -- the policy phase's host side: the table of kernel
// variants the autotuner chooses from, shared-memory sizing and the launch.
// The kernel itself is eco_policy_kernel.cuh, instantiated per precision in
// eco_policy_fp32.cu, eco_policy_bf16.cu and eco_policy_fp8.cu.
#include "eco_internal.cuh"
#include "eco_kernels.h"

namespace eco {

struct VariantDesc {
  const char *name;
  int warps, unroll;
  bool sparse;
};

// The launch bounds of each (warps, units in flight, resident CTAs) are in
// policy_pick_variant (eco_policy_kernel.cuh).
static const VariantDesc kVariants[] = {
    {"warp-per-agent, 4 warps/CTA, 8 units in flight per lane", 4, 8, false},
    {"warp-per-agent, 8 warps/CTA, 8 units in flight per lane", 8, 8, false},
    {"warp-per-agent, 8 warps/CTA, 4 units in flight per lane", 8, 4, false},
    {"warp-per-agent, 16 warps/CTA, 4 units in flight per lane", 16, 4, false},
    {"warp-per-agent, 8 warps/CTA, 4 units in flight per lane, 64 registers", 8, 4, false},
    {"warp-per-agent, 4 warps/CTA, 8 units in flight per lane, 64 registers", 4, 8, false},
    {"input-sparse W_in rows, 8 warps/CTA, 4 units in flight per lane", 8, 4, true},
    {"input-sparse W_in rows, 4 warps/CTA, 8 units in flight per lane, 64 registers", 4, 8, true},
    {"warp-per-agent, 4 warps/CTA, 8 units in flight per lane, 56 registers", 4, 8, false},
    {"warp-per-agent, 4 warps/CTA, 4 units in flight per lane, 56 registers", 4, 4, false},
};
static const int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int policy_variant_count() { return kNumVariants; }
const char *policy_variant_name(int k) {
  if (k < 1 || k > kNumVariants) return "invalid";
  return kVariants[k - 1].name;
}
bool policy_variant_sparse(int k) { return k >= 1 && k <= kNumVariants && kVariants[k - 1].sparse; }

static PolicyFn pick(int prec, int H, int variant) {
  if (prec == PREC_FP32) return policy_pick_fp32(H, variant);
  if (prec == PREC_BF16) return policy_pick_bf16(H, variant);
  return policy_pick_fp8(H, variant);
}

int policy_xs_floats(const Layout &L) { return ((L.D > L.H ? L.D : L.H) + 3) & ~3; }

cudaError_t policy_prepare(const Layout &L, const Rules &R, int variant, PolicyLaunch *pl) {
  if (variant < 1 || variant > kNumVariants) return cudaErrorInvalidValue;
  PolicyFn fn = pick(R.precision, L.H, variant);
  if (!fn) return cudaErrorInvalidValue;
  const VariantDesc &v = kVariants[variant - 1];
  const int xs = policy_xs_floats(L);
  // per warp: observation, hidden activation, logits (+ the sparse input list)
  const size_t smem = (size_t)v.warps * policy_warp_floats(xs, L.H, v.sparse) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, v.warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  pl->fn = (void *)fn;
  pl->threads = v.warps * 32;
  pl->blocks = sms * per_sm;  // one full wave of resident CTAs on every SM
  pl->smem = smem;
  pl->xs_floats = xs;
  return cudaSuccess;
}

cudaError_t policy_launch(const PolicyLaunch &pl, const Dev &d, const Layout &L, const Rules &R,
                          cudaStream_t s, bool apply_moves) {
  PolicyFn fn = (PolicyFn)pl.fn;
  fn<<<pl.blocks, pl.threads, pl.smem, s>>>(d, L, R, pl.xs_floats, apply_moves ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace eco
