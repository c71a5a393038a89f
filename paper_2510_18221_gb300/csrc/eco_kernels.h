// eco_kernels.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "eco_internal.cuh"

namespace eco {

// Policy phase (eco_policy.cu).
struct PolicyLaunch {
  void *fn;
  int threads, blocks;
  size_t smem;
  int xs_floats;
};
int policy_variant_count();
const char *policy_variant_name(int k);
// Variants that stream only the W_in rows of nonzero inputs (opt-in: the
// autotuner chooses among them only when asked to, policy_variant = -1).
bool policy_variant_sparse(int k);
typedef void (*PolicyFn)(Dev, Layout, Rules, int, int);
// Floats of one warp's shared-memory slice: observation (xs_floats, a
// multiple of 4), hidden activation (H), logits (16) and, for the sparse
// variants, the list of nonzero inputs (xs_floats shorts, rounded up to whole
// 16-byte units).  Every part is a multiple of 4 floats, so each warp's
// slice and the float4 reads of its activations stay 16-byte aligned.
__host__ __device__ inline int policy_warp_floats(int xs_floats, int H, bool sparse) {
  return xs_floats + H + 16 + (sparse ? ((xs_floats / 2 + 3) & ~3) : 0);
}
// Kernel instance of variant k for a hidden width (one translation unit per
// precision: eco_policy_fp32.cu, eco_policy_bf16.cu, eco_policy_fp8.cu).
PolicyFn policy_pick_fp32(int H, int variant);
PolicyFn policy_pick_bf16(int H, int variant);
PolicyFn policy_pick_fp8(int H, int variant);
cudaError_t policy_prepare(const Layout &L, const Rules &R, int variant, PolicyLaunch *pl);
// apply_moves: also apply facing / turns and file move claims (the step);
// false leaves the world state untouched (timing, parity of the policy).
cudaError_t policy_launch(const PolicyLaunch &pl, const Dev &d, const Layout &L, const Rules &R,
                          cudaStream_t s, bool apply_moves);

// Environment phases (eco_env.cu).
struct EnvGrid {
  int sms;                // SM count
  int slot_blocks;        // blocks of 256 threads for per-agent phases
  int cell_blocks;        // blocks of 256 threads for per-cell phases
  int birth_blocks;       // CTAs of the mutation kernel
  int persistent_blocks;  // co-resident CTAs of the persistent form (0: unavailable)
  int use_persistent;     // run the environment phases as one persistent kernel
};
__host__ __device__ int compact_tiles(int total_slots);
// Alive list of the current state (ascending slots) and its count.
cudaError_t launch_compact(const Dev &d, cudaStream_t s);
// Shared-memory attributes and the persistent form's grid size.
cudaError_t env_prepare(const Layout &L, EnvGrid *g);
cudaError_t launch_env_phases(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                              cudaStream_t s);

// Reset and parameter maintenance (eco_init.cu).
cudaError_t launch_reset(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                         cudaStream_t s);
// Static per-slot tables (environment of every slot) at create.
cudaError_t launch_init_static(const Dev &d, const EnvGrid &g, cudaStream_t s);
// Recompute the "now" statistics (alive, food, energy, step) from the state.
cudaError_t launch_recount(const Dev &d, const Rules &R, cudaStream_t s);
cudaError_t launch_requant(const Dev &d, const Layout &L, const Rules &R, int slot0, int n,
                           cudaStream_t s);

}  // namespace eco
