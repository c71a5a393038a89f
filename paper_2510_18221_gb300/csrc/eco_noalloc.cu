// eco_noalloc.cu -- move-claim resolution for one world that allocates no
// device memory: the claim scratch lives in a fixed file-scope __device__
// array instead of the caller's workspace.
//
// It applies the same rule as the movement phase of eco_step: a move action
// faces its direction; a move into a blocked cell (wall, or occupied when
// the step began) fails; among movers into one free cell the highest
// CLAIM_MOVE draw wins, ties to the lower agent index; turn-left/right
// (actions 6, 7) rotate the facing.  Agent i plays the role of slot i.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/eco.h"
#include "eco_internal.cuh"

namespace eco {
namespace {

// Claim scratch shared by every call on a device (8 MiB, held until exit).
static __device__ __align__(256) unsigned long long g_move_claims[ECO_NOALLOC_MAX_CELLS];

// Device address of g_move_claims per device, looked up once.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned long long *g_claims_ptr[kMaxDevices] = {};

__global__ void k_na_clear(unsigned long long *claims, int n_cells) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
    claims[c] = 0ull;
}

__global__ void k_na_claim(unsigned long long *claims, int side, int n, const int32_t *pos,
                           const uint8_t *act, const uint8_t *facing_in, const uint8_t *blocked,
                           uint32_t seed, uint32_t step, uint8_t *facing_out, int32_t *pos_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int a = act[i];
    int f = facing_in[i] & 3;
    int tc = -1;
    if (a >= ACT_N && a <= ACT_W) {
      f = (a == ACT_N) ? 0 : (a == ACT_S) ? 2 : (a == ACT_E) ? 1 : 3;
      const int c = step_cell(pos[i], f, side);
      if (!blocked[c]) {
        const U4 r = philox(step, (uint32_t)i, 0u, 0u, seed, S_CLAIM_MOVE);
        atomicMax(&claims[c], claim_key(r.x, i));
        tc = c;
      }
    } else if (a == ACT_LEFT) {
      f = (f + 3) & 3;
    } else if (a == ACT_RIGHT) {
      f = (f + 1) & 3;
    }
    facing_out[i] = (uint8_t)f;
    pos_out[i] = tc;  // the target for now; resolved below
  }
}

__global__ void k_na_apply(const unsigned long long *claims, int n, const int32_t *pos,
                           int32_t *pos_out, uint8_t *moved) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tc = pos_out[i];
    const bool won = tc >= 0 && claim_local_slot(claims[tc]) == i;
    pos_out[i] = won ? tc : pos[i];
    moved[i] = won ? 1 : 0;
  }
}

}  // namespace
}  // namespace eco

using namespace eco;

extern "C" int eco_move_claims_noalloc(int32_t side, int32_t n_agents, const int32_t *pos,
                                       const uint8_t *act, const uint8_t *facing_in,
                                       const uint8_t *blocked, uint32_t seed, uint32_t step,
                                       uint8_t *facing_out, int32_t *pos_out, uint8_t *moved,
                                       void *stream) {
  if (side < 4 || (side & 1) || n_agents < 0) return ECO_EINVAL;
  if ((long long)side * side > ECO_NOALLOC_MAX_CELLS) return ECO_EINVAL;
  if (n_agents > 0 && (!pos || !act || !facing_in || !blocked || !facing_out || !pos_out || !moved))
    return ECO_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECO_ECUDA;
  unsigned long long *claims = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_claims_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_move_claims) != cudaSuccess || !p) return ECO_ECUDA;
      g_claims_ptr[dev] = reinterpret_cast<unsigned long long *>(p);
    }
    claims = g_claims_ptr[dev];
  }
  if (n_agents == 0) return ECO_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n_cells = side * side;
  k_na_clear<<<grid_for(n_cells, 256, 1024), 256, 0, s>>>(claims, n_cells);
  k_na_claim<<<grid_for(n_agents, 256, 1024), 256, 0, s>>>(claims, side, n_agents, pos, act,
                                                           facing_in, blocked, seed, step,
                                                           facing_out, pos_out);
  k_na_apply<<<grid_for(n_agents, 256, 1024), 256, 0, s>>>(claims, n_agents, pos, pos_out, moved);
  return cudaGetLastError() == cudaSuccess ? ECO_OK : ECO_ECUDA;
}
