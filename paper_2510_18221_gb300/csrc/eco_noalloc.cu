// eco_noalloc.cu -- move-claim resolution for one world that allocates no
// device memory: the claim scratch lives in a fixed file-scope __device__
// array instead of the caller's workspace.
//
// It applies the same rule as the movement phase of eco_step under the
// simple rule set without ECO_CANCEL_ALL: a move action
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

// Target cell of agent i's move, or -1: a move action (1 N, 2 S, 3 E, 4 W)
// into a neighbour that is not blocked.  An agent whose pos lies outside
// [0, side * side) does not move, so no array is indexed out of range.
__device__ __forceinline__ int na_target(int side, int p, int a, const uint8_t *blocked) {
  if (a < ACT_N || a > ACT_W) return -1;
  if ((unsigned)p >= (unsigned)(side * side)) return -1;
  const int f = (a == ACT_N) ? 0 : (a == ACT_S) ? 2 : (a == ACT_E) ? 1 : 3;
  const int c = step_cell(p, f, side);
  return blocked[c] ? -1 : c;
}

// Facing, and the claim of every mover on its target cell.  Reads act[i],
// facing_in[i] and pos[i] before writing facing_out[i], and writes nothing
// else per agent, so facing_out may alias facing_in.
__global__ void k_na_claim(unsigned long long *claims, int side, int n, const int32_t *pos,
                           const uint8_t *act, const uint8_t *facing_in, const uint8_t *blocked,
                           uint32_t seed, uint32_t step, uint8_t *facing_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int a = act[i];
    int f = facing_in[i] & 3;
    if (a >= ACT_N && a <= ACT_W) {
      f = (a == ACT_N) ? 0 : (a == ACT_S) ? 2 : (a == ACT_E) ? 1 : 3;
      const int tc = na_target(side, pos[i], a, blocked);
      if (tc >= 0) {
        const U4 r = philox(step, (uint32_t)i, 0u, 0u, seed, S_CLAIM_MOVE);
        atomicMax(&claims[tc], claim_key(r.x, i));
      }
    } else if (a == ACT_LEFT) {
      f = (f + 3) & 3;
    } else if (a == ACT_RIGHT) {
      f = (f + 1) & 3;
    }
    facing_out[i] = (uint8_t)f;
  }
}

// Winners move.  The target is recomputed from act[i], pos[i] and blocked
// (unchanged since the claims), and pos[i] is read before pos_out[i] is
// written, so pos_out may alias pos.
__global__ void k_na_apply(const unsigned long long *claims, int side, int n, const int32_t *pos,
                           const uint8_t *act, const uint8_t *blocked, int32_t *pos_out,
                           uint8_t *moved) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = pos[i];
    const int tc = na_target(side, p, act[i], blocked);
    const bool won = tc >= 0 && claim_local_slot(claims[tc]) == i;
    pos_out[i] = won ? tc : p;
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
  if (side < 4 || (side & 1) || n_agents < 0)
    return set_global_error(ECO_EINVAL, "noalloc: side must be even and >= 4, n_agents >= 0");
  if ((long long)side * side > ECO_NOALLOC_MAX_CELLS)
    return set_global_error(ECO_EINVAL, "noalloc: side * side exceeds ECO_NOALLOC_MAX_CELLS (%d)",
                            ECO_NOALLOC_MAX_CELLS);
  if (n_agents > 0 && (!pos || !act || !facing_in || !blocked || !facing_out || !pos_out || !moved))
    return set_global_error(ECO_EINVAL, "noalloc: null array");
  // An error left by earlier, unrelated work is not this call's: report it
  // as pending without clearing it, and launch nothing.
  cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return set_global_error(ECO_ECUDA, "noalloc: a CUDA error was pending before the call: %s",
                            cudaGetErrorString(pending));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_global_error(ECO_ECUDA, "noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_global_error(ECO_ECUDA, "noalloc: device %d out of range", dev);
  unsigned long long *claims = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_claims_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_move_claims);
      if (e != cudaSuccess || !p)
        return set_global_error(ECO_ECUDA, "noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_claims_ptr[dev] = reinterpret_cast<unsigned long long *>(p);
    }
    claims = g_claims_ptr[dev];
  }
  if (n_agents == 0) return ECO_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n_cells = side * side;
  k_na_clear<<<grid_for(n_cells, 256, 1024), 256, 0, s>>>(claims, n_cells);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_global_error(ECO_ECUDA, "noalloc: clear launch: %s", cudaGetErrorString(e));
  k_na_claim<<<grid_for(n_agents, 256, 1024), 256, 0, s>>>(claims, side, n_agents, pos, act,
                                                           facing_in, blocked, seed, step, facing_out);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_global_error(ECO_ECUDA, "noalloc: claim launch: %s", cudaGetErrorString(e));
  k_na_apply<<<grid_for(n_agents, 256, 1024), 256, 0, s>>>(claims, side, n_agents, pos, act, blocked,
                                                           pos_out, moved);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_global_error(ECO_ECUDA, "noalloc: apply launch: %s", cudaGetErrorString(e));
  return ECO_OK;
}
