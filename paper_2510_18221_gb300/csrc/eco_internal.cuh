// eco_internal.cuh -- device-side data layout and helpers shared by the
// library's translation units (not part of the C-ABI).
//
// Layout in HBM (one workspace, carved at create):
//   per cell (all environments concatenated): cellf u8 (bit0 food, bit1
//     wall, bit2 agent), occ i32 (global slot or -1), claim_move u64,
//     cnt_move u32, claim_birth u64, att_cell u64 (this step's attack claim);
//   per slot (all environments concatenated): alive u8, pos i32 (env-local
//     cell y*L+x), facing u8, energy i32, parent i32 (env-local), birth i32,
//     act u8, env u16, tgt i32, gain i32, logits f32[A], hp i32, age i32
//     (paper rules);
//   per cell, paper rules: res i32 (energy lying on the cell; the food bit
//     of cellf is res > 0);
//   per slot: colour f32x4 (the colour trait, RGB + padding);
//   terrain rules: per cell rock, water, bio, flow i32 and photo u32; per
//     slot a_water, a_bio i32;
//   weights: FP32 masters [slot][mstride] and, for BF16/FP8, the streamed
//     copy [slot][stride], both in the kernel's tiled block layout below.
//
// Block layout of one agent's parameters (Sec. 3.3 MLP D -> H -> H -> A),
// element size es (4 FP32, 2 BF16, 1 FP8), E = 16 / es elements per 16-byte
// unit:
//   W1: D x H elements, input-major: element (j, o) at j*H + o.  A 16-byte
//       unit holds E consecutive outputs o of one input j, so one warp load
//       of 32 units is 512 contiguous bytes and each lane keeps a fixed
//       group of E outputs.
//   W2: H x H elements, input-major, the same way.
//   W3: A x H elements, output-major: element (a, j) at a*H + j.
//   [FP8 only] row scales: s1[H], s2[H], s3[A] (FP32), padded to 16 bytes.
//   biases: b1[H], b2[H], b3[A] (FP32), padded to 16 bytes.
//   The block stride is padded to 128 bytes (whole cache lines).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eco.h"

namespace eco {

enum : uint32_t {
  CELL_FOOD = 1u,
  CELL_WALL = 2u,
  CELL_AGENT = 4u,
};

enum : uint32_t {
  S_WALL = 1,
  S_FOOD_INIT = 2,
  S_PLACE = 3,
  S_FACING_INIT = 4,
  S_W_INIT = 5,
  S_SAMPLE = 6,
  S_CLAIM_MOVE = 7,
  S_CLAIM_ATTACK = 8,
  S_CLAIM_BIRTH = 9,
  S_MUTATE = 10,
  S_REGROW = 11,
  S_COLOUR = 12,
  S_BIOMASS = 13,
};

enum : int {
  VISION_CHANNELS = 0,
  VISION_RGB = 1,
  VIEW_AROUND = 0,
  VIEW_FRONT = 1,
};

enum : int {
  ACT_STAY = 0,
  ACT_N = 1,
  ACT_S = 2,
  ACT_E = 3,
  ACT_W = 4,
  ACT_ATTACK = 5,
  ACT_LEFT = 6,
  ACT_RIGHT = 7,
  ACT_EAT = 8,
};

// Paper rule set (Sec. 3.2 "Actions", one resource).
enum : int {
  PA_REST = 0,
  PA_CW = 1,
  PA_CCW = 2,
  PA_FORWARD = 3,
  PA_ATTACK = 4,
  PA_EAT = 5,
  PA_REPRODUCE = 6,
  PA_N = 7,
  TA_DRINK = 7,      // terrain rules
  TA_EAT_BIO = 8,
  TA_N = 9,
};

enum : int {
  RULES_SIMPLE = 0,
  RULES_PAPER = 1,
  RULES_TERRAIN = 2,  // the paper rules plus rock, water and biomass
};

enum : int {
  PREC_FP32 = 0,
  PREC_BF16 = 1,
  PREC_FP8 = 2,
};

enum : int {
  F_AUTO_EAT = 1,
  F_ROTATE_OBS = 2,
  F_CANCEL_ALL = 4,
  F_GREEDY = 8,
};

// Statistic indices (same meaning and order as the public enum).
enum : int {
  ST_STEP = 0,
  ST_AGENT_STEPS,
  ST_ACT0,
  ST_MOVES = ST_ACT0 + 16,
  ST_MOVE_BLOCKED,
  ST_MOVE_LOST,
  ST_EATEN,
  ST_ATTACKS,
  ST_ATTACK_HITS,
  ST_ENERGY_TRANSFERRED,
  ST_DEATHS,
  ST_DEAD_ENERGY,
  ST_BIRTHS,
  ST_FAILED_BIRTHS,
  ST_REGROWN,
  ST_ALIVE,
  ST_FOOD_TOTAL,
  ST_ENERGY_TOTAL,
  ST_RES_TOTAL,
  ST_EATEN_ENERGY,
  ST_METAB_PAID,
  ST_HEALS,
  ST_STARVED,
  ST_DAMAGE,
  ST_FOOD_EMPTIED,
  ST_FOOD_REFILLED,
  ST_WATER_CELLS,
  ST_WATER_AGENTS,
  ST_BIO_CELLS,
  ST_BIO_AGENTS,
  ST_DRUNK,
  ST_WATER_SPENT,
  ST_THIRSTY,
  ST_BIO_EATEN,
  ST_PHOTO,
  ST_DEAD_WATER,
  ST_DEAD_BIO,
  N_ST
};

struct EnvDesc {
  int32_t side;
  int32_t slot_off;   // first global slot of the environment
  int32_t n_slots;
  int32_t cell_off;   // first global cell of the environment
  int32_t init_alive;
  uint32_t seed;
};

// Shape and block layout of one agent's parameters.  Logical order (the
// order of eco_read_params): W_in [H][D], one input bias [H] per sensor,
// L hidden layers (W_l [H][H], b_l [H]), W_out [A][H], b_out [A] (plain form
// only), tau (paper form only).  The plain form is one sensor, L = 1, tanh,
// a biased head and no temperature (W1 b1 W2 b2 W3 b3); the paper form
// (Sec. 3.3) is 2-3 sensors, L hidden layers, ReLU, an unbiased head and
// the log-temperature tau (logits are divided by exp(tau)).
// Tiled block (streamed and master): W_in | W_1..W_L | W_out | [FP8 row
// scales: H + L*H + A] | biases: b_in (ns*H) | b_1..b_L (L*H) | [b_out (A)]
// | [tau].
struct Layout {
  int D, H, A, P;     // observation size, hidden, actions, parameter count
  int L;              // hidden H -> H layers
  int ns;             // sensors (input bias vectors summed into layer 1)
  int relu;           // 1: ReLU, 0: tanh
  int out_bias;       // head has a bias
  int temp;           // a log-temperature parameter follows the biases
  int patch;          // nch k^2: inputs of the vision sensor
  int nch;            // channels per patch cell: 3, or 4 under the terrain rules
  int n_scalars;      // 4, 8 or 16
  int nW, nB;         // weight elements, bias (+ tau) elements
  int es;             // bytes per streamed weight element
  int64_t stride;     // bytes per slot, streamed copy
  int off_w1, off_w2, off_w3, off_scale, off_bias;  // byte offsets, streamed
                                                    // (off_w2: first hidden layer)
  int64_t mstride;    // bytes per slot, FP32 masters
  int moff_w1, moff_w2, moff_w3, moff_bias;          // byte offsets, masters
};

// Logical index of master element q of the tiled block (or -1 for padding).
__host__ __device__ __forceinline__ int layout_logical(const Layout &L, int q) {
  const int D = L.D, H = L.H, A = L.A;
  const int n1 = D * H, nh = L.L * H * H, n3 = A * H;
  const int hid0 = D * H + L.ns * H;  // logical start of hidden layer 0
  if (q < n1) {  // W_in (j, o) at j*H + o
    const int j = q / H, o = q - j * H;
    return o * D + j;
  }
  q -= n1;
  if (q < nh) {  // hidden layer l: (j, o) at l*H*H + j*H + o
    const int l = q / (H * H), r = q - l * H * H;
    const int j = r / H, o = r - j * H;
    return hid0 + l * (H * H + H) + o * H + j;
  }
  q -= nh;
  const int out0 = hid0 + L.L * (H * H + H);
  if (q < n3) return out0 + q;  // W_out (a, j) at a*H + j
  q -= n3;
  if (q < L.ns * H) return D * H + q;  // input biases
  q -= L.ns * H;
  if (q < L.L * H) {  // hidden biases
    const int l = q / H;
    return hid0 + l * (H * H + H) + H * H + (q - l * H);
  }
  q -= L.L * H;
  int k = out0 + n3;
  if (L.out_bias) {
    if (q < A) return k + q;
    q -= A;
    k += A;
  }
  if (L.temp && q == 0) return k;
  return -1;
}

// Fan-in of master weight element q (q < nW): the vision patch, the compass
// one-hot (4 inputs, 8-scalar form) or the internal scalars for W_in in the
// paper form; D for W_in in the plain form; H for hidden layers and the head.
__host__ __device__ __forceinline__ int layout_fan_in(const Layout &L, int q) {
  if (q >= L.D * L.H) return L.H;
  if (!L.relu) return L.D;  // the plain (tanh) form: one input layer over all of x
  const int j = q / L.H;
  if (j < L.patch) return L.patch;
  if (L.n_scalars >= 8 && j >= L.patch + 1 && j < L.patch + 5) return 4;
  return L.n_scalars >= 8 ? L.n_scalars - 4 : L.n_scalars;
}

struct Rules {
  int patch_k, n_scalars, flags, precision;
  float sigma;
  uint32_t thr_food, thr_regrow, thr_wall;
  int e_init, e_metab, e_food, e_repro, attack_num, attack_den;
  int rules;  // RULES_SIMPLE / RULES_PAPER; the rest is paper rules only
  int hp_max, hp_child, attack_damage, heal_rate, heal_cost, age_div, starve_damage;
  int e_act, e_cap, e_child;
  int vision, view;  // VISION_*, VIEW_*
  // terrain rules
  int sea_level, w_init, w_metab, w_bite, w_cap, w_child, heal_water;
  int b_body, b_child, b_bite, b_cap, b_site;
  uint32_t thr_bio;
  int photo_q16, res_cap;
};

// Device pointers (all inside the caller's workspace).
struct Dev {
  const EnvDesc *env;   // [n_envs]
  int n_envs;
  int total_slots;
  int total_cells;
  uint8_t *cellf;
  int32_t *occ;
  unsigned long long *claim_move;
  uint32_t *cnt_move;
  unsigned long long *claim_birth;
  uint8_t *alive;
  int32_t *pos;
  uint8_t *facing;
  int32_t *energy;
  int32_t *parent;
  int32_t *birth;
  uint8_t *act;
  uint16_t *env_of;
  int32_t *tgt;
  int32_t *gain;
  unsigned long long *att_cell;  // [total_cells] this step's attack claim (simple rules:
                                 // the best key; paper rules: the attacker count)
  float *logits;
  int32_t *alive_list;
  int32_t *tile_counts;  // [2][compact tiles] alive slots per tile of 4096, per step parity
                         // (kept by deaths and births)
  unsigned *barrier;     // [BAR_N] grid barrier of the persistent form and its test words
  unsigned long long *trace;  // [kTraceSteps][kTraceWords] phase trace (written only when on)
  int32_t *counters;    // [0] n_alive, [1] n_births, [2] status, [3..] spare
  int2 *births;         // (parent global, child global)
  int32_t *free_list;   // per env: slot_off + rank (free slots in ascending order); one
                        // world's fast birth path: tile * 256 + rank, per tile of 4096 slots
  int32_t *free_tiles;  // [compact tiles] one world: free slots per tile of 4096
  int32_t *birth_contenders;  // [n_envs] count of this step's birth claimants
  int32_t *contenders;        // per env: slot_off + k -> k-th claimant (global slot)
  int32_t *bcell;             // per env: slot_off + k -> its birth cell (env-local)
  long long *stats_step;   // [n_envs][N_ST] this step
  long long *stats_total;  // [n_envs][N_ST]
  long long *stats_last;   // [n_envs][N_ST]
  long long *step;         // [1] current step t (all environments)
  int32_t *alive_at_step;  // [kAliveRing] agents alive at the start of step t, at t % kAliveRing
  float *master;           // [total_slots][mstride / 4]
  uint8_t *wq;             // [total_slots][stride] streamed copy (or == master)
  uint32_t *hist;          // [n_envs][65536] placement radix select
  unsigned long long *place_prefix;  // [n_envs] (prefix, remaining)
  int32_t *place_remaining; // [n_envs] placement radix select
  uint8_t *bflag;          // [total_slots] birth pass flags
  int32_t *hp;             // [total_slots] paper rules: HP (quarter points)
  int32_t *age;            // [total_slots] paper rules: steps survived
  int32_t *res;            // [total_cells] paper rules: energy on the cell
  float4 *colour;          // [total_slots] colour trait (x, y, z = RGB; w = 0)
  // terrain rules
  int32_t *rock;           // [total_cells] rock height (caller's input)
  int32_t *water;          // [total_cells] water on the cell
  int32_t *bio;            // [total_cells] free biomass
  uint32_t *photo;         // [total_cells] photosynthesis remainder (2^-16)
  uint32_t *flow;          // [total_cells] this step's transfer: amount << 2 | direction
  int32_t *a_water;        // [total_slots] water carried
  int32_t *a_bio;          // [total_slots] biomass carried
};

constexpr int kAliveRing = 4096;
// Readable workspace bytes after the last slot's weight block: the policy
// kernel's last, partial FP8 batch of a layer loads up to 32 lanes x 8 units
// x 16 B past the layer's end (and skips those products).
constexpr int kStreamSlack = 4096;

// Words of Dev::barrier: the persistent form's grid-barrier arrival counts
// (one per step parity: a launch uses its step's word and clears the other
// for the next launch) and two failure-detection test words (0 = off: one
// more than the index of a CTA that leaves before its first barrier, and the
// poll budget of the barrier's waits), and the phase-trace switch (0 = off).
enum : int {
  BAR_COUNT0 = 0,
  BAR_COUNT1 = 1,
  BAR_ABSENT_CTA = 2,
  BAR_BUDGET = 3,
  BAR_TRACE = 4,
  BAR_N = 5,
};

// Phase trace of the persistent environment kernel (off unless switched
// on): one row of kTraceWords globaltimer values (ns) per step, row
// step % kTraceSteps.  Words: TR_START CTA 0's start; TR_ARRIVE0 + k the
// last CTA's arrival at grid barrier k (0..3; a CTA records its arrival once
// all its threads are there); TR_PASS0 + k CTA 0's pass through barrier k;
// TR_END the last CTA's end; TR_STEP the step; TR_CLAIMANTS this step's
// birth claimants; TR_BARRIERS the grid barriers the step used.
constexpr int kTraceSteps = ECO_TRACE_STEPS;
constexpr int kTraceWords = ECO_TRACE_WORDS;
enum : int {
  TR_START = 0,
  TR_ARRIVE0 = 1,  // .. 4
  TR_PASS0 = 5,    // .. 8
  TR_END = 9,
  TR_STEP = 10,
  TR_CLAIMANTS = 11,
  TR_BARRIERS = 12,
};

enum : int {
  CNT_N_ALIVE = 0,
  CNT_N_BIRTHS = 1,
  CNT_STATUS = 2,
  CNT_CONTENDERS = 3,  // this step's birth claimants over all environments
  CNT_N = 8,
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds; each round
// multiplies words 0 and 2 by the two round constants, forms the new words
// from the high/low halves xor the other words and the key, then bumps the
// key by the Weyl constants.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t a0 = 0xD2511F53u * c0;
    const uint32_t h0 = __umulhi(0xD2511F53u, c0);
    const uint32_t a2 = 0xCD9E8D57u * c2;
    const uint32_t h2 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = h2 ^ c1 ^ k0;
    const uint32_t n2 = h0 ^ c3 ^ k1;
    c0 = n0;
    c1 = a2;
    c2 = n2;
    c3 = a0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t word_of(const U4 &r, int i) {
  return i == 0 ? r.x : (i == 1 ? r.y : (i == 2 ? r.z : r.w));
}

// Uniform in (0,1): ((r >> 8) | 1) * 2^-24, exact in binary32.
__device__ __forceinline__ float uniform01(uint32_t r) {
  return __uint2float_rn((r >> 8) | 1u) * 5.9604644775390625e-8f;
}

// Standard normal number i (0..3) of a Philox block by Box-Muller on the
// pairs (u0,u1) and (u2,u3).  Uses the CUDA math library's logf, sqrtf and
// sincospif.
__device__ __forceinline__ float normal_of(const U4 &r, int i) {
  const float ua = uniform01(i < 2 ? r.x : r.z);
  const float ub = uniform01(i < 2 ? r.y : r.w);
  const float rad = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  return rad * ((i & 1) ? s : c);
}

// All four normals of a block.
__device__ __forceinline__ void normals4(const U4 &r, float n[4]) {
  const float u0 = uniform01(r.x), u1 = uniform01(r.y);
  const float u2 = uniform01(r.z), u3 = uniform01(r.w);
  const float ra = sqrtf(-2.0f * logf(u0));
  const float rb = sqrtf(-2.0f * logf(u2));
  float s0, c0, s1, c1;
  sincospif(2.0f * u1, &s0, &c0);
  sincospif(2.0f * u3, &s1, &c1);
  n[0] = ra * c0;
  n[1] = ra * s0;
  n[2] = rb * c1;
  n[3] = rb * s1;
}

// Direction vectors N E S W.
__device__ __forceinline__ int dir_dx(int d) { return d == 1 ? 1 : (d == 3 ? -1 : 0); }
__device__ __forceinline__ int dir_dy(int d) { return d == 0 ? -1 : (d == 2 ? 1 : 0); }

__device__ __forceinline__ int wrapi(int v, int L) {
  v %= L;
  return v < 0 ? v + L : v;
}

// Env-local cell one step from local cell c in direction d.
__device__ __forceinline__ int step_cell(int c, int d, int L) {
  const int x = c % L, y = c / L;
  return wrapi(y + dir_dy(d), L) * L + wrapi(x + dir_dx(d), L);
}

// Claim key: the larger wins; the draw first, then the lower env-local slot.
__device__ __forceinline__ unsigned long long claim_key(uint32_t draw, int local_slot) {
  return ((unsigned long long)draw << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)local_slot);
}

__device__ __forceinline__ int claim_local_slot(unsigned long long key) {
  return (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}

// Warp-aggregated add of v to stats[env][idx]: lanes with the same
// (env, idx) combine before one 64-bit atomic.  Integer adds commute, so
// totals do not depend on thread order.  The per-warp partial sum must fit
// in 32 bits (every counter here does).
__device__ __forceinline__ void stat_add(long long *stats, int env, int idx, int v) {
  const unsigned active = __activemask();
  const int key = env * N_ST + idx;
  const unsigned peers = __match_any_sync(active, key);
  const int tot = __reduce_add_sync(peers, v);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && tot != 0)
    atomicAdd((unsigned long long *)&stats[key], (unsigned long long)(long long)tot);
}

// Find the environment of a global cell (environments are sorted by cell
// offset; a short binary search).
__device__ __forceinline__ int env_of_cell(const EnvDesc *env, int n_envs, int cell) {
  int lo = 0, hi = n_envs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (env[mid].cell_off <= cell)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one int per thread (blockDim.x multiple of 32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int *total, int *sh /* >= 33 ints */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  int incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nwarps ? sh[lane] : 0;
    int wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xFFFFFFFFu, wi, off);
      if (lane >= off) wi += o;
    }
    if (lane < nwarps) sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const int excl = sh[warp] + incl - v;
  *total = sh[32];
  __syncthreads();
  return excl;
}

// Launch helpers (host).
int grid_for(long long n, int threads, int max_blocks);

// Record the message eco_last_error(NULL) returns (entry points without a
// handle); returns code.
int set_global_error(int code, const char *fmt, ...);

}  // namespace eco
