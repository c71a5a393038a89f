// eco_env.cu -- the environment phases of one step (Sec. 3.2 "Actions",
// "Resources and Agent Health"; Sec. 3.3 mutation), for every environment
// of the batch at once.
//
// Phase order: alive compaction -> policy (+ facing, turns and move claims,
// fused into its epilogue) -> move apply + eat -> attack claims -> attack
// gains -> metabolism + death -> birth claims -> slot assignment ->
// mutation of the children -> regrowth -> statistics.
//
// Conflicts (two movers into one free cell, two attackers on one victim,
// two parents onto one birth cell) are resolved by a 64-bit atomicMax of
// (Philox draw << 32 | ~local slot): the highest draw wins, equal draws go
// to the lower slot.  A maximum does not depend on the order of the
// atomics, every other atomic is an integer add, and no phase's result
// depends on the order of the alive list, so all integer state is bit-identical from
// run to run and equal to the plain sequential rule.
#include "eco_internal.cuh"
#include "eco_kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace eco {

int grid_for(long long n, int threads, int max_blocks) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// A0: list of alive slots in ascending slot order (Sec. 3.1: the population
// function names the alive agents).  Two kernels over tiles of kCompactTile
// slots: each tile counts its alive slots; then each tile adds up the
// counts of the tiles before it (a few dozen numbers) and writes its slots.
// Slot order keeps the warps of the policy kernel streaming neighbouring
// weight blocks at the same time.
constexpr int kCompactTile = 4096;  // 256 threads x 16 slots

__device__ __forceinline__ uint32_t alive_mask16(const Dev &d, int s0) {
  const int S = d.total_slots;
  uint32_t mask = 0;
  if (s0 + 16 <= S) {
    const uint4 v = *reinterpret_cast<const uint4 *>(d.alive + s0);  // 16-byte aligned
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if ((w[k >> 2] >> ((k & 3) * 8)) & 0xFFu) mask |= 1u << k;
  } else {
    for (int k = 0; k < 16 && s0 + k < S; ++k)
      if (d.alive[s0 + k]) mask |= 1u << k;
  }
  return mask;
}

__global__ void __launch_bounds__(256) k_compact_count(Dev d) {
  __shared__ int sh[33];
  const uint32_t mask = alive_mask16(d, blockIdx.x * kCompactTile + threadIdx.x * 16);
  int total;
  block_exclusive_scan(__popc(mask), &total, sh);
  if (threadIdx.x == 0) d.tile_counts[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_compact_scatter(Dev d) {
  __shared__ int sh[33];
  int before = 0;
  for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) before += d.tile_counts[k];
  int base;
  block_exclusive_scan(before, &base, sh);  // base = sum over the earlier tiles
  const int s0 = blockIdx.x * kCompactTile + threadIdx.x * 16;
  uint32_t mask = alive_mask16(d, s0);
  int total;
  int at = base + block_exclusive_scan(__popc(mask), &total, sh);
  while (mask) {
    const int k = __ffs(mask) - 1;
    d.alive_list[at++] = s0 + k;
    mask &= mask - 1;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) d.counters[CNT_N_ALIVE] = base + total;
}

// A6 (part 2) + A7: winners move (only the winner of a cell writes it, and
// a winner's old cell was occupied when the step began, so nobody moves
// into it); then every agent eats the food of its post-move cell, when the
// rules say it eats.  Nobody else can be on that cell.
__global__ void k_move_apply_eat(Dev d, Rules R, int n_actions) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    const int e = d.env_of[slot];
    const EnvDesc ed = d.env[e];
    const int tc = d.tgt[slot];
    int pos = d.pos[slot];
    if (tc >= 0) {
      const int gc = ed.cell_off + tc;
      bool won = claim_local_slot(d.claim_move[gc]) == slot - ed.slot_off;
      if (R.flags & F_CANCEL_ALL) won = won && d.cnt_move[gc] == 1u;
      if (won) {
        const int old = ed.cell_off + pos;
        d.occ[old] = -1;
        d.cellf[old] &= (uint8_t)~CELL_AGENT;
        d.occ[gc] = slot;
        d.cellf[gc] |= (uint8_t)CELL_AGENT;
        d.pos[slot] = tc;
        pos = tc;
        stat_add(d.stats_step, e, ST_MOVES, 1);
      } else {
        stat_add(d.stats_step, e, ST_MOVE_LOST, 1);
      }
    }
    const int a = d.act[slot];
    if ((R.flags & F_AUTO_EAT) || (n_actions > ACT_EAT && a == ACT_EAT)) {
      const int gpos = ed.cell_off + pos;
      const uint8_t cf = d.cellf[gpos];
      if (cf & CELL_FOOD) {
        d.cellf[gpos] = (uint8_t)(cf & ~CELL_FOOD);
        d.energy[slot] += R.e_food;
        stat_add(d.stats_step, e, ST_EATEN, 1);
      }
    }
  }
}

// A8 (part 1): clear this step's move claims; attackers claim the agent on
// the faced cell (post-move occupancy).
__global__ void k_attack_claim(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  const uint32_t t = (uint32_t)d.step[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    const int e = d.env_of[slot];
    const EnvDesc ed = d.env[e];
    const int tc = d.tgt[slot];
    if (tc >= 0) {
      d.claim_move[ed.cell_off + tc] = 0ull;
      if (R.flags & F_CANCEL_ALL) d.cnt_move[ed.cell_off + tc] = 0u;
    }
    int victim = -1;
    if (d.act[slot] == ACT_ATTACK) {
      const int c = step_cell(d.pos[slot], d.facing[slot], ed.side);
      const int v = d.occ[ed.cell_off + c];
      if (v >= 0) {
        const int local = slot - ed.slot_off;
        const U4 r = philox(t, (uint32_t)local, 0u, 0u, ed.seed, S_CLAIM_ATTACK);
        atomicMax(&d.claim_att[v], claim_key(r.x, local));
        victim = v;
      }
    }
    d.tgt[slot] = victim;
  }
}

// A8 (part 2): the winning attacker of each victim takes floor(e * num /
// den) of the victim's post-eat energy (read here, written only later).
__global__ void k_attack_gain(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    const int v = d.tgt[slot];
    int g = 0;
    if (v >= 0) {
      const int e = d.env_of[slot];
      const int local = slot - d.env[e].slot_off;
      if (claim_local_slot(d.claim_att[v]) == local) {
        g = (int)(((long long)d.energy[v] * R.attack_num) / R.attack_den);
        stat_add(d.stats_step, e, ST_ATTACK_HITS, 1);
        stat_add(d.stats_step, e, ST_ENERGY_TRANSFERRED, g);
      }
    }
    d.gain[slot] = g;
  }
}

// A8 (part 3) + A9: apply the transfer, pay metabolism, die at e <= 0.
__global__ void k_metab_death(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    int en = d.energy[slot];
    const unsigned long long ca = d.claim_att[slot];
    const int loss = ca ? (int)(((long long)en * R.attack_num) / R.attack_den) : 0;
    if (ca) d.claim_att[slot] = 0ull;
    en = en - loss + d.gain[slot] - R.e_metab;
    if (en <= 0) {
      const int e = d.env_of[slot];
      const int gpos = d.env[e].cell_off + d.pos[slot];
      d.alive[slot] = 0;
      d.occ[gpos] = -1;
      d.cellf[gpos] &= (uint8_t)~CELL_AGENT;
      stat_add(d.stats_step, e, ST_DEATHS, 1);
      stat_add(d.stats_step, e, ST_DEAD_ENERGY, en);
      en = 0;
    }
    d.energy[slot] = en;
  }
}

// A10 (part 1): agents with e >= e_repro claim the free non-wall cell
// behind them and join their environment's contender list.
__global__ void k_birth_claim(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  const uint32_t t = (uint32_t)d.step[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    int bt = -1;
    if (d.alive[slot] && d.energy[slot] >= R.e_repro) {
      const int e = d.env_of[slot];
      const EnvDesc ed = d.env[e];
      const int c = step_cell(d.pos[slot], (d.facing[slot] + 2) & 3, ed.side);
      const int gc = ed.cell_off + c;
      if (!(d.cellf[gc] & (CELL_WALL | CELL_AGENT))) {
        const int local = slot - ed.slot_off;
        const U4 r = philox(t, (uint32_t)local, 0u, 0u, ed.seed, S_CLAIM_BIRTH);
        atomicMax(&d.claim_birth[gc], claim_key(r.x, local));
        const int k = atomicAdd(&d.birth_contenders[e], 1);
        d.contenders[ed.slot_off + k] = slot;
        bt = c;
      }
    }
    d.tgt[slot] = bt;
  }
}

// Give winner p (global slot) the child slot c (global) behind it.
__device__ __forceinline__ void make_child(const Dev &d, const EnvDesc &ed, int p, int c, int bt,
                                           uint32_t t) {
  const int en = d.energy[p];
  const int ce = en / 2;
  d.energy[p] = en - ce;
  d.energy[c] = ce;
  d.alive[c] = 1;
  d.pos[c] = bt;
  d.facing[c] = d.facing[p];
  d.parent[c] = p - ed.slot_off;
  d.birth[c] = (int)t;
  d.occ[ed.cell_off + bt] = c;
  d.cellf[ed.cell_off + bt] |= (uint8_t)CELL_AGENT;
  const int b = atomicAdd(&d.counters[CNT_N_BIRTHS], 1);
  d.births[b] = make_int2(p, c);
}

// A10 (part 2): one CTA per environment.  Cell winners in ascending slot
// order take the free slots in ascending order; the child gets floor(e/2)
// of the parent's energy, the parent's facing, and the cell behind.
// Winners (at most kBirthCap per step) are sorted in shared memory; only
// the first n_winners free slots are searched for.  More contenders than
// kBirthCap fall back to a full scan of the environment's slots.
constexpr int kBirthCap = 2048;

__global__ void __launch_bounds__(1024) k_birth_assign(Dev d) {
  __shared__ int sh[33];
  __shared__ int s_win[kBirthCap];
  __shared__ int s_free[kBirthCap];
  __shared__ int s_nwin, s_nfree;
  const int e = blockIdx.x;
  const int nc = d.birth_contenders[e];
  if (nc == 0) return;  // uniform across the CTA
  const EnvDesc ed = d.env[e];
  const uint32_t t = (uint32_t)d.step[0];
  const int tid = threadIdx.x, nt = blockDim.x;

  if (nc <= kBirthCap) {
    int p2 = 1;
    while (p2 < nc) p2 <<= 1;
    for (int i = tid; i < p2; i += nt) {
      int v = 0x7FFFFFFF;
      if (i < nc) {
        const int g = d.contenders[ed.slot_off + i];
        const int bt = d.tgt[g];
        if (claim_local_slot(d.claim_birth[ed.cell_off + bt]) == g - ed.slot_off) v = g;
      }
      s_win[i] = v;
    }
    __syncthreads();
    // bitonic sort of s_win[0, p2) ascending
    for (int k = 2; k <= p2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < p2; i += nt) {
          const int l = i ^ j;
          if (l > i) {
            const int a = s_win[i], b = s_win[l];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              s_win[i] = b;
              s_win[l] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      int nw = 0;
      while (nw < p2 && s_win[nw] != 0x7FFFFFFF) ++nw;
      s_nwin = nw;
    }
    __syncthreads();
    const int nwin = s_nwin;
    // the first nwin free slots, 16 slots per thread per pass
    int found = 0;
    for (int base = 0; base < ed.n_slots && found < nwin; base += nt * 16) {
      const int s0 = base + tid * 16;
      uint32_t mask = 0;
      for (int k = 0; k < 16; ++k) {
        const int s = s0 + k;
        if (s < ed.n_slots && !d.alive[ed.slot_off + s]) mask |= 1u << k;
      }
      int total;
      int r = found + block_exclusive_scan(__popc(mask), &total, sh);
      while (mask && r < nwin) {
        const int k = __ffs(mask) - 1;
        s_free[r++] = s0 + k;
        mask &= mask - 1;
      }
      found += total;
      __syncthreads();
    }
    const int nfree = found < nwin ? found : nwin;
    int born = 0, failed = 0;
    for (int i = tid; i < nwin; i += nt) {
      const int p = s_win[i];
      const int bt = d.tgt[p];
      d.claim_birth[ed.cell_off + bt] = 0ull;
      if (i < nfree) {
        make_child(d, ed, p, ed.slot_off + s_free[i], bt, t);
        ++born;
      } else {
        ++failed;
      }
    }
    if (born) atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_BIRTHS], (unsigned long long)born);
    if (failed)
      atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_FAILED_BIRTHS], (unsigned long long)failed);
    return;
  }

  // Fallback: full scan over the environment's slots (more than kBirthCap
  // contenders this step).
  const int n = ed.n_slots;
  const int per = (n + nt - 1) / nt;
  const int beg = min(n, tid * per), end = min(n, beg + per);
  int nfree = 0, nwin = 0;
  for (int s = beg; s < end; ++s) {
    const int g = ed.slot_off + s;
    uint8_t fl = 0;
    if (!d.alive[g]) {
      fl = 1;
      ++nfree;
    } else {
      const int bt = d.tgt[g];
      if (bt >= 0 && claim_local_slot(d.claim_birth[ed.cell_off + bt]) == s) {
        fl = 2;
        ++nwin;
      }
    }
    d.bflag[g] = fl;
  }
  int free_total, win_total;
  int free_off = block_exclusive_scan(nfree, &free_total, sh);
  int win_off = block_exclusive_scan(nwin, &win_total, sh);
  for (int s = beg; s < end; ++s)
    if (d.bflag[ed.slot_off + s] == 1) d.free_list[ed.slot_off + free_off++] = s;
  __syncthreads();
  int failed = 0, born = 0;
  for (int s = beg; s < end; ++s) {
    const int p = ed.slot_off + s;
    if (d.bflag[p] != 2) continue;
    const int r = win_off++;
    const int bt = d.tgt[p];
    d.claim_birth[ed.cell_off + bt] = 0ull;
    if (r >= free_total) {
      ++failed;
      continue;
    }
    make_child(d, ed, p, ed.slot_off + d.free_list[ed.slot_off + r], bt, t);
    ++born;
  }
  if (born) atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_BIRTHS], (unsigned long long)born);
  if (failed)
    atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_FAILED_BIRTHS], (unsigned long long)failed);
}

// ---------------------------------------------------------------------------
// A11: mutation (Sec. 3.3): child = fl32(parent + sigma * n) on every
// parameter, n ~ N(0,1) from stream MUTATE at counter (step, parent's local
// slot, p / 4) for logical parameter p; then the child's streamed BF16 /
// FP8 copy is re-derived from its new master.
//
// Work items per birth: H/16 tiles of W1 (16 output rows x all D inputs),
// H/16 tiles of W2, and one item for W3 and the biases.  A tile draws its
// normals in logical order (one Philox block per four parameters) into
// shared memory, then walks the master in its physical (input-major) order
// so global reads and writes are contiguous; FP8 row scales come from the
// tile's complete rows.
// ---------------------------------------------------------------------------
constexpr int kMutRows = 16;

__device__ __forceinline__ uint8_t e4m3_sat(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__global__ void __launch_bounds__(256) k_mutate(Dev d, Layout L, Rules R) {
  extern __shared__ __align__(16) float msm[];
  __shared__ float s_scale[kMutRows + 16];
  const int D = L.D, H = L.H, A = L.A;
  const int nb = d.counters[CNT_N_BIRTHS];
  const int tiles = H / kMutRows;
  const int items = 2 * tiles + 1;
  const uint32_t t = (uint32_t)d.step[0];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int64_t mper = L.mstride / 4;

  for (int w = blockIdx.x; w < nb * items; w += gridDim.x) {
    const int b = w / items, it = w - b * items;
    const int2 pc = d.births[b];
    const EnvDesc ed = d.env[d.env_of[pc.y]];
    const uint32_t lp = (uint32_t)(pc.x - ed.slot_off);
    const float *pm = d.master + (int64_t)pc.x * mper;
    float *cm = d.master + (int64_t)pc.y * mper;
    uint8_t *cq = d.wq + (int64_t)pc.y * L.stride;
    if (it < 2 * tiles) {
      const bool l1 = it < tiles;
      const int o0 = (l1 ? it : it - tiles) * kMutRows;
      const int nin = l1 ? D : H;
      const int rs = nin + 1;  // padded shared-memory row stride
      const int lbase = l1 ? o0 * D : D * H + H + o0 * H;  // logical (o0, 0)
      const int qbase = l1 ? 0 : D * H;                    // physical layer start
      const int nel = kMutRows * nin;
      const int g0 = lbase >> 2, g1 = (lbase + nel - 1) >> 2;
      for (int g = g0 + tid; g <= g1; g += nt) {
        const U4 r = philox(t, lp, (uint32_t)g, 0u, ed.seed, S_MUTATE);
        float n4[4];
        normals4(r, n4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int off = 4 * g + k - lbase;
          if (off >= 0 && off < nel) {
            const int rr = off / nin, j = off - rr * nin;
            msm[rr * rs + j] = n4[k];
          }
        }
      }
      __syncthreads();
      for (int idx = tid; idx < nel; idx += nt) {
        const int j = idx >> 4, rr = idx & (kMutRows - 1);
        const int q = qbase + j * H + o0 + rr;
        const float v = fmaf(R.sigma, msm[rr * rs + j], pm[q]);
        cm[q] = v;
        msm[rr * rs + j] = v;
      }
      __syncthreads();
      if (R.precision == PREC_BF16) {
        __nv_bfloat16 *qw = reinterpret_cast<__nv_bfloat16 *>(cq);
        for (int idx = tid; idx < nel; idx += nt) {
          const int j = idx >> 4, rr = idx & (kMutRows - 1);
          qw[qbase + j * H + o0 + rr] = __float2bfloat16_rn(msm[rr * rs + j]);
        }
      } else if (R.precision == PREC_FP8) {
        for (int rr = warp; rr < kMutRows; rr += nw) {
          float mx = 0.0f;
          for (int j = lane; j < nin; j += 32) mx = fmaxf(mx, fabsf(msm[rr * rs + j]));
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
          float s = __fdiv_rn(mx, 448.0f);
          if (s == 0.0f) s = 1.0f;
          if (lane == 0) {
            s_scale[rr] = s;
            reinterpret_cast<float *>(cq + L.off_scale)[(l1 ? 0 : H) + o0 + rr] = s;
          }
        }
        __syncthreads();
        for (int idx = tid; idx < nel; idx += nt) {
          const int j = idx >> 4, rr = idx & (kMutRows - 1);
          cq[qbase + j * H + o0 + rr] = e4m3_sat(__fdiv_rn(msm[rr * rs + j], s_scale[rr]));
        }
      }
      __syncthreads();
    } else {
      // W3 (output-major, logical order = physical order) and the biases
      const int n3 = A * H, nbias = 2 * H + A;
      const int l3 = D * H + 2 * H + H * H;  // logical start of W3
      const int q3 = D * H + H * H;          // physical start of W3
      const int qb = L.moff_bias / 4;
      for (int e = tid; e < n3 + nbias; e += nt) {
        int p, q;
        if (e < n3) {
          p = l3 + e;
          q = q3 + e;
        } else {
          const int k = e - n3;
          q = qb + k;
          p = (k < H) ? D * H + k : (k < 2 * H) ? D * H + H + H * H + (k - H)
                                               : D * H + 2 * H + H * H + A * H + (k - 2 * H);
        }
        const U4 r = philox(t, lp, (uint32_t)(p >> 2), 0u, ed.seed, S_MUTATE);
        const float v = fmaf(R.sigma, normal_of(r, p & 3), pm[q]);
        cm[q] = v;
        if (e < n3) msm[e] = v;
        else if (R.precision != PREC_FP32) reinterpret_cast<float *>(cq + L.off_bias)[e - n3] = v;
      }
      __syncthreads();
      if (R.precision == PREC_BF16) {
        __nv_bfloat16 *qw = reinterpret_cast<__nv_bfloat16 *>(cq);
        for (int e = tid; e < n3; e += nt) qw[q3 + e] = __float2bfloat16_rn(msm[e]);
      } else if (R.precision == PREC_FP8) {
        for (int a = warp; a < A; a += nw) {
          float mx = 0.0f;
          for (int j = lane; j < H; j += 32) mx = fmaxf(mx, fabsf(msm[a * H + j]));
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
          float s = __fdiv_rn(mx, 448.0f);
          if (s == 0.0f) s = 1.0f;
          if (lane == 0) reinterpret_cast<float *>(cq + L.off_scale)[2 * H + a] = s;
          for (int j = lane; j < H; j += 32) cq[q3 + a * H + j] = e4m3_sat(__fdiv_rn(msm[a * H + j], s));
        }
      }
      __syncthreads();
    }
  }
}

size_t mutate_smem_bytes(const Layout &L) {
  const size_t tile = (size_t)kMutRows * (L.D + 1);
  const size_t head = (size_t)L.A * L.H;
  return 4 * (tile > head ? tile : head);
}

// A12: regrowth of food on non-wall food-less cells; four cells per thread
// share one Philox block (counter (step, local cell / 4)).
__global__ void k_regrow(Dev d, Rules R) {
  const int groups = d.total_cells >> 2;
  const uint32_t t = (uint32_t)d.step[0];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
    const int c0 = g << 2;
    const int e = env_of_cell(d.env, d.n_envs, c0);
    const EnvDesc ed = d.env[e];
    uchar4 cf = reinterpret_cast<uchar4 *>(d.cellf)[g];
    int grown = 0;
    const bool any = !((cf.x & (CELL_WALL | CELL_FOOD)) && (cf.y & (CELL_WALL | CELL_FOOD)) &&
                       (cf.z & (CELL_WALL | CELL_FOOD)) && (cf.w & (CELL_WALL | CELL_FOOD)));
    if (any) {
      const U4 r = philox(t, (uint32_t)((c0 - ed.cell_off) >> 2), 0u, 0u, ed.seed, S_REGROW);
      if (!(cf.x & (CELL_WALL | CELL_FOOD)) && r.x < R.thr_regrow) { cf.x |= CELL_FOOD; ++grown; }
      if (!(cf.y & (CELL_WALL | CELL_FOOD)) && r.y < R.thr_regrow) { cf.y |= CELL_FOOD; ++grown; }
      if (!(cf.z & (CELL_WALL | CELL_FOOD)) && r.z < R.thr_regrow) { cf.z |= CELL_FOOD; ++grown; }
      if (!(cf.w & (CELL_WALL | CELL_FOOD)) && r.w < R.thr_regrow) { cf.w |= CELL_FOOD; ++grown; }
      if (grown) reinterpret_cast<uchar4 *>(d.cellf)[g] = cf;
    }
    stat_add(d.stats_step, e, ST_REGROWN, grown);
  }
}

// A13: fold this step's counters into the per-environment records and
// advance the step counter.  Agent-steps and attacks come from the action
// histogram the policy kernel counted.
__global__ void k_finish(Dev d, Rules R) {
  const long long t = d.step[0];
  for (int i = threadIdx.x; i < d.n_envs; i += blockDim.x) {
    long long *st = d.stats_step + i * N_ST;
    long long as = 0;
    for (int a = 0; a < 16; ++a) as += st[ST_ACT0 + a];
    st[ST_AGENT_STEPS] = as;
    st[ST_ATTACKS] = st[ST_ACT0 + ACT_ATTACK];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_envs * N_ST; i += blockDim.x) {
    const int e = i / N_ST, k = i - e * N_ST;
    long long *st = d.stats_step + e * N_ST;
    long long *tot = d.stats_total + e * N_ST;
    long long *last = d.stats_last + e * N_ST;
    long long v;
    if (k == ST_STEP) {
      v = t + 1;
    } else if (k == ST_ALIVE) {
      v = tot[k] + st[ST_BIRTHS] - st[ST_DEATHS];
    } else if (k == ST_FOOD_TOTAL) {
      v = tot[k] + st[ST_REGROWN] - st[ST_EATEN];
    } else if (k == ST_ENERGY_TOTAL) {
      v = tot[k] + (long long)R.e_food * st[ST_EATEN] - (long long)R.e_metab * st[ST_AGENT_STEPS] -
          st[ST_DEAD_ENERGY];
    } else {
      last[k] = st[k];
      tot[k] += st[k];
      continue;
    }
    last[k] = v;
    tot[k] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_envs * N_ST; i += blockDim.x) d.stats_step[i] = 0;
  for (int i = threadIdx.x; i < d.n_envs; i += blockDim.x) d.birth_contenders[i] = 0;
  if (threadIdx.x == 0) {
    d.step[0] = t + 1;
    d.counters[CNT_N_BIRTHS] = 0;
  }
}

int compact_tiles(int total_slots) { return (total_slots + kCompactTile - 1) / kCompactTile; }

cudaError_t launch_compact(const Dev &d, cudaStream_t s) {
  const int tiles = compact_tiles(d.total_slots);
  k_compact_count<<<tiles, 256, 0, s>>>(d);
  k_compact_scatter<<<tiles, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t env_prepare(const Layout &L) {
  const size_t smem = mutate_smem_bytes(L);
  return cudaFuncSetAttribute((const void *)k_mutate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t launch_env_phases(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                              cudaStream_t s) {
  const int T = 256;
  k_move_apply_eat<<<g.slot_blocks, T, 0, s>>>(d, R, L.A);
  k_attack_claim<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_attack_gain<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_metab_death<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_claim<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_assign<<<d.n_envs, 1024, 0, s>>>(d);
  k_mutate<<<g.birth_blocks, 256, mutate_smem_bytes(L), s>>>(d, L, R);
  k_regrow<<<g.cell_blocks, T, 0, s>>>(d, R);
  k_finish<<<1, 1024, 0, s>>>(d, R);
  return cudaGetLastError();
}

}  // namespace eco
