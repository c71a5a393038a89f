// eco_env.cu -- the environment phases of one step (Sec. 3.2 "Actions",
// "Resources and Agent Health"; Sec. 3.3 mutation), for every environment
// of the batch at once.
//
// Phase order: alive compaction -> [policy] -> face/turn + move claims ->
// move apply -> eat + attack claims -> attack gains -> metabolism + death ->
// birth claims -> slot assignment -> mutation of the children -> regrowth
// -> statistics.
//
// Conflicts (two movers into one free cell, two attackers on one victim,
// two parents onto one birth cell) are resolved by a 64-bit atomicMax of
// (Philox draw << 32 | ~local slot): the highest draw wins, equal draws go
// to the lower slot.  A maximum does not depend on the order of the
// atomics, and every other atomic is an integer add, so all integer state
// is bit-identical from run to run and equal to the plain sequential rule.
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
// function names the alive agents).  One CTA; each thread owns a contiguous
// chunk of slots.
__global__ void __launch_bounds__(1024) k_compact(Dev d) {
  __shared__ int sh[33];
  const int S = d.total_slots;
  const int per = (S + blockDim.x - 1) / blockDim.x;
  const int beg = min(S, (int)threadIdx.x * per), end = min(S, beg + per);
  int cnt = 0;
  for (int s = beg; s < end; ++s) cnt += d.alive[s];
  int total;
  int off = block_exclusive_scan(cnt, &total, sh);
  for (int s = beg; s < end; ++s)
    if (d.alive[s]) d.alive_list[off++] = s;
  if (threadIdx.x == 0) d.counters[CNT_N_ALIVE] = total;
}

// A6 (part 1): facing and turns; move claims on cells that are free and not
// walls when the step begins.
__global__ void k_move_claim(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  const uint32_t t = (uint32_t)d.step[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    const int e = d.env_of[slot];
    const EnvDesc ed = d.env[e];
    const int a = d.act[slot];
    int f = d.facing[slot];
    stat_add(d.stats_step, e, ST_AGENT_STEPS, 1);
    stat_add(d.stats_step, e, ST_ACT0 + a, 1);
    int tc = -1;
    if (a >= ACT_N && a <= ACT_W) {
      f = (a == ACT_N) ? 0 : (a == ACT_S) ? 2 : (a == ACT_E) ? 1 : 3;
      const int c = step_cell(d.pos[slot], f, ed.side);
      const int gc = ed.cell_off + c;
      if (d.cellf[gc] & (CELL_WALL | CELL_AGENT)) {
        stat_add(d.stats_step, e, ST_MOVE_BLOCKED, 1);
      } else {
        const int local = slot - ed.slot_off;
        const U4 r = philox(t, (uint32_t)local, 0u, 0u, ed.seed, S_CLAIM_MOVE);
        atomicMax(&d.claim_move[gc], claim_key(r.x, local));
        if (R.flags & F_CANCEL_ALL) atomicAdd(&d.cnt_move[gc], 1u);
        tc = c;
      }
    } else if (a == ACT_LEFT) {
      f = (f + 3) & 3;
    } else if (a == ACT_RIGHT) {
      f = (f + 1) & 3;
    } else if (a == ACT_ATTACK) {
      stat_add(d.stats_step, e, ST_ATTACKS, 1);
    }
    d.facing[slot] = (uint8_t)f;
    d.tgt[slot] = tc;
  }
}

// A6 (part 2): winners move.  Only the winner of a cell writes it, and a
// winner's old cell was occupied at the start of the step, so nobody else
// moves into it.
__global__ void k_move_apply(Dev d, Rules R) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = d.alive_list[i];
    const int tc = d.tgt[slot];
    if (tc < 0) continue;
    const int e = d.env_of[slot];
    const EnvDesc ed = d.env[e];
    const int local = slot - ed.slot_off;
    const int gc = ed.cell_off + tc;
    bool won = claim_local_slot(d.claim_move[gc]) == local;
    if (R.flags & F_CANCEL_ALL) won = won && d.cnt_move[gc] == 1u;
    if (won) {
      const int old = ed.cell_off + d.pos[slot];
      d.occ[old] = -1;
      d.cellf[old] &= (uint8_t)~CELL_AGENT;
      d.occ[gc] = slot;
      d.cellf[gc] |= (uint8_t)CELL_AGENT;
      d.pos[slot] = tc;
      stat_add(d.stats_step, e, ST_MOVES, 1);
    } else {
      stat_add(d.stats_step, e, ST_MOVE_LOST, 1);
    }
  }
}

// A7 + A8 (part 1): clear this step's move claims, eat, and claim victims.
__global__ void k_eat_attack_claim(Dev d, Rules R, int n_actions) {
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
    const int a = d.act[slot];
    const int pos = d.pos[slot];
    const int gpos = ed.cell_off + pos;
    if ((R.flags & F_AUTO_EAT) || (n_actions > ACT_EAT && a == ACT_EAT)) {
      const uint8_t cf = d.cellf[gpos];
      if (cf & CELL_FOOD) {
        d.cellf[gpos] = (uint8_t)(cf & ~CELL_FOOD);
        d.energy[slot] += R.e_food;
        stat_add(d.stats_step, e, ST_EATEN, 1);
      }
    }
    int victim = -1;
    if (a == ACT_ATTACK) {
      const int c = step_cell(pos, d.facing[slot], ed.side);
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

// A10 (part 1): agents with e >= e_repro claim the free non-wall cell behind.
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
        atomicAdd(&d.birth_contenders[e], 1);
        bt = c;
      }
    }
    d.tgt[slot] = bt;
  }
}

// A10 (part 2): one CTA per environment.  Cell winners in ascending slot
// order take the free slots in ascending order; the child gets floor(e/2)
// of the parent's energy, the parent's facing, and the cell behind.
__global__ void __launch_bounds__(1024) k_birth_assign(Dev d) {
  __shared__ int sh[33];
  const int e = blockIdx.x;
  if (d.birth_contenders[e] == 0) return;  // uniform across the CTA
  const EnvDesc ed = d.env[e];
  const uint32_t t = (uint32_t)d.step[0];
  const int n = ed.n_slots;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per), end = min(n, beg + per);
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
    const int c = ed.slot_off + d.free_list[ed.slot_off + r];
    const int en = d.energy[p];
    const int ce = en / 2;
    d.energy[p] = en - ce;
    d.energy[c] = ce;
    d.alive[c] = 1;
    d.pos[c] = bt;
    d.facing[c] = d.facing[p];
    d.parent[c] = s;
    d.birth[c] = (int)t;
    d.occ[ed.cell_off + bt] = c;
    d.cellf[ed.cell_off + bt] |= (uint8_t)CELL_AGENT;
    const int b = atomicAdd(&d.counters[CNT_N_BIRTHS], 1);
    d.births[b] = make_int2(p, c);
    ++born;
  }
  if (born) atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_BIRTHS], (unsigned long long)born);
  if (failed)
    atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_FAILED_BIRTHS], (unsigned long long)failed);
}

// ---------------------------------------------------------------------------
// A11: mutation (Sec. 3.3).  One CTA per birth: child = fl32(parent + sigma
// * n) on every parameter, n ~ N(0,1) from stream MUTATE at counter (step,
// parent's local slot, p / 4) for logical parameter p; then the streamed
// BF16 / FP8 copy of the child is re-derived.
// ---------------------------------------------------------------------------

// Logical index (W1, b1, W2, b2, W3, b3 order) of master element q of the
// tiled block, or -1 for padding.
__device__ __forceinline__ int master_logical(const Layout &L, int q) {
  const int D = L.D, H = L.H, A = L.A;
  const int n1 = D * H, n2 = H * H, n3 = A * H;
  if (q < n1) {  // W1 (j, o) at j*H + o
    const int j = q / H, o = q - j * H;
    return o * D + j;
  }
  q -= n1;
  if (q < n2) {  // W2 (j, o)
    const int j = q / H, o = q - j * H;
    return D * H + H + o * H + j;
  }
  q -= n2;
  if (q < n3) return D * H + 2 * H + H * H + q;  // W3 (a, j) at a*H + j
  q -= n3;
  if (q < H) return D * H + q;                      // b1
  if (q < 2 * H) return D * H + H + H * H + (q - H); // b2
  if (q < 2 * H + A) return D * H + 2 * H + H * H + A * H + (q - 2 * H);  // b3
  return -1;
}

__device__ __forceinline__ uint8_t e4m3_sat(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// Re-derive the streamed copy of one slot from its FP32 master (whole CTA).
__device__ void requant_slot(const Dev &d, const Layout &L, int prec, int slot) {
  if (prec == PREC_FP32) return;
  const int H = L.H, A = L.A;
  const int nW = L.D * H + H * H + A * H;  // weight elements, same order in both
  const float *m = d.master + (int64_t)slot * (L.mstride / 4);
  uint8_t *q = d.wq + (int64_t)slot * L.stride;
  const float *mb = m + L.moff_bias / 4;
  float *qb = reinterpret_cast<float *>(q + L.off_bias);
  for (int i = threadIdx.x; i < 2 * H + A; i += blockDim.x) qb[i] = mb[i];
  if (prec == PREC_BF16) {
    __nv_bfloat16 *qw = reinterpret_cast<__nv_bfloat16 *>(q);
    for (int i = threadIdx.x; i < nW; i += blockDim.x) qw[i] = __float2bfloat16_rn(m[i]);
    return;
  }
  // FP8: one warp per output row; s = max|w| / 448 (IEEE binary32 division),
  // 1 for an all-zero row; codes = satfinite RNE e4m3(w / s).
  float *qs = reinterpret_cast<float *>(q + L.off_scale);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < 2 * H + A; row += nw) {
    int base, stride, n;
    if (row < H) { base = row; stride = H; n = L.D; }                        // W1 row o
    else if (row < 2 * H) { base = L.D * H + (row - H); stride = H; n = H; }  // W2 row o
    else { base = L.D * H + H * H + (row - 2 * H) * H; stride = 1; n = H; }  // W3 row a
    float mx = 0.0f;
    for (int j = lane; j < n; j += 32) mx = fmaxf(mx, fabsf(m[base + j * stride]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    float s = __fdiv_rn(mx, 448.0f);
    if (s == 0.0f) s = 1.0f;
    if (lane == 0) qs[row] = s;
    for (int j = lane; j < n; j += 32) {
      const int idx = base + j * stride;
      q[idx] = e4m3_sat(__fdiv_rn(m[idx], s));
    }
  }
}

__global__ void __launch_bounds__(256) k_mutate(Dev d, Layout L, Rules R) {
  const int nb = d.counters[CNT_N_BIRTHS];
  const uint32_t t = (uint32_t)d.step[0];
  const int total = L.D * L.H + L.H * L.H + L.A * L.H + 2 * L.H + L.A;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const int2 pc = d.births[b];
    const EnvDesc ed = d.env[d.env_of[pc.y]];
    const uint32_t lp = (uint32_t)(pc.x - ed.slot_off);
    const float *pm = d.master + (int64_t)pc.x * (L.mstride / 4);
    float *cm = d.master + (int64_t)pc.y * (L.mstride / 4);
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int p = master_logical(L, q);
      const U4 r = philox(t, lp, (uint32_t)(p >> 2), 0u, ed.seed, S_MUTATE);
      const float nrm = normal_of(r, p & 3);
      cm[q] = fmaf(R.sigma, nrm, pm[q]);
    }
    __syncthreads();
    requant_slot(d, L, R.precision, pc.y);
    __syncthreads();
  }
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
// advance the step counter.
__global__ void k_finish(Dev d, Rules R) {
  const long long t = d.step[0];
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

cudaError_t launch_compact(const Dev &d, cudaStream_t s) {
  k_compact<<<1, 1024, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_env_phases(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                              cudaStream_t s) {
  const int T = 256;
  k_move_claim<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_move_apply<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_eat_attack_claim<<<g.slot_blocks, T, 0, s>>>(d, R, L.A);
  k_attack_gain<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_metab_death<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_claim<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_assign<<<d.n_envs, 1024, 0, s>>>(d);
  k_mutate<<<g.birth_blocks, 256, 0, s>>>(d, L, R);
  k_regrow<<<g.cell_blocks, T, 0, s>>>(d, R);
  k_finish<<<1, 1024, 0, s>>>(d, R);
  return cudaGetLastError();
}

}  // namespace eco
