// eco_init.cu -- reset of every environment (Sec. 3.2: grid world with
// randomly distributed resources and a founding population; Sec. 3.3:
// Kaiming-style initial weights, zero biases) and re-derivation of the
// streamed BF16 / FP8 weight copy from the FP32 masters.
//
// Founders: the K non-wall cells with the smallest 64-bit keys
// (PLACE draw << 32 | local cell) -- all keys are distinct -- found by a
// four-round radix select on 16-bit digits (one histogram pass over the
// cells per round), then numbered in ascending cell order by a block scan.
#include "eco_internal.cuh"
#include "eco_kernels.h"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace eco {

__device__ __forceinline__ unsigned long long place_key(const EnvDesc &ed, int local_cell) {
  const U4 r = philox((uint32_t)(local_cell >> 2), 0u, 0u, 0u, ed.seed, S_PLACE);
  return ((unsigned long long)word_of(r, local_cell & 3) << 32) | (unsigned long long)(uint32_t)local_cell;
}

// Walls, food, empty occupancy, cleared claims.  Paper rules: a food cell
// holds one bite, e_food energy.
__global__ void k_init_cells(Dev d, Rules R) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.total_cells; c += gridDim.x * blockDim.x) {
    const int e = env_of_cell(d.env, d.n_envs, c);
    const EnvDesc ed = d.env[e];
    const int lc = c - ed.cell_off;
    const U4 rw = philox((uint32_t)(lc >> 2), 0u, 0u, 0u, ed.seed, S_WALL);
    const bool wall = word_of(rw, lc & 3) < R.thr_wall;
    const U4 rf = philox((uint32_t)(lc >> 2), 0u, 0u, 0u, ed.seed, S_FOOD_INIT);
    const bool food = !wall && word_of(rf, lc & 3) < R.thr_food;
    d.cellf[c] = (uint8_t)((wall ? CELL_WALL : 0u) | (food ? CELL_FOOD : 0u));
    d.res[c] = (R.rules != RULES_SIMPLE && food) ? R.e_food : 0;
    d.occ[c] = -1;
    // terrain rules: water fills the cells whose rock lies below sea level;
    // a Bernoulli(biomass_density) site (stream BIOMASS) holds b_site
    int water = 0, bio = 0;
    if (R.rules == RULES_TERRAIN && !wall) {
      const int rk = d.rock[c];
      if (rk < R.sea_level) water = R.sea_level - rk;
      const U4 rb = philox((uint32_t)(lc >> 2), 0u, 0u, 0u, ed.seed, S_BIOMASS);
      if (word_of(rb, lc & 3) < R.thr_bio) bio = R.b_site;
    }
    d.water[c] = water;
    d.bio[c] = bio;
    d.photo[c] = 0u;
    d.flow[c] = 0u;
    d.claim_move[c] = 0ull;
    d.cnt_move[c] = 0u;
    d.claim_birth[c] = 0ull;
    d.att_cell[c] = 0ull;
  }
}

// Per-slot agent fields (founders get alive / facing / energy here; their
// cells come from the placement below).
__global__ void k_init_agents(Dev d, Rules R) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.total_slots; s += gridDim.x * blockDim.x) {
    int e = 0;
    while (e + 1 < d.n_envs && d.env[e + 1].slot_off <= s) ++e;
    const EnvDesc ed = d.env[e];
    const int ls = s - ed.slot_off;
    const bool founder = ls < ed.init_alive;
    d.env_of[s] = (uint16_t)e;
    d.alive[s] = founder ? 1 : 0;
    d.pos[s] = 0;
    uint8_t f = 0;
    if (founder) {
      const U4 r = philox((uint32_t)(ls >> 2), 0u, 0u, 0u, ed.seed, S_FACING_INIT);
      f = (uint8_t)(word_of(r, ls & 3) >> 30);
    }
    d.facing[s] = f;
    d.energy[s] = founder ? R.e_init : 0;
    d.parent[s] = -1;
    d.birth[s] = -1;
    d.act[s] = 0;
    d.tgt[s] = -1;
    d.gain[s] = 0;
    d.hp[s] = (founder && R.rules != RULES_SIMPLE) ? R.hp_max : 0;
    d.a_water[s] = (founder && R.rules == RULES_TERRAIN) ? R.w_init : 0;
    d.a_bio[s] = (founder && R.rules == RULES_TERRAIN) ? R.b_body : 0;
    d.age[s] = 0;
    // colour trait (Sec. 3.3): three uniforms of COLOUR at counter (slot, 0, 0, 0)
    float4 col = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (founder) {
      const U4 r = philox((uint32_t)ls, 0u, 0u, 0u, ed.seed, S_COLOUR);
      col = make_float4(uniform01(r.x), uniform01(r.y), uniform01(r.z), 0.0f);
    }
    d.colour[s] = col;
  }
}

// Sum of a 64-bit value over the CTA (every thread gets the total).
__device__ long long block_sum_ll(long long v, unsigned long long *acc) {
  if (threadIdx.x == 0) *acc = 0ull;
  __syncthreads();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, (unsigned long long)v);
  __syncthreads();
  const long long total = (long long)*acc;
  __syncthreads();
  return total;
}

// Radix-select round: histogram of the 16-bit digit at `shift` among the
// non-wall cells whose higher digits equal the prefix found so far.
__global__ void k_place_hist(Dev d, int shift) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.total_cells; c += gridDim.x * blockDim.x) {
    if (d.cellf[c] & CELL_WALL) continue;
    const int e = env_of_cell(d.env, d.n_envs, c);
    const EnvDesc ed = d.env[e];
    if (ed.init_alive == 0) continue;
    const unsigned long long key = place_key(ed, c - ed.cell_off);
    if (shift < 48 && (key >> (shift + 16)) != d.place_prefix[e]) continue;
    atomicAdd(&d.hist[(size_t)e * 65536 + ((key >> shift) & 0xFFFFull)], 1u);
  }
}

// One CTA per environment: find the bin holding the remaining-th smallest
// key, extend the prefix, clear the histogram.  A missing bin (fewer than K
// non-wall cells) sets the status word.
__global__ void __launch_bounds__(1024) k_place_find(Dev d) {
  __shared__ int sh[33];
  __shared__ int found_bin, found_before;
  const int e = blockIdx.x;
  uint32_t *h = d.hist + (size_t)e * 65536;
  const int remaining = d.place_remaining[e];
  if (d.env[e].init_alive == 0) return;
  const int per = 65536 / blockDim.x;  // 64 bins per thread
  const int beg = threadIdx.x * per;
  int cnt = 0;
  for (int i = 0; i < per; ++i) cnt += (int)h[beg + i];
  int total;
  int before = block_exclusive_scan(cnt, &total, sh);
  if (threadIdx.x == 0) {
    found_bin = -1;
    found_before = 0;
  }
  __syncthreads();
  if (before < remaining && before + cnt >= remaining) {
    int run = before;
    for (int i = 0; i < per; ++i) {
      const int c = (int)h[beg + i];
      if (run + c >= remaining) {
        found_bin = beg + i;
        found_before = run;
        break;
      }
      run += c;
    }
  }
  __syncthreads();
  for (int i = 0; i < per; ++i) h[beg + i] = 0u;
  if (threadIdx.x == 0) {
    if (found_bin < 0) {
      atomicOr(&d.counters[CNT_STATUS], 1);
    } else {
      d.place_prefix[e] = (d.place_prefix[e] << 16) | (unsigned long long)found_bin;
      d.place_remaining[e] = remaining - found_before;
    }
  }
}

// One CTA per environment: founders are the non-wall cells with key <= the
// selected threshold; slot = rank in ascending cell order.
__global__ void __launch_bounds__(1024) k_place_assign(Dev d) {
  __shared__ int sh[33];
  const int e = blockIdx.x;
  const EnvDesc ed = d.env[e];
  if (ed.init_alive == 0) return;
  const unsigned long long thr = d.place_prefix[e];
  const int n = ed.side * ed.side;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = min(n, (int)threadIdx.x * per), end = min(n, beg + per);
  int cnt = 0;
  for (int c = beg; c < end; ++c)
    if (!(d.cellf[ed.cell_off + c] & CELL_WALL) && place_key(ed, c) <= thr) ++cnt;
  int total;
  int off = block_exclusive_scan(cnt, &total, sh);
  for (int c = beg; c < end; ++c) {
    const int gc = ed.cell_off + c;
    if (!(d.cellf[gc] & CELL_WALL) && place_key(ed, c) <= thr) {
      // the guard only matters when the select failed (status already set)
      if (off < ed.init_alive) {
        const int slot = ed.slot_off + off;
        d.pos[slot] = c;
        d.occ[gc] = slot;
        d.cellf[gc] |= (uint8_t)CELL_AGENT;
      }
      ++off;
    }
  }
  if (threadIdx.x == 0 && total != ed.init_alive) atomicOr(&d.counters[CNT_STATUS], 2);
}

// Founders' weights (Sec. 3.3: Kaiming initialisation, zero biases): weight
// p = N(0,1) * sqrt(gain / fan_in) from stream W_INIT at counter (local
// slot, p / 4), gain 1 for the plain (tanh) form and 2 for the paper (ReLU)
// form; biases and tau zero; every other slot all zero.
__global__ void k_init_params(Dev d, Layout L) {
  const int64_t per_slot = L.mstride / 4;
  const int64_t total = (int64_t)d.total_slots * per_slot;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / per_slot);
    const int q = (int)(i - (int64_t)s * per_slot);
    const EnvDesc ed = d.env[d.env_of[s]];
    const int ls = s - ed.slot_off;
    float w = 0.0f;
    if (ls < ed.init_alive && q < L.nW) {
      const int p = layout_logical(L, q);
      const U4 r = philox((uint32_t)ls, (uint32_t)(p >> 2), 0u, 0u, ed.seed, S_W_INIT);
      const float fan = (float)layout_fan_in(L, q);
      const float n = normal_of(r, p & 3);
      w = L.relu ? n * sqrtf(__fdiv_rn(2.0f, fan)) : __fdiv_rn(n, sqrtf(fan));
    }
    d.master[i] = w;
  }
}

// Streamed copy of slots [slot0, slot0 + n): BF16 elementwise (RNE), FP8 per
// output row (scale = max|w| / 448, satfinite RNE codes), biases FP32.
__global__ void k_requant_bf16(Dev d, Layout L, int slot0, int n) {
  const int nW = L.nW;
  const int per = L.nW + L.nB;
  const int64_t total = (int64_t)n * per;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = slot0 + (int)(i / per);
    const int q = (int)(i % per);
    const float *m = d.master + (int64_t)s * (L.mstride / 4);
    uint8_t *blk = d.wq + (int64_t)s * L.stride;
    if (q < nW) {
      reinterpret_cast<__nv_bfloat16 *>(blk)[q] = __float2bfloat16_rn(m[q]);
    } else {
      reinterpret_cast<float *>(blk + L.off_bias)[q - nW] = m[L.moff_bias / 4 + (q - nW)];
    }
  }
}

__global__ void k_requant_fp8(Dev d, Layout L, int slot0, int n) {
  const int H = L.H, rows = H + L.L * H + L.A;
  const int lane = threadIdx.x & 31;
  // biases (and tau) are copied unchanged
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * L.nB;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = slot0 + (int)(i / L.nB), k = (int)(i % L.nB);
    reinterpret_cast<float *>(d.wq + (int64_t)s * L.stride + L.off_bias)[k] =
        d.master[(int64_t)s * (L.mstride / 4) + L.moff_bias / 4 + k];
  }
  const int64_t warps = (int64_t)n * rows;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < warps;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int s = slot0 + (int)(w / rows);
    const int row = (int)(w % rows);
    const float *m = d.master + (int64_t)s * (L.mstride / 4);
    uint8_t *blk = d.wq + (int64_t)s * L.stride;
    int base, stride, cnt;
    if (row < H) {  // W_in row o: elements (j, o), j < D
      base = row; stride = H; cnt = L.D;
    } else if (row < H + L.L * H) {  // hidden layer l, row o
      const int l = (row - H) / H, o = (row - H) - l * H;
      base = L.D * H + l * H * H + o; stride = H; cnt = H;
    } else {  // head row a
      base = L.D * H + L.L * H * H + (row - H - L.L * H) * H; stride = 1; cnt = H;
    }
    float mx = 0.0f;
    for (int j = lane; j < cnt; j += 32) mx = fmaxf(mx, fabsf(m[base + j * stride]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    float sc = __fdiv_rn(mx, 448.0f);
    if (sc == 0.0f) sc = 1.0f;
    for (int j = lane; j < cnt; j += 32) {
      const int idx = base + j * stride;
      blk[idx] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(m[idx], sc), __NV_SATFINITE, __NV_E4M3);
    }
    if (lane == 0) reinterpret_cast<float *>(blk + L.off_scale)[row] = sc;
  }
}

// Initial statistics: alive = K, food count, energy = K * e_init, step 0;
// paper rules: energy on cells = food count * e_food; terrain rules: water
// and biomass on cells (summed) and carried (K * w_init, K * b_body).
__global__ void __launch_bounds__(1024) k_init_stats(Dev d, Rules R) {
  __shared__ unsigned long long acc;
  const int e = blockIdx.x;
  const EnvDesc ed = d.env[e];
  const int n = ed.side * ed.side;
  long long cnt = 0, water = 0, bio = 0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    cnt += (d.cellf[ed.cell_off + c] & CELL_FOOD) ? 1 : 0;
    water += d.water[ed.cell_off + c];
    bio += d.bio[ed.cell_off + c];
  }
  const long long total = block_sum_ll(cnt, &acc);
  const long long wt = block_sum_ll(water, &acc);
  const long long bt = block_sum_ll(bio, &acc);
  const bool terrain = R.rules == RULES_TERRAIN;
  for (int k = threadIdx.x; k < N_ST; k += blockDim.x) {
    long long v = 0;
    if (k == ST_ALIVE) v = ed.init_alive;
    else if (k == ST_FOOD_TOTAL) v = total;
    else if (k == ST_ENERGY_TOTAL) v = (long long)ed.init_alive * R.e_init;
    else if (k == ST_RES_TOTAL && R.rules != RULES_SIMPLE) v = total * R.e_food;
    else if (k == ST_WATER_CELLS && terrain) v = wt;
    else if (k == ST_BIO_CELLS && terrain) v = bt;
    else if (k == ST_WATER_AGENTS && terrain) v = (long long)ed.init_alive * R.w_init;
    else if (k == ST_BIO_AGENTS && terrain) v = (long long)ed.init_alive * R.b_body;
    d.stats_total[e * N_ST + k] = v;
    d.stats_last[e * N_ST + k] = v;
    d.stats_step[e * N_ST + k] = 0;
  }
  if (threadIdx.x == 0) {
    d.birth_contenders[e] = 0;
    if (e == 0) d.counters[CNT_CONTENDERS] = 0;
    d.place_prefix[e] = 0ull;
    d.place_remaining[e] = ed.init_alive;
  }
}

__global__ void k_init_static(Dev d) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.total_slots; s += gridDim.x * blockDim.x) {
    int e = 0;
    while (e + 1 < d.n_envs && d.env[e + 1].slot_off <= s) ++e;
    d.env_of[s] = (uint16_t)e;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.total_cells; c += gridDim.x * blockDim.x)
    d.occ[c] = -1;
}

// One CTA per environment: alive count, food count, energy sum (and, under
// the paper rules, the energy lying on cells) of the current state become
// the "now" statistics; the step counter is copied.
__global__ void __launch_bounds__(1024) k_recount(Dev d, Rules R) {
  __shared__ unsigned long long acc;
  const int e = blockIdx.x;
  const EnvDesc ed = d.env[e];
  const int n = ed.side * ed.side;
  long long food = 0, alive = 0, energy = 0, res = 0, wc = 0, bc = 0, wa = 0, ba = 0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    food += (d.cellf[ed.cell_off + c] & CELL_FOOD) ? 1 : 0;
    res += d.res[ed.cell_off + c];
    wc += d.water[ed.cell_off + c];
    bc += d.bio[ed.cell_off + c];
  }
  for (int s = threadIdx.x; s < ed.n_slots; s += blockDim.x) {
    const int g = ed.slot_off + s;
    if (d.alive[g]) {
      ++alive;
      energy += d.energy[g];
      wa += d.a_water[g];
      ba += d.a_bio[g];
    }
  }
  const bool terrain = R.rules == RULES_TERRAIN;
  const long long wct = block_sum_ll(wc, &acc), bct = block_sum_ll(bc, &acc);
  const long long wat = block_sum_ll(wa, &acc), bat = block_sum_ll(ba, &acc);
  const long long ft = block_sum_ll(food, &acc);
  const long long at = block_sum_ll(alive, &acc);
  const long long et = block_sum_ll(energy, &acc);
  const long long rt = block_sum_ll(res, &acc);
  if (threadIdx.x == 0) {
    const long long t = d.step[0];
    long long *tot = d.stats_total + e * N_ST, *last = d.stats_last + e * N_ST;
    tot[ST_ALIVE] = last[ST_ALIVE] = at;
    tot[ST_FOOD_TOTAL] = last[ST_FOOD_TOTAL] = ft;
    tot[ST_ENERGY_TOTAL] = last[ST_ENERGY_TOTAL] = et;
    tot[ST_RES_TOTAL] = last[ST_RES_TOTAL] = R.rules != RULES_SIMPLE ? rt : 0;
    tot[ST_WATER_CELLS] = last[ST_WATER_CELLS] = terrain ? wct : 0;
    tot[ST_BIO_CELLS] = last[ST_BIO_CELLS] = terrain ? bct : 0;
    tot[ST_WATER_AGENTS] = last[ST_WATER_AGENTS] = terrain ? wat : 0;
    tot[ST_BIO_AGENTS] = last[ST_BIO_AGENTS] = terrain ? bat : 0;
    tot[ST_STEP] = last[ST_STEP] = t;
  }
}

cudaError_t launch_init_static(const Dev &d, const EnvGrid &g, cudaStream_t s) {
  const long long n = d.total_slots > d.total_cells ? d.total_slots : d.total_cells;
  k_init_static<<<grid_for(n, 256, g.sms * 16), 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_recount(const Dev &d, const Rules &R, cudaStream_t s) {
  k_recount<<<d.n_envs, 1024, 0, s>>>(d, R);
  return cudaGetLastError();
}

cudaError_t launch_requant(const Dev &d, const Layout &L, const Rules &R, int slot0, int n,
                           cudaStream_t s) {
  if (R.precision == PREC_FP32 || n <= 0) return cudaSuccess;
  if (R.precision == PREC_BF16) {
    const long long work = (long long)n * (L.nW + L.nB);
    k_requant_bf16<<<grid_for(work, 256, 152 * 32), 256, 0, s>>>(d, L, slot0, n);
  } else {
    const long long work = (long long)n * (L.H + L.L * L.H + L.A) * 32;
    k_requant_fp8<<<grid_for(work, 256, 152 * 32), 256, 0, s>>>(d, L, slot0, n);
  }
  return cudaGetLastError();
}

cudaError_t launch_reset(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                         cudaStream_t s) {
  cudaError_t err;
  const int T = 256;
  const int cb = grid_for(d.total_cells, T, g.sms * 16);
  const int sb = grid_for(d.total_slots, T, g.sms * 16);
  if ((err = cudaMemsetAsync(d.counters, 0, sizeof(int32_t) * CNT_N, s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(d.step, 0, sizeof(long long), s)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(d.hist, 0, sizeof(uint32_t) * 65536 * (size_t)d.n_envs, s)) != cudaSuccess)
    return err;
  k_init_cells<<<cb, T, 0, s>>>(d, R);
  k_init_agents<<<sb, T, 0, s>>>(d, R);
  k_init_stats<<<d.n_envs, 1024, 0, s>>>(d, R);  // also zeroes the placement prefix
  for (int round = 0; round < 4; ++round) {
    const int shift = 48 - 16 * round;
    k_place_hist<<<cb, T, 0, s>>>(d, shift);
    k_place_find<<<d.n_envs, 1024, 0, s>>>(d);
  }
  k_place_assign<<<d.n_envs, 1024, 0, s>>>(d);
  const long long pw = (long long)d.total_slots * (L.mstride / 4);
  k_init_params<<<grid_for(pw, T, g.sms * 64), T, 0, s>>>(d, L);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_requant(d, L, R, 0, d.total_slots, s);
}

}  // namespace eco
