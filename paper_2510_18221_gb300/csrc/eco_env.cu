// eco_env.cu -- the environment phases of one step (Sec. 3.2 "Actions",
// "Resources and Agent Health"; Sec. 3.3 mutation), for every environment
// of the batch at once.
//
// Phase order: policy (+ facing, turns and move claims, fused into its
// epilogue; eco_policy.cu) -> move apply + eat + attack claims on cells ->
// attack transfers + metabolism + death -> birth claims (+ regrowth, which
// commutes with them) -> slot assignment -> mutation of the children, the
// alive list of the next step and the statistics.
//
// Two launch forms run the same phase functions: one persistent kernel
// (cooperative launch; phases separated by grid barriers whose waits are
// bounded, so a stuck barrier sets the status word and every CTA exits), and
// one kernel per phase.  Both give bit-identical results.
//
// Conflicts (two movers into one free cell, two attackers on one victim's
// cell, two parents onto one birth cell) are resolved by a 64-bit atomicMax
// of (Philox draw << 32 | ~local slot): the highest draw wins, equal draws
// go to the lower slot.  A maximum does not depend on the order of the
// atomics, every other atomic is an integer add, and no phase's result
// depends on the order in which agents are visited, so all integer state
// is bit-identical from run to run and equal to the plain sequential rule.
#include "eco_internal.cuh"
#include "eco_kernels.h"

#include <cuda/atomic>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace eco {

int grid_for(long long n, int threads, int max_blocks) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// ---------------------------------------------------------------------------
// A0: list of alive slots in ascending slot order (Sec. 3.1: the population
// function names the alive agents).  Two passes over tiles of kCompactTile
// slots: each tile counts its alive slots; then each tile adds up the
// counts of the tiles before it (a few dozen numbers) and writes its slots.
// The step itself runs only the second pass: every death and birth adjusts
// its tile's count as it happens (the fast birth path's children are added
// by the scatter itself), so the counts are exact when the alive set is
// final (the first pass runs after reset and state writes).
// Slot order keeps the warps of the policy kernel streaming neighbouring
// weight blocks at the same time.  Block-level: the first 256 threads of a
// CTA of any size >= 256 cover a tile.
// ---------------------------------------------------------------------------
constexpr int kCompactTile = 4096;  // 256 threads x 16 slots

__host__ __device__ int compact_tiles(int total_slots) {
  return (total_slots + kCompactTile - 1) / kCompactTile;
}

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

// Tile counts are kept per step parity: step t's deaths and births adjust
// counts[t & 1], and its scatter writes counts[(t + 1) & 1] for the next
// step (so a scatter never reads a count another CTA is writing).
__device__ __forceinline__ int32_t *tile_counts_of(const Dev &d, uint32_t t) {
  return d.tile_counts + (t & 1u) * compact_tiles(d.total_slots);
}

__device__ void ph_compact_count(const Dev &d, int b0, int bs, int *sh) {
  const int tiles = compact_tiles(d.total_slots);
  int32_t *cur = tile_counts_of(d, (uint32_t)d.step[0]);
  for (int tile = b0; tile < tiles; tile += bs) {
    const uint32_t mask =
        threadIdx.x < kCompactTile / 16 ? alive_mask16(d, tile * kCompactTile + threadIdx.x * 16) : 0u;
    int total;
    block_exclusive_scan(__popc(mask), &total, sh);
    if (threadIdx.x == 0) cur[tile] = total;
  }
}

// children (global slots, ascending, nchild of them) are this step's
// births that the alive bytes may not show yet (the fast birth path writes
// them concurrently); cmask is a 4096-bit shared-memory scratch.
__device__ void ph_compact_scatter(const Dev &d, int b0, int bs, int *sh, uint32_t t, const int *children,
                                   int nchild, uint32_t *cmask) {
  const int tiles = compact_tiles(d.total_slots);
  const int32_t *cur = tile_counts_of(d, t);
  int32_t *nxt = tile_counts_of(d, t + 1u);
  for (int tile = b0; tile < tiles; tile += bs) {
    const int t0 = tile * kCompactTile;
    int before = 0;
    for (int k = threadIdx.x; k < tile; k += blockDim.x) before += cur[k];
    for (int i = threadIdx.x; i < nchild; i += blockDim.x) before += children[i] < t0 ? 1 : 0;
    if (nchild > 0) {
      for (int w = threadIdx.x; w < kCompactTile / 32; w += blockDim.x) cmask[w] = 0u;
      __syncthreads();
      for (int i = threadIdx.x; i < nchild; i += blockDim.x) {
        const int c = children[i] - t0;
        if (c >= 0 && c < kCompactTile) atomicOr(&cmask[c >> 5], 1u << (c & 31));
      }
    }
    int base;
    block_exclusive_scan(before, &base, sh);  // base = sum over the earlier tiles
    const int s0 = t0 + threadIdx.x * 16;
    uint32_t mask = threadIdx.x < kCompactTile / 16 ? alive_mask16(d, s0) : 0u;
    if (nchild > 0 && threadIdx.x < kCompactTile / 16)
      mask |= (cmask[threadIdx.x >> 1] >> ((threadIdx.x & 1) * 16)) & 0xFFFFu;
    int total;
    int at = base + block_exclusive_scan(__popc(mask), &total, sh);
    while (mask) {
      const int k = __ffs(mask) - 1;
      d.alive_list[at++] = s0 + k;
      mask &= mask - 1;
    }
    if (threadIdx.x == 0) nxt[tile] = total;
    if (tile == tiles - 1 && threadIdx.x == 0) d.counters[CNT_N_ALIVE] = base + total;
  }
}

// ---------------------------------------------------------------------------
// Per-agent phases (grid-stride over the alive list).  The alive list does
// not change until the compaction at the end of the step, so a persistent
// thread loads the slot of its first entry once and passes it in (`first`;
// -1 in the one-kernel-per-phase form).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int agent_slot(const Dev &d, int i, int g0, int first) {
  return (i == g0 && first >= 0) ? first : d.alive_list[i];
}

// Environment of a slot (no lookup when there is one environment).
__device__ __forceinline__ int env_index(const Dev &d, int slot) {
  return d.n_envs == 1 ? 0 : (int)d.env_of[slot];
}


// A6 (part 2) + A7 + A8 (part 1): winners move (only the winner of a cell
// writes it, and a winner's old cell was occupied when the step began, so
// nobody moves into it); then every agent eats the food of its post-move
// cell, when the rules say it eats (nobody else can be on that cell); then
// attackers claim their target cells.
__device__ void ph_move_apply_eat(const Dev &d, const Rules &R, int n_actions, int g0, int gs, int first,
                                  uint32_t t) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = g0; i < n; i += gs) {
    const int slot = agent_slot(d, i, g0, first);
    const int e = env_index(d, slot);
    const EnvDesc ed = d.env[e];
    const int tc = d.tgt[slot];
    int pos = d.pos[slot];
    const int a = d.act[slot];
    // read with the slot's other words, before this phase's stores: only
    // this thread writes them in this phase
    int en = d.energy[slot];
    const int fac = d.facing[slot];
    // simple rules: the food bits of the cells this agent can end on, read
    // with the claim (no other agent changes them in this phase: only the
    // agent on a cell eats its food, and regrowth comes later)
    const bool eats_simple = R.rules == RULES_SIMPLE &&
                             ((R.flags & F_AUTO_EAT) || (n_actions > ACT_EAT && a == ACT_EAT));
    uint32_t cf_stay = 0u, cf_move = 0u;
    if (eats_simple) {
      cf_stay = d.cellf[ed.cell_off + pos];
      if (tc >= 0) cf_move = d.cellf[ed.cell_off + tc];
    }
    bool moved = false;
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
        moved = true;
        stat_add(d.stats_step, e, ST_MOVES, 1);
      } else {
        stat_add(d.stats_step, e, ST_MOVE_LOST, 1);
      }
    }
    if (R.rules == RULES_TERRAIN && (a == TA_DRINK || a == TA_EAT_BIO)) {
      // terrain rules: drink or eat biomass, min(bite, on the cell, room)
      const int gpos = ed.cell_off + pos;
      if (a == TA_DRINK) {
        const int w = d.water[gpos];
        const int sip = min(min(R.w_bite, w), R.w_cap - d.a_water[slot]);
        if (sip > 0) {
          d.water[gpos] = w - sip;
          d.a_water[slot] += sip;
          stat_add(d.stats_step, e, ST_DRUNK, sip);
        }
      } else {
        const int b = d.bio[gpos];
        const int bite = min(min(R.b_bite, b), R.b_cap - d.a_bio[slot]);
        if (bite > 0) {
          d.bio[gpos] = b - bite;
          d.a_bio[slot] += bite;
          stat_add(d.stats_step, e, ST_BIO_EATEN, bite);
        }
      }
    } else if (R.rules != RULES_SIMPLE) {
      // one bite: min(e_food, energy on the cell, room in the stomach)
      if (a == PA_EAT) {
        const int gpos = ed.cell_off + pos;
        const int r = d.res[gpos];
        const int bite = min(min(R.e_food, r), R.e_cap - d.energy[slot]);
        if (bite > 0) {
          d.res[gpos] = r - bite;
          d.energy[slot] += bite;
          stat_add(d.stats_step, e, ST_EATEN, 1);
          stat_add(d.stats_step, e, ST_EATEN_ENERGY, bite);
          if (r == bite) {
            d.cellf[gpos] &= (uint8_t)~CELL_FOOD;
            stat_add(d.stats_step, e, ST_FOOD_EMPTIED, 1);
          }
        }
      }
    } else if (eats_simple) {
      const uint32_t cf = moved ? cf_move : cf_stay;
      if (cf & CELL_FOOD) {
        // the agent stands on this cell: its agent bit is set
        d.cellf[ed.cell_off + pos] = (uint8_t)((cf & ~CELL_FOOD) | CELL_AGENT);
        en += R.e_food;
        d.energy[slot] = en;
        stat_add(d.stats_step, e, ST_EATEN, 1);
      }
    }
    // simple rules: the post-eat energy, which attack transfers are computed
    // from, kept where an attacker can read it while the owner updates its
    // own energy in the metabolism phase
    if (R.rules == RULES_SIMPLE) d.gain[slot] = en;
    // A8 (part 1): attacks claim their target cells.  An attacker does not
    // move (attack and move are different actions), so its cell and facing
    // are final here, while the agents it hits are only known once every
    // move is in; they are looked up after the barrier (metabolism phase).
    // Simple rules: the faced cell, claimed by the highest CLAIM_ATTACK
    // draw; paper rules: every cell of the 3x3 square in front (1..3 cells
    // ahead, one to either side) counts one more attacker.
    if (R.rules != RULES_SIMPLE) {
      if (a == PA_ATTACK) {
        const int side = ed.side;
        const int px = pos % side, py = pos / side;
        const int f = fac, rt = (f + 1) & 3;
        for (int fw = 1; fw <= 3; ++fw)
          for (int lat = -1; lat <= 1; ++lat) {
            const int cx = wrapi(px + fw * dir_dx(f) + lat * dir_dx(rt), side);
            const int cy = wrapi(py + fw * dir_dy(f) + lat * dir_dy(rt), side);
            atomicAdd(&d.att_cell[ed.cell_off + cy * side + cx], 1ull);
          }
      }
    } else if (a == ACT_ATTACK) {
      const int c = step_cell(pos, fac, ed.side);
      const int local = slot - ed.slot_off;
      const U4 r = philox(t, (uint32_t)local, 0u, 0u, ed.seed, S_CLAIM_ATTACK);
      atomicMax(&d.att_cell[ed.cell_off + c], claim_key(r.x, local));
    }
  }
}

// Paper rules, one agent: pay the action's cost (starving when it exceeds
// the energy), take the attack and age damage, heal from energy, and die at
// HP <= 0, dropping the energy on the cell; survivors age by one step.
// Terrain rules: also spend w_metab water onto the cell (thirst: what there
// is, and starve_damage HP), heal only with heal_water water (spent onto the
// cell too), and drop water and biomass at death.  One agent per cell, so
// the cell's counters are this agent's to change here.
__device__ __forceinline__ void health_paper(const Dev &d, const Rules &R, int slot, uint32_t t) {
  int en = d.energy[slot];
  int hp = d.hp[slot];
  const int age = d.age[slot];
  const int cost = R.e_metab + (d.act[slot] != PA_REST ? R.e_act : 0);
  int paid = cost, starved = 0, healed = 0;
  if (en >= cost) {
    en -= cost;
  } else {
    paid = en;
    en = 0;
    hp -= R.starve_damage;
    starved = 1;
  }
  const bool terrain = R.rules == RULES_TERRAIN;
  const int e = env_index(d, slot);
  const int gpos = d.env[e].cell_off + d.pos[slot];
  int aw = terrain ? d.a_water[slot] : 0, spent = 0, thirsty = 0;
  if (terrain) {
    spent = R.w_metab;
    if (aw < spent) {
      spent = aw;
      hp -= R.starve_damage;
      thirsty = 1;
    }
    aw -= spent;
  }
  // every attacker whose square covers this cell takes attack_damage
  const int hits = (int)d.att_cell[gpos];
  hp -= hits * R.attack_damage;
  stat_add(d.stats_step, e, ST_ATTACK_HITS, hits);
  stat_add(d.stats_step, e, ST_DAMAGE, hits * R.attack_damage);
  hp -= age / R.age_div;
  if (hp > 0 && hp < R.hp_max && R.heal_rate > 0 && en >= R.heal_cost && (!terrain || aw >= R.heal_water)) {
    hp = min(hp + R.heal_rate, R.hp_max);
    en -= R.heal_cost;
    if (terrain) {
      aw -= R.heal_water;
      spent += R.heal_water;
    }
    healed = 1;
  }
  if (terrain) {
    int back = spent;  // spent water, and at death everything carried
    if (hp <= 0) {
      back += aw;
      const int ab = d.a_bio[slot];
      d.bio[gpos] += ab;
      d.a_bio[slot] = 0;
      stat_add(d.stats_step, e, ST_DEAD_WATER, aw);
      stat_add(d.stats_step, e, ST_DEAD_BIO, ab);
      aw = 0;
    }
    d.water[gpos] += back;
    d.a_water[slot] = aw;
    stat_add(d.stats_step, e, ST_WATER_SPENT, spent);
    stat_add(d.stats_step, e, ST_THIRSTY, thirsty);
  }
  stat_add(d.stats_step, e, ST_METAB_PAID, paid);
  stat_add(d.stats_step, e, ST_STARVED, starved);
  stat_add(d.stats_step, e, ST_HEALS, healed);
  if (hp <= 0) {
    uint8_t cf = (uint8_t)(d.cellf[gpos] & ~CELL_AGENT);
    if (en > 0) {
      const int r = d.res[gpos];
      d.res[gpos] = r + en;
      if (r == 0) {
        cf |= (uint8_t)CELL_FOOD;
        stat_add(d.stats_step, e, ST_FOOD_REFILLED, 1);
      }
    }
    d.cellf[gpos] = cf;  // occ keeps the slot until the birth-claim phase
    d.alive[slot] = 0;
    atomicSub(&tile_counts_of(d, t)[slot / kCompactTile], 1);
    stat_add(d.stats_step, e, ST_DEATHS, 1);
    stat_add(d.stats_step, e, ST_DEAD_ENERGY, en);
    en = 0;
    hp = 0;
  } else {
    d.age[slot] = age + 1;
  }
  d.hp[slot] = hp;
  d.energy[slot] = en;
}

// A8 (part 2) + A9: the attack transfer, metabolism, death at e <= 0
// (paper rules: health_paper).  Also clears this step's move claims.
// A dying agent clears its alive flag and its cell's agent bit here, but
// its occ entry only in the birth-claim phase, so that an attacker that
// won the agent's cell still finds it in this phase.
__device__ void ph_metab_death(const Dev &d, const Rules &R, int g0, int gs, int first, uint32_t t) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = g0; i < n; i += gs) {
    const int slot = agent_slot(d, i, g0, first);
    const int e = env_index(d, slot);
    const EnvDesc ed = d.env[e];
    const int tc = d.tgt[slot];
    if (R.rules != RULES_SIMPLE) {
      if (tc >= 0) {
        d.claim_move[ed.cell_off + tc] = 0ull;
        if (R.flags & F_CANCEL_ALL) d.cnt_move[ed.cell_off + tc] = 0u;
      }
      health_paper(d, R, slot, t);
      continue;
    }
    // A8 (part 2): a victim -- an agent on a claimed cell -- loses
    // floor(e * num / den) of its post-eat energy to the attacker that won
    // the cell's claim, which gains the same amount (read from the victim's
    // post-eat snapshot); claims are cleared in the birth-claim phase.
    // Every word this needs is final in this phase (attack claims, cells'
    // occupants and the snapshots were written before the barrier), so all
    // are requested before the phase's first store: the slot's own words,
    // then the claims on its own and its target cell with the target's
    // occupant, then the occupant's snapshot.
    int en = d.energy[slot];
    const int pos = d.pos[slot];
    const bool attacker = d.act[slot] == ACT_ATTACK;
    const int fac = d.facing[slot];
    const unsigned long long hit = d.att_cell[ed.cell_off + pos];
    const int c = ed.cell_off + step_cell(pos, fac, ed.side);
    const bool won = attacker && claim_local_slot(d.att_cell[c]) == slot - ed.slot_off;
    const int v = attacker ? d.occ[c] : -1;
    if (tc >= 0) {
      d.claim_move[ed.cell_off + tc] = 0ull;
      if (R.flags & F_CANCEL_ALL) d.cnt_move[ed.cell_off + tc] = 0u;
    }
    const int loss = hit ? (int)(((long long)en * R.attack_num) / R.attack_den) : 0;
    int g = 0;
    if (won && v >= 0) {
      g = (int)(((long long)d.gain[v] * R.attack_num) / R.attack_den);
      stat_add(d.stats_step, e, ST_ATTACK_HITS, 1);
      stat_add(d.stats_step, e, ST_ENERGY_TRANSFERRED, g);
    }
    en = en - loss + g - R.e_metab;
    if (en <= 0) {
      const int gpos = ed.cell_off + pos;
      d.alive[slot] = 0;
      atomicSub(&tile_counts_of(d, t)[slot / kCompactTile], 1);
      d.cellf[gpos] &= (uint8_t)~CELL_AGENT;
      stat_add(d.stats_step, e, ST_DEATHS, 1);
      stat_add(d.stats_step, e, ST_DEAD_ENERGY, en);
      en = 0;
    }
    d.energy[slot] = en;
  }
}

// A10 (part 1): agents with e >= e_repro (paper rules: that chose to
// reproduce; terrain rules: that also carry b_body + b_child biomass and
// w_child water) claim the free non-wall cell behind them and join their
// environment's contender list.
__device__ void ph_birth_claim(const Dev &d, const Rules &R, int g0, int gs, int first, uint32_t t) {
  const int n = d.counters[CNT_N_ALIVE];
  for (int i = g0; i < n; i += gs) {
    const int slot = agent_slot(d, i, g0, first);
    {
      // clear this step's attack claims and, for an agent that died, its
      // cell's occupant (kept for the attackers of the metabolism phase)
      const EnvDesc ed = d.env[env_index(d, slot)];
      const int pos = d.pos[slot];
      const int a = d.act[slot];
      if (!d.alive[slot]) d.occ[ed.cell_off + pos] = -1;
      if (R.rules != RULES_SIMPLE) {
        if (a == PA_ATTACK) {
          const int side = ed.side;
          const int px = pos % side, py = pos / side;
          const int f = d.facing[slot], rt = (f + 1) & 3;
          for (int fw = 1; fw <= 3; ++fw)
            for (int lat = -1; lat <= 1; ++lat) {
              const int cx = wrapi(px + fw * dir_dx(f) + lat * dir_dx(rt), side);
              const int cy = wrapi(py + fw * dir_dy(f) + lat * dir_dy(rt), side);
              d.att_cell[ed.cell_off + cy * side + cx] = 0ull;
            }
        }
      } else if (a == ACT_ATTACK) {
        d.att_cell[ed.cell_off + step_cell(pos, d.facing[slot], ed.side)] = 0ull;
      }
    }
    int bt = -1;
    if (d.alive[slot] && d.energy[slot] >= R.e_repro &&
        (R.rules == RULES_SIMPLE || d.act[slot] == PA_REPRODUCE) &&
        (R.rules != RULES_TERRAIN ||
         (d.a_bio[slot] >= R.b_body + R.b_child && d.a_water[slot] >= R.w_child))) {
      const int e = env_index(d, slot);
      const EnvDesc ed = d.env[e];
      const int c = step_cell(d.pos[slot], (d.facing[slot] + 2) & 3, ed.side);
      const int gc = ed.cell_off + c;
      if (!(d.cellf[gc] & (CELL_WALL | CELL_AGENT))) {
        const int local = slot - ed.slot_off;
        const U4 r = philox(t, (uint32_t)local, 0u, 0u, ed.seed, S_CLAIM_BIRTH);
        atomicMax(&d.claim_birth[gc], claim_key(r.x, local));
        const int k = atomicAdd(&d.birth_contenders[e], 1);
        atomicAdd(&d.counters[CNT_CONTENDERS], 1);
        d.contenders[ed.slot_off + k] = slot;
        d.bcell[ed.slot_off + k] = c;
        bt = c;
      }
    }
    d.tgt[slot] = bt;
  }
}

// ---------------------------------------------------------------------------
// A10 (part 2): slot assignment, one CTA per environment.  Cell winners in
// ascending slot order take the free slots in ascending order; the child
// gets floor(e/2) of the parent's energy (paper rules: e_child, and hp_child
// HP), the parent's facing, and the cell behind.  Winners (at most kBirthCap per step) are sorted in shared memory
// and only the first n_winners free slots are searched for; more
// contenders than kBirthCap fall back to a full scan of the slots.
// ---------------------------------------------------------------------------
constexpr int kBirthCap = 2048;
// Claimants of one step up to which a single world takes the fast birth
// path (each compaction tile lists this many of its free slots), and the
// most compaction tiles (4096 slots each) such a world may have.
constexpr int kFastBirths = 256;
constexpr int kMaxFastTiles = 256;

struct BirthSmem {
  int sh[33];
  int win[kBirthCap];
  int free_[kBirthCap];
  int nwin, nborn, nfree;
  int tile_first[kMaxFastTiles];  // fast path: free slots before each tile
  uint32_t cmask[kCompactTile / 32];  // the scatter's children of one tile
};

// A child at the free slot c (global) of the parent p (global), on the birth
// cell bt (env-local).  record: also bump the tile count of step t and
// append (p, c) to the births list (the general path; the fast path's
// scatter and mutation take the pairs from shared memory instead).
__device__ __forceinline__ void make_child(const Dev &d, const Rules &R, const EnvDesc &ed, int p,
                                           int c, int bt, uint32_t t, bool record) {
  const bool paper = R.rules != RULES_SIMPLE;
  const int en = d.energy[p];
  const int ce = paper ? R.e_child : en / 2;
  d.energy[p] = en - ce;
  d.energy[c] = ce;
  d.hp[c] = paper ? R.hp_child : 0;
  d.age[c] = 0;
  if (R.rules == RULES_TERRAIN) {  // the child's water and body
    d.a_water[p] -= R.w_child;
    d.a_water[c] = R.w_child;
    d.a_bio[p] -= R.b_child;
    d.a_bio[c] = R.b_child;
  }
  {
    // colour trait: clamp(parent + sigma * n, 0, 1), n the first three
    // normals of COLOUR at counter (step, parent's local slot, 1, 0)
    float n[4];
    normals4(philox(t, (uint32_t)(p - ed.slot_off), 1u, 0u, ed.seed, S_COLOUR), n);
    const float4 pc = d.colour[p];
    d.colour[c] = make_float4(fminf(fmaxf(fmaf(R.sigma, n[0], pc.x), 0.0f), 1.0f),
                              fminf(fmaxf(fmaf(R.sigma, n[1], pc.y), 0.0f), 1.0f),
                              fminf(fmaxf(fmaf(R.sigma, n[2], pc.z), 0.0f), 1.0f), 0.0f);
  }
  d.alive[c] = 1;
  d.pos[c] = bt;
  d.facing[c] = d.facing[p];
  d.parent[c] = p - ed.slot_off;
  d.birth[c] = (int)t;
  d.occ[ed.cell_off + bt] = c;
  d.cellf[ed.cell_off + bt] |= (uint8_t)CELL_AGENT;
  if (record) {
    atomicAdd(&tile_counts_of(d, t)[c / kCompactTile], 1);
    const int b = atomicAdd(&d.counters[CNT_N_BIRTHS], 1);
    d.births[b] = make_int2(p, c);
  }
}

// Block-level: the nc contenders of environment e that won their birth
// cell's claim, in ascending slot order, into S.win (INT_MAX fills the
// sorted tail up to a power of two); returns their count (every thread).
__device__ int sort_winners(const Dev &d, const EnvDesc &ed, int nc, BirthSmem &S) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int p2 = 1;
  while (p2 < nc) p2 <<= 1;
  for (int i = tid; i < p2; i += nt) {
    int v = 0x7FFFFFFF;
    if (i < nc) {
      const int g = d.contenders[ed.slot_off + i];
      const int bt = d.bcell[ed.slot_off + i];
      if (claim_local_slot(d.claim_birth[ed.cell_off + bt]) == g - ed.slot_off) v = g;
    }
    S.win[i] = v;
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {  // bitonic sort, ascending
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < p2; i += nt) {
        const int l = i ^ j;
        if (l > i) {
          const int a = S.win[i], b = S.win[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            S.win[i] = b;
            S.win[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    int nw = 0;
    while (nw < p2 && S.win[nw] != 0x7FFFFFFF) ++nw;
    S.nwin = nw;
  }
  __syncthreads();
  return S.nwin;
}

// Block-level: the first (at most limit) free slots of environment e, env-
// local and ascending, into out; returns how many (every thread).  64
// slots per thread per pass.
__device__ int scan_free_slots(const Dev &d, const EnvDesc &ed, int limit, int *out, int *sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int found = 0;
  for (int base = 0; base < ed.n_slots && found < limit; base += nt * 64) {
    const int s0 = base + tid * 64;
    unsigned long long mask = 0ull;
    const uint8_t *al = d.alive + ed.slot_off + s0;
    if (s0 + 64 <= ed.n_slots && ((reinterpret_cast<uintptr_t>(al) & 15) == 0)) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = reinterpret_cast<const uint4 *>(al)[q];
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // 0xFF in each byte that is 0 (a free slot); its top bits, gathered
          // by the multiply, are the four slots' free bits
          const uint32_t z = __vcmpeq4(w4[k], 0u) & 0x80808080u;
          mask |= (unsigned long long)((z * 0x00204081u) >> 28) << (q * 16 + 4 * k);
        }
      }
    } else {
      for (int k = 0; k < 64; ++k)
        if (s0 + k < ed.n_slots && !al[k]) mask |= 1ull << k;
    }
    int total;
    int r = found + block_exclusive_scan(__popcll(mask), &total, sh);
    while (mask && r < limit) {
      const int k = __ffsll(mask) - 1;
      out[r++] = s0 + k;
      mask &= mask - 1;
    }
    found += total;
    __syncthreads();
  }
  return found < limit ? found : limit;
}

__device__ void birth_assign_env(const Dev &d, const Rules &R, int e, BirthSmem &S, uint32_t t) {
  const int nc = d.birth_contenders[e];
  if (nc == 0) return;  // uniform across the CTA
  const EnvDesc ed = d.env[e];
  const int tid = threadIdx.x, nt = blockDim.x;
  int born = 0, failed = 0;

  if (nc <= kBirthCap) {
    const int nwin = sort_winners(d, ed, nc, S);
    const int nfree = scan_free_slots(d, ed, nwin, S.free_, S.sh);
    for (int i = tid; i < nwin; i += nt) {
      const int p = S.win[i];
      const int bt = d.tgt[p];
      d.claim_birth[ed.cell_off + bt] = 0ull;
      if (i < nfree) {
        make_child(d, R, ed, p, ed.slot_off + S.free_[i], bt, t, true);
        ++born;
      } else {
        ++failed;
      }
    }
  } else {
    // full scan over the environment's slots
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
    int free_off = block_exclusive_scan(nfree, &free_total, S.sh);
    int win_off = block_exclusive_scan(nwin, &win_total, S.sh);
    for (int s = beg; s < end; ++s)
      if (d.bflag[ed.slot_off + s] == 1) d.free_list[ed.slot_off + free_off++] = s;
    __syncthreads();
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
      make_child(d, R, ed, p, ed.slot_off + d.free_list[ed.slot_off + r], bt, t, true);
      ++born;
    }
  }
  if (born) atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_BIRTHS], (unsigned long long)born);
  if (failed)
    atomicAdd((unsigned long long *)&d.stats_step[e * N_ST + ST_FAILED_BIRTHS], (unsigned long long)failed);
  __syncthreads();  // S is reused by the next environment of this CTA
}

__device__ void ph_birth_assign(const Dev &d, const Rules &R, int b0, int bs, BirthSmem &S, uint32_t t) {
  for (int e = b0; e < d.n_envs; e += bs) birth_assign_env(d, R, e, S, t);
}

// ---------------------------------------------------------------------------
// A11: mutation (Sec. 3.3): child = fl32(parent + sigma * n) on every
// parameter, n ~ N(0,1) from stream MUTATE at counter (step, parent's local
// slot, p / 4) for logical parameter p; then the child's streamed BF16 /
// FP8 copy is re-derived from its new master.
//
// Work items per birth: H/8 tiles of W_in (8 output rows x all D inputs),
// H/8 tiles of each hidden layer, and one item for W_out and the biases
// (small tiles: a step's few births spread over many CTAs).  A tile draws its
// normals in logical order (one Philox block per four parameters) into
// shared memory, then walks the master in its physical (input-major) order
// so global reads and writes are contiguous; FP8 row scales come from the
// tile's complete rows.  Block-level (any multiple of 32 threads).
// ---------------------------------------------------------------------------
constexpr int kMutRows = 8;
constexpr int kMutRowsLog2 = 3;
static_assert((1 << kMutRowsLog2) == kMutRows, "kMutRows is a power of two");

__device__ __forceinline__ uint8_t e4m3_sat(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// The births are (par[b], chi[b]) for b < nbirths when par is given (the
// fast path's pairs in shared memory), else the births list.
__device__ void ph_mutate(const Dev &d, const Layout &L, const Rules &R, int b0, int bs, float *msm,
                          float *s_scale, uint32_t t, const int *par, const int *chi, int nbirths) {
  const int D = L.D, H = L.H, A = L.A;
  const int nb = par ? nbirths : d.counters[CNT_N_BIRTHS];
  const int tiles = H / kMutRows;
  const int wtiles = (1 + L.L) * tiles;  // W_in, then each hidden layer
  const int items = wtiles + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int64_t mper = L.mstride / 4;

  for (int w = b0; w < nb * items; w += bs) {
    const int b = w / items, it = w - b * items;
    const int2 pc = par ? make_int2(par[b], chi[b]) : d.births[b];
    const EnvDesc ed = d.env[env_index(d, pc.y)];
    const uint32_t lp = (uint32_t)(pc.x - ed.slot_off);
    const float *pm = d.master + (int64_t)pc.x * mper;
    float *cm = d.master + (int64_t)pc.y * mper;
    uint8_t *cq = d.wq + (int64_t)pc.y * L.stride;
    if (it < wtiles) {
      const int layer = it / tiles;  // 0: W_in; l + 1: hidden layer l
      const bool l1 = layer == 0;
      const int o0 = (it - layer * tiles) * kMutRows;
      const int nin = l1 ? D : H;
      const int rs = nin + 1;  // padded shared-memory row stride
      // logical (o0, 0) and the physical start of the layer
      const int lbase = l1 ? o0 * D : D * H + L.ns * H + (layer - 1) * (H * H + H) + o0 * H;
      const int qbase = l1 ? 0 : D * H + (layer - 1) * H * H;
      const int srow = l1 ? 0 : H + (layer - 1) * H;  // first FP8 scale row of the layer
      const int nel = kMutRows * nin;
      const int g0 = lbase >> 2, g1 = (lbase + nel - 1) >> 2;
      for (int g = g0 + tid; g <= g1; g += nt) {
        const U4 r = philox(t, lp, (uint32_t)g, 0u, ed.seed, S_MUTATE);
        float n4[4];
        normals4(r, n4);
        // tile position (row rr, input j) of the group's first element,
        // then stepped: a group of four crosses at most one row end
        const int off0 = 4 * g - lbase;
        int rr = off0 >= 0 ? off0 / nin : 0, j = off0 - rr * nin;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int off = off0 + k;
          if (off >= 0 && off < nel) msm[rr * rs + j] = n4[k];
          if (++j == nin) {
            j = 0;
            ++rr;
          }
        }
      }
      __syncthreads();
      // the parent's master is read-only in this launch (parents and
      // children are different slots), so its loads need not wait for the
      // child's stores
#pragma unroll 4
      for (int idx = tid; idx < nel; idx += nt) {
        const int j = idx >> kMutRowsLog2, rr = idx & (kMutRows - 1);
        const int q = qbase + j * H + o0 + rr;
        const float v = fmaf(R.sigma, msm[rr * rs + j], __ldg(pm + q));
        cm[q] = v;
        msm[rr * rs + j] = v;
      }
      __syncthreads();
      if (R.precision == PREC_BF16) {
        __nv_bfloat16 *qw = reinterpret_cast<__nv_bfloat16 *>(cq);
        for (int idx = tid; idx < nel; idx += nt) {
          const int j = idx >> kMutRowsLog2, rr = idx & (kMutRows - 1);
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
            reinterpret_cast<float *>(cq + L.off_scale)[srow + o0 + rr] = s;
          }
        }
        __syncthreads();
        for (int idx = tid; idx < nel; idx += nt) {
          const int j = idx >> kMutRowsLog2, rr = idx & (kMutRows - 1);
          cq[qbase + j * H + o0 + rr] = e4m3_sat(__fdiv_rn(msm[rr * rs + j], s_scale[rr]));
        }
      }
      __syncthreads();
    } else {
      // the head (output-major) and every bias (and tau): master elements
      // [q3, q3 + n3) and [nW, nW + nB)
      const int n3 = A * H, nbias = L.nB;
      const int q3 = D * H + L.L * H * H;  // physical start of W_out
      for (int e = tid; e < n3 + nbias; e += nt) {
        const int q = e < n3 ? q3 + e : L.nW + (e - n3);
        const int p = layout_logical(L, q);
        const U4 r = philox(t, lp, (uint32_t)(p >> 2), 0u, ed.seed, S_MUTATE);
        const float v = fmaf(R.sigma, normal_of(r, p & 3), __ldg(pm + q));
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
          if (lane == 0) reinterpret_cast<float *>(cq + L.off_scale)[H + L.L * H + a] = s;
          for (int j = lane; j < H; j += 32) cq[q3 + a * H + j] = e4m3_sat(__fdiv_rn(msm[a * H + j], s));
        }
      }
      __syncthreads();
    }
  }
}

// The mutation in the persistent kernel, FP32 and BF16 forms (FP8 needs
// each row's maximum first and keeps ph_mutate's tiles): every parameter of
// every child is an independent element -- its normal comes from the
// Philox block of its logical index, as in ph_mutate -- so the grid's
// threads (g0, stride gs) take elements across children and layers with
// no block barrier between tiles.  The same draws and fmaf as ph_mutate,
// so the same values bit for bit; each element draws its own Philox block
// (four times the arithmetic of the tiled form, which the tiles' barriers
// and dependent loads outweigh).
__device__ void ph_mutate_flat(const Dev &d, const Layout &L, const Rules &R, uint32_t t, const int *par,
                               const int *chi, int nbirths, int g0, int gs) {
  const int nb = par ? nbirths : d.counters[CNT_N_BIRTHS];
  const int P = L.nW + L.nB;  // physical master elements: weights, then biases (and tau)
  const int64_t mper = L.mstride / 4;
  for (int w = g0; w < nb * P; w += gs) {
    const int b = w / P, q = w - b * P;
    const int2 pc = par ? make_int2(par[b], chi[b]) : d.births[b];
    const EnvDesc ed = d.env[env_index(d, pc.y)];
    const uint32_t lp = (uint32_t)(pc.x - ed.slot_off);
    const int p = layout_logical(L, q);
    const U4 r = philox(t, lp, (uint32_t)(p >> 2), 0u, ed.seed, S_MUTATE);
    const float v = fmaf(R.sigma, normal_of(r, p & 3), __ldg(d.master + (int64_t)pc.x * mper + q));
    d.master[(int64_t)pc.y * mper + q] = v;
    if (R.precision == PREC_BF16) {
      uint8_t *cq = d.wq + (int64_t)pc.y * L.stride;
      if (q < L.nW)
        reinterpret_cast<__nv_bfloat16 *>(cq)[q] = __float2bfloat16_rn(v);
      else
        reinterpret_cast<float *>(cq + L.off_bias)[q - L.nW] = v;
    }
  }
}

// Shared memory of the mutation: a tile of kMutRows rows of nin + 1 floats,
// where nin is D for W_in and H for the hidden layers (D may be below H: an
// agent without a vision sensor), or the head's A x H rows.
size_t mutate_smem_bytes(const Layout &L) {
  const size_t tile = (size_t)kMutRows * ((L.D > L.H ? L.D : L.H) + 1);
  const size_t head = (size_t)L.A * L.H;
  return 4 * (tile > head ? tile : head);
}

// A12: regrowth of food on non-wall food-less cells; four cells per thread
// share one Philox block (counter (step, local cell / 4)).
__device__ void ph_regrow(const Dev &d, const Rules &R, int g0, int gs, uint32_t t) {
  const int groups = d.total_cells >> 2;
  if (R.rules != RULES_TERRAIN) {
    // kRG of this thread's groups per round, their cell bytes loaded
    // together (the loop's stores would otherwise hold each load behind the
    // previous group's); the regrown count is kept per environment and
    // added once per environment (groups ascend, so environments do).
    constexpr int kRG = 4;
    int e = -1, grown_e = 0;
    EnvDesc ed = d.env[0];
    for (int gb = g0; gb < groups; gb += kRG * gs) {
      uchar4 cfv[kRG];
#pragma unroll
      for (int k = 0; k < kRG; ++k) {
        const int g = gb + k * gs;
        cfv[k] = g < groups ? reinterpret_cast<const uchar4 *>(d.cellf)[g] : make_uchar4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < kRG; ++k) {
        const int g = gb + k * gs;
        if (g >= groups) break;
        const int c0 = g << 2;
        if (e < 0 || (e + 1 < d.n_envs && d.env[e + 1].cell_off <= c0)) {
          if (e >= 0) stat_add(d.stats_step, e, ST_REGROWN, grown_e);
          grown_e = 0;
          e = env_of_cell(d.env, d.n_envs, c0);
          ed = d.env[e];
        }
        uchar4 cf = cfv[k];
        const bool any = !((cf.x & (CELL_WALL | CELL_FOOD)) && (cf.y & (CELL_WALL | CELL_FOOD)) &&
                           (cf.z & (CELL_WALL | CELL_FOOD)) && (cf.w & (CELL_WALL | CELL_FOOD)));
        if (!any) continue;
        const U4 r = philox(t, (uint32_t)((c0 - ed.cell_off) >> 2), 0u, 0u, ed.seed, S_REGROW);
        int mask = 0;
        if (!(cf.x & (CELL_WALL | CELL_FOOD)) && r.x < R.thr_regrow) { cf.x |= CELL_FOOD; mask |= 1; }
        if (!(cf.y & (CELL_WALL | CELL_FOOD)) && r.y < R.thr_regrow) { cf.y |= CELL_FOOD; mask |= 2; }
        if (!(cf.z & (CELL_WALL | CELL_FOOD)) && r.z < R.thr_regrow) { cf.z |= CELL_FOOD; mask |= 4; }
        if (!(cf.w & (CELL_WALL | CELL_FOOD)) && r.w < R.thr_regrow) { cf.w |= CELL_FOOD; mask |= 8; }
        if (!mask) continue;
        grown_e += __popc(mask);
        if (R.rules == RULES_PAPER)  // one bite of energy on each regrown cell
          for (int q = 0; q < 4; ++q)
            if (mask & (1 << q)) d.res[c0 + q] = R.e_food;
        reinterpret_cast<uchar4 *>(d.cellf)[g] = cf;
      }
    }
    if (e >= 0) stat_add(d.stats_step, e, ST_REGROWN, grown_e);
    return;
  }
  // terrain rules: one group per round (its biomass, energy and remainders
  // are loaded as 16-byte vectors); the counts are kept per environment
  int e = -1, grown_e = 0, refilled_e = 0;
  long long photo_e = 0;
  EnvDesc ed = d.env[0];
  auto flush = [&]() {
    if (e < 0) return;
    stat_add(d.stats_step, e, ST_REGROWN, grown_e);
    stat_add(d.stats_step, e, ST_FOOD_REFILLED, refilled_e);
    stat_add(d.stats_step, e, ST_PHOTO, (int)photo_e);
    grown_e = refilled_e = 0;
    photo_e = 0;
  };
  for (int g = g0; g < groups; g += gs) {
    const int c0 = g << 2;
    if (e < 0 || (e + 1 < d.n_envs && d.env[e + 1].cell_off <= c0)) {
      flush();
      e = env_of_cell(d.env, d.n_envs, c0);
      ed = d.env[e];
    }
    uchar4 cf = reinterpret_cast<uchar4 *>(d.cellf)[g];
    // the group's biomass, remainders and energy, loaded together (the
    // loads are independent; the chain per cell was the phase's cost)
    int bio[4], res[4];
    uint32_t pho[4];
    {
      const int4 b4 = reinterpret_cast<const int4 *>(d.bio)[g];
      const int4 r4 = reinterpret_cast<const int4 *>(d.res)[g];
      const uint4 p4 = reinterpret_cast<const uint4 *>(d.photo)[g];
      bio[0] = b4.x, bio[1] = b4.y, bio[2] = b4.z, bio[3] = b4.w;
      res[0] = r4.x, res[1] = r4.y, res[2] = r4.z, res[3] = r4.w;
      pho[0] = p4.x, pho[1] = p4.y, pho[2] = p4.z, pho[3] = p4.w;
    }
    int grown = 0;
    const bool any = !((cf.x & (CELL_WALL | CELL_FOOD)) && (cf.y & (CELL_WALL | CELL_FOOD)) &&
                       (cf.z & (CELL_WALL | CELL_FOOD)) && (cf.w & (CELL_WALL | CELL_FOOD)));
    // a zero threshold (no random regrowth) grows nothing: no draw needed
    if (any && R.thr_regrow != 0u) {
      const U4 r = philox(t, (uint32_t)((c0 - ed.cell_off) >> 2), 0u, 0u, ed.seed, S_REGROW);
      int mask = 0;
      if (!(cf.x & (CELL_WALL | CELL_FOOD)) && r.x < R.thr_regrow) { cf.x |= CELL_FOOD; mask |= 1; }
      if (!(cf.y & (CELL_WALL | CELL_FOOD)) && r.y < R.thr_regrow) { cf.y |= CELL_FOOD; mask |= 2; }
      if (!(cf.z & (CELL_WALL | CELL_FOOD)) && r.z < R.thr_regrow) { cf.z |= CELL_FOOD; mask |= 4; }
      if (!(cf.w & (CELL_WALL | CELL_FOOD)) && r.w < R.thr_regrow) { cf.w |= CELL_FOOD; mask |= 8; }
      grown = __popc(mask);
      for (int k = 0; k < 4; ++k)  // one bite of energy on each regrown cell, in the group's registers
        if (mask & (1 << k)) res[k] = R.e_food;
    }
    bool changed = grown != 0;
    // energy grows on free biomass: a 2^-16 fixed-point remainder per cell
    // makes the sum over steps exact; at most res_cap energy per cell
    uint8_t *cfb = reinterpret_cast<uint8_t *>(&cf);
    bool touched = grown != 0;
    for (int k = 0; k < 4; ++k) {
      const int b = bio[k];
      if ((cfb[k] & CELL_WALL) || b <= 0) continue;
      const unsigned long long acc = (unsigned long long)pho[k] + (unsigned long long)b * (unsigned)R.photo_q16;
      pho[k] = (uint32_t)(acc & 0xFFFFull);
      touched = true;
      const int r = res[k];
      const long long gain = min((long long)(acc >> 16), (long long)R.res_cap - r);
      if (gain <= 0) continue;
      if (r == 0) {
        cfb[k] |= (uint8_t)CELL_FOOD;
        ++refilled_e;
        changed = true;
      }
      res[k] = r + (int)gain;
      photo_e += gain;
    }
    if (touched) {
      reinterpret_cast<int4 *>(d.res)[g] = make_int4(res[0], res[1], res[2], res[3]);
      reinterpret_cast<uint4 *>(d.photo)[g] = make_uint4(pho[0], pho[1], pho[2], pho[3]);
    }
    if (changed) reinterpret_cast<uchar4 *>(d.cellf)[g] = cf;
    grown_e += grown;
  }
  flush();
}

// Terrain rules, water flow (Sec. 3.2 "Terrain"), part 1: each cell's
// transfer from the surfaces (rock + water) before the step.  A wet
// non-wall cell sends min(water, floor(drop / 5)) to its lowest non-wall
// neighbour (the first of N, E, S, W on ties) when that one lies `drop`
// below it.  Stored as amount << 2 | direction (amount 0: none); the total
// water of an environment is below 2^30, so the amount fits.
//
// Both parts take cells in groups of four along a row (cell offsets and
// sides are even; a group stays in one row when the side is a multiple of
// four): the group, the four cells above and below it (16-byte loads) and
// the two at its ends are loaded together, so a group costs one round
// trip of independent loads.  Other sides take the neighbours one by one.
__device__ __forceinline__ uint32_t flow_pick(int w, long long here, const long long hn[4], const bool wn[4]) {
  long long lowest = 0;
  int best = -1;
#pragma unroll
  for (int dir = 0; dir < 4; ++dir) {
    if (wn[dir]) continue;
    if (best < 0 || hn[dir] < lowest) {
      best = dir;
      lowest = hn[dir];
    }
  }
  if (best >= 0 && lowest < here) {
    const long long amount = min((here - lowest) / 5, (long long)w);
    return ((uint32_t)amount << 2) | (uint32_t)best;
  }
  return 0u;
}

// The four cells of a group and their neighbours: global indices of the
// group start, the rows above and below (same columns) and the cells west
// of the first and east of the last.
struct FlowGroup {
  int c0, up0, dn0, west, east;
};

__device__ __forceinline__ FlowGroup flow_group(const EnvDesc &ed, int c0) {
  const int lc = c0 - ed.cell_off, L = ed.side;
  const int x0 = lc % L, y = lc / L;
  const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
  FlowGroup fg;
  fg.c0 = c0;
  fg.up0 = ed.cell_off + yu * L + x0;
  fg.dn0 = ed.cell_off + yd * L + x0;
  fg.west = ed.cell_off + y * L + (x0 == 0 ? L - 1 : x0 - 1);
  fg.east = ed.cell_off + y * L + (x0 + 4 == L ? 0 : x0 + 4);
  return fg;
}

__device__ __forceinline__ void unpack4(const int4 v, int o[4]) { o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w; }

__device__ void ph_flow_out(const Dev &d, int g0, int gs) {
  const int groups = d.total_cells >> 2;
  for (int g = g0; g < groups; g += gs) {
    const int c0 = g << 2;
    int w[4];
    unpack4(reinterpret_cast<const int4 *>(d.water)[g], w);
    const uchar4 cf4 = reinterpret_cast<const uchar4 *>(d.cellf)[g];
    const uint8_t cf[4] = {cf4.x, cf4.y, cf4.z, cf4.w};
    bool wet[4], any = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      wet[k] = w[k] > 0 && !(cf[k] & CELL_WALL);
      any |= wet[k];
    }
    uint32_t f[4] = {0u, 0u, 0u, 0u};
    if (any) {
      const EnvDesc ed = d.env[env_of_cell(d.env, d.n_envs, c0)];
      int rk[4];
      unpack4(reinterpret_cast<const int4 *>(d.rock)[g], rk);
      if ((ed.side & 3) == 0) {
        const FlowGroup fg = flow_group(ed, c0);
        int wu[4], ru[4], wd[4], rd[4];
        unpack4(*reinterpret_cast<const int4 *>(d.water + fg.up0), wu);
        unpack4(*reinterpret_cast<const int4 *>(d.rock + fg.up0), ru);
        unpack4(*reinterpret_cast<const int4 *>(d.water + fg.dn0), wd);
        unpack4(*reinterpret_cast<const int4 *>(d.rock + fg.dn0), rd);
        const uchar4 cu = *reinterpret_cast<const uchar4 *>(d.cellf + fg.up0);
        const uchar4 cd = *reinterpret_cast<const uchar4 *>(d.cellf + fg.dn0);
        const uint8_t cuv[4] = {cu.x, cu.y, cu.z, cu.w}, cdv[4] = {cd.x, cd.y, cd.z, cd.w};
        const long long hw = (long long)d.rock[fg.west] + d.water[fg.west];
        const long long he = (long long)d.rock[fg.east] + d.water[fg.east];
        const bool ww = (d.cellf[fg.west] & CELL_WALL) != 0, we = (d.cellf[fg.east] & CELL_WALL) != 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!wet[k]) continue;
          // N, E, S, W
          const long long hn[4] = {(long long)ru[k] + wu[k],
                                   k < 3 ? (long long)rk[k + 1] + w[k + 1] : he,
                                   (long long)rd[k] + wd[k],
                                   k > 0 ? (long long)rk[k - 1] + w[k - 1] : hw};
          const bool wn[4] = {(cuv[k] & CELL_WALL) != 0, k < 3 ? (cf[k + 1] & CELL_WALL) != 0 : we,
                              (cdv[k] & CELL_WALL) != 0, k > 0 ? (cf[k - 1] & CELL_WALL) != 0 : ww};
          f[k] = flow_pick(w[k], (long long)rk[k] + w[k], hn, wn);
        }
      } else {
        for (int k = 0; k < 4; ++k) {
          if (!wet[k]) continue;
          const int lc = c0 + k - ed.cell_off;
          long long hn[4];
          bool wn[4];
          for (int dir = 0; dir < 4; ++dir) {
            const int n = ed.cell_off + step_cell(lc, dir, ed.side);
            wn[dir] = (d.cellf[n] & CELL_WALL) != 0;
            hn[dir] = (long long)d.rock[n] + d.water[n];
          }
          f[k] = flow_pick(w[k], (long long)rk[k] + w[k], hn, wn);
        }
      }
    }
    reinterpret_cast<uint4 *>(d.flow)[g] = make_uint4(f[0], f[1], f[2], f[3]);
  }
}

// Part 2: every cell gives its transfer and takes those of the neighbours
// that point at it (a neighbour in direction dir points back with dir + 2).
// Only this cell's water is written, from the transfers alone.
__device__ __forceinline__ int flow_in_of(uint32_t fn, int dir) {
  return ((fn >> 2) && (int)(fn & 3u) == ((dir + 2) & 3)) ? (int)(fn >> 2) : 0;
}

__device__ void ph_flow_in(const Dev &d, int g0, int gs) {
  const int groups = d.total_cells >> 2;
  for (int g = g0; g < groups; g += gs) {
    const int c0 = g << 2;
    const uchar4 cf4 = reinterpret_cast<const uchar4 *>(d.cellf)[g];
    const uint8_t cf[4] = {cf4.x, cf4.y, cf4.z, cf4.w};
    if ((cf[0] & cf[1] & cf[2] & cf[3]) & CELL_WALL) continue;
    int w[4];
    unpack4(reinterpret_cast<const int4 *>(d.water)[g], w);
    const uint4 f4 = reinterpret_cast<const uint4 *>(d.flow)[g];
    const uint32_t f[4] = {f4.x, f4.y, f4.z, f4.w};
    const EnvDesc ed = d.env[env_of_cell(d.env, d.n_envs, c0)];
    if ((ed.side & 3) == 0) {
      const FlowGroup fg = flow_group(ed, c0);
      const uint4 fu4 = *reinterpret_cast<const uint4 *>(d.flow + fg.up0);
      const uint4 fd4 = *reinterpret_cast<const uint4 *>(d.flow + fg.dn0);
      const uint32_t fu[4] = {fu4.x, fu4.y, fu4.z, fu4.w}, fd[4] = {fd4.x, fd4.y, fd4.z, fd4.w};
      const uint32_t fw = d.flow[fg.west], fe = d.flow[fg.east];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (cf[k] & CELL_WALL) continue;
        int v = w[k] - (int)(f[k] >> 2);
        v += flow_in_of(fu[k], 0);
        v += flow_in_of(k < 3 ? f[k + 1] : fe, 1);
        v += flow_in_of(fd[k], 2);
        v += flow_in_of(k > 0 ? f[k - 1] : fw, 3);
        w[k] = v;
      }
    } else {
      for (int k = 0; k < 4; ++k) {
        if (cf[k] & CELL_WALL) continue;
        const int lc = c0 + k - ed.cell_off;
        int v = w[k] - (int)(f[k] >> 2);
        for (int dir = 0; dir < 4; ++dir) v += flow_in_of(d.flow[ed.cell_off + step_cell(lc, dir, ed.side)], dir);
        w[k] = v;
      }
    }
    reinterpret_cast<int4 *>(d.water)[g] = make_int4(w[0], w[1], w[2], w[3]);
  }
}

// The step's birth counters back to zero (block-level), after clearing the
// birth-cell claims of the step's claimants (the fast birth path leaves
// them: its CTAs read them until the launch ends).
__device__ void reset_birth_counters(const Dev &d) {
  for (int e = 0; e < d.n_envs; ++e) {
    const EnvDesc ed = d.env[e];
    const int nc = d.birth_contenders[e];
    for (int i = threadIdx.x; i < nc; i += blockDim.x) d.claim_birth[ed.cell_off + d.bcell[ed.slot_off + i]] = 0ull;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_envs; i += blockDim.x) d.birth_contenders[i] = 0;
  if (threadIdx.x == 0) {
    d.counters[CNT_N_BIRTHS] = 0;
    d.counters[CNT_CONTENDERS] = 0;
  }
}

// A13: fold this step's counters into the per-environment records and
// advance the step counter (one CTA).  Agent-steps and attacks come from the
// action histogram the policy kernel counted.
// reset_counters: also clear this step's birth counters (the one-kernel-
// per-phase form; the persistent form clears them at its next launch's
// start, because its other CTAs may still read them here).
__device__ void ph_finish(const Dev &d, const Rules &R, bool reset_counters) {
  const long long t = d.step[0];
  for (int i = threadIdx.x; i < d.n_envs; i += blockDim.x) {
    long long *st = d.stats_step + i * N_ST;
    long long as = 0;
    for (int a = 0; a < 16; ++a) as += st[ST_ACT0 + a];
    st[ST_AGENT_STEPS] = as;
    st[ST_ATTACKS] = st[ST_ACT0 + (R.rules != RULES_SIMPLE ? PA_ATTACK : ACT_ATTACK)];
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
      v = R.rules != RULES_SIMPLE ? tot[k] + st[ST_REGROWN] - st[ST_FOOD_EMPTIED] + st[ST_FOOD_REFILLED]
                                 : tot[k] + st[ST_REGROWN] - st[ST_EATEN];
    } else if (k == ST_ENERGY_TOTAL) {
      v = R.rules != RULES_SIMPLE
              ? tot[k] + st[ST_EATEN_ENERGY] - st[ST_METAB_PAID] - (long long)R.heal_cost * st[ST_HEALS] -
                    st[ST_DEAD_ENERGY]
              : tot[k] + (long long)R.e_food * st[ST_EATEN] - (long long)R.e_metab * st[ST_AGENT_STEPS] -
                    st[ST_DEAD_ENERGY];
    } else if (k == ST_RES_TOTAL) {
      v = R.rules != RULES_SIMPLE ? tot[k] + (long long)R.e_food * st[ST_REGROWN] - st[ST_EATEN_ENERGY] +
                                        st[ST_DEAD_ENERGY] + st[ST_PHOTO]
                                  : 0;
    } else if (k == ST_WATER_CELLS || k == ST_WATER_AGENTS) {
      // the flow moves water between cells only
      const long long to_cells = st[ST_WATER_SPENT] + st[ST_DEAD_WATER] - st[ST_DRUNK];
      v = tot[k] + (k == ST_WATER_CELLS ? to_cells : -to_cells);
    } else if (k == ST_BIO_CELLS || k == ST_BIO_AGENTS) {
      const long long to_cells = st[ST_DEAD_BIO] - st[ST_BIO_EATEN];
      v = tot[k] + (k == ST_BIO_CELLS ? to_cells : -to_cells);
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
  if (threadIdx.x == 0) d.step[0] = t + 1;
  if (reset_counters) reset_birth_counters(d);
}

// ---------------------------------------------------------------------------
// One kernel per phase.
// ---------------------------------------------------------------------------
#define GRID_ARGS blockIdx.x *blockDim.x + threadIdx.x, gridDim.x *blockDim.x

__global__ void __launch_bounds__(256) k_compact_count(Dev d) {
  __shared__ int sh[33];
  ph_compact_count(d, blockIdx.x, gridDim.x, sh);
}
__global__ void __launch_bounds__(256) k_compact_scatter(Dev d) {
  __shared__ int sh[33];
  ph_compact_scatter(d, blockIdx.x, gridDim.x, sh, (uint32_t)d.step[0], nullptr, 0, nullptr);
}
#define STEP_T ((uint32_t)d.step[0])
__global__ void k_move_apply_eat(Dev d, Rules R, int A) { ph_move_apply_eat(d, R, A, GRID_ARGS, -1, STEP_T); }
__global__ void k_metab_death(Dev d, Rules R) { ph_metab_death(d, R, GRID_ARGS, -1, STEP_T); }
__global__ void k_birth_claim(Dev d, Rules R) { ph_birth_claim(d, R, GRID_ARGS, -1, STEP_T); }
__global__ void __launch_bounds__(1024) k_birth_assign(Dev d, Rules R) {
  __shared__ BirthSmem S;
  ph_birth_assign(d, R, blockIdx.x, gridDim.x, S, STEP_T);
}
__global__ void __launch_bounds__(256) k_mutate(Dev d, Layout L, Rules R) {
  extern __shared__ __align__(16) float msm[];
  __shared__ float s_scale[kMutRows];
  ph_mutate(d, L, R, blockIdx.x, gridDim.x, msm, s_scale, STEP_T, nullptr, nullptr, 0);
}
__global__ void k_regrow(Dev d, Rules R) { ph_regrow(d, R, GRID_ARGS, STEP_T); }
__global__ void k_flow_out(Dev d) { ph_flow_out(d, GRID_ARGS); }
__global__ void k_flow_in(Dev d) { ph_flow_in(d, GRID_ARGS); }
__global__ void k_finish(Dev d, Rules R) { ph_finish(d, R, true); }
#undef STEP_T

// ---------------------------------------------------------------------------
// The persistent form: all phases in one cooperative launch.
// ---------------------------------------------------------------------------
constexpr unsigned kBarrierSpinLimit = 40u * 1000u * 1000u;  // x >= 64 ns: > 2.5 s
constexpr int kStatusTimeout = 4;

// Grid-wide barrier for a co-resident (cooperative) grid.  One arrival
// count per launch (count = the word of the step's parity; the launch of
// step t clears the word of step t + 1 at its start): at its k-th barrier
// every CTA adds 1 (a reduction whose result it does not wait for) and
// waits until the count reaches k * nblocks.  The wait is bounded by
// `budget` polls: when it runs out, the status word records a timeout and
// the CTA adds kBroken to the count, which releases every present and
// later wait of the launch as failed, so every CTA leaves the kernel at its
// next barrier.  Returns false when the kernel must stop.
constexpr unsigned kBroken = 1u << 30;  // above any k * nblocks

__device__ bool grid_sync(unsigned *count, int *status_word, unsigned nblocks, unsigned budget, unsigned &k,
                          int *s_flag) {
  __syncthreads();
  ++k;
  if (nblocks == 1) return true;  // one CTA: the block barrier is the grid barrier
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(*count);
    const unsigned target = k * nblocks;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    unsigned it = 0, v;
    int ok = 1;
    while ((v = cnt.load(cuda::memory_order_acquire)) < target) {
      if (++it > budget) {
        cuda::atomic_ref<int, cuda::thread_scope_device>(*status_word)
            .fetch_or(kStatusTimeout, cuda::memory_order_relaxed);
        cnt.fetch_add(kBroken, cuda::memory_order_relaxed);
        ok = 0;
        break;
      }
      if (it > 2048) __nanosleep(64);  // spin first: most waits are short
    }
    if (v >= kBroken) ok = 0;
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// One world, for the fast birth path: the first free slots of every
// compaction tile of 4096 slots (at most kFastBirths, env-local, ascending)
// into free_list[tile * kFastBirths + i], and the tile's free count into
// free_tiles[tile]; once the deaths are final and before any birth.  Tile k
// is scanned by CTA nb - 1 - k (the last CTAs have the least grid-stride
// work in the birth-claim interval), four slots per thread.
__device__ void list_free_slots(const Dev &d, int *sh) {
  const int n = d.env[0].n_slots;
  const int tiles = (n + kCompactTile - 1) / kCompactTile;
  for (int tile = (int)gridDim.x - 1 - (int)blockIdx.x; tile >= 0 && tile < tiles; tile += gridDim.x) {
    const int s0 = tile * kCompactTile + threadIdx.x * 4;
    uint32_t mask = 0u;  // free bits of slots s0 .. s0 + 3
    if (threadIdx.x < kCompactTile / 4) {
      if (s0 + 4 <= n) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(d.alive + s0);  // 4-byte aligned
        mask = ((__vcmpeq4(w, 0u) & 0x80808080u) * 0x00204081u) >> 28;
      } else {
        for (int k = 0; k < 4; ++k)
          if (s0 + k < n && !d.alive[s0 + k]) mask |= 1u << k;
      }
    }
    int total;
    int r = block_exclusive_scan(__popc(mask), &total, sh);
    while (mask && r < kFastBirths) {
      const int k = __ffs(mask) - 1;
      d.free_list[tile * kFastBirths + r++] = s0 + k;
      mask &= mask - 1;
    }
    if (threadIdx.x == 0) d.free_tiles[tile] = total;
  }
}

// The fast birth path (one environment, at most kFastBirths claimants):
// every CTA derives the same births from the claims and the free-slot list
// (written in the birth-claim phase, when the deaths were final), so no
// barrier separates the slot assignment
// from the mutation and the alive list: pair i is (S.win[i], S.free_[i]),
// i < S.nborn, of S.nwin winners.
__device__ void fast_births(const Dev &d, BirthSmem &S, int nc) {
  const EnvDesc ed = d.env[0];
  // The first nc free slots (at most nc are needed), read with the claims
  // rather than after the sort: from the per-tile lists of list_free_slots,
  // tile k's entries covering ranks [before_k, before_k + min(free_k, cap)).
  const int tiles = (ed.n_slots + kCompactTile - 1) / kCompactTile;
  if (threadIdx.x == 0) {
    int before = 0;
    for (int k = 0; k < tiles; ++k) {
      S.tile_first[k] = before;
      before += d.free_tiles[k];
    }
    S.nfree = before;
  }
  __syncthreads();
  const int want = nc < S.nfree ? nc : S.nfree;
  for (int i = threadIdx.x; i < want; i += blockDim.x) {
    int k = 0;
    while (k + 1 < tiles && S.tile_first[k + 1] <= i) ++k;
    S.free_[i] = ed.slot_off + d.free_list[k * kFastBirths + (i - S.tile_first[k])];
  }
  const int nwin = sort_winners(d, ed, nc, S);  // synchronises the CTA
  const int nborn = nwin < S.nfree ? nwin : S.nfree;
  if (threadIdx.x == 0) S.nborn = nborn;
  __syncthreads();
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

__global__ void __launch_bounds__(1024, 1) k_env_persistent(Dev d, Layout L, Rules R) {
  extern __shared__ __align__(16) float msm[];
  __shared__ BirthSmem S;
  __shared__ float s_scale[kMutRows];
  __shared__ int s_flag;
  const unsigned nb = gridDim.x;
  const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  // The launch's first reads, issued together: the step, the failure-
  // detection test words (0 unless armed by eco_arm_barrier_timeout,
  // cleared by eco_reset: a CTA that leaves before its first barrier, and the
  // poll budget of every wait), the phase-trace switch, the alive count and
  // each thread's first alive-list entry (loaded once for all phases; the
  // list has total_slots entries, so the read stays in bounds even past the
  // count).  Every phase takes the step from here: the statistics CTA
  // advances the step word in the last interval while other CTAs still work
  // on this step.
  const uint32_t t = (uint32_t)d.step[0];
  const unsigned absent = d.barrier[BAR_ABSENT_CTA], budget_word = d.barrier[BAR_BUDGET];
  const unsigned trace_on = d.barrier[BAR_TRACE];
  const int n_alive = d.counters[CNT_N_ALIVE];
  const int first_entry = g0 < d.total_slots ? d.alive_list[g0] : -1;
  // A timeout recorded by an earlier launch (the status word keeps it until
  // eco_reset) stops this step at once, before any barrier count changes;
  // one read per CTA decides for all its threads.
  if (threadIdx.x == 0) {
    s_flag = cuda::atomic_ref<int, cuda::thread_scope_device>(d.counters[CNT_STATUS]).load(
                 cuda::memory_order_relaxed) & kStatusTimeout;
  }
  __syncthreads();
  if (s_flag) return;
  if (absent == blockIdx.x + 1u) return;
  const unsigned budget = budget_word ? budget_word : kBarrierSpinLimit;
  unsigned *count = d.barrier + BAR_COUNT0 + (t & 1u);
  unsigned bar = 0;  // barriers passed in this launch (the same sequence in every CTA)
  // Phase trace (eco_trace_phases): this step's row; CTA 0 clears the next
  // step's row (its maxima must start at 0).
  unsigned long long *trow = trace_on ? d.trace + (size_t)(t % kTraceSteps) * kTraceWords : nullptr;
  if (trow && blockIdx.x == 0) {
    if (threadIdx.x < kTraceWords) d.trace[(size_t)((t + 1u) % kTraceSteps) * kTraceWords + threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
      trow[TR_START] = global_ns();
      trow[TR_STEP] = (unsigned long long)t;
    }
  }
  // the grid barrier, with the trace's arrival and pass stamps
  auto sync = [&]() -> bool {
    if (trow) {
      __syncthreads();
      if (threadIdx.x == 0) atomicMax(trow + TR_ARRIVE0 + bar, global_ns());
    }
    const bool ok = grid_sync(count, d.counters + CNT_STATUS, nb, budget, bar, &s_flag);
    if (trow && blockIdx.x == 0 && threadIdx.x == 0) trow[TR_PASS0 + bar - 1] = global_ns();
    return ok;
  };
  // Housekeeping goes to CTAs with little else to do in its interval: the
  // per-agent phases take one agent per thread from CTA 0 on, and the
  // alive list's tiles go to CTAs 0 .. tiles - 1.
  const int tiles = compact_tiles(d.total_slots);
  const unsigned last = nb - 1u;
  const unsigned fold_cta = (unsigned)tiles < nb ? (unsigned)tiles : 0u;      // statistics
  const unsigned birth_cta = fold_cta + 1u < nb ? fold_cta + 1u : 0u;         // fast-path births
  if (blockIdx.x == last) {
    // the previous launch is over: clear its birth counters and the next
    // launch's arrival count (this launch's was cleared by the previous one,
    // or by eco_reset); nothing reads them before the second barrier
    reset_birth_counters(d);
    if (threadIdx.x == 0) d.barrier[BAR_COUNT0 + ((t + 1u) & 1u)] = 0u;
  }
  const int first = g0 < n_alive ? first_entry : -1;
  ph_move_apply_eat(d, R, L.A, g0, gs, first, t);
  if (!sync()) return;
  ph_metab_death(d, R, g0, gs, first, t);
  if (!sync()) return;
  // regrowth (with photosynthesis and the flow's transfers) needs only the
  // state after the deaths, and birth claims read only wall and agent bits,
  // which regrowth keeps: the two share an interval
  ph_birth_claim(d, R, g0, gs, first, t);
  if (d.n_envs == 1 && compact_tiles(d.total_slots) <= kMaxFastTiles) list_free_slots(d, S.sh);
  ph_regrow(d, R, g0, gs, t);
  if (R.rules == RULES_TERRAIN) ph_flow_out(d, g0, gs);
  if (!sync()) return;
  // Every claim is in, and the count of claimants does not change again
  // in this launch, so every CTA takes the same branch.
  const int claimants = cuda::atomic_ref<int, cuda::thread_scope_device>(d.counters[CNT_CONTENDERS]).load(
      cuda::memory_order_relaxed);
  const bool fast = claimants > 0 && d.n_envs == 1 && claimants <= kFastBirths &&
                    compact_tiles(d.total_slots) <= kMaxFastTiles;
  if (trow && blockIdx.x == 0 && threadIdx.x == 0) trow[TR_CLAIMANTS] = (unsigned long long)claimants;
  if (claimants > 0 && !fast) {
    // general path: one CTA per environment assigns the slots, then a barrier
    ph_birth_assign(d, R, blockIdx.x, gridDim.x, S, t);
    if (!sync()) return;
  } else if (fast) {
    fast_births(d, S, claimants);
  }
  // Every statistic of the step is in (the fast path's births are counted
  // here): one CTA folds them while the others go on.
  if (blockIdx.x == fold_cta) {
    if (fast && threadIdx.x == 0) {
      d.stats_step[ST_BIRTHS] += S.nborn;
      d.stats_step[ST_FAILED_BIRTHS] += S.nwin - S.nborn;
    }
    __syncthreads();
    ph_finish(d, R, false);
  }
  if (fast) {
    // the births' side effects, pair by pair over every thread of the grid
    // (the claims stay until the next launch clears them: other CTAs may
    // still be reading them in fast_births)
    const EnvDesc ed = d.env[0];
    const int gb = (int)((blockIdx.x + nb - birth_cta) % nb) * (int)blockDim.x + (int)threadIdx.x;
    for (int i = gb; i < S.nborn; i += gs) {
      const int p = S.win[i];
      make_child(d, R, ed, p, S.free_[i], d.tgt[p], t, false);
    }
  }
  // The rest -- the water flow's second pass, the next step's alive list,
  // the children's weights -- writes nothing that another CTA reads in this
  // launch, so no barrier follows.  Mutation work starts from the last CTA,
  // the alive list from the first.
  if (R.rules == RULES_TERRAIN) ph_flow_in(d, g0, gs);
  ph_compact_scatter(d, blockIdx.x, gridDim.x, S.sh, t, fast ? S.free_ : nullptr, fast ? S.nborn : 0, S.cmask);
  if (claimants > 0) {
    if (R.precision != PREC_FP8)
      ph_mutate_flat(d, L, R, t, fast ? S.win : nullptr, fast ? S.free_ : nullptr, fast ? S.nborn : 0,
                     (int)((gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x));
    else
      ph_mutate(d, L, R, gridDim.x - 1 - blockIdx.x, gridDim.x, msm, s_scale, t, fast ? S.win : nullptr,
                fast ? S.free_ : nullptr, fast ? S.nborn : 0);
  }
  if (trow) {
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicMax(trow + TR_END, global_ns());
      if (blockIdx.x == 0) trow[TR_BARRIERS] = bar;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_compact(const Dev &d, cudaStream_t s) {
  const int tiles = compact_tiles(d.total_slots);
  k_compact_count<<<tiles, 256, 0, s>>>(d);
  k_compact_scatter<<<tiles, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t env_prepare(const Layout &L, EnvGrid *g) {
  const size_t smem = mutate_smem_bytes(L);
  cudaError_t e = cudaFuncSetAttribute((const void *)k_mutate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void *)k_env_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, coop = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_env_persistent, 1024,
                                                         smem)) != cudaSuccess)
    return e;
  // one CTA per SM: fewer arrivals on the barrier counter
  g->persistent_blocks = (coop && per_sm >= 1) ? g->sms : 0;
  return cudaSuccess;
}

// The step's phases after the policy kernel, ending with the alive list of
// the next step.
cudaError_t launch_env_phases(const Dev &d, const Layout &L, const Rules &R, const EnvGrid &g,
                              cudaStream_t s) {
  const size_t msmem = mutate_smem_bytes(L);
  if (g.persistent_blocks > 0 && g.use_persistent) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.persistent_blocks);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = msmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_env_persistent, d, L, R);
  }
  const int T = 256;
  k_move_apply_eat<<<g.slot_blocks, T, 0, s>>>(d, R, L.A);
  k_metab_death<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_claim<<<g.slot_blocks, T, 0, s>>>(d, R);
  k_birth_assign<<<d.n_envs, 1024, 0, s>>>(d, R);
  k_mutate<<<g.birth_blocks, 256, msmem, s>>>(d, L, R);
  k_regrow<<<g.cell_blocks, T, 0, s>>>(d, R);
  if (R.rules == RULES_TERRAIN) {
    const int fb = grid_for(d.total_cells / 4, T, g.sms * 8);
    k_flow_out<<<fb, T, 0, s>>>(d);
    k_flow_in<<<fb, T, 0, s>>>(d);
  }
  // the tile counts are current: the second pass of the compaction only,
  // before k_finish advances the step (the counts are kept per step parity)
  k_compact_scatter<<<compact_tiles(d.total_slots), 256, 0, s>>>(d);
  k_finish<<<1, 1024, 0, s>>>(d, R);
  return cudaGetLastError();
}

}  // namespace eco
