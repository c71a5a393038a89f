// eco_api.cu -- the C-ABI declared in include/eco.h: configuration checks,
// the parameter-block layout, carving of the caller's workspace, the CUDA
// graph of one step, the policy-variant autotuner, and host <-> device
// state and parameter I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/eco.h"
#include "eco_internal.cuh"
#include "eco_kernels.h"

using namespace eco;

static_assert((int)ECO_STAT_ACT0 == (int)eco::ST_ACT0, "stat enum");
static_assert((int)ECO_STAT_ENERGY_TOTAL == (int)eco::ST_ENERGY_TOTAL, "stat enum");
static_assert((int)ECO_N_STATS == (int)eco::N_ST, "stat enum");
static_assert(sizeof(eco_stats) == sizeof(long long) * eco::N_ST, "stat record");

static char g_err[512] = "";

struct eco_handle {
  // configuration
  int n_envs;
  std::vector<int32_t> side, slots, init_alive;
  std::vector<uint32_t> seed;
  Layout L;
  Rules R;
  // device
  Dev d;
  std::vector<EnvDesc> env_host;
  EnvDesc *env_dev;
  uint8_t *ws;
  size_t ws_bytes;
  cudaStream_t stream;
  bool own_stream;
  EnvGrid grid;
  // policy
  int variant;       // chosen variant (0 = not chosen yet)
  int forced;        // variant forced by the configuration (0 = autotune the dense
                     // variants, -1 = autotune the input-sparse ones)
  PolicyLaunch pl;
  // step graphs: [GRAPH_TIMED] one step with event-record nodes around the
  // policy kernel (eco_step_timed), [GRAPH_ONE] one step, [GRAPH_MANY]
  // kStepsPerGraph steps (eco_step).  An event-record node costs a few us
  // on the critical path between two kernels, so the untimed graphs have
  // none, and a graph of several steps saves the launch gap between graphs.
  // [GRAPH_READ1], [GRAPH_READ2]: one step, then a copy of the statistics
  // into pinned slot 1 or 2 (eco_step_read); [GRAPH_TIMED_MANY]:
  // kStepsPerGraph steps with event-record nodes around the first step's
  // policy kernel only (eco_step_timed: one timed launch per graph)
  cudaGraphExec_t graph[6];
  cudaGraph_t graph_src[6];  // kept alive: their node handles address the execs' nodes
  cudaGraphNode_t ev_node[6][2];  // in the timed graphs
  // steps run since reset (a host shadow of the device's step counter) and
  // the first step of every timed launch not yet reported
  long long steps_done;
  std::vector<long long> timed_steps;
  cudaEvent_t ev_dummy[2];
  std::vector<cudaEvent_t> ev_pool;  // pairs
  int ev_used;
  // pinned host mirrors of [stats_total, stats_last, counters], contiguous
  // in the workspace, rd_bytes each: slot 0 for eco_read_stats, slots 1 and
  // 2 for eco_step_read, whose copy of slot rd_pending (0: none) may still
  // be in flight, completion marked by rd_ev[slot - 1]
  uint8_t *rd_host;
  size_t rd_bytes;
  int rd_pending;
  cudaEvent_t rd_ev[2];
  char err[512];
};

static int fail(eco_handle *h, int code, const char *fmt, ...) {
  char *dst = h ? h->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  if (h) snprintf(g_err, sizeof(g_err), "%s", h->err);
  return code;
}

int eco::set_global_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(h, call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail((h), ECO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static int64_t pad(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Bernoulli threshold floor(p * 2^32) (same definition as the method's).
static uint32_t threshold_of(float p) {
  const double v = (double)p;
  if (!(v > 0.0)) return 0u;
  if (v >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)std::floor(v * 4294967296.0);
}

static int validate(const eco_config *c, char *msg, size_t n) {
  if (!c) return snprintf(msg, n, "null config"), ECO_EINVAL;
  if (c->abi_version != ECO_ABI_VERSION) return snprintf(msg, n, "abi_version %d != %d", c->abi_version, ECO_ABI_VERSION), ECO_EABI;
  if (c->n_envs < 1 || c->n_envs > 4096) return snprintf(msg, n, "n_envs out of range"), ECO_EINVAL;
  if (!c->env_side || !c->env_slots || !c->env_init_alive || !c->env_seed)
    return snprintf(msg, n, "null per-environment array"), ECO_EINVAL;
  if (c->patch_k < 0 || (c->patch_k > 0 && (c->patch_k & 1) == 0) || c->patch_k > 31)
    return snprintf(msg, n, "patch_k must be 0 (no vision) or odd in [1, 31]"), ECO_EINVAL;
  const bool terrain = c->rules == ECO_RULES_TERRAIN;
  if (terrain ? c->n_scalars != 16 : (c->n_scalars != 4 && c->n_scalars != 8))
    return snprintf(msg, n, "n_scalars must be 4 or 8 (16 under the terrain rules)"), ECO_EINVAL;
  if (c->hidden != 32 && c->hidden != 64 && c->hidden != 128) return snprintf(msg, n, "hidden must be 32, 64 or 128"), ECO_EINVAL;
  if (c->rules != ECO_RULES_SIMPLE && c->rules != ECO_RULES_PAPER && c->rules != ECO_RULES_TERRAIN)
    return snprintf(msg, n, "bad rules"), ECO_EINVAL;
  if (c->vision != ECO_VISION_CHANNELS && c->vision != ECO_VISION_RGB) return snprintf(msg, n, "bad vision"), ECO_EINVAL;
  if (c->view != ECO_VIEW_AROUND && c->view != ECO_VIEW_FRONT) return snprintf(msg, n, "bad view"), ECO_EINVAL;
  if (c->view == ECO_VIEW_FRONT && !(c->flags & ECO_ROTATE_OBS))
    return snprintf(msg, n, "the front view needs ECO_ROTATE_OBS"), ECO_EINVAL;
  if (c->rules == ECO_RULES_SIMPLE && c->n_actions != 6 && c->n_actions != 9)
    return snprintf(msg, n, "n_actions must be 6 or 9 under the simple rules"), ECO_EINVAL;
  if (c->rules != ECO_RULES_SIMPLE) {
    if (c->n_actions != (terrain ? TA_N : PA_N))
      return snprintf(msg, n, "n_actions must be 7 under the paper rules, 9 under the terrain rules"), ECO_EINVAL;
    if (c->flags & ECO_AUTO_EAT) return snprintf(msg, n, "the paper rules eat only by the eat action"), ECO_EINVAL;
    if (c->hp_max < 1 || c->hp_child < 1 || c->hp_child > c->hp_max || c->attack_damage < 0 ||
        c->heal_rate < 0 || c->heal_cost < 0 || c->age_div < 1 || c->starve_damage < 0 || c->e_act < 0)
      return snprintf(msg, n, "bad HP constants"), ECO_EINVAL;
    if (c->e_food < 1 || c->e_init < 0 || c->e_cap < 1 || c->e_cap < c->e_init || c->e_child < 1 ||
        c->e_child > c->e_repro)
      return snprintf(msg, n, "bad energy constants for the paper rules"), ECO_EINVAL;
  }
  if (c->precision < ECO_FP32 || c->precision > ECO_FP8_E4M3) return snprintf(msg, n, "bad precision"), ECO_EINVAL;
  if (c->e_repro <= 0 || c->attack_den <= 0 || c->attack_num < 0 || c->e_metab < 0)
    return snprintf(msg, n, "bad energy constants"), ECO_EINVAL;
  if (!(c->sigma >= 0.0f) || !std::isfinite(c->sigma)) return snprintf(msg, n, "bad sigma"), ECO_EINVAL;
  if (c->launch_mode < 0 || c->launch_mode > 1) return snprintf(msg, n, "launch_mode must be 0 or 1"), ECO_EINVAL;
  if (c->policy_form != ECO_POLICY_PLAIN && c->policy_form != ECO_POLICY_PAPER)
    return snprintf(msg, n, "bad policy_form"), ECO_EINVAL;
  if (c->policy_form == ECO_POLICY_PAPER && (c->n_hidden < 1 || c->n_hidden > 4))
    return snprintf(msg, n, "n_hidden must be in [1, 4] for the paper form"), ECO_EINVAL;
  if (terrain) {
    if (c->vision != ECO_VISION_RGB) return snprintf(msg, n, "the terrain rules need RGB vision"), ECO_EINVAL;
    if (c->sea_level < 0 || c->sea_level > 1024) return snprintf(msg, n, "sea_level must be in [0, 1024]"), ECO_EINVAL;
    if (c->w_bite < 1 || c->w_cap < 1 || c->b_bite < 1 || c->b_cap < 1 || c->w_init < 0 || c->w_init > c->w_cap ||
        c->b_body < 0 || c->b_body > c->b_cap || c->w_metab < 0 || c->w_child < 0 || c->heal_water < 0 ||
        c->b_child < 0 || c->b_site < 0 || c->photo_q16 < 0 || c->photo_q16 > 65536 || c->res_cap < c->e_food ||
        !(c->biomass_density >= 0.0f && c->biomass_density <= 1.0f))
      return snprintf(msg, n, "bad terrain constants"), ECO_EINVAL;
    if (c->w_child > c->w_cap || c->b_child > c->b_cap)
      return snprintf(msg, n, "a child's water and biomass must fit its capacities"), ECO_EINVAL;
  }
  if (c->policy_variant < -1 || c->policy_variant > policy_variant_count())
    return snprintf(msg, n, "policy_variant out of range"), ECO_EINVAL;
  long long cells = 0, slots = 0;
  for (int e = 0; e < c->n_envs; ++e) {
    const int L = c->env_side[e];
    if (L < 4 || (L & 1) || L > 16384) return snprintf(msg, n, "env %d: side must be even in [4, 16384]", e), ECO_EINVAL;
    if (c->patch_k > L) return snprintf(msg, n, "env %d: patch larger than the grid", e), ECO_EINVAL;
    if (c->env_slots[e] < 1) return snprintf(msg, n, "env %d: slots must be >= 1", e), ECO_EINVAL;
    if (c->env_init_alive[e] < 0 || c->env_init_alive[e] > c->env_slots[e] || c->env_init_alive[e] > L * L)
      return snprintf(msg, n, "env %d: init_alive out of range", e), ECO_EINVAL;
    cells += (long long)L * L;
    slots += c->env_slots[e];
    // terrain: all water of an environment must fit one int32 cell
    if (terrain && (long long)L * L * (c->sea_level + 1) + (long long)c->env_slots[e] * c->w_cap > (1ll << 30))
      return snprintf(msg, n, "env %d: too much water for int32 cells", e), ECO_EINVAL;
  }
  if (cells > (1ll << 30) || slots > (1ll << 28)) return snprintf(msg, n, "too many cells or slots"), ECO_EINVAL;
  return ECO_OK;
}

static Layout make_layout(const eco_config *c) {
  Layout L;
  L.nch = c->rules == ECO_RULES_TERRAIN ? 4 : 3;
  L.D = L.nch * c->patch_k * c->patch_k + c->n_scalars;
  L.H = c->hidden;
  L.A = c->n_actions;
  L.patch = L.nch * c->patch_k * c->patch_k;
  L.n_scalars = c->n_scalars;
  if (c->policy_form == ECO_POLICY_PAPER) {
    L.L = c->n_hidden;
    // sensors: vision (when there is a patch), compass (8+ scalars), internal
    L.ns = (c->patch_k > 0 ? 1 : 0) + (c->n_scalars >= 8 ? 1 : 0) + 1;
    L.relu = 1;
    L.out_bias = 0;
    L.temp = 1;
  } else {
    L.L = 1;
    L.ns = 1;
    L.relu = 0;
    L.out_bias = 1;
    L.temp = 0;
  }
  L.nW = L.D * L.H + L.L * L.H * L.H + L.A * L.H;
  L.nB = L.ns * L.H + L.L * L.H + (L.out_bias ? L.A : 0) + (L.temp ? 1 : 0);
  L.P = L.nW + L.nB;
  const int rows = L.H + L.L * L.H + L.A;  // FP8 row scales
  // FP32 masters: W_in | hidden | W_out | biases (W sections are multiples of 4 floats)
  L.moff_w1 = 0;
  L.moff_w2 = L.D * L.H * 4;
  L.moff_w3 = L.moff_w2 + L.L * L.H * L.H * 4;
  L.moff_bias = L.nW * 4;
  L.mstride = pad((int64_t)L.P * 4, 128);
  L.es = c->precision == ECO_FP32 ? 4 : (c->precision == ECO_BF16 ? 2 : 1);
  L.off_w1 = 0;
  L.off_w2 = L.D * L.H * L.es;
  L.off_w3 = L.off_w2 + L.L * L.H * L.H * L.es;
  const int wend = L.off_w3 + L.A * L.H * L.es;
  L.off_scale = wend;
  L.off_bias = (c->precision == ECO_FP8_E4M3) ? (int)(wend + pad(rows * 4, 16)) : wend;
  L.stride = (c->precision == ECO_FP32) ? L.mstride : pad(L.off_bias + pad(L.nB * 4, 16), 128);
  return L;
}

// Workspace carving (256-byte aligned regions).
struct Carve {
  size_t off = 0;
  uint8_t *base = nullptr;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

static size_t carve(const eco_config *c, const Layout &L, uint8_t *base, Dev *d, EnvDesc **env_dev) {
  Carve k;
  k.base = base;
  long long cells = 0, slots = 0;
  for (int e = 0; e < c->n_envs; ++e) {
    cells += (long long)c->env_side[e] * c->env_side[e];
    slots += c->env_slots[e];
  }
  const int E = c->n_envs;
  Dev &D = *d;
  memset(&D, 0, sizeof(D));
  D.n_envs = E;
  D.total_cells = (int)cells;
  D.total_slots = (int)slots;
  // weights first: the big arrays start at the workspace base
  D.master = k.take<float>((size_t)slots * (L.mstride / 4));
  if (c->precision == ECO_FP32)
    D.wq = reinterpret_cast<uint8_t *>(D.master);
  else
    D.wq = k.take<uint8_t>((size_t)slots * L.stride);
  const size_t wq_end = k.off;
  *env_dev = k.take<EnvDesc>(E);
  D.env = *env_dev;
  D.cellf = k.take<uint8_t>(cells);
  D.occ = k.take<int32_t>(cells);
  D.claim_move = k.take<unsigned long long>(cells);
  D.cnt_move = k.take<uint32_t>(cells);
  D.claim_birth = k.take<unsigned long long>(cells);
  D.att_cell = k.take<unsigned long long>(cells);
  D.alive = k.take<uint8_t>(slots);
  D.pos = k.take<int32_t>(slots);
  D.facing = k.take<uint8_t>(slots);
  D.energy = k.take<int32_t>(slots);
  D.parent = k.take<int32_t>(slots);
  D.birth = k.take<int32_t>(slots);
  D.act = k.take<uint8_t>(slots);
  D.env_of = k.take<uint16_t>(slots);
  D.tgt = k.take<int32_t>(slots);
  D.gain = k.take<int32_t>(slots);
  D.logits = k.take<float>((size_t)slots * L.A);
  D.alive_list = k.take<int32_t>(slots);
  D.tile_counts = k.take<int32_t>(2 * compact_tiles((int)slots));
  D.barrier = k.take<unsigned>(BAR_N);
  D.births = k.take<int2>(slots);
  D.free_list = k.take<int32_t>(std::max((long long)slots, (long long)compact_tiles((int)slots) * 256));
  D.free_tiles = k.take<int32_t>(compact_tiles((int)slots));
  D.bflag = k.take<uint8_t>(slots);
  D.birth_contenders = k.take<int32_t>(E);
  D.contenders = k.take<int32_t>(slots);
  D.bcell = k.take<int32_t>(slots);
  D.stats_step = k.take<long long>((size_t)E * N_ST);
  D.stats_total = k.take<long long>((size_t)E * N_ST);
  D.stats_last = k.take<long long>((size_t)E * N_ST);
  // the counters (with the status word) follow the statistics, so that one
  // copy brings both to the host
  D.counters = k.take<int32_t>(CNT_N);
  D.step = k.take<long long>(1);
  D.alive_at_step = k.take<int32_t>(kAliveRing);
  D.hist = k.take<uint32_t>((size_t)E * 65536);
  D.place_prefix = k.take<unsigned long long>(E);
  D.place_remaining = k.take<int32_t>(E);
  D.hp = k.take<int32_t>(slots);
  D.age = k.take<int32_t>(slots);
  D.res = k.take<int32_t>(cells);
  D.colour = k.take<float4>(slots);
  D.rock = k.take<int32_t>(cells);
  D.water = k.take<int32_t>(cells);
  D.bio = k.take<int32_t>(cells);
  D.photo = k.take<uint32_t>(cells);
  D.flow = k.take<uint32_t>(cells);
  D.a_water = k.take<int32_t>(slots);
  D.a_bio = k.take<int32_t>(slots);
  D.trace = k.take<unsigned long long>((size_t)kTraceSteps * kTraceWords);
  // The policy kernel's FP8 tail batches load up to kStreamSlack bytes past
  // the last weight block (their products are skipped): the regions after
  // the weights (the histogram alone is 256 KB per world) keep those loads
  // inside the workspace, and this keeps that true for any layout.
  if (k.off < wq_end + kStreamSlack) k.take<uint8_t>(wq_end + kStreamSlack - k.off);
  return (k.off + 255) & ~(size_t)255;
}

extern "C" int eco_param_count(const eco_config *cfg, int32_t *n_params, int32_t *obs_dim) {
  char msg[256];
  int rc = validate(cfg, msg, sizeof msg);
  if (rc) return fail(nullptr, rc, "%s", msg);
  Layout L = make_layout(cfg);
  if (n_params) *n_params = L.P;
  if (obs_dim) *obs_dim = L.D;
  return ECO_OK;
}

extern "C" int eco_workspace_bytes(const eco_config *cfg, size_t *bytes) {
  char msg[256];
  int rc = validate(cfg, msg, sizeof msg);
  if (rc) return fail(nullptr, rc, "%s", msg);
  if (!bytes) return fail(nullptr, ECO_EINVAL, "null bytes");
  Layout L = make_layout(cfg);
  Dev d;
  EnvDesc *ed;
  *bytes = carve(cfg, L, nullptr, &d, &ed);
  return ECO_OK;
}

enum { GRAPH_TIMED = 0, GRAPH_ONE = 1, GRAPH_MANY = 2, GRAPH_READ1 = 3, GRAPH_READ2 = 4, GRAPH_TIMED_MANY = 5 };
constexpr int kNumGraphs = 6;
constexpr int kStepsPerGraph = 8;

static void destroy_graph(eco_handle *h) {
  for (int k = 0; k < kNumGraphs; ++k) {
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    if (h->graph_src[k]) cudaGraphDestroy(h->graph_src[k]);
    h->graph[k] = nullptr;
    h->graph_src[k] = nullptr;
  }
}

extern "C" int eco_create(const eco_config *cfg, void *dev_workspace, size_t bytes, void *stream,
                          eco_handle **out) {
  if (!out) return fail(nullptr, ECO_EINVAL, "null out");
  *out = nullptr;
  char msg[256];
  int rc = validate(cfg, msg, sizeof msg);
  if (rc) return fail(nullptr, rc, "%s", msg);
  size_t need = 0;
  eco_workspace_bytes(cfg, &need);
  if (!dev_workspace || bytes < need) return fail(nullptr, ECO_ENOMEM, "workspace of %zu bytes < %zu needed", bytes, need);
  if ((reinterpret_cast<uintptr_t>(dev_workspace) & 255) != 0) return fail(nullptr, ECO_EINVAL, "workspace not 256-byte aligned");

  eco_handle *h = new eco_handle();
  h->n_envs = cfg->n_envs;
  h->side.assign(cfg->env_side, cfg->env_side + cfg->n_envs);
  h->slots.assign(cfg->env_slots, cfg->env_slots + cfg->n_envs);
  h->init_alive.assign(cfg->env_init_alive, cfg->env_init_alive + cfg->n_envs);
  h->seed.assign(cfg->env_seed, cfg->env_seed + cfg->n_envs);
  h->L = make_layout(cfg);
  Rules &R = h->R;
  R.patch_k = cfg->patch_k;
  R.n_scalars = cfg->n_scalars;
  R.flags = cfg->flags;
  R.precision = cfg->precision;
  R.sigma = cfg->sigma;
  R.thr_food = threshold_of(cfg->food_density);
  R.thr_regrow = threshold_of(cfg->regrow_p);
  R.thr_wall = threshold_of(cfg->wall_density);
  R.e_init = cfg->e_init;
  R.e_metab = cfg->e_metab;
  R.e_food = cfg->e_food;
  R.e_repro = cfg->e_repro;
  R.attack_num = cfg->attack_num;
  R.attack_den = cfg->attack_den;
  R.rules = cfg->rules;
  R.hp_max = cfg->hp_max;
  R.hp_child = cfg->hp_child;
  R.attack_damage = cfg->attack_damage;
  R.heal_rate = cfg->heal_rate;
  R.heal_cost = cfg->heal_cost;
  R.age_div = cfg->age_div;
  R.starve_damage = cfg->starve_damage;
  R.e_act = cfg->e_act;
  R.e_cap = cfg->e_cap;
  R.e_child = cfg->e_child;
  R.vision = cfg->vision;
  R.view = cfg->view;
  R.sea_level = cfg->sea_level;
  R.w_init = cfg->w_init;
  R.w_metab = cfg->w_metab;
  R.w_bite = cfg->w_bite;
  R.w_cap = cfg->w_cap;
  R.w_child = cfg->w_child;
  R.heal_water = cfg->heal_water;
  R.b_body = cfg->b_body;
  R.b_child = cfg->b_child;
  R.b_bite = cfg->b_bite;
  R.b_cap = cfg->b_cap;
  R.b_site = cfg->b_site;
  R.thr_bio = threshold_of(cfg->biomass_density);
  R.photo_q16 = cfg->photo_q16;
  R.res_cap = cfg->res_cap;
  h->ws = reinterpret_cast<uint8_t *>(dev_workspace);
  h->ws_bytes = bytes;
  carve(cfg, h->L, h->ws, &h->d, &h->env_dev);
  int so = 0, co = 0;
  for (int e = 0; e < cfg->n_envs; ++e) {
    EnvDesc ed;
    ed.side = cfg->env_side[e];
    ed.slot_off = so;
    ed.n_slots = cfg->env_slots[e];
    ed.cell_off = co;
    ed.init_alive = cfg->env_init_alive[e];
    ed.seed = cfg->env_seed[e];
    h->env_host.push_back(ed);
    so += ed.n_slots;
    co += ed.side * ed.side;
  }
  h->own_stream = (stream == nullptr);
  if (h->own_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, ECO_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
  } else {
    h->stream = reinterpret_cast<cudaStream_t>(stream);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->grid.sms, cudaDevAttrMultiProcessorCount, dev);
  h->grid.slot_blocks = grid_for(h->d.total_slots, 256, h->grid.sms * 8);
  h->grid.cell_blocks = grid_for(h->d.total_cells / 4, 256, h->grid.sms * 8);
  h->grid.birth_blocks = h->grid.sms * 2;
  h->grid.persistent_blocks = 0;
  h->grid.use_persistent = cfg->launch_mode == 0;
  h->forced = cfg->policy_variant;
  h->variant = 0;
  for (int k = 0; k < kNumGraphs; ++k) {
    h->graph[k] = nullptr;
    h->graph_src[k] = nullptr;
  }
  h->ev_used = 0;
  h->steps_done = 0;
  h->rd_pending = 0;
  h->rd_ev[0] = h->rd_ev[1] = nullptr;
  h->err[0] = 0;
  h->rd_bytes = (size_t)(reinterpret_cast<uint8_t *>(h->d.counters + CNT_N) -
                         reinterpret_cast<uint8_t *>(h->d.stats_total));
  h->rd_host = nullptr;
  // zero the whole workspace first, then install the environment table
  cudaError_t e = cudaMemsetAsync(h->ws, 0, need, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->env_dev, h->env_host.data(), sizeof(EnvDesc) * h->n_envs,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_init_static(h->d, h->grid, h->stream);
  if (e == cudaSuccess) e = env_prepare(h->L, &h->grid);
  if (e == cudaSuccess && h->grid.persistent_blocks > 0) {
    // a batch of at most 4,096 slots and 16,384 cells runs the persistent
    // form on one CTA (at most four slots or cell groups per thread), whose
    // phases need no grid barrier; anything larger keeps one CTA per SM
    // (fewer CTAs only made the barriers' waits longer)
    const long long work = std::max((long long)h->d.total_slots, (long long)h->d.total_cells / 4);
    if (work <= 4096) h->grid.persistent_blocks = 1;
  }
  if (e == cudaSuccess) e = cudaMallocHost(&h->rd_host, 3 * h->rd_bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rd_ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rd_ev[1], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev_dummy[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev_dummy[1]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    int r = fail(nullptr, ECO_ECUDA, "create: %s", cudaGetErrorString(e));
    if (h->rd_host) cudaFreeHost(h->rd_host);
    for (cudaEvent_t ev : h->rd_ev)
      if (ev) cudaEventDestroy(ev);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return r;
  }
  if (h->forced > 0) {
    e = policy_prepare(h->L, h->R, h->forced, &h->pl);
    if (e != cudaSuccess) {
      int r = fail(nullptr, ECO_ECUDA, "policy variant %d: %s", h->forced, cudaGetErrorString(e));
      eco_destroy(h);
      return r;
    }
    h->variant = h->forced;
  }
  *out = h;
  return ECO_OK;
}

extern "C" void eco_destroy(eco_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_graph(h);
  for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
  if (h->ev_dummy[0]) cudaEventDestroy(h->ev_dummy[0]);
  if (h->ev_dummy[1]) cudaEventDestroy(h->ev_dummy[1]);
  if (h->rd_host) cudaFreeHost(h->rd_host);
  for (cudaEvent_t ev : h->rd_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" const char *eco_last_error(const eco_handle *h) { return h ? h->err : g_err; }

static int check_status(eco_handle *h) {
  int32_t st = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&st, h->d.counters + CNT_STATUS, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (st & 3) return fail(h, ECO_EINVAL, "reset: fewer non-wall cells than founders (status %d)", st);
  if (st & 4) return fail(h, ECO_ETIMEOUT, "a device-side wait ran out of its budget");
  return ECO_OK;
}

extern "C" int eco_reset(eco_handle *h) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  // also clears the status word, the persistent form's barrier and its
  // failure-detection test words
  CUDA_TRY(h, cudaMemsetAsync(h->d.barrier, 0, BAR_N * sizeof(unsigned), h->stream));
  CUDA_TRY(h, launch_reset(h->d, h->L, h->R, h->grid, h->stream));
  CUDA_TRY(h, launch_compact(h->d, h->stream));
  h->rd_pending = 0;  // eco_step_read starts over from the reset records
  h->steps_done = 0;
  return check_status(h);
}

extern "C" int eco_reset_seed(eco_handle *h, uint64_t seed) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  for (int e = 0; e < h->n_envs; ++e) {
    const uint32_t se = (uint32_t)(seed + (uint64_t)e);
    h->seed[e] = se;
    h->env_host[e].seed = se;
  }
  // the step graphs read the environment table from device memory, so the
  // new seeds reach them without a re-capture
  CUDA_TRY(h, cudaMemcpyAsync(h->env_dev, h->env_host.data(), sizeof(EnvDesc) * h->n_envs,
                              cudaMemcpyHostToDevice, h->stream));
  return eco_reset(h);
}

// Choose the fastest policy variant on the current state (autotuner).
static int autotune(eco_handle *h) {
  if (h->variant) return ECO_OK;
  CUDA_TRY(h, launch_compact(h->d, h->stream));
  // candidates of the requested family
  const bool sparse = h->forced < 0;
  std::vector<int> ids;
  std::vector<PolicyLaunch> pls;
  for (int v = 1; v <= policy_variant_count(); ++v) {
    if (policy_variant_sparse(v) != sparse) continue;
    PolicyLaunch pl;
    if (policy_prepare(h->L, h->R, v, &pl) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    ids.push_back(v);
    pls.push_back(pl);
  }
  if (ids.empty()) return fail(h, ECO_ECUDA, "no policy variant could be prepared");
  // policy-only launches (no state changes) on the current state: one
  // warm-up each, then kRounds rounds that time kPerRound launches of every
  // candidate in turn, so that a drift in clocks or memory state over the
  // tuning affects every candidate alike; the lowest total wins
  constexpr int kRounds = 5, kPerRound = 3;
  struct EventPair {  // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CUDA_TRY(h, cudaEventCreate(&ev.a));
  CUDA_TRY(h, cudaEventCreate(&ev.b));
  cudaEvent_t a = ev.a, b = ev.b;
  for (const PolicyLaunch &pl : pls) CUDA_TRY(h, policy_launch(pl, h->d, h->L, h->R, h->stream, false));
  std::vector<double> total(ids.size(), 0.0);
  for (int r = 0; r < kRounds; ++r) {
    for (size_t c = 0; c < ids.size(); ++c) {
      CUDA_TRY(h, cudaEventRecord(a, h->stream));
      for (int k = 0; k < kPerRound; ++k) CUDA_TRY(h, policy_launch(pls[c], h->d, h->L, h->R, h->stream, false));
      CUDA_TRY(h, cudaEventRecord(b, h->stream));
      CUDA_TRY(h, cudaEventSynchronize(b));
      float ms = 0;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, a, b));
      total[c] += ms;
    }
  }
  size_t best = 0;
  for (size_t c = 1; c < ids.size(); ++c)
    if (total[c] < total[best]) best = c;
  h->variant = ids[best];
  h->pl = pls[best];
  return ECO_OK;
}

// One step: the alive list was built by the previous step (or by reset /
// write_state), so the step is the policy kernel and the environment
// phases, which end by building the next step's alive list.  timed: an
// event-record node on each side of the policy kernel.
static cudaError_t enqueue_step(eco_handle *h, bool timed) {
  cudaError_t e = cudaSuccess;
  // "external" records become event-record nodes of the captured graph
  if (timed) e = cudaEventRecordWithFlags(h->ev_dummy[0], h->stream, cudaEventRecordExternal);
  if (e == cudaSuccess) e = policy_launch(h->pl, h->d, h->L, h->R, h->stream, true);
  if (e == cudaSuccess && timed)
    e = cudaEventRecordWithFlags(h->ev_dummy[1], h->stream, cudaEventRecordExternal);
  if (e == cudaSuccess) e = launch_env_phases(h->d, h->L, h->R, h->grid, h->stream);
  return e;
}

static int build_graph(eco_handle *h, int kind) {
  if (h->graph[kind]) return ECO_OK;
  int rc = autotune(h);
  if (rc) return rc;
  const bool timed = kind == GRAPH_TIMED || kind == GRAPH_TIMED_MANY;
  const int steps = (kind == GRAPH_MANY || kind == GRAPH_TIMED_MANY) ? kStepsPerGraph : 1;
  const int copy_slot = kind == GRAPH_READ1 ? 1 : (kind == GRAPH_READ2 ? 2 : 0);
  cudaGraph_t g = nullptr;
  for (;;) {
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = enqueue_step(h, timed && k == 0);
    if (e == cudaSuccess && copy_slot)
      e = cudaMemcpyAsync(h->rd_host + copy_slot * h->rd_bytes, h->d.stats_total, h->rd_bytes,
                          cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) break;
    if (e2 == cudaSuccess && g) cudaGraphDestroy(g);
    g = nullptr;
    cudaGetLastError();
    if (h->grid.use_persistent && h->grid.persistent_blocks > 0) {
      // the persistent form could not be captured: fall back to one
      // kernel per phase (identical results) in every graph
      h->grid.use_persistent = 0;
      CUDA_TRY(h, cudaStreamSynchronize(h->stream));
      destroy_graph(h);
      continue;
    }
    if (e != cudaSuccess) return fail(h, ECO_ECUDA, "capture: %s", cudaGetErrorString(e));
    return fail(h, ECO_ECUDA, "end capture: %s", cudaGetErrorString(e2));
  }
  if (timed) {
    // locate the two event-record nodes
    size_t n = 0;
    CUDA_TRY(h, cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CUDA_TRY(h, cudaGraphGetNodes(g, nodes.data(), &n));
    int found = 0;
    for (size_t i = 0; i < n; ++i) {
      cudaGraphNodeType t;
      CUDA_TRY(h, cudaGraphNodeGetType(nodes[i], &t));
      if (t == cudaGraphNodeTypeEventRecord) {
        cudaEvent_t ev;
        CUDA_TRY(h, cudaGraphEventRecordNodeGetEvent(nodes[i], &ev));
        if (ev == h->ev_dummy[0]) h->ev_node[kind][0] = nodes[i], ++found;
        if (ev == h->ev_dummy[1]) h->ev_node[kind][1] = nodes[i], ++found;
      }
    }
    if (found != 2) {
      cudaGraphDestroy(g);
      return fail(h, ECO_ECUDA, "step graph: event nodes not found");
    }
  }
  cudaError_t ie = cudaGraphInstantiate(&h->graph[kind], g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    h->graph[kind] = nullptr;
    return fail(h, ECO_ECUDA, "instantiate: %s", cudaGetErrorString(ie));
  }
  h->graph_src[kind] = g;
  return ECO_OK;
}

static int step_impl(eco_handle *h, int32_t n_steps, bool timed) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  if (n_steps < 0) return fail(h, ECO_EINVAL, "n_steps < 0");
  if (n_steps == 0) return ECO_OK;
  const int many = n_steps / kStepsPerGraph, rest = n_steps % kStepsPerGraph;
  if (!timed) {
    int rc = many ? build_graph(h, GRAPH_MANY) : ECO_OK;
    if (rc == ECO_OK && rest) rc = build_graph(h, GRAPH_ONE);
    if (rc) return rc;
    for (int i = 0; i < many; ++i) CUDA_TRY(h, cudaGraphLaunch(h->graph[GRAPH_MANY], h->stream));
    for (int i = 0; i < rest; ++i) CUDA_TRY(h, cudaGraphLaunch(h->graph[GRAPH_ONE], h->stream));
    h->steps_done += n_steps;
    return ECO_OK;
  }
  // one timed launch per graph of kStepsPerGraph steps (the first step's
  // policy kernel), the remaining steps untimed; fewer steps than a graph:
  // every step timed, in one-step graphs
  const int kind = many ? GRAPH_TIMED_MANY : GRAPH_TIMED;
  const int launches = many ? many : rest;
  const int per = many ? kStepsPerGraph : 1;
  int rc = build_graph(h, kind);
  if (rc == ECO_OK && many && rest) rc = build_graph(h, GRAPH_ONE);
  if (rc) return rc;
  cudaGraphExec_t gx = h->graph[kind];
  if (h->ev_used + launches > 4096) return fail(h, ECO_EINVAL, "more than 4096 timed launches buffered");
  while ((int)h->ev_pool.size() < 2 * (h->ev_used + launches)) {
    cudaEvent_t ev;
    CUDA_TRY(h, cudaEventCreate(&ev));
    h->ev_pool.push_back(ev);
  }
  for (int i = 0; i < launches; ++i) {
    CUDA_TRY(h, cudaGraphExecEventRecordNodeSetEvent(gx, h->ev_node[kind][0], h->ev_pool[2 * h->ev_used]));
    CUDA_TRY(h, cudaGraphExecEventRecordNodeSetEvent(gx, h->ev_node[kind][1], h->ev_pool[2 * h->ev_used + 1]));
    ++h->ev_used;
    h->timed_steps.push_back(h->steps_done);
    CUDA_TRY(h, cudaGraphLaunch(gx, h->stream));
    h->steps_done += per;
  }
  CUDA_TRY(h, cudaGraphExecEventRecordNodeSetEvent(gx, h->ev_node[kind][0], h->ev_dummy[0]));
  CUDA_TRY(h, cudaGraphExecEventRecordNodeSetEvent(gx, h->ev_node[kind][1], h->ev_dummy[1]));
  if (many && rest) {
    for (int i = 0; i < rest; ++i) CUDA_TRY(h, cudaGraphLaunch(h->graph[GRAPH_ONE], h->stream));
    h->steps_done += rest;
  }
  return ECO_OK;
}

extern "C" int eco_step(eco_handle *h, int32_t n_steps) { return step_impl(h, n_steps, false); }

extern "C" int eco_prepare(eco_handle *h) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  int rc = build_graph(h, GRAPH_ONE);
  if (rc == ECO_OK) rc = build_graph(h, GRAPH_MANY);
  if (rc == ECO_OK) rc = build_graph(h, GRAPH_TIMED);
  if (rc == ECO_OK) rc = build_graph(h, GRAPH_TIMED_MANY);
  if (rc == ECO_OK) rc = build_graph(h, GRAPH_READ1);
  if (rc == ECO_OK) rc = build_graph(h, GRAPH_READ2);
  if (rc == ECO_OK) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return rc;
}
extern "C" int eco_step_timed(eco_handle *h, int32_t n_steps) { return step_impl(h, n_steps, true); }

extern "C" int eco_policy_timing(eco_handle *h, double *total_ms, int32_t *n_timed, int64_t *agents) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  double tot = 0;
  for (int i = 0; i < h->ev_used; ++i) {
    float ms = 0;
    CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
    tot += ms;
  }
  if (agents) {
    // the agent counts the policy kernel wrote at the timed steps
    std::vector<int32_t> ring(kAliveRing);
    CUDA_TRY(h, cudaMemcpy(ring.data(), h->d.alive_at_step, sizeof(int32_t) * kAliveRing, cudaMemcpyDeviceToHost));
    long long a = 0;
    for (long long t : h->timed_steps) a += ring[(size_t)(t & (kAliveRing - 1))];
    *agents = a;
  }
  if (total_ms) *total_ms = tot;
  if (n_timed) *n_timed = h->ev_used;
  h->ev_used = 0;
  h->timed_steps.clear();
  return ECO_OK;
}

extern "C" int eco_policy_only(eco_handle *h, int32_t n_iters) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  int rc = autotune(h);
  if (rc) return rc;
  CUDA_TRY(h, launch_compact(h->d, h->stream));
  for (int i = 0; i < n_iters; ++i) CUDA_TRY(h, policy_launch(h->pl, h->d, h->L, h->R, h->stream, false));
  return ECO_OK;
}

extern "C" int eco_arm_barrier_timeout(eco_handle *h, int32_t absent_cta, int32_t poll_budget) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  const bool pers = h->grid.use_persistent && h->grid.persistent_blocks > 1;
  if (!pers) return fail(h, ECO_EINVAL, "the persistent launch form with more than one CTA is not in use");
  if (absent_cta < 0 || absent_cta >= h->grid.persistent_blocks) return fail(h, ECO_EINVAL, "absent_cta out of range");
  if (poll_budget < 1) return fail(h, ECO_EINVAL, "poll_budget must be >= 1");
  const unsigned words[2] = {(unsigned)absent_cta + 1u, (unsigned)poll_budget};
  CUDA_TRY(h, cudaMemcpyAsync(h->d.barrier + BAR_ABSENT_CTA, words, sizeof words, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}

extern "C" int eco_trace_phases(eco_handle *h, int32_t on) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  const bool pers = h->grid.use_persistent && h->grid.persistent_blocks > 0;
  if (!pers) return fail(h, ECO_EINVAL, "the phase trace needs the persistent launch form");
  const unsigned word = on ? 1u : 0u;
  CUDA_TRY(h, cudaMemsetAsync(h->d.trace, 0, sizeof(unsigned long long) * kTraceSteps * kTraceWords, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d.barrier + BAR_TRACE, &word, sizeof word, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}

extern "C" int eco_read_phase_trace(eco_handle *h, uint64_t *rows, int32_t max_rows, int32_t *n_rows) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  if (!rows || max_rows < 0) return fail(h, ECO_EINVAL, "null rows or negative max_rows");
  const int n = max_rows < kTraceSteps ? max_rows : kTraceSteps;
  CUDA_TRY(h, cudaMemcpyAsync(rows, h->d.trace, sizeof(uint64_t) * kTraceWords * (size_t)n, cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (n_rows) *n_rows = n;
  return ECO_OK;
}

extern "C" int eco_policy_variants(const eco_handle *h, int32_t *count, int32_t *chosen) {
  if (count) *count = policy_variant_count();
  if (chosen) *chosen = h ? h->variant : 0;
  return ECO_OK;
}

extern "C" const char *eco_policy_variant_name(int32_t k) { return policy_variant_name(k); }

extern "C" int eco_launch_mode(const eco_handle *h, int32_t *mode, int32_t *blocks) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  const bool pers = h->grid.use_persistent && h->grid.persistent_blocks > 0;
  if (mode) *mode = pers ? 0 : 1;
  if (blocks) *blocks = pers ? h->grid.persistent_blocks : 0;
  return ECO_OK;
}

extern "C" int eco_policy_bytes(eco_handle *h, int64_t *bytes, int64_t *n_alive) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  int32_t n = 0;
  CUDA_TRY(h, launch_compact(h->d, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&n, h->d.counters + CNT_N_ALIVE, sizeof n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  const Layout &L = h->L;
  int64_t per = (int64_t)L.nW * L.es + (int64_t)L.nB * 4;
  if (h->R.precision == ECO_FP8_E4M3) per += (int64_t)(L.H + L.L * L.H + L.A) * 4;  // row scales
  if (bytes) *bytes = per * n;
  if (n_alive) *n_alive = n;
  return ECO_OK;
}

// Records of the pinned mirror slot `slot` to the caller's buffers, and the
// status word's verdict.
static int stats_from_mirror(eco_handle *h, int slot, eco_stats *total, eco_stats *last, int32_t n_envs) {
  const uint8_t *base = reinterpret_cast<const uint8_t *>(h->d.stats_total);
  const uint8_t *m = h->rd_host + (size_t)slot * h->rd_bytes;
  auto mirror = [&](const void *dev) { return m + (reinterpret_cast<const uint8_t *>(dev) - base); };
  if (total) memcpy(total, mirror(h->d.stats_total), sizeof(eco_stats) * n_envs);
  if (last) memcpy(last, mirror(h->d.stats_last), sizeof(eco_stats) * n_envs);
  int32_t st = 0;
  memcpy(&st, mirror(h->d.counters + CNT_STATUS), sizeof st);
  if (st & 3) return fail(h, ECO_EINVAL, "reset: fewer non-wall cells than founders (status %d)", st);
  if (st & 4) return fail(h, ECO_ETIMEOUT, "a device-side wait ran out of its budget");
  return ECO_OK;
}

extern "C" int eco_read_stats(eco_handle *h, eco_stats *total, eco_stats *last, int32_t n_envs) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  if (n_envs < 0 || n_envs > h->n_envs) return fail(h, ECO_EINVAL, "n_envs out of range");
  // one asynchronous copy of the statistics and the status word into pinned
  // memory, one synchronisation, then host-side copies
  CUDA_TRY(h, cudaMemcpyAsync(h->rd_host, h->d.stats_total, h->rd_bytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return stats_from_mirror(h, 0, total, last, n_envs);
}

extern "C" int eco_step_read(eco_handle *h, eco_stats *total, eco_stats *last, int32_t n_envs) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  if (n_envs < 0 || n_envs > h->n_envs) return fail(h, ECO_EINVAL, "n_envs out of range");
  int prev = h->rd_pending;
  if (prev == 0) {
    // nothing in flight: the records as they stand now go to slot 2
    CUDA_TRY(h, cudaMemcpyAsync(h->rd_host + 2 * h->rd_bytes, h->d.stats_total, h->rd_bytes,
                                cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaEventRecord(h->rd_ev[1], h->stream));
    prev = 2;
  }
  const int slot = prev == 1 ? 2 : 1;
  int rc = build_graph(h, slot == 1 ? GRAPH_READ1 : GRAPH_READ2);
  if (rc) return rc;
  CUDA_TRY(h, cudaGraphLaunch(h->graph[slot == 1 ? GRAPH_READ1 : GRAPH_READ2], h->stream));
  h->steps_done += 1;
  CUDA_TRY(h, cudaEventRecord(h->rd_ev[slot - 1], h->stream));
  h->rd_pending = slot;
  // the step just enqueued runs while the host waits for the previous copy
  CUDA_TRY(h, cudaEventSynchronize(h->rd_ev[prev - 1]));
  return stats_from_mirror(h, prev, total, last, n_envs);
}

// ---------------------------------------------------------------------------
// State and parameter I/O (host-side marshalling between the library's
// layout and the plain views of the header).
// ---------------------------------------------------------------------------

static int check_env(eco_handle *h, int32_t env) {
  if (!h) return fail(nullptr, ECO_EINVAL, "null handle");
  if (env < 0 || env >= h->n_envs) return fail(h, ECO_EINVAL, "env %d out of range", env);
  return ECO_OK;
}

extern "C" int eco_read_state(eco_handle *h, int32_t env, eco_state_view *out) {
  int rc = check_env(h, env);
  if (rc) return rc;
  if (!out) return fail(h, ECO_EINVAL, "null view");
  const EnvDesc &ed = h->env_host[env];
  const int N = ed.side * ed.side, S = ed.n_slots;
  std::vector<uint8_t> cellf(N), alive(S), facing(S);
  std::vector<int32_t> occ(N), pos(S), energy(S), parent(S), birth(S);
  long long step = 0;
  cudaStream_t s = h->stream;
  if (out->hp) CUDA_TRY(h, cudaMemcpyAsync(out->hp, h->d.hp + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  if (out->age) CUDA_TRY(h, cudaMemcpyAsync(out->age, h->d.age + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  if (out->res) CUDA_TRY(h, cudaMemcpyAsync(out->res, h->d.res + ed.cell_off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
  if (out->water) CUDA_TRY(h, cudaMemcpyAsync(out->water, h->d.water + ed.cell_off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
  if (out->bio) CUDA_TRY(h, cudaMemcpyAsync(out->bio, h->d.bio + ed.cell_off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
  if (out->photo) CUDA_TRY(h, cudaMemcpyAsync(out->photo, h->d.photo + ed.cell_off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
  if (out->a_water) CUDA_TRY(h, cudaMemcpyAsync(out->a_water, h->d.a_water + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  if (out->a_bio) CUDA_TRY(h, cudaMemcpyAsync(out->a_bio, h->d.a_bio + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  std::vector<float4> colour(out->colour ? S : 0);
  if (out->colour)
    CUDA_TRY(h, cudaMemcpyAsync(colour.data(), h->d.colour + ed.slot_off, sizeof(float4) * (size_t)S,
                                cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(cellf.data(), h->d.cellf + ed.cell_off, N, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(occ.data(), h->d.occ + ed.cell_off, 4 * (size_t)N, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(alive.data(), h->d.alive + ed.slot_off, S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(facing.data(), h->d.facing + ed.slot_off, S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(pos.data(), h->d.pos + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(energy.data(), h->d.energy + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(parent.data(), h->d.parent + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(birth.data(), h->d.birth + ed.slot_off, 4 * (size_t)S, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaMemcpyAsync(&step, h->d.step, sizeof step, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  for (int c = 0; c < N; ++c) {
    if (out->food) out->food[c] = (cellf[c] & CELL_FOOD) ? 1 : 0;
    if (out->wall) out->wall[c] = (cellf[c] & CELL_WALL) ? 1 : 0;
    if (out->occ) out->occ[c] = occ[c] < 0 ? -1 : occ[c] - ed.slot_off;
  }
  for (int i = 0; i < S; ++i) {
    if (out->alive) out->alive[i] = alive[i];
    if (out->x) out->x[i] = pos[i] % ed.side;
    if (out->y) out->y[i] = pos[i] / ed.side;
    if (out->facing) out->facing[i] = facing[i];
    if (out->energy) out->energy[i] = energy[i];
    if (out->parent) out->parent[i] = parent[i];
    if (out->birth_step) out->birth_step[i] = birth[i];
    if (out->colour) {
      out->colour[3 * i + 0] = colour[i].x;
      out->colour[3 * i + 1] = colour[i].y;
      out->colour[3 * i + 2] = colour[i].z;
    }
  }
  if (out->step) *out->step = step;
  return ECO_OK;
}

extern "C" int eco_write_state(eco_handle *h, int32_t env, const eco_state_view *in) {
  int rc = check_env(h, env);
  if (rc) return rc;
  if (!in) return fail(h, ECO_EINVAL, "null view");
  const EnvDesc &ed = h->env_host[env];
  const int N = ed.side * ed.side, S = ed.n_slots;
  cudaStream_t s = h->stream;
  const bool cells = in->food || in->wall || in->occ;
  if (cells && !(in->food && in->wall && in->occ)) return fail(h, ECO_EINVAL, "food, wall and occ must be written together");
  const bool where = in->alive || in->x || in->y;
  if (where && !(in->alive && in->x && in->y)) return fail(h, ECO_EINVAL, "alive, x and y must be written together");
  const bool paper = h->R.rules != RULES_SIMPLE;
  if (paper && (cells || in->res) && !(cells && in->res))
    return fail(h, ECO_EINVAL, "under the paper rules res is written together with food, wall and occ");
  std::vector<uint8_t> cellf, alive;
  std::vector<int32_t> occ, pos;
  if (cells) {
    cellf.resize(N);
    occ.resize(N);
    for (int c = 0; c < N; ++c) {
      if (in->occ[c] < -1 || in->occ[c] >= S) return fail(h, ECO_EINVAL, "occ[%d] out of range", c);
      if (paper && in->res[c] < 0) return fail(h, ECO_EINVAL, "res[%d] negative", c);
      const bool food = paper ? in->res[c] > 0 : in->food[c] != 0;
      cellf[c] = (uint8_t)((food ? CELL_FOOD : 0) | (in->wall[c] ? CELL_WALL : 0) | (in->occ[c] >= 0 ? CELL_AGENT : 0));
      occ[c] = in->occ[c] < 0 ? -1 : in->occ[c] + ed.slot_off;
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->d.cellf + ed.cell_off, cellf.data(), N, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d.occ + ed.cell_off, occ.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, s));
    if (paper) CUDA_TRY(h, cudaMemcpyAsync(h->d.res + ed.cell_off, in->res, 4 * (size_t)N, cudaMemcpyHostToDevice, s));
  }
  if (where) {
    alive.assign(in->alive, in->alive + S);
    pos.resize(S);
    for (int i = 0; i < S; ++i) {
      if (in->x[i] < 0 || in->x[i] >= ed.side || in->y[i] < 0 || in->y[i] >= ed.side)
        return fail(h, ECO_EINVAL, "slot %d position out of range", i);
      pos[i] = in->y[i] * ed.side + in->x[i];
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->d.alive + ed.slot_off, alive.data(), S, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d.pos + ed.slot_off, pos.data(), 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  }
  if (in->facing) CUDA_TRY(h, cudaMemcpyAsync(h->d.facing + ed.slot_off, in->facing, S, cudaMemcpyHostToDevice, s));
  if (in->energy) CUDA_TRY(h, cudaMemcpyAsync(h->d.energy + ed.slot_off, in->energy, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  if (in->parent) CUDA_TRY(h, cudaMemcpyAsync(h->d.parent + ed.slot_off, in->parent, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  if (in->birth_step) CUDA_TRY(h, cudaMemcpyAsync(h->d.birth + ed.slot_off, in->birth_step, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  if (in->hp) CUDA_TRY(h, cudaMemcpyAsync(h->d.hp + ed.slot_off, in->hp, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  if (in->age) CUDA_TRY(h, cudaMemcpyAsync(h->d.age + ed.slot_off, in->age, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  if (h->R.rules == RULES_TERRAIN) {
    // terrain arrays: counts must be non-negative
    const int32_t *cellv[2] = {in->water, in->bio};
    for (int q = 0; q < 2; ++q)
      if (cellv[q])
        for (int c = 0; c < N; ++c)
          if (cellv[q][c] < 0) return fail(h, ECO_EINVAL, "negative water or biomass at cell %d", c);
    const int32_t *slotv[2] = {in->a_water, in->a_bio};
    for (int q = 0; q < 2; ++q)
      if (slotv[q])
        for (int i = 0; i < S; ++i)
          if (slotv[q][i] < 0) return fail(h, ECO_EINVAL, "negative carried water or biomass at slot %d", i);
    if (in->water) CUDA_TRY(h, cudaMemcpyAsync(h->d.water + ed.cell_off, in->water, 4 * (size_t)N, cudaMemcpyHostToDevice, s));
    if (in->bio) CUDA_TRY(h, cudaMemcpyAsync(h->d.bio + ed.cell_off, in->bio, 4 * (size_t)N, cudaMemcpyHostToDevice, s));
    if (in->photo) CUDA_TRY(h, cudaMemcpyAsync(h->d.photo + ed.cell_off, in->photo, 4 * (size_t)N, cudaMemcpyHostToDevice, s));
    if (in->a_water) CUDA_TRY(h, cudaMemcpyAsync(h->d.a_water + ed.slot_off, in->a_water, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
    if (in->a_bio) CUDA_TRY(h, cudaMemcpyAsync(h->d.a_bio + ed.slot_off, in->a_bio, 4 * (size_t)S, cudaMemcpyHostToDevice, s));
  }
  std::vector<float4> colour;
  if (in->colour) {
    colour.resize(S);
    for (int i = 0; i < S; ++i) {
      const float r = in->colour[3 * i], g = in->colour[3 * i + 1], b = in->colour[3 * i + 2];
      if (!(r >= 0.0f && r <= 1.0f && g >= 0.0f && g <= 1.0f && b >= 0.0f && b <= 1.0f))
        return fail(h, ECO_EINVAL, "colour of slot %d outside [0, 1]", i);
      colour[i] = make_float4(r, g, b, 0.0f);
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->d.colour + ed.slot_off, colour.data(), sizeof(float4) * (size_t)S,
                                cudaMemcpyHostToDevice, s));
  }
  if (in->step) {
    // all environments share one step counter
    long long st = *in->step;
    CUDA_TRY(h, cudaMemcpyAsync(h->d.step, &st, sizeof st, cudaMemcpyHostToDevice, s));
    h->steps_done = st;
    CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  CUDA_TRY(h, launch_recount(h->d, h->R, s));
  CUDA_TRY(h, launch_compact(h->d, s));
  // the persistent form's arrival counts are kept per step parity, which a
  // written step may change: both start from zero
  CUDA_TRY(h, cudaMemsetAsync(h->d.barrier + BAR_COUNT0, 0, 2 * sizeof(unsigned), s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  return ECO_OK;
}

extern "C" int eco_set_rock(eco_handle *h, int32_t env, const int32_t *rock) {
  int rc = check_env(h, env);
  if (rc) return rc;
  if (h->R.rules != RULES_TERRAIN) return fail(h, ECO_EINVAL, "a rock layer needs the terrain rules");
  if (!rock) return fail(h, ECO_EINVAL, "null rock");
  const EnvDesc &ed = h->env_host[env];
  const int N = ed.side * ed.side;
  for (int c = 0; c < N; ++c)
    if (rock[c] < 0 || rock[c] > 65535) return fail(h, ECO_EINVAL, "rock[%d] outside [0, 65535]", c);
  CUDA_TRY(h, cudaMemcpyAsync(h->d.rock + ed.cell_off, rock, 4 * (size_t)N, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}

extern "C" int eco_get_rock(eco_handle *h, int32_t env, int32_t *rock) {
  int rc = check_env(h, env);
  if (rc) return rc;
  if (!rock) return fail(h, ECO_EINVAL, "null rock");
  const EnvDesc &ed = h->env_host[env];
  CUDA_TRY(h, cudaMemcpyAsync(rock, h->d.rock + ed.cell_off, 4 * (size_t)ed.side * ed.side, cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}

// Logical index of every master element of the tiled block (host copy of
// the layout map), or -1 for padding.
static void logical_map(const Layout &L, std::vector<int> &map) {
  const int per = (int)(L.mstride / 4);
  map.assign(per, -1);
  for (int q = 0; q < L.P; ++q) map[q] = layout_logical(L, q);
}

static int check_range(eco_handle *h, int32_t env, int32_t slot0, int32_t n) {
  int rc = check_env(h, env);
  if (rc) return rc;
  if (slot0 < 0 || n < 0 || slot0 + n > h->env_host[env].n_slots) return fail(h, ECO_EINVAL, "slot range out of bounds");
  return ECO_OK;
}

extern "C" int eco_read_params(eco_handle *h, int32_t env, int32_t slot0, int32_t n, float *out) {
  int rc = check_range(h, env, slot0, n);
  if (rc) return rc;
  if (n == 0) return ECO_OK;
  if (!out) return fail(h, ECO_EINVAL, "null output");
  const Layout &L = h->L;
  const int per = (int)(L.mstride / 4);
  std::vector<float> buf((size_t)n * per);
  const int g0 = h->env_host[env].slot_off + slot0;
  CUDA_TRY(h, cudaMemcpyAsync(buf.data(), h->d.master + (size_t)g0 * per, buf.size() * 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  std::vector<int> map;
  logical_map(L, map);
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < per; ++q)
      if (map[q] >= 0) out[(size_t)i * L.P + map[q]] = buf[(size_t)i * per + q];
  return ECO_OK;
}

extern "C" int eco_write_params(eco_handle *h, int32_t env, int32_t slot0, int32_t n, const float *in) {
  int rc = check_range(h, env, slot0, n);
  if (rc) return rc;
  if (n == 0) return ECO_OK;
  if (!in) return fail(h, ECO_EINVAL, "null input");
  const Layout &L = h->L;
  const int per = (int)(L.mstride / 4);
  std::vector<float> buf((size_t)n * per, 0.0f);
  std::vector<int> map;
  logical_map(L, map);
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < per; ++q)
      if (map[q] >= 0) buf[(size_t)i * per + q] = in[(size_t)i * L.P + map[q]];
  const int g0 = h->env_host[env].slot_off + slot0;
  CUDA_TRY(h, cudaMemcpyAsync(h->d.master + (size_t)g0 * per, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, launch_requant(h->d, h->L, h->R, g0, n, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}

extern "C" int eco_read_streamed(eco_handle *h, int32_t env, int32_t slot0, int32_t n, void *codes,
                                 float *row_scales) {
  int rc = check_range(h, env, slot0, n);
  if (rc) return rc;
  if (h->R.precision == ECO_FP32) return fail(h, ECO_EINVAL, "no streamed copy in the FP32 form");
  if (n == 0) return ECO_OK;
  const Layout &L = h->L;
  std::vector<uint8_t> buf((size_t)n * L.stride);
  const int g0 = h->env_host[env].slot_off + slot0;
  CUDA_TRY(h, cudaMemcpyAsync(buf.data(), h->d.wq + (size_t)g0 * L.stride, buf.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  std::vector<int> map;
  logical_map(L, map);
  const int nW = L.nW;
  const int nB = L.H + L.L * L.H + L.A;  // row scales
  for (int i = 0; i < n; ++i) {
    const uint8_t *blk = buf.data() + (size_t)i * L.stride;
    if (codes) {
      if (L.es == 2) {
        uint16_t *c = reinterpret_cast<uint16_t *>(codes) + (size_t)i * L.P;
        for (int q = 0; q < L.P; ++q) c[q] = 0;
        for (int q = 0; q < nW; ++q) {
          uint16_t v;
          memcpy(&v, blk + 2 * q, 2);
          c[map[q]] = v;
        }
      } else {
        uint8_t *c = reinterpret_cast<uint8_t *>(codes) + (size_t)i * L.P;
        for (int q = 0; q < L.P; ++q) c[q] = 0;
        for (int q = 0; q < nW; ++q) c[map[q]] = blk[q];
      }
    }
    if (row_scales && L.es == 1) memcpy(row_scales + (size_t)i * nB, blk + L.off_scale, 4 * (size_t)nB);
  }
  return ECO_OK;
}

extern "C" int eco_read_streamed_bias(eco_handle *h, int32_t env, int32_t slot0, int32_t n, float *bias) {
  int rc = check_range(h, env, slot0, n);
  if (rc) return rc;
  if (h->R.precision == ECO_FP32) return fail(h, ECO_EINVAL, "no streamed copy in the FP32 form");
  if (n == 0) return ECO_OK;
  if (!bias) return fail(h, ECO_EINVAL, "null output");
  const Layout &L = h->L;
  std::vector<uint8_t> buf((size_t)n * L.stride);
  const int g0 = h->env_host[env].slot_off + slot0;
  CUDA_TRY(h, cudaMemcpyAsync(buf.data(), h->d.wq + (size_t)g0 * L.stride, buf.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  // the block holds the biases in physical order k (master element nW + k);
  // the caller gets them in ascending logical position
  std::vector<std::pair<int, int>> order((size_t)L.nB);
  for (int k = 0; k < L.nB; ++k) order[k] = {layout_logical(L, L.nW + k), k};
  std::sort(order.begin(), order.end());
  for (int i = 0; i < n; ++i) {
    const uint8_t *blk = buf.data() + (size_t)i * L.stride + L.off_bias;
    for (int r = 0; r < L.nB; ++r) memcpy(bias + (size_t)i * L.nB + r, blk + 4 * (size_t)order[r].second, 4);
  }
  return ECO_OK;
}

extern "C" int eco_read_policy_io(eco_handle *h, int32_t env, float *logits, uint8_t *actions) {
  int rc = check_env(h, env);
  if (rc) return rc;
  const EnvDesc &ed = h->env_host[env];
  if (logits)
    CUDA_TRY(h, cudaMemcpyAsync(logits, h->d.logits + (size_t)ed.slot_off * h->L.A,
                                sizeof(float) * (size_t)ed.n_slots * h->L.A, cudaMemcpyDeviceToHost, h->stream));
  if (actions)
    CUDA_TRY(h, cudaMemcpyAsync(actions, h->d.act + ed.slot_off, ed.n_slots, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ECO_OK;
}
