/*
 * eco.h -- C-ABI of the GB300 (sm_103a) ecological-simulator step library.
 *
 * The library runs the environment step of arXiv 2510.18221 ("The Emergence
 * of Complex Behavior in Large-Scale Ecological Environments") on one GPU,
 * for one or many independent environments at once.  App. E of the paper
 * describes the same split: a population-level interface where the map
 * state, agent states and heritable traits go in, and the actions, births,
 * deaths and environment transitions happen inside.
 * Every phase of the step runs in the library's own CUDA kernels:
 *   observe (Sec. 3.2 "Sensors") -> per-agent MLP (Sec. 3.3) -> sample
 *   (Sec. 3.3) -> turn/move with claim conflicts (Sec. 3.2 "Actions") -> eat
 *   -> attack -> metabolism and death (Sec. 3.2 "Resources and Agent
 *   Health") -> reproduction with Gaussian mutation (Sec. 3.2, 3.3) ->
 *   regrowth -> statistics (App. E measurement API).
 *
 * Conventions
 *   - Every function that can fail returns an int status: ECO_OK (0) or a
 *     negative ECO_E* code.  The message of the last failure on a handle is
 *     returned by eco_last_error().
 *   - Device memory: the caller allocates ONE workspace of the size
 *     eco_workspace_bytes() reports, 256-byte aligned, and keeps it alive
 *     until eco_destroy().  The library carves every device array out of
 *     it, allocates no other device memory, and never frees caller memory.
 *     Each handle holds three small pinned host buffers for the statistics
 *     and status word (about 2 x n_envs x 8 x ECO_N_STATS bytes each; one
 *     for eco_read_stats(), two for eco_step_read()), freed by
 *     eco_destroy(); a read copies into one of them in one transfer.
 *   - Streams: all device work is enqueued on the stream given to
 *     eco_create() (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  eco_reset() and eco_step() are asynchronous.  eco_read_*()
 *     and eco_write_*() synchronise that stream.
 *   - Host buffers passed to eco_read_* / eco_write_* are caller-owned,
 *     sized as documented per function, and are not retained.
 *   - Environments are independent: environment e, run alone or batched
 *     with others, produces identical results.
 */
#ifndef ECO_H
#define ECO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ECO_ABI_VERSION 5

/* Status codes. */
#define ECO_OK 0
#define ECO_EINVAL (-1)   /* bad argument or configuration                  */
#define ECO_ENOMEM (-2)   /* workspace too small or device memory exhausted */
#define ECO_ECUDA (-3)    /* a CUDA runtime call failed                     */
#define ECO_ETIMEOUT (-4) /* a device-side wait ran out of its budget       */
#define ECO_EABI (-5)     /* abi_version mismatch                           */

/* Precision of the weights the policy kernel streams (Sec. 3.3 uses
 * bfloat16 weights; FP8 e4m3 with a per-output-row FP32 scale is the
 * second reduced form).  FP32 master weights always exist and receive the
 * mutations; the streamed copy is re-derived from them. */
#define ECO_FP32 0
#define ECO_BF16 1
#define ECO_FP8_E4M3 2

/* Rule flags. */
#define ECO_AUTO_EAT 1   /* eat automatically on the post-move cell        */
#define ECO_ROTATE_OBS 2 /* rotate the patch so the facing is the top row  */
#define ECO_CANCEL_ALL 4 /* the paper's rule: every contested move fails   */
#define ECO_GREEDY 8     /* argmax of the logits instead of sampling       */

/* Policy forms.  Plain: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2),
 * logits = W3 h2 + b3 (the workloads' MLP).  Paper (Sec. 3.3): each sensor
 * (vision patch, internal scalars, compass one-hot) has its own input linear
 * layer; their outputs are summed and passed through ReLU, then n_hidden
 * ReLU layers of width H, then an unbiased linear head; logits are divided
 * by the evolvable temperature exp(tau).  Kaiming initialisation, zero
 * biases and tau. */
#define ECO_POLICY_PLAIN 0
#define ECO_POLICY_PAPER 1

/* Rule sets.  Simple: the workloads' rules -- energy is life (death at
 * e <= 0), the attack takes a fraction of the faced agent's energy,
 * reproduction happens at e >= e_repro.  Paper (Sec. 3.2 "Resources and
 * Agent Health" and "Actions"; App. F.7 attack strength, App. F.8 agent HP),
 * with one resource, energy, lying on cells and carried in a stomach:
 *   - HP (quarter points) is life; founders start at hp_max, children at
 *     hp_child;
 *   - each step costs e_metab (rest) or e_metab + e_act (any other action);
 *     a cost above the energy empties the stomach and costs starve_damage
 *     HP; attacks and age (floor(age / age_div) per step) take HP; a
 *     survivor below hp_max with >= heal_cost energy heals heal_rate HP for
 *     heal_cost energy; at HP <= 0 the agent dies and its energy is added to
 *     its cell;
 *   - attack: every agent in the 3x3 square in front (1..3 cells ahead, one
 *     to either side) loses attack_damage HP per attacker;
 *   - eat: moves min(e_food, energy on the cell, e_cap - energy) into the
 *     stomach; a cell "has food" while it holds energy;
 *   - reproduce (the action, at energy >= e_repro): the child on the cell
 *     behind gets e_child energy from the parent;
 *   - regrowth puts e_food energy on an empty cell with probability
 *     regrow_p. */
#define ECO_RULES_SIMPLE 0
#define ECO_RULES_PAPER 1
/* Terrain rules (Sec. 3.2 "Terrain", "Resources and Agent Health"; App.
 * F.2): the paper rules plus
 *   - a rock layer (eco_set_rock) and water: eco_reset fills every non-wall
 *     cell below sea_level to the sea level; each step the water flows: a
 *     cell with water sends min(water, floor(drop / 5)) to its lowest open
 *     neighbour (first of N, E, S, W) when that neighbour's surface
 *     (rock + water) lies `drop` below its own, all computed from the
 *     surfaces before the step;
 *   - biomass: a Bernoulli(biomass_density) site holds b_site at reset;
 *     free biomass grows energy at photo_q16 / 2^16 per unit per step (a
 *     per-cell fixed-point remainder keeps the sum exact), up to res_cap
 *     energy per cell;
 *   - agents carry water and biomass: founders w_init and b_body; every step
 *     spends w_metab water onto the agent's cell (not enough: it spends what
 *     it has and loses starve_damage HP); healing also needs and spends
 *     heal_water; drink / eat-biomass take min(bite, on the cell, room);
 *     reproduction also needs b_body + b_child biomass and w_child water and
 *     hands b_child and w_child to the child; a dying agent drops its
 *     energy, water and biomass on its cell;
 *   - vision: RGB (needs ECO_VISION_RGB) with 4 channels per cell -- an
 *     agent's colour, a wall's grey, else (B/(B+b_bite), r/(r+e_food),
 *     W/(W+w_bite)) of the cell's biomass, energy and water -- and the rock
 *     difference d to the agent's cell as d/(|d|+16); 16 scalars:
 *     [e/e_repro, compass x4, HP/hp_max, age/(age+age_div), r/(r+e_food),
 *     water/w_cap, biomass/b_cap, W/(W+w_bite), B/(B+b_bite) of its own
 *     cell, 0, 0, 0, 0]. */
#define ECO_RULES_TERRAIN 2

/* Vision (Sec. 3.2 "Sensors": a top-down patch with three colour channels)
 * and viewing configuration (App. F.6).  Channels: per cell (food, agent,
 * wall) as 0/1.  RGB: a cell holding an agent shows that agent's colour
 * trait; otherwise a wall is (0.5, 0.5, 0.5), food (0, 1, 0), an empty cell
 * (0, 0, 0).  Around: the k x k window is centred on the agent.  Front
 * (needs ECO_ROTATE_OBS): the window lies ahead, the agent in the middle of
 * its bottom row, so nothing behind it is visible.
 * Every agent carries a colour trait (Sec. 3.3), RGB in [0, 1]: uniform at
 * reset, and at birth clamp(parent + sigma * n, 0, 1) per channel. */
#define ECO_VISION_CHANNELS 0
#define ECO_VISION_RGB 1
#define ECO_VIEW_AROUND 0
#define ECO_VIEW_FRONT 1

/* Action codes.  Simple rules: 0 stay, 1 north, 2 south, 3 east, 4 west,
 * 5 attack; nine-action sets add 6 turn-left, 7 turn-right, 8 eat.  Paper
 * rules (7 actions): 0 rest, 1 rotate clockwise, 2 rotate counter-
 * clockwise, 3 forward, 4 attack, 5 eat, 6 reproduce.  Terrain rules (9):
 * those and 7 drink, 8 eat biomass. */

typedef struct eco_handle eco_handle;

/* Configuration, copied at eco_create().  All environments share the
 * observation, MLP shape, precision, rules and constants; each has its own
 * grid side (even, >= 4), slot count, founder count and seed. */
typedef struct {
  int32_t abi_version;           /* must be ECO_ABI_VERSION                  */
  int32_t n_envs;                /* >= 1                                     */
  const int32_t *env_side;       /* [n_envs] grid side L (torus L x L)       */
  const int32_t *env_slots;      /* [n_envs] agent slots                     */
  const int32_t *env_init_alive; /* [n_envs] founders placed by eco_reset    */
  const uint32_t *env_seed;      /* [n_envs] Philox seed                     */
  int32_t patch_k;               /* odd patch side k: D = 3k^2 + n_scalars
                                    (4k^2 under the terrain rules); 0 = no
                                    vision sensor (App. F.6 "Blind")        */
  int32_t n_scalars;             /* 4 or 8; 16 under the terrain rules       */
  int32_t hidden;                /* H in {32, 64, 128}                       */
  int32_t n_actions;             /* A in {6, 9}; 7 under the paper rules     */
  int32_t precision;             /* ECO_FP32 / ECO_BF16 / ECO_FP8_E4M3       */
  int32_t flags;                 /* ECO_AUTO_EAT | ECO_ROTATE_OBS | ...      */
  float sigma;                   /* mutation standard deviation              */
  float food_density;            /* initial food probability per cell        */
  float regrow_p;                /* food regrowth probability per step       */
  float wall_density;            /* wall probability per cell                */
  int32_t e_init;                /* founders' energy                         */
  int32_t e_metab;               /* energy paid per step                     */
  int32_t e_food;                /* energy per food unit eaten               */
  int32_t e_repro;               /* reproduction threshold; also the energy
                                    scale of the observation scalar          */
  int32_t attack_num, attack_den;/* transferred fraction of victim energy    */
  int32_t policy_variant;        /* 0 = autotune over the dense variants;
                                    -1 = autotune over the input-sparse
                                    variants, which stream only the W_in
                                    rows of nonzero inputs (same result up to
                                    the order of FP32 additions); k > 0 =
                                    force variant k (eco_policy_variants) */
  int32_t launch_mode;           /* environment phases: 0 = one persistent
                                    cooperative kernel when the device
                                    supports it, 1 = one kernel per phase
                                    (identical results)                     */
  int32_t policy_form;           /* ECO_POLICY_PLAIN or ECO_POLICY_PAPER     */
  int32_t n_hidden;              /* paper form: hidden H -> H layers (1..4);
                                    the plain form ignores it (one layer)   */
  /* Rule set, and the constants only the paper rules use (HP in quarter
   * points: the paper's 10 HP maximum is 40). */
  int32_t rules;                 /* ECO_RULES_SIMPLE or ECO_RULES_PAPER      */
  int32_t hp_max;                /* >= 1                                     */
  int32_t hp_child;              /* in [1, hp_max]                           */
  int32_t attack_damage;         /* HP per attacker covering a victim, >= 0  */
  int32_t heal_rate;             /* HP healed per step, >= 0                 */
  int32_t heal_cost;             /* energy per step of healing, >= 0         */
  int32_t age_div;               /* age damage floor(age / age_div), >= 1    */
  int32_t starve_damage;         /* HP lost when the cost exceeds the energy */
  int32_t e_act;                 /* extra cost of any action but rest, >= 0  */
  int32_t e_cap;                 /* stomach capacity, >= max(e_init, 1)      */
  int32_t e_child;               /* energy handed to a child, in [1, e_repro] */
  int32_t vision;                /* ECO_VISION_CHANNELS or ECO_VISION_RGB    */
  int32_t view;                  /* ECO_VIEW_AROUND or ECO_VIEW_FRONT        */
  /* Terrain rules only (whole units of water and biomass). */
  int32_t sea_level;             /* water level at reset                     */
  int32_t w_init;                /* founders' water, in [0, w_cap]           */
  int32_t w_metab;               /* water spent per step, >= 0               */
  int32_t w_bite, w_cap;         /* drink amount, water capacity, >= 1       */
  int32_t w_child;               /* water handed to a child, >= 0            */
  int32_t heal_water;            /* water per step of healing, >= 0          */
  int32_t b_body;                /* founders' biomass, in [0, b_cap]         */
  int32_t b_child;               /* biomass handed to a child, >= 0          */
  int32_t b_bite, b_cap;         /* eat-biomass amount, capacity, >= 1       */
  int32_t b_site;                /* biomass on an initial site, >= 0         */
  float biomass_density;         /* initial biomass site probability         */
  int32_t photo_q16;             /* energy per biomass unit per step, 2^-16  */
  int32_t res_cap;               /* most energy a cell holds, >= e_food      */
} eco_config;

/* Statistics, one record per environment (App. E measurement API).
 * Counters marked (sum) accumulate over steps in the "total" record and
 * hold the last step's value in the "last" record; (now) values describe
 * the state after the last step in both records. */
enum {
  ECO_STAT_STEP = 0,          /* (now) steps completed since reset          */
  ECO_STAT_AGENT_STEPS,       /* (sum) agents alive when a step began       */
  ECO_STAT_ACT0,              /* (sum) ECO_STAT_ACT0 + a: action a chosen   */
  ECO_STAT_MOVES = ECO_STAT_ACT0 + 16, /* (sum) successful moves             */
  ECO_STAT_MOVE_BLOCKED,      /* (sum) move into wall / occupied cell       */
  ECO_STAT_MOVE_LOST,         /* (sum) lost a contested cell                */
  ECO_STAT_EATEN,             /* (sum) food units eaten                     */
  ECO_STAT_ATTACKS,           /* (sum) attack actions                       */
  ECO_STAT_ATTACK_HITS,       /* (sum) energy transfers (paper rules: agents
                                 hit, counted once per attacker)           */
  ECO_STAT_ENERGY_TRANSFERRED,/* (sum) energy moved by attacks              */
  ECO_STAT_DEATHS,            /* (sum)                                      */
  ECO_STAT_DEAD_ENERGY,       /* (sum) energies of agents that died (<= 0
                                 under the simple rules; dropped on the
                                 cell under the paper rules)              */
  ECO_STAT_BIRTHS,            /* (sum)                                      */
  ECO_STAT_FAILED_BIRTHS,     /* (sum) birth-cell winners without a slot    */
  ECO_STAT_REGROWN,           /* (sum) cells that regrew food               */
  ECO_STAT_ALIVE,             /* (now) alive agents                         */
  ECO_STAT_FOOD_TOTAL,        /* (now) cells holding food                   */
  ECO_STAT_ENERGY_TOTAL,      /* (now) summed energy of alive agents        */
  /* paper rules only (0 under the simple rules) */
  ECO_STAT_RES_TOTAL,         /* (now) energy lying on cells                */
  ECO_STAT_EATEN_ENERGY,      /* (sum) energy moved from cells to stomachs  */
  ECO_STAT_METAB_PAID,        /* (sum) energy paid for actions              */
  ECO_STAT_HEALS,             /* (sum) agent-steps of healing               */
  ECO_STAT_STARVED,           /* (sum) agent-steps whose cost exceeded e    */
  ECO_STAT_DAMAGE,            /* (sum) HP dealt by attacks                  */
  ECO_STAT_FOOD_EMPTIED,      /* (sum) cells emptied by eating              */
  ECO_STAT_FOOD_REFILLED,     /* (sum) empty cells that received a drop
                                 (terrain: or grew energy)                  */
  /* terrain rules only (0 otherwise) */
  ECO_STAT_WATER_CELLS,       /* (now) water on cells                       */
  ECO_STAT_WATER_AGENTS,      /* (now) water carried                        */
  ECO_STAT_BIO_CELLS,         /* (now) free biomass                         */
  ECO_STAT_BIO_AGENTS,        /* (now) biomass carried                      */
  ECO_STAT_DRUNK,             /* (sum) water moved from cells into agents   */
  ECO_STAT_WATER_SPENT,       /* (sum) water agents spent onto their cells  */
  ECO_STAT_THIRSTY,           /* (sum) agent-steps without w_metab water    */
  ECO_STAT_BIO_EATEN,         /* (sum) biomass moved from cells into agents */
  ECO_STAT_PHOTO,             /* (sum) energy grown on free biomass         */
  ECO_STAT_DEAD_WATER,        /* (sum) water dropped by agents that died    */
  ECO_STAT_DEAD_BIO,          /* (sum) biomass dropped by agents that died  */
  ECO_N_STATS
};

typedef struct {
  int64_t v[ECO_N_STATS];
} eco_stats;

/* Host view of one environment's world state (all arrays caller-owned).
 * Cells are indexed c = y * L + x (x = column, grows east; y = row, grows
 * south).  Any pointer may be NULL to skip that array. */
typedef struct {
  uint8_t *food;       /* [L*L] 0/1                                         */
  uint8_t *wall;       /* [L*L] 0/1                                         */
  int32_t *occ;        /* [L*L] slot on the cell or -1                      */
  uint8_t *alive;      /* [slots] 0/1                                       */
  int32_t *x, *y;      /* [slots]                                           */
  uint8_t *facing;     /* [slots] 0 N, 1 E, 2 S, 3 W                        */
  int32_t *energy;     /* [slots]                                           */
  int32_t *parent;     /* [slots] parent slot, -1 for founders              */
  int32_t *birth_step; /* [slots] step of birth, -1 for founders            */
  int64_t *step;       /* [1] steps completed                               */
  int32_t *hp;         /* [slots] paper rules: HP (quarter points)          */
  int32_t *age;        /* [slots] paper rules: steps survived               */
  int32_t *res;        /* [L*L] paper rules: energy lying on the cell; on
                          write, food is taken as res > 0 (the food array
                          is then ignored)                                  */
  float *colour;       /* [slots][3] colour trait, RGB in [0, 1]            */
  int32_t *water;      /* [L*L] terrain rules: water on the cell            */
  int32_t *bio;        /* [L*L] terrain rules: free biomass on the cell     */
  uint32_t *photo;     /* [L*L] terrain rules: photosynthesis remainder     */
  int32_t *a_water;    /* [slots] terrain rules: water carried              */
  int32_t *a_bio;      /* [slots] terrain rules: biomass carried            */
} eco_state_view;

/* Parameter count P and observation size D for a configuration.
 * Parameters in "logical order" are W1[H][D], b1[H], W2[H][H], b2[H],
 * W3[A][H], b3[A] (Sec. 3.3 MLP: tanh hidden layers, linear head). */
int eco_param_count(const eco_config *cfg, int32_t *n_params, int32_t *obs_dim);

/* Bytes of device workspace eco_create() needs for cfg.  Returns
 * ECO_EINVAL for an invalid configuration. */
int eco_workspace_bytes(const eco_config *cfg, size_t *bytes);

/* Create a handle.  dev_workspace: caller-allocated device memory of at
 * least the reported size (256-byte aligned); stream: cudaStream_t or
 * NULL.  A variant forced by cfg->policy_variant > 0 is set up here; with
 * 0 or -1 the variant is autotuned on the state at eco_prepare or at the
 * first step.  On failure *out is NULL. */
int eco_create(const eco_config *cfg, void *dev_workspace, size_t bytes,
               void *stream, eco_handle **out);

/* Reset every environment (Sec. 3.2, 3.3), each from its own Philox seed
 * (env_seed, or the last eco_reset_seed): walls and food by Bernoulli
 * draws, founders on the K non-wall cells with the smallest placement keys
 * (slots 0..K-1 in ascending cell order), random facings, energy e_init,
 * weights N(0, 1/fan_in), zero biases; statistics cleared.  Asynchronous. */
int eco_reset(eco_handle *h);

/* eco_reset after re-seeding: environment e takes the Philox seed
 * (uint32_t)(seed + e) (the low 32 bits; Philox keys are (seed, stream)
 * word pairs) in place of its env_seed, for this reset and every step after
 * it, until the next eco_reset_seed.  A new seed needs no new handle and no
 * new capture of the step graphs.  Asynchronous, except that it waits for
 * the host-to-device copy of the environment table. */
int eco_reset_seed(eco_handle *h, uint64_t seed);

/* Advance every environment by n_steps >= 0 steps.  Asynchronous; replays
 * CUDA graphs of 8 steps and of one step (built at the first call that
 * needs them; the first call should not come inside a stream capture).
 * A device-side wait that ran out of its budget in a step is reported as
 * ECO_ETIMEOUT by the next eco_read_stats(). */
int eco_step(eco_handle *h, int32_t n_steps);

/* Pipelined step and read: enqueue one step whose graph ends by copying
 * the statistics and status word into one of two pinned buffers the handle
 * owns, then wait for the copy made by the PREVIOUS eco_step_read call and
 * return those records.  So a call returns the records as of the end of
 * the step enqueued by the previous call (on the first call after
 * eco_create or eco_reset: the records as they stood when the call was
 * made), while the step it enqueued runs; eco_read_stats afterwards gives
 * the last step's.  The host never waits for the step it has just
 * enqueued, so the GPU stays busy across the read.  Buffers as for
 * eco_read_stats; the status word is checked as there (ECO_ETIMEOUT). */
int eco_step_read(eco_handle *h, eco_stats *total, eco_stats *last, int32_t n_envs);

/* Optional: choose the policy-kernel variant (autotuned on the current
 * state, so call it after eco_reset) and build every step graph now rather
 * than in the first eco_step / eco_step_timed that needs them.  Steps
 * nothing.  Synchronises the stream. */
int eco_prepare(eco_handle *h);

/* Copy statistics of environments [0, n_envs) to host records (either
 * pointer may be NULL).  Synchronises the stream. */
int eco_read_stats(eco_handle *h, eco_stats *total, eco_stats *last, int32_t n_envs);

/* Copy environment env's world state to / from the host (App. E,
 * "Simulator design": the simulator's population-level interface hands the
 * map state and the agent states to the population algorithm and takes
 * them back; here they also serve checkpoints and the oracle's lock-step).
 * Writing replaces
 * the listed arrays (NULL arrays are left unchanged; food, wall and occ
 * must be written together if any of them is written, as must alive / x /
 * y), then re-derives the derived device tables.  Both synchronise. */
int eco_read_state(eco_handle *h, int32_t env, eco_state_view *out);
int eco_write_state(eco_handle *h, int32_t env, const eco_state_view *in);

/* Terrain rules: the rock layer of env (Sec. 3.2 "Terrain": each map has a
 * rock layer defining the height of each cell), host array rock[L*L] of
 * heights in [0, 65535], cells indexed y * L + x.  The paper gives no
 * generator for its terrains: the caller supplies the heights.  Kept until
 * the next eco_set_rock (eco_create starts from a flat 0 layer); the next
 * eco_reset fills the cells below sea_level, and the flow and the vision's
 * elevation channel use it at once.  ECO_EINVAL under the other rule sets
 * or for heights out of range.  Synchronises. */
int eco_set_rock(eco_handle *h, int32_t env, const int32_t *rock);
int eco_get_rock(eco_handle *h, int32_t env, int32_t *rock);

/* FP32 master parameters of slots [slot0, slot0 + n) of env, logical
 * order, host array [n][P]: the agents' heritable traits that App. E's
 * population-level interface exchanges with the population algorithm
 * (Sec. 3.3: the per-agent policy weights that mutation perturbs).  Writing also re-derives the streamed
 * BF16/FP8 copy of those slots.  Both synchronise. */
int eco_read_params(eco_handle *h, int32_t env, int32_t slot0, int32_t n, float *out);
int eco_write_params(eco_handle *h, int32_t env, int32_t slot0, int32_t n, const float *in);

/* Streamed copy of slots [slot0, slot0 + n), logical order: BF16 codes as
 * uint16 [n][P] or e4m3 codes as uint8 [n][P] (bias positions hold the
 * code of 0), plus for FP8 the row scales [n][H + Lh*H + A], Lh the
 * number of hidden layers (1 in the plain form, n_hidden in the paper
 * form): the output rows of W_in, of each hidden layer, then of the head.
 * row_scales must hold that many floats per slot.  ECO_EINVAL for the
 * FP32 precision.  Synchronises. */
int eco_read_streamed(eco_handle *h, int32_t env, int32_t slot0, int32_t n,
                      void *codes, float *row_scales);

/* The FP32 biases (and tau) that the streamed copy of slots
 * [slot0, slot0 + n) of env carries beside its codes, which the policy
 * kernel reads instead of the masters' (Sec. 3.3: only the weights are
 * streamed in the reduced precision).  Host array bias [n][nB], nB = P
 * minus the weight count, each slot's values in ascending logical
 * parameter position.  ECO_EINVAL for the FP32 precision.  Synchronises. */
int eco_read_streamed_bias(eco_handle *h, int32_t env, int32_t slot0, int32_t n, float *bias);

/* Logits [slots][A] (FP32) and actions [slots] of the last step's policy
 * phase for env (dead slots hold stale values).  Synchronises. */
int eco_read_policy_io(eco_handle *h, int32_t env, float *logits, uint8_t *actions);

/* Policy-kernel variants: *count variants exist; *chosen is the one in use.
 * eco_policy_variant_name() describes variant k (static string). */
int eco_policy_variants(const eco_handle *h, int32_t *count, int32_t *chosen);
const char *eco_policy_variant_name(int32_t k);

/* Launch form of the environment phases in use: *mode 0 = one persistent
 * cooperative kernel of *blocks CTAs, 1 = one kernel per phase.  Decided at
 * the first eco_step (falls back to 1 when the device or the graph capture
 * does not support the cooperative form). */
int eco_launch_mode(const eco_handle *h, int32_t *mode, int32_t *blocks);

/* Like eco_step, and also times policy-kernel launches with a CUDA-event
 * pair on the library stream, inside the step graphs: the first step of
 * every graph of 8 steps (the rest of n_steps untimed), or, for n_steps
 * below 8, every step in one-step graphs.  The results are identical; an
 * event-record node adds a few us to its step, so only one step in 8
 * carries them and eco_step's graphs have none.
 * eco_policy_timing() synchronises, then returns, over the launches timed
 * since its last call: the summed policy-kernel time in milliseconds, their
 * number, and (agents may be NULL) the summed count of agents they
 * processed (at most 4096 launches are buffered, and eco_policy_timing must
 * come within 4096 steps of them; more launches return ECO_EINVAL). */
int eco_step_timed(eco_handle *h, int32_t n_steps);
int eco_policy_timing(eco_handle *h, double *total_ms, int32_t *n_timed, int64_t *agents);

/* Run only the policy phase (observe + MLP + sample) of the current state
 * n_iters times, for timing and for the policy-parity tests; the world
 * state does not change.  Asynchronous. */
int eco_policy_only(eco_handle *h, int32_t n_iters);

/* Failure-detection test hook (off unless called; cleared by eco_reset).
 * The persistent environment kernel separates its phases with grid
 * barriers whose waits are bounded; this arms the next steps so that CTA
 * absent_cta leaves that kernel before its first barrier and every wait
 * gives up after poll_budget polls (a few ms for 10^5).  The other CTAs'
 * waits then run out: the status word records the timeout, every CTA
 * leaves at its barrier, the later steps' environment kernels return at
 * once, and the next eco_read_stats / eco_step_read returns ECO_ETIMEOUT.
 * The world state is then partly stepped; eco_reset (or eco_reset_seed)
 * clears the barrier, the status word and these test words.  ECO_EINVAL
 * when the persistent form with more than one CTA is not in use
 * (eco_launch_mode; it is decided at the first eco_step) or for an
 * argument out of range.  Synchronises. */
int eco_arm_barrier_timeout(eco_handle *h, int32_t absent_cta, int32_t poll_budget);

/* Phase trace of the persistent environment kernel (a tracing aid; App. E
 * describes the simulator's measurement tooling, not this).  on = 1 clears
 * the trace table and makes every following step record, in the row
 * step % ECO_TRACE_STEPS, ECO_TRACE_WORDS globaltimer values in ns:
 *   [0] CTA 0's start; [1 + k] the last CTA's arrival at grid barrier k
 *   (k = 0..3, 0 when unused; a CTA arrives once all its threads are
 *   there); [5 + k] CTA 0's pass through barrier k; [9] the last CTA's end;
 *   [10] the step; [11] the step's birth claimants; [12] the number of grid
 *   barriers the step used; [13..15] 0.
 * on = 0 clears the table and stops recording.  Traced steps compute the
 * same results (the stamps add a block barrier and a few stores per grid
 * barrier).  eco_reset switches the trace off.  ECO_EINVAL when the
 * persistent form is not in use (eco_launch_mode; it is decided by
 * eco_prepare or the first eco_step).  Synchronises. */
#define ECO_TRACE_STEPS 64
#define ECO_TRACE_WORDS 16
int eco_trace_phases(eco_handle *h, int32_t on);

/* Copy the first max_rows (at most ECO_TRACE_STEPS) rows of the trace
 * table to rows[max_rows][ECO_TRACE_WORDS] (host); *n_rows = rows copied.
 * Rows of steps not traced since the last eco_trace_phases hold 0.
 * Synchronises. */
int eco_read_phase_trace(eco_handle *h, uint64_t *rows, int32_t max_rows, int32_t *n_rows);

/* Algorithmic bytes the policy phase must read for the current alive
 * population (weights of every alive agent in the streamed precision,
 * biases and scales in FP32); synchronises. */
int eco_policy_bytes(eco_handle *h, int64_t *bytes, int64_t *n_alive);

/* Movement-claim resolution for one world, allocating nothing.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code running where every byte of
 * device memory is owned by a host framework's own pool, loops that must
 * not call cudaMalloc because it can synchronise the whole device, and
 * callers that cannot hold a workspace for the lifetime of a handle.  It
 * needs no handle and no workspace: its scratch (one 64-bit claim per
 * cell) is a fixed file-scope device array of ECO_NOALLOC_MAX_CELLS
 * entries (8 MiB), which every GPU that loads the library holds until the
 * process exits.
 *
 * Rule (the movement phase of eco_step for one world, under
 * ECO_RULES_SIMPLE without ECO_CANCEL_ALL; the paper and terrain rules'
 * forward / rotate actions and the cancel-all rule are not covered): agent
 * i at cell pos[i] (y * side + x) with action act[i] and facing
 * facing_in[i]; a move action (1 N, 2 S, 3 E, 4 W) faces its direction and
 * claims the neighbouring cell unless blocked[cell] is nonzero (a wall, or
 * an agent there when the step began); among claimants of one cell the
 * highest Philox draw of stream CLAIM_MOVE at counter (step, i, 0, 0)
 * under key (seed, 7) wins, ties to the lower i; actions 6 / 7 turn left /
 * right.  An agent whose pos[i] lies outside [0, side * side) does not
 * move (its facing still follows its action).  Outputs: facing_out[i],
 * pos_out[i] (the new cell, or pos[i]) and moved[i] (0/1).  pos_out may be
 * pos and facing_out may be facing_in (an in-place update).
 *
 * All array arguments are device pointers the caller allocates: pos,
 * pos_out int32[n_agents]; act, facing_in, facing_out, moved
 * uint8[n_agents]; blocked uint8[side * side].  Work is enqueued on
 * stream (cudaStream_t or NULL) and is asynchronous.
 * Returns ECO_EINVAL if side is odd or < 4, if side * side exceeds
 * ECO_NOALLOC_MAX_CELLS, or for a null array with n_agents > 0;
 * ECO_ECUDA if a CUDA call or launch fails, and also, without launching
 * anything or clearing it, when a CUDA error left by earlier work is
 * already pending on the calling thread.  The message is
 * eco_last_error(NULL).  It calls no cudaMalloc / cudaFree.
 *
 * The first call on each device looks up the scratch array's device
 * address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call on a device shares the
 * one scratch array (each call clears the cells it uses before claiming),
 * so calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race and give wrong results; serialise them. */
#define ECO_NOALLOC_MAX_CELLS (1 << 20)
int eco_move_claims_noalloc(int32_t side, int32_t n_agents, const int32_t *pos,
                            const uint8_t *act, const uint8_t *facing_in,
                            const uint8_t *blocked, uint32_t seed, uint32_t step,
                            uint8_t *facing_out, int32_t *pos_out, uint8_t *moved,
                            void *stream);

/* Release the handle (not the workspace).  Accepts NULL. */
void eco_destroy(eco_handle *h);

/* Message of the last failure on h (or a global message when h is NULL). */
const char *eco_last_error(const eco_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* ECO_H */
