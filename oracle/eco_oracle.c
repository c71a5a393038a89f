/*
 * eco_oracle.c -- plain, slow, obviously-correct CPU oracle for one environment
 * step of the ecological simulator of arXiv 2510.18221 ("The Emergence of
 * Complex Behavior in Large-Scale Ecological Environments").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant generator
 * with the CUDA library; every rule below is restated from the paper (and the
 * concrete rule set the build fixes where the paper leaves a gap; each such
 * reading is listed in the design notes).
 *
 * Paper passages followed (sections of the paper):
 *   Sec. 3.1  Ecological Games: population function (alive mask + parents).
 *   Sec. 3.2  Environment: grid world, resources, sensors, actions, move
 *             cancellation, attack, eat, single-parent reproduction behind
 *             the parent.
 *   Sec. 3.3  Policies: per-agent MLP, softmax sampling, bfloat16 weights,
 *             Kaiming init with zero biases, Gaussian mutation of all
 *             parameters of the child.
 *   Sec. 3.2 "Resources and Agent Health", "Actions", App. F.7 (attack
 *             strength), App. F.8 (agent HP): the paper's rule set -- HP with
 *             starvation, attack and age damage and healing from energy,
 *             rotate / forward moves, a 3x3 attack in front that can kill,
 *             explicit eat and reproduce actions, resources dropped where an
 *             agent dies.  One resource (energy lying on cells) stands in for
 *             the paper's water / energy / biomass.
 *   App. E    the step runs every phase of the environment each step.
 *
 * Precision: the policy runs in FP64 on the FP32-stored master parameters
 * (or on their exact dequantised BF16 / FP8-e4m3 forms).  All world state is
 * integer.  Random numbers are Philox4x32-10 (Salmon et al., SC'11), keyed by
 * (seed, stream) and counted by (step, index, sub, 0), so no draw depends on
 * evaluation order.
 *
 * Build: gcc -std=c99 -O2 -ffp-contract=off -fopenmp -fPIC -shared -lm.
 * OpenMP is used only across agents in the policy phase and across slots in
 * weight initialisation; every agent's result is independent of the thread
 * count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Configuration and state (all arrays are owned by the caller).            */
/* ------------------------------------------------------------------------ */

enum {
  ORC_FP32 = 0,
  ORC_BF16 = 1,
  ORC_FP8 = 2
};

enum {
  ORC_AUTO_EAT = 1,     /* small config: eating is automatic on the cell   */
  ORC_ROTATE_OBS = 2,   /* egocentric patch rotated so facing is "up"      */
  ORC_CANCEL_ALL = 4,   /* the paper's rule: any contested move is cancelled */
  ORC_GREEDY = 8        /* argmax of the logits, no Gumbel noise           */
};

/* Philox stream identifiers (key word 1). */
enum {
  ST_WALL = 1,
  ST_FOOD_INIT = 2,
  ST_PLACE = 3,
  ST_FACING_INIT = 4,
  ST_W_INIT = 5,
  ST_SAMPLE = 6,
  ST_CLAIM_MOVE = 7,
  ST_CLAIM_ATTACK = 8,
  ST_CLAIM_BIRTH = 9,
  ST_MUTATE = 10,
  ST_REGROW = 11,
  ST_COLOUR = 12,  /* colour trait: initial colour, and its mutation */
  ST_BIOMASS = 13  /* terrain rules: initial biomass sites              */
};

/* Vision (Sec. 3.2 "Sensors"; App. F.6 viewing configurations). */
enum {
  ORC_VISION_CHANNELS = 0, /* one-hot channels (food, agent, wall)          */
  ORC_VISION_RGB = 1       /* rendered colours: an agent shows its colour   */
                           /* trait, a wall grey, food green, empty black   */
};
enum {
  ORC_VIEW_AROUND = 0,     /* the window is centred on the agent             */
  ORC_VIEW_FRONT = 1       /* the window lies ahead: the agent in the middle */
                           /* of its bottom row, nothing behind it visible   */
};

/* Rule sets.  Simple: the workloads' rules (death at zero energy, a
 * 50% energy-stealing attack on the faced cell, reproduction at a
 * threshold).  Paper (Sec. 3.2, App. F.7-F.8): HP, rotate / forward moves,
 * a 3x3 attack in front, eat and reproduce actions, resource drop at death. */
enum {
  ORC_RULES_SIMPLE = 0,
  ORC_RULES_PAPER = 1,
  ORC_RULES_TERRAIN = 2  /* the paper rules plus rock, flowing water and
                            biomass (Sec. 3.2 "Terrain", "Resources")     */
};

/* Action codes of the paper rule set (Sec. 3.2 "Actions": rest, three
 * moves, attack, eat -- one resource here, so one eat action -- and
 * reproduce). */
enum {
  P_REST = 0,
  P_ROT_CW = 1,
  P_ROT_CCW = 2,
  P_FORWARD = 3,
  P_ATTACK = 4,
  P_EAT = 5,
  P_REPRODUCE = 6,
  P_N_ACTIONS = 7,
  T_DRINK = 7,      /* terrain rules: the eat action of water            */
  T_EAT_BIO = 8,    /* terrain rules: the eat action of biomass          */
  T_N_ACTIONS = 9
};

/* Action codes of the simple rule set.  Small config: 0..5; mid and larger
 * configs add 6..8. */
enum {
  A_STAY = 0,
  A_NORTH = 1,
  A_SOUTH = 2,
  A_EAST = 3,
  A_WEST = 4,
  A_ATTACK = 5,
  A_TURN_LEFT = 6,
  A_TURN_RIGHT = 7,
  A_EAT = 8
};

typedef struct {
  int32_t side;        /* L: the grid is L x L and toroidal              */
  int32_t slots;       /* S: agent slots (alive or free)                 */
  int32_t init_alive;  /* K: agents placed at reset                      */
  int32_t patch_k;     /* k: odd side of the egocentric patch; 0 = no     */
                       /* vision sensor ("Blind", App. F.6)               */
  int32_t n_scalars;   /* 4 (energy + 3 zeros) or 8 (+ facing one-hot)   */
  int32_t hidden;      /* H                                              */
  int32_t n_actions;   /* A: 6 or 9                                      */
  int32_t precision;   /* ORC_FP32 / ORC_BF16 / ORC_FP8                  */
  int32_t flags;       /* ORC_* flags                                    */
  uint32_t seed;
  float sigma;         /* mutation standard deviation                    */
  float food_density;  /* initial Bernoulli food probability             */
  float regrow_p;      /* per-step Bernoulli regrowth probability        */
  float wall_density;  /* Bernoulli wall probability                     */
  int32_t e_init, e_metab, e_food, e_repro, attack_num, attack_den;
  int32_t policy_form; /* ORC_PLAIN or ORC_PAPER_FORM (see the layout below) */
  int32_t n_hidden;    /* paper form: hidden H -> H layers (plain form: 1)  */
  /* Paper rule set only (ORC_RULES_PAPER).  HP is counted in quarter
   * points, so that the paper's 10 HP maximum, 5 HP child, full / half /
   * quarter attack (10 / 5 / 2.5 HP) are whole numbers: 40, 20, 40/20/10. */
  int32_t rules;         /* ORC_RULES_SIMPLE or ORC_RULES_PAPER            */
  int32_t hp_max;        /* HP ceiling; founders start at it               */
  int32_t hp_child;      /* HP of a newborn                                */
  int32_t attack_damage; /* HP taken from every agent in the 3x3 square    */
  int32_t heal_rate;     /* HP regained per step while energy allows       */
  int32_t heal_cost;     /* energy paid for one step of healing            */
  int32_t age_div;       /* age damage per step = floor(age / age_div)     */
  int32_t starve_damage; /* HP lost in a step whose cost exceeds the energy */
  int32_t e_act;         /* extra energy cost of any action but rest       */
  int32_t e_cap;         /* stomach capacity: eating stops at this energy  */
  int32_t e_child;       /* energy a parent hands to its child             */
  int32_t vision;        /* ORC_VISION_CHANNELS or ORC_VISION_RGB          */
  int32_t view;          /* ORC_VIEW_AROUND or ORC_VIEW_FRONT              */
  /* Terrain rule set only (water and biomass in whole units). */
  int32_t sea_level;     /* reset: water depth sea_level - rock below it   */
  int32_t w_init;        /* founders' water                                */
  int32_t w_metab;       /* water spent per step, returned to the cell     */
  int32_t w_bite, w_cap; /* water drunk per drink action; water capacity   */
  int32_t w_child;       /* water a parent hands to its child              */
  int32_t heal_water;    /* water spent (returned) per step of healing     */
  int32_t b_body;        /* biomass of a body: founders carry it           */
  int32_t b_child;       /* biomass a parent hands to its child            */
  int32_t b_bite, b_cap; /* biomass per eat-biomass action; capacity       */
  int32_t b_site;        /* biomass on an initial biomass site             */
  float biomass_density; /* probability that a cell is a biomass site      */
  int32_t photo_q16;     /* energy grown per biomass unit per step, 2^-16  */
  int32_t res_cap;       /* most energy a cell holds                       */
} orc_config;

enum {
  ORC_PLAIN = 0,      /* tanh MLP D -> H -> H -> A with biases everywhere   */
  ORC_PAPER_FORM = 1  /* Sec. 3.3: per-sensor input linears summed, ReLU,
                         L hidden layers, unbiased head, temperature       */
};

typedef struct {
  uint8_t *food;       /* [L*L] 0/1                                      */
  uint8_t *wall;       /* [L*L] 0/1                                      */
  int32_t *occ;        /* [L*L] slot standing on the cell, or -1         */
  uint8_t *alive;      /* [S]                                            */
  int32_t *x, *y;      /* [S] column, row                                */
  uint8_t *facing;     /* [S] 0 N, 1 E, 2 S, 3 W                         */
  int32_t *energy;     /* [S]                                            */
  int32_t *parent;     /* [S] parent slot, -1 for founders               */
  int32_t *birth_step; /* [S] step of birth, -1 for founders             */
  float *master;       /* [S][P] parameters, logical order (see below)   */
  int64_t *step;       /* the step counter t                             */
  int32_t *hp;         /* [S] paper rules: HP in quarter points           */
  int32_t *age;        /* [S] paper rules: steps survived                 */
  int32_t *res;        /* [L*L] paper rules: energy lying on the cell;    */
                       /*   food[c] == (res[c] > 0)                       */
  float *colour;       /* [S][3] colour trait (Sec. 3.3), RGB in [0, 1]   */
  int32_t *rock;       /* [L*L] terrain: rock height (an input)           */
  int32_t *water;      /* [L*L] terrain: water on the cell                */
  int32_t *bio;        /* [L*L] terrain: free biomass on the cell         */
  uint32_t *photo;     /* [L*L] terrain: photosynthesis remainder, 2^-16  */
  int32_t *a_water;    /* [S] terrain: water carried                      */
  int32_t *a_bio;      /* [S] terrain: biomass carried                    */
} orc_state;

typedef struct {
  int64_t agent_steps;        /* agents alive when the step began        */
  int64_t act[16];            /* histogram of chosen actions             */
  int64_t moves;              /* successful moves                        */
  int64_t move_blocked;       /* target wall or occupied at step start   */
  int64_t move_lost;          /* lost the claim (or cancelled)           */
  int64_t eaten;              /* food units eaten                        */
  int64_t attacks;            /* attack actions taken                    */
  int64_t attack_hits;        /* energy transfers made                   */
  int64_t energy_transferred; /* energy moved by attacks                 */
  int64_t deaths;
  int64_t dead_energy;        /* sum of energies (<= 0) of agents that died */
  int64_t births;
  int64_t failed_births;      /* birth-cell winners left without a slot   */
  int64_t regrown;            /* cells that regrew food                  */
  int64_t alive;              /* alive at the end of the step            */
  int64_t food_total;         /* food cells at the end of the step       */
  int64_t energy_total;       /* sum of alive energies at the end        */
  /* paper rules only (0 under the simple rules) */
  int64_t res_total;          /* energy lying on cells at the end        */
  int64_t eaten_energy;       /* energy moved from cells into stomachs   */
  int64_t metab_paid;         /* energy paid for actions                 */
  int64_t heals;              /* agents that healed this step            */
  int64_t starved;            /* agents whose cost exceeded their energy */
  int64_t damage;             /* HP dealt by attacks                     */
  int64_t food_emptied;       /* cells emptied by eating                 */
  int64_t food_refilled;      /* empty cells that received a death drop  */
                              /* (terrain: or grew energy)               */
  /* terrain rules only */
  int64_t water_cells;        /* water on cells at the end               */
  int64_t water_agents;       /* water carried at the end                */
  int64_t bio_cells;          /* free biomass at the end                 */
  int64_t bio_agents;         /* biomass carried at the end              */
  int64_t drunk;              /* water moved from cells into agents      */
  int64_t water_spent;        /* water agents spent (back on their cell) */
  int64_t thirsty;            /* agent-steps without the water to spend  */
  int64_t bio_eaten;          /* biomass moved from cells into agents    */
  int64_t photo;              /* energy grown on free biomass            */
  int64_t dead_water;         /* water dropped by agents that died       */
  int64_t dead_bio;           /* biomass dropped by agents that died     */
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Parameter layout (logical order).  Sec. 3.3: a per-agent MLP.             */
/*   W_in [H][D] row-major, then one bias vector [H] per sensor (the        */
/*   paper's separate per-sensor input linears, whose outputs are summed:   */
/*   the weights of all sensors together form W_in), then L hidden layers   */
/*   W_l [H][H], b_l [H], then the head W_out [A][H], its bias b_out [A]     */
/*   (plain form only), then the log-temperature tau (paper form only).     */
/* Plain form: one sensor, L = 1, tanh, biased head, no temperature         */
/* (= W1, b1, W2, b2, W3, b3).  Paper form: sensors vision / internal       */
/* (+ compass with 8 scalars), L = n_hidden, ReLU, unbiased head, tau.      */
/* ------------------------------------------------------------------------ */

/* Channels per patch cell: 3, or 4 under the terrain rules (Sec. 3.2:
 * three colour channels and the local difference in elevation). */
static int patch_channels(const orc_config *c) {
  return c->rules == ORC_RULES_TERRAIN ? 4 : 3;
}

int orc_obs_dim(const orc_config *c) {
  return patch_channels(c) * c->patch_k * c->patch_k + c->n_scalars;
}

typedef struct {
  int D, H, A, L;       /* inputs, hidden width, actions, hidden layers     */
  int ns;               /* sensors, each with its own input bias            */
  int relu, out_bias, temp;
  int oWin, obin, oWh, oWout, obout, otau, P;
} orc_shape;

/* Parameter count for explicit shape numbers (the paper's table of network
 * sizes is written in these terms). */
int orc_param_count_shape(int D, int H, int A, int L, int ns, int out_bias, int temp) {
  return H * D + ns * H + L * (H * H + H) + A * H + (out_bias ? A : 0) + (temp ? 1 : 0);
}

static void shape_of(const orc_config *c, orc_shape *s) {
  s->D = orc_obs_dim(c);
  s->H = c->hidden;
  s->A = c->n_actions;
  if (c->policy_form == ORC_PAPER_FORM) {
    s->L = c->n_hidden;
    /* sensors: vision (when there is a patch), compass (8+ scalars), internal */
    s->ns = (c->patch_k > 0 ? 1 : 0) + (c->n_scalars >= 8 ? 1 : 0) + 1;
    s->relu = 1;
    s->out_bias = 0;
    s->temp = 1;
  } else {
    s->L = 1;
    s->ns = 1;
    s->relu = 0;
    s->out_bias = 1;
    s->temp = 0;
  }
  s->oWin = 0;
  s->obin = s->H * s->D;
  s->oWh = s->obin + s->ns * s->H; /* layer l: W at oWh + l*(H*H+H), b after */
  s->oWout = s->oWh + s->L * (s->H * s->H + s->H);
  s->obout = s->oWout + s->A * s->H;
  s->otau = s->obout + (s->out_bias ? s->A : 0);
  s->P = s->otau + (s->temp ? 1 : 0);
}

int orc_n_params(const orc_config *c) {
  orc_shape s;
  shape_of(c, &s);
  return s.P;
}

/* Is parameter p a weight (part of W_in, a hidden W_l or W_out)? */
static int is_weight(const orc_shape *s, int p) {
  int l;
  if (p < s->obin) return 1;
  for (l = 0; l < s->L; l++) {
    int w0 = s->oWh + l * (s->H * s->H + s->H);
    if (p >= w0 && p < w0 + s->H * s->H) return 1;
  }
  return p >= s->oWout && p < s->obout;
}

/* Number of inputs of the sensor that input j of W_in belongs to: the
 * patch (3k^2), the compass one-hot (4 inputs, 8-scalar form), and the
 * internal scalars (energy and the reserved zeros).  The plain form treats
 * the whole observation as one input. */
static int sensor_fan_in(const orc_config *c, const orc_shape *s, int j) {
  int patch = patch_channels(c) * c->patch_k * c->patch_k;
  if (c->policy_form != ORC_PAPER_FORM) return s->D;
  if (j < patch) return patch;
  if (c->n_scalars >= 8 && j >= patch + 1 && j < patch + 5) return 4;
  return c->n_scalars >= 8 ? c->n_scalars - 4 : c->n_scalars;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies with  */
/* a Weyl-sequence key schedule.                                            */
/* ------------------------------------------------------------------------ */

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int round;
  for (round = 0; round < 10; round++) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ x1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ x3 ^ k1;
    uint32_t n3 = lo0;
    x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    k0 += 0x9E3779B9u; /* golden ratio            */
    k1 += 0xBB67AE85u; /* sqrt(3) - 1             */
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One draw: key = (seed, stream), counter = (a, b, d, 0). */
static void draw4(const orc_config *c, uint32_t stream, uint32_t a, uint32_t b,
                  uint32_t d, uint32_t out[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = a; ctr[1] = b; ctr[2] = d; ctr[3] = 0;
  key[0] = c->seed; key[1] = stream;
  orc_philox(ctr, key, out);
}

/* Uniform in (0,1): the top 24 bits with the lowest forced to one, times
 * 2^-24.  An odd integer below 2^24 times a power of two is exact in FP32
 * and FP64, and the value is never 0 or 1. */
double orc_uniform(uint32_t r) {
  return (double)((r >> 8) | 1u) * (1.0 / 16777216.0);
}

/* Four standard normals from one Philox block by Box-Muller
 * (Box & Muller, 1958): pairs (u0,u1) and (u2,u3). */
void orc_normals4(const uint32_t r[4], double n[4]) {
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = orc_uniform(r[0]), u1 = orc_uniform(r[1]);
  double u2 = orc_uniform(r[2]), u3 = orc_uniform(r[3]);
  double rad0 = sqrt(-2.0 * log(u0));
  double rad1 = sqrt(-2.0 * log(u2));
  n[0] = rad0 * cos(two_pi * u1);
  n[1] = rad0 * sin(two_pi * u1);
  n[2] = rad1 * cos(two_pi * u3);
  n[3] = rad1 * sin(two_pi * u3);
}

/* Standard Gumbel by inversion: -ln(-ln u). */
double orc_gumbel(uint32_t r) {
  double u = orc_uniform(r);
  return -log(-log(u));
}

/* Bernoulli threshold: an event of probability p happens when a 32-bit
 * draw is below floor(p * 2^32). */
uint32_t orc_threshold(float p) {
  double v = (double)p;
  if (!(v > 0.0)) return 0u;
  if (v >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)floor(v * 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Number formats (Sec. 3.3: bfloat16 weights; FP8 e4m3 with a per-row      */
/* scale is the build's second streamed form).                              */
/* ------------------------------------------------------------------------ */

/* bfloat16 = the top 16 bits of an IEEE binary32, rounded to nearest with
 * ties to even on the 16 dropped bits.  NaNs stay quiet NaNs. */
uint16_t orc_bf16_rne(float f) {
  uint32_t u, upper, lower;
  memcpy(&u, &f, 4);
  if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x0040u);
  upper = u >> 16;
  lower = u & 0xFFFFu;
  if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1u;
  return (uint16_t)upper;
}

double orc_bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* Round half to even of a non-negative double. */
static double round_half_even(double v) {
  double fl = floor(v);
  double diff = v - fl;
  if (diff > 0.5) return fl + 1.0;
  if (diff < 0.5) return fl;
  return (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
}

/* OCP 8-bit floating point, E4M3 variant: 1 sign bit, 4 exponent bits with
 * bias 7, 3 mantissa bits; no infinities; S.1111.111 is NaN, so the largest
 * finite magnitude is 1.75 * 2^8 = 448.  Encoding rounds to nearest-even and
 * saturates finite values beyond 448 to +-448 ("satfinite"). */
uint8_t orc_e4m3_encode(float f) {
  uint8_t sign = signbit(f) ? 0x80u : 0x00u;
  double a;
  int e;
  double mant, q;
  if (isnan(f)) return (uint8_t)(sign | 0x7Fu);
  a = fabs((double)f);
  if (a >= 448.0) return (uint8_t)(sign | 0x7Eu);
  if (a < ldexp(1.0, -6)) {
    /* subnormals: multiples of 2^-9; 8 * 2^-9 = 2^-6 is the least normal,
     * whose code (exponent field 1, mantissa 0) is also 8 */
    q = round_half_even(a * 512.0);
    return (uint8_t)(sign | (uint8_t)q);
  }
  frexp(a, &e);  /* a = m * 2^e with m in [0.5, 1) */
  e -= 1;        /* now a in [2^e, 2^(e+1)) */
  mant = a / ldexp(1.0, e) - 1.0; /* in [0, 1), exact */
  q = round_half_even(mant * 8.0);
  if (q >= 8.0) {
    q = 0.0;
    e += 1;
  }
  return (uint8_t)(sign | (uint8_t)((e + 7) << 3) | (uint8_t)q);
}

double orc_e4m3_value(uint8_t b) {
  int s = (b >> 7) & 1, ef = (b >> 3) & 15, m = b & 7;
  double v;
  if (ef == 15 && m == 7) return NAN;
  if (ef == 0)
    v = (double)m * ldexp(1.0, -9);
  else
    v = (1.0 + (double)m / 8.0) * ldexp(1.0, ef - 7);
  return s ? -v : v;
}

/* Per-output-row scale of the FP8 form: the row's largest magnitude maps to
 * the largest finite e4m3 value (IEEE binary32 division); an all-zero row
 * uses scale 1. */
float orc_fp8_row_scale(const float *row, int n) {
  float mx = 0.0f, s;
  int j;
  for (j = 0; j < n; j++) {
    float a = fabsf(row[j]);
    if (a > mx) mx = a;
  }
  s = mx / 448.0f;
  if (s == 0.0f) s = 1.0f;
  return s;
}

/* ------------------------------------------------------------------------ */
/* Geometry.  Column x grows to the east, row y to the south; the grid      */
/* wraps around in both directions.                                         */
/* ------------------------------------------------------------------------ */

static const int DIR_DX[4] = {0, 1, 0, -1}; /* N E S W */
static const int DIR_DY[4] = {-1, 0, 1, 0};

static int wrap(int v, int L) {
  int m = v % L;
  return m < 0 ? m + L : m;
}

static int cell_of(int x, int y, int L) { return y * L + x; }

/* The cell one step from (x, y) in direction dir. */
static int neighbour(int x, int y, int dir, int L) {
  return cell_of(wrap(x + DIR_DX[dir], L), wrap(y + DIR_DY[dir], L), L);
}

/* ------------------------------------------------------------------------ */
/* Reset (Sec. 3.2 / 3.3): walls, food, founders on distinct free cells,     */
/* random facings, Kaiming-style N(0, 1/fan_in) weights and zero biases.     */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Initial parameters of one founder (Sec. 3.3: Kaiming initialisation, zero
 * biases): weight p = N(0,1) * sqrt(gain / fan_in), the normal drawn from
 * stream W_INIT at counter (slot, p/4); gain 1 in the plain (tanh) form and
 * 2 in the paper (ReLU) form; fan_in is the input count of the weight's
 * sensor (W_in) or H (hidden layers and head).  Biases and the
 * log-temperature start at zero. */
void orc_init_params(const orc_config *c, int32_t slot, float *row) {
  orc_shape s;
  int p;
  uint32_t r[4];
  double n[4];
  double gain;
  shape_of(c, &s);
  gain = s.relu ? 2.0 : 1.0;
  for (p = 0; p < s.P; p++) {
    double fan_in;
    if ((p & 3) == 0) {
      draw4(c, ST_W_INIT, (uint32_t)slot, (uint32_t)(p >> 2), 0u, r);
      orc_normals4(r, n);
    }
    if (!is_weight(&s, p)) {
      row[p] = 0.0f;
      continue;
    }
    if (p < s.obin) fan_in = (double)sensor_fan_in(c, &s, p % s.D);
    else fan_in = (double)s.H;
    if (gain == 1.0)
      row[p] = (float)(n[p & 3] / sqrt(fan_in));
    else
      row[p] = (float)(n[p & 3] * sqrt(gain / fan_in));
  }
}

int orc_reset(const orc_config *c, orc_state *s) {
  int L = c->side, N = L * L, S = c->slots, K = c->init_alive;
  int P = orc_n_params(c);
  uint32_t thr_wall = orc_threshold(c->wall_density);
  uint32_t thr_food = orc_threshold(c->food_density);
  uint32_t thr_bio = orc_threshold(c->biomass_density);
  int terrain = c->rules == ORC_RULES_TERRAIN;
  uint64_t *keys;
  int32_t *chosen;
  int cell, nfree = 0, i, slot;
  uint32_t r[4];

  if (K > S || K < 0) return -1;
  for (cell = 0; cell < N; cell++) {
    draw4(c, ST_WALL, (uint32_t)(cell >> 2), 0u, 0u, r);
    s->wall[cell] = (uint8_t)(r[cell & 3] < thr_wall);
    draw4(c, ST_FOOD_INIT, (uint32_t)(cell >> 2), 0u, 0u, r);
    s->food[cell] = (uint8_t)(!s->wall[cell] && r[cell & 3] < thr_food);
    /* paper rules: a food cell holds one bite, e_food energy */
    s->res[cell] = (c->rules != ORC_RULES_SIMPLE && s->food[cell]) ? c->e_food : 0;
    s->occ[cell] = -1;
    /* terrain rules: water fills the cells whose rock lies below sea level
     * (Sec. 3.2 "Terrain"); a Bernoulli(biomass_density) site (stream
     * BIOMASS) holds b_site biomass.  The rock itself is an input. */
    s->water[cell] = 0;
    s->bio[cell] = 0;
    s->photo[cell] = 0;
    if (terrain && !s->wall[cell]) {
      if (s->rock[cell] < c->sea_level) s->water[cell] = c->sea_level - s->rock[cell];
      draw4(c, ST_BIOMASS, (uint32_t)(cell >> 2), 0u, 0u, r);
      if (r[cell & 3] < thr_bio) s->bio[cell] = c->b_site;
    }
  }

  /* Founders: the K non-wall cells with the smallest (PLACE draw, cell)
   * keys, then slots 0..K-1 in ascending cell order. */
  keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(N > 0 ? N : 1));
  chosen = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
  for (cell = 0; cell < N; cell++) {
    if (s->wall[cell]) continue;
    draw4(c, ST_PLACE, (uint32_t)(cell >> 2), 0u, 0u, r);
    keys[nfree++] = ((uint64_t)r[cell & 3] << 32) | (uint64_t)(uint32_t)cell;
  }
  if (nfree < K) {
    free(keys);
    free(chosen);
    return -2;
  }
  qsort(keys, (size_t)nfree, sizeof(uint64_t), cmp_u64);
  for (i = 0; i < K; i++) chosen[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
  qsort(chosen, (size_t)K, sizeof(int32_t), cmp_i32);

  for (slot = 0; slot < S; slot++) {
    s->alive[slot] = 0;
    s->x[slot] = 0;
    s->y[slot] = 0;
    s->facing[slot] = 0;
    s->energy[slot] = 0;
    s->parent[slot] = -1;
    s->birth_step[slot] = -1;
    s->hp[slot] = 0;
    s->age[slot] = 0;
    s->a_water[slot] = 0;
    s->a_bio[slot] = 0;
    s->colour[3 * slot + 0] = s->colour[3 * slot + 1] = s->colour[3 * slot + 2] = 0.0f;
  }
  for (i = 0; i < K; i++) {
    cell = chosen[i];
    s->alive[i] = 1;
    s->x[i] = cell % L;
    s->y[i] = cell / L;
    draw4(c, ST_FACING_INIT, (uint32_t)(i >> 2), 0u, 0u, r);
    s->facing[i] = (uint8_t)(r[i & 3] >> 30);
    s->energy[i] = c->e_init;
    s->hp[i] = c->rules != ORC_RULES_SIMPLE ? c->hp_max : 0;
    s->a_water[i] = terrain ? c->w_init : 0;
    s->a_bio[i] = terrain ? c->b_body : 0;
    /* colour trait: three uniforms of COLOUR at counter (slot, 0, 0, 0) */
    draw4(c, ST_COLOUR, (uint32_t)i, 0u, 0u, r);
    s->colour[3 * i + 0] = (float)orc_uniform(r[0]);
    s->colour[3 * i + 1] = (float)orc_uniform(r[1]);
    s->colour[3 * i + 2] = (float)orc_uniform(r[2]);
    s->occ[cell] = i;
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (slot = 0; slot < S; slot++) {
    float *row = s->master + (size_t)slot * (size_t)P;
    if (slot < K)
      orc_init_params(c, slot, row);
    else
      memset(row, 0, sizeof(float) * (size_t)P);
  }
  *s->step = 0;
  free(keys);
  free(chosen);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Observation (Sec. 3.2 "Sensors"): a k x k patch around the agent with     */
/* channels (food, agent, wall), rotated so that the agent's facing is the  */
/* top row, flattened (row, column, channel), then the scalars             */
/* [energy / e_repro, one-hot facing (8-scalar form), zeros].  Under the    */
/* paper rules the zeros become the internal and external sensors: HP /     */
/* hp_max, age / (age + age_div), and the energy r lying on the agent's     */
/* cell as r / (r + e_food), all in [0, 1).                                 */
/* Front view (App. F.6): the window lies ahead of the agent, which sits in  */
/* the middle of its bottom row.  RGB vision (Sec. 3.2: a rendered patch     */
/* with three colour channels): a cell with an agent shows that agent's      */
/* colour trait, otherwise a wall is grey (0.5, 0.5, 0.5), food is green     */
/* (0, 1, 0) and an empty cell black.                                        */
/* ------------------------------------------------------------------------ */

/* Terrain rules: 4 channels per cell.  RGB as above, except that a cell
 * with neither agent nor wall shows its resources: (B / (B + b_bite),
 * r / (r + e_food), W / (W + w_bite)) for its biomass B, energy r and water
 * W; the fourth channel is the rock height difference d to the agent's own
 * cell as d / (|d| + 16).  16 scalars: [e / e_repro, compass x4, HP, age,
 * r, carried water / w_cap, carried biomass / b_cap, W / (W + w_bite),
 * B / (B + b_bite) of the agent's cell, zeros]. */
static double ratio(double v, double scale) { return v / (v + scale); }

void orc_observe(const orc_config *c, const orc_state *s, int32_t slot, double *x) {
  int L = c->side, k = c->patch_k, R = k / 2, nch = patch_channels(c);
  int terrain = c->rules == ORC_RULES_TERRAIN;
  int f = s->facing[slot];
  int right = (f + 1) & 3;
  int here = cell_of(s->x[slot], s->y[slot], L);
  int r, col, i, base = nch * k * k;
  for (r = 0; r < k; r++) {
    for (col = 0; col < k; col++) {
      int dx, dy, cell, idx = (r * k + col) * nch;
      if (c->flags & ORC_ROTATE_OBS) {
        /* rows run from far ahead (top) to behind (Around) or to the
         * agent's own row (Front); columns from its left to its right */
        int fwd = (c->view == ORC_VIEW_FRONT ? k - 1 : R) - r, rt = col - R;
        dx = fwd * DIR_DX[f] + rt * DIR_DX[right];
        dy = fwd * DIR_DY[f] + rt * DIR_DY[right];
      } else {
        dx = col - R;
        dy = r - R;
      }
      cell = cell_of(wrap(s->x[slot] + dx, L), wrap(s->y[slot] + dy, L), L);
      if (c->vision == ORC_VISION_RGB) {
        int who = s->occ[cell], ch;
        for (ch = 0; ch < 3; ch++) {
          if (who >= 0) x[idx + ch] = (double)s->colour[3 * who + ch];
          else if (s->wall[cell]) x[idx + ch] = 0.5;
          else if (terrain)
            x[idx + ch] = ch == 0 ? ratio(s->bio[cell], c->b_bite)
                        : ch == 1 ? ratio(s->res[cell], c->e_food)
                                  : ratio(s->water[cell], c->w_bite);
          else if (s->food[cell]) x[idx + ch] = ch == 1 ? 1.0 : 0.0;
          else x[idx + ch] = 0.0;
        }
        if (terrain) {
          double d = (double)s->rock[cell] - (double)s->rock[here];
          x[idx + 3] = d / (fabs(d) + 16.0);
        }
        continue;
      }
      x[idx + 0] = s->food[cell] ? 1.0 : 0.0;
      x[idx + 1] = s->occ[cell] >= 0 ? 1.0 : 0.0;
      x[idx + 2] = s->wall[cell] ? 1.0 : 0.0;
    }
  }
  for (i = 0; i < c->n_scalars; i++) x[base + i] = 0.0;
  x[base] = (double)s->energy[slot] / (double)c->e_repro;
  if (c->n_scalars >= 8) x[base + 1 + f] = 1.0;
  if (c->rules != ORC_RULES_SIMPLE) {
    int extra = c->n_scalars >= 8 ? base + 5 : base + 1;
    double age = (double)s->age[slot];
    x[extra + 0] = (double)s->hp[slot] / (double)c->hp_max;
    x[extra + 1] = age / (age + (double)c->age_div);
    x[extra + 2] = ratio(s->res[here], c->e_food);
  }
  if (terrain) {
    x[base + 8] = (double)s->a_water[slot] / (double)c->w_cap;
    x[base + 9] = (double)s->a_bio[slot] / (double)c->b_cap;
    x[base + 10] = ratio(s->water[here], c->w_bite);
    x[base + 11] = ratio(s->bio[here], c->b_bite);
  }
}

/* ------------------------------------------------------------------------ */
/* Policy (Sec. 3.3).  Plain form: h1 = tanh(W1 x + b1),                  */
/* h2 = tanh(W2 h1 + b2), logits = W3 h2 + b3.  Paper form: h0 =             */
/* ReLU(sum over sensors of (W_s x_s + b_s)), L layers h = ReLU(W_l h + b_l), */
/* logits = (W_out h) / T with T = exp(tau).  The action is sampled from     */
/* softmax(logits) by Gumbel-max.                                            */
/* ------------------------------------------------------------------------ */

/* The parameters the policy actually multiplies with, in FP64:
 *   FP32 form (or use_master): the master values;
 *   BF16 form: every weight rounded to bfloat16, biases FP32;
 *   FP8 form:  every weight row r of each layer quantised as
 *              s_r * e4m3(w / s_r), biases FP32. */
void orc_effective_params(const orc_config *c, const float *m, int use_master, double *w) {
  orc_shape s;
  int p, row;
  shape_of(c, &s);
  for (p = 0; p < s.P; p++) w[p] = (double)m[p];
  if (use_master || c->precision == ORC_FP32) return;
  if (c->precision == ORC_BF16) {
    for (p = 0; p < s.P; p++)
      if (is_weight(&s, p)) w[p] = orc_bf16_value(orc_bf16_rne(m[p]));
    return;
  }
  /* FP8: rows of W_in have D entries; rows of the hidden layers and of
   * the head have H entries */
  for (row = 0; row < s.H + s.L * s.H + s.A; row++) {
    int start, n, j;
    float sc;
    if (row < s.H) {
      start = s.oWin + row * s.D;
      n = s.D;
    } else if (row < s.H + s.L * s.H) {
      int l = (row - s.H) / s.H, o = (row - s.H) % s.H;
      start = s.oWh + l * (s.H * s.H + s.H) + o * s.H;
      n = s.H;
    } else {
      start = s.oWout + (row - s.H - s.L * s.H) * s.H;
      n = s.H;
    }
    sc = orc_fp8_row_scale(m + start, n);
    for (j = 0; j < n; j++) {
      float q = m[start + j] / sc; /* IEEE binary32 division */
      w[start + j] = (double)sc * orc_e4m3_value(orc_e4m3_encode(q));
    }
  }
}

/* Is logical parameter p a weight (1) or a bias / the temperature (0)?
 * mask[p] for every p < P. */
void orc_weight_mask(const orc_config *c, uint8_t *mask) {
  orc_shape s;
  int p;
  shape_of(c, &s);
  for (p = 0; p < s.P; p++) mask[p] = (uint8_t)is_weight(&s, p);
}

/* The streamed copy of one master row, as codes in logical order (the
 * weights the reduced-precision policy multiplies with, Sec. 3.3):
 *   BF16 form: codes is uint16_t[P], the bfloat16 RNE code of every weight;
 *   FP8 form:  codes is uint8_t[P]; weight row r of each layer (W_in rows of
 *              D entries, then every hidden layer's rows of H, then the
 *              head's rows of H) has scale s_r = max|w| / 448 (1 for an
 *              all-zero row), written to scales[r], and the e4m3 code of
 *              w / s_r (IEEE binary32 division, satfinite RNE).
 * Bias and temperature positions hold the code of 0 (they stay FP32 in the
 * streamed copy).  Nothing is written for the FP32 form. */
void orc_quantise(const orc_config *c, const float *m, void *codes, float *scales) {
  orc_shape s;
  int p, row;
  shape_of(c, &s);
  if (c->precision == ORC_BF16) {
    uint16_t *q = (uint16_t *)codes;
    for (p = 0; p < s.P; p++) q[p] = is_weight(&s, p) ? orc_bf16_rne(m[p]) : 0;
    return;
  }
  if (c->precision != ORC_FP8) return;
  {
    uint8_t *q = (uint8_t *)codes;
    for (p = 0; p < s.P; p++) q[p] = 0;
    for (row = 0; row < s.H + s.L * s.H + s.A; row++) {
      int start, n, j;
      float sc;
      if (row < s.H) {
        start = s.oWin + row * s.D;
        n = s.D;
      } else if (row < s.H + s.L * s.H) {
        int l = (row - s.H) / s.H, o = (row - s.H) % s.H;
        start = s.oWh + l * (s.H * s.H + s.H) + o * s.H;
        n = s.H;
      } else {
        start = s.oWout + (row - s.H - s.L * s.H) * s.H;
        n = s.H;
      }
      sc = orc_fp8_row_scale(m + start, n);
      scales[row] = sc;
      for (j = 0; j < n; j++) q[start + j] = orc_e4m3_encode(m[start + j] / sc);
    }
  }
}

static double activate(const orc_shape *s, double v) {
  if (s->relu) return v > 0.0 ? v : 0.0;
  return tanh(v);
}

/* Forward pass of one agent's MLP on observation x (FP64).  The returned
 * logits already carry the temperature (logit / T with T = exp(tau)), so
 * the action is sampled from softmax(logits). */
void orc_mlp(const orc_config *c, const double *w, const double *x, double *logits) {
  orc_shape s;
  int o, j, l, k;
  double ha[512], hb[512];
  double *h = ha, *h2 = hb, *tmp;
  shape_of(c, &s);
  for (o = 0; o < s.H; o++) {
    double acc = 0.0;
    for (k = 0; k < s.ns; k++) acc += w[s.obin + k * s.H + o];  /* summed sensor biases */
    for (j = 0; j < s.D; j++) acc += w[s.oWin + o * s.D + j] * x[j];
    h[o] = activate(&s, acc);
  }
  for (l = 0; l < s.L; l++) {
    int oW = s.oWh + l * (s.H * s.H + s.H), ob = oW + s.H * s.H;
    for (o = 0; o < s.H; o++) {
      double acc = w[ob + o];
      for (j = 0; j < s.H; j++) acc += w[oW + o * s.H + j] * h[j];
      h2[o] = activate(&s, acc);
    }
    tmp = h;
    h = h2;
    h2 = tmp;
  }
  for (o = 0; o < s.A; o++) {
    double acc = s.out_bias ? w[s.obout + o] : 0.0;
    for (j = 0; j < s.H; j++) acc += w[s.oWout + o * s.H + j] * h[j];
    if (s.temp) acc = acc * exp(-w[s.otau]);
    logits[o] = acc;
  }
}

/* Policy phase for every alive agent.  For each agent: the logits, the
 * sampled scores (logit + Gumbel, or the logit alone in GREEDY mode), the
 * chosen action (the first maximum) and a bit mask of every action whose
 * score lies within tol of the maximum: when more than one bit is set, the
 * choice is not determined at that resolution and any flagged action is a
 * valid outcome.  Dead slots get zeros and action 0. */
int orc_policy(const orc_config *c, const orc_state *s, int use_master, double tol,
               double *logits, double *scores, uint8_t *action, uint32_t *valid) {
  int S = c->slots, A = c->n_actions, D = orc_obs_dim(c), P = orc_n_params(c);
  int64_t t = *s->step;
  int bad = 0;
  if (A > 16 || c->hidden > 512 || c->e_repro <= 0) return -1;
  if (c->policy_form == ORC_PAPER_FORM && (c->n_hidden < 1 || c->n_hidden > 8)) return -1;
#pragma omp parallel
  {
    double *w = (double *)malloc(sizeof(double) * (size_t)P);
    double *x = (double *)malloc(sizeof(double) * (size_t)D);
    int slot;
#pragma omp for schedule(dynamic, 32)
    for (slot = 0; slot < S; slot++) {
      double *lg = logits + (size_t)slot * A;
      double *sc = scores + (size_t)slot * A;
      int a, best = 0;
      uint32_t mask = 0;
      if (!w || !x) {
        bad = 1;
        continue;
      }
      if (!s->alive[slot]) {
        for (a = 0; a < A; a++) { lg[a] = 0.0; sc[a] = 0.0; }
        action[slot] = 0;
        valid[slot] = 0;
        continue;
      }
      orc_observe(c, s, slot, x);
      orc_effective_params(c, s->master + (size_t)slot * (size_t)P, use_master, w);
      orc_mlp(c, w, x, lg);
      for (a = 0; a < A; a++) {
        double g = 0.0;
        if (!(c->flags & ORC_GREEDY)) {
          uint32_t r[4];
          draw4(c, ST_SAMPLE, (uint32_t)t, (uint32_t)slot, (uint32_t)(a >> 2), r);
          g = orc_gumbel(r[a & 3]);
        }
        sc[a] = lg[a] + g;
      }
      for (a = 1; a < A; a++)
        if (sc[a] > sc[best]) best = a;
      for (a = 0; a < A; a++)
        if (sc[best] - sc[a] <= tol) mask |= 1u << a;
      action[slot] = (uint8_t)best;
      valid[slot] = mask;
    }
    free(w);
    free(x);
  }
  return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Mutation (Sec. 3.3): the child's parameters are the parent's plus          */
/* sigma * N(0,1) on every parameter; the normal for parameter p comes from  */
/* stream MUTATE at counter (step, parent slot, p/4).                        */
/* ------------------------------------------------------------------------ */

void orc_mutate(const orc_config *c, int64_t step, int32_t parent_slot,
                const float *parent_row, float *child_row) {
  int P = orc_n_params(c), p;
  uint32_t r[4];
  double n[4];
  for (p = 0; p < P; p++) {
    if ((p & 3) == 0) {
      draw4(c, ST_MUTATE, (uint32_t)step, (uint32_t)parent_slot, (uint32_t)(p >> 2), r);
      orc_normals4(r, n);
    }
    child_row[p] = (float)((double)parent_row[p] + (double)c->sigma * n[p & 3]);
  }
}

/* Colour trait (Sec. 3.3: a 3-channel colour that mutates like the network
 * weights): child = clamp(fl32(parent + sigma * n), 0, 1) per channel, with
 * n the first three normals of COLOUR at counter (step, parent slot, 1, 0). */
void orc_mutate_colour(const orc_config *c, int64_t step, int32_t parent_slot,
                       const float *parent_rgb, float *child_rgb) {
  uint32_t r[4];
  double n[4];
  int ch;
  draw4(c, ST_COLOUR, (uint32_t)step, (uint32_t)parent_slot, 1u, r);
  orc_normals4(r, n);
  for (ch = 0; ch < 3; ch++) {
    float v = (float)((double)parent_rgb[ch] + (double)c->sigma * n[ch]);
    child_rgb[ch] = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
  }
}

/* ------------------------------------------------------------------------ */
/* Transition (Sec. 3.2 "Actions", "Resources and Agent Health").  Phase    */
/* order: face/turn, move, eat, attack, metabolism + death (health under    */
/* the paper rules), reproduction + mutation, regrowth.                     */
/* ------------------------------------------------------------------------ */

static uint64_t claim_key(const orc_config *c, uint32_t stream, int64_t t, int32_t slot) {
  uint32_t r[4];
  draw4(c, stream, (uint32_t)t, (uint32_t)slot, 0u, r);
  /* the highest draw wins; equal draws go to the lower slot */
  return ((uint64_t)r[0] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)slot);
}

static int32_t claim_slot(uint64_t key) {
  return (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
}


/* The cell at `fwd` steps ahead and `lat` steps to the right of an agent at
 * (x, y) facing f, on the torus. */
static int cell_ahead(int x, int y, int f, int fwd, int lat, int L) {
  int right = (f + 1) & 3;
  int dx = fwd * DIR_DX[f] + lat * DIR_DX[right];
  int dy = fwd * DIR_DY[f] + lat * DIR_DY[right];
  return cell_of(wrap(x + dx, L), wrap(y + dy, L), L);
}

/* One step of the water flow (Sec. 3.2 "Terrain": water flows downhill
 * over the rock layer in a discrete flow simulation).  Reading: each
 * non-wall cell holding water compares its surface, rock + water, with the
 * surfaces of its four non-wall neighbours; the lowest (the first of N, E,
 * S, W on ties) receives min(water, floor((surface - lowest) / 5)) when it
 * is strictly lower.  Every transfer is computed from the surfaces before
 * the step, so no order of the cells matters.  Sending at most a fifth of
 * the drop (one more than the number of neighbours) keeps a cell that
 * receives from all four neighbours from rising above them. */
int orc_water_flow(const orc_config *c, orc_state *s) {
  int L = c->side, N = L * L, cell, d;
  int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  int32_t *to = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  if (!out || !to) {
    free(out);
    free(to);
    return -1;
  }
  for (cell = 0; cell < N; cell++) {
    int64_t here, lowest = 0;
    int best = -1;
    out[cell] = 0;
    to[cell] = -1;
    if (s->wall[cell] || s->water[cell] <= 0) continue;
    here = (int64_t)s->rock[cell] + s->water[cell];
    for (d = 0; d < 4; d++) {
      int n = neighbour(cell % L, cell / L, d, L);
      int64_t h;
      if (s->wall[n]) continue;
      h = (int64_t)s->rock[n] + s->water[n];
      if (best < 0 || h < lowest) {
        best = n;
        lowest = h;
      }
    }
    if (best >= 0 && lowest < here) {
      int64_t amount = (here - lowest) / 5;
      if (amount > s->water[cell]) amount = s->water[cell];
      out[cell] = (int32_t)amount;
      to[cell] = best;
    }
  }
  for (cell = 0; cell < N; cell++) s->water[cell] -= out[cell];
  for (cell = 0; cell < N; cell++)
    if (to[cell] >= 0) s->water[to[cell]] += out[cell];
  free(out);
  free(to);
  return 0;
}

int orc_transition(const orc_config *c, orc_state *s, const uint8_t *action,
                   orc_stats *st, int32_t *birth_parent, int32_t *birth_child) {
  int L = c->side, N = L * L, S = c->slots, A = c->n_actions;
  int P = orc_n_params(c);
  int paper = c->rules != ORC_RULES_SIMPLE;  /* the paper or the terrain rules */
  int terrain = c->rules == ORC_RULES_TERRAIN;
  int64_t t = *s->step;
  uint32_t thr_regrow = orc_threshold(c->regrow_p);
  uint64_t *best_cell = (uint64_t *)calloc((size_t)N, sizeof(uint64_t));
  int32_t *count_cell = (int32_t *)calloc((size_t)N, sizeof(int32_t));
  uint64_t *best_victim = (uint64_t *)calloc((size_t)S, sizeof(uint64_t));
  int32_t *target = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  int32_t *esnap = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  int32_t *dmg = (int32_t *)calloc((size_t)S, sizeof(int32_t));
  int32_t *winners = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  int32_t *free_slots = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
  int slot, cell, nwin = 0, nfree = 0, i, rc = 0;
  static const int MOVE_DIR[5] = {-1, 0, 2, 1, 3}; /* action -> N S E W dir */

  memset(st, 0, sizeof(*st));
  if (!best_cell || !count_cell || !best_victim || !target || !esnap || !dmg || !winners ||
      !free_slots) {
    rc = -1;
    goto done;
  }
  for (slot = 0; slot < S; slot++) {
    if (!s->alive[slot]) continue;
    if (action[slot] >= A) {
      rc = -2;
      goto done;
    }
    st->agent_steps++;
    st->act[action[slot]]++;
  }

  /* 1. Facing.  Simple rules: a move action faces its direction whether or
   *    not the move succeeds; turn-left / turn-right rotate by a quarter.
   *    Paper rules: rotate clockwise / counter-clockwise by a quarter. */
  for (slot = 0; slot < S; slot++) {
    int a = action[slot];
    if (!s->alive[slot]) continue;
    if (paper) {
      if (a == P_ROT_CW) s->facing[slot] = (uint8_t)((s->facing[slot] + 1) & 3);
      else if (a == P_ROT_CCW) s->facing[slot] = (uint8_t)((s->facing[slot] + 3) & 3);
    } else if (a >= A_NORTH && a <= A_WEST) {
      s->facing[slot] = (uint8_t)MOVE_DIR[a];
    } else if (A > A_TURN_LEFT && a == A_TURN_LEFT) {
      s->facing[slot] = (uint8_t)((s->facing[slot] + 3) & 3);
    } else if (A > A_TURN_RIGHT && a == A_TURN_RIGHT) {
      s->facing[slot] = (uint8_t)((s->facing[slot] + 1) & 3);
    }
  }

  /* 2. Moves, one cell in the facing direction (N/S/E/W actions, or move
   *    forward under the paper rules).  A move into a wall or into a cell
   *    occupied when the step began is cancelled.  Several agents moving
   *    into one free cell: the highest CLAIM_MOVE draw wins (ties to the
   *    lower slot), or, with the paper's cancel-all rule, every contested
   *    move is cancelled. */
  for (slot = 0; slot < S; slot++) {
    int a = action[slot], tc;
    uint64_t key;
    target[slot] = -1;
    if (!s->alive[slot]) continue;
    if (paper ? a != P_FORWARD : (a < A_NORTH || a > A_WEST)) continue;
    tc = neighbour(s->x[slot], s->y[slot], s->facing[slot], L);
    if (s->wall[tc] || s->occ[tc] != -1) {
      st->move_blocked++;
      continue;
    }
    target[slot] = tc;
    key = claim_key(c, ST_CLAIM_MOVE, t, slot);
    if (key > best_cell[tc]) best_cell[tc] = key;
    count_cell[tc]++;
  }
  for (slot = 0; slot < S; slot++) {
    int tc = target[slot];
    int won;
    if (tc < 0) continue;
    won = claim_slot(best_cell[tc]) == slot;
    if ((c->flags & ORC_CANCEL_ALL) && count_cell[tc] > 1) won = 0;
    if (!won) {
      st->move_lost++;
      continue;
    }
    s->occ[cell_of(s->x[slot], s->y[slot], L)] = -1;
    s->occ[tc] = slot;
    s->x[slot] = tc % L;
    s->y[slot] = tc / L;
    st->moves++;
  }

  /* 3. Eat.  Simple rules: the food on the agent's cell (automatic in the
   *    small rule set, the eat action otherwise) becomes e_food energy.
   *    Paper rules: the eat action moves one bite, min(e_food, energy on
   *    the cell, e_cap - energy), from the cell into the stomach.  Terrain
   *    rules add the eat actions of the other two resources: drink moves
   *    min(w_bite, water on the cell, w_cap - water carried), eat-biomass
   *    min(b_bite, biomass on the cell, b_cap - biomass carried). */
  for (slot = 0; slot < S; slot++) {
    int here;
    if (!s->alive[slot]) continue;
    here = cell_of(s->x[slot], s->y[slot], L);
    if (terrain && action[slot] == T_DRINK) {
      int32_t sip = c->w_bite;
      if (s->water[here] < sip) sip = s->water[here];
      if (c->w_cap - s->a_water[slot] < sip) sip = c->w_cap - s->a_water[slot];
      if (sip > 0) {
        s->water[here] -= sip;
        s->a_water[slot] += sip;
        st->drunk += sip;
      }
      continue;
    }
    if (terrain && action[slot] == T_EAT_BIO) {
      int32_t bite = c->b_bite;
      if (s->bio[here] < bite) bite = s->bio[here];
      if (c->b_cap - s->a_bio[slot] < bite) bite = c->b_cap - s->a_bio[slot];
      if (bite > 0) {
        s->bio[here] -= bite;
        s->a_bio[slot] += bite;
        st->bio_eaten += bite;
      }
      continue;
    }
    if (paper) {
      int32_t bite = c->e_food;
      if (action[slot] != P_EAT) continue;
      if (s->res[here] < bite) bite = s->res[here];
      if (c->e_cap - s->energy[slot] < bite) bite = c->e_cap - s->energy[slot];
      if (bite <= 0) continue;
      s->res[here] -= bite;
      s->energy[slot] += bite;
      st->eaten++;
      st->eaten_energy += bite;
      if (s->res[here] == 0) {
        s->food[here] = 0;
        st->food_emptied++;
      }
      continue;
    }
    if (!((c->flags & ORC_AUTO_EAT) || (A > A_EAT && action[slot] == A_EAT))) continue;
    if (s->food[here]) {
      s->food[here] = 0;
      s->energy[slot] += c->e_food;
      st->eaten++;
    }
  }

  /* 4. Attack.  Simple rules: on the faced cell; a victim yields to one
   *    attacker (highest CLAIM_ATTACK draw, ties to the lower slot), which
   *    takes floor(e * num / den) of the victim's post-eat energy.  Every
   *    amount is computed from the post-eat snapshot, so the outcome does
   *    not depend on any order.  Paper rules: every agent in the 3x3 square
   *    directly in front (1..3 cells ahead, one to either side) loses
   *    attack_damage HP per attacker. */
  if (paper) {
    for (slot = 0; slot < S; slot++) {
      int fwd, lat;
      if (!s->alive[slot] || action[slot] != P_ATTACK) continue;
      st->attacks++;
      for (fwd = 1; fwd <= 3; fwd++) {
        for (lat = -1; lat <= 1; lat++) {
          int v = s->occ[cell_ahead(s->x[slot], s->y[slot], s->facing[slot], fwd, lat, L)];
          if (v < 0) continue;
          dmg[v] += c->attack_damage;
          st->attack_hits++;
          st->damage += c->attack_damage;
        }
      }
    }
  } else {
    for (slot = 0; slot < S; slot++) esnap[slot] = s->energy[slot];
    for (slot = 0; slot < S; slot++) {
      int tc, v;
      uint64_t key;
      if (!s->alive[slot] || action[slot] != A_ATTACK) continue;
      st->attacks++;
      tc = neighbour(s->x[slot], s->y[slot], s->facing[slot], L);
      v = s->occ[tc];
      if (v < 0) continue;
      key = claim_key(c, ST_CLAIM_ATTACK, t, slot);
      if (key > best_victim[v]) best_victim[v] = key;
    }
    for (slot = 0; slot < S; slot++) {
      int32_t w, amount;
      if (best_victim[slot] == 0) continue;
      w = claim_slot(best_victim[slot]);
      amount = (int32_t)(((int64_t)esnap[slot] * c->attack_num) / c->attack_den);
      s->energy[slot] -= amount;
      s->energy[w] += amount;
      st->attack_hits++;
      st->energy_transferred += amount;
    }
  }

  /* 5. Simple rules: every agent pays e_metab; an agent whose energy is then
   *    <= 0 dies and frees its cell and slot.
   *    Paper rules, per agent in this order: pay the action's cost
   *    (e_metab, plus e_act for anything but rest); a cost above the
   *    energy empties the stomach and costs starve_damage HP.  Then the
   *    attack damage and the age damage floor(age / age_div) come off the
   *    HP.  A survivor below hp_max with at least heal_cost energy heals
   *    heal_rate HP (capped at hp_max) for heal_cost energy.  At HP <= 0 the
   *    agent dies and its energy is dropped on its cell; otherwise it ages
   *    by one step.
   *    Terrain rules: after the energy, every agent spends w_metab water,
   *    which goes back onto its cell (Sec. 3.2: spent water returns to the
   *    landscape); without enough water it spends what it has and loses
   *    starve_damage HP.  Healing also needs, and spends onto the cell,
   *    heal_water water.  A dying agent drops its energy, water and
   *    biomass on its cell. */
  for (slot = 0; slot < S; slot++) {
    int here;
    if (!s->alive[slot]) continue;
    here = cell_of(s->x[slot], s->y[slot], L);
    if (paper) {
      int32_t cost = c->e_metab + (action[slot] != P_REST ? c->e_act : 0);
      int32_t hp = s->hp[slot];
      if (s->energy[slot] >= cost) {
        s->energy[slot] -= cost;
        st->metab_paid += cost;
      } else {
        st->metab_paid += s->energy[slot];
        s->energy[slot] = 0;
        hp -= c->starve_damage;
        st->starved++;
      }
      if (terrain) {
        int32_t spend = c->w_metab;
        if (s->a_water[slot] < spend) {
          spend = s->a_water[slot];
          hp -= c->starve_damage;
          st->thirsty++;
        }
        s->a_water[slot] -= spend;
        s->water[here] += spend;
        st->water_spent += spend;
      }
      hp -= dmg[slot];
      hp -= s->age[slot] / c->age_div;
      if (hp > 0 && hp < c->hp_max && c->heal_rate > 0 && s->energy[slot] >= c->heal_cost &&
          (!terrain || s->a_water[slot] >= c->heal_water)) {
        hp += c->heal_rate;
        if (hp > c->hp_max) hp = c->hp_max;
        s->energy[slot] -= c->heal_cost;
        if (terrain) {
          s->a_water[slot] -= c->heal_water;
          s->water[here] += c->heal_water;
          st->water_spent += c->heal_water;
        }
        st->heals++;
      }
      if (hp <= 0) {
        int32_t e = s->energy[slot];
        st->deaths++;
        st->dead_energy += e;
        if (terrain) {
          s->water[here] += s->a_water[slot];
          s->bio[here] += s->a_bio[slot];
          st->dead_water += s->a_water[slot];
          st->dead_bio += s->a_bio[slot];
          s->a_water[slot] = 0;
          s->a_bio[slot] = 0;
        }
        if (e > 0 && s->res[here] == 0) {
          s->food[here] = 1;
          st->food_refilled++;
        }
        s->res[here] += e;
        s->alive[slot] = 0;
        s->occ[here] = -1;
        s->energy[slot] = 0;
        s->hp[slot] = 0;
      } else {
        s->hp[slot] = hp;
        s->age[slot]++;
      }
      continue;
    }
    s->energy[slot] -= c->e_metab;
    if (s->energy[slot] <= 0) {
      st->deaths++;
      st->dead_energy += s->energy[slot];
      s->alive[slot] = 0;
      s->occ[here] = -1;
      s->energy[slot] = 0;
    }
  }

  /* 6. Reproduction: an agent with energy >= e_repro (under the paper rules:
   *    that also took the reproduce action) places one child on the cell
   *    behind it, if that cell is not a wall and is free after the deaths.
   *    One winner per cell (highest CLAIM_BIRTH draw, ties to the lower
   *    slot).  Winners, in ascending slot order, take the free slots in
   *    ascending order; winners left without a slot keep their energy.
   *    Simple rules: the child gets floor(e/2), the parent keeps the rest.
   *    Paper rules: the parent hands e_child to the child, which starts at
   *    hp_child HP and age 0.  Terrain rules: the parent must also carry
   *    b_body + b_child biomass (its own body and the child's: Sec. 3.2,
   *    biomass is needed to exist) and w_child water, and hands b_child and
   *    w_child to the child.  The child faces as the parent did and
   *    carries the parent's parameters mutated by sigma * N(0,1). */
  for (i = 0; i < N; i++) best_cell[i] = 0;
  for (slot = 0; slot < S; slot++) {
    int tc;
    uint64_t key;
    target[slot] = -1;
    if (!s->alive[slot] || s->energy[slot] < c->e_repro) continue;
    if (paper && action[slot] != P_REPRODUCE) continue;
    if (terrain && (s->a_bio[slot] < c->b_body + c->b_child || s->a_water[slot] < c->w_child)) continue;
    tc = neighbour(s->x[slot], s->y[slot], (s->facing[slot] + 2) & 3, L);
    if (s->wall[tc] || s->occ[tc] != -1) continue;
    target[slot] = tc;
    key = claim_key(c, ST_CLAIM_BIRTH, t, slot);
    if (key > best_cell[tc]) best_cell[tc] = key;
  }
  for (slot = 0; slot < S; slot++) {
    if (target[slot] >= 0 && claim_slot(best_cell[target[slot]]) == slot) winners[nwin++] = slot;
    if (!s->alive[slot]) free_slots[nfree++] = slot;
  }
  for (i = 0; i < nwin; i++) {
    int32_t p = winners[i], ch, e, ce, tc;
    if (i >= nfree) {
      st->failed_births++;
      continue;
    }
    ch = free_slots[i];
    tc = target[p];
    e = s->energy[p];
    ce = paper ? c->e_child : e / 2;
    s->energy[p] = e - ce;
    s->energy[ch] = ce;
    s->hp[ch] = paper ? c->hp_child : 0;
    s->age[ch] = 0;
    if (terrain) {
      s->a_water[p] -= c->w_child;
      s->a_water[ch] = c->w_child;
      s->a_bio[p] -= c->b_child;
      s->a_bio[ch] = c->b_child;
    }
    s->alive[ch] = 1;
    s->x[ch] = tc % L;
    s->y[ch] = tc / L;
    s->facing[ch] = s->facing[p];
    s->parent[ch] = p;
    s->birth_step[ch] = (int32_t)t;
    s->occ[tc] = ch;
    orc_mutate(c, t, p, s->master + (size_t)p * (size_t)P, s->master + (size_t)ch * (size_t)P);
    orc_mutate_colour(c, t, p, s->colour + 3 * p, s->colour + 3 * ch);
    if (birth_parent) birth_parent[st->births] = p;
    if (birth_child) birth_child[st->births] = ch;
    st->births++;
  }

  /* 7. Regrowth: every non-wall cell without food regrows with probability
   *    regrow_p (stream REGROW at counter (step, cell/4)): one food unit, or
   *    under the paper rules one bite of e_food energy. */
  for (cell = 0; cell < N; cell++) {
    uint32_t r[4];
    if (s->wall[cell] || s->food[cell]) continue;
    draw4(c, ST_REGROW, (uint32_t)t, (uint32_t)(cell >> 2), 0u, r);
    if (r[cell & 3] < thr_regrow) {
      s->food[cell] = 1;
      if (paper) s->res[cell] = c->e_food;
      st->regrown++;
    }
  }

  /* 8. Terrain rules: energy grows on free biomass (Sec. 3.2; App. F.2
   *    "biomass photosynthesis rate"), then the water flows one step. */
  if (terrain) {
    for (cell = 0; cell < N; cell++) {
      uint64_t acc;
      int64_t gain, room;
      if (s->wall[cell] || s->bio[cell] <= 0) continue;
      acc = (uint64_t)s->photo[cell] + (uint64_t)s->bio[cell] * (uint64_t)c->photo_q16;
      gain = (int64_t)(acc >> 16);
      s->photo[cell] = (uint32_t)(acc & 0xFFFFu);
      room = (int64_t)c->res_cap - s->res[cell];
      if (gain > room) gain = room;
      if (gain <= 0) continue;
      if (s->res[cell] == 0) {
        s->food[cell] = 1;
        st->food_refilled++;
      }
      s->res[cell] += (int32_t)gain;
      st->photo += gain;
    }
    if (orc_water_flow(c, s) != 0) {
      rc = -1;
      goto done;
    }
  }

  for (slot = 0; slot < S; slot++) {
    if (!s->alive[slot]) continue;
    st->alive++;
    st->energy_total += s->energy[slot];
    if (terrain) {
      st->water_agents += s->a_water[slot];
      st->bio_agents += s->a_bio[slot];
    }
  }
  for (cell = 0; cell < N; cell++) {
    st->food_total += s->food[cell];
    if (paper) st->res_total += s->res[cell];
    if (terrain) {
      st->water_cells += s->water[cell];
      st->bio_cells += s->bio[cell];
    }
  }
  *s->step = t + 1;

done:
  free(best_cell); free(count_cell); free(best_victim); free(target);
  free(esnap); free(dmg); free(winners); free(free_slots);
  return rc;
}
