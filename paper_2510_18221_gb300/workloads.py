"""Seeded synthetic workload definitions (inputs only, no simulation arithmetic).

Each workload is a plain dictionary describing one environment: grid side,
agent slots, founders, observation patch, MLP shape, streamed precision,
rule flags and the constants of the rule set.  Both the CUDA library (through
the binding) and the CPU oracle (in the tests) consume these dictionaries;
neither derives anything from the other.

The five workloads mirror the paper's scales (Sec. 3.2: grids from 64^2 to
1024^2 with the initial population scaled with the area; App. E: runs of up
to ~131k agent slots at 1024^2) with the concrete rule set the build fixes:
binary food, int32 energy, a tanh MLP and fixed constants.
"""
from __future__ import annotations

import copy

import numpy as np

_COMMON = dict(
    e_init=100, e_metab=1, e_food=20, e_repro=200, attack_num=1, attack_den=2,
)

# 64x64 toroidal grid, 256 slots, 200 founders, 5x5x3 patch + 4 scalars = 79
# inputs, MLP 79 -> 32 -> 32 -> 6, FP32, automatic eating.
SMALL = dict(
    name="small-64x64-256slots-79-32-32-6-fp32",
    side=64, slots=256, init_alive=200, patch_k=5, n_scalars=4, hidden=32,
    n_actions=6, precision="fp32", flags=("auto_eat", "rotate_obs"), seed=0,
    sigma=0.02, food_density=0.1, regrow_p=0.01, wall_density=0.0, steps=100,
    **_COMMON)

# 512x512, 16,384 slots, 12,000 founders, 11x11x3 patch + 8 scalars = 371
# inputs, MLP 371 -> 64 -> 64 -> 9, FP32, 2% walls.
MID = dict(
    name="mid-512x512-16384slots-371-64-64-9-fp32",
    side=512, slots=16384, init_alive=12000, patch_k=11, n_scalars=8, hidden=64,
    n_actions=9, precision="fp32", flags=("rotate_obs",), seed=0, sigma=0.01,
    food_density=0.05, regrow_p=0.005, wall_density=0.02, steps=1000, **_COMMON)

# 1024x1024, 65,536 slots, 50,000 founders, same MLP, weights streamed as BF16.
PAPER = dict(MID, name="paper-1024x1024-65536slots-371-64-64-9-bf16",
             side=1024, slots=65536, init_alive=50000, precision="bf16")

# 2048x2048, 262,144 slots, 200,000 founders, 15x15x3 + 8 = 683 inputs,
# MLP 683 -> 128 -> 128 -> 9, FP8 e4m3 with a per-row scale.
LARGE = dict(MID, name="large-2048x2048-262144slots-683-128-128-9-fp8",
             side=2048, slots=262144, init_alive=200000, patch_k=15, hidden=128,
             precision="fp8", steps=500)

# The paper's own policy form (Sec. 3.3) on the paper-scale world: separate
# input linears for the vision patch, the internal scalars and the compass,
# summed; two hidden ReLU layers of 64; an unbiased head; an evolvable
# softmax temperature; weights streamed as BF16.
PAPER_FORM = dict(PAPER, name="paperform-1024x1024-65536slots-RCV-2x64-bf16",
                  policy_form="paper", n_hidden=2)

# The paper's rule set (Sec. 3.2 "Resources and Agent Health", "Actions";
# App. F.7-F.8), one resource: HP in quarter points (10 HP maximum, children
# start at 5 HP, the full attack takes 10 HP, healing 1 HP per step for one
# energy unit), age damage floor(age / 1000) quarter points per step, 2 HP
# per step while starving; actions rest, rotate cw / ccw, forward, attack
# (the 3x3 square in front), eat (one bite of up to 20 energy, stomach 400),
# reproduce (at >= 200 energy, handing 100 to the child).
PAPER_RULES = dict(rules="paper", n_actions=7, hp_max=40, hp_child=20, attack_damage=40,
                   heal_rate=4, heal_cost=1, age_div=1000, starve_damage=8, e_act=1,
                   e_cap=400, e_child=100)

# The paper's rules and policy form together on the paper-scale world
# (RCV+A agents: vision, compass, internal sensors; attack enabled).  The
# vision patch is rendered in colour (Sec. 3.2), each agent showing its
# evolvable colour trait (Sec. 3.3); the window is centred on the agent
# ("Around", the paper's main setting, App. F.6).
ECOLOGY = dict(PAPER_FORM, name="ecology-1024x1024-65536slots-RCV+A-rgb-2x64-7act-bf16",
               vision="rgb", view="around", **PAPER_RULES)

# The terrain rules (Sec. 3.2 "Terrain", "Resources and Agent Health"; App.
# F.2): the paper rules plus a rock layer with sea level 32, water that
# flows downhill, and biomass.  Agents carry water (60 at birth of a
# founder, 1 spent per step back onto their cell, drinks of 10, capacity
# 100) and biomass (a body of 10; children get a body of 10 from their
# parent; bites of 5, capacity 50).  A quarter of the cells start as
# biomass sites of 20 (App. F.2: initial site density 1/4), on which energy
# grows at 0.01 per biomass unit per step (App. F.2: photosynthesis rate
# 0.01; 655 / 2^16), up to 100 per cell; there is no random regrowth.
# Vision: RGB plus the elevation channel; 16 scalars (internal and
# external sensors of all three resources).
TERRAIN_RULES = dict(PAPER_RULES, rules="terrain", n_actions=9, n_scalars=16, vision="rgb",
                     sea_level=32, w_init=60, w_metab=1, w_bite=10, w_cap=100, w_child=30,
                     heal_water=1, b_body=10, b_child=10, b_bite=5, b_cap=50, b_site=20,
                     biomass_density=0.25, photo_q16=655, res_cap=100, regrow_p=0.0)

# The terrain rules on the paper-scale world, "beach" terrain.
TERRAIN = dict(ECOLOGY, name="terrain-beach-1024x1024-65536slots-RCV+A-2x64-9act-bf16",
               terrain="beach", **TERRAIN_RULES)

WORKLOADS = {"small": SMALL, "mid": MID, "paper": PAPER, "large": LARGE,
             "paperform": PAPER_FORM, "ecology": ECOLOGY, "terrain": TERRAIN}

TERRAINS = ("ocean", "beach", "island", "lake", "isthmus", "channel")


def terrain(preset: str, side: int, seed: int = 0) -> np.ndarray:
    """A synthetic rock layer (int32 heights, [side * side], row-major) for
    the paper's named terrains (Sec. 3.2 "Terrain": Ocean, Beach, Island,
    Lake, Isthmus, Channel), whose generator the paper does not give.  A
    base shape in [0, 64] against sea level 32 -- ocean: all below; beach:
    rising from west to east; island: a central hill; lake: a central
    basin; isthmus: a north-south ridge between two seas; channel: an
    east-west trough through land -- plus value noise of amplitude 8
    (uniform draws of numpy's seeded generator on a 16-cell lattice,
    bilinearly interpolated), rounded and clipped to [0, 96].  An input
    generator: none of the simulator's arithmetic."""
    u = (np.arange(side) + 0.5) / side
    X, Y = np.meshgrid(u, u)           # X: column (east), Y: row (south)
    r = np.hypot(X - 0.5, Y - 0.5)
    base = {
        "ocean": np.full_like(X, 16.0),
        "beach": 64.0 * X,
        "island": 64.0 - 128.0 * r,
        "lake": 128.0 * r,
        "isthmus": 64.0 - 256.0 * np.abs(X - 0.5),
        "channel": 256.0 * np.abs(Y - 0.5),
    }[preset]
    rng = np.random.default_rng(seed)
    n = side // 16 + 2
    lattice = rng.uniform(-8.0, 8.0, size=(n, n))
    g = np.arange(side) / 16.0
    i0 = np.floor(g).astype(int)
    f = g - i0
    rows = lattice[i0] * (1 - f)[:, None] + lattice[i0 + 1] * f[:, None]
    noise = rows[:, i0] * (1 - f)[None, :] + rows[:, i0 + 1] * f[None, :]
    rock = np.clip(np.rint(np.maximum(base, 0.0) + noise), 0, 96).astype(np.int32)
    return rock.ravel()


def get(key: str, **overrides) -> dict:
    """A copy of a named workload with fields overridden.  A workload with a
    terrain preset gets its rock layer (key "rock") for its side and seed."""
    w = copy.deepcopy(WORKLOADS[key])
    w.update(overrides)
    if w.get("terrain") and "rock" not in overrides:
        w["rock"] = terrain(w["terrain"], w["side"], w.get("seed", 0))
    return w


def scaled(base: str, side: int, slots: int, init_alive: int, **overrides) -> dict:
    """A named workload's rules and MLP on a different grid / population."""
    w = get(base, side=side, slots=slots, init_alive=init_alive)
    w["name"] = "%s-%dx%d-%dslots" % (base, side, side, slots)
    w.update(overrides)
    if w.get("terrain") and "rock" not in overrides:
        w["rock"] = terrain(w["terrain"], w["side"], w.get("seed", 0))
    return w


def batched(n_envs: int = 64, seed: int = 0, base_seed: int = 0,
            precision: str = "bf16") -> list:
    """Independent environments of uneven size (the many-small-worlds shape of
    the paper's self-averaging study, App. F.3): sides uniform over
    {128, 256, 512, 1024}; founders lognormal with median 4,096 and log-sd 1,
    clipped to [512, 32768] and to a quarter of the cells; slots = founders
    * 1.3 rounded up to a multiple of 256.  Environment e uses seed
    base_seed + e.  Sizes come from numpy's seeded generator (an input
    generator, not a draw of the method)."""
    rng = np.random.default_rng(seed)
    envs = []
    for e in range(n_envs):
        side = int(rng.choice([128, 256, 512, 1024]))
        n = int(round(float(np.exp(rng.normal(np.log(4096.0), 1.0)))))
        n = max(512, min(32768, n))
        n = min(n, side * side // 4)
        slots = ((int(np.ceil(n * 1.3)) + 255) // 256) * 256
        envs.append(get("mid", side=side, slots=slots, init_alive=n, seed=base_seed + e,
                        precision=precision,
                        name="batched-env%d-%dx%d-%dslots" % (e, side, side, slots)))
    return envs
