"""Pins for the oracle's terrain rule set (not GPU).

Sec. 3.2 "Terrain" (a rock layer, water filling the cells below sea level
and flowing downhill) and "Resources and Agent Health" (water, energy and
biomass; spent water returns to the landscape; biomass is conserved and
needed to exist and to reproduce; energy grows on free biomass), App. F.2
(photosynthesis rate, initial biomass site density).

* Water flow, hand-worked: a single column of water spreading to the first
  of its equal neighbours; two cells draining into one lower cell; a wall
  that neither sends nor receives; a cell one unit above its neighbour
  that stays put (a fifth of the drop rounds to zero).
* Water flow, invariants on random terrains: total water conserved, no
  negative water, none on walls, the highest surface never rises and the
  lowest never sinks, a level lake stays level, and water on a slope ends
  in the basin.
* Photosynthesis, closed form: after t steps a cell with B biomass and no
  eating holds floor(t * B * q / 2^16) energy (q = photo_q16), capped at
  res_cap.
* Hand-worked agent scenarios: drink and eat-biomass bites with their
  capacities; spent water goes back onto the cell; thirst costs HP;
  healing needs water; death drops energy, water and biomass; reproduction
  needs the action, energy, b_body + b_child biomass and w_child water, and
  hands over e_child, w_child and b_child.
* Reset: water = sea_level - rock below sea level; biomass sites are the
  Bernoulli draws of stream BIOMASS; founders carry w_init and b_body.
* Observation: 4 channels (RGB of the cell's resources, elevation
  difference d / (|d| + 16)) and the 16 scalars, hand-worked.
* Ledgers every step of random runs: water and biomass conserved; energy
  in stomachs and on cells changes only by photosynthesis, regrowth,
  action costs and healing; food == (energy on the cell > 0).
"""
import numpy as np
import pytest

import oracle
from paper_2510_18221_gb300 import workloads
from tests import scenarios
from tests.scenarios import cell

N_, E_, S_, W_ = 0, 1, 2, 3
REST, CW, CCW, FWD, ATK, EAT, REPRO, DRINK, EAT_BIO = range(9)
ST_BIOMASS = 13


def world(side=6, slots=8, **kw):
    rules = dict(workloads.TERRAIN_RULES)
    rules.update(kw)
    return scenarios.empty_world(scenarios.tiny_cfg(side=side, slots=slots, **rules))


def put(o, slot, x, y, facing=N_, energy=100, hp=40, water=50, bio=10, age=0):
    scenarios.place(o, slot, x, y, facing=facing, energy=energy)
    o.hp[slot] = hp
    o.age[slot] = age
    o.a_water[slot] = water
    o.a_bio[slot] = bio


def acts(o, mapping, default=REST):
    return scenarios.actions(o, mapping, default=default)


def grid(o, a):
    return a.reshape(o.side, o.side)


# ----------------------------------------------------------------------------- flow, hand-worked

def test_flow_single_column_goes_to_the_first_lowest_neighbour():
    o = world(side=5)
    o.water[cell(o, 2, 2)] = 10
    o.water_flow()
    # all four neighbours are at surface 0: N wins the tie and gets 10 // 5
    assert o.water[cell(o, 2, 2)] == 8 and o.water[cell(o, 2, 1)] == 2
    assert o.water.sum() == 10
    o.water_flow()
    # (2,2): surface 8, N is at 2, E/S/W at 0 -> E gets 8 // 5 = 1;
    # (2,1): surface 2, lowest neighbour N (2,0) at 0, but 2 // 5 = 0: stays
    assert o.water[cell(o, 2, 2)] == 7 and o.water[cell(o, 3, 2)] == 1
    assert o.water[cell(o, 2, 0)] == 0 and o.water[cell(o, 2, 1)] == 2


def test_flow_two_cells_drain_into_one_lower_cell():
    o = world(side=5)
    o.rock[:] = 50
    o.rock[cell(o, 2, 2)] = 0
    o.water[cell(o, 1, 2)] = 5          # surface 55, lowest neighbour (2,2) at 0
    o.water[cell(o, 3, 2)] = 20         # surface 70
    o.water_flow()
    assert o.water[cell(o, 1, 2)] == 0          # min(5, 55 // 5)
    assert o.water[cell(o, 3, 2)] == 6          # 20 - min(20, 70 // 5)
    assert o.water[cell(o, 2, 2)] == 5 + 14
    assert o.water.sum() == 25


def test_flow_walls_neither_send_nor_receive_and_small_drops_stay():
    o = world(side=5)
    o.wall[cell(o, 2, 1)] = 1
    o.wall[cell(o, 3, 2)] = 1
    o.wall[cell(o, 2, 3)] = 1
    o.water[cell(o, 2, 2)] = 10          # only W (1,2) is open
    o.water[cell(o, 0, 0)] = 1           # one unit above its neighbours: stays
    o.water_flow()
    assert o.water[cell(o, 1, 2)] == 2 and o.water[cell(o, 2, 2)] == 8
    assert o.water[cell(o, 0, 0)] == 1
    assert not (o.water * o.wall).any()


def _random_terrain_oracle(seed, side=24):
    rng = np.random.default_rng(seed)
    o = world(side=side)
    o.rock[:] = rng.integers(0, 60, side * side)
    o.wall[:] = (rng.random(side * side) < 0.1).astype(np.uint8)
    o.water[:] = np.where(o.wall == 1, 0, rng.integers(0, 40, side * side))
    return o


@pytest.mark.parametrize("seed", range(8))
def test_flow_invariants_on_random_terrain(seed):
    o = _random_terrain_oracle(seed)
    total = int(o.water.sum())
    open_ = o.wall == 0
    for _ in range(60):
        surf = (o.rock + o.water)[open_]
        hi, lo = int(surf.max()), int(surf.min())
        o.water_flow()
        surf = (o.rock + o.water)[open_]
        assert int(o.water.sum()) == total
        assert (o.water >= 0).all() and not (o.water * o.wall).any()
        assert int(surf.max()) <= hi and int(surf.min()) >= lo


def test_level_lake_stays_level():
    o = world(side=8)
    o.rock[:] = np.arange(64) % 7
    o.water[:] = 20 - o.rock           # every surface at 20
    before = o.water.copy()
    o.water_flow()
    assert np.array_equal(o.water, before)


def test_water_runs_down_a_slope_into_the_basin():
    side = 16
    o = world(side=side)
    x = np.arange(side * side) % side
    o.rock[:] = np.where(x < 4, 0, 8 * (x - 3))   # basin in columns 0..3, slope east
    o.water[:] = np.where(x >= 4, 3, 0)
    total = int(o.water.sum())
    for _ in range(400):
        o.water_flow()
    assert int(o.water.sum()) == total
    # a fixed point: one more step moves nothing, and no wet cell has a
    # neighbour whose surface is 5 or more below its own
    before = o.water.copy()
    o.water_flow()
    assert np.array_equal(o.water, before)
    surf = (o.rock + o.water).reshape(side, side)
    wet = (o.water > 0).reshape(side, side)
    for sh, ax in ((1, 0), (-1, 0), (1, 1), (-1, 1)):
        drop = surf - np.roll(surf, sh, axis=ax)
        assert not (wet & (drop >= 5)).any()
    # so water stays only in the basin and at the foot of the slope (each
    # slope cell above it drops 8 in rock to its western neighbour)
    assert not o.water[x >= 6].any()
    assert int(o.water[x < 4].sum()) > total // 2


# ----------------------------------------------------------------------------- photosynthesis

def test_photosynthesis_closed_form_and_cap():
    o = world(side=6, photo_q16=655, res_cap=100)
    for B, xy in ((20, (1, 1)), (7, (3, 3)), (1, (5, 0))):
        o.bio[cell(o, *xy)] = B
    photo = 0
    for t in range(1, 301):
        st, _ = o.transition(acts(o, {}))
        photo += st["photo"]
        for B, xy in ((20, (1, 1)), (7, (3, 3)), (1, (5, 0))):
            want = min((t * B * 655) >> 16, 100)
            assert o.res[cell(o, *xy)] == want, (t, B)
            assert o.food[cell(o, *xy)] == (1 if want > 0 else 0)
    assert photo == int(o.res.sum())


# ----------------------------------------------------------------------------- agents

def test_drink_and_eat_biomass_bites_and_capacities():
    o = world(w_metab=0, heal_rate=0)
    put(o, 0, 1, 1, water=95, bio=10)
    put(o, 1, 3, 3, water=20, bio=48)
    o.water[cell(o, 1, 1)] = 30
    o.bio[cell(o, 3, 3)] = 4
    st, _ = o.transition(acts(o, {0: DRINK, 1: EAT_BIO}))
    assert o.a_water[0] == 100 and st["drunk"] == 5          # capacity 100
    assert o.a_bio[1] == 50 and o.bio[cell(o, 3, 3)] == 2     # capacity 50
    assert st["bio_eaten"] == 2


def test_spent_water_returns_to_the_cell_and_thirst_costs_hp():
    o = world(heal_rate=0, w_metab=2)
    o.rock[:] = 90                                          # dry land, high
    put(o, 0, 1, 1, water=10)
    put(o, 1, 4, 4, water=1, hp=40)
    st, _ = o.transition(acts(o, {}))
    assert o.a_water[0] == 8
    assert o.a_water[1] == 0 and o.hp[1] == 32 and st["thirsty"] == 1
    assert st["water_spent"] == 3
    assert int(o.water.sum()) == 3                          # on the cells (and flowing)


def test_healing_needs_and_spends_water():
    o = world(w_metab=0, heal_water=2)
    put(o, 0, 1, 1, hp=30, water=2)
    put(o, 1, 4, 4, hp=30, water=1)
    st, _ = o.transition(acts(o, {}))
    assert (o.hp[0], o.hp[1]) == (34, 30)
    assert o.a_water[0] == 0 and st["heals"] == 1 and st["water_spent"] == 2


def test_death_drops_energy_water_and_biomass():
    o = world(w_metab=0)
    o.rock[:] = 90
    put(o, 0, 2, 4, facing=N_)
    put(o, 1, 2, 3, energy=50, water=33, bio=17)
    st, _ = o.transition(acts(o, {0: ATK}))
    c = cell(o, 2, 3)
    assert not o.alive[1]
    assert o.res[c] == 49 and o.bio[c] == 17
    assert st["dead_water"] == 33 and st["dead_bio"] == 17
    assert o.a_water[1] == 0 and o.a_bio[1] == 0
    assert int(o.water.sum()) == 33


def test_reproduction_needs_biomass_and_water_and_hands_them_over():
    o = world(slots=6, w_metab=0, e_repro=150, e_child=60)
    o.rock[:] = 90
    put(o, 0, 1, 1, facing=N_, energy=300, water=80, bio=20)     # enough
    put(o, 1, 4, 1, facing=N_, energy=300, water=80, bio=19)     # biomass short
    put(o, 2, 1, 4, facing=N_, energy=300, water=29, bio=40)     # water short
    st, births = o.transition(acts(o, {0: REPRO, 1: REPRO, 2: REPRO}))
    assert births == [(0, 3)]
    assert (o.a_water[0], o.a_bio[0], o.energy[0]) == (50, 10, 300 - 2 - 60)
    assert (o.a_water[3], o.a_bio[3], o.energy[3]) == (30, 10, 60)


# ----------------------------------------------------------------------------- reset, observation

def test_reset_water_biomass_and_founders():
    w = workloads.scaled("terrain", 32, 200, 150)
    o = oracle.Oracle(w)
    o.reset()
    open_ = o.wall == 0
    np.testing.assert_array_equal(o.water, np.where(open_, np.maximum(0, 32 - o.rock), 0))
    for c in (0, 5, 77, 1023):
        r = oracle.philox((c >> 2, 0, 0, 0), (w["seed"], ST_BIOMASS))[c & 3]
        want = 20 if (open_[c] and r < oracle.threshold(0.25)) else 0
        assert o.bio[c] == want
    assert (o.a_water[:150] == 60).all() and (o.a_bio[:150] == 10).all()
    assert (o.a_water[150:] == 0).all() and (o.a_bio[150:] == 0).all()
    assert (o.photo == 0).all()


def test_observation_channels_and_scalars():
    o = world(side=5, patch_k=3)
    o.rock[:] = 40
    put(o, 0, 2, 2, facing=N_, energy=50, hp=30, water=25, bio=10, age=1000)
    o.colour[0] = (0.25, 0.5, 0.75)
    c = cell(o, 2, 1)                         # the cell ahead
    o.rock[c] = 48
    o.bio[c], o.res[c], o.water[c] = 5, 20, 30
    o.food[c] = 1
    here = cell(o, 2, 2)
    o.water[here], o.bio[here], o.res[here] = 10, 15, 0
    x = o.observe(0)
    ahead = x[(0 * 3 + 1) * 4:(0 * 3 + 2) * 4]
    np.testing.assert_allclose(ahead, [5 / 10, 20 / 40, 30 / 40, 8 / 24], rtol=0, atol=1e-15)
    me = x[(1 * 3 + 1) * 4:(1 * 3 + 2) * 4]
    np.testing.assert_allclose(me, [0.25, 0.5, 0.75, 0.0], rtol=0, atol=1e-15)
    base = 4 * 9
    want = [50 / 200, 1, 0, 0, 0, 30 / 40, 1000 / 2000, 0.0, 25 / 100, 10 / 50,
            10 / 20, 15 / 20, 0, 0, 0, 0]
    np.testing.assert_allclose(x[base:], want, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- ledgers

@pytest.mark.parametrize("preset,over", [
    ("beach", dict(e_repro=90, e_child=30, e_init=100, w_init=30)),
    ("island", dict(e_repro=50, e_child=30, e_init=60, w_init=20, w_child=10, attack_damage=10)),
    ("lake", dict(e_repro=80, e_child=20, policy_form="plain", n_hidden=1, patch_k=5,
                  hidden=32, heal_water=2, w_metab=2)),
])
def test_ledgers_every_step(preset, over):
    over = dict(over, b_child=5, b_bite=10)   # one bite of biomass makes a parent
    o = oracle.Oracle(workloads.scaled("terrain", 40, 700, 500, terrain=preset, **over))
    o.reset()
    c = o.cfg
    water = int(o.water.sum() + o.a_water.sum())
    bio = int(o.bio.sum() + o.a_bio.sum())
    seen = dict(births=0, deaths=0, drunk=0, bio_eaten=0, photo=0, thirsty=0, heals=0,
                dead_water=0, dead_bio=0)
    for _ in range(40):
        alive = o.alive == 1
        e0 = int(o.energy[alive].sum()) + int(o.res.sum())
        _, st, _ = o.step_once()
        for k in seen:
            seen[k] += st[k]
        alive = o.alive == 1
        assert int(o.water.sum()) + int(o.a_water[alive].sum()) == water
        assert int(o.bio.sum()) + int(o.a_bio[alive].sum()) == bio
        assert (o.a_water[~alive] == 0).all() and (o.a_bio[~alive] == 0).all()
        e1 = int(o.energy[alive].sum()) + int(o.res.sum())
        assert e1 - e0 == (st["photo"] + c["e_food"] * st["regrown"] - st["metab_paid"]
                           - c["heal_cost"] * st["heals"])
        assert st["water_cells"] + st["water_agents"] == water
        assert st["bio_cells"] + st["bio_agents"] == bio
        assert np.array_equal(o.food, (o.res > 0).astype(np.uint8))
        assert (o.water >= 0).all() and (o.bio >= 0).all() and not (o.water * o.wall).any()
        assert ((o.a_water[alive] <= c["w_cap"]) & (o.a_bio[alive] <= c["b_cap"])).all()
        assert (o.a_bio[alive] >= c["b_child"]).all()
    assert all(v > 0 for v in seen.values()), seen
