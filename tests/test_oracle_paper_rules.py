"""Pins for the oracle's paper rule set (not GPU).

Sec. 3.2 "Resources and Agent Health" and "Actions", App. F.7 (attack
strength) and App. F.8 (agent HP), with one resource (energy lying on
cells).  HP is in quarter points.

* Hand-worked scenarios: rotate clockwise / counter-clockwise, move forward
  (free, wall, contested), the 3x3 attack square in front for each facing
  and across the torus seam, damage adding up over attackers, a full attack
  killing and the victim's energy dropped on its cell, starvation, age
  damage, healing and its cap, eating in bites up to the stomach capacity,
  reproduction only through the reproduce action, regrowth only on empty
  cells, and the observation's internal / external scalars.
* Brute force: on random tiny worlds, every agent's HP loss equals
  attack_damage times the number of attackers whose square (recomputed here
  from the geometry) covers it.
* Ledgers every step of random runs: energy in stomachs plus energy on
  cells changes only by regrowth, action costs and healing; the food map is
  exactly the cells holding energy; population; HP in (0, hp_max]; energy
  in [0, e_cap]; age = steps survived.
"""
import numpy as np
import pytest

import oracle
from paper_2510_18221_gb300 import workloads
from tests import scenarios
from tests.scenarios import cell

N_, E_, S_, W_ = 0, 1, 2, 3
DX = {N_: 0, E_: 1, S_: 0, W_: -1}
DY = {N_: -1, E_: 0, S_: 1, W_: 0}
ST_MOVE, ST_BIRTH = 7, 9
REST, CW, CCW, FWD, ATK, EAT, REPRO = range(7)


def claim(o, stream, slot):
    r = oracle.philox((int(o.step[0]), slot, 0, 0), (o.cfg["seed"], stream))[0]
    return (r << 32) | (0xFFFFFFFF - slot)


def world(side=7, slots=8, **kw):
    rules = dict(workloads.PAPER_RULES)
    rules.update(kw)
    return scenarios.empty_world(scenarios.tiny_cfg(side=side, slots=slots, **rules))


def put(o, slot, x, y, facing=N_, energy=100, hp=40, age=0):
    scenarios.place(o, slot, x, y, facing=facing, energy=energy)
    o.hp[slot] = hp
    o.age[slot] = age


def acts(o, mapping, default=REST):
    return scenarios.actions(o, mapping, default=default)


def drop_energy(o, x, y, amount):
    o.res[cell(o, x, y)] = amount
    o.food[cell(o, x, y)] = 1 if amount > 0 else 0


# ----------------------------------------------------------------------------- moves

def test_rotations():
    o = world()
    put(o, 0, 1, 1, facing=N_)
    put(o, 1, 4, 4, facing=N_)
    put(o, 2, 2, 5, facing=W_)
    o.transition(acts(o, {0: CW, 1: CCW, 2: CW}))
    assert (o.facing[0], o.facing[1], o.facing[2]) == (E_, W_, N_)
    assert (o.x[0], o.y[0]) == (1, 1)


def test_forward_free_wall_and_seam():
    o = world()
    put(o, 0, 1, 1, facing=E_)
    put(o, 1, 3, 3, facing=S_)
    put(o, 2, 0, 5, facing=W_)                    # wraps to x = 6
    o.wall[cell(o, 3, 4)] = 1
    st, _ = o.transition(acts(o, {0: FWD, 1: FWD, 2: FWD}))
    assert (o.x[0], o.y[0]) == (2, 1)
    assert (o.x[1], o.y[1]) == (3, 3)
    assert (o.x[2], o.y[2]) == (6, 5)
    assert st["moves"] == 2 and st["move_blocked"] == 1
    assert o.facing[0] == E_ and o.facing[1] == S_


def test_forward_contest_highest_claim_or_cancel_all():
    for flags in (("rotate_obs",), ("rotate_obs", "cancel_all")):
        o = world(flags=flags)
        put(o, 0, 1, 2, facing=E_)
        put(o, 1, 3, 2, facing=W_)
        winner = 0 if claim(o, ST_MOVE, 0) > claim(o, ST_MOVE, 1) else 1
        st, _ = o.transition(acts(o, {0: FWD, 1: FWD}))
        if "cancel_all" in flags:
            assert o.occ[cell(o, 2, 2)] == -1 and st["move_lost"] == 2
        else:
            assert o.occ[cell(o, 2, 2)] == winner and st["moves"] == 1


# ----------------------------------------------------------------------------- attack

@pytest.mark.parametrize("facing", [N_, E_, S_, W_])
def test_attack_square_in_front(facing):
    """Every cell holds an agent; only the one in the middle attacks.  The
    nine agents 1..3 cells ahead and at most one to the side lose HP."""
    side = 7
    o = world(side=side, slots=side * side, attack_damage=10, heal_rate=0)
    for y in range(side):
        for x in range(side):
            put(o, y * side + x, x, y, facing=N_)
    me = 3 * side + 3
    o.facing[me] = facing
    st, _ = o.transition(acts(o, {me: ATK}))
    right = (facing + 1) % 4
    hit = set()
    for fwd in (1, 2, 3):
        for lat in (-1, 0, 1):
            x = (3 + fwd * DX[facing] + lat * DX[right]) % side
            y = (3 + fwd * DY[facing] + lat * DY[right]) % side
            hit.add(y * side + x)
    for s in range(side * side):
        assert o.hp[s] == (30 if s in hit else 40), s
    assert st["attacks"] == 1 and st["attack_hits"] == 9 and st["damage"] == 90


def test_attack_wraps_across_the_seam():
    o = world(side=6, attack_damage=10, heal_rate=0)
    put(o, 0, 0, 0, facing=N_)
    put(o, 1, 5, 5)           # one ahead (y = -1 -> 5), one to the left (x = -1 -> 5)
    put(o, 2, 1, 3)           # three ahead (y = -3 -> 3), one to the right
    put(o, 3, 0, 2)           # four ahead: outside
    o.transition(acts(o, {0: ATK}))
    assert (o.hp[1], o.hp[2], o.hp[3]) == (30, 30, 40)


def test_damage_adds_over_attackers_and_full_attack_kills_with_drop():
    o = world(attack_damage=10, heal_rate=0)
    put(o, 0, 3, 5, facing=N_)
    put(o, 1, 2, 5, facing=N_)
    put(o, 2, 3, 3, energy=77)        # in both squares
    o.transition(acts(o, {0: ATK, 1: ATK}))
    assert o.hp[2] == 20 and o.alive[2]

    o = world()                        # attack_damage = hp_max: a kill
    put(o, 0, 3, 5, facing=N_)
    put(o, 1, 3, 4, energy=77)
    st, _ = o.transition(acts(o, {0: ATK, 1: FWD}))
    # the victim moved first (to (3, 3), still in the square), paid 2 for
    # its action, died, and dropped the rest on its cell
    assert not o.alive[1] and o.occ[cell(o, 3, 3)] == -1
    assert o.res[cell(o, 3, 3)] == 75 and o.food[cell(o, 3, 3)] == 1
    assert st["deaths"] == 1 and st["dead_energy"] == 75 and st["food_refilled"] == 1
    assert o.energy[1] == 0 and o.hp[1] == 0


def test_drop_onto_a_cell_that_already_holds_energy():
    o = world()
    put(o, 0, 3, 5, facing=N_)
    put(o, 1, 3, 4, energy=50)
    drop_energy(o, 3, 4, 15)
    st, _ = o.transition(acts(o, {0: ATK}))
    assert o.res[cell(o, 3, 4)] == 15 + 49 and st["food_refilled"] == 0


# ----------------------------------------------------------------------------- health

def test_action_costs_and_starvation():
    o = world(heal_rate=0)
    put(o, 0, 1, 1, energy=10)
    put(o, 1, 3, 3, energy=10)
    put(o, 2, 5, 5, energy=1, hp=40)      # cannot pay 2 for a rotation
    put(o, 3, 1, 5, energy=1, hp=8)       # starving kills at 8 quarter points
    st, _ = o.transition(acts(o, {1: CW, 2: CW, 3: CW}))
    assert (o.energy[0], o.energy[1]) == (9, 8)
    assert o.energy[2] == 0 and o.hp[2] == 32
    assert not o.alive[3]
    assert st["starved"] == 2 and st["metab_paid"] == 1 + 2 + 1 + 1


def test_age_damage_and_ageing():
    o = world(heal_rate=0)
    put(o, 0, 1, 1, age=2500)     # floor(2500 / 1000) = 2
    put(o, 1, 3, 3, age=999)
    o.transition(acts(o, {}))
    assert (o.hp[0], o.hp[1]) == (38, 40)
    assert (o.age[0], o.age[1]) == (2501, 1000)
    o.transition(acts(o, {}))
    assert o.hp[1] == 39


def test_healing_cap_and_cost():
    o = world()
    put(o, 0, 1, 1, hp=30, energy=10)
    put(o, 1, 3, 3, hp=38, energy=10)
    put(o, 2, 5, 5, hp=40, energy=10)
    put(o, 3, 1, 5, hp=30, energy=1)      # pays 1 to rest, nothing left to heal
    st, _ = o.transition(acts(o, {}))
    assert (o.hp[0], o.hp[1], o.hp[2], o.hp[3]) == (34, 40, 40, 30)
    assert (o.energy[0], o.energy[1], o.energy[2], o.energy[3]) == (8, 8, 9, 0)
    assert st["heals"] == 2


def test_damage_then_heal_in_one_step():
    o = world(attack_damage=10)
    put(o, 0, 3, 5, facing=N_)
    put(o, 1, 3, 4, energy=50)
    o.transition(acts(o, {0: ATK}))
    assert o.hp[1] == 40 - 10 + 4 and o.energy[1] == 50 - 1 - 1


# ----------------------------------------------------------------------------- eat

def test_eat_in_bites_up_to_capacity():
    o = world(heal_rate=0)
    put(o, 0, 2, 2, energy=100)
    drop_energy(o, 2, 2, 50)
    for want_res, want_e in ((30, 100 + 20 - 2), (10, 118 + 20 - 2), (0, 136 + 10 - 2)):
        st, _ = o.transition(acts(o, {0: EAT}))
        assert o.res[cell(o, 2, 2)] == want_res and o.energy[0] == want_e
    assert o.food[cell(o, 2, 2)] == 0 and st["food_emptied"] == 1 and st["eaten_energy"] == 10
    o = world(heal_rate=0)
    put(o, 0, 2, 2, energy=395)
    drop_energy(o, 2, 2, 20)
    st, _ = o.transition(acts(o, {0: EAT}))
    assert o.energy[0] == 400 - 2 and o.res[cell(o, 2, 2)] == 15 and st["eaten"] == 1
    st, _ = o.transition(acts(o, {0: EAT}))    # 398 -> bite of 2
    assert o.res[cell(o, 2, 2)] == 13


def test_no_eat_without_the_action():
    o = world()
    put(o, 0, 2, 2)
    drop_energy(o, 2, 2, 20)
    o.transition(acts(o, {0: FWD}))
    o.transition(acts(o, {0: CW}))
    assert o.res[cell(o, 2, 2)] == 20


# ----------------------------------------------------------------------------- reproduce

def test_reproduce_only_with_the_action_and_enough_energy():
    o = world(slots=6)
    put(o, 0, 2, 2, facing=N_, energy=300)
    put(o, 1, 4, 4, facing=E_, energy=300)
    put(o, 2, 1, 5, facing=N_, energy=201)   # 201 - 2 < 200 after paying
    st, births = o.transition(acts(o, {0: REPRO, 2: REPRO}))
    assert births == [(0, 3)]
    assert (o.x[3], o.y[3]) == (2, 3) and o.facing[3] == N_
    assert o.energy[0] == 300 - 2 - 100 and o.energy[3] == 100
    assert o.hp[3] == 20 and o.age[3] == 0 and o.parent[3] == 0 and o.birth_step[3] == 0
    assert o.energy[1] == 299 and o.energy[2] == 199
    np.testing.assert_array_equal(o.master[3], o.mutate(0, 0, o.master[0]))


def test_two_reproducers_one_cell():
    o = world(slots=6)
    put(o, 0, 2, 1, facing=N_, energy=300)   # behind: (2, 2)
    put(o, 1, 2, 3, facing=S_, energy=300)   # behind: (2, 2)
    w = 0 if claim(o, ST_BIRTH, 0) > claim(o, ST_BIRTH, 1) else 1
    st, births = o.transition(acts(o, {0: REPRO, 1: REPRO}))
    assert births == [(w, 2)] and o.occ[cell(o, 2, 2)] == 2


# ----------------------------------------------------------------------------- regrowth, observation

def test_regrowth_only_on_empty_cells():
    o = world(regrow_p=1.0)
    drop_energy(o, 1, 1, 7)
    o.wall[cell(o, 2, 2)] = 1
    st, _ = o.transition(acts(o, {}))
    assert o.res[cell(o, 1, 1)] == 7
    assert o.res[cell(o, 2, 2)] == 0
    assert o.res[cell(o, 3, 3)] == 20
    assert st["regrown"] == 49 - 2 and st["res_total"] == 7 + 20 * 47


@pytest.mark.parametrize("n_scalars", [4, 8])
def test_observation_scalars(n_scalars):
    o = world(n_scalars=n_scalars)
    put(o, 0, 2, 2, facing=S_, energy=50, hp=30, age=3000)
    drop_energy(o, 2, 2, 60)
    x = o.observe(0)
    base = 3 * 3 * 3
    want = [50 / 200]
    if n_scalars == 8:
        want += [0, 0, 1, 0]
    want += [30 / 40, 3000 / 4000, 60 / 80]
    np.testing.assert_allclose(x[base:], want, rtol=0, atol=1e-15)
    centre = (1 * 3 + 1) * 3
    assert x[centre] == 1.0 and x[centre + 1] == 1.0    # food and self on the cell


def test_reset_paper_rules():
    o = oracle.Oracle(workloads.scaled("ecology", 64, 600, 400))
    o.reset()
    assert np.array_equal(o.res, np.where(o.food == 1, 20, 0))
    assert (o.hp[:400] == 40).all() and (o.hp[400:] == 0).all() and (o.age == 0).all()


# ----------------------------------------------------------------------------- brute force

def _square_cells(x, y, f, side):
    right = (f + 1) % 4
    return {((x + a * DX[f] + b * DX[right]) % side, (y + a * DY[f] + b * DY[right]) % side)
            for a in (1, 2, 3) for b in (-1, 0, 1)}


@pytest.mark.parametrize("trial", range(30))
def test_attack_damage_brute_force(trial):
    rng = np.random.default_rng(1000 + trial)
    side = int(rng.integers(5, 9))
    n = int(rng.integers(2, side * side // 2))
    o = world(side=side, slots=n, attack_damage=3, heal_rate=0)
    cells = rng.choice(side * side, n, replace=False)
    for s, c in enumerate(cells):
        put(o, s, int(c % side), int(c // side), facing=int(rng.integers(4)))
    act = rng.choice([REST, ATK, CW, CCW], n).astype(np.uint8)
    facing_after = [(int(o.facing[s]) + (1 if act[s] == CW else 3 if act[s] == CCW else 0)) % 4
                    for s in range(n)]
    where = {(int(o.x[s]), int(o.y[s])): s for s in range(n)}
    count = np.zeros(n, int)
    for s in range(n):
        if act[s] == ATK:
            for xy in _square_cells(int(o.x[s]), int(o.y[s]), facing_after[s], side):
                if xy in where:
                    count[where[xy]] += 1
    o.transition(act)
    assert np.array_equal(o.hp, 40 - 3 * count)


# ----------------------------------------------------------------------------- ledgers

def _check(o, before, st):
    c = o.cfg
    L = o.side
    alive = np.flatnonzero(o.alive)
    cells = o.y[alive] * L + o.x[alive]
    assert len(set(cells.tolist())) == len(alive)
    assert np.array_equal(o.occ[cells], alive) and (o.occ >= 0).sum() == len(alive)
    assert not o.wall[cells].any()
    assert ((o.hp[alive] > 0) & (o.hp[alive] <= c["hp_max"])).all()
    assert ((o.energy[alive] >= 0) & (o.energy[alive] <= c["e_cap"])).all()
    assert np.array_equal(o.food, (o.res > 0).astype(np.uint8)) and (o.res >= 0).all()
    assert not (o.res * o.wall).any()
    t = int(o.step[0])
    founders = alive[o.birth_step[alive] < 0]
    kids = alive[o.birth_step[alive] >= 0]
    assert (o.age[founders] == t).all()
    assert (o.age[kids] == t - o.birth_step[kids] - 1).all()
    e0, r0, f0, n0 = before
    e1, r1 = int(o.energy[alive].sum()), int(o.res.sum())
    assert (e1 + r1) - (e0 + r0) == c["e_food"] * st["regrown"] - st["metab_paid"] - c["heal_cost"] * st["heals"]
    assert st["energy_total"] == e1 and st["res_total"] == r1
    assert st["energy_total"] == e0 + st["eaten_energy"] - st["metab_paid"] - c["heal_cost"] * st["heals"] - st["dead_energy"]
    assert st["food_total"] == f0 + st["regrown"] - st["food_emptied"] + st["food_refilled"]
    assert st["food_total"] == int(o.food.sum())
    assert st["alive"] == n0 + st["births"] - st["deaths"] == len(alive)


@pytest.mark.parametrize("over", [
    dict(side=48, slots=800, init_alive=500, e_repro=60, e_child=25, e_init=60),
    dict(side=32, slots=300, init_alive=250, e_repro=90, e_child=30, precision="bf16",
         flags=("rotate_obs", "cancel_all"), attack_damage=10, age_div=20),
    dict(side=40, slots=400, init_alive=300, e_repro=70, e_child=50, n_scalars=4, patch_k=5,
         policy_form="plain", n_hidden=1, food_density=0.3, regrow_p=0.05, e_init=40),
])
def test_ledgers_every_step(over):
    base = {k: over.pop(k) for k in ("side", "slots", "init_alive")}
    o = oracle.Oracle(workloads.scaled("ecology", base["side"], base["slots"], base["init_alive"],
                                       **over))
    o.reset()
    seen = dict(births=0, deaths=0, heals=0, starved=0, food_refilled=0, food_emptied=0)
    for _ in range(40):
        alive = o.alive == 1
        before = (int(o.energy[alive].sum()), int(o.res.sum()), int(o.food.sum()), int(alive.sum()))
        _, st, _ = o.step_once()
        for k in seen:
            seen[k] += st[k]
        _check(o, before, st)
    assert all(v > 0 for v in seen.values()), seen
