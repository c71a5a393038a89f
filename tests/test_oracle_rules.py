"""Pins for the oracle's transition rules (not GPU).

Hand-worked scenarios (Sec. 3.2 "Actions": moves into occupied cells or into
the same cell are cancelled; attack; eat; single-parent reproduction directly
behind the parent; Sec. 3.1 population function), brute-force conflict
resolution on random tiny grids, a brute-force re-derivation of the founders'
placement, and ledger invariants over many steps.
"""
import numpy as np
import pytest

import oracle
from paper_2510_18221_gb300 import workloads
from tests import scenarios
from tests.scenarios import place, cell, actions

N_, E_, S_, W_ = 0, 1, 2, 3
ST_WALL, ST_FOOD, ST_PLACE, ST_FACING = 1, 2, 3, 4
ST_MOVE, ST_ATTACK, ST_BIRTH, ST_REGROW = 7, 8, 9, 11


def claim(o, stream, slot):
    """The claim key of a slot in the coming step: a larger key wins (draw
    first, then the lower slot).  Call it before the transition."""
    r = oracle.philox((int(o.step[0]), slot, 0, 0), (o.cfg["seed"], stream))[0]
    return (r << 32) | (0xFFFFFFFF - slot)


def world(**kw):
    return scenarios.empty_world(scenarios.tiny_cfg(**kw))


# ----------------------------------------------------------------------------- moves

def test_two_movers_one_cell_highest_claim_wins():
    o = world(side=6, slots=4)
    place(o, 0, 1, 2)
    place(o, 1, 3, 2)
    winner = 0 if claim(o, ST_MOVE, 0) > claim(o, ST_MOVE, 1) else 1
    st, _ = o.transition(actions(o, {0: oracle.EAST, 1: oracle.WEST}))
    loser = 1 - winner
    assert o.occ[cell(o, 2, 2)] == winner
    assert (o.x[loser], o.y[loser]) == ((1, 2) if loser == 0 else (3, 2))
    assert st["moves"] == 1 and st["move_lost"] == 1
    assert o.facing[0] == E_ and o.facing[1] == W_


def test_swap_is_cancelled():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=N_)
    place(o, 1, 2, 1, facing=N_)
    st, _ = o.transition(actions(o, {0: oracle.EAST, 1: oracle.WEST}))
    assert (o.x[0], o.x[1]) == (1, 2)
    assert st["move_blocked"] == 2 and st["moves"] == 0
    assert o.facing[0] == E_ and o.facing[1] == W_   # facing turns even when blocked


def test_chain_front_moves_back_blocked():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1)
    place(o, 1, 2, 1)
    st, _ = o.transition(actions(o, {0: oracle.EAST, 1: oracle.EAST}))
    assert (o.x[0], o.x[1]) == (1, 3)
    assert o.occ[cell(o, 2, 1)] == -1 and o.occ[cell(o, 3, 1)] == 1 and o.occ[cell(o, 1, 1)] == 0
    assert st["moves"] == 1 and st["move_blocked"] == 1


def test_wall_blocks_and_wraps():
    o = world(side=5, slots=4)
    place(o, 0, 2, 2)
    place(o, 1, 0, 0)
    o.wall[cell(o, 2, 1)] = 1
    st, _ = o.transition(actions(o, {0: oracle.NORTH, 1: oracle.WEST}))
    assert (o.x[0], o.y[0], o.facing[0]) == (2, 2, N_)
    assert (o.x[1], o.y[1]) == (4, 0)                 # wrapped west
    assert st["move_blocked"] == 1 and st["moves"] == 1


def test_cancel_all_rule():
    o = world(side=6, slots=4, flags=("rotate_obs", "cancel_all"))
    place(o, 0, 1, 2)
    place(o, 1, 3, 2)
    place(o, 2, 0, 5)
    st, _ = o.transition(actions(o, {0: oracle.EAST, 1: oracle.WEST, 2: oracle.NORTH}))
    assert (o.x[0], o.x[1]) == (1, 3) and o.occ[cell(o, 2, 2)] == -1
    assert (o.x[2], o.y[2]) == (0, 4)
    assert st["move_lost"] == 2 and st["moves"] == 1


def test_turns():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=N_)
    place(o, 1, 3, 3, facing=N_)
    place(o, 2, 4, 4, facing=W_)
    o.transition(actions(o, {0: oracle.TURN_LEFT, 1: oracle.TURN_RIGHT, 2: oracle.TURN_RIGHT}))
    assert list(o.facing[:3]) == [W_, E_, N_]
    assert (o.x[0], o.y[0]) == (1, 1)


def _brute_force_moves(o0, act):
    """O(N^2) restatement: mover i succeeds iff its target is no wall, was free
    at the start, and no other mover to the same target has a larger key."""
    L = o0.side
    dirs = {oracle.NORTH: (0, -1), oracle.SOUTH: (0, 1), oracle.EAST: (1, 0), oracle.WEST: (-1, 0)}
    alive = [s for s in range(o0.S) if o0.alive[s]]
    tgt = {}
    for s in alive:
        if act[s] in dirs:
            dx, dy = dirs[act[s]]
            t = ((o0.y[s] + dy) % L) * L + (o0.x[s] + dx) % L
            if not o0.wall[t] and o0.occ[t] == -1:
                tgt[s] = t
    pos = {s: (int(o0.x[s]), int(o0.y[s])) for s in alive}
    for s, t in tgt.items():
        if all(claim(o0, ST_MOVE, s) > claim(o0, ST_MOVE, q) for q, u in tgt.items() if u == t and q != s):
            pos[s] = (t % L, t // L)
    return pos


@pytest.mark.parametrize("trial", range(60))
def test_moves_brute_force(trial):
    g = np.random.default_rng(1000 + trial)
    side = int(g.integers(3, 7))
    o = world(side=side, slots=12, seed=int(g.integers(0, 2**31)))
    o.step[0] = int(g.integers(0, 1000))
    free = list(g.permutation(side * side))
    for c in free[:3]:
        o.wall[c] = 1
    n = min(10, side * side - 3)
    for s in range(n):
        c = int(free[3 + s])
        place(o, s, c % side, c // side)
    act = g.integers(0, 5, o.S).astype(np.uint8)
    want = _brute_force_moves(o.copy(), act)
    o.transition(act)
    for s, (x, y) in want.items():
        assert (o.x[s], o.y[s]) == (x, y)
        assert o.occ[y * side + x] == s


# ----------------------------------------------------------------------------- eat

def test_eat_explicit_and_auto():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, energy=50)
    place(o, 1, 3, 3, energy=50)
    o.food[cell(o, 1, 1)] = 1
    o.food[cell(o, 3, 3)] = 1
    st, _ = o.transition(actions(o, {0: oracle.EAT, 1: oracle.STAY}))
    assert (o.energy[0], o.energy[1]) == (69, 49)
    assert o.food[cell(o, 1, 1)] == 0 and o.food[cell(o, 3, 3)] == 1
    assert st["eaten"] == 1

    o = world(side=6, slots=4, n_actions=6, n_scalars=4, flags=("auto_eat", "rotate_obs"))
    place(o, 0, 1, 1, energy=50)
    o.food[cell(o, 2, 1)] = 1
    o.transition(actions(o, {0: oracle.EAST}))   # moves onto the food and eats it
    assert (o.x[0], o.energy[0], o.food[cell(o, 2, 1)]) == (2, 69, 0)


# ----------------------------------------------------------------------------- attack

def test_attack_transfers_half_of_post_eat_energy():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=E_, energy=100)
    place(o, 1, 2, 1, facing=N_, energy=81)
    o.food[cell(o, 2, 1)] = 1
    st, _ = o.transition(actions(o, {0: oracle.ATTACK, 1: oracle.EAT}))
    # victim: 81 + 20 = 101 after eating; loses 50; both pay 1
    assert (o.energy[0], o.energy[1]) == (149, 50)
    assert st["attacks"] == 1 and st["attack_hits"] == 1 and st["energy_transferred"] == 50


def test_mutual_attack_is_symmetric():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=E_, energy=100)
    place(o, 1, 2, 1, facing=W_, energy=60)
    o.transition(actions(o, {0: oracle.ATTACK, 1: oracle.ATTACK}))
    assert (o.energy[0], o.energy[1]) == (100 - 50 + 30 - 1, 60 - 30 + 50 - 1)


def test_one_attacker_per_victim_and_empty_target():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=E_, energy=100)
    place(o, 1, 2, 1, facing=N_, energy=100)
    place(o, 2, 3, 1, facing=W_, energy=100)
    place(o, 3, 5, 5, facing=N_, energy=100)
    w = 0 if claim(o, ST_ATTACK, 0) > claim(o, ST_ATTACK, 2) else 2
    st, _ = o.transition(actions(o, {0: oracle.ATTACK, 2: oracle.ATTACK, 3: oracle.ATTACK}))
    assert o.energy[w] == 149 and o.energy[2 - w] == 99 and o.energy[1] == 49
    assert st["attacks"] == 3 and st["attack_hits"] == 1


# ----------------------------------------------------------------------------- death

def test_death_frees_cell_and_slot():
    o = world(side=6, slots=4)
    place(o, 0, 1, 1, facing=E_, energy=1)
    place(o, 1, 3, 3, facing=E_, energy=100)
    place(o, 2, 4, 3, facing=N_, energy=2)
    st, _ = o.transition(actions(o, {1: oracle.ATTACK}))
    assert o.alive[0] == 0 and o.occ[cell(o, 1, 1)] == -1 and o.energy[0] == 0
    assert o.alive[2] == 0 and o.occ[cell(o, 4, 3)] == -1   # 2 -> 1 by attack -> 0
    assert st["deaths"] == 2 and st["dead_energy"] == 0 and o.energy[1] == 100


# ----------------------------------------------------------------------------- birth

def test_birth_behind_parent_into_lowest_free_slot():
    o = world(side=6, slots=4, sigma=0.0)
    place(o, 0, 0, 0, energy=100)
    place(o, 2, 2, 2, facing=N_, energy=250)
    o.master[2] = np.arange(o.P, dtype=np.float32) * 0.001
    o.step[0] = 7
    st, births = o.transition(actions(o, {}))
    assert births == [(2, 1)]
    assert o.alive[1] == 1 and (o.x[1], o.y[1]) == (2, 3) and o.occ[cell(o, 2, 3)] == 1
    assert (o.energy[2], o.energy[1]) == (125, 124)        # 249 split
    assert o.facing[1] == N_ and o.parent[1] == 2 and o.birth_step[1] == 7
    assert np.array_equal(o.master[1], o.master[2])         # sigma = 0
    assert st["births"] == 1


def test_birth_child_is_mutated_copy():
    o = world(side=6, slots=4, sigma=0.01)
    place(o, 0, 2, 2, facing=E_, energy=220)
    o.master[0] = np.linspace(-1, 1, o.P).astype(np.float32)
    o.step[0] = 3
    _, births = o.transition(actions(o, {}))
    assert births == [(0, 1)] and (o.x[1], o.y[1]) == (1, 2)
    assert np.array_equal(o.master[1], o.mutate(3, 0, o.master[0]))


def test_birth_blocked_by_wall_or_agent():
    o = world(side=6, slots=4)
    place(o, 0, 2, 2, facing=N_, energy=250)
    o.wall[cell(o, 2, 3)] = 1
    place(o, 1, 4, 4, facing=E_, energy=250)
    place(o, 2, 3, 4, facing=N_, energy=50)
    st, births = o.transition(actions(o, {}))
    assert births == [] and st["births"] == 0 and o.energy[0] == 249


def test_birth_into_cell_freed_by_death_and_slot_reuse():
    o = world(side=6, slots=2)
    place(o, 0, 2, 2, facing=N_, energy=250)
    place(o, 1, 2, 3, facing=N_, energy=1)        # dies this step, behind the parent
    st, births = o.transition(actions(o, {}))
    assert births == [(0, 1)] and (o.x[1], o.y[1]) == (2, 3) and o.energy[1] == 124


def test_two_parents_one_cell():
    o = world(side=6, slots=4)
    place(o, 0, 2, 1, facing=N_, energy=300)
    place(o, 1, 2, 3, facing=S_, energy=300)
    w = 0 if claim(o, ST_BIRTH, 0) > claim(o, ST_BIRTH, 1) else 1
    st, births = o.transition(actions(o, {}))
    assert births == [(w, 2)] and o.occ[cell(o, 2, 2)] == 2
    assert o.energy[1 - w] == 299 and st["failed_births"] == 0


def test_slot_exhaustion_lowest_parents_win():
    o = world(side=8, slots=4)
    place(o, 3, 1, 1, facing=N_, energy=300)
    place(o, 1, 4, 4, facing=N_, energy=300)
    place(o, 2, 6, 1, facing=N_, energy=300)
    st, births = o.transition(actions(o, {}))
    assert births == [(1, 0)] and st["failed_births"] == 2
    assert o.energy[2] == 299 and o.energy[3] == 299 and o.energy[1] == 150


# ----------------------------------------------------------------------------- regrowth

def test_regrowth_probability_one_and_zero():
    o = world(side=8, slots=2, regrow_p=1.0)
    o.wall[5] = 1
    o.transition(actions(o, {}))
    assert o.food.sum() == 63 and o.food[5] == 0
    o = world(side=8, slots=2, regrow_p=0.0)
    st, _ = o.transition(actions(o, {}))
    assert o.food.sum() == 0 and st["regrown"] == 0


def test_regrowth_rate_and_formula():
    o = world(side=256, slots=2, regrow_p=0.05)
    o.step[0] = 9
    st, _ = o.transition(actions(o, {}))
    assert abs(st["regrown"] / 65536 - 0.05) < 0.004
    thr = oracle.threshold(0.05)
    for c in [0, 1, 2, 3, 4, 1000, 65535]:
        r = oracle.philox((9, c >> 2, 0, 0), (o.cfg["seed"], ST_REGROW))[c & 3]
        assert o.food[c] == (r < thr)


# ----------------------------------------------------------------------------- reset

def test_reset_placement_brute_force():
    cfg = workloads.get("small", wall_density=0.1, seed=5)
    o = oracle.Oracle(cfg)
    o.reset()
    L, K, seed = cfg["side"], cfg["init_alive"], cfg["seed"]
    def word(stream, idx):
        return oracle.philox((idx >> 2, 0, 0, 0), (seed, stream))[idx & 3]
    walls = [c for c in range(L * L) if word(ST_WALL, c) < oracle.threshold(0.1)]
    assert sorted(np.flatnonzero(o.wall).tolist()) == walls
    food = [c for c in range(L * L) if c not in set(walls) and word(ST_FOOD, c) < oracle.threshold(0.1)]
    assert sorted(np.flatnonzero(o.food).tolist()) == food
    wallset = set(walls)
    keys = sorted((word(ST_PLACE, c), c) for c in range(L * L) if c not in wallset)
    cells = sorted(c for _, c in keys[:K])
    for s, c in enumerate(cells):
        assert o.alive[s] == 1 and (o.x[s], o.y[s]) == (c % L, c // L) and o.occ[c] == s
        assert o.facing[s] == word(ST_FACING, s) >> 30 and o.energy[s] == 100
    assert o.alive[K:].sum() == 0 and not o.master[K:].any()


# ----------------------------------------------------------------------------- invariants

def _check_invariants(o, before, st):
    L = o.side
    alive = np.flatnonzero(o.alive)
    cells = o.y[alive] * L + o.x[alive]
    assert len(set(cells.tolist())) == len(alive)               # one agent per cell
    assert np.array_equal(o.occ[cells], alive)                  # occupancy map agrees
    assert (o.occ >= 0).sum() == len(alive)
    assert not o.wall[cells].any()                              # nobody on a wall
    assert (o.energy[alive] > 0).all()
    e0, f0 = before
    c = o.cfg
    assert st["energy_total"] == e0 + c["e_food"] * st["eaten"] - c["e_metab"] * st["agent_steps"] - st["dead_energy"]
    assert st["food_total"] == f0 - st["eaten"] + st["regrown"]
    assert st["alive"] == st["agent_steps"] + st["births"] - st["deaths"]
    assert st["food_total"] == int(o.food.sum()) and st["alive"] == len(alive)


@pytest.mark.parametrize("name,steps,over", [
    ("small", 100, {}),
    ("mid", 40, dict(side=64, slots=512, init_alive=300)),
    ("mid", 40, dict(side=48, slots=600, init_alive=500, precision="fp8", e_init=190)),
])
def test_ledgers_hold_every_step(name, steps, over):
    o = oracle.Oracle(workloads.get(name, **over))
    o.reset()
    births = 0
    for _ in range(steps):
        before = (int(o.energy[o.alive == 1].sum()), int(o.food.sum()))
        _, st, b = o.step_once()
        births += len(b)
        _check_invariants(o, before, st)
    assert births > 0
