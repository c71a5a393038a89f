"""Pins for the oracle's vision variants and colour trait (not GPU).

* Front view (App. F.6 viewing configurations): the hand-worked 5x5 torus
  fixture in tests/golden, for each of the four facings, with wrap-around.
* RGB vision (Sec. 3.2: a rendered patch with three colour channels): a
  hand-worked patch -- an agent shows its colour trait (also when it stands
  on food), walls are grey, food green, empty cells black -- for two
  facings and both views.
* Colour trait (Sec. 3.3): founders' colours are the uniforms u = ((r >> 8)
  | 1) 2^-24 of their COLOUR draws (exact odd multiples of 2^-24, KS against
  U(0,1)); free slots are black; mutation with sigma = 0 is an exact copy,
  (child - parent) / sigma is N(0,1) (KS) away from the bounds, and the
  clamp keeps every channel in [0, 1] with about half the mass of a
  parent at 1 landing exactly on 1; a child born in the world carries
  mutate_colour of its parent's colour.
* Blind agents (App. F.6; the R and RC agents of the main experiments):
  the observation is the scalars alone, and the paper form has the compass
  and internal sensors only -- the parameter count of App. F.5's form with
  their sensor count, Kaiming fan-ins 4 and n_scalars - 4, zero biases.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2510_18221_gb300 import workloads
from tests import scenarios
from tests.scenarios import cell, place

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "observe_front_5x5_k3.txt")
DIRS = {"N": 0, "E": 1, "S": 2, "W": 3}
ST_COLOUR = 12


def _load_golden():
    world = {"food": [], "wall": [], "agent": []}
    blocks, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "world":
            if parts[1] in ("food", "wall"):
                world[parts[1]] += [tuple(map(int, p.split(","))) for p in parts[2:]]
            else:
                world["agent"].append((int(parts[2]), *map(int, parts[3].split(",")), int(parts[4])))
        elif parts[0] == "facing":
            cur = parts[1]
            blocks[cur] = []
        else:
            blocks[cur].append([tuple(map(int, c.split(","))) for c in parts])
    return world, blocks


@pytest.mark.parametrize("facing", ["N", "E", "S", "W"])
def test_front_view_golden(facing):
    world, blocks = _load_golden()
    o = scenarios.empty_world(scenarios.tiny_cfg(side=5, patch_k=3, view="front"))
    for x, y in world["food"]:
        o.food[cell(o, x, y)] = 1
    for x, y in world["wall"]:
        o.wall[cell(o, x, y)] = 1
    for slot, x, y, e in world["agent"]:
        place(o, slot, x, y, facing=0, energy=e)
    o.facing[0] = DIRS[facing]
    x = o.observe(0)
    want = np.array([v for row in blocks[facing] for c in row for v in c], np.float64)
    np.testing.assert_array_equal(x[:27], want)


def _rgb_world(view="around"):
    o = scenarios.empty_world(scenarios.tiny_cfg(side=5, patch_k=3, vision="rgb", view=view))
    place(o, 0, 2, 2, facing=0)
    place(o, 1, 2, 1, facing=0)
    o.colour[0] = (0.25, 0.5, 0.75)
    o.colour[1] = (1.0, 0.0, 0.125)
    for xy in ((2, 2), (2, 1), (3, 1)):
        o.food[cell(o, *xy)] = 1
    o.wall[cell(o, 1, 1)] = 1
    return o


K_, G_, W_, R_ = (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.5, 0.5, 0.5), None
A_, B_ = (0.25, 0.5, 0.75), (1.0, 0.0, 0.125)


@pytest.mark.parametrize("view,facing,rows", [
    # Around, facing N: ahead is row y = 1, left is x - 1
    ("around", 0, [[W_, B_, G_], [K_, A_, K_], [K_, K_, K_]]),
    # Around, facing S: ahead is y = 3, left is x + 1; behind (y = 1) reversed
    ("around", 2, [[K_, K_, K_], [K_, A_, K_], [G_, B_, W_]]),
    # Front, facing N: two rows ahead (y = 0, y = 1), then the agent's row
    ("front", 0, [[K_, K_, K_], [W_, B_, G_], [K_, A_, K_]]),
    # Front, facing S: y = 4, y = 3, then the agent's row (left is x + 1)
    ("front", 2, [[K_, K_, K_], [K_, K_, K_], [K_, A_, K_]]),
])
def test_rgb_patch_hand_worked(view, facing, rows):
    o = _rgb_world(view)
    o.facing[0] = facing
    x = o.observe(0)
    want = np.array([v for row in rows for c in row for v in c], np.float64)
    np.testing.assert_array_equal(x[:27], want)


def test_channels_vision_ignores_colour():
    o = _rgb_world()
    o.cfg["vision"] = "channels"
    o2 = scenarios.empty_world(scenarios.tiny_cfg(side=5, patch_k=3))
    for n in oracle.Oracle.ARRAYS:
        if n != "master":
            setattr(o2, n, getattr(o, n).copy())
    x = o2.observe(0)
    assert set(np.unique(x[:27]).tolist()) <= {0.0, 1.0}


def test_founder_colours_are_uniforms_of_their_draws():
    w = workloads.scaled("mid", 64, 600, 500)
    o = oracle.Oracle(w)
    o.reset()
    for slot in (0, 1, 77, 499):
        r = oracle.philox((slot, 0, 0, 0), (w["seed"], ST_COLOUR))
        want = [((v >> 8) | 1) * 2.0 ** -24 for v in r[:3]]
        assert o.colour[slot].tolist() == want
    assert (o.colour[500:] == 0).all()
    founders = o.colour[:500].astype(np.float64)
    assert ((founders > 0) & (founders < 1)).all()
    q = founders * 2.0 ** 24
    assert np.array_equal(q, np.round(q)) and (np.round(q) % 2 == 1).all()
    assert scipy.stats.kstest(founders.ravel(), "uniform").pvalue > 1e-3


def _mut_oracle(sigma):
    return oracle.Oracle(workloads.scaled("mid", 16, 8, 4, sigma=sigma))


def test_colour_mutation_sigma_zero_is_a_copy():
    o = _mut_oracle(0.0)
    p = np.array([0.0, 0.3, 1.0], np.float32)
    for step in range(20):
        assert np.array_equal(o.mutate_colour(step, 3, p), p)


def test_colour_mutation_is_gaussian_away_from_the_bounds():
    sigma = 0.01
    o = _mut_oracle(sigma)
    p = np.full(3, 0.5, np.float32)
    z = np.array([(o.mutate_colour(step, slot, p).astype(np.float64) - 0.5) / sigma
                  for step in range(400) for slot in range(25)]).ravel()
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.05 and abs(z.var() - 1) < 0.05


def test_colour_mutation_draws_are_the_colour_stream_normals():
    sigma = 0.02
    o = _mut_oracle(sigma)
    p = np.array([0.4, 0.5, 0.6], np.float32)
    for step, slot in ((0, 0), (5, 3), (1234, 7)):
        r = oracle.philox((step, slot, 1, 0), (o.cfg["seed"], ST_COLOUR))
        n = oracle.normals4(r)
        want = [np.float32(float(p[c]) + np.float32(sigma).item() * n[c]) for c in range(3)]
        assert o.mutate_colour(step, slot, p).tolist() == [float(v) for v in want]


def test_colour_mutation_clamps_to_the_unit_interval():
    o = _mut_oracle(0.5)
    kids = np.array([o.mutate_colour(step, 1, np.array([1.0, 0.0, 1.0], np.float32))
                     for step in range(2000)])
    assert ((kids >= 0) & (kids <= 1)).all()
    at_one = float((kids[:, 0] == 1.0).mean())
    at_zero = float((kids[:, 1] == 0.0).mean())
    assert abs(at_one - 0.5) < 0.05 and abs(at_zero - 0.5) < 0.05


def test_child_carries_the_mutated_colour():
    o = scenarios.empty_world(scenarios.tiny_cfg(side=6, slots=4, vision="rgb", sigma=0.05))
    place(o, 0, 2, 2, facing=0, energy=250)
    o.colour[0] = (0.2, 0.9, 0.5)
    _, births = o.transition(scenarios.actions(o, {}))
    assert births == [(0, 1)]
    np.testing.assert_array_equal(o.colour[1], o.mutate_colour(0, 0, o.colour[0]))
    assert not np.array_equal(o.colour[1], o.colour[0])


def test_colours_stay_in_range_over_a_run():
    o = oracle.Oracle(workloads.scaled("mid", 48, 600, 500, e_init=190, vision="rgb",
                                       view="front", sigma=0.2))
    o.reset()
    births = 0
    for _ in range(20):
        _, _, b = o.step_once()
        births += len(b)
        alive = o.alive == 1
        assert ((o.colour[alive] >= 0) & (o.colour[alive] <= 1)).all()
    assert births > 0


# ----------------------------------------------------------------------------- blind agents

@pytest.mark.parametrize("n_scalars", [4, 8])
def test_blind_observation_is_the_scalars(n_scalars):
    """App. F.6 "Blind" (the R / RC agents of the main experiments): no
    vision sensor, so the observation is the scalars alone."""
    o = scenarios.empty_world(scenarios.tiny_cfg(side=5, patch_k=0, n_scalars=n_scalars))
    place(o, 0, 2, 2, facing=3, energy=150)
    o.food[cell(o, 2, 1)] = 1
    x = o.observe(0)
    want = [150 / 200] + ([0, 0, 0, 1] if n_scalars == 8 else []) + [0, 0, 0]
    np.testing.assert_array_equal(x, np.array(want, np.float64))


@pytest.mark.parametrize("n_scalars,L,H", [(8, 2, 64), (4, 2, 64), (8, 1, 32), (8, 3, 128)])
def test_blind_paper_form_sensors_and_count(n_scalars, L, H):
    """Without a vision sensor the paper form has the compass (8 scalars)
    and the internal sensor: L(H^2+H) + H(D + n_sensors + A) + 1 parameters
    (the form of App. F.5's table), and Kaiming fan-ins of 4 and
    n_scalars - 4 (or n_scalars)."""
    w = workloads.scaled("paperform", 32, 64, 40, patch_k=0, n_scalars=n_scalars,
                         n_hidden=L, hidden=H)
    o = oracle.Oracle(w)
    ns = 2 if n_scalars == 8 else 1
    A = w["n_actions"]
    assert o.D == n_scalars
    assert o.P == L * (H * H + H) + H * (n_scalars + ns + A) + 1
    rows = np.array([o.init_params(s) for s in range(40)], np.float64)
    w_in = rows[:, :H * n_scalars].reshape(40, H, n_scalars)
    if n_scalars == 8:
        compass = w_in[:, :, 1:5].ravel()
        internal = np.concatenate([w_in[:, :, :1].ravel(), w_in[:, :, 5:].ravel()])
        assert scipy.stats.kstest(compass / np.sqrt(2.0 / 4), "norm").pvalue > 1e-3
        assert scipy.stats.kstest(internal / np.sqrt(2.0 / 4), "norm").pvalue > 1e-3
    else:
        assert scipy.stats.kstest(w_in.ravel() / np.sqrt(2.0 / 4), "norm").pvalue > 1e-3
    assert not rows[:, H * n_scalars:H * n_scalars + ns * H].any()   # sensor biases zero
