"""Hand-built worlds for rule tests.  Only array assignments: no rule
arithmetic lives here."""
import numpy as np

import oracle


def tiny_cfg(side=5, slots=8, patch_k=3, n_scalars=8, hidden=8, n_actions=9,
             flags=("rotate_obs",), **kw):
    cfg = dict(name="tiny", side=side, slots=slots, init_alive=0, patch_k=patch_k,
               n_scalars=n_scalars, hidden=hidden, n_actions=n_actions,
               precision="fp32", flags=flags, seed=kw.pop("seed", 11), sigma=0.01,
               food_density=0.0, regrow_p=0.0, wall_density=0.0, e_init=100,
               e_metab=1, e_food=20, e_repro=200, attack_num=1, attack_den=2)
    cfg.update(kw)
    return cfg


def empty_world(cfg):
    """An oracle with no food, walls or agents."""
    return oracle.Oracle(cfg)


def place(o, slot, x, y, facing=0, energy=100):
    o.alive[slot] = 1
    o.x[slot] = x
    o.y[slot] = y
    o.facing[slot] = facing
    o.energy[slot] = energy
    o.occ[y * o.side + x] = slot


def cell(o, x, y):
    return y * o.side + x


def actions(o, mapping, default=0):
    a = np.full(o.S, default, np.uint8)
    for s, v in mapping.items():
        a[s] = v
    return a
