"""Pins for the oracle's paper-form policy (Sec. 3.3), not GPU.

* Parameter counts: the paper's table of network sizes (App. F.5, R and RC
  agents, (layers, channels) in {(1,32), (2,32), (2,64), (2,128), (3,128)})
  is reproduced by the count of the paper form: per-sensor input linears
  (weights + one bias per sensor), L hidden layers with biases, an unbiased
  head and one temperature parameter.  The paper does not list its sensor
  sizes; the table fixes D + n_sensors + n_actions = 216 for R, and the
  compass adds 4 inputs and one bias (RC).
* Forward pass: against numpy float64 (a library routine) on random
  parameters: ReLU(sum of sensor linears) -> L x ReLU(W h + b) -> W_out h,
  divided by the temperature exp(tau).
* Temperature: closed form (tau = ln 2 halves every logit).
* Kaiming initialisation (Sec. 3.3): per-sensor fan-in, std sqrt(2/fan_in);
  zero biases and tau.
* Streamed forms: BF16 / FP8 effective weights of every layer (including
  the extra hidden layers) against torch's conversions, row by row.
* Ledgers every step of an oracle run with the paper-form policy.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2510_18221_gb300 import workloads
from tests import inputs

TABLE = {  # (layers, channels): (RC, R) -- App. F.5, network-size table
    (1, 32): (8129, 7969),
    (2, 32): (9185, 9025),
    (2, 64): (22465, 22145),
    (2, 128): (61313, 60673),
    (3, 128): (77825, 77185),
}


@pytest.mark.parametrize("lc", sorted(TABLE))
def test_param_counts_match_paper_table(lc):
    L, c = lc
    rc, r = TABLE[lc]
    A = 8               # rest, 3 moves, 3 eats, reproduce (no attack)
    ns_r, D_r = 2, 216 - 2 - A   # internal + external sensors
    assert oracle.param_count_shape(D_r, c, A, L, ns_r, 0, 1) == r
    assert oracle.param_count_shape(D_r + 4, c, A, L, ns_r + 1, 0, 1) == rc  # + compass


def _cfg(**kw):
    w = workloads.get("mid", policy_form="paper", n_hidden=2, slots=4, side=16, init_alive=0)
    w.update(kw)
    return w


def _split(w, D, H, A, L, ns):
    out = {}
    i = 0
    out["Win"] = w[i:i + H * D].reshape(H, D); i += H * D
    out["bin"] = w[i:i + ns * H].reshape(ns, H); i += ns * H
    out["hid"] = []
    for _ in range(L):
        W = w[i:i + H * H].reshape(H, H); i += H * H
        b = w[i:i + H]; i += H
        out["hid"].append((W, b))
    out["Wout"] = w[i:i + A * H].reshape(A, H); i += A * H
    out["tau"] = w[i]; i += 1
    assert i == len(w)
    return out


def test_paper_form_count_for_the_mid_observation():
    o = oracle.Oracle(_cfg())
    D, H, A = 371, 64, 9
    assert o.P == H * D + 3 * H + 2 * (H * H + H) + A * H + 1 == 32833


@pytest.mark.parametrize("L", [1, 2, 3])
def test_paper_form_forward_matches_numpy(L):
    o = oracle.Oracle(_cfg(n_hidden=L))
    D, H, A, ns = o.D, 64, 9, 3
    for seed in range(3):
        w = inputs.random_params(o.P, seed=20 + seed, scale=0.2)[0].astype(np.float64)
        w[-1] = 0.3 * (seed - 1)              # tau
        x = inputs.random_obs(D, seed=30 + seed)
        p = _split(w, D, H, A, L, ns)
        h = np.maximum(p["Win"] @ x + p["bin"].sum(axis=0), 0.0)
        for W, b in p["hid"]:
            h = np.maximum(W @ h + b, 0.0)
        want = (p["Wout"] @ h) / math.exp(p["tau"])
        assert np.allclose(o.mlp(w, x), want, rtol=0, atol=1e-12)


def test_temperature_halves_logits():
    o = oracle.Oracle(_cfg())
    w = inputs.random_params(o.P, seed=41, scale=0.2)[0].astype(np.float64)
    x = inputs.random_obs(o.D, seed=42)
    w[-1] = 0.0
    l0 = o.mlp(w, x)
    w[-1] = math.log(2.0)
    assert np.allclose(o.mlp(w, x), l0 / 2.0, rtol=1e-13, atol=0)


def test_kaiming_init_per_sensor():
    from scipy import stats
    o = oracle.Oracle(_cfg(slots=8))
    D, H, A, L, ns = o.D, 64, 9, 2, 3
    rows = [o.init_params(s) for s in range(6)]
    p = _split(rows[0].astype(np.float64), D, H, A, L, ns)
    vis = np.concatenate([_split(r.astype(np.float64), D, H, A, L, ns)["Win"][:, :363].ravel() for r in rows])
    assert stats.kstest(vis * math.sqrt(363 / 2.0), "norm").pvalue > 1e-3
    comp = np.concatenate([_split(r.astype(np.float64), D, H, A, L, ns)["Win"][:, 364:368].ravel() for r in rows])
    assert abs(comp.var() - 2.0 / 4) < 0.1                      # compass: fan-in 4
    hid = np.concatenate([_split(r.astype(np.float64), D, H, A, L, ns)["hid"][1][0].ravel() for r in rows])
    assert abs(hid.var() * H / 2.0 - 1.0) < 0.05
    assert not p["bin"].any() and p["tau"] == 0.0
    assert all(not b.any() for _, b in p["hid"])


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_paper_form_effective_params(prec):
    o = oracle.Oracle(_cfg(precision=prec, n_hidden=3))
    D, H, A, L, ns = o.D, 64, 9, 3, 3
    o.master[0] = inputs.random_params(o.P, seed=50)[0]
    w = o.effective_params(0)
    m = _split(o.master[0].astype(np.float64), D, H, A, L, ns)
    e = _split(w, D, H, A, L, ns)
    mats = [("Win", m["Win"], e["Win"])] + [("h%d" % i, m["hid"][i][0], e["hid"][i][0]) for i in range(L)] \
        + [("Wout", m["Wout"], e["Wout"])]
    for name, M, E in mats:
        for r in range(M.shape[0]):
            row = M[r].astype(np.float32)
            if prec == "bf16":
                want = torch.from_numpy(row.copy()).to(torch.bfloat16).float().numpy().astype(np.float64)
            else:
                s = np.float32(np.max(np.abs(row))) / np.float32(448.0)
                q = torch.from_numpy((row / s).astype(np.float32)).to(torch.float8_e4m3fn)
                want = float(s) * q.float().numpy().astype(np.float64)
            assert np.array_equal(E[r], want), (name, r)
    assert np.array_equal(e["bin"], m["bin"]) and e["tau"] == m["tau"]
    for i in range(L):
        assert np.array_equal(e["hid"][i][1], m["hid"][i][1])


def test_paper_form_ledgers():
    w = workloads.scaled("mid", 48, 600, 500, policy_form="paper", n_hidden=2, e_init=190)
    o = oracle.Oracle(w)
    o.reset()
    births = 0
    for _ in range(30):
        e0 = int(o.energy[o.alive == 1].sum())
        f0 = int(o.food.sum())
        _, st, b = o.step_once()
        births += len(b)
        assert st["energy_total"] == e0 + 20 * st["eaten"] - st["agent_steps"] - st["dead_energy"]
        assert st["food_total"] == f0 - st["eaten"] + st["regrown"]
        assert st["alive"] == st["agent_steps"] + st["births"] - st["deaths"]
    assert births > 0
