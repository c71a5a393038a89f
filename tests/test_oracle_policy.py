"""Pins for the oracle's observation and policy (not GPU).

* Observation: the hand-worked 5x5 torus fixture in tests/golden (Sec. 3.2
  "Sensors"), for each of the four facings, with wrap-around.
* MLP (Sec. 3.3): against numpy float64 matrix products (a library routine,
  not the oracle's loops) on random parameters, and a closed form with
  one-hot weights.
* Parameter count: H*D + H + H*H + H + A*H + A for each workload.
* Streamed forms: BF16 / FP8 effective weights against PyTorch's conversions
  applied per row.
* Initialisation and mutation (Sec. 3.3): zero biases, N(0, 1/fan_in)
  weights, sigma = 0 gives an exact copy, (child - parent) / sigma is N(0,1).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2510_18221_gb300 import workloads
from tests import inputs, scenarios

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "observe_5x5_k3.txt")
DIRS = {"N": 0, "E": 1, "S": 2, "W": 3}


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


def _golden_world(facing, flags=("rotate_obs",)):
    world, _ = _load_golden()
    o = scenarios.empty_world(scenarios.tiny_cfg(side=5, patch_k=3, flags=flags))
    for x, y in world["food"]:
        o.food[scenarios.cell(o, x, y)] = 1
    for x, y in world["wall"]:
        o.wall[scenarios.cell(o, x, y)] = 1
    for slot, x, y, e in world["agent"]:
        scenarios.place(o, slot, x, y, facing=0, energy=e)
    o.facing[0] = facing
    return o


@pytest.mark.parametrize("name", ["N", "E", "S", "W"])
def test_observation_hand_worked(name):
    _, blocks = _load_golden()
    o = _golden_world(DIRS[name])
    x = o.observe(0)
    want = np.array(blocks[name], dtype=np.float64).reshape(-1)
    assert np.array_equal(x[:27], want)
    scal = np.zeros(8)
    scal[0] = 50 / 200
    scal[1 + DIRS[name]] = 1.0
    assert np.array_equal(x[27:], scal)


@pytest.mark.parametrize("name", ["E", "S", "W"])
def test_observation_unrotated_is_north_up(name):
    _, blocks = _load_golden()
    o = _golden_world(DIRS[name], flags=())
    want = np.array(blocks["N"], dtype=np.float64).reshape(-1)
    assert np.array_equal(o.observe(0)[:27], want)


def test_observation_small_scalars():
    cfg = scenarios.tiny_cfg(side=5, patch_k=3, n_scalars=4)
    o = scenarios.empty_world(cfg)
    scenarios.place(o, 0, 2, 2, facing=3, energy=137)
    x = o.observe(0)
    assert np.array_equal(x[27:], np.array([137 / 200, 0, 0, 0]))


def _split(w, D, H, A):
    i = 0
    out = []
    for shape in [(H, D), (H,), (H, H), (H,), (A, H), (A,)]:
        n = int(np.prod(shape))
        out.append(w[i:i + n].reshape(shape))
        i += n
    return out


@pytest.mark.parametrize("name", ["small", "mid", "large"])
def test_param_count(name):
    cfg = workloads.get(name)
    o = oracle.Oracle(dict(cfg, slots=1, side=8, init_alive=0))
    D = 3 * cfg["patch_k"] ** 2 + cfg["n_scalars"]
    H, A = cfg["hidden"], cfg["n_actions"]
    assert o.D == D
    assert o.P == H * D + H + H * H + H + A * H + A
    assert {"small": 3814, "mid": 28553, "large": 105225}[name] == o.P


@pytest.mark.parametrize("name", ["small", "mid"])
def test_mlp_matches_numpy_float64(name):
    cfg = workloads.get(name)
    o = oracle.Oracle(dict(cfg, slots=1, side=8, init_alive=0))
    D, H, A = o.D, cfg["hidden"], cfg["n_actions"]
    for seed in range(5):
        w = inputs.random_params(o.P, seed=seed)[0].astype(np.float64)
        x = inputs.random_obs(D, seed=100 + seed)
        W1, b1, W2, b2, W3, b3 = _split(w, D, H, A)
        h1 = np.tanh(W1 @ x + b1)
        h2 = np.tanh(W2 @ h1 + b2)
        want = W3 @ h2 + b3
        got = o.mlp(w, x)
        assert np.allclose(got, want, rtol=0, atol=1e-12)


def test_mlp_closed_form_one_hot():
    cfg = workloads.get("small")
    o = oracle.Oracle(dict(cfg, slots=1, side=8, init_alive=0))
    D, H, A = o.D, 32, 6
    W1 = np.zeros((H, D)); W2 = np.eye(H); W3 = np.zeros((A, H))
    for k in range(H):
        W1[k, k] = 1.0
    for a in range(A):
        W3[a, a] = 2.0
    b3 = np.arange(A) * 0.5
    w = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(), b3])
    x = np.zeros(D)
    x[[0, 2, 5]] = 1.0
    got = o.mlp(w, x)
    t = math.tanh(math.tanh(1.0))
    want = np.array([2 * t, 0, 2 * t, 0, 0, 2 * t]) + b3
    assert np.allclose(got, want, atol=1e-15)


def test_effective_params_bf16_matches_torch():
    cfg = workloads.get("mid", precision="bf16", slots=2, side=16, init_alive=0)
    o = oracle.Oracle(cfg)
    o.master[0] = inputs.random_params(o.P, seed=9)[0]
    w = o.effective_params(0)
    D, H, A = o.D, 64, 9
    m = o.master[0]
    bf = torch.from_numpy(m.copy()).to(torch.bfloat16).float().numpy().astype(np.float64)
    parts_m = _split(m.astype(np.float64), D, H, A)
    parts_b = _split(bf, D, H, A)
    parts_w = _split(w, D, H, A)
    for i in (0, 2, 4):
        assert np.array_equal(parts_w[i], parts_b[i])
    for i in (1, 3, 5):
        assert np.array_equal(parts_w[i], parts_m[i])  # biases stay FP32


def test_effective_params_fp8_matches_torch_rowwise():
    cfg = workloads.get("mid", precision="fp8", slots=2, side=16, init_alive=0)
    o = oracle.Oracle(cfg)
    o.master[0] = inputs.random_params(o.P, seed=10)[0]
    w = o.effective_params(0)
    D, H, A = o.D, 64, 9
    pm = _split(o.master[0], D, H, A)
    pw = _split(w, D, H, A)
    for i in (0, 2, 4):
        for r in range(pm[i].shape[0]):
            row = pm[i][r]
            s = np.float32(np.max(np.abs(row))) / np.float32(448.0)
            q = torch.from_numpy((row / s).astype(np.float32)).to(torch.float8_e4m3fn)
            want = float(s) * q.float().numpy().astype(np.float64)
            assert np.array_equal(pw[i][r], want), (i, r)
    for i in (1, 3, 5):
        assert np.array_equal(pw[i], pm[i].astype(np.float64))


def test_init_params_statistics():
    cfg = workloads.get("mid", slots=4, side=16, init_alive=0)
    o = oracle.Oracle(cfg)
    D, H, A = o.D, 64, 9
    rows = [o.init_params(s) for s in range(3)]
    assert not np.array_equal(rows[0], rows[1])
    assert np.array_equal(rows[0], o.init_params(0))
    for row in rows:
        W1, b1, W2, b2, W3, b3 = _split(row.astype(np.float64), D, H, A)
        assert not b1.any() and not b2.any() and not b3.any()
        assert abs(W1.var() * D - 1.0) < 0.05 and abs(W1.mean()) < 0.01
        assert abs(W2.var() * H - 1.0) < 0.1
    from scipy import stats
    W1 = _split(rows[0].astype(np.float64), D, H, A)[0].ravel() * math.sqrt(D)
    assert stats.kstest(W1, "norm").pvalue > 1e-3


def test_mutation_sigma_zero_copies_exactly():
    cfg = workloads.get("mid", slots=4, side=16, init_alive=0, sigma=0.0)
    o = oracle.Oracle(cfg)
    parent = inputs.random_params(o.P, seed=12)[0]
    assert np.array_equal(o.mutate(17, 3, parent), parent)


def test_mutation_noise_is_sigma_times_standard_normal():
    from scipy import stats
    cfg = workloads.get("mid", slots=4, side=16, init_alive=0, sigma=1.0)
    o = oracle.Oracle(cfg)
    zero = np.zeros(o.P, np.float32)
    n = np.concatenate([o.mutate(5, s, zero) for s in range(4)]).astype(np.float64)
    assert stats.kstest(n, "norm").pvalue > 1e-3
    # different parents or steps give different noise; the same gives the same
    assert not np.array_equal(o.mutate(5, 0, zero), o.mutate(5, 1, zero))
    assert not np.array_equal(o.mutate(5, 0, zero), o.mutate(6, 0, zero))
    assert np.array_equal(o.mutate(5, 0, zero), o.mutate(5, 0, zero))
    cfg2 = workloads.get("mid", slots=4, side=16, init_alive=0, sigma=0.01)
    o2 = oracle.Oracle(cfg2)
    parent = inputs.random_params(o2.P, seed=13)[0]
    d = (o2.mutate(5, 0, parent).astype(np.float64) - parent) / 0.01
    assert abs(d.std() - 1.0) < 0.02 and abs(d.mean()) < 0.02


def test_greedy_policy_takes_argmax_and_flags_ties():
    cfg = scenarios.tiny_cfg(side=6, slots=4, hidden=8, flags=("rotate_obs", "greedy"))
    o = scenarios.empty_world(cfg)
    scenarios.place(o, 1, 2, 2, facing=0, energy=80)
    P = o.P
    b3 = P - 9
    o.master[1, b3 + 4] = 5.0          # head bias forces action 4
    pol = o.policy(tol=1e-3)
    assert pol["action"][1] == 4 and pol["valid"][1] == 1 << 4
    assert np.allclose(pol["logits"][1], o.master[1, b3:b3 + 9])
    assert pol["action"][0] == 0 and pol["valid"][0] == 0  # dead slot
    o.master[1, b3 + 7] = 5.0          # an exact tie: first maximum, both valid
    pol = o.policy(tol=1e-3)
    assert pol["action"][1] == 4 and pol["valid"][1] == (1 << 4) | (1 << 7)
