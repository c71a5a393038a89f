"""CPU oracle for one step of the ecological simulator (arXiv 2510.18221).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import this module.
The product path (the CUDA library and its binding) never imports it, and it
imports nothing from the product package: the two implementations share no
code.  Workload configurations reach both as plain dictionaries.

The arithmetic lives in ``eco_oracle.c`` (plain C99, FP64 policy, integer
world state), which follows the paper's Sec. 3.2 (environment, sensors,
actions) and Sec. 3.3 (per-agent MLP, sampling, initialisation, mutation).
This module only allocates the state as numpy arrays and marshals calls.

Parity status per function (see the pins in ``tests/test_oracle_*.py``):
every function below has at least one pin (library routine, closed form,
hand-worked fixture, brute force or invariant); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eco_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FP32, BF16, FP8 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8}

AUTO_EAT, ROTATE_OBS, CANCEL_ALL, GREEDY = 1, 2, 4, 8
PLAIN, PAPER_FORM = 0, 1
POLICY_FORMS = {"plain": PLAIN, "paper": PAPER_FORM}
FLAG_NAMES = {"auto_eat": AUTO_EAT, "rotate_obs": ROTATE_OBS,
              "cancel_all": CANCEL_ALL, "greedy": GREEDY}

# Action codes (the build's reading of the configs' action sets).
STAY, NORTH, SOUTH, EAST, WEST, ATTACK, TURN_LEFT, TURN_RIGHT, EAT = range(9)

# Rule sets, and the paper rule set's action codes (Sec. 3.2 "Actions").
RULES_SIMPLE, RULES_PAPER, RULES_TERRAIN = 0, 1, 2
RULES = {"simple": RULES_SIMPLE, "paper": RULES_PAPER, "terrain": RULES_TERRAIN}
P_REST, P_ROT_CW, P_ROT_CCW, P_FORWARD, P_ATTACK, P_EAT, P_REPRODUCE = range(7)
T_DRINK, T_EAT_BIO = 7, 8
TERRAIN_FIELDS = ("sea_level", "w_init", "w_metab", "w_bite", "w_cap", "w_child", "heal_water",
                  "b_body", "b_child", "b_bite", "b_cap", "b_site")

# Constants of the paper rule set, read from the workload dictionary (0 when
# absent: the simple rule set ignores them).
# Vision (Sec. 3.2 "Sensors") and viewing configuration (App. F.6).
VISIONS = {"channels": 0, "rgb": 1}
VIEWS = {"around": 0, "front": 1}
PAPER_RULE_FIELDS = ("hp_max", "hp_child", "attack_damage", "heal_rate", "heal_cost",
                     "age_div", "starve_damage", "e_act", "e_cap", "e_child")


def build(force: bool = False) -> str:
    """Compile ``eco_oracle.c`` into ``liboracle.so`` next to it."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [
        ("side", ctypes.c_int32), ("slots", ctypes.c_int32),
        ("init_alive", ctypes.c_int32), ("patch_k", ctypes.c_int32),
        ("n_scalars", ctypes.c_int32), ("hidden", ctypes.c_int32),
        ("n_actions", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("seed", ctypes.c_uint32),
        ("sigma", ctypes.c_float), ("food_density", ctypes.c_float),
        ("regrow_p", ctypes.c_float), ("wall_density", ctypes.c_float),
        ("e_init", ctypes.c_int32), ("e_metab", ctypes.c_int32),
        ("e_food", ctypes.c_int32), ("e_repro", ctypes.c_int32),
        ("attack_num", ctypes.c_int32), ("attack_den", ctypes.c_int32),
        ("policy_form", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
        ("rules", ctypes.c_int32), ("hp_max", ctypes.c_int32),
        ("hp_child", ctypes.c_int32), ("attack_damage", ctypes.c_int32),
        ("heal_rate", ctypes.c_int32), ("heal_cost", ctypes.c_int32),
        ("age_div", ctypes.c_int32), ("starve_damage", ctypes.c_int32),
        ("e_act", ctypes.c_int32), ("e_cap", ctypes.c_int32),
        ("e_child", ctypes.c_int32),
        ("vision", ctypes.c_int32), ("view", ctypes.c_int32),
    ] + [(k, ctypes.c_int32) for k in TERRAIN_FIELDS] + [
        ("biomass_density", ctypes.c_float), ("photo_q16", ctypes.c_int32),
        ("res_cap", ctypes.c_int32),
    ]


_P = ctypes.c_void_p


class State(ctypes.Structure):
    _fields_ = [(n, _P) for n in ("food", "wall", "occ", "alive", "x", "y", "facing",
                                  "energy", "parent", "birth_step", "master", "step",
                                  "hp", "age", "res", "colour", "rock", "water", "bio",
                                  "photo", "a_water", "a_bio")]


STAT_FIELDS = ["agent_steps"] + ["act%d" % i for i in range(16)] + [
    "moves", "move_blocked", "move_lost", "eaten", "attacks", "attack_hits",
    "energy_transferred", "deaths", "dead_energy", "births", "failed_births",
    "regrown", "alive", "food_total", "energy_total",
    "res_total", "eaten_energy", "metab_paid", "heals", "starved", "damage",
    "food_emptied", "food_refilled",
    "water_cells", "water_agents", "bio_cells", "bio_agents", "drunk", "water_spent",
    "thirsty", "bio_eaten", "photo", "dead_water", "dead_bio"]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in STAT_FIELDS]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.argtypes = [ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_gumbel.argtypes = [ctypes.c_uint32]
            L.orc_gumbel.restype = ctypes.c_double
            L.orc_normals4.argtypes = [u32p, ctypes.POINTER(ctypes.c_double)]
            L.orc_threshold.argtypes = [ctypes.c_float]
            L.orc_threshold.restype = ctypes.c_uint32
            L.orc_bf16_rne.argtypes = [ctypes.c_float]
            L.orc_bf16_rne.restype = ctypes.c_uint16
            L.orc_bf16_value.argtypes = [ctypes.c_uint16]
            L.orc_bf16_value.restype = ctypes.c_double
            L.orc_e4m3_encode.argtypes = [ctypes.c_float]
            L.orc_e4m3_encode.restype = ctypes.c_uint8
            L.orc_e4m3_value.argtypes = [ctypes.c_uint8]
            L.orc_e4m3_value.restype = ctypes.c_double
            L.orc_fp8_row_scale.argtypes = [_P, ctypes.c_int]
            L.orc_fp8_row_scale.restype = ctypes.c_float
            cfgp = ctypes.POINTER(Config)
            stp = ctypes.POINTER(State)
            L.orc_param_count_shape.argtypes = [ctypes.c_int] * 7
            L.orc_obs_dim.argtypes = [cfgp]
            L.orc_n_params.argtypes = [cfgp]
            L.orc_reset.argtypes = [cfgp, stp]
            L.orc_init_params.argtypes = [cfgp, ctypes.c_int32, _P]
            L.orc_observe.argtypes = [cfgp, stp, ctypes.c_int32, _P]
            L.orc_effective_params.argtypes = [cfgp, _P, ctypes.c_int, _P]
            L.orc_weight_mask.argtypes = [cfgp, _P]
            L.orc_quantise.argtypes = [cfgp, _P, _P, _P]
            L.orc_mlp.argtypes = [cfgp, _P, _P, _P]
            L.orc_policy.argtypes = [cfgp, stp, ctypes.c_int, ctypes.c_double, _P, _P, _P, _P]
            L.orc_mutate.argtypes = [cfgp, ctypes.c_int64, ctypes.c_int32, _P, _P]
            L.orc_mutate_colour.argtypes = [cfgp, ctypes.c_int64, ctypes.c_int32, _P, _P]
            L.orc_water_flow.argtypes = [cfgp, stp]
            L.orc_transition.argtypes = [cfgp, stp, _P, ctypes.POINTER(Stats), _P, _P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ---------------------------------------------------------------------------
# Scalar helpers (each a thin call into the C oracle)
# ---------------------------------------------------------------------------

def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter and 2-word key -> 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(v) for v in o]


def uniform(r: int) -> float:
    return lib().orc_uniform(int(r) & 0xFFFFFFFF)


def gumbel(r: int) -> float:
    return lib().orc_gumbel(int(r) & 0xFFFFFFFF)


def normals4(words):
    r = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in words])
    n = (ctypes.c_double * 4)()
    lib().orc_normals4(r, n)
    return [float(v) for v in n]


def param_count_shape(D, H, A, L, ns, out_bias, temp) -> int:
    """Parameter count of a policy with D inputs, ns sensors (one input
    bias each), L hidden H -> H layers, A actions, an optional head bias
    and an optional temperature parameter."""
    return int(lib().orc_param_count_shape(D, H, A, L, ns, int(out_bias), int(temp)))


def threshold(p: float) -> int:
    return int(lib().orc_threshold(float(p)))


def bf16_rne(f: float) -> int:
    return int(lib().orc_bf16_rne(float(f)))


def bf16_value(b: int) -> float:
    return float(lib().orc_bf16_value(int(b)))


def e4m3_encode(f: float) -> int:
    return int(lib().orc_e4m3_encode(float(f)))


def e4m3_value(b: int) -> float:
    return float(lib().orc_e4m3_value(int(b)))


def fp8_row_scale(row: np.ndarray) -> float:
    row = np.ascontiguousarray(row, dtype=np.float32)
    return float(lib().orc_fp8_row_scale(_ptr(row), int(row.size)))


# ---------------------------------------------------------------------------
# World state
# ---------------------------------------------------------------------------

def make_config(cfg: dict) -> Config:
    """Build the C config from a workload dictionary (one environment)."""
    flags = cfg.get("flags", 0)
    if not isinstance(flags, int):
        flags = sum(FLAG_NAMES[f] for f in flags)
    prec = cfg.get("precision", "fp32")
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    return Config(
        side=cfg["side"], slots=cfg["slots"], init_alive=cfg["init_alive"],
        patch_k=cfg["patch_k"], n_scalars=cfg["n_scalars"], hidden=cfg["hidden"],
        n_actions=cfg["n_actions"], precision=prec, flags=flags,
        seed=cfg.get("seed", 0) & 0xFFFFFFFF, sigma=cfg["sigma"],
        food_density=cfg["food_density"], regrow_p=cfg["regrow_p"],
        wall_density=cfg["wall_density"], e_init=cfg["e_init"],
        e_metab=cfg["e_metab"], e_food=cfg["e_food"], e_repro=cfg["e_repro"],
        attack_num=cfg["attack_num"], attack_den=cfg["attack_den"],
        policy_form=POLICY_FORMS[cfg.get("policy_form", "plain")]
        if isinstance(cfg.get("policy_form", "plain"), str) else int(cfg["policy_form"]),
        n_hidden=cfg.get("n_hidden", 1),
        rules=RULES[cfg.get("rules", "simple")],
        biomass_density=float(cfg.get("biomass_density", 0.0)),
        photo_q16=int(cfg.get("photo_q16", 0)), res_cap=int(cfg.get("res_cap", 0)),
        vision=VISIONS[cfg.get("vision", "channels")],
        view=VIEWS[cfg.get("view", "around")],
        **{k: int(cfg.get(k, 0)) for k in PAPER_RULE_FIELDS + TERRAIN_FIELDS})


class Oracle:
    """One environment held as numpy arrays, stepped by the C oracle."""

    ARRAYS = ("food", "wall", "occ", "alive", "x", "y", "facing", "energy",
              "parent", "birth_step", "master", "step", "hp", "age", "res", "colour",
              "rock", "water", "bio", "photo", "a_water", "a_bio")

    def __init__(self, cfg: dict, allocate: bool = True):
        self.cfg = dict(cfg)
        self.c = make_config(cfg)
        L = lib()
        self.D = L.orc_obs_dim(ctypes.byref(self.c))
        self.P = L.orc_n_params(ctypes.byref(self.c))
        self.side = cfg["side"]
        self.S = cfg["slots"]
        self.A = cfg["n_actions"]
        if allocate:
            N = self.side * self.side
            S = self.S
            self.food = np.zeros(N, np.uint8)
            self.wall = np.zeros(N, np.uint8)
            self.occ = np.full(N, -1, np.int32)
            self.alive = np.zeros(S, np.uint8)
            self.x = np.zeros(S, np.int32)
            self.y = np.zeros(S, np.int32)
            self.facing = np.zeros(S, np.uint8)
            self.energy = np.zeros(S, np.int32)
            self.parent = np.full(S, -1, np.int32)
            self.birth_step = np.full(S, -1, np.int32)
            self.master = np.zeros((S, self.P), np.float32)
            self.step = np.zeros(1, np.int64)
            self.hp = np.zeros(S, np.int32)
            self.age = np.zeros(S, np.int32)
            self.res = np.zeros(N, np.int32)
            self.colour = np.zeros((S, 3), np.float32)
            # terrain: the rock layer is an input (cfg["rock"], else flat 0)
            rock = cfg.get("rock")
            self.rock = (np.zeros(N, np.int32) if rock is None
                         else np.ascontiguousarray(rock, np.int32).ravel().copy())
            assert self.rock.size == N
            self.water = np.zeros(N, np.int32)
            self.bio = np.zeros(N, np.int32)
            self.photo = np.zeros(N, np.uint32)
            self.a_water = np.zeros(S, np.int32)
            self.a_bio = np.zeros(S, np.int32)

    # -- plumbing ----------------------------------------------------------
    def _state(self) -> State:
        return State(**{n: _ptr(getattr(self, n)) for n in self.ARRAYS})

    def copy(self) -> "Oracle":
        o = Oracle(self.cfg, allocate=False)
        for n in self.ARRAYS:
            setattr(o, n, getattr(self, n).copy())
        return o

    def arrays(self) -> dict:
        return {n: getattr(self, n) for n in self.ARRAYS}

    # -- the method --------------------------------------------------------
    def reset(self) -> None:
        st = self._state()
        rc = lib().orc_reset(ctypes.byref(self.c), ctypes.byref(st))
        if rc != 0:
            raise ValueError("oracle reset failed (%d)" % rc)

    def observe(self, slot: int) -> np.ndarray:
        x = np.zeros(self.D, np.float64)
        st = self._state()
        lib().orc_observe(ctypes.byref(self.c), ctypes.byref(st), int(slot), _ptr(x))
        return x

    def effective_params(self, slot: int, use_master: bool = False) -> np.ndarray:
        w = np.zeros(self.P, np.float64)
        row = np.ascontiguousarray(self.master[slot])
        lib().orc_effective_params(ctypes.byref(self.c), _ptr(row), int(use_master), _ptr(w))
        return w

    def weight_mask(self) -> np.ndarray:
        """bool[P]: True where logical parameter p is a weight (False: a
        bias or the temperature)."""
        m = np.zeros(self.P, np.uint8)
        lib().orc_weight_mask(ctypes.byref(self.c), _ptr(m))
        return m.astype(bool)

    def fp8_rows(self) -> int:
        """Weight rows that carry an FP8 scale: W_in, every hidden layer, the head."""
        L = self.cfg.get("n_hidden", 1) if self.c.policy_form == PAPER_FORM else 1
        H = self.cfg["hidden"]
        return H + L * H + self.A

    def quantise(self, rows: np.ndarray):
        """The streamed copy of master rows [n][P] (float32) in logical
        order: (codes, scales).  BF16: codes uint16 [n][P], scales None.
        FP8: codes uint8 [n][P] and row scales float32 [n][fp8_rows()].
        Bias positions hold the code of 0."""
        rows = np.ascontiguousarray(rows, np.float32).reshape(-1, self.P)
        n = rows.shape[0]
        if self.c.precision == BF16:
            codes, scales = np.zeros((n, self.P), np.uint16), None
        elif self.c.precision == FP8:
            codes, scales = np.zeros((n, self.P), np.uint8), np.zeros((n, self.fp8_rows()), np.float32)
        else:
            raise ValueError("the FP32 form has no streamed copy")
        for i in range(n):
            lib().orc_quantise(ctypes.byref(self.c), _ptr(rows[i]), _ptr(codes[i]),
                               _ptr(scales[i]) if scales is not None else None)
        return codes, scales

    def mlp(self, w: np.ndarray, x: np.ndarray) -> np.ndarray:
        w = np.ascontiguousarray(w, np.float64)
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros(self.A, np.float64)
        lib().orc_mlp(ctypes.byref(self.c), _ptr(w), _ptr(x), _ptr(out))
        return out

    def init_params(self, slot: int) -> np.ndarray:
        row = np.zeros(self.P, np.float32)
        lib().orc_init_params(ctypes.byref(self.c), int(slot), _ptr(row))
        return row

    def mutate(self, step: int, parent_slot: int, parent_row: np.ndarray) -> np.ndarray:
        parent_row = np.ascontiguousarray(parent_row, np.float32)
        child = np.zeros(self.P, np.float32)
        lib().orc_mutate(ctypes.byref(self.c), int(step), int(parent_slot),
                         _ptr(parent_row), _ptr(child))
        return child

    def mutate_colour(self, step: int, parent_slot: int, parent_rgb) -> np.ndarray:
        parent_rgb = np.ascontiguousarray(parent_rgb, np.float32)
        child = np.zeros(3, np.float32)
        lib().orc_mutate_colour(ctypes.byref(self.c), int(step), int(parent_slot),
                                _ptr(parent_rgb), _ptr(child))
        return child

    def water_flow(self) -> None:
        """One step of the terrain rules' water flow, alone."""
        st = self._state()
        if lib().orc_water_flow(ctypes.byref(self.c), ctypes.byref(st)) != 0:
            raise RuntimeError("oracle water flow failed")

    def policy(self, use_master: bool = False, tol: float = 1e-3) -> dict:
        S, A = self.S, self.A
        out = {"logits": np.zeros((S, A), np.float64),
               "scores": np.zeros((S, A), np.float64),
               "action": np.zeros(S, np.uint8),
               "valid": np.zeros(S, np.uint32)}
        st = self._state()
        rc = lib().orc_policy(ctypes.byref(self.c), ctypes.byref(st), int(use_master),
                              float(tol), _ptr(out["logits"]), _ptr(out["scores"]),
                              _ptr(out["action"]), _ptr(out["valid"]))
        if rc != 0:
            raise RuntimeError("oracle policy failed (%d)" % rc)
        return out

    def transition(self, action: np.ndarray):
        action = np.ascontiguousarray(action, np.uint8)
        stats = Stats()
        bp = np.zeros(self.S, np.int32)
        bc = np.zeros(self.S, np.int32)
        st = self._state()
        rc = lib().orc_transition(ctypes.byref(self.c), ctypes.byref(st), _ptr(action),
                                  ctypes.byref(stats), _ptr(bp), _ptr(bc))
        if rc != 0:
            raise RuntimeError("oracle transition failed (%d)" % rc)
        d = {n: int(getattr(stats, n)) for n in STAT_FIELDS}
        nb = d["births"]
        return d, list(zip(bp[:nb].tolist(), bc[:nb].tolist()))

    def step_once(self, tol: float = 1e-3):
        pol = self.policy(tol=tol)
        stats, births = self.transition(pol["action"])
        return pol, stats, births
