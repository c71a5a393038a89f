"""Python binding of libeco.so, the C-ABI in include/eco.h.

The module-level functions carry the C names (``eco_create``, ``eco_reset``,
``eco_step``, ``eco_read_stats`` ...) and only marshal arguments; every
phase of the simulation step runs in the library's CUDA kernels.  PyTorch
supplies the device workspace (one ``torch.empty`` allocation) and the CUDA
stream.  There is no CPU fallback: if the library is missing the binding
raises.

``Env`` wraps a handle for one batch of environments described by workload
dictionaries (see ``workloads.py``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeco.so")

ECO_ABI_VERSION = 5
ECO_OK, ECO_EINVAL, ECO_ENOMEM, ECO_ECUDA, ECO_ETIMEOUT, ECO_EABI = 0, -1, -2, -3, -4, -5
ECO_FP32, ECO_BF16, ECO_FP8_E4M3 = 0, 1, 2
ECO_AUTO_EAT, ECO_ROTATE_OBS, ECO_CANCEL_ALL, ECO_GREEDY = 1, 2, 4, 8
PRECISIONS = {"fp32": ECO_FP32, "bf16": ECO_BF16, "fp8": ECO_FP8_E4M3}
ECO_POLICY_PLAIN, ECO_POLICY_PAPER = 0, 1
POLICY_FORMS = {"plain": ECO_POLICY_PLAIN, "paper": ECO_POLICY_PAPER}
ECO_RULES_SIMPLE, ECO_RULES_PAPER, ECO_RULES_TERRAIN = 0, 1, 2
RULES = {"simple": ECO_RULES_SIMPLE, "paper": ECO_RULES_PAPER, "terrain": ECO_RULES_TERRAIN}
TERRAIN_FIELDS = ("sea_level", "w_init", "w_metab", "w_bite", "w_cap", "w_child", "heal_water",
                  "b_body", "b_child", "b_bite", "b_cap", "b_site")
VISIONS = {"channels": 0, "rgb": 1}
VIEWS = {"around": 0, "front": 1}
PAPER_RULE_FIELDS = ("hp_max", "hp_child", "attack_damage", "heal_rate", "heal_cost",
                     "age_div", "starve_damage", "e_act", "e_cap", "e_child")
FLAGS = {"auto_eat": ECO_AUTO_EAT, "rotate_obs": ECO_ROTATE_OBS,
         "cancel_all": ECO_CANCEL_ALL, "greedy": ECO_GREEDY}

STAT_NAMES = (["step", "agent_steps"] + ["act%d" % i for i in range(16)] +
              ["moves", "move_blocked", "move_lost", "eaten", "attacks", "attack_hits",
               "energy_transferred", "deaths", "dead_energy", "births", "failed_births",
               "regrown", "alive", "food_total", "energy_total",
               "res_total", "eaten_energy", "metab_paid", "heals", "starved", "damage",
               "food_emptied", "food_refilled",
               "water_cells", "water_agents", "bio_cells", "bio_agents", "drunk", "water_spent",
               "thirsty", "bio_eaten", "photo", "dead_water", "dead_bio"])
ECO_N_STATS = len(STAT_NAMES)

_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p


class eco_config(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32), ("n_envs", ctypes.c_int32),
        ("env_side", _i32p), ("env_slots", _i32p), ("env_init_alive", _i32p),
        ("env_seed", _u32p),
        ("patch_k", ctypes.c_int32), ("n_scalars", ctypes.c_int32),
        ("hidden", ctypes.c_int32), ("n_actions", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("sigma", ctypes.c_float), ("food_density", ctypes.c_float),
        ("regrow_p", ctypes.c_float), ("wall_density", ctypes.c_float),
        ("e_init", ctypes.c_int32), ("e_metab", ctypes.c_int32),
        ("e_food", ctypes.c_int32), ("e_repro", ctypes.c_int32),
        ("attack_num", ctypes.c_int32), ("attack_den", ctypes.c_int32),
        ("policy_variant", ctypes.c_int32), ("launch_mode", ctypes.c_int32),
        ("policy_form", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
        ("rules", ctypes.c_int32),
    ] + [(k, ctypes.c_int32) for k in PAPER_RULE_FIELDS] + [
        ("vision", ctypes.c_int32), ("view", ctypes.c_int32)] + [
        (k, ctypes.c_int32) for k in TERRAIN_FIELDS] + [
        ("biomass_density", ctypes.c_float), ("photo_q16", ctypes.c_int32),
        ("res_cap", ctypes.c_int32)]


class eco_stats(ctypes.Structure):
    _fields_ = [("v", ctypes.c_int64 * ECO_N_STATS)]


class eco_state_view(ctypes.Structure):
    _fields_ = [(n, _vp) for n in ("food", "wall", "occ", "alive", "x", "y", "facing",
                                   "energy", "parent", "birth_step", "step", "hp", "age",
                                   "res", "colour", "water", "bio", "photo", "a_water",
                                   "a_bio")]


_lib = None


class EcoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("eco error %d: %s" % (code, msg))
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libeco.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libeco.so is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        cp = ctypes.POINTER(eco_config)
        H = _vp
        L.eco_param_count.argtypes = [cp, _i32p, _i32p]
        L.eco_workspace_bytes.argtypes = [cp, ctypes.POINTER(ctypes.c_size_t)]
        L.eco_create.argtypes = [cp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
        L.eco_reset.argtypes = [H]
        L.eco_reset_seed.argtypes = [H, ctypes.c_uint64]
        L.eco_arm_barrier_timeout.argtypes = [H, ctypes.c_int32, ctypes.c_int32]
        L.eco_trace_phases.argtypes = [H, ctypes.c_int32]
        L.eco_read_phase_trace.argtypes = [H, _vp, ctypes.c_int32, _i32p]
        L.eco_step.argtypes = [H, ctypes.c_int32]
        L.eco_step_timed.argtypes = [H, ctypes.c_int32]
        L.eco_prepare.argtypes = [H]
        L.eco_step_read.argtypes = [H, _vp, _vp, ctypes.c_int32]
        L.eco_policy_timing.argtypes = [H, ctypes.POINTER(ctypes.c_double), _i32p,
                                        ctypes.POINTER(ctypes.c_int64)]
        L.eco_read_stats.argtypes = [H, _vp, _vp, ctypes.c_int32]
        L.eco_read_state.argtypes = [H, ctypes.c_int32, ctypes.POINTER(eco_state_view)]
        L.eco_write_state.argtypes = [H, ctypes.c_int32, ctypes.POINTER(eco_state_view)]
        L.eco_set_rock.argtypes = [H, ctypes.c_int32, _vp]
        L.eco_get_rock.argtypes = [H, ctypes.c_int32, _vp]
        L.eco_read_params.argtypes = [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]
        L.eco_write_params.argtypes = [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]
        L.eco_read_streamed.argtypes = [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
        L.eco_read_streamed_bias.argtypes = [H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]
        L.eco_read_policy_io.argtypes = [H, ctypes.c_int32, _vp, _vp]
        L.eco_policy_variants.argtypes = [H, _i32p, _i32p]
        L.eco_policy_variant_name.argtypes = [ctypes.c_int32]
        L.eco_policy_variant_name.restype = ctypes.c_char_p
        L.eco_policy_only.argtypes = [H, ctypes.c_int32]
        L.eco_launch_mode.argtypes = [H, _i32p, _i32p]
        L.eco_policy_bytes.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.eco_move_claims_noalloc.argtypes = [
            ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32,
            _vp, _vp, _vp, _vp]
        L.eco_destroy.argtypes = [H]
        L.eco_destroy.restype = None
        L.eco_last_error.argtypes = [H]
        L.eco_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, h=None) -> None:
    if rc != ECO_OK:
        msg = lib().eco_last_error(h)
        raise EcoError(rc, msg.decode() if msg else "")


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# Thin wrappers with the C names
# ---------------------------------------------------------------------------

def eco_param_count(cfg: eco_config):
    p, d = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().eco_param_count(ctypes.byref(cfg), ctypes.byref(p), ctypes.byref(d)))
    return p.value, d.value


def eco_workspace_bytes(cfg: eco_config) -> int:
    n = ctypes.c_size_t()
    _check(lib().eco_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def eco_create(cfg: eco_config, workspace_ptr: int, nbytes: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(lib().eco_create(ctypes.byref(cfg), ctypes.c_void_p(workspace_ptr), nbytes,
                            ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h


def eco_reset(h) -> None:
    _check(lib().eco_reset(h), h)


def eco_reset_seed(h, seed: int) -> None:
    _check(lib().eco_reset_seed(h, int(seed) & 0xFFFFFFFFFFFFFFFF), h)


def eco_arm_barrier_timeout(h, absent_cta: int, poll_budget: int) -> None:
    """Failure-detection test hook (see include/eco.h)."""
    _check(lib().eco_arm_barrier_timeout(h, int(absent_cta), int(poll_budget)), h)


ECO_TRACE_STEPS = 64
ECO_TRACE_WORDS = 16


def eco_trace_phases(h, on: bool) -> None:
    """Switch the environment kernel's phase trace on or off (see include/eco.h)."""
    _check(lib().eco_trace_phases(h, 1 if on else 0), h)


def eco_read_phase_trace(h) -> np.ndarray:
    """The trace table, uint64 [ECO_TRACE_STEPS][ECO_TRACE_WORDS]."""
    rows = np.zeros((ECO_TRACE_STEPS, ECO_TRACE_WORDS), np.uint64)
    n = ctypes.c_int32()
    _check(lib().eco_read_phase_trace(h, rows.ctypes.data, ECO_TRACE_STEPS, ctypes.byref(n)), h)
    return rows[:n.value]


def eco_step(h, n_steps: int) -> None:
    _check(lib().eco_step(h, int(n_steps)), h)


def eco_prepare(h) -> None:
    _check(lib().eco_prepare(h), h)


def eco_step_read(h, n_envs: int):
    """One pipelined step: returns the (total, last) records of the step the
    previous call enqueued, while this call's step runs."""
    tot = np.zeros((n_envs, ECO_N_STATS), np.int64)
    last = np.zeros((n_envs, ECO_N_STATS), np.int64)
    _check(lib().eco_step_read(h, _p(tot), _p(last), int(n_envs)), h)
    return tot, last


def eco_step_timed(h, n_steps: int) -> None:
    _check(lib().eco_step_timed(h, int(n_steps)), h)


def eco_policy_timing(h):
    """(summed policy-kernel ms, timed launches, agents in those launches)."""
    ms, n, ag = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().eco_policy_timing(h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(ag)), h)
    return ms.value, n.value, ag.value


def eco_read_stats(h, n_envs: int):
    tot = np.zeros((n_envs, ECO_N_STATS), np.int64)
    last = np.zeros((n_envs, ECO_N_STATS), np.int64)
    _check(lib().eco_read_stats(h, _p(tot), _p(last), int(n_envs)), h)
    return tot, last


def eco_policy_only(h, n_iters: int) -> None:
    _check(lib().eco_policy_only(h, int(n_iters)), h)


def eco_policy_bytes(h):
    b, n = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().eco_policy_bytes(h, ctypes.byref(b), ctypes.byref(n)), h)
    return b.value, n.value


def eco_policy_variants(h):
    c, ch = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().eco_policy_variants(h, ctypes.byref(c), ctypes.byref(ch)))
    return c.value, ch.value


def eco_launch_mode(h):
    m, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().eco_launch_mode(h, ctypes.byref(m), ctypes.byref(b)), h)
    return m.value, b.value


def eco_policy_variant_name(k: int) -> str:
    return lib().eco_policy_variant_name(int(k)).decode()


def eco_destroy(h) -> None:
    lib().eco_destroy(h)


def eco_move_claims_noalloc(side: int, n_agents: int, pos: int, act: int, facing_in: int,
                            blocked: int, seed: int, step: int, facing_out: int, pos_out: int,
                            moved: int, stream: int) -> None:
    """Movement-claim resolution with no device allocation (all array
    arguments are device pointers owned by the caller; see include/eco.h
    for who needs it and its limits)."""
    _check(lib().eco_move_claims_noalloc(
        int(side), int(n_agents), _vp(pos), _vp(act), _vp(facing_in), _vp(blocked),
        int(seed) & 0xFFFFFFFF, int(step) & 0xFFFFFFFF, _vp(facing_out), _vp(pos_out),
        _vp(moved), _vp(stream)))


# ---------------------------------------------------------------------------
# Env: a handle plus its torch-owned workspace and stream
# ---------------------------------------------------------------------------

_SHARED = ("patch_k", "n_scalars", "hidden", "n_actions", "precision", "flags", "sigma",
           "food_density", "regrow_p", "wall_density", "e_init", "e_metab", "e_food",
           "e_repro", "attack_num", "attack_den", "policy_form", "n_hidden",
           "rules", "vision", "view", "biomass_density", "photo_q16",
           "res_cap") + PAPER_RULE_FIELDS + TERRAIN_FIELDS


def make_config(envs: Sequence[dict], policy_variant: int = 0, launch_mode: int = 0):
    """An eco_config for environments sharing rules and MLP shape (the
    per-environment arrays are returned too, to keep them alive)."""
    envs = list(envs)
    w0 = envs[0]
    for w in envs[1:]:
        for k in _SHARED:
            if w.get(k) != w0.get(k):
                raise ValueError("environments differ in %r" % k)
    side = (ctypes.c_int32 * len(envs))(*[w["side"] for w in envs])
    slots = (ctypes.c_int32 * len(envs))(*[w["slots"] for w in envs])
    alive = (ctypes.c_int32 * len(envs))(*[w["init_alive"] for w in envs])
    seed = (ctypes.c_uint32 * len(envs))(*[w.get("seed", 0) & 0xFFFFFFFF for w in envs])
    flags = w0.get("flags", 0)
    if not isinstance(flags, int):
        flags = sum(FLAGS[f] for f in flags)
    prec = w0.get("precision", "fp32")
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    cfg = eco_config(
        abi_version=ECO_ABI_VERSION, n_envs=len(envs), env_side=side, env_slots=slots,
        env_init_alive=alive, env_seed=seed, patch_k=w0["patch_k"], n_scalars=w0["n_scalars"],
        hidden=w0["hidden"], n_actions=w0["n_actions"], precision=prec, flags=flags,
        sigma=w0["sigma"], food_density=w0["food_density"], regrow_p=w0["regrow_p"],
        wall_density=w0["wall_density"], e_init=w0["e_init"], e_metab=w0["e_metab"],
        e_food=w0["e_food"], e_repro=w0["e_repro"], attack_num=w0["attack_num"],
        attack_den=w0["attack_den"], policy_variant=policy_variant, launch_mode=launch_mode,
        policy_form=POLICY_FORMS[w0.get("policy_form", "plain")], n_hidden=w0.get("n_hidden", 1),
        rules=RULES[w0.get("rules", "simple")],
        vision=VISIONS[w0.get("vision", "channels")], view=VIEWS[w0.get("view", "around")],
        biomass_density=float(w0.get("biomass_density", 0.0)),
        photo_q16=int(w0.get("photo_q16", 0)), res_cap=int(w0.get("res_cap", 0)),
        **{k: int(w0.get(k, 0)) for k in TERRAIN_FIELDS},
        **{k: int(w0.get(k, 0)) for k in PAPER_RULE_FIELDS})
    return cfg, (side, slots, alive, seed)


class Env:
    """One or more environments advanced together on the current GPU."""

    def __init__(self, envs, policy_variant: int = 0, stream=None, launch_mode: int = 0):
        import torch
        if isinstance(envs, dict):
            envs = [envs]
        self.envs = list(envs)
        self.cfg, self._keep = make_config(self.envs, policy_variant, launch_mode)
        self.P, self.D = eco_param_count(self.cfg)
        self.A = self.cfg.n_actions
        self.H = self.cfg.hidden
        self.n_envs = len(self.envs)
        nbytes = eco_workspace_bytes(self.cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.h = eco_create(self.cfg, aligned, nbytes, self.stream.cuda_stream)
        self.workspace_bytes = nbytes
        for e, w in enumerate(self.envs):   # terrain rules: the rock layers
            if w.get("rock") is not None:
                self.set_rock(e, w["rock"])

    # -- lifecycle ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "h", None):
            eco_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the step ------------------------------------------------------------
    def reset(self) -> None:
        eco_reset(self.h)

    def reset_seed(self, seed: int) -> None:
        """Reset with environment e seeded (seed + e) mod 2^32."""
        eco_reset_seed(self.h, seed)

    def step(self, n: int = 1) -> None:
        eco_step(self.h, n)

    def prepare(self) -> None:
        eco_prepare(self.h)

    def step_timed(self, n: int = 1) -> None:
        eco_step_timed(self.h, n)

    def policy_timing(self):
        return eco_policy_timing(self.h)

    def policy_only(self, n: int = 1) -> None:
        eco_policy_only(self.h, n)

    def policy_bytes(self):
        return eco_policy_bytes(self.h)

    def trace_phases(self, on: bool = True) -> None:
        eco_trace_phases(self.h, on)

    def phase_trace(self) -> np.ndarray:
        return eco_read_phase_trace(self.h)

    def launch_mode(self):
        """(0 persistent / 1 one kernel per phase, persistent CTAs)."""
        return eco_launch_mode(self.h)

    def variants(self):
        return eco_policy_variants(self.h)

    # -- statistics and state ----------------------------------------------
    def stats(self, which: str = "total"):
        tot, last = eco_read_stats(self.h, self.n_envs)
        arr = tot if which == "total" else last
        return [dict(zip(STAT_NAMES, row.tolist())) for row in arr]

    def read_state(self, env: int = 0) -> dict:
        w = self.envs[env]
        N, S = w["side"] * w["side"], w["slots"]
        out = {"food": np.zeros(N, np.uint8), "wall": np.zeros(N, np.uint8),
               "occ": np.zeros(N, np.int32), "alive": np.zeros(S, np.uint8),
               "x": np.zeros(S, np.int32), "y": np.zeros(S, np.int32),
               "facing": np.zeros(S, np.uint8), "energy": np.zeros(S, np.int32),
               "parent": np.zeros(S, np.int32), "birth_step": np.zeros(S, np.int32),
               "step": np.zeros(1, np.int64), "hp": np.zeros(S, np.int32),
               "age": np.zeros(S, np.int32), "res": np.zeros(N, np.int32),
               "colour": np.zeros((S, 3), np.float32), "water": np.zeros(N, np.int32),
               "bio": np.zeros(N, np.int32), "photo": np.zeros(N, np.uint32),
               "a_water": np.zeros(S, np.int32), "a_bio": np.zeros(S, np.int32)}
        v = eco_state_view(**{k: _p(a) for k, a in out.items()})
        _check(lib().eco_read_state(self.h, int(env), ctypes.byref(v)), self.h)
        return out

    def write_state(self, env: int, arrays: dict) -> None:
        keep = {}
        kw = {}
        for k in eco_state_view._fields_:
            name = k[0]
            if name in arrays and arrays[name] is not None:
                dt = {"food": np.uint8, "wall": np.uint8, "occ": np.int32, "alive": np.uint8,
                      "x": np.int32, "y": np.int32, "facing": np.uint8, "energy": np.int32,
                      "parent": np.int32, "birth_step": np.int32, "step": np.int64,
                      "hp": np.int32, "age": np.int32, "res": np.int32,
                      "colour": np.float32, "water": np.int32, "bio": np.int32,
                      "photo": np.uint32, "a_water": np.int32, "a_bio": np.int32}[name]
                a = np.ascontiguousarray(arrays[name], dtype=dt)
                keep[name] = a
                kw[name] = _p(a)
        v = eco_state_view(**kw)
        _check(lib().eco_write_state(self.h, int(env), ctypes.byref(v)), self.h)

    def set_rock(self, env: int, rock) -> None:
        side = self.envs[env]["side"]
        rock = np.ascontiguousarray(rock, np.int32).ravel()
        if rock.size != side * side:
            raise ValueError("rock must hold side * side heights")
        _check(lib().eco_set_rock(self.h, int(env), _p(rock)), self.h)

    def get_rock(self, env: int = 0) -> np.ndarray:
        side = self.envs[env]["side"]
        out = np.zeros(side * side, np.int32)
        _check(lib().eco_get_rock(self.h, int(env), _p(out)), self.h)
        return out

    def read_params(self, env: int = 0, slot0: int = 0, n: int | None = None) -> np.ndarray:
        if n is None:
            n = self.envs[env]["slots"] - slot0
        out = np.zeros((n, self.P), np.float32)
        _check(lib().eco_read_params(self.h, int(env), int(slot0), int(n), _p(out)), self.h)
        return out

    def write_params(self, env: int, slot0: int, params: np.ndarray) -> None:
        params = np.ascontiguousarray(params, np.float32).reshape(-1, self.P)
        _check(lib().eco_write_params(self.h, int(env), int(slot0), int(params.shape[0]),
                                      _p(params)), self.h)

    def read_streamed(self, env: int = 0, slot0: int = 0, n: int = 1):
        prec = self.cfg.precision
        codes = np.zeros((n, self.P), np.uint16 if prec == ECO_BF16 else np.uint8)
        layers = self.cfg.n_hidden if self.cfg.policy_form == ECO_POLICY_PAPER else 1
        scales = np.zeros((n, self.H + layers * self.H + self.A), np.float32)
        _check(lib().eco_read_streamed(self.h, int(env), int(slot0), int(n), _p(codes),
                                       _p(scales)), self.h)
        return codes, (scales if prec == ECO_FP8_E4M3 else None)

    def read_streamed_bias(self, env: int = 0, slot0: int = 0, n: int = 1) -> np.ndarray:
        """FP32 biases of the streamed copy, [n][nB] in ascending logical
        position (nB = P minus the weights)."""
        H, A = self.H, self.A
        layers = self.cfg.n_hidden if self.cfg.policy_form == ECO_POLICY_PAPER else 1
        n_w = self.D * H + layers * H * H + A * H
        out = np.zeros((n, self.P - n_w), np.float32)
        _check(lib().eco_read_streamed_bias(self.h, int(env), int(slot0), int(n), _p(out)), self.h)
        return out

    def read_policy_io(self, env: int = 0):
        S = self.envs[env]["slots"]
        logits = np.zeros((S, self.A), np.float32)
        act = np.zeros(S, np.uint8)
        _check(lib().eco_read_policy_io(self.h, int(env), _p(logits), _p(act)), self.h)
        return logits, act
