"""Lock-step comparison of the CUDA step (through the C-ABI) with the oracle.

Data flows from the oracle to the GPU only: after reset the oracle's
founders' parameters are written into the GPU, and after every step the
oracle's children's parameters are, so both sides always start a step from
identical states.  The GPU's output is compared, never copied into the
oracle.

Rules (written in the tests):
  * integer state and every statistic: bit-exact;
  * logits: |gpu - oracle| <= 1e-5 * max(1, max_a |oracle logit|) per agent;
  * actions: equal wherever the oracle's top-two gap of (logit + Gumbel)
    exceeds 1e-3; inside the gap the GPU's action must be one of the
    oracle's valid set, and the GPU state must then equal the oracle's
    transition taken with that valid choice (after which the GPU is reset to
    the oracle's own trajectory);
  * child parameters: |gpu - oracle| <= 2^-19 * (|parent| + |child - parent|)
    (FP32 Box-Muller on the GPU vs FP64 in the oracle, a few ulp);
  * colour traits: bit-exact, except a newborn's, which is held to the
    child-parameter bound (the same Box-Muller difference) and then
    replaced by the oracle's.
"""
import numpy as np

import oracle

STATE_KEYS = ("food", "wall", "occ", "alive", "x", "y", "facing", "energy", "parent",
              "birth_step", "hp", "age", "res", "water", "bio", "photo", "a_water", "a_bio")
LOGIT_RTOL = 1e-5
GAP_TOL = 1e-3
PARAM_RTOL = 2.0 ** -19

# statistic names shared by the GPU record and the oracle's per-step record
STEP_STATS = (["agent_steps"] + ["act%d" % i for i in range(16)] +
              ["moves", "move_blocked", "move_lost", "eaten", "attacks", "attack_hits",
               "energy_transferred", "deaths", "dead_energy", "births", "failed_births",
               "regrown", "alive", "food_total", "energy_total",
               "res_total", "eaten_energy", "metab_paid", "heals", "starved", "damage",
               "food_emptied", "food_refilled",
               "water_cells", "water_agents", "bio_cells", "bio_agents", "drunk", "water_spent",
               "thirsty", "bio_eaten", "photo", "dead_water", "dead_bio"])


def runs(slots):
    """Contiguous runs [a, b) of a sorted slot list."""
    out = []
    for s in sorted(set(int(v) for v in slots)):
        if out and out[-1][1] == s:
            out[-1][1] = s + 1
        else:
            out.append([s, s + 1])
    return out


def push_params(env, orc, slots, e=0, chunk=4096):
    for a, b in runs(slots):
        for c in range(a, b, chunk):
            env.write_params(e, c, orc.master[c:min(b, c + chunk)])


def compare_state(gs, orc, where=""):
    for k in STATE_KEYS:
        g, o = gs[k], getattr(orc, k)
        if not np.array_equal(g, o):
            idx = np.flatnonzero(g != o)[:8]
            raise AssertionError("%s: %s differs at %s: gpu %s oracle %s" %
                                 (where, k, idx.tolist(), g[idx].tolist(), o[idx].tolist()))
    assert int(gs["step"][0]) == int(orc.step[0]), where


def compare_stats(last, st, where=""):
    for k in STEP_STATS:
        assert last[k] == st[k], "%s: stat %s gpu %d oracle %d" % (where, k, last[k], st[k])


def compare_colours(gs, orc, births=(), where=""):
    got, want = gs["colour"], orc.colour
    fresh = np.zeros(len(want), bool)
    fresh[[c for _, c in births]] = True
    if not np.array_equal(got[~fresh], want[~fresh]):
        idx = np.flatnonzero((got != want).any(axis=1) & ~fresh)[:8]
        raise AssertionError("%s: colour differs at %s: gpu %s oracle %s" %
                             (where, idx.tolist(), got[idx].tolist(), want[idx].tolist()))
    err = 0.0
    for p, c in births:
        err = max(err, check_params(got[c], want[c], want[p], where + " colour of child %d" % c))
    return err


def push_colours(env, orc, e=0):
    env.write_state(e, {"colour": orc.colour})


def check_params(got, want, parent=None, where=""):
    ref = np.abs(want.astype(np.float64))
    if parent is not None:
        ref = np.abs(parent.astype(np.float64)) + np.abs(want.astype(np.float64) - parent)
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    bad = err > PARAM_RTOL * ref + 1e-30
    if bad.any():
        i = np.flatnonzero(bad.ravel())[:5]
        raise AssertionError("%s: params differ beyond tolerance at %s: gpu %s oracle %s" %
                             (where, i.tolist(), got.ravel()[i].tolist(), want.ravel()[i].tolist()))
    return float((err / np.maximum(ref, 1e-30)).max()) if err.size else 0.0


def start_pair(env, orc, e=0, check_init=True, sample=None):
    """Reset both sides, check the reset state, then give the GPU the
    oracle's founders' parameters."""
    env.reset()
    orc.reset()
    gs = env.read_state(e)
    compare_state(gs, orc, "reset")
    compare_colours(gs, orc, (), "reset")
    K = int(orc.alive.sum())
    if check_init and K:
        slots = np.arange(K) if sample is None else np.unique(
            np.random.default_rng(0).integers(0, K, size=min(sample, K)))
        for a, b in runs(slots):
            check_params(env.read_params(e, a, b - a), orc.master[a:b], where="init params")
    push_params(env, orc, range(orc.S), e)


def check_policy(env, orc, pol, alive0, e=0, where=""):
    logits, act = env.read_policy_io(e)
    ref = pol["logits"][alive0]
    got = logits[alive0].astype(np.float64)
    if ref.size:
        scale = np.maximum(1.0, np.abs(ref).max(axis=1))
        err = float((np.abs(got - ref).max(axis=1) / scale).max())
        assert err <= LOGIT_RTOL, "%s: logit error %.3g" % (where, err)
    else:
        err = 0.0
    diff = alive0 & (act != pol["action"])
    if diff.any():
        ok = (pol["valid"][diff] >> act[diff].astype(np.uint32)) & 1
        assert ok.all(), "%s: action outside the oracle's valid set at %s" % (
            where, np.flatnonzero(diff)[ok == 0][:8].tolist())
    return err, act, diff


def lockstep(env, orc, steps, e=0, where="", vs_master=False):
    """Advance both sides `steps` steps in lock-step; returns a report.

    With vs_master, every step also evaluates the oracle on the FP32 master
    parameters (the unquantised policy) and records how far the GPU's
    logits are from it and how often the GPU's action agrees with it
    (quantisation error: reported, not bounded)."""
    rep = {"steps": 0, "ambiguous": 0, "births": 0, "max_logit_err": 0.0, "max_param_err": 0.0}
    if vs_master:
        rep.update({"agents": 0, "agree": 0, "master_err_max": 0.0, "master_err_sum": 0.0})
    for t in range(steps):
        tag = "%s step %d" % (where, int(orc.step[0]))
        alive0 = orc.alive.astype(bool).copy()
        pol = orc.policy(tol=GAP_TOL)
        ref = orc.policy(use_master=True, tol=GAP_TOL) if vs_master else None
        env.step(1)
        err, act, diff = check_policy(env, orc, pol, alive0, e, tag)
        rep["max_logit_err"] = max(rep["max_logit_err"], err)
        if vs_master and alive0.any():
            lg, _ = env.read_policy_io(e)
            r = ref["logits"][alive0]
            rel = np.abs(lg[alive0].astype(np.float64) - r).max(axis=1) / np.maximum(1.0, np.abs(r).max(axis=1))
            rep["master_err_max"] = max(rep["master_err_max"], float(rel.max()))
            rep["master_err_sum"] += float(rel.sum())
            rep["agents"] += int(alive0.sum())
            rep["agree"] += int((act[alive0] == ref["action"][alive0]).sum())
        last = env.stats("last")[e]
        gs = env.read_state(e)
        if diff.any():
            rep["ambiguous"] += int(diff.sum())
            alt = orc.copy()
            alt_act = pol["action"].copy()
            alt_act[diff] = act[diff]
            st_alt, births_alt = alt.transition(alt_act)
            compare_state(gs, alt, tag + " (valid alternative)")
            compare_stats(last, st_alt, tag + " (valid alternative)")
            compare_colours(gs, alt, births_alt, tag + " (valid alternative)")
            st, births = orc.transition(pol["action"])
            env.write_state(e, orc.arrays())
            push_params(env, orc, [c for _, c in births] + [c for _, c in births_alt], e)
        else:
            st, births = orc.transition(pol["action"])
            compare_state(gs, orc, tag)
            compare_stats(last, st, tag)
            rep["max_param_err"] = max(rep["max_param_err"], compare_colours(gs, orc, births, tag))
            if births:
                push_colours(env, orc, e)
                kids = [c for _, c in births]
                for p, c in births:
                    got = env.read_params(e, c, 1)[0]
                    rep["max_param_err"] = max(rep["max_param_err"], check_params(
                        got, orc.master[c], orc.master[p], tag + " child %d" % c))
                push_params(env, orc, kids, e)
        rep["births"] += len(births)
        rep["steps"] += 1
    return rep
