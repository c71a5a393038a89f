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
    replaced by the oracle's;
  * a child's streamed BF16 / FP8 copy, which the mutation kernel derives
    from the child's new FP32 master: codes, FP8 row scales and FP32 biases
    bit-exact against the oracle's quantiser applied to that same GPU
    master (RNE and IEEE division are deterministic), checked before the
    oracle's child replaces it.
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


def read_rows(env, slots, e=0):
    """GPU FP32 masters of `slots`, read run by run: {slot: row}."""
    out = {}
    for a, b in runs(slots):
        rows = env.read_params(e, a, b - a)
        for i in range(b - a):
            out[a + i] = rows[i]
    return out


def check_streamed(env, orc, masters, e=0, where=""):
    """The streamed copy of every slot in `masters` ({slot: GPU master row})
    against the oracle's quantiser applied to that master: codes, FP8 row
    scales and the FP32 biases, bit for bit.  Returns the slots checked."""
    if orc.c.precision == oracle.FP32 or not masters:
        return 0
    wmask = orc.weight_mask()
    for a, b in runs(masters):
        m = np.stack([masters[s] for s in range(a, b)])
        codes, scales = env.read_streamed(e, a, b - a)
        bias = env.read_streamed_bias(e, a, b - a)
        want_codes, want_scales = orc.quantise(m)
        if not np.array_equal(codes, want_codes):
            i, p = np.argwhere(codes != want_codes)[0]
            raise AssertionError("%s: streamed code of slot %d param %d: gpu %d oracle %d (master %r)" %
                                 (where, a + i, p, codes[i, p], want_codes[i, p], float(m[i, p])))
        if want_scales is not None and not np.array_equal(scales.view(np.uint32), want_scales.view(np.uint32)):
            i, r = np.argwhere(scales.view(np.uint32) != want_scales.view(np.uint32))[0]
            raise AssertionError("%s: FP8 row scale %d of slot %d: gpu %r oracle %r" %
                                 (where, r, a + i, float(scales[i, r]), float(want_scales[i, r])))
        want_bias = np.ascontiguousarray(m[:, ~wmask])
        if not np.array_equal(bias.view(np.uint32), want_bias.view(np.uint32)):
            i, k = np.argwhere(bias.view(np.uint32) != want_bias.view(np.uint32))[0]
            raise AssertionError("%s: streamed bias %d of slot %d: gpu %r master %r" %
                                 (where, k, a + i, float(bias[i, k]), float(want_bias[i, k])))
    return len(masters)


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


def new_report(vs_master=False):
    rep = {"steps": 0, "ambiguous": 0, "births": 0, "gpu_births": 0, "max_logit_err": 0.0,
           "max_param_err": 0.0, "streamed_checked": 0}
    if vs_master:
        rep.update({"agents": 0, "agree": 0, "master_err_max": 0.0, "master_err_sum": 0.0})
    return rep


def check_step(env, orc, pol, alive0, rep, e=0, tag="", ref=None):
    """After env stepped once from the state orc holds (pol: the oracle's
    policy on that state, alive0 its alive mask): check world e of env
    against the oracle's step, advance the oracle, and bring the GPU back
    onto the oracle's trajectory where the two may differ (near-ties,
    children's parameters).  ref: the oracle's policy on the FP32 masters,
    for the precision report."""
    err, act, diff = check_policy(env, orc, pol, alive0, e, tag)
    rep["max_logit_err"] = max(rep["max_logit_err"], err)
    if ref is not None and alive0.any():
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
        rep["streamed_checked"] += check_streamed(
            env, orc, read_rows(env, [c for _, c in births_alt], e), e, tag + " (valid alternative)")
        rep["gpu_births"] += len(births_alt)
        st, births = orc.transition(pol["action"])
        env.write_state(e, orc.arrays())
        push_params(env, orc, [c for _, c in births] + [c for _, c in births_alt], e)
    else:
        st, births = orc.transition(pol["action"])
        compare_state(gs, orc, tag)
        compare_stats(last, st, tag)
        rep["max_param_err"] = max(rep["max_param_err"], compare_colours(gs, orc, births, tag))
        rep["gpu_births"] += len(births)
        if births:
            push_colours(env, orc, e)
            kids = [c for _, c in births]
            got = read_rows(env, kids, e)
            for p, c in births:
                rep["max_param_err"] = max(rep["max_param_err"], check_params(
                    got[c], orc.master[c], orc.master[p], tag + " child %d" % c))
            rep["streamed_checked"] += check_streamed(env, orc, got, e, tag)
            push_params(env, orc, kids, e)
    rep["births"] += len(births)
    rep["steps"] += 1
    return st


def lockstep(env, orc, steps, e=0, where="", vs_master=False):
    """Advance both sides `steps` steps in lock-step; returns a report.

    With vs_master, every step also evaluates the oracle on the FP32 master
    parameters (the unquantised policy) and records how far the GPU's
    logits are from it and how often the GPU's action agrees with it
    (quantisation error: reported, not bounded)."""
    rep = new_report(vs_master)
    for t in range(steps):
        tag = "%s step %d" % (where, int(orc.step[0]))
        alive0 = orc.alive.astype(bool).copy()
        pol = orc.policy(tol=GAP_TOL)
        ref = orc.policy(use_master=True, tol=GAP_TOL) if vs_master else None
        env.step(1)
        check_step(env, orc, pol, alive0, rep, e, tag, ref)
    return rep


def lockstep_batch(env, orcs, steps, where=""):
    """Lock-step of a batched handle: every step advances all its worlds at
    once, then each world e is checked against its own oracle orcs[e] as
    lockstep checks a single world.  Returns one report per world, each
    with the statistics of every step ("per_step")."""
    reps = [new_report() for _ in orcs]
    for r in reps:
        r["per_step"] = []
    for t in range(steps):
        alive0 = [o.alive.astype(bool).copy() for o in orcs]
        pols = [o.policy(tol=GAP_TOL) for o in orcs]
        env.step(1)
        for e, o in enumerate(orcs):
            tag = "%s world %d step %d" % (where, e, int(o.step[0]))
            reps[e]["per_step"].append(check_step(env, o, pols[e], alive0[e], reps[e], e, tag))
    return reps
