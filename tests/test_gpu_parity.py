"""Parity of the CUDA step (through the C-ABI) with the CPU oracle, on the
GPU.  Lock-step rules are in tests/harness.py."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2510_18221_gb300 import workloads
from tests import harness

pytestmark = pytest.mark.gpu


def _pair(w, **kw):
    from paper_2510_18221_gb300 import eco
    return eco.Env(w, **kw), oracle.Oracle(w)


def _run(w, steps, **kw):
    env, orc = _pair(w, **kw)
    try:
        harness.start_pair(env, orc)
        return harness.lockstep(env, orc, steps, where=w["name"])
    finally:
        env.close()


def test_small_workload_100_steps():
    rep = _run(workloads.get("small"), 100)
    assert rep["steps"] == 100 and rep["births"] > 0


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_mid_rules_scaled_with_births(prec):
    # mid rules on a 128x128 grid; founders start near the reproduction
    # threshold so births, slot reuse and mutation happen within the run
    w = workloads.scaled("mid", 128, 2048, 1500, precision=prec, e_init=190)
    rep = _run(w, 25)
    assert rep["births"] > 20


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_mid_workload_seeds(seed):
    # 512x512, 16,384 slots, 12,000 founders, 371 -> 64 -> 64 -> 9, FP32
    rep = _run(workloads.get("mid", seed=seed), 3)
    assert rep["steps"] == 3


def test_large_rules_fp8_scaled():
    # 15x15 patch, 683 -> 128 -> 128 -> 9, FP8 e4m3 + row scales
    w = workloads.scaled("large", 128, 1024, 900, e_init=195)
    rep = _run(w, 6)
    assert rep["steps"] == 6


@pytest.mark.parametrize("flags", [("rotate_obs", "cancel_all"), ("greedy",), ()])
def test_rule_flags(flags):
    w = workloads.scaled("mid", 64, 512, 400, flags=flags, e_init=190)
    _run(w, 10)


@pytest.mark.parametrize("variant", list(range(1, 11)))
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_every_policy_variant(variant, prec):
    w = workloads.scaled("mid", 64, 512, 450, precision=prec)
    _run(w, 3, policy_variant=variant)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_policy_variants_bit_identical(prec):
    """Every dense variant computes each agent in the same order (units in
    ascending order per lane, a fixed reduce-scatter), whatever its warps,
    units in flight or registers, and whichever warp takes the agent: the
    autotuner's choice does not change a single bit of logits or state."""
    from paper_2510_18221_gb300 import eco
    w = workloads.scaled("mid", 128, 2048, 1500, precision=prec, e_init=185)
    envs = [eco.Env(w, policy_variant=v) for v in (1, 2, 4, 6, 9, 10)]
    for x in envs:
        x.reset()
    for t in range(6):
        for x in envs:
            x.step(1)
        ref_l, ref_a = envs[0].read_policy_io(0)
        ref_s = envs[0].read_state(0)
        for x in envs[1:]:
            lg, ac = x.read_policy_io(0)
            assert np.array_equal(lg, ref_l) and np.array_equal(ac, ref_a), t
            st = x.read_state(0)
            for k in harness.STATE_KEYS:
                assert np.array_equal(st[k], ref_s[k]), (t, k)
    for x in envs:
        x.close()


def test_edge_no_founders_and_full_slots():
    _run(workloads.get("small", init_alive=0), 3)
    _run(workloads.get("small", init_alive=256, e_init=250), 5)   # births with no free slot
    _run(workloads.get("small", side=6, slots=40, init_alive=10), 10)   # tiny 6x6 torus, patch wraps


def test_ragged_slot_counts():
    for slots, k in [(1, 1), (33, 20), (257, 200), (1000, 999)]:
        _run(workloads.scaled("mid", 64, slots, k, precision="bf16"), 3)


def test_quantised_copy_bit_exact():
    from paper_2510_18221_gb300 import eco
    from tests import inputs
    for prec in ("bf16", "fp8"):
        w = workloads.scaled("mid", 32, 16, 8, precision=prec)
        env = eco.Env(w)
        orc = oracle.Oracle(w)
        rows = inputs.random_params(orc.P, n_rows=16, seed=3)
        rows[5] = 0.0                                          # all-zero rows
        rows[6, :100] *= 1e-3
        env.write_params(0, 0, rows)
        assert np.array_equal(env.read_params(0, 0, 16), rows)
        codes, scales = env.read_streamed(0, 0, 16)
        D, H, A = orc.D, orc.cfg["hidden"], orc.A
        nW1 = H * D
        for s in range(16):
            m = rows[s]
            if prec == "bf16":
                want = [oracle.bf16_rne(v) for v in m[:nW1]]
                assert np.array_equal(codes[s, :nW1], np.array(want, np.uint16))
            else:
                for o in range(H):
                    row = m[o * D:(o + 1) * D]
                    sc = oracle.fp8_row_scale(row)
                    assert scales[s, o] == np.float32(sc)
                    want = [oracle.e4m3_encode(float(np.float32(v) / np.float32(sc))) for v in row]
                    assert np.array_equal(codes[s, o * D:(o + 1) * D], np.array(want, np.uint8))
        env.close()


def test_batched_equals_single_and_oracle():
    from paper_2510_18221_gb300 import eco
    envs = [workloads.scaled("mid", s, n, k, seed=10 + i, precision="bf16", e_init=190)
            for i, (s, n, k) in enumerate([(64, 512, 300), (128, 1280, 1000), (32, 256, 200), (64, 768, 700)])]
    batch = eco.Env(envs)
    batch.reset()
    singles = [eco.Env(w) for w in envs]
    orcs = [oracle.Oracle(w) for w in envs]
    for e, (s, o) in enumerate(zip(singles, orcs)):
        s.reset()
        o.reset()
        harness.push_params(batch, o, range(o.S), e)
        harness.push_params(s, o, range(o.S), 0)
    for t in range(8):
        batch.step(1)
        for e, s in enumerate(singles):
            s.step(1)
            a, b = batch.read_state(e), s.read_state(0)
            for k in harness.STATE_KEYS:
                assert np.array_equal(a[k], b[k]), (t, e, k)
            la, aa = batch.read_policy_io(e)
            lb, ab = s.read_policy_io(0)
            alive = a["alive"].astype(bool)
            assert np.array_equal(aa[alive], ab[alive])
            assert np.array_equal(la[b["alive"].astype(bool) | alive], lb[b["alive"].astype(bool) | alive])
            assert batch.stats("last")[e] == s.stats("last")[0]
    # and every environment of the batch against its oracle, with its
    # statistics, through near-ties (the harness's valid-set rule)
    batch2 = eco.Env(envs)
    for o in orcs:
        o.reset()
    batch2.reset()
    for e, o in enumerate(orcs):
        harness.compare_state(batch2.read_state(e), o, "batched reset env %d" % e)
        harness.push_params(batch2, o, range(o.S), e)
    reps = harness.lockstep_batch(batch2, orcs, 8, where="batched")
    assert all(r["steps"] == 8 for r in reps)
    assert sum(r["births"] for r in reps) > 0
    batch.close()
    batch2.close()
    for s in singles:
        s.close()


@pytest.mark.parametrize("e_init", [100, 195])
def test_batched_workload_lockstep(e_init):
    """Twelve worlds of the batched workload's distribution (sides 128 to
    1024, lognormal populations; the many-worlds shape of App. F.3) in one
    handle, each in lock-step with its own oracle for 6 steps: state,
    actions, logits and every statistic per world.  e_init 195 puts most
    founders near the reproduction threshold, so births happen in every
    world within the run."""
    from paper_2510_18221_gb300 import eco
    ws = [dict(w, e_init=e_init) for w in workloads.batched(n_envs=12, seed=0)]
    assert {w["side"] for w in ws} == {128, 256, 512, 1024}
    env = eco.Env(ws)
    orcs = [oracle.Oracle(w) for w in ws]
    try:
        env.reset()
        for e, o in enumerate(orcs):
            o.reset()
            harness.compare_state(env.read_state(e), o, "batched reset env %d" % e)
            harness.push_params(env, o, range(o.S), e)
        reps = harness.lockstep_batch(env, orcs, 6, where="batched-12")
    finally:
        env.close()
    assert all(r["steps"] == 6 for r in reps)
    if e_init == 195:
        assert all(r["births"] > 0 for r in reps)
        assert sum(r["streamed_checked"] for r in reps) == sum(r["gpu_births"] for r in reps)
    print("batched lock-step:", [(r["births"], r["ambiguous"], r["max_logit_err"]) for r in reps])


@pytest.mark.parametrize("slots,launch_mode", [(8192, 0), (8192, 1), (5000, 0)])
def test_full_scan_birth_assignment(slots, launch_mode):
    """More than 2,048 birth contenders in one world in one step: slot
    assignment leaves the sorted-winner path for the full scan of the
    world's slots (winners in ascending slot order take the free slots in
    ascending order; Sec. 3.2, reproduction onto the cell behind).  4,000
    founders at e_init 250 on a 128x128 world all reach the threshold in the
    first step.  With 5,000 slots only 1,000 are free, so most winners fail
    (counted) on the same path."""
    w = workloads.scaled("mid", 128, slots, 4000, precision="bf16", e_init=250)
    env, orc = _pair(w, launch_mode=launch_mode)
    try:
        harness.start_pair(env, orc)
        rep = harness.lockstep(env, orc, 1, where=w["name"])
        first = env.stats("last")[0]
        assert first["births"] + first["failed_births"] > 2048, first
        if slots == 5000:
            assert first["births"] == 1000 and first["failed_births"] > 1000
        rep2 = harness.lockstep(env, orc, 5, where=w["name"])
        assert rep["streamed_checked"] + rep2["streamed_checked"] == rep["gpu_births"] + rep2["gpu_births"]
    finally:
        env.close()


def test_phase_trace_changes_nothing_and_is_ordered():
    """Steps with the environment kernel's phase trace on give the same
    state and statistics bit for bit as steps without it, and every traced
    row is ordered: the last CTA arrives at a barrier before CTA 0 passes
    it, arrives at the next barrier after that, and ends last."""
    from paper_2510_18221_gb300 import eco
    w = workloads.scaled("mid", 256, 8192, 6000, precision="bf16", e_init=185, seed=3)
    a, b = eco.Env(w), eco.Env(w)
    try:
        for x in (a, b):
            x.reset()
            x.prepare()
        if a.launch_mode()[0] != 0:
            pytest.skip("the persistent launch form is not in use")
        a.trace_phases(True)
        a.step(12)
        b.step(12)
        sa, sb = a.read_state(0), b.read_state(0)
        for k in harness.STATE_KEYS:
            assert np.array_equal(sa[k], sb[k]), k
        assert a.stats()[0] == b.stats()[0]
        assert np.array_equal(a.read_params(0), b.read_params(0))
        rows = a.phase_trace().astype(np.int64)
        rows = rows[rows[:, 0] > 0]
        assert len(rows) == 12
        assert sorted(rows[:, 10].tolist()) == list(range(int(rows[:, 10].min()), int(rows[:, 10].min()) + 12))
        for r in rows:
            nbar = int(r[12])
            assert nbar in (3, 4)
            prev = r[0]                         # CTA 0's start
            for k in range(nbar):
                # the last arrival at k follows CTA 0's pass through k - 1
                # (CTA 0 arrives at k after it), and CTA 0 passes k after it
                assert r[1 + k] >= prev and r[5 + k] >= r[1 + k], (r.tolist(), k)
                prev = r[5 + k]
            assert r[9] >= prev
        assert (rows[:, 11] > 0).any()          # births were claimed in some traced steps
        a.trace_phases(False)
        a.step(2)
        assert (a.phase_trace() == 0).all()     # off: nothing recorded
    finally:
        a.close()
        b.close()


def test_barrier_timeout_is_reported_and_reset_recovers():
    """Failure detection without a GPU fault: one CTA of the persistent
    environment kernel leaves before its first grid barrier (the hook
    eco_arm_barrier_timeout), so the other CTAs' bounded waits run out
    after 10^5 polls.  The status word reaches the host as ECO_ETIMEOUT,
    nothing waits without bound, and eco_reset clears the barrier, the
    status and the hook: the next steps are in lock-step with the oracle."""
    from paper_2510_18221_gb300 import eco
    w = workloads.scaled("mid", 128, 8192, 4000, precision="bf16", e_init=190)
    env, orc = _pair(w)
    try:
        env.reset()
        env.step(2)
        mode, blocks = env.launch_mode()
        assert mode == 0 and blocks > 1
        eco.eco_arm_barrier_timeout(env.h, blocks - 1, 100000)
        env.step(9)          # a graph of 8 steps, then one more
        with pytest.raises(eco.EcoError) as ex:
            env.stats()
        assert ex.value.code == eco.ECO_ETIMEOUT and "budget" in str(ex.value)
        with pytest.raises(eco.EcoError) as ex:
            eco.eco_step_read(env.h, 1)
        assert ex.value.code == eco.ECO_ETIMEOUT
        harness.start_pair(env, orc)
        rep = harness.lockstep(env, orc, 6, where="after a timeout")
        assert rep["steps"] == 6 and rep["births"] > 0
        assert env.stats()[0]["step"] == 6
    finally:
        env.close()
    b = eco.Env(w, launch_mode=1)   # the per-phase form has no grid barrier
    try:
        b.reset()
        b.step(1)
        with pytest.raises(eco.EcoError) as ex:
            eco.eco_arm_barrier_timeout(b.h, 0, 1000)
        assert ex.value.code == eco.ECO_EINVAL
    finally:
        b.close()


def test_reset_seed_matches_config_seeds():
    """eco_reset_seed(s) gives world e the seed s + e: the same reset and
    steps as a handle created with those seeds in its configuration, and as
    the oracle."""
    from paper_2510_18221_gb300 import eco
    ws = [workloads.scaled("mid", 64, 600, 500, precision="bf16", seed=1),
          workloads.scaled("mid", 32, 300, 200, precision="bf16", seed=2)]
    a = eco.Env(ws)
    b = eco.Env([dict(w, seed=77 + e) for e, w in enumerate(ws)])
    try:
        a.reset()
        a.step(3)
        a.reset_seed(77)
        b.reset()
        for e in range(2):
            harness.compare_state(a.read_state(e), _reset_oracle(dict(ws[e], seed=77 + e)),
                                  "reset_seed env %d" % e)
            assert np.array_equal(a.read_params(e), b.read_params(e))
        a.step(5)
        b.step(5)
        for e in range(2):
            sa, sb = a.read_state(e), b.read_state(e)
            for k in harness.STATE_KEYS:
                assert np.array_equal(sa[k], sb[k]), (e, k)
            assert a.stats()[e] == b.stats()[e]
    finally:
        a.close()
        b.close()


def _reset_oracle(w):
    o = oracle.Oracle(w)
    o.reset()
    return o


def test_launch_forms_bit_identical():
    """The persistent cooperative kernel and one kernel per phase run the
    same phase functions: every array and statistic must match."""
    from paper_2510_18221_gb300 import eco
    envs = [workloads.scaled("mid", s, n, k, seed=40 + i, precision="bf16", e_init=185)
            for i, (s, n, k) in enumerate([(64, 600, 500), (128, 2048, 1500), (32, 300, 250)])]
    a = eco.Env(envs, launch_mode=0)
    b = eco.Env(envs, launch_mode=1)
    a.reset()
    b.reset()
    a.step(1)
    b.step(1)
    assert b.launch_mode()[0] == 1
    assert a.launch_mode()[0] == 0 and a.launch_mode()[1] > 0   # GB300 supports the persistent form
    for t in range(6):
        a.step(5)
        b.step(5)
        for e in range(len(envs)):
            sa, sb = a.read_state(e), b.read_state(e)
            for k in harness.STATE_KEYS:
                assert np.array_equal(sa[k], sb[k]), (t, e, k)
            assert a.stats()[e] == b.stats()[e]
            assert np.array_equal(a.read_params(e), b.read_params(e))
    assert sum(s["births"] for s in a.stats()) > 0
    a.close()
    b.close()


@pytest.mark.parametrize("launch_mode", [0, 1])
def test_step_graph_forms_bit_identical(launch_mode):
    """eco_step(n) replays graphs of 8 steps and of one step, eco_step_timed
    a one-step graph with event-record nodes around the policy kernel, and
    eco_prepare builds them ahead: every array and statistic must match
    after 8k + r steps taken in each of these ways, and eco_policy_timing
    reports the timed launches' agents."""
    from paper_2510_18221_gb300 import eco
    envs = [workloads.scaled("mid", s, n, k, seed=50 + i, precision="bf16", e_init=185)
            for i, (s, n, k) in enumerate([(64, 600, 500), (128, 2048, 1500)])]
    many, ones, timed = (eco.Env(envs, launch_mode=launch_mode) for _ in range(3))
    for x in (many, ones, timed):
        x.reset()
    many.prepare()
    many.step(19)                 # 2 x 8 steps + 3 x 1
    per_step = []                 # agents processed by each step
    for _ in range(19):
        ones.step(1)
        per_step.append(sum(st["agent_steps"] for st in ones.stats("last")))
    timed.step_timed(19)          # 2 x 8 steps, the first of each timed, + 3 x 1
    ms, n_timed, agents = timed.policy_timing()
    # the timed launches are the policy kernels of steps 0 and 8
    assert n_timed == 2 and ms > 0 and agents == per_step[0] + per_step[8]
    for e in range(len(envs)):
        sm, so, st = many.read_state(e), ones.read_state(e), timed.read_state(e)
        for k in harness.STATE_KEYS:
            assert np.array_equal(sm[k], so[k]) and np.array_equal(sm[k], st[k]), (e, k)
        assert many.stats()[e] == ones.stats()[e] == timed.stats()[e]
        assert np.array_equal(many.read_params(e), ones.read_params(e))
        assert np.array_equal(many.read_params(e), timed.read_params(e))
    assert many.stats()[0]["step"] == 19 and sum(s["births"] for s in many.stats()) > 0
    # fewer steps than a graph: every step timed, in one-step graphs
    timed.reset()
    timed.step_timed(3)
    ms, n_timed, agents = timed.policy_timing()
    assert n_timed == 3 and ms > 0 and agents == sum(per_step[:3])
    for x in (many, ones, timed):
        x.close()


def test_step_read_pipelined_records():
    """eco_step_read returns, at each call, the records of the step that the
    previous call enqueued (at the first call after reset, the records as
    they stand), with the state equal to eco_step's throughout."""
    from paper_2510_18221_gb300 import eco
    w = [workloads.scaled("mid", 64, 600, 500, precision="bf16", e_init=185),
         workloads.scaled("mid", 32, 300, 250, seed=7, precision="bf16", e_init=185)]
    a, b = eco.Env(w), eco.Env(w)
    for x in (a, b):
        x.reset()
    want = [eco.eco_read_stats(b.h, 2)]
    for _ in range(12):
        b.step(1)
        want.append(eco.eco_read_stats(b.h, 2))
    for k in range(12):
        tot, last = eco.eco_step_read(a.h, 2)
        assert np.array_equal(tot, want[k][0]) and np.array_equal(last, want[k][1]), k
    tot, last = eco.eco_read_stats(a.h, 2)
    assert np.array_equal(tot, want[12][0]) and np.array_equal(last, want[12][1])
    for e in range(2):
        sa, sb = a.read_state(e), b.read_state(e)
        for k in harness.STATE_KEYS:
            assert np.array_equal(sa[k], sb[k]), (e, k)
    a.reset()   # the pipeline starts over
    tot, _ = eco.eco_step_read(a.h, 2)
    assert np.array_equal(tot, want[0][0])
    a.close()
    b.close()


def test_api_argument_errors():
    """Bad arguments come back as ECO_EINVAL with a message, and the handle
    stays usable."""
    from paper_2510_18221_gb300 import eco
    w = workloads.get("small")
    env = eco.Env(w)
    env.reset()
    for call in (lambda: eco.eco_step(env.h, -1),
                 lambda: eco.eco_read_stats(env.h, 2),
                 lambda: eco.eco_step_read(env.h, 2)):
        with pytest.raises(eco.EcoError) as ex:
            call()
        assert ex.value.code == eco.ECO_EINVAL and str(ex.value)
    view = eco.eco_state_view()
    assert eco.lib().eco_read_state(env.h, 1, ctypes.byref(view)) == eco.ECO_EINVAL   # no env 1
    env.step(2)
    assert env.stats()[0]["step"] == 2
    env.close()


def test_per_phase_launch_form_lockstep():
    w = workloads.scaled("mid", 128, 2048, 1500, precision="fp8", e_init=190)
    rep = _run(w, 15, launch_mode=1)
    assert rep["births"] > 10


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_paper_form_policy_lockstep(prec):
    """Sec. 3.3's policy: per-sensor input linears summed, two ReLU hidden
    layers, unbiased head, evolvable temperature."""
    w = workloads.scaled("mid", 128, 2048, 1500, precision=prec, e_init=190,
                         policy_form="paper", n_hidden=2)
    rep = _run(w, 20)
    assert rep["births"] > 10


@pytest.mark.parametrize("L,base", [(1, "small"), (3, "mid"), (2, "large")])
def test_paper_form_shapes(L, base):
    side, slots, k = (64, 256, 200) if base == "small" else (64, 600, 500)
    w = workloads.scaled(base, side, slots, k, policy_form="paper", n_hidden=L, e_init=190,
                         precision="bf16" if base != "large" else "fp8")
    _run(w, 8)


def test_paper_form_quantised_copy_bit_exact():
    from paper_2510_18221_gb300 import eco
    from tests import inputs
    w = workloads.scaled("mid", 32, 8, 4, precision="fp8", policy_form="paper", n_hidden=3)
    env = eco.Env(w)
    orc = oracle.Oracle(w)
    rows = inputs.random_params(orc.P, n_rows=8, seed=8)
    env.write_params(0, 0, rows)
    assert np.array_equal(env.read_params(0, 0, 8), rows)
    codes, scales = env.read_streamed(0, 0, 8)
    D, H, A = orc.D, 64, 9
    starts = [(0, D)] + [(H * D + 3 * H + l * (H * H + H), H) for l in range(3)]
    head = H * D + 3 * H + 3 * (H * H + H)
    for s in range(8):
        m = rows[s]
        r = 0
        for st, n in starts:
            for o in range(H):
                row = m[st + o * n:st + (o + 1) * n]
                sc = oracle.fp8_row_scale(row)
                assert scales[s, r] == np.float32(sc)
                want = [oracle.e4m3_encode(float(np.float32(v) / np.float32(sc))) for v in row]
                assert np.array_equal(codes[s, st + o * n:st + (o + 1) * n], np.array(want, np.uint8))
                r += 1
        for a in range(A):
            row = m[head + a * H:head + (a + 1) * H]
            assert scales[s, r] == np.float32(oracle.fp8_row_scale(row))
            r += 1
    env.close()


def _ecology(side, slots, k, **kw):
    """The paper's rule set (HP, 3x3 attack, eat / reproduce actions, drops)
    with the paper's policy form, on a reduced world; founders start with
    little energy and a low reproduction threshold so that births,
    starvation, kills, drops and healing all happen within a short run."""
    over = dict(e_init=60, e_repro=50, e_child=20)
    over.update(kw)
    return workloads.scaled("ecology", side, slots, k, **over)


def _run_totals(w, steps, **kw):
    env, orc = _pair(w, **kw)
    try:
        harness.start_pair(env, orc)
        rep = harness.lockstep(env, orc, steps, where=w["name"])
        return rep, env.stats()[0]
    finally:
        env.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_paper_rules_lockstep(prec):
    """Sec. 3.2 "Resources and Agent Health" / "Actions", App. F.7-F.8."""
    rep, tot = _run_totals(_ecology(128, 2048, 1500, precision=prec), 30)
    assert rep["births"] > 50
    for k in ("deaths", "food_refilled", "heals", "starved", "eaten", "food_emptied", "damage"):
        assert tot[k] > 0, k


@pytest.mark.parametrize("over", [
    dict(policy_form="plain", n_hidden=1, n_scalars=4, patch_k=5, hidden=32),
    dict(flags=("rotate_obs", "cancel_all"), attack_damage=10, age_div=5),
    dict(flags=(), heal_rate=0, e_cap=70),
    dict(slots=1200, e_repro=40, e_child=10),      # slot exhaustion: failed births
])
def test_paper_rules_variants(over):
    over = dict(over)
    slots = over.pop("slots", 600)
    rep, tot = _run_totals(_ecology(64, slots, 500, **over), 15)
    assert rep["steps"] == 15 and tot["deaths"] > 0


def test_paper_rules_launch_forms_bit_identical():
    from paper_2510_18221_gb300 import eco
    w = _ecology(128, 2048, 1500, precision="fp8")
    a, b = eco.Env(w, launch_mode=0), eco.Env(w, launch_mode=1)
    a.reset()
    b.reset()
    for t in range(25):
        a.step(1)
        b.step(1)
        sa, sb = a.read_state(0), b.read_state(0)
        for k in harness.STATE_KEYS:
            assert np.array_equal(sa[k], sb[k]), (t, k)
        assert a.stats()[0] == b.stats()[0]
    assert a.stats()[0]["births"] > 0
    a.close()
    b.close()


def test_paper_rules_state_roundtrip():
    """eco_write_state / eco_read_state carry HP, age and the energy on
    cells; the food bits follow the energy."""
    from paper_2510_18221_gb300 import eco
    w = _ecology(32, 64, 40)
    env = eco.Env(w)
    orc = oracle.Oracle(w)
    orc.reset()
    for _ in range(5):
        orc.step_once()
    rng = np.random.default_rng(5)
    orc.hp[orc.alive == 1] = rng.integers(1, 41, int(orc.alive.sum()))
    orc.age[:] = rng.integers(0, 5000, orc.S)
    orc.res[:] = np.where(orc.wall == 1, 0, rng.integers(0, 3, orc.res.size) * 7)
    orc.food[:] = (orc.res > 0).astype(np.uint8)
    env.reset()
    env.write_state(0, orc.arrays())
    gs = env.read_state(0)
    harness.compare_state(gs, orc, "roundtrip")
    harness.compare_colours(gs, orc, (), "roundtrip")
    st = env.stats()[0]
    assert st["res_total"] == int(orc.res.sum()) and st["food_total"] == int(orc.food.sum())
    env.close()


@pytest.mark.parametrize("vision,view", [("rgb", "around"), ("channels", "front"), ("rgb", "front")])
@pytest.mark.parametrize("rules", ["simple", "paper"])
def test_vision_variants_lockstep(vision, view, rules):
    """RGB vision with the colour trait (Sec. 3.2, 3.3) and the Front
    viewing configuration (App. F.6), under both rule sets."""
    if rules == "simple":
        w = workloads.scaled("mid", 64, 600, 500, precision="bf16", e_init=190, sigma=0.05,
                             vision=vision, view=view)
    else:
        w = _ecology(64, 600, 500, precision="bf16", vision=vision, view=view)
    rep = _run(w, 12)
    assert rep["births"] > 0


@pytest.mark.parametrize("k,hidden,view", [(3, 32, "around"), (3, 32, "front"), (7, 64, "front"),
                                           (9, 64, "around")])
def test_vision_ranges(k, hidden, view):
    """The paper's vision ranges 3x3, 7x7 and 9x9 (App. F.6), Around and
    Front, RGB, paper rules and policy form."""
    w = _ecology(64, 600, 500, patch_k=k, hidden=hidden, view=view, precision="fp8")
    rep = _run(w, 10)
    assert rep["steps"] == 10


def _terrain(side, slots, k, **kw):
    """The terrain rules (rock, flowing water, biomass, photosynthesis) with
    the paper form, on a reduced world; weak attacks, little water at birth
    and a low reproduction threshold so that births, thirst, drinking,
    eating biomass, photosynthesis and deaths all happen within a short run."""
    over = dict(e_repro=50, e_child=25, e_init=80, b_child=5, b_bite=10, w_init=12, w_child=5,
                attack_damage=10)
    over.update(kw)
    return workloads.scaled("terrain", side, slots, k, **over)


@pytest.mark.parametrize("preset,prec", [("beach", "bf16"), ("island", "fp8"), ("lake", "fp32"),
                                         ("isthmus", "bf16"), ("channel", "fp8"), ("ocean", "bf16")])
def test_terrain_lockstep(preset, prec):
    """Sec. 3.2 "Terrain", "Resources and Agent Health"; App. F.2."""
    rep, tot = _run_totals(_terrain(64, 1200, 800, terrain=preset, precision=prec), 25)
    assert rep["births"] > 5
    for k in ("deaths", "drunk", "bio_eaten", "photo", "thirsty", "heals", "dead_water", "dead_bio"):
        assert tot[k] > 0, k


@pytest.mark.parametrize("over", [
    dict(policy_form="plain", n_hidden=1, patch_k=5, hidden=32),
    dict(wall_density=0.08, flags=("rotate_obs", "cancel_all")),
    dict(view="front", heal_water=2, w_metab=2, photo_q16=6553),
])
def test_terrain_variants(over):
    rep, tot = _run_totals(_terrain(48, 900, 600, **over), 15)
    assert rep["steps"] == 15 and tot["deaths"] > 0


@pytest.mark.parametrize("side,preset,launch_mode", [(50, "beach", 0), (50, "beach", 1), (30, "lake", 0)])
def test_terrain_sides_two_mod_four(side, preset, launch_mode):
    """The flow and photosynthesis phases take cells in groups of four; on a
    side that is 2 mod 4 a group straddles two rows and the neighbours are
    found cell by cell.  Both launch forms, against the oracle."""
    slots, k = (700, 450) if side == 50 else (300, 200)
    rep, tot = _run_totals(_terrain(side, slots, k, terrain=preset), 15, launch_mode=launch_mode)
    assert rep["steps"] == 15 and tot["photo"] > 0 and tot["deaths"] > 0


def test_terrain_launch_forms_bit_identical():
    from paper_2510_18221_gb300 import eco
    w = _terrain(128, 4096, 3000, terrain="island", precision="fp8", wall_density=0.03)
    a, b = eco.Env(w, launch_mode=0), eco.Env(w, launch_mode=1)
    a.reset()
    b.reset()
    for t in range(25):
        a.step(1)
        b.step(1)
        sa, sb = a.read_state(0), b.read_state(0)
        for k in harness.STATE_KEYS:
            assert np.array_equal(sa[k], sb[k]), (t, k)
        assert a.stats()[0] == b.stats()[0]
    assert a.stats()[0]["births"] > 0
    a.close()
    b.close()


def test_terrain_rock_and_state_roundtrip():
    from paper_2510_18221_gb300 import eco
    w = _terrain(32, 64, 40, terrain="lake")
    env = eco.Env(w)
    assert np.array_equal(env.get_rock(0), w["rock"])
    orc = oracle.Oracle(w)
    orc.reset()
    for _ in range(4):
        orc.step_once()
    env.reset()
    env.write_state(0, orc.arrays())
    gs = env.read_state(0)
    harness.compare_state(gs, orc, "roundtrip")
    st = env.stats()[0]
    assert st["water_cells"] == int(orc.water.sum())
    assert st["water_agents"] == int(orc.a_water[orc.alive == 1].sum())
    assert st["bio_cells"] == int(orc.bio.sum())
    env.close()


@pytest.mark.parametrize("base", ["ecology", "terrain", "paperform"])
def test_input_sparse_variants_on_dense_inputs(base):
    """The input-sparse variants (7, 8) on worlds whose observations are
    mostly nonzero (RGB, elevation) and on the paper form's sensors."""
    w = workloads.scaled(base, 64, 600, 450, e_init=60, e_repro=50, e_child=20, precision="bf16")
    if base == "paperform":
        w = workloads.scaled(base, 64, 600, 450, e_init=190, precision="fp8")
    for v in (7, 8):
        _run(w, 5, policy_variant=v)


@pytest.mark.parametrize("base,over", [
    ("mid", dict(e_init=190, precision="bf16")),
    ("paperform", dict(e_init=190, precision="fp8")),
    ("paperform", dict(e_init=190, n_scalars=4, precision="bf16")),
    ("ecology", dict(e_init=60, e_repro=50, e_child=20, precision="bf16")),
    ("terrain", dict(e_init=80, e_repro=50, e_child=25, b_child=5, b_bite=10, w_init=12,
                     w_child=5, attack_damage=10, precision="bf16")),
])
def test_blind_agents(base, over):
    """Agents without a vision sensor (App. F.6 "Blind"; the paper's R / RC
    agents): the observation is the scalars alone, so D is below H."""
    w = workloads.scaled(base, 64, 600, 450, patch_k=0, **over)
    rep = _run(w, 12)
    assert rep["steps"] == 12
