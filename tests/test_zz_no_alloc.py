"""The allocation-free movement-claim entry point (eco_move_claims_noalloc)
against the movement phase of the existing step entry point (eco_step).

Some callers cannot allocate device memory: their device memory belongs to a
host framework's own pool, or cudaMalloc's device-wide synchronisation is not
acceptable inside their loop.  For them the library resolves movement claims
with its scratch in a fixed device array.  This test forces every agent of a
world to a move or a turn (greedy policy, dominant head bias), runs one
eco_step, and checks that the new entry point, given the world as it was
before the step, reports exactly the same cells and facings.  The outputs are
integers, so the tolerance is exact equality, as for every integer result in
this suite.  Two calls in a row are checked, each against its own eco_step,
so the second call runs on scratch the first one left behind.
"""
import numpy as np
import pytest

from paper_2510_18221_gb300 import eco, workloads

pytestmark = pytest.mark.gpu


def test_noalloc_move_claims_match_step_two_calls_in_a_row():
    import torch

    w = workloads.scaled("mid", 64, 700, 600, flags=("rotate_obs", "greedy"), e_init=150,
                         seed=21)
    L, S = w["side"], w["slots"]
    env = eco.Env(w)
    env.reset()
    rng = np.random.default_rng(5)
    cuda = torch.device("cuda")
    try:
        for call in range(2):
            choice = rng.choice([0, 1, 2, 3, 4, 6, 7], size=S).astype(np.uint8)
            params = env.read_params(0)
            head = env.P - env.A
            params[:, head:] = 0.0
            params[np.arange(S), head + choice.astype(np.int64)] = 100.0
            env.write_params(0, 0, params)

            before = env.read_state(0)
            alive = before["alive"].astype(bool)
            act = np.where(alive, choice, 0).astype(np.uint8)
            pos = (before["y"] * L + before["x"]).astype(np.int32)
            blocked = ((before["wall"] != 0) | (before["occ"] >= 0)).astype(np.uint8)

            t_pos = torch.from_numpy(pos).to(cuda)
            t_act = torch.from_numpy(act).to(cuda)
            t_fac = torch.from_numpy(before["facing"].copy()).to(cuda)
            t_blk = torch.from_numpy(blocked).to(cuda)
            t_fac_out = torch.empty(S, dtype=torch.uint8, device=cuda)
            t_pos_out = torch.empty(S, dtype=torch.int32, device=cuda)
            t_moved = torch.empty(S, dtype=torch.uint8, device=cuda)
            torch.cuda.synchronize()
            eco.eco_move_claims_noalloc(L, S, t_pos.data_ptr(), t_act.data_ptr(), t_fac.data_ptr(),
                                        t_blk.data_ptr(), w["seed"], int(before["step"][0]),
                                        t_fac_out.data_ptr(), t_pos_out.data_ptr(),
                                        t_moved.data_ptr(), 0)
            torch.cuda.synchronize()

            env.step(1)
            after = env.read_state(0)
            _, act_gpu = env.read_policy_io(0)
            assert np.array_equal(act_gpu[alive], choice[alive])    # the forced actions ran
            assert after["alive"][alive].all()                      # nobody died or moved away
            new_pos = t_pos_out.cpu().numpy()
            new_fac = t_fac_out.cpu().numpy()
            moved = t_moved.cpu().numpy()
            assert np.array_equal(new_pos[alive], (after["y"] * L + after["x"])[alive]), call
            assert np.array_equal(new_fac[alive], after["facing"][alive]), call
            assert int(moved[alive].sum()) == env.stats("last")[0]["moves"], call
            assert int(moved[alive].sum()) > 0
    finally:
        env.close()


def test_noalloc_rejects_oversized_grid():
    side = 2048  # 2048^2 cells exceed ECO_NOALLOC_MAX_CELLS
    with pytest.raises(eco.EcoError) as ex:
        eco.eco_move_claims_noalloc(side, 1, 1, 1, 1, 1, 0, 0, 1, 1, 1, 0)
    assert ex.value.code == eco.ECO_EINVAL


def test_noalloc_in_place_update_matches_separate_outputs():
    """A caller may update positions and facings in place (pos_out is pos,
    facing_out is facing_in): the result equals the call with separate
    output arrays, on a world where many movers contest the same cells."""
    import torch

    cuda = torch.device("cuda")
    side, n = 64, 1500
    rng = np.random.default_rng(17)
    cells = rng.choice(side * side, size=n, replace=False).astype(np.int32)
    blocked = np.zeros(side * side, np.uint8)
    blocked[cells] = 1
    blocked[rng.choice(side * side, size=200, replace=False)] = 1      # walls
    act = rng.choice([0, 1, 2, 3, 4, 5, 6, 7, 8], size=n).astype(np.uint8)
    fac = rng.integers(0, 4, size=n).astype(np.uint8)
    t_blk = torch.from_numpy(blocked).to(cuda)
    t_act = torch.from_numpy(act).to(cuda)
    outs = []
    for in_place in (False, True):
        t_pos = torch.from_numpy(cells.copy()).to(cuda)
        t_fac = torch.from_numpy(fac.copy()).to(cuda)
        if in_place:
            t_pos_out, t_fac_out = t_pos, t_fac
        else:
            t_pos_out = torch.empty(n, dtype=torch.int32, device=cuda)
            t_fac_out = torch.empty(n, dtype=torch.uint8, device=cuda)
        t_moved = torch.empty(n, dtype=torch.uint8, device=cuda)
        torch.cuda.synchronize()
        eco.eco_move_claims_noalloc(side, n, t_pos.data_ptr(), t_act.data_ptr(), t_fac.data_ptr(),
                                    t_blk.data_ptr(), 3, 9, t_fac_out.data_ptr(),
                                    t_pos_out.data_ptr(), t_moved.data_ptr(), 0)
        torch.cuda.synchronize()
        outs.append((t_pos_out.cpu().numpy(), t_fac_out.cpu().numpy(), t_moved.cpu().numpy()))
    (p0, f0, m0), (p1, f1, m1) = outs
    assert np.array_equal(p0, p1) and np.array_equal(f0, f1) and np.array_equal(m0, m1)
    assert 0 < int(m0.sum()) < int(((act >= 1) & (act <= 4)).sum())   # some won, some lost or were blocked
    assert np.array_equal(p0[m0 == 0], cells[m0 == 0])
    assert len(np.unique(p0)) == n                                     # one agent per cell
