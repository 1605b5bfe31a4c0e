"""Torque map with the recursive Newton-Euler algorithm over each agent's
kinematic tree (paper Eq. rnea) against the FP64 oracle's spatial RNEA, in
both solver forms; the tree's lifetime (cleared by a model upload) and its
argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import agents, device_inputs, oracle_view, torque_close  # noqa: E402


@pytest.fixture(scope="module")
def mpcgpu():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu as m
    m.load()
    return m


def _solve(s, ids, inp32):
    return s.solve_host(ids.astype(np.int32), inp32["x0"], inp32["qd_meas"], inp32["cmd"], inp32["phase"])


def _oracle(model, inp32):
    from oracle.solve import solve_batch
    m, i = oracle_view(model, inp32)
    return solve_batch(m, i)


@pytest.mark.parametrize("form", [1, 0], ids=["fused", "plain"])
def test_tree_torques_match_oracle(mpcgpu, form):
    from workload import make_trees
    ids = np.arange(24)
    model, _ = agents("uneven", ids)
    trees = make_trees("uneven", ids)
    tmodel = dict(model)
    tmodel.update(trees)
    s = mpcgpu.Solver(max_agents=24, max_horizon=20, form=form, stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, ids)
    s.set_trees(trees, ids)
    for replan in (0, 1):
        _, inp = agents("uneven", ids, replan=replan)
        inp32 = device_inputs(inp)
        r = _solve(s, ids, inp32)
        ref = _oracle(tmodel, inp32)
        assert (r["status"] == 0).all()
        err = np.abs(r["tau"] - ref["tau"])
        print(f"\n[tree torques, form {form}, replan {replan}] max |dtau| {err.max():.2e} N m, "
              f"|tau| up to {np.abs(ref['tau']).max():.1f}")
        ok = torque_close(r["tau"], ref["tau"])
        assert ok.all(), np.argwhere(~ok)
    s.close()


def test_model_upload_clears_the_tree(mpcgpu):
    from workload import make_trees
    ids = np.arange(8)
    model, inp = agents("small", ids)
    inp32 = device_inputs(inp)
    s = mpcgpu.Solver(max_agents=8, max_horizon=20, stream=torch.cuda.current_stream().cuda_stream, warm_start=0)
    s.set_models(model, ids)
    s.set_trees(make_trees("small", ids), ids)
    with_tree = _solve(s, ids, inp32)["tau"].copy()
    s.set_models(model, ids[:4], idx=ids[:4])    # agents 0-3 lose their trees
    r = _solve(s, ids, inp32)
    ref = _oracle(model, inp32)                  # diagonal joint model
    assert torque_close(r["tau"][:4], ref["tau"][:4]).all()
    np.testing.assert_array_equal(r["tau"][4:], with_tree[4:])
    assert np.abs(with_tree[:4] - r["tau"][:4]).max() > 1e-3
    s.close()


def test_tree_argument_checks(mpcgpu):
    from workload import make_trees
    ids = np.arange(2)
    model, _ = agents("small", ids)
    s = mpcgpu.Solver(max_agents=2, max_horizon=20, stream=torch.cuda.current_stream().cuda_stream)
    s.set_models(model, ids)
    bad = make_trees("small", ids)
    bad["tree_axis"][1, 3] *= 1.01                # not a unit vector
    with pytest.raises(mpcgpu.MpcError) as e:
        s.set_trees(bad, ids)
    assert e.value.status == mpcgpu.MPC_ERR_INVALID
    with pytest.raises(mpcgpu.MpcError):
        s.set_trees(make_trees("small", ids), np.array([0, 5]))   # id out of range
    s.close()
