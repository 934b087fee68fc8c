"""GPU jerk j = dg/dt (Sec. 2.2: same pass and lists as g, pairs with the
softened kernel, nodes by monopole) against the oracle on identical lists.

Tolerance: j is summed in FP32 per lane and per work item from FP32
velocities and positions; its terms cancel more than the field's (velocity
differences, the (d . w) projection), so the per-row error relative to |j|
is held to a median of 2e-5 and a 99th percentile of 5e-4, twice the force
tolerance; the field of the jerk call equals sfg_accel's."""
import numpy as np
import pytest

import gen
from _helpers import edge_clouds, oracle_tree, rel_err, to_dev

pytestmark = pytest.mark.gpu

J_MEDIAN = 2e-5
J_P99 = 5e-4


def _vel(n, seed):
    return np.random.default_rng(seed).normal(size=(n, 3)) * 0.5


def _run(c, vel, active, theta, leaf_size=16, group_size=32, quad=True):
    import torch
    import paper_2010_11254_gb300 as sfg
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=leaf_size, group_size=group_size, quadrupole=quad)
    act = torch.from_numpy(np.asarray(active, np.int64)).cuda()
    acc, phi, jerk = t.accel_jerk(torch.from_numpy(vel).cuda(), act)
    assert t.status() == sfg.SFG_OK
    acc2, phi2 = t.accel(act)
    t.close()
    o = oracle_tree(c, leaf_size)
    o.walk(active, group_size, theta)
    Jo = o.jerk_group(vel, active)
    return jerk.cpu().numpy(), Jo, acc.cpu().numpy(), acc2.cpu().numpy(), phi.cpu().numpy(), phi2.cpu().numpy()


def _check(J, Jo, acc, acc2, phi, phi2):
    e = rel_err(J, Jo)
    assert np.median(e) <= J_MEDIAN, np.median(e)
    assert np.percentile(e, 99) <= J_P99, np.percentile(e, 99)
    assert rel_err(acc, acc2).max() <= 1e-5
    assert rel_err(phi, phi2).max() <= 1e-6


@pytest.mark.parametrize("quad", [True, False])
def test_uniform_4096_all_active(quad):
    c = gen.uniform_cloud(4096)
    _check(*_run(c, _vel(c.n, 1), np.arange(c.n), 0.7, quad=quad))


def test_clumpy_with_sinks_partial_active():
    c = gen.clumpy_cloud(30000, n_clumps=24, n_sink=32, seed=15)
    _check(*_run(c, _vel(c.n, 2), gen.active_subset(c.n, 0.2, seed=4), 0.5))


@pytest.mark.parametrize("leaf_size,group_size", [(1, 1), (8, 13)])
def test_leaf_and_group_sizes(leaf_size, group_size):
    c = gen.uniform_cloud(5000, seed=22, n_sink=7)
    _check(*_run(c, _vel(c.n, 3), gen.active_subset(c.n, 0.5, seed=6), 0.5, leaf_size, group_size))


def test_sinks_only_pass():
    """The sinks-only tree pass of Sec. 2.3: a tree of the sinks alone."""
    rng = np.random.default_rng(5)
    m = 200
    c = gen.Cloud(rng.normal(size=(m, 3)), rng.lognormal(np.log(1e-4), 1.2, m), np.full(m, 1e-3),
                  np.ones(m, np.uint8), 0, "sinks")
    _check(*_run(c, _vel(m, 4), np.arange(m), 0.5, leaf_size=4, group_size=8))


@pytest.mark.parametrize("name", ["n2", "duplicates", "massless"])
def test_edge_clouds(name):
    c = edge_clouds()[name]
    J, Jo, *_ = _run(c, _vel(c.n, 5), np.arange(c.n), 0.5, leaf_size=8, group_size=16)
    np.testing.assert_allclose(J, Jo, rtol=0, atol=5e-4 * np.abs(Jo).max())
