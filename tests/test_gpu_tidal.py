"""GPU tidal tensor T = -grad grad Phi (Sec. 2.2, same pass and lists as g;
Sec. 2.2.1, same softened kernel) and tidal timestep (Sec. 2.3) against the
oracle on identical lists.

Tolerance: T is summed in FP32 per lane and per work item (thousands of
terms, each rounded once; the isotropic part is summed apart and subtracted
at the end, which can cancel one decimal digit), so the per-row Frobenius
error relative to |T| is held to a median of 2e-5 and a 99th percentile of
5e-4, twice the force tolerance.  The timestep is FP64 arithmetic on the same
T: 1e-13 relative."""
import numpy as np
import pytest

import gen
from _helpers import edge_clouds, oracle_tree, rel_err, to_dev

pytestmark = pytest.mark.gpu

T_MEDIAN = 2e-5
T_P99 = 5e-4


def _frob_err(T, To):
    def full(x):
        return np.concatenate([x[:, :3], np.sqrt(2.0) * x[:, 3:]], 1)
    return np.linalg.norm(full(T) - full(To), axis=1) / np.maximum(np.linalg.norm(full(To), axis=1), 1e-300)


def _run(c, active, theta, leaf_size=16, group_size=32, quad=True, G=1.0):
    import torch
    import paper_2010_11254_gb300 as sfg
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=leaf_size, group_size=group_size, quadrupole=quad,
                 G=G)
    act = torch.from_numpy(np.asarray(active, np.int64)).cuda()
    acc, phi, tid = t.accel_tidal(act)
    assert t.status() == sfg.SFG_OK
    acc2, phi2 = t.accel(act)
    t.close()
    o = oracle_tree(c, leaf_size)
    o.walk(active, group_size, theta)
    ao, po = o.accel_group(active, G=G, quadrupole=quad)
    To = o.tidal_group(active, G=G, quadrupole=quad)
    return (acc.cpu().numpy(), phi.cpu().numpy(), tid.cpu().numpy(), acc2.cpu().numpy(), phi2.cpu().numpy(),
            ao, po, To)


def _check(acc, phi, tid, acc2, phi2, ao, po, To):
    e = _frob_err(tid, To)
    assert np.median(e) <= T_MEDIAN, np.median(e)
    assert np.percentile(e, 99) <= T_P99, np.percentile(e, 99)
    # the field of the tidal call is the field of sfg_accel
    ea = rel_err(acc, ao)
    assert np.median(ea) <= 1e-5 and np.percentile(ea, 99) <= 2e-4
    assert rel_err(phi, po).max() <= 1e-6
    assert rel_err(acc, acc2).max() <= 1e-5
    assert rel_err(phi, phi2).max() <= 1e-6


@pytest.mark.parametrize("quad", [True, False])
def test_uniform_4096_theta07_all_active(quad):
    c = gen.uniform_cloud(4096)
    _check(*_run(c, np.arange(c.n), 0.7, quad=quad))


def test_clumpy_with_sinks_partial_active():
    c = gen.clumpy_cloud(30000, n_clumps=24, n_sink=32, seed=12)
    act = gen.active_subset(c.n, 0.2, seed=4)
    _check(*_run(c, act, 0.5))


@pytest.mark.parametrize("leaf_size,group_size", [(1, 1), (8, 13), (32, 32)])
def test_leaf_and_group_sizes(leaf_size, group_size):
    c = gen.uniform_cloud(5000, seed=21, n_sink=7)
    act = gen.active_subset(c.n, 0.5, seed=6)
    _check(*_run(c, act, 0.5, leaf_size=leaf_size, group_size=group_size))


@pytest.mark.parametrize("name", ["n2", "duplicates", "sinks_only", "massless"])
def test_edge_clouds(name):
    c = edge_clouds()[name]
    acc, phi, tid, acc2, phi2, ao, po, To = _run(c, np.arange(c.n), 0.5, leaf_size=8, group_size=16)
    scale = np.abs(To).max()
    np.testing.assert_allclose(tid, To, rtol=0, atol=5e-4 * scale)


def test_timestep_matches_oracle():
    import torch
    import oracle
    import paper_2010_11254_gb300 as sfg
    rng = np.random.default_rng(9)
    T = rng.normal(size=(1000, 6)) * 10.0 ** rng.uniform(-3, 3, size=(1000, 1))
    T[0] = 0.0
    dt = sfg.tidal_timestep(torch.from_numpy(T).cuda(), 0.02).cpu().numpy()
    do = oracle.tidal_dt(T, 0.02)
    assert np.isinf(dt[0]) and np.isinf(do[0])
    np.testing.assert_allclose(dt[1:], do[1:], rtol=1e-13)


def test_error_paths():
    """The stored-list passes refuse an all-FP64 tree; empty active sets are no-ops."""
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.uniform_cloud(500, seed=3)
    pos, mass, soft, sink = to_dev(c, torch)
    t64 = sfg.Tree(pos, mass, soft, sink, precision=1)
    with pytest.raises(sfg.SfgError) as e:
        t64.accel_tidal(None)
    assert e.value.code == sfg.SFG_EINVAL
    vel = torch.zeros((c.n, 3), dtype=torch.float64, device=pos.device)
    with pytest.raises(sfg.SfgError):
        t64.accel_jerk(vel)
    with pytest.raises(sfg.SfgError):
        t64.sink_timestep(vel, 0.01)
    t64.close()
    t = sfg.Tree(pos, mass, soft, sink)
    empty = torch.zeros(0, dtype=torch.int64, device=pos.device)
    a, p, T = t.accel_tidal(empty)
    assert a.shape == (0, 3) and T.shape == (0, 6)
    with pytest.raises(sfg.SfgError):
        t.sink_timestep(vel, -1.0)
    with pytest.raises(sfg.SfgError):
        t.set_relative(torch.ones(c.n, dtype=torch.float64, device=pos.device), -0.5)
    assert t.status() == sfg.SFG_OK
    t.close()
