"""GPU sink two-body timestep (Sec. 2.3, minima over the tree lists with the
masses of accepted nodes combined) against the oracle on identical lists.
The terms are FP32 (a division and a square root each) and the output FP64:
relative error <= 1e-5 per row."""
import numpy as np
import pytest

from _helpers import oracle_tree
import gen

pytestmark = pytest.mark.gpu


def _sinks(n, seed):
    rng = np.random.default_rng(seed)
    return gen.Cloud(rng.normal(size=(n, 3)), rng.lognormal(np.log(1e-3), 1.0, n), np.full(n, 1e-3),
                     np.ones(n, np.uint8), seed, "sinks"), rng.normal(size=(n, 3)) * 0.2


@pytest.mark.parametrize("n,theta,leaf,group", [(300, 0.5, 4, 8), (2000, 0.7, 8, 32), (64, 0.0, 4, 4)])
def test_sink_timestep_matches_oracle(n, theta, leaf, group):
    import torch
    import paper_2010_11254_gb300 as sfg
    from _helpers import to_dev
    c, vel = _sinks(n, n)
    pos, mass, soft, sink = to_dev(c, torch)
    t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=leaf, group_size=group)
    act = np.arange(c.n)
    dt = t.sink_timestep(torch.from_numpy(vel).cuda(), 0.01, torch.from_numpy(act).cuda()).cpu().numpy()
    assert t.status() == sfg.SFG_OK
    t.close()
    o = oracle_tree(c, leaf)
    o.walk(act, group, theta)
    do = o.tstep_group(vel, 0.01, act)
    np.testing.assert_allclose(dt, do, rtol=1e-5)


def test_single_sink_has_no_limit():
    import torch
    import paper_2010_11254_gb300 as sfg
    dev = torch.device("cuda:0")
    t = sfg.Tree(torch.zeros((1, 3), dtype=torch.float64, device=dev), torch.ones(1, dtype=torch.float64, device=dev),
                 torch.full((1,), 1e-3, dtype=torch.float64, device=dev), torch.ones(1, dtype=torch.uint8, device=dev))
    dt = t.sink_timestep(torch.zeros((1, 3), dtype=torch.float64, device=dev), 0.01)
    t.close()
    assert torch.isinf(dt).all()
