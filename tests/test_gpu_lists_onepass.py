"""Stored lists built in one pass (each group's lists staged per warp and
placed where the walk reserved space) and by the sizes-first path (a walk
for the sizes, then one that writes) give the fields of the oracle on the
same lists.  A run of calls whose list sizes jump (Theta 0.9, then 0.15
repeatedly) takes both paths: a sizing hint or a staging area that is
short sends a call down the sizes-first path, which raises them for the
next call."""
import numpy as np
import pytest

import gen
from _helpers import oracle_tree, rel_err, to_dev

pytestmark = pytest.mark.gpu


def test_one_pass_and_sizes_first_lists_agree_with_oracle():
    import torch
    import paper_2010_11254_gb300 as sfg
    c = gen.clumpy_cloud(30000, n_clumps=16, n_sink=16, seed=41)
    act = gen.active_subset(c.n, 0.3, seed=7)
    pos, mass, soft, sink = to_dev(c, torch)
    a_t = torch.from_numpy(act).cuda()
    o = oracle_tree(c, 16)
    ref = {}
    walks = []
    for theta in [0.9, 0.15, 0.15, 0.15, 0.15, 0.15, 0.9]:
        t = sfg.Tree(pos, mass, soft, sink, theta=theta, leaf_size=16, group_size=32)
        acc, phi = t.accel(a_t)
        assert t.status() == sfg.SFG_OK
        walks.append(t.stats()["list_walks"])
        t.close()
        if theta not in ref:
            o.walk(act, 32, theta)
            ref[theta] = o.accel_group(act)
        ao, po = ref[theta]
        e = rel_err(acc.cpu().numpy(), ao)
        assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 2e-4, (theta, walks)
        assert rel_err(phi.cpu().numpy(), po).max() <= 1e-6, (theta, walks)
    # the jump to Theta = 0.15 outgrew the hint, and the hint then caught up
    assert walks[1] == 2, walks
    assert 1 in walks[2:], walks
