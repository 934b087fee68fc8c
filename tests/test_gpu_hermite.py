"""The e = 0.9 binary of Sec. 2.3 integrated with the modified Hermite step,
its field and jerk from the library's sinks-only pass (a tree of the two
sinks, sfg_accel_jerk, FP32 pair arithmetic on group-centred offsets), and
the sink two-body timestep: the relative energy error per orbit stays below
the paper's 1e-6 at eta = 0.01."""
import math

import numpy as np
import pytest

from paper_2010_11254_gb300.hermite import modified_hermite_step, two_body_dt

pytestmark = pytest.mark.gpu

G = 1.0
M2 = np.array([0.6, 0.4])
HS = 1e-6


def test_binary_energy_error_sinks_only_pass():
    import torch
    import paper_2010_11254_gb300 as sfg
    dev = torch.device("cuda:0")
    mass = torch.tensor(M2, dtype=torch.float64, device=dev)
    soft = torch.full((2,), HS, dtype=torch.float64, device=dev)
    sink = torch.ones(2, dtype=torch.uint8, device=dev)

    def fj(x, v):
        t = sfg.Tree(torch.from_numpy(x).to(dev), mass, soft, sink, G=G, theta=0.5, leaf_size=4, group_size=8)
        a, _, j = t.accel_jerk(torch.from_numpy(v).to(dev))
        assert t.status() == sfg.SFG_OK
        t.close()
        return a.cpu().numpy(), j.cpu().numpy()

    e, a_ax = 0.9, 1.0
    M = M2.sum()
    ra = a_ax * (1 + e)
    va = math.sqrt(G * M * (1 - e) / (a_ax * (1 + e)))
    x = np.array([[-M2[1] / M * ra, 0, 0], [M2[0] / M * ra, 0, 0]])
    v = np.array([[0, -M2[1] / M * va, 0], [0, M2[0] / M * va, 0]])
    period = 2 * math.pi * math.sqrt(a_ax ** 3 / (G * M))

    def energy(x, v):
        return 0.5 * (M2 * (v * v).sum(1)).sum() - G * M2[0] * M2[1] / np.linalg.norm(x[1] - x[0])

    e0 = energy(x, v)
    t, orbits = 0.0, 2
    while t < orbits * period:
        dt = two_body_dt(x, v, M2, HS, 0.01, G)
        x, v, _, _ = modified_hermite_step(x, v, fj, dt)
        t += dt
    assert abs(energy(x, v) - e0) / abs(e0) / orbits < 1e-6
