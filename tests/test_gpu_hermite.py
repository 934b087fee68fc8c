"""The library's modified Hermite step of sink particles (sfg_hermite_step,
Sec. 2.3: predictor, a second field + jerk evaluation, corrector; both
evaluations by the sinks-only tree pass on the GPU) against the oracle's
FP64 step on direct sums, and the e = 0.9 binary of Sec. 2.3 integrated
entirely by the library (step and two-body timestep): the relative energy
error per orbit stays below the paper's 1e-6 at eta = 0.01."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

G = 1.0


def _cluster(n=64, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x *= rng.random((n, 1)) ** (1 / 3)
    v = 0.3 * rng.standard_normal((n, 3))
    m = rng.lognormal(math.log(1e-2), 1.0, n)
    h = np.full(n, 0.02)
    return x, v, m, h


@pytest.mark.parametrize("seed", [3, 4])
def test_step_matches_oracle_step(oracle_lib, seed):
    import torch
    import paper_2010_11254_gb300 as sfg
    x, v, m, h = _cluster(seed=seed)
    dt = 1e-2
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # theta = 0 opens every node: the tree pass sums every pair, like the oracle's direct sums
    x1, v1 = sfg.hermite_step(t(x), t(v), t(m), t(h), dt, G=G, theta=0.0, leaf_size=8, group_size=16)
    xo, vo = oracle_lib.hermite_step(x, v, m, h, dt, G=G)
    x1, v1 = x1.cpu().numpy(), v1.cpu().numpy()
    # compare the parts the field drives: the velocity change and the position change beyond dt v0
    dv_g, dv_o = v1 - v, vo - v
    dx_g, dx_o = x1 - x - dt * v, xo - x - dt * v
    ev = np.linalg.norm(dv_g - dv_o, axis=1) / np.linalg.norm(dv_o, axis=1)
    ex = np.linalg.norm(dx_g - dx_o, axis=1) / np.linalg.norm(dx_o, axis=1)
    assert np.median(ev) <= 1e-5 and ev.max() <= 1e-3, (np.median(ev), ev.max())
    assert np.median(ex) <= 1e-5 and ex.max() <= 1e-3, (np.median(ex), ex.max())


def test_step_rejects_bad_arguments():
    import torch
    import paper_2010_11254_gb300 as sfg
    x = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    x[1, 0] = 1.0
    m = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sfg.SfgError) as e:
        sfg.hermite_step(x, x.clone(), m, m.clone(), float("nan"))
    assert e.value.code == sfg.SFG_EINVAL


def test_binary_energy_error_library_only():
    import torch
    import paper_2010_11254_gb300 as sfg
    M2 = np.array([0.6, 0.4])
    HS = 1e-6
    dev = torch.device("cuda:0")
    mass = torch.tensor(M2, dtype=torch.float64, device=dev)
    soft = torch.full((2,), HS, dtype=torch.float64, device=dev)
    sink = torch.ones(2, dtype=torch.uint8, device=dev)
    e, a_ax = 0.9, 1.0
    M = M2.sum()
    ra = a_ax * (1 + e)
    va = math.sqrt(G * M * (1 - e) / (a_ax * (1 + e)))
    x = torch.tensor([[-M2[1] / M * ra, 0, 0], [M2[0] / M * ra, 0, 0]], dtype=torch.float64, device=dev)
    v = torch.tensor([[0, -M2[1] / M * va, 0], [0, M2[0] / M * va, 0]], dtype=torch.float64, device=dev)
    period = 2 * math.pi * math.sqrt(a_ax ** 3 / (G * M))

    def energy(x, v):
        x, v = x.cpu().numpy(), v.cpu().numpy()
        return 0.5 * (M2 * (v * v).sum(1)).sum() - G * M2[0] * M2[1] / np.linalg.norm(x[1] - x[0])

    e0 = energy(x, v)
    t, orbits = 0.0, 2
    while t < orbits * period:
        tr = sfg.Tree(x, mass, soft, sink, G=G, theta=0.5, leaf_size=4, group_size=8)
        dt = float(tr.sink_timestep(v, 0.01).min().item())
        tr.check()
        tr.close()
        x, v = sfg.hermite_step(x, v, mass, soft, dt, G=G, theta=0.5, leaf_size=4, group_size=8)
        t += dt
    assert abs(energy(x, v) - e0) / abs(e0) / orbits < 1e-6
