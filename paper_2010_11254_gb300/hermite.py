"""Modified 4th-order Hermite step for sink particles (STARFORGE methods paper,
Sec. 2.3, the predictor and corrector equations) and the sink two-body
timestep (Sec. 2.3, Delta t_2-body).

The step takes two field + jerk evaluations: at the start of the step and
after the prediction.  ``force_jerk(x, v) -> (a, j)`` supplies them; with
this library that is a tree over the sinks alone (the paper's sinks-only
pass) evaluated by ``Tree.accel_jerk``.  The arithmetic is elementwise and
works on numpy arrays or torch tensors alike.
"""
from __future__ import annotations

import math


def modified_hermite_step(x0, v0, force_jerk, dt: float, aj0=None):
    """One step of length dt from (x0, v0).  Returns (x, v, a0, j0).

    Prediction with the field and jerk at the start,
      x_p = x0 + dt v0 + dt^2/2 a0 + dt^3/6 j0,   v_p = v0 + dt a0 + dt^2/2 j0,
    a second evaluation at (x_p, v_p), then the correction, velocity first
    (the position update uses the corrected velocity):
      v = v0 + dt/2 (a + a0) + dt^2/12 (j0 - j),
      x = x0 + dt/2 (v + v0) + dt^2/12 (a0 - a).
    aj0 may carry (a0, j0) when the caller already has them."""
    a0, j0 = force_jerk(x0, v0) if aj0 is None else aj0
    xp = x0 + dt * v0 + (dt * dt / 2.0) * a0 + (dt ** 3 / 6.0) * j0
    vp = v0 + dt * a0 + (dt * dt / 2.0) * j0
    a1, j1 = force_jerk(xp, vp)
    v1 = v0 + (dt / 2.0) * (a1 + a0) + (dt * dt / 12.0) * (j0 - j1)
    x1 = x0 + (dt / 2.0) * (v1 + v0) + (dt * dt / 12.0) * (a0 - a1)
    return x1, v1, a0, j0


def two_body_dt(x, v, m, h_sink: float, eta: float, G: float = 1.0) -> float:
    """Smallest two-body timestep over the sinks (Sec. 2.3):
    sqrt(eta) / (1 / t_c,min + 1 / t_dyn,min) per sink, with
    t_c = sqrt(r^2 + eps^2) / |v_ss'| and t_dyn = sqrt((r^2 + eps^2)^{3/2} / (G (m_s + m_s'))),
    eps = h_sink / 2.8 the Plummer-equivalent softening.  x, v, m are host
    sequences of the sinks (a direct O(N_s^2) loop: sinks are few)."""
    eps2 = (h_sink / 2.8) ** 2
    n = len(m)
    best = math.inf
    for s in range(n):
        tc, td = math.inf, math.inf
        for q in range(n):
            if q == s:
                continue
            d = [x[q][k] - x[s][k] for k in range(3)]
            w = [v[q][k] - v[s][k] for k in range(3)]
            r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2
            vw = math.sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2])
            if vw > 0.0:
                tc = min(tc, math.sqrt(r2) / vw)
            td = min(td, math.sqrt(r2 ** 1.5 / (G * (m[s] + m[q]))))
        best = min(best, math.sqrt(eta) / (1.0 / tc + 1.0 / td))
    return best
