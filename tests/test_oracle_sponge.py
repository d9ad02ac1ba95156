"""Pin of the oracle's absorbing layer by its physics, not by its formula (reading R8: a
layer of nbl cells with damping rate sigma = sigma0 (d/nbl)^2, sigma0 = 3 v_d ln(1000) /
(2 nbl h), in m (u_tt + sigma u_t) - Laplacian(u) = q, zero values beyond the grid).

A line of sources across the whole padded width launches a plane wave; the up-going half
crosses the top layer, reflects off the zero boundary beyond it and crosses the layer
again.  Along the way sigma u_t makes the amplitude decay like exp(-sigma t / 2), so in the
WKB (slowly varying) limit the round trip multiplies the amplitude by
    exp(-(1/2) * 2 * integral_0^L sigma(d) / v dd) = exp(-sigma0 L / (3 v))
                                                 = exp(-ln(1000) v_d / (2 v)),
with the sign flipped by the zero boundary.  The recorded reflection against the direct
pulse must follow this law: a wrong sigma0 factor, a linear instead of quadratic profile
or a damping term without the 1/2 would move the log-amplitude by at least 0.5.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_06914_gb300 import inputs as I


@pytest.mark.parametrize("damp_v", [1000.0, 2000.0])
def test_sponge_round_trip_attenuation_follows_wkb(damp_v):
    v, h, nbl, nx, nz = 2000.0, 10.0, 40, 500, 80
    dt, nt, f0 = 0.4 * h / v, 500, 15.0
    g = O.Grid(2, nx, 1, nz, nbl, nt, h, h, h, dt, damp_v)
    NX, NZ = nx + 2 * nbl, nz + 2 * nbl
    m = np.full((NZ, NX), 1.0 / v ** 2)
    # sources at every on-grid column at 400 m depth; receiver 200 m above, mid-width (the
    # disturbance from the side layers needs 1.25 s to reach it, beyond the 1 s recorded)
    src = np.array([[(i - nbl) * h, 0.0, 400.0] for i in range(NX - 1)])
    rec = np.array([[0.5 * (nx - 1) * h, 0.0, 200.0]])
    d = O.forward(g, m, src, I.ricker(nt, dt, f0), rec)["d"][:, 0]
    t = np.arange(nt) * dt
    direct = d[(t >= 0.1) & (t < 0.4)]          # arrives at ~0.2 s
    refl = d[(t >= 0.5) & (t < 0.95)]           # 1200 m more path: ~0.8 s
    kd, kr = np.argmax(np.abs(direct)), np.argmax(np.abs(refl))
    ln_ratio = math.log(abs(refl[kr]) / abs(direct[kd]))
    wkb = -math.log(1000.0) * damp_v / (2.0 * v)
    assert abs(ln_ratio - wkb) < 0.25, (ln_ratio, wkb)
    assert np.sign(refl[kr]) == -np.sign(direct[kd])   # reflected off the zero boundary
    # the reflection arrives when the extra 1200 m of path says it should
    assert abs(t[(t >= 0.5) & (t < 0.95)][kr] - t[(t >= 0.1) & (t < 0.4)][kd] - 1200.0 / v) < 0.02
