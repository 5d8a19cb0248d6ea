"""The seeded input generator: Philox known answers, RAMBO kinematics, cuts."""
import math
import os

import numpy as np
import pytest

from paper_2312_07440_gb300 import events as ev

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = ev.philox4x32_10(([w[0]], [w[1]], [w[2]], [w[3]]), (w[4], w[5]))
        assert [int(x) for x in out[:, 0]] == w[6:10]


@pytest.mark.parametrize("name", list(ev.WORKLOADS))
def test_rambo_kinematics_and_cuts(name):
    wl = ev.WORKLOADS[name]
    mom, w = ev.generate(wl, 2000)
    N = ev.N_EXTERNAL[wl.process]
    assert mom.shape == (N, 4, 2000) and mom.dtype == np.float64 and mom.flags.c_contiguous
    # momentum conservation and mass shells
    assert np.abs(mom[0] + mom[1] - mom[2:].sum(axis=0)).max() < 1e-10 * mom[0, 0].max()
    m2 = mom[:, 0] ** 2 - mom[:, 1] ** 2 - mom[:, 2] ** 2 - mom[:, 3] ** 2
    for i, m in enumerate((0.0, 0.0) + wl.final_masses):
        assert np.allclose(m2[i], m * m, atol=1e-8 * mom[i, 0].max() ** 2)
    rs = mom[0, 0] + mom[1, 0]
    assert rs.min() >= wl.sqrt_s[0] - 1e-9 and rs.max() <= wl.sqrt_s[1] + 1e-9
    first = 2 if wl.process == "ee_5a" else 4  # cut particles: photons / outgoing gluons

    def eta(p):
        a = np.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
        return 0.5 * np.log((a + p[3]) / (a - p[3]))
    if wl.pt_min:
        for i in range(first, N):
            assert np.hypot(mom[i, 1], mom[i, 2]).min() > wl.pt_min
    if wl.eta_max:
        for i in range(first, N):
            assert np.abs(eta(mom[i])).max() < wl.eta_max
    if wl.dr_min:
        for i in range(first, N):
            for j in range(i + 1, N):
                pa, pb = mom[i], mom[j]
                dphi = np.angle(np.exp(1j * (np.arctan2(pa[2], pa[1]) - np.arctan2(pb[2], pb[1]))))
                assert np.sqrt((eta(pa) - eta(pb)) ** 2 + dphi ** 2).min() > wl.dr_min
    # lognormal weights: log w ~ N(0, 1)
    lw = np.log(w)
    assert abs(lw.mean()) < 0.1 and abs(lw.std() - 1) < 0.1


def test_counter_based_subranges_match():
    wl = ev.WORKLOADS["gg_ttgg_1m"]
    a, wa = ev.generate(wl, 300)
    b, wb = ev.generate(wl, 100, start=150)
    assert np.array_equal(a[:, :, 150:250], b[:, :, :100]) and np.array_equal(wa[150:250], wb[:100])


def test_boost_rotation_preserve_invariants():
    mom, _ = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 10)
    b = ev.rotate(ev.boost(mom, (0.1, 0.2, -0.3)), (1, 1, 0), 1.0)

    def inv(p, q):
        return p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3]
    for i in range(5):
        for j in range(5):
            assert np.allclose(inv(mom[i], mom[j]), inv(b[i], b[j]), rtol=1e-10, atol=1e-6)
    assert math.isclose(1.0, 1.0)
