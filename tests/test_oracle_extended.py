"""The oracle's extended-precision build, and how far the FP64 oracle is from it.

The GPU parity tests compare FP64 results per event at 1e-12 (relative).  On
a few ill-conditioned events (a top propagator close to its mass shell, where
p^2 - m^2 of order 1e3 GeV^2 is formed from terms of order 1e7 GeV^2) the FP64
oracle's own rounding error is a sizable part of that bound.  There the GPU
tests evaluate the event again with the same oracle source compiled with a
long double significand (64 bits on x86-64, 113 on AArch64) and compare with
that; everywhere else they use the FP64 oracle, which is sound where the FP64
oracle is within a quarter of the bound of the extended result.  The events of
the GPU tests' seeded FP64 samples where it is not are listed in
tests/golden/fp64_oracle_flags.json (written from the oracle alone); this file
checks that list and pins the extended build itself against a closed form at
exactly on-shell kinematics.
"""
import math
import os
import sys

import numpy as np

from paper_2312_07440_gb300 import events as ev

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
from parity_helpers import load_flags  # noqa: E402

TOL = 1e-12


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.where(a == b, 0.0, np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def per_event_error(a, b):
    e = rel(a["me0"], b["me0"])
    for k in ("me", "ratio", "wnew"):
        e = np.maximum(e, rel(a[k], b[k]).max(axis=0))
    return e


def on_shell_integer_event(m, E):
    """g g -> Q Qbar in the centre-of-mass frame with integer momenta that are
    exactly on shell and exactly conserve momentum: E^2 - (a^2 + b^2 + c^2)
    = m^2 for integers a >= b >= c > 0 (found by search)."""
    target = E * E - m * m
    for a in range(int(math.isqrt(target)), 0, -1):
        r = target - a * a
        for b in range(min(a, int(math.isqrt(r))), 0, -1):
            c2 = r - b * b
            c = math.isqrt(c2)
            if c > 0 and c * c == c2:
                p = np.zeros((4, 4))
                p[0] = [E, 0, 0, E]
                p[1] = [E, 0, 0, -E]
                p[2] = [E, a, b, c]
                p[3] = [E, -a, -b, -c]
                return p
    return None


def test_extended_build_matches_closed_form_on_shell(oracle_mod):
    """Averaged g g -> Q Qbar (Combridge; Ellis, Stirling & Webber) evaluated in
    long double: at kinematics that are exactly consistent in binary the
    extended oracle agrees to a few units of its own precision, far below what
    the FP64 build can reach."""
    eps = float(np.finfo(np.longdouble).eps)
    L = np.longdouble
    pi = L("3.141592653589793238462643383279502884197")
    worst = 0.0
    for E, m in ((301, 173), (450, 173), (777, 173), (1500, 0), (650, 0)):
        p = on_shell_integer_event(m, E)
        assert p is not None
        pl = p.astype(L)

        def dot(x, y):
            return x[0] * y[0] - x[1] * y[1] - x[2] * y[2] - x[3] * y[3]
        s = dot(pl[0] + pl[1], pl[0] + pl[1])
        t1, t2, rho = 2 * dot(pl[0], pl[2]) / s, 2 * dot(pl[1], pl[2]) / s, 4 * L(m) * L(m) / s
        g2 = 4 * pi * L(0.118)
        cf = g2 * g2 * (1 / (6 * t1 * t2) - L(3) / 8) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4 * t1 * t2))
        mom = np.ascontiguousarray(p[:, :, None])
        x = oracle_mod.me("gg_tt", ev.param_vector(m_t=float(m)), mom, precision="extended")[0]
        d = oracle_mod.me("gg_tt", ev.param_vector(m_t=float(m)), mom)[0]
        e_ext = abs(L(x) / cf - 1)
        worst = max(worst, float(e_ext))
        assert e_ext < 256 * eps + 4e-16  # the result is rounded to float64 once
        assert abs(d / float(cf) - 1) < 1e-13
    assert worst < 1e-15


def test_fp64_oracle_flags_are_current(oracle_mod):
    """The committed list of events (tests/golden/fp64_oracle_flags.json) on
    which the FP64 oracle is a quarter of the bound or more from the extended
    result is exactly what the oracle gives now; on every other event of the
    GPU tests' FP64 sets it is closer than that, which is what lets those
    tests use the FP64 oracle there."""
    import make_fp64_oracle_flags as mk
    flags, worst = mk.compute_flags()
    stored = load_flags()
    assert set(stored) == set(flags)
    for name in flags:
        assert list(stored[name]) == flags[name], name
    assert max(worst.values()) < 2 * TOL  # the FP64 oracle stays usable as a first filter


def test_fp64_oracle_error_on_an_ill_conditioned_event(oracle_mod):
    """The reason for the re-evaluation: on event 110 of the g g -> t tbar g g
    sample (m_t 173 -> 207.6 GeV) the FP64 oracle's own ratio is off by more
    than a fifth of the 1e-12 bound, while on typical events it is ~1e-14."""
    mom, w = ev.generate(ev.WORKLOADS["gg_ttgg_1m"], 111)
    pts = ev.reweight_points("gg_ttgg_1m", "mt")
    o = oracle_mod.reweight("gg_ttgg", ev.param_vector(), pts, mom, w)
    x = oracle_mod.reweight("gg_ttgg", ev.param_vector(), pts, mom, w, precision="extended")
    err = per_event_error(o, x)
    assert err[110] > 0.2 * TOL
    assert np.median(err) < 0.05 * TOL
