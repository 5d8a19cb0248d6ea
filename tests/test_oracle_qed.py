"""Pins of the oracle's e- e+ -> n photons (the paper's benchmark process,
Table 1): textbook closed forms, helicity-amplitude closed forms, the Ward
identity, Lorentz and Bose symmetry, the soft-photon limit and the coupling
scaling.  None of them uses the oracle to check itself."""
import itertools
import math

import numpy as np
import pytest

from paper_2312_07440_gb300 import events as ev

PAR = ev.param_vector()
E2 = 4 * math.pi / PAR[4]  # e^2 with alpha = 1/alpha_em_inv


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def event(n, seed, rs=500.0):
    """AoS momenta [n+2][4]: e- along +z, e+ along -z, n massless photons."""
    u = ev._uniforms(seed, np.arange(1), 0, 4 * n)
    pf = ev.rambo_massless(u, np.full(1, rs))
    p = np.zeros((n + 2, 4))
    p[0] = [rs / 2, 0, 0, rs / 2]
    p[1] = [rs / 2, 0, 0, -rs / 2]
    p[2:] = pf[:, :, 0]
    return p


def test_two_photons_textbook(oracle_mod):
    """e+ e- -> gamma gamma, massless: 1/4 sum |M|^2 = 2 e^4 (u/t + t/u)
    (Peskin & Schroeder Eq. 5.105 at m -> 0), times 1/2! here."""
    for seed in range(6):
        p = event(2, seed)
        t = mdot(p[0] - p[2], p[0] - p[2])
        u = mdot(p[0] - p[3], p[0] - p[3])
        me2, _ = oracle_mod.ee_photons(2, PAR, p)
        assert abs(me2 / (E2 ** 2 * (u / t + t / u)) - 1) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_mhv_closed_form(oracle_mod, n):
    """Helicity amplitudes (all-outgoing helicities): configurations with the
    fermions at equal helicity, or fewer than two of either sign, vanish; MHV
    ones (two negative: a fermion x and photon j) and their parity conjugates
    obey |A|^2 = (2 e^2)^n s_xj^3 s_yj s_xy^(n-2) / prod_i (s_xi s_yi) -- the
    Parke-Taylor quark-line amplitude summed over the n! photon orders with
    the eikonal identity (U(1) decoupling).  The helicity sum equals the
    spin-summed |M|^2 of the linear basis."""
    for seed in (21, 22):
        p = event(n, seed)
        out = [-p[0], -p[1]] + [p[i] for i in range(2, n + 2)]

        def S(a, b):
            return abs(mdot(out[a] + out[b], out[a] + out[b]))
        total, checked, scale, zeros = 0.0, 0, 0.0, []
        me2 = None
        for hel in itertools.product([0, 1], repeat=n + 2):
            me2, A = oracle_mod.ee_photons(n, PAR, p, 1, hel)
            total += abs(A) ** 2
            scale = max(scale, abs(A))
            lam = [(1 if hel[i] == 0 else -1) * (-1 if i < 2 else 1) for i in range(n + 2)]
            neg = [i for i in range(n + 2) if lam[i] < 0]
            pos = [i for i in range(n + 2) if lam[i] > 0]
            if lam[0] == lam[1] or len(neg) < 2 or len(pos) < 2:
                zeros.append(abs(A))
                continue
            if len(neg) == 2:
                j, x = [i for i in neg if i > 1][0], (0 if lam[0] < 0 else 1)
            elif len(pos) == 2:
                j, x = [i for i in pos if i > 1][0], (0 if lam[0] > 0 else 1)
            else:
                continue  # NMHV: no one-term formula
            y = 1 - x
            F = (2 * E2) ** n * S(x, j) ** 3 * S(y, j) * S(0, 1) ** (n - 2) / \
                np.prod([S(0, i) * S(1, i) for i in range(2, n + 2)])
            assert abs(abs(A) ** 2 / F - 1) < 1e-11
            checked += 1
        assert checked == (4 if n == 2 else 4 * n)  # n = 2: MHV and MHV-bar coincide
        assert max(zeros) < 1e-13 * scale
        assert abs(total / (4 * math.factorial(n)) / me2 - 1) < 1e-13


@pytest.mark.parametrize("n", [3, 5])
def test_ward_identity(oracle_mod, n):
    """Replacing one photon's polarisation by its momentum (the others
    physical) makes the amplitude vanish: only the sum over all n! attachment
    orders is gauge invariant, so a missing or mis-signed diagram fails."""
    rng = np.random.default_rng(n)
    for seed in (31, 32):
        p = event(n, seed)
        hel = [0, 1] + list(rng.integers(0, 2, n))
        eps = np.array([np.conj(oracle_mod.polvec(p[2 + i], 1, hel[2 + i])) for i in range(n)])
        _, A0 = oracle_mod.ee_photons(n, PAR, p, 1, hel, eps=eps)
        for j in range(n):
            e2 = eps.copy()
            e2[j] = p[2 + j] / p[2 + j][0]
            _, A = oracle_mod.ee_photons(n, PAR, p, 1, hel, eps=e2)
            assert abs(A) < 1e-12 * abs(A0)


def test_lorentz_and_bose_symmetry(oracle_mod):
    """The spin-summed |M|^2 of e- e+ -> 5 photons is unchanged by a boost and
    a rotation of the whole event, and by any relabelling of the photons."""
    wl = ev.WORKLOADS["ee_5a_1m"]
    mom, _ = ev.generate(wl, 24)
    me = oracle_mod.me("ee_5a", PAR, mom)
    moved = ev.rotate(ev.boost(mom, (0.3, -0.2, 0.5)), (1.0, 2.0, -0.5), 0.9)
    assert np.allclose(oracle_mod.me("ee_5a", PAR, moved), me, rtol=1e-12, atol=0)
    perm = [0, 1, 4, 6, 2, 5, 3]
    assert np.allclose(oracle_mod.me("ee_5a", PAR, np.ascontiguousarray(mom[perm])), me, rtol=1e-13, atol=0)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_soft_photon_limit(oracle_mod, n):
    """A soft photon k factorises the spin-summed squared amplitude:
    sum |A_n|^2 -> e^2 2 p0.p1 / ((p0.k)(p1.k)) sum |A_(n-1)|^2 (eikonal
    factor of the two massless beams, summed over the photon's polarisations);
    the deviation vanishes linearly in |k|.  The oracle's |M|^2 carries 1/n!
    for n identical photons, so |M_n|^2 n -> |M_(n-1)|^2 x eikonal.  With
    n = 2 fixed by the textbook cross section (test_two_photons_textbook),
    the chain n = 3, 4, 5 pins the identical-photon factor 1/5! of the
    e- e+ -> 5 photon workload."""
    rs = 500.0

    def deviation(seed, soft):
        rng = np.random.default_rng(seed)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        k = soft * rs * np.array([1.0, *d])
        # four hard photons recoiling against k: generated at rest with mass
        # M^2 = (P - k)^2, then boosted to momentum -k
        P = np.array([rs, 0.0, 0.0, 0.0]) - k
        hard = event(n - 1, seed, rs=math.sqrt(mdot(P, P)))[2:]
        hard = ev.boost(hard[:, :, None], tuple(P[1:] / P[0]))[:, :, 0]
        beams = event(n - 1, seed)[:2]
        pn = np.vstack([beams, hard, k])
        assert np.abs(pn[0] + pn[1] - pn[2:].sum(axis=0)).max() < 1e-9
        me_n, _ = oracle_mod.ee_photons(n, PAR, pn)
        me_m, _ = oracle_mod.ee_photons(n - 1, PAR, np.vstack([beams, hard]))
        eik = E2 * 2 * mdot(pn[0], pn[1]) / (mdot(pn[0], k) * mdot(pn[1], k))
        return me_n * n / (me_m * eik) - 1
    for seed in (41, 42, 43):
        d5, d6 = deviation(seed, 1e-5), deviation(seed, 1e-6)
        assert abs(d6) < 1e-4
        assert 8 < d5 / d6 < 12


def test_coupling_scaling(oracle_mod):
    """Only e enters: r = (alpha'/alpha)^5 for every event of a reweight."""
    wl = ev.WORKLOADS["ee_5a_1m"]
    mom, w = ev.generate(wl, 32)
    pts = ev.reweight_points("ee_5a_1m")
    o = oracle_mod.reweight("ee_5a", PAR, pts, mom, w)
    for j in range(pts.shape[0]):
        assert np.allclose(o["ratio"][j], (PAR[4] / pts[j, 4]) ** 5, rtol=1e-13, atol=0)
