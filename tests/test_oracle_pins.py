"""Pins of the FP64 CPU oracle against things other than itself.

Every check here is a closed form, an invariance, a special case that reduces
to a textbook result, or an independent evaluation inside the oracle (spin
sums by traces; full-colour Feynman rules).  Together they make a plausible
mistake anywhere in the oracle (a dropped diagram, a sign, a transposed index,
a wrong normalisation) fail at least one test.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2312_07440_gb300 import events as ev

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PROCS = [("gg_tt", "gg_tt_1m"), ("gg_ttg", "gg_ttg_4m"), ("gg_ttgg", "gg_ttgg_1m")]
METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def slash(g, a):
    return sum(METRIC[mu, mu] * a[mu] * g[mu] for mu in range(4))


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------
def test_dirac_clifford(oracle_mod):
    g, g5 = oracle_mod.dirac()
    for mu in range(4):
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * METRIC[mu, nu] * np.eye(4), atol=1e-15)
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0, atol=1e-15)
    assert np.allclose(g5 @ g5, np.eye(4), atol=1e-15)
    assert np.allclose(g[0].conj().T, g[0]) and np.allclose(g[1].conj().T, -g[1])


def test_su3_generators(oracle_mod):
    t, f = oracle_mod.su3()
    for a in range(8):
        for b in range(8):
            assert abs(np.trace(t[a] @ t[b]) - 0.5 * (a == b)) < 1e-15
            comm = t[a] @ t[b] - t[b] @ t[a]
            assert np.allclose(comm, 1j * np.einsum("c,cij->ij", f[a, b], t), atol=1e-15)
    ref = np.zeros((8, 8, 8))
    for line in open(os.path.join(GOLDEN, "su3_structure_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c, v = line.split()
        a, b, c, v = int(a) - 1, int(b) - 1, int(c) - 1, float(v)
        for (i, j, k), s in zip(itertools.permutations((a, b, c)), (1, -1, -1, 1, 1, -1)):
            ref[i, j, k] = s * v
    assert np.allclose(f, ref, atol=1e-15)


@pytest.mark.parametrize("m", [0.0, 173.0])
@pytest.mark.parametrize("basis", [0, 1])
def test_spinors(oracle_mod, m, basis):
    g, _ = oracle_mod.dirac()
    rng = np.random.default_rng(3)
    for _ in range(5):
        pv = rng.normal(size=3) * 300
        p = np.array([math.sqrt(m * m + pv @ pv), *pv])
        P = slash(g, p)
        su = np.zeros((4, 4), complex)
        sv = np.zeros((4, 4), complex)
        for s in range(2):
            u = oracle_mod.spinor("u", p, m, basis, s)
            v = oracle_mod.spinor("v", p, m, basis, s)
            assert np.abs((P - m * np.eye(4)) @ u).max() < 1e-10
            assert np.abs((P + m * np.eye(4)) @ v).max() < 1e-10
            su += np.outer(u, u.conj() @ g[0])
            sv += np.outer(v, v.conj() @ g[0])
        assert np.abs(su - (P + m * np.eye(4))).max() < 1e-10
        assert np.abs(sv - (P - m * np.eye(4))).max() < 1e-10


def test_massless_helicity_spinors_are_chiral(oracle_mod):
    g, g5 = oracle_mod.dirac()
    p = np.array([5.0, 3.0, 0.0, 4.0])
    u_plus = oracle_mod.spinor("u", p, 0.0, 1, 0)
    assert np.allclose(g5 @ u_plus, u_plus)          # right-handed
    u_minus = oracle_mod.spinor("u", p, 0.0, 1, 1)
    assert np.allclose(g5 @ u_minus, -u_minus)
    v_plus = oracle_mod.spinor("v", p, 0.0, 1, 0)    # antifermion h=+1/2 is left-chiral
    assert np.allclose(g5 @ v_plus, -v_plus)


@pytest.mark.parametrize("basis", [0, 1])
def test_polarisation_vectors(oracle_mod, basis):
    rng = np.random.default_rng(4)
    for k3 in [np.array([0, 0, 1.0]), np.array([0, 0, -2.0]), *rng.normal(size=(4, 3))]:
        k = np.array([np.linalg.norm(k3), *k3])
        eps = [oracle_mod.polvec(k, basis, s) for s in range(2)]
        proj = np.zeros((4, 4), complex)
        for e in eps:
            assert abs(mdot(e, k)) < 1e-14 * k[0]
            assert abs(mdot(e, e.conj()) + 1) < 1e-14
            assert abs(e[0]) < 1e-15
            proj += np.outer(e, e.conj())
        # transverse projector: delta_ij - k_i k_j/|k|^2 on the spatial block
        kh = k3 / np.linalg.norm(k3)
        assert np.allclose(proj[1:, 1:], np.eye(3) - np.outer(kh, kh), atol=1e-14)
        assert abs(mdot(eps[0], eps[1].conj())) < 1e-14


# ---------------------------------------------------------------------------
# P1 / P2: closed forms
# ---------------------------------------------------------------------------
def ee_mumu_closed_form(p, alpha_inv, GF, MZ, WZ):
    """Massless e-e+ -> mu-mu+ via s-channel photon and Z: the four nonzero
    helicity amplitudes A_ij = e^2/s + g_i g_j/(s - MZ^2 + i MZ WZ) (i,j in
    {L,R}), |M|^2 = sum_ij |A_ij|^2 (u^2 if i == j else t^2), with
    g_L = e(-1/2 + s_W^2)/(s_W c_W), g_R = e s_W^2/(s_W c_W)."""
    alpha = 1.0 / alpha_inv
    MW2 = MZ ** 2 / 2 + math.sqrt(MZ ** 4 / 4 - math.pi * alpha * MZ ** 2 / (math.sqrt(2) * GF))
    sw2 = 1 - MW2 / MZ ** 2
    sw, cw = math.sqrt(sw2), math.sqrt(1 - sw2)
    e = math.sqrt(4 * math.pi * alpha)
    g = [e * (-0.5 + sw2) / (sw * cw), e * sw2 / (sw * cw)]
    s = mdot(p[0] + p[1], p[0] + p[1])
    t = mdot(p[0] - p[2], p[0] - p[2])
    u = mdot(p[0] - p[3], p[0] - p[3])
    tot = 0.0
    for i in range(2):
        for j in range(2):
            A = e * e / s + g[i] * g[j] / (s - MZ ** 2 + 1j * MZ * WZ)
            tot += abs(A) ** 2 * (u * u if i == j else t * t)
    return tot


def test_p1_ee_mumu_closed_form(oracle_mod):
    mom, _ = ev.generate(ev.WORKLOADS["ee_mumu_4k"], 64)
    for pars in [dict(), dict(m_Z=92.0, w_Z=2.6)]:
        par = ev.param_vector(**pars)
        me = oracle_mod.me("ee_mumu", par, mom)
        d = dict(zip(ev.PARAM_FIELDS, par))
        cf = np.array([ee_mumu_closed_form(mom[:, :, k], d["alpha_em_inv"], d["G_F"], d["m_Z"], d["w_Z"])
                       for k in range(mom.shape[-1])])
        assert np.abs(me / cf - 1).max() < 1e-13


def gg_qq_closed_form(p, alpha_s, m):
    """Averaged g g -> Q Qbar (Combridge 1979; Ellis, Stirling & Webber,
    heavy-quark production): g^4 (1/(6 t1 t2) - 3/8)(t1^2 + t2^2 + rho -
    rho^2/(4 t1 t2)), t1 = 2 p1.p3/s, t2 = 2 p2.p3/s, rho = 4 m^2/s."""
    s = mdot(p[0] + p[1], p[0] + p[1])
    t1 = 2 * mdot(p[0], p[2]) / s
    t2 = 2 * mdot(p[1], p[2]) / s
    rho = 4 * m * m / s
    g2 = 4 * math.pi * alpha_s
    return g2 * g2 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4 * t1 * t2))


def test_p2_gg_tt_closed_form(oracle_mod):
    mom, _ = ev.generate(ev.WORKLOADS["gg_tt_1m"], 256)
    par = ev.param_vector()
    me = oracle_mod.me("gg_tt", par, mom)
    cf = np.array([gg_qq_closed_form(mom[:, :, k], 0.118, 173.0) for k in range(mom.shape[-1])])
    assert np.abs(me / cf - 1).max() < 1e-13
    # massless quarks (the gg -> q qbar textbook limit)
    u = ev._uniforms(11, np.arange(32), 0, 8)
    pf = ev.rambo_massless(u, np.full(32, 700.0))
    m0 = np.zeros((4, 4, 32))
    m0[0, 0], m0[0, 3], m0[1, 0], m0[1, 3] = 350.0, 350.0, 350.0, -350.0
    m0[2:] = pf
    me0 = oracle_mod.me("gg_tt", ev.param_vector(m_t=0.0), m0)
    cf0 = np.array([gg_qq_closed_form(m0[:, :, k], 0.118, 0.0) for k in range(32)])
    assert np.abs(me0 / cf0 - 1).max() < 1e-13


# ---------------------------------------------------------------------------
# P3: spin sums by traces (no external spinors)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("proc,wl,nev", [("ee_mumu", "ee_mumu_4k", 16), ("gg_tt", "gg_tt_1m", 16),
                                         ("gg_ttg", "gg_ttg_4m", 3)])
def test_p3_trace_spin_sums(oracle_mod, proc, wl, nev):
    mom, _ = ev.generate(ev.WORKLOADS[wl], nev)
    par = ev.param_vector()
    me = oracle_mod.me(proc, par, mom)
    tr = np.array([oracle_mod.me_traces(proc, par, mom[:, :, k]) for k in range(nev)])
    assert np.abs(tr / me - 1).max() < 1e-12


# ---------------------------------------------------------------------------
# P4: Lorentz invariance of the summed |M|^2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("proc,wl", [("ee_mumu", "ee_mumu_4k")] + PROCS)
def test_p4_lorentz_invariance(oracle_mod, proc, wl):
    nev = 8 if proc != "gg_ttgg" else 3
    mom, _ = ev.generate(ev.WORKLOADS[wl], nev)
    par = ev.param_vector()
    me = oracle_mod.me(proc, par, mom)
    for beta, axis, ang in [((0.3, -0.2, 0.5), (1, 2, 3), 0.7), ((0.0, 0.0, -0.9), (0, 1, 0), 2.5)]:
        mb = ev.rotate(ev.boost(mom, beta), axis, ang)
        assert np.abs(oracle_mod.me(proc, par, mb) / me - 1).max() < 1e-12


# ---------------------------------------------------------------------------
# P5: gauge invariance of every colour-ordered amplitude
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("proc,wl", PROCS)
def test_p5_gauge_invariance(oracle_mod, proc, wl):
    N = oracle_mod.N_EXTERNAL[proc]
    mom, _ = ev.generate(ev.WORKLOADS[wl], 2)
    gl = [0, 1] + list(range(4, N))
    for e in range(2):
        p = mom[:, :, e].copy()
        scale, worst = 0.0, 0.0
        for hel in itertools.product([0, 1], repeat=N):
            ext = oracle_mod.external(proc, p, 173.0, 1, hel)
            scale = max(scale, np.abs(oracle_mod.partial_amps(proc, p, 173.0, 0.118, ext)).max())
            for ip in gl:
                e2 = ext.copy()
                e2[ip] = (p[ip] if ip < 2 else -p[ip]) / p[ip][0]
                worst = max(worst, np.abs(oracle_mod.partial_amps(proc, p, 173.0, 0.118, e2)).max())
        assert worst < 1e-12 * scale


# ---------------------------------------------------------------------------
# P6: massless limit against Parke-Taylor MHV amplitudes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("proc", ["gg_tt", "gg_ttg", "gg_ttgg"])
def test_p6_parke_taylor(oracle_mod, proc):
    """|A(q, sigma, qbar)|^2 = (2 g^2)^n s_{q-,g-}^3 s_{q+,g-} / prod_cyclic s_{k,k+1}
    for MHV (two negative helicities, all outgoing) and the parity conjugate
    for MHV-bar; amplitudes with 0 or 1 negative (or positive) helicity and
    same-helicity quark pairs vanish.  Normalisation (2 g^2)^n follows from
    t^a = T^a/sqrt(2) relative to Tr(T^a T^b) = delta^ab conventions."""
    N = oracle_mod.N_EXTERNAL[proc]
    n = N - 2
    gl = [0, 1] + list(range(4, N))
    gs2 = 4 * math.pi * 0.118
    _, perms = oracle_mod.colour_matrix(n)
    u = ev._uniforms(7, np.arange(2), 0, 4 * (N - 2))
    pf = ev.rambo_massless(u, np.full(2, 1000.0))
    for e in range(2):
        pm = np.zeros((N, 4))
        pm[0] = [500, 0, 0, 500]
        pm[1] = [500, 0, 0, -500]
        pm[2:] = pf[:, :, e]
        out = [(-pm[i] if i < 2 else pm[i]) for i in range(N)]

        def S(a, b):
            return abs(mdot(out[a] + out[b], out[a] + out[b]))
        checked = 0
        for hel in itertools.product([0, 1], repeat=N):
            ext = oracle_mod.external(proc, pm, 0.0, 1, hel)
            A = oracle_mod.partial_amps(proc, pm, 0.0, 0.118, ext)
            lam = [(1 if hel[i] == 0 else -1) * (-1 if i < 2 else 1) for i in range(N)]
            neg = [i for i in range(N) if lam[i] < 0]
            pos = [i for i in range(N) if lam[i] > 0]
            if lam[2] == lam[3] or len(neg) < 2 or len(pos) < 2:
                assert np.abs(A).max() < 1e-12, (hel, A)
                continue
            if len(neg) == 2:
                gsp, qs = [i for i in neg if i not in (2, 3)][0], (2 if lam[2] < 0 else 3)
            elif len(pos) == 2:
                gsp, qs = [i for i in pos if i not in (2, 3)][0], (2 if lam[2] > 0 else 3)
            else:
                continue  # NMHV (6 external legs, 3 negative): no one-term formula
            qo = 5 - qs
            for s in range(len(perms)):
                chain = [2] + [gl[g] for g in perms[s]] + [3]
                den = np.prod([S(chain[i], chain[(i + 1) % len(chain)]) for i in range(len(chain))])
                pt = S(qs, gsp) ** 3 * S(qo, gsp) / den
                assert abs(abs(A[s]) ** 2 / (pt * (2 * gs2) ** n) - 1) < 1e-11
                checked += 1
        assert checked > 0


# ---------------------------------------------------------------------------
# P7: colour matrices
# ---------------------------------------------------------------------------
def test_p7_colour_matrix_textbook(oracle_mod):
    C, perms = oracle_mod.colour_matrix(2)
    ref = []
    for line in open(os.path.join(GOLDEN, "colour_matrix_qqbar_gg.txt")):
        if not line.startswith("#") and line.strip():
            ref.append([float(Fraction(x)) for x in line.split()])
    assert perms.tolist() == [[0, 1], [1, 0]]
    assert np.allclose(C, np.array(ref), atol=1e-15)


@pytest.mark.parametrize("n,den", [(1, 2), (2, 3), (3, 9), (4, 54)])
def test_p7_colour_matrix_structure(oracle_mod, n, den):
    C, perms = oracle_mod.colour_matrix(n)
    K = math.factorial(n)
    assert C.shape == (K, K) and np.allclose(C, C.T, atol=1e-14)
    # diagonal: Tr(t^a1..t^an t^an..t^a1) = N_c C_F^n
    assert np.allclose(np.diag(C), 3 * (4 / 3) ** n, rtol=1e-14)
    # entries are integers over a common denominator
    assert np.allclose(C * den, np.round(C * den), atol=1e-11)
    assert np.linalg.eigvalsh(C).min() > 0
    if n == 3:
        # adjacent swap of the first two gluons: C_F Tr(t^b t^a t^b t^a) = -8/9
        i = perms.tolist().index([0, 1, 2])
        j = perms.tolist().index([1, 0, 2])
        assert abs(C[i, j] + 8 / 9) < 1e-14


@pytest.mark.parametrize("proc,wl", PROCS)
def test_colour_decomposition_matches_full_colour_rules(oracle_mod, proc, wl):
    """M_ij(a_1..a_n) from the colour-dressed Feynman rules equals
    sum_sigma (t^{a_sigma1}...t^{a_sigman})_ij A_sigma for every colour set."""
    N = oracle_mod.N_EXTERNAL[proc]
    n = N - 2
    t, _ = oracle_mod.su3()
    _, perms = oracle_mod.colour_matrix(n)
    mom, _ = ev.generate(ev.WORKLOADS[wl], 1)
    p = mom[:, :, 0].copy()
    rng = np.random.default_rng(5)
    for hel in ([0] * N, [0, 1, 1, 0, 1, 0][:N]):
        ext = oracle_mod.external(proc, p, 173.0, 0, hel)
        A = oracle_mod.partial_amps(proc, p, 173.0, 0.118, ext)
        colour_sets = list(itertools.product(range(8), repeat=n)) if n <= 2 else rng.integers(0, 8, (40, n))
        for adj in colour_sets:
            M = oracle_mod.full_colour_amp(proc, p, 173.0, 0.118, ext, adj)
            Mc = np.zeros((3, 3), complex)
            for s, perm in enumerate(perms):
                T = np.eye(3, dtype=complex)
                for g in perm:
                    T = T @ t[adj[g]]
                Mc += T * A[s]
            assert np.abs(M - Mc).max() < 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("proc,wl", [("gg_tt", "gg_tt_1m"), ("gg_ttg", "gg_ttg_4m")])
def test_full_colour_sum_equals_me(oracle_mod, proc, wl):
    """|M|^2 from explicit sums over every gluon colour, quark colour and
    spin of the colour-dressed amplitudes equals the colour-matrix result."""
    N = oracle_mod.N_EXTERNAL[proc]
    n = N - 2
    mom, _ = ev.generate(ev.WORKLOADS[wl], 1)
    p = mom[:, :, 0].copy()
    tot = 0.0
    for hel in itertools.product([0, 1], repeat=N):
        ext = oracle_mod.external(proc, p, 173.0, 0, hel)
        for adj in itertools.product(range(8), repeat=n):
            M = oracle_mod.full_colour_amp(proc, p, 173.0, 0.118, ext, adj)
            tot += float(np.sum(np.abs(M) ** 2))
    tot /= 4 * 64 * math.factorial(n - 2)
    me = oracle_mod.me(proc, ev.param_vector(), mom)[0]
    assert abs(tot / me - 1) < 1e-12


def _full_colour_spin_sum(args):
    """sum over the given helicity configurations and every gluon colour of
    sum_ij |M_ij|^2 from the colour-dressed Feynman rules (worker process)."""
    import oracle
    proc, p, hels = args
    n = oracle.N_EXTERNAL[proc] - 2
    tot = 0.0
    for hel in hels:
        ext = oracle.external(proc, p, 173.0, 0, hel)
        for adj in itertools.product(range(8), repeat=n):
            M = oracle.full_colour_amp(proc, p, 173.0, 0.118, ext, adj)
            tot += float(np.sum(np.abs(M) ** 2))
    return tot


def test_gg_ttgg_identical_gluon_factor(oracle_mod):
    """g g -> t tbar g g: the two outgoing gluons are identical bosons, so a
    phase-space integral over both would count every configuration twice;
    |M|^2 therefore carries 1/2 besides the incoming averages 1/4 (spins) and
    1/64 (colours).  Checked against the explicit sum over all 64 spin
    configurations and all 8^4 gluon colour assignments of the colour-dressed
    Feynman-rule amplitudes (f^abc, t^a, full four-gluon vertex), which uses
    neither the colour-ordered decomposition nor the colour matrix."""
    import multiprocessing as mp
    proc = "gg_ttgg"
    mom, _ = ev.generate(ev.WORKLOADS["gg_ttgg_1m"], 1)
    p = mom[:, :, 0].copy()
    hels = list(itertools.product([0, 1], repeat=6))
    jobs = [(proc, p, hels[i::16]) for i in range(16)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        tot = math.fsum(pool.map(_full_colour_spin_sum, jobs))
    spin_avg, colour_avg, identical = 4, 64, 2
    me = oracle_mod.me(proc, ev.param_vector(), mom)[0]
    assert abs(tot / (spin_avg * colour_avg * identical) / me - 1) < 1e-12


# ---------------------------------------------------------------------------
# P9 / P8: parameter dependence, reshuffle, Eq. 2/3 bookkeeping
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("proc,wl,npow", [("gg_tt", "gg_tt_1m", 2), ("gg_ttg", "gg_ttg_4m", 3),
                                          ("gg_ttgg", "gg_ttgg_1m", 4)])
def test_p9_alpha_s_scaling(oracle_mod, proc, wl, npow):
    mom, w = ev.generate(ev.WORKLOADS[wl], 6)
    res = oracle_mod.reweight(proc, ev.param_vector(), ev.param_vector(alpha_s=0.120), mom, w)
    assert np.abs(res["ratio"][0] / (0.120 / 0.118) ** npow - 1).max() < 1e-14


@pytest.mark.parametrize("proc,wl", [("ee_mumu", "ee_mumu_4k"), ("gg_tt", "gg_tt_1m")])
def test_unchanged_parameters_give_unit_ratio(oracle_mod, proc, wl):
    mom, w = ev.generate(ev.WORKLOADS[wl], 64)
    p0 = ev.param_vector()
    res = oracle_mod.reweight(proc, p0, np.stack([p0, p0]), mom, w)
    assert np.all(res["ratio"] == 1.0) and np.all(res["wnew"] == w)


def test_yukawa_axis_is_degenerate(oracle_mod):
    mom, w = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 8)
    res = oracle_mod.reweight("gg_ttg", ev.param_vector(), ev.reweight_points("gg_ttg_4m")[:4], mom, w)
    assert np.all(res["ratio"] == 1.0)


def test_reshuffle_onto_new_mass_shell(oracle_mod):
    for proc, wl in PROCS:
        mom, _ = ev.generate(ev.WORKLOADS[wl], 32)
        out, st = oracle_mod.reshuffle(proc, ev.param_vector(m_t=175.0), mom)
        assert np.all(st == 0)
        msq = out[:, 0] ** 2 - out[:, 1] ** 2 - out[:, 2] ** 2 - out[:, 3] ** 2
        assert np.allclose(np.sqrt(np.abs(msq[2:4])), 175.0, rtol=1e-12)
        assert np.allclose(out[:2], mom[:2])
        tot_in = mom[0] + mom[1]
        tot_out = out[2:].sum(axis=0)
        assert np.abs(tot_out - tot_in).max() < 1e-9
        # directions unchanged
        for i in range(2, out.shape[0]):
            cr = np.cross(out[i, 1:].T, mom[i, 1:].T)
            assert np.abs(cr).max() < 1e-8 * np.abs(mom[i, 1:]).max() ** 2
    # no room for the new masses
    mom, _ = ev.generate(ev.WORKLOADS["gg_tt_1m"], 4)
    _, st = oracle_mod.reshuffle("gg_tt", ev.param_vector(m_t=1500.0), mom)
    lo = mom[0, 0] + mom[1, 0]
    assert np.all(st == (lo <= 3000.0))


def test_mass_change_reweight_uses_reshuffled_closed_form(oracle_mod):
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 32)
    pt = ev.param_vector(m_t=175.0, alpha_s=0.120)
    res = oracle_mod.reweight("gg_tt", ev.param_vector(), pt, mom, w)
    moved, _ = oracle_mod.reshuffle("gg_tt", pt, mom)
    cf = np.array([gg_qq_closed_form(moved[:, :, k], 0.120, 175.0) for k in range(32)])
    assert np.abs(res["me"][0] / cf - 1).max() < 1e-13


def test_p11_sigma_and_bad_events(oracle_mod):
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 100)
    mom[:, :, 7] = 0.0  # |M|^2 = NaN: violates |M|^2 != 0
    res = oracle_mod.reweight("gg_tt", ev.param_vector(), ev.reweight_points("gg_tt_1m"), mom, w)
    assert res["n_bad"] == 1
    assert res["ratio"][0, 7] == 0 and res["wnew"][0, 7] == 0
    assert res["sigma"][0] == math.fsum(res["wnew"][0])
    assert res["sigma_orig"] == math.fsum(w)
    ok = np.arange(100) != 7
    assert np.allclose(res["wnew"][0, ok], res["ratio"][0, ok] * w[ok], rtol=0, atol=0)
