"""Seeded synthetic event batches (momenta + weights) for the reweighting path.

This module only produces INPUTS: partonic phase-space points and synthetic
event weights.  It holds none of the reweighting arithmetic (no matrix
elements, no ratios, no cross sections); both the CUDA path and the FP64 CPU
oracle consume the arrays it returns.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), implemented here from
its published definition, so every event is a pure function of
(seed, event index, attempt) and any sub-range of a batch can be regenerated
on its own.

Kinematics follow RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40
(1986) 359): isotropic massless momenta boosted and scaled to the partonic
centre-of-mass energy, then rescaled onto the mass shell with a Newton solve
for the common 3-momentum scale.  Events live in the partonic centre-of-mass
frame with the two incoming partons along +z and -z.  The paper's event
weights (Sec. 2.1, Eq. 1) need parton densities and a phase-space integrator
that this library does not reproduce; the weights here are lognormal,
W = exp(z) with z ~ N(0, 1) drawn by Box-Muller.

Layout returned: momenta as float64 structure-of-arrays ``mom[N][4][E]``
(particle, Lorentz component (E, px, py, pz), event), weights ``w[E]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: uint32-valued array of shape (4, n); key: (k0, k1) python ints or
    uint32 arrays of shape (n,).  Returns a uint32 array of shape (4, n).
    """
    c = [np.asarray(ctr[i], dtype=np.uint64) & _MASK32 for i in range(4)]
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK32
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(_PHILOX_W1)) & _MASK32
        p0 = _PHILOX_M0 * c[0]
        p1 = _PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c).astype(np.uint32)


def _uniforms(seed, event, attempt, n_doubles, stream=0):
    """Open-interval (0,1) doubles with 53-bit resolution.

    Counter word 0/1 = event index (64 bit), word 2 = attempt, word 3 packs
    (stream << 16) | block; key = 64-bit seed.  Returns (n_doubles, n).
    """
    event = np.asarray(event, dtype=np.uint64)
    n = event.shape[0]
    nblk = (n_doubles + 1) // 2
    out = np.empty((2 * nblk, n), dtype=np.float64)
    lo = event & _MASK32
    hi = event >> np.uint64(32)
    att = np.broadcast_to(np.asarray(attempt, dtype=np.uint64), (n,))
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    for b in range(nblk):
        w3 = np.full(n, ((stream & 0xFFFF) << 16) | b, dtype=np.uint64)
        r = philox4x32_10((lo, hi, att, w3), key).astype(np.uint64)
        for j in range(2):
            a = r[2 * j] >> np.uint64(5)  # 27 bits
            bb = r[2 * j + 1] >> np.uint64(6)  # 26 bits
            u = (a.astype(np.float64) * 67108864.0 + bb.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
            out[2 * b + j] = u
    return out[:n_doubles]


# --------------------------------------------------------------------------
# RAMBO
# --------------------------------------------------------------------------
def rambo_massless(u, sqrt_s):
    """RAMBO for n massless momenta at total energy sqrt_s (array (n_ev,)).

    u: uniforms of shape (4*n, n_ev).  Returns p of shape (n, 4, n_ev) in the
    rest frame of the total momentum.
    """
    n = u.shape[0] // 4
    nev = u.shape[1]
    q = np.empty((n, 4, nev))
    for i in range(n):
        r1, r2, r3, r4 = u[4 * i: 4 * i + 4]
        c = 2.0 * r3 - 1.0
        s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
        f = 2.0 * math.pi * r4
        e = -np.log(r1 * r2)
        q[i, 0] = e
        q[i, 1] = e * s * np.cos(f)
        q[i, 2] = e * s * np.sin(f)
        q[i, 3] = e * c
    Q = q.sum(axis=0)
    M = np.sqrt(Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2)
    b = -Q[1:] / M
    x = sqrt_s / M
    gam = Q[0] / M
    a = 1.0 / (1.0 + gam)
    p = np.empty_like(q)
    for i in range(n):
        bq = b[0] * q[i, 1] + b[1] * q[i, 2] + b[2] * q[i, 3]
        p[i, 0] = x * (gam * q[i, 0] + bq)
        for k in range(3):
            p[i, 1 + k] = x * (q[i, 1 + k] + b[k] * q[i, 0] + a * bq * b[k])
    # The boost loses digits when the q_i are nearly collinear (large gamma):
    # restore sum p = (sqrt_s, 0) to rounding by removing the residual
    # 3-momentum, putting the energies back on the light cone and rescaling.
    p[:, 1:] -= p[:, 1:].sum(axis=0, keepdims=True) / n
    p[:, 0] = np.sqrt(p[:, 1] ** 2 + p[:, 2] ** 2 + p[:, 3] ** 2)
    p *= (sqrt_s / p[:, 0].sum(axis=0))[None, None]
    return p


def rambo_to_masses(p, masses, sqrt_s):
    """Put RAMBO massless momenta on their mass shells (common 3-momentum
    scale xi from sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt_s, Newton)."""
    m2 = np.asarray(masses, dtype=np.float64) ** 2
    if not np.any(m2 > 0):
        return p
    p3sq = p[:, 1] ** 2 + p[:, 2] ** 2 + p[:, 3] ** 2  # (n, nev)
    xi = np.sqrt(np.maximum(1e-12, 1.0 - (np.sum(np.sqrt(m2)) / sqrt_s) ** 2)) * np.ones_like(sqrt_s)
    live = np.ones(xi.shape, dtype=bool)  # per-event convergence: batch independent
    for _ in range(100):
        e = np.sqrt(m2[:, None] + xi[None] ** 2 * p3sq)
        f = e.sum(axis=0) - sqrt_s
        df = (xi[None] * p3sq / e).sum(axis=0)
        step = np.where(live, f / df, 0.0)
        xi = xi - step
        live &= np.abs(step) > 4e-16 * xi
        if not live.any():
            break
    out = np.empty_like(p)
    out[:, 1:] = xi[None, None] * p[:, 1:]
    out[:, 0] = np.sqrt(m2[:, None] + xi[None] ** 2 * p3sq)
    return out


# --------------------------------------------------------------------------
# processes and workloads
# --------------------------------------------------------------------------
M_TOP = 173.0


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic event sample: process, sizes, kinematic ranges and cuts."""
    name: str
    process: str          # 'ee_mumu' | 'gg_tt' | 'gg_ttg' | 'gg_ttgg' | 'ee_5a'
    n_events: int
    sqrt_s: tuple         # (lo, hi); lo == hi for a fixed energy
    final_masses: tuple   # masses of the outgoing particles, in order
    pt_min: float = 0.0   # applied to the outgoing gluons / photons
    dr_min: float = 0.0   # applied to outgoing gluon / photon pairs
    seed: int = 231207440
    eta_max: float = 0.0  # |pseudorapidity| bound on the same particles (0: none)


N_EXTERNAL = {"ee_mumu": 4, "gg_tt": 4, "gg_ttg": 5, "gg_ttgg": 6, "ee_5a": 7}
# index of the first outgoing particle the cuts apply to (gluons follow t,
# tbar; the five photons of e- e+ -> 5 photons are particles 2..6)
_FIRST_FINAL_GLUON = {"ee_mumu": None, "gg_tt": None, "gg_ttg": 4, "gg_ttgg": 4, "ee_5a": 2}

# The five sample definitions (events, energies, cuts) the library is
# benchmarked and tested on; seeds are 231207440 + index.
WORKLOADS = {
    "ee_mumu_4k": Workload("ee_mumu_4k", "ee_mumu", 4096, (200.0, 200.0), (0.0, 0.0), seed=231207440 + 0),
    "gg_tt_1m": Workload("gg_tt_1m", "gg_tt", 1 << 20, (400.0, 2000.0), (M_TOP, M_TOP), seed=231207440 + 1),
    "gg_ttg_4m": Workload("gg_ttg_4m", "gg_ttg", 1 << 22, (500.0, 3000.0), (M_TOP, M_TOP, 0.0), pt_min=20.0,
                          seed=231207440 + 2),
    "gg_ttgg_1m": Workload("gg_ttgg_1m", "gg_ttgg", 1 << 20, (600.0, 4000.0), (M_TOP, M_TOP, 0.0, 0.0),
                           pt_min=20.0, dr_min=0.4, seed=231207440 + 3),
    # the paper's own benchmark process (Table 1), e- e+ -> 5 photons; photon
    # cuts p_T > 10 GeV, |eta| < 2.5, Delta R > 0.4 (the usual generator-level
    # photon cuts), sqrt(s) = 500 GeV
    "ee_5a_1m": Workload("ee_5a_1m", "ee_5a", 1 << 20, (500.0, 500.0), (0.0,) * 5, pt_min=10.0, dr_min=0.4,
                         seed=231207440 + 5, eta_max=2.5),
}


def _cuts_pass(p, wl):
    first = _FIRST_FINAL_GLUON[wl.process]
    ok = np.ones(p.shape[-1], dtype=bool)
    if first is None:
        return ok
    gl = list(range(first, p.shape[0]))
    pt = {i: np.hypot(p[i, 1], p[i, 2]) for i in gl}
    if wl.pt_min > 0:
        for i in gl:
            ok &= pt[i] > wl.pt_min
    if wl.eta_max > 0:
        for i in gl:
            pa = np.sqrt(p[i, 1] ** 2 + p[i, 2] ** 2 + p[i, 3] ** 2)
            with np.errstate(divide="ignore", invalid="ignore"):
                ok &= np.abs(0.5 * np.log((pa + p[i, 3]) / (pa - p[i, 3]))) < wl.eta_max
    if wl.dr_min > 0 and len(gl) > 1:
        for a in range(len(gl)):
            for b in range(a + 1, len(gl)):
                i, j = gl[a], gl[b]
                pa = np.sqrt(p[i, 1] ** 2 + p[i, 2] ** 2 + p[i, 3] ** 2)
                pb = np.sqrt(p[j, 1] ** 2 + p[j, 2] ** 2 + p[j, 3] ** 2)
                with np.errstate(divide="ignore", invalid="ignore"):
                    eta_a = 0.5 * np.log((pa + p[i, 3]) / (pa - p[i, 3]))
                    eta_b = 0.5 * np.log((pb + p[j, 3]) / (pb - p[j, 3]))
                dphi = np.arctan2(p[i, 2], p[i, 1]) - np.arctan2(p[j, 2], p[j, 1])
                dphi = (dphi + math.pi) % (2 * math.pi) - math.pi
                ok &= np.sqrt((eta_a - eta_b) ** 2 + dphi ** 2) > wl.dr_min
    return ok & np.all(np.isfinite(p), axis=(0, 1))


def _draw(wl, events, attempt):
    nfin = N_EXTERNAL[wl.process] - 2
    u = _uniforms(wl.seed, events, attempt, 1 + 4 * nfin, stream=0)
    lo, hi = wl.sqrt_s
    rs = lo + (hi - lo) * u[0]
    pf = rambo_to_masses(rambo_massless(u[1:], rs), wl.final_masses, rs)
    p = np.empty((nfin + 2, 4, len(events)))
    half = 0.5 * rs
    p[0, 0], p[0, 1], p[0, 2], p[0, 3] = half, 0.0, 0.0, half
    p[1, 0], p[1, 1], p[1, 2], p[1, 3] = half, 0.0, 0.0, -half
    p[2:] = pf
    return p


def generate(wl: Workload, n_events: int | None = None, start: int = 0):
    """Events [start, start+n_events) of workload ``wl``.

    Returns (mom[N][4][E] float64 C-contiguous, w[E] float64).  Events
    failing the cuts are redrawn (same event index, next attempt counter), so
    event k is identical whatever batch it is generated in.
    """
    n = wl.n_events if n_events is None else int(n_events)
    N = N_EXTERNAL[wl.process]
    mom = np.empty((N, 4, n), dtype=np.float64)
    idx = np.arange(start, start + n, dtype=np.uint64)
    todo = np.arange(n)
    attempt = 0
    while todo.size:
        p = _draw(wl, idx[todo], attempt)
        ok = _cuts_pass(p, wl)
        mom[:, :, todo[ok]] = p[:, :, ok]
        todo = todo[~ok]
        attempt += 1
        if attempt > 10000:
            raise RuntimeError("cut acceptance too low")
    uw = _uniforms(wl.seed, idx, 0xFFFFFFFF, 2, stream=1)
    z = np.sqrt(-2.0 * np.log(uw[0])) * np.cos(2.0 * math.pi * uw[1])
    w = np.exp(z)
    return np.ascontiguousarray(mom), np.ascontiguousarray(w)


def boost(mom, beta):
    """Lorentz boost of every momentum of every event by velocity beta
    (3-vector).  Test helper: the summed |M|^2 is boost invariant."""
    bx, by, bz = beta
    b2 = bx * bx + by * by + bz * bz
    g = 1.0 / math.sqrt(1.0 - b2)
    out = np.empty_like(mom)
    e = mom[:, 0]
    bp = bx * mom[:, 1] + by * mom[:, 2] + bz * mom[:, 3]
    out[:, 0] = g * (e + bp)
    f = (g - 1.0) / b2 if b2 > 0 else 0.0
    for k, bk in enumerate((bx, by, bz)):
        out[:, 1 + k] = mom[:, 1 + k] + (f * bp + g * e) * bk
    return out


def rotate(mom, axis, angle):
    """Rotation of all 3-momenta about a unit axis (Rodrigues)."""
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    c, s = math.cos(angle), math.sin(angle)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + s * K + (1 - c) * (K @ K)
    out = mom.copy()
    out[:, 1:] = np.einsum("ij,njk->nik", R, mom[:, 1:])
    return out


# --------------------------------------------------------------------------
# model parameter points (inputs, not arithmetic)
# --------------------------------------------------------------------------
PARAM_FIELDS = ("alpha_s", "m_t", "w_t", "yt_scale", "alpha_em_inv", "G_F", "m_Z", "w_Z")

# Standard Model inputs of the original sample: alpha_s(M_Z), pole top mass,
# top width 0 (every top propagator here is off shell), alpha(M_Z)^-1, G_F,
# M_Z and Gamma_Z.
SM_PARAMS = dict(alpha_s=0.118, m_t=173.0, w_t=0.0, yt_scale=1.0, alpha_em_inv=132.507, G_F=1.16639e-5,
                 m_Z=91.1876, w_Z=2.4952)


def param_vector(**overrides):
    """float64[8] parameter vector (SM_PARAMS with overrides)."""
    d = dict(SM_PARAMS)
    for k, v in overrides.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return np.array([d[f] for f in PARAM_FIELDS], dtype=np.float64)


def coupling_points(n: int):
    """n points with a random electroweak coupling each, alpha' = alpha (0.5 + u),
    u ~ U[0, 1) from the e- e+ -> 5 photons sample's Philox stream 2 (point i
    is the same for every n)."""
    wl = WORKLOADS["ee_5a_1m"]
    u = _uniforms(wl.seed, np.arange(n, dtype=np.uint64), 0, 1, stream=2)[0]
    inv0 = SM_PARAMS["alpha_em_inv"]
    return np.stack([param_vector(alpha_em_inv=inv0 / (0.5 + x)) for x in u])


def reweight_points(workload_name: str, variant: str = "default"):
    """Modified parameter points of each sample, float64[P][8].

    ee_mumu_4k: (M_Z, Gamma_Z) 91.1876/2.4952 -> 92.0/2.6.
    gg_tt_1m:   m_t 173 -> 175 and alpha_s 0.118 -> 0.120 as one point.
    gg_ttg_4m:  64 points kappa = 0.8 + 0.4 i/63; 'default' scales the top
                Yukawa (absent from these tree amplitudes, so r = 1), 'mt'
                scales m_t = kappa * 173 GeV instead.
    gg_ttgg_1m: one point kappa = 1.2, same two variants.
    ee_5a_1m:   8 points with a random electroweak coupling each (the paper's
                benchmark, Table 1): alpha' = alpha (0.5 + u), u ~ U[0, 1)
                from the sample's Philox stream 2.
    """
    if workload_name == "ee_mumu_4k":
        return param_vector(m_Z=92.0, w_Z=2.6)[None]
    if workload_name == "gg_tt_1m":
        return param_vector(m_t=175.0, alpha_s=0.120)[None]
    if workload_name == "ee_5a_1m":
        return coupling_points(8)
    if workload_name in ("gg_ttg_4m", "gg_ttgg_1m"):
        ks = [0.8 + 0.4 * i / 63 for i in range(64)] if workload_name == "gg_ttg_4m" else [1.2]
        if variant == "mt":
            return np.stack([param_vector(m_t=k * M_TOP) for k in ks])
        return np.stack([param_vector(yt_scale=k) for k in ks])
    raise KeyError(workload_name)
