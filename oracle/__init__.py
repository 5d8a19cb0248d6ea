"""FP64 CPU oracle for leading-order event reweighting -- TEST INFRASTRUCTURE.

Plain, slow, independently written reference for what the CUDA library
computes (arXiv:2312.07440, Sec. 2: Eq. 2 cross section, Eq. 3 reweighting).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference arms may import it; the product path never does, and it never
imports the product package.  The arithmetic lives in ``oracle.c`` (compiled
here on first use with gcc/OpenMP); the cross-section sums are exact
(``math.fsum``, Shewchuk's adaptive-precision summation).

Parameter vectors are 8 float64 in this order (the same field order as the
library's parameter struct): alpha_s, m_t, w_t, yt_scale, alpha_em_inv, G_F,
m_Z, w_Z.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

PROCESS_ID = {"ee_mumu": 0, "gg_tt": 1, "gg_ttg": 2, "gg_ttgg": 3, "ee_5a": 4}
N_EXTERNAL = {"ee_mumu": 4, "gg_tt": 4, "gg_ttg": 5, "gg_ttgg": 6, "ee_5a": 7}
PARAM_FIELDS = ("alpha_s", "m_t", "w_t", "yt_scale", "alpha_em_inv", "G_F", "m_Z", "w_Z")

_EXT_PATH = os.path.join(_BUILD, "liboracle_ext.so")

_lib = None
_ext = None


def _compile(path, defines, force):
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC", *defines, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (FP64) and
    _build/liboracle_ext.so (the same formulas in long double: 64-bit
    significand on x86-64, 113-bit on AArch64), atomic replace."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_EXT_PATH, ["-DORACLE_EXTENDED"], force)
    return _compile(_LIB_PATH, [], force)


def _batch_signatures(lib):
    i, l, P = ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    lib.oracle_set_threads.argtypes = [i]
    lib.oracle_set_threads.restype = i
    lib.oracle_me.argtypes = [i, P, l, P, P]
    lib.oracle_me.restype = i
    lib.oracle_reshuffle.argtypes = [i, P, l, P, P, P]
    lib.oracle_reshuffle.restype = i
    lib.oracle_reweight.argtypes = [i, P, i, P, l, P, P, P, P, P, P, P]
    lib.oracle_reweight.restype = i


def _load_ext():
    """The extended-precision build (batch entry points only)."""
    global _ext
    if _ext is None:
        build()
        lib = ctypes.CDLL(_EXT_PATH)
        _batch_signatures(lib)
        lib.oracle_init()
        _ext = lib
    return _ext


def _pick(precision):
    if precision == "fp64":
        return _load()
    if precision == "extended":
        return _load_ext()
    raise ValueError(f"precision must be 'fp64' or 'extended', not {precision!r}")


def extended_digits() -> int:
    """Significand bits of the extended build's long double (64 on x86-64,
    113 on AArch64)."""
    return int(np.finfo(np.longdouble).nmant) + 1


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
    P = ctypes.c_void_p
    lib.oracle_set_threads.argtypes = [i]
    lib.oracle_set_threads.restype = i
    lib.oracle_me.argtypes = [i, P, l, P, P]
    lib.oracle_me.restype = i
    lib.oracle_reshuffle.argtypes = [i, P, l, P, P, P]
    lib.oracle_reshuffle.restype = i
    lib.oracle_reweight.argtypes = [i, P, i, P, l, P, P, P, P, P, P, P]
    lib.oracle_reweight.restype = i
    lib.oracle_colour_matrix.argtypes = [i, P, P]
    lib.oracle_colour_matrix.restype = i
    lib.oracle_su3.argtypes = [P, P]
    lib.oracle_su3.restype = None
    lib.oracle_dirac.argtypes = [P, P]
    lib.oracle_dirac.restype = None
    lib.oracle_external.argtypes = [i, P, d, i, P, P]
    lib.oracle_external.restype = i
    lib.oracle_spinor.argtypes = [i, P, d, i, i, P]
    lib.oracle_spinor.restype = None
    lib.oracle_polvec.argtypes = [P, i, i, P]
    lib.oracle_polvec.restype = None
    lib.oracle_partial_amps.argtypes = [i, P, d, d, P, P]
    lib.oracle_partial_amps.restype = i
    lib.oracle_me_traces.argtypes = [i, P, P]
    lib.oracle_me_traces.restype = d
    lib.oracle_full_colour_amp.argtypes = [i, P, d, d, P, P, P]
    lib.oracle_full_colour_amp.restype = i
    lib.oracle_ee_photons.argtypes = [i, P, P, i, P, P, P]
    lib.oracle_ee_photons.restype = d
    lib.oracle_init()
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def params(**kw) -> np.ndarray:
    """Parameter vector from keyword arguments (missing fields raise)."""
    return np.array([float(kw[f]) for f in PARAM_FIELDS], dtype=np.float64)


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (n <= 0 keeps it); returns the count."""
    return _load().oracle_set_threads(int(n))


def me(process: str, par, mom, precision: str = "fp64") -> np.ndarray:
    """|M|^2 per event.  mom: float64 [N][4][E].  precision "extended"
    evaluates the same formulas in long double (result rounded to float64)."""
    lib = _pick(precision)
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    E = mom.shape[-1]
    out = np.empty(E)
    par = np.ascontiguousarray(par, dtype=np.float64)
    rc = lib.oracle_me(PROCESS_ID[process], _ptr(par), E, _ptr(mom), _ptr(out))
    assert rc == 0
    return out


def reshuffle(process: str, par_new, mom):
    """Move events onto the mass shells of ``par_new`` (status 1 = no fit)."""
    lib = _load()
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    out = np.empty_like(mom)
    st = np.empty(mom.shape[-1], dtype=np.int32)
    par_new = np.ascontiguousarray(par_new, dtype=np.float64)
    lib.oracle_reshuffle(PROCESS_ID[process], _ptr(par_new), mom.shape[-1], _ptr(mom), _ptr(out), _ptr(st))
    return out, st


def reweight(process: str, par0, points, mom, w, precision: str = "fp64"):
    """Eq. 3 for every parameter point and Eq. 2 sums.

    Returns dict(me0[E], me[P][E], ratio[P][E], wnew[P][E], sigma[P],
    sigma_orig, n_bad); sigma are exactly rounded sums (math.fsum).
    precision "extended": the same formulas in long double, every result
    rounded to float64 once at the end.
    """
    lib = _pick(precision)
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    par0 = np.ascontiguousarray(par0, dtype=np.float64)
    pts = np.ascontiguousarray(np.atleast_2d(points), dtype=np.float64)
    P, E = pts.shape[0], mom.shape[-1]
    me0 = np.empty(E)
    mep = np.empty((P, E))
    ratio = np.empty((P, E))
    wnew = np.empty((P, E))
    nbad = ctypes.c_long(0)
    rc = lib.oracle_reweight(PROCESS_ID[process], _ptr(par0), P, _ptr(pts), E, _ptr(mom), _ptr(w), _ptr(me0),
                             _ptr(mep), _ptr(ratio), _ptr(wnew), ctypes.byref(nbad))
    assert rc == 0
    return {
        "me0": me0, "me": mep, "ratio": ratio, "wnew": wnew,
        "sigma": np.array([math.fsum(wnew[j]) for j in range(P)]),
        "sigma_orig": math.fsum(w), "n_bad": int(nbad.value),
    }


def colour_matrix(n: int):
    """(C[K][K], orderings[K][n]) for n gluons; orderings lexicographic."""
    lib = _load()
    K = math.factorial(n)
    C = np.empty((K, K))
    perms = np.empty((K, n), dtype=np.int32)
    lib.oracle_colour_matrix(n, _ptr(C), _ptr(perms))
    return C, perms


def su3():
    """(t[8][3][3] complex, f[8][8][8]) as used by the oracle."""
    lib = _load()
    t = np.empty((8, 3, 3), dtype=np.complex128)
    f = np.empty((8, 8, 8))
    lib.oracle_su3(_ptr(t), _ptr(f))
    return t, f


def dirac():
    lib = _load()
    g = np.empty((4, 4, 4), dtype=np.complex128)
    g5 = np.empty((4, 4), dtype=np.complex128)
    lib.oracle_dirac(_ptr(g), _ptr(g5))
    return g, g5


def external(process: str, p_aos, m: float, basis: int, hel) -> np.ndarray:
    """External wavefunctions ext[N][4] of one event (AoS momenta p[N][4])."""
    lib = _load()
    p = np.ascontiguousarray(p_aos, dtype=np.float64)
    h = np.ascontiguousarray(hel, dtype=np.int32)
    ext = np.empty((p.shape[0], 4), dtype=np.complex128)
    rc = lib.oracle_external(PROCESS_ID[process], _ptr(p), m, basis, _ptr(h), _ptr(ext))
    assert rc == 0
    return ext


def spinor(kind: str, p, m: float, basis: int, s: int) -> np.ndarray:
    lib = _load()
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty(4, dtype=np.complex128)
    lib.oracle_spinor(0 if kind == "u" else 1, _ptr(p), m, basis, s, _ptr(out))
    return out


def polvec(k, basis: int, s: int) -> np.ndarray:
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.float64)
    out = np.empty(4, dtype=np.complex128)
    lib.oracle_polvec(_ptr(k), basis, s, _ptr(out))
    return out


def partial_amps(process: str, p_aos, m: float, alpha_s: float, ext) -> np.ndarray:
    """Colour-ordered partial amplitudes A[K] (orderings as colour_matrix)."""
    lib = _load()
    p = np.ascontiguousarray(p_aos, dtype=np.float64)
    ext = np.ascontiguousarray(ext, dtype=np.complex128)
    n = N_EXTERNAL[process] - 2
    A = np.empty(math.factorial(n), dtype=np.complex128)
    lib.oracle_partial_amps(PROCESS_ID[process], _ptr(p), m, alpha_s, _ptr(ext), _ptr(A))
    return A


def me_traces(process: str, par, p_aos) -> float:
    """|M|^2 of one event from spin-sum traces (independent of the spinors)."""
    lib = _load()
    p = np.ascontiguousarray(p_aos, dtype=np.float64)
    par = np.ascontiguousarray(par, dtype=np.float64)
    return lib.oracle_me_traces(PROCESS_ID[process], _ptr(par), _ptr(p))


def full_colour_amp(process: str, p_aos, m: float, alpha_s: float, ext, adj) -> np.ndarray:
    """M[3][3] from the colour-dressed Feynman rules for gluon colours adj."""
    lib = _load()
    p = np.ascontiguousarray(p_aos, dtype=np.float64)
    ext = np.ascontiguousarray(ext, dtype=np.complex128)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    M = np.empty(9, dtype=np.complex128)
    lib.oracle_full_colour_amp(PROCESS_ID[process], _ptr(p), m, alpha_s, _ptr(ext), _ptr(adj), _ptr(M))
    return M.reshape(3, 3)


def ee_photons(n: int, par, p_aos, basis: int = 0, hel=None, eps=None):
    """e- e+ -> n photons for one event p_aos[n+2][4]: (|M|^2 spin-averaged
    with 1/4 and 1/n!, helicity amplitude for hel[n+2] in ``basis`` or None).
    ``eps`` (complex [n][4], used as given) replaces the photon polarisations
    of the amplitude (gauge tests)."""
    lib = _load()
    par = np.ascontiguousarray(par, dtype=np.float64)
    p = np.ascontiguousarray(p_aos, dtype=np.float64).reshape(n + 2, 4)
    amp = np.zeros(1, dtype=np.complex128)
    h = None if hel is None else np.ascontiguousarray(hel, dtype=np.int32)
    ep = None if eps is None else np.ascontiguousarray(eps, dtype=np.complex128).reshape(n, 4)
    me2 = lib.oracle_ee_photons(n, _ptr(par), _ptr(p), basis, _ptr(h) if h is not None else None,
                                _ptr(amp) if h is not None else None, _ptr(ep) if ep is not None else None)
    return me2, (complex(amp[0]) if h is not None else None)
