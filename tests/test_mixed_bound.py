"""The mixed-precision error statement (the colour sum of the mixed modes):
J scaled by a power of two so that max |J_k| lies in [0.5, 1), each real and
imaginary part rounded to FP16 (11 significant bits) or BF16 (8), then
J16^dagger C J16 with the exact colour matrix.  The stated bound on the
relative change of J^dagger C J is 2 u sqrt(kappa(C)), u = 2^-11 or 2^-8 and
kappa the condition number of the positive-definite C.  Checked here with the
roundings done bit-exactly on the CPU, for colour vectors of the kinds the
amplitudes produce (comparable orderings, one dominant ordering, orderings
spread over decades), on the colour matrices of two, three and four gluons."""
import math

import numpy as np
import pytest

import oracle


def round_fp16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def round_bf16(x):
    """Round to nearest even BF16 (the top 16 bits of an FP32 word)."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded(J, rnd):
    """The scaled, rounded vector back in the original scale (the power of two
    is exact), as the colour passes see it."""
    mx = np.max(np.abs(np.concatenate([J.real, J.imag])))
    e = math.frexp(mx)[1] if mx > 0 else 0
    s = 2.0 ** -e
    return (rnd(J.real * s) + 1j * rnd(J.imag * s)) / s


def quad(C, J):
    return float(np.real(np.conj(J) @ C @ J))


@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("mode", ["fp16", "bf16"])
def test_rounding_j_stays_within_the_stated_bound(n, mode):
    C, _ = oracle.colour_matrix(n)
    K = C.shape[0]
    ev = np.linalg.eigvalsh(C)
    assert ev.min() > 0  # positive definite: J^dagger C J > 0 for J != 0
    u = 2.0 ** -11 if mode == "fp16" else 2.0 ** -8
    bound = 2 * u * math.sqrt(ev.max() / ev.min())
    rnd = round_fp16 if mode == "fp16" else round_bf16
    rng = np.random.default_rng(17 + n)
    worst = 0.0
    for trial in range(3000):
        kind = trial % 3
        J = rng.normal(size=K) + 1j * rng.normal(size=K)
        if kind == 1:
            J[rng.integers(K)] *= 50.0  # one dominant ordering
        elif kind == 2:
            J *= 10.0 ** rng.uniform(-6, 0, size=K)  # orderings spread over decades
        J *= 10.0 ** rng.uniform(-8, 3)  # any overall scale: the power of two removes it
        exact = quad(C, J)
        err = abs(quad(C, rounded(J, rnd)) - exact) / exact
        worst = max(worst, err)
        assert err <= bound, (trial, err, bound)
    # the bound is not loose by orders of magnitude: rounding errors reach a
    # visible part of it
    assert worst > bound / 100


def test_bf16_rounding_helper():
    """Round to nearest even at the 8th significant bit, checked on values
    whose BF16 neighbours are known."""
    one_ulp = 2.0 ** -7  # BF16 spacing in [1, 2)
    assert round_bf16(1.0) == 1.0
    assert round_bf16(1.0 + one_ulp) == 1.0 + one_ulp
    assert round_bf16(1.0 + one_ulp / 2) == 1.0  # tie to even
    assert round_bf16(1.0 + 3 * one_ulp / 2) == 1.0 + 2 * one_ulp  # tie to even
    assert round_bf16(1.0 + 0.6 * one_ulp) == 1.0 + one_ulp
    assert round_bf16(-3.0) == -3.0
