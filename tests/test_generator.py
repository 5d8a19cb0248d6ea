"""The build-time process generator (CUDA side): diagram counts, colour
matrices against the oracle's brute-force SU(3) sums, emitted code in sync."""
import os

import numpy as np
import pytest

from paper_2312_07440_gb300.gen import qcd_gen


@pytest.mark.parametrize("n,count", [(1, 1), (2, 3), (3, 16), (4, 123)])
def test_p10_diagram_counts(n, count):
    assert qcd_gen.diagram_count(n) == count


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_p7_colour_matrix_matches_oracle(oracle_mod, n):
    Ci, den = qcd_gen.colour_matrix_int(n)
    C, perms = oracle_mod.colour_matrix(n)
    assert [tuple(p) for p in perms] == qcd_gen.orderings(n)
    assert np.abs(np.array(Ci) / den - C).max() < 1e-12 * np.abs(C).max()
    # every integer entry is exact in fp16 and bf16 (8-bit mantissa: |x| <= 256 or a multiple of 2^k)
    import torch
    t = torch.tensor(np.array(Ci, dtype=np.float64))
    assert torch.equal(t.to(torch.float16).double(), t)
    assert torch.equal(t.to(torch.bfloat16).double(), t)


def test_generated_headers_are_current():
    here = os.path.join(os.path.dirname(qcd_gen.__file__), "..", "csrc")
    for name, spec in qcd_gen.PROCESSES.items():
        src, _ = qcd_gen.emit_process(name, *spec)
        with open(os.path.join(here, f"gen_qcd_{name}.cuh")) as f:
            assert f.read() == src, f"regenerate gen_qcd_{name}.cuh"


def test_colour_sum_forms_equal_the_quadratic_form():
    """The two FMA forms the generator emits for J^dagger Cint J (pairs with one
    accumulator per distinct entry; rows z = C A with the helicity-flip factor 2
    folded in) against the plain quadratic form, for random complex amplitudes."""
    rng = np.random.default_rng(11)
    for n in (2, 3, 4):
        Cint, _ = qcd_gen.colour_matrix_int(n)
        C = np.array(Cint, dtype=np.float64)
        K = len(Cint)
        for _ in range(5):
            A = rng.normal(size=K) + 1j * rng.normal(size=K)
            q = float(np.real(np.conj(A) @ C @ A))
            scale = float(np.abs(A) @ np.abs(C) @ np.abs(A))
            pairs = sum(c * np.real(np.conj(A[i]) * A[j]) for i, j, c in qcd_gen.colour_pairs(Cint))
            rows = sum(np.real(np.conj(A[i]) * sum(cf * A[j] for j, cf in row)) for i, row in qcd_gen.colour_rows(Cint))
            assert abs(pairs - q) <= 1e-12 * scale
            assert abs(rows - 2 * q) <= 1e-12 * scale
