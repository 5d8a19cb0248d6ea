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
