"""GPU: the whole procedure of the paper from an event file -- parse the LHE
events, reweight on the GPU, write the new weights -- against the oracle.

The files are written in the partonic centre-of-mass frame, so the momenta
read back are the seeded sample's bit for bit and the FP64 bound of 1e-12 and
the oracle's extended-precision re-check apply as in the other parity tests
(the reader's boost from a lab frame is tested on the CPU, tests/test_lhe.py).
The weights are written in the shortest form that reads back as the same
double, so the file itself is compared exactly with the kernel's W'.
"""
import math
import re

import numpy as np
import pytest

import oracle
from paper_2312_07440_gb300 import events as ev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_07440_gb300 import rwgt  # noqa: E402
from parity_helpers import POINT_SETS, check_against_oracle  # noqa: E402
from test_lhe import write_lhe  # noqa: E402

DEV = torch.device("cuda", 0)


def file_weights(path, P):
    vals = re.findall(r"<wgt id='p(\d+)'> (\S+) </wgt>", path.read_text())
    return np.array([float(v) for _, v in vals]).reshape(-1, P).T


@pytest.mark.parametrize("process,wl,n,pts_name,set_name", [
    ("gg_ttg", "gg_ttg_4m", 611, "gg_ttg_mt4", "gg_ttg_611"),
    ("ee_5a", "ee_5a_1m", 517, "ee_5a_3", "ee_5a_517"),
])
def test_lhe_file_reweighted(tmp_path, process, wl, n, pts_name, set_name):
    mom, w = ev.generate(ev.WORKLOADS[wl], n)
    pts = POINT_SETS[pts_name]()
    src, dst = tmp_path / "in.lhe", tmp_path / "out.lhe"
    write_lhe(src, process, mom, w, beta=0.0)
    with rwgt.Lhe(src) as f:
        m, wf = f.read(process, threads=4)
        assert np.array_equal(m, mom) and np.array_equal(wf, w)
        g = rwgt.reweight(process, "fp64", torch.from_numpy(m).to(DEV), torch.from_numpy(wf).to(DEV),
                          ev.param_vector(), pts)
        g = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in g.items()}
        f.write(dst, g["wnew"], [f"p{j}" for j in range(len(pts))])
    o = oracle.reweight(process, ev.param_vector(), pts, m, wf)
    check_against_oracle(g, o, "fp64", (process, pts, m, wf), set_name)
    assert np.array_equal(file_weights(dst, len(pts)), g["wnew"])


@pytest.mark.parametrize("chunk", [1237, 5003, 100000])
def test_pipelined_file_reweight(tmp_path, chunk):
    """rw_lhe_reweight (parsing of chunk k+1 and writing of chunk k-1 on the
    host while the GPU reweights chunk k) writes the same file, byte for
    byte, as parsing everything, reweighting and writing in turn; its weights
    match the oracle per event and its sums are the exact sums of the
    written weights."""
    n = 5003
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], n)
    pts = POINT_SETS["gg_tt_five"]()[:2]
    ids = ["p0", "p1"]
    src = tmp_path / "in.lhe"
    write_lhe(src, "gg_tt", mom, w, beta=0.0)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    with rwgt.Context(0, stream) as c, rwgt.Lhe(src) as f:
        c.set_process("gg_tt", "fp64")
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        nb = rwgt.lhe_workspace_bytes(c, chunk)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        sig, so, nbad, _ = rwgt.lhe_reweight(c, f, tmp_path / "piped.lhe", ids, chunk, ws, nb, threads=3)
        # the same steps one after the other
        m, wf = f.read("gg_tt", threads=3)
        g = rwgt.reweight("gg_tt", "fp64", torch.from_numpy(m).to(DEV), torch.from_numpy(wf).to(DEV),
                          ev.param_vector(), pts)
        f.write(tmp_path / "plain.lhe", g["wnew"].cpu().numpy(), ids)
    assert (tmp_path / "piped.lhe").read_bytes() == (tmp_path / "plain.lhe").read_bytes()
    wnew = file_weights(tmp_path / "piped.lhe", 2)
    o = oracle.reweight("gg_tt", ev.param_vector(), pts, mom, w)
    assert np.max(np.abs(wnew / o["wnew"] - 1)) < 1e-12
    assert nbad == 0
    for j in range(2):
        exact = math.fsum(wnew[j])
        assert abs(sig[j] - exact) <= 2 * np.spacing(exact)
    assert abs(so - math.fsum(w)) <= 2 * np.spacing(so)
