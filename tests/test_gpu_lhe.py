"""GPU: the whole procedure of the paper from an event file -- parse the LHE
events, reweight on the GPU, write the new weights -- against the oracle."""
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
from test_lhe import write_lhe  # noqa: E402


@pytest.mark.parametrize("process,wl", [("gg_ttg", "gg_ttg_4m"), ("ee_5a", "ee_5a_1m")])
def test_lhe_file_reweighted(tmp_path, process, wl):
    mom, w = ev.generate(ev.WORKLOADS[wl], 1500)
    pts = ev.reweight_points(wl, "mt")[::21] if process == "gg_ttg" else ev.reweight_points(wl)[:3]
    src, dst = tmp_path / "in.lhe", tmp_path / "out.lhe"
    write_lhe(src, process, mom, w)
    with rwgt.Lhe(src) as f:
        m, wf = f.read(process, threads=4)
        dev = torch.device("cuda", 0)
        g = rwgt.reweight(process, "fp64", torch.from_numpy(m).to(dev), torch.from_numpy(wf).to(dev),
                          ev.param_vector(), pts)
        wnew = g["wnew"].cpu().numpy()
        f.write(dst, wnew, [f"p{j}" for j in range(len(pts))])
    o = oracle.reweight(process, ev.param_vector(), pts, mom, w)  # the original centre-of-mass events
    assert np.abs(wnew / o["wnew"] - 1).max() < 1e-11
    vals = re.findall(r"<wgt id='p(\d+)'> (\S+) </wgt>", dst.read_text())
    got = np.array([float(v) for _, v in vals]).reshape(1500, len(pts)).T
    assert np.allclose(got, wnew, rtol=1e-10, atol=0)
    for j in range(len(pts)):
        assert abs(g["sigma"][j] / math.fsum(o["wnew"][j]) - 1) < 1e-11
