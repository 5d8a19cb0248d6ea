"""GPU: the interpolation surrogate (rw_reweight_interp) against the oracle's
exact ratios and the library's exact kernel."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_07440_gb300 import events as ev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_07440_gb300 import rwgt  # noqa: E402

DEV = torch.device("cuda", 0)
BOUND = 1e-3  # |log r_surrogate - log r| per event and point


def run_interp(proc, mode, mom, w, pts, n_nodes, tol, lane_bits=-1):
    with rwgt.Context(0, torch.cuda.current_stream(DEV).cuda_stream) as c:
        c.set_process(proc, mode)
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        if lane_bits >= 0:
            c.set_tuning(lane_bits, 0)
        E = mom.shape[-1]
        dm, dw = torch.from_numpy(mom).to(DEV), torch.from_numpy(w).to(DEV)
        nb = c.workspace_bytes(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        c.load_events(dm, dw, E, ws, nb)
        wn = torch.empty((pts.shape[0], E), dtype=torch.float64, device=DEV)
        fl = torch.empty(E, dtype=torch.uint8, device=DEV)
        out = rwgt.reweight_interp(c, n_nodes, tol, wn, fl)
        torch.cuda.synchronize()
    out["wnew"] = wn.cpu().numpy()
    out["flag"] = fl.cpu().numpy().astype(bool)
    return out


def exact_gpu(proc, mode, mom, w, pts, lane_bits=-1):
    g = rwgt.reweight(proc, mode, torch.from_numpy(mom).to(DEV), torch.from_numpy(w).to(DEV), ev.param_vector(), pts,
                      lane_bits=lane_bits)
    torch.cuda.synchronize()
    return g["wnew"].cpu().numpy()


def check(out, o, w, exact):
    wn, fl = out["wnew"], out["flag"]
    acc = ~fl
    err = np.abs(np.log(wn[:, acc] / o["wnew"][:, acc]))
    assert err.max() <= BOUND
    # recomputed events: the exact kernel (same launch variant), bit for bit
    assert np.array_equal(wn[:, fl], exact[:, fl])
    assert out["n_fallback"] == int(fl.sum()) and out["n_bad"] == o["n_bad"]
    for j in range(wn.shape[0]):
        s = math.fsum(wn[j])
        assert abs(out["sigma"][j] - s) <= 2 * np.spacing(s)
    assert abs(out["sigma_orig"] - math.fsum(w)) <= 2 * np.spacing(out["sigma_orig"])
    return err.max(), fl.mean()


@pytest.mark.parametrize("mode,lb", [("fp32", 0), ("fp32", 1), ("fp64", 0)])
def test_top_mass_axis_64_points(mode, lb):
    """g g -> t tbar g, m_t = kappa 173 GeV for 64 kappa in [0.8, 1.2]: 1 + 7
    exact evaluations per event instead of 65."""
    pts = ev.reweight_points("gg_ttg_4m", "mt")
    mom, w = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 611)
    o = oracle.reweight("gg_ttg", ev.param_vector(), pts, mom, w)
    out = run_interp("gg_ttg", mode, mom, w, pts, 7, 2.5e-4, lane_bits=lb)
    err, ffb = check(out, o, w, exact_gpu("gg_ttg", mode, mom, w, pts, lane_bits=lb))
    print(f"max |d log r| {err:.2e}, recomputed {ffb:.3%}")
    assert ffb < 0.05


def test_coupling_axis_ee_5a():
    """e- e+ -> 5 photons, 8 random couplings: log r = 5 log(alpha'/alpha),
    analytic in alpha_em_inv on the points' range [112, 258] with the nearest
    singularity at 0 (Chebyshev ratio ~4.9): 5 nodes leave ~4e-3, so every
    event is recomputed; 10 nodes ~1e-6 and none is."""
    pts = ev.reweight_points("ee_5a_1m")
    mom, w = ev.generate(ev.WORKLOADS["ee_5a_1m"], 300)
    exact = 5 * np.log(ev.SM_PARAMS["alpha_em_inv"] / pts[:, 4])[:, None]
    out = run_interp("ee_5a", "fp64", mom, w, pts, 5, 2.5e-4)
    assert out["flag"].all() and out["n_fallback"] == 300
    assert np.abs(np.log(out["wnew"] / w[None, :]) - exact).max() < 1e-13
    out = run_interp("ee_5a", "fp64", mom, w, pts, 10, 2.5e-4)
    assert not out["flag"].any()
    assert np.abs(np.log(out["wnew"] / w[None, :]) - exact).max() < 1e-5


def test_points_must_lie_on_one_axis():
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 64)
    pts = ev.reweight_points("gg_tt_1m")  # m_t and alpha_s move together
    with pytest.raises(rwgt.RwError):
        run_interp("gg_tt", "fp64", mom, w, pts, 5, 1e-4)
    pts = np.stack([ev.param_vector(m_t=170.0), ev.param_vector(m_t=176.0)])
    for bad_nodes in (2, 17):
        with pytest.raises(rwgt.RwError):
            run_interp("gg_tt", "fp64", mom, w, pts, bad_nodes, 1e-4)
