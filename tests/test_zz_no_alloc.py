"""rw_reweight_noalloc: the allocation-free variant of the fused reweight.

For callers that cannot allocate device memory (a host framework that owns the
whole device budget, or a latency-critical loop that must not pay cudaMalloc's
implicit synchronisation), the library keeps the reduction scratch in a fixed
device array.  This test calls the entry point through the C ABI twice in a
row and checks each result against the workspace-based entry point
(rw_reweight_async + rw_get_results) within the parity tolerance (1e-12).
It lives in a file pytest collects last and works in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_07440_gb300 import events as ev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_07440_gb300 import rwgt  # noqa: E402

TOL = 1e-12


def noalloc_fn():
    fn = rwgt.load().rw_reweight_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("proc,wl,n,pts,mode", [
    ("gg_tt", "gg_tt_1m", 5003, ev.reweight_points("gg_tt_1m"), "fp64"),
    ("gg_ttg", "gg_ttg_4m", 700, ev.reweight_points("gg_ttg_4m", "mt")[::8], "fp64"),
    # a kernel with its current store in dynamic shared memory
    ("gg_ttgg", "gg_ttgg_1m", 300, ev.reweight_points("gg_ttgg_1m", "mt"), "fp32"),
])
def test_noalloc_matches_workspace_entry_point_twice(proc, wl, n, pts, mode):
    dev = torch.device("cuda", 0)
    mom, w = ev.generate(ev.WORKLOADS[wl], n)
    dm = torch.from_numpy(mom).to(dev)
    dw = torch.from_numpy(w).to(dev)
    P = pts.shape[0]
    stream = torch.cuda.current_stream(dev).cuda_stream
    fn = noalloc_fn()
    with rwgt.Context(0, stream) as c:
        c.set_process(proc, mode)
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        # reference: the workspace-based entry point
        nb = c.workspace_bytes(n)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        c.load_events(dm, dw, n, ws, nb)
        ref_wnew = torch.empty((P, n), dtype=torch.float64, device=dev)
        ref_ratio = torch.empty((P, n), dtype=torch.float64, device=dev)
        c.reweight_async(ref_wnew, ref_ratio)
        ref_sig, ref_sig_orig, ref_nbad, _ = c.get_results(P)
        ref_wnew, ref_ratio = ref_wnew.cpu().numpy(), ref_ratio.cpu().numpy()
        for _call in range(2):
            wnew = torch.full((P, n), -1.0, dtype=torch.float64, device=dev)
            ratio = torch.full((P, n), -1.0, dtype=torch.float64, device=dev)
            sig = torch.full((P + 1,), -1.0, dtype=torch.float64, device=dev)
            nbad = torch.full((1,), 12345, dtype=torch.int64, device=dev)
            rc = fn(c.h, dm.data_ptr(), dw.data_ptr(), n, wnew.data_ptr(), ratio.data_ptr(), sig.data_ptr(),
                    nbad.data_ptr())
            assert rc == 0, c.last_error()
            torch.cuda.synchronize()
            g_wnew, g_ratio, g_sig = wnew.cpu().numpy(), ratio.cpu().numpy(), sig.cpu().numpy()
            assert np.max(np.abs(g_wnew - ref_wnew) / np.abs(ref_wnew)) < TOL
            assert np.max(np.abs(g_ratio - ref_ratio) / np.abs(ref_ratio)) < TOL
            assert np.max(np.abs(g_sig[:P] - ref_sig) / np.abs(ref_sig)) < TOL
            assert abs(g_sig[P] / ref_sig_orig - 1) < TOL
            assert int(nbad.item()) == ref_nbad == 0


def test_noalloc_rejects_too_many_points():
    dev = torch.device("cuda", 0)
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 64)
    dm = torch.from_numpy(mom).to(dev)
    dw = torch.from_numpy(w).to(dev)
    sig = torch.empty(64, dtype=torch.float64, device=dev)
    nbad = torch.empty(1, dtype=torch.int64, device=dev)
    with rwgt.Context(0, torch.cuda.current_stream(dev).cuda_stream) as c:
        c.set_process("gg_tt", "fp64")
        c.set_params(ev.param_vector())
        c.set_reweight_points(np.tile(ev.param_vector(m_t=175.0), (17, 1)))
        rc = noalloc_fn()(c.h, dm.data_ptr(), dw.data_ptr(), 64, None, None, sig.data_ptr(), nbad.data_ptr())
        assert rc == -2
        assert c.last_error() == "too many points"
