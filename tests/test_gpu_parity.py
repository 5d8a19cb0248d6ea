"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (per event, relative): 1e-12 in FP64 mode, 1e-5 in FP32 mode, on
|M|^2, |M'|^2, r and W', flat for every event (FP64 mode: against the
extended-precision oracle where the FP64 oracle's own rounding matters, see
check_against_oracle).  Cross sections: the GPU sigma' must equal the exactly
rounded sum of the GPU's own W' to 2 ulp (compensated summation), and agree
with the oracle's exact sum to the per-event tolerance.
"""
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
from parity_helpers import POINT_SETS, TOL, check_against_oracle, rel  # noqa: E402

DEV = torch.device("cuda", 0)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


_ORACLE_CACHE = {}


def oracle_run(proc, wl_name, n, pts, start=0):
    key = (proc, wl_name, n, start, pts.tobytes())
    if key not in _ORACLE_CACHE:
        mom, w = ev.generate(ev.WORKLOADS[wl_name], n, start=start)
        _ORACLE_CACHE[key] = (mom, w, oracle.reweight(proc, ev.param_vector(), pts, mom, w))
    return _ORACLE_CACHE[key]


def run_gpu(proc, mode, mom, w, pts, lane_bits=-1, block=0):
    out = rwgt.reweight(proc, mode, to_dev(mom), to_dev(w), ev.param_vector(), pts, lane_bits=lane_bits,
                        block=block)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


# --------------------------------------------------------------------------
# g g -> t tbar (the 1M-event workload's process), every launch variant
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("lane_bits", [0, 1, 2])
def test_gg_tt_parity(mode, lane_bits):
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 5003, pts)  # several blocks + a ragged tail
    g = run_gpu("gg_tt", mode, mom, w, pts, lane_bits=lane_bits)
    check_against_oracle(g, o, mode, ("gg_tt", pts, mom, w), "gg_tt_5003")


@pytest.mark.parametrize("block", [32, 64, 256])
def test_gg_tt_block_sizes(block):
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 5003, pts)
    g = run_gpu("gg_tt", "fp64", mom, w, pts, block=block)
    check_against_oracle(g, o, "fp64", ("gg_tt", pts, mom, w), "gg_tt_5003")


def test_gg_tt_several_points_and_alpha_s_scaling():
    pts = np.stack([ev.param_vector(alpha_s=0.120), ev.param_vector(m_t=175.0), ev.param_vector(),
                    ev.param_vector(m_t=175.0, alpha_s=0.120), ev.param_vector(m_t=160.0)])
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 777, pts)
    g = run_gpu("gg_tt", "fp64", mom, w, pts)
    check_against_oracle(g, o, "fp64", ("gg_tt", pts, mom, w), "gg_tt_777_five")
    assert np.abs(g["ratio"][0] / (0.120 / 0.118) ** 2 - 1).max() < 1e-14   # P9
    assert np.all(g["ratio"][2] == 1.0) and np.all(g["wnew"][2] == w)       # P8 (bitwise)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_ee_mumu_parity_full_sample(mode):
    pts = ev.reweight_points("ee_mumu_4k")
    mom, w, o = oracle_run("ee_mumu", "ee_mumu_4k", 4096, pts)
    for lb in ([0, 2, 4] if mode == "fp64" else [0]):
        g = run_gpu("ee_mumu", mode, mom, w, pts, lane_bits=lb)
        check_against_oracle(g, o, mode, ("ee_mumu", pts, mom, w), "ee_mumu_4096")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("lane_bits", [0, 1, 2, 3])
def test_gg_ttg_parity(mode, lane_bits):
    pts = ev.reweight_points("gg_ttg_4m", "mt")[::21]  # kappa = 0.8, 0.933, 1.067, 1.2 (m_t = kappa 173)
    mom, w, o = oracle_run("gg_ttg", "gg_ttg_4m", 611, pts)
    g = run_gpu("gg_ttg", mode, mom, w, pts, lane_bits=lane_bits)
    check_against_oracle(g, o, mode, ("gg_ttg", pts, mom, w), "gg_ttg_611")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_gg_ttgg_parity(mode):
    pts = ev.reweight_points("gg_ttgg_1m", "mt")
    mom, w, o = oracle_run("gg_ttgg", "gg_ttgg_1m", 197, pts)
    for lb in (1, 2, 3, 4) if mode == "fp32" else (1, 2, 3):
        g = run_gpu("gg_ttgg", mode, mom, w, pts, lane_bits=lb)
        check_against_oracle(g, o, mode, ("gg_ttgg", pts, mom, w), "gg_ttgg_197")


@pytest.mark.parametrize("lane_bits,block", [(2, 64), (2, 128), (3, 64), (3, 256), (4, 64), (4, 256)])
def test_gg_ttgg_fp32_shared_event_constants(lane_bits, block):
    """FP32 with 4-16 lanes per event keeps each event's constants in one
    shared-memory slot per event group: every slot placement (groups of 4, 8
    and 16 lanes; up to the largest block that fits, 128 threads with 4 lanes
    per event and 256 with 8 or 16; a ragged last block) against the oracle,
    for the original point and a moved top mass (the slot is rewritten between
    the two evaluations)."""
    pts = ev.reweight_points("gg_ttgg_1m", "mt")
    mom, w, o = oracle_run("gg_ttgg", "gg_ttgg_1m", 197, pts)
    g = run_gpu("gg_ttgg", "fp32", mom, w, pts, lane_bits=lane_bits, block=block)
    check_against_oracle(g, o, "fp32", ("gg_ttgg", pts, mom, w), "gg_ttgg_197")


# --------------------------------------------------------------------------
# e- e+ -> 5 photons (the paper's benchmark process), random coupling points
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("lane_bits", [0, 1, 2, 3])
def test_ee_5a_parity(mode, lane_bits):
    pts = ev.reweight_points("ee_5a_1m")[:3]
    mom, w, o = oracle_run("ee_5a", "ee_5a_1m", 517, pts)  # several blocks + a ragged tail
    g = run_gpu("ee_5a", mode, mom, w, pts, lane_bits=lane_bits)
    check_against_oracle(g, o, mode, ("ee_5a", pts, mom, w), "ee_5a_517")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_ee_5a_coupling_only_points(mode):
    """Unchanged parameters give r == 1 bitwise (P8); a coupling change gives
    r = (alpha'/alpha)^5 for every event (only e enters)."""
    pts = np.stack([ev.param_vector(), ev.param_vector(alpha_em_inv=100.0)])
    mom, w = ev.generate(ev.WORKLOADS["ee_5a_1m"], 300)
    g = run_gpu("ee_5a", mode, mom, w, pts)
    assert np.all(g["ratio"][0] == 1.0) and np.all(g["wnew"][0] == w)
    assert np.abs(g["ratio"][1] / (ev.SM_PARAMS["alpha_em_inv"] / 100.0) ** 5 - 1).max() < 1e-14


def test_ee_5a_has_no_mixed_mode():
    mom, w = ev.generate(ev.WORKLOADS["ee_5a_1m"], 64)
    with pytest.raises(rwgt.RwError):
        run_gpu("ee_5a", "mixed_fp16", mom, w, ev.reweight_points("ee_5a_1m"))


def test_yukawa_axis_gives_unit_ratio():
    pts = ev.reweight_points("gg_ttg_4m")[:8]
    mom, w = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 300)
    g = run_gpu("gg_ttg", "fp64", mom, w, pts)
    assert np.all(g["ratio"] == 1.0)


# --------------------------------------------------------------------------
# edge cases and error behaviour
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 31, 33, 129])
def test_tiny_batches(n):
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", n, pts)
    g = run_gpu("gg_tt", "fp64", mom, w, pts)
    check_against_oracle(g, o, "fp64", ("gg_tt", pts, mom, w), "gg_tt_5003")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_maximum_number_of_points(mode):
    """256 parameter points in one launch (the most a context takes): m_t and
    alpha_s on a 16 x 16 grid, a ragged number of events."""
    mts = np.linspace(165.0, 181.0, 16)
    als = np.linspace(0.110, 0.126, 16)
    pts = np.stack([ev.param_vector(m_t=m, alpha_s=a) for m in mts for a in als])
    assert pts.shape[0] == 256
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 77, pts)
    g = run_gpu("gg_tt", mode, mom, w, pts)
    check_against_oracle(g, o, mode, ("gg_tt", pts, mom, w), "gg_tt_77_256")


def test_bad_events_are_counted_and_excluded():
    pts = ev.reweight_points("gg_tt_1m")
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 500)
    mom[:, :, 17] = 0.0      # |M|^2 = NaN
    mom[:, :, 400] = np.nan
    o = oracle.reweight("gg_tt", ev.param_vector(), pts, mom, w)
    g = run_gpu("gg_tt", "fp64", mom, w, pts)
    assert g["status"] == rwgt.RW_WARN_BAD_EVENTS and g["n_bad"] == 2 == o["n_bad"]
    for k in (17, 400):
        assert g["ratio"][0, k] == 0.0 and g["wnew"][0, k] == 0.0
    ok = np.ones(500, bool)
    ok[[17, 400]] = False
    assert rel(g["wnew"][0, ok], o["wnew"][0, ok]).max() < 1e-12
    assert abs(g["sigma"][0] / o["sigma"][0] - 1) < 1e-12


def test_mass_that_does_not_fit_gives_zero_weight():
    pts = ev.param_vector(m_t=700.0)[None]
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 400)
    o = oracle.reweight("gg_tt", ev.param_vector(), pts, mom, w)
    g = run_gpu("gg_tt", "fp64", mom, w, pts)
    out = (mom[0, 0] + mom[1, 0]) <= 1400.0
    assert out.any() and np.all(g["wnew"][0, out] == 0.0) and np.all(o["wnew"][0, out] == 0.0)
    assert rel(g["wnew"][0], o["wnew"][0]).max() < 1e-12


def test_deterministic_results():
    pts = ev.reweight_points("gg_tt_1m")
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 20000)
    a = run_gpu("gg_tt", "fp64", mom, w, pts)
    b = run_gpu("gg_tt", "fp64", mom, w, pts)
    assert np.array_equal(a["wnew"], b["wnew"]) and np.array_equal(a["sigma"], b["sigma"])


def test_eval_me_matches_fused_path():
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 1000, pts)
    dm, dw = to_dev(mom), to_dev(w)
    stream = torch.cuda.current_stream().cuda_stream
    with rwgt.Context(0, stream) as c:
        c.set_process("gg_tt", "fp64")
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        nb = c.workspace_bytes(1000)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        c.load_events(dm, dw, 1000, ws, nb)
        me0 = torch.empty(1000, dtype=torch.float64, device=DEV)
        me1 = torch.empty(1000, dtype=torch.float64, device=DEV)
        c.eval_me(-1, me0)
        c.eval_me(0, me1)
        torch.cuda.synchronize()
    assert rel(me0.cpu().numpy(), o["me0"]).max() < 1e-12
    assert rel(me1.cpu().numpy(), o["me"][0]).max() < 1e-12


def test_host_entry_point_matches_device_path():
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 3001, pts)
    with rwgt.Context(0, torch.cuda.current_stream().cuda_stream) as c:
        c.set_process("gg_tt", "fp64")
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        nb = c.workspace_bytes_host(3001)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        hw = np.empty((1, 3001))
        sig, so, nbad, rc = c.reweight_host(np.ascontiguousarray(mom), np.ascontiguousarray(w), 3001, hw, 1, ws, nb)
    assert rc == 0 and nbad == 0
    assert rel(hw, o["wnew"]).max() < 1e-12
    assert abs(sig[0] - math.fsum(hw[0])) <= 2 * np.spacing(sig[0])


@pytest.mark.parametrize("proc,wl,mode,E", [
    ("gg_tt", "gg_tt_1m", "fp64", 300001),   # several chunks and a ragged last one
    ("gg_ttgg", "gg_ttgg_1m", "fp32", 30001),  # a kernel with its current store in shared memory
])
def test_host_entry_point_pipelined_chunks(proc, wl, mode, E):
    """A batch larger than one launch's resident threads goes through the
    chunked copy/compute pipeline: W' bit-identical to the device path, the
    carried sums within 2 ulp of the exact sums, and the same result without
    the W' copy-out."""
    pts = np.stack([ev.param_vector(m_t=175.0, alpha_s=0.120), ev.param_vector(m_t=170.0)])
    mom, w = ev.generate(ev.WORKLOADS[wl], E)
    g = run_gpu(proc, mode, mom, w, pts)
    with rwgt.Context(0, torch.cuda.current_stream().cuda_stream) as c:
        c.set_process(proc, mode)
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        nb = c.workspace_bytes_host(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        hm, hwt = torch.from_numpy(mom).pin_memory(), torch.from_numpy(w).pin_memory()
        hw = torch.empty((2, E), dtype=torch.float64).pin_memory()
        sig, so, nbad, rc = c.reweight_host(hm, hwt, E, hw, 2, ws, nb)
        sig2, so2, _, _ = c.reweight_host(hm, hwt, E, None, 2, ws, nb)
    hw = hw.numpy()
    assert rc == 0 and nbad == 0
    assert np.array_equal(hw, g["wnew"])
    for j in range(2):
        assert abs(sig[j] - math.fsum(hw[j])) <= 2 * np.spacing(sig[j])
    assert abs(so - math.fsum(w)) <= 2 * np.spacing(so)
    assert np.array_equal(sig, sig2) and so == so2


def test_argument_errors():
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 64)
    dm, dw = to_dev(mom), to_dev(w)
    with rwgt.Context(0, torch.cuda.current_stream().cuda_stream) as c:
        with pytest.raises(rwgt.RwError) as e:
            c.load_events(dm, dw, 64, None, 0)
        assert e.value.code == -6  # no process yet
        c.set_process("gg_tt", "fp64")
        for bad in (dict(w_t=1.5), dict(alpha_s=-0.1), dict(m_t=float("nan"))):
            with pytest.raises(rwgt.RwError) as e:
                c.set_params(ev.param_vector(**bad))
            assert e.value.code == -4
        c.set_params(ev.param_vector())
        with pytest.raises(rwgt.RwError) as e:
            c.set_reweight_points(np.zeros((0, 8)))
        assert e.value.code == -2
        with pytest.raises(rwgt.RwError) as e:
            c.set_reweight_points(np.tile(ev.param_vector(), (300, 1)))
        assert e.value.code == -2
        c.set_reweight_points(ev.reweight_points("gg_tt_1m"))
        nb = c.workspace_bytes(64)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        with pytest.raises(rwgt.RwError) as e:
            c.load_events(dm, dw, 0, ws, nb)
        assert e.value.code == -2
        with pytest.raises(rwgt.RwError) as e:
            c.load_events(dm, dw, 64, ws, nb - 1)
        assert e.value.code == -8
        with pytest.raises(rwgt.RwError) as e:
            c.load_events(dm.data_ptr() + 4, dw, 64, ws, nb)
        assert e.value.code == -7
        with pytest.raises(rwgt.RwError) as e:
            c.load_events(np.ascontiguousarray(mom), dw, 64, ws, nb)  # host pointer
        assert e.value.code in (-2, -5)
        with pytest.raises(rwgt.RwError) as e:
            c.reweight_async()
        assert e.value.code == -6  # no events
        with pytest.raises(rwgt.RwError) as e:
            c.set_tuning(7, 0)
        assert e.value.code == -3


# --------------------------------------------------------------------------
# full size, in the benchmark's launch configuration: sampled events
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_gg_tt_full_size_sampled(mode):
    wl = ev.WORKLOADS["gg_tt_1m"]
    pts = ev.reweight_points("gg_tt_1m")
    mom, w = ev.generate(wl)
    g = run_gpu("gg_tt", mode, mom, w, pts)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, wl.n_events, 1500), np.argsort(g["me0"])[:50],
                                    np.argsort(g["me0"])[-50:], [0, wl.n_events - 1]]))
    o = oracle.reweight("gg_tt", ev.param_vector(), pts, np.ascontiguousarray(mom[:, :, idx]), w[idx])
    tol = TOL[mode]
    assert rel(g["me0"][idx], o["me0"]).max() < tol
    assert rel(g["wnew"][0, idx], o["wnew"][0]).max() < tol
    exact = math.fsum(g["wnew"][0])
    assert abs(g["sigma"][0] - exact) <= 2 * np.spacing(exact)
    assert g["n_bad"] == 0


# --------------------------------------------------------------------------
# autotuner
# --------------------------------------------------------------------------
def test_autotune_keeps_parity_and_uses_its_cache(tmp_path):
    pts = ev.reweight_points("gg_tt_1m")
    mom, w, o = oracle_run("gg_tt", "gg_tt_1m", 5003, pts)
    dm, dw = to_dev(mom), to_dev(w)
    cache = str(tmp_path / "tune.jsonl")
    chosen = []
    for _ in range(2):
        with rwgt.Context(0, torch.cuda.current_stream().cuda_stream) as c:
            c.set_process("gg_tt", "fp64")
            c.set_params(ev.param_vector())
            c.set_reweight_points(pts)
            nb = c.workspace_bytes(5003)
            ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
            c.load_events(dm, dw, 5003, ws, nb)
            ms = c.autotune(max_events=1000, cache_path=cache)  # a sub-range of a longer batch
            assert ms > 0
            lb, bl = c.get_tuning()
            assert 0 <= lb <= 3 and bl in (64, 128, 256)
            chosen.append((lb, bl))
            wnew = torch.empty((1, 5003), dtype=torch.float64, device=DEV)
            c.reweight_async(wnew)
            sig, so, nbad, rc = c.get_results(1)
            assert rel(wnew.cpu().numpy(), o["wnew"]).max() < 1e-12
            assert abs(sig[0] / o["sigma"][0] - 1) < 1e-12
    assert chosen[0] == chosen[1]
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and '"lane_bits"' in lines[0]


# --------------------------------------------------------------------------
# mixed precision: FP32 amplitudes, tensor-core colour sum in FP16 / BF16
# --------------------------------------------------------------------------
def mixed_bound(mode, n_gluons):
    """Rounding J to p significant bits changes J^dagger C J by at most
    2 u sqrt(kappa(C)) relative (u = 2^-p, kappa the colour matrix's condition
    number), plus the FP32 amplitude error (1e-5)."""
    C, _ = oracle.colour_matrix(n_gluons)
    ev_ = np.linalg.eigvalsh(C)
    u = 2.0 ** -11 if mode == "mixed_fp16" else 2.0 ** -8
    return 2 * u * math.sqrt(ev_.max() / ev_.min()) + 1e-5


@pytest.mark.parametrize("mode", ["mixed_fp16", "mixed_bf16"])
@pytest.mark.parametrize("proc,wl,n,lbs,pts", [
    ("gg_tt", "gg_tt_1m", 5003, (0, 1), ev.reweight_points("gg_tt_1m")),
    ("gg_ttg", "gg_ttg_4m", 611, (0, 1, 2), ev.reweight_points("gg_ttg_4m", "mt")[::21]),
    ("gg_ttgg", "gg_ttgg_1m", 197, (1, 2, 3), ev.reweight_points("gg_ttgg_1m", "mt")),
])
def test_mixed_precision_colour_sum(mode, proc, wl, n, lbs, pts):
    mom, w, o = oracle_run(proc, wl, n, pts)
    b = mixed_bound(mode, ev.N_EXTERNAL[proc] - 2)
    for lb in lbs:
        g = run_gpu(proc, mode, mom, w, pts, lane_bits=lb)
        assert rel(g["me0"], o["me0"]).max() < b
        assert rel(g["me"], o["me"]).max() < b
        assert rel(g["ratio"], o["ratio"]).max() < 2 * b
        for j in range(len(g["sigma"])):
            exact_gpu = math.fsum(g["wnew"][j])
            assert abs(g["sigma"][j] - exact_gpu) <= 2 * np.spacing(exact_gpu)
            assert abs(g["sigma"][j] / o["sigma"][j] - 1) < 2 * b
        # the rounding is not systematic: the mean error is far below the bound
        assert rel(g["me0"], o["me0"]).mean() < b / 4


def test_host_entry_point_mixed_gg_ttgg_keeps_its_buffers():
    """The host-buffer entry point lays out its own buffers after the
    workspace's core, so a mixed mode of g g -> t tbar g g sums colours inside
    the amplitude kernel there (no separate pass writing over them): W' within
    the stated bound of the oracle over two chunks, sums within 2 ulp of the
    exact sums of the returned W', and within twice the bound of the device
    path, which takes the separate tensor-core pass."""
    pts = np.stack([ev.param_vector(m_t=0.9 * ev.M_TOP), ev.param_vector(m_t=1.2 * ev.M_TOP)])
    E = 3001
    mom, w, o = oracle_run("gg_ttgg", "gg_ttgg_1m", E, pts, start=9000)
    b = mixed_bound("mixed_bf16", 4)
    with rwgt.Context(0, torch.cuda.current_stream().cuda_stream) as c:
        c.set_process("gg_ttgg", "mixed_bf16")
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        c.set_tuning(3, 128)
        nb = c.workspace_bytes_host(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        hm, hwt = torch.from_numpy(mom).pin_memory(), torch.from_numpy(w).pin_memory()
        hw = torch.empty((2, E), dtype=torch.float64).pin_memory()
        sig, so, nbad, rc = c.reweight_host(hm, hwt, E, hw, 2, ws, nb)
    hw = hw.numpy()
    assert rc == 0 and nbad == 0
    assert rel(hw, o["wnew"]).max() < 2 * b
    for j in range(2):
        assert abs(sig[j] - math.fsum(hw[j])) <= 2 * np.spacing(sig[j])
    g = run_gpu("gg_ttgg", "mixed_bf16", mom, w, pts, lane_bits=3, block=128)
    assert rel(g["wnew"], hw).max() < 4 * b


@pytest.mark.parametrize("mode", ["mixed_fp16", "mixed_bf16"])
def test_separate_colour_pass_gg_ttgg(mode):
    """g g -> t tbar g g in a mixed mode with 4 or 8 lanes per event runs the
    amplitudes as in FP32 mode, stores the J vectors in 16 bits and sums
    colours in a separate tcgen05 pass: per event within the stated bound of
    the oracle for 1, 2 and 3 points, over 12 tiles with a ragged last one and
    grid-stride trips; unchanged parameters give r == 1 exactly; eval_me gives
    the reweight's |M|^2 bit for bit; and it agrees with the in-kernel
    tensor-core colour sum (2 lanes per event) within twice the bound."""
    pts = np.stack([ev.param_vector(m_t=k * ev.M_TOP) for k in (0.9, 1.1, 1.2)])
    mom, w, o = oracle_run("gg_ttgg", "gg_ttgg_1m", 1500, pts, start=3000)
    b = mixed_bound(mode, 4)
    fused = run_gpu("gg_ttgg", mode, mom, w, pts, lane_bits=1, block=128)
    for lb, block in ((2, 128), (3, 256), (3, 64)):
        g = run_gpu("gg_ttgg", mode, mom, w, pts, lane_bits=lb, block=block)
        assert rel(g["me0"], o["me0"]).max() < b
        assert rel(g["me"], o["me"]).max() < b
        assert rel(g["ratio"], o["ratio"]).max() < 2 * b
        assert rel(g["me0"], fused["me0"]).max() < 2 * b
        assert rel(g["me0"], o["me0"]).mean() < b / 4
        for j in range(3):
            exact_gpu = math.fsum(g["wnew"][j])
            assert abs(g["sigma"][j] - exact_gpu) <= 2 * np.spacing(exact_gpu)
            assert abs(g["sigma"][j] / o["sigma"][j] - 1) < 2 * b
        assert g["sigma_orig"] == pytest.approx(math.fsum(w), rel=1e-15)
    for P in (1, 2):
        g = run_gpu("gg_ttgg", mode, mom, w, pts[:P], lane_bits=3, block=128)
        assert rel(g["me"], o["me"][:P]).max() < b
    same = run_gpu("gg_ttgg", mode, mom, w, ev.param_vector()[None], lane_bits=3, block=128)
    assert np.all(same["ratio"] == 1.0)
    st = torch.cuda.current_stream(DEV).cuda_stream
    with rwgt.Context(0, st) as c:
        c.set_process("gg_ttgg", mode)
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        c.set_tuning(3, 128)
        E = mom.shape[-1]
        nb = c.workspace_bytes(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        c.load_events(to_dev(mom), to_dev(w), E, ws, nb)
        me = torch.empty(E, dtype=torch.float64, device=DEV)
        c.eval_me(-1, me)
        torch.cuda.synchronize()
    g = run_gpu("gg_ttgg", mode, mom, w, pts, lane_bits=3, block=128)
    assert np.array_equal(me.cpu().numpy(), g["me0"])


@pytest.mark.parametrize("block", [32, 256])
def test_mixed_modes_every_block_size(block):
    """Each warp's colour staging lives in the block's dynamic shared memory,
    so the tensor-core colour sum runs with any block size."""
    pts = POINT_SETS["gg_ttg_mt4"]()
    mom, w, o = oracle_run("gg_ttg", "gg_ttg_4m", 611, pts)
    b = mixed_bound("mixed_fp16", 3)
    g = run_gpu("gg_ttg", "mixed_fp16", mom, w, pts, lane_bits=1, block=block)
    assert rel(g["me0"], o["me0"]).max() < b and rel(g["me"], o["me"]).max() < b


def test_point_count_changes_on_one_context():
    """A kernel whose shared memory is far above the 48 KB default, launched on
    one context with 2 points, then 1, then 2 again: every launch runs (a
    kernel's shared-memory limit is only ever raised) and gives the same W' as
    a fresh context with that point set, bit for bit.  With 3 points the block
    (its static shared memory included) no longer fits: an argument error,
    after which the context still works."""
    wl = ev.WORKLOADS["gg_ttgg_1m"]
    E = 300
    mom, w = ev.generate(wl, E, start=777)
    sets = [np.stack([ev.param_vector(m_t=k * ev.M_TOP) for k in ks]) for ks in ((0.9, 1.2), (1.1,))]
    three = np.stack([ev.param_vector(m_t=k * ev.M_TOP) for k in (0.9, 1.1, 1.2)])
    dm, dw = to_dev(mom), to_dev(w)
    st = torch.cuda.current_stream(DEV).cuda_stream
    with rwgt.Context(0, st) as c:
        c.set_process("gg_ttgg", "fp32")
        c.set_params(ev.param_vector())
        c.set_reweight_points(three)  # the workspace sized for up to 3 points
        c.set_tuning(3, 256)  # 256 threads x (current store + constants): about 227 KB
        nb = c.workspace_bytes(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        c.load_events(dm, dw, E, ws, nb)
        for pts in (sets[0], sets[1], sets[0]):
            c.set_reweight_points(pts)
            wn = torch.empty((pts.shape[0], E), dtype=torch.float64, device=DEV)
            c.reweight_async(wn)
            torch.cuda.synchronize()
            ref = run_gpu("gg_ttgg", "fp32", mom, w, pts, lane_bits=3, block=256)
            assert np.array_equal(wn.cpu().numpy(), ref["wnew"])
        c.set_reweight_points(three)
        wn = torch.empty((3, E), dtype=torch.float64, device=DEV)
        with pytest.raises(rwgt.RwError) as x:
            c.reweight_async(wn)
        assert x.value.code == -2
        c.set_reweight_points(sets[1])
        wn = torch.empty((1, E), dtype=torch.float64, device=DEV)
        c.reweight_async(wn)
        torch.cuda.synchronize()
        assert np.array_equal(wn.cpu().numpy(), run_gpu("gg_ttgg", "fp32", mom, w, sets[1], lane_bits=3,
                                                         block=256)["wnew"])


def test_block_too_large_for_shared_memory_is_an_argument_error():
    """g g -> t tbar g g in a mixed mode keeps 936 bytes per thread in shared
    memory: a 256-thread block does not fit, and asking for one is an argument
    error that leaves the CUDA context clean (the next call and the autotuner's
    choice run normally)."""
    pts = POINT_SETS["gg_ttgg_mt"]()[:4]
    mom, w = ev.generate(ev.WORKLOADS["gg_ttgg_1m"], 64)
    with pytest.raises(rwgt.RwError) as x:
        run_gpu("gg_ttgg", "mixed_bf16", mom, w, pts, lane_bits=1, block=256)
    assert x.value.code == -2
    torch.cuda.synchronize()
    assert float(torch.ones(4, device=DEV).sum()) == 4.0
    g = run_gpu("gg_ttgg", "mixed_bf16", mom, w, pts, lane_bits=1, block=128)
    assert np.all(np.isfinite(g["me0"])) and g["n_bad"] == 0


# --------------------------------------------------------------------------
# CUDA-graph batching: several processes and point sets in one replay
# --------------------------------------------------------------------------
def test_graph_batches_processes_and_replays():
    side = torch.cuda.Stream(DEV)
    jobs = [("gg_tt", "fp64", "gg_tt_1m", 3001, ev.reweight_points("gg_tt_1m")),
            ("ee_mumu", "fp64", "ee_mumu_4k", 4096, ev.reweight_points("ee_mumu_4k")),
            ("gg_ttg", "fp32", "gg_ttg_4m", 500, ev.reweight_points("gg_ttg_4m", "mt")[::9])]
    ctxs, outs, refs, keep = [], [], [], []
    for proc, mode, wl, n, pts in jobs:
        mom, w, o = oracle_run(proc, wl, n, pts)
        dm, dw = to_dev(mom), to_dev(w)
        c = rwgt.Context(0, side.cuda_stream)
        c.set_process(proc, mode)
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        nb = c.workspace_bytes(n)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        c.load_events(dm, dw, n, ws, nb)
        out = torch.full((pts.shape[0], n), -1.0, dtype=torch.float64, device=DEV)
        ctxs.append(c)
        outs.append(out)
        refs.append((o, mode))
        keep += [dm, dw, ws]
    torch.cuda.synchronize()
    g = rwgt.Graph(side.cuda_stream)
    g.begin()
    for c, out in zip(ctxs, outs):
        c.reweight_async(out)
    g.end()
    for rep in range(2):
        for out in outs:
            out.fill_(-1.0)
        torch.cuda.synchronize()
        g.launch()
        side.synchronize()
        for c, out, (o, mode), job in zip(ctxs, outs, refs, jobs):
            assert rel(out.cpu().numpy(), o["wnew"]).max() < TOL[mode]
            sig, so, nbad, _ = c.get_results(job[4].shape[0])
            assert np.abs(sig / o["sigma"] - 1).max() < TOL[mode]
    g.close()
    for c in ctxs:
        c.close()
