"""Several processes in one persistent launch, and a Born + real-emission
sample reweighted through it (the real-emission trees of an NLO sample as LO
processes of one more parton, Sec. 4).

Every process's W', r and sums are compared with the oracle per event (FP64
1e-12, re-evaluated in extended precision where the FP64 oracle's rounding
matters; FP32 1e-5); the sample's totals are the exact sums of both
processes' W'.  FKS subtraction counterterms are not specified by the paper
and are not part of the sample's weights here.
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
from parity_helpers import POINT_SETS, TOL, check_against_oracle  # noqa: E402

DEV = torch.device("cuda", 0)
# the points every process is reweighted to (the last one unchanged: r == 1)
POINTS = POINT_SETS["multi"]()
FP64_SET = {"gg_tt": "gg_tt_3001_multi", "gg_ttg": "gg_ttg_611_multi", "gg_ttgg": "gg_ttgg_197_multi"}
SAMPLES = {"gg_tt": ("gg_tt_1m", 3001), "gg_ttg": ("gg_ttg_4m", 611), "gg_ttgg": ("gg_ttgg_1m", 197)}


def prepared(proc, mode, stream, mom=None, w=None):
    if mom is None:
        wl, n = SAMPLES[proc]
        mom, w = ev.generate(ev.WORKLOADS[wl], n)
    E = mom.shape[-1]
    dm, dw = torch.from_numpy(np.ascontiguousarray(mom)).to(DEV), torch.from_numpy(np.ascontiguousarray(w)).to(DEV)
    c = rwgt.Context(0, stream)
    c.set_process(proc, mode)
    c.set_params(ev.param_vector())
    c.set_reweight_points(POINTS)
    nb = c.workspace_bytes(E)
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    c.load_events(dm, dw, E, ws, nb)
    wnew = torch.full((len(POINTS), E), -1.0, dtype=torch.float64, device=DEV)
    ratio = torch.full((len(POINTS), E), -1.0, dtype=torch.float64, device=DEV)
    return {"ctx": c, "keep": (dm, dw, ws), "wnew": wnew, "ratio": ratio, "mom": mom, "w": w, "proc": proc}


def check_item(it, mode):
    c, proc = it["ctx"], it["proc"]
    o = oracle.reweight(proc, ev.param_vector(), POINTS, it["mom"], it["w"])
    sig, so, nbad, _ = c.get_results(len(POINTS))
    g = {"wnew": it["wnew"].cpu().numpy(), "ratio": it["ratio"].cpu().numpy(), "sigma": sig, "sigma_orig": so,
         "n_bad": nbad}
    # the events are prefixes of each process's multi-point FP64 set
    check_against_oracle(g, o, mode, (proc, POINTS, it["mom"], it["w"]), FP64_SET[proc])
    assert np.all(g["ratio"][-1] == 1.0) and np.all(g["wnew"][-1] == it["w"])  # unchanged point, bitwise
    return g, o


@pytest.mark.parametrize("mode,procs", [("fp64", ("gg_tt", "gg_ttg")), ("fp32", ("gg_tt", "gg_ttg")),
                                        ("fp64", ("gg_tt", "gg_ttg", "gg_ttgg"))])
def test_one_launch_for_several_processes(mode, procs):
    stream = torch.cuda.current_stream(DEV).cuda_stream
    items = [prepared(p, mode, stream) for p in procs]
    with rwgt.Multi(0, stream) as m:
        for it in items:
            m.add(it["ctx"], it["wnew"], it["ratio"])
        nb = m.workspace_bytes()
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        m.reweight_async(ws, nb)
        tot, tot_orig, nbad, _ = m.get_results(len(POINTS))
    gs = [check_item(it, mode)[0] for it in items]
    for j in range(len(POINTS)):  # the sample's totals: exact sums over every process's W'
        exact = math.fsum(np.concatenate([g["wnew"][j] for g in gs]))
        assert abs(tot[j] - exact) <= 2 * np.spacing(exact)
    assert abs(tot_orig - math.fsum(np.concatenate([it["w"] for it in items]))) <= 2 * np.spacing(tot_orig)
    assert nbad == 0
    for it in items:
        it["ctx"].close()


def test_multi_launch_replays_in_a_cuda_graph():
    side = torch.cuda.Stream(DEV)
    items = [prepared(p, "fp64", side.cuda_stream) for p in ("gg_tt", "gg_ttg")]
    m = rwgt.Multi(0, side.cuda_stream)
    for it in items:
        m.add(it["ctx"], it["wnew"], it["ratio"])
    nb = m.workspace_bytes()
    ws = torch.zeros(nb, dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    g = rwgt.Graph(side.cuda_stream)
    g.begin()
    m.reweight_async(ws, nb)
    g.end()
    for _ in range(2):
        for it in items:
            it["wnew"].fill_(-1.0)
            it["ratio"].fill_(-1.0)
        torch.cuda.synchronize()
        g.launch()
        side.synchronize()
        for it in items:
            check_item(it, "fp64")
    g.close()
    m.close()
    for it in items:
        it["ctx"].close()


def test_multi_argument_errors():
    stream = torch.cuda.current_stream(DEV).cuda_stream
    a = prepared("gg_tt", "fp64", stream)
    b = prepared("gg_ttg", "fp32", stream)
    c = prepared("gg_tt", "fp64", stream)
    e = prepared("ee_mumu", "fp64", stream, *ev.generate(ev.WORKLOADS["ee_mumu_4k"], 64))
    with rwgt.Multi(0, stream) as m:
        m.add(a["ctx"], a["wnew"])
        with pytest.raises(rwgt.RwError) as x:
            m.add(b["ctx"], b["wnew"])
        assert x.value.code == -3  # modes differ
        with pytest.raises(rwgt.RwError) as x:
            m.add(c["ctx"], c["wnew"])
        assert x.value.code == -2  # the same process twice
        m.add(e["ctx"], e["wnew"])
        ws = torch.empty(m.workspace_bytes(), dtype=torch.uint8, device=DEV)
        with pytest.raises(rwgt.RwError) as x:
            m.reweight_async(ws, m.workspace_bytes())
        assert x.value.code == -3  # no kernel for this process set
    with rwgt.Multi(0, stream) as m:
        with pytest.raises(rwgt.RwError) as x:
            m.reweight_async(torch.empty(256, dtype=torch.uint8, device=DEV), 256)
        assert x.value.code == -6  # nothing added
    for it in (a, b, c, e):
        it["ctx"].close()


# --------------------------------------------------------------------------
# A Born + real-emission sample in one event file
# --------------------------------------------------------------------------
def _write_event_file(path, blocks_by_kind, kinds):
    it = {k: iter(v) for k, v in blocks_by_kind.items()}
    head = ('<LesHouchesEvents version="3.0">\n<header>\n</header>\n<init>\n2212 2212 6.5e3 6.5e3 0 0 0 0 3 1\n'
            '1.0 0.1 1.0 1\n</init>\n')
    path.write_text(head + "\n".join(next(it[k]) for k in kinds) + "\n</LesHouchesEvents>\n")


def _event_blocks(codes, mom, w):
    out = []
    N, _, E = mom.shape
    for e in range(E):
        lines = [f"{N} 1 {float(w[e])!r} 91.188 7.546771e-03 1.18e-01"]
        for i in range(N):
            st = -1 if i < 2 else 1
            px, py, pz, en = (float(mom[i, m, e]) for m in (1, 2, 3, 0))
            lines.append(f" {codes[i]} {st} 0 0 0 0 {px!r} {py!r} {pz!r} {en!r} 0.0 0. 9.")
        out.append("<event>\n" + "\n".join(lines) + "\n</event>")
    return out


def test_born_and_real_emission_sample_from_one_event_file(tmp_path):
    """An NLO-style sample: g g -> t tbar events (Born kinematics) and
    g g -> t tbar g events (real emission) interleaved in one file.  The file
    is classified by process, each process's events are read into its own
    batch, both are reweighted in one launch, and the new weights go back into
    the file in file order; each event's weight matches the oracle's for its
    own process, and the sample's cross section is the sum over both."""
    mb, wb = ev.generate(ev.WORKLOADS["gg_tt_1m"], 700)
    mr, wr = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 300)
    kinds = np.random.default_rng(5).permutation([0] * 700 + [1] * 300)
    src = tmp_path / "nlo.lhe"
    _write_event_file(src, {0: _event_blocks([21, 21, 6, -6], mb, wb),
                            1: _event_blocks([21, 21, 6, -6, 21], mr, wr)}, kinds)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    with rwgt.Lhe(src) as f:
        lab = f.classify(["gg_tt", "gg_ttg"])
        assert np.array_equal(lab, kinds)
        idx = [np.nonzero(lab == k)[0] for k in (0, 1)]
        batches = [f.read_list(p, i) for p, i in zip(("gg_tt", "gg_ttg"), idx)]
        items = [prepared(p, "fp64", stream, m, w) for p, (m, w) in zip(("gg_tt", "gg_ttg"), batches)]
        with rwgt.Multi(0, stream) as m:
            for it in items:
                m.add(it["ctx"], it["wnew"], it["ratio"])
            ws = torch.empty(m.workspace_bytes(), dtype=torch.uint8, device=DEV)
            m.reweight_async(ws, m.workspace_bytes())
            tot, tot_orig, nbad, _ = m.get_results(len(POINTS))
        wfile = np.empty((len(POINTS), len(f)))
        for it, i in zip(items, idx):
            wfile[:, i] = it["wnew"].cpu().numpy()
        ids = ["mt175_as120", "mt170", "as116", "same"]
        f.write(tmp_path / "out.lhe", wfile, ids)
    ref = np.empty_like(wfile)
    for it, i in zip(items, idx):
        g, o = check_item(it, "fp64")
        ref[:, i] = o["wnew"]
    assert nbad == 0
    for j in range(len(POINTS)):
        assert abs(tot[j] / math.fsum(ref[j]) - 1) < TOL["fp64"]
    assert abs(tot_orig - math.fsum(np.concatenate([wb, wr]))) <= 2 * np.spacing(tot_orig)
    # the written weights (shortest form that reads back as the same double),
    # event by event in file order: the kernel's W' exactly
    text = (tmp_path / "out.lhe").read_text()
    for j, name in enumerate(ids):
        vals = np.array([float(v) for v in re.findall(rf"<wgt id='{name}'>\s*(\S+)\s*</wgt>", text)])
        assert vals.shape == (len(kinds),)
        assert np.array_equal(vals, wfile[j])
    for it in items:
        it["ctx"].close()
