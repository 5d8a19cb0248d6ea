"""Les Houches Event files through the library's reader and writer (host
only): round trip of momenta and weights from a lab-frame file with shuffled
particle order, intermediate lines and existing weight blocks; the weights
written back; error reporting."""
import math
import os
import re

import numpy as np
import pytest

from paper_2312_07440_gb300 import events as ev

rwgt = pytest.importorskip("paper_2312_07440_gb300.rwgt")
try:
    rwgt.load()
except (RuntimeError, OSError) as e:  # the library is built by __graft_entry__.build()
    pytest.skip(f"library not built: {e}", allow_module_level=True)

PDG = {"gg_tt": [21, 21, 6, -6], "gg_ttg": [21, 21, 6, -6, 21], "ee_5a": [11, -11, 22, 22, 22, 22, 22]}


def boost_z(p, beta):
    g = 1.0 / math.sqrt(1.0 - beta * beta)
    q = p.copy()
    q[..., 0] = g * (p[..., 0] + beta * p[..., 3])
    q[..., 3] = g * (p[..., 3] + beta * p[..., 0])
    return q


def write_lhe(path, process, mom, w, beta=0.3, extra=True):
    """A minimal LHE 3.0 file: lab frame (boost beta along z), outgoing
    particles before incoming ones and antiparticles first, an intermediate
    resonance line, a comment and, every third event, an existing <rwgt>."""
    codes = PDG[process]
    N, _, E = mom.shape
    out = ['<LesHouchesEvents version="3.0">', "<header>", "<!-- synthetic -->", "</header>", "<init>",
           "2212 2212 6.5e3 6.5e3 0 0 0 0 3 1", "1.0 0.1 1.0 1", "</init>"]
    order = list(range(2, N))[::-1] + [1, 0]
    # identical particles keep their relative order (the reader matches in file order)
    order = sorted(order, key=lambda i: (codes[i], i)) if process != "gg_tt" else [3, 2, 0, 1]
    for e in range(E):
        p = boost_z(mom[:, :, e], beta)
        lines = [f"{N + (1 if extra else 0)} 1 {float(w[e])!r} 91.1880000e+00 7.546771e-03 1.180000e-01"]
        if extra:
            lines.append(" 23 2 1 2 0 0 0.0 0.0 0.0 91.1876 91.1876 0. 0.")
        for i in order:
            st = -1 if i < 2 else 1
            px, py, pz, en = (float(p[i, m]) for m in (1, 2, 3, 0))
            lines.append(f" {codes[i]} {st} 0 0 0 0 {px!r} {py!r} {pz!r} {en!r} 0.0 0. 9.")
        if extra:
            lines.append("# a comment line")
        if extra and e % 3 == 0:
            lines += ["<rwgt>", "<wgt id='old'> 1.0 </wgt>", "</rwgt>"]
        out += ["<event>"] + lines + ["</event>"]
    out.append("</LesHouchesEvents>")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


@pytest.mark.parametrize("process,wl", [("gg_ttg", "gg_ttg_4m"), ("ee_5a", "ee_5a_1m"), ("gg_tt", "gg_tt_1m")])
def test_read_round_trip(tmp_path, process, wl):
    mom, w = ev.generate(ev.WORKLOADS[wl], 2500)
    path = tmp_path / "in.lhe"
    write_lhe(path, process, mom, w)
    with rwgt.Lhe(path) as f:
        assert len(f) == 2500
        m1, w1 = f.read(process, threads=1)
        m4, w4 = f.read(process, threads=4)
        m_part, w_part = f.read(process, first=100, n=50)
    assert np.array_equal(m1, m4) and np.array_equal(w1, w4)
    assert np.array_equal(w1, w)  # the weight text is exact
    # back in the centre-of-mass frame: the boost there and back costs a few ulp
    scale = mom[0, 0][None, None, :]
    assert np.abs(m1 - mom).max() <= 1e-13 * scale.max()
    assert np.array_equal(m_part, m1[:, :, 100:150]) and np.array_equal(w_part, w1[100:150])


def test_write_new_weights(tmp_path):
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 300)
    src, dst = tmp_path / "in.lhe", tmp_path / "out.lhe"
    write_lhe(src, "gg_tt", mom, w)
    rng = np.random.default_rng(4)
    wnew = rng.lognormal(size=(3, 300))
    with rwgt.Lhe(src) as f:
        f.write(dst, wnew, ["mt175", "as120", "both"])
    text = dst.read_text()
    # every event carries its three new weights, in order, after any old ones
    blocks = re.findall(r"<event>(.*?)</event>", text, re.S)
    assert len(blocks) == 300
    for k, b in enumerate(blocks):
        vals = re.findall(r"<wgt id='(\w+)'> (\S+) </wgt>", b)
        names = [n for n, _ in vals if n != "old"]
        assert names == ["mt175", "as120", "both"]
        got = [float(v) for n, v in vals if n != "old"]
        assert np.allclose(got, wnew[:, k], rtol=1e-10, atol=0)
        assert b.count("<rwgt>") == 1
    # removing the added lines (and the blocks created for them) gives the input back
    stripped = re.sub(r"<wgt id='(mt175|as120|both)'> \S+ </wgt>\n", "", text)
    stripped = stripped.replace("<rwgt>\n</rwgt>\n", "")
    assert stripped == src.read_text()
    # and the written file reads back to the same events
    with rwgt.Lhe(dst) as g:
        m2, w2 = g.read("gg_tt")
    with rwgt.Lhe(src) as f:
        m1, w1 = f.read("gg_tt")
    assert np.array_equal(m1, m2) and np.array_equal(w1, w2)


def test_errors(tmp_path):
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 10)
    path = tmp_path / "in.lhe"
    write_lhe(path, "gg_tt", mom, w)
    with pytest.raises(rwgt.RwError):
        rwgt.Lhe(tmp_path / "missing.lhe")
    with rwgt.Lhe(path) as f:
        with pytest.raises(rwgt.RwError, match="event 0"):
            f.read("ee_5a")
        with pytest.raises(rwgt.RwError):
            f.read("gg_tt", first=5, n=6)
        with pytest.raises(rwgt.RwError):
            f.write(tmp_path / "o.lhe", np.ones((1, 10)), ["bad'id"])
    bad = path.read_text().replace(f"{float(w[3])!r}", "bad-number", 1)
    (tmp_path / "bad.lhe").write_text(bad)
    with rwgt.Lhe(tmp_path / "bad.lhe") as f:
        with pytest.raises(rwgt.RwError, match="event 3"):
            f.read("gg_tt", threads=1)
    (tmp_path / "open.lhe").write_text("<LesHouchesEvents>\n<event>\n1 1 1.0 0 0 0\n")
    with pytest.raises(rwgt.RwError):
        rwgt.Lhe(tmp_path / "open.lhe")


def test_write_needs_one_id_per_row(tmp_path):
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 20)
    path = tmp_path / "in.lhe"
    write_lhe(path, "gg_tt", mom, w)
    with rwgt.Lhe(path) as f:
        with pytest.raises(ValueError):
            f.write(tmp_path / "o.lhe", np.ones((2, 20)), ["only_one"])


def test_fortran_d_exponents(tmp_path):
    """Fortran writers may print 1.2345678901D+02: read exactly as the E form."""
    mom, w = ev.generate(ev.WORKLOADS["gg_ttg_4m"], 40)
    path_e, path_d = tmp_path / "e.lhe", tmp_path / "d.lhe"
    write_lhe(path_e, "gg_ttg", mom, w)
    text = path_e.read_text()
    # re-print every float of the event blocks in Fortran E/D form
    head, rest = text.split("<event>", 1)

    def fortran(m):
        x = float(m.group(0))
        return f"{x:.15E}"

    body = re.sub(r"-?\d+\.\d+(?:e[+-]?\d+)?", fortran, "<event>" + rest)
    path_e.write_text(head + body)
    path_d.write_text(head + body.replace("E+", "D+").replace("E-", "d-"))
    with rwgt.Lhe(path_e) as f:
        m_e, w_e = f.read("gg_ttg")
    with rwgt.Lhe(path_d) as f:
        m_d, w_d = f.read("gg_ttg")
    assert np.array_equal(m_e, m_d) and np.array_equal(w_e, w_d)
    bad = head + body.replace("E+", "D", 1).replace("D", "D ", 1)
    (tmp_path / "bad.lhe").write_text(bad)
    with rwgt.Lhe(tmp_path / "bad.lhe") as f:
        with pytest.raises(rwgt.RwError, match="event 0"):
            f.read("gg_ttg", threads=1)


def test_gzip_files(tmp_path):
    """.lhe.gz in and out: the same events and weights as the plain file."""
    import gzip
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 50)
    plain, packed = tmp_path / "in.lhe", tmp_path / "in.lhe.gz"
    write_lhe(plain, "gg_tt", mom, w)
    packed.write_bytes(gzip.compress(plain.read_bytes()))
    with rwgt.Lhe(plain) as f:
        m1, w1 = f.read("gg_tt")
        wnew = np.vstack([w1 * 1.5])
        f.write(tmp_path / "out.lhe", wnew, ["x"])
    with rwgt.Lhe(packed) as f:
        assert f._tmp is None  # the decompressed copy is gone once the text is in memory
        m2, w2 = f.read("gg_tt")
        f.write(tmp_path / "out.lhe.gz", wnew, ["x"])
    assert np.array_equal(m1, m2) and np.array_equal(w1, w2)
    assert gzip.decompress((tmp_path / "out.lhe.gz").read_bytes()) == (tmp_path / "out.lhe").read_bytes()


def test_event_attributes_extra_tags_and_comments(tmp_path):
    """<event> attributes, <mgrwt>/<scales> blocks after the particle lines and
    "<event>" inside header comments leave the events and weights unchanged."""
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 30)
    plain, fancy = tmp_path / "a.lhe", tmp_path / "b.lhe"
    write_lhe(plain, "gg_tt", mom, w)
    t = plain.read_text()
    t = t.replace("<event>", '<event npLO=" -1 " npNLO=" 1 ">')
    t = t.replace("</event>", "<mgrwt>\n<rscale> 0 0.1E+03 </rscale>\n</mgrwt>\n"
                              "<scales pt_clust_1=\"0.1E+03\"></scales>\n</event>")
    t = t.replace("<header>", "<header>\n<!-- an <event> mentioned in a comment -->\n<!-- and </event> -->")
    t = t.replace("</init>", "</init>\n<!-- <event> between init and events -->")
    fancy.write_text(t)
    with rwgt.Lhe(plain) as f:
        m1, w1 = f.read("gg_tt")
    with rwgt.Lhe(fancy) as f:
        assert len(f) == 30
        m2, w2 = f.read("gg_tt")
        f.write(tmp_path / "c.lhe", np.vstack([w2]), ["same"])
    assert np.array_equal(m1, m2) and np.array_equal(w1, w2)
    with rwgt.Lhe(tmp_path / "c.lhe") as g:
        m3, w3 = g.read("gg_tt")
    assert np.array_equal(m3, m2) and np.array_equal(w3, w2)


def test_write_without_weight_blocks_is_linear(tmp_path):
    """Events without an <rwgt> block get one; the search for it stays inside
    each event (it once ran ahead through the rest of the file: quadratic)."""
    import time
    E = 20000
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], E)
    src, dst = tmp_path / "in.lhe", tmp_path / "out.lhe"
    write_lhe(src, "gg_tt", mom, w, extra=False)
    with rwgt.Lhe(src) as f:
        t0 = time.perf_counter()
        f.write(dst, np.vstack([w * 2.0]), ["twice"])
        dt = time.perf_counter() - t0
    assert dt < 2.0  # ~10 ms linear, ~5 s quadratic
    text = dst.read_text()
    assert text.count("<rwgt>") == E and text.count("<wgt id='twice'>") == E


def test_unclosed_comment_is_an_error(tmp_path):
    """A comment that is never closed hides every event after it: the file is
    rejected instead of being read short."""
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 10)
    path = tmp_path / "in.lhe"
    write_lhe(path, "gg_tt", mom, w)
    t = path.read_text()
    cut = [m.end() for m in re.finditer("</event>", t)][3]
    (tmp_path / "oops.lhe").write_text(t[:cut] + "\n<!-- oops\n" + t[cut:])
    with pytest.raises(rwgt.RwError, match="not closed"):
        rwgt.Lhe(tmp_path / "oops.lhe")


def test_end_tag_inside_a_comment_of_an_event(tmp_path):
    """'</event>' inside a comment of an event block does not end the block:
    the event is read whole and the new weights go before the real end tag."""
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 6)
    plain, tricky = tmp_path / "a.lhe", tmp_path / "b.lhe"
    write_lhe(plain, "gg_tt", mom, w, extra=False)
    t = plain.read_text().replace("</event>", "<!-- a </event> in a comment -->\n</event>")
    tricky.write_text(t)
    with rwgt.Lhe(plain) as f:
        m1, w1 = f.read("gg_tt")
    with rwgt.Lhe(tricky) as f:
        assert len(f) == 6
        m2, w2 = f.read("gg_tt")
        f.write(tmp_path / "c.lhe", np.vstack([2 * w2]), ["twice"])
    assert np.array_equal(m1, m2) and np.array_equal(w1, w2)
    out = (tmp_path / "c.lhe").read_text()
    for blk in re.findall(r"<event>(.*?)\n</event>", out, flags=re.S):
        assert blk.index("<!-- a </event> in a comment -->") < blk.index("<rwgt>")
        assert blk.rstrip().endswith("</rwgt>")


def test_many_comments_index_in_linear_time(tmp_path):
    """Many comments between two events, and inside one event, are skipped in
    one pass (each used to restart the search for the next tag)."""
    import time
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], 4)
    path = tmp_path / "in.lhe"
    write_lhe(path, "gg_tt", mom, w, extra=False)
    t = path.read_text()
    many = "<!-- c -->\n" * 100000
    k = t.index("</event>") + len("</event>")
    t = t[:k] + "\n" + many + t[k:]
    k = t.rindex("</event>")
    t = t[:k] + many + t[k:]
    (tmp_path / "many.lhe").write_text(t)
    t0 = time.perf_counter()
    with rwgt.Lhe(tmp_path / "many.lhe") as f:
        assert len(f) == 4
        m2, w2 = f.read("gg_tt")
    assert time.perf_counter() - t0 < 2.0  # ~10 ms linear, minutes quadratic
    assert np.array_equal(w2, w)


def mixed_file(tmp_path, n_born=40, n_real=25):
    """An event file whose events come from two processes, interleaved as in
    an NLO sample (g g -> t tbar Born-like events and g g -> t tbar g
    real-emission events)."""
    mb, wb = ev.generate(ev.WORKLOADS["gg_tt_1m"], n_born)
    mr, wr = ev.generate(ev.WORKLOADS["gg_ttg_4m"], n_real)
    write_lhe(tmp_path / "b.lhe", "gg_tt", mb, wb)
    write_lhe(tmp_path / "r.lhe", "gg_ttg", mr, wr)
    tb, tr = (tmp_path / "b.lhe").read_text(), (tmp_path / "r.lhe").read_text()
    blocks_b = re.findall(r"<event>.*?</event>", tb, flags=re.S)
    blocks_r = re.findall(r"<event>.*?</event>", tr, flags=re.S)
    rng = np.random.default_rng(3)
    kinds = rng.permutation([0] * n_born + [1] * n_real)
    it = {0: iter(blocks_b), 1: iter(blocks_r)}
    body = "\n".join(next(it[k]) for k in kinds)
    head = tb[:tb.index("<event>")]
    (tmp_path / "mixed.lhe").write_text(head + body + "\n</LesHouchesEvents>\n")
    return tmp_path / "mixed.lhe", kinds, (mb, wb), (mr, wr)


def test_mixed_process_file_is_classified_and_read_by_lists(tmp_path):
    path, kinds, (mb, wb), (mr, wr) = mixed_file(tmp_path)
    with rwgt.Lhe(path) as f:
        lab = f.classify(["gg_tt", "gg_ttg"])
        assert np.array_equal(lab, kinds)
        assert np.all(f.classify(["ee_5a"]) == -1)
        m1, w1 = f.read_list("gg_tt", np.nonzero(lab == 0)[0])
        m2, w2 = f.read_list("gg_ttg", np.nonzero(lab == 1)[0])
        # reversed order of the list: the columns follow the list
        m3, w3 = f.read_list("gg_ttg", np.nonzero(lab == 1)[0][::-1])
        with pytest.raises(rwgt.RwError, match="outside"):
            f.read_list("gg_tt", [len(f)])
        with pytest.raises(rwgt.RwError, match="extra external particles"):
            f.read_list("gg_tt", np.nonzero(lab == 1)[0][:1])
    assert np.array_equal(w1, wb) and np.array_equal(w2, wr) and np.array_equal(w3, wr[::-1])
    # the lab-frame boost back to the centre-of-mass frame: the same momenta to rounding
    assert np.allclose(m1, mb, rtol=0, atol=1e-9) and np.allclose(m2, mr, rtol=0, atol=1e-9)
    assert np.array_equal(m3, m2[:, :, ::-1])
