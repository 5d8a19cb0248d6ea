"""The C ABI: the library builds for sm_103a, loads, and exports every entry
point include/rwgt.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w]+\**\s+\**(rw_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2312_07440_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("rw_create", "rw_destroy", "rw_set_process", "rw_set_params", "rw_set_reweight_points",
                 "rw_load_events", "rw_eval_me", "rw_reweight", "rw_reweight_async", "rw_get_results",
                 "rw_reweight_host", "rw_last_error", "rw_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_process_info_without_gpu():
    from paper_2312_07440_gb300 import rwgt
    from paper_2312_07440_gb300.gen import qcd_gen
    for name, ndiag in (("gg_tt", 3), ("gg_ttg", 16), ("gg_ttgg", 123)):
        info = rwgt.process_info(name)
        assert info.n_diagrams == ndiag == qcd_gen.diagram_count(info.n_external - 2)
        assert info.n_helicities == 2 ** info.n_external
        assert info.flops_hel_sum > 0
    info = rwgt.process_info("ee_mumu")
    assert (info.n_external, info.n_helicities, info.n_diagrams) == (4, 16, 2)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2312_07440_gb300 import rwgt
    with pytest.raises(rwgt.RwError):
        rwgt.Context(0)
