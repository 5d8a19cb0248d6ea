"""Host-side checks of the Python binding: buffers are checked for element type,
contiguity and size before their addresses reach the library (which takes plain
pointers and cannot check them)."""
import numpy as np
import pytest

rwgt = pytest.importorskip("paper_2312_07440_gb300.rwgt")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("make", [np.zeros, lambda n, dtype: torch.zeros(n, dtype=getattr(torch, dtype))])
def test_buffer_checks(make):
    ok = make(12, dtype="float64")
    rwgt._check_buffer(ok, "x", 12)
    rwgt._check_buffer(None, "x", 12)      # optional outputs
    rwgt._check_buffer(12345, "x", 12)     # raw addresses pass through
    with pytest.raises(ValueError, match="float64"):
        rwgt._check_buffer(make(12, dtype="float32"), "x", 12)
    with pytest.raises(ValueError, match="at least 13"):
        rwgt._check_buffer(ok, "x", 13)
    strided = ok.reshape(3, 4)[:, ::2]
    with pytest.raises(ValueError, match="contiguous"):
        rwgt._check_buffer(strided, "x", 6)


def test_float32_and_int_buffers_named_in_the_message():
    with pytest.raises(ValueError, match="mom: expected float64 elements, got int64"):
        rwgt._check_buffer(np.zeros(4, dtype=np.int64), "mom", 4)


class _NoLibrary:
    """Stands in for the library: every call succeeds and does nothing, so the
    binding's own checks are what the test exercises (no GPU needed)."""

    def __getattr__(self, name):
        return lambda *args: 0

    def rw_last_error(self, h):
        return b""


def _context(process, n_points):
    c = object.__new__(rwgt.Context)
    c.h, c.lib = 1, _NoLibrary()
    c.n_external, c.n_points, c.n_events = rwgt.process_info(process).n_external, n_points, 0
    return c


@pytest.mark.parametrize("process,n_ext", [("gg_tt", 4), ("ee_5a", 7)])
def test_context_checks_event_and_output_buffers(process, n_ext):
    E, P = 100, 3
    c = _context(process, P)
    f64 = dict(dtype=torch.float64)
    mom, w = torch.zeros((n_ext, 4, E), **f64), torch.zeros(E, **f64)
    with pytest.raises(ValueError, match="mom"):
        c.load_events(mom.float(), w, E, None, 0)
    with pytest.raises(ValueError, match="mom"):
        c.load_events(mom[:, :, :E - 1].contiguous(), w, E, None, 0)
    with pytest.raises(ValueError, match="contiguous"):
        c.load_events(mom.transpose(0, 1), w, E, None, 0)
    c.load_events(mom, w, E, None, 0)
    assert c.n_events == E
    c.reweight_async(torch.zeros((P, E), **f64), None, torch.zeros(E, **f64))
    with pytest.raises(ValueError, match="wnew"):
        c.reweight_async(torch.zeros((P - 1, E), **f64))
    with pytest.raises(ValueError, match="out"):
        c.eval_me(0, torch.zeros(E - 1, **f64))
    with pytest.raises(ValueError, match="h_wnew"):
        c.reweight_host(mom.numpy(), w.numpy(), E, np.zeros((P, E), np.float32), P, None, 0)
    with pytest.raises(ValueError, match="d_fallback"):
        rwgt.reweight_interp(c, 5, 1e-4, torch.zeros((P, E), **f64), torch.zeros(E, dtype=torch.int32))
