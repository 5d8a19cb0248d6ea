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
