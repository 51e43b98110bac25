"""Host-side logic of the Python binding that needs no GPU: the row layout handed to the C ABI
(rows that overlap are refused, since the library would read past the tensor's storage) and
the choice of context (a call without an explicit context runs on the GPU that holds its data,
not on torch's current device: kernels of one GPU reading another GPU's memory would fault)."""
import types

import pytest

torch = pytest.importorskip("torch")

import paper_1204_5041_gb300 as isw  # noqa: E402


def test_rows_layout():
    t = torch.zeros(10, 7, dtype=torch.float64)
    assert isw._rows(t, 10, "t") == (7, 7)
    big = torch.zeros(10, 16, dtype=torch.float64)[:, :7]        # a column slice keeps ld = 16
    assert isw._rows(big, 10, "t") == (7, 16)
    assert isw._rows(torch.zeros(1, 5), 1, "t") == (5, 5)
    assert isw._rows(torch.zeros(10, 0), 10, "t") == (0, 1)


@pytest.mark.parametrize("make", [
    lambda: torch.zeros(1, 5, dtype=torch.float64).expand(10, 5),     # row stride 0
    lambda: torch.zeros(50, dtype=torch.float64).as_strided((10, 8), (4, 1)),   # rows overlap
])
def test_rows_refuse_overlapping_rows(make):
    with pytest.raises(ValueError, match="overlap"):
        isw._rows(make(), 10, "t")


def test_rows_refuse_bad_shapes():
    with pytest.raises(ValueError):
        isw._rows(torch.zeros(9, 5), 10, "t")
    with pytest.raises(ValueError):
        isw._rows(torch.zeros(5, 10).t(), 10, "t")                    # column-major


def test_default_context_follows_the_data(monkeypatch):
    asked = []
    monkeypatch.setattr(isw, "default_context", lambda device=None: asked.append(device) or f"ctx{device}")
    on_gpu1 = types.SimpleNamespace(is_cuda=True, device=torch.device("cuda", 1))
    assert isw._ctx(None, on_gpu1) == "ctx1"
    explicit = object()
    assert isw._ctx(explicit, on_gpu1) is explicit
    host = torch.zeros(3)
    assert isw._ctx(None, host) == "ctxNone"                         # no device tensor: current device
    assert asked == [1, None]
