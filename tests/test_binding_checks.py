"""The Python binding checks the type, size and device of every tensor before its address goes to the
library, so that a mismatched buffer raises ValueError instead of reaching a kernel (CPU only: a fake
context stands in for the library's shape queries)."""
import numpy as np
import pytest
import torch

from paper_1401_7494_gb300 import rct

L, W, H = 8, 16, 12


@pytest.fixture
def fake_ctx(monkeypatch):
    state = {"dtype": rct.RCT_PROJ_F32, "slab": (0, L)}
    monkeypatch.setattr(rct, "rct_get_shape", lambda ctx: (L, W, H, 4))
    monkeypatch.setattr(rct, "rct_get_slab", lambda ctx: state["slab"])
    monkeypatch.setattr(rct, "rct_get_precision", lambda ctx: (state["dtype"], rct.RCT_INTERP_SOFT))

    def never(*a, **k):
        raise AssertionError("the library was called with a buffer the binding should have refused")
    monkeypatch.setattr(rct, "lib", never)
    return state


def test_device_projections_must_be_cuda_tensors(fake_ctx):
    with pytest.raises(ValueError, match="CUDA tensor"):
        rct.rct_backproject(1, torch.zeros(4 * H * W), 0, 4)
    with pytest.raises(ValueError, match="CUDA tensor"):
        rct.rct_backproject(1, np.zeros(4 * H * W, np.float32), 0, 4)


def test_host_projections_must_match_dtype_and_size(fake_ctx):
    with pytest.raises(ValueError, match="dtype"):
        rct.rct_backproject_host(1, torch.zeros(4 * H * W, dtype=torch.float16), 0, 4)
    with pytest.raises(ValueError, match="elements"):
        rct.rct_backproject_host(1, torch.zeros(3 * H * W), 0, 4)
    fake_ctx["dtype"] = rct.RCT_PROJ_F16
    with pytest.raises(ValueError, match="dtype"):
        rct.rct_backproject_host(1, torch.zeros(4 * H * W), 0, 4)
    with pytest.raises(ValueError, match="dtype"):
        rct.rct_backproject_host(1, np.zeros(4 * H * W, np.float32), 0, 4)


def test_volume_buffers_must_hold_the_context_planes(fake_ctx):
    with pytest.raises(ValueError, match="elements"):
        rct.rct_read_volume(1, torch.zeros(L ** 3 - 1))
    with pytest.raises(ValueError, match="dtype"):
        rct.rct_write_volume(1, torch.zeros(L ** 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="dtype"):
        rct.rct_read_volume(1, np.zeros(L ** 3, np.float64))
    fake_ctx["slab"] = (0, 3)                       # a slab context holds 3 planes
    with pytest.raises(ValueError, match="elements"):
        rct.rct_read_volume(1, torch.zeros(3 * L * L - 1))
    with pytest.raises(ValueError, match="elements"):
        rct.rct_backproject_host_read(1, torch.zeros(4 * H * W), 0, 4, torch.zeros(2 * L * L))


def test_conversion_and_filter_buffers(fake_ctx):
    with pytest.raises(ValueError):
        rct.rct_convert_projections(torch.zeros(10), torch.zeros(10, dtype=torch.float16), 10, rct.RCT_PROJ_F16)
    with pytest.raises(ValueError):
        rct.rct_filter_projections(1, torch.zeros(4 * H * W), torch.zeros(4 * H * W), rct.RCT_PROJ_F32, 0, 4)


def test_noalloc_entry_point_checks_its_buffers(monkeypatch):
    monkeypatch.setattr(rct, "lib", lambda: (_ for _ in ()).throw(AssertionError("library called")))
    m, o, s = np.zeros((1, 3, 4)), np.zeros(3), np.ones(3)
    with pytest.raises(ValueError, match="CUDA tensor"):
        rct.rct_backproject_f16_noalloc(L, W, H, m, o, s, torch.zeros(H * W), 1, torch.zeros(L ** 3))
    with pytest.raises(ValueError):
        rct.rct_backproject_f16_noalloc(L, W, H, m, o, s, torch.zeros(H * W, dtype=torch.float16), 1,
                                        torch.zeros(L ** 3))


def test_raw_addresses_pass_through_unchecked():
    rct._check_buffer(12345, "x", code=rct.RCT_PROJ_F32, min_elems=10 ** 9, where="device")
    rct._check_buffer(None, "x", code=rct.RCT_PROJ_F32, min_elems=10 ** 9, where="device")
