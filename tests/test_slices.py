"""Host-side plane output (paper_2505_20911_b300/slices.py): axis and index
conventions of the [5][N][N][N] layout (x fastest), the offset encoding's base
state added back, and the files written.  CPU only."""
import os

import numpy as np
import pytest
import torch

from paper_2505_20911_b300 import Config, slices


def _state(n, dtype):
    # q[c, z, y, x] = 1000 c + 100 z + 10 y + x (exact in FP32; FP16 rounds c >= 2)
    c, z, y, x = torch.meshgrid(*(torch.arange(s, dtype=torch.float64) for s in (5, n, n, n)),
                                indexing="ij")
    return (1000 * c + 100 * z + 10 * y + x).to(dtype)


def test_plane_axes_and_plain_encoding():
    n = 8
    cfg = Config(n=n, mode="fp32")
    q = _state(n, torch.float32)
    zp = slices.plane(cfg, q, "z", 3)
    yp = slices.plane(cfg, q, "y", 5)
    xp = slices.plane(cfg, q, "x", 6)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for c, f in enumerate(slices.FIELDS):
        assert zp[f].dtype == np.float64 and zp[f].shape == (n, n)
        np.testing.assert_array_equal(zp[f], 1000 * c + 100 * 3 + 10 * j + i)   # [y, x]
        np.testing.assert_array_equal(yp[f], 1000 * c + 100 * j + 10 * 5 + i)   # [z, x]
        np.testing.assert_array_equal(xp[f], 1000 * c + 100 * j + 10 * i + 6)   # [z, y]


def test_offset_encoding_adds_the_base_state_back():
    n = 8
    cfg = Config(n=n, mode="fp16_fp32", encoding="offset", mach=0.1, gamma=1.4)
    q = _state(n, torch.float16)
    p = slices.plane(cfg, q)  # the mid-plane z = N/2
    rho_e0 = 1.0 / (1.4 * 0.4 * 0.01)
    assert slices.encoding_offsets(cfg) == (1.0, pytest.approx(rho_e0, rel=1e-15))
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    base = 100 * (n // 2) + 10 * j + i
    np.testing.assert_array_equal(p["rho"], base + 1.0)
    np.testing.assert_array_equal(p["rho_u"], 1000 + base)
    # the stored FP16 value (rounded from 4000 + base), widened, plus the base state
    np.testing.assert_array_equal(p["rho_E"], q[4, n // 2].double().numpy() + rho_e0)


def test_save_midplane_slices(tmp_path):
    n = 8
    cfg = Config(n=n, mode="fp64")
    q = _state(n, torch.float64)
    paths = slices.save_midplane_slices(str(tmp_path), cfg, q, axes=("z", "x"),
                                        fields=("rho", "rho_E"), step=40)
    names = sorted(os.path.basename(p) for p in paths)
    assert names == ["rho_E_x4_s40.npy", "rho_E_z4_s40.npy", "rho_x4_s40.npy", "rho_z4_s40.npy"]
    a = np.load(os.path.join(str(tmp_path), "rho_E_z4_s40.npy"))
    np.testing.assert_array_equal(a, q[4, n // 2].numpy())


def test_plane_refuses_bad_arguments():
    cfg = Config(n=8, mode="fp32")
    q = _state(8, torch.float32)
    with pytest.raises(ValueError):
        slices.plane(cfg, q[:, :4])
    with pytest.raises(ValueError):
        slices.plane(cfg, q, "w")
    with pytest.raises(ValueError):
        slices.plane(cfg, q, "z", 8)
    with pytest.raises(ValueError):
        slices.plane(cfg, q, "z", 0, fields=("pressure",))
