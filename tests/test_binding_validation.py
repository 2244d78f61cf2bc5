"""The Python binding refuses a buffer whose dtype, size, layout or device
does not match what the library will read or write, before any library call
(a mismatched buffer would otherwise be read or written out of bounds by the
kernels).  Runs on the CPU with stand-in CUDA tensors and a library guard
that fails the test if any device entry point is reached."""
import pytest
import torch

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import _abi

HOST_ONLY = {"tgv_state_bytes", "tgv_qt_bytes", "tgv_workspace_bytes", "tgv_check_config",
             "tgv_adjoint_workspace_bytes", "tgv_grad_workspace_bytes", "tgv_dt_max",
             "tgv_run_host_workspace_bytes", "tgv_run_host_stream_workspace_bytes",
             "tgv_strerror", "tgv_abi_version"}


class FakeCuda:
    """Looks like a contiguous CUDA tensor to the binding's checks."""

    def __init__(self, shape, dtype, index=0, contiguous=True):
        self.shape, self.dtype, self.index, self.contig = tuple(shape), dtype, index, contiguous
        self.is_cuda = True
        self.device = torch.device("cuda", index)

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def element_size(self):
        return torch.tensor([], dtype=self.dtype).element_size()

    def is_contiguous(self):
        return self.contig

    def data_ptr(self):
        return 1 << 20


class Guard:
    def __init__(self, real):
        self.real = real

    def __getattr__(self, name):
        if name in HOST_ONLY:
            return getattr(self.real, name)
        raise AssertionError(f"device entry point {name} reached with an invalid buffer")


@pytest.fixture
def guarded(monkeypatch):
    real = _abi.lib()
    monkeypatch.setattr(_abi, "_lib", Guard(real))
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(tgv, "_stream", lambda s: None)
    yield


N = 16


def state(cfg, dtype=None, fields=5, **kw):
    return FakeCuda((fields, N, N, N), dtype or cfg.q_dtype, **kw)


def test_wrong_dtype_is_refused(guarded):
    c64 = tgv.Config(n=N, mode="fp64")
    with pytest.raises(ValueError, match="expected torch.float64"):
        tgv.tgv_init(c64, state(c64, torch.float32))
    with pytest.raises(ValueError, match="q_b"):
        tgv.rk_step(c64, state(c64), state(c64, torch.float32), state(c64), 0.004, 1)
    c16 = tgv.Config(n=N, mode="hpsp")
    with pytest.raises(ValueError, match="qt"):
        tgv.rk_substep(c16, state(c16), state(c16), state(c16, torch.float32), 0, 0.004)
    with pytest.raises(ValueError, match="r:"):
        tgv.rhs_eval(c16, state(c16), state(c16, torch.float16))


def test_short_buffers_are_refused(guarded):
    c = tgv.Config(n=N, mode="fp32")
    short = FakeCuda((5, N, N, N - 1), torch.float32)
    with pytest.raises(ValueError, match="bytes"):
        tgv.tgv_init(c, short)
    with pytest.raises(ValueError, match="diag"):
        tgv.rk_step(c, state(c), state(c), state(c), 0.004, 20, 10,
                    FakeCuda((2, tgv.TGV_DIAG_COUNT), torch.float64),
                    FakeCuda((tgv.tgv_workspace_bytes(c),), torch.uint8))
    with pytest.raises(ValueError, match="out"):
        tgv.diagnostics_reduce_noalloc(c, state(c), FakeCuda((9,), torch.float64))
    with pytest.raises(ValueError, match="out"):
        tgv.diagnostics_reduce(c, state(c), FakeCuda((4,), torch.float64),
                               FakeCuda((1 << 20,), torch.uint8))


def test_adjoint_buffers_are_checked(guarded):
    c = tgv.Config(n=N, mode="fp64")
    with pytest.raises(ValueError, match="grad_mom"):
        tgv.tgv_grad_final_ke(c, state(c), 0.004, 4, 2, FakeCuda((2, N, N, N), torch.float64),
                              FakeCuda((1,), torch.float64), FakeCuda((1 << 24,), torch.uint8))
    with pytest.raises(ValueError, match="stage_inputs"):
        tgv.rk_step_adjoint(c, FakeCuda((2, 5, N, N, N), torch.float64), state(c), 0.004,
                            FakeCuda((1 << 24,), torch.uint8))
    with pytest.raises(ValueError, match="lam"):
        tgv.rhs_vjp(c, state(c), state(c, torch.float32), state(c),
                    FakeCuda((1 << 24,), torch.uint8))


def test_other_device_and_layout_are_refused(guarded):
    c = tgv.Config(n=N, mode="fp32")
    with pytest.raises(ValueError, match="cuda:1"):
        tgv.tgv_init(c, state(c, index=1))
    with pytest.raises(ValueError, match="contiguous"):
        tgv.tgv_init(c, state(c, contiguous=False))
    with pytest.raises(ValueError, match="CUDA tensor"):
        tgv.tgv_init(c, torch.empty(5, N, N, N))


def test_host_buffers_are_checked(guarded):
    c = tgv.Config(n=N, mode="fp16_fp32")
    good = torch.empty(5, N, N, N, dtype=torch.float16)
    ws = FakeCuda((tgv.tgv_run_host_workspace_bytes(c, 2, 1),), torch.uint8)
    with pytest.raises(ValueError, match="q_host_out"):
        tgv.tgv_run_host(c, good, torch.empty(5, N, N, N, dtype=torch.float32), 0.004, 2, 1,
                         None, ws)
    with pytest.raises(ValueError, match="diag_host"):
        tgv.tgv_run_host(c, good, good, 0.004, 2, 1, torch.empty(2, tgv.TGV_DIAG_COUNT,
                                                                 dtype=torch.float64), ws)
    with pytest.raises(ValueError, match=r"q_host_in\[1\]"):
        tgv.tgv_run_host_stream(c, [good, good[:, :1]], [good, good], 0.004, 2, 0, None, ws,
                                None, object())
