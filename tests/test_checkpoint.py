"""Checkpoint files (paper_2505_20911_b300.checkpoint): round trip of the
state, configuration, step and time; refusal of damaged files (host only)."""
import os

import pytest
import torch

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import checkpoint


@pytest.mark.parametrize("mode", ["fp64", "hpsp", "fp16_fp32", "bf16_fp32"])
def test_round_trip_is_exact(tmp_path, mode):
    cfg = tgv.Config(n=8, mode=mode, mach=0.2, re=800.0, split="kgp", encoding="offset")
    q = torch.randn(5, 8, 8, 8, dtype=torch.float64,
                    generator=torch.Generator().manual_seed(1)).to(cfg.q_dtype)
    path = os.path.join(tmp_path, "s.tgvq")
    checkpoint.save_state(path, cfg, q, step=1234, time=1.5425)
    cfg2, q2, step, t = checkpoint.load_state(path, device="cpu")
    assert cfg2 == cfg and step == 1234 and t == 1.5425
    assert q2.dtype == q.dtype and torch.equal(q2.view(torch.uint8), q.view(torch.uint8))
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]


def test_damaged_files_are_refused(tmp_path):
    cfg = tgv.Config(n=8, mode="fp32")
    q = torch.zeros(5, 8, 8, 8, dtype=torch.float32)
    path = os.path.join(tmp_path, "s.tgvq")
    checkpoint.save_state(path, cfg, q, step=3)
    blob = bytearray(open(path, "rb").read())
    blob[-1] ^= 0x40                                    # one flipped bit in the state
    open(path, "wb").write(bytes(blob))
    with pytest.raises(checkpoint.CheckpointError, match="checksum"):
        checkpoint.load_state(path, device="cpu")
    open(path, "wb").write(bytes(blob[:-10]))           # truncated
    with pytest.raises(checkpoint.CheckpointError, match="truncated"):
        checkpoint.load_state(path, device="cpu")
    open(path, "wb").write(b"not a checkpoint")
    with pytest.raises(checkpoint.CheckpointError, match="not a TGV"):
        checkpoint.load_state(path, device="cpu")


def test_wrong_state_type_is_refused_on_save(tmp_path):
    cfg = tgv.Config(n=8, mode="fp16_fp32")
    with pytest.raises(ValueError):
        checkpoint.save_state(os.path.join(tmp_path, "s"), cfg, torch.zeros(5, 8, 8, 8), 0)
