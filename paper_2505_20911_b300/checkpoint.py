"""Save and resume a run: the state Q, the step count, the simulated time and
the configuration (precision mode included) in one self-describing file.

Q alone determines the rest of a run: the RK increment is scratch that the
first stage of every step restarts (A_1 = 0 in the 2N scheme of Sec. 3.1,
Eqs. 3-4), so a run resumed from a saved Q continues bit for bit as if it had
never stopped.

File format (little-endian):
  8 bytes   magic b"TGVQ\\x00\\x01\\r\\n"
  8 bytes   length L of the header (unsigned)
  L bytes   UTF-8 JSON header: {"config": {...}, "step": int, "time": float,
            "shape": [5, N, N, N], "dtype": "float32", "bytes": int,
            "crc32": int}
  `bytes`   the state in the storage type, in the library's layout (x fastest)
The file is written to a temporary name next to the target and renamed into
place, so an interrupted save never leaves a truncated checkpoint under the
target name.
"""
from __future__ import annotations

import dataclasses
import json
import os
import struct
import zlib

import torch

MAGIC = b"TGVQ\x00\x01\r\n"
_DTYPES = {"float64": torch.float64, "float32": torch.float32, "bfloat16": torch.bfloat16,
           "float16": torch.float16}


class CheckpointError(RuntimeError):
    pass


def save_state(path: str, cfg, q: torch.Tensor, step: int, time: float = 0.0) -> None:
    """Write the state q (device or host tensor of cfg's storage type) with
    its configuration, step count and time to `path`."""
    from . import Config
    if not isinstance(cfg, Config):
        raise TypeError("cfg must be a Config")
    if q.dtype != cfg.q_dtype or tuple(q.shape) != (5, cfg.n, cfg.n, cfg.n):
        raise ValueError(f"q must be a (5, {cfg.n}, {cfg.n}, {cfg.n}) tensor of {cfg.q_dtype}")
    data = q.detach().contiguous().cpu().view(torch.uint8).numpy().tobytes()
    header = {"config": dataclasses.asdict(cfg), "step": int(step), "time": float(time),
              "shape": list(q.shape), "dtype": str(q.dtype).replace("torch.", ""),
              "bytes": len(data), "crc32": zlib.crc32(data)}
    hb = json.dumps(header, sort_keys=True).encode()
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as fh:
        fh.write(MAGIC)
        fh.write(struct.pack("<Q", len(hb)))
        fh.write(hb)
        fh.write(data)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)


def load_state(path: str, device="cuda"):
    """(cfg, q, step, time) from a file written by save_state; q is placed on
    `device`.  Raises CheckpointError on a wrong magic, a short file or a
    checksum mismatch."""
    from . import Config
    with open(path, "rb") as fh:
        if fh.read(len(MAGIC)) != MAGIC:
            raise CheckpointError(f"{path}: not a TGV state checkpoint")
        raw = fh.read(8)
        if len(raw) != 8:
            raise CheckpointError(f"{path}: truncated header")
        (hl,) = struct.unpack("<Q", raw)
        try:
            header = json.loads(fh.read(hl).decode())
        except (UnicodeDecodeError, json.JSONDecodeError) as exc:
            raise CheckpointError(f"{path}: unreadable header") from exc
        data = fh.read(header["bytes"])
    if len(data) != header["bytes"]:
        raise CheckpointError(f"{path}: truncated state ({len(data)} of {header['bytes']} bytes)")
    if zlib.crc32(data) != header["crc32"]:
        raise CheckpointError(f"{path}: checksum mismatch")
    cfg = Config(**header["config"])
    dtype = _DTYPES[header["dtype"]]
    if dtype != cfg.q_dtype:
        raise CheckpointError(f"{path}: state type {dtype} does not match mode {cfg.mode}")
    q = torch.frombuffer(bytearray(data), dtype=torch.uint8).view(dtype).reshape(header["shape"])
    return cfg, q.to(device), header["step"], header["time"]
