"""Test helpers: tensor <-> numpy views with the ABI's key types."""
import numpy as np
import torch

NP_KEY = {"u32": np.uint32, "i32": np.int32, "u64": np.uint64, "f32": np.float32}


def to_np(t: torch.Tensor, kt: str | None = None) -> np.ndarray:
    """Host numpy copy; int32 tensors viewed as uint32 for u32 keys and payloads."""
    a = t.detach().cpu().numpy()
    if kt is not None:
        return a.view(NP_KEY[kt]) if a.dtype.itemsize == np.dtype(NP_KEY[kt]).itemsize else a.astype(NP_KEY[kt])
    return a


def vals_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def first_mismatch(x: np.ndarray, y: np.ndarray):
    bad = np.nonzero(x != y)[0]
    return None if len(bad) == 0 else int(bad[0])
