"""Test helpers: move numpy arrays of unsigned keys to and from the GPU
bit for bit (through the signed torch dtype of the same width)."""
import numpy as np

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64, np.dtype(np.int32): np.int32,
           np.dtype(np.int64): np.int64}


def to_dev(a: np.ndarray, device="cuda"):
    import torch

    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(_SIGNED[a.dtype])).to(device)


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def assert_same(got: np.ndarray, want: np.ndarray, what: str = ""):
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        i = int(bad[0])
        raise AssertionError(f"{what}: {bad.size} of {want.size} differ; first at {i}: got {got[i]} want {want[i]}")
