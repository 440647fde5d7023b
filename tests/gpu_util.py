"""Helpers shared by the GPU tests: moving seeded numpy images to the device
and results back (no arithmetic of the method lives here)."""
import numpy as np
import pytest

try:
    import torch
except ImportError:     # pragma: no cover
    torch = None


def require_gpu():
    if torch is None or not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def to_device(img, pad_cols=0, offset_px=0):
    """Copy a uint8/uint16 numpy image to the GPU as a 2-D tensor view whose
    row pitch is (cols + pad_cols) pixels and whose first pixel sits
    offset_px pixels into its allocation (to exercise unaligned rows)."""
    r, c = img.shape
    pitch = c + pad_cols
    flat = np.zeros(r * pitch + offset_px + 16, dtype=img.dtype)
    view = flat[offset_px:offset_px + r * pitch].reshape(r, pitch)
    view[:, :c] = img
    if img.dtype == np.uint16:
        t = torch.from_numpy(flat.view(np.int16)).cuda()
    else:
        t = torch.from_numpy(flat).cuda()
    return t[offset_px:offset_px + r * pitch].view(r, pitch)[:, :c]


def u64(t):
    """A device tensor holding uint64 bit patterns -> numpy uint64 array."""
    if t.dtype != torch.int64:
        t = t.view(torch.int64)
    return t.cpu().numpy().view(np.uint64)


def f64(t):
    return t.cpu().numpy()
