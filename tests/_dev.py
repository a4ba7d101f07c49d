"""Device-buffer helpers for the GPU tests (torch is used only for memory)."""
import numpy as np


def torch_mod():
    import torch
    return torch


def upload(frame: np.ndarray, pitch_elems: int = None, offset_elems: int = 0):
    """Copy a (H, W) uint8/uint16 frame into a fresh device buffer with the
    given row pitch (in elements) and base offset. Returns (buffer, address,
    pitch_bytes); the buffer keeps the memory alive."""
    torch = torch_mod()
    H, W = frame.shape
    pitch_elems = W if pitch_elems is None else pitch_elems
    es = frame.itemsize
    host = np.zeros(offset_elems + H * pitch_elems + 64, dtype=frame.dtype)
    view = np.lib.stride_tricks.as_strided(host[offset_elems:], shape=(H, W),
                                           strides=(pitch_elems * es, es))
    view[...] = frame
    t = torch.from_numpy(host.view(np.uint8).copy()).cuda()
    return t, int(t.data_ptr()) + offset_elems * es, pitch_elems * es


def empty_like_frame(frame: np.ndarray, pitch_elems: int = None, offset_elems: int = 0, fill: int = 0xA5):
    torch = torch_mod()
    H, W = frame.shape
    pitch_elems = W if pitch_elems is None else pitch_elems
    es = frame.itemsize
    nbytes = (offset_elems + H * pitch_elems + 64) * es
    t = torch.full((nbytes,), fill, dtype=torch.uint8, device="cuda")
    return t, int(t.data_ptr()) + offset_elems * es, pitch_elems * es


def download(buf, addr: int, pitch_bytes: int, H: int, W: int, dtype) -> np.ndarray:
    torch = torch_mod()
    torch.cuda.synchronize()
    host = buf.cpu().numpy()
    base = addr - int(buf.data_ptr())
    es = np.dtype(dtype).itemsize
    out = np.empty((H, W), dtype=dtype)
    for y in range(H):
        row = host[base + y * pitch_bytes: base + y * pitch_bytes + W * es]
        out[y] = row.view(dtype)
    return out


def guard_bytes_intact(buf, addr: int, pitch_bytes: int, H: int, W: int, es: int, fill: int = 0xA5) -> bool:
    """Every byte of `buf` outside the frame's rows must still hold `fill`."""
    host = buf.cpu().numpy()
    mask = np.ones(host.size, dtype=bool)
    base = addr - int(buf.data_ptr())
    for y in range(H):
        s = base + y * pitch_bytes
        mask[s:s + W * es] = False
    return bool(np.all(host[mask] == fill))
