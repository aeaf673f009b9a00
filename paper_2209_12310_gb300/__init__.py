"""GB300 convex hull by GPU-heaphull filtering (arXiv 2209.12310), C ABI + binding.

The compute path is libconvhull.so (hand-written sm_103a CUDA behind the C
ABI of include/ch.h).  This package only marshals arguments: the ``ch_*``
functions take raw addresses exactly like the C functions, and the tensor
helpers below pass PyTorch-allocated device memory and the current CUDA
stream to them.  There is no CPU fallback.
"""
from __future__ import annotations

from ._native import (CH_EBUSY, CH_ECUDA, CH_EINVAL, CH_ENOMEM, CH_ERANGE, CH_ETIMEOUT, CH_OK,  # noqa: F401
                      CH_MAX_POINTS, CH_PENDING, CHError, LIB_PATH, ch_batched_config, ch_batched_counters, ch_filter, ch_filter16, ch_filter_manhattan, ch_hull,
                      ch_hull_batched, ch_hull_counters, ch_hull_host,
                      ch_poll, ch_profile_enable, ch_profile_read, ch_profile_reset, ch_release,
                      ch_reserve, ch_server_create, ch_server_destroy, ch_server_stats, ch_server_trace, ch_strerror,
                      ch_submit, ch_workspace_bytes, load, strerror)


def build(force: bool = False):
    from .build import build as _b
    return _b(force=force)


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _points(pts):
    import torch
    if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float32):
        raise TypeError("pts must be a CUDA float32 tensor of shape (n, 2)")
    if pts.dim() != 2 or pts.shape[1] != 2 or not pts.is_contiguous():
        raise ValueError("pts must be a contiguous (n, 2) tensor")
    return pts


def hull(pts, out_idx=None, out_n=None, stream=None, sync=True):
    """Hull of a (n, 2) CUDA float32 tensor.  Returns the int32 index tensor
    (counter-clockwise, from the lexicographically smallest vertex); with
    ``sync=False`` returns (out_idx, out_n) device tensors without waiting."""
    import torch
    pts = _points(pts)
    n = pts.shape[0]
    dev = pts.device
    if out_idx is None:
        out_idx = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if out_n is None:
        out_n = torch.empty(1, dtype=torch.int64, device=dev)
    ch_hull(pts.data_ptr(), n, out_idx.data_ptr(), out_n.data_ptr(), _stream(stream))
    if not sync:
        return out_idx, out_n
    h = int(out_n.item())
    if h < 0:
        raise CHError(h, "ch_hull")
    return out_idx[:h]


def hull_batched(pts, offsets, stream=None, sync=True):
    """k hulls of sets packed in ``pts`` with int64 ``offsets`` (k + 1).
    Returns a list of int32 index tensors (local indices)."""
    import torch
    pts = _points(pts)
    offsets_t = offsets if isinstance(offsets, torch.Tensor) else torch.as_tensor(offsets, dtype=torch.int64)
    host_off = offsets_t.to("cpu", torch.int64).contiguous()
    dev_off = offsets_t.to(pts.device, torch.int64).contiguous()
    k = host_off.numel() - 1
    total = int(host_off[-1])
    out_idx = torch.empty(max(total, 1), dtype=torch.int32, device=pts.device)
    out_n = torch.empty(max(k, 1), dtype=torch.int64, device=pts.device)
    ch_hull_batched(pts.data_ptr(), dev_off.data_ptr(), k, out_idx.data_ptr(), out_n.data_ptr(),
                    host_off.data_ptr(), _stream(stream))
    if not sync:
        return out_idx, out_n
    ns = out_n[:k].cpu().tolist()
    res = []
    for i in range(k):
        if ns[i] < 0:
            raise CHError(int(ns[i]), f"ch_hull_batched set {i}")
        o = int(host_off[i])
        res.append(out_idx[o:o + ns[i]])
    return res


def filter_labels(pts, labels=True, stream=None):
    """The paper's GPUfilter: (ext8 int32[8], labels uint8[n] or None, counts int64[4])."""
    import torch
    pts = _points(pts)
    n = pts.shape[0]
    ext = torch.empty(8, dtype=torch.int32, device=pts.device)
    lab = torch.empty(max(n, 1), dtype=torch.uint8, device=pts.device) if labels else None
    cnt = torch.empty(4, dtype=torch.int64, device=pts.device)
    ch_filter(pts.data_ptr(), n, ext.data_ptr(), lab.data_ptr() if lab is not None else None,
              cnt.data_ptr(), _stream(stream))
    return ext, (lab[:n] if lab is not None else None), cnt


def filter16_labels(pts, labels=True, stream=None):
    """The filter with the 16-direction polygon: (ext16 int32[16], labels
    uint8[n] or None, counts int64[4])."""
    import torch
    pts = _points(pts)
    n = pts.shape[0]
    ext = torch.empty(16, dtype=torch.int32, device=pts.device)
    lab = torch.empty(max(n, 1), dtype=torch.uint8, device=pts.device) if labels else None
    cnt = torch.empty(4, dtype=torch.int64, device=pts.device)
    ch_filter16(pts.data_ptr(), n, ext.data_ptr(), lab.data_ptr() if lab is not None else None,
                cnt.data_ptr(), _stream(stream))
    return ext, (lab[:n] if lab is not None else None), cnt
