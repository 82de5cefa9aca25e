"""Helpers for the GPU tests: move bit arrays to the device and read results
back as bit patterns.  Inputs always come from the seeded generators in
``paper_1605_05436_gb300.workloads``; expected values always come from the
oracle or from exact rationals."""
from __future__ import annotations

import numpy as np

F64, F32, BF16 = 0, 1, 2
NP_UNSIGNED = {F64: np.uint64, F32: np.uint32, BF16: np.uint16}
NP_SIGNED = {F64: np.int64, F32: np.int32, BF16: np.int16}


def torch_bits_dtype(dt):
    import torch
    return {F64: torch.int64, F32: torch.int32, BF16: torch.int16}[dt]


def to_device(bits: np.ndarray, dt: int, device="cuda:0", offset_elems: int = 0):
    """Copy a bit array to the device.  With offset_elems > 0 the returned
    tensor is a view starting that many elements into a larger buffer, so
    that the data pointer is not 16-byte aligned."""
    import torch
    a = np.ascontiguousarray(bits).view(NP_SIGNED[dt])
    if offset_elems:
        buf = torch.zeros(len(a) + offset_elems, dtype=torch_bits_dtype(dt), device=device)
        buf[offset_elems:] = torch.from_numpy(a).to(device)
        return buf[offset_elems:]
    return torch.from_numpy(a).to(device)


def result_bits(t, dt: int) -> list:
    """Bit patterns of a result tensor of format dt (float64/float32/bfloat16)."""
    import torch
    host = t.view(torch_bits_dtype(dt)).cpu().numpy()
    return [int(v) for v in host.view(NP_UNSIGNED[dt])]
