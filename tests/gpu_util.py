"""Helpers for the GPU tests: move +/-1 planes between the host and device
planes of either layout (pure data movement)."""
import numpy as np
import torch

import paper_1908_07341_gb300 as shk


def to_device_plane(spins: np.ndarray, L: int, layout: str) -> torch.Tensor:
    plane = shk.alloc_plane(L, layout)
    plane.zero_()
    if layout == "bitpack":
        raw = shk.pack_bits(spins).view(np.uint8)
    else:
        raw = np.ascontiguousarray(spins, dtype=np.int8).view(np.uint8)
    plane[: raw.size].copy_(torch.from_numpy(raw.copy()))
    return plane


def from_device_plane(plane: torch.Tensor, L: int, layout: str) -> np.ndarray:
    raw = plane.cpu().numpy()
    if layout == "bitpack":
        return shk.unpack_bits(raw[: L * L // 8], L).reshape(-1)
    return raw[: L * L].view(np.int8).copy()
