"""PyTorch plumbing around the C ABI: a device arena and a context handle.

PyTorch owns the device memory (one uint8 tensor, the arena that libscl
sub-allocates) and supplies streams; every computation goes through
``scl``'s C entry points.
"""
from __future__ import annotations

import torch

from . import scl


class Context:
    """One libscl context over a torch-allocated arena on ``device``."""

    def __init__(self, arena_bytes: int, device: int = 0, hbm_budget_bytes: int = 0,
                 inflight_batches: int = 4, tune_cache_path: str | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libscl needs a CUDA device")
        self.device = device
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda:%d" % device)
        self.handle = scl.scl_create(device, self.arena.data_ptr(), self.arena.numel(),
                                     hbm_budget_bytes, inflight_batches, tune_cache_path)

    def close(self) -> None:
        if self.handle:
            torch.cuda.synchronize(self.device)
            scl.scl_destroy(self.handle)
            self.handle = 0
        self.arena = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def current_stream(device: int = 0) -> int:
    """cudaStream_t of torch's current stream on ``device``."""
    return torch.cuda.current_stream(device).cuda_stream
