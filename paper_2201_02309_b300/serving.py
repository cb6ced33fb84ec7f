"""Serving loop binding: torch host tensors in and out of the library's
continuous-batching server (``katsevich_server_*``).  Marshalling only: the
admission, plan cache, streams and all computation are in the C++/CUDA
library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import native
from .native import KATS_OK, KATS_PREC_FP32, KATS_ETIMEOUT, KatsevichError


def _torch():
    import torch
    return torch


@dataclass
class Ticket:
    """A submitted request; keeps its host buffers alive until it is waited for."""
    id: int
    sino: object
    vol: object
    geom: dict = field(repr=False)


class Server:
    """Reconstruction requests of any geometry, admitted by device memory.

    ``arena_bytes`` bounds the device memory of the running requests (view
    window + volume + workspace each), ``plan_cache_bytes`` the cached plans,
    ``slots`` the number of concurrent requests (one CUDA stream each).
    """

    def __init__(self, arena_bytes: int, plan_cache_bytes: int, slots: int = 4, max_bypass: int = 8):
        self.handle = native.katsevich_server_create(arena_bytes, plan_cache_bytes, slots, max_bypass)

    def submit(self, geom: dict, sino, vol=None, precision: int = KATS_PREC_FP32) -> Ticket:
        """Queue one reconstruction of ``sino`` [n_views][n_rows][n_cols] (float32 CPU
        tensor, page-locked for overlap); returns at once."""
        torch = _torch()
        shape = (geom["n_views"], geom["n_rows"], geom["n_cols"])
        if sino.dtype != torch.float32 or sino.is_cuda or not sino.is_contiguous() or tuple(sino.shape) != shape:
            raise ValueError(f"expected a contiguous float32 CPU tensor of shape {shape}")
        vshape = (geom["nz"], geom["ny"], geom["nx"])
        if vol is None:
            vol = torch.empty(vshape, dtype=torch.float32, pin_memory=sino.is_pinned())
        elif vol.dtype != torch.float32 or vol.is_cuda or not vol.is_contiguous() or tuple(vol.shape) != vshape:
            raise ValueError(f"expected a contiguous float32 CPU output of shape {vshape}")
        t = native.katsevich_server_submit(self.handle, geom, sino.data_ptr(), vol.data_ptr(), precision)
        return Ticket(t, sino, vol, geom)

    def wait(self, ticket: Ticket, timeout_ms: int = 600_000):
        """(volume, stats) of a finished request; raises KatsevichError with the
        request's status if it failed, or KATS_ETIMEOUT (ticket still valid)."""
        rc, stats, msg = native.katsevich_server_wait(self.handle, ticket.id, timeout_ms)
        if rc != KATS_OK:
            raise KatsevichError(rc, msg)
        return ticket.vol, stats

    def stats(self) -> dict:
        return native.katsevich_server_stats(self.handle)

    def close(self) -> None:
        if self.handle:
            native.katsevich_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "Ticket", "KATS_ETIMEOUT"]
