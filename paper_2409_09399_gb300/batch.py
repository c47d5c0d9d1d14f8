"""Many cells in one launch (gint_batch_*) and a brick-shape autotuner.

The autotuner times the three calls of candidate brick shapes on a sample of
cells (each candidate set up on each sampled cell; shapes the tensor-core
path cannot take are skipped) and keeps the shape with the least total time,
in the spirit of the paper's start-up tile autotuning (Section 2.3.3).
"""
from __future__ import annotations

import ctypes
import time
from typing import Sequence

import numpy as np

from . import gint as _g

CANDIDATE_BRICKS = ((8, 8, 8), (8, 8, 4), (4, 8, 8), (4, 4, 8), (4, 4, 4), (3, 3, 4))


def _time_calls(h, V, D, reps=1):
    import torch
    h.vlocal(V); h.rho(D); h.force_stress(V, D)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        h.vlocal(V); h.rho(D); h.force_stress(V, D)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def autotune_brick(systems: Sequence, precision="fp16x3", candidates=CANDIDATE_BRICKS, sample=6, seed=0):
    """Brick shape with the least vlocal + rho + force time over a sample of the systems.

    Returns (brick, {brick: seconds or None}) -- None where the shape is not supported.
    """
    import torch

    import synth
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(systems), size=min(sample, len(systems)), replace=False)
    times = {}
    for brick in candidates:
        tot = 0.0
        ok = True
        for i in idx:
            s = systems[int(i)]
            try:
                h = _g.from_system(s, precision=precision, brick=brick)
                V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
                bl, off = h.pattern()
                D = synth.d_fill_torch(bl, off[:-1], h.n_values, s.pos, s.cell, s.nw(), "cuda")
                tot += _time_calls(h, V, D)
                h.sync()
                h.close()
            except _g.GintError:
                ok = False
                break
        times[brick] = tot if ok else None
    best = min((t, b) for b, t in times.items() if t is not None)[1]
    return best, times


class GintBatch:
    """Handles for many cells and one graph launch of all their calls."""

    def __init__(self, systems: Sequence, precision="fp16x3", brick=(8, 8, 8)):
        self.handles = [_g.from_system(s, precision=precision, brick=brick) for s in systems]
        L = _g.load()
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        out = ctypes.c_void_p()
        _g._check(L.gint_batch_create(len(self.handles), arr, ctypes.byref(out)))
        self._b = out

    def close(self):
        if getattr(self, "_b", None):
            _g.load().gint_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, V, D, H=None, rho=None, F=None, sigma=None, E=None, stream=None):
        """Run every cell's calls as one graph launch; arguments are lists of CUDA tensors (or None)."""
        n = len(self.handles)

        def ptrs(lst):
            if lst is None:
                return None
            return (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in lst])

        _g._check(_g.load().gint_batch_run(self._b, ptrs(V), ptrs(D), ptrs(H), ptrs(rho), ptrs(F), ptrs(sigma),
                                           ptrs(E), _g.Gint._stream(stream)))
