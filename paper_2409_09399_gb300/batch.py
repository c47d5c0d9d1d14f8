"""Many cells in one launch (gint_batch_*) and the brick-shape autotuner.

The autotuner times the three calls (H^V, rho, force/stress) for each
candidate brick shape on a sample of the cells.  It ranks the shapes by total
time. Each cell of a batch then takes the best-ranked shape that the kernels of
its precision accept.  The start-up tile tuning of Section 2.3.3 is the model.
"""
from __future__ import annotations

import ctypes
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gint as _g

# the small shapes keep the densest cells (up to ~0.19 atoms per cubic angstrom, 63 atom images
# within the cutoff of a 2 x 2 x 4 brick) inside the tensor-core limits
CANDIDATE_BRICKS: Tuple[Tuple[int, int, int], ...] = ((8, 8, 8), (4, 8, 8), (4, 4, 8), (4, 4, 4), (3, 3, 4), (2, 2, 4),
                                                      (2, 2, 2))


def _timing_inputs(g, seed=0):
    """V and D for timing only: seeded uniform values of the right sizes (the kernels' work does not
    depend on the values), so the autotuner needs nothing from the caller's inputs."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    V = torch.rand(g.grid, dtype=torch.float64, device="cuda", generator=gen) - 0.5
    D = torch.rand(g.n_values, dtype=torch.float64, device="cuda", generator=gen) - 0.5
    return V, D


def _time_calls(g, V, D, reps=2):
    import torch
    g.vlocal(V); g.rho(D); g.force_stress(V, D)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        g.vlocal(V); g.rho(D); g.force_stress(V, D)
    torch.cuda.synchronize()
    g.sync()
    return (time.perf_counter() - t0) / reps


def autotune_brick(systems: Sequence, precision="fp16x3", candidates=CANDIDATE_BRICKS, sample=4, seed=0):
    """Rank candidate brick shapes by the time of vlocal + rho + force on a sample of the systems.

    Returns (ranking, table): ranking lists the shapes from fastest to slowest
    (shapes that some sampled system cannot take come last, by their time on
    the systems that take them), table maps shape -> {system index: seconds or None}.
    """
    rng = np.random.default_rng(seed)
    idx = [int(i) for i in rng.choice(len(systems), size=min(sample, len(systems)), replace=False)]
    table: Dict[tuple, Dict[int, Optional[float]]] = {}
    for brick in candidates:
        brick = tuple(brick)
        table[brick] = {}
        for i in idx:
            try:
                g = _g.from_system(systems[i], precision=precision, brick=brick)
            except _g.GintError:
                table[brick][i] = None  # the brick tables do not fit (setup rejects the shape)
                continue
            try:
                if not g.supported():
                    table[brick][i] = None
                    continue
                V, D = _timing_inputs(g)
                table[brick][i] = _time_calls(g, V, D)
            finally:
                g.close()
    return rank_shapes(table), table


def rank_shapes(table: Dict[tuple, Dict[int, Optional[float]]]) -> List[tuple]:
    """Shapes from fastest to slowest: first by how many sampled systems cannot take the
    shape (None), then by the summed time on the systems that can (ties keep table order)."""
    def key(b):
        t = table[b]
        missing = sum(v is None for v in t.values())
        return (missing, sum(v for v in t.values() if v is not None))
    return sorted(table, key=key)


def brick_for(system, precision, ranking) -> Tuple[int, int, int]:
    """The first shape of the ranking that the kernels of `precision` accept for `system`."""
    for brick in ranking:
        try:
            g = _g.from_system(system, precision=precision, brick=brick)
        except _g.GintError:
            continue
        ok = g.supported()
        g.close()
        if ok:
            return tuple(brick)
    raise _g.GintError(6, f"no candidate brick shape fits {system.name} in precision {precision}")


class GintBatch:
    """Handles for many cells and one CUDA-graph launch of all their calls.

    brick: one shape for every cell, a list with one shape per cell, or "auto"
    (autotune on a sample, then each cell takes the best shape it supports).
    """

    def __init__(self, systems: Sequence, precision="fp16x3", brick="auto", candidates=CANDIDATE_BRICKS,
                 sample=4):
        self.ranking = None
        if isinstance(brick, str):
            if brick != "auto":
                raise ValueError("brick must be a shape, a list of shapes or 'auto'")
            self.ranking, self.tuning = autotune_brick(systems, precision, candidates, sample)
            bricks = [brick_for(s, precision, self.ranking) for s in systems]
        elif len(brick) == 3 and all(isinstance(x, (int, np.integer)) for x in brick):
            bricks = [tuple(brick)] * len(systems)
        else:
            bricks = [tuple(b) for b in brick]
        self.bricks: List[tuple] = bricks
        self.handles = [_g.from_system(s, precision=precision, brick=b) for s, b in zip(systems, bricks)]
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
        """All cells' calls as one graph launch; each argument is a list of CUDA float64 tensors (or None)."""
        n = len(self.handles)

        def ptrs(lst, name, numel=None):
            if lst is None:
                return None
            if len(lst) != n:
                raise ValueError(f"{name}: need {n} tensors")
            out = (ctypes.c_void_p * n)()
            for i, t in enumerate(lst):
                if t is None:
                    continue
                if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
                    raise TypeError(f"{name}[{i}] must be a contiguous CUDA float64 tensor")
                if numel is not None and t.numel() < numel(i):
                    raise ValueError(f"{name}[{i}] holds {t.numel()} values, needs {numel(i)}")
                out[i] = t.data_ptr()
            return out

        h = self.handles
        args = [ptrs(V, "V", lambda i: h[i].n_grid), ptrs(D, "D", lambda i: h[i].n_values),
                ptrs(H, "H", lambda i: h[i].n_values), ptrs(rho, "rho", lambda i: h[i].n_grid),
                ptrs(F, "F", lambda i: 3 * h[i].n_atoms), ptrs(sigma, "sigma", lambda _: 9), ptrs(E, "E", lambda _: 1)]
        _g._check(_g.load().gint_batch_run(self._b, *args, _g.Gint._stream(stream)))
