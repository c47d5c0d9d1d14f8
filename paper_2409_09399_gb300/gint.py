"""Thin ctypes binding of libgint (the C ABI declared in include/gint.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libgint.so.  Torch provides device memory and streams.  There is
no CPU fallback: if libgint.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

GINT_FP64, GINT_FP32, GINT_TF32, GINT_BF16X3, GINT_BF16X6, GINT_FP16X3, GINT_FP16X4 = range(7)
PRECISIONS = {"fp64": GINT_FP64, "fp32": GINT_FP32, "tf32": GINT_TF32, "bf16x3": GINT_BF16X3,
              "bf16x6": GINT_BF16X6, "fp16x3": GINT_FP16X3, "fp16x4": GINT_FP16X4}
STATUS = {0: "GINT_OK", 1: "GINT_ERR_INVALID_ARG", 2: "GINT_ERR_CUDA", 3: "GINT_ERR_OOM",
          4: "GINT_ERR_PATTERN_MISMATCH", 5: "GINT_ERR_TIMEOUT", 6: "GINT_ERR_UNSUPPORTED", 7: "GINT_ERR_DEVICE"}

# exported symbols, in the order include/gint.h declares them
SYMBOLS = ["gint_setup", "gint_destroy", "gint_pattern", "gint_set_precision", "gint_vlocal", "gint_rho",
           "gint_force_stress", "gint_energy_grads", "gint_update_positions", "gint_select_bricks", "gint_brick_loads",
           "gint_set_wait_limit", "gint_debug_fail_alloc", "gint_local_potential", "gint_vlocal_static", "gint_fold_k", "gint_check",
           "gint_batch_create", "gint_batch_run", "gint_batch_destroy", "gint_sync", "gint_get_info",
           "gint_work_stats", "gint_last_error"]


class GintError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Radial(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("n_knots", ctypes.c_int), ("dr", ctypes.c_double),
                ("y", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double))]


class _Species(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_double), ("n_radial", ctypes.c_int), ("radial", ctypes.POINTER(_Radial))]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("brick", ctypes.c_int * 3), ("device", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class _Info(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int64), ("n_values", ctypes.c_int64), ("n_ext_atoms", ctypes.c_int64),
                ("n_bricks", ctypes.c_int64), ("n_bricks_nonempty", ctypes.c_int64),
                ("n_brick_atoms", ctypes.c_int64), ("n_brick_pairs", ctypes.c_int64),
                ("max_brick_atoms", ctypes.c_int), ("max_brick_orbitals", ctypes.c_int),
                ("brick", ctypes.c_int * 3), ("precision", ctypes.c_int), ("scratch_bytes", ctypes.c_int64),
                ("n_orbitals", ctypes.c_int64)]


_lib = None


def load(build: bool = True) -> ctypes.CDLL:
    """Load libgint.so (building it first if needed).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise OSError(f"libgint.so not found at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.gint_setup.restype = i32
    L.gint_setup.argtypes = [i32, vp, vp, vp, i32, ctypes.POINTER(_Species), vp, ctypes.POINTER(_Options),
                             ctypes.POINTER(vp)]
    L.gint_destroy.restype = None
    L.gint_destroy.argtypes = [vp]
    L.gint_pattern.restype = i32
    L.gint_pattern.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.gint_set_precision.restype = i32
    L.gint_set_precision.argtypes = [vp, i32]
    L.gint_vlocal.restype = i32
    L.gint_vlocal.argtypes = [vp, vp, vp, i32, vp]
    L.gint_rho.restype = i32
    L.gint_rho.argtypes = [vp, vp, vp, vp]
    L.gint_force_stress.restype = i32
    L.gint_force_stress.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.gint_energy_grads.restype = i32
    L.gint_energy_grads.argtypes = [vp] * 10
    L.gint_update_positions.restype = i32
    L.gint_update_positions.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32)]
    L.gint_select_bricks.restype = i32
    L.gint_select_bricks.argtypes = [vp, i64, vp]
    L.gint_brick_loads.restype = i32
    L.gint_brick_loads.argtypes = [vp, vp]
    L.gint_set_wait_limit.restype = i32
    L.gint_set_wait_limit.argtypes = [vp, i64]
    L.gint_debug_fail_alloc.restype = i32
    L.gint_debug_fail_alloc.argtypes = [i32]
    L.gint_local_potential.restype = i32
    L.gint_local_potential.argtypes = [vp] * 7
    L.gint_vlocal_static.restype = i32
    L.gint_vlocal_static.argtypes = [vp, vp, vp, vp]
    L.gint_fold_k.restype = i32
    L.gint_fold_k.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double * 3), vp, i64, vp]
    L.gint_check.restype = i32
    L.gint_check.argtypes = [vp]
    L.gint_batch_create.restype = i32
    L.gint_batch_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.gint_batch_run.restype = i32
    L.gint_batch_run.argtypes = [vp] + [ctypes.POINTER(vp)] * 7 + [vp]
    L.gint_batch_destroy.restype = None
    L.gint_batch_destroy.argtypes = [vp]
    L.gint_sync.restype = i32
    L.gint_sync.argtypes = [vp, vp]
    L.gint_get_info.restype = i32
    L.gint_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.gint_work_stats.restype = i32
    L.gint_work_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.gint_last_error.restype = ctypes.c_char_p
    L.gint_last_error.argtypes = []
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        msg = load().gint_last_error().decode(errors="replace")
        raise GintError(status, msg)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


class _DevArray:
    """__cuda_array_interface__ view of memory owned by a handle."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}
        self._owner = owner


class Gint:
    """One geometry on one GPU: pattern, bricks, tables (gint_setup)."""

    def __init__(self, pos, species_index, cell, species: Sequence, grid, precision="fp64",
                 brick=(0, 0, 0), device: int = -1):
        L = load()
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        spi = np.ascontiguousarray(species_index, dtype=np.int32)
        cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
        grid = np.ascontiguousarray(grid, dtype=np.int32).reshape(3)
        self.n_atoms = pos.shape[0]
        self.grid = tuple(int(x) for x in grid)
        self.n_grid = self.grid[0] * self.grid[1] * self.grid[2]
        self.pos = pos.copy()
        self.cell = cell.reshape(3, 3).copy()
        self.omega = float(abs(np.linalg.det(self.cell)))
        self.dV = self.omega / float(self.grid[0] * self.grid[1] * self.grid[2])
        keep = []
        sps = (_Species * len(species))()
        for s, S in enumerate(species):
            rads = (_Radial * len(S.radials))()
            for j, R in enumerate(S.radials):
                y = np.ascontiguousarray(R.y, dtype=np.float64)
                dy = np.ascontiguousarray(R.dy, dtype=np.float64)
                keep += [y, dy]
                rads[j].l = int(R.l)
                rads[j].n_knots = int(y.size)
                rads[j].dr = float(R.dr)
                rads[j].y = y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                rads[j].dy = dy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            keep.append(rads)
            sps[s].rc = float(S.rc)
            sps[s].n_radial = len(S.radials)
            sps[s].radial = rads
        opt = _Options()
        opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        for i in range(3):
            opt.brick[i] = int(brick[i])
        opt.device = int(device)
        h = ctypes.c_void_p()
        _check(L.gint_setup(self.n_atoms, pos.ctypes.data, spi.ctypes.data, cell.ctypes.data, len(species), sps,
                            grid.ctypes.data, ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.nw = np.array([species[s].n_orb for s in spi], dtype=np.int64)
        nb, nv = ctypes.c_int64(), ctypes.c_int64()
        _check(L.gint_pattern(self._h, ctypes.byref(nb), ctypes.byref(nv), None, None))
        self.n_blocks, self.n_values = nb.value, nv.value
        self.n_orbitals = int(self.nw.sum())
        self._pattern = None

    # -------------------------------------------------------------- basics
    def close(self):
        if getattr(self, "_h", None):
            load().gint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(load().gint_set_precision(self._h, p))

    def fold_k(self, H, kfrac, Hk=None, stream=None):
        """Bloch sum H(k) = sum_t exp(2 pi i kfrac . t) H(t): dense complex128 CUDA tensor (N, N)."""
        import torch
        self._need(H, self.n_values, "H")
        n = self.n_orbitals
        if Hk is None:
            Hk = torch.empty((n, n), dtype=torch.complex128, device=H.device)
        if not (Hk.is_cuda and Hk.dtype == torch.complex128 and Hk.dim() == 2 and Hk.shape[0] >= n
                and Hk.shape[1] >= n and Hk.stride(1) == 1):
            raise TypeError("Hk must be a row-major complex128 CUDA matrix of at least n_orbitals x n_orbitals")
        k = (ctypes.c_double * 3)(*[float(x) for x in kfrac])
        _check(load().gint_fold_k(self._h, _ptr(H), ctypes.byref(k), Hk.data_ptr(), Hk.stride(0),
                                  self._stream(stream)))
        return Hk

    def update_positions(self, pos, cell=None, keep_pattern: bool = False) -> bool:
        """New positions (bohr) and optionally a new cell for this handle (gint_update_positions).

        Returns True if the pair pattern changed (then D and H must be laid out anew).  With
        keep_pattern the pattern must stay the same, else GintError (GINT_ERR_PATTERN_MISMATCH)
        and the handle keeps its old geometry."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n_atoms, 3)
        c = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
        changed = ctypes.c_int(0)
        _check(load().gint_update_positions(self._h, pos.ctypes.data, None if c is None else c.ctypes.data,
                                            1 if keep_pattern else 0, ctypes.byref(changed)))
        self.pos = pos.copy()
        if c is not None:
            self.cell = c.reshape(3, 3).copy()
            self.omega = float(abs(np.linalg.det(self.cell)))
            self.dV = self.omega / float(self.n_grid)
        nb, nv = ctypes.c_int64(), ctypes.c_int64()
        _check(load().gint_pattern(self._h, ctypes.byref(nb), ctypes.byref(nv), None, None))
        self.n_blocks, self.n_values = nb.value, nv.value
        self._pattern = None
        return bool(changed.value)

    def select_bricks(self, bricks=None):
        """Restrict later calls to the bricks with the given ids (None: every brick)."""
        if bricks is None:
            _check(load().gint_select_bricks(self._h, 0, None))
            return
        b = np.ascontiguousarray(bricks, dtype=np.int64).reshape(-1)
        _check(load().gint_select_bricks(self._h, b.size, b.ctypes.data))

    def brick_loads(self) -> np.ndarray:
        """Atom images meeting each brick (int64, one entry per brick)."""
        out = np.zeros(int(self.info()["n_bricks"]), dtype=np.int64)
        _check(load().gint_brick_loads(self._h, out.ctypes.data))
        return out

    def set_wait_limit(self, polls: int = 0):
        _check(load().gint_set_wait_limit(self._h, int(polls)))

    def energy_grads(self, V, D, grad_E=None, want=("R", "eps", "V", "D", "E"), stream=None):
        """Gradients of E = sum V rho dV (gint_energy_grads): dict with the requested entries of
        R: dE/dR (n, 3), eps: dE/d(strain) (3, 3), V: dE/dV (grid), D: dE/dD (n_values), E: (1,).
        grad_E: optional device scalar multiplying every gradient."""
        import torch
        self._need(V, self.n_grid, "V")
        self._need(D, self.n_values, "D")
        dev = V.device
        f64 = torch.float64
        out = {}
        if "R" in want:
            out["R"] = torch.empty((self.n_atoms, 3), dtype=f64, device=dev)
        if "eps" in want:
            out["eps"] = torch.empty((3, 3), dtype=f64, device=dev)
        if "V" in want:
            out["V"] = torch.empty(self.grid, dtype=f64, device=dev)
        if "D" in want:
            out["D"] = torch.empty(self.n_values, dtype=f64, device=dev)
        if "E" in want:
            out["E"] = torch.empty(1, dtype=f64, device=dev)
        if grad_E is not None:
            grad_E = grad_E.to(device=dev, dtype=f64).reshape(1).contiguous()
        _check(load().gint_energy_grads(self._h, _ptr(V), _ptr(D), _ptr(grad_E), _ptr(out.get("R")),
                                        _ptr(out.get("eps")), _ptr(out.get("V")), _ptr(out.get("D")),
                                        _ptr(out.get("E")), self._stream(stream)))
        return out

    def local_potential(self, rho, V_ext=None, V_out=None, want_vh=False, stream=None):
        """(V_out, V_H or None, energies (2,) = (E_H, E_xc)): V_out = V_ext + V_H + v_xc from rho."""
        import torch
        self._need(rho, self.n_grid, "rho")
        if V_ext is not None:
            self._need(V_ext, self.n_grid, "V_ext")
        if V_out is None:
            V_out = torch.empty(self.grid, dtype=torch.float64, device=rho.device)
        self._need(V_out, self.n_grid, "V_out")
        vh = torch.empty(self.grid, dtype=torch.float64, device=rho.device) if want_vh else None
        en = torch.empty(2, dtype=torch.float64, device=rho.device)
        _check(load().gint_local_potential(self._h, _ptr(rho), _ptr(V_ext), _ptr(V_out), _ptr(vh), _ptr(en),
                                           self._stream(stream)))
        return V_out, vh, en

    def supported(self) -> bool:
        """Whether the kernels of the current precision accept this handle's bricks."""
        st = load().gint_check(self._h)
        if st == 0:
            return True
        if st == 6:  # GINT_ERR_UNSUPPORTED
            return False
        _check(st)

    def info(self) -> dict:
        inf = _Info()
        _check(load().gint_get_info(self._h, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in _Info._fields_}
        d["brick"] = tuple(inf.brick)
        return d

    def work_stats(self):
        """(sum_r n_o(r), sum_r n_o(r)^2) over all grid points (exact orbital counts)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().gint_work_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def pattern(self):
        """(blocks int64 (n_blocks, 5) numpy, offsets int64 (n_blocks+1,) numpy), copied from the device."""
        if self._pattern is None:
            import torch
            L = load()
            bp, op = ctypes.c_void_p(), ctypes.c_void_p()
            _check(L.gint_pattern(self._h, None, None, ctypes.byref(bp), ctypes.byref(op)))
            nb = self.n_blocks
            if nb == 0:
                self._pattern = (np.zeros((0, 5), np.int64), np.zeros(1, np.int64))
            else:
                b = torch.as_tensor(_DevArray(bp.value, (nb, 5), "<i4", self), device="cuda")
                o = torch.as_tensor(_DevArray(op.value, (nb + 1,), "<i8", self), device="cuda")
                self._pattern = (b.cpu().numpy().astype(np.int64), o.cpu().numpy().copy())
        return self._pattern

    def sync(self, stream=None):
        _check(load().gint_sync(self._h, self._stream(stream)))

    @staticmethod
    def _stream(stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return ctypes.c_void_p(int(stream.cuda_stream))

    @staticmethod
    def _need(t, numel, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        if t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")

    # --------------------------------------------------------------- calls
    def vlocal(self, V, H=None, accumulate: bool = False, stream=None):
        """H^V on the pattern (Eq. 2); returns the float64 CUDA tensor H."""
        import torch
        ng = self.grid[0] * self.grid[1] * self.grid[2]
        self._need(V, ng, "V")
        if H is None:
            H = torch.empty(self.n_values, dtype=torch.float64, device=V.device)
        self._need(H, self.n_values, "H")
        _check(load().gint_vlocal(self._h, _ptr(V), _ptr(H), 1 if accumulate else 0, self._stream(stream)))
        return H

    def rho(self, D, rho=None, stream=None):
        """Density on the grid (Eq. 3); returns a (n1, n2, n3) float64 CUDA tensor."""
        import torch
        self._need(D, self.n_values, "D")
        if rho is None:
            rho = torch.empty(self.grid, dtype=torch.float64, device=D.device)
        self._need(rho, self.grid[0] * self.grid[1] * self.grid[2], "rho")
        _check(load().gint_rho(self._h, _ptr(D), _ptr(rho), self._stream(stream)))
        return rho

    def force_stress(self, V, D, out=None, stream=None):
        """(F (n,3), sigma (3,3), virial per atom (n,3,3), E (1,)) as float64 CUDA tensors (Eq. 4, 5)."""
        import torch
        ng = self.grid[0] * self.grid[1] * self.grid[2]
        self._need(V, ng, "V")
        self._need(D, self.n_values, "D")
        if out is None:
            dev = V.device
            out = (torch.empty((self.n_atoms, 3), dtype=torch.float64, device=dev),
                   torch.empty((3, 3), dtype=torch.float64, device=dev),
                   torch.empty((self.n_atoms, 3, 3), dtype=torch.float64, device=dev),
                   torch.empty(1, dtype=torch.float64, device=dev))
        F, sigma, vir, E = out
        _check(load().gint_force_stress(self._h, _ptr(V), _ptr(D), _ptr(F), _ptr(sigma), _ptr(vir), _ptr(E),
                                        self._stream(stream)))
        return F, sigma, vir, E


def debug_fail_alloc(n: int):
    """Test hook: make the n-th device allocation of the library from now on fail (0 disables)."""
    _check(load().gint_debug_fail_alloc(int(n)))


def from_system(system, precision="fp64", brick=(0, 0, 0), device=-1, pos=None, cell=None) -> Gint:
    """Gint handle for a ``synth.System``-like object (pos, species_index, cell, species, grid)."""
    return Gint(system.pos if pos is None else pos, system.species_index, system.cell if cell is None else cell,
                system.species, system.grid, precision=precision, brick=brick, device=device)
