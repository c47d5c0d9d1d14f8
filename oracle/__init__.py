"""ctypes binding of the FP64 brute-force oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.

``Oracle(system)`` builds the oracle's own pair pattern (blocks (I, J, t1, t2, t3)
sorted lexicographically, each block row-major nw_I x nw_J) and exposes:
  vlocal(V)                 -> H on the oracle layout            (paper Eq. 2)
  vlocal_blocks(V, keys)    -> selected blocks of H
  rho(D) / rho_points(D, g) -> density on the grid / at points   (Eq. 3)
  force(V, D, atoms)        -> F_I and per-atom virial Pi_I      (Eq. 4, 5)
  energy(V, D)              -> sum_g V rho dV
  vlocal_masked / force_masked -> the same sums over a subset (shard) of the grid points
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, OpenMP, IEEE arithmetic, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.c_int, _f64p, _i32p, _f64p, _i32p, ctypes.c_int, _f64p, _i32p,
                                 _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_destroy.argtypes = [vp]
        L.orc_error.argtypes = [vp]
        L.orc_n_blocks.restype = ctypes.c_int64
        L.orc_n_blocks.argtypes = [vp]
        L.orc_n_values.restype = ctypes.c_int64
        L.orc_n_values.argtypes = [vp]
        L.orc_blocks.argtypes = [vp, _i64p, _i64p]
        L.orc_dV.restype = ctypes.c_double
        L.orc_dV.argtypes = [vp]
        L.orc_omega.restype = ctypes.c_double
        L.orc_omega.argtypes = [vp]
        L.orc_vlocal.argtypes = [vp, _f64p, _f64p]
        L.orc_vlocal_blocks.argtypes = [vp, _f64p, ctypes.c_int64, _i64p, _f64p]
        L.orc_rho.argtypes = [vp, _f64p, _f64p]
        L.orc_rho_points.argtypes = [vp, _f64p, ctypes.c_int64, _i64p, _f64p]
        L.orc_energy.argtypes = [vp, _f64p, _f64p, ctypes.POINTER(ctypes.c_double)]
        L.orc_force.argtypes = [vp, _f64p, _f64p, ctypes.c_int, _i32p, _f64p, _f64p]
        _u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        L.orc_vlocal_masked.argtypes = [vp, _f64p, _u8p, _f64p]
        L.orc_force_masked.argtypes = [vp, _f64p, _f64p, _u8p, ctypes.c_int, _i32p, _f64p, _f64p]
        L.orc_eval_orbitals.argtypes = [vp, ctypes.c_int, ctypes.c_int64, _f64p, _f64p, _f64p]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int):
    """OpenMP threads of later oracle calls (n >= 1)."""
    lib().orc_set_num_threads(int(n))


class Oracle:
    """FP64 oracle bound to one system (geometry, species, grid)."""

    def __init__(self, system, pos=None, cell=None):
        L = lib()
        self.system = system
        pos = np.ascontiguousarray(system.pos if pos is None else pos, dtype=np.float64)
        cell = np.ascontiguousarray(system.cell if cell is None else cell, dtype=np.float64)
        self.pos, self.cell = pos, cell
        sp = np.ascontiguousarray(system.species_index, dtype=np.int32)
        rc = np.array([s.rc for s in system.species], dtype=np.float64)
        n_rad = np.array([len(s.radials) for s in system.species], dtype=np.int32)
        rads = [r for s in system.species for r in s.radials]
        rl = np.array([r.l for r in rads], dtype=np.int32)
        rnk = np.array([len(r.y) for r in rads], dtype=np.int32)
        rdr = np.array([r.dr for r in rads], dtype=np.float64)
        y = np.ascontiguousarray(np.concatenate([r.y for r in rads]), dtype=np.float64)
        dy = np.ascontiguousarray(np.concatenate([r.dy for r in rads]), dtype=np.float64)
        grid = np.array(system.grid, dtype=np.int32)
        self._h = L.orc_create(int(pos.shape[0]), pos.reshape(-1), sp, cell.reshape(-1), grid,
                               len(system.species), rc, n_rad, rl, rnk, rdr, y, dy)
        if L.orc_error(self._h):
            raise ValueError("oracle: unsupported basis (l > 3 or too many orbitals)")
        nb = L.orc_n_blocks(self._h)
        self.blocks = np.zeros((nb, 5), dtype=np.int64)
        self.offsets = np.zeros(nb + 1, dtype=np.int64)
        if nb:
            L.orc_blocks(self._h, self.blocks, self.offsets)
        self.n_values = int(L.orc_n_values(self._h))
        self.dV = float(L.orc_dV(self._h))
        self.omega = float(L.orc_omega(self._h))
        self.nw = system.nw()
        self._index = None

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().orc_destroy(self._h)
        except Exception:
            pass

    # -------------------------------------------------------------- layout
    def block_index(self):
        """dict (I, J, t1, t2, t3) -> block number."""
        if self._index is None:
            self._index = {tuple(int(x) for x in row): b for b, row in enumerate(self.blocks)}
        return self._index

    def block(self, flat, b):
        I, J = int(self.blocks[b, 0]), int(self.blocks[b, 1])
        return flat[self.offsets[b]:self.offsets[b + 1]].reshape(int(self.nw[I]), int(self.nw[J]))

    def d_fill(self, seed: int = 3, pos=None):
        """Synthetic density matrix on this pattern (values from ``synth``)."""
        import synth
        p = self.pos if pos is None else pos
        return synth.d_fill(self.blocks, self.offsets, self.n_values, p, self.cell, self.nw, seed=seed)

    # ------------------------------------------------------------- results
    def vlocal(self, V):
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        H = np.zeros(self.n_values, dtype=np.float64)
        if self.n_values:
            lib().orc_vlocal(self._h, V, H)
        return H

    def vlocal_blocks(self, V, keys):
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        keys = np.ascontiguousarray(keys, dtype=np.int64).reshape(-1, 5)
        sizes = self.nw[keys[:, 0]] * self.nw[keys[:, 1]]
        out = np.zeros(int(sizes.sum()), dtype=np.float64)
        rc = lib().orc_vlocal_blocks(self._h, V, keys.shape[0], keys.reshape(-1), out)
        if rc != 0:
            raise KeyError("requested block not in the oracle pattern")
        res, o = [], 0
        for k, s in zip(keys, sizes):
            res.append(out[o:o + s].reshape(int(self.nw[k[0]]), int(self.nw[k[1]])))
            o += int(s)
        return res

    def rho(self, D):
        D = np.ascontiguousarray(D, dtype=np.float64)
        n = self.system.n_grid
        out = np.zeros(n, dtype=np.float64)
        if lib().orc_rho(self._h, D, out) != 0:
            raise RuntimeError("oracle rho: neighbour pair missing from the pattern")
        return out.reshape(self.system.grid)

    def rho_points(self, D, idx):
        D = np.ascontiguousarray(D, dtype=np.float64)
        idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1, 3)
        out = np.zeros(idx.shape[0], dtype=np.float64)
        if lib().orc_rho_points(self._h, D, idx.shape[0], idx.reshape(-1), out) != 0:
            raise RuntimeError("oracle rho: neighbour pair missing from the pattern")
        return out

    def energy(self, V, D):
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        D = np.ascontiguousarray(D, dtype=np.float64)
        E = ctypes.c_double(0.0)
        if lib().orc_energy(self._h, V, D, ctypes.byref(E)) != 0:
            raise RuntimeError("oracle energy: neighbour pair missing from the pattern")
        return E.value

    def force(self, V, D, atoms=None):
        """(F (n_sel, 3), per-atom virial Pi_I (n_sel, 3, 3)); stress = -sum Pi / Omega."""
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        D = np.ascontiguousarray(D, dtype=np.float64)
        if atoms is None:
            atoms = np.arange(self.pos.shape[0])
        atoms = np.ascontiguousarray(atoms, dtype=np.int32)
        F = np.zeros((atoms.size, 3), dtype=np.float64)
        W = np.zeros((atoms.size, 9), dtype=np.float64)
        if lib().orc_force(self._h, V, D, atoms.size, atoms, F.reshape(-1), W.reshape(-1)) != 0:
            raise RuntimeError("oracle force: neighbour pair missing from the pattern")
        return F, W.reshape(-1, 3, 3)

    def fold_k(self, H, kfrac):
        """Bloch sum H(k) = sum over blocks (I, J, t) of exp(2 pi i k . t) H_IJ(t) (Eq. 6-8 setting).

        k = sum_i kfrac_i b_i with b_i the reciprocal vectors (b_i . a_j = 2 pi delta_ij), so
        k . T = 2 pi kfrac . t for T = t . A.  Dense N x N complex matrix, N = sum of orbitals;
        rows and columns in atom order, each atom's orbitals in the pattern's order.
        """
        H = np.asarray(H, dtype=np.float64)
        kf = np.asarray(kfrac, dtype=np.float64).reshape(3)
        off = np.concatenate([[0], np.cumsum(self.nw)]).astype(np.int64)
        N = int(off[-1])
        Hk = np.zeros((N, N), dtype=np.complex128)
        for b in range(self.blocks.shape[0]):
            I, J = int(self.blocks[b, 0]), int(self.blocks[b, 1])
            t = self.blocks[b, 2:5].astype(np.float64)
            ph = np.exp(2j * np.pi * float(kf @ t))
            Hk[off[I]:off[I + 1], off[J]:off[J + 1]] += ph * self.block(H, b)
        return Hk

    def vlocal_masked(self, V, mask):
        """H^V summed over the grid points with mask != 0 only (mask: bool/uint8 grid array)."""
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        H = np.zeros(self.n_values, dtype=np.float64)
        if self.n_values:
            lib().orc_vlocal_masked(self._h, V, m, H)
        return H

    def force_masked(self, V, D, mask, atoms=None):
        """(F, per-atom virial) summed over the grid points with mask != 0 only."""
        V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1)
        D = np.ascontiguousarray(D, dtype=np.float64)
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        if atoms is None:
            atoms = np.arange(self.pos.shape[0])
        atoms = np.ascontiguousarray(atoms, dtype=np.int32)
        F = np.zeros((atoms.size, 3), dtype=np.float64)
        W = np.zeros((atoms.size, 9), dtype=np.float64)
        if lib().orc_force_masked(self._h, V, D, m, atoms.size, atoms, F.reshape(-1), W.reshape(-1)) != 0:
            raise RuntimeError("oracle force: neighbour pair missing from the pattern")
        return F, W.reshape(-1, 3, 3)

    def stress(self, V, D):
        F, W = self.force(V, D)
        return -W.sum(0) / self.omega, F

    def eval_orbitals(self, species, d):
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        no = self.system.species[species].n_orb
        phi = np.zeros(d.shape[0] * no, dtype=np.float64)
        g = np.zeros(d.shape[0] * no * 3, dtype=np.float64)
        lib().orc_eval_orbitals(self._h, species, d.shape[0], d.reshape(-1), phi, g)
        return phi.reshape(-1, no), g.reshape(-1, no, 3)
