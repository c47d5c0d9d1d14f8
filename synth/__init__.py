"""Seeded synthetic inputs for real-space grid integration (gint).

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2409_09399_gb300``).  It builds *inputs* only: geometries,
tabulated radial functions, the local potential V on the grid and the density
matrix D on a block list supplied by the caller.  It holds none of the
method's arithmetic: no interpolation of the radial tables, no spherical
harmonics, no neighbour search, no grid sums.

Units are bohr and hartree; angstrom inputs are converted with the lattice
constant 1 angstrom = 1.8897259886 bohr that the paper states for its tests
(Section 3, testing systems).

Random numbers come from one counter-based generator, the SplitMix64
finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), iterated over a key sequence, so every value is a
pure function of (seed, key) and does not depend on numpy's generator streams.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

BOHR_PER_ANG = 1.8897259886

# ---------------------------------------------------------------------------
# counter-based random numbers
# ---------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 ``x`` (wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def hash_keys(seed: int, *keys) -> np.ndarray:
    """Iterated SplitMix64 over (seed, k0, k1, ...); keys are broadcast int arrays.

    Negative keys are offset by 2^20 so that every key is a non-negative
    integer before mixing.
    """
    with np.errstate(over="ignore"):
        h = splitmix64(np.uint64(seed))
        for k in keys:
            k = np.asarray(k, dtype=np.int64) + (1 << 20)
            h = splitmix64(h ^ k.astype(np.uint64))
    return h


def uniform01(seed: int, *keys) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of ``hash_keys``."""
    h = hash_keys(seed, *keys)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# radial functions (numerical atomic orbitals, tabulated)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Radial:
    """One tabulated radial function R_{zeta l}(r) on knots r_k = k*dr."""
    l: int
    zeta: int
    dr: float
    y: np.ndarray   # R(r_k), k = 0 .. n_knots-1
    dy: np.ndarray  # R'(r_k)


@dataclasses.dataclass
class Species:
    name: str
    rc: float
    radials: List[Radial]

    @property
    def n_orb(self) -> int:
        return sum(2 * r.l + 1 for r in self.radials)


def _taper(r, r0, rc):
    """Quintic smoothstep taper f and f' (C2, f(rc)=f'(rc)=0) over [r0, rc]."""
    w = rc - r0
    t = np.clip((r - r0) / w, 0.0, 1.0)
    f = 1.0 - 10.0 * t**3 + 15.0 * t**4 - 6.0 * t**5
    fp = (-30.0 * t**2 + 60.0 * t**3 - 30.0 * t**4) / w
    inside = (r > r0) & (r < rc)
    fp = np.where(inside, fp, 0.0)
    f = np.where(r >= rc, 0.0, f)
    return f, fp


def gaussian_radial(l: int, alphas: Sequence[float], coeffs: Sequence[float],
                    rc: float = 7.0, taper_start: float = 6.0, dr: float = 0.01,
                    normalize: bool = True, taper: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """Tabulate R(r) = r^l * sum_k c_k exp(-a_k r^2) * taper(r) and R'(r).

    Knots r_k = k*dr for k = 0..round(rc/dr).  With ``normalize`` the
    coefficients are scaled so that int_0^rc R^2 r^2 dr = 1 (Gauss-Legendre
    quadrature on [0, taper_start] and [taper_start, rc], both smooth pieces).
    """
    alphas = np.asarray(alphas, dtype=np.float64)
    coeffs = np.asarray(coeffs, dtype=np.float64)

    def g_and_dg(r):
        e = np.exp(-alphas[None, :] * (r[:, None] ** 2))
        g = (coeffs[None, :] * e).sum(1)
        dg = (coeffs[None, :] * (-2.0 * alphas[None, :] * r[:, None]) * e).sum(1)
        return g, dg

    def radial(r):
        g, dg = g_and_dg(r)
        if taper:
            f, fp = _taper(r, taper_start, rc)
        else:
            f, fp = np.ones_like(r), np.zeros_like(r)
        rl = r**l
        drl = l * r ** (l - 1) if l > 0 else np.zeros_like(r)
        R = rl * g * f
        dR = drl * g * f + rl * dg * f + rl * g * fp
        return R, dR

    if normalize:
        x, w = np.polynomial.legendre.leggauss(400)
        norm2 = 0.0
        for a, b in ((0.0, taper_start), (taper_start, rc)):
            r = 0.5 * (b - a) * x + 0.5 * (b + a)
            R, _ = radial(r)
            norm2 += 0.5 * (b - a) * np.sum(w * R * R * r * r)
        coeffs = coeffs / math.sqrt(norm2)
    n_knots = int(round(rc / dr)) + 1
    r = np.arange(n_knots, dtype=np.float64) * dr
    y, dy = radial(r)
    y[-1] = 0.0 if taper else y[-1]
    dy[-1] = 0.0 if taper else dy[-1]
    return y, dy


# (l, zeta) shells per element for the basis sets named in the workloads:
# C DZP = 2s2p1d (13 orbitals), H DZP = 2s1p (5), O SZP = 1s1p1d (9).
BASIS_SHELLS = {
    ("C", "DZP"): [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0)],
    ("H", "DZP"): [(0, 0), (0, 1), (1, 0)],
    ("O", "SZP"): [(0, 0), (1, 0), (2, 0)],
}
_Z = {"H": 1, "C": 6, "O": 8}


def make_species(element: str, basis: str, seed: int = 4, rc: float = 7.0,
                 dr: float = 0.01, taper_start: float = 6.0) -> Species:
    """Seeded two-Gaussian radial functions for one element and basis.

    Per (element, l, zeta): alpha_1, alpha_2 log-uniform in [0.2, 3.0],
    c_1 = 1, c_2 uniform in (-1, 1); tapered to zero over [6, 7] bohr and
    normalised.
    """
    radials = []
    for (l, zeta) in BASIS_SHELLS[(element, basis)]:
        u = uniform01(seed, _Z[element], l, zeta, np.arange(3))
        a1 = math.exp(math.log(0.2) + (math.log(3.0) - math.log(0.2)) * u[0])
        a2 = math.exp(math.log(0.2) + (math.log(3.0) - math.log(0.2)) * u[1])
        c2 = 2.0 * u[2] - 1.0
        y, dy = gaussian_radial(l, [a1, a2], [1.0, c2], rc=rc, taper_start=taper_start, dr=dr)
        radials.append(Radial(l=l, zeta=zeta, dr=dr, y=y, dy=dy))
    return Species(name=element, rc=rc, radials=radials)


# ---------------------------------------------------------------------------
# geometries
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class System:
    """A periodic cell: rows of ``cell`` are a1, a2, a3 (bohr); pos in bohr."""
    name: str
    cell: np.ndarray          # (3, 3)
    pos: np.ndarray           # (n, 3)
    species_index: np.ndarray  # (n,) int32
    species: List[Species]
    grid: Tuple[int, int, int]

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_grid(self) -> int:
        return int(self.grid[0]) * int(self.grid[1]) * int(self.grid[2])

    def nw(self) -> np.ndarray:
        return np.array([self.species[s].n_orb for s in self.species_index], dtype=np.int64)


def diamond(seed: int = 1, a_ang: float = 3.567, disp_ang: float = 0.05, grid=(36, 36, 36),
            species: Species | None = None) -> System:
    """8-atom conventional diamond-C cell with seeded uniform displacements."""
    frac = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                     [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    a = a_ang * BOHR_PER_ANG
    cell = np.eye(3) * a
    u = uniform01(seed, np.arange(8)[:, None], np.arange(3)[None, :])
    pos = frac * a + (2.0 * u - 1.0) * disp_ang * BOHR_PER_ANG
    sp = species if species is not None else make_species("C", "DZP")
    return System("diamond", cell, pos, np.zeros(8, np.int32), [sp], tuple(grid))


def tbg_counts(m: int) -> int:
    """Atom count of the commensurate (m, m+1) twisted bilayer: 4(3m^2+3m+1)."""
    return 4 * (3 * m * m + 3 * m + 1)


def tbg_angle(m: int) -> float:
    """Twist angle (radians): cos(theta) = (3m^2+3m+1/2)/(3m^2+3m+1)."""
    n = 3 * m * m + 3 * m + 1
    return math.acos((n - 0.5) / n)


def _graphene_layer(a1, a2, basis, t1, t2, rot):
    """Sites of a (rotated) graphene layer inside the supercell spanned by t1, t2."""
    T = np.stack([t1, t2], 1)  # columns
    Tinv = np.linalg.inv(T)
    R = np.array([[math.cos(rot), -math.sin(rot)], [math.sin(rot), math.cos(rot)]])
    a1r, a2r = R @ a1, R @ a2
    br = [R @ b for b in basis]
    L = np.stack([a1r, a2r], 1)
    # corners of the supercell in rotated-lattice coordinates bound the search
    corners = np.array([[0, 0], t1, t2, t1 + t2]).T
    c = np.linalg.solve(L, corners)
    lo = np.floor(c.min(1)).astype(int) - 2
    hi = np.ceil(c.max(1)).astype(int) + 2
    n1, n2 = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1), indexing="ij")
    pts = []
    for b in br:
        p = n1[..., None] * a1r + n2[..., None] * a2r + b
        pts.append(p.reshape(-1, 2))
    p = np.concatenate(pts, 0)
    f = p @ Tinv.T
    eps = 1e-9
    keep = (f[:, 0] >= -eps) & (f[:, 0] < 1 - eps) & (f[:, 1] >= -eps) & (f[:, 1] < 1 - eps)
    return p[keep]


def tbg(m: int, cc_ang: float = 1.42, d_ang: float = 3.35, vacuum_ang: float = 20.0,
        h_bohr: float = math.pi / 20.0, grid=None, species: Species | None = None) -> System:
    """Commensurate twisted bilayer graphene of index m (AA origin, layers centred in c).

    Supercell t1 = m a1 + (m+1) a2, t2 = -(m+1) a1 + (2m+1) a2 with
    a = cc*sqrt(3) and a1, a2 at 60 degrees; layer 2 is layer 1 rotated by the
    commensurate angle about the shared site at the origin.  c = d + vacuum.
    Grid n_i = ceil(|a_i| / h) with h = pi/20 bohr (400 Ry density cutoff).
    """
    a = cc_ang * math.sqrt(3.0)
    a1 = np.array([a, 0.0])
    a2 = np.array([0.5 * a, 0.5 * math.sqrt(3.0) * a])
    basis = [np.zeros(2), (a1 + a2) / 3.0]
    t1 = m * a1 + (m + 1) * a2
    t2 = -(m + 1) * a1 + (2 * m + 1) * a2
    theta = tbg_angle(m)
    # pick the rotation sense that keeps t1 a lattice vector of layer 2
    L = np.stack([a1, a2], 1)
    sign = None
    for s in (1.0, -1.0):
        R = np.array([[math.cos(-s * theta), -math.sin(-s * theta)],
                      [math.sin(-s * theta), math.cos(-s * theta)]])
        c = np.linalg.solve(L, R @ t1)
        if np.allclose(c, np.round(c), atol=1e-6):
            sign = s
            break
    assert sign is not None
    l1 = _graphene_layer(a1, a2, basis, t1, t2, 0.0)
    l2 = _graphene_layer(a1, a2, basis, t1, t2, sign * theta)
    n_layer = 2 * (3 * m * m + 3 * m + 1)
    assert l1.shape[0] == n_layer and l2.shape[0] == n_layer, (l1.shape, l2.shape, n_layer)
    c = d_ang + vacuum_ang
    z1, z2 = 0.5 * c - 0.5 * d_ang, 0.5 * c + 0.5 * d_ang
    pos = np.concatenate([np.c_[l1, np.full(n_layer, z1)], np.c_[l2, np.full(n_layer, z2)]], 0)
    cell = np.array([[t1[0], t1[1], 0.0], [t2[0], t2[1], 0.0], [0.0, 0.0, c]])
    cell_b = cell * BOHR_PER_ANG
    pos_b = pos * BOHR_PER_ANG
    if grid is None:
        grid = tuple(int(math.ceil(np.linalg.norm(cell_b[i]) / h_bohr - 1e-9)) for i in range(3))
    sp = species if species is not None else make_species("C", "DZP")
    return System(f"tbg_m{m}", cell_b, pos_b, np.zeros(pos.shape[0], np.int32), [sp], tuple(grid))


def random_cell(i: int, n_atoms_range=(8, 96), box_ang=(8.0, 16.0), min_sep_ang: float = 1.0) -> System:
    """One cubic C/H/O cell of the uneven multi-cell workload (seed 1000 + i).

    Box L ~ U[8, 16] angstrom, grid n = round(24 + 40 (L-8)/8) per axis,
    atom count uniform in [8, 96], species uniform over C (DZP), H (DZP),
    O (SZP), positions by random sequential placement with a periodic
    minimum separation of 1 angstrom.
    """
    seed = 1000 + i
    u = uniform01(seed, 0, np.arange(3))
    L = box_ang[0] + (box_ang[1] - box_ang[0]) * u[0]
    n = int(round(24 + 40 * (L - 8.0) / 8.0))
    n_at = n_atoms_range[0] + int(u[1] * (n_atoms_range[1] - n_atoms_range[0] + 1))
    sps = [make_species("C", "DZP"), make_species("H", "DZP"), make_species("O", "SZP")]
    spi = np.minimum((uniform01(seed, 1, np.arange(n_at)) * 3).astype(np.int32), 2)
    pos = []
    k = 0
    while len(pos) < n_at:
        p = uniform01(seed, 2, k, np.arange(3)) * L
        k += 1
        ok = True
        for q in pos:
            d = p - q
            d -= L * np.round(d / L)
            if np.dot(d, d) < min_sep_ang**2:
                ok = False
                break
        if ok:
            pos.append(p)
        assert k < 100000
    cell = np.eye(3) * L * BOHR_PER_ANG
    return System(f"cell{i}", cell, np.array(pos) * BOHR_PER_ANG, spi.astype(np.int32), sps, (n, n, n))


# ---------------------------------------------------------------------------
# local potential V on the grid
# ---------------------------------------------------------------------------
def plane_wave_params(seed: int = 2, n_waves: int = 16, mmax: int = 4, amp: float = 0.5):
    """Integer wave vectors m_k (|m_ki| <= 4, m_k != 0) and phases phi_k in [0, 2 pi)."""
    ms = []
    k = 0
    while len(ms) < n_waves:
        u = uniform01(seed, k, np.arange(4))
        k += 1
        mk = np.minimum((u[:3] * (2 * mmax + 1)).astype(np.int64), 2 * mmax) - mmax
        if np.all(mk == 0):
            continue
        ms.append((mk, 2.0 * math.pi * u[3]))
    m = np.array([x[0] for x in ms], dtype=np.int64)
    phi = np.array([x[1] for x in ms], dtype=np.float64)
    return m, phi, amp


def v_at(idx: np.ndarray, grid, params) -> np.ndarray:
    """V at grid indices ``idx`` (..., 3): sum_k amp cos(2 pi m_k . f + phi_k), f_i = g_i/n_i."""
    m, phi, amp = params
    idx = np.asarray(idx, dtype=np.int64)
    f = idx / np.asarray(grid, dtype=np.float64)
    arg = 2.0 * math.pi * (f @ m.T.astype(np.float64)) + phi
    return amp * np.cos(arg).sum(-1)


def v_grid(grid, params, device=None, dtype=None):
    """V on the whole grid as a torch tensor of shape (n1, n2, n3), C order.

    Uses the same per-point formula as ``v_at`` evaluated in float64 with
    torch (on ``device``, e.g. a CUDA device for the 6.4e8-point cell).
    """
    import torch
    m, phi, amp = params
    dev = torch.device(device) if device is not None else torch.device("cpu")
    n1, n2, n3 = (int(x) for x in grid)
    out = torch.zeros((n1, n2, n3), dtype=torch.float64, device=dev)
    f1 = torch.arange(n1, dtype=torch.float64, device=dev) / n1
    f2 = torch.arange(n2, dtype=torch.float64, device=dev) / n2
    f3 = torch.arange(n3, dtype=torch.float64, device=dev) / n3
    two_pi = 2.0 * math.pi
    for k in range(m.shape[0]):
        a1 = two_pi * float(m[k, 0]) * f1
        a2 = two_pi * float(m[k, 1]) * f2
        a3 = two_pi * float(m[k, 2]) * f3
        # chunk over the first axis to bound temporaries
        step = max(1, (1 << 26) // (n2 * n3))
        for s in range(0, n1, step):
            e = min(n1, s + step)
            arg = (a1[s:e, None, None] + a2[None, :, None]) + a3[None, None, :] + float(phi[k])
            out[s:e] += amp * torch.cos(arg)
    if dtype is not None:
        out = out.to(dtype)
    return out


# ---------------------------------------------------------------------------
# density matrix D on a caller-supplied block list
# ---------------------------------------------------------------------------
def is_canonical(I, J, T) -> np.ndarray:
    """(I < J) or (I == J and T >= 0 lexicographically)."""
    I = np.asarray(I); J = np.asarray(J); T = np.asarray(T)
    t1, t2, t3 = T[..., 0], T[..., 1], T[..., 2]
    lex_nonneg = (t1 > 0) | ((t1 == 0) & ((t2 > 0) | ((t2 == 0) & (t3 >= 0))))
    return (I < J) | ((I == J) & lex_nonneg)


def d_blocks(blocks: np.ndarray, pos: np.ndarray, cell: np.ndarray, nw: np.ndarray,
             seed: int = 3, scale: float = 0.5, decay: float = 4.0) -> List[np.ndarray]:
    """Density-matrix blocks for the block list ``blocks`` (rows I, J, t1, t2, t3).

    For a canonical block (I, J, T): entries U(-1, 1) * scale * exp(-|R_J + T - R_I| / decay)
    with U from the counter-based generator keyed by (I, J, T, mu, nu);
    D_II(0) is symmetrised.  Non-canonical blocks are the transpose of their
    canonical mirror, D_JI(-T) = D_IJ(T)^T, so D is symmetric.
    Returns one (nw_I, nw_J) array per block (the values of ``d_fill``).
    """
    blocks = np.asarray(blocks, dtype=np.int64).reshape(-1, 5)
    nw = np.asarray(nw, dtype=np.int64)
    sizes = nw[blocks[:, 0]] * nw[blocks[:, 1]]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    flat = d_fill(blocks, offs[:-1], int(offs[-1]), pos, cell, nw, seed, scale, decay)
    return [flat[offs[k]:offs[k + 1]].reshape(int(nw[blocks[k, 0]]), int(nw[blocks[k, 1]]))
            for k in range(blocks.shape[0])]


def d_fill(blocks: np.ndarray, offsets: np.ndarray, total: int, pos, cell, nw, seed: int = 3,
           scale: float = 0.5, decay: float = 4.0) -> np.ndarray:
    """D laid out as a flat float64 array: block b row-major at offsets[b].

    Vectorised over blocks of equal shape; same values as ``d_blocks``.
    """
    blocks = np.asarray(blocks, dtype=np.int64)
    offsets = np.asarray(offsets, dtype=np.int64)
    nw = np.asarray(nw, dtype=np.int64)
    pos = np.asarray(pos, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    out = np.zeros(int(total), dtype=np.float64)
    if blocks.shape[0] == 0:
        return out
    I, J, T = blocks[:, 0], blocks[:, 1], blocks[:, 2:5]
    canon = is_canonical(I, J, T)
    Ic = np.where(canon, I, J)
    Jc = np.where(canon, J, I)
    Tc = np.where(canon[:, None], T, -T)
    ni, nj = nw[Ic], nw[Jc]
    dvec = pos[Jc] + Tc @ cell - pos[Ic]
    amp = scale * np.exp(-np.sqrt((dvec * dvec).sum(1)) / decay)
    rect_mirror = (~canon) & (ni != nj)
    for a in np.unique(ni):
        for bsz in np.unique(nj):
            sel = np.nonzero((ni == a) & (nj == bsz) & ~rect_mirror)[0]
            if sel.size == 0:
                continue
            for s0 in range(0, sel.size, 1 << 16):
                s = sel[s0:s0 + (1 << 16)]
                mu = np.arange(a)[None, :, None]
                nu = np.arange(bsz)[None, None, :]
                X = (2.0 * uniform01(seed, Ic[s][:, None, None], Jc[s][:, None, None],
                                     Tc[s, 0][:, None, None], Tc[s, 1][:, None, None],
                                     Tc[s, 2][:, None, None], mu, nu) - 1.0)
                X = X * amp[s][:, None, None]
                diag = (Ic[s] == Jc[s]) & (~Tc[s].any(1))
                if diag.any():
                    X[diag] = 0.5 * (X[diag] + np.swapaxes(X[diag], 1, 2))
                # square mirrors of a canonical block are its transpose
                nc = ~canon[s]
                if nc.any():
                    X[nc] = np.swapaxes(X[nc], 1, 2)
                idx = offsets[s][:, None] + np.arange(a * bsz)[None, :]
                out[idx] = X.reshape(s.size, a * bsz)
    # rectangular mirror blocks (nw_I != nw_J, non-canonical): the transpose
    # of the canonical block, generated with the same keys
    for b in np.nonzero(rect_mirror)[0]:
        a, bsz = int(ni[b]), int(nj[b])
        mu = np.arange(a)[:, None]
        nu = np.arange(bsz)[None, :]
        X = (2.0 * uniform01(seed, Ic[b], Jc[b], Tc[b, 0], Tc[b, 1], Tc[b, 2], mu, nu) - 1.0) * amp[b]
        out[offsets[b]:offsets[b] + a * bsz] = X.T.reshape(-1)
    return out


# ---------------------------------------------------------------------------
# torch versions (same definitions, for large grids and patterns on a device)
# ---------------------------------------------------------------------------
def _t_splitmix64(z):
    """SplitMix64 finaliser on int64 tensors holding uint64 bit patterns."""
    import torch  # noqa: F401
    z = z + (-7046029254386353131)  # 0x9E3779B97F4A7C15 as int64
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * (-4658895280553007687)  # 0xBF58476D1CE4E5B9
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * (-7723592293110705685)  # 0x94D049BB133111EB
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def uniform01_torch(seed: int, *keys):
    """Same values as ``uniform01`` for int64 tensor keys (broadcast)."""
    import torch
    h0 = int(splitmix64(np.uint64(seed)))
    if h0 >= 1 << 63:
        h0 -= 1 << 64
    dev = keys[0].device
    h = torch.tensor(h0, dtype=torch.int64, device=dev)
    for k in keys:
        h = _t_splitmix64(h ^ (k.to(torch.int64) + (1 << 20)))
    top = (h >> 11) & ((1 << 53) - 1)
    return top.to(torch.float64) * (1.0 / 9007199254740992.0)


def d_fill_torch(blocks, offsets, total: int, pos, cell, nw, device, seed: int = 3, scale: float = 0.5,
                 decay: float = 4.0):
    """``d_fill`` evaluated with torch on ``device`` (identical definition).

    stored[b][mu][nu] = amp_b (2 U(seed, Ic, Jc, Tc, mu_c, nu_c) - 1) with
    (mu_c, nu_c) = (mu, nu) for a canonical block and (nu, mu) for its mirror;
    the self-mirror blocks D_II(0) are symmetrised.
    """
    import torch
    dev = torch.device(device)
    blocks = torch.as_tensor(np.asarray(blocks, dtype=np.int64), device=dev)
    offsets = torch.as_tensor(np.asarray(offsets, dtype=np.int64), device=dev)
    nw_t = torch.as_tensor(np.asarray(nw, dtype=np.int64), device=dev)
    pos_t = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=dev)
    cell_t = torch.as_tensor(np.asarray(cell, dtype=np.float64), device=dev)
    out = torch.zeros(int(total), dtype=torch.float64, device=dev)
    if blocks.shape[0] == 0:
        return out
    I, J, T = blocks[:, 0], blocks[:, 1], blocks[:, 2:5]
    t1, t2, t3 = T[:, 0], T[:, 1], T[:, 2]
    lex = (t1 > 0) | ((t1 == 0) & ((t2 > 0) | ((t2 == 0) & (t3 >= 0))))
    canon = (I < J) | ((I == J) & lex)
    Ic = torch.where(canon, I, J)
    Jc = torch.where(canon, J, I)
    Tc = torch.where(canon[:, None], T, -T)
    dvec = pos_t[Jc] + Tc.to(torch.float64) @ cell_t - pos_t[Ic]
    amp = scale * torch.exp(-torch.sqrt((dvec * dvec).sum(1)) / decay)
    selfm = (Ic == Jc) & (Tc == 0).all(1)
    ni, nj = nw_t[I], nw_t[J]
    shapes = torch.unique(torch.stack([ni, nj], 1), dim=0).cpu().numpy()
    for a, bsz in shapes:
        sel_all = torch.nonzero((ni == int(a)) & (nj == int(bsz))).flatten()
        for s0 in range(0, sel_all.numel(), 1 << 15):
            s = sel_all[s0:s0 + (1 << 15)]
            mu = torch.arange(int(a), device=dev)[None, :, None]
            nu = torch.arange(int(bsz), device=dev)[None, None, :]
            c = canon[s][:, None, None]
            muc = torch.where(c, mu, nu)
            nuc = torch.where(c, nu, mu)
            X = 2.0 * uniform01_torch(seed, Ic[s][:, None, None], Jc[s][:, None, None], Tc[s, 0][:, None, None],
                                      Tc[s, 1][:, None, None], Tc[s, 2][:, None, None], muc, nuc) - 1.0
            X = X * amp[s][:, None, None]
            sm = selfm[s]
            if bool(sm.any()):
                X[sm] = 0.5 * (X[sm] + X[sm].transpose(1, 2))
            idx = offsets[s][:, None] + torch.arange(int(a) * int(bsz), device=dev)[None, :]
            out[idx.reshape(-1)] = X.reshape(-1)
    return out
