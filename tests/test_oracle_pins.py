"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms
(analytic Gaussian overlaps, the spherical-harmonic sum rule and
orthonormality, exact Hermite reproduction of cubics), identities the
definitions imply (H symmetry, Tr(D H^V) = sum rho V dV, grid-shift and
supercell invariance) and finite differences of the energy (forces, stress).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------------------ helpers
def gaussian_species(shells, rc=7.0, dr=0.01, taper=False):
    """Species whose radial functions are r^l sum_k c_k exp(-a_k r^2) (exact tables)."""
    rads = []
    for z, (l, alphas, coeffs) in enumerate(shells):
        y, dy = synth.gaussian_radial(l, alphas, coeffs, rc=rc, dr=dr, normalize=False, taper=taper)
        rads.append(synth.Radial(l=l, zeta=z, dr=dr, y=y, dy=dy))
    return synth.Species("G", rc, rads)


def system(pos, cell, species, grid, spi=None):
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    spi = np.zeros(len(pos), np.int32) if spi is None else np.asarray(spi, np.int32)
    return synth.System("t", np.asarray(cell, dtype=np.float64), pos, spi,
                        species if isinstance(species, list) else [species], tuple(grid))


# Real solid harmonics r^l Y_lm (normalised, no Condon-Shortley phase) as
# Cartesian polynomials {(i, j, k): coefficient}, m = -l..l.
def solid_harmonic_polys(l):
    pi = math.pi
    if l == 0:
        return [{(0, 0, 0): math.sqrt(1 / (4 * pi))}]
    if l == 1:
        c = math.sqrt(3 / (4 * pi))
        return [{(0, 1, 0): c}, {(0, 0, 1): c}, {(1, 0, 0): c}]
    if l == 2:
        a, b, c = math.sqrt(15 / (4 * pi)), math.sqrt(5 / (16 * pi)), math.sqrt(15 / (16 * pi))
        return [{(1, 1, 0): a}, {(0, 1, 1): a}, {(0, 0, 2): 2 * b, (2, 0, 0): -b, (0, 2, 0): -b},
                {(1, 0, 1): a}, {(2, 0, 0): c, (0, 2, 0): -c}]
    if l == 3:
        a, b = math.sqrt(35 / (32 * pi)), math.sqrt(105 / (4 * pi))
        c, d, e = math.sqrt(21 / (32 * pi)), math.sqrt(7 / (16 * pi)), math.sqrt(105 / (16 * pi))
        return [{(2, 1, 0): 3 * a, (0, 3, 0): -a}, {(1, 1, 1): b},
                {(0, 1, 2): 4 * c, (2, 1, 0): -c, (0, 3, 0): -c},
                {(0, 0, 3): 2 * d, (2, 0, 1): -3 * d, (0, 2, 1): -3 * d},
                {(1, 0, 2): 4 * c, (3, 0, 0): -c, (1, 2, 0): -c},
                {(2, 0, 1): e, (0, 2, 1): -e}, {(3, 0, 0): a, (1, 2, 0): -3 * a}]
    raise ValueError(l)


def _moment(n, p):
    """int u^n exp(-p u^2) du over the real line."""
    if n % 2:
        return 0.0
    return math.gamma((n + 1) / 2) / p ** ((n + 1) / 2)


def _overlap_1d(i, j, a, b, A, B):
    """int (x-A)^i (x-B)^j exp(-a (x-A)^2 - b (x-B)^2) dx (Gaussian product theorem)."""
    p = a + b
    P = (a * A + b * B) / p
    pref = math.exp(-a * b / p * (A - B) ** 2)
    s = 0.0
    for u in range(i + 1):
        for v in range(j + 1):
            s += (math.comb(i, u) * math.comb(j, v) * (P - A) ** (i - u) * (P - B) ** (j - v)
                  * _moment(u + v, p))
    return pref * s


def analytic_overlap(shellsA, A, shellsB, B):
    """Overlap matrix of two contracted Gaussian shells sets in the oracle's orbital order."""
    def orbitals(shells):
        out = []
        for l in range(4):
            for (ll, al, co) in shells:
                if ll != l:
                    continue
                for poly in solid_harmonic_polys(l):
                    out.append((al, co, poly))
        return out
    oa, ob = orbitals(shellsA), orbitals(shellsB)
    S = np.zeros((len(oa), len(ob)))
    for m, (aa, ca, pa) in enumerate(oa):
        for n, (ab, cb, pb) in enumerate(ob):
            s = 0.0
            for x, cx in zip(aa, ca):
                for y, cy in zip(ab, cb):
                    for (i, j, k), u in pa.items():
                        for (i2, j2, k2), v in pb.items():
                            s += cx * cy * u * v * (_overlap_1d(i, i2, x, y, A[0], B[0])
                                                    * _overlap_1d(j, j2, x, y, A[1], B[1])
                                                    * _overlap_1d(k, k2, x, y, A[2], B[2]))
            S[m, n] = s
    return S


SHELLS = [(0, [1.3, 0.8], [1.0, -0.4]), (1, [1.1], [1.0]), (2, [0.9, 1.6], [0.7, 0.5]), (3, [1.2], [1.0])]


# ------------------------------------------------------------ basis pins
def test_hermite_reproduces_cubic_exactly():
    # a table sampled from a cubic polynomial is interpolated exactly
    c = [0.3, -1.2, 0.7, -0.15]
    dr = 0.25
    r = np.arange(29) * dr
    y = c[0] + c[1] * r + c[2] * r ** 2 + c[3] * r ** 3
    dy = c[1] + 2 * c[2] * r + 3 * c[3] * r ** 2
    sp = synth.Species("cub", 7.0, [synth.Radial(0, 0, dr, y, dy)])
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    rs = np.linspace(0.01, 6.9, 301)
    d = np.c_[rs, np.zeros_like(rs), np.zeros_like(rs)]
    phi, g = o.eval_orbitals(0, d)
    y00 = 1 / math.sqrt(4 * math.pi)
    exact = (c[0] + c[1] * rs + c[2] * rs ** 2 + c[3] * rs ** 3) * y00
    dexact = (c[1] + 2 * c[2] * rs + 3 * c[3] * rs ** 2) * y00
    assert np.max(np.abs(phi[:, 0] - exact)) < 1e-13
    assert np.max(np.abs(g[:, 0, 0] - dexact)) < 1e-12
    # outside rc the orbital vanishes
    phi, g = o.eval_orbitals(0, [[7.0, 0, 0], [0, 7.5, 0]])
    assert np.all(phi == 0) and np.all(g == 0)


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_spherical_harmonic_sum_rule(l):
    # at a knot (r = 1.0 = 4 * 0.25, t = 0) R(r) is the tabulated value exactly
    dr = 0.25
    y = np.linspace(0.5, 0.0, 29)
    dy = np.full(29, -0.5 / 7.0)
    sp = synth.Species("s", 7.0, [synth.Radial(l, 0, dr, y, dy)])
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    rng = np.random.default_rng(1)
    v = rng.normal(size=(50, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    phi, _ = o.eval_orbitals(0, v * 1.0)
    R = y[4]
    assert np.allclose((phi ** 2).sum(1), R * R * (2 * l + 1) / (4 * math.pi), rtol=1e-13, atol=0)


def test_spherical_harmonics_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform in phi is exact for these degrees
    dr = 0.25
    y = np.ones(29)
    dy = np.zeros(29)
    rads = [synth.Radial(l, 0, dr, y, dy) for l in range(4)]
    sp = synth.Species("s", 7.0, rads)
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    x, w = np.polynomial.legendre.leggauss(16)
    ph = np.arange(32) * 2 * math.pi / 32
    ct = np.repeat(x, 32)
    st = np.sqrt(1 - ct ** 2)
    pp = np.tile(ph, 16)
    d = np.c_[st * np.cos(pp), st * np.sin(pp), ct] * 2.0  # r = 2.0, a knot
    W = np.repeat(w, 32) * (2 * math.pi / 32)
    phi, _ = o.eval_orbitals(0, d)
    M = (phi * W[:, None]).T @ phi
    assert np.allclose(M, np.eye(16), atol=1e-13)


def test_gradient_matches_finite_differences():
    sp = gaussian_species(SHELLS)
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    rng = np.random.default_rng(3)
    d = rng.normal(size=(40, 3)) * 1.5
    h = 1e-5
    _, g = o.eval_orbitals(0, d)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        p1, _ = o.eval_orbitals(0, d + e)
        p0, _ = o.eval_orbitals(0, d - e)
        assert np.allclose(g[:, :, a], (p1 - p0) / (2 * h), atol=2e-8)


def test_orbital_values_closed_form():
    # phi = sum c exp(-a r^2) S_lm(d) for the Gaussian test shells (no taper)
    sp = gaussian_species(SHELLS)
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    rng = np.random.default_rng(4)
    d = rng.normal(size=(30, 3)) * 1.3
    phi, _ = o.eval_orbitals(0, d)
    ref = []
    for l in range(4):
        for (ll, al, co) in SHELLS:
            if ll != l:
                continue
            for poly in solid_harmonic_polys(l):
                r2 = (d ** 2).sum(1)
                rad = sum(c * np.exp(-a * r2) for a, c in zip(al, co))
                S = sum(v * d[:, 0] ** i * d[:, 1] ** j * d[:, 2] ** k for (i, j, k), v in poly.items())
                ref.append(rad * S)
    ref = np.array(ref).T
    assert np.max(np.abs(phi - ref)) < 5e-8  # cubic Hermite error at dr = 0.01


# --------------------------------------------------------------- H^V pins
@pytest.mark.parametrize("cellkind", ["cubic", "hexagonal"])
def test_overlap_matches_analytic_gaussians(cellkind):
    """V = 1: the grid integral converges to the analytic overlap S (Eq. 2)."""
    sp = gaussian_species(SHELLS)
    if cellkind == "cubic":
        cell = np.eye(3) * 24.0
        grid = (120, 120, 120)
    else:
        a = 25.0
        cell = np.array([[a, 0, 0], [0.5 * a, 0.5 * math.sqrt(3) * a, 0], [0, 0, 24.0]])
        grid = (128, 128, 120)
    A = np.array([11.3, 9.1, 12.2])
    B = A + np.array([1.1, -0.7, 0.9])
    o = oracle.Oracle(system([A, B], cell, sp, grid))
    V = np.ones(grid)
    (H,) = o.vlocal_blocks(V, [[0, 1, 0, 0, 0]])
    S = analytic_overlap(SHELLS, A, SHELLS, B)
    assert np.max(np.abs(H - S)) < 1e-9, np.max(np.abs(H - S))
    (H0,) = o.vlocal_blocks(V, [[0, 0, 0, 0, 0]])
    S0 = analytic_overlap(SHELLS, A, SHELLS, A)
    assert np.max(np.abs(H0 - S0)) < 1e-9


def test_overlap_error_is_fourth_order_in_table_spacing():
    """Halving dr cuts the Hermite error ~16x: the interpolant is the cubic Hermite one."""
    errs = []
    for dr in (0.04, 0.02):
        sp = gaussian_species([(0, [2.5], [1.0]), (1, [2.2], [1.0])], dr=dr)
        A = np.array([10.0, 10.4, 9.7])
        B = A + np.array([0.8, 0.5, -0.6])
        o = oracle.Oracle(system([A, B], np.eye(3) * 20.0, sp, (160, 160, 160)))
        (H,) = o.vlocal_blocks(np.ones((160, 160, 160)), [[0, 1, 0, 0, 0]])
        S = analytic_overlap([(0, [2.5], [1.0]), (1, [2.2], [1.0])], A, [(0, [2.5], [1.0]), (1, [2.2], [1.0])], B)
        errs.append(np.max(np.abs(H - S)))
    ratio = errs[0] / errs[1]
    assert 10.0 < ratio < 24.0, (errs, ratio)


def test_single_atom_onsite_overlap():
    """One atom, V = 1: S = delta_ll' delta_mm' int R_z R_z' r^2 dr (C DZP tables)."""
    sp = synth.make_species("C", "DZP")
    o = oracle.Oracle(system([[9.9, 10.2, 10.05]], np.eye(3) * 20.0, sp, (140, 140, 140)))
    (H,) = o.vlocal_blocks(np.ones((140, 140, 140)), [[0, 0, 0, 0, 0]])
    rads = sp.radials
    r = np.arange(len(rads[0].y)) * rads[0].dr

    def simpson(f):
        return rads[0].dr / 3.0 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())

    ref = np.zeros((13, 13))
    orb = []
    for l in range(3):
        for j, R in enumerate(rads):
            if R.l == l:
                orb += [(j, l, m) for m in range(2 * l + 1)]
    for a, (j, l, m) in enumerate(orb):
        for b, (j2, l2, m2) in enumerate(orb):
            if l == l2 and m == m2:
                ref[a, b] = simpson(rads[j].y * rads[j2].y * r * r)
    assert np.max(np.abs(H - ref)) < 2e-4, np.max(np.abs(H - ref))
    assert np.allclose(np.diag(H), 1.0, atol=2e-4)


# ---------------------------------------------- diamond-like small systems
def small_diamond(grid=(20, 20, 20), basis="SZP"):
    sp = synth.make_species("O", "SZP") if basis == "SZP" else synth.make_species("C", "DZP")
    s = synth.diamond(grid=grid, species=sp)
    return s


def test_h_symmetry_and_trace_identity():
    """H_JI(-T) = H_IJ(T)^T; sum_g rho_g V_g dV = sum_blocks D . H  (Eq. 2, 3)."""
    s = small_diamond()
    o = oracle.Oracle(s)
    params = synth.plane_wave_params()
    V = synth.v_grid(s.grid, params).numpy()
    H = o.vlocal(V)
    idx = o.block_index()
    worst = 0.0
    for b, key in enumerate(o.blocks):
        I, J, t = key[0], key[1], key[2:]
        m = idx[(J, I, -t[0], -t[1], -t[2])]
        worst = max(worst, np.max(np.abs(o.block(H, b) - o.block(H, m).T)))
    assert worst <= 1e-14 * np.max(np.abs(H))
    D = o.d_fill()
    rho = o.rho(D)
    E_grid = float((rho * V).sum() * o.dV)
    E_tr = float(np.dot(D, H))
    assert abs(E_grid - E_tr) <= 1e-12 * max(1.0, abs(E_tr))
    assert abs(o.energy(V, D) - E_grid) <= 1e-13 * max(1.0, abs(E_grid))


def test_forces_match_energy_finite_differences():
    """F = -dE/dR at fixed V and D (Eq. 4): central differences, delta = 1e-4 bohr."""
    s = small_diamond(grid=(18, 18, 18))
    o = oracle.Oracle(s)
    params = synth.plane_wave_params()
    V = synth.v_grid(s.grid, params).numpy()
    D0 = o.d_fill()
    Dmap = {tuple(int(x) for x in k): o.block(D0, b).copy() for b, k in enumerate(o.blocks)}
    F, _ = o.force(V, D0, atoms=[1, 5])

    def energy_at(pos):
        op = oracle.Oracle(s, pos=pos)
        D = np.zeros(op.n_values)
        for b, k in enumerate(op.blocks):
            blk = Dmap.get(tuple(int(x) for x in k))
            if blk is not None:
                D[op.offsets[b]:op.offsets[b + 1]] = blk.reshape(-1)
        return op.energy(V, D)

    delta = 1e-4
    scale = np.max(np.abs(F))
    for q, I in enumerate([1, 5]):
        for a in range(3):
            p1 = s.pos.copy(); p1[I, a] += delta
            p0 = s.pos.copy(); p0[I, a] -= delta
            fd = -(energy_at(p1) - energy_at(p0)) / (2 * delta)
            assert abs(fd - F[q, a]) < 1e-6 * scale + 1e-9, (I, a, fd, F[q, a])


def test_stress_matches_strain_finite_differences():
    """Pi_ab = dE/d(eps_ab) at fixed V_g and dV (Eq. 5 read as the strain derivative)."""
    s = small_diamond(grid=(16, 16, 16))
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    D0 = o.d_fill()
    Dmap = {tuple(int(x) for x in k): o.block(D0, b).copy() for b, k in enumerate(o.blocks)}
    sigma, _ = o.stress(V, D0)
    Pi = -sigma * o.omega

    def energy_strained(eps):
        Fm = np.eye(3) + eps
        cell = s.cell @ Fm.T
        pos = s.pos @ Fm.T
        op = oracle.Oracle(s, pos=pos, cell=cell)
        D = np.zeros(op.n_values)
        for b, k in enumerate(op.blocks):
            blk = Dmap.get(tuple(int(x) for x in k))
            if blk is not None:
                D[op.offsets[b]:op.offsets[b + 1]] = blk.reshape(-1)
        return op.energy(V, D) * (o.dV / op.dV)  # fixed dV

    eta = 1e-5
    scale = np.max(np.abs(Pi))
    for a, b in [(0, 0), (1, 2), (2, 1), (0, 2)]:
        e = np.zeros((3, 3)); e[a, b] = eta
        fd = (energy_strained(e) - energy_strained(-e)) / (2 * eta)
        assert abs(fd - Pi[a, b]) < 1e-5 * scale, (a, b, fd, Pi[a, b])


def test_grid_shift_invariance():
    """Shift atoms by a grid vector and roll V: H unchanged, rho rolls."""
    s = small_diamond(grid=(16, 18, 20))
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    shift = np.array([3, -2, 5])
    sv = (shift / np.array(s.grid)) @ s.cell
    o2 = oracle.Oracle(s, pos=s.pos + sv)
    V2 = np.roll(V, tuple(shift), axis=(0, 1, 2))
    assert np.array_equal(o.blocks, o2.blocks)
    H, H2 = o.vlocal(V), o2.vlocal(V2)
    assert np.max(np.abs(H - H2)) < 1e-12 * np.max(np.abs(H))
    D = o.d_fill()
    rho, rho2 = o.rho(D), o2.rho(D)
    assert np.max(np.abs(np.roll(rho, tuple(shift), axis=(0, 1, 2)) - rho2)) < 1e-12 * np.max(np.abs(rho))


def test_supercell_consistency():
    """The 2x1x1 replica reproduces H blocks mapped by T and doubles E (periodic images)."""
    s = small_diamond(grid=(14, 14, 14))
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    H = o.vlocal(V)
    D = o.d_fill()
    E = o.energy(V, D)
    n = s.n_atoms
    cell2 = s.cell.copy(); cell2[0] *= 2
    pos2 = np.concatenate([s.pos, s.pos + s.cell[0]])
    s2 = synth.System("sc", cell2, pos2, np.zeros(2 * n, np.int32), s.species, (28, 14, 14))
    o2 = oracle.Oracle(s2)
    V2 = np.concatenate([V, V], axis=0)
    H2 = o2.vlocal(V2)
    idx = o.block_index()
    D2 = np.zeros(o2.n_values)
    worst = 0.0
    for b, (I2, J2, t1, t2, t3) in enumerate(o2.blocks):
        I, kI, J, kJ = I2 % n, I2 // n, J2 % n, J2 // n
        key = (I, J, kJ - kI + 2 * t1, t2, t3)
        ub = idx[key]
        worst = max(worst, np.max(np.abs(o2.block(H2, b) - o.block(H, ub))))
        D2[o2.offsets[b]:o2.offsets[b + 1]] = o.block(D, ub).reshape(-1)
    assert worst < 1e-13 * np.max(np.abs(H))
    assert abs(o2.energy(V2, D2) - 2 * E) < 1e-12 * abs(E)


# --------------------------------------------- atom-centre limit (|d| -> 0)
def _centre_closed_form(shells):
    """phi(0) and grad phi(0) of r^l sum_k c_k exp(-a_k r^2) Y_lm, oracle orbital order.

    phi = (sum_k c_k exp(-a_k r^2)) S_lm(d) with S_lm = r^l Y_lm a polynomial of
    degree l, so at d = 0: phi = sum c / sqrt(4 pi) for l = 0 and 0 for l >= 1;
    grad phi = sum c grad S_1m for l = 1 (the constant gradient of the linear
    polynomial) and 0 for l = 0 (the Gaussian is flat at the centre) and l >= 2.
    """
    phi, grad = [], []
    for l in range(4):
        for (ll, al, co) in shells:
            if ll != l:
                continue
            csum = float(sum(co))
            for poly in solid_harmonic_polys(l):
                g = np.zeros(3)
                if l == 1:
                    (i, j, k), v = next(iter(poly.items()))
                    g[[i, j, k].index(1)] = csum * v
                phi.append(csum * poly.get((0, 0, 0), 0.0))
                grad.append(g)
    return np.array(phi), np.array(grad)


def test_orbitals_at_atom_centre_closed_form():
    """At d = 0 the oracle returns the limits of Eq. 2's orbitals, not 0/0."""
    sp = gaussian_species(SHELLS)
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    phi, g = o.eval_orbitals(0, np.zeros((1, 3)))
    phi_ref, g_ref = _centre_closed_form(SHELLS)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
    # the Hermite table reproduces R(0) = y_0 and R'(0) = y'_0 exactly at the first knot
    assert np.max(np.abs(phi[0] - phi_ref)) < 1e-14, (phi[0], phi_ref)
    assert np.max(np.abs(g[0] - g_ref)) < 1e-14, (g[0], g_ref)
    # the p orbitals (y, z, x order) carry the only non-zero gradients
    assert np.count_nonzero(np.abs(g[0]).sum(1) > 0) == 3


@pytest.mark.parametrize("basis", ["gauss", "C_DZP"])
def test_orbitals_continuous_at_atom_centre(basis):
    """phi and grad phi at |d| = 1e-7 and 1e-9 along several directions equal their values at d = 0."""
    sp = gaussian_species(SHELLS) if basis == "gauss" else synth.make_species("C", "DZP")
    o = oracle.Oracle(system([[0, 0, 0]], np.eye(3) * 30, sp, (4, 4, 4)))
    p0, g0 = o.eval_orbitals(0, np.zeros((1, 3)))
    rng = np.random.default_rng(11)
    n = rng.normal(size=(12, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    for r in (1e-7, 1e-9):
        p, g = o.eval_orbitals(0, n * r)
        assert np.max(np.abs(p - p0)) < 1e-5, (r, np.max(np.abs(p - p0)))
        assert np.max(np.abs(g - g0)) < 1e-5, (r, np.max(np.abs(g - g0)))
    # and away from the limit branch the same values are approached smoothly (FD of phi at 1e-4)
    h = 1e-5
    for a in range(3):
        e = np.zeros((1, 3)); e[0, a] = h
        pp, _ = o.eval_orbitals(0, e)
        pm, _ = o.eval_orbitals(0, -e)
        assert np.max(np.abs((pp - pm) / (2 * h) - g0[:, :, a])) < 1e-4


def test_density_and_force_with_atom_on_grid_point():
    """An atom exactly on a grid point: rho there is finite and the force equals -dE/dR (Eq. 3, 4)."""
    sp = synth.make_species("O", "SZP")
    cell = np.eye(3) * 9.0
    grid = (18, 18, 18)
    pos = np.array([[0.0, 0.0, 0.0], [4.5, 3.0, 5.5]])  # atom 0 on grid point (0, 0, 0)
    s = system(pos, cell, sp, grid)
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    D = o.d_fill()
    rho0 = o.rho_points(D, [[0, 0, 0]])
    assert np.isfinite(rho0).all()
    F, _ = o.force(V, D, atoms=[0])
    Dmap = {tuple(int(x) for x in k): o.block(D, b).copy() for b, k in enumerate(o.blocks)}

    def energy_at(p):
        op = oracle.Oracle(s, pos=p)
        Dp = np.zeros(op.n_values)
        for b, k in enumerate(op.blocks):
            blk = Dmap.get(tuple(int(x) for x in k))
            if blk is not None:
                Dp[op.offsets[b]:op.offsets[b + 1]] = blk.reshape(-1)
        return op.energy(V, Dp)

    delta = 1e-4
    scale = max(1e-3, np.max(np.abs(F)))
    for a in range(3):
        p1 = pos.copy(); p1[0, a] += delta
        p0 = pos.copy(); p0[0, a] -= delta
        fd = -(energy_at(p1) - energy_at(p0)) / (2 * delta)
        assert abs(fd - F[0, a]) < 2e-6 * scale + 1e-9, (a, fd, F[0, a])


# ----------------------------------------------------- pattern enumeration
def brute_force_pattern(pos, cell, rc, tmax):
    """All (I, J, t) with |R_J + t A - R_I| < rc_I + rc_J for |t_i| <= tmax, sorted (plain numpy)."""
    rng_t = np.arange(-tmax, tmax + 1)
    T = np.stack(np.meshgrid(rng_t, rng_t, rng_t, indexing="ij"), -1).reshape(-1, 3)
    TA = T @ cell
    rows = []
    for I in range(len(pos)):
        for J in range(len(pos)):
            d = pos[J] + TA - pos[I]
            keep = np.sqrt((d * d).sum(1)) < rc[I] + rc[J]
            for t in T[keep]:
                rows.append((I, J, int(t[0]), int(t[1]), int(t[2])))
    rows.sort()
    return np.array(rows, dtype=np.int64).reshape(-1, 5)


def test_pattern_diamond_block_count():
    """Diamond (8 C, rc = 7 bohr): 2,344 blocks, equal to a brute force over |t_i| <= 5 (Section 2.2 sparsity)."""
    s = synth.diamond()
    o = oracle.Oracle(s)
    ref = brute_force_pattern(s.pos, s.cell, np.full(s.n_atoms, 7.0), 5)
    assert len(ref) == 2344
    assert np.array_equal(o.blocks, ref)
    nw = s.nw()
    assert o.offsets[-1] == int(np.sum(nw[ref[:, 0]] * nw[ref[:, 1]]))


def test_pattern_hexagonal_two_species():
    """A skewed hexagonal two-species cell with different cutoffs: the oracle's pattern equals the brute force."""
    a = 8.3
    cell = np.array([[a, 0, 0], [0.5 * a, 0.5 * math.sqrt(3) * a, 0], [0.7, -0.4, 12.0]])
    sps = [synth.make_species("C", "DZP"), synth.make_species("H", "DZP", rc=5.5, taper_start=4.5)]
    pos = np.array([[0.3, 0.2, 1.0], [4.1, 2.2, 6.5], [6.6, 5.0, 3.3], [1.7, 3.9, 9.8]])
    spi = np.array([0, 1, 0, 1], np.int32)
    s = system(pos, cell, sps, (16, 16, 24), spi=spi)
    o = oracle.Oracle(s)
    rc = np.array([sps[k].rc for k in spi])
    ref = brute_force_pattern(pos, cell, rc, 6)
    assert np.array_equal(o.blocks, ref)
    # closed under (I, J, T) -> (J, I, -T)
    keys = {tuple(r) for r in ref.tolist()}
    assert all((J, I, -t1, -t2, -t3) in keys for (I, J, t1, t2, t3) in keys)
