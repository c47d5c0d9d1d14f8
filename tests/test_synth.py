"""Pins of the seeded input generators (no GPU)."""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tbg_lattice_tab2.txt")


def _tab2():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [float(x) for x in line.split()]
        rows.append((int(v[0]), np.array(v[1:4]), np.array(v[4:7]), np.array(v[7:10])))
    return rows


def test_splitmix64_reference_sequence():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 1234567: the first five
    # outputs of the published reference implementation.
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        xs = np.array([np.uint64(1234567) + np.uint64(k) * g for k in range(5)], dtype=np.uint64)
    out = [int(v) for v in synth.splitmix64(xs)]
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_range_and_determinism():
    u = synth.uniform01(7, np.arange(10000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(u, synth.uniform01(7, np.arange(10000)))


@pytest.mark.parametrize("row", range(4))
def test_tbg_matches_table2(row):
    """Twisted bilayer supercells reproduce the paper's Table 2 (Section 3)."""
    n_atoms, X, Y, Z = _tab2()[row]
    m = {76: 2, 508: 6, 1876: 12, 10444: 29}[n_atoms]
    assert synth.tbg_counts(m) == n_atoms
    s = synth.tbg(m)
    assert s.n_atoms == n_atoms
    A = s.cell / synth.BOHR_PER_ANG
    # in-plane Gram matrix against the table's X and Z columns (3-decimal print)
    G_ours = np.array([[A[0] @ A[0], A[0] @ A[1]], [A[1] @ A[0], A[1] @ A[1]]])
    G_tab = np.array([[X @ X, X @ Z], [Z @ X, Z @ Z]])
    assert np.allclose(np.sqrt(np.diag(G_ours)), np.sqrt(np.diag(G_tab)), atol=2e-3)
    assert abs(G_ours[0, 1] / G_ours[0, 0] - G_tab[0, 1] / G_tab[0, 0]) < 1e-4
    # the table's remaining column is the 30-angstrom perpendicular vector
    assert abs(np.linalg.norm(Y) - 30.0) < 2e-3
    assert abs(Y @ X) < 0.05 and abs(Y @ Z) < 0.05


def test_tbg_geometry_rules():
    s = synth.tbg(5)
    assert s.grid == (283, 283, 281)
    pos = s.pos / synth.BOHR_PER_ANG
    z = np.unique(np.round(pos[:, 2], 6))
    assert len(z) == 2 and abs(z[1] - z[0] - 3.35) < 1e-9
    # nearest-neighbour C-C distance within a layer is 1.42 angstrom
    lay = pos[pos[:, 2] == z[0]]
    A = s.cell / synth.BOHR_PER_ANG
    d = lay[None, :, None, :] - lay[:, None, None, :] - np.array(
        [i * A[0] + j * A[1] for i in (-1, 0, 1) for j in (-1, 0, 1)])[None, None]
    r = np.sqrt((d ** 2).sum(-1)).reshape(len(lay), -1)
    r[r < 1e-6] = np.inf
    assert np.allclose(r.min(1), 1.42, atol=1e-6)
    assert abs(math.degrees(synth.tbg_angle(5)) - 6.0089831977) < 1e-6


def test_radial_tables_normalised_and_smooth():
    sp = synth.make_species("C", "DZP")
    assert sp.n_orb == 13
    for R in sp.radials:
        r = np.arange(len(R.y)) * R.dr
        # composite Simpson on the knots (700 intervals, even) of R^2 r^2
        f = R.y ** 2 * r ** 2
        simpson = R.dr / 3.0 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        assert abs(simpson - 1.0) < 1e-6
        assert R.y[-1] == 0.0 and R.dy[-1] == 0.0
        # tabulated derivative agrees with central differences of the values
        fd = (R.y[2:] - R.y[:-2]) / (2 * R.dr)
        assert np.max(np.abs(fd - R.dy[1:-1])) < 2e-3 * max(1.0, np.abs(R.dy).max())
        if R.l >= 1:
            assert R.y[0] == 0.0


def test_d_blocks_symmetric():
    s = synth.diamond()
    nw = s.nw()
    keys = np.array([[0, 3, 1, 0, -1], [3, 0, -1, 0, 1], [2, 2, 0, 0, 0], [2, 2, 0, 1, 0], [2, 2, 0, -1, 0]])
    b = synth.d_blocks(keys, s.pos, s.cell, nw)
    assert np.array_equal(b[0], b[1].T)
    assert np.array_equal(b[2], b[2].T)
    assert np.array_equal(b[3], b[4].T)
    offs = np.concatenate([[0], np.cumsum(nw[keys[:, 0]] * nw[keys[:, 1]])])
    flat = synth.d_fill(keys, offs[:-1], offs[-1], s.pos, s.cell, nw)
    for k in range(len(keys)):
        assert np.array_equal(flat[offs[k]:offs[k + 1]].reshape(b[k].shape), b[k])


def test_v_grid_matches_pointwise():
    params = synth.plane_wave_params()
    grid = (12, 10, 14)
    V = synth.v_grid(grid, params).numpy()
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in grid], indexing="ij"), -1).reshape(-1, 3)
    assert np.allclose(V.reshape(-1), synth.v_at(idx, grid, params), atol=1e-13, rtol=0)
    assert abs(V.mean()) < 1e-12  # each cosine has a non-zero integer wave vector resolved by the grid


def test_d_fill_torch_matches_numpy():
    import oracle
    s = synth.random_cell(5)  # C/H/O: rectangular and square blocks, mirrors, self-mirrors
    o = oracle.Oracle(s)
    Dn = synth.d_fill(o.blocks, o.offsets[:-1], o.n_values, s.pos, s.cell, s.nw())
    Dt = synth.d_fill_torch(o.blocks, o.offsets[:-1], o.n_values, s.pos, s.cell, s.nw(), "cpu").numpy()
    assert np.max(np.abs(Dn - Dt)) <= 1e-15 * np.max(np.abs(Dn))
    # symmetric on the pattern
    idx = o.block_index()
    for b, k in enumerate(o.blocks[:200]):
        m = idx[(k[1], k[0], -k[2], -k[3], -k[4])]
        assert np.array_equal(o.block(Dn, b), o.block(Dn, m).T)
