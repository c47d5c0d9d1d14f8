"""Pins of the oracle's Bloch sum H(T) -> H(k) (the step after the grid integrals):
Hermiticity, periodicity in k, the real k = 0 sum, and the inverse transform over a
k grid finer than the pattern's image range, which must return every block and zero
for pairs outside the pattern."""
import itertools

import numpy as np

import oracle
import synth


def _case():
    s = synth.diamond(grid=(18, 18, 18))
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    return s, o, o.vlocal(V)


def test_fold_hermitian_and_periodic():
    s, o, H = _case()
    for kf in [(0.1, 0.2, 0.3), (0.5, 0.0, 0.25)]:
        Hk = o.fold_k(H, kf)
        assert np.max(np.abs(Hk - Hk.conj().T)) < 1e-12 * np.max(np.abs(Hk))
        Hk2 = o.fold_k(H, np.array(kf) + np.array([1.0, -2.0, 3.0]))
        assert np.max(np.abs(Hk - Hk2)) < 1e-10 * np.max(np.abs(Hk))
    H0 = o.fold_k(H, (0, 0, 0))
    assert np.max(np.abs(H0.imag)) == 0.0
    # k = 0: every block of a pair added without phase
    off = np.concatenate([[0], np.cumsum(o.nw)])
    I, J = 0, 1
    ref = sum(o.block(H, b) for b in range(len(o.blocks)) if o.blocks[b, 0] == I and o.blocks[b, 1] == J)
    assert np.max(np.abs(H0[off[I]:off[I + 1], off[J]:off[J + 1]].real - ref)) < 1e-12


def test_fold_inverse_transform():
    s, o, H = _case()
    tmax = int(np.max(np.abs(o.blocks[:, 2:5])))
    M = 2 * tmax + 1  # finer than the image range: no aliasing
    off = np.concatenate([[0], np.cumsum(o.nw)])
    ks = [np.array(k, dtype=np.float64) / M for k in itertools.product(range(M), repeat=3)]
    folds = [o.fold_k(H, k) for k in ks]
    idx = o.block_index()
    rng = np.random.default_rng(0)
    n_atoms = len(o.nw)
    for _ in range(12):
        I, J = int(rng.integers(n_atoms)), int(rng.integers(n_atoms))
        t = tuple(int(x) for x in rng.integers(-tmax, tmax + 1, 3))
        back = sum(np.exp(-2j * np.pi * float(k @ np.array(t))) * Hk[off[I]:off[I + 1], off[J]:off[J + 1]]
                   for k, Hk in zip(ks, folds)) / len(ks)
        b = idx.get((I, J) + t)
        ref = o.block(H, b) if b is not None else np.zeros((o.nw[I], o.nw[J]))
        assert np.max(np.abs(back - ref)) < 1e-12 * max(1.0, np.max(np.abs(H)))
