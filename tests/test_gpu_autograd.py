"""The differentiable energy (torch.autograd.Function over the hand-written kernels)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _d_on(g, s, dmap):
    """D on handle g's pattern with the values of the reference pattern (zero for new blocks)."""
    import torch
    blocks, offsets = g.pattern()
    D = np.zeros(g.n_values)
    for b, k in enumerate(blocks):
        v = dmap.get(tuple(int(x) for x in k))
        if v is not None:
            D[offsets[b]:offsets[b + 1]] = v
    return torch.from_numpy(D).cuda()


def test_energy_gradients_fp64(cuda):
    import torch
    from paper_2409_09399_gb300 import gint, energy
    s = synth.diamond(grid=(22, 20, 18), species=synth.make_species("O", "SZP"))
    o = oracle.Oracle(s)
    Vn = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    Dor = o.d_fill()
    dmap = {tuple(int(x) for x in k): o.block(Dor, b).reshape(-1).copy() for b, k in enumerate(o.blocks)}
    g = gint.from_system(s, precision="fp64")
    V = torch.from_numpy(Vn).cuda().requires_grad_(True)
    D = _d_on(g, s, dmap).requires_grad_(True)
    pos = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
    E = energy(g, pos, V, D)
    E.backward()
    # forward against the oracle
    E_ref = o.energy(Vn, Dor)
    assert abs(E.item() - E_ref) < 1e-11 * abs(E_ref)
    # dE/dV = rho dV and dE/dD = H (linear in each: exact)
    rho_ref = o.rho(Dor)
    assert np.max(np.abs(V.grad.cpu().numpy() - rho_ref * o.dV)) < 1e-11 * np.max(np.abs(rho_ref * o.dV))
    H_ref = o.vlocal(Vn)
    assert np.max(np.abs(D.grad.detach().cpu().numpy() - H_ref)) < 1e-11 * np.max(np.abs(H_ref))
    # dE/dR against central finite differences of E (new geometry, D held fixed)
    grad = pos.grad.numpy()
    delta = 1e-4
    scale = np.max(np.abs(grad))
    for I, a in [(1, 0), (5, 2), (6, 1)]:
        es = []
        for sgn in (1, -1):
            p = s.pos.copy()
            p[I, a] += sgn * delta
            gp = gint.from_system(s, precision="fp64", pos=p)
            _, _, _, Ep = gp.force_stress(V.detach(), _d_on(gp, s, dmap))
            es.append(Ep.item())
        fd = (es[0] - es[1]) / (2 * delta)
        assert abs(fd - grad[I, a]) < 1e-6 * scale, (I, a, fd, grad[I, a])


def test_strain_derivative_fp64(cuda):
    import torch
    from paper_2409_09399_gb300 import gint, energy_and_strain
    s = synth.diamond(grid=(20, 20, 20), species=synth.make_species("O", "SZP"))
    o = oracle.Oracle(s)
    Vn = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    Dor = o.d_fill()
    dmap = {tuple(int(x) for x in k): o.block(Dor, b).reshape(-1).copy() for b, k in enumerate(o.blocks)}
    g = gint.from_system(s, precision="fp64")
    V = torch.from_numpy(Vn).cuda()
    E, dEde = energy_and_strain(g, V, _d_on(g, s, dmap))
    dEde = dEde.cpu().numpy()
    eta = 1e-5
    scale = np.max(np.abs(dEde))
    for a, b in [(0, 0), (1, 2), (2, 0)]:
        es = []
        for sgn in (1, -1):
            e = np.zeros((3, 3)); e[a, b] = sgn * eta
            Fm = np.eye(3) + e
            gp = gint.from_system(s, precision="fp64", pos=s.pos @ Fm.T, cell=s.cell @ Fm.T)
            _, _, _, Ep = gp.force_stress(V, _d_on(gp, s, dmap))
            es.append(Ep.item() * (g.dV / gp.dV))  # fixed dV
        fd = (es[0] - es[1]) / (2 * eta)
        assert abs(fd - dEde[a, b]) < 1e-5 * scale, (a, b, fd, dEde[a, b])


def test_mixed_gradient_against_oracle_tbg15(cuda):
    """TBG m=15: dE/dR from the tensor-core form against the oracle on 8 random atoms."""
    import torch
    from paper_2409_09399_gb300 import gint, energy
    s = synth.tbg(15)
    g = gint.from_system(s, precision="fp16x3", brick=(8, 8, 8))
    blocks, offsets = g.pattern()
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    pos = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
    E = energy(g, pos, V, D)
    E.backward()
    o = oracle.Oracle(s)
    atoms = np.random.default_rng(5).choice(s.n_atoms, 8, replace=False)
    F_ref, _ = o.force(V.cpu().numpy(), synth.d_fill(o.blocks, o.offsets[:-1], o.n_values, s.pos, s.cell, s.nw()),
                       atoms=atoms)
    err = np.max(np.abs(-pos.grad.numpy()[atoms] - F_ref))
    print(f"TBG m=15 fp16x3 dE/dR vs oracle: {err:.2e} (max |F| {np.abs(F_ref).max():.2f})")
    assert err < 1e-5  # the stated force target (Ha/bohr)


def test_energy_moves_one_handle(cuda):
    """The autograd energy follows the positions it is given: central differences of E taken
    through the same handle (gint_update_positions, pattern kept) equal dE/dR (Eq. 4)."""
    import torch
    from paper_2409_09399_gb300 import gint, energy
    s = synth.diamond(grid=(22, 20, 18), species=synth.make_species("O", "SZP"))
    g = gint.from_system(s, precision="fp64")
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    pos = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
    E = energy(g, pos, V, D)
    E.backward()
    grad = pos.grad.numpy().copy()
    delta = 1e-4
    scale = np.max(np.abs(grad))
    for I, a in [(0, 0), (3, 1), (7, 2)]:
        es = []
        for sgn in (1, -1):
            p = torch.tensor(s.pos, dtype=torch.float64)
            p[I, a] += sgn * delta
            es.append(energy(g, p, V, D).item())
        fd = (es[0] - es[1]) / (2 * delta)
        assert abs(fd - grad[I, a]) < 1e-6 * scale, (I, a, fd, grad[I, a])
    # back at the original positions the handle gives the original energy
    assert abs(energy(g, torch.tensor(s.pos), V, D).item() - E.item()) <= 1e-12 * abs(E.item())


def _bricks_near(g, s, point, radius):
    """Ids of the bricks with a grid point within `radius` of `point` or one of its images
    (a superset: brick centre distance below radius + half the brick diagonal)."""
    B = np.array(g.info()["brick"])
    n = np.array(s.grid)
    nb = -(-n // B)
    ids = np.arange(int(np.prod(nb)))
    bc = np.stack([ids // (nb[1] * nb[2]), (ids // nb[2]) % nb[1], ids % nb[2]], 1)
    fc = (bc * B + 0.5 * (B - 1)) / n
    fa = np.linalg.solve(s.cell.T, point)
    df = fc - fa
    df -= np.round(df)
    d = np.linalg.norm(df @ s.cell, axis=1)
    half = 0.5 * np.sum(np.linalg.norm((B / n)[:, None] * s.cell, axis=1))
    return ids[d < radius + half]


def test_mixed_gradient_vs_finite_differences_tbg15(cuda):
    """TBG m=15: dE/dR of the three-product form (autograd) against central differences
    (delta = 1e-4 bohr) of the FP64 energy on 8 random atoms.  The energy change of a moved atom
    comes only from the bricks within reach of it, so each difference is taken over those
    bricks (gint_select_bricks) on one FP64 handle moved with gint_update_positions."""
    import torch
    from paper_2409_09399_gb300 import gint, energy
    s = synth.tbg(15)
    g = gint.from_system(s, precision="fp16x3", brick=(8, 8, 8))
    blocks, offsets = g.pattern()
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    pos = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
    E = energy(g, pos, V, D)
    E.backward()
    grad = pos.grad.numpy()
    g64 = gint.from_system(s, precision="fp64", brick=(8, 8, 8))
    atoms = np.random.default_rng(5).choice(s.n_atoms, 8, replace=False)
    delta = 1e-4
    worst = 0.0
    for I in atoms:
        g64.select_bricks(_bricks_near(g64, s, s.pos[I], 7.0 + 0.05))
        for a in range(3):
            es = []
            for sgn in (1, -1):
                p = s.pos.copy()
                p[I, a] += sgn * delta
                g64.update_positions(p, keep_pattern=False)
                bl, of = g64.pattern()
                Dp = synth.d_fill_torch(bl, of[:-1], g64.n_values, s.pos, s.cell, s.nw(), "cuda")  # D held fixed
                es.append(g64.energy_grads(V, Dp, want=("E",))["E"].item())
            fd = (es[0] - es[1]) / (2 * delta)
            worst = max(worst, abs(fd - grad[I, a]))
    g64.update_positions(s.pos)
    g64.select_bricks(None)
    print(f"TBG m=15 fp16x3 dE/dR vs FP64 central differences on 8 atoms: max {worst:.2e} Ha/bohr "
          f"(max |dE/dR| {np.abs(grad[atoms]).max():.2f})")
    assert worst < 1e-5  # the stated force target (Ha/bohr)
