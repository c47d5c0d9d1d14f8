"""The grid decomposition's library side on one GPU: the bricks of a TBG cell dealt to three
slabs by cost (the partition the ranks of a multi-GPU run take), each slab computed on its own
(gint_select_bricks); the slabs' H^V, forces, stress and energy add up to the whole cell's and
their rho slabs tile its rho (Section 2.3.1, Fig. 5).  The reductions between ranks are
checked on CPU ranks (test_shard_dist.py)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp16x4"])
def test_slabs_add_up_to_the_cell(precision, cuda):
    import torch
    from paper_2409_09399_gb300 import gint, shard
    s = synth.tbg(2)
    g = gint.from_system(s, precision=precision, brick=(8, 8, 8))
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    H0 = g.vlocal(V).clone()
    rho0 = g.rho(D).clone()
    F0, sig0, _, E0 = [t.clone() for t in g.force_stress(V, D)]
    g.sync()
    brick = g.info()["brick"]
    nb = shard.bricks_per_axis(s.grid, brick)
    loads = g.brick_loads()
    assert loads.shape == (int(np.prod(nb)),) and loads.sum() == g.info()["n_brick_atoms"]
    parts = shard.partition_slabs(shard.brick_costs(loads), nb, 3)
    costs = shard.brick_costs(loads)
    print("slab costs", [float(costs[p].sum() / costs.sum()) for p in parts])
    H = torch.zeros_like(H0)
    F = torch.zeros_like(F0)
    sig = torch.zeros_like(sig0)
    E = torch.zeros_like(E0)
    rho = torch.full_like(rho0, float("nan"))
    for p in parts:
        g.select_bricks(p)
        H += g.vlocal(V)
        g.rho(D, rho)  # writes this slab's points only
        Fp, sp, _, Ep = g.force_stress(V, D)
        F += Fp
        sig += sp
        E += Ep
        g.sync()
        covered = torch.from_numpy(shard.brick_point_mask(p, s.grid, brick)).cuda()
        assert not torch.isnan(rho[covered]).any()
    g.select_bricks(None)
    assert not torch.isnan(rho).any()
    tol = 1e-12
    eH = float((H - H0).abs().max() / H0.abs().max())
    eR = float((rho - rho0).abs().max() / rho0.abs().max())
    eF = float((F - F0).abs().max() / max(1.0, float(F0.abs().max())))
    eS = float((sig - sig0).abs().max() / max(1e-30, float(sig0.abs().max())))
    eE = float((E - E0).abs().max() / E0.abs().max())
    print(f"{precision}: slabs vs whole cell: H {eH:.1e} rho {eR:.1e} F {eF:.1e} sigma {eS:.1e} E {eE:.1e}")
    assert eH < tol and eR < tol and eF < tol and eS < 1e-10 and eE < 1e-10
    # with every brick selected again the handle gives the whole-cell results
    H1 = g.vlocal(V)
    g.sync()
    assert float((H1 - H0).abs().max() / H0.abs().max()) < tol


def test_sharded_step_single_rank_equals_the_cell(cuda):
    """shard.sharded_step with one rank needs no process group and returns the whole cell."""
    from paper_2409_09399_gb300 import gint, shard
    s = synth.tbg(2)
    g = gint.from_system(s, precision="fp64", brick=(8, 8, 8))
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    H0 = g.vlocal(V).clone()
    _, _, _, E0 = g.force_stress(V, D)
    E0 = E0.clone()
    H, (v0, v1), rho, F, sigma, E = shard.sharded_step(g, 0, 1, V, D)
    g.sync()
    assert (v0, v1) == (0, g.n_values)
    assert float((H - H0).abs().max() / H0.abs().max()) < 1e-12
    assert abs(float(E) - float(E0)) < 1e-10 * abs(float(E0))
