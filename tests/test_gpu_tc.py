"""Tensor-core (tcgen05) forms against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

_cache = {}

# Stated accuracy of each form: max abs for H and F, normwise for rho.  The
# three-product forms carry the bias of the tensor-core FP32 accumulation; the
# exact form (fp16x4) meets the target accuracy H <= 1e-7 Ha, rho <= 1e-6
# (normwise), F <= 1e-5 Ha/bohr.
TOL = {
    "fp16x3": {"H": 5e-5, "rho": 1e-4, "F": 1e-5, "sigma": 1e-4},
    "bf16x3": {"H": 5e-5, "rho": 1e-4, "F": 1e-4, "sigma": 1e-4},
    "fp16x4": {"H": 1e-7, "rho": 1e-6, "F": 1e-5, "sigma": 1e-6},
}


def diamond_case():
    if "diamond" not in _cache:
        s = synth.diamond()
        o = oracle.Oracle(s)
        V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
        _cache["diamond"] = (s, o, V, o.vlocal(V))
    return _cache["diamond"]


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "fp16x4"])
@pytest.mark.parametrize("brick", [(3, 3, 4), (4, 3, 3)])
def test_tc_vlocal_diamond_full(precision, brick, cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s, o, V, H_ref = diamond_case()
    g = gint.from_system(s, precision=precision, brick=brick)
    H = g.vlocal(torch.from_numpy(V).cuda())
    g.sync()
    err = np.max(np.abs(H.cpu().numpy() - H_ref))
    print(f"{precision} brick {brick}: max |H - H_ref| = {err:.3e} (max |H_ref| {np.abs(H_ref).max():.3f})")
    # split 16-bit operands with FP32 accumulation in tensor memory: the error is
    # set by the accumulator (~2^-23 |partial| per accumulation step)
    assert err < TOL[precision]["H"]


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "fp16x4"])
def test_tc_vlocal_tbg_sampled(precision, cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.tbg(2)
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    g = gint.from_system(s, precision=precision, brick=(8, 8, 8))
    H = g.vlocal(torch.from_numpy(V).cuda()).cpu().numpy()
    g.sync()
    blocks, offsets = g.pattern()
    rng = np.random.default_rng(7)
    # on-site blocks (largest elements) and random blocks
    onsite = np.nonzero((blocks[:, 0] == blocks[:, 1]) & (blocks[:, 2:] == 0).all(1))[0][:8]
    sel = np.concatenate([onsite, rng.choice(len(blocks), 40, replace=False)])
    ref = o.vlocal_blocks(V, blocks[sel])
    err = 0.0
    for k, b in enumerate(sel):
        got = H[offsets[b]:offsets[b + 1]].reshape(ref[k].shape)
        err = max(err, np.max(np.abs(got - ref[k])))
    print(f"{precision} TBG m=2: max |H - H_ref| over {len(sel)} blocks = {err:.3e}")
    assert err < TOL[precision]["H"]


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "fp16x4"])
def test_tc_rho_force_diamond(precision, cuda):
    """rho and force/stress on the tensor cores against the oracle (diamond, 3x3x4 bricks)."""
    import torch
    from paper_2409_09399_gb300 import gint
    s, o, V, _ = diamond_case()
    if "diamond_rf" not in _cache:
        D = o.d_fill()
        F, W = o.force(V, D)
        _cache["diamond_rf"] = (D, o.rho(D), F, W)
    D_or, rho_ref, F_ref, W_ref = _cache["diamond_rf"]
    g = gint.from_system(s, precision=precision, brick=(3, 3, 4))
    blocks, offsets = g.pattern()
    assert np.array_equal(blocks, o.blocks)
    D = torch.from_numpy(D_or).cuda()
    Vt = torch.from_numpy(V).cuda()
    rho = g.rho(D)
    F, sigma, vir, E = g.force_stress(Vt, D)
    g.sync()
    e_rho = np.max(np.abs(rho.cpu().numpy() - rho_ref)) / np.max(np.abs(rho_ref))
    e_F = np.max(np.abs(F.cpu().numpy() - F_ref))
    sig_ref = -W_ref.sum(0) / o.omega
    e_sig = np.max(np.abs(sigma.cpu().numpy() - sig_ref))
    print(f"{precision}: rho normwise {e_rho:.3e}  F abs {e_F:.3e} (max {np.abs(F_ref).max():.3f})  sigma abs {e_sig:.3e}")
    tol = TOL[precision]
    assert e_rho < tol["rho"]
    assert e_F < tol["F"]
    assert e_sig < tol["sigma"]


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "fp16x4"])
def test_tc_rho_force_tbg_sampled(precision, cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.tbg(2)
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    g = gint.from_system(s, precision=precision, brick=(8, 8, 8))
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    Vt = torch.from_numpy(V).cuda()
    rho = g.rho(D).cpu().numpy()
    F, sigma, vir, E = g.force_stress(Vt, D)
    g.sync()
    rng = np.random.default_rng(3)
    D_or = o.d_fill()
    idx = np.stack([rng.integers(0, n, 2000) for n in s.grid], 1)
    # points near the layers, where rho is not zero
    idx[:, 2] = rng.integers(100, 180, 2000)
    r_ref = o.rho_points(D_or, idx)
    r_got = rho[idx[:, 0], idx[:, 1], idx[:, 2]]
    e_rho = np.max(np.abs(r_got - r_ref)) / np.max(np.abs(r_ref))
    atoms = np.array([0, 17, 40, 75])
    F_ref, _ = o.force(V, D_or, atoms=atoms)
    e_F = np.max(np.abs(F.cpu().numpy()[atoms] - F_ref))
    print(f"{precision} TBG m=2: rho normwise {e_rho:.3e}  F abs {e_F:.3e} (max {np.abs(F_ref).max():.3f})")
    assert e_rho < TOL[precision]["rho"]
    assert e_F < TOL[precision]["F"]


def test_tc_exact_accumulate(cuda):
    """Exact form with accumulate = 1 (normalisation in the FP64 epilogue) adds the same H."""
    import torch
    from paper_2409_09399_gb300 import gint
    s, o, V, H_ref = diamond_case()
    g = gint.from_system(s, precision="fp16x4", brick=(3, 3, 4))
    Vt = torch.from_numpy(V).cuda()
    H1 = g.vlocal(Vt)
    H2 = g.vlocal(Vt, H=H1.clone(), accumulate=True)
    g.sync()
    e_acc = float((H2 - 2 * H1).abs().max())
    e_ref = float(np.max(np.abs(H2.cpu().numpy() - 2 * H_ref)))
    print(f"fp16x4 accumulate: |H2 - 2 H1| {e_acc:.2e}, |H2 - 2 H_ref| {e_ref:.2e}")
    assert e_acc < 1e-7 and e_ref < 2e-7
