"""Tensor-core (tcgen05) forms against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

_cache = {}


def diamond_case():
    if "diamond" not in _cache:
        s = synth.diamond()
        o = oracle.Oracle(s)
        V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
        _cache["diamond"] = (s, o, V, o.vlocal(V))
    return _cache["diamond"]


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
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
    assert err < 5e-5


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
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
    assert err < 5e-5
