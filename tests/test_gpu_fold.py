"""Bloch sum H(T) -> H(k) on the GPU (gint_fold_k) against the oracle's fold_k."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kf", [(0.0, 0.0, 0.0), (0.125, -0.25, 0.375), (0.5, 0.5, 0.0)])
def test_fold_diamond_vs_oracle(kf, cuda):
    """FP64 H from the GPU, folded on the GPU, against the oracle's H folded by the oracle."""
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.diamond(grid=(18, 18, 18))
    o = oracle.Oracle(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    g = gint.from_system(s, precision="fp64")
    H = g.vlocal(torch.from_numpy(V).cuda())
    Hk = g.fold_k(H, kf)
    g.sync()
    ref = o.fold_k(o.vlocal(V), kf)
    err = np.max(np.abs(Hk.cpu().numpy() - ref)) / np.max(np.abs(ref))
    print(f"diamond k={kf}: |Hk - Hk_ref| / max = {err:.2e}")
    assert err < 1e-11


def test_fold_tbg_same_input(cuda):
    """The kernel alone: GPU fold of the GPU H against the oracle's fold of the same H (TBG m=2),
    with a padded leading dimension; and the time of one fold at TBG m=5 (N = 4732)."""
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.tbg(2)
    o = oracle.Oracle(s)
    g = gint.from_system(s, precision="fp64", brick=(8, 8, 8))
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    H = g.vlocal(V)
    n = g.n_orbitals
    Hk_pad = torch.full((n, n + 7), complex(7.0, -3.0), dtype=torch.complex128, device="cuda")
    kf = (0.3, -0.1, 0.0)
    g.fold_k(H, kf, Hk=Hk_pad)
    g.sync()
    ref = o.fold_k(H.cpu().numpy(), kf)
    got = Hk_pad.cpu().numpy()
    err = np.max(np.abs(got[:, :n] - ref)) / np.max(np.abs(ref))
    assert err < 1e-13
    assert np.all(got[:, n:] == 0)  # the whole leading-dimension stride is written
    s5 = synth.tbg(5)
    g5 = gint.from_system(s5, precision="fp16x3", brick=(8, 8, 8))
    H5 = g5.vlocal(synth.v_grid(s5.grid, synth.plane_wave_params(), device="cuda"))
    Hk5 = torch.empty((g5.n_orbitals, g5.n_orbitals), dtype=torch.complex128, device="cuda")
    g5.fold_k(H5, kf, Hk=Hk5)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        g5.fold_k(H5, kf, Hk=Hk5)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    gb = (g5.n_values * 8 + g5.n_orbitals ** 2 * 16) / 1e9
    print(f"fold at TBG m=5: N = {g5.n_orbitals}, {ms:.2f} ms, {gb / (ms / 1e3):.0f} GB/s (H read + H(k) written)")
    assert np.all(np.abs(Hk5.cpu().numpy() - Hk5.cpu().numpy().conj().T) < 1e-9)
