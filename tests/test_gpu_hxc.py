"""The local potential from rho on the GPU (gint_local_potential: Hartree by FFT, LDA
exchange-correlation, FP64 energies) against the oracle's plain definitions (oracle/hxc.py),
element by element, on a skewed cell (even and odd axes, so Nyquist planes are covered) and on
the TBG m=5 grid with a seeded density that vanishes in the vacuum and changes sign."""
import math

import numpy as np
import pytest

import synth
from oracle import hxc

pytestmark = pytest.mark.gpu

SKEWED = np.array([[9.0, 0.0, 0.0], [2.5, 8.0, 0.0], [1.5, -2.0, 10.0]])


def _handle(cell, grid):
    from paper_2409_09399_gb300 import gint
    s = synth.System("hxc", np.asarray(cell, dtype=np.float64), np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32),
                     [synth.make_species("O", "SZP")], tuple(grid))
    return gint.from_system(s)


def _compare(g, rho, v_ext):
    import torch
    V_ref_h, E_h = hxc.hartree(rho, g.cell)
    eps, vxc = hxc.lda_xc(rho)
    E_xc = float(np.sum(rho * eps)) * g.dV
    V_ref = v_ext + V_ref_h + vxc
    r = torch.from_numpy(rho).cuda()
    ve = torch.from_numpy(v_ext).cuda()
    V, VH, en = g.local_potential(r, V_ext=ve, want_vh=True)
    g.sync()
    V, VH, en = V.cpu().numpy(), VH.cpu().numpy(), en.cpu().numpy()
    e_vh = np.max(np.abs(VH - V_ref_h)) / np.max(np.abs(V_ref_h))
    e_v = np.max(np.abs(V - V_ref)) / np.max(np.abs(V_ref))
    e_eh = abs(en[0] - E_h) / abs(E_h)
    e_ex = abs(en[1] - E_xc) / abs(E_xc)
    return e_vh, e_v, e_eh, e_ex


@pytest.mark.parametrize("grid", [(18, 16, 20), (17, 15, 21), (16, 19, 12)])
def test_local_potential_skewed_cell(grid, cuda):
    g = _handle(SKEWED, grid)
    f = np.meshgrid(*[np.arange(n) / n for n in grid], indexing="ij")
    rng = np.random.default_rng(3)
    rho = 0.05 + 0.02 * rng.random(grid)  # positive: every point takes the XC branch
    for m, a in (((1, 0, 2), 0.03), ((0, -2, 1), 0.02), ((3, 1, -1), 0.01)):
        rho += a * np.cos(2 * math.pi * (m[0] * f[0] + m[1] * f[1] + m[2] * f[2]) + 0.3)
    rho[0, 0, 0] = 3.0  # rs < 1 at one point: the other Perdew-Zunger branch
    v_ext = 0.1 * np.sin(2 * math.pi * f[1])
    e_vh, e_v, e_eh, e_ex = _compare(g, rho, v_ext)
    print(f"skewed {grid}: V_H {e_vh:.2e} V {e_v:.2e} E_H {e_eh:.2e} E_xc {e_ex:.2e}")
    assert e_vh < 1e-12 and e_v < 1e-12 and e_eh < 1e-12 and e_ex < 1e-12


def test_local_potential_tbg5(cuda):
    import torch
    s = synth.tbg(5)
    g = _handle(s.cell, s.grid)
    v = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    z = (np.arange(s.grid[2]) / s.grid[2]) * s.cell[2, 2]
    zc = 0.5 * s.cell[2, 2]
    envelope = np.exp(-((z - zc) / 4.0) ** 2)
    envelope[np.abs(z - zc) > 9.0] = 0.0  # vacuum: rho = 0 exactly
    rho = 0.02 * (v + 1.5) * envelope[None, None, :]  # changes sign where v < -1.5
    assert (rho < 0).any() and (rho == 0).any() and (rho > 0).any()
    e_vh, e_v, e_eh, e_ex = _compare(g, rho, np.zeros_like(rho))
    print(f"TBG m=5 grid {s.grid}: V_H {e_vh:.2e} V {e_v:.2e} E_H {e_eh:.2e} E_xc {e_ex:.2e}")
    assert e_vh < 1e-12 and e_v < 1e-12 and e_eh < 1e-12 and e_ex < 1e-12
    # time the call (FFTs included) on the resident inputs
    r = torch.from_numpy(rho).cuda()
    out = torch.empty_like(r)
    g.local_potential(r, V_out=out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        g.local_potential(r, V_out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    print(f"TBG m=5 local potential: {ms:.3f} ms per call ({s.n_grid / ms / 1e6:.2f} Gpoints/s, FFTs included)")
