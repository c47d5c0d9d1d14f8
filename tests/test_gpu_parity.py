"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Element by element on small systems that span many bricks and ragged brick
tails; FP64 form to 1e-11 normwise relative (max|x - x_ref| / max|x_ref|).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def normwise(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def make_case(kind):
    if kind == "diamond":
        return synth.diamond()  # 36^3 grid, 8 atoms, C DZP
    if kind == "diamond_szp":
        return synth.diamond(grid=(30, 26, 22), species=synth.make_species("O", "SZP"))
    if kind == "cell":
        return synth.random_cell(3)
    raise ValueError(kind)


_cache = {}


def oracle_results(kind):
    if kind not in _cache:
        s = make_case(kind)
        o = oracle.Oracle(s)
        V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
        D = o.d_fill()
        H = o.vlocal(V)
        rho = o.rho(D)
        F, W = o.force(V, D)
        E = float((rho * V).sum() * o.dV)
        _cache[kind] = (s, o, V, D, H, rho, F, W, E)
    return _cache[kind]


def gpu_handle(s, precision="fp64", brick=(0, 0, 0)):
    from paper_2409_09399_gb300 import gint
    return gint.from_system(s, precision=precision, brick=brick)


def gpu_d(g, s):
    import torch
    blocks, offsets = g.pattern()
    D = synth.d_fill(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw())
    return torch.from_numpy(D).cuda()


@pytest.mark.parametrize("kind", ["diamond", "diamond_szp", "cell"])
def test_pattern_identical(kind, cuda):
    s = make_case(kind)
    o = oracle.Oracle(s)
    g = gpu_handle(s)
    blocks, offsets = g.pattern()
    assert np.array_equal(blocks, o.blocks)
    assert np.array_equal(offsets, o.offsets)
    assert g.n_values == o.n_values


@pytest.mark.parametrize("kind,brick", [("diamond", (0, 0, 0)), ("diamond", (5, 7, 3)), ("diamond", (4, 4, 4)),
                                        ("diamond_szp", (8, 8, 8)), ("cell", (0, 0, 0))])
def test_fp64_parity(kind, brick, cuda):
    import torch
    s, o, V, Dor, H_ref, rho_ref, F_ref, W_ref, E_ref = oracle_results(kind)
    g = gpu_handle(s, "fp64", brick)
    Vt = torch.from_numpy(V).cuda()
    D = gpu_d(g, s)
    assert np.array_equal(D.cpu().numpy(), Dor)
    H = g.vlocal(Vt)
    rho = g.rho(D)
    F, sigma, vir, E = g.force_stress(Vt, D)
    g.sync()
    assert normwise(H.cpu().numpy(), H_ref) < TOL_FP64
    assert normwise(rho.cpu().numpy(), rho_ref) < TOL_FP64
    assert normwise(F.cpu().numpy(), F_ref) < TOL_FP64
    assert normwise(vir.cpu().numpy(), W_ref) < TOL_FP64
    sig_ref = -W_ref.sum(0) / o.omega
    assert normwise(sigma.cpu().numpy(), sig_ref) < TOL_FP64
    assert abs(E.item() - E_ref) < TOL_FP64 * abs(E_ref)


def test_fp64_accumulate_and_repeat(cuda):
    import torch
    s, o, V, Dor, H_ref, *_ = oracle_results("diamond")
    g = gpu_handle(s)
    Vt = torch.from_numpy(V).cuda()
    H1 = g.vlocal(Vt).clone()
    H2 = g.vlocal(Vt)
    g.vlocal(Vt, H=H2, accumulate=True)
    g.sync()
    assert normwise(H1.cpu().numpy(), H_ref) < TOL_FP64
    assert normwise(H2.cpu().numpy(), 2 * H_ref) < TOL_FP64


def test_trace_identity_on_gpu(cuda):
    """sum_g rho V dV (from gint_rho) = sum D . H (from gint_vlocal) = E (from gint_force_stress)."""
    import torch
    s, o, V, *_ = oracle_results("cell")
    g = gpu_handle(s)
    Vt = torch.from_numpy(V).cuda()
    D = gpu_d(g, s)
    H = g.vlocal(Vt)
    rho = g.rho(D)
    _, _, _, E = g.force_stress(Vt, D)
    g.sync()
    e1 = float((rho * Vt).sum().item() * o.dV)
    e2 = float(torch.dot(D, H).item())
    assert abs(e1 - e2) < 1e-11 * abs(e2)
    assert abs(E.item() - e2) < 1e-11 * abs(e2)


@pytest.mark.parametrize("kind", ["diamond", "cell"])
def test_fp32_form_error(kind, cuda):
    """FP32 orbital values and contractions; FP64 accumulation (mixed form)."""
    import torch
    s, o, V, Dor, H_ref, rho_ref, F_ref, W_ref, E_ref = oracle_results(kind)
    g = gpu_handle(s, "fp32")
    Vt = torch.from_numpy(V).cuda()
    D = gpu_d(g, s)
    H = g.vlocal(Vt)
    rho = g.rho(D)
    F, sigma, vir, E = g.force_stress(Vt, D)
    g.sync()
    # FP32 products summed in FP32 over one brick (<= 512 points), FP64 across
    # bricks: per-brick error ~ sqrt(512) * 2^-24 * |partial|, |partial| <= ~2
    assert np.max(np.abs(H.cpu().numpy() - H_ref)) < 1e-5
    assert normwise(rho.cpu().numpy(), rho_ref) < 1e-5
    assert np.max(np.abs(F.cpu().numpy() - F_ref)) < 1e-4
