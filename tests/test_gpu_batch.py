"""Batched launch over many uneven cells (gint_batch_*): one CUDA graph holding
every cell's H^V, rho and force/stress calls, brick shapes from the autotuner,
per-cell error of the mixed form against the FP64 form, and the FP64 batch
against the oracle on the smallest cells."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N_CELLS = 12


def _cells():
    return [synth.random_cell(i) for i in range(N_CELLS)]


def _run_batch(b, systems, Vs, Ds):
    import torch
    H = [torch.empty(h.n_values, dtype=torch.float64, device="cuda") for h in b.handles]
    rho = [torch.empty(h.grid, dtype=torch.float64, device="cuda") for h in b.handles]
    F = [torch.empty((h.n_atoms, 3), dtype=torch.float64, device="cuda") for h in b.handles]
    sig = [torch.empty((3, 3), dtype=torch.float64, device="cuda") for h in b.handles]
    E = [torch.empty(1, dtype=torch.float64, device="cuda") for h in b.handles]
    b.run(Vs, Ds, H, rho, F, sig, E)
    torch.cuda.synchronize()
    for h in b.handles:
        h.sync()
    return H, rho, F, sig, E


def test_batch_mixed_vs_single_and_fp64(cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    from paper_2409_09399_gb300.batch import GintBatch
    systems = _cells()
    b = GintBatch(systems, precision="fp16x3", brick="auto", candidates=((8, 8, 8), (4, 4, 8), (4, 4, 4)), sample=3)
    print("autotuner ranking", b.ranking, "bricks", b.bricks)
    Vs, Ds = [], []
    for s, h in zip(systems, b.handles):
        blocks, offsets = h.pattern()
        Vs.append(synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda"))
        Ds.append(synth.d_fill_torch(blocks, offsets[:-1], h.n_values, s.pos, s.cell, s.nw(), "cuda"))
    H, rho, F, sig, E = _run_batch(b, systems, Vs, Ds)
    # a second launch with new output buffers re-captures; with the same ones it replays
    H2, rho2, F2, sig2, E2 = _run_batch(b, systems, Vs, Ds)
    # time the graph (replays) against the same calls made one cell at a time
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(3):
        b.run(Vs, Ds, H2, rho2, F2, sig2, E2)
    e.record()
    torch.cuda.synchronize()
    t_graph = a.elapsed_time(e) / 3
    a.record()
    for _ in range(3):
        for i, h in enumerate(b.handles):
            h.vlocal(Vs[i], H2[i])
            h.rho(Ds[i], rho2[i])
            h.force_stress(Vs[i], Ds[i], out=(F2[i], sig2[i], torch.empty((h.n_atoms, 3, 3), dtype=torch.float64,
                                                                          device="cuda"), E2[i]))
    e.record()
    torch.cuda.synchronize()
    t_cells = a.elapsed_time(e) / 3
    print(f"batch of {len(systems)} cells: one graph launch {t_graph:.2f} ms, cell by cell {t_cells:.2f} ms")
    worst = {"H": 0.0, "rho": 0.0, "F": 0.0}
    for i, (s, h) in enumerate(zip(systems, b.handles)):
        # same kernels one cell at a time: equal up to the order of FP64 atomics
        Hs = h.vlocal(Vs[i])
        rs = h.rho(Ds[i])
        Fs, ss, _, Es = h.force_stress(Vs[i], Ds[i])
        h.sync()
        for got in (H[i], H2[i]):
            assert torch.allclose(got, Hs, rtol=0, atol=1e-12 * float(Hs.abs().max()))
        for got in (rho[i], rho2[i]):
            assert torch.allclose(got, rs, rtol=0, atol=1e-12 * float(rs.abs().max()))
        assert torch.allclose(F[i], Fs, rtol=0, atol=1e-12 * max(1.0, float(Fs.abs().max())))
        assert torch.allclose(sig[i], ss, rtol=0, atol=1e-12)
        assert abs(float(E[i]) - float(Es)) <= 1e-12 * abs(float(Es))
        # per-cell error against the FP64 form
        g64 = gint.from_system(s, precision="fp64", brick=b.bricks[i])
        H64 = g64.vlocal(Vs[i])
        r64 = g64.rho(Ds[i])
        F64, s64, _, E64 = g64.force_stress(Vs[i], Ds[i])
        g64.sync()
        eH = float((H[i] - H64).abs().max())
        eR = float((rho[i] - r64).abs().max() / r64.abs().max())
        eF = float((F[i] - F64).abs().max())
        print(f"cell {i}: {s.n_atoms} atoms grid {s.grid[0]} brick {b.bricks[i]}: H {eH:.2e} rho {eR:.2e} F {eF:.2e}")
        worst["H"] = max(worst["H"], eH)
        worst["rho"] = max(worst["rho"], eR)
        worst["F"] = max(worst["F"], eF)
        g64.close()
    print("worst per-cell error vs FP64:", worst)
    # fp16x3 meets the force target (F <= 1e-5 Ha/bohr); H and rho carry its accumulation bias
    assert worst["H"] < 5e-5 and worst["rho"] < 1e-4 and worst["F"] < 1e-5


def test_batch_fp64_vs_oracle(cuda):
    """FP64 cells through the batch graph against the oracle (the two smallest grids)."""
    import torch
    from paper_2409_09399_gb300.batch import GintBatch
    systems = _cells()
    order = np.argsort([np.prod(s.grid) for s in systems])[:2]
    sel = [systems[i] for i in order]
    b = GintBatch(sel, precision="fp64", brick=(4, 4, 4))
    Vs = [synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda") for s in sel]
    Ds = []
    for s, h in zip(sel, b.handles):
        blocks, offsets = h.pattern()
        Ds.append(synth.d_fill_torch(blocks, offsets[:-1], h.n_values, s.pos, s.cell, s.nw(), "cuda"))
    H, rho, F, sig, E = _run_batch(b, sel, Vs, Ds)
    for i, s in enumerate(sel):
        o = oracle.Oracle(s)
        Vn = Vs[i].cpu().numpy()
        Dn = o.d_fill()
        H_ref = o.vlocal(Vn)
        r_ref = o.rho(Dn)
        F_ref, W_ref = o.force(Vn, Dn)
        eH = np.max(np.abs(H[i].cpu().numpy() - H_ref)) / np.max(np.abs(H_ref))
        eR = np.max(np.abs(rho[i].cpu().numpy() - r_ref)) / np.max(np.abs(r_ref))
        eF = np.max(np.abs(F[i].cpu().numpy() - F_ref)) / max(1.0, np.max(np.abs(F_ref)))
        print(f"fp64 cell {s.name}: H {eH:.2e} rho {eR:.2e} F {eF:.2e}")
        assert eH < 1e-11 and eR < 1e-11 and eF < 1e-10


# per-result bounds of the queue path against the oracle.  These cells have coarse grids
# (0.47-0.63 bohr against the TBG workloads' 0.157), where the exact form's H error is set by
# the FP32 orbital values (|r| in FP32, about 3e-7 relative per value) and averages out over
# fewer points: bounded by 5e-7 x max(1, max|H|) as in the other coarse-grid tests.
QUEUE_TOL = {"fp16x4": {"H": 5e-7, "rho": 1e-6, "F": 1e-5, "sigma": 1e-5},
             "fp16x3": {"H": 5e-5, "rho": 1e-4, "F": 1e-5, "sigma": 1e-4}}
QUEUE_CELLS = (5, 21, 3, 15, 7)  # two dense cells (0.09 atoms per cubic angstrom), 20-81 atoms, grids 24^3-39^3
_oracle_cache = {}


def _oracle_cell(i):
    if i not in _oracle_cache:
        s = synth.random_cell(i)
        o = oracle.Oracle(s)
        V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
        D = o.d_fill()
        F, W = o.force(V, D)
        _oracle_cache[i] = (s, o, V, D, o.vlocal(V), o.rho(D), F, W, o.energy(V, D))
    return _oracle_cache[i]


@pytest.mark.parametrize("precision", ["fp16x4", "fp16x3"])
def test_batch_queue_vs_oracle(precision, cuda):
    """The multi-cell persistent queue (one launch per call over every cell's bricks) against the
    oracle, element by element, for uneven C/H/O cells."""
    import torch
    from paper_2409_09399_gb300.batch import GintBatch, brick_for
    cases = [_oracle_cell(i) for i in QUEUE_CELLS]
    systems = [c[0] for c in cases]
    order = ((4, 4, 8), (4, 4, 4), (2, 4, 4), (2, 2, 4), (2, 2, 2))
    bricks = [brick_for(s, precision, order) for s in systems]
    b = GintBatch(systems, precision=precision, brick=bricks)
    # every cell takes the same tensor-core form and passes its limits: the batch runs the
    # (cell, brick) queue, not per-cell calls
    assert all(h.supported() for h in b.handles)
    Vs = [torch.from_numpy(c[2]).cuda() for c in cases]
    Ds = [torch.from_numpy(c[3]).cuda() for c in cases]
    for h, c in zip(b.handles, cases):
        blocks, offsets = h.pattern()
        assert np.array_equal(blocks, c[1].blocks) and np.array_equal(offsets, c[1].offsets)
    H, rho, F, sig, E = _run_batch(b, systems, Vs, Ds)
    tol = QUEUE_TOL[precision]
    for i, (s, o, V, D, H_ref, r_ref, F_ref, W_ref, E_ref) in enumerate(cases):
        eH = float(np.max(np.abs(H[i].cpu().numpy() - H_ref)))
        eR = float(np.max(np.abs(rho[i].cpu().numpy() - r_ref)) / np.max(np.abs(r_ref)))
        eF = float(np.max(np.abs(F[i].cpu().numpy() - F_ref)))
        s_ref = -W_ref.sum(0) / o.omega
        eS = float(np.max(np.abs(sig[i].cpu().numpy() - s_ref)))
        # E = sum V rho dV cancels (V and rho change sign): relative to sum |V rho| dV
        eE = abs(float(E[i]) - E_ref) / (float(np.sum(np.abs(V * r_ref))) * o.dV)
        print(f"{precision} cell {QUEUE_CELLS[i]} ({s.n_atoms} atoms, grid {s.grid[0]}^3, brick {bricks[i]}): "
              f"H {eH:.2e} (max {np.abs(H_ref).max():.2f}) rho {eR:.2e} F {eF:.2e} sigma {eS:.2e} E {eE:.2e}")
        assert eH < tol["H"] * max(1.0, float(np.max(np.abs(H_ref))))
        assert eR < tol["rho"]
        assert eF < tol["F"] * max(1.0, float(np.max(np.abs(F_ref))))
        assert eS < tol["sigma"] * max(1.0, float(np.max(np.abs(s_ref))))
        assert eE < tol["rho"]
