"""Failure detection through the C ABI, made on the host or by a bounded wait (no GPU fault):

* an allocation that fails (the library's test hook makes the n-th device allocation fail
  the way cudaMalloc fails on a full device): gint_setup returns GINT_ERR_OOM and releases
  what it had allocated;
* new positions that need a different pair pattern with the pattern kept:
  GINT_ERR_PATTERN_MISMATCH, the handle unchanged;
* bricks beyond the tensor-core limits: GINT_ERR_UNSUPPORTED from gint_check and from every
  compute call, nothing enqueued;
* a tensor-core pipeline wait that runs out (a wait limit of one poll, far below the time the
  producers need): the kernel stops, gint_sync reports GINT_ERR_TIMEOUT, and the next call with
  the default limit gives correct results on the same context.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _status(fn):
    from paper_2409_09399_gb300 import gint
    try:
        fn()
    except gint.GintError as e:
        return e.status, str(e)
    return 0, ""


def test_setup_out_of_memory_releases_everything(cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.diamond(grid=(20, 20, 20), species=synth.make_species("O", "SZP"))
    g = gint.from_system(s)  # loads the library's modules before memory is measured
    g.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n_fail = 0
    for n in range(1, 200):
        gint.debug_fail_alloc(n)
        st, msg = _status(lambda: gint.from_system(s).close())
        gint.debug_fail_alloc(0)
        if st == 0:
            break
        assert st == 3, (n, st, msg)  # GINT_ERR_OOM
        assert "out of memory" in msg, msg
        n_fail += 1
    assert n_fail >= 10  # every allocation of the set-up was made to fail once
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    print(f"{n_fail} failed set-ups; device free memory before {free0 / 2**20:.1f} MiB, after {free1 / 2**20:.1f} MiB")
    assert free1 >= free0 - (2 << 20)  # nothing kept beyond allocator granularity
    # the library still works after the failures
    g = gint.from_system(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    H = g.vlocal(V)
    g.sync()
    assert torch.isfinite(H).all()


def test_update_positions_pattern_mismatch(cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.diamond(grid=(20, 20, 20), species=synth.make_species("O", "SZP"))
    g = gint.from_system(s)
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    H0 = g.vlocal(V).clone()
    nb0 = g.n_blocks
    far = s.pos.copy()
    far[0] += np.array([2.1, -1.7, 1.3])  # new pairs come within the cutoff sum
    st, msg = _status(lambda: g.update_positions(far, keep_pattern=True))
    assert st == 4, (st, msg)  # GINT_ERR_PATTERN_MISMATCH
    assert g.n_blocks == nb0
    H1 = g.vlocal(V)
    g.sync()
    assert torch.equal(H0, H1) or float((H0 - H1).abs().max()) < 1e-13 * float(H0.abs().max())
    # without keeping the pattern the update goes through and reports the change
    assert g.update_positions(far, keep_pattern=False) is True
    g2 = gint.from_system(s, pos=far)
    assert g.n_blocks == g2.n_blocks
    H2, H3 = g.vlocal(V), g2.vlocal(V)
    g.sync()
    assert float((H2 - H3).abs().max()) < 1e-13 * float(H3.abs().max())


def test_unsupported_bricks_on_tensor_cores(cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.diamond()  # dense: an 8^3 brick meets far more than 64 atom images
    g = gint.from_system(s, precision="fp16x4", brick=(8, 8, 8))
    assert not g.supported()
    L = gint.load()
    assert L.gint_check(g._h) == 6
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    H = torch.full((g.n_values,), 7.0, dtype=torch.float64, device="cuda")
    for call in (lambda: g.vlocal(V, H), lambda: g.rho(D), lambda: g.force_stress(V, D),
                 lambda: g.energy_grads(V, D)):
        st, msg = _status(call)
        assert st == 6, (st, msg)  # GINT_ERR_UNSUPPORTED
        assert "use smaller bricks" in msg
    g.sync()
    assert float(H.min()) == 7.0  # nothing was enqueued on H (not even the zero fill)


@pytest.mark.parametrize("call", ["vlocal", "rho", "force"])
def test_pipeline_wait_timeout(call, cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.tbg(2)
    g = gint.from_system(s, precision="fp16x4", brick=(8, 8, 8))
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")
    run = {"vlocal": lambda: g.vlocal(V), "rho": lambda: g.rho(D), "force": lambda: g.force_stress(V, D)[0]}[call]
    ref = run().clone()
    g.sync()
    g.set_wait_limit(1)
    run()
    st, msg = _status(g.sync)
    assert st == 5, (st, msg)  # GINT_ERR_TIMEOUT
    # the context is still usable: the default limit gives the reference results again
    g.set_wait_limit(0)
    out = run()
    g.sync()
    scale = float(ref.abs().max())
    assert float((out - ref).abs().max()) <= 1e-12 * scale
