"""The benchmark's end-to-end step through the public API (inputs in pinned host memory,
copies inside every step): the variant that overlaps each step's copies with the neighbouring
steps' compute (two copy streams, two sets of device buffers, ordered by events) downloads the
same H, rho, F, sigma and E as the variant with the copies in line."""
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_overlapped_copies_match_inline(cuda):
    import torch
    import bench
    from paper_2409_09399_gb300 import gint
    s = synth.tbg(2)
    g = gint.from_system(s, precision="fp16x4", brick=(8, 8, 8))
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device="cuda")
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, s.pos, s.cell, s.nw(), "cuda")

    def use(call):
        g.set_precision("fp16x3" if call == "force" else "fp16x4")

    runner = bench.EndToEnd(g, V, D, use, torch.cuda.current_stream(), torch.device("cuda"))
    runner.inline(1)
    ref = [t.clone() for t in (runner.Hh, runner.rhoh, runner.Fh, runner.sigh, runner.Eh)]
    for t in (runner.Hh, runner.rhoh, runner.Fh, runner.sigh, runner.Eh):
        t.fill_(float("nan"))
    ms = runner.overlapped(3)
    g.sync()
    got = (runner.Hh, runner.rhoh, runner.Fh, runner.sigh, runner.Eh)
    for name, a, b in zip(("H", "rho", "F", "sigma", "E"), got, ref):
        scale = float(b.abs().max())
        err = float((a - b).abs().max())
        assert err <= 1e-12 * max(scale, 1e-30), (name, err, scale)
    print(f"overlapped end-to-end step: {ms:.2f} ms on TBG m=2")
