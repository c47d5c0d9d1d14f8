"""gint_vlocal_static: the H^V entry point that allocates nothing.

Callers that cannot let a library call cudaMalloc (it synchronises the
device and fails once a framework's caching allocator holds the free memory)
use gint_vlocal_static, whose kernel scratch is a fixed array inside the
library.  This file is collected last so that a run stopping at the first
failure has run every other test first.  The test calls the entry point
through the C ABI twice in a row, checks that neither call changes the
device's free memory or torch's reserved memory, and compares each result
with gint_vlocal in the FP64 form.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_vlocal_static_matches_vlocal_twice(cuda):
    import torch
    from paper_2409_09399_gb300 import gint
    s = synth.diamond(grid=(30, 28, 26))
    g = gint.from_system(s, precision="fp64")
    V = synth.v_grid(s.grid, synth.plane_wave_params(), device=cuda)
    H_ref = g.vlocal(V)
    g.sync()
    L = gint.load()
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    ref = H_ref.cpu().numpy()
    scale = np.max(np.abs(ref))
    outs = [torch.full((g.n_values,), float("nan"), dtype=torch.float64, device=cuda) for _ in range(2)]
    torch.cuda.synchronize()
    # the call's defining property: no device memory is taken, neither from the device (free
    # bytes) nor from torch's caching allocator (reserved bytes)
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for call, H in enumerate(outs):
        st = L.gint_vlocal_static(g._h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(H.data_ptr()), stream)
        assert st == 0, L.gint_last_error()
        g.sync()
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0, call
    for call, H in enumerate(outs):
        err = np.max(np.abs(H.cpu().numpy() - ref)) / scale
        assert err < 1e-11, (call, err)


def test_vlocal_static_rejects_null(cuda):
    from paper_2409_09399_gb300 import gint
    L = gint.load()
    assert L.gint_vlocal_static(None, None, None, None) == 1
