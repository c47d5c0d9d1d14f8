"""Host-side logic of bench.py: the per-call form specification and the launch count."""
import pytest

import bench


def test_one_form_for_every_call():
    assert bench.parse_forms("fp16x4") == {"vlocal": "fp16x4", "rho": "fp16x4", "force": "fp16x4"}


def test_one_form_per_call():
    f = bench.parse_forms("vlocal=fp16x4,rho=fp16x4,force=fp16x3")
    assert f == {"vlocal": "fp16x4", "rho": "fp16x4", "force": "fp16x3"}
    assert bench.parse_forms(bench.DEFAULT_FORMS) == f


@pytest.mark.parametrize("spec", ["vlocal=fp16x4,rho=fp16x4", "vlocal=fp16x4,rho=fp16x4,forces=fp16x3"])
def test_incomplete_or_unknown_call_is_rejected(spec):
    with pytest.raises(SystemExit):
        bench.parse_forms(spec)


@pytest.mark.parametrize("spec,n", [
    ("fp64", 6),      # vlocal + mirror, rho + empty-brick fill, force + finalize
    ("fp32", 6),
    ("fp16x3", 8),    # + the D format before the rho and force kernels
    ("fp16x4", 11),   # + the H normalisation and the D row maxima before each D format
    ("vlocal=fp16x4,rho=fp16x4,force=fp16x3", 10),
])
def test_launches_per_step(spec, n):
    assert bench.launches_per_step(bench.parse_forms(spec)) == n
