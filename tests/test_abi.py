"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
symbol include/gfdtd.h declares; host-only entry points behave as documented."""
import os
import re

import numpy as np
import pytest

from paper_2304_06586_gb300 import binding as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gfdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gfdtd_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gfdtd_create", "gfdtd_set_medium", "gfdtd_add_source", "gfdtd_add_probe",
                     "gfdtd_step", "gfdtd_read_fields", "gfdtd_read_spectrum", "gfdtd_stability",
                     "gfdtd_last_error", "gfdtd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = gb.load()
    for name in _declared():
        assert hasattr(L, name), name
    # the binding marshals every declared entry point
    assert set(_declared()) <= set(gb.SIGNATURES), set(_declared()) - set(gb.SIGNATURES)


@pytest.mark.parametrize("kind", [gb.PERTURBATION, gb.MATTER])
def test_host_stability_matches_oracle_von_neumann(kind):
    from oracle import vonneumann as vn
    for S, beta, eps in [(0.5, 0.3, 4.0), (0.5, -0.45, 4.0), (0.5, 0.8, 4.0), (0.5, 0.7, 6.0),
                         (0.2, -0.3, 2.0), (0.5, 0.5, 9.0), (0.9, 0.1, 1.0)]:
        g = gb.stability(S, beta, eps, 1.0, kind)
        ref = vn.max_growth(S, beta, eps, 1.0, kind=kind, n_theta=4096)
        assert abs(g - ref) < 1e-9, (S, beta, eps, g, ref)


def test_stability_rejects_bad_arguments():
    with pytest.raises(gb.GfdtdError):
        gb.stability(0.0, 0.3, 4.0)
    with pytest.raises(gb.GfdtdError):
        gb.stability(0.5, 1.0, 4.0)


def test_create_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gb.GfdtdError):
        gb.Simulation([100], 0.5, stream=0)


def test_workloads_are_seeded_and_shaped():
    from paper_2304_06586_gb300 import workloads as w
    a = w.config3(n_inst=16)
    b = w.config3(n_inst=16)
    assert [i.nz for i in a.instances] == [i.nz for i in b.instances]
    assert all(4096 <= i.nz <= 262144 for i in a.instances)
    assert all(abs(i.beta) <= 0.8 for i in a.instances)
    for i in a.instances:
        assert np.all(np.diff(i.z) >= 20) and len(i.eps) == len(i.z) + 1
    c5 = w.config5(n_inst=2)
    assert len(c5.instances[0].eps) == 514 and len(c5.instances[0].z) == 514
