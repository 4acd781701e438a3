"""Every precision tier against the FP64 oracle at full size: the moving-gradient
workload (stable variant: linear eps ramp 1 -> 2 over 2^18 of 2^20 cells, v =
0.7c, S = 0.5; Fig. 8 geometry scaled up) after 20000 steps from rest, with its
source and probe.  The oracle's state comes from tests/golden/
gradient_2p20_20000.npz, written by make_gradient_reference.py beside it
(oracle only); the fields are exactly zero outside the stored window, and
the GPU's must be too.  Relative L2 of D, B and the probe spectrum per tier,
bounds a few times the measured values."""
import os

import numpy as np
import pytest

from helpers import make_sim
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gradient_2p20_20000.npz")
BOUNDS = {gb.F64: 1e-11, gb.F32_KAHAN: 1e-5, gb.F32: 1e-4, gb.F16: 1e-2, gb.BF16: 8e-2}
NAMES = {gb.F64: "F64", gb.F32_KAHAN: "F32_KAHAN", gb.F32: "F32", gb.F16: "F16", gb.BF16: "BF16"}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


@pytest.fixture(scope="module")
def reference():
    return np.load(GOLDEN)


@pytest.mark.parametrize("prec", sorted(BOUNDS))
def test_gradient_full_size_error_per_tier(prec, reference):
    ref = reference
    n_steps = int(ref["n_steps"])
    wl = w.config4("stable", n_steps=n_steps)
    assert wl.instances[0].nz == int(ref["nz"])
    assert np.array_equal(wl.instances[0].probes[0][1], ref["bins"])
    sim = make_sim(wl, prec=prec, allow_unstable=False)
    sim.step(n_steps)
    lo, hi = int(ref["lo"]), int(ref["hi"])
    errs = []
    for which, key in ((gb.FIELD_D, "D"), (gb.FIELD_B, "B")):
        f = sim.read_fields(0, which)
        assert not np.any(f[:lo]) and not np.any(f[hi:]), key
        errs.append(np.linalg.norm(f[lo:hi] - ref[key]) / np.linalg.norm(ref[key]))
    X = sim.read_spectrum(0, 0, len(ref["bins"]))
    errs.append(np.linalg.norm(X - ref["spectrum"]) / np.linalg.norm(ref["spectrum"]))
    print("gradient 2^20 cells, %d steps, tier %-9s D %.2e  B %.2e  spectrum %.2e"
          % (n_steps, NAMES[prec], *errs))
    sim.close()
    assert max(errs) <= BOUNDS[prec], (NAMES[prec], errs)
