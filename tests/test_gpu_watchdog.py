"""Failure detection on the GPU without a GPU fault.

* The runtime stability watchdog (gfdtd_watchdog): an instance run where the
  scheme is unstable (n|v| > 1, Sec. 5) is flagged once its fields pass the
  limit, its measured growth per step equals the von Neumann max|zeta| of the
  medium (App. A), a non-finite value written into an instance is flagged as
  such, and stable instances are not flagged.
* The bounded waits of the fast kernel (gfdtd_test_stall): with the hook on,
  every tile barrier is armed but no copy is started, each wait gives up
  after its limit, the step reports E_TIMEOUT, and the same context then
  steps correctly again (checked against the oracle).  No copy is ever in
  flight, so nothing lands after a block has exited.
"""
import time

import numpy as np
import pytest

from helpers import make_oracle, make_sim, rel_l2
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def _uniform(nz, beta, eps):
    return w.InstanceSpec(nz=nz, beta=beta, eps=np.array([eps]), mu=np.ones(1))


def test_watchdog_flags_growth_and_non_finite_values():
    wl = w.Workload("watch", 0.5, 0, [_uniform(4000, 0.3, 4.0), _uniform(4000, 0.8, 4.0),
                                      _uniform(3000, -0.2, 2.0)])
    sim = make_sim(wl, tuning=(16, 16, 4), allow_unstable=True)
    rng = np.random.default_rng(4)
    for k, I in enumerate(wl.instances):
        B, D = (f.astype(np.float32).astype(np.float64) for f in w.random_fields(I.nz, rng, 1e-3))
        if k == 2:
            D[1500] = np.nan
        sim.write_fields(k, gb.FIELD_B, B)
        sim.write_fields(k, gb.FIELD_D, D)
    sim.step(2000)
    flags, a1 = sim.watchdog(limit=1e3, reset=True)
    sim.step(2000)
    flags2, a2 = sim.watchdog(limit=1e3)
    # the stable instance decays from its 1e-3 start; the unstable one grows past the limit
    assert flags[0] == 0 and flags2[0] == 0, (flags, a1)
    assert flags2[1] & 2 and not flags2[1] & 1, (flags2, a2)
    assert flags[2] & 1 and flags2[2] & 1, flags
    # growth per step of the largest field, after the fastest-growing mode has taken over
    rate = (a2[1] / a1[1]) ** (1.0 / 2000)
    zeta = gb.stability(0.5, 0.8, 4.0, 1.0, gb.PERTURBATION)
    print("watchdog: measured growth per step %.6f, von Neumann max|zeta| %.6f" % (rate, zeta))
    assert zeta > 1.005
    assert abs(rate - zeta) < 1e-3 * zeta, (rate, zeta)
    sim.close()


def test_watchdog_quiet_on_a_stable_batch():
    wl = w.config3(n_inst=16, nz_lo=1 << 11, nz_hi=1 << 13, n_steps=2000, stable_only=True)
    sim = make_sim(wl, allow_unstable=False, tuning=(20, 24, 7))
    sim.step(wl.n_steps)
    flags, amax = sim.watchdog(limit=1e3)
    assert not flags.any(), flags
    assert (amax > 0).all() and (amax < 10).all(), amax
    sim.close()


def test_bounded_wait_gives_up_and_the_context_recovers():
    wl = w.config3(n_inst=6, nz_lo=1 << 12, nz_hi=1 << 13, n_steps=0, stable_only=True)
    sim = make_sim(wl, allow_unstable=False, tuning=(16, 16, 4))
    assert sim.stats()["n_tiles"] > 0
    sim.test_stall(True)
    t0 = time.time()
    sim.step(16)
    with pytest.raises(gb.GfdtdError) as err:
        sim.synchronize()
    waited = time.time() - t0
    assert err.value.status == gb.E_TIMEOUT
    assert waited < 60.0, waited
    sim.synchronize()                  # reported once
    sim.test_stall(False)
    # the context is usable again: fresh fields, steps, parity with the oracle
    orcs = make_oracle(wl)
    rng = np.random.default_rng(9)
    for k, I in enumerate(wl.instances):
        B, D = (f.astype(np.float32).astype(np.float64) for f in w.random_fields(I.nz, rng))
        sim.write_fields(k, gb.FIELD_B, B)
        sim.write_fields(k, gb.FIELD_D, D)
        orcs[k].B[:], orcs[k].D[:] = B, D
        orcs[k].n_done = 16
    sim.step(100)
    sim.synchronize()
    for k, o in enumerate(orcs):
        o.run(100)
        assert rel_l2(sim.read_fields(k, gb.FIELD_D), o.D) <= 1e-4
        assert rel_l2(sim.read_fields(k, gb.FIELD_B), o.B) <= 1e-4
    print("bounded wait: E_TIMEOUT after %.2f s" % waited)
    sim.close()
