"""Space-time capture (the z-t field maps of Fig. 5(a)): frames recorded by
gfdtd_step against gfdtd_read_fields at the same steps (exact after the
frame's rounding) and against the FP64 oracle (1e-4 relative L2)."""
import numpy as np
import pytest

from helpers import make_oracle, make_sim, rel_l2
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TUNING = (20, 24, 7)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def _workload():
    """Three moving layered instances of a few thousand cells, sources and probes."""
    out = []
    for nz, v in ((3000, 0.3), (2500, -0.25), (4100, 0.1)):
        z = 800.0 + np.cumsum(np.full(12, 60.0)) + 0.37
        eps = np.where(np.arange(13) % 2 == 0, 1.0, 3.0)
        out.append(w.InstanceSpec(nz=nz, beta=v, z=z, eps=eps, mu=np.ones(13),
                                  sources=[w.gaussian_source(600, 20.0, 3.0)],
                                  probes=[(nz - 200, np.linspace(0.2, 0.4, 3))]))
    return w.Workload("capture", 0.5, 0, out)


@pytest.mark.parametrize("which", [gb.FIELD_D, gb.FIELD_B, gb.FIELD_E])
@pytest.mark.parametrize("half", [False, True])
def test_frames_equal_read_fields(which, half):
    wl = _workload()
    a = make_sim(wl, allow_unstable=False, tuning=TUNING)
    b = make_sim(wl, allow_unstable=False, tuning=TUNING)
    inst, z0, z1, zs, ts, nf = 1, 37, 2410, 3, 7, 40
    a.set_capture(inst, which, z0, z1, zs, ts, max_frames=nf, half=half)
    a.step(ts * nf)
    frames, dropped = a.capture()
    assert frames.shape == (nf, len(range(z0, z1, zs))) and dropped == 0
    rnd = np.float16 if half else np.float32
    for f in range(nf):
        b.step(ts)        # the same chunks, so the same launches and roundings
        ref = b.read_fields(inst, which)[z0:z1:zs].astype(rnd).astype(np.float64)
        assert np.array_equal(frames[f], ref), (f, np.abs(frames[f] - ref).max())


def test_frames_match_oracle():
    wl = _workload()
    sim = make_sim(wl, allow_unstable=False, tuning=TUNING)
    orcs = make_oracle(wl)
    inst, ts, nf = 0, 50, 12
    sim.set_capture(inst, gb.FIELD_D, 0, wl.instances[inst].nz, 2, ts, max_frames=nf)
    sim.step(ts * nf)
    frames, _ = sim.capture()
    for f in range(nf):
        orcs[inst].run(ts)
        ref = orcs[inst].D[::2]
        if np.abs(ref).max() > 0:
            assert rel_l2(frames[f], ref) <= 1e-4, f


def test_capture_bookkeeping():
    """Dropped frames past max_frames, off with t_stride 0, a new capture
    replaces the old one, frames counted from the call, bad ranges rejected."""
    wl = _workload()
    sim = make_sim(wl, allow_unstable=False, tuning=TUNING)
    sim.step(5)
    sim.set_capture(2, gb.FIELD_D, 0, 10, 1, 4, max_frames=3)
    sim.step(17)                 # frames after 4, 8, 12, 16 steps: one dropped
    frames, dropped = sim.capture()
    assert frames.shape == (3, 10) and dropped == 1
    sim.set_capture(2, gb.FIELD_D, 0, 10, 1, 0)    # off: frames kept
    sim.step(8)
    assert sim.capture()[0].shape == (3, 10)
    sim.set_capture(0, gb.FIELD_B, 5, 6, 1, 1, max_frames=4)
    assert sim.capture()[0].shape == (0, 1)
    sim.step(2)
    assert sim.capture()[0].shape == (2, 1)
    for bad in ((0, gb.FIELD_D, 0, 3001, 1, 1), (0, gb.FIELD_D, 10, 10, 1, 1), (0, gb.FIELD_D, 0, 5, 0, 1),
                (7, gb.FIELD_D, 0, 5, 1, 1)):
        with pytest.raises(gb.GfdtdError):
            sim.set_capture(*bad)
