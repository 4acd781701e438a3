"""GPU one-way (total-field / scattered-field) sources against the FP64 oracle
with the same sources: fields and spectra at 1e-4 relative L2 in FP32 (1e-11
in FP64), through several tile shapes, over more than one chunk of steps (the
auxiliary grids carry their state across chunks), with scatterers in the
total-field region and probes on both sides."""
import numpy as np
import pytest

from helpers import make_oracle, make_sim, rel_l2
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def _pulse(lam0=40.0, periods=3.0):
    w0 = 2 * np.pi / lam0
    tau = periods * lam0 / (2 * np.sqrt(np.log(2)))
    return w0, tau, 4 * tau


def _workload(kind=w.PERTURBATION):
    """Instances with a one-way source at q and a layered scatterer further on:
    both signs of v, a wide-layer instance whose other tiles take the fast
    kernel, a linear ramp, and a boundary near the domain start."""
    out, tf = [], []
    bg = 2.0 if kind == w.PERTURBATION else 1.0    # moving matter with n' > 1 damps the pulse (reading R3)
    specs = [(3000, 0.3, 800, [1000.0, 1200.0], [1.0, 4.0, 1.0]),
             (2500, -0.25, 600, [800.0, 860.0, 920.0], [1.0, 2.5, 1.0, 2.5]),
             (6000, 0.1, 1000, [1250.0, 1850.0], [1.0, 4.0, 1.0]),
             (4000, 0.45, 3, [150.0, 250.0], [1.0, 3.0, 1.0]),
             (5000, -0.4, 2100, [2300.0, 2700.0], [bg, 5.0, bg])]
    for nz, v, q, z, eps in specs:
        out.append(w.InstanceSpec(nz=nz, beta=v, kind=kind, z=np.array(z), eps=np.array(eps),
                                  mu=np.ones(len(eps)),
                                  probes=[(max(q - 150, 0), np.linspace(0.1, 0.2, 4)),
                                          (min(q + 300, nz - 1), np.linspace(0.1, 0.2, 4))]))
        tf.append(q)
    out.append(w.InstanceSpec(nz=3000, beta=0.2, kind=kind, interp=w.LINEAR,
                              z=np.array([850.0, 1400.0]), eps=np.array([1.0, 3.0]), mu=np.ones(2),
                              probes=[(500, np.linspace(0.1, 0.2, 4))]))
    tf.append(700)
    return w.Workload("tfsf", 0.5, 0, out), tf


def _pair(wl, tf, prec=gb.F32, tuning=None):
    sim = make_sim(wl, prec=prec, allow_unstable=False, tuning=tuning)
    orcs = make_oracle(wl)
    w0, tau, t0 = _pulse()
    for k, q in enumerate(tf):
        sim.add_tfsf(k, q, w0, tau, t0, 0.8)
        orcs[k].add_tfsf(q, w0, tau, t0, 0.8)
    return sim, orcs


def _compare(wl, sim, orcs, tol):
    # spectra: relative L2, with probes that saw little (a pulse damped by
    # moving matter, a weak reflection) measured against 1 % of the largest
    # probe spectrum of the workload (an FP32 rounding of the incident wave is
    # 1e-7 of that)
    scale = max(np.linalg.norm(o.spectrum(p)) for o in orcs for p in range(len(o.probes)))
    for k, I in enumerate(wl.instances):
        for which, ref in ((gb.FIELD_B, orcs[k].B), (gb.FIELD_D, orcs[k].D)):
            assert np.abs(ref).max() > 1e-3, (k, which)
            e = rel_l2(sim.read_fields(k, which), ref)
            assert e <= tol, (k, I.nz, I.beta, which, e)
        for p, (node, om) in enumerate(I.probes):
            ref = orcs[k].spectrum(p)
            e = np.linalg.norm(sim.read_spectrum(k, p, len(om)) - ref) / max(np.linalg.norm(ref), 1e-2 * scale)
            assert e <= tol, (k, "probe", p, e)


@pytest.mark.parametrize("tuning", [None, (16, 24, 8), (8, 16), (20, 32, 7)])
@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_tfsf_matches_oracle(kind, tuning):
    wl, tf = _workload(kind)
    sim, orcs = _pair(wl, tf, tuning=tuning)
    n = 2400                    # three chunks
    sim.step(700)
    sim.step(n - 700)
    import oracle
    oracle.run_many(orcs, n)
    _compare(wl, sim, orcs, TOL32)


def test_tfsf_with_absorbing_layers():
    """One-way sources and graded absorbing layers together (the layers damp
    after each update, the corrections are added after the damping, on both
    sides)."""
    wl, tf = _workload()
    sim, orcs = _pair(wl, tf)
    for k, I in enumerate(wl.instances):
        sim.set_absorber(k, 48, 0.2)
        orcs[k].set_absorber(48, 0.2)
    sim.step(2400)
    import oracle
    oracle.run_many(orcs, 2400)
    _compare(wl, sim, orcs, TOL32)


def test_tfsf_fp64_tier():
    wl, tf = _workload()
    sim, orcs = _pair(wl, tf, prec=gb.F64)
    sim.step(2400)
    import oracle
    oracle.run_many(orcs, 2400)
    _compare(wl, sim, orcs, 1e-11)


def test_tfsf_scattered_region_empty_in_uniform_medium():
    """No scatterer: the scattered-field region holds only rounding (FP32) and
    what the auxiliary layers reflect."""
    insts = [w.InstanceSpec(nz=3000, beta=v, z=np.zeros(0), eps=np.array([e]), mu=np.ones(1))
             for v, e in ((0.0, 1.0), (0.3, 1.0), (-0.3, 2.0), (0.5, 1.5))]
    wl = w.Workload("tfsf_uniform", 0.5, 0, insts)
    sim, _ = _pair(wl, [900] * len(insts))
    sim.step(1800)
    for k in range(len(insts)):
        D = sim.read_fields(k, gb.FIELD_D)
        assert np.abs(D[900:]).max() > 0.05
        assert np.abs(D[:899]).max() <= 1e-5 * np.abs(D[900:]).max(), k


def test_tfsf_arguments_and_rejections():
    wl, tf = _workload()
    sim = make_sim(wl, allow_unstable=False)
    w0, tau, t0 = _pulse()
    for bad in ((0, -1, w0, tau, t0), (0, 3000, w0, tau, t0), (0, 10, w0, 0.0, t0), (0, 10, w0, tau, np.nan),
                (99, 10, w0, tau, t0)):
        with pytest.raises(gb.GfdtdError):
            sim.add_tfsf(*bad)
    sim.add_tfsf(0, 800, w0, tau, t0)
    with pytest.raises(gb.GfdtdError):
        sim.step_plain(2)
    with pytest.raises(gb.GfdtdError):
        sim.adjoint(10, 0, 0, 1, [len(I.eps) for I in wl.instances])
    for _ in range(4):
        sim.add_tfsf(1, 700, w0, tau, t0)
    with pytest.raises(gb.GfdtdError):          # at most 4 per instance
        sim.add_tfsf(1, 701, w0, tau, t0)
