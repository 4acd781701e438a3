"""GPU absorbing layers against the FP64 oracle with the same layers
(relative L2 <= 1e-4 on fields and spectra), through the batched kernels of
several tile shapes and the plain kernel."""
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


def _workload(kind=w.PERTURBATION, seed=9):
    rng = np.random.default_rng(seed)
    out, layers = [], []
    for nz, v, width in ((300, 0.3, 8), (1000, -0.3, 64), (3001, 0.45, 64), (9000, -0.2, 128),
                         (20000, 0.1, 64), (5000, 0.0, 40)):
        z = rng.uniform(0.2, 0.4) * nz + np.cumsum(rng.integers(30, 90, size=6)) + 0.3
        eps = rng.uniform(1.0, 3.0, size=7)
        out.append(w.InstanceSpec(nz=nz, beta=v, kind=kind, z=z, eps=eps, mu=np.ones(7),
                                  sources=[w.gaussian_source(nz // 2, 20.0, 3.0)],
                                  probes=[(nz // 2 + 60, np.linspace(0.1, 0.5, 5))]))
        layers.append(width)
    return w.Workload("absorber", 0.5, 0, out), layers


def _pair(wl, layers, tuning=None, seed_fields=True):
    sim = make_sim(wl, allow_unstable=False, tuning=tuning)
    orcs = make_oracle(wl)
    rng = np.random.default_rng(1)
    for k, (I, width) in enumerate(zip(wl.instances, layers)):
        sim.set_absorber(k, width, 0.2)
        orcs[k].set_absorber(width, 0.2)
        if seed_fields:
            for f, which in ((orcs[k].B, gb.FIELD_B), (orcs[k].D, gb.FIELD_D)):
                x = rng.standard_normal(I.nz).astype(np.float32).astype(np.float64)
                f[:] = x
                sim.write_fields(k, which, x)
    return sim, orcs


def _compare(wl, sim, orcs, spectra=True):
    for k, I in enumerate(wl.instances):
        for which, ref in ((gb.FIELD_B, orcs[k].B), (gb.FIELD_D, orcs[k].D)):
            e = rel_l2(sim.read_fields(k, which), ref)
            assert e <= TOL32, (k, I.nz, which, e)
        if spectra:
            for p, (node, om) in enumerate(I.probes):
                e = rel_l2(sim.read_spectrum(k, p, len(om)), orcs[k].spectrum(p))
                assert e <= TOL32, (k, "probe", p, e)


@pytest.mark.parametrize("tuning", [None, (16, 24, 8), (24, 24, 6), (8, 16)])
@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_absorber_random_fields(tuning, kind):
    wl, layers = _workload(kind)
    sim, orcs = _pair(wl, layers, tuning)
    n = 77
    sim.step(n)
    for o in orcs:
        o.run(n)
    _compare(wl, sim, orcs)


def test_absorber_long_run_from_rest():
    """A pulse from each source travels into the layers and is absorbed there."""
    wl, layers = _workload()
    sim, orcs = _pair(wl, layers, seed_fields=False)
    sim.step(1500)
    import oracle
    oracle.run_many(orcs, 1500)
    _compare(wl, sim, orcs)


def test_absorber_plain_kernel():
    wl, layers = _workload()
    sim, orcs = _pair(wl, layers)
    sim.step_plain(30)
    for o in orcs:
        o.run(30)
    _compare(wl, sim, orcs, spectra=False)


def test_absorber_arguments_and_adjoint():
    wl, layers = _workload()
    sim = make_sim(wl, allow_unstable=False)
    for bad in ((0, -1, 0.2), (0, 150, 0.2), (0, 8, -1.0), (0, 8, float("nan")), (9, 8, 0.2)):
        with pytest.raises(gb.GfdtdError):
            sim.set_absorber(*bad)
    sim.set_absorber(1, 64, 0.2)
    with pytest.raises(gb.GfdtdError):
        sim.adjoint(10, 0, 0, 1, [7] * len(wl.instances))
    sim.set_absorber(1, 0, 0.0)
