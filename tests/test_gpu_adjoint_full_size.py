"""The adjoint at the adjoint workload's full size: 256 instances of 2^14
cells, piecewise-linear eps over 514 knots (512 controls uniform in [1, 4]),
v = 0.4c, 16000 steps, loss = transmitted DFT power over a 16-bin band.  The
GPU runs the whole batch (as the benchmark does); two sampled instances are
checked against the oracle's FP64 discrete adjoint on every knot, and one of
them against central finite differences of the oracle's FP64 loss (h = 1e-4)
on eight controls whose derivative is not small, per component."""
import numpy as np
import pytest

from helpers import make_oracle, make_sim
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

SAMPLE = (7, 131)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


@pytest.fixture(scope="module")
def gpu_adjoint():
    wl = w.config5()
    sim = make_sim(wl, allow_unstable=False)
    nv = [len(I.eps) for I in wl.instances]
    loss, grads = sim.adjoint(wl.n_steps, 0, 0, 16, nv)
    sim.close()
    return wl, loss, grads


@pytest.fixture(scope="module")
def oracle_adjoint(gpu_adjoint):
    from concurrent.futures import ThreadPoolExecutor
    wl = gpu_adjoint[0]
    orcs = make_oracle(w.Workload("sample", wl.S, wl.n_steps, [wl.instances[k] for k in SAMPLE]))
    with ThreadPoolExecutor(len(orcs)) as ex:
        return list(ex.map(lambda o: o.adjoint(0, range(16), wl.n_steps), orcs))


def test_adjoint_matches_oracle_adjoint_on_every_knot(gpu_adjoint, oracle_adjoint):
    wl, loss, grads = gpu_adjoint
    for (L, g), k in zip(oracle_adjoint, SAMPLE):
        gg = grads[k]
        assert abs(loss[k] - L) <= 1e-4 * L, (k, loss[k], L)
        rel = np.linalg.norm(gg - g) / np.linalg.norm(g)
        big = np.abs(g) >= 1e-2 * np.abs(g).max()
        comp = np.abs(gg - g)[big] / np.abs(g)[big]
        print("adjoint instance %d: loss %.6e (oracle %.6e), gradient relative L2 %.2e, "
              "per component (|g| >= 1e-2 max, %d of %d): largest %.2e"
              % (k, loss[k], L, rel, int(big.sum()), len(g), comp.max()))
        assert rel <= 1e-3, (k, rel)
        assert comp.max() <= 1e-3, (k, comp.max())
        assert np.all(np.abs(gg - g)[~big] <= 1e-5 * np.abs(g).max())


def test_adjoint_matches_central_differences(gpu_adjoint, oracle_adjoint):
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    wl, loss, grads = gpu_adjoint
    k = SAMPLE[0]
    I = wl.instances[k]
    g_orc = oracle_adjoint[0][1]
    ctrl = np.arange(1, len(I.eps) - 1)
    cand = ctrl[np.abs(g_orc[ctrl]) >= 0.1 * np.abs(g_orc[ctrl]).max()]
    pick = cand[np.linspace(0, len(cand) - 1, 8).astype(int)]
    h = 1e-4

    def L_of(j, sign):
        eps = I.eps.copy()
        eps[j] += sign * h
        o = oracle.Instance(I.nz, wl.S, I.beta, interp=I.interp, z=I.z, eps=eps, mu=I.mu)
        o.add_source(*I.sources[0])
        o.add_probe(I.probes[0][0], I.probes[0][1])
        o.run(wl.n_steps)
        return float(np.sum(np.abs(o.spectrum(0)[:16]) ** 2))

    jobs = [(j, s) for j in pick for s in (1, -1)]
    with ThreadPoolExecutor(len(jobs)) as ex:
        vals = list(ex.map(lambda a: L_of(*a), jobs))
    for i, j in enumerate(pick):
        fd = (vals[2 * i] - vals[2 * i + 1]) / (2 * h)
        print("control %3d: GPU adjoint %+.6e, oracle adjoint %+.6e, central difference %+.6e"
              % (j, grads[k][j], g_orc[j], fd))
        assert abs(g_orc[j] - fd) <= 1e-6 * abs(fd), (j, g_orc[j], fd)
        assert abs(grads[k][j] - fd) <= 1e-3 * abs(fd), (j, grads[k][j], fd)
