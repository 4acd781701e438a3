"""The allocation-free entry point (gfdtd_step_noalloc) against gfdtd_step.

gfdtd_step_noalloc serves callers that cannot allocate device memory (their
GPU memory is reserved by another framework's pool, or their host gives them
buffers but no allocator): it keeps its working buffers in one static device
array shared by all calls.  Each case makes two calls in a row, the second
continuing the first, and compares both with a context stepped by
gfdtd_step on the same tile shape (16 x 16 x 4), within the FP32 parity
tolerance; the second call must leave the device's free memory unchanged.
Collected last so that a failure here comes after every other test has run;
passes alone in a fresh process or after the rest of the suite.
"""
import numpy as np
import pytest

from helpers import make_sim, rel_l2
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


def _medium(kind, interp, nz, rng):
    """Layers of 25-90 cells, or a piecewise-linear profile of 40 knots, in the
    middle of the grid; eps in [1, 2] (moving matter: eps' in [1, 2])."""
    if interp == w.LAYERS:
        widths = rng.integers(25, 90, size=30)
        z = nz * 0.2 + np.cumsum(widths).astype(float)
        z = z[z < nz * 0.9]
        eps = rng.uniform(1.0, 2.0, size=len(z) + 1)
    else:
        z = np.sort(rng.uniform(0.2, 0.8, size=40)) * nz + np.arange(40) * 0.5
        eps = rng.uniform(1.0, 2.0, size=40)
    return z, eps


@pytest.mark.parametrize("kind,interp,beta,nz", [
    (w.PERTURBATION, w.LAYERS, 0.35, 5000), (w.PERTURBATION, w.LAYERS, -0.4, 777),
    (w.PERTURBATION, w.LAYERS, 0.0, 40000), (w.MATTER, w.LAYERS, 0.3, 3001),
    (w.MATTER, w.LAYERS, -0.45, 6000), (w.PERTURBATION, w.LINEAR, -0.25, 6000),
    (w.PERTURBATION, w.LINEAR, 0.4, 2500), (w.MATTER, w.LINEAR, 0.2, 4000)])
def test_noalloc_matches_context_step_on_two_calls(kind, interp, beta, nz):
    import torch
    rng = np.random.default_rng(61)
    z, eps = _medium(kind, interp, nz, rng)
    spec = w.InstanceSpec(nz=nz, beta=beta, kind=kind, interp=interp, z=z, eps=eps, mu=np.ones(len(eps)))
    wl = w.Workload("noalloc", 0.5, 0, [spec])
    B0 = rng.standard_normal(nz).astype(np.float32).astype(np.float64)
    D0 = rng.standard_normal(nz).astype(np.float32).astype(np.float64)

    sim = make_sim(wl, tuning=(16, 16, 4), allow_unstable=False)
    sim.write_fields(0, gb.FIELD_B, B0)
    sim.write_fields(0, gb.FIELD_D, D0)

    dev = torch.device("cuda", 0)
    Bd = torch.tensor(B0, dtype=torch.float32, device=dev)
    Dd = torch.tensor(D0, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    done = 0
    for call, n_steps in enumerate((50, 37)):   # two calls in a row, the second continuing the first
        sim.step(n_steps)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        gb.step_noalloc(Bd.data_ptr(), Dd.data_ptr(), nz, wl.S, kind, beta, interp,
                        z, eps, None, n_done=done, n_steps=n_steps, stream=stream)
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:
            # (the first call may load the library's device module, which holds the array)
            assert free_after == free_before, (free_before, free_after)
        done += n_steps
        for which, dev_field in ((gb.FIELD_B, Bd), (gb.FIELD_D, Dd)):
            ref = sim.read_fields(0, which)
            got = dev_field.double().cpu().numpy()
            assert rel_l2(got, ref) <= TOL32, (n_steps, which, rel_l2(got, ref))
    sim.close()


def test_noalloc_rejects_oversized_problem():
    import torch
    Bd = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(gb.GfdtdError):
        gb.step_noalloc(Bd.data_ptr(), Bd.data_ptr(), (1 << 18) + 1, 0.5, n_steps=1)
