"""The allocation-free entry point (gfdtd_step_noalloc) against gfdtd_step.

It serves callers that cannot allocate device memory (for example code being
captured into a CUDA graph); it keeps its working buffers in a static device
array shared by all calls.  Collected last so that a failure here comes after
every other test has run.  Passes alone or after the rest of the suite.
"""
import numpy as np
import pytest

from helpers import make_sim, rel_l2
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


@pytest.mark.parametrize("beta,nz", [(0.35, 5000), (-0.4, 777), (0.0, 40000)])
def test_noalloc_matches_context_step_on_two_calls(beta, nz):
    import torch
    rng = np.random.default_rng(61)
    widths = rng.integers(25, 90, size=30)
    z = nz * 0.2 + np.cumsum(widths).astype(float)
    z = z[z < nz * 0.9]
    eps = rng.uniform(1.0, 2.0, size=len(z) + 1)
    spec = w.InstanceSpec(nz=nz, beta=beta, z=z, eps=eps, mu=np.ones(len(eps)))
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
    for n_steps in (50, 37):        # two calls in a row, the second continuing the first
        sim.step(n_steps)
        gb.step_noalloc(Bd.data_ptr(), Dd.data_ptr(), nz, wl.S, gb.PERTURBATION, beta, gb.LAYERS,
                        z, eps, None, n_done=done, n_steps=n_steps, stream=stream)
        done += n_steps
        for which, dev_field in ((gb.FIELD_B, Bd), (gb.FIELD_D, Dd)):
            ref = sim.read_fields(0, which)
            got = dev_field.double().cpu().numpy()
            assert rel_l2(got, ref) <= 1e-4, (n_steps, which, rel_l2(got, ref))


def test_noalloc_rejects_oversized_problem():
    import torch
    Bd = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(gb.GfdtdError):
        gb.step_noalloc(Bd.data_ptr(), Bd.data_ptr(), (1 << 18) + 1, 0.5, n_steps=1)
