"""The moving-matter slab workload as written, on the GPU against the FP64
oracle: five instances of 2^16 cells (rest eps' = 9, an 800-cell slab, v in
{-0.5, -0.2, 0, 0.2, 0.5}c; moving matter by reading R3 of the solved star
relations of Eq. const_3d), 40000 steps from rest with their Gaussian sources
and both 256-bin probes (Sec. 4, Table 1).

Fields within 1e-10 (FP64 tier) and 1e-4 (FP32 tier, autotuned as the
benchmark's examples run it) relative L2; each spectrum within the same
bounds of the oracle's, relative to its norm floored at 1 % of the instance's
larger probe spectrum (reading R18): behind the slab the transmitted pulse
arrives damped by the first-order dissipation of reading R3 inside moving
matter, at v = -0.5c some 1e-7 of the incident one, which the fields carry only
to their rounding level (plain relative L2 of that spectrum: 6e-8 in FP64, 10
in FP32)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _run(wl, prec):
    sim = gb.Simulation([I.nz for I in wl.instances], wl.S, prec)
    for k, I in enumerate(wl.instances):
        sim.set_medium(k, I.kind, I.beta, I.interp, I.z, I.eps, I.mu)
        for s in I.sources:
            sim.add_source(k, *s)
        for p in I.probes:
            sim.add_probe(k, p[0], p[1])
    sim.step(wl.n_steps)
    assert sim.steps_done() == wl.n_steps
    out = []
    for k, I in enumerate(wl.instances):
        out.append((sim.read_fields(k, gb.FIELD_D), sim.read_fields(k, gb.FIELD_B),
                    [sim.read_spectrum(k, p, len(I.probes[p][1])) for p in range(len(I.probes))]))
    sim.close()
    return out


def test_slab_as_written_matches_oracle():
    wl = w.config2()
    orcs = []
    for I in wl.instances:
        o = oracle.Instance(I.nz, wl.S, I.beta, kind=I.kind, interp=I.interp, z=I.z, eps=I.eps, mu=I.mu)
        for s in I.sources:
            o.add_source(*s)
        for p in I.probes:
            o.add_probe(p[0], p[1])
        orcs.append(o)
    with ThreadPoolExecutor(len(orcs)) as ex:          # the oracle's C loop runs outside the GIL
        list(ex.map(lambda o: o.run(wl.n_steps), orcs))
    f64, f32 = _run(wl, gb.F64), _run(wl, gb.F32)
    worst = 0.0
    for I, o, (D8, B8, X8), (D4, B4, X4) in zip(wl.instances, orcs, f64, f32):
        spectra = [o.spectrum(p) for p in range(len(I.probes))]
        floor = 0.01 * max(np.linalg.norm(y) for y in spectra)

        def rel_floor(x, y):
            return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), floor))
        e64 = [rel(D8, o.D), rel(B8, o.B)] + [rel_floor(x, y) for x, y in zip(X8, spectra)]
        e32 = [rel(D4, o.D), rel(B4, o.B)] + [rel_floor(x, y) for x, y in zip(X4, spectra)]
        plain = [rel(x, y) for x, y in zip(X4, spectra)]
        print("slab v = %+.1fc: FP64 max %.1e; FP32 D %.2e, B %.2e, spectra %s (plain %s)" % (
            I.beta, max(e64), e32[0], e32[1], ", ".join("%.2e" % e for e in e32[2:]),
            ", ".join("%.2e" % e for e in plain)))
        assert max(e64) <= 1e-10, (I.beta, e64)
        assert max(e32) <= TOL, (I.beta, e32)
        worst = max(worst, max(e32))
    print("FP32: largest relative L2 over fields and spectra: %.2e" % worst)
