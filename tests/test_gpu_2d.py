"""GPU parity of the 2D TE generalized scheme (gfdtd2d_*) against the FP64
oracle's 2D scheme (Sec. 3 and Sec. 4 before the 1D reduction), through the
C ABI: random fields in slanted moving layers (both signs of v, several
column counts, ragged z sizes spanning several tiles, both tile shapes, time
blocks plus a partial one), line sources and probes from rest, FP32 at 1e-4
and FP64 at 1e-11 relative L2; the reflection of an obliquely incident pulse
off a co-moving interface against the closed form derived from Eq. cont and
Eq. star; argument errors."""
import numpy as np
import pytest

from oracle.core import Instance2D
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FIELDS = ((gb.FIELD2D_D, "D"), (gb.FIELD2D_BX, "Bx"), (gb.FIELD2D_BZ, "Bz"))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _pair(nx, nz, dx, beta, slope, z, eps, mu, prec, tuning=None):
    g = gb.Simulation2D(nx, nz, dx, 0.5, prec)
    g.set_medium(beta, slope, z, eps, mu)
    if tuning:
        g.set_tuning(*tuning)
    o = Instance2D(nx, nz, 0.5, beta, dx=dx, z=z, eps=eps, mu=mu, slope=slope)
    return g, o


def _round(x, prec):
    return x.astype(np.float32).astype(np.float64) if prec == gb.F32 else x


CASES = [  # nx, nz, dx, beta, slope
    (1, 700, 1.0, 0.3, 0.0), (5, 1301, 2.5, -0.35, 0.4), (8, 3000, 1.5, 0.45, -0.7),
    (16, 999, 3.0, -0.2, 1.3), (32, 2100, 2.0, 0.25, 0.2)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,tuning", [(gb.F32, (8, 16)), (gb.F32, (8, 8)), (gb.F64, (8, 8))])
def test_random_fields_in_slanted_moving_layers(case, prec, tuning):
    nx, nz, dx, beta, slope = case
    rng = np.random.default_rng(nx * 7 + nz)
    widths = rng.integers(3, 60, size=12)
    z = 0.2 * nz + np.cumsum(widths) + rng.uniform(0, 1)
    eps = rng.uniform(1.0, 2.5, size=len(z) + 1)
    mu = rng.uniform(1.0, 1.3, size=len(z) + 1)
    g, o = _pair(nx, nz, dx, beta, slope, z, eps, mu, prec, tuning)
    for which, name in FIELDS:
        f = _round(rng.standard_normal((nx, nz)), prec)
        g.write_fields(which, f)
        getattr(o, name)[:] = f
    n = 2 * tuning[1] + 5            # two time blocks and a partial one
    g.step(n)
    o.run(n)
    tol = 1e-11 if prec == gb.F64 else 1e-4
    for which, name in FIELDS:
        e = rel(g.read_fields(which), getattr(o, name))
        assert e <= tol, (case, name, e)
    g.close()


@pytest.mark.parametrize("prec", [gb.F32, gb.F64])
def test_line_source_and_probes_from_rest(prec):
    """An oblique pulse (30 degrees) from a line source onto a co-moving slanted
    slab, 800 steps, probes before and behind it: fields and spectra."""
    nx, nz, S = 8, 2400, 0.5
    lam0 = 40.0
    w0 = 2 * np.pi / lam0
    kx = w0 * np.sin(np.radians(30.0))
    dx = 2 * np.pi / kx / nx
    _, _, tau, t0, _ = w.gaussian_source(0, lam0, 3.0)
    z, eps = [900.0, 1100.0], [1.0, 3.0, 1.0]
    g, o = _pair(nx, nz, dx, 0.3, 0.15, z, eps, [1.0] * 3, prec)
    bins = np.linspace(0.6, 1.4, 9) * w0
    for k in (600,):
        g.add_source(k, kx, w0, tau, t0)
        o.add_source(k, kx, w0, tau, t0)
    for i, k in ((0, 700), (3, 1500), (7, 2300)):
        g.add_probe(i, k, bins)
        o.add_probe(i, k, bins)
    g.step(800)
    o.run(800)
    tol = 1e-11 if prec == gb.F64 else 1e-4
    for which, name in FIELDS:
        e = rel(g.read_fields(which), getattr(o, name))
        assert e <= tol, (name, e)
    for p in range(3):
        e = rel(g.read_spectrum(p, len(bins)), o.spectrum(p))
        assert e <= tol, (p, e)
    g.close()


def test_oblique_moving_interface_reflection_on_gpu():
    """|Gamma| of a TE pulse at 30 degrees off an interface co-moving at 0.3c
    (eps 1 | 4, 40 cells per carrier wavelength) against
    exact.oblique_interface within 1 %, on the GPU in FP32 (the oracle's own
    run of the same case is a pin in test_oracle_2d)."""
    import test_oracle_2d as t2
    runs, fs, w0, kxe, steps = t2.oblique_reflection(0.3, 30.0)
    X = []
    for I in runs:
        g = gb.Simulation2D(I.nx, I.nz, I.dx, I.S, gb.F32)
        g.set_medium(I.beta, I.slope, I.z if len(I.eps) > 1 else (), I.eps, I.mu)
        for src in I.sources:
            g.add_source(*src)
        p = I.probes[0]
        g.add_probe(p["i"], p["k"], p["omega"])
        g.step(steps)
        X.append(g.read_spectrum(0, len(p["omega"])))
        g.close()
    err = t2.reflection_errors(X[0], X[1], 0.3, fs, w0, kxe)
    print("oblique reflection on the GPU, errors at 0.9, 1.0, 1.1 w0:", np.round(err, 4))
    assert np.all(np.abs(err) < 0.01), err


def test_argument_errors():
    with pytest.raises(gb.GfdtdError):
        gb.Simulation2D(33, 100, 1.0, 0.5)                 # more columns than a block holds
    with pytest.raises(gb.GfdtdError):
        gb.Simulation2D(4, 100, 1.0, 0.8)                  # beyond the 2D Yee limit
    with pytest.raises(gb.GfdtdError):
        gb.Simulation2D(4, 100, 1.0, 0.5, gb.F16)
    g = gb.Simulation2D(4, 100, 2.0, 0.5)
    with pytest.raises(gb.GfdtdError):
        g.set_medium(0.6, 0.0, [50.0], [1.0, 4.0])        # n|v| > 1
    with pytest.raises(gb.GfdtdError):
        g.set_tuning(16, 16)
    with pytest.raises(gb.GfdtdError):
        g.add_probe(4, 10, [0.1])
    for q in range(32):                                    # at most 32 line sources and 32 probes
        g.add_source(10 + q, 0.0, 0.3, 20.0, 60.0)
        g.add_probe(q % 4, 20 + q, [0.3])
    with pytest.raises(gb.GfdtdError):
        g.add_source(60, 0.0, 0.3, 20.0, 60.0)
    with pytest.raises(gb.GfdtdError):
        g.add_probe(0, 60, [0.3])
    g.close()
