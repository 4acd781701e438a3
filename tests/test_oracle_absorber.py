"""The oracle's graded absorbing layers (an option of this library; the
paper is silent on the domain ends): reflection measured against a domain too
long for any reflection to return, and the layers' absence when width = 0."""
import numpy as np
import pytest

import oracle
from paper_2304_06586_gb300 import workloads as w


def _series(nz, src, prb, beta, width, sigma, steps, eps=1.0):
    o = oracle.Instance(nz, 0.5, beta, z=(), eps=(eps,))
    o.add_source(*w.gaussian_source(src, 40.0, 3.0))
    o.add_probe(prb, np.array([0.1]))
    o.set_absorber(width, sigma)
    o.run(steps, record=True)
    return o.series(0)


@pytest.mark.parametrize("beta,width,sigma,bound", [(0.0, 64, 0.2, 1e-6), (0.3, 64, 0.2, 3e-4),
                                                     (-0.3, 64, 0.2, 3e-4), (0.0, 128, 0.1, 1e-7),
                                                     (0.3, 128, 0.1, 5e-5)])
def test_reflection_below_bound(beta, width, sigma, bound):
    """A pulse 600 cells from the left end: the probe series equals that of a
    12000-cell domain until the echo of the layer would arrive; the difference
    is the layer's reflection (the echo from the left end reaches the probe
    by step 4100, the one from the right end after step 5300).  Without the
    layer the zero-field end reflects the pulse, which the same measurement
    shows."""
    steps = 4400
    ref = _series(12000, 6000, 5600, beta, 0, 0.0, steps)
    got = _series(2000, 1000, 600, beta, width, sigma, steps)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= bound
    bare = _series(2000, 1000, 600, beta, 0, 0.0, steps)
    assert np.abs(bare - ref).max() / np.abs(ref).max() > 0.3


def test_zero_width_is_no_layer():
    rng = np.random.default_rng(2)
    a = oracle.Instance(300, 0.5, 0.2, z=(100.0, 180.0), eps=(1.0, 3.0, 1.0))
    b = oracle.Instance(300, 0.5, 0.2, z=(100.0, 180.0), eps=(1.0, 3.0, 1.0)).set_absorber(0, 5.0)
    a.B[:] = rng.standard_normal(300)
    a.D[:] = rng.standard_normal(300)
    b.B[:], b.D[:] = a.B, a.D
    a.run(50)
    b.run(50)
    assert np.array_equal(a.B, b.B) and np.array_equal(a.D, b.D)


def test_damping_is_local():
    """Fields away from the layers are untouched until a wave reaches them:
    with the layers, a field seeded in the middle evolves identically for as
    many steps as it takes a disturbance from the layers to travel back."""
    rng = np.random.default_rng(3)
    nz, width = 2000, 64
    a = oracle.Instance(nz, 0.5, 0.0)
    b = oracle.Instance(nz, 0.5, 0.0).set_absorber(width, 0.3)
    seed = np.zeros(nz)
    seed[900:1100] = rng.standard_normal(200)
    for o in (a, b):
        o.D[:] = seed
    a.run(100)
    b.run(100)
    # 100 steps reach at most 2 cells per step: 200 cells from each layer
    mid = slice(width + 250, nz - width - 250)
    assert np.array_equal(a.D[mid], b.D[mid]) and np.array_equal(a.B[mid], b.B[mid])
