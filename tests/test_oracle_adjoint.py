"""Pins of the oracle's discrete adjoint: the transpose identity of one step,
and central finite differences of the loss (the gradient target of the
method's differentiation path)."""
import numpy as np
import pytest

from oracle import Instance
from paper_2304_06586_gb300 import workloads as w


@pytest.mark.parametrize("beta", [0.4, -0.35, 0.0])
@pytest.mark.parametrize("interp", [0, 1])
def test_step_transpose_dot_product(beta, interp):
    """<A x, y> = <x, A^T y> for one step (no source), to rounding."""
    rng = np.random.default_rng(21)
    nz, S = 120, 0.5
    if interp == 0:
        z, eps = [30.5, 61.0, 77.25], [1.0, 3.0, 2.0, 4.0]
    else:
        z, eps = [20.0, 40.5, 41.0, 90.0], [1.0, 3.5, 2.0, 1.5]
    mu = [1.0] * len(eps)
    I = Instance(nz, S, beta, interp=interp, z=z, eps=eps, mu=mu)
    n = 17
    B, D = rng.standard_normal(nz), rng.standard_normal(nz)
    yB, yD = rng.standard_normal(nz), rng.standard_normal(nz)
    I.B[:], I.D[:] = B, D
    I.n_done = n - 1
    I.run(1)
    lhs = I.B @ yB + I.D @ yD
    aB, aD, _ = I.step_transpose(n, yB, yD, D)
    rhs = B @ aB + D @ aD
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(B) * np.linalg.norm(yB))


def test_eps_gradient_of_one_step_matches_differences():
    """geps from the transpose equals d<A(eps) x, y>/d eps_k (by central differences)."""
    rng = np.random.default_rng(22)
    nz, S, beta = 40, 0.5, 0.3
    z = np.arange(nz - 1) + 0.25          # one layer per cell: node k lies in layer k
    eps = rng.uniform(1.0, 3.0, size=nz)
    I = Instance(nz, S, beta, z=z, eps=eps)
    B, D = rng.standard_normal(nz), rng.standard_normal(nz)
    yB, yD = rng.standard_normal(nz), rng.standard_normal(nz)
    n = 1                                  # no motion yet at level 1/2 matters little: beta S/2 < 0.25
    _, _, geps = I.step_transpose(n, yB, yD, D)
    h = 1e-6
    for k in (0, 5, 17, nz - 1):
        vals = []
        for sgn in (1, -1):
            e2 = eps.copy()
            e2[k] += sgn * h
            J = Instance(nz, S, beta, z=z, eps=e2)
            J.B[:], J.D[:] = B, D
            J.n_done = n - 1
            J.run(1)
            vals.append(J.B @ yB + J.D @ yD)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - geps[k]) <= 1e-6 * (1 + abs(fd)), (k, fd, geps[k])


@pytest.mark.slow
def test_adjoint_gradient_matches_central_differences():
    """Config-5 shape at reduced size: dL/d(control eps) vs central differences (h = 1e-4)."""
    wl = w.config5(n_inst=1, nz=1 << 11, n_steps=1400, n_ctrl=48)
    I0 = wl.instances[0]
    # shift the geometry into the reduced grid: region at [400, 496), source 100, probe 1200
    z = I0.z - 2046.0 + 400.0
    spec = dict(nz=I0.nz, S=wl.S, beta=I0.beta, interp=1, z=z, eps=I0.eps, mu=I0.mu)
    node, om = 1200, I0.probes[0][1]
    src = w.gaussian_source(100, 40.0, 3.0)

    def make(eps):
        J = Instance(spec["nz"], spec["S"], spec["beta"], interp=1, z=spec["z"], eps=eps, mu=spec["mu"])
        J.add_source(*src)
        J.add_probe(node, om)
        return J

    I = make(I0.eps)
    L, grad = I.adjoint(0, range(len(om)), wl.n_steps)

    def loss(eps):
        J = make(eps)
        J.run(wl.n_steps)
        return float(np.sum(np.abs(J.spectrum(0)) ** 2))

    assert abs(loss(I0.eps) - L) <= 1e-12 * L
    assert np.abs(grad[1:-1]).max() > 0
    h = 1e-4
    for j in (1, 7, 20, 33, 48):
        ep, em = I0.eps.copy(), I0.eps.copy()
        ep[j] += h
        em[j] -= h
        fd = (loss(ep) - loss(em)) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-6 * np.abs(grad).max() + 1e-6 * abs(fd), (j, fd, grad[j])
