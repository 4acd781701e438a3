"""GPU results against the exact solutions the paper gives (App. B): the
moving-interface reflection and transmission coefficients of Eq.
coef_interface within 1 % at 150 cells per wavelength (Fig. 5 parameters),
measured with a one-way source so that the scattered-field probe records the
reflected pulse alone, and the Doppler factors of Eq. comp_exp."""
import numpy as np
import pytest

from paper_2304_06586_gb300 import binding as gb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


@pytest.mark.parametrize("prec", [gb.F32, gb.F32_KAHAN])
def test_moving_interface_coefficients_on_gpu(prec):
    from oracle import exact
    from oracle import vonneumann as vn
    beta, e1, e2, S, lam0 = -0.3, 2.0, 4.0, 0.2, 150.0
    w0 = 2 * np.pi / lam0
    tau = 3 * lam0 / (2 * np.sqrt(np.log(2)))
    t0 = 4 * tau
    q, zI, zr, zi, zt, nz, t_end = 1000, 3000, 950, 1050, 2800, 4500, 6000.0
    steps = int(t_end / S)
    ex = exact.interface(e1, e2, beta)
    fs = np.array([0.95, 1.0, 1.05])
    # instance 0: the interface; instance 1: the same background without it (incident wave alone)
    sim = gb.Simulation([nz, nz], S, prec)
    sim.set_medium(0, gb.PERTURBATION, beta, gb.LAYERS, [zI], [e1, e2], [1.0, 1.0])
    sim.set_medium(1, gb.PERTURBATION, beta, gb.LAYERS, [], [e1], [1.0])
    for k in (0, 1):
        sim.add_tfsf(k, q, w0, tau, t0)
        sim.set_absorber(k, 64, 0.2)
    sim.add_probe(0, zr, ex["a_r"] * fs * w0)        # probe 0: reflected (scattered field)
    sim.add_probe(0, zt, ex["a_t"] * fs * w0)        # probe 1: transmitted
    sim.add_probe(1, zi, fs * w0)                    # incident, total field without scatterer
    sim.step(steps)
    Xr = np.abs(sim.read_spectrum(0, 0, 3))
    Xt = np.abs(sim.read_spectrum(0, 1, 3))
    Xi = np.abs(sim.read_spectrum(1, 0, 3))
    n1 = np.sqrt(e1)
    src = q - 12                                     # the auxiliary soft source's position
    tm = (zI - src + t0 / n1) / (1 / n1 - beta)      # pulse centre meets the interface
    zm = zI + beta * tm
    for j, f in enumerate(fs):
        w = f * w0
        li = vn.propagation_loss(S, beta, e1, 1.0, w, zm - zi, +1)
        lr = vn.propagation_loss(S, beta, e1, 1.0, ex["a_r"] * w, zm - zr, -1)
        lt = vn.propagation_loss(S, beta, e2, 1.0, ex["a_t"] * w, zt - zm, +1)
        G = ex["a_r"] * Xr[j] / Xi[j] / (li * lr)
        T = ex["a_t"] * Xt[j] / Xi[j] / (li * lt)
        assert abs(G / abs(ex["Gamma"]) - 1) < 0.01, (f, G, ex["Gamma"])
        assert abs(T / abs(ex["T"]) - 1) < 0.01, (f, T, ex["T"])


@pytest.mark.parametrize("beta", [0.2, -0.2])
def test_moving_slab_transmission_on_gpu(beta):
    """|T| of a moving slab (eps 1 | 4 | 1, 450 cells, Eq. coef_slab) at 300
    cells per vacuum wavelength: the transmitted spectrum over that of the
    same background without the slab, within 1 % over 0.9-1.1 w0 (the
    Fabry-Perot phase inside the slab makes |T| sensitive to the scheme's
    phase error, which falls with the square of the resolution)."""
    from oracle import exact
    e1, e2, S, lam0 = 1.0, 4.0, 0.5, 300.0
    w0 = 2 * np.pi / lam0
    tau = 6 * lam0 / (2 * np.sqrt(np.log(2)))
    t0 = 4 * tau
    q, z0, ell, zt, nz, steps = 2400, 7000.0, 450.0, 17200, 20000, 80000
    fs = np.array([0.9, 0.95, 1.0, 1.05, 1.1])
    sim = gb.Simulation([nz, nz], S, gb.F32_KAHAN)
    sim.set_medium(0, gb.PERTURBATION, beta, gb.LAYERS, [z0, z0 + ell], [e1, e2, e1], [1.0] * 3)
    sim.set_medium(1, gb.PERTURBATION, beta, gb.LAYERS, [], [e1], [1.0])
    for k in (0, 1):
        sim.add_tfsf(k, q, w0, tau, t0)
        sim.set_absorber(k, 64, 0.2)
        sim.add_probe(k, zt, fs * w0)
    sim.step(steps)
    T = np.abs(sim.read_spectrum(0, 0, len(fs))) / np.abs(sim.read_spectrum(1, 0, len(fs)))
    for j, f in enumerate(fs):
        Tex, _ = exact.slab_closed_form(e1, e2, beta, ell, f * w0)
        assert abs(T[j] / abs(Tex) - 1) < 0.01, (beta, f, T[j], abs(Tex))
