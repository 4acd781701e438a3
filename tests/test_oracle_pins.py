"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the worked
example printed in Sec. 5, textbook Yee, exact symmetries of Table 1, the
closed-form scattering coefficients of Appendix B, the Doppler/compression
factors of Eq. comp_exp, and library routines for the DFT probes.
"""
import json
import os

import numpy as np
import pytest

from oracle import Instance, exact
from oracle import vonneumann as vn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Sec. 5 pin

def test_worked_example_zeta_matches_paper():
    """Sec. 5 worked example: the amplification eigenvalues, to the printed digits."""
    g = json.load(open(os.path.join(GOLDEN, "worked_example_sec5.json")))
    zp, zm = vn.zeta_pm(g["S"], g["beta"], g["eps"], g["mu"], g["kz_dz_over_pi"] * np.pi)
    assert abs(zp.real - g["zeta_plus"][0]) <= 0.0005
    assert abs(zp.imag - g["zeta_plus"][1]) <= 0.005
    assert abs(zm.real - g["zeta_minus"][0]) <= 0.0005
    assert abs(zm.imag - g["zeta_minus"][1]) <= 0.005
    assert abs(abs(zp) - g["abs_zeta_plus"]) <= 0.005
    assert abs(abs(zm) - g["abs_zeta_minus"]) <= 0.005


@pytest.mark.parametrize("beta", [0.3, -0.3, 0.0, 0.7])
@pytest.mark.parametrize("which", ["+", "-"])
def test_oracle_step_multiplies_eigenmode_by_zeta(beta, which):
    """One oracle step applied to a discrete plane wave multiplies it by zeta (Eq. PW_test_field)."""
    S, eps, mu, th = 0.5, 4.0, 1.0, 2 * np.pi / 5
    z, Bh, Dh = vn.eigenmode(S, beta, eps, mu, th, which)
    nz = 64
    k = np.arange(nz)
    out = []
    for part in (np.real, np.imag):   # the scheme is real-linear: step real and imaginary parts
        I = Instance(nz, S, beta, eps=[eps], mu=[mu])
        I.B[:] = part(Bh * np.exp(1j * th * (k + 0.5)))
        I.D[:] = part(Dh * np.exp(1j * th * k))
        I.run(1)
        out.append((I.B.copy(), I.D.copy()))
    Bc = out[0][0] + 1j * out[1][0]
    Dc = out[0][1] + 1j * out[1][1]
    sl = slice(4, nz - 4)               # away from the zero ghost cells
    np.testing.assert_allclose(Bc[sl], z * Bh * np.exp(1j * th * (k[sl] + 0.5)), atol=1e-13)
    np.testing.assert_allclose(Dc[sl], z * Dh * np.exp(1j * th * k[sl]), atol=1e-13)


def test_negative_velocity_gives_conjugate_pair():
    """App. A: the characteristic polynomial for v < 0 gives the same |zeta| (conjugate pair)."""
    for th in np.linspace(0.1, 3.0, 7):
        a = np.sort_complex(vn.zetas(0.5, 0.3, 4.0, 1.0, th))
        b = np.sort_complex(np.conj(vn.zetas(0.5, -0.3, 4.0, 1.0, th)))
        np.testing.assert_allclose(a, b, atol=1e-12)


# ------------------------------------------------------ v = 0: textbook Yee

def _textbook_yee(B, D, eps_k, mu_j, S, n_steps):
    """Standard 1D Yee (E = D/eps, H = B/mu), zero fields outside the grid."""
    B, D = B.copy(), D.copy()
    for _ in range(n_steps):
        E = np.append(D / eps_k, 0.0)
        B = B - S * (E[1:] - E[:-1])
        H = np.concatenate(([0.0], B / mu_j))
        D = D - S * (H[1:] - H[:-1])
    return B, D


def test_zero_velocity_is_textbook_yee():
    """Sec. 3: with v = 0 the generalized cell is the standard Yee cell."""
    rng = np.random.default_rng(1)
    nz, S = 300, 0.7
    z = [80.0, 150.5, 222.0]
    eps, mu = [1.0, 3.0, 2.0, 5.0], [1.0, 1.5, 1.0, 2.0]
    I = Instance(nz, S, 0.0, eps=eps, mu=mu, z=z)
    B0, D0 = rng.standard_normal(nz), rng.standard_normal(nz)
    I.B[:], I.D[:] = B0, D0
    I.run(50)
    ek = I.material("eps", half_node=False, h=1)
    mj = I.material("mu", half_node=True, h=0)
    # static medium: sampled directly from the layer boundaries
    kk = np.arange(nz)
    ek_ref = np.array(eps)[np.searchsorted(z, kk, side="right")]
    mj_ref = np.array(mu)[np.searchsorted(z, kk + 0.5, side="right")]
    np.testing.assert_array_equal(ek, ek_ref)
    np.testing.assert_array_equal(mj, mj_ref)
    Br, Dr = _textbook_yee(B0, D0, ek_ref, mj_ref, S, 50)
    np.testing.assert_allclose(I.B, Br, rtol=0, atol=1e-12)
    np.testing.assert_allclose(I.D, Dr, rtol=0, atol=1e-12)


# ----------------------------------------------------- Table 1 mirror symmetry

def test_mirror_symmetry_between_table_columns():
    """Table 1's v<0 column is the mirror image of the v>0 column (z -> -z, B -> -B).

    A compactly supported random field run with +beta and its mirror image run
    with -beta stay mirror images (the domain ends are never reached).
    """
    rng = np.random.default_rng(2)
    nz, S, beta, steps = 400, 0.5, 0.37, 40
    B0 = np.zeros(nz)
    D0 = np.zeros(nz)
    B0[180:220] = rng.standard_normal(40)
    D0[180:220] = rng.standard_normal(40)
    # moving layers around the centre; mirror of boundary z is (nz-1) - z for D nodes
    zb = [190.25, 205.5]
    eps = [1.0, 4.0, 2.0]
    A = Instance(nz, S, beta, eps=eps, z=zb)
    A.B[:], A.D[:] = B0, D0
    A.run(steps)
    # mirror: D'_k = D_{nz-1-k}, B'_j = -B_{nz-2-j}; profile mirrored about node (nz-1)/2
    zm = sorted((nz - 1) - np.array(zb))
    M = Instance(nz, S, -beta, eps=eps[::-1], z=zm)
    M.D[:] = D0[::-1]
    M.B[:-1] = -B0[:-1][::-1]
    M.run(steps)
    # half-open layers flip to half-closed under the mirror; boundaries here never hit nodes
    np.testing.assert_allclose(M.D, A.D[::-1], atol=1e-13)
    np.testing.assert_allclose(M.B[:-1], -A.B[:-1][::-1], atol=1e-13)


# ------------------------------------------------------------ stability (S2)

def test_stability_threshold_n_beta_equals_one():
    """The scheme is von Neumann stable iff n|beta| <= 1 (checked on both sides)."""
    for eps, beta in [(4.0, 0.45), (4.0, -0.45), (1.0, 0.95), (2.0, 0.7)]:
        assert vn.max_growth(0.5, beta, eps, 1.0) <= 1 + 1e-9
    for eps, beta in [(4.0, 0.6), (4.0, -0.6), (6.0, 0.7)]:
        assert vn.max_growth(0.5, beta, eps, 1.0) > 1 + 1e-5


def test_unstable_run_grows_at_von_neumann_rate():
    """In an unstable uniform medium the oracle's field grows at max|zeta| per step."""
    S, beta, eps = 0.5, 0.8, 4.0
    g = vn.max_growth(S, beta, eps, 1.0, n_theta=8192)
    nz = 4096
    rng = np.random.default_rng(3)
    I = Instance(nz, S, beta, eps=[eps])
    I.B[:] = rng.standard_normal(nz) * 1e-6
    I.D[:] = rng.standard_normal(nz) * 1e-6
    I.run(1500)
    a = np.linalg.norm(I.D[1024:3072])
    I.run(500)
    b = np.linalg.norm(I.D[1024:3072])
    rate = (b / a) ** (1 / 500)
    assert abs(rate - g) < 2e-4, (rate, g)


# -------------------------------------------------------------- DFT probes

def test_dft_probe_matches_library_fft():
    """Probe accumulators equal sum F_n exp(i w t_n) dt, checked against numpy's FFT."""
    rng = np.random.default_rng(4)
    nz, S, N = 50, 0.5, 256
    I = Instance(nz, S, 0.2, eps=[1.0])
    I.B[:] = rng.standard_normal(nz)
    I.D[:] = rng.standard_normal(nz)
    w = 2 * np.pi * np.arange(N) / (N * S)   # FFT grid frequencies
    pid = I.add_probe(25, w)
    I.run(N, record=True)
    F = I.series(pid)
    t = (np.arange(N) + 1.5) * S            # t_{n+1/2}, n = 1..N
    # sum_n F_n e^{i w_m t_n} S = S e^{i w_m t_1} * sum_n F_n e^{2 pi i m n / N}
    ref = S * np.exp(1j * w * t[0]) * np.fft.ifft(F) * N
    np.testing.assert_allclose(I.spectrum(pid), ref, rtol=1e-11, atol=1e-11)


def test_source_radiates_closed_form_spectrum():
    """A soft source radiates the Gaussian-modulated carrier of Eq. spectrum_incident.

    Adding s(t) to D at one node every step is a current sheet of strength
    s/dt; in 1D it radiates E = s(t - |z|/c) / (2 dt) each way.  The probe
    spectrum therefore equals the continuous transform of
    s(t) = sin(w0 (t - t0)) exp(-((t - t0)/tau)^2), which is
    exp(i w t0) tau sqrt(pi)/(2i) [exp(-tau^2 (w + w0)^2/4) - exp(-tau^2 (w - w0)^2/4)],
    delayed by the path and divided by 2 dt.
    """
    S, lam0 = 0.5, 80.0
    w0 = 2 * np.pi / lam0
    tau = 3 * lam0 / (2 * np.sqrt(np.log(2)))
    t0 = 4 * tau
    N = int(2 * t0 / S) + 400
    k = 120
    J = Instance(4001, S, 0.0, eps=[1.0])
    J.add_source(2000, w0, tau, t0, 1.0)
    for w in (0.9 * w0, w0, 1.1 * w0):
        J.add_probe(2000 + k, [w])
    J.run(N)
    for i, w in enumerate((0.9 * w0, w0, 1.1 * w0)):
        F = (np.exp(1j * w * t0) * tau * np.sqrt(np.pi) / 2j
             * (np.exp(-tau ** 2 * (w + w0) ** 2 / 4) - np.exp(-tau ** 2 * (w - w0) ** 2 / 4)))
        expect = F * np.exp(1j * w * k) / (2 * S)
        got = J.spectrum(i)[0]
        assert abs(abs(got) / abs(expect) - 1) < 5e-3, (w, got, expect)
        assert abs(np.angle(got / expect)) < 0.02, (w, got, expect)


# ------------------------------------------- moving interface (App. B.2)

def _gauss_source(lam0, fwhm_periods):
    w0 = 2 * np.pi / lam0
    tau = fwhm_periods * lam0 / (2 * np.sqrt(np.log(2)))
    return w0, tau, 4 * tau


@pytest.mark.slow
def test_contra_moving_interface_coefficients():
    """Fig. 5 parameters (v=-0.3c, eps1=2, eps2=4, S=0.2, dz=lambda0/150).

    |Gamma| and |T| from ratios of probe spectra (Eq. spectrum_scat_interface)
    match Eq. coef_interface within 1% after removing the scheme's own
    propagation loss (Sec. 5 analysis) over the probe paths.  The peak
    frequencies follow the compression factors of Eq. comp_exp, i.e. the
    moving-frame frequency omega - v k is conserved.
    """
    beta, e1, e2, S, lam0 = -0.3, 2.0, 4.0, 0.2, 150.0
    w0, tau, t0 = _gauss_source(lam0, 3)
    zs, zI, zr, zt, nz, t_end = 1000, 3000, 1800, 2800, 4500, 4800.0
    steps = int(t_end / S)
    ex = exact.interface(e1, e2, beta)
    runs = {}
    for tag, eps, z in (("A", [e1, e2], [zI]), ("R", [e1], [])):
        I = Instance(nz, S, beta, eps=eps, z=z)
        I.add_source(zs, w0, tau, t0)
        I.add_probe(zr, [w0])
        I.add_probe(zt, [w0])
        I.run(steps, record=True)
        runs[tag] = (I.series(0), I.series(1))
    t = (np.arange(steps) + 1.5) * S

    def X(f, w, mask=None):
        f = f if mask is None else f * mask
        return np.sum(f * np.exp(1j * w * t)) * S

    n1 = np.sqrt(e1)
    # meeting point of the pulse centre with the interface
    tm = (zI - zs + t0 / n1) / (1 / n1 - beta)
    zm = zI + beta * tm
    for f in (0.95, 1.0, 1.05):
        w = f * w0
        Xi = X(runs["R"][0], w, t < 3800)
        Xr = X(runs["A"][0] - runs["R"][0], ex["a_r"] * w, t < 3950)
        Xt = X(runs["A"][1], ex["a_t"] * w)
        li = vn.propagation_loss(S, beta, e1, 1.0, w, zm - zr, +1)
        lr = vn.propagation_loss(S, beta, e1, 1.0, ex["a_r"] * w, zm - zr, -1)
        lt = vn.propagation_loss(S, beta, e2, 1.0, ex["a_t"] * w, zt - zm, +1)
        G = ex["a_r"] * abs(Xr) / abs(Xi) / (li * lr)
        T = ex["a_t"] * abs(Xt) / abs(Xi) / (li * lt)
        assert abs(G / abs(ex["Gamma"]) - 1) < 0.01, (f, G, ex["Gamma"])
        assert abs(T / abs(ex["T"]) - 1) < 0.01, (f, T, ex["T"])
    # Doppler: spectral peaks at a_r w0 (reflected) and a_t w0 (transmitted)
    ws = np.linspace(0.2 * w0, 4 * w0, 1500)
    Pr = np.abs([X(runs["A"][0] - runs["R"][0], w, t < 3950) for w in ws])
    Pt = np.abs([X(runs["A"][1], w) for w in ws])
    Pi = np.abs([X(runs["R"][0], w, t < 3800) for w in ws])
    wi, wr, wt = ws[np.argmax(Pi)], ws[np.argmax(Pr)], ws[np.argmax(Pt)]
    assert abs(wr / wi - ex["a_r"]) < 0.02 * ex["a_r"]
    assert abs(wt / wi - ex["a_t"]) < 0.02 * ex["a_t"]
    # conserved moving-frame frequency: omega (1 - n beta) for +z waves, (1 + n beta) for -z
    n2 = np.sqrt(e2)
    Om_i, Om_r, Om_t = wi * (1 - n1 * beta), wr * (1 + n1 * beta), wt * (1 - n2 * beta)
    assert abs(Om_r / Om_i - 1) < 0.02 and abs(Om_t / Om_i - 1) < 0.02


# -------------------------------------------------- transfer matrix (App. B)

def test_star_tmm_reduces_to_interface_and_slab():
    """The star-amplitude TMM reproduces Eq. coef_interface and Eq. coef_slab, and
    with beta = 0 the textbook transfer matrix."""
    for beta in (-0.3, 0.0, 0.3):
        ex = exact.interface(2.0, 4.0, beta)
        T, G = exact.star_tmm([2.0, 4.0], [1.0, 1.0], [], beta, 0.05)
        assert abs(T - ex["T"]) < 1e-12 and abs(G - ex["Gamma"]) < 1e-12
        for ell in (17.0, 55.5):
            Ts, Gs = exact.slab_closed_form(1.0, 4.0, beta, ell, 0.05)
            T3, G3 = exact.star_tmm([1.0, 4.0, 1.0], [1.0] * 3, [ell], beta, 0.05)
            assert abs(abs(T3) - abs(Ts)) < 1e-12 and abs(abs(G3) - abs(Gs)) < 1e-12
    # beta = 0 slab: |t|^2 + |r|^2 = 1 (energy) and quarter-wave closed form
    n2, w = 2.0, 0.05
    ell = np.pi / (2 * n2 * w)
    T, G = exact.star_tmm([1.0, 4.0, 1.0], [1.0] * 3, [ell], 0.0, w)
    assert abs(abs(T) ** 2 + abs(G) ** 2 - 1) < 1e-12
    assert abs(abs(G) - (n2 ** 2 - 1) / (n2 ** 2 + 1)) < 1e-12


def test_matter_slab_lorentz_limits():
    """Moving-matter slab: beta = 0 is the rest Fabry-Perot slab; |t|^2 + |r'|^2 = 1 in the rest frame."""
    t, r, wr = exact.matter_slab(3.0, 800.0, 0.0, 0.1)
    T, G = exact.star_tmm([1.0, 9.0, 1.0], [1.0] * 3, [800.0], 0.0, 0.1)
    assert abs(abs(t) - abs(T)) < 1e-12 and abs(abs(r) - abs(G)) < 1e-12 and wr == 0.1
    for beta in (-0.5, 0.2, 0.5):
        t, r, wr = exact.matter_slab(3.0, 800.0, beta, 0.1)
        rp = r * (1 + beta) / (1 - beta)
        assert abs(abs(t) ** 2 + abs(rp) ** 2 - 1) < 1e-12


# --------------------------------------------------------- moving matter

def test_matter_scheme_at_rest_is_textbook_yee():
    """Moving matter with beta = 0 reduces to Yee with E* = D/eps'."""
    rng = np.random.default_rng(5)
    nz, S = 200, 0.5
    z, eps, mu = [60.0, 130.0], [1.0, 9.0, 2.0], [1.0, 1.0, 1.5]
    I = Instance(nz, S, 0.0, kind=1, eps=eps, mu=mu, z=z)
    B0, D0 = rng.standard_normal(nz), rng.standard_normal(nz)
    kk = np.arange(nz)
    ek = np.array(eps)[np.searchsorted(z, kk, side="right")]
    mj = np.array(mu)[np.searchsorted(z, kk + 0.5, side="right")]
    I.B[:], I.D[:] = B0, D0
    I.run(30)
    Br, Dr = _textbook_yee(B0, D0, ek, mj, S, 30)
    np.testing.assert_allclose(I.B, Br, atol=1e-12)
    np.testing.assert_allclose(I.D, Dr, atol=1e-12)


def test_matter_phase_velocity_is_fizeau():
    """In uniform moving matter the scheme's phase velocity converges to relativistic
    velocity addition (Fizeau drag), for both propagation directions."""
    S, n = 0.5, 3.0
    for beta in (-0.5, 0.2, 0.5):
        th = 2 * np.pi / 800
        z = np.linalg.eigvals(vn.amplification_matter(S, beta, n * n, 1.0, th))
        vp = sorted(-np.angle(z[np.abs(z) > 0.5]) / S / th)
        assert abs(vp[0] - exact.fizeau_velocity(n, beta, False)) < 1e-4
        assert abs(vp[1] - exact.fizeau_velocity(n, beta, True)) < 1e-4


def test_matter_scheme_stable_at_config_velocities():
    for beta in (-0.5, -0.2, 0.0, 0.2, 0.5):
        for eps in (1.0, 9.0):
            assert vn.max_growth(0.5, beta, eps, 1.0, kind=1, n_theta=1024) <= 1 + 1e-9


def test_oracle_matter_step_matches_amplification_matrix():
    """One oracle step of moving matter applied to each eigenmode of its amplification matrix."""
    S, beta, eps, th = 0.5, 0.4, 9.0, 2 * np.pi / 7
    G = vn.amplification_matter(S, beta, eps, 1.0, th)
    zs, V = np.linalg.eig(G)
    nz = 64
    k = np.arange(nz)
    sl = slice(4, nz - 4)
    for i in range(2):
        out = []
        for part in (np.real, np.imag):
            I = Instance(nz, S, beta, kind=1, eps=[eps])
            I.B[:] = part(V[0, i] * np.exp(1j * th * (k + 0.5)))
            I.D[:] = part(V[1, i] * np.exp(1j * th * k))
            I.run(1)
            out.append((I.B.copy(), I.D.copy()))
        for f, ph in ((0, 0.5), (1, 0.0)):
            got = out[0][f] + 1j * out[1][f]
            np.testing.assert_allclose(got[sl], zs[i] * V[f, i] * np.exp(1j * th * (k[sl] + ph)),
                                       atol=1e-13)


def test_matter_in_moving_vacuum_is_the_perturbation_scheme():
    """Moving matter with eps' = mu' = 1 is vacuum; the update equals the moving-perturbation one."""
    rng = np.random.default_rng(6)
    nz, S = 200, 0.5
    for beta in (0.45, -0.3):
        A = Instance(nz, S, beta, kind=1, eps=[1.0])
        P = Instance(nz, S, beta, kind=0, eps=[1.0])
        B0, D0 = rng.standard_normal(nz), rng.standard_normal(nz)
        A.B[:], A.D[:] = B0, D0
        P.B[:], P.D[:] = B0, D0
        A.run(25)
        P.run(25)
        np.testing.assert_allclose(A.B, P.B, atol=1e-12)
        np.testing.assert_allclose(A.D, P.D, atol=1e-12)


@pytest.mark.slow
def test_matter_interface_first_pass_reflection():
    """A pulse hitting a moving-matter half space (n'=3) reflects with
    r = r12' (1-beta)/(1+beta) at frequency w (1-beta)/(1+beta) (Lorentz
    transformation of the rest-frame Fresnel coefficient)."""
    S, lam0, n = 0.5, 160.0, 3.0
    w0, tau, t0 = _gauss_source(lam0, 2)
    # windows end before the source's echo off z = 0 returns from the interface
    for beta, steps, t_win in ((-0.2, 9000, 3950.0), (0.2, 14000, 7000.0)):
        zs, zI, zr, nz = 800, 3000, 1600, 6000
        runs = {}
        for tag, eps, z in (("A", [1.0, n * n], [float(zI)]), ("R", [1.0], [])):
            I = Instance(nz, S, beta, kind=1, eps=eps, z=z)
            I.add_source(zs, w0, tau, t0)
            I.add_probe(zr, [w0])
            I.run(steps, record=True)
            runs[tag] = I.series(0)
        t = (np.arange(steps) + 1.5) * S
        ar = (1 - beta) / (1 + beta)
        Xi = np.sum(runs["R"] * (t < 2500.0) * np.exp(1j * w0 * t)) * S   # before the echo
        Xr = np.sum((runs["A"] - runs["R"]) * (t < t_win) * np.exp(1j * ar * w0 * t)) * S
        r = ar * abs(Xr) / abs(Xi)
        assert abs(r / abs(exact.matter_interface_reflection(n, beta)) - 1) < 0.01, (beta, r)


def test_scheme_doppler_factor_tends_to_eq_comp_exp():
    """The scheme's own Doppler factors (w - v k conserved across the moving
    interface with the scheme's wavenumbers) converge to Eq. comp_exp's a_t, a_r
    as the mesh is refined, at second order (error x 1/100 per 10x finer)."""
    from oracle import vonneumann as vn
    for beta, e1, e2 in ((0.3, 1.0, 4.0), (-0.3, 2.0, 4.0), (0.45, 1.5, 2.0)):
        ex = exact.interface(e1, e2, beta)
        err = {}
        for lam in (400.0, 4000.0):
            om = 2 * np.pi / lam
            err[lam] = (vn.doppler_factor(0.5, beta, e1, e2, om, +1) / ex["a_t"] - 1,
                        vn.doppler_factor(0.5, beta, e1, e1, om, -1) / ex["a_r"] - 1)
        for j in (0, 1):
            assert abs(err[4000.0][j]) < 1e-5, (beta, err)
            assert 80 < err[400.0][j] / err[4000.0][j] < 120, (beta, err)
