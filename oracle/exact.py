"""Exact scattering results for moving structures (test infrastructure only).

Closed forms of Appendix B of the paper, plus two results the paper relies on
but does not print in usable form:

* ``interface``: Eq. coef_interface (T_21, Gamma_121) and Eq. comp_exp
  (compression factors a_t, a_r).
* ``slab_closed_form``: Eq. coef_slab with the omega_2^+/- expressions under it.
  The text prints exp(+i...) in the denominator of Gamma and exp(-i...) in
  that of T; the multiple-reflection sum gives the same exponent in both, which
  is what is used here (only the magnitudes are compared in tests, and those do
  not depend on the sign convention once it is consistent).
* ``star_tmm``: transfer-matrix method for a stack of moving-perturbation
  layers (Appendix B.3).  The printed matrices carry typos (gamma_nmn reduces
  to 1, Gamma = -A/D); this version is derived from the interface conditions
  Eq. cont and the star fields Eq. star.  In the frame that moves with the
  structure every wave has the same frequency Omega = omega_i (1 - n_1 beta)
  (the invariant behind Eq. comp_exp), and the star amplitudes
  u+ = E+ (1 - n beta), u- = E- (1 + n beta) obey ordinary Fresnel matching
  with impedance eta = sqrt(mu/eps), because E* = u+ + u- and
  H* = (u+ - u-)/eta.  With three layers it reduces to the slab closed form,
  and with beta = 0 to the textbook transfer matrix.
* ``matter_slab``: a moving-matter slab (rest index n', lab thickness L) in
  vacuum, from the Lorentz transformation of the rest-frame Fabry-Perot
  solution: t = t'(omega'), r = r'(omega') (1 - beta)/(1 + beta), with
  omega' = omega sqrt((1 - beta)/(1 + beta)) and rest thickness gamma L.

Units: c = 1, beta = v/c, lengths in cells, omega in rad per unit time.
"""
import numpy as np


def interface(eps1, eps2, beta, mu1=1.0, mu2=1.0):
    """Eq. coef_interface and Eq. comp_exp for incidence from medium 1 onto medium 2."""
    n1, n2 = np.sqrt(eps1 * mu1), np.sqrt(eps2 * mu2)
    eta1, eta2 = np.sqrt(mu1 / eps1), np.sqrt(mu2 / eps2)
    T = 2 * eta2 / (eta1 + eta2) * (1 - n1 * beta) / (1 - n2 * beta)
    G = (eta2 - eta1) / (eta1 + eta2) * (1 - n1 * beta) / (1 + n1 * beta)
    a_t = (1 - n1 * beta) / (1 - n2 * beta)
    a_r = (1 - n1 * beta) / (1 + n1 * beta)
    return {"T": T, "Gamma": G, "a_t": a_t, "a_r": a_r}


def slab_closed_form(eps1, eps2, beta, ell, omega_i, mu1=1.0, mu2=1.0):
    """Eq. coef_slab: medium 1 | slab of medium 2, lab length ell | medium 1."""
    n1, n2 = np.sqrt(eps1 * mu1), np.sqrt(eps2 * mu2)
    f12 = interface(eps1, eps2, beta, mu1, mu2)
    f21 = interface(eps2, eps1, beta, mu2, mu1)
    T21, G121 = f12["T"], f12["Gamma"]
    T12 = f21["T"]
    G212 = f21["Gamma"]
    G212m = interface(eps2, eps1, -beta, mu2, mu1)["Gamma"]
    w2p = (1 - n1 * beta) / (1 - n2 * beta) * omega_i
    w2m = (1 - n1 * beta) / (1 + n2 * beta) * omega_i
    rt = np.exp(-1j * (w2p + w2m) * n2 * ell)
    T = T21 * T12 * np.exp(-1j * w2p * n2 * ell) / (1 - G212 * G212m * rt)
    G = G121 * (1 - rt) / (1 - G212 * G212m * rt)
    return T, G


def star_tmm(eps, mu, thick, beta, omega_i):
    """Scattering of a moving stack: layers 0 and N-1 are the semi-infinite media.

    eps, mu: per layer; thick: lengths of layers 1..N-2 (moving frame);
    omega_i: lab frequency of the incident wave in layer 0 (travelling +z).
    Returns (T, Gamma) as ratios of physical E amplitudes at the first and last
    interfaces.
    """
    eps = np.asarray(eps, float)
    mu = np.asarray(mu, float)
    n = np.sqrt(eps * mu)
    eta = np.sqrt(mu / eps)
    Om = omega_i * (1 - n[0] * beta)
    kp = n * Om / (1 - n * beta)      # lab wavenumber of the +z wave in each layer
    km = n * Om / (1 + n * beta)      # lab wavenumber magnitude of the -z wave
    # M maps (u+, u-) just left of the first interface to just right of the last one
    M = np.eye(2, dtype=complex)
    for m in range(len(eps) - 1):
        a, b = eta[m], eta[m + 1]
        # continuity of E* = u+ + u- and H* = (u+ - u-)/eta
        I = 0.5 * np.array([[1 + b / a, 1 - b / a], [1 - b / a, 1 + b / a]])
        M = I @ M
        if m + 1 < len(eps) - 1:
            L = thick[m]
            P = np.diag([np.exp(1j * kp[m + 1] * L), np.exp(-1j * km[m + 1] * L)])
            M = P @ M
    # right side: u_N- = 0.  [uN+, 0] = M [u1+, u1-]
    u1p = 1 - n[0] * beta
    u1m = -M[1, 0] * u1p / M[1, 1]
    uNp = M[0, 0] * u1p + M[0, 1] * u1m
    T = uNp / (1 - n[-1] * beta)
    G = u1m / (1 + n[0] * beta)
    return T, G


def matter_slab(n_rest, L, beta, omega):
    """Moving-matter slab in vacuum (rest index n_rest, lab length L, velocity beta).

    Returns (t, r, omega_r): transmission at the incident frequency and
    reflection at the Doppler-shifted frequency omega_r.
    """
    gam = 1.0 / np.sqrt(1 - beta * beta)
    wp = omega * np.sqrt((1 - beta) / (1 + beta))
    Lp = gam * L
    r12 = (1 - n_rest) / (1 + n_rest)
    e2 = np.exp(2j * n_rest * wp * Lp)
    rp = r12 * (1 - e2) / (1 - r12 * r12 * e2)
    tp = (1 - r12 * r12) * np.exp(1j * n_rest * wp * Lp) / (1 - r12 * r12 * e2)
    return tp, rp * (1 - beta) / (1 + beta), omega * (1 - beta) / (1 + beta)


def matter_interface_reflection(n_rest, beta):
    """First-pass reflection from vacuum onto a moving-matter half space."""
    return (1 - n_rest) / (1 + n_rest) * (1 - beta) / (1 + beta)


def fizeau_velocity(n_rest, beta, forward=True):
    """Lab-frame phase velocity in matter moving at beta (relativistic velocity addition)."""
    u = 1.0 / n_rest if forward else -1.0 / n_rest
    return (u + beta) / (1 + u * beta)


def oblique_interface(eps1, eps2, beta, kx, omega, mu1=1.0, mu2=1.0):
    """TE (E along y) plane wave of lab frequency omega and transverse
    wavenumber kx arriving from medium 1 on a moving-perturbation interface
    z = z0 + beta t (normal along the motion, oblique incidence).  Derived
    from Eq. cont and Eq. star: in each uniform medium the wave is an ordinary
    plane wave (kx^2 + kz^2 = omega^2 n^2, B = k x E / omega), all waves share kx
    and the frequency seen by the interface, Omega = omega - beta kz, and the
    tangential star fields E*_y = E_y (1 - beta kz/omega) and
    H*_x = E_y (-kz/(omega mu) + beta eps) are continuous.  Returns
    (Gamma, T, omega_r, omega_t, domega_r/domega): reflection and transmission
    as ratios of E_y amplitudes, the reflected and transmitted lab frequencies
    and the slope of omega_r(omega) at fixed kx (the spectral compression of
    the reflected pulse).  kx = 0 gives Eq. coef_interface and Eq. comp_exp;
    beta = 0 the TE Fresnel coefficients."""
    n1, n2 = np.sqrt(eps1 * mu1), np.sqrt(eps2 * mu2)

    def kz(w, n, sign):
        return sign * np.sqrt(w * w * n * n - kx * kx + 0j)

    kz1 = kz(omega, n1, 1).real
    Om = omega - beta * kz1

    def leaving(n, sign):
        # omega_out - beta kz_out = Om with kz_out = sign sqrt(omega_out^2 n^2 - kx^2)
        a = 1 - beta * beta * n * n
        b = -2 * Om
        c = Om * Om + beta * beta * kx * kx
        disc = np.sqrt(b * b - 4 * a * c)
        for w in ((-b - disc) / (2 * a), (-b + disc) / (2 * a)):
            if w > 0 and w * n >= abs(kx):
                k = kz(w, n, sign).real
                if abs(w - beta * k - Om) < 1e-9 * abs(Om):
                    return w, k
        raise ValueError("no propagating wave leaves the interface")

    wr, kzr = leaving(n1, -1)
    wt, kzt = leaving(n2, +1)

    def star(w, k, eps, mu):
        return 1 - beta * k / w, -k / (w * mu) + beta * eps

    ei, hi = star(omega, kz1, eps1, mu1)
    er, hr = star(wr, kzr, eps1, mu1)
    et, ht = star(wt, kzt, eps2, mu2)
    M = np.array([[er, -et], [hr, -ht]])
    G, T = np.linalg.solve(M, -np.array([ei, hi]))
    dw = 1e-7 * omega
    wr_p = oblique_interface_frequency(eps1, beta, kx, omega + dw, mu1)
    wr_m = oblique_interface_frequency(eps1, beta, kx, omega - dw, mu1)
    return G, T, wr, wt, (wr_p - wr_m) / (2 * dw)


def oblique_interface_frequency(eps1, beta, kx, omega, mu1=1.0):
    """Lab frequency of the wave reflected by the moving interface (see
    oblique_interface): omega_r - beta kz_r = omega - beta kz_i, kz_r < 0."""
    n1 = np.sqrt(eps1 * mu1)
    kz1 = np.sqrt(omega * omega * n1 * n1 - kx * kx)
    Om = omega - beta * kz1
    a = 1 - beta * beta * n1 * n1
    b = -2 * Om
    c = Om * Om + beta * beta * kx * kx
    disc = np.sqrt(b * b - 4 * a * c)
    for w in ((-b - disc) / (2 * a), (-b + disc) / (2 * a)):
        if w > 0 and w * n1 >= abs(kx):
            k = -np.sqrt(w * w * n1 * n1 - kx * kx)
            if abs(w - beta * k - Om) < 1e-9 * abs(Om):
                return w
    raise ValueError("no reflected wave")
