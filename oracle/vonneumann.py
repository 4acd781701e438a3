"""Von Neumann amplification of the generalized FDTD scheme (test infrastructure only).

Sec. 5 and Appendix A of the paper insert the plane-wave test field
Psi_k^n = Psi_0 xi^k zeta^n, xi = exp(i kz dz) (Eq. PW_test_field) into the
update equations and look for the zeta that the homogeneous system admits.
The closed forms the paper prints for zeta (Eqs. zeta_stability and
zeta_polynom) are garbled in the available text, so this module assembles the
one-step amplification matrix G(kz dz) directly from the discrete updates of
Sec. 4 and Table 1 and takes its eigenvalues; the two eigenvalues of the
moving-perturbation matrix are the paper's zeta_+ and zeta_-.  The worked
example of Sec. 5 (S = 0.5, beta = 0.3, eps = 4, mu = 1, kz dz = 2 pi / 5 gives
zeta_+ = 0.925 - 0.33i and zeta_- = 0.917 + 0.23i) pins this construction.

State vectors are the complex amplitudes of one Fourier mode: B (at half
nodes k+1/2) and D (at nodes k), for moving perturbation and moving matter
alike.  theta = kz dz.
"""
import numpy as np


def _shifts(beta, theta):
    """Fourier symbols of the Table 1 stencils for the column selected by sign(beta).

    Returns (bsum, adv): bsum multiplies B-hat in the Ba/Bb average seen from an
    integer node (without the factor 1/2); adv multiplies a field in the upwind
    difference dBa/dBb (identically dDa/dDb).
    """
    if beta >= 0:   # Ba: B_{k-1/2} + B_{k-3/2};  dBa: B_{k+1/2} - B_{k-1/2}
        bsum = np.exp(-0.5j * theta) + np.exp(-1.5j * theta)
        adv = 1.0 - np.exp(-1j * theta)
    else:           # Bb: B_{k+3/2} + B_{k+1/2};  dBb: B_{k+3/2} - B_{k+1/2}
        bsum = np.exp(1.5j * theta) + np.exp(0.5j * theta)
        adv = np.exp(1j * theta) - 1.0
    return bsum, adv


def amplification_perturbation(S, beta, eps, mu, theta):
    """2x2 matrix mapping (B^{n-1}, D^{n-1/2}) to (B^n, D^{n+1/2}) for one mode."""
    bsum, adv = _shifts(beta, theta)
    curl = 2j * np.sin(theta / 2)          # symbol of f_{+1/2} - f_{-1/2}
    avg = np.cos(theta / 2)                # symbol of (f_{-1/2} + f_{+1/2}) / 2
    # E* = D/eps - beta * bsum/2 * B            (columns: B, D)
    Es = np.array([-beta * 0.5 * bsum, 1.0 / eps])
    # B' = B - S curl E* - beta S adv B
    Bn = np.array([1.0 - beta * S * adv, 0.0]) - S * curl * Es
    # H* = B'/mu - beta * avg * D
    Hs = Bn / mu - beta * avg * np.array([0.0, 1.0])
    # D' = D - S curl H* - beta S adv D
    Dn = np.array([0.0, 1.0 - beta * S * adv]) - S * curl * Hs
    return np.array([Bn, Dn])


def matter_coefficients(beta, eps_r, mu_r):
    """(1/eps_m, 1/mu_m, beta_c) of the solved moving-matter star relations.

    Eq. const_3d with the footnote tensors gives, in 1D,
    eps' E* = (1 - beta^2) D - beta H* and mu' H* = (1 - beta^2) B - beta E*;
    solving the pair: E* = D/eps_m - beta_c B, H* = B/mu_m - beta_c D.
    """
    den = eps_r * mu_r - beta * beta
    g = 1.0 - beta * beta
    return g * mu_r / den, g * eps_r / den, beta * g / den


def amplification_matter(S, beta, eps_r, mu_r, theta):
    """2x2 matrix for moving matter (rest eps_r, mu_r): Table 1 with beta_c in the averages."""
    ie, im, bc = matter_coefficients(beta, eps_r, mu_r)
    bsum, adv = _shifts(beta, theta)
    curl = 2j * np.sin(theta / 2)
    avg = np.cos(theta / 2)
    Es = np.array([-bc * 0.5 * bsum, ie])
    Bn = np.array([1.0 - beta * S * adv, 0.0]) - S * curl * Es
    Hs = im * Bn - bc * avg * np.array([0.0, 1.0])
    Dn = np.array([0.0, 1.0 - beta * S * adv]) - S * curl * Hs
    return np.array([Bn, Dn])


def zetas(S, beta, eps, mu, theta, kind=0):
    """Eigenvalues of the amplification matrix (sorted by decreasing modulus)."""
    G = (amplification_perturbation if kind == 0 else amplification_matter)(S, beta, eps, mu, theta)
    z = np.linalg.eigvals(G)
    return z[np.argsort(-np.abs(z))]


def zeta_pm(S, beta, eps, mu, theta):
    """(zeta_+, zeta_-) of Eq. PW_anal: zeta_+ is the mode travelling towards +z.

    With xi = exp(i theta) and zeta = exp(-alpha dt), a +z travelling wave has
    a negative temporal phase, so zeta_+ is the eigenvalue with arg < 0.
    """
    z = np.linalg.eigvals(amplification_perturbation(S, beta, eps, mu, theta))
    zp = z[np.argmin(np.angle(z))]
    zm = z[np.argmax(np.angle(z))]
    return zp, zm


def max_growth(S, beta, eps, mu, kind=0, n_theta=2048):
    """max over kz dz in (0, pi] of |zeta| (the von Neumann stability measure)."""
    thetas = np.linspace(np.pi / n_theta, np.pi, n_theta)
    return max(np.abs(zetas(S, beta, eps, mu, t, kind)).max() for t in thetas)


def eigenmode(S, beta, eps, mu, theta, which="+"):
    """(zeta, B-hat, D-hat) of the +z (which='+') or -z travelling eigenmode."""
    G = amplification_perturbation(S, beta, eps, mu, theta)
    z, V = np.linalg.eig(G)
    i = np.argmin(np.angle(z)) if which == "+" else np.argmax(np.angle(z))
    return z[i], V[0, i], V[1, i]


def mode_for_frequency(S, beta, eps, mu, omega, direction=+1):
    """Real wavenumber theta = kz dz of the discrete mode with lab frequency omega.

    direction +1 selects the +z travelling branch, -1 the -z branch.  Returns
    (theta, zeta, group_velocity) where the group velocity is in cells per
    unit time.
    """
    def branch(theta):
        z = zetas(S, beta, eps, mu, direction * theta)
        # a wave travelling along sign(theta) has zeta = exp(-i omega S), omega > 0
        w = -np.angle(z) / S
        i = np.argmax(w)
        return w[i], z[i]
    lo, hi = 1e-6, np.pi * 0.9
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if branch(mid)[0] < omega:
            lo = mid
        else:
            hi = mid
    theta = 0.5 * (lo + hi)
    w, z = branch(theta)
    dth = 1e-6
    vg = (branch(theta + dth)[0] - branch(theta - dth)[0]) / (2 * dth)
    return theta, z, vg


def propagation_loss(S, beta, eps, mu, omega, distance, direction=+1):
    """Amplitude factor the discrete scheme applies to a wave of frequency omega
    over ``distance`` cells in a uniform moving-perturbation medium."""
    theta, z, vg = mode_for_frequency(S, beta, eps, mu, omega, direction)
    steps = abs(distance) / (abs(vg) * S)
    return abs(z) ** steps


def doppler_factor(S, beta, eps_in, eps_out, omega, direction_out=+1, mu_in=1.0, mu_out=1.0):
    """Lab frequency ratio omega_out / omega of the wave that leaves a moving
    interface (velocity beta) when a +z wave of lab frequency omega arrives in
    medium `in`: the interface moves rigidly, so the frequency seen in its frame,
    Omega = omega - beta k, is the same on both sides (the invariant behind
    Eq. comp_exp), here with k taken from the scheme's own dispersion relation
    (mode_for_frequency) in each uniform medium.  direction_out = +1: the
    transmitted wave in medium `out`; -1: the reflected wave (medium `out` =
    medium `in`).  As omega -> 0 it tends to Eq. comp_exp's a_t and a_r."""
    th_in, _, _ = mode_for_frequency(S, beta, eps_in, mu_in, omega, +1)
    Om = omega - beta * th_in
    lo, hi = 0.05 * omega, 20.0 * omega
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        th, _, _ = mode_for_frequency(S, beta, eps_out, mu_out, mid, direction_out)
        if mid - beta * direction_out * th < Om:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi) / omega
