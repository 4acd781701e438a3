"""GPU parameter sweeps against the FP64 oracle: the von Neumann stability map
(Sec. 5, App. A) and the star transfer-matrix scattering of moving stacks
(App. B.3).  Both sides are FP64; the bar is 1e-12 relative (1e-11 for the
transfer matrices, whose propagation phases reach ~1e3 rad)."""
import numpy as np
import pytest

from paper_2304_06586_gb300 import binding as gb

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def _points(rng, n):
    S = rng.uniform(0.1, 1.0, n)
    beta = rng.uniform(-0.9, 0.9, n)
    eps = rng.uniform(1.0, 9.0, n)
    mu = np.where(rng.uniform(size=n) < 0.5, 1.0, rng.uniform(1.0, 2.0, n))
    kind = rng.integers(0, 2, n)
    # moving matter needs eps mu > beta^2 (true here) and |beta| S < 1
    return S, beta, eps, mu, kind


def test_stability_map_matches_oracle():
    from oracle import vonneumann as vn
    rng = np.random.default_rng(3)
    S, beta, eps, mu, kind = _points(rng, 48)
    n_theta = 384
    got = gb.stability_map(S, beta, eps, mu, kind, n_theta=n_theta).cpu().numpy()
    for i in range(len(S)):
        ref = vn.max_growth(S[i], beta[i], eps[i], mu[i], kind=int(kind[i]), n_theta=n_theta)
        assert abs(got[i] - ref) <= TOL * max(1.0, ref), (i, got[i], ref)


def test_stability_map_threshold_and_edges():
    """Either side of n |beta| = 1 for a moving perturbation (the scheme's
    stability limit), v = 0, the S = 1 magic step, and an empty call."""
    from oracle import vonneumann as vn
    eps = 4.0
    b = np.array([0.45, 0.49, 0.51, 0.55, -0.45, -0.55, 0.0, 0.0])
    S = np.array([0.5] * 6 + [0.5, 1.0])
    got = gb.stability_map(S, b, eps, 1.0, gb.PERTURBATION, n_theta=1024).cpu().numpy()
    for i in range(len(b)):
        ref = vn.max_growth(S[i], b[i], eps, 1.0, n_theta=1024)
        assert abs(got[i] - ref) <= TOL * max(1.0, ref)
    assert np.all(got[[0, 1, 4]] <= 1.0 + 1e-12) and np.all(got[[2, 3, 5]] > 1.0 + 1e-7)
    assert gb.stability_map(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0)).numel() == 0


def test_stability_map_large_sampled():
    """A 2^18-point sweep checked on sampled points."""
    from oracle import vonneumann as vn
    rng = np.random.default_rng(4)
    S, beta, eps, mu, kind = _points(rng, 1 << 18)
    got = gb.stability_map(S, beta, eps, mu, kind, n_theta=256).cpu().numpy()
    for i in rng.choice(len(S), size=12, replace=False):
        ref = vn.max_growth(S[i], beta[i], eps[i], mu[i], kind=int(kind[i]), n_theta=256)
        assert abs(got[i] - ref) <= TOL * max(1.0, ref)


def _stacks(rng, n):
    out = []
    for _ in range(n):
        nl = int(rng.integers(2, 13))
        eps = rng.uniform(1.0, 6.0, nl)
        mu = np.where(rng.uniform(size=nl) < 0.7, 1.0, rng.uniform(1.0, 1.5, nl))
        thick = rng.uniform(5.0, 80.0, nl)
        out.append((eps, mu, thick))
    return out


def test_star_tmm_matches_oracle():
    from oracle import exact
    rng = np.random.default_rng(6)
    stacks = _stacks(rng, 40)
    beta = rng.uniform(-0.3, 0.3, len(stacks))      # n |beta| <= 0.9 in every layer
    omega = np.linspace(0.05, 0.6, 9)
    T, G = gb.star_tmm(stacks, beta, omega)
    T, G = T.cpu().numpy(), G.cpu().numpy()
    for s, (eps, mu, thick) in enumerate(stacks):
        for f, w in enumerate(omega):
            t, g = exact.star_tmm(eps, mu, thick[1:-1], beta[s], w)
            # phases reach ~1e3 rad, so argument rounding costs ~1 digit of the 1e-12 bar
            assert abs(T[s, f] - t) <= 10 * TOL * max(1.0, abs(t)), (s, f, T[s, f], t)
            assert abs(G[s, f] - g) <= 10 * TOL * max(1.0, abs(g)), (s, f, G[s, f], g)


def test_star_tmm_single_interface_and_degenerate_stack():
    """Two layers reduce to Eq. coef_interface; a one-layer stack gives NaN."""
    from oracle import exact
    stacks = [(np.array([1.0, 4.0]), np.ones(2), np.zeros(2)), (np.array([2.0]), np.ones(1), np.zeros(1))]
    T, G = gb.star_tmm(stacks, [0.2, 0.2], [0.3])
    ref = exact.interface(1.0, 4.0, 0.2)
    assert abs(T[0, 0].item() - ref["T"]) <= 1e-13 and abs(G[0, 0].item() - ref["Gamma"]) <= 1e-13
    assert np.isnan(T[1, 0].real.item()) and np.isnan(G[1, 0].real.item())
