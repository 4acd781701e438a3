"""Seeded synthetic workloads shaped like the paper's examples (Figs. 5-8).

This module only draws geometry and parameters: grid sizes, velocities,
layer profiles, source and probe placement.  It holds none of the scheme's
arithmetic and is the one module that both the CUDA path (through the
binding) and the FP64 oracle (through the tests) consume.

Units: cells for lengths, c = 1, so a carrier of wavelength lam0 cells has
angular frequency 2 pi / lam0 and period lam0.  Sources are Gaussian-modulated
carriers with a full width at half maximum of `fwhm_periods` periods,
tau = FWHM / (2 sqrt(ln 2)) (Eq. spectrum_incident) and centre t0 = 4 tau.
Seeds: numpy default_rng(20230413 + config number).
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

PERTURBATION, MATTER = 0, 1
LAYERS, LINEAR = 0, 1
SEED0 = 20230413


@dataclass
class InstanceSpec:
    nz: int
    beta: float
    kind: int = PERTURBATION
    interp: int = LAYERS
    z: np.ndarray = field(default_factory=lambda: np.zeros(0))
    eps: np.ndarray = field(default_factory=lambda: np.ones(1))
    mu: np.ndarray = field(default_factory=lambda: np.ones(1))
    sources: List[Tuple[int, float, float, float, float]] = field(default_factory=list)
    probes: List[Tuple[int, np.ndarray]] = field(default_factory=list)


@dataclass
class Workload:
    name: str
    S: float
    n_steps: int
    instances: List[InstanceSpec]
    description: str = ""

    @property
    def cells(self):
        return int(sum(i.nz for i in self.instances))

    @property
    def cell_updates(self):
        return self.cells * self.n_steps


def gaussian_source(node, lam0, fwhm_periods=10.0, amp=1.0):
    w0 = 2 * np.pi / lam0
    tau = fwhm_periods * lam0 / (2 * np.sqrt(np.log(2)))
    return (int(node), w0, tau, 4 * tau, amp)


def random_fields(nz, rng, scale=1.0):
    """Random initial (B, D) for parity tests."""
    return rng.standard_normal(nz) * scale, rng.standard_normal(nz) * scale


# ------------------------------------------------------------------ configs

def config1(lam0=40.0, scale=1):
    """Moving interface, moving perturbation (Fig. 5 geometry, co-moving v = +0.3c).

    Nz = 4000, dz = lam0/40, S = 0.5, 8000 steps; eps = 1 ahead of the
    interface (xi < 2000), eps = 4 behind it; source 500 cells ahead of the
    interface; probes on both sides with 64 bins over [0, 4 w0).
    """
    s = int(scale)
    lam = lam0 * s
    w0 = 2 * np.pi / lam
    bins = np.arange(64) * (4 * w0 / 64)
    inst = InstanceSpec(nz=4000 * s, beta=0.3, z=np.array([2000.0 * s]), eps=np.array([1.0, 4.0]),
                        mu=np.ones(2), sources=[gaussian_source(1500 * s, lam, 10.0)],
                        probes=[(1900 * s, bins), (3300 * s, bins)])
    return Workload("interface", 0.5, 8000 * s, [inst],
                    "1D moving-perturbation interface, v=+0.3c, eps 1|4, Nz=4000, 8000 steps")


def config2(velocities=(-0.5, -0.2, 0.0, 0.2, 0.5), nz=1 << 16, n_steps=40000, slab=800, lam0=40.0,
            src_gap=1024):
    """Moving-matter slab (Fig. 6 geometry): rest eps' = 9, mu' = 1, one instance per velocity.

    Slab [32768, 32768 + 800) of the moving frame at t = 0 (scaled with nz);
    source src_gap cells before it; reflected / transmitted probes at 5/16 and
    11/16 of the grid; 256 bins over [0, 4 w0).
    """
    w0 = 2 * np.pi / lam0
    bins = np.arange(256) * (4 * w0 / 256)
    z0 = nz // 2
    out = []
    for v in velocities:
        out.append(InstanceSpec(nz=nz, beta=float(v), kind=MATTER, z=np.array([z0, z0 + slab], float),
                                eps=np.array([1.0, 9.0, 1.0]), mu=np.ones(3),
                                sources=[gaussian_source(z0 - src_gap, lam0, 10.0)],
                                probes=[(nz * 5 // 16, bins), (nz * 11 // 16, bins)]))
    return Workload("matter_slab", 0.5, n_steps, out,
                    "5 x 2^16 moving-matter slab, eps'=9, v in {-0.5,-0.2,0,0.2,0.5}c, 40000 steps")


def config3(n_inst=4096, nz_lo=1 << 12, nz_hi=1 << 18, periods=64, v_max=0.8, n_steps=20000,
            lam0=40.0, seed=SEED0 + 3, stable_only=False):
    """Batched moving bilayer crystal (Fig. 7 geometry, scaled up).

    Per instance: Nz log-uniform in [nz_lo, nz_hi]; velocity uniform in
    [-v_max, v_max] (|v| < 0.5 when stable_only: n|v| <= 1 in the eps = 4
    layers); `periods` periods of layers alternating eps = 1 and eps = 4 with
    lengths uniform in [20, 120] cells, starting at Nz/8 of the moving frame
    and truncated at 7 Nz / 8; a source at Nz/16 and a transmitted probe at
    15 Nz / 16 with 16 bins over [0.75, 1.25] w0.
    """
    rng = np.random.default_rng(seed)
    w0 = 2 * np.pi / lam0
    bins = np.linspace(0.75, 1.25, 16) * w0
    out = []
    for _ in range(n_inst):
        nz = int(np.exp(rng.uniform(np.log(nz_lo), np.log(nz_hi))))
        hi = 0.5 if stable_only else v_max
        v = float(rng.uniform(-hi, hi))
        if stable_only:
            v = float(np.clip(v, -0.499, 0.499))
        lengths = rng.integers(20, 121, size=2 * periods)
        z = nz / 8 + np.cumsum(lengths)
        z = z[z < 7 * nz / 8]
        bounds = np.concatenate(([nz / 8], z)).astype(float)
        eps = np.array([1.0] + [4.0 if i % 2 == 0 else 1.0 for i in range(len(bounds))])
        out.append(InstanceSpec(nz=nz, beta=v, z=bounds, eps=eps, mu=np.ones(len(eps)),
                                sources=[gaussian_source(nz // 16, lam0, 10.0)],
                                probes=[(nz * 15 // 16, bins)]))
    return Workload("crystal", 0.5, n_steps, out,
                    "%d moving bilayer crystals, Nz log-uniform in [%d, %d], v in [-%.2f, %.2f]c, "
                    "%d steps" % (n_inst, nz_lo, nz_hi, v_max, v_max, n_steps))


def config4(variant="as_written", nz=1 << 20, n_steps=200000, lam0=40.0):
    """Moving gradient (Fig. 8 geometry, scaled up): linear eps ramp over
    [nz/4, nz/2) of the moving frame, v = 0.7c (co-moving with the pulse).

    as_written: eps 1 -> 6 (n|v| exceeds 1 beyond eps = 2.04: unstable there);
    stable: eps 1 -> 2 (n|v| <= 0.99).  The source sits g = min(1024, nz/16)
    cells behind the ramp, so that the pulse, chasing the ramp at 0.3c,
    reaches it early in the run; the probe sits 2g behind it and records the
    source's backward pulse and what the ramp reflects.
    """
    e2 = 6.0 if variant == "as_written" else 2.0
    w0 = 2 * np.pi / lam0
    bins = np.linspace(0.5, 1.5, 16) * w0
    g = min(1024, nz // 16)
    inst = InstanceSpec(nz=nz, beta=0.7, interp=LINEAR, z=np.array([nz / 4, nz / 2], float),
                        eps=np.array([1.0, e2]), mu=np.ones(2),
                        sources=[gaussian_source(nz // 4 - g, lam0, 10.0)],
                        probes=[(nz // 4 - 2 * g, bins)])
    return Workload("gradient_" + variant, 0.5, n_steps, [inst],
                    "Nz=2^20 linear ramp eps 1->%g over 2^18 cells, v=0.7c, %d steps" % (e2, n_steps))


def config5(n_inst=256, nz=1 << 14, n_steps=16000, n_ctrl=512, lam0=40.0, seed=SEED0 + 5):
    """Adjoint workload: piecewise-linear eps over a 1024-cell moving region, v = 0.4c.

    Knots: 2046 (eps 1), 2048 + 2j for j < n_ctrl (eps uniform in [1, 4]),
    2048 + 2 n_ctrl (eps 1); source at 1024, transmitted probe at 6656 with
    16 bins of spacing w0/64 centred on the transmitted carrier.
    """
    rng = np.random.default_rng(seed)
    w0 = 2 * np.pi / lam0
    out = []
    z = np.concatenate(([2046.0], 2048.0 + 2.0 * np.arange(n_ctrl), [2048.0 + 2.0 * n_ctrl]))
    for _ in range(n_inst):
        ctrl = rng.uniform(1.0, 4.0, size=n_ctrl)
        eps = np.concatenate(([1.0], ctrl, [1.0]))
        bins = w0 + (np.arange(16) - 7.5) * (w0 / 64)
        out.append(InstanceSpec(nz=nz, beta=0.4, interp=LINEAR, z=z.copy(), eps=eps,
                                mu=np.ones(len(eps)), sources=[gaussian_source(1024, lam0, 10.0)],
                                probes=[(6656, bins)]))
    return Workload("adjoint", 0.5, n_steps, out,
                    "%d x 2^14 PWL eps profiles (%d control points), v=0.4c, %d steps"
                    % (n_inst, n_ctrl, n_steps))
