"""Scattering coefficients of a moving interface measured from DFT probes
(test helper, shared by the oracle and GPU tests).

Geometry: the moving-interface workload (v = +0.3c, eps 1 | 4, S = 0.5,
interface at 2000, soft source 500 cells ahead of it, probes at 1900 and
3300, 8000 steps, carrier of 40 cells), every length and the step count
multiplied by `scale` (scale 1 is the workload as stated).  Three instances:

* A: the interface, zero fields beyond both ends;
* B: the same without the interface (uniform eps 1): the reflected spectrum is
  A - B at the probe before the interface (both share the source's backward
  pulse and its echo off z = 0, which cancel);
* C: B with absorbing layers at both ends: the incident spectrum at that
  probe, free of the echo.

Coefficients (Eqs. coef_interface and comp_exp, App. B; reading of
Eq. spectrum_scat_interface: a scattered spectrum is the coefficient times the
incident spectrum compressed by the Doppler factor a): |Gamma| =
a_r |X_r(a_r w)| / |X_i(w)|, |T| = a_t |X_t(a_t w)| / |X_i(w)|, with two
properties of the scheme itself removed: its propagation loss over the paths
between the probes and the point where the pulse meets the interface (von
Neumann amplification factor, Sec. 5), and its own Doppler factors -- the
interface conserves w - v k with the scheme's wavenumbers k (oracle
vonneumann.doppler_factor), which differ from Eq. comp_exp's by a second-order
term (-2.6 % for the transmitted wave of the stated workload, 11.4 cells per
transmitted wavelength).  The spectral peaks are compared with both factors.
"""
import numpy as np

from paper_2304_06586_gb300 import workloads as w

FREQS = (0.95, 1.0, 1.05)        # multiples of the carrier frequency
FINE = np.linspace(0.8, 1.2, 81)  # grid for the spectral peaks


class Interface:
    def __init__(self, scale=1.0, beta=0.3, e1=1.0, e2=4.0, S=0.5):
        from oracle import exact
        from oracle import vonneumann as vn
        s = float(scale)
        self.beta, self.e1, self.e2, self.S = beta, e1, e2, S
        self.lam0 = 40.0 * s
        self.nz, self.zI, self.src = int(4000 * s), 2000.0 * s, int(1500 * s)
        self.zr, self.zt, self.steps = int(1900 * s), int(3300 * s), int(8000 * s)
        self.absorber = (int(64 * s), 0.2)
        self.source = w.gaussian_source(self.src, self.lam0, 10.0)
        _, self.w0, tau, t0, _ = self.source
        self.ex = exact.interface(e1, e2, beta)
        n1 = np.sqrt(e1)
        tm = (self.zI - self.src + t0 / n1) / (1 / n1 - beta)   # pulse centre meets the interface
        self.zm = self.zI + beta * tm
        om = np.array(FREQS) * self.w0
        self.ar = np.array([vn.doppler_factor(S, beta, e1, e1, x, -1) for x in om])
        self.at = np.array([vn.doppler_factor(S, beta, e1, e2, x, +1) for x in om])
        self.li = np.array([vn.propagation_loss(S, beta, e1, 1.0, x, self.zm - self.zr, +1) for x in om])
        self.lr = np.array([vn.propagation_loss(S, beta, e1, 1.0, a * x, self.zm - self.zr, -1)
                            for a, x in zip(self.ar, om)])
        self.lt = np.array([vn.propagation_loss(S, beta, e2, 1.0, a * x, self.zt - self.zm, +1)
                            for a, x in zip(self.at, om)])
        g = FINE * self.w0
        self.bins_i = np.concatenate((om, g))
        self.bins_r = np.concatenate((self.ar * om, self.ex["a_r"] * g))
        self.bins_t = np.concatenate((self.at * om, self.ex["a_t"] * g))
        self.specs = [
            w.InstanceSpec(nz=self.nz, beta=beta, z=np.array([self.zI]), eps=np.array([e1, e2]), mu=np.ones(2),
                           sources=[self.source], probes=[(self.zr, self.bins_r), (self.zt, self.bins_t)]),
            w.InstanceSpec(nz=self.nz, beta=beta, eps=np.array([e1]), mu=np.ones(1),
                           sources=[self.source], probes=[(self.zr, self.bins_r)]),
            w.InstanceSpec(nz=self.nz, beta=beta, eps=np.array([e1]), mu=np.ones(1),
                           sources=[self.source], probes=[(self.zr, self.bins_i)]),
        ]

    def workload(self):
        return w.Workload("interface x%g" % (self.lam0 / 40.0), self.S, self.steps, self.specs)

    def coefficients(self, XA_r, XB_r, XA_t, XC_i):
        """Relative errors of |Gamma| and |T| against Eq. coef_interface at each
        frequency of FREQS, and the measured Doppler factors from the peaks."""
        n = len(FREQS)
        Xr, Xt, Xi = XA_r - XB_r, XA_t, XC_i
        G = self.ar * np.abs(Xr[:n]) / np.abs(Xi[:n]) / (self.li * self.lr)
        T = self.at * np.abs(Xt[:n]) / np.abs(Xi[:n]) / (self.li * self.lt)

        def peak(X):
            a = np.abs(X[n:])
            k = int(np.clip(np.argmax(a), 1, len(a) - 2))
            d = 0.5 * (a[k - 1] - a[k + 1]) / (a[k - 1] - 2 * a[k] + a[k + 1])
            return np.interp(k + d, np.arange(len(FINE)), FINE)

        pi, pr, pt = peak(Xi), peak(Xr), peak(Xt)
        return {"Gamma": G / abs(self.ex["Gamma"]) - 1, "T": T / abs(self.ex["T"]) - 1,
                "a_r": self.ex["a_r"] * pr / pi, "a_t": self.ex["a_t"] * pt / pi,
                "a_r_scheme": self.ar[1], "a_t_scheme": self.at[1],
                "cells_per_transmitted_wavelength": self.lam0 / (np.sqrt(self.e2) * self.ex["a_t"])}

    def run_oracle(self):
        import oracle
        from helpers import make_oracle
        A, B, C = make_oracle(self.workload())
        C.set_absorber(*self.absorber)
        oracle.run_many([A, B, C], self.steps)
        return self.coefficients(A.spectrum(0), B.spectrum(0), A.spectrum(1), C.spectrum(0))

    def run_gpu(self, prec):
        from helpers import make_sim
        sim = make_sim(self.workload(), prec=prec, allow_unstable=False)
        sim.set_absorber(2, *self.absorber)
        sim.step(self.steps)
        nr, nt, ni = len(self.bins_r), len(self.bins_t), len(self.bins_i)
        res = self.coefficients(sim.read_spectrum(0, 0, nr), sim.read_spectrum(1, 0, nr),
                                sim.read_spectrum(0, 1, nt), sim.read_spectrum(2, 0, ni))
        sim.close()
        return res
