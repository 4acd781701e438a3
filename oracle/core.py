"""ctypes wrapper around the FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It drives ``gfdtd_oracle.c``, which follows Sec. 4 of the paper
(Eqs. Farad_discr, Ampere_discr, Dconst_discr, Bconst_discr and Table 1) and,
for moving matter, the star-form constitutive relations obtained from
Eq. const_3d with the footnote tensors.  See the C file's header for the exact
statement of every update.
"""
import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("interp", C.c_int32), ("n", C.c_int32),
                ("reserved", C.c_int32), ("z", _dp), ("eps", _dp), ("mu", _dp),
                ("beta", C.c_double), ("S", C.c_double), ("nz", C.c_int64),
                ("absorb_width", C.c_int64), ("absorb_sigma", C.c_double)]


class _Source(C.Structure):
    _fields_ = [("node", C.c_int64), ("omega0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("amp", C.c_double)]


class _Probe(C.Structure):
    _fields_ = [("node", C.c_int64), ("n_bins", C.c_int32), ("reserved", C.c_int32),
                ("omega", _dp), ("re", _dp), ("im", _dp), ("series", _dp)]


class _Problem2(C.Structure):
    _fields_ = [("nx", C.c_int64), ("nz", C.c_int64), ("dx", C.c_double), ("S", C.c_double),
                ("beta", C.c_double), ("slope", C.c_double), ("n", C.c_int32), ("reserved", C.c_int32),
                ("z", _dp), ("eps", _dp), ("mu", _dp)]


class _Source2(C.Structure):
    _fields_ = [("k", C.c_int64), ("kx", C.c_double), ("omega0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("amp", C.c_double)]


class _Probe2(C.Structure):
    _fields_ = [("i", C.c_int64), ("k", C.c_int64), ("n_bins", C.c_int32), ("reserved", C.c_int32),
                ("omega", _dp), ("re", _dp), ("im", _dp)]


class _Tfsf(C.Structure):
    _fields_ = [("node", C.c_int64), ("omega0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("amp", C.c_double), ("aux_B", _dp), ("aux_D", _dp)]


AUX_N = 1064   # cells of a one-way source's auxiliary grid (see the C header)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_run.restype = C.c_int
        L.orc_run.argtypes = [C.POINTER(_Problem), C.c_int, C.POINTER(_Source), C.c_int,
                              C.POINTER(_Probe), C.c_int64, C.c_int64, _dp, _dp]
        L.orc_run_tfsf.restype = C.c_int
        L.orc_run_tfsf.argtypes = [C.POINTER(_Problem), C.c_int, C.POINTER(_Source), C.c_int,
                                   C.POINTER(_Probe), C.c_int, C.POINTER(_Tfsf), C.c_int64, C.c_int64,
                                   _dp, _dp]
        L.orc_sample_material.restype = C.c_int
        L.orc_sample_material.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_int64, _dp]
        L.orc_step_transpose.restype = C.c_int
        L.orc_step_transpose.argtypes = [C.POINTER(_Problem), C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc2_run.restype = C.c_int
        L.orc2_run.argtypes = [C.POINTER(_Problem2), C.c_int, C.POINTER(_Source2), C.c_int,
                               C.POINTER(_Probe2), C.c_int64, C.c_int64, _dp, _dp, _dp]
        L.orc_adjoint.restype = C.c_int
        L.orc_adjoint.argtypes = [C.POINTER(_Problem), C.c_int, C.POINTER(_Source), C.POINTER(_Probe),
                                  C.c_int64, C.c_int64, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Instance:
    """One 1D problem: grid, moving medium, sources and DFT probes, with FP64 state.

    ``kind`` 0 = moving perturbation, 1 = moving matter; ``interp`` 0 = layers
    (``z`` holds n-1 boundaries for n values), 1 = piecewise linear (``z`` holds
    n knots).  Positions are in cells of the moving frame at t = 0.
    """

    def __init__(self, nz, S, beta, kind=0, interp=0, z=(), eps=(1.0,), mu=None):
        self.nz = int(nz)
        self.S = float(S)
        self.beta = float(beta)
        self.kind = int(kind)
        self.interp = int(interp)
        self.eps = _f64(eps)
        self.mu = _f64(np.ones_like(self.eps) if mu is None else mu)
        self.z = _f64(z) if len(z) else np.zeros(1)
        n = len(self.eps)
        assert len(self.mu) == n
        assert len(z) == (n - 1 if interp == 0 else n)
        self.B = np.zeros(self.nz)
        self.D = np.zeros(self.nz)
        self.n_done = 0
        self.sources = []
        self.probes = []
        self.absorb_width, self.absorb_sigma = 0, 0.0
        self.tfsf = []

    def set_absorber(self, width, sigma):
        """Graded absorbing layers of `width` cells at both ends (0: none); see the C header."""
        self.absorb_width, self.absorb_sigma = int(width), float(sigma)
        return self

    def add_source(self, node, omega0, tau, t0, amp=1.0):
        self.sources.append((int(node), float(omega0), float(tau), float(t0), float(amp)))

    def add_tfsf(self, node, omega0, tau, t0, amp=1.0):
        """One-way source: total field at nodes >= node, the incident wave being the
        right-going wave of a soft source with this waveform (see the C header)."""
        self.tfsf.append({"args": (int(node), float(omega0), float(tau), float(t0), float(amp)),
                          "B": np.zeros(AUX_N), "D": np.zeros(AUX_N)})

    def add_probe(self, node, omega):
        omega = _f64(omega)
        self.probes.append({"node": int(node), "omega": omega,
                            "re": np.zeros(len(omega)), "im": np.zeros(len(omega)),
                            "series": []})
        return len(self.probes) - 1

    def _problem(self):
        return _Problem(self.kind, self.interp, len(self.eps), 0, _ptr(self.z), _ptr(self.eps),
                        _ptr(self.mu), self.beta, self.S, self.nz, self.absorb_width, self.absorb_sigma)

    def run(self, n_steps, record=False):
        """Advance ``n_steps`` leapfrog steps in FP64."""
        n_steps = int(n_steps)
        prob = self._problem()
        srcs = (_Source * max(1, len(self.sources)))(*[_Source(*s) for s in self.sources])
        series = [np.zeros(n_steps) if record else None for _ in self.probes]
        prbs = (_Probe * max(1, len(self.probes)))(*[
            _Probe(p["node"], len(p["omega"]), 0, _ptr(p["omega"]), _ptr(p["re"]),
                   _ptr(p["im"]), _ptr(series[i]))
            for i, p in enumerate(self.probes)])
        tfs = (_Tfsf * max(1, len(self.tfsf)))(*[
            _Tfsf(*t["args"], _ptr(t["B"]), _ptr(t["D"])) for t in self.tfsf])
        rc = lib().orc_run_tfsf(C.byref(prob), len(self.sources), srcs, len(self.probes), prbs,
                                len(self.tfsf), tfs, self.n_done, n_steps, _ptr(self.B), _ptr(self.D))
        if rc != 0:
            raise ValueError("oracle rejected the problem")
        self.n_done += n_steps
        if record:
            for i, p in enumerate(self.probes):
                p["series"].append(series[i])
        return self

    def spectrum(self, probe_id):
        p = self.probes[probe_id]
        return p["re"] + 1j * p["im"]

    def series(self, probe_id):
        s = self.probes[probe_id]["series"]
        return np.concatenate(s) if s else np.zeros(0)

    def step_transpose(self, n, aBn, aDn, D_old):
        """Transpose of step n (the linear map (B^{n-1}, D^{n-1/2}) -> (B^n, D^{n+1/2})).

        Returns (aB, aD, geps) with geps[k] = dL/deps_k at level n-1/2.
        """
        aB, aD, g = np.zeros(self.nz), np.zeros(self.nz), np.zeros(self.nz)
        rc = lib().orc_step_transpose(C.byref(self._problem()), int(n), _ptr(_f64(aBn)), _ptr(_f64(aDn)),
                                      _ptr(_f64(D_old)), _ptr(aB), _ptr(aD), _ptr(g))
        if rc != 0:
            raise ValueError("transpose needs a moving-perturbation problem")
        return aB, aD, g

    def adjoint(self, probe_id, bins, n_steps):
        """L = sum over `bins` of |X_f|^2 of probe `probe_id`, accumulated over the next
        n_steps from the current state, and dL/d(eps value) of every profile value.
        The instance's state is left unchanged."""
        if self.tfsf:
            raise ValueError("the adjoint covers soft sources only")
        p = self.probes[probe_id]
        om = _f64(np.asarray(p["omega"])[list(bins)])
        scratch = np.zeros(len(om))
        prb = _Probe(p["node"], len(om), 0, _ptr(om), _ptr(scratch), _ptr(scratch), None)
        srcs = (_Source * max(1, len(self.sources)))(*[_Source(*s) for s in self.sources])
        loss = C.c_double()
        grad = np.zeros(len(self.eps))
        rc = lib().orc_adjoint(C.byref(self._problem()), len(self.sources), srcs, C.byref(prb),
                               self.n_done, int(n_steps), _ptr(self.B), _ptr(self.D),
                               C.byref(loss), _ptr(grad))
        if rc != 0:
            raise ValueError("adjoint needs a moving-perturbation problem and n_steps >= 1")
        return loss.value, grad

    def material(self, which="eps", half_node=False, h=0):
        """eps (or mu) at every node at half level ``h`` (time h*S/2)."""
        out = np.zeros(self.nz)
        prob = self._problem()
        lib().orc_sample_material(C.byref(prob), 0 if which == "eps" else 1, int(half_node),
                                  int(h), _ptr(out))
        return out


def run_many(instances, n_steps, threads=None, record=False):
    """Run independent instances concurrently on host threads (ctypes drops the GIL)."""
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda inst: inst.run(n_steps, record=record), instances))
    return instances


class Instance2D:
    """The 2D TE generalized scheme (see the C file): nx columns (periodic in x,
    width dx each), nz cells along the motion (zero fields beyond the ends),
    moving-perturbation layers whose boundaries are the lines
    z - beta t - slope x = z_b.  State: Bx, Bz, D as [nx, nz] FP64 arrays
    (D at (i, k), Bx at (i, k + 1/2), Bz at (i + 1/2, k))."""

    def __init__(self, nx, nz, S, beta, dx=1.0, z=(), eps=(1.0,), mu=None, slope=0.0):
        self.nx, self.nz, self.S, self.beta, self.dx, self.slope = int(nx), int(nz), float(S), float(beta), \
            float(dx), float(slope)
        self.eps = _f64(eps)
        self.mu = _f64(np.ones_like(self.eps) if mu is None else mu)
        assert len(z) == len(self.eps) - 1
        self.z = _f64(z) if len(z) else np.zeros(1)
        self.Bx = np.zeros((self.nx, self.nz))
        self.Bz = np.zeros((self.nx, self.nz))
        self.D = np.zeros((self.nx, self.nz))
        self.n_done = 0
        self.sources = []
        self.probes = []

    def add_source(self, k, kx, omega0, tau, t0, amp=1.0):
        self.sources.append((int(k), float(kx), float(omega0), float(tau), float(t0), float(amp)))

    def add_probe(self, i, k, omega):
        omega = _f64(omega)
        self.probes.append({"i": int(i), "k": int(k), "omega": omega,
                            "re": np.zeros(len(omega)), "im": np.zeros(len(omega))})
        return len(self.probes) - 1

    def run(self, n_steps):
        prob = _Problem2(self.nx, self.nz, self.dx, self.S, self.beta, self.slope, len(self.eps), 0,
                         _ptr(self.z), _ptr(self.eps), _ptr(self.mu))
        srcs = (_Source2 * max(1, len(self.sources)))(*[_Source2(*s) for s in self.sources])
        prbs = (_Probe2 * max(1, len(self.probes)))(*[
            _Probe2(p["i"], p["k"], len(p["omega"]), 0, _ptr(p["omega"]), _ptr(p["re"]), _ptr(p["im"]))
            for p in self.probes])
        for a in (self.Bx, self.Bz, self.D):
            assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
        rc = lib().orc2_run(C.byref(prob), len(self.sources), srcs, len(self.probes), prbs, self.n_done,
                            int(n_steps), _ptr(self.Bx), _ptr(self.Bz), _ptr(self.D))
        if rc != 0:
            raise ValueError("oracle rejected the 2D problem")
        self.n_done += int(n_steps)
        return self

    def spectrum(self, probe_id):
        p = self.probes[probe_id]
        return p["re"] + 1j * p["im"]
