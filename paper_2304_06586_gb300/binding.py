"""Thin ctypes binding of the C ABI in include/gfdtd.h.

Only argument marshalling lives here; every step of the method runs in the
CUDA library.  There is no fallback: if ``libgfdtd.so`` cannot be loaded, or
no GPU is present when a context is created, the call raises.

PyTorch supplies the CUDA stream (the current stream at creation) and, through
``use_torch_allocator()``, the device memory of the contexts.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))

OK, E_ARG, E_OOM, E_CUDA, E_UNSTABLE, E_TIMEOUT, E_STATE, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
PERTURBATION, MATTER = 0, 1
F32, F32_KAHAN, BF16, F16, F64 = 0, 1, 2, 3, 4
LAYERS, LINEAR = 0, 1
FIELD_D, FIELD_B, FIELD_E, FIELD_H, FIELD_ESTAR = 0, 1, 2, 3, 4

_STATUS = {E_ARG: "E_ARG", E_OOM: "E_OOM", E_CUDA: "E_CUDA", E_UNSTABLE: "E_UNSTABLE",
           E_TIMEOUT: "E_TIMEOUT", E_STATE: "E_STATE", E_UNSUPPORTED: "E_UNSUPPORTED"}

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Stats(C.Structure):
    _fields_ = [("cells_per_lane", C.c_int), ("time_block", C.c_int), ("blocks_per_sm", C.c_int),
                ("n_tiles", C.c_int64),
                ("kernel_launches", C.c_int64), ("cells", C.c_int64), ("uniform_split", C.c_int)]


class KernelTimes(C.Structure):
    _fields_ = [("launches", C.c_int64 * 3), ("ms", C.c_double * 3), ("cell_updates", C.c_int64 * 3)]


KERNEL_VARIANTS = ("general_perturbation", "general_matter", "fast")


# every symbol of include/gfdtd.h with its (restype, argtypes)
SIGNATURES = {
    "gfdtd_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "gfdtd_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _i64p, C.c_double, C.c_int, C.c_void_p]),
    "gfdtd_set_medium": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, _dp, _dp,
                                   _dp, C.c_int]),
    "gfdtd_add_source": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_double, C.c_double,
                                   C.c_double]),
    "gfdtd_add_tfsf": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_double, C.c_double,
                                   C.c_double]),
    "gfdtd_add_probe": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, _dp, C.POINTER(C.c_int)]),
    "gfdtd_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "gfdtd_step_plain": (C.c_int, [C.c_void_p, C.c_int64]),
    "gfdtd_plain_floor": (C.c_int, [C.c_void_p, C.c_int64]),
    "gfdtd_read_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, C.c_int64]),
    "gfdtd_write_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, C.c_int64]),
    "gfdtd_read_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "gfdtd_write_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "gfdtd_state_layout": (C.c_int, [C.c_void_p, _i64p, C.POINTER(C.c_int), _i64p]),
    "gfdtd_read_spectrum": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, _dp]),
    "gfdtd_steps_done": (C.c_int, [C.c_void_p, _i64p]),
    "gfdtd_stability": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _dp]),
    "gfdtd_stability_map": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int, C.c_void_p, C.c_void_p]),
    "gfdtd_star_tmm": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gfdtd_adjoint": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, _dp, _dp]),
    "gfdtd_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "gfdtd_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "gfdtd_set_absorber": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_double]),
    "gfdtd_set_capture": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int64, C.c_int]),
    "gfdtd_capture_info": (C.c_int, [C.c_void_p, _i64p, _i64p, _i64p]),
    "gfdtd_read_capture": (C.c_int, [C.c_void_p, _dp, C.c_int64]),
    "gfdtd_profile_kernels": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(KernelTimes)]),
    "gfdtd_synchronize": (C.c_int, [C.c_void_p]),
    "gfdtd_watchdog": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int), _dp]),
    "gfdtd_test_stall": (C.c_int, [C.c_void_p, C.c_int]),
    "gfdtd2d_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int64, C.c_double, C.c_double, C.c_int,
                                 C.c_void_p]),
    "gfdtd2d_set_medium": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, C.c_int]),
    "gfdtd2d_add_source": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double]),
    "gfdtd2d_add_probe": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, _dp, C.POINTER(C.c_int)]),
    "gfdtd2d_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "gfdtd2d_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "gfdtd2d_read_fields": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_int64]),
    "gfdtd2d_write_fields": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_int64]),
    "gfdtd2d_read_spectrum": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp]),
    "gfdtd2d_synchronize": (C.c_int, [C.c_void_p]),
    "gfdtd2d_last_error": (C.c_char_p, [C.c_void_p]),
    "gfdtd2d_destroy": (None, [C.c_void_p]),
    "gfdtd_last_error": (C.c_char_p, [C.c_void_p]),
    "gfdtd_destroy": (None, [C.c_void_p]),
    "gfdtd_step_noalloc": (C.c_int, [C.c_int64, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int, _dp,
                                     _dp, _dp, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) the C-ABI library; raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libgfdtd.so is not built: %s" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class GfdtdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_dp)


# ------------------------------------------------------------ torch memory

_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    import torch
    L = load()

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:   # noqa: BLE001 -- reported to the library as a NULL pointer
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    rc = L.gfdtd_set_allocator(_alloc_refs[0], _alloc_refs[1], None)
    if rc != OK:
        raise GfdtdError(rc, "gfdtd_set_allocator")


def stability(S, beta, eps_r, mu_r=1.0, kind=PERTURBATION):
    """gfdtd_stability: max |zeta| of a uniform moving medium (host computation)."""
    out = C.c_double()
    rc = load().gfdtd_stability(S, beta, eps_r, mu_r, kind, C.byref(out))
    if rc != OK:
        raise GfdtdError(rc, "gfdtd_stability")
    return out.value


def _dev(x, dtype):
    """A contiguous CUDA tensor of x (argument marshalling for the sweep entry points)."""
    import torch
    t = torch.as_tensor(x, dtype=dtype)
    return t.to("cuda").contiguous()


def stability_map(S, beta, eps_r, mu_r, kind=PERTURBATION, n_theta=2048, stream=None):
    """gfdtd_stability_map: max |zeta| for every point of the (broadcast) parameter
    arrays, on the GPU.  Accepts numpy arrays or CUDA tensors; returns a CUDA
    float64 tensor (call .cpu() for numpy)."""
    import torch
    S, beta, eps_r, mu_r, kind = torch.broadcast_tensors(
        *[torch.as_tensor(v, dtype=torch.float64) for v in (S, beta, eps_r, mu_r, kind)])
    n = S.numel()
    a = [_dev(v.reshape(-1), torch.float64) for v in (S, beta, eps_r, mu_r)]
    k = _dev(kind.reshape(-1), torch.int32)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = load().gfdtd_stability_map(n, *[t.data_ptr() for t in a], k.data_ptr(), int(n_theta),
                                    out.data_ptr(), st)
    if rc != OK:
        raise GfdtdError(rc, "gfdtd_stability_map")
    return out.reshape(S.shape)


def star_tmm(stacks, beta, omega, stream=None):
    """gfdtd_star_tmm: (T, Gamma) of moving stacks for every incident frequency.

    stacks: list of (eps, mu, thick) per stack (eps, mu per layer, first and
    last semi-infinite; thick per layer, inner layers used); beta: per stack;
    omega: frequencies.  Returns two complex CUDA tensors [n_stacks, n_freq]."""
    import torch
    off = np.zeros(len(stacks) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(e) for e, _, _ in stacks])
    cat = lambda i: np.concatenate([np.asarray(st[i], float) for st in stacks]) if stacks else np.zeros(0)
    d_off = _dev(off, torch.int64)
    d_eps, d_mu, d_th = (_dev(cat(i), torch.float64) for i in range(3))
    d_beta = _dev(np.broadcast_to(np.asarray(beta, float), (len(stacks),)).copy(), torch.float64)
    d_om = _dev(np.asarray(omega, float).reshape(-1), torch.float64)
    n_s, n_f = len(stacks), d_om.numel()
    T = torch.empty(n_s * n_f * 2, dtype=torch.float64, device="cuda")
    G = torch.empty_like(T)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = load().gfdtd_star_tmm(n_s, d_off.data_ptr(), d_eps.data_ptr(), d_mu.data_ptr(), d_th.data_ptr(),
                               d_beta.data_ptr(), n_f, d_om.data_ptr(), T.data_ptr(), G.data_ptr(), st)
    if rc != OK:
        raise GfdtdError(rc, "gfdtd_star_tmm")
    as_c = lambda x: torch.view_as_complex(x.reshape(n_s, n_f, 2))
    return as_c(T), as_c(G)


def step_noalloc(B_ptr, D_ptr, nz, S, kind=PERTURBATION, beta=0.0, interp=LAYERS, z=(), eps=(1.0,),
                 mu=None, n_done=0, n_steps=1, stream=0):
    """gfdtd_step_noalloc: advance one instance held in caller-owned device buffers
    (FP32 device pointers B_ptr, D_ptr of nz elements) without allocating."""
    eps = _f64(eps)
    mu = _f64(np.ones_like(eps) if mu is None else mu)
    z = _f64(z) if len(z) else np.zeros(1)
    rc = load().gfdtd_step_noalloc(int(nz), float(S), kind, float(beta), interp, len(eps), _ptr(z),
                                   _ptr(eps), _ptr(mu), C.c_void_p(B_ptr), C.c_void_p(D_ptr),
                                   int(n_done), int(n_steps), C.c_void_p(stream))
    if rc != OK:
        raise GfdtdError(rc, "gfdtd_step_noalloc")


class Simulation:
    """A gfdtd_ctx: a batch of independent 1D instances on the current CUDA device."""

    def __init__(self, nz, S, prec=F32, stream=None):
        L = load()
        self._L = L
        nz = np.ascontiguousarray(np.atleast_1d(np.asarray(nz, dtype=np.int64)))
        self.nz = nz
        self.S = float(S)
        self.prec = prec
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        rc = L.gfdtd_create(C.byref(h), len(nz), nz.ctypes.data_as(_i64p), self.S, prec,
                            C.c_void_p(stream))
        if rc != OK:
            raise GfdtdError(rc, L.gfdtd_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, rc, what):
        if rc != OK:
            raise GfdtdError(rc, "%s: %s" % (what, self._L.gfdtd_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._L.gfdtd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- ABI calls
    def set_medium(self, inst, kind=PERTURBATION, beta=0.0, interp=LAYERS, z=(), eps=(1.0,), mu=None,
                   allow_unstable=False):
        eps = _f64(eps)
        mu = _f64(np.ones_like(eps) if mu is None else mu)
        z = _f64(z) if len(z) else np.zeros(1)
        self._check(self._L.gfdtd_set_medium(self._h, inst, kind, float(beta), interp, len(eps), _ptr(z),
                                             _ptr(eps), _ptr(mu), int(bool(allow_unstable))),
                    "set_medium")

    def add_source(self, inst, node, omega0, tau, t0, amp=1.0):
        self._check(self._L.gfdtd_add_source(self._h, inst, int(node), float(omega0), float(tau),
                                             float(t0), float(amp)), "add_source")

    def add_tfsf(self, inst, node, omega0, tau, t0, amp=1.0):
        """One-way source: total field at nodes >= node, the incident wave being the
        right-going wave of a soft source with this waveform (gfdtd_add_tfsf)."""
        self._check(self._L.gfdtd_add_tfsf(self._h, inst, int(node), float(omega0), float(tau),
                                           float(t0), float(amp)), "add_tfsf")

    def add_probe(self, inst, node, omega):
        omega = _f64(np.atleast_1d(omega))
        pid = C.c_int()
        self._check(self._L.gfdtd_add_probe(self._h, inst, int(node), len(omega), _ptr(omega),
                                            C.byref(pid)), "add_probe")
        return pid.value

    def step(self, n):
        self._check(self._L.gfdtd_step(self._h, int(n)), "step")

    def step_plain(self, n):
        self._check(self._L.gfdtd_step_plain(self._h, int(n)), "step_plain")

    def plain_floor(self, n):
        """The plain path's launch structure without its arithmetic (gfdtd_plain_floor):
        n steps' worth of launches that read and write back B and D; the state is unchanged."""
        self._check(self._L.gfdtd_plain_floor(self._h, int(n)), "plain_floor")

    def read_fields(self, inst, which=FIELD_D):
        out = np.empty(int(self.nz[inst]))
        self._check(self._L.gfdtd_read_fields(self._h, inst, which, _ptr(out), len(out)), "read_fields")
        return out

    def write_fields(self, inst, which, values):
        v = _f64(values)
        self._check(self._L.gfdtd_write_fields(self._h, inst, which, _ptr(v), len(v)), "write_fields")

    def state_layout(self):
        n, eb = C.c_int64(), C.c_int()
        offs = np.zeros(len(self.nz), dtype=np.int64)
        self._check(self._L.gfdtd_state_layout(self._h, C.byref(n), C.byref(eb), offs.ctypes.data_as(_i64p)),
                    "state_layout")
        return n.value, eb.value, offs

    def read_state(self, which, host_ptr, nbytes):
        self._check(self._L.gfdtd_read_state(self._h, which, C.c_void_p(host_ptr), int(nbytes)), "read_state")

    def write_state(self, which, host_ptr, nbytes):
        self._check(self._L.gfdtd_write_state(self._h, which, C.c_void_p(host_ptr), int(nbytes)), "write_state")

    def read_spectrum(self, inst, probe_id, n_bins):
        re, im = np.zeros(n_bins), np.zeros(n_bins)
        self._check(self._L.gfdtd_read_spectrum(self._h, inst, probe_id, _ptr(re), _ptr(im)), "read_spectrum")
        return re + 1j * im

    def adjoint(self, n_steps, probe_id, bin_lo, bin_hi, n_values):
        """gfdtd_adjoint: per-instance loss and d loss / d eps values (list of arrays)."""
        loss = np.zeros(len(self.nz))
        grad = np.zeros(int(sum(n_values)))
        self._check(self._L.gfdtd_adjoint(self._h, int(n_steps), int(probe_id), int(bin_lo), int(bin_hi),
                                          _ptr(loss), _ptr(grad)), "adjoint")
        out, o = [], 0
        for n in n_values:
            out.append(grad[o:o + n])
            o += n
        return loss, out

    def steps_done(self):
        n = C.c_int64()
        self._check(self._L.gfdtd_steps_done(self._h, C.byref(n)), "steps_done")
        return n.value

    def set_tuning(self, cells_per_lane=0, time_block=0, blocks_per_sm=0):
        self._check(self._L.gfdtd_set_tuning(self._h, cells_per_lane, time_block, blocks_per_sm),
                    "set_tuning")

    def stats(self):
        s = Stats()
        self._check(self._L.gfdtd_get_stats(self._h, C.byref(s)), "get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_absorber(self, inst, width=64, sigma=0.2):
        """Graded absorbing layers of `width` cells at both ends of instance inst (0: none)."""
        self._check(self._L.gfdtd_set_absorber(self._h, inst, int(width), float(sigma)), "set_absorber")

    def set_capture(self, inst, which, z0, z1, z_stride=1, t_stride=1, max_frames=1024, half=False):
        """Record field `which` of instance inst at cells z0:z1:z_stride after every
        t_stride steps (t_stride=0 turns capture off)."""
        self._check(self._L.gfdtd_set_capture(self._h, inst, which, z0, z1, z_stride, t_stride, max_frames,
                                              1 if half else 0), "set_capture")

    def capture(self):
        """The recorded frames as a [frames, cells] float64 array, and the dropped count."""
        f, m, d = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.gfdtd_capture_info(self._h, C.byref(f), C.byref(m), C.byref(d)), "capture_info")
        out = np.empty(f.value * m.value)
        self._check(self._L.gfdtd_read_capture(self._h, _ptr(out), len(out)), "read_capture")
        return out.reshape(f.value, m.value), d.value

    def profile_kernels(self, n):
        """Advance n steps like step(), timing each batched-kernel launch with
        CUDA events; per kernel variant: launches, total ms, cell-updates."""
        t = KernelTimes()
        self._check(self._L.gfdtd_profile_kernels(self._h, int(n), C.byref(t)), "profile_kernels")
        return {name: {"launches": t.launches[i], "ms": t.ms[i], "cell_updates": t.cell_updates[i]}
                for i, name in enumerate(KERNEL_VARIANTS)}

    def synchronize(self):
        self._check(self._L.gfdtd_synchronize(self._h), "synchronize")

    def watchdog(self, limit=1e30, reset=False):
        """gfdtd_watchdog: per-instance flags (bit 0 non-finite, bit 1 above
        `limit`) and largest |B|, |D| written since creation or the last reset.
        Returns (flags, amax); an E_UNSTABLE status is the flags themselves."""
        n = len(self.nz)
        flags = np.zeros(n, dtype=np.int32)
        amax = np.zeros(n)
        rc = self._L.gfdtd_watchdog(self._h, float(limit), int(bool(reset)),
                                    flags.ctypes.data_as(C.POINTER(C.c_int)), _ptr(amax))
        if rc not in (OK, E_UNSTABLE):
            self._check(rc, "watchdog")
        return flags, amax

    def test_stall(self, on):
        """gfdtd_test_stall: make the fast kernel's bounded waits run out (test hook)."""
        self._check(self._L.gfdtd_test_stall(self._h, int(bool(on))), "test_stall")


# ------------------------------------------------------------- 2D TE

FIELD2D_D, FIELD2D_BX, FIELD2D_BZ = 0, 1, 2


class Simulation2D:
    """A gfdtd2d_ctx: the 2D TE generalized scheme on nx periodic columns (width
    dx) of nz cells along the motion, on the current CUDA device.  Fields are
    [nx, nz] arrays: D_y at (i, k), B_x at (i, k + 1/2), B_z at (i + 1/2, k)."""

    def __init__(self, nx, nz, dx, S, prec=F32, stream=None):
        L = load()
        self._L = L
        self.nx, self.nz, self.dx, self.S, self.prec = int(nx), int(nz), float(dx), float(S), prec
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        rc = L.gfdtd2d_create(C.byref(h), self.nx, self.nz, self.dx, self.S, prec, C.c_void_p(stream))
        if rc != OK:
            raise GfdtdError(rc, "gfdtd2d_create")
        self._h = h

    def _check(self, rc, what):
        if rc != OK:
            raise GfdtdError(rc, "%s: %s" % (what, self._L.gfdtd2d_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._L.gfdtd2d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_medium(self, beta=0.0, slope=0.0, z=(), eps=(1.0,), mu=None, allow_unstable=False):
        eps = _f64(eps)
        mu = _f64(np.ones_like(eps) if mu is None else mu)
        z = _f64(z) if len(z) else np.zeros(1)
        self._check(self._L.gfdtd2d_set_medium(self._h, float(beta), float(slope), len(eps), _ptr(z), _ptr(eps),
                                               _ptr(mu), int(bool(allow_unstable))), "set_medium")

    def add_source(self, k, kx, omega0, tau, t0, amp=1.0):
        self._check(self._L.gfdtd2d_add_source(self._h, int(k), float(kx), float(omega0), float(tau), float(t0),
                                               float(amp)), "add_source")

    def add_probe(self, i, k, omega):
        omega = _f64(np.atleast_1d(omega))
        pid = C.c_int()
        self._check(self._L.gfdtd2d_add_probe(self._h, int(i), int(k), len(omega), _ptr(omega), C.byref(pid)),
                    "add_probe")
        return pid.value

    def set_tuning(self, cells_per_lane, time_block):
        self._check(self._L.gfdtd2d_set_tuning(self._h, int(cells_per_lane), int(time_block)), "set_tuning")

    def step(self, n):
        self._check(self._L.gfdtd2d_step(self._h, int(n)), "step")

    def read_fields(self, which=FIELD2D_D):
        out = np.empty(self.nx * self.nz)
        self._check(self._L.gfdtd2d_read_fields(self._h, int(which), _ptr(out), len(out)), "read_fields")
        return out.reshape(self.nx, self.nz)

    def write_fields(self, which, values):
        v = _f64(np.asarray(values).reshape(-1))
        self._check(self._L.gfdtd2d_write_fields(self._h, int(which), _ptr(v), len(v)), "write_fields")

    def read_spectrum(self, probe_id, n_bins):
        re, im = np.zeros(n_bins), np.zeros(n_bins)
        self._check(self._L.gfdtd2d_read_spectrum(self._h, int(probe_id), _ptr(re), _ptr(im)), "read_spectrum")
        return re + 1j * im

    def synchronize(self):
        self._check(self._L.gfdtd2d_synchronize(self._h), "synchronize")


# ------------------------------------------------------------- autograd

def _autograd():
    import torch

    class ProbePower(torch.autograd.Function):
        """Per-instance probe power L_i = sum_{f = bin_lo}^{bin_hi - 1} |X_f|^2 over
        n_steps from rest, as a differentiable function of every instance's
        permittivity profile values (concatenated in instance order).  The forward
        runs gfdtd_adjoint on a fresh context built by make_sim(eps_per_instance),
        which returns dL_i / d eps with the loss; backward scales those by the
        incoming gradient of each L_i."""

        @staticmethod
        def forward(ctx, eps, make_sim, n_values, n_steps, probe_id, bin_lo, bin_hi):
            e = eps.detach().to("cpu", torch.float64).numpy()
            parts = np.split(e, np.cumsum(n_values)[:-1])
            sim = make_sim(parts)
            try:
                loss, grads = sim.adjoint(n_steps, probe_id, bin_lo, bin_hi, list(n_values))
            finally:
                sim.close()
            g = torch.from_numpy(np.concatenate(grads)).to(eps.device, eps.dtype)
            owner = torch.repeat_interleave(torch.arange(len(n_values)),
                                            torch.tensor(list(n_values))).to(eps.device)
            ctx.save_for_backward(g, owner)
            return torch.from_numpy(loss).to(eps.device, eps.dtype)

        @staticmethod
        def backward(ctx, grad_loss):
            g, owner = ctx.saved_tensors
            return grad_loss[owner] * g, None, None, None, None, None, None

    return ProbePower


_probe_power_fn = None


def probe_power(eps, make_sim, n_values, n_steps, probe_id=0, bin_lo=0, bin_hi=1):
    """Differentiable per-instance probe power (see ProbePower above): `eps` is a
    1-D tensor holding the profile values of all instances (n_values[i] for
    instance i), `make_sim(list_of_eps_arrays)` returns a configured Simulation
    (media, sources, probes) at rest.  Returns a tensor of n_inst losses whose
    backward gives d loss / d eps from the GPU adjoint."""
    global _probe_power_fn
    if _probe_power_fn is None:
        _probe_power_fn = _autograd()
    return _probe_power_fn.apply(eps, make_sim, tuple(int(n) for n in n_values), int(n_steps),
                                 int(probe_id), int(bin_lo), int(bin_hi))
