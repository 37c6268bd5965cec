"""Thin ctypes binding of libpmace.so (include/pmace.h).

The functions keep the C names and only marshal arguments: array arguments
may be torch tensors (host or CUDA; their data pointers are passed through)
or numpy arrays (host).  Every step of the hot path runs in the library's
CUDA kernels; if the library is missing this module raises at import.
`Reconstruction` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# PMACE_LIBRARY selects another build of the library (for example the
# bounds-checking libpmace_debug.so); default: the in-tree libpmace.so
_LIB_PATH = os.environ.get("PMACE_LIBRARY") or os.path.join(_PKG, "libpmace.so")

PMACE_OK = 0
PMACE_ERR_INVALID_ARG = 1
PMACE_ERR_OOM = 2
PMACE_ERR_CUDA = 3
PMACE_ERR_UNSUPPORTED_SIZE = 4
PMACE_ERR_TIMEOUT = 5
PMACE_ERR_STATE = 6
PMACE_AMP_F32 = 0
PMACE_AMP_F16_SCALED = 1


class pmace_dims(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("np", ctypes.c_int32),
                ("J", ctypes.c_int32), ("kappa", ctypes.c_float)]


class pmace_step(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("rho", ctypes.c_float)]


class pmace_state_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("rho_pending", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class pmace_plan(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("cols_per_thread", ctypes.c_int32), ("stage_y", ctypes.c_int32),
                ("max_clusters", ctypes.c_int32), ("exchange", ctypes.c_int32),
                ("windows_per_cluster", ctypes.c_int32)]


class pmace_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active_jobs", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("fill_pixels", ctypes.c_int64)]


class pmace_request(ctypes.Structure):
    _fields_ = [("dims", pmace_dims), ("probe", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("amps", ctypes.c_void_p), ("fmt", ctypes.c_int32), ("scales", ctypes.c_void_p),
                ("init", ctypes.c_void_p), ("step", pmace_step), ("iterations", ctypes.c_int32)]


class pmace_job_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("finish_ms", ctypes.c_double),
                ("device_bytes", ctypes.c_int64)]


class pmace_server_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("queued", "active", "completed", "ticks", "device_bytes", "budget_bytes")]


EXPORTS = ["pmace_create", "pmace_iterate", "pmace_get_image", "pmace_get_patches",
           "pmace_residual", "pmace_get_state", "pmace_set_state", "pmace_set_profiling",
           "pmace_kernel_times", "pmace_get_plan", "pmace_device_bytes", "pmace_destroy",
           "pmace_last_error", "pmace_status_string", "pmace_abi_version",
           "pmace_amplitude_energy_noalloc", "pmace_set_plan", "pmace_autotune",
           "pmace_server_create", "pmace_server_submit", "pmace_server_poll", "pmace_server_wait",
           "pmace_server_release", "pmace_server_stats", "pmace_server_destroy",
           "pmace_simulate", "pmace_photon_noise", "pmace_selftest_bounded_wait", "pmace_debug_spectra"]


# ABI version of include/pmace.h that the structures below mirror
ABI_VERSION = 2


def load_library(path: str = _LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_2111_14240_gb300.build` "
            "(there is no CPU fallback for the PMACE hot path)")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "pmace_create": (i32, [P(pmace_dims), vp, vp, vp, i32, vp, vp, ctypes.c_int, vp, P(vp)]),
        "pmace_iterate": (i32, [vp, i32, P(pmace_step), vp]),
        "pmace_get_image": (i32, [vp, vp, ctypes.c_int, vp]),
        "pmace_get_patches": (i32, [vp, vp, ctypes.c_int, vp]),
        "pmace_residual": (i32, [vp, P(ctypes.c_double), vp]),
        "pmace_get_state": (i32, [vp, vp, vp, P(pmace_state_info), ctypes.c_int, vp]),
        "pmace_set_state": (i32, [vp, vp, vp, P(pmace_state_info), ctypes.c_int, vp]),
        "pmace_set_profiling": (i32, [vp, ctypes.c_int]),
        "pmace_kernel_times": (i32, [vp, P(ctypes.c_double), P(i64), P(ctypes.c_double), P(i64),
                                     ctypes.c_int]),
        "pmace_get_plan": (i32, [vp, P(pmace_plan)]),
        "pmace_device_bytes": (i64, [vp]),
        "pmace_destroy": (None, [vp]),
        "pmace_last_error": (ctypes.c_char_p, [vp]),
        "pmace_status_string": (ctypes.c_char_p, [i32]),
        "pmace_abi_version": (i32, []),
        "pmace_amplitude_energy_noalloc": (i32, [vp, i32, vp, i32, i32, vp, vp]),
        "pmace_set_plan": (i32, [vp, i32, i32, vp]),
        "pmace_autotune": (i32, [vp, P(pmace_step), i32, vp, P(pmace_plan)]),
        "pmace_server_create": (i32, [P(pmace_server_config), P(vp)]),
        "pmace_server_submit": (i32, [vp, P(pmace_request), P(i64)]),
        "pmace_server_poll": (i32, [vp, i64, P(pmace_job_result), vp]),
        "pmace_server_wait": (i32, [vp, i64, i32, P(pmace_job_result), vp]),
        "pmace_server_release": (i32, [vp, i64]),
        "pmace_server_stats": (i32, [vp, P(pmace_server_counters)]),
        "pmace_server_destroy": (None, [vp]),
        "pmace_simulate": (i32, [P(pmace_dims), vp, vp, vp, ctypes.c_double, ctypes.c_uint64, vp,
                                 ctypes.c_int, vp]),
        "pmace_photon_noise": (i32, [vp, i32, i32, ctypes.c_double, ctypes.c_uint64, vp, ctypes.c_int, vp]),
        "pmace_selftest_bounded_wait": (i32, [vp]),
        "pmace_debug_spectra": (i32, [vp, P(pmace_step), vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.pmace_abi_version() != ABI_VERSION:
        raise ImportError(f"{path} has ABI version {lib.pmace_abi_version()}, this binding expects "
                          f"{ABI_VERSION}: rebuild it with `python -m paper_2111_14240_gb300.build`")
    return lib


_lib = load_library()


class PmaceError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.pmace_status_string(status).decode()}: {msg}")
        self.status = status


def _check(status: int, handle=None):
    if status != PMACE_OK:
        raise PmaceError(status, _lib.pmace_last_error(handle).decode(errors="replace"))


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _on_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ----------------------------------------------------------------- C names
def pmace_abi_version() -> int:
    return _lib.pmace_abi_version()


def pmace_create(n1, n2, np_, J, kappa, probe, offsets, amps, amp_format=PMACE_AMP_F32,
                 scales=None, init=None, inputs_on_device=None, stream=None):
    """probe: (np, np) complex64 as float32 pairs; offsets: (J, 2) int32 host;
    amps: (J, np, np) float32 or float16 codes; returns the handle (c_void_p)."""
    if inputs_on_device is None:
        inputs_on_device = _on_device(amps)
    offs = offsets.cpu().numpy() if hasattr(offsets, "cpu") else np.asarray(offsets)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    dims = pmace_dims(int(n1), int(n2), int(np_), int(J), float(kappa))
    h = ctypes.c_void_p()
    st = _lib.pmace_create(ctypes.byref(dims), _ptr(probe), _ptr(offs), _ptr(amps), int(amp_format),
                           _ptr(scales), _ptr(init), int(bool(inputs_on_device)), _stream(stream),
                           ctypes.byref(h))
    _check(st, None)
    return h


def pmace_iterate(h, n, alpha, rho, stream=None):
    step = pmace_step(float(alpha), float(rho))
    _check(_lib.pmace_iterate(h, int(n), ctypes.byref(step), _stream(stream)), h)


def pmace_get_image(h, out, stream=None):
    _check(_lib.pmace_get_image(h, _ptr(out), int(_on_device(out)), _stream(stream)), h)


def pmace_get_patches(h, out, stream=None):
    _check(_lib.pmace_get_patches(h, _ptr(out), int(_on_device(out)), _stream(stream)), h)


def pmace_residual(h, stream=None):
    out = (ctypes.c_double * 2)()
    _check(_lib.pmace_residual(h, out, _stream(stream)), h)
    return float(out[0]), float(out[1])


def pmace_get_state(h, q, xbar, stream=None):
    info = pmace_state_info()
    on_dev = int(_on_device(q))
    _check(_lib.pmace_get_state(h, _ptr(q), _ptr(xbar), ctypes.byref(info), on_dev, _stream(stream)), h)
    return info


def pmace_set_state(h, q, xbar, info, stream=None):
    on_dev = int(_on_device(q))
    _check(_lib.pmace_set_state(h, _ptr(q), _ptr(xbar), ctypes.byref(info), on_dev, _stream(stream)), h)


def pmace_set_profiling(h, enable: bool):
    _check(_lib.pmace_set_profiling(h, int(bool(enable))), h)


def pmace_kernel_times(h, reset=False):
    am, cm = ctypes.c_double(), ctypes.c_double()
    an, cn = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pmace_kernel_times(h, ctypes.byref(am), ctypes.byref(an), ctypes.byref(cm),
                                   ctypes.byref(cn), int(bool(reset))), h)
    return dict(agent_ms=am.value, agent_launches=an.value, consensus_ms=cm.value,
                consensus_launches=cn.value)


def pmace_get_plan(h):
    p = pmace_plan()
    _check(_lib.pmace_get_plan(h, ctypes.byref(p)), h)
    return {k: getattr(p, k) for k, _ in pmace_plan._fields_}


def pmace_amplitude_energy_noalloc(amps, J, np_, out, amp_format=PMACE_AMP_F32, scales=None,
                                   stream=None):
    """Sum of y^2 over J np x np patterns into the device double `out`,
    allocating nothing (see include/pmace.h)."""
    _check(_lib.pmace_amplitude_energy_noalloc(_ptr(amps), int(amp_format), _ptr(scales), int(J),
                                               int(np_), _ptr(out), _stream(stream)), None)


def simulate(obj, probe, offsets, peak=None, seed=0, stream=None):
    """Measured amplitudes (J, Np, Np) float32 of `obj` (n1 x n2 complex) seen
    through `probe` at `offsets` on the GPU (include/pmace.h, pmace_simulate);
    peak None or <= 0: noiseless.  numpy in, numpy out."""
    obj = np.ascontiguousarray(obj, dtype=np.complex64)
    probe = np.ascontiguousarray(probe, dtype=np.complex64)
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    n1, n2 = obj.shape
    np_ = probe.shape[0]
    out = np.empty((offs.shape[0], np_, np_), np.float32)
    dims = pmace_dims(n1, n2, np_, offs.shape[0], 1.0)
    _check(_lib.pmace_simulate(ctypes.byref(dims), _ptr(probe), _ptr(offs), _ptr(obj),
                               float(peak) if peak else 0.0, int(seed) & (2**64 - 1), _ptr(out), 0,
                               _stream(stream)), None)
    return out


def photon_noise(intensity, peak, seed=0, stream=None):
    """Section IV photon scaling of float32 intensities (J, Np, Np) on the GPU
    (include/pmace.h, pmace_photon_noise).  numpy in, numpy out."""
    inten = np.ascontiguousarray(intensity, dtype=np.float32)
    J, n1, n2 = inten.shape
    if n1 != n2:
        raise ValueError("patterns must be square")
    out = np.empty_like(inten)
    _check(_lib.pmace_photon_noise(_ptr(inten), int(J), int(n1), float(peak), int(seed) & (2**64 - 1),
                                   _ptr(out), 0, _stream(stream)), None)
    return out


def pmace_debug_spectra(h, alpha, rho, out, stream=None):
    """One iteration that also writes every window's forward 2-D DFT
    F (d v_j), unnormalised, natural order, into the device tensor `out`
    (J, np, np, 2) float32 (include/pmace.h)."""
    step = pmace_step(float(alpha), float(rho))
    _check(_lib.pmace_debug_spectra(h, ctypes.byref(step), _ptr(out), _stream(stream)), h)


def pmace_set_plan(h, variant, tile_h, stream=None):
    _check(_lib.pmace_set_plan(h, int(variant), int(tile_h), _stream(stream)), h)


def pmace_autotune(h, alpha, rho, iters=10, stream=None):
    step = pmace_step(float(alpha), float(rho))
    p = pmace_plan()
    _check(_lib.pmace_autotune(h, ctypes.byref(step), int(iters), _stream(stream), ctypes.byref(p)), h)
    return {k: getattr(p, k) for k, _ in pmace_plan._fields_}


def pmace_device_bytes(h) -> int:
    return int(_lib.pmace_device_bytes(h))


def pmace_destroy(h):
    _lib.pmace_destroy(h)


def pmace_last_error(h=None) -> str:
    return _lib.pmace_last_error(h).decode(errors="replace")


# ----------------------------------------------------------------- wrapper
class Reconstruction:
    """One PMACE job resident on the current CUDA device (torch tensors in/out)."""

    def __init__(self, probe, offsets, amps, image_shape, *, kappa=1.25, amp_format=PMACE_AMP_F32,
                 scales=None, init=None, stream=None):
        import torch
        self.n1, self.n2 = int(image_shape[0]), int(image_shape[1])
        self.np = int(probe.shape[0])
        self.J = int(offsets.shape[0])
        self.stream = stream
        dev = torch.device("cuda", torch.cuda.current_device())
        self._probe = _as_pairs(probe, dev)
        self._amps = amps if hasattr(amps, "is_cuda") and amps.is_cuda else _to_dev(amps, dev)
        self._scales = None if scales is None else _to_dev(scales, dev).float().contiguous()
        self._init = None if init is None else _as_pairs(init, dev)
        self.h = pmace_create(self.n1, self.n2, self.np, self.J, kappa, self._probe, offsets,
                              self._amps, amp_format, self._scales, self._init, True, stream)
        self._probe = self._amps = self._scales = self._init = None

    def iterate(self, n, alpha, rho=0.5):
        pmace_iterate(self.h, n, alpha, rho, self.stream)

    def image(self):
        import torch
        out = torch.empty((self.n1, self.n2, 2), dtype=torch.float32, device="cuda")
        pmace_get_image(self.h, out, self.stream)
        return torch.view_as_complex(out)

    def patches(self):
        import torch
        out = torch.empty((self.J, self.np, self.np, 2), dtype=torch.float32, device="cuda")
        pmace_get_patches(self.h, out, self.stream)
        return torch.view_as_complex(out)

    def residual(self):
        return pmace_residual(self.h, self.stream)

    def plan(self):
        return pmace_get_plan(self.h)

    def set_plan(self, variant, tile_h=16):
        pmace_set_plan(self.h, variant, tile_h, self.stream)

    def autotune(self, alpha, rho=0.5, iters=10):
        return pmace_autotune(self.h, alpha, rho, iters, self.stream)

    def close(self):
        if self.h:
            pmace_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _to_dev(a, dev):
    import torch
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    return a.to(dev).contiguous()


def _as_pairs(z, dev):
    """Complex array -> contiguous float32 (..., 2) tensor on dev."""
    import torch
    if isinstance(z, np.ndarray):
        z = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64)))
    if z.is_complex():
        z = torch.view_as_real(z.to(torch.complex64).contiguous())
    return z.to(dev).float().contiguous()


# ----------------------------------------------------------------- serving
def _result_dict(r):
    return {k: getattr(r, k) for k, _ in pmace_job_result._fields_}


class Server:
    """Continuous-batching server (pmace_server_*): jobs are submitted with
    host arrays and read back as host images."""

    def __init__(self, hbm_budget_bytes=0, max_active_jobs=0, tile_h=0, fill_pixels=0):
        cfg = pmace_server_config(int(hbm_budget_bytes), int(max_active_jobs), int(tile_h),
                                  int(fill_pixels))
        self.h = ctypes.c_void_p()
        _check(_lib.pmace_server_create(ctypes.byref(cfg), ctypes.byref(self.h)), None)
        self.shapes = {}

    def submit(self, probe, offsets, amps, image_shape, iterations, alpha, rho=0.5, kappa=1.25,
               amp_format=PMACE_AMP_F32, scales=None, init=None):
        probe = np.ascontiguousarray(np.asarray(probe, dtype=np.complex64)).view(np.float32)
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        amps = np.ascontiguousarray(amps)
        n1, n2 = int(image_shape[0]), int(image_shape[1])
        sc = None if scales is None else np.ascontiguousarray(np.asarray(scales, dtype=np.float32))
        ini = None if init is None else np.ascontiguousarray(
            np.asarray(init, dtype=np.complex64)).view(np.float32)
        req = pmace_request(pmace_dims(n1, n2, int(probe.shape[0]), int(offs.shape[0]), float(kappa)),
                            _ptr(probe), _ptr(offs), _ptr(amps), int(amp_format), _ptr(sc), _ptr(ini),
                            pmace_step(float(alpha), float(rho)), int(iterations))
        jid = ctypes.c_int64()
        _check(_lib.pmace_server_submit(self.h, ctypes.byref(req), ctypes.byref(jid)), None)
        self.shapes[jid.value] = (n1, n2)
        return jid.value

    def _image_buf(self, jid):
        n1, n2 = self.shapes[jid]
        return np.empty((n1, n2), dtype=np.complex64)

    def poll(self, jid):
        res = pmace_job_result()
        img = self._image_buf(jid)
        _check(_lib.pmace_server_poll(self.h, jid, ctypes.byref(res), _ptr(img)), None)
        return _result_dict(res), (img if res.done and res.status == PMACE_OK else None)

    def wait(self, jid, timeout_ms=600000):
        res = pmace_job_result()
        img = self._image_buf(jid)
        _check(_lib.pmace_server_wait(self.h, jid, int(timeout_ms), ctypes.byref(res), _ptr(img)), None)
        return _result_dict(res), (img if res.status == PMACE_OK else None)

    def release(self, jid):
        _check(_lib.pmace_server_release(self.h, jid), None)
        self.shapes.pop(jid, None)

    def stats(self):
        c = pmace_server_counters()
        _check(_lib.pmace_server_stats(self.h, ctypes.byref(c)), None)
        return {k: getattr(c, k) for k, _ in pmace_server_counters._fields_}

    def close(self):
        if self.h:
            _lib.pmace_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
