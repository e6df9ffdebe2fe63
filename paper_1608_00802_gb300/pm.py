"""Python binding of the C ABI in include/pm.h (argument marshalling only).

Every stage of the step runs in the CUDA kernels of libpm.so; PyTorch only
provides the device arena and the stream.  There is no CPU fallback: if the
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpm.so")

PM_OK = 0
STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_NO_MEMORY", 3: "PM_ERR_CUDA",
          4: "PM_ERR_CUFFT", 5: "PM_ERR_NONFINITE", 6: "PM_ERR_STATE", 7: "PM_ERR_TIMEOUT"}
FORCE_MESHGRAD, FORCE_HYBRID, FORCE_LAGRANGIAN = 0, 1, 2
LAP_COMPACT, LAP_WIDE = 0, 1
FP32, FP64 = 0, 1
KERNEL_CIC, KERNEL_SPLINE = 0, 1
FIELD_RHO, FIELD_PHI, FIELD_Q = 0, 1, 2

# every entry point declared in include/pm.h
EXPORTS = ["pm_config_default", "pm_hbar_over_m", "pm_arena_bytes", "pm_create", "pm_destroy",
           "pm_set_particles", "pm_get_particles", "pm_deposit", "pm_forces", "pm_step", "pm_run",
           "pm_energy", "pm_power_spectrum", "pm_get_field", "pm_set_density", "pm_get_order",
           "pm_profile_begin", "pm_profile_end", "pm_deposit_noalloc", "pm_last_error",
           "pm_batch_arena_bytes", "pm_batch_create", "pm_batch_destroy", "pm_batch_member", "pm_batch_run",
           "pm_batch_last_error", "pm_get_tuning", "pm_set_tuning", "pm_autotune", "pm_run_adaptive",
           "pm_sort_stats", "pm_batch_info", "pm_debug_sort_timeout", "pm_checkpoint_bytes", "pm_save", "pm_load"]
NOALLOC_MAX_PARTICLES = 65536
NOALLOC_MAX_MESH = 128
STAGES = ["sort_histogram", "sort_pass", "row_start", "deposit", "fft_r2c", "green", "fft_c2r", "stencil",
          "kick", "sort_partition", "sort_merge", "other"]
CUFFT_STAGES = ("fft_r2c", "fft_c2r")


class pm_config(C.Structure):
    _fields_ = [("n_part", C.c_int64), ("n_mesh", C.c_int32), ("precision", C.c_int32),
                ("box", C.c_double), ("omega_m", C.c_double), ("omega_l", C.c_double),
                ("h", C.c_double), ("m22", C.c_double), ("quantum", C.c_int32),
                ("force_mode", C.c_int32), ("lap", C.c_int32), ("cosmological", C.c_int32),
                ("rho_floor", C.c_double), ("rho_fp64", C.c_double), ("kernel", C.c_int32),
                ("reserved", C.c_int32), ("smooth_h", C.c_double), ("fft_jit", C.c_int32),
                ("smooth_real", C.c_int32)]


class pm_tuning(C.Structure):
    _fields_ = [("stencil_rows", C.c_int32), ("stencil_planes", C.c_int32), ("stencil_stages", C.c_int32),
                ("kick_threads", C.c_int32), ("deposit_warps", C.c_int32), ("green_fused", C.c_int32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for name, _ in cls._fields_:
            setattr(t, name, int(d[name]))
        return t


class PMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError("libpm.so not built (run paper_1608_00802_gb300.build.build()): %s" % path)
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    cfgp = C.POINTER(pm_config)
    sig = {
        "pm_config_default": (None, [cfgp]),
        "pm_hbar_over_m": (C.c_double, [cfgp]),
        "pm_arena_bytes": (C.c_size_t, [cfgp]),
        "pm_create": (C.c_int, [cfgp, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "pm_destroy": (C.c_int, [vp]),
        "pm_set_particles": (C.c_int, [vp, dp, dp]),
        "pm_get_particles": (C.c_int, [vp, dp, dp]),
        "pm_deposit": (C.c_int, [vp, dp]),
        "pm_forces": (C.c_int, [vp, C.c_double, dp]),
        "pm_step": (C.c_int, [vp, C.c_double, C.c_double]),
        "pm_run": (C.c_int, [vp, C.c_int32, C.c_double, C.c_double]),
        "pm_run_adaptive": (C.c_int, [vp, C.c_double, C.c_double, C.c_double, C.c_int32, dp,
                                      C.POINTER(C.c_int32)]),
        "pm_energy": (C.c_int, [vp, C.c_double, dp]),
        "pm_power_spectrum": (C.c_int, [vp, C.c_int32, dp, dp, C.POINTER(C.c_int64)]),
        "pm_get_field": (C.c_int, [vp, C.c_int32, dp]),
        "pm_set_density": (C.c_int, [vp, dp]),
        "pm_get_order": (C.c_int, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
        "pm_sort_stats": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "pm_debug_sort_timeout": (C.c_int, [vp, C.c_int32]),
        "pm_checkpoint_bytes": (C.c_size_t, [vp]),
        "pm_save": (C.c_int, [vp, vp, C.c_size_t]),
        "pm_load": (C.c_int, [vp, vp, C.c_size_t]),
        "pm_profile_begin": (C.c_int, [vp, C.c_int32]),
        "pm_profile_end": (C.c_int, [vp, dp, C.POINTER(C.c_int64)]),
        "pm_deposit_noalloc": (C.c_int, [vp, C.c_int64, C.c_int32, C.c_double, vp, vp, vp]),
        "pm_last_error": (C.c_char_p, [vp]),
        "pm_batch_arena_bytes": (C.c_size_t, [cfgp, C.c_int32]),
        "pm_batch_create": (C.c_int, [cfgp, C.c_int32, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "pm_batch_destroy": (C.c_int, [vp]),
        "pm_batch_member": (vp, [vp, C.c_int32]),
        "pm_batch_run": (C.c_int, [vp, C.c_int32, dp, dp]),
        "pm_batch_last_error": (C.c_char_p, [vp]),
        "pm_batch_info": (C.c_int, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "pm_get_tuning": (C.c_int, [vp, C.POINTER(pm_tuning)]),
        "pm_set_tuning": (C.c_int, [vp, C.POINTER(pm_tuning)]),
        "pm_autotune": (C.c_int, [vp, C.c_int32, C.POINTER(pm_tuning)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(n_part, n_mesh, box, precision=FP32, omega_m=0.3, omega_l=0.7, h=0.7, m22=2.5,
                quantum=True, force_mode=FORCE_MESHGRAD, lap=LAP_COMPACT, cosmological=True,
                rho_floor=1e-6, rho_fp64=1e-2, kernel=KERNEL_CIC, smooth_h=3.5, fft_jit=False,
                smooth_real=False) -> pm_config:
    cfg = pm_config()
    lib().pm_config_default(C.byref(cfg))
    cfg.n_part, cfg.n_mesh, cfg.box = int(n_part), int(n_mesh), float(box)
    cfg.precision = int(precision)
    cfg.omega_m, cfg.omega_l, cfg.h, cfg.m22 = float(omega_m), float(omega_l), float(h), float(m22)
    cfg.quantum, cfg.force_mode, cfg.lap = int(bool(quantum)), int(force_mode), int(lap)
    cfg.cosmological = int(bool(cosmological))
    cfg.rho_floor, cfg.rho_fp64 = float(rho_floor), float(rho_fp64)
    cfg.kernel, cfg.smooth_h = int(kernel), float(smooth_h)
    cfg.fft_jit = int(bool(fft_jit))
    cfg.smooth_real = int(bool(smooth_real))
    return cfg


def arena_bytes(cfg: pm_config) -> int:
    return int(lib().pm_arena_bytes(C.byref(cfg)))


def tuning_key(cfg: pm_config) -> str:
    """Configurations with the same key share launch shapes."""
    return "n%d_N%d_p%d_q%d_f%d_l%d_k%d" % (cfg.n_part, cfg.n_mesh, cfg.precision, cfg.quantum, cfg.force_mode,
                                           cfg.lap, cfg.kernel)


class TuningCache(dict):
    """Autotuner results by configuration key, optionally kept in a JSON file
    (written after every new entry)."""

    def __init__(self, path=None):
        super().__init__()
        self.path = path
        if path and os.path.exists(path):
            import json
            with open(path) as fh:
                self.update(json.load(fh))

    def __setitem__(self, key, value):
        super().__setitem__(key, dict(value))
        if self.path:
            import json
            tmp = self.path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(dict(self), fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


class Sim:
    """One simulation: a device arena (a torch uint8 tensor) and a stream.

    Methods mirror the C entry points; arrays are numpy float64 (n, 3) or
    (N, N, N) indexed [z, y, x].
    """

    def __init__(self, cfg: pm_config, device=None, stream=None, arena=None, handle=None):
        import torch
        self.cfg = cfg
        if handle is not None:  # a batch member: the batch owns the handle and the arena
            self.n, self.N, self.handle, self.owned = int(cfg.n_part), int(cfg.n_mesh), handle, False
            return
        self.owned = True
        self.n = int(cfg.n_part)
        self.N = int(cfg.n_mesh)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = arena_bytes(cfg)
        if nbytes == 0:
            raise PMError(1, lib().pm_last_error(None).decode())
        if arena is None:
            arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        elif arena.numel() * arena.element_size() < nbytes:
            raise PMError(2, "arena too small")
        self.arena = arena
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = lib().pm_create(C.byref(cfg), C.c_void_p(arena.data_ptr()), C.c_size_t(nbytes),
                             C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != PM_OK:
            raise PMError(st, lib().pm_last_error(None).decode())
        self.handle = h

    # -- helpers
    def _check(self, st):
        if st != PM_OK:
            raise PMError(st, lib().pm_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None) and getattr(self, "owned", True):
            lib().pm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI
    def set_particles(self, x, p):
        x = np.ascontiguousarray(x, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        assert x.shape == (self.n, 3) and p.shape == (self.n, 3)
        self._check(lib().pm_set_particles(self.handle, _dptr(x), _dptr(p)))

    def get_particles(self, x=None, p=None):
        """Positions and momenta in id order; x, p may be preallocated (e.g.
        pinned) float64 (n, 3) arrays."""
        x = np.empty((self.n, 3)) if x is None else x
        p = np.empty((self.n, 3)) if p is None else p
        assert x.dtype == np.float64 and x.flags.c_contiguous and x.shape == (self.n, 3)
        assert p.dtype == np.float64 and p.flags.c_contiguous and p.shape == (self.n, 3)
        self._check(lib().pm_get_particles(self.handle, _dptr(x), _dptr(p)))
        return x, p

    def deposit(self, copy=True):
        if not copy:
            self._check(lib().pm_deposit(self.handle, None))
            return None
        rho = np.empty((self.N, self.N, self.N))
        self._check(lib().pm_deposit(self.handle, _dptr(rho)))
        return rho

    def forces(self, a):
        acc = np.empty((self.n, 3))
        self._check(lib().pm_forces(self.handle, float(a), _dptr(acc)))
        return acc

    def step(self, a0, a1):
        self._check(lib().pm_step(self.handle, float(a0), float(a1)))

    def run(self, nsteps, a_start, a_end):
        self._check(lib().pm_run(self.handle, int(nsteps), float(a_start), float(a_end)))

    def run_adaptive(self, a_start, a_end, cfl=0.5, max_steps=100000):
        """Adaptive leapfrog to a_end; returns the step boundaries (a or t)."""
        bounds = np.empty(int(max_steps) + 1)
        done = C.c_int32(0)
        self._check(lib().pm_run_adaptive(self.handle, float(a_start), float(a_end), float(cfl), int(max_steps),
                                          _dptr(bounds), C.byref(done)))
        return bounds[:done.value + 1].copy()

    def energy(self, a):
        out = np.empty(6)
        self._check(lib().pm_energy(self.handle, float(a), _dptr(out)))
        return out

    def power_spectrum(self, nbins=None):
        nbins = self.N // 2 if nbins is None else int(nbins)
        k = np.empty(nbins)
        pk = np.empty(nbins)
        cnt = np.empty(nbins, dtype=np.int64)
        self._check(lib().pm_power_spectrum(self.handle, nbins, _dptr(k), _dptr(pk),
                                            cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        return k, pk, cnt

    def get_field(self, which):
        f = np.empty((self.N, self.N, self.N))
        self._check(lib().pm_get_field(self.handle, int(which), _dptr(f)))
        return f

    def set_density(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (self.N, self.N, self.N)
        self._check(lib().pm_set_density(self.handle, _dptr(rho)))

    def get_order(self):
        cell = np.empty(self.n, dtype=np.uint32)
        ids = np.empty(self.n, dtype=np.uint32)
        self._check(lib().pm_get_order(self.handle, cell.ctypes.data_as(C.POINTER(C.c_uint32)),
                                       ids.ctypes.data_as(C.POINTER(C.c_uint32))))
        return cell, ids

    def get_tuning(self):
        t = pm_tuning()
        self._check(lib().pm_get_tuning(self.handle, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, shapes):
        """Sets the launch shapes; keys missing from `shapes` keep their values."""
        cur = self.get_tuning()
        cur.update(shapes)
        t = pm_tuning.from_dict(cur)
        self._check(lib().pm_set_tuning(self.handle, C.byref(t)))

    def autotune(self, reps=5, cache=None):
        """Launch shapes for this simulation: taken from `cache` (a TuningCache)
        when it holds this configuration, else measured on the current state
        (particles must be set) and stored there.  Returns the shapes."""
        key = tuning_key(self.cfg)
        if cache is not None and key in cache:
            self.set_tuning(cache[key])
            return cache[key]
        t = pm_tuning()
        self._check(lib().pm_autotune(self.handle, int(reps), C.byref(t)))
        if cache is not None:
            cache[key] = t.as_dict()
        return t.as_dict()

    def debug_sort_timeout(self, spin_limit=64):
        """Status of a radix pass whose look-back waits on a tile that never
        publishes (a test of the bounded device waits; PM_ERR_TIMEOUT)."""
        return int(lib().pm_debug_sort_timeout(self.handle, int(spin_limit)))

    def sort_stats(self):
        """(incremental re-sorts, particles they moved) since creation."""
        r, m = C.c_int64(0), C.c_int64(0)
        self._check(lib().pm_sort_stats(self.handle, C.byref(r), C.byref(m)))
        return int(r.value), int(m.value)

    def save(self):
        """The checkpoint (numpy uint8 array) this simulation continues from:
        records in storage order, keys, statistics, launch shapes."""
        buf = np.empty(int(lib().pm_checkpoint_bytes(self.handle)), dtype=np.uint8)
        self._check(lib().pm_save(self.handle, buf.ctypes.data_as(C.c_void_p), buf.nbytes))
        return buf

    def load(self, buf):
        """Continues from a checkpoint of `save` (same n_part, n_mesh, precision, kernel)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(lib().pm_load(self.handle, buf.ctypes.data_as(C.c_void_p), buf.nbytes))

    def profile_begin(self, capacity):
        self._check(lib().pm_profile_begin(self.handle, int(capacity)))

    def profile_end(self):
        """{stage: (total ms, launches)} of the launches since profile_begin."""
        ms = np.zeros(len(STAGES))
        cnt = np.zeros(len(STAGES), dtype=np.int64)
        self._check(lib().pm_profile_end(self.handle, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(STAGES)}


def deposit_noalloc(x_dev, n_mesh, box, rho_dev, stream=None, err_dev=None):
    """pm_deposit_noalloc on torch CUDA tensors: x_dev float64 (n, 3), rho_dev
    float32 (N, N, N); enqueued on `stream` (default: the current stream).
    err_dev (optional): a one-element int32 CUDA tensor that receives the
    call's device error bits in stream order (0 = ok)."""
    import torch
    assert x_dev.is_cuda and x_dev.dtype == torch.float64 and x_dev.is_contiguous() and x_dev.shape[1] == 3
    assert rho_dev.is_cuda and rho_dev.dtype == torch.float32 and rho_dev.is_contiguous()
    assert rho_dev.numel() == n_mesh ** 3
    err_ptr = None
    if err_dev is not None:
        assert err_dev.is_cuda and err_dev.dtype == torch.int32 and err_dev.numel() >= 1
        err_ptr = C.c_void_p(err_dev.data_ptr())
    st_obj = stream if stream is not None else torch.cuda.current_stream(x_dev.device)
    st = lib().pm_deposit_noalloc(C.c_void_p(x_dev.data_ptr()), int(x_dev.shape[0]), int(n_mesh), float(box),
                                  C.c_void_p(rho_dev.data_ptr()), err_ptr, C.c_void_p(st_obj.cuda_stream))
    if st != PM_OK:
        raise PMError(st, lib().pm_last_error(None).decode())


class Batch:
    """Many independent simulations stepped together (pm_batch_*)."""

    def __init__(self, cfgs, device=None, stream=None):
        import torch
        self.cfgs = list(cfgs)
        arr = (pm_config * len(self.cfgs))(*self.cfgs)
        self._arr = arr
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = int(lib().pm_batch_arena_bytes(arr, len(self.cfgs)))
        if nbytes == 0:
            raise PMError(1, lib().pm_last_error(None).decode())
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = lib().pm_batch_create(arr, len(self.cfgs), C.c_void_p(self.arena.data_ptr()), C.c_size_t(nbytes),
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != PM_OK:
            raise PMError(st, lib().pm_last_error(None).decode())
        self.handle = h
        self.members = [Sim(c, handle=C.c_void_p(lib().pm_batch_member(h, i))) for i, c in enumerate(self.cfgs)]

    def run(self, nsteps, a_start, a_end):
        a0 = np.ascontiguousarray(np.broadcast_to(np.asarray(a_start, dtype=np.float64), (len(self.cfgs),)))
        a1 = np.ascontiguousarray(np.broadcast_to(np.asarray(a_end, dtype=np.float64), (len(self.cfgs),)))
        st = lib().pm_batch_run(self.handle, int(nsteps), _dptr(a0), _dptr(a1))
        if st != PM_OK:
            raise PMError(st, lib().pm_batch_last_error(self.handle).decode())

    def info(self):
        """(classes, members the last run stepped by packed launches)."""
        c, p = C.c_int32(0), C.c_int32(0)
        st = lib().pm_batch_info(self.handle, C.byref(c), C.byref(p))
        if st != PM_OK:
            raise PMError(st, lib().pm_batch_last_error(self.handle).decode())
        return int(c.value), int(p.value)

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.handle = None
            lib().pm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
