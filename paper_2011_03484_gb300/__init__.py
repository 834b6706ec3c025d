"""GB300-native GLISSE test-particle map: Python binding of libglisse.so.

Thin ctypes layer over the C ABI in ``include/glisse.h``: the functions keep
the C names and only marshal arguments (numpy arrays for host buffers, torch
tensors or raw integers for device pointers).  Every step of the map runs in
the library's CUDA kernels; there is no CPU fallback.  If the library has not
been built (``paper_2011_03484_gb300._build.build()``) or no CUDA device is
usable, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GLISSE_OK = 0
GLISSE_E_INVAL = -1
GLISSE_E_NOMEM = -2
GLISSE_E_CUDA = -3
GLISSE_E_KEPLER = -4
GLISSE_E_TIMEOUT = -5
GLISSE_E_STATE = -6
GLISSE_MAX_PLANETS = 8
GLISSE_ALIVE = 0
GLISSE_REMOVED_ESCAPE = -1
GLISSE_REMOVED_KEPLER = -2
GLISSE_REMOVED_NONFINITE = -3
GLISSE_KEPLER_CONVERGE = 0
GLISSE_KEPLER_PAPER_FIXED = 1
GLISSE_PAPER_KEPLER_TOL = 1e-14
GLISSE_MAX_KEPLER_ITERS = 64
GLISSE_ENC_HILL = 0
GLISSE_ENC_FIXED = 1
GLISSE_SORT_NONE = 0
GLISSE_SORT_COST = 1
GLISSE_LAUNCH_AUTO, GLISSE_LAUNCH_PLAIN, GLISSE_LAUNCH_TASKS = 0, 1, 2
GLISSE_DIFF_AUTO = -1
GLISSE_DIFF_TAPE_TANGENT = -2
GLISSE_MATH_RSQRT, GLISSE_MATH_RCP, GLISSE_MATH_RCP40, GLISSE_MATH_KRCUBE = 0, 1, 2, 3
GLISSE_MATH_FLOAT_SQUARE, GLISSE_MATH_FLOAT_CUBE, GLISSE_MATH_D2F = 4, 5, 6
GLISSE_WAIT_PARTICLE_TASKS, GLISSE_WAIT_DIFF_FORWARD, GLISSE_WAIT_DIFF_BACKWARD = 0, 1, 2
GLISSE_FRAME_HELIO = 0
GLISSE_FRAME_BARY = 1

# every symbol the header declares (checked by the tests against the built library)
EXPORTED = (
    "glisse_opts_default", "glisse_create", "glisse_advance", "glisse_read", "glisse_status",
    "glisse_read_planets", "glisse_set_ephemeris", "glisse_destroy", "glisse_strerror",
    "glisse_partition_device", "glisse_fp64_peak", "glisse_timings", "glisse_partition_device_noalloc",
    "glisse_batch_create", "glisse_batch_advance", "glisse_batch_read", "glisse_batch_status",
    "glisse_batch_timings", "glisse_batch_steps_done", "glisse_batch_tune", "glisse_batch_set_launch",
    "glisse_batch_destroy",
    "glisse_diff_create", "glisse_diff_forward", "glisse_diff_backward", "glisse_diff_backward_growth",
    "glisse_diff_growth_gradient", "glisse_diff_checkpoint_every",
    "glisse_diff_destroy",
    "glisse_set_sampling", "glisse_read_elements", "glisse_read_libration", "glisse_selftest_math",
    "glisse_selftest_wait",
    "glisse_checkpoint_size", "glisse_checkpoint", "glisse_resume", "glisse_sizes",
    "glisse_batch_checkpoint_size", "glisse_batch_checkpoint", "glisse_batch_resume", "glisse_batch_sizes",
)

GLISSE_PARTITION_NOALLOC_MAX = 67108864


class glisse_timing(C.Structure):
    _fields_ = [
        ("particle_ms", C.c_double),
        ("particle_launches", C.c_int64),
        ("particle_steps", C.c_int64),
        ("ephemeris_ms", C.c_double),
        ("ephemeris_launches", C.c_int64),
        ("compact_ms", C.c_double),
        ("compact_launches", C.c_int64),
    ]


class glisse_opts(C.Structure):
    _fields_ = [
        ("chunk_steps", C.c_int32),
        ("resync_chunks", C.c_int32),
        ("kepler_mode", C.c_int32),
        ("kepler_iters", C.c_int32),
        ("enc_mode", C.c_int32),
        ("timing", C.c_int32),
        ("sort_mode", C.c_int32),
        ("launch_mode", C.c_int32),
        ("enc_value", C.c_double),
        ("r_max", C.c_double),
        ("cuda_stream", C.c_void_p),
    ]


class glisse_sampling(C.Structure):
    _fields_ = [
        ("every", C.c_int32),
        ("frame", C.c_int32),
        ("max_samples", C.c_int64),
        ("res_planet", C.c_int32),
        ("res_p", C.c_int32),
        ("res_q", C.c_int32),
        ("pad_", C.c_int32),
        ("avoid_deg", C.c_double),
    ]


class GlisseError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libglisse.so (optionally building it first).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(
            "libglisse.so is not built; run paper_2011_03484_gb300._build.build() (needs nvcc for sm_103a)")
    L = C.CDLL(_build.LIB)
    dp, i64p, i32p, u8p, vp = (C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                               C.POINTER(C.c_uint8), C.c_void_p)
    L.glisse_opts_default.argtypes = [C.POINTER(glisse_opts)]
    L.glisse_opts_default.restype = None
    L.glisse_create.argtypes = [C.POINTER(vp), C.c_double, dp, C.c_int32, dp, C.c_int64, C.c_double,
                                C.POINTER(glisse_opts)]
    L.glisse_create.restype = C.c_int
    L.glisse_advance.argtypes = [vp, C.c_int64]
    L.glisse_advance.restype = C.c_int
    L.glisse_read.argtypes = [vp, dp, u8p, i64p, i32p]
    L.glisse_read.restype = C.c_int
    L.glisse_status.argtypes = [vp, i64p, i64p, dp]
    L.glisse_status.restype = C.c_int
    L.glisse_read_planets.argtypes = [vp, dp, dp]
    L.glisse_read_planets.restype = C.c_int
    L.glisse_set_ephemeris.argtypes = [vp, dp, C.c_int64]
    L.glisse_set_ephemeris.restype = C.c_int
    L.glisse_destroy.argtypes = [vp]
    L.glisse_destroy.restype = None
    L.glisse_checkpoint_size.argtypes = [vp, i64p]
    L.glisse_checkpoint_size.restype = C.c_int
    L.glisse_checkpoint.argtypes = [vp, vp, C.c_int64]
    L.glisse_checkpoint.restype = C.c_int
    L.glisse_resume.argtypes = [C.POINTER(vp), vp, C.c_int64, C.POINTER(glisse_opts)]
    L.glisse_resume.restype = C.c_int
    L.glisse_sizes.argtypes = [vp, i64p, i32p]
    L.glisse_sizes.restype = C.c_int
    L.glisse_batch_checkpoint_size.argtypes = [vp, i64p]
    L.glisse_batch_checkpoint_size.restype = C.c_int
    L.glisse_batch_checkpoint.argtypes = [vp, vp, C.c_int64]
    L.glisse_batch_checkpoint.restype = C.c_int
    L.glisse_batch_resume.argtypes = [C.POINTER(vp), vp, C.c_int64, C.POINTER(glisse_opts)]
    L.glisse_batch_resume.restype = C.c_int
    L.glisse_batch_sizes.argtypes = [vp, i64p, i32p]
    L.glisse_batch_sizes.restype = C.c_int
    L.glisse_strerror.argtypes = [C.c_int]
    L.glisse_strerror.restype = C.c_char_p
    L.glisse_partition_device.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
    L.glisse_partition_device.restype = C.c_int
    L.glisse_partition_device_noalloc.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
    L.glisse_partition_device_noalloc.restype = C.c_int
    L.glisse_fp64_peak.argtypes = [C.c_int32, dp, dp]
    L.glisse_fp64_peak.restype = C.c_int
    L.glisse_timings.argtypes = [vp, C.POINTER(glisse_timing), C.c_int32]
    L.glisse_timings.restype = C.c_int
    L.glisse_batch_create.argtypes = [C.POINTER(vp), C.c_int32, dp, i32p, dp, i64p, dp, dp, C.POINTER(glisse_opts)]
    L.glisse_batch_create.restype = C.c_int
    L.glisse_batch_advance.argtypes = [vp, C.c_int64]
    L.glisse_batch_advance.restype = C.c_int
    L.glisse_batch_read.argtypes = [vp, dp, u8p, i64p, i32p]
    L.glisse_batch_read.restype = C.c_int
    L.glisse_batch_status.argtypes = [vp, i64p, i64p]
    L.glisse_batch_status.restype = C.c_int
    L.glisse_batch_timings.argtypes = [vp, C.POINTER(glisse_timing), C.c_int32]
    L.glisse_batch_timings.restype = C.c_int
    L.glisse_batch_steps_done.argtypes = [vp, C.POINTER(C.c_int64)]
    L.glisse_batch_steps_done.restype = C.c_int
    L.glisse_batch_tune.argtypes = [vp, C.c_int32, i32p, i32p, i32p]
    L.glisse_batch_tune.restype = C.c_int
    L.glisse_batch_set_launch.argtypes = [vp, C.c_int32, C.c_int32]
    L.glisse_batch_set_launch.restype = C.c_int
    L.glisse_batch_destroy.argtypes = [vp]
    L.glisse_batch_destroy.restype = None
    L.glisse_diff_create.argtypes = [C.POINTER(vp), C.c_double, dp, C.c_int32, C.c_int64, C.c_double, C.c_int64,
                                     C.c_int32, C.POINTER(glisse_opts)]
    L.glisse_diff_create.restype = C.c_int
    L.glisse_diff_forward.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp, vp, vp, vp]
    L.glisse_diff_forward.restype = C.c_int
    L.glisse_diff_backward.argtypes = [vp, vp, vp, vp]
    L.glisse_diff_backward.restype = C.c_int
    L.glisse_diff_backward_growth.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.glisse_diff_backward_growth.restype = C.c_int
    L.glisse_diff_growth_gradient.argtypes = [vp, vp, vp, vp, vp, vp]
    L.glisse_diff_growth_gradient.restype = C.c_int
    L.glisse_diff_destroy.argtypes = [vp]
    L.glisse_diff_destroy.restype = None
    L.glisse_diff_checkpoint_every.argtypes = [vp, C.POINTER(C.c_int32)]
    L.glisse_diff_checkpoint_every.restype = C.c_int
    L.glisse_set_sampling.argtypes = [vp, C.POINTER(glisse_sampling)]
    L.glisse_set_sampling.restype = C.c_int
    L.glisse_read_elements.argtypes = [vp, dp, i64p, C.c_int64, i64p]
    L.glisse_read_elements.restype = C.c_int
    L.glisse_read_libration.argtypes = [vp, u8p, u8p, i32p]
    L.glisse_read_libration.restype = C.c_int
    L.glisse_selftest_math.argtypes = [C.c_int32, vp, vp, vp, C.c_int64, vp]
    L.glisse_selftest_math.restype = C.c_int
    L.glisse_selftest_wait.argtypes = [C.c_int32, C.c_int32, i32p, vp]
    L.glisse_selftest_wait.restype = C.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _check(rc, what):
    if rc != GLISSE_OK:
        raise GlisseError(rc, what)


def strerror(code: int) -> str:
    try:
        return load().glisse_strerror(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def glisse_opts_default() -> glisse_opts:
    o = glisse_opts()
    load().glisse_opts_default(C.byref(o))
    return o


def glisse_create(star_mass, planets, particles, dt, opts: glisse_opts | None = None):
    """Create a context from host arrays planets [np][7] and particles [n][6]; returns a handle."""
    L = load()
    pl = np.ascontiguousarray(planets, dtype=np.float64).reshape(-1, 7)
    pa = np.ascontiguousarray(particles, dtype=np.float64).reshape(-1, 6)
    h = C.c_void_p()
    rc = L.glisse_create(C.byref(h), float(star_mass), _dp(pl) if pl.size else None, pl.shape[0],
                         _dp(pa) if pa.size else None, pa.shape[0], float(dt),
                         C.byref(opts) if opts is not None else None)
    _check(rc, "glisse_create")
    return h


def glisse_advance(h, n_steps: int):
    _check(load().glisse_advance(h, int(n_steps)), "glisse_advance")


def glisse_read(h, n: int, out=None):
    """Returns dict(state [n][6], alive [n] bool, removal_step [n], removal_reason [n]).
    out: optional dict of preallocated host arrays (state float64 [n][6], alive uint8 [n],
    removal_step int64 [n], removal_reason int32 [n]), e.g. in pinned memory, written in place."""
    if out is not None:
        st, alive, steps, rsn = out["state"], out["alive"], out["removal_step"], out["removal_reason"]
        assert st.dtype == np.float64 and st.shape == (n, 6) and st.flags.c_contiguous
        assert alive.dtype == np.uint8 and steps.dtype == np.int64 and rsn.dtype == np.int32
    else:
        st = np.empty((n, 6))
        alive = np.empty(n, dtype=np.uint8)
        steps = np.empty(n, dtype=np.int64)
        rsn = np.empty(n, dtype=np.int32)
    rc = load().glisse_read(h, _dp(st), alive.ctypes.data_as(C.POINTER(C.c_uint8)),
                            steps.ctypes.data_as(C.POINTER(C.c_int64)), rsn.ctypes.data_as(C.POINTER(C.c_int32)))
    _check(rc, "glisse_read")
    return {"state": st, "alive": alive.astype(bool), "removal_step": steps, "removal_reason": rsn}


def glisse_set_sampling(h, every=None, frame=GLISSE_FRAME_BARY, max_samples=0, res_planet=-1, res_p=0, res_q=0,
                        avoid_deg=10.0):
    """Start element sampling every `every` steps (None: stop sampling)."""
    if every is None:
        _check(load().glisse_set_sampling(h, None), "glisse_set_sampling")
        return
    sp = glisse_sampling(int(every), int(frame), int(max_samples), int(res_planet), int(res_p), int(res_q), 0,
                         float(avoid_deg))
    _check(load().glisse_set_sampling(h, C.byref(sp)), "glisse_set_sampling")


def glisse_read_elements(h, n: int, max_samples: int):
    """Returns (elements [k][n][6], sample_steps [k]) for the k <= max_samples kept samples."""
    el = np.empty((max(max_samples, 0), n, 6))
    steps = np.empty(max(max_samples, 0), dtype=np.int64)
    k = C.c_int64()
    _check(load().glisse_read_elements(h, _dp(el) if max_samples > 0 else None,
                                       steps.ctypes.data_as(C.POINTER(C.c_int64)), int(max_samples),
                                       C.byref(k)), "glisse_read_elements")
    return el[:k.value], steps[:k.value]


def glisse_read_libration(h, n: int):
    """Returns dict(near0, near180 [n] bool, count [n], librating [n] bool)."""
    n0 = np.zeros(n, dtype=np.uint8)
    n1 = np.zeros(n, dtype=np.uint8)
    cnt = np.zeros(n, dtype=np.int32)
    _check(load().glisse_read_libration(h, n0.ctypes.data_as(C.POINTER(C.c_uint8)),
                                        n1.ctypes.data_as(C.POINTER(C.c_uint8)),
                                        cnt.ctypes.data_as(C.POINTER(C.c_int32))), "glisse_read_libration")
    return {"near0": n0.astype(bool), "near180": n1.astype(bool), "count": cnt,
            "librating": (cnt > 0) & ~(n0.astype(bool) & n1.astype(bool))}


def glisse_selftest_math(fn, a, b=None):
    """Evaluate a device arithmetic helper on CUDA float64 tensors a (and b); returns a tensor."""
    import torch

    a = a.contiguous()
    out = torch.empty_like(a)
    bp = b.contiguous().data_ptr() if b is not None else None
    stream = torch.cuda.current_stream(a.device).cuda_stream
    _check(load().glisse_selftest_math(int(fn), a.data_ptr(), bp, out.data_ptr(), a.numel(), stream),
           "glisse_selftest_math")
    return out


def glisse_selftest_wait(which, polls=1000, stream=None) -> int:
    """Run one task launch whose bounded wait is made to run out (see include/glisse.h);
    returns the kernel's status word (GLISSE_E_TIMEOUT expected)."""
    st = C.c_int32(0)
    _check(load().glisse_selftest_wait(int(which), int(polls), C.byref(st), stream), "glisse_selftest_wait")
    return st.value


def glisse_status(h):
    nl, st, t = C.c_int64(), C.c_int64(), C.c_double()
    _check(load().glisse_status(h, C.byref(nl), C.byref(st), C.byref(t)), "glisse_status")
    return nl.value, st.value, t.value


def glisse_read_planets(h, n_planets: int):
    out = np.empty((n_planets, 7))
    t = C.c_double()
    _check(load().glisse_read_planets(h, _dp(out), C.byref(t)), "glisse_read_planets")
    return out, t.value


def glisse_set_ephemeris(h, log):
    lg = np.ascontiguousarray(log, dtype=np.float64)
    n = lg.shape[0] - 1
    _check(load().glisse_set_ephemeris(h, _dp(lg) if lg.size else None, n), "glisse_set_ephemeris")


def glisse_destroy(h):
    if h:
        load().glisse_destroy(h)


def glisse_checkpoint(h) -> np.ndarray:
    """The context's checkpoint as a uint8 array (host bytes; see glisse_resume)."""
    L = load()
    n = C.c_int64()
    _check(L.glisse_checkpoint_size(h, C.byref(n)), "glisse_checkpoint_size")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(L.glisse_checkpoint(h, buf.ctypes.data, n.value), "glisse_checkpoint")
    return buf


def glisse_resume(buf, opts: glisse_opts | None = None):
    """A new context from a checkpoint (bytes or uint8 array); returns a handle.  Of opts
    only cuda_stream and timing are used."""
    b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray)) else buf,
                             dtype=np.uint8)
    h = C.c_void_p()
    rc = load().glisse_resume(C.byref(h), b.ctypes.data, b.size, C.byref(opts) if opts is not None else None)
    _check(rc, "glisse_resume")
    return h


def glisse_batch_checkpoint(h) -> np.ndarray:
    """The batch's checkpoint as a uint8 array (host bytes; see glisse_batch_resume)."""
    L = load()
    n = C.c_int64()
    _check(L.glisse_batch_checkpoint_size(h, C.byref(n)), "glisse_batch_checkpoint_size")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(L.glisse_batch_checkpoint(h, buf.ctypes.data, n.value), "glisse_batch_checkpoint")
    return buf


def glisse_batch_resume(buf, opts: glisse_opts | None = None):
    """A new batch from a checkpoint (bytes or uint8 array); returns a handle.  Of opts only
    cuda_stream and timing are used."""
    b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray)) else buf,
                             dtype=np.uint8)
    h = C.c_void_p()
    rc = load().glisse_batch_resume(C.byref(h), b.ctypes.data, b.size, C.byref(opts) if opts is not None else None)
    _check(rc, "glisse_batch_resume")
    return h


def glisse_batch_sizes(h):
    """(number of particles, number of systems) of a batch."""
    n, ns = C.c_int64(), C.c_int32()
    _check(load().glisse_batch_sizes(h, C.byref(n), C.byref(ns)), "glisse_batch_sizes")
    return n.value, ns.value


def glisse_sizes(h):
    """(number of particles, number of planets) of a context."""
    n, npl = C.c_int64(), C.c_int32()
    _check(load().glisse_sizes(h, C.byref(n), C.byref(npl)), "glisse_sizes")
    return n.value, npl.value


def glisse_partition_device(n, ld, alive_ptr, src_ptr, src_id_ptr, dst_ptr, dst_id_ptr, n_out_ptr, stream=0):
    """Device-level stable partition; all pointers are device addresses (ints)."""
    rc = load().glisse_partition_device(int(n), int(ld), alive_ptr, src_ptr, src_id_ptr, dst_ptr, dst_id_ptr,
                                        n_out_ptr, stream)
    _check(rc, "glisse_partition_device")


def glisse_partition_device_noalloc(n, ld, alive_ptr, src_ptr, src_id_ptr, dst_ptr, dst_id_ptr, n_out_ptr,
                                    stream=0):
    """Stable partition without allocating: the scratch is a fixed array in the library's
    device image (limit GLISSE_PARTITION_NOALLOC_MAX slots).  For callers that must not
    allocate device memory.  Calls that overlap on the GPU share that array and race."""
    rc = load().glisse_partition_device_noalloc(int(n), int(ld), alive_ptr, src_ptr, src_id_ptr, dst_ptr,
                                                dst_id_ptr, n_out_ptr, stream)
    _check(rc, "glisse_partition_device_noalloc")


def glisse_timings(h, reset: bool = False) -> dict:
    t = glisse_timing()
    _check(load().glisse_timings(h, C.byref(t), 1 if reset else 0), "glisse_timings")
    return {name: getattr(t, name) for name, _ in glisse_timing._fields_}


def glisse_fp64_peak(iterations: int = 20000):
    """(DFMA instructions per second, SM MHz) measured on the current device."""
    r, mhz = C.c_double(), C.c_double()
    _check(load().glisse_fp64_peak(int(iterations), C.byref(r), C.byref(mhz)), "glisse_fp64_peak")
    return r.value, mhz.value


def glisse_batch_create(star_mass, n_planets, planets, n_particles, particles, dt, opts: glisse_opts | None = None):
    """Batch of independent systems from concatenated host arrays; returns a handle."""
    L = load()
    m0 = np.ascontiguousarray(star_mass, dtype=np.float64)
    npl = np.ascontiguousarray(n_planets, dtype=np.int32)
    npa = np.ascontiguousarray(n_particles, dtype=np.int64)
    pl = np.ascontiguousarray(planets, dtype=np.float64).reshape(-1, 7)
    pa = np.ascontiguousarray(particles, dtype=np.float64).reshape(-1, 6)
    d = np.ascontiguousarray(dt, dtype=np.float64)
    h = C.c_void_p()
    rc = L.glisse_batch_create(C.byref(h), len(m0), _dp(m0), npl.ctypes.data_as(C.POINTER(C.c_int32)),
                               _dp(pl) if pl.size else None, npa.ctypes.data_as(C.POINTER(C.c_int64)),
                               _dp(pa) if pa.size else None, _dp(d), C.byref(opts) if opts is not None else None)
    _check(rc, "glisse_batch_create")
    return h


def glisse_batch_advance(h, n_steps: int):
    _check(load().glisse_batch_advance(h, int(n_steps)), "glisse_batch_advance")


def glisse_batch_read(h, n: int, out=None):
    """Returns dict(state [n][6], alive [n] bool, removal_step [n], removal_reason [n]) in the
    batch's particle order.  out: optional dict of preallocated host arrays (as for glisse_read,
    e.g. in pinned memory), written in place."""
    if out is not None:
        st, alive, steps, rsn = out["state"], out["alive"], out["removal_step"], out["removal_reason"]
        assert st.shape == (n, 6) and st.dtype == np.float64 and st.flags.c_contiguous
        assert alive.shape == (n,) and alive.dtype == np.uint8 and steps.dtype == np.int64
        assert rsn.dtype == np.int32
    else:
        st = np.empty((n, 6))
        alive = np.empty(n, dtype=np.uint8)
        steps = np.empty(n, dtype=np.int64)
        rsn = np.empty(n, dtype=np.int32)
    rc = load().glisse_batch_read(h, _dp(st), alive.ctypes.data_as(C.POINTER(C.c_uint8)),
                                  steps.ctypes.data_as(C.POINTER(C.c_int64)),
                                  rsn.ctypes.data_as(C.POINTER(C.c_int32)))
    _check(rc, "glisse_batch_read")
    return {"state": st, "alive": alive.astype(bool), "removal_step": steps, "removal_reason": rsn}


def glisse_batch_status(h):
    nl, st = C.c_int64(), C.c_int64()
    _check(load().glisse_batch_status(h, C.byref(nl), C.byref(st)), "glisse_batch_status")
    return nl.value, st.value


def glisse_batch_steps_done(h) -> int:
    v = C.c_int64()
    _check(load().glisse_batch_steps_done(h, C.byref(v)), "glisse_batch_steps_done")
    return v.value


def glisse_batch_timings(h, reset: bool = False) -> dict:
    t = glisse_timing()
    _check(load().glisse_batch_timings(h, C.byref(t), 1 if reset else 0), "glisse_batch_timings")
    return {name: getattr(t, name) for name, _ in glisse_timing._fields_}


def glisse_batch_tune(h, trial_steps: int = 256):
    """(chunk steps, block threads, threads per particle) chosen by the autotuner."""
    c, t, p = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().glisse_batch_tune(h, int(trial_steps), C.byref(c), C.byref(t), C.byref(p)), "glisse_batch_tune")
    return c.value, t.value, p.value


def glisse_batch_set_launch(h, block_threads: int, threads_per_particle: int = 1):
    _check(load().glisse_batch_set_launch(h, int(block_threads), int(threads_per_particle)), "glisse_batch_set_launch")


def glisse_batch_destroy(h):
    if h:
        load().glisse_batch_destroy(h)


class BatchSimulation:
    """Owner of a batch of independent systems (same calls, Python lifetime)."""

    def __init__(self, star_mass, n_planets, planets, n_particles, particles, dt, **opt):
        o = glisse_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        self.n = int(np.sum(n_particles))
        self.h = None
        self.h = glisse_batch_create(star_mass, n_planets, planets, n_particles, particles, dt, o)

    def advance(self, n_steps):
        glisse_batch_advance(self.h, n_steps)
        return self

    def read(self, out=None):
        return glisse_batch_read(self.h, self.n, out)

    def status(self):
        return glisse_batch_status(self.h)

    def timings(self, reset=False):
        return glisse_batch_timings(self.h, reset)

    def steps_done(self):
        """Particle-steps advanced since creation over all systems (exact)."""
        return glisse_batch_steps_done(self.h)

    def tune(self, trial_steps=256):
        return glisse_batch_tune(self.h, trial_steps)

    def set_launch(self, block_threads, threads_per_particle=1):
        glisse_batch_set_launch(self.h, block_threads, threads_per_particle)

    def checkpoint(self) -> np.ndarray:
        """Everything needed to go on exactly from here (see BatchSimulation.resume)."""
        return glisse_batch_checkpoint(self.h)

    @classmethod
    def resume(cls, buf, **opt):
        """A BatchSimulation continuing from a checkpoint; opt may set cuda_stream and timing."""
        o = glisse_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        self = cls.__new__(cls)
        self.h = None
        b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray))
                                 else buf, dtype=np.uint8)
        self.h = glisse_batch_resume(b, o)
        self.n = glisse_batch_sizes(self.h)[0]
        return self

    def close(self):
        if self.h:
            glisse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Convenience owner of a context (same calls, Python lifetime)."""

    def __init__(self, star_mass, planets, particles, dt, **opt):
        o = glisse_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        self.n = int(np.asarray(particles).reshape(-1, 6).shape[0])
        self.n_planets = int(np.asarray(planets).reshape(-1, 7).shape[0])
        self.h = None
        self.h = glisse_create(star_mass, planets, particles, dt, o)

    def advance(self, n_steps):
        glisse_advance(self.h, n_steps)
        return self

    def read(self, out=None):
        return glisse_read(self.h, self.n, out)

    def status(self):
        return glisse_status(self.h)

    def planets(self):
        return glisse_read_planets(self.h, self.n_planets)

    def set_ephemeris(self, log):
        glisse_set_ephemeris(self.h, log)

    def checkpoint(self) -> np.ndarray:
        """Everything needed to go on exactly from here (see Simulation.resume)."""
        return glisse_checkpoint(self.h)

    @classmethod
    def resume(cls, buf, **opt):
        """A Simulation continuing from a checkpoint; opt may set cuda_stream and timing."""
        o = glisse_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        self = cls.__new__(cls)
        self.h = None
        self.h = glisse_resume(buf, o)
        self.n, self.n_planets = glisse_sizes(self.h)
        return self

    def timings(self, reset=False):
        return glisse_timings(self.h, reset)

    def set_sampling(self, every=None, **kw):
        self.max_samples = int(kw.get("max_samples", 0)) if every is not None else 0
        glisse_set_sampling(self.h, every, **kw)

    def elements(self, max_samples=None):
        """(elements [k][n][6], sample steps [k]) of the kept samples; max_samples bounds k (default:
        the max_samples given to set_sampling on this object; pass it for a resumed context)."""
        k = getattr(self, "max_samples", 0) if max_samples is None else int(max_samples)
        return glisse_read_elements(self.h, self.n, k)

    def libration(self):
        return glisse_read_libration(self.h, self.n)

    def close(self):
        if self.h:
            glisse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Derivatives of the map (device arrays are torch CUDA float64 tensors)
# ---------------------------------------------------------------------------
def glisse_diff_create(star_mass, planets, n_particles, dt, n_steps, checkpoint_every=256, opts=None):
    L = load()
    pl = np.ascontiguousarray(planets, dtype=np.float64).reshape(-1, 7)
    h = C.c_void_p()
    rc = L.glisse_diff_create(C.byref(h), float(star_mass), _dp(pl) if pl.size else None, pl.shape[0],
                              int(n_particles), float(dt), int(n_steps), int(checkpoint_every),
                              C.byref(opts) if opts is not None else None)
    _check(rc, "glisse_diff_create")
    return h


def glisse_diff_checkpoint_every(h) -> int:
    """Checkpoint interval in effect (0: tape mode)."""
    k = C.c_int32()
    _check(load().glisse_diff_checkpoint_every(h, C.byref(k)), "glisse_diff_checkpoint_every")
    return int(k.value)


def glisse_diff_forward(h, state0, state1, tangent0=None, tangent1=None, log_growth=None, removal_step=None,
                        removal_reason=None, stream=0):
    """All arguments after h are device addresses (ints) or None; see include/glisse.h."""
    T = 0 if tangent0 is None else tangent0[1]
    rc = load().glisse_diff_forward(h, state0, state1, T, None if tangent0 is None else tangent0[0],
                                    tangent1, log_growth, removal_step, removal_reason, stream)
    _check(rc, "glisse_diff_forward")


def glisse_diff_backward(h, grad_state1, grad_state0, stream=0):
    _check(load().glisse_diff_backward(h, grad_state1, grad_state0, stream), "glisse_diff_backward")


def glisse_diff_backward_growth(h, grad_state1, grad_growth, tangent1, grad_state0, grad_tangent0, stream=0):
    _check(load().glisse_diff_backward_growth(h, grad_state1, grad_growth, tangent1, grad_state0, grad_tangent0,
                                              stream), "glisse_diff_backward_growth")


def glisse_diff_growth_gradient(h, state0, tangent0, grad_state0, log_growth=None, stream=0):
    _check(load().glisse_diff_growth_gradient(h, state0, tangent0, grad_state0, log_growth, stream),
           "glisse_diff_growth_gradient")


def glisse_diff_destroy(h):
    if h:
        load().glisse_diff_destroy(h)


class DiffMap:
    """Differentiable run of the map over a fixed number of steps for n particles.

    forward(state0 [n, 6]) -> state1 [n, 6] (plus tangents J t and a growth
    indicator); backward(g [n, 6]) -> J^T g for the last forward call.  Both run
    in the library's kernels; tensors must be CUDA float64 and contiguous.

    checkpoint_every: K >= 1 stores the state every K steps and recomputes each
    segment in the backward pass; 0 (tape) records every step in the forward
    pass ((112 + 16 N_p) B per particle-step) so the backward pass is the reverse
    sweep alone (about half the cost); GLISSE_DIFF_AUTO takes the tape when it
    fits in half of the free device memory.  The reverse sweep for the growth
    indicator's gradient needs checkpoints, or GLISSE_DIFF_TAPE_TANGENT: a tape
    that also keeps tangent 0 ((184 + 16 N_p) B per particle-step), after which
    that sweep recomputes nothing either.  The default stays K = 256."""

    def __init__(self, star_mass, planets, n_particles, dt, n_steps, checkpoint_every=256, **opt):
        o = glisse_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        self.n = int(n_particles)
        self.h = None
        self.h = glisse_diff_create(star_mass, planets, n_particles, dt, n_steps, checkpoint_every, o)
        self.checkpoint_every = glisse_diff_checkpoint_every(self.h)  # GLISSE_DIFF_AUTO resolved
        self.tape = self.checkpoint_every in (0, GLISSE_DIFF_TAPE_TANGENT)
        # the growth gradient's reverse sweep needs checkpoints or a record that keeps tangent 0
        self.reverse_growth = self.checkpoint_every != 0
        self.forward_calls = 0

    @staticmethod
    def _ptr(t):
        return None if t is None else t.data_ptr()

    def forward(self, state0, tangents=None):
        import torch

        state0 = state0.contiguous()
        assert state0.is_cuda and state0.dtype == torch.float64 and state0.shape == (self.n, 6)
        state1 = torch.empty_like(state0)
        growth = torch.empty(self.n, dtype=torch.float64, device=state0.device)
        rstep = torch.empty(self.n, dtype=torch.int64, device=state0.device)
        reason = torch.empty(self.n, dtype=torch.int32, device=state0.device)
        tan1 = None
        tan0 = None
        if tangents is not None:
            tangents = tangents.contiguous()
            assert tangents.dim() == 3 and tangents.shape[1:] == (self.n, 6)
            tan1 = torch.empty_like(tangents)
            tan0 = (tangents.data_ptr(), tangents.shape[0])
        stream = torch.cuda.current_stream(state0.device).cuda_stream
        glisse_diff_forward(self.h, state0.data_ptr(), state1.data_ptr(), tan0, self._ptr(tan1),
                            growth.data_ptr() if tangents is not None else None, rstep.data_ptr(),
                            reason.data_ptr(), stream)
        self.forward_calls += 1
        return state1, tan1, (growth if tangents is not None else None), rstep, reason

    def backward(self, grad_state1):
        import torch

        g = grad_state1.contiguous()
        out = torch.empty_like(g)
        stream = torch.cuda.current_stream(g.device).cuda_stream
        glisse_diff_backward(self.h, g.data_ptr(), out.data_ptr(), stream)
        return out

    def backward_growth(self, grad_state1, grad_growth, tangent1):
        """One reverse sweep for the last forward call (which carried tangent 0 = t0):
        (J^T grad_state1 + grad_growth dg/dstate0, grad_growth dg/dt0) for
        g = log(|J t0| / |t0|); tangent1 = J t0 from that call [n, 6].  Needs
        checkpoints or GLISSE_DIFF_TAPE_TANGENT (not the plain tape).
        grad_state1 / grad_growth may be None."""
        import torch

        t1 = tangent1.contiguous()
        g1 = None if grad_state1 is None else grad_state1.contiguous()
        gg = None if grad_growth is None else grad_growth.contiguous()
        gs0 = torch.empty_like(t1)
        gt0 = torch.empty_like(t1)
        stream = torch.cuda.current_stream(t1.device).cuda_stream
        glisse_diff_backward_growth(self.h, self._ptr(g1), self._ptr(gg), t1.data_ptr(), gs0.data_ptr(),
                                    gt0.data_ptr(), stream)
        return gs0, gt0

    def growth_gradient(self, state0, tangent0):
        """(d g / d state0 [n, 6] with the seed held fixed, g [n]) for
        g = log(|J t0| / |t0|); independent of forward()."""
        import torch

        state0 = state0.contiguous()
        tangent0 = tangent0.contiguous()
        assert state0.is_cuda and state0.dtype == torch.float64 and state0.shape == (self.n, 6)
        assert tangent0.shape == (self.n, 6) and tangent0.dtype == torch.float64
        grad = torch.empty_like(state0)
        growth = torch.empty(self.n, dtype=torch.float64, device=state0.device)
        stream = torch.cuda.current_stream(state0.device).cuda_stream
        glisse_diff_growth_gradient(self.h, state0.data_ptr(), tangent0.data_ptr(), grad.data_ptr(),
                                    growth.data_ptr(), stream)
        return grad, growth

    def close(self):
        if self.h:
            glisse_diff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _growth_seed(state0):
    """Default tangent for the growth indicator: unit vectors along r and along v."""
    import torch

    r = state0[:, :3] / state0[:, :3].norm(dim=1, keepdim=True)
    v = state0[:, 3:] / state0[:, 3:].norm(dim=1, keepdim=True)
    return (torch.cat([r, v], dim=1) / 2**0.5).unsqueeze(0)


def _make_autograd():
    import torch

    class GlisseMap(torch.autograd.Function):
        """state1, log_growth = GlisseMap.apply(state0, diff_map[, tangent0]).

        Both outputs are differentiable with respect to state0 (and tangent0).
        log_growth = log(|J t0| / |t0|) for the seed tangent0 [n, 6], by default
        unit vectors along r and v (_growth_seed, whose own dependence on state0
        is included).  Gradients: with checkpoints, one reverse sweep of the map
        extended by its tangent (glisse_diff_backward_growth) gives both parts;
        without the growth, or in tape mode, J^T from the adjoint kernel
        (glisse_diff_backward), the growth's gradient at fixed seed from the
        forward-mode second-order kernel (glisse_diff_growth_gradient), and with
        respect to the seed J^T (J t0) / |J t0|^2 - t0 / |t0|^2 from the adjoint."""

        @staticmethod
        def forward(ctx, state0, dmap, *rest):
            tangent0 = rest[0] if rest else None
            ctx.n_inputs = 2 + len(rest)
            ctx.default_seed = tangent0 is None
            seed = _growth_seed(state0.detach())[0] if tangent0 is None else tangent0.detach()
            state1, tan1, growth, _, _ = dmap.forward(state0.detach(), seed.unsqueeze(0).contiguous())
            ctx.dmap = dmap
            ctx.call = dmap.forward_calls
            ctx.save_for_backward(state0.detach(), seed, tan1[0])
            return state1, growth

        @staticmethod
        def backward(ctx, grad_state1, grad_growth):
            if ctx.dmap.forward_calls != ctx.call:
                raise RuntimeError("DiffMap was run forward again before this backward; use one DiffMap per use")
            state0, seed, tn = ctx.saved_tensors
            g1 = torch.zeros_like(state0) if grad_state1 is None else grad_state1
            grad_seed = None
            has_growth = grad_growth is not None and bool((grad_growth != 0).any())
            if has_growth and ctx.dmap.reverse_growth:
                # one reverse sweep of the map extended by its tangent
                grad_state0, grad_seed = ctx.dmap.backward_growth(g1, grad_growth, tn)
                if ctx.default_seed:
                    with torch.enable_grad():
                        s0 = state0.clone().requires_grad_(True)
                        (gs,) = torch.autograd.grad(_growth_seed(s0)[0], s0, grad_seed)
                    grad_state0 = grad_state0 + gs
                    grad_seed = None
                return (grad_state0, None, grad_seed)[: ctx.n_inputs]
            grad_state0 = ctx.dmap.backward(g1)
            if has_growth:
                gg = grad_growth.unsqueeze(1)
                H, _ = ctx.dmap.growth_gradient(state0, seed)
                grad_state0 = grad_state0 + gg * H
                if ctx.default_seed or ctx.needs_input_grad[2]:
                    nn = (tn * tn).sum(dim=1, keepdim=True)
                    u = torch.where(nn > 0, tn / torch.where(nn > 0, nn, torch.ones_like(nn)), torch.zeros_like(tn))
                    n0 = (seed * seed).sum(dim=1, keepdim=True)
                    grad_seed = ctx.dmap.backward((gg * u).contiguous()) - gg * seed / n0
                if ctx.default_seed and grad_seed is not None:
                    with torch.enable_grad():
                        s0 = state0.clone().requires_grad_(True)
                        (gs,) = torch.autograd.grad(_growth_seed(s0)[0], s0, grad_seed)
                    grad_state0 = grad_state0 + gs
                    grad_seed = None
            return (grad_state0, None, grad_seed)[: ctx.n_inputs]

    return GlisseMap


_glisse_map_cls = None


def glisse_map():
    """The torch.autograd.Function of the differentiable map (created on first use)."""
    global _glisse_map_cls
    if _glisse_map_cls is None:
        _glisse_map_cls = _make_autograd()
    return _glisse_map_cls
