"""Python binding of the plain FP64 CPU oracle (``glisse_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline / reference leg may import this module.  The product
path (the CUDA library and its binding) never imports, links or calls it.

``build()`` compiles the C file with gcc (no FMA contraction, no fast-math,
OpenMP over particles) into ``oracle/_build/liboracle.so``.

Every function here is pinned to something other than itself: closed forms,
exact two-body motion, reversibility, the Jacobi constant, convergence
against an N-body integration and the paper's statements
(tests/test_oracle_pins.py, planted mistakes in tests/test_oracle_mutants.py);
the tangent map (tests/test_oracle_tangent.py); the growth gradient
(tests/test_oracle_growth.py); the fixed-iteration solve
(tests/test_oracle_paper_mode.py); elements and the libration test
(tests/test_oracle_elements.py); the integrated map, elements and libration
test together against the resonance locations, the 3:1 resonance and the
solver range that the paper prints (tests/golden/paper_values.txt,
tests/test_oracle_golden.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glisse_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ALIVE, ESCAPE, KEPLER, NONFINITE = 0, -1, -2, -3

# convergence required of the paper's fixed-iteration Kepler solve (section 2.2)
PAPER_KEPLER_TOL = 1e-14


CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC"]


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into a shared object (used by build() and the mutant tests)."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or older than the source
    (and its op-counting build, opcount.cpp)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        compile_source(_SRC, _OUT)
    build_opcount(force)
    return _OUT


_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_OUT = os.path.join(_HERE, "_build", "libopcount.so")


def build_opcount(force: bool = False) -> str:
    """Compile opcount.cpp (the oracle's particle map over a counting double) with g++,
    the same floating-point flags as the oracle, single-threaded."""
    os.makedirs(os.path.dirname(_OPC_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_OPC_SRC), os.path.getmtime(_SRC))
    if force or not os.path.exists(_OPC_OUT) or os.path.getmtime(_OPC_OUT) < newest:
        tmp = _OPC_OUT + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-shared", "-fPIC",
                        "-o", tmp, _OPC_SRC, "-lm"], check=True)
        os.replace(tmp, _OPC_OUT)
    return _OPC_OUT


OPCOUNT_FIELDS = ("add", "mul", "div", "sqrt", "trans", "cmp", "other")


def opcount_particles(star_mass, planet_masses, log, dt, state0, rcrit_, r_max):
    """The particle map of ParticleRun.advance over log (test at t_0 first), run through the
    op-counting build.  Returns (final state [n][6], removal_step, reason, counts dict with
    OPCOUNT_FIELDS over the whole run)."""
    L = C.CDLL(build_opcount())
    dp = C.POINTER(C.c_double)
    L.orc_opcount_particles.argtypes = [C.c_double, C.c_int, dp, dp, C.c_int64, C.c_double, dp, C.c_double, dp,
                                        C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_uint64)]
    L.orc_opcount_particles.restype = C.c_int
    pm = _f64(planet_masses)
    log = _f64(log)
    st = _f64(state0).reshape(-1, 6).copy()
    n = st.shape[0]
    rs = np.empty(n, dtype=np.int64)
    rn = np.empty(n, dtype=np.int32)
    cnt = np.zeros(len(OPCOUNT_FIELDS), dtype=np.uint64)
    rc = L.orc_opcount_particles(float(star_mass), pm.shape[0], _dp(pm), _dp(log), log.shape[0] - 1, float(dt),
                                 _dp(_f64(rcrit_)), float(r_max), _dp(st), n,
                                 rs.ctypes.data_as(C.POINTER(C.c_int64)), rn.ctypes.data_as(C.POINTER(C.c_int32)),
                                 cnt.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc != 0:
        raise RuntimeError(f"orc_opcount_particles failed: {rc}")
    return st, rs, rn, dict(zip(OPCOUNT_FIELDS, (int(c) for c in cnt)))


SOURCE = _SRC


_override = []


class using:
    """Context manager: route this module's calls to another build of the oracle
    (tests use it to check that the pins catch planted mistakes)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        _override.append(_bind(C.CDLL(self.path)))
        return self

    def __exit__(self, *exc):
        _override.pop()
        return False


def lib():
    global _lib
    if _override:
        return _override[-1]
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L):
    """Declare the C signatures on a loaded oracle library."""
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    i32p = C.POINTER(C.c_int32)
    L.orc_G.restype = C.c_double
    L.orc_kepler_drift.argtypes = [C.c_double, C.c_double, dp]
    L.orc_kepler_drift.restype = C.c_int
    L.orc_last_iters.restype = C.c_int
    L.orc_planet_wh.argtypes = [C.c_double, C.c_int, dp, C.c_double, C.c_int64, dp, dp]
    L.orc_planet_wh.restype = C.c_int
    L.orc_rcrit.argtypes = [C.c_double, C.c_int, dp, C.c_int, C.c_double, dp]
    L.orc_rcrit.restype = C.c_int
    L.orc_particles.argtypes = [C.c_double, C.c_int, dp, dp, C.c_int64, C.c_double, dp, C.c_double, dp,
                                C.c_int64, i64p, i32p, dp, dp, C.c_int64, C.c_int, C.c_int]
    L.orc_particles.restype = C.c_int
    L.orc_kepler_drift_fixed.argtypes = [C.c_double, C.c_double, dp, C.c_int, C.c_double, dp]
    L.orc_kepler_drift_fixed.restype = C.c_int
    L.orc_particles_ex.argtypes = [C.c_double, C.c_int, dp, dp, C.c_int64, C.c_double, dp, C.c_double, dp,
                                   C.c_int64, i64p, i32p, dp, dp, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_double,
                                   dp]
    L.orc_particles_ex.restype = C.c_int
    u8p = C.POINTER(C.c_uint8)
    L.orc_elements.argtypes = [C.c_double, dp, dp]
    L.orc_elements.restype = C.c_int
    L.orc_barycentre.argtypes = [C.c_double, C.c_int, dp, dp, dp]
    L.orc_barycentre.restype = None
    L.orc_sample.argtypes = [C.c_double, C.c_int, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, u8p,
                             C.c_int64, dp, dp, u8p, u8p, i32p]
    L.orc_sample.restype = C.c_int
    L.orc_max_threads.restype = C.c_int
    L.orc_particles_jvp.argtypes = [C.c_double, C.c_int, dp, dp, C.c_int64, C.c_double, dp, C.c_double, dp, dp,
                                    C.c_int64, dp, dp, i64p, i32p, C.c_int, C.c_int]
    L.orc_particles_jvp.restype = C.c_int
    return L



def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a



def grav():
    return lib().orc_G()


def kepler_drift(mu: float, state, dt: float):
    """Drift one heliocentric state [6] by dt about mu. Returns (new_state, status, newton_iters)."""
    st = _f64(state, (6,)).copy()
    rc = lib().orc_kepler_drift(float(mu), float(dt), _dp(st))
    return st, rc, lib().orc_last_iters()


def kepler_drift_fixed(mu: float, state, dt: float, iters: int = 5, tol: float = PAPER_KEPLER_TOL):
    """The paper's fixed-iteration drift. Returns (new_state, status, |last Newton step|)."""
    st = _f64(state, (6,)).copy()
    ldx = C.c_double()
    rc = lib().orc_kepler_drift_fixed(float(mu), float(dt), _dp(st), int(iters), float(tol), C.byref(ldx))
    return st, rc, ldx.value


def planet_wh(star_mass: float, planets, dt: float, n_steps: int, want_log: bool = True, want_energy: bool = False):
    """Advance the planets n_steps.  Returns (planets_out [np][7], log [n+1][np][3] or None, energy or None)."""
    pl = _f64(planets).copy()
    np_ = pl.shape[0]
    log = np.empty((n_steps + 1, np_, 3)) if want_log else None
    en = np.empty(n_steps + 1) if want_energy else None
    rc = lib().orc_planet_wh(float(star_mass), np_, _dp(pl), float(dt), int(n_steps),
                             _dp(log) if log is not None else None, _dp(en) if en is not None else None)
    if rc != 0:
        raise RuntimeError(f"orc_planet_wh failed: {rc}")
    return pl, log, en


def rcrit(star_mass: float, planets, mode: int = 0, value: float = 1.0):
    pl = _f64(planets)
    out = np.empty(pl.shape[0])
    rc = lib().orc_rcrit(float(star_mass), pl.shape[0], _dp(pl), int(mode), float(value), _dp(out))
    if rc != 0:
        raise ValueError("unbound planet")
    return out


class ParticleRun:
    """State of an oracle particle integration that can be advanced in pieces."""

    def __init__(self, star_mass, planet_masses, state, rcrit_, r_max, kepler_iters=0,
                 kepler_tol=PAPER_KEPLER_TOL):
        """kepler_iters > 0 selects the paper's fixed-iteration Kepler solve with that many
        Newton steps (kepler_dx then records the largest |last step| seen per particle)."""
        self.m0 = float(star_mass)
        self.pm = _f64(planet_masses).copy()
        self.state = _f64(state).reshape(-1, 6).copy()
        n = self.state.shape[0]
        self.removal_step = np.full(n, -1, dtype=np.int64)
        self.reason = np.zeros(n, dtype=np.int32)
        self.margin = np.full(n, np.inf)
        self.closest = np.full(n, np.inf)
        self.rcrit = _f64(rcrit_).copy()
        self.r_max = float(r_max)
        self.step = 0
        self.tested_first = False
        self.kepler_iters = int(kepler_iters)
        self.kepler_tol = float(kepler_tol)
        self.kepler_dx = np.zeros(n)

    def advance(self, log, dt: float, nthreads: int = 0):
        """Advance by len(log)-1 steps using planet positions log[0..n] (log[0] at the current step)."""
        log = _f64(log)
        n = log.shape[0] - 1
        npl = self.pm.shape[0]
        rc = lib().orc_particles_ex(self.m0, npl, _dp(self.pm), _dp(log), int(n), float(dt), _dp(self.rcrit),
                                    self.r_max, _dp(self.state), self.state.shape[0],
                                    self.removal_step.ctypes.data_as(C.POINTER(C.c_int64)),
                                    self.reason.ctypes.data_as(C.POINTER(C.c_int32)), _dp(self.margin),
                                    _dp(self.closest), int(self.step), 0 if self.tested_first else 1, int(nthreads),
                                    self.kepler_iters, self.kepler_tol, _dp(self.kepler_dx))
        if rc != 0:
            raise RuntimeError(f"orc_particles_ex failed: {rc}")
        self.tested_first = True
        self.step += n
        return self


def run(star_mass, planets, particles, dt, n_steps, k_hill=1.0, r_max=1000.0, enc_mode=0, nthreads=0,
        kepler_iters=0):
    """Whole-run convenience: planets and particles from a heliocentric start.

    Returns a dict with the final particle state [n][6], removal_step, reason, margin, closest,
    kepler_dx (fixed-iteration mode only), the planet log [n+1][np][3] and the final planets [np][7]."""
    pl0 = _f64(planets)
    rc_ = rcrit(star_mass, pl0, enc_mode, k_hill)
    pl1, log, _ = planet_wh(star_mass, pl0, dt, n_steps)
    pr = ParticleRun(star_mass, pl0[:, 0], particles, rc_, r_max, kepler_iters=kepler_iters)
    pr.advance(log, dt, nthreads)
    return {"state": pr.state, "removal_step": pr.removal_step, "reason": pr.reason, "margin": pr.margin,
            "closest": pr.closest, "kepler_dx": pr.kepler_dx, "log": log, "planets": pl1, "rcrit": rc_}


def particles_jvp(star_mass, planet_masses, log, dt, state0, direction, rcrit_, r_max, test_first=True,
                  nthreads=0):
    """Tangent map by complex step: (final state [n][6], J @ direction [n][6], removal_step, reason)."""
    pm = _f64(planet_masses)
    log = _f64(log)
    s0 = _f64(state0).reshape(-1, 6)
    dr = _f64(direction).reshape(-1, 6)
    n = s0.shape[0]
    s1 = np.empty_like(s0)
    jv = np.empty_like(s0)
    rs = np.empty(n, dtype=np.int64)
    rn = np.empty(n, dtype=np.int32)
    rc = lib().orc_particles_jvp(float(star_mass), pm.shape[0], _dp(pm), _dp(log), log.shape[0] - 1, float(dt),
                                 _dp(_f64(rcrit_)), float(r_max), _dp(s0), _dp(dr), n, _dp(s1), _dp(jv),
                                 rs.ctypes.data_as(C.POINTER(C.c_int64)), rn.ctypes.data_as(C.POINTER(C.c_int32)),
                                 1 if test_first else 0, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_particles_jvp failed: {rc}")
    return s1, jv, rs, rn


def growth(star_mass, planet_masses, log, dt, state0, tangent0, rcrit_, r_max, nthreads=0):
    """Tangent-growth indicator g = log(|J t0| / |t0|) per particle, J t0 from the
    complex-step tangent map; also the removal steps of that run."""
    t0 = _f64(tangent0).reshape(-1, 6)
    _, jv, rs, _ = particles_jvp(star_mass, planet_masses, log, dt, state0, t0, rcrit_, r_max, nthreads=nthreads)
    return 0.5 * np.log((jv * jv).sum(axis=1) / (t0 * t0).sum(axis=1)), rs


def growth_gradient(star_mass, planet_masses, log, dt, state0, tangent0, rcrit_, r_max, h_pos=1e-5, h_vel=1e-6,
                    nthreads=0):
    """d g / d state0 [n][6] at fixed tangent0, by central differences of growth()
    with steps h and h/2 per coordinate (h_pos AU for positions, h_vel AU/yr for
    velocities) combined by Richardson extrapolation, (4 D(h/2) - D(h)) / 3.

    Returns (gradient, error estimate |R - D(h/2)| per entry, ok [n]); ok is False
    for particles whose removal step differs between the perturbed runs (there
    the difference quotient is not a derivative)."""
    s0 = _f64(state0).reshape(-1, 6)
    n = s0.shape[0]
    _, rs0 = growth(star_mass, planet_masses, log, dt, s0, tangent0, rcrit_, r_max, nthreads)
    ok = np.ones(n, dtype=bool)
    grad = np.empty((n, 6))
    err = np.empty((n, 6))
    for c in range(6):
        h = h_pos if c < 3 else h_vel
        d = []
        for hh in (h, 0.5 * h):
            e = np.zeros_like(s0)
            e[:, c] = hh
            gp, rp = growth(star_mass, planet_masses, log, dt, s0 + e, tangent0, rcrit_, r_max, nthreads)
            gm, rm = growth(star_mass, planet_masses, log, dt, s0 - e, tangent0, rcrit_, r_max, nthreads)
            ok &= (rp == rs0) & (rm == rs0)
            d.append((gp - gm) / (2.0 * hh))
        grad[:, c] = (4.0 * d[1] - d[0]) / 3.0
        err[:, c] = np.abs(grad[:, c] - d[1])
    return grad, err, ok


def particles_jacobian(star_mass, planet_masses, log, dt, state0, rcrit_, r_max, nthreads=0):
    """Full 6x6 Jacobian per particle [n][6][6] (column c = derivative along input coordinate c)."""
    s0 = _f64(state0).reshape(-1, 6)
    n = s0.shape[0]
    J = np.empty((n, 6, 6))
    for c in range(6):
        e = np.zeros_like(s0)
        e[:, c] = 1.0
        _, jv, _, _ = particles_jvp(star_mass, planet_masses, log, dt, s0, e, rcrit_, r_max, nthreads=nthreads)
        J[:, :, c] = jv
    return J


def elements(mu: float, states):
    """Osculating elements [n][6] (a, e, i, Omega, omega, M) of states [n][6] about mu."""
    st = _f64(states).reshape(-1, 6)
    out = np.empty_like(st)
    for p in range(st.shape[0]):
        row = np.ascontiguousarray(st[p])
        el = np.empty(6)
        if lib().orc_elements(float(mu), _dp(row), _dp(el)) != 0:
            el[:] = np.nan
        out[p] = el
    return out


def barycentre(star_mass, planet_masses, planet_states):
    """Heliocentric state [6] of the barycentre of the star and planets ([np][6] heliocentric states)."""
    pm = _f64(planet_masses).reshape(-1)
    pl = _f64(planet_states).reshape(-1, 6)
    R = np.empty(6)
    lib().orc_barycentre(float(star_mass), pm.shape[0], _dp(pm), _dp(pl), _dp(R))
    return R


def run_sampled(star_mass, planets, particles, dt, n_steps, every, frame=1, res_planet=-1, res_p=0, res_q=0,
                avoid_deg=10.0, k_hill=1.0, r_max=1000.0, nthreads=0):
    """run() with an element sample every `every` steps (at steps every, 2 every, ... <= n_steps).

    Returns the run() dict plus elements [n_samples][n][6] (NaN rows for particles not live at the
    sample), sample_steps, phi [n_samples][n] (NaN where not used), near0, near180, count."""
    pl = _f64(planets).copy()
    pa = _f64(particles).reshape(-1, 6)
    n = pa.shape[0]
    pm = np.ascontiguousarray(pl[:, 0])
    rc_ = rcrit(star_mass, pl, 0, k_hill)
    pr = ParticleRun(star_mass, pm, pa, rc_, r_max)
    near0 = np.zeros(n, dtype=np.uint8)
    near180 = np.zeros(n, dtype=np.uint8)
    count = np.zeros(n, dtype=np.int32)
    elems, phis, steps, logs = [], [], [], []
    done = 0
    while done < n_steps:
        m = min(every - done % every, n_steps - done)
        pl, log, _ = planet_wh(star_mass, pl, dt, m)
        logs.append(log if not logs else log[1:])
        pr.advance(log, dt, nthreads)
        done += m
        if done % every == 0:
            live = (pr.removal_step < 0).astype(np.uint8)
            el = np.empty((n, 6))
            ph = np.empty(n)
            hel = np.ascontiguousarray(pl[:, 1:])
            rc = lib().orc_sample(float(star_mass), pl.shape[0], _dp(pm), _dp(hel), int(frame), int(res_planet),
                                  int(res_p), int(res_q), float(np.radians(avoid_deg)), _dp(pr.state),
                                  live.ctypes.data_as(C.POINTER(C.c_uint8)), n, _dp(el), _dp(ph),
                                  near0.ctypes.data_as(C.POINTER(C.c_uint8)),
                                  near180.ctypes.data_as(C.POINTER(C.c_uint8)),
                                  count.ctypes.data_as(C.POINTER(C.c_int32)))
            if rc != 0:
                raise RuntimeError(f"orc_sample failed: {rc}")
            elems.append(el)
            phis.append(ph)
            steps.append(done)
    return {"state": pr.state, "removal_step": pr.removal_step, "reason": pr.reason, "margin": pr.margin,
            "closest": pr.closest, "planets": pl, "log": np.concatenate(logs) if logs else None,
            "elements": np.array(elems).reshape(-1, n, 6), "phi": np.array(phis).reshape(-1, n),
            "sample_steps": np.array(steps, dtype=np.int64), "near0": near0, "near180": near180, "count": count}


def max_threads() -> int:
    return lib().orc_max_threads()
