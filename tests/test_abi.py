"""The C-ABI library builds, loads and exports every declared entry point (no GPU needed).

Only calls that do not reach the GPU are made here: option defaults, status
strings and argument validation, which happens before any CUDA call.
"""
import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "glisse.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(glisse_\w+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def G():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2011_03484_gb300 as G

    G._build.build()
    return G


def test_library_exports_every_declared_symbol(G):
    L = C.CDLL(G.library_path())
    names = _declared()
    assert names, "no declarations found"
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(G.EXPORTED) == names


def test_opts_defaults(G):
    o = G.glisse_opts_default()
    assert o.chunk_steps == 1024 and o.resync_chunks == 1
    assert o.kepler_mode == G.GLISSE_KEPLER_CONVERGE and o.kepler_iters == 5
    assert o.enc_mode == G.GLISSE_ENC_HILL and o.enc_value == 1.0 and o.r_max == 1000.0
    assert o.sort_mode == G.GLISSE_SORT_NONE and o.timing == 0
    assert o.launch_mode == G.GLISSE_LAUNCH_AUTO


def test_strerror_names_every_code(G):
    for code in range(0, -7, -1):
        s = G.strerror(code)
        assert s and "unknown" not in s
    assert "unknown" in G.strerror(-99)


def test_argument_errors_before_any_cuda_call(G):
    import glisse_inputs as gi

    w = gi.make("tiny", n=4)
    bad = [
        dict(star_mass=0.0),
        dict(star_mass=float("nan")),
        dict(dt=0.0),
        dict(dt=float("inf")),
        dict(planets=np.zeros((9, 7))),  # more than GLISSE_MAX_PLANETS
        dict(planets=np.vstack([w["planets"][:1] * [[-1, 1, 1, 1, 1, 1, 1]]])),  # negative mass
        dict(planets=np.where(np.arange(7) == 2, np.nan, w["planets"])),
    ]
    for kw in bad:
        args = dict(star_mass=1.0, planets=w["planets"], particles=w["particles"], dt=0.5)
        args.update(kw)
        with pytest.raises(G.GlisseError) as ei:
            G.glisse_create(**args)
        assert ei.value.code == G.GLISSE_E_INVAL, kw
    o = G.glisse_opts_default()
    o.chunk_steps = 0
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_create(1.0, w["planets"], w["particles"], 0.5, o)
    assert ei.value.code == G.GLISSE_E_INVAL
    # Kepler modes: unknown mode, iteration counts outside 1..GLISSE_MAX_KEPLER_ITERS
    for mode, iters in ((7, 5), (G.GLISSE_KEPLER_PAPER_FIXED, 0), (G.GLISSE_KEPLER_PAPER_FIXED, 65)):
        o = G.glisse_opts_default()
        o.kepler_mode, o.kepler_iters = mode, iters
        with pytest.raises(G.GlisseError) as ei:
            G.glisse_create(1.0, w["planets"], w["particles"], 0.5, o)
        assert ei.value.code == G.GLISSE_E_INVAL, (mode, iters)
    o = G.glisse_opts_default()
    o.sort_mode = 2
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_create(1.0, w["planets"], w["particles"], 0.5, o)
    assert ei.value.code == G.GLISSE_E_INVAL
    for lm in (-1, 3):
        o = G.glisse_opts_default()
        o.launch_mode = lm
        with pytest.raises(G.GlisseError) as ei:
            G.glisse_create(1.0, w["planets"], w["particles"], 0.5, o)
        assert ei.value.code == G.GLISSE_E_INVAL, lm
    # checkpoint intervals below GLISSE_DIFF_TAPE_TANGENT
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_diff_create(1.0, w["planets"], 4, 0.5, 10, -3)
    assert ei.value.code == G.GLISSE_E_INVAL
    # the fixed-iteration mode is for glisse_create only
    o = G.glisse_opts_default()
    o.kepler_mode = G.GLISSE_KEPLER_PAPER_FIXED
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_diff_create(1.0, w["planets"], 4, 0.5, 10, 4, o)
    assert ei.value.code == G.GLISSE_E_INVAL
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_batch_create([1.0], [4], w["planets"], [4], w["particles"], [0.5], o)
    assert ei.value.code == G.GLISSE_E_INVAL
    L = G.load()
    assert L.glisse_advance(None, 1) == G.GLISSE_E_INVAL
    assert L.glisse_read(None, None, None, None, None) == G.GLISSE_E_INVAL
    assert L.glisse_partition_device(-1, 0, None, None, None, None, None, None, None) == G.GLISSE_E_INVAL
    assert L.glisse_fp64_peak(0, None, None) == G.GLISSE_E_INVAL
    st = C.c_int32(7)
    for which, polls in ((-1, 10), (3, 10), (G.GLISSE_WAIT_PARTICLE_TASKS, 0)):
        assert L.glisse_selftest_wait(which, polls, C.byref(st), None) == G.GLISSE_E_INVAL, (which, polls)
    assert L.glisse_selftest_wait(G.GLISSE_WAIT_DIFF_FORWARD, 10, None, None) == G.GLISSE_E_INVAL
    assert st.value == 7
    L.glisse_destroy(None)


def test_null_handles_are_rejected(G):
    """Every call that takes a context returns GLISSE_E_INVAL for a NULL one (no CUDA call)."""
    L = G.load()
    E = G.GLISSE_E_INVAL
    calls = [
        lambda: L.glisse_status(None, None, None, None),
        lambda: L.glisse_read_planets(None, None, None),
        lambda: L.glisse_set_ephemeris(None, None, 1),
        lambda: L.glisse_timings(None, None, 0),
        lambda: L.glisse_set_sampling(None, None),
        lambda: L.glisse_read_elements(None, None, None, 0, None),
        lambda: L.glisse_read_libration(None, None, None, None),
        lambda: L.glisse_batch_advance(None, 1),
        lambda: L.glisse_batch_read(None, None, None, None, None),
        lambda: L.glisse_batch_status(None, None, None),
        lambda: L.glisse_batch_timings(None, None, 0),
        lambda: L.glisse_batch_steps_done(None, None),
        lambda: L.glisse_batch_tune(None, 0, None, None, None),
        lambda: L.glisse_batch_set_launch(None, 128, 1),
        lambda: L.glisse_diff_forward(None, None, None, 0, None, None, None, None, None, None),
        lambda: L.glisse_diff_backward(None, None, None, None),
        lambda: L.glisse_diff_backward_growth(None, None, None, None, None, None, None),
        lambda: L.glisse_diff_growth_gradient(None, None, None, None, None, None),
        lambda: L.glisse_checkpoint_size(None, None),
        lambda: L.glisse_checkpoint(None, None, 0),
        lambda: L.glisse_sizes(None, None, None),
        lambda: L.glisse_batch_checkpoint_size(None, None),
        lambda: L.glisse_batch_checkpoint(None, None, 0),
        lambda: L.glisse_batch_sizes(None, None, None),
    ]
    for k, call in enumerate(calls):
        assert call() == E, k
    L.glisse_batch_destroy(None)
    L.glisse_diff_destroy(None)


def test_no_cpu_fallback_without_a_device(G):
    """On a machine without a usable GPU a valid create fails with GLISSE_E_CUDA instead of computing."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import glisse_inputs as gi

    w = gi.make("tiny", n=4)
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_create(1.0, w["planets"], w["particles"], 0.5)
    assert ei.value.code == G.GLISSE_E_CUDA


def test_package_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2011_03484_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f


def test_resume_rejects_what_is_not_a_checkpoint(G):
    """glisse_resume validates the buffer on the host before any CUDA call."""
    import ctypes as C

    L = G.load()
    h = C.c_void_p()
    E = G.GLISSE_E_INVAL
    assert L.glisse_resume(None, None, 0, None) == E
    assert L.glisse_resume(C.byref(h), None, 0, None) == E
    for buf in (b"", b"GLISSECK", bytes(4096), b"GLISSECK" + bytes(4088), np.random.default_rng(0).bytes(4096)):
        arr = np.frombuffer(buf, dtype=np.uint8).copy() if buf else np.zeros(1, dtype=np.uint8)
        assert L.glisse_resume(C.byref(h), arr.ctypes.data, len(buf), None) == E
        assert not h.value
    with pytest.raises(G.GlisseError) as ei:
        G.glisse_resume(bytes(64))
    assert ei.value.code == E
    # the batched resume, and neither accepts the other's checkpoints' magic
    assert L.glisse_batch_resume(None, None, 0, None) == E
    for buf in (b"", b"GLISSEBK" + bytes(4088), b"GLISSECK" + bytes(4088), np.random.default_rng(1).bytes(4096)):
        arr = np.frombuffer(buf, dtype=np.uint8).copy() if buf else np.zeros(1, dtype=np.uint8)
        assert L.glisse_batch_resume(C.byref(h), arr.ctypes.data, len(buf), None) == E
        assert not h.value
