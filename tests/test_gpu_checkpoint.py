"""Checkpoint and resume through the C ABI (GPU).

The paper continues runs from their output states (sections 4.2.2, 4.3.2).
A context resumed from a checkpoint and advanced must give exactly what the
original context gives with the same calls: states (live and frozen), flags,
removal steps and reasons, planets, live count and step, all bit for bit.
Cases: a resume in the middle of a chunk, inside the first chunk (whose
particles run in segments behind the planets' progress), right after
create (the removal test at t_0 still to come), with removals, a compaction
interval of several chunks, the cost-sorted particle order and the paper's
fixed-iteration solver.  A checkpoint taken right after resume equals the
one resumed from, byte for byte.  Buffers that are not checkpoints, or hold
an id outside the particle range, are rejected.  Batches of independent
systems resume the same way (graph-replayed or timed chunks, lane pairs).
"""
import numpy as np
import pytest

import glisse_inputs as gi
import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_03484_gb300 as G

    G._build.build()
    G.load()
    return G


def _snapshot(sim):
    out = sim.read()
    out["planets"] = sim.planets()[0] if sim.n_planets else None
    out["status"] = sim.status()
    return out


def _assert_identical(a, b):
    for k in ("state", "alive", "removal_step", "removal_reason"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    if a["planets"] is not None:
        assert np.array_equal(a["planets"], b["planets"])
    assert a["status"] == b["status"]


CASES = [
    # (workload, particles, first call, second call, options)
    ("tiny", 1024, 300, 700, dict(chunk_steps=128)),          # resume in the middle of a chunk
    ("tiny", 1024, 40, 500, dict(chunk_steps=128)),           # inside the first chunk (its segments)
    ("tiny", 1024, 0, 400, dict(chunk_steps=128)),            # before the first step: t_0 test pending
    ("eccentric", 4096, 600, 900, dict(chunk_steps=256, resync_chunks=3)),
    ("eccentric", 4096, 700, 600, dict(chunk_steps=256, sort_mode=1)),
    ("eccentric", 2048, 300, 300, dict(chunk_steps=100, kepler_mode=1, kepler_iters=3)),
]


@pytest.mark.parametrize("name,n,first,second,opt", CASES)
def test_resume_continues_bit_for_bit(G, name, n, first, second, opt):
    w = gi.make(name, n=n)
    a = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], **opt)
    if first:
        a.advance(first)
    ck = a.checkpoint()
    a.advance(second)
    ref = _snapshot(a)
    a.close()

    b = G.Simulation.resume(ck)
    assert (b.n, b.n_planets) == (n, w["planets"].shape[0])
    assert np.array_equal(b.checkpoint(), ck)  # nothing lost or changed on the way in
    b.advance(second)
    got = _snapshot(b)
    b.close()
    _assert_identical(ref, got)
    if name == "eccentric" and first:
        assert (~ref["alive"]).sum() > 0  # the case exercises removed particles


def test_resume_on_another_stream_with_timing(G):
    import torch

    w = gi.make("tiny", n=512)
    a = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=64)
    a.advance(100)
    ck = a.checkpoint()
    a.advance(200)
    ref = _snapshot(a)
    a.close()
    s = torch.cuda.Stream()
    b = G.Simulation.resume(ck, cuda_stream=s.cuda_stream, timing=1)
    b.advance(200)
    got = _snapshot(b)
    t = b.timings()
    b.close()
    _assert_identical(ref, got)
    assert t["particle_launches"] > 0 and t["particle_steps"] > 0


def test_chained_checkpoints_equal_one_run(G):
    w = gi.make("tiny", n=1024)
    a = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=128)
    a.advance(900)
    ref = _snapshot(a)
    a.close()
    sim = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=128)
    for m in (100, 250, 300, 250):
        sim.advance(m)
        ck = sim.checkpoint()
        sim.close()
        sim = G.Simulation.resume(ck)
    got = _snapshot(sim)
    sim.close()
    # the calls differ from the single 900-step call only where they cut the run (two half
    # kicks instead of one merged kick, and a compaction): the split-invariance criteria
    # hold, removal steps exactly and live states to rounding; the planets are bit for bit
    assert np.array_equal(ref["removal_step"], got["removal_step"])
    assert np.array_equal(ref["removal_reason"], got["removal_reason"])
    live = ref["alive"]
    e = parity.rel_err(got["state"][live], ref["state"][live])
    assert np.median(e) < 1e-12, np.median(e)
    assert e.max() < 1e3 * parity.state_tol(900), e.max()
    assert np.array_equal(ref["planets"], got["planets"])


def test_checkpoint_errors(G):
    import ctypes as C

    L = G.load()
    w = gi.make("tiny", n=256)
    sim = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=64)
    ck = sim.checkpoint()
    # a buffer smaller than the checkpoint
    n = C.c_int64()
    assert L.glisse_checkpoint_size(sim.h, C.byref(n)) == G.GLISSE_OK and n.value == ck.size
    small = np.empty(ck.size - 1, dtype=np.uint8)
    assert L.glisse_checkpoint(sim.h, small.ctypes.data, small.size) == G.GLISSE_E_INVAL
    # truncated, wrong magic, an id outside 0..n-1, a repeated id
    h = C.c_void_p()
    assert L.glisse_resume(C.byref(h), ck.ctypes.data, ck.size - 1, None) == G.GLISSE_E_INVAL
    bad = ck.copy()
    bad[0] ^= 0xFF
    assert L.glisse_resume(C.byref(h), bad.ctypes.data, bad.size, None) == G.GLISSE_E_INVAL
    ids = np.arange(256, dtype=np.int32).tobytes()
    off = ck.tobytes().find(ids)
    assert off > 0 and off % 4 == 0
    for k, v in ((17, 256), (17, -1), (17, 3)):
        bad = ck.copy()
        bad[off + 4 * k: off + 4 * k + 4] = np.frombuffer(np.int32(v).tobytes(), dtype=np.uint8)
        assert L.glisse_resume(C.byref(h), bad.ctypes.data, bad.size, None) == G.GLISSE_E_INVAL, v
    assert not h.value
    sim.close()
    # state that a checkpoint does not hold: an external ephemeris
    sim = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=64)
    sim.set_ephemeris(np.tile(w["planets"][:, 1:4], (11, 1, 1)))
    with pytest.raises(G.GlisseError) as ei:
        sim.checkpoint()
    assert ei.value.code == G.GLISSE_E_STATE
    sim.close()


def test_resume_rejects_oversized_sample_count(G):
    """A checkpoint whose header claims more kept element samples than its buffer can hold
    (here 2^40 samples of 256 particles, 12.6 PB) is rejected before any array is read."""
    import ctypes as C

    L = G.load()
    w = gi.make("tiny", n=256)
    sim = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=64)
    sim.set_sampling(25, max_samples=9)
    sim.advance(130)  # 5 samples taken, 5 kept
    ck = sim.checkpoint()
    sim.close()
    h = C.c_void_p()
    assert L.glisse_resume(C.byref(h), ck.ctypes.data, ck.size, None) == G.GLISSE_OK
    L.glisse_destroy(h)
    # header fields: samples taken, samples kept (int64 each), then the sampling settings
    # (every = 25 as int32, frame int32, max_samples int64)
    pat = np.int64(5).tobytes() + np.int64(5).tobytes() + np.int32(25).tobytes()
    off = ck.tobytes().find(pat)
    assert 0 < off < 512 and off % 8 == 0
    big = np.int64(1 << 40).tobytes()
    bad = ck.copy()
    for o in (off, off + 8, off + 24):  # seen, kept, max_samples
        bad[o:o + 8] = np.frombuffer(big, dtype=np.uint8)
    h = C.c_void_p()
    assert L.glisse_resume(C.byref(h), bad.ctypes.data, bad.size, None) == G.GLISSE_E_INVAL
    assert not h.value


def test_empty_and_planet_free_checkpoints(G):
    w = gi.make("tiny", n=300)
    for planets, particles in ((w["planets"], w["particles"][:0]), (w["planets"][:0], w["particles"])):
        a = G.Simulation(1.0, planets, particles, w["dt"], chunk_steps=50)
        a.advance(75)
        ck = a.checkpoint()
        a.advance(60)
        ref = _snapshot(a)
        a.close()
        b = G.Simulation.resume(ck)
        b.advance(60)
        got = _snapshot(b)
        b.close()
        _assert_identical(ref, got)


# ---------------------------------------------------------------------------
# batches of independent systems
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("first,second,chunk,shape,timing", [
    (300, 700, 256, None, 0),       # mid-chunk, graph-replayed chunks
    (0, 500, 128, None, 0),         # before the first step: the removal test at t_0 pending
    (512, 512, 256, (64, 2), 1),    # lane pairs, 64-thread blocks; the resumed batch times its launches
])
def test_batch_resume_continues_bit_for_bit(G, first, second, chunk, shape, timing):
    b = gi.make_batched(seed=4, n_systems=12, n_max=4096)
    args = (b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"])
    a = G.BatchSimulation(*args, chunk_steps=chunk)
    if shape:
        a.set_launch(*shape)
    if first:
        a.advance(first)
    ck = a.checkpoint()
    a.advance(second)
    ref, ref_status = a.read(), a.status()
    a.close()

    r = G.BatchSimulation.resume(ck, timing=timing)
    assert r.n == a.n == int(np.sum(b["n_particles"]))
    assert np.array_equal(r.checkpoint(), ck)  # nothing lost or changed on the way in
    r.advance(second)
    got, got_status = r.read(), r.status()
    r.close()
    for k in ("state", "alive", "removal_step", "removal_reason"):
        assert np.array_equal(ref[k], got[k], equal_nan=True), k
    assert ref_status == got_status


def test_batch_checkpoint_errors(G):
    import ctypes as C

    L = G.load()
    b = gi.make_batched(seed=4, n_systems=6, n_max=2048)
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"],
                            b["dt"], chunk_steps=128)
    sim.advance(200)
    ck = sim.checkpoint()
    small = np.empty(ck.size - 1, dtype=np.uint8)
    assert L.glisse_batch_checkpoint(sim.h, small.ctypes.data, small.size) == G.GLISSE_E_INVAL
    sim.close()
    h = C.c_void_p()
    assert L.glisse_batch_resume(C.byref(h), ck.ctypes.data, ck.size - 1, None) == G.GLISSE_E_INVAL
    for pos in (0, 8):  # magic, version
        bad = ck.copy()
        bad[pos] ^= 0xFF
        assert L.glisse_batch_resume(C.byref(h), bad.ctypes.data, bad.size, None) == G.GLISSE_E_INVAL
    # a single-system checkpoint is not a batch checkpoint, nor the reverse
    w = gi.make("tiny", n=64)
    s1 = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"])
    ck1 = s1.checkpoint()
    s1.close()
    assert L.glisse_batch_resume(C.byref(h), ck1.ctypes.data, ck1.size, None) == G.GLISSE_E_INVAL
    assert L.glisse_resume(C.byref(h), ck.ctypes.data, ck.size, None) == G.GLISSE_E_INVAL
    assert not h.value


def test_continuation_with_libration_detection(G):
    """The paper's continuation runs: a long run, then more steps that log elements and test
    libration (section 4.2.2).  A resumed context that starts sampling gives the same
    elements, sample steps and libration flags as the original context sampling from the
    same step, bit for bit (the sampled planet states come from the recomputed chunk)."""
    w = gi.make("tiny", n=512)
    samp = dict(max_samples=12, res_planet=3, res_p=3, res_q=2, avoid_deg=10.0)
    a = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=128)
    a.advance(1000)
    ck = a.checkpoint()
    a.set_sampling(20, **samp)
    a.advance(230)
    ref_el, ref_steps = a.elements()
    ref_lib = a.libration()
    ref = _snapshot(a)
    a.close()

    b = G.Simulation.resume(ck)
    b.set_sampling(20, **samp)
    b.advance(230)
    el, steps = b.elements()
    lib = b.libration()
    got = _snapshot(b)
    b.close()
    assert len(steps) == 11 and np.array_equal(steps, ref_steps)
    assert np.array_equal(el, ref_el, equal_nan=True)
    for k in ref_lib:
        assert np.array_equal(np.asarray(lib[k]), np.asarray(ref_lib[k])), k
    _assert_identical(ref, got)


def test_checkpoint_while_sampling(G):
    """A checkpoint taken between samples carries the sampling: the resumed context's
    elements, sample steps and libration flags over the whole run equal the original's."""
    w = gi.make("tiny", n=512)
    samp = dict(max_samples=9, res_planet=3, res_p=3, res_q=2, avoid_deg=10.0)
    a = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], chunk_steps=128)
    a.set_sampling(25, **samp)
    a.advance(130)
    ck = a.checkpoint()
    a.advance(200)  # 13 samples in all: 9 kept, every one counted by the libration test
    ref_el, ref_steps = a.elements()
    ref_lib = a.libration()
    ref = _snapshot(a)
    a.close()
    b = G.Simulation.resume(ck)
    b.advance(200)
    el, steps = b.elements(samp["max_samples"])
    lib = b.libration()
    got = _snapshot(b)
    b.close()
    assert len(steps) == 9 and np.array_equal(steps, ref_steps)
    assert np.array_equal(el, ref_el, equal_nan=True)
    for k in ref_lib:
        assert np.array_equal(np.asarray(lib[k]), np.asarray(ref_lib[k])), k
    assert int(np.asarray(ref_lib["count"]).max()) == 13
    _assert_identical(ref, got)
