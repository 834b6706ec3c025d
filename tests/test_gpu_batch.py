"""Batched independent systems (many stars, planet sets, particle sets and dt in one
context) on the GPU, checked against the oracle system by system and against the
single-system path on the same inputs."""
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


def small_batch(n_systems=10, seed=7, n_min=20, n_max=700):
    b = gi.make_batched(seed=seed, n_systems=n_systems, n_min=n_min, n_max=n_max)
    # add a planet-free system and a one-planet system (edge cases of the planet count)
    extra_pl = b["planets"][:1].copy()
    b2 = {
        "star_mass": np.concatenate([b["star_mass"], [1.0, 1.0]]),
        "n_planets": np.concatenate([b["n_planets"], [0, 1]]).astype(np.int32),
        "planets": np.concatenate([b["planets"], extra_pl]),
        "n_particles": np.concatenate([b["n_particles"], [33, 65]]).astype(np.int64),
        "dt": np.concatenate([b["dt"], [0.3, 0.2]]),
    }
    rng = np.random.default_rng(seed)
    a = rng.uniform(3.0, 9.0, 98)
    extra_pa = gi.elements_to_cartesian(gi.G, a, rng.uniform(0, 0.05, 98), np.radians(rng.uniform(0, 2, 98)),
                                        *rng.uniform(0, 2 * np.pi, (3, 98)))
    b2["particles"] = np.concatenate([b["particles"], extra_pa])
    return b2


def offsets(b):
    po = np.concatenate([[0], np.cumsum(b["n_planets"])])
    ao = np.concatenate([[0], np.cumsum(b["n_particles"])])
    return po, ao


def oracle_batch(orc, b, n_steps, ids_per_system=None):
    """Oracle run system by system; returns concatenated results, sensitivity, unstable mask,
    particle ids and the mean anomaly each particle advances (for the phase-scaled bounds)."""
    po, ao = offsets(b)
    keys = ("state", "removal_step", "reason", "margin", "closest")
    outs = {k: [] for k in keys}
    sens_all, unst_all, idx, phase = [], [], [], []
    for s in range(len(b["star_mass"])):
        pl = b["planets"][po[s]:po[s + 1]]
        rows = np.arange(ao[s], ao[s + 1]) if ids_per_system is None else ids_per_system[s]
        if len(rows) == 0:
            continue
        pa = b["particles"][rows]
        base = orc.run(b["star_mass"][s], pl, pa, b["dt"][s], n_steps)
        runs = [orc.run(b["star_mass"][s], pl, p, b["dt"][s], n_steps) for p in parity.perturbed_inputs(pa)]
        runs.append(orc.run(b["star_mass"][s], parity.perturbed_planets(pl), pa, b["dt"][s], n_steps))
        sens, unst = parity.sensitivity(base, runs)
        for k in keys:
            outs[k].append(base[k])
        sens_all.append(sens)
        unst_all.append(unst)
        idx.append(rows)
        phase.append(parity.phase_advance(pa, gi.G * b["star_mass"][s], b["dt"][s], n_steps))
    o = {k: np.concatenate(v) for k, v in outs.items()}
    return (o, np.concatenate(sens_all), np.concatenate(unst_all), np.concatenate(idx),
            np.concatenate(phase))


def run_batch(G, b, n_steps, splits=None, **opt):
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"],
                            **opt)
    for m in (splits or [n_steps]):
        sim.advance(m)
    out = sim.read()
    out["n_live"], out["step"] = sim.status()
    sim.close()
    return out


def sub(g, ids):
    return {k: g[k][ids] for k in ("state", "alive", "removal_step", "removal_reason")}


def test_batch_matches_oracle_system_by_system(G, orc):
    b = small_batch()
    n = 1500
    g = run_batch(G, b, n, chunk_steps=256)
    o, sens, unst, ids, ph = oracle_batch(orc, b, n)
    rep = parity.compare(sub(g, ids), o, n, sens, unst, ph)
    print(rep)
    parity.assert_parity(rep)
    assert rep["removed"] > 0
    assert g["n_live"] == int(g["alive"].sum()) and g["step"] == n


@pytest.mark.parametrize("chunk", [128, 1024])
def test_batch_equals_single_system_runs(G, chunk):
    """Each system of a batch evolves as the single-system path evolves it: same removal
    steps, and, within one chunk (chunk >= n), bit-identical states except on lanes that
    needed the general Kepler solver, whose plain expressions the compiler may contract
    into FMAs differently in the two kernels (rounding-level differences).  The
    single-system path runs its first chunk in segments (cut at steps 64, 128, 256, 512)
    that pass the open kick between them; the batch path does not cut, so this also checks
    that the cuts leave no trace.  With several chunks (chunk 128) the batch closes every
    chunk with a half kick while the single-system path keeps its chunk ends open: the
    states then differ by rounding at each chunk end, within the parity tolerance."""
    b = small_batch(n_systems=6, seed=8)
    n = 700
    g = run_batch(G, b, n, chunk_steps=chunk)
    po, ao = offsets(b)
    for s in range(len(b["star_mass"])):
        sim = G.Simulation(b["star_mass"][s], b["planets"][po[s]:po[s + 1]], b["particles"][ao[s]:ao[s + 1]],
                           b["dt"][s], chunk_steps=chunk)
        sim.advance(n)
        r = sim.read()
        sim.close()
        rows = slice(ao[s], ao[s + 1])
        np.testing.assert_array_equal(g["removal_step"][rows], r["removal_step"])
        np.testing.assert_array_equal(g["removal_reason"][rows], r["removal_reason"])
        e = parity.rel_err(g["state"][rows], r["state"])
        if chunk >= n:
            assert np.mean(e == 0.0) > 0.5, (s, np.mean(e == 0.0))
        assert e.max() <= parity.state_tol(n), (s, e.max())


def test_graph_replay_equals_direct_launches(G):
    b = small_batch(n_systems=5, seed=9)
    g1 = run_batch(G, b, 900, splits=[300, 300, 300], chunk_steps=256)  # captured chunk graphs
    g2 = run_batch(G, b, 900, splits=[300, 300, 300], chunk_steps=256, timing=1)  # direct launches with events
    for k in ("state", "removal_step", "removal_reason"):
        np.testing.assert_array_equal(g1[k], g2[k])


def test_batch_split_invariance(G):
    b = small_batch(n_systems=5, seed=10)
    ref = run_batch(G, b, 1000, chunk_steps=512)
    g = run_batch(G, b, 1000, splits=[1, 399, 600], chunk_steps=512)
    np.testing.assert_array_equal(g["removal_step"], ref["removal_step"])
    alive = g["alive"]
    e = parity.rel_err(g["state"][alive], ref["state"][alive])
    assert np.median(e) < 1e-12 and e.max() < 1e3 * parity.state_tol(1000)


def test_autotuner_keeps_the_state(G, orc):
    b = small_batch(n_systems=8, seed=11, n_min=200, n_max=3000)
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"])
    sim.advance(100)
    before = sim.read()
    c, t, p = sim.tune(trial_steps=64)
    assert c in (256, 512, 1024) and t in (64, 128, 256) and p in (1, 2)
    after = sim.read()
    for k in ("state", "removal_step", "removal_reason"):
        np.testing.assert_array_equal(before[k], after[k])
    assert sim.status()[1] == 100
    sim.advance(900)
    g = sim.read()
    g["n_live"], g["step"] = sim.status()
    sim.close()
    o, sens, unst, ids, ph = oracle_batch(orc, b, 1000)
    parity.assert_parity(parity.compare(sub(g, ids), o, 1000, sens, unst, ph))


def test_full_batched_workload_sampled(G, orc):
    """The 256-system, ~3.4e6-particle workload in its default launch shape, sampled."""
    b = gi.make_batched()
    n = 2048
    g = run_batch(G, b, n)
    po, ao = offsets(b)
    rng = np.random.default_rng(12)
    systems = rng.choice(len(b["star_mass"]), 24, replace=False)
    per = {s: np.sort(rng.choice(np.arange(ao[s], ao[s + 1]), min(40, ao[s + 1] - ao[s]), replace=False))
           for s in systems}
    bb = dict(b)
    ids_per_system = [per.get(s, np.zeros(0, dtype=np.int64)) for s in range(len(b["star_mass"]))]
    o, sens, unst, ids, ph = oracle_batch(orc, bb, n, ids_per_system)
    rep = parity.compare(sub(g, ids), o, n, sens, unst, ph)
    print(rep)
    parity.assert_parity(rep)
    assert g["n_live"] == int(g["alive"].sum())
    assert np.all((g["removal_step"] >= 0) == ~g["alive"])


def test_batch_long_horizon_against_the_oracle(G, orc):
    """Six systems of the batched workload's shape (2-8 planets, dt = P_inner / 20) over
    10^4 steps, in 1024-step chunks with graph replay, against the oracle system by system
    under the phase-scaled bounds."""
    b = small_batch(n_systems=6, seed=21, n_min=20, n_max=64)
    n = 10_000
    g = run_batch(G, b, n, chunk_steps=1024)
    o, sens, unst, ids, ph = oracle_batch(orc, b, n)
    rep = parity.compare(sub(g, ids), o, n, sens, unst, ph)
    print(rep)
    parity.assert_parity(rep)
    assert rep["n"] >= 200 and rep["regular"] >= 20


def test_steps_done_counts_each_particles_steps(G):
    """glisse_batch_steps_done (graph-replayed chunks) equals the particle-steps implied
    by the removal steps: a removed particle advanced removal_step steps, a live one all."""
    b = small_batch(n_systems=5, seed=12)
    n = 1300
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"],
                            chunk_steps=256)
    sim.advance(700)
    sim.advance(600)
    done = sim.steps_done()
    g = sim.read()
    sim.close()
    rs = g["removal_step"]
    assert done == int(np.where(rs >= 0, rs, n).sum())
    assert (rs >= 0).sum() > 0


def test_two_lanes_per_particle_match_the_oracle(G, orc):
    """The lane-pair kernel (threads_per_particle = 2: each lane of the pair takes half of
    the planets in the kick) against the oracle, system by system."""
    b = small_batch()
    n = 1500
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"],
                            chunk_steps=256)
    sim.set_launch(128, 2)
    sim.advance(n)
    g = sim.read()
    g["n_live"], g["step"] = sim.status()
    done = sim.steps_done()
    sim.close()
    o, sens, unst, ids, ph = oracle_batch(orc, b, n)
    rep = parity.compare(sub(g, ids), o, n, sens, unst, ph)
    print(rep)
    parity.assert_parity(rep)
    assert rep["removed"] > 0
    rs = g["removal_step"]
    assert done == int(np.where(rs >= 0, rs, n).sum())  # each particle counted once


def test_two_lanes_equal_one_lane_up_to_rounding(G, orc):
    """The pair sums its two partial kicks, so states differ from the one-lane kernel by
    rounding only; removal steps agree, and states agree within the parity bound (the
    regular-orbit tolerance, or sens_factor(n) times the oracle's one-ulp sensitivity for
    orbits a planet passage makes chaotic)."""
    b = small_batch(n_systems=5, seed=13)
    n = 800
    out = []
    for tpp in (1, 2):
        sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"],
                                b["dt"], chunk_steps=256)
        sim.set_launch(64, tpp)
        sim.advance(n)
        out.append(sim.read())
        sim.close()
    assert np.mean(out[0]["removal_step"] == out[1]["removal_step"]) > 0.999
    _, sens, _, ids, _ = oracle_batch(orc, b, n)
    s_by_id = np.zeros(len(out[0]["alive"]))
    s_by_id[ids] = sens
    both = out[0]["alive"] & out[1]["alive"]
    e = parity.rel_err(out[0]["state"][both], out[1]["state"][both])
    bound = np.maximum(parity.state_tol(n), parity.sens_factor(n) * s_by_id[both])
    assert np.median(e) < 1e-12 and (e <= bound).all(), (np.median(e), e.max(), (e / bound).max())


def test_set_launch_rejects_bad_shapes(G):
    b = small_batch(n_systems=2, seed=14)
    sim = G.BatchSimulation(b["star_mass"], b["n_planets"], b["planets"], b["n_particles"], b["particles"], b["dt"])
    for bad in ((48, 1), (512, 1), (128, 3), (128, 0)):
        with pytest.raises(RuntimeError):
            sim.set_launch(*bad)
    sim.close()
