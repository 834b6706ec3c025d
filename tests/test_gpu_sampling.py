"""Element sampling and the resonance libration test on the GPU (glisse_set_sampling,
glisse_read_elements, glisse_read_libration) against the oracle's run_sampled."""
import numpy as np
import pytest

import glisse_inputs as gi
import parity
import test_oracle_elements as TE

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


def _ang(x, y):
    return np.abs(np.mod(x - y + np.pi, 2 * np.pi) - np.pi)


def run_gpu(G, pl, pa, dt, n, every, max_samples, chunk=1024, **samp):
    sim = G.Simulation(1.0, pl, pa, dt, chunk_steps=chunk)
    sim.set_sampling(every, max_samples=max_samples, **samp)
    sim.advance(n)
    out = sim.read()
    out["elements"], out["sample_steps"] = sim.elements()
    if samp.get("res_planet", -1) >= 0:
        out.update(sim.libration())
    sim.close()
    return out


def borderline(phi, avoid_deg, eps=1e-6):
    """Particles with some sample of phi within eps of a window edge (the GPU and the oracle
    may then decide the flag differently)."""
    a = np.radians(avoid_deg)
    d0 = np.minimum(phi, 2 * np.pi - phi)
    d180 = np.abs(phi - np.pi)
    near = (np.abs(d0 - a) < eps) | (np.abs(d180 - a) < eps)
    return np.any(np.nan_to_num(near, nan=False), axis=0)


def test_elements_and_flags_match_the_oracle(G, orc):
    """1024 particles, 3000 steps, a sample every 500 steps (not aligned with the 1024-step
    chunks), barycentric elements, Neptune's 2:3 inner resonance phi = 2 lambda - 3 lambda_N + varpi."""
    w = gi.make("tiny")
    pl, pa = w["planets"], w["particles"]
    n, every = 3000, 500
    samp = dict(frame=G.GLISSE_FRAME_BARY, res_planet=3, res_p=2, res_q=3, avoid_deg=10.0)
    g = run_gpu(G, pl, pa, w["dt"], n, every, 16, **samp)
    o = orc.run_sampled(1.0, pl, pa, w["dt"], n, every, frame=1, res_planet=3, res_p=2, res_q=3, avoid_deg=10.0)
    np.testing.assert_array_equal(g["sample_steps"], o["sample_steps"])
    assert g["elements"].shape == o["elements"].shape == (6, 1024, 6)
    # rows of particles live in the oracle at each sample (removal steps agree outside the band)
    border = o["margin"] < parity.BAND
    live_o = ~np.isnan(o["elements"][..., 0])
    live_g = ~np.isnan(g["elements"][..., 0])
    assert np.array_equal(live_o[:, ~border], live_g[:, ~border])
    # regular particles: elements as close as the states (FP64 phase noise after 3000 steps)
    reg = (o["closest"] >= 25.0) & ~border
    m = live_o & live_g & reg[None, :]
    eg, eo = g["elements"][m], o["elements"][m]
    tol = 1e-9
    assert np.abs(eg[:, 0] / eo[:, 0] - 1).max() < tol
    assert np.abs(eg[:, 1] - eo[:, 1]).max() < tol
    assert np.abs(eg[:, 2] - eo[:, 2]).max() < tol
    assert (_ang(eg[:, 3] + eg[:, 4], eo[:, 3] + eo[:, 4]) * eo[:, 1]).max() < tol
    assert _ang(eg[:, 3] + eg[:, 4] + eg[:, 5], eo[:, 3] + eo[:, 4] + eo[:, 5]).max() < tol
    # libration flags: exact for regular particles away from the window edges
    ok = reg & ~borderline(o["phi"], 10.0)
    np.testing.assert_array_equal(g["count"][ok], o["count"][ok])
    np.testing.assert_array_equal(g["near0"][ok], o["near0"][ok].astype(bool))
    np.testing.assert_array_equal(g["near180"][ok], o["near180"][ok].astype(bool))
    assert ok.sum() > 400 and (g["count"][ok] > 0).all()


def test_resonant_particles_librate_on_the_gpu(G, orc):
    pl, pa = TE._resonant_and_circulating(orc)
    g = run_gpu(G, pl, pa, 0.5, 40000, 10, 0, frame=G.GLISSE_FRAME_HELIO, res_planet=3, res_p=3, res_q=2)
    assert np.all(g["count"] == 4000)
    assert g["librating"][:6].all() and not g["librating"][6:].any(), (g["near0"], g["near180"])
    assert g["elements"].shape[0] == 0


def test_sampling_leaves_the_map_unchanged(G):
    """Sampling ends segments at the sample steps; those cuts are open (the merged kick is
    applied as in an uncut run, the sampled state is computed beside it), so the run is the
    unsampled run bit for bit."""
    w = gi.make("tiny")
    n = 2000
    a = run_gpu(G, w["planets"], w["particles"], w["dt"], n, 300, 2, frame=G.GLISSE_FRAME_HELIO)
    sim = G.Simulation(1.0, w["planets"], w["particles"], w["dt"])
    sim.advance(n)
    b = sim.read()
    sim.close()
    for k in ("state", "alive", "removal_step", "removal_reason"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_element_log_capacity_and_flags_count(G):
    w = gi.make("tiny", n=200)
    g = run_gpu(G, w["planets"], w["particles"], w["dt"], 1200, 200, 3, frame=G.GLISSE_FRAME_HELIO, res_planet=3,
                res_p=2, res_q=3)
    np.testing.assert_array_equal(g["sample_steps"], [200, 400, 600])
    live_end = g["removal_step"] < 0
    assert np.all(g["count"][live_end] == 6)  # every sample of a bound live particle counts
    # removed particles have NaN rows from the first sample after their removal
    for k, st in enumerate(g["sample_steps"]):
        gone = (g["removal_step"] >= 0) & (g["removal_step"] <= st)
        assert np.isnan(g["elements"][k][gone]).all()
        assert not np.isnan(g["elements"][k][~gone & live_end]).any()


def test_sampling_argument_and_state_errors(G):
    w = gi.make("tiny", n=8)
    sim = G.Simulation(1.0, w["planets"], w["particles"], w["dt"])
    with pytest.raises(G.GlisseError) as ei:
        sim.libration()
    assert ei.value.code == G.GLISSE_E_STATE
    for kw in (dict(every=0), dict(every=10, frame=5), dict(every=10, res_planet=4, res_p=3, res_q=1),
               dict(every=10, res_planet=3, res_p=0, res_q=1), dict(every=10, res_planet=3, res_p=3, res_q=1,
                                                                    avoid_deg=95.0)):
        with pytest.raises(G.GlisseError) as ei:
            sim.set_sampling(**kw)
        assert ei.value.code == G.GLISSE_E_INVAL, kw
    sim.set_sampling(10, max_samples=1)
    with pytest.raises(G.GlisseError) as ei:
        sim.set_ephemeris(np.zeros((11, 4, 3)))
    assert ei.value.code == G.GLISSE_E_STATE
    with pytest.raises(G.GlisseError) as ei:
        sim.libration()  # sampling set without a libration test
    assert ei.value.code == G.GLISSE_E_STATE
    sim.set_sampling(None)
    sim.close()
