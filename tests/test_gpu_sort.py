"""Ordering live particles by expected Kepler-solve cost (GLISSE_SORT_COST; section 2.2's
sorting suggestion) on the GPU: results stay those of the oracle, and differ from the
unsorted run only by rounding (a warp's polynomial degree depends on its members)."""
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


def run_gpu(G, w, pa, n, **opt):
    sim = G.Simulation(1.0, w["planets"], pa, w["dt"], **opt)
    sim.advance(n)
    g = sim.read()
    sim.close()
    return g


def test_sorted_run_matches_the_oracle(G, orc):
    w = gi.make("eccentric")
    ids = gi.subset_ids("eccentric", 3000)
    pa = w["particles"][ids]
    n = 2000
    g = run_gpu(G, w, pa, n, sort_mode=G.GLISSE_SORT_COST, chunk_steps=256)
    base = orc.run(1.0, w["planets"], pa, w["dt"], n)
    runs = [orc.run(1.0, w["planets"], p, w["dt"], n) for p in parity.perturbed_inputs(pa)]
    runs.append(orc.run(1.0, parity.perturbed_planets(w["planets"]), pa, w["dt"], n))
    sens, unstable = parity.sensitivity(base, runs)
    rep = parity.compare(g, base, n, sens, unstable, ecc=parity.eccentricity(pa, gi.G))
    print(rep)
    parity.assert_parity(rep)
    assert rep["removed"] > 100


@pytest.mark.parametrize("resync", [1, 3])
def test_sorted_equals_unsorted_up_to_rounding(G, resync):
    w = gi.make("eccentric")
    pa = w["particles"][:20000]
    n = 3000
    a = run_gpu(G, w, pa, n, sort_mode=G.GLISSE_SORT_COST, chunk_steps=512, resync_chunks=resync)
    b = run_gpu(G, w, pa, n, chunk_steps=512, resync_chunks=resync)
    assert np.mean(a["removal_step"] == b["removal_step"]) > 0.99
    both = a["alive"] & b["alive"]
    e = parity.rel_err(a["state"][both], b["state"][both])
    assert np.median(e) < 1e-12, np.median(e)
