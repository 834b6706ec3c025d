"""Bounded device waits give up with an error status, and the context stays usable.

The task launches (glisse_advance's particle map, the differentiable forward
pass and the reverse sweep) order each 32-slot group's sub-chunks with a
device-side wait on the group's counter, limited to seconds of polling.  No
real run should ever reach that limit, so glisse_selftest_wait runs the same
kernels on two groups whose first sub-chunks no task runs, with the limit cut
to a few thousand polls: every wait must give up, the kernel must report
GLISSE_E_TIMEOUT through its status word and return, and the GPU must go on
computing the same results as before.  Nothing here faults or hangs the GPU.
"""
import time

import numpy as np
import pytest

import glisse_inputs as gi

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


def _short_run(G):
    w = gi.make("tiny", n=96)
    sim = G.Simulation(w["star_mass"], w["planets"], w["particles"], w["dt"], launch_mode=G.GLISSE_LAUNCH_TASKS)
    sim.advance(256)
    out = sim.read()
    sim.close()
    return out


@pytest.mark.parametrize("which", ["GLISSE_WAIT_PARTICLE_TASKS", "GLISSE_WAIT_DIFF_FORWARD",
                                   "GLISSE_WAIT_DIFF_BACKWARD"])
def test_bounded_wait_gives_up_and_the_context_stays_usable(G, which):
    before = _short_run(G)
    t0 = time.perf_counter()
    status = G.glisse_selftest_wait(getattr(G, which), polls=4000)
    elapsed = time.perf_counter() - t0
    assert status == G.GLISSE_E_TIMEOUT, status
    assert elapsed < 5.0, elapsed  # 4000 polls of ~64 ns; seconds would mean the limit was ignored
    after = _short_run(G)
    for k in ("state", "removal_step", "removal_reason"):
        np.testing.assert_array_equal(after[k], before[k], err_msg=k)
