"""Tangent and adjoint maps on the GPU (glisse_diff_*), through the C ABI.

Checked against the oracle's complex-step tangent map, central finite
differences (h = 1e-7 AU), the symplectic structure of the Jacobian, the
dot-product identity <g, J t> = <J^T g, t> between the two kernels, the
gradient of the tangent-growth indicator against the oracle's difference
quotients and the GPU's own, and the
independence of the gradient from the checkpoint interval; the
torch.autograd.Function is checked against the tangent kernel.
"""
import numpy as np
import pytest

import glisse_inputs as gi
import parity

pytestmark = pytest.mark.gpu

OMEGA = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_03484_gb300 as G

    G._build.build()
    G.load()
    return G


def _workload(n):
    w = gi.make("diff", n=n)
    return w, w["planets"], w["particles"]


def _cuda(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_jacobian(G, pl, s0, dt, n_steps, K=256):
    import torch

    n = s0.shape[0]
    dm = G.DiffMap(1.0, pl, n, dt, n_steps, K)
    e = np.zeros((6, n, 6))
    for c in range(6):
        e[c, :, c] = 1.0
    s1, t1, growth, rstep, reason = dm.forward(_cuda(s0), _cuda(e))
    dm.close()
    J = t1.cpu().numpy().transpose(1, 2, 0)  # [n][6 out][6 in]
    return s1.cpu().numpy(), J, rstep.cpu().numpy(), reason.cpu().numpy()


def test_tangent_matches_oracle_complex_step(G, orc):
    """64 particles of the 65536-particle differentiation workload over 10^4 steps."""
    w, pl, s0 = _workload(64)
    n = 10_000
    s1, J, rstep, reason = gpu_jacobian(G, pl, s0, w["dt"], n)
    _, log, _ = orc.planet_wh(1.0, pl, w["dt"], n)
    rc = orc.rcrit(1.0, pl)
    Jo = orc.particles_jacobian(1.0, pl[:, 0], log, w["dt"], s0, rc, 1000.0)
    o = orc.run(1.0, pl, s0, w["dt"], n)
    np.testing.assert_array_equal(rstep, o["removal_step"])
    # relative to each particle's Jacobian scale; chaotic particles amplify rounding in J as in the state
    err = np.abs(J - Jo).max(axis=(1, 2)) / np.abs(Jo).max(axis=(1, 2))
    regular = (o["closest"] >= 25.0) & (o["removal_step"] < 0)
    print("tangent rel err: regular max", err[regular].max(), "all median", np.median(err))
    assert regular.sum() > 10
    assert err[regular].max() < 1e-8
    assert np.median(err) < 1e-8


def test_jacobian_is_symplectic(G):
    w, pl, s0 = _workload(128)
    _, J, rstep, _ = gpu_jacobian(G, pl, s0, w["dt"], 3000)
    for p in np.where(rstep < 0)[0]:
        M = J[p].T @ OMEGA @ J[p]
        assert np.abs(M - OMEGA).max() < 1e-12 * max(1.0, np.abs(J[p]).max() ** 2), p


def test_tangent_matches_central_differences(G):
    """Every column of the Jacobian (positions and velocities) against central differences of the
    map: h = 1e-7 AU for positions and 1e-8 AU/yr for velocities (about 4e-9 and 8e-9 of the
    coordinates).  Such a quotient is good to about eps |x| / h (rounding, ~3e-8 here) plus
    h^2 times the third derivative, relative to the Jacobian's scale."""
    w, pl, s0 = _workload(32)
    n = 2000
    _, J, rstep, _ = gpu_jacobian(G, pl, s0, w["dt"], n)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n)
    scale = np.abs(J).max(axis=(1, 2))
    for c in range(6):
        h = 1e-7 if c < 3 else 1e-8
        e = np.zeros_like(s0)
        e[:, c] = h
        sp = dm.forward(_cuda(s0 + e))[0].cpu().numpy()
        sm = dm.forward(_cuda(s0 - e))[0].cpu().numpy()
        fd = (sp - sm) / (2 * h)
        err = np.abs(fd - J[:, :, c]).max(axis=1) / scale
        print("column", c, "max", err[rstep < 0].max(), "median", np.median(err[rstep < 0]))
        assert err[rstep < 0].max() < 1e-5, (c, err.max())
    dm.close()


def test_adjoint_is_the_transpose_of_the_tangent(G):
    """<g, J t> = <J^T g, t> per particle, with J t from the forward kernel and J^T g from the backward one."""
    import torch

    w, pl, s0 = _workload(2048)
    n = 3000
    rng = np.random.default_rng(5)
    t = rng.normal(size=s0.shape)
    g = rng.normal(size=s0.shape)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 128)
    s1, t1, _, rstep, _ = dm.forward(_cuda(s0), _cuda(t[None]))
    gT = dm.backward(_cuda(g)).cpu().numpy()
    dm.close()
    Jt = t1[0].cpu().numpy()
    lhs = (g * Jt).sum(axis=1)
    rhs = (gT * t).sum(axis=1)
    scale = np.abs(g).sum(axis=1) * np.abs(Jt).max(axis=1) + np.abs(gT).max(axis=1) * np.abs(t).sum(axis=1)
    rel = np.abs(lhs - rhs) / scale
    print("dot-product test: max", rel.max(), "removed", int((rstep.cpu().numpy() >= 0).sum()))
    assert rel.max() < 1e-11


def test_gradient_independent_of_checkpoint_interval(G):
    """Interior kicks merge inside a checkpoint segment and stay half kicks at its
    boundaries, so the trajectory, and with it the gradient, depends on K only by
    rounding (chaotic particles amplify it, as they do state differences)."""
    w, pl, s0 = _workload(256)
    n = 700
    g = np.random.default_rng(6).normal(size=s0.shape)
    outs = []
    for K in (1, 7, 256, 1000):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K)
        dm.forward(_cuda(s0))
        outs.append(dm.backward(_cuda(g)).cpu().numpy())
        dm.close()
    for o in outs[1:]:
        rel = np.abs(o - outs[0]).max(axis=1) / np.abs(outs[0]).max(axis=1)
        assert np.median(rel) < 1e-12 and np.quantile(rel, 0.99) < 1e-8, (np.median(rel), rel.max())
    # the same K twice: bit-identical (the backward pass recomputes the forward trajectory exactly)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 7)
    dm.forward(_cuda(s0))
    again = dm.backward(_cuda(g)).cpu().numpy()
    dm.close()
    np.testing.assert_array_equal(again, outs[1])


def test_tape_mode_equals_one_recomputed_segment(G):
    """checkpoint_every = 0 records every step in the forward pass; the backward pass then
    skips the recompute.  With a single segment (K = n) the recompute produces the same
    record, so the two gradients are bit-identical."""
    w, pl, s0 = _workload(512)
    n = 900
    g = np.random.default_rng(8).normal(size=s0.shape)
    outs = []
    for K in (0, n):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K)
        s1, _, _, rstep, _ = dm.forward(_cuda(s0))
        outs.append((s1.cpu().numpy(), dm.backward(_cuda(g)).cpu().numpy(), rstep.cpu().numpy()))
        dm.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert (outs[0][2] >= 0).sum() > 0  # removals on the way (frozen-state derivatives on the tape)
    # a tape written by a forward pass that carries a tangent (another kernel, the same arithmetic
    # for the state and the record) gives the same bits too
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 0)
    s1, _, _, _, _ = dm.forward(_cuda(s0), _cuda(_seed(s0)[None]))
    np.testing.assert_array_equal(s1.cpu().numpy(), outs[0][0])
    np.testing.assert_array_equal(dm.backward(_cuda(g)).cpu().numpy(), outs[0][1])
    dm.close()


def test_autograd_function(G):
    import torch

    w, pl, s0 = _workload(64)
    n = 1000
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n)
    x = _cuda(s0).requires_grad_(True)
    s1, growth = G.glisse_map().apply(x, dm)
    wgt = _cuda(np.random.default_rng(7).normal(size=s0.shape))
    (s1 * wgt).sum().backward()
    _, J, rstep, _ = gpu_jacobian(G, pl, s0, w["dt"], n)
    ref = np.einsum("pij,pi->pj", J, wgt.cpu().numpy())
    got = x.grad.cpu().numpy()
    err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert err.max() < 1e-10, err.max()
    assert torch.isfinite(growth).all() and growth.requires_grad  # differentiable too (tests below)
    dm.close()


def test_removed_particles_have_frozen_state_derivatives(G, orc):
    """Particles removed at t_0 map to themselves: identity Jacobian and gradient."""
    w, pl, s0 = _workload(16)
    rc = orc.rcrit(1.0, pl)
    s0 = s0.copy()
    s0[0, :3] = pl[2, 1:4] + [0.3 * rc[2], 0, 0]
    s0[0, 3:] = pl[2, 4:7]
    s1, J, rstep, reason = gpu_jacobian(G, pl, s0, w["dt"], 200)
    assert rstep[0] == 0 and reason[0] == 3
    np.testing.assert_array_equal(s1[0], s0[0])
    np.testing.assert_array_equal(J[0], np.eye(6))


# ---------------------------------------------------------------------------
# gradient of the tangent-growth indicator (glisse_diff_growth_gradient)
# ---------------------------------------------------------------------------
def _seed(s0):
    r = s0[:, :3] / np.linalg.norm(s0[:, :3], axis=1, keepdims=True)
    v = s0[:, 3:] / np.linalg.norm(s0[:, 3:], axis=1, keepdims=True)
    return np.ascontiguousarray(np.hstack([r, v]) / 2**0.5)


def test_growth_gradient_matches_oracle(G, orc):
    """d log(|J t0| / |t0|) / d state0 at fixed t0 on 32 particles over 2000 steps,
    against the oracle's Richardson-extrapolated difference quotients of its
    complex-step growth (good to ~1e-8 relative on regular orbits)."""
    w, pl, s0 = _workload(32)
    n = 2000
    t0 = _seed(s0)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n)
    grad, growth = dm.growth_gradient(_cuda(s0), _cuda(t0))
    _, _, g_fwd, rstep, _ = dm.forward(_cuda(s0), _cuda(t0[None]))
    # the value part of the dual tangent is the forward pass's tangent, bit for bit
    np.testing.assert_array_equal(growth.cpu().numpy(), g_fwd.cpu().numpy())
    dm.close()
    _, log, _ = orc.planet_wh(1.0, pl, w["dt"], n)
    rc = orc.rcrit(1.0, pl)
    ref, err, ok = orc.growth_gradient(1.0, pl[:, 0], log, w["dt"], s0, t0, rc, 1000.0)
    o = orc.run(1.0, pl, s0, w["dt"], n)
    regular = ok & (o["closest"] >= 25.0) & (o["removal_step"] < 0)
    got = grad.cpu().numpy()
    rel = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
    print("growth gradient rel err: regular max", rel[regular].max(), "median", np.median(rel), "regular",
          int(regular.sum()))
    assert regular.sum() >= 16
    assert rel[regular].max() < 1e-6


@pytest.mark.parametrize("K", [0, 128])
def test_launch_shapes_are_bit_identical(G, K):
    """The task launches of the forward and backward passes (32-particle groups over sub-chunks
    of the run, the state, tangent and cotangent handed on through memory) equal the plain
    launches bit for bit: states, the tangent, the growth indicator, removal steps and J^T g, in
    tape mode (sub-chunks of one segment) and with checkpoints; eccentric particles among them
    are removed part-way."""
    w, pl, s0 = _workload(2000)
    ecc = gi.make("eccentric", n=1000)["particles"]
    s0 = np.concatenate([s0, ecc])
    n = 700
    rng = np.random.default_rng(7)
    g = _cuda(rng.normal(size=s0.shape))
    t0 = _cuda(rng.normal(size=(1,) + s0.shape))
    outs = []
    for m in (G.GLISSE_LAUNCH_PLAIN, G.GLISSE_LAUNCH_TASKS, G.GLISSE_LAUNCH_AUTO):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K, launch_mode=m)
        s1t, tan1, growth, _, _ = dm.forward(_cuda(s0), t0)
        s1, _, _, rstep, reason = dm.forward(_cuda(s0))
        outs.append([x.cpu().numpy() for x in (s1t, tan1, growth, s1, rstep, reason, dm.backward(g))])
        dm.close()
    assert (outs[0][4] >= 0).sum() > 10
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            np.testing.assert_array_equal(x, y)


def test_auto_storage_picks_the_record_when_it_fits(G):
    """GLISSE_DIFF_AUTO on a small map resolves to tape mode (its record is far below half the
    free memory) and gives what explicit tape mode gives, bit for bit."""
    import torch

    w, pl, s0 = _workload(512)
    n = 700
    g = _cuda(np.random.default_rng(4).normal(size=s0.shape))
    outs = []
    for k in (G.GLISSE_DIFF_AUTO, 0):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, k)
        assert dm.checkpoint_every == 0 and dm.tape
        s1 = dm.forward(_cuda(s0))[0]
        outs.append((s1.cpu().numpy(), dm.backward(g).cpu().numpy()))
        dm.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 128)
    assert dm.checkpoint_every == 128 and not dm.tape
    dm.close()


def test_growth_gradient_long_horizon(G, orc):
    """The gradient of the growth indicator on 128 particles over the differentiation workload's
    full 10^4 steps, by both GPU routes (forward mode, and the reverse sweep after a
    checkpointed forward pass), against the oracle's difference quotients, on orbits that never
    came within 5 R_crit.  Over 10^4 steps the growth is strongly nonlinear in the state and
    the quotients are the limit: with steps of 1e-5 and 1e-6 AU (Richardson-extrapolated) they
    differ from each other by a median 4e-7 and at most 4e-6 of the gradient, so the GPU is held
    to 1e-5 of each particle's gradient scale (median 1e-6) against the 1e-6 AU quotients."""
    w, pl, s0 = _workload(128)
    n = 10_000
    t0 = _seed(s0)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 256)
    fwd, _ = dm.growth_gradient(_cuda(s0), _cuda(t0))
    _, tan1, _, _, _ = dm.forward(_cuda(s0), _cuda(t0[None]))
    rev, _ = dm.backward_growth(None, _cuda(np.ones(len(s0))), tan1[0])
    dm.close()
    _, log, _ = orc.planet_wh(1.0, pl, w["dt"], n)
    rc = orc.rcrit(1.0, pl)
    ref, _, ok = orc.growth_gradient(1.0, pl[:, 0], log, w["dt"], s0, t0, rc, 1000.0, h_pos=1e-6, h_vel=1e-7)
    o = orc.run(1.0, pl, s0, w["dt"], n)
    scale = np.abs(ref).max(axis=1)
    good = ok & (o["closest"] >= 25.0) & (o["removal_step"] < 0)
    for name, got in (("forward", fwd.cpu().numpy()), ("reverse", rev.cpu().numpy())):
        rel = np.abs(got - ref).max(axis=1) / scale
        print(name, "growth gradient over 1e4 steps: max", rel[good].max(), "median", np.median(rel[good]),
              "compared", int(good.sum()))
        assert rel[good].max() < 1e-5 and np.median(rel[good]) < 1e-6
    assert good.sum() >= 48


def test_growth_gradient_gives_the_directional_derivative(G):
    """grad . a against difference quotients of the GPU's own growth along a random a."""
    w, pl, s0 = _workload(128)
    n = 1000
    t0 = _seed(s0)
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n)
    grad, g0 = dm.growth_gradient(_cuda(s0), _cuda(t0))
    a = np.random.default_rng(8).normal(size=s0.shape) * [1e-5, 1e-5, 1e-5, 1e-6, 1e-6, 1e-6]
    d, same = [], None
    _, _, _, r0, _ = dm.forward(_cuda(s0), _cuda(t0[None]))
    r0 = r0.cpu().numpy()
    for hh in (1.0, 0.5):
        gs = []
        for sg in (1.0, -1.0):
            _, _, g, rs, _ = dm.forward(_cuda(s0 + sg * hh * a), _cuda(t0[None]))
            gs.append(g.cpu().numpy())
            eq = rs.cpu().numpy() == r0
            same = eq if same is None else same & eq
        d.append((gs[0] - gs[1]) / (2 * hh))
    dm.close()
    fd = (4 * d[1] - d[0]) / 3
    pred = (grad.cpu().numpy() * a).sum(axis=1)
    scale = np.abs(grad.cpu().numpy() * a).sum(axis=1)
    rel = np.abs(pred - fd) / scale
    print("directional: max", rel[same].max(), "median", np.median(rel[same]))
    assert same.sum() > 100
    assert np.median(rel[same]) < 1e-7 and rel[same].max() < 1e-4


def test_autograd_growth_gradient(G):
    """(s1 . w + growth).sum() through glisse_map() with the default seed (unit
    vectors along r and v, whose dependence on the state is part of the
    gradient), against difference quotients of the same loss."""
    import torch

    w, pl, s0 = _workload(64)
    n = 1000
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n)
    wgt = _cuda(np.random.default_rng(9).normal(size=s0.shape))
    x = _cuda(s0).requires_grad_(True)
    s1, growth = G.glisse_map().apply(x, dm)
    assert growth.requires_grad
    ((s1 * wgt).sum(dim=1) + growth).sum().backward()
    got = x.grad.cpu().numpy()

    def loss(xx):
        y, _, g, rs, _ = dm.forward(xx, G._growth_seed(xx).contiguous())
        return ((y * wgt).sum(dim=1) + g).cpu().numpy(), rs.cpu().numpy()

    a = np.random.default_rng(10).normal(size=s0.shape) * [1e-5, 1e-5, 1e-5, 1e-6, 1e-6, 1e-6]
    base, r0 = loss(_cuda(s0))
    d, same = [], np.ones(len(s0), dtype=bool)
    for hh in (1.0, 0.5):
        lp, rp = loss(_cuda(s0 + hh * a))
        lm, rm = loss(_cuda(s0 - hh * a))
        same &= (rp == r0) & (rm == r0)
        d.append((lp - lm) / (2 * hh))
    dm.close()
    fd = (4 * d[1] - d[0]) / 3
    pred = (got * a).sum(axis=1)
    rel = np.abs(pred - fd) / np.abs(got * a).sum(axis=1)
    print("autograd growth: max", rel[same].max(), "median", np.median(rel[same]))
    assert same.sum() > 50
    assert np.median(rel[same]) < 1e-7 and rel[same].max() < 1e-4


def test_growth_gradient_of_particle_removed_at_t0(G, orc):
    w, pl, s0 = _workload(8)
    rc = orc.rcrit(1.0, pl)
    s0 = s0.copy()
    s0[0, :3] = pl[2, 1:4] + [0.3 * rc[2], 0, 0]
    s0[0, 3:] = pl[2, 4:7]
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], 300)
    grad, growth = dm.growth_gradient(_cuda(s0), _cuda(_seed(s0)))
    dm.close()
    assert growth[0].item() == 0.0
    np.testing.assert_array_equal(grad[0].cpu().numpy(), np.zeros(6))
    assert np.isfinite(grad.cpu().numpy()).all() and np.abs(grad[1:].cpu().numpy()).max() > 0


def test_reverse_growth_sweep_matches_forward_mode(G):
    """glisse_diff_backward_growth (one reverse sweep of the map extended by its
    tangent, dual-number adjoints) against the forward-mode growth gradient plus
    the plain adjoint: J^T g1 + gg dg/dx0, and gg (J^T (J t0)/|J t0|^2 - t0/|t0|^2)."""
    import torch

    w, pl, s0 = _workload(256)
    n = 1500
    t0 = _seed(s0)
    rng = np.random.default_rng(11)
    g1 = _cuda(rng.normal(size=s0.shape))
    gg = _cuda(rng.normal(size=len(s0)))
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, 128)
    _, tan1, _, rstep, _ = dm.forward(_cuda(s0), _cuda(t0[None]))
    gs_rev, gt_rev = dm.backward_growth(g1, gg, tan1[0])
    H, _ = dm.growth_gradient(_cuda(s0), _cuda(t0))
    ref_s = dm.backward(g1) + gg[:, None] * H
    tn = tan1[0]
    u = tn / (tn * tn).sum(dim=1, keepdim=True)
    tt = _cuda(t0)
    ref_t = dm.backward((gg[:, None] * u).contiguous()) - gg[:, None] * tt / (tt * tt).sum(dim=1, keepdim=True)
    dm.close()
    a, b = gs_rev.cpu().numpy(), ref_s.cpu().numpy()
    rel_s = np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)
    c, d = gt_rev.cpu().numpy(), ref_t.cpu().numpy()
    rel_t = np.abs(c - d).max(axis=1) / np.maximum(np.abs(d).max(axis=1), 1e-300)
    print("reverse vs forward mode: state median", np.median(rel_s), "max", rel_s.max(), "seed median",
          np.median(rel_t), "max", rel_t.max(), "removed", int((rstep.cpu().numpy() >= 0).sum()))
    assert np.median(rel_s) < 1e-11 and np.median(rel_t) < 1e-11
    assert np.mean(rel_s < 1e-8) > 0.95 and np.mean(rel_t < 1e-8) > 0.95


def test_autograd_growth_tape_mode_matches_checkpoints(G):
    """Tape mode takes the forward-mode route for the growth; the gradient agrees with
    the checkpointed reverse sweep."""
    import torch

    w, pl, s0 = _workload(64)
    n = 800
    out = []
    for K in (100, 0):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K)
        x = _cuda(s0).requires_grad_(True)
        s1, growth = G.glisse_map().apply(x, dm)
        (s1.sum(dim=1) + 2.0 * growth).sum().backward()
        out.append(x.grad.cpu().numpy())
        dm.close()
    rel = np.abs(out[0] - out[1]).max(axis=1) / np.abs(out[1]).max(axis=1)
    assert np.median(rel) < 1e-11 and rel.max() < 1e-7, (np.median(rel), rel.max())


def test_reverse_growth_sweep_needs_a_tangent_and_checkpoints(G):
    import torch

    w, pl, s0 = _workload(8)
    t = _cuda(_seed(s0))
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], 100, 50)
    with pytest.raises(RuntimeError):
        dm.backward_growth(None, None, t)  # no forward call yet
    dm.forward(_cuda(s0))
    with pytest.raises(RuntimeError):
        dm.backward_growth(None, None, t)  # the forward call carried no tangent
    dm.close()
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], 100, 0)
    dm.forward(_cuda(s0), t[None])
    with pytest.raises(RuntimeError):
        dm.backward_growth(None, None, t)  # tape mode without tangent 0 in the record
    dm.close()
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], 100, G.GLISSE_DIFF_TAPE_TANGENT)
    assert dm.checkpoint_every == G.GLISSE_DIFF_TAPE_TANGENT and dm.tape and dm.reverse_growth
    dm.forward(_cuda(s0))
    with pytest.raises(RuntimeError):
        dm.backward_growth(None, None, t)  # the forward call wrote no tangent rows
    dm.forward(_cuda(s0), t[None])
    dm.backward_growth(None, None, t)
    dm.close()


def test_tangent_tape_gives_the_recomputed_growth_gradient(G):
    """GLISSE_DIFF_TAPE_TANGENT keeps tangent 0 in the forward call's record of every step, so
    the growth gradient's reverse sweep recomputes nothing.  With one checkpoint segment
    (K = n) the recompute writes the same rows, so the two routes give the same bits: the
    growth sweep's state and seed gradients, and the plain adjoint, removals included."""
    w, pl, s0 = _workload(512)
    n = 900
    t0 = _seed(s0)
    rng = np.random.default_rng(11)
    g = rng.normal(size=s0.shape)
    gg = rng.normal(size=len(s0))
    outs = []
    for K in (G.GLISSE_DIFF_TAPE_TANGENT, n):
        dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K)
        s1, tan1, _, rstep, _ = dm.forward(_cuda(s0), _cuda(t0[None]))
        gs, gt = dm.backward_growth(_cuda(g), _cuda(gg), tan1[0])
        jtg = dm.backward(_cuda(g))
        outs.append([x.cpu().numpy() for x in (s1, tan1[0], gs, gt, jtg, rstep)])
        dm.close()
    for a, b, name in zip(outs[0], outs[1], ("state1", "J t0", "growth sweep lx", "growth sweep lt", "J^T g",
                                             "removal step")):
        np.testing.assert_array_equal(a, b, err_msg=name)
    assert (outs[0][5] >= 0).sum() > 0  # removals on the way


@pytest.mark.parametrize("K", [256, 0])
def test_forward_pass_reproduces_the_map(G, orc, K):
    """The differentiable forward pass (its own drift arithmetic: one Halley step from the
    FP32 root, the G-functions from two series and their recurrence; half kicks at the
    checkpoint boundaries) meets the plain map's parity criteria against the oracle:
    256 particles over 10^4 steps, with checkpoints and in tape mode."""
    import parity

    w, pl, s0 = _workload(256)
    n = 10_000
    dm = G.DiffMap(1.0, pl, len(s0), w["dt"], n, K)
    s1, _, _, rstep, reason = dm.forward(_cuda(s0))
    dm.close()
    rs = rstep.cpu().numpy()
    g = {"state": s1.cpu().numpy(), "alive": rs < 0, "removal_step": rs, "removal_reason": reason.cpu().numpy()}
    base = orc.run(1.0, pl, s0, w["dt"], n)
    runs = [orc.run(1.0, pl, p, w["dt"], n) for p in parity.perturbed_inputs(s0)]
    runs.append(orc.run(1.0, parity.perturbed_planets(pl), s0, w["dt"], n))
    sens, unstable = parity.sensitivity(base, runs)
    rep = parity.compare(g, base, n, sens, unstable)
    print(rep)
    parity.assert_parity(rep)
