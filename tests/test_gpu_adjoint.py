"""Hand-written adjoint (mx_adjoint_step behind torch.autograd) against the
oracle's forward-mode reference derivative and against central differences.

Loss: weighted squared change of the planetesimals' semimajor axes after a
checkpointed run (4 giant cores + planetesimals with gas drag, the shape of
the adjoint workload).  Gradients w.r.t. the initial heliocentric state and
(Sigma1, gamma, C_D factor) are checked along random directions:
  * planetesimals that met a core masked out of the loss: against the
    oracle's dual-number JVP, relative error <= 1e-8, and against central
    differences of the GPU loss (recorded C_D branches replayed), <= 1e-5 at
    a step on the plateau;
  * every planetesimal in the loss, so the derivative runs through the
    Bulirsch-Stoer groups (accepted sub-steps held fixed): against the
    oracle's JVP, whose dual numbers follow its own integrator's steps,
    relative error <= 1e-6 (the two integrators' sequences agree only to the
    Bulirsch-Stoer tolerance).
"""
import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import mx, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2601_16791_gb300.autograd import Trajectory, semimajor_loss  # noqa: E402


def _setup(nsmall=300, nsteps=40, every=10, seed=4):
    w = W.adjoint_4core_50k(seed=seed, nsmall=nsmall, nsteps=nsteps, checkpoint_every=every)
    traj = Trajectory(w)
    g = w.params["gas"]
    xv0 = torch.tensor(w.xv_helio, dtype=torch.float64, device="cuda")
    gas = torch.tensor([g["sigma1_gcm2"], g["gamma"], g["cd_scale"]], dtype=torch.float64,
                       device="cuda")
    wts = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    wts[w.nbig:] = 1.0 / w.nsmall
    return w, traj, xv0, gas, wts


def _directions(w, k, rng):
    out = []
    for _ in range(k):
        dxv = np.zeros((6, w.n))
        dxv[:3] = rng.normal(0, 1e-4, (3, w.n))
        dxv[3:] = rng.normal(0, 1e-6, (3, w.n))
        dpar = np.array([17.0, 0.01, 0.01]) * rng.normal(0, 1, 3)
        out.append((dxv, dpar))
    return out


def _grad(traj, xv0, gas, wts, nsteps, every, mask=True):
    x = xv0.clone().requires_grad_(True)
    p = gas.clone().requires_grad_(True)
    L = semimajor_loss(traj, x, p, wts, nsteps, every, mask_encounters=mask)
    L.backward()
    return float(L.detach()), x.grad.detach().cpu().numpy(), p.grad.detach().cpu().numpy()


def test_adjoint_vs_oracle_jvp():
    w, traj, xv0, gas, wts = _setup()
    L, gx, gp = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every)
    ever_gpu = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever_gpu)
    # the oracle's own encounter mask
    p = orc.make_params(w.params)
    xvd, mu, rc = orc.init(p, w.nbig, w.nsmall, w.m_big, w.xv_helio)
    _, ever_o, _, _ = orc.step(p, w.nbig, xvd, mu, rc, w.rp_km, w.rhop, w.nsteps)
    assert np.array_equal(ever_o[w.nbig:], ever_gpu.cpu().numpy()[w.nbig:])
    w_small = (1.0 / w.nsmall) * (1 - ever_o[w.nbig:].astype(float))
    assert ever_o[w.nbig:].sum() > 0 and w_small.sum() > 0
    rng = np.random.default_rng(12)
    for dxv, dpar in _directions(w, 4, rng):
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, w_small,
                               w.nsteps, dxv, dpar)
        ours = float((gx * dxv).sum() + (gp * dpar).sum())
        assert abs(Lo - L) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-8 * abs(jvp), (ours, jvp)
    traj.close()


def test_adjoint_through_encounters_vs_oracle_jvp():
    w, traj, xv0, gas, wts = _setup()
    L, gx, gp = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask=False)
    _, gxm, gpm = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask=True)
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever)
    met = ever.cpu().numpy()[w.nbig:].astype(bool)
    assert met.sum() > 0
    # the bodies that met a core now carry a gradient
    assert np.abs(gx[:, w.nbig:][:, met]).max() > 0 and not np.abs(gxm[:, w.nbig:][:, met]).any()
    p = orc.make_params(w.params)
    w_small = np.full(w.nsmall, 1.0 / w.nsmall)
    rng = np.random.default_rng(13)
    for dxv, dpar in _directions(w, 4, rng):
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, w_small,
                               w.nsteps, dxv, dpar)
        ours = float((gx * dxv).sum() + (gp * dpar).sum())
        assert abs(Lo - L) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-6 * abs(jvp), (ours, jvp)
    traj.close()


def test_adjoint_vs_central_differences():
    w, traj, xv0, gas, wts = _setup(nsmall=200, nsteps=30)
    L, gx, gp = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every)
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever)
    w_eff = wts * (1.0 - ever.to(torch.float64))
    rng = np.random.default_rng(5)
    for dxv, dpar in _directions(w, 3, rng):
        ours = float((gx * dxv).sum() + (gp * dpar).sum())
        best = np.inf
        for t in (1e-1, 3e-2, 1e-2, 3e-3):
            dx_t = torch.tensor(dxv, dtype=torch.float64, device="cuda")
            dp_t = torch.tensor(dpar, dtype=torch.float64, device="cuda")
            Lp = traj.loss_at(xv0 + t * dx_t, gas + t * dp_t, w_eff, w.nsteps, w.checkpoint_every)
            Lm = traj.loss_at(xv0 - t * dx_t, gas - t * dp_t, w_eff, w.nsteps, w.checkpoint_every)
            fd = (Lp - Lm) / (2 * t)
            best = min(best, abs(fd - ours) / abs(ours))
        assert best <= 1e-5, best
    traj.close()


def test_adjoint_is_deterministic():
    w, traj, xv0, gas, wts = _setup(nsmall=150, nsteps=20)
    a = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask=False)
    b = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask=False)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    traj.close()


def test_full_size_adjoint_workload():
    """The adjoint workload at its full size: 4 cores + 50,000 planetesimals,
    2,000 steps checkpointed every 50.
      * The mean over every planetesimal that met no core: the gradient along
        16 random directions against central differences of the GPU loss
        (recorded C_D branches replayed), <= 1e-5.
      * A loss on 200 sampled planetesimals (weight 1/N on them, 0 elsewhere;
        the GPU still integrates all 50,000): against the oracle's JVP over
        the cores and that sample, which, being massless, moves as inside the
        full disk, <= 1e-8.  The other planetesimals get a zero gradient."""
    w, traj, xv0, gas, wts = _setup(nsmall=50_000, nsteps=2000, every=50)
    L, gx, gp = _grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every)
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever)
    ev = ever.cpu().numpy()[w.nbig:].astype(bool)
    assert 0 < ev.sum() < w.nsmall // 4
    w_eff = wts * (1.0 - ever.to(torch.float64))
    rng = np.random.default_rng(21)
    for dxv, dpar in _directions(w, 16, rng):
        ours = float((gx * dxv).sum() + (gp * dpar).sum())
        dx_t = torch.tensor(dxv, dtype=torch.float64, device="cuda")
        dp_t = torch.tensor(dpar, dtype=torch.float64, device="cuda")
        best = np.inf
        for t in (1e-2, 3e-2, 3e-3, 1e-1):
            Lp = traj.loss_at(xv0 + t * dx_t, gas + t * dp_t, w_eff, w.nsteps, w.checkpoint_every)
            Lm = traj.loss_at(xv0 - t * dx_t, gas - t * dp_t, w_eff, w.nsteps, w.checkpoint_every)
            best = min(best, abs((Lp - Lm) / (2 * t) - ours) / abs(ours))
            if best <= 1e-5:
                break
        assert best <= 1e-5, best
    # the sampled loss against the oracle
    quiet = np.flatnonzero(~ev)
    sel = np.sort(rng.choice(quiet, 200, replace=False))
    cols = np.concatenate([np.arange(w.nbig), w.nbig + sel])
    p = orc.make_params(w.params)
    xh = w.xv_helio[:, cols].copy()
    xv, mu, rc = orc.init(p, w.nbig, len(sel), w.m_big, xh)
    _, ever_o, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[sel], w.rhop[sel], w.nsteps)
    w_o = np.where(ever_o[w.nbig:] == 0, 1.0 / w.nsmall, 0.0)
    assert (w_o > 0).sum() >= 190
    w_s = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    w_s[torch.as_tensor(w.nbig + sel, device="cuda")] = torch.as_tensor(w_o, device="cuda")
    L2, gx2, gp2 = _grad(traj, xv0, gas, w_s, w.nsteps, w.checkpoint_every)
    rest = np.ones(w.n, dtype=bool)
    rest[cols] = False
    assert not gx2[:, rest].any()
    for dxv, dpar in _directions(w, 4, rng):
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, xh, w.rp_km[sel], w.rhop[sel], w_o, w.nsteps,
                               dxv[:, cols], dpar)
        ours = float((gx2[:, cols] * dxv[:, cols]).sum() + (gp2 * dpar).sum())
        assert abs(Lo - L2) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-8 * abs(jvp), (ours, jvp)
    traj.close()


def test_adjoint_does_not_depend_on_the_forward_tiling():
    """The forward step gives the same bits for any tiling, and the adjoint
    runs on its own tiling, so the loss and gradient are bit-identical
    whatever tile size the forward autotuner picked."""
    w, traj, xv0, gas, wts = _setup(nsmall=700, nsteps=20, every=10)
    out = []
    for tile in (64, 256, 128):
        mx.mx_set_tiling(traj.h, tile, 0)
        out.append(_grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every))
    for o in out[1:]:
        assert o[0] == out[0][0] and np.array_equal(o[1], out[0][1]) and np.array_equal(o[2], out[0][2])
    traj.close()


def test_adjoint_kept_and_recomputed_substeps_agree_bitwise():
    """The reverse of a two-body group reads the Stoermer sub-steps the
    forward kept, or recomputes them when the pool is used up: with the
    default pool, a pool of one chunk (8 slots: the first records kept, the
    rest recomputed) and no pool, the loss and gradient through the groups are
    the same to the bit."""
    w, traj, xv0, gas, wts = _setup(nsmall=300, nsteps=40, every=10)
    out = []
    for slots in (1 << 14, 8, 0):
        mx._check(mx.load().mx_adjoint_store(traj.h, slots), "mx_adjoint_store")
        out.append(_grad(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask=False))
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    mx.mx_encounter_log(traj.h, ever)
    assert ever.cpu().numpy()[w.nbig:].sum() > 0
    for o in out[1:]:
        assert o[0] == out[0][0] and np.array_equal(o[1], out[0][1]) and np.array_equal(o[2], out[0][2])
    assert np.abs(out[0][1]).max() > 0
    traj.close()


@pytest.mark.parametrize("mask", [False, True])
def test_adjoint_through_big_body_encounters_vs_oracle_jvp(mask):
    """A swarm of 1,000 embryos with 1,000 planetesimals over 30 steps, where
    embryos meet each other (groups of big bodies, every member's state from
    the group) and planetesimals meet embryos (test-particle groups with the
    whole big groups).  The gradient of the planetesimals' loss against the
    oracle's dual-number JVP, which follows its own integrator's steps:
    relative <= 1e-6.  mask=True leaves out the planetesimals that met a big
    body (mode 2: the big groups only); mask=False takes every group."""
    from paper_2601_16791_gb300.autograd import Trajectory, semimajor_loss
    w = W.semiactive_2000big_200k(nbig=1000, nsmall=1000, nsteps=30)
    w.checkpoint_every = 10
    traj = Trajectory(w)
    g = w.params["gas"]
    xv0 = torch.tensor(w.xv_helio, dtype=torch.float64, device="cuda", requires_grad=True)
    gas = torch.tensor([g["sigma1_gcm2"], g["gamma"], g["cd_scale"]], dtype=torch.float64,
                       device="cuda", requires_grad=True)
    wts = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    wts[w.nbig:] = 1.0 / w.nsmall
    L = semimajor_loss(traj, xv0, gas, wts, w.nsteps, w.checkpoint_every, mask_encounters=mask)
    L.backward()
    gx = xv0.grad.cpu().numpy()
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    nbb = mx.mx_encounter_log(traj.h, ever)
    traj.close()
    ever = ever.cpu().numpy().astype(bool)
    assert nbb > 20 and ever[:w.nbig].sum() > 20, "no big-body groups: the test is vacuous"
    w_small = np.full(w.nsmall, 1.0 / w.nsmall)
    if mask:
        w_small = w_small * (1 - ever[w.nbig:].astype(float))
    p = orc.make_params(w.params)
    rng = np.random.default_rng(17)
    for _ in range(3):
        dxv = np.zeros((6, w.n))
        dxv[:3] = rng.normal(0, 1e-4, (3, w.n))
        dxv[3:] = rng.normal(0, 1e-6, (3, w.n))
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, w.xv_helio, w.rp_km, w.rhop, w_small,
                               w.nsteps, dxv, np.zeros(3))
        ours = float((gx * dxv).sum())
        assert abs(Lo - float(L.detach())) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-6 * abs(jvp), (ours, jvp)


@pytest.mark.parametrize("mask", [True, False])
def test_semiactive_full_size_adjoint_sampled(mask):
    """The semi-active disk at full size (2,000 embryos, which meet each other
    every step, + 200,000 planetesimals), 20 steps checkpointed every 10, with
    the loss on a sample of planetesimals.  mask=True: 300 that met no embryo,
    the masked loss (mode 2: the groups of big bodies only).  mask=False: 150
    that met no embryo and 150 that did, every group differentiated (mode 1:
    thousands of test-particle groups a step, more than the adjoint's first
    record holds).  Being massless, the sample moves as inside the full disk,
    so the oracle's JVP over the embryos and the sample is the reference:
    relative <= 1e-6 (the groups run on each side's own integrator).  The
    other planetesimals get a zero gradient."""
    from paper_2601_16791_gb300.autograd import Trajectory, semimajor_loss
    w = W.semiactive_2000big_200k(nsteps=20)
    w.checkpoint_every = 10
    rng = np.random.default_rng(23)
    p = orc.make_params(w.params)
    cand = np.sort(rng.choice(w.nsmall, 400 if mask else 1500, replace=False))
    cols0 = np.concatenate([np.arange(w.nbig), w.nbig + cand])
    xv, mu, rc = orc.init(p, w.nbig, len(cand), w.m_big, w.xv_helio[:, cols0].copy())
    _, ever_o, _, _ = orc.step(p, w.nbig, xv, mu, rc, w.rp_km[cand], w.rhop[cand], w.nsteps)
    assert ever_o[:w.nbig].sum() > 100, "no big-body groups: the test is vacuous"
    met = ever_o[w.nbig:] != 0
    if mask:
        sel = cand[~met][:300]
        assert len(sel) == 300
    else:
        assert met.sum() >= 50, "too few planetesimals met an embryo: the test is vacuous"
        sel = np.sort(np.concatenate([cand[~met][:150], cand[met][:150]]))
    cols = np.concatenate([np.arange(w.nbig), w.nbig + sel])
    traj = Trajectory(w)
    g = w.params["gas"]
    xv0 = torch.tensor(w.xv_helio, dtype=torch.float64, device="cuda", requires_grad=True)
    gas = torch.tensor([g["sigma1_gcm2"], g["gamma"], g["cd_scale"]], dtype=torch.float64,
                       device="cuda", requires_grad=True)
    w_s = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    w_s[torch.as_tensor(w.nbig + sel, device="cuda")] = 1.0 / len(sel)
    L = semimajor_loss(traj, xv0, gas, w_s, w.nsteps, w.checkpoint_every, mask_encounters=mask)
    L.backward()
    gx = xv0.grad.cpu().numpy()
    ever = torch.zeros(w.n, dtype=torch.uint8, device="cuda")
    nbb = mx.mx_encounter_log(traj.h, ever)
    traj.close()
    ever = ever.cpu().numpy()
    assert nbb > 100
    assert np.array_equal(ever[w.nbig + sel] != 0, met[np.searchsorted(cand, sel)])
    rest = np.ones(w.n, dtype=bool)
    rest[cols] = False
    assert not gx[:, rest].any()
    w_o = np.full(len(sel), 1.0 / len(sel))
    xh = w.xv_helio[:, cols].copy()
    for _ in range(3):
        dxv = np.zeros((6, len(cols)))
        dxv[:3] = rng.normal(0, 1e-4, (3, len(cols)))
        dxv[3:] = rng.normal(0, 1e-6, (3, len(cols)))
        Lo, jvp = orc.jvp_loss(p, w.nbig, w.m_big, xh, w.rp_km[sel], w.rhop[sel], w_o, w.nsteps,
                               dxv, np.zeros(3))
        ours = float((gx[:, cols] * dxv).sum())
        assert abs(Lo - float(L.detach())) <= 1e-9 * abs(Lo)
        assert abs(ours - jvp) <= 1e-6 * abs(jvp), (ours, jvp)


def _raw_adjoint(h, n, nsys, xv_h0, w_host, nsteps, mode, merge=False, flush_at=None,
                 predrift=False):
    """Forward run of nsteps from the heliocentric state xv_h0 (every state
    kept), the loss of weights w_host (bodies that met a big body left out
    in modes 0 and 2, whose reverse assumes it), and its reverse through the
    C ABI: (L per system, the
    gradient w.r.t. xv_h0, d/d(params) per system, the encounter log).  With
    merge, consecutive steps are reversed with mx_adjoint_merge on; with
    flush_at = k, the cotangent after step k's reverse is also returned (read
    after mx_adjoint_flush).  With predrift, each step's pre-drift state from
    the forward run replaces the adjoint's recomputation of it."""
    mx.mx_set_state(h, xv_h0, mx.MX_COORD_HELIO, 0)
    mx.mx_encounter_log(h, None, reset=True)
    mx.mx_kick_branches(h, 1, 2 * nsteps + 2)
    seg, pre = [], []
    for _ in range(nsteps):
        z = torch.empty((6, n), dtype=torch.float64, device="cuda")
        mx.mx_get_state_device(h, z)
        seg.append(z)
        mx.mx_step(h, 1)
        if predrift:   # (recording branches keeps deferral off)
            pre.append(torch.empty((6, n), dtype=torch.float64, device="cuda"))
            mx.mx_predrift_state(h, pre[-1])
    ever = torch.zeros(n, dtype=torch.uint8, device="cuda")
    nbb = mx.mx_encounter_log(h, ever)
    wt = torch.tensor(w_host, dtype=torch.float64, device="cuda")
    if mode in (0, 2):
        wt = wt * (1.0 - ever.to(torch.float64))
    xv0 = torch.tensor(xv_h0, dtype=torch.float64, device="cuda")
    seed_f = torch.empty((6, n), dtype=torch.float64, device="cuda")
    seed_i = torch.empty((6, n), dtype=torch.float64, device="cuda")
    L = mx.mx_loss_semimajor(h, xv0, wt, seed_f, seed_i, nsys)
    mx.mx_kick_branches(h, 2)
    mx._check(mx.load().mx_adjoint_encounters(h, mode), "mx_adjoint_encounters")
    lam = seed_f.clone()
    dpar = torch.zeros(3 * nsys, dtype=torch.float64, device="cuda")
    mx.mx_adjoint_merge(h, merge)
    mid = None
    for k in reversed(range(nsteps)):
        if predrift:
            mx.mx_adjoint_step_predrift(h, seg[k], pre[k], k, lam, dpar)
        else:
            mx.mx_adjoint_step(h, seg[k], k, lam, dpar)
        if k == flush_at:
            mx.mx_adjoint_flush(h)
            mid = lam.cpu().numpy()
    grad = torch.empty((6, n), dtype=torch.float64, device="cuda")
    mx.mx_adjoint_init(h, lam, grad)
    mx.mx_adjoint_merge(h, False)
    grad += seed_i
    out = (L, grad.cpu().numpy(), dpar.cpu().numpy(), nbb, ever.cpu().numpy())
    return out if flush_at is None else out + (mid,)


def test_batched_adjoint_matches_each_system_alone():
    """Three gas disks of different sizes and gas (gamma = 1; gamma = 1.5 with
    a larger C_D factor; gamma = 1 with an inner edge at 1.5 AU and the disk's
    gravity) differentiated as
    one batched mx_system, against each differentiated alone over the same 8
    steps.  The adjoint's tiles, partial records and folds are per system, so
    with the encounter groups skipped (the masked loss) the loss, the
    gradient and the parameter cotangents are the same bits.  Through every
    group the groups' shares are summed over the batch's one work list, in
    another order than alone: relative 1e-12."""
    ws = []
    for seed, nb, ns, gam, cds, rin in ((11, 4, 3000, 1.0, 1.0, None), (12, 3, 2000, 1.5, 1.3, None),
                                         (13, 5, 2500, 1.0, 0.8, 1.5)):
        w = W.gas_4core_100k(seed=seed, nbig=nb, nsmall=ns, nsteps=8)
        w.params["gas"].update(gamma=gam, cd_scale=cds)
        if rin is not None:   # the disk's gravity, the gamma = 1 edge form
            w.params["gas"].update(r_in_au=rin, disk_gravity=True)
        ws.append(w)
    nsteps = 8
    rng = np.random.default_rng(29)
    b = mx.Batch(ws)
    off = b.offsets
    xv_all = np.concatenate([w.xv_helio for w in ws], axis=1)
    w_all = rng.uniform(0.5, 1.5, b.n) / b.n
    for i, w in enumerate(ws):   # the loss over the planetesimals only
        w_all[off[i]:off[i] + w.nbig] = 0.0
    out = {}
    for mode in (0, 1):
        out[mode] = _raw_adjoint(b.h, b.n, len(ws), xv_all, w_all, nsteps, mode)
    b.close()
    met = 0
    for i, w in enumerate(ws):
        s = mx.System(w)
        sl = slice(off[i], off[i + 1])
        for mode in (0, 1):
            L, g, dp, nbb, ever = _raw_adjoint(s.h, w.n, 1, w.xv_helio, w_all[sl], nsteps, mode)
            Lb, gb, dpb, _, everb = out[mode]
            assert nbb == 0, "big bodies met: mode 0 does not apply"
            assert np.array_equal(ever, everb[sl])
            met += int(ever.sum())
            if mode == 0:
                assert Lb[i] == L[0]
                assert np.array_equal(gb[:, sl], g)
                assert np.array_equal(dpb[3 * i:3 * i + 3], dp)
            else:
                assert abs(Lb[i] - L[0]) <= 1e-15 * abs(L[0])
                assert np.abs(gb[:, sl] - g).max() <= 1e-12 * np.abs(g).max()
                assert np.allclose(dpb[3 * i:3 * i + 3], dp, rtol=1e-12, atol=0)
            assert np.abs(g).max() > 0 and np.abs(dp).max() > 0
        s.close()
    assert met > 0, "no planetesimal met a core: the groups' case is vacuous"


@pytest.mark.parametrize("disk", ["gas", "semiactive"])
def test_merged_reverse_matches_unmerged(disk):
    """mx_adjoint_merge: the pair pass of each step's first half kick taken
    with the previous step's last one (same positions, summed cotangents)
    against separate passes, with the groups skipped or every group
    differentiated.  The gas disk (4 cores + 3,000 planetesimals, 12 steps)
    and 1,000 embryos + 2,000 planetesimals (20 steps), whose embryos meet
    (mode 2 instead of 0).
    The sums are the same terms grouped otherwise: relative 1e-12.  A flush
    after step 6's reverse (mx_adjoint_flush) gives the unmerged cotangent
    there, and the run goes on merged to the same gradient."""
    if disk == "gas":
        nsteps = 12
        w = W.adjoint_4core_50k(seed=4, nsmall=3000, nsteps=nsteps)
        modes = (0, 1)
    else:
        nsteps = 20
        w = W.semiactive_2000big_200k(nbig=1000, nsmall=2000, nsteps=nsteps)
        modes = (2, 1)
    s = mx.System(w)
    wts = np.zeros(w.n)
    wts[w.nbig:] = 1.0 / w.nsmall
    for mode in modes:
        L0, g0, d0, nbb, _, mid0 = _raw_adjoint(s.h, w.n, 1, w.xv_helio, wts, nsteps, mode,
                                                flush_at=6)
        L1, g1, d1, _, _, mid1 = _raw_adjoint(s.h, w.n, 1, w.xv_helio, wts, nsteps, mode,
                                              merge=True, flush_at=6)
        assert (nbb == 0) == (disk == "gas")
        assert L0[0] == L1[0]
        assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max()
        assert np.allclose(d1, d0, rtol=1e-12, atol=0)
        for r in range(6):
            assert np.abs(mid1[r] - mid0[r]).max() <= 1e-12 * np.abs(mid0[r]).max()
        assert np.abs(g0).max() > 0
        assert (np.abs(d0).max() > 0) == (disk == "gas")   # no gas on the embryos' disk
    s.close()


@pytest.mark.parametrize("disk", ["gas", "semiactive"])
def test_adjoint_from_the_forward_predrift_state(disk):
    """mx_adjoint_step_predrift takes each step's pre-drift state (x2, v1)
    from the forward run (mx_predrift_state) instead of recomputing the first
    half kick and jump: the same gradient, with the groups skipped or every
    group differentiated (relative 1e-12; the recomputation repeats the
    forward's arithmetic).  mx_predrift_state refuses after a step with
    deferral on, whose deferred bodies the catch-up drifts."""
    if disk == "gas":
        nsteps = 12
        w = W.adjoint_4core_50k(seed=4, nsmall=3000, nsteps=nsteps)
        modes = (0, 1)
    else:
        nsteps = 10
        w = W.semiactive_2000big_200k(nbig=1000, nsmall=2000, nsteps=nsteps)
        modes = (2, 1)
    s = mx.System(w)
    wts = np.zeros(w.n)
    wts[w.nbig:] = 1.0 / w.nsmall
    for mode in modes:
        L0, g0, d0, _, _ = _raw_adjoint(s.h, w.n, 1, w.xv_helio, wts, nsteps, mode)
        L1, g1, d1, _, _ = _raw_adjoint(s.h, w.n, 1, w.xv_helio, wts, nsteps, mode, predrift=True)
        assert L0[0] == L1[0]
        assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max()
        assert np.allclose(d1, d0, rtol=1e-12, atol=0)
    if disk == "gas":   # deferral on (the default window, no branch recording)
        mx.mx_kick_branches(s.h, 0)
        mx.mx_set_state(s.h, w.xv_helio, mx.MX_COORD_HELIO, 0)
        mx.mx_step(s.h, 1)
        buf = torch.empty((6, w.n), dtype=torch.float64, device="cuda")
        with pytest.raises(mx.MxError):
            mx.mx_predrift_state(s.h, buf)
    s.close()
