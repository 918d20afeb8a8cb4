"""Differentiable runs of the hybrid step: a torch.autograd.Function whose
backward is the library's hand-written adjoint (mx_adjoint_step), with the
state checkpointed every k steps and each segment recomputed before its
reverse sweep.

The loss is the weighted squared change of semimajor axes,
    L = sum_j w_j (a_final,j - a_initial,j)^2,
with a from the heliocentric state (mx_loss_semimajor).  A planetesimal's
close encounters are differentiated through the Bulirsch-Stoer groups of the
step, with the accepted sub-steps and extrapolation rows held fixed (the
adjoint's k_adj_bs.cu).  With mask_encounters=True (the default), bodies
flagged for an encounter in any step get weight 0 instead, and the adjoint
skips the test-particle groups (mx_adjoint_encounters): the derivative is
exact for that loss, since those planetesimals are massless, and costs about
as much as the forward step, where differentiating the groups costs their
recorded Bulirsch-Stoer integration and its reverse.  Groups of big bodies
(big-big encounters) are always differentiated: every body feels them.  The
k switch of the drag coefficient is
recorded in the forward run and replayed in the recomputation, so the
reverse sweep sees the branches the forward run took.  Consecutive steps are
reversed with mx_adjoint_merge on: the pair pass of a step's first half kick
joins that of the previous step's last half kick, at the same positions.  The
recomputation keeps each step's pre-drift state (mx_predrift_state), so the
adjoint does not recompute the first half kick (mx_adjoint_step_predrift).

Inputs: the initial heliocentric state (6 x N float64 CUDA tensor) and the
gas parameters (sigma1 [g/cm^2], gamma, cd_scale) as a 3-vector.
"""
from __future__ import annotations

import torch

from . import mx


def _dev(t):
    return t.contiguous()


class Trajectory:
    """An mx_system kept for differentiable runs of one workload."""

    def __init__(self, workload, stream=None):
        self.w = workload
        self.sys = mx.System(workload, stream)
        self.h = self.sys.h
        self.n = workload.n

    def run(self, xv_helio0, gas, nsteps, every, record=True, replay=False, keep=True):
        """Forward run from xv_helio0 with gas parameters; returns the
        checkpoints [(step, state)] and the encounter mask (N bytes)."""
        mx.mx_set_gas_params(self.h, 0, float(gas[0]), float(gas[1]), float(gas[2]))
        mx.mx_set_state(self.h, xv_helio0.detach().cpu().numpy(), mx.MX_COORD_HELIO, 0)
        mx.mx_encounter_log(self.h, None, reset=True)
        if record:
            mx.mx_kick_branches(self.h, 1, 2 * nsteps + 2)
        elif replay:
            mx.mx_kick_branches(self.h, 2)
        ckpts = []
        for start in range(0, nsteps, every):
            if keep:
                ck = torch.empty((6, self.n), dtype=torch.float64, device="cuda")
                mx.mx_get_state_device(self.h, ck)
                ckpts.append((start, ck))
            mx.mx_step(self.h, min(every, nsteps - start))
        ever = torch.zeros(self.n, dtype=torch.uint8, device="cuda")
        nbb = mx.mx_encounter_log(self.h, ever, reset=False)
        return ckpts, ever, nbb

    def loss(self, xv_helio0, w_eff):
        """Loss at the current state and its seeds (final DH, initial helio)."""
        seed_f = torch.empty((6, self.n), dtype=torch.float64, device="cuda")
        seed_i = torch.empty((6, self.n), dtype=torch.float64, device="cuda")
        L = mx.mx_loss_semimajor(self.h, _dev(xv_helio0), _dev(w_eff), seed_f, seed_i)
        return float(L[0]), seed_f, seed_i

    def loss_at(self, xv_helio0, gas, w_eff, nsteps, every):
        """Loss of a run that replays the recorded branches (finite differences)."""
        self.run(xv_helio0, gas, nsteps, every, record=False, replay=True, keep=False)
        return self.loss(xv_helio0, w_eff)[0]

    def close(self):
        self.sys.close()


class SemimajorLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xv_helio0, gas, traj, w, nsteps, every, mask_encounters):
        ckpts, ever, nbb = traj.run(xv_helio0, gas, nsteps, every, record=True)
        w_eff = w * (1.0 - ever.to(torch.float64)) if mask_encounters else w
        # masked: the groups of big bodies only, and none when no big bodies met
        ctx.groups = (2 if nbb > 0 else 0) if mask_encounters else 1
        L, seed_f, seed_i = traj.loss(xv_helio0, w_eff)
        ctx.traj, ctx.nsteps, ctx.every, ctx.nbb = traj, nsteps, every, nbb
        ctx.ckpts = ckpts
        ctx.save_for_backward(seed_f, seed_i)
        ctx.w_eff = w_eff
        return torch.tensor(L, dtype=torch.float64, device=xv_helio0.device)

    @staticmethod
    def backward(ctx, gL):
        traj = ctx.traj
        seed_f, seed_i = ctx.saved_tensors
        g = float(gL)
        h = traj.h
        mx.mx_kick_branches(h, 2)
        mx._check(mx.load().mx_adjoint_encounters(h, ctx.groups), "mx_adjoint_encounters")
        # consecutive steps share the pair pass of their adjoining half kicks;
        # mx_adjoint_init adds the last pending one
        mx.mx_adjoint_merge(h, True)
        lam = (seed_f * g).contiguous()
        dpar = torch.zeros(3, dtype=torch.float64, device="cuda")
        seg = torch.empty((ctx.every, 6, traj.n), dtype=torch.float64, device="cuda")
        pre = torch.empty((ctx.every, 6, traj.n), dtype=torch.float64, device="cuda")
        for start, ck in reversed(ctx.ckpts):
            length = min(ctx.every, ctx.nsteps - start)
            mx.mx_set_state_device(h, ck)
            mx.mx_set_step_index(h, start)
            # each step's start and pre-drift state (the branch replay keeps
            # deferral off, so the step leaves every body's)
            for k in range(length):
                mx.mx_get_state_device(h, seg[k])
                mx.mx_step(h, 1)
                mx.mx_predrift_state(h, pre[k])
            for k in reversed(range(length)):
                mx.mx_adjoint_step_predrift(h, seg[k], pre[k], start + k, lam, dpar)
        grad0 = torch.empty((6, traj.n), dtype=torch.float64, device="cuda")
        mx.mx_adjoint_init(h, lam, grad0)
        mx.mx_adjoint_merge(h, False)
        grad0 += g * seed_i
        return grad0, dpar, None, None, None, None, None


def semimajor_loss(traj, xv_helio0, gas, w, nsteps, every, mask_encounters=True):
    """Differentiable loss of a run of nsteps steps checkpointed every `every`."""
    return SemimajorLoss.apply(xv_helio0, gas, traj, w, int(nsteps), int(every),
                               bool(mask_encounters))
