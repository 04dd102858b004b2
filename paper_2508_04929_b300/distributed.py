"""Data-parallel training across GPUs: particles are split over the ranks, Theta is
replicated, and one all-reduce of dL/dTheta (11 N floats) per step precedes a replicated Adam
step, so every rank keeps the same Theta.  The paper trains on one GPU (Sec. 4.1); the loss
is a sum over particles (Sec. 3.3.5), so the summed gradient of the ranks' batches is the
gradient of the whole batch.

``DataParallelStep`` takes the two halves of a step as callables: ``local_grad(theta, dtheta)``
fills dtheta with this rank's batch gradient (on a GPU: a GraphStep replay without Adam),
``adam(theta, dtheta)`` applies the update (on a GPU: gs_step_counted).  The collective is
torch.distributed's all-reduce (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def init_from_env(backend=None):
    """Join the process group described by RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT
    (as torchrun sets them).  Returns (rank, world)."""
    if not dist.is_initialized():
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size()


def broadcast_params(theta, src=0):
    """Make every rank's Theta equal to rank src's (in place)."""
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.broadcast(theta, src)
    return theta


def allreduce_gradients(dtheta, average=False):
    """Sum (or mean) of dtheta over the ranks, in place."""
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(dtheta, op=dist.ReduceOp.SUM)
        if average:
            dtheta /= dist.get_world_size()
    return dtheta


class DataParallelStep:
    """One data-parallel training step: local gradient, all-reduce, replicated update."""

    def __init__(self, theta, local_grad, adam, average=False):
        self.theta = theta
        self.dtheta = torch.zeros_like(theta)
        self.local_grad = local_grad
        self.adam = adam
        self.average = average
        broadcast_params(self.theta)

    def __call__(self):
        self.dtheta.zero_()
        out = self.local_grad(self.theta, self.dtheta)
        allreduce_gradients(self.dtheta, self.average)
        self.adam(self.theta, self.dtheta)
        return out


def graph_step_parts(gs, lr=1e-3):
    """(local_grad, adam) for a single-problem GraphStep recorded with adam=False: the graph
    replay leaves this rank's gradient in the problem's dtheta buffer, which the step hands
    over; Adam runs with the step counter on the device."""
    from . import _lib as L
    p = gs.problems[0]

    def local_grad(theta, dtheta):
        assert theta.data_ptr() == p.theta.data_ptr()
        losses = gs.replay()[0]
        dtheta.copy_(p.dtheta)
        return losses

    def adam(theta, dtheta):
        L.gs_step_counted(theta, dtheta, p.m, p.v, p.t, lr=lr)

    return local_grad, adam


def world_from_env():
    return int(os.environ.get("WORLD_SIZE", "1"))
