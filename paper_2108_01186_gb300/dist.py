"""Host-side multi-GPU logic: one process per GPU.

Two partitions of the FLO-SIC step:

* independent units (systems of a batch, or whole replicas of a workload):
  no data-path collective, only a barrier around the timed region and the
  maximum of the per-rank times;
* the orbital units of one system (Sec. II.A solves one Poisson problem per
  orbital): every rank builds all Fermi-Loewdin orbitals of the system (the
  N x N coupling of a spin stays on every rank), solves and scores only its
  own orbitals through the library's orbital mask, and the partial results
  are summed over ranks -- E_SIC and the per-orbital U, E_xc (Eq. 1 sums over
  orbitals), the averaged potential V_avg (Eq. 13's numerator sums over
  orbitals over the same denominator), and in reverse mode the FOD gradient
  and dE/dpsi (linear in the per-orbital adjoint seeds).

Works with NCCL on GPUs and with gloo on CPU (used by the tests).
"""
import datetime
import os

import torch
import torch.distributed as dist


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, timeout_s=600):
    """Initialise the default process group from the environment (no-op for
    a single process)."""
    rank, world, _ = env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
    return rank, world


def shard(n_units, rank, world):
    """Contiguous balanced split of range(n_units): the units of this rank.
    Every unit is owned by exactly one rank; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(value, device=None):
    """Maximum of a per-rank scalar (the step time of the slowest rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device_sync=None):
    """Barrier across ranks, then wait for this rank's device work."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
    if device_sync is not None:
        device_sync()


def orbital_mask(norb, rank, world):
    """One 0/1 entry per orbital: 1 for the orbitals of this rank (the
    contiguous balanced split of shard())."""
    mine = set(shard(norb, rank, world))
    return [1 if o in mine else 0 for o in range(norb)]


def allreduce_sum(tensors):
    """Sums each tensor over ranks in place (nothing to do for one process);
    returns the list."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tensors
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors


class OrbitalShardedStep:
    """One FLO-SIC step of a context's systems with their orbitals split over
    the ranks (the orbital-unit partition described in the module docstring).
    forward() and backward() return the full results on every rank; V is
    this rank's potentials (zero for the orbitals of other ranks)."""

    def __init__(self, ctx, rank=None, world=None):
        r, w, _ = env()
        self.rank = r if rank is None else rank
        self.world = w if world is None else world
        self.ctx = ctx
        self.mask = orbital_mask(ctx.norb, self.rank, self.world)
        ctx.set_orbital_mask(self.mask if self.world > 1 else None)

    def forward(self, psi, fods, scale=1.0):
        ctx = self.ctx
        phi, _, _ = ctx.build_flos(psi, fods, want_matrices=False)
        V, iters, conv = ctx.orbital_poisson(phi)
        E, Vavg, U, Exc = ctx.sic_energy_potential(psi, phi, V, scale)
        allreduce_sum([E, Vavg, U, Exc, iters])
        if self.world > 1 and dist.is_initialized():
            dist.all_reduce(conv, op=dist.ReduceOp.MIN)   # masked orbitals report 1
        return dict(phi=phi, V=V, iters=iters, conv=conv, E_sic=E, V_avg=Vavg, U=U, Exc=Exc)

    def backward(self, psi, fods, phi, V, gE, want_dpsi=True):
        dpsi, dfod = self.ctx.sic_backward(psi, fods, phi, V, gE, want_dpsi=want_dpsi)
        allreduce_sum([dfod, dpsi])
        return dpsi, dfod
