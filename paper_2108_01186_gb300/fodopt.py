"""FOD optimisation: relax the Fermi-orbital descriptors of each system to a
minimum of E_SIC using the FOD forces (Sec. II: the FOD positions are found
by minimising the SIC energy with the forces of Eq. 9; Sec. III converges
every FOD to a force below 1e-3 Eh/bohr).

The paper does not say which minimiser it uses.  This module uses FIRE (the
fast inertial relaxation engine of Bitzek, Koskinen, Gaehler, Moseler and
Gumbsch, Phys. Rev. Lett. 97, 170201 (2006)) with unit masses and a
semi-implicit Euler step, one independent FIRE state per system:

  F = -dE/da;  stop when max |F| < fmax;
  P = F . v:
    P > 0:  v <- (1 - alpha) v + alpha |v| F/|F|;  after more than n_min
            such steps in a row: dt <- min(f_inc dt, dt_max), alpha <- f_alpha alpha
    P <= 0: v <- 0, dt <- f_dec dt, alpha <- alpha_start, counter reset
  v <- v + dt F;  a <- a + dt v.

Every energy and gradient comes from the CUDA library (forward, Poisson,
energy and reverse mode of the step); each Poisson solve starts from the
previous step's potentials (warm start).  Host work is the FIRE update of
3N numbers per system, done on the device with torch.
"""
from dataclasses import dataclass

import torch


@dataclass
class FireParams:
    dt0: float = 0.2          # initial time step (bohr / sqrt(Eh/bohr) units, unit mass)
    dt_max: float = 1.0
    n_min: int = 5
    f_inc: float = 1.1
    f_dec: float = 0.5
    alpha0: float = 0.1
    f_alpha: float = 0.99


class Fire:
    """FIRE state of several independent systems.  x: [n] flat positions,
    seg: [n] system index of each coordinate (0 .. nsys-1)."""

    def __init__(self, x, seg, nsys, params=None):
        self.p = params or FireParams()
        self.seg = seg
        self.nsys = nsys
        dev, dt = x.device, x.dtype
        self.v = torch.zeros_like(x)
        self.dt = torch.full((nsys,), self.p.dt0, dtype=dt, device=dev)
        self.alpha = torch.full((nsys,), self.p.alpha0, dtype=dt, device=dev)
        self.npos = torch.zeros(nsys, dtype=torch.int64, device=dev)

    def _segsum(self, a):
        out = torch.zeros(self.nsys, dtype=a.dtype, device=a.device)
        return out.index_add_(0, self.seg, a)

    def step(self, x, F, active):
        """One FIRE update of the systems with active[s] true; returns new x."""
        p = self.p
        P = self._segsum(F * self.v)
        vn = torch.sqrt(self._segsum(self.v * self.v))
        fn = torch.sqrt(self._segsum(F * F))
        up = active & (P > 0)
        down = active & ~(P > 0)
        s = self.seg
        mix_v = (1 - self.alpha)[s] * self.v + (self.alpha * vn / torch.clamp(fn, min=1e-300))[s] * F
        self.v = torch.where(up[s], mix_v, self.v)
        self.npos = torch.where(up, self.npos + 1, self.npos)
        grow = up & (self.npos > p.n_min)
        self.dt = torch.where(grow, torch.clamp(self.dt * p.f_inc, max=p.dt_max), self.dt)
        self.alpha = torch.where(grow, self.alpha * p.f_alpha, self.alpha)
        self.v = torch.where(down[s], torch.zeros_like(self.v), self.v)
        self.dt = torch.where(down, self.dt * p.f_dec, self.dt)
        self.alpha = torch.where(down, torch.full_like(self.alpha, p.alpha0), self.alpha)
        self.npos = torch.where(down, torch.zeros_like(self.npos), self.npos)
        dt = self.dt[s]
        act = active[s]
        self.v = torch.where(act, self.v + dt * F, self.v)
        return torch.where(act, x + dt * self.v, x)


def fire_minimize(energy_grad, x0, seg, nsys, fmax=1e-3, max_steps=500, params=None, callback=None):
    """Generic batched FIRE.  energy_grad(x) -> (E [nsys], grad [n]).
    Returns (x, E, max|F| per system, steps taken per system)."""
    x = x0.clone()
    fire = Fire(x, seg, nsys, params)
    steps = torch.zeros(nsys, dtype=torch.int64, device=x.device)
    active = torch.ones(nsys, dtype=torch.bool, device=x.device)
    E = fm = None
    for k in range(max_steps + 1):
        E, g = energy_grad(x)
        F = -g
        fm = torch.zeros(nsys, dtype=x.dtype, device=x.device).scatter_reduce_(
            0, seg, F.abs(), reduce="amax", include_self=True)
        active = active & (fm >= fmax)
        if callback is not None:
            callback(k, x, E, fm, active)
        if k == max_steps or not bool(active.any()):
            break
        x = fire.step(x, F, active)
        steps = steps + active.to(torch.int64)
    return x, E, fm, steps


def optimize_fods(ctx, psi, fods, fmax=1e-3, max_steps=500, scale=1.0, params=None, warm_start=True,
                  callback=None):
    """Relax the FODs of every system of the context (flat [sum orbitals x 3]
    float64 tensor on the device).  Returns dict(fods, E_sic, fmax, steps,
    cg_iters) where cg_iters lists the mean CG iterations per orbital of each
    step's Poisson solves."""
    blk_sys, norb = [], []
    for si, s in enumerate(ctx.systems):
        for N in s["norb"]:
            norb.append(N)
            blk_sys.append(si)
    seg = torch.cat([torch.full((3 * N,), b, dtype=torch.int64) for N, b in zip(norb, blk_sys)]).to(fods.device)
    nsys = len(ctx.systems)
    state = {"V": None, "iters": []}
    gE = torch.ones(nsys, dtype=torch.float64, device=fods.device)

    def energy_grad(x):
        out = ctx.forward(psi, x, scale=scale, V0=state["V"] if warm_start else None)
        state["V"] = out["V"]
        state["iters"].append(float(out["iters"].double().mean()))
        _, dfod = ctx.sic_backward(psi, x, out["phi"], out["V"], gE, want_dpsi=False)
        return out["E_sic"], dfod

    x, E, fm, steps = fire_minimize(energy_grad, fods, seg, nsys, fmax, max_steps, params, callback)
    return dict(fods=x, E_sic=E, fmax=fm, steps=steps, cg_iters=state["iters"])
