"""Seeded synthetic inputs: Kohn-Sham-like orbitals and FOD positions.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds none of the FLO-SIC arithmetic: it only samples Gaussian s/p functions
on a uniform grid, orthonormalises their random combinations with a QR
factorisation (a different route from the method's Loewdin step; the SIC
energy is invariant under the rotation this leaves), and draws FOD positions
near the atoms.

Recipe (the paper's molecules are not available, so these stand in for them
with its grid spacings and sp-shell orbitals):

* grid: n^3 interior points, spacing h, box side L = n*h centred at 0;
* atoms: uniform in the central cube of half-width L/2 - p, p = min(6, 0.4 L)
  bohr, pairwise at least 2 bohr apart (rejection sampling);
* basis: per atom one normalised s Gaussian (2a/pi)^{3/4} exp(-a r^2) and
  three p Gaussians 2 sqrt(a) (2a/pi)^{3/4} x exp(-a r^2), each with its own
  exponent a uniform in [0.3, 3.0] bohr^-2;
* orbitals: N combinations with standard-normal coefficients, sampled on the
  grid and orthonormalised so that dV psi psi^T = I;
* FODs: FOD i sits within 0.5 bohr of atom (i mod n_atoms) (uniform in the
  ball); redrawn when closer than 0.3 bohr to another FOD of the same spin or
  within 1e-3 h of a grid plane.
* seeds: ``seed = 1000 * config + system``; spin s uses seed + 7919 s for its
  coefficients and FODs.
* extended systems (``make_extended_system``): the same recipe on a periodic
  cell; along periodic directions atoms lie anywhere in the cell and each
  basis function is summed over its periodic images.
"""
import math
from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class System:
    n: int                       # points per side (nx = ny = nz = n)
    h: float                     # grid spacing, bohr
    norb: List[int]              # occupied orbitals per spin
    atoms: np.ndarray            # [natoms, 3]
    psi: List[np.ndarray] = field(default_factory=list)   # per spin [N, G] float64
    fods: List[np.ndarray] = field(default_factory=list)  # per spin [N, 3] float64

    @property
    def origin(self):
        o = -0.5 * self.h * (self.n - 1)
        return np.array([o, o, o])

    @property
    def G(self):
        return self.n ** 3

    @property
    def grid(self):
        return (self.n, self.n, self.n, self.h, self.origin)

    @property
    def nspin(self):
        return len(self.norb)


def _place_atoms(rng, L, natoms, min_sep=2.0, max_tries=200000):
    pad = min(6.0, 0.4 * L)
    half = L / 2.0 - pad
    atoms = []
    tries = 0
    while len(atoms) < natoms:
        tries += 1
        if tries > max_tries:
            raise ValueError("cannot place %d atoms %.1f bohr apart in a cube of half-width %.2f"
                             % (natoms, min_sep, half))
        x = rng.uniform(-half, half, size=3)
        if all(np.linalg.norm(x - a) >= min_sep for a in atoms):
            atoms.append(x)
    return np.array(atoms)


def max_atoms(n, h, min_sep=2.0):
    """Atoms that random rejection sampling places reliably (about 30 % of
    the simple-cubic packing bound); used to cap orbital counts."""
    L = n * h
    half = L / 2.0 - min(6.0, 0.4 * L)
    per_side = 2.0 * half / min_sep + 1.0
    return max(1, int(0.3 * per_side ** 3))


def _basis(atoms, rng, x1d):
    funcs = []
    X = x1d[None, None, :]
    Y = x1d[None, :, None]
    Z = x1d[:, None, None]
    for a in atoms:
        for lm in range(4):
            alpha = rng.uniform(0.3, 3.0)
            dx, dy, dz = X - a[0], Y - a[1], Z - a[2]
            r2 = dx * dx + dy * dy + dz * dz
            norm = (2.0 * alpha / math.pi) ** 0.75
            g = norm * np.exp(-alpha * r2)
            if lm == 1:
                g = 2.0 * math.sqrt(alpha) * dx * g
            elif lm == 2:
                g = 2.0 * math.sqrt(alpha) * dy * g
            elif lm == 3:
                g = 2.0 * math.sqrt(alpha) * dz * g
            funcs.append(g.reshape(-1))
    return np.stack(funcs)


def _near_plane(x, origin, h, frac=1e-3):
    u = (x - origin) / h
    return np.any(np.abs(u - np.round(u)) < frac)


def _draw_fods(rng, atoms, N, origin, h, min_sep=0.3, max_tries=100000):
    fods = []
    for i in range(N):
        a = atoms[i % len(atoms)]
        for _ in range(max_tries):
            d = rng.normal(size=3)
            d *= rng.uniform() ** (1.0 / 3.0) * 0.5 / np.linalg.norm(d)
            x = a + d
            if _near_plane(x, origin, h):
                continue
            if any(np.linalg.norm(x - f) < min_sep for f in fods):
                continue
            fods.append(x)
            break
        else:
            raise ValueError("cannot place FOD %d" % i)
    return np.array(fods)


def make_system(n, h, natoms, norb, seed):
    """One system: n^3 grid, spacing h, natoms atoms, norb = [N_up(, N_dn)]."""
    rng = np.random.default_rng(seed)
    L = n * h
    atoms = _place_atoms(rng, L, natoms)
    sysm = System(n=n, h=h, norb=list(norb), atoms=atoms)
    x1d = sysm.origin[0] + h * np.arange(n)
    dV = h ** 3
    for s, N in enumerate(norb):
        srng = np.random.default_rng(seed + 7919 * s)
        B = _basis(atoms, srng, x1d)                     # [nb, G]
        if N > B.shape[0]:
            raise ValueError("more orbitals than basis functions")
        C = srng.normal(size=(N, B.shape[0]))
        M = (C @ B).T * math.sqrt(dV)                     # [G, N]
        Qm, _ = np.linalg.qr(M)
        psi = np.ascontiguousarray((Qm / math.sqrt(dV)).T)
        sysm.psi.append(psi)
        sysm.fods.append(_draw_fods(srng, atoms, N, sysm.origin, h))
    return sysm


_PERIODIC_AXES = {"periodic": (0, 1, 2), "slab": (0, 1)}


def make_extended_system(n, h, natoms, norb, seed, bc, images=2):
    """One extended system on an n^3 cell (bc "periodic": all directions
    periodic; "slab": x and y periodic, z finite).  As make_system, except:
    along the periodic directions atoms are placed anywhere in the cell (at
    least 2 bohr apart by the minimum-image distance) and every basis
    function is summed over its periodic images up to ``images`` cells away,
    so orbitals and FODs cross the cell faces; along a finite z atoms keep
    make_system's padding."""
    axes = _PERIODIC_AXES[bc]
    rng = np.random.default_rng(seed)
    L = n * h
    pad = min(6.0, 0.4 * L)
    lo = np.array([-L / 2 if d in axes else -L / 2 + pad for d in range(3)])
    hi = np.array([L / 2 if d in axes else L / 2 - pad for d in range(3)])
    atoms = []
    tries = 0
    while len(atoms) < natoms:
        tries += 1
        if tries > 200000:
            raise ValueError("cannot place %d atoms in the cell" % natoms)
        x = rng.uniform(lo, hi)
        ok = True
        for a in atoms:
            d = x - a
            for ax in axes:
                d[ax] -= L * np.round(d[ax] / L)
            if np.linalg.norm(d) < 2.0:
                ok = False
                break
        if ok:
            atoms.append(x)
    atoms = np.array(atoms)
    sysm = System(n=n, h=h, norb=list(norb), atoms=atoms)
    x1d = sysm.origin[0] + h * np.arange(n)
    dV = h ** 3
    rng_img = range(-images, images + 1)
    shifts = [np.array([i if 0 in axes else 0, j if 1 in axes else 0, k if 2 in axes else 0]) * L
              for i in (rng_img if 0 in axes else (0,))
              for j in (rng_img if 1 in axes else (0,))
              for k in (rng_img if 2 in axes else (0,))]
    for sp, N in enumerate(norb):
        srng = np.random.default_rng(seed + 7919 * sp)
        B = None
        # the same exponents for every image of a function: draw them once
        state = srng.bit_generator.state
        for sh in shifts:
            srng.bit_generator.state = state
            Bi = _basis(atoms + sh, srng, x1d)
            B = Bi if B is None else B + Bi
        if N > B.shape[0]:
            raise ValueError("more orbitals than basis functions")
        C = srng.normal(size=(N, B.shape[0]))
        M = (C @ B).T * math.sqrt(dV)
        Qm, _ = np.linalg.qr(M)
        sysm.psi.append(np.ascontiguousarray((Qm / math.sqrt(dV)).T))
        sysm.fods.append(_draw_fods(srng, atoms, N, sysm.origin, h))
    return sysm


# Workloads of the FLO-SIC step (grid, spacing, atoms, orbitals per spin).
CONFIGS = {
    0: dict(n=40, h=0.3, natoms=3, norb=[5], desc="40^3 h=0.3, 5 orbitals, one spin, FP64"),
    1: dict(n=96, h=0.2, natoms=8, norb=[16, 16], desc="96^3 h=0.2, 16+16 orbitals, scale 0.5"),
    3: dict(n=128, h=0.2, natoms=16, norb=[32, 32], desc="128^3 h=0.2, 32+32 orbitals, forward+adjoint"),
    4: dict(n=192, h=0.15, natoms=60, norb=[120, 120], desc="192^3 h=0.15, 120+120 orbitals"),
}


def make_config(idx, system=0):
    c = CONFIGS[idx]
    return make_system(c["n"], c["h"], c["natoms"], c["norb"], seed=1000 * idx + system)


def make_uneven_batch(nsys=64, seed_base=2000, n_range=(48, 128), h_range=(0.15, 0.3),
                      norb_range=(2, 40)):
    """Many independent one-spin systems of uneven grid and orbital counts."""
    out = []
    for s in range(nsys):
        rng = np.random.default_rng(seed_base + s + 500000)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        h = float(rng.uniform(*h_range))
        N = int(rng.integers(norb_range[0], norb_range[1] + 1))
        natoms = min(int(math.ceil(N / 2)), max_atoms(n, h))
        N = min(N, 4 * natoms)
        out.append(make_system(n, h, natoms, [N], seed=seed_base + s))
    return out
