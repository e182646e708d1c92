"""FP64 oracle: the FLO-SIC step written out in the paper's order.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Every array is
float64.  A *grid* is the tuple ``(nx, ny, nz, h, origin)`` with interior
points ``origin + h*(i, j, k)``; a field on it is a flat array of length
``G = nx*ny*nz`` with x fastest.  Orbitals vanish outside the interior.

Steps and the passages they follow:

* ``fd_weights``/``laplacian``: centred high-order finite differences and the
  trapezoid rule on a uniform grid (Sec. II.A).
* ``poisson``: -Delta_h V = 4 pi rho with multipole Dirichlet values
  (Sec. II.A); the result is the exact solution of the discrete system,
  reached by plain CG to a relative residual of ``tol``.
* ``build_flos``: psi at the FODs by cubic interpolation, rho(a_i) with unit
  occupations (Sec. II.B), T (Eq. 8), Fermi orbitals F = T psi (Eqs. 6-7),
  overlap S = dV F F^T, symmetric Loewdin phi = S^{-1/2} F (Sec. I.B).
* ``sic_forward``: orbital densities, per-orbital Hartree U and fully
  polarised LSDA E_xc, E_SIC (Eq. 1), V_i^SIC = -(V_i + v_xc^i) (Eq. 5,
  bracketed term), and the scaled averaged SIC potential (Eq. 13).
* ``sic_backward``: reverse mode of the above; FOD gradient dE_SIC/da and
  dE_SIC/dpsi on the grid.
* ``pederson_fod_gradient``: the same FOD gradient by Eq. 9, with
  d phi/d a from Eqs. 10-11 and a forward derivative of S^{-1/2}.

Extended systems (``bc`` argument; Sec. II.A: periodic conditions along
extended directions, Dirichlet values from a dipole correction for surfaces):
``"isolated"`` (default; zero outside, multipole Dirichlet values),
``"periodic"`` (every direction periodic; the orbital density is neutralised
by a uniform background and V has zero mean), ``"slab"`` (periodic along x
and y; along z the dipole-corrected planar potential of ``slab_bc_rhs``).
Along a periodic direction the stencil, the interpolation nodes and the FOD
coordinates wrap around the box.
"""
import ctypes
import os
import subprocess

import numpy as np

__all__ = [
    "fd_weights", "laplacian", "multipole_moments", "multipole_value", "bc_rhs",
    "bc_rhs_adjoint", "cg_zero_bc", "poisson", "interp", "interp_scatter",
    "grad_central", "lsda_pol", "pw92_ferro", "build_flos", "sic_forward",
    "sic_backward", "pederson_fod_gradient", "max_threads", "eigh_sym", "hamiltonian_apply",
    "BC_MASK", "slab_bc_rhs", "slab_moments",
]

# bit d set = periodic along direction d (x = bit 0)
BC_MASK = {"isolated": 0, "periodic": 7, "slab": 3}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flosic_oracle.c")
_SO = os.path.join(_HERE, "_flosic_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build_library(force=False):
    """Compile flosic_oracle.c with gcc (OpenMP over independent orbitals)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build_library()
        L = ctypes.CDLL(_SO)
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "orc_fd_weights": (None, [i, _D]),
            "orc_laplacian": (None, [i, i, i, d, _D, _D]),
            "orc_laplacian_bc": (None, [i, i, i, d, i, _D, _D]),
            "orc_cg_batch_bc": (None, [i, i, i, i, d, i, _D, _D, d, i, _I]),
            "orc_slab_bc_rhs": (None, [i, i, i, d, _D, d, d, _D]),
            "orc_interp_bc": (None, [i, i, i, d, _D, i, i, _D, _D, _D, _D]),
            "orc_interp_scatter_bc": (None, [i, i, i, d, _D, i, _D, d, _D]),
            "orc_multipole_moments": (None, [i, i, i, d, _D, _D, _D]),
            "orc_multipole_value": (d, [_D, _D]),
            "orc_bc_rhs": (None, [i, i, i, d, _D, _D, _D]),
            "orc_bc_rhs_adjoint": (None, [i, i, i, d, _D, _D, _D]),
            "orc_cg_batch": (None, [i, i, i, i, d, _D, _D, d, i, _I]),
            "orc_poisson_batch": (None, [i, i, i, i, d, _D, _D, _D, d, i, _I]),
            "orc_interp": (None, [i, i, i, d, _D, i, _D, _D, _D, _D]),
            "orc_interp_scatter": (None, [i, i, i, d, _D, _D, d, _D]),
            "orc_grad_central": (None, [i, i, i, d, _D, _D]),
            "orc_pw92_ferro": (None, [d, _D, _D]),
            "orc_lsda_pol_grid": (None, [i64, _D, d, _D, _D]),
            "orc_max_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(grid):
    nx, ny, nz, h, origin = grid
    return int(nx), int(ny), int(nz), float(h), _f64(origin).reshape(3)


def max_threads():
    return lib().orc_max_threads()


# ---------------------------------------------------------------------------
# Grid operators (Sec. II.A)
# ---------------------------------------------------------------------------

def fd_weights(M=6):
    w = np.zeros(M + 1)
    lib().orc_fd_weights(M, _p(w))
    return w


def laplacian(u, grid, bc="isolated"):
    nx, ny, nz, h, _ = _grid(grid)
    u = _f64(u)
    out = np.empty_like(u)
    lib().orc_laplacian_bc(nx, ny, nz, h, BC_MASK[bc], _p(u), _p(out))
    return out


def hamiltonian_apply(psi, grid, vloc=None, vavg=None, bc="isolated"):
    """The SC_AvgSIC Kohn-Sham Hamiltonian of one spin (Sec. II.C, Eq. 13) on
    the orbitals psi [N, G]: H psi_a = -1/2 Delta_h psi_a + (v_loc + V_avg)
    psi_a, orbitals zero outside the box (periodic along the periodic
    directions of bc); v_loc stands for the other local terms of Eq. 13
    (external, Hartree, exchange-correlation)."""
    psi = np.atleast_2d(_f64(psi))
    v = np.zeros(psi.shape[1])
    if vloc is not None:
        v = v + _f64(vloc)
    if vavg is not None:
        v = v + _f64(vavg)
    return np.stack([-0.5 * laplacian(p, grid, bc) + v * p for p in psi])


def multipole_moments(rho, grid):
    nx, ny, nz, h, origin = _grid(grid)
    rho = _f64(rho)
    mom = np.zeros(10)
    lib().orc_multipole_moments(nx, ny, nz, h, _p(origin), _p(rho), _p(mom))
    return mom


def multipole_value(mom, R):
    return lib().orc_multipole_value(_p(_f64(mom)), _p(_f64(R)))


def bc_rhs(mom, grid):
    nx, ny, nz, h, origin = _grid(grid)
    out = np.zeros(nx * ny * nz)
    lib().orc_bc_rhs(nx, ny, nz, h, _p(origin), _p(_f64(mom)), _p(out))
    return out


def bc_rhs_adjoint(y, grid):
    nx, ny, nz, h, origin = _grid(grid)
    out = np.zeros(nx * ny * nz)
    lib().orc_bc_rhs_adjoint(nx, ny, nz, h, _p(origin), _p(_f64(y)), _p(out))
    return out


def cg_zero_bc(b, grid, tol=1e-12, max_iter=100000):
    """Solve (-Delta_h) x = b with zero ghost values for each row of b."""
    nx, ny, nz, h, _ = _grid(grid)
    b = _f64(np.atleast_2d(b))
    x = np.zeros_like(b)
    it = np.zeros(b.shape[0], dtype=np.int32)
    lib().orc_cg_batch(b.shape[0], nx, ny, nz, h, _p(b), _p(x), tol, max_iter,
                       it.ctypes.data_as(_I))
    return x, it


def slab_moments(rho, grid):
    """Charge Q = dV sum rho and dipole p_z = dV sum rho (z - c_z) of each row
    of rho about the box centre c_z (the two numbers the slab boundary needs)."""
    nx, ny, nz, h, origin = _grid(grid)
    rho = _f64(np.atleast_2d(rho)).reshape(-1, nz, ny, nx)
    dV = h ** 3
    Z = origin[2] + h * np.arange(nz) - (origin[2] + 0.5 * h * (nz - 1))
    planes = rho.sum(axis=(2, 3))
    return dV * planes.sum(axis=1), dV * planes @ Z


def slab_bc_rhs(Q, pz, grid):
    """Boundary term of the slab problem for charge Q and dipole p_z: the
    ghost planes along z hold V_b(z) = -(2 pi/A)(Q |z - c_z| - sgn(z - c_z) p_z),
    A = nx ny h^2 (Sec. II.A: dipole-corrected Dirichlet values)."""
    nx, ny, nz, h, origin = _grid(grid)
    out = np.zeros(nx * ny * nz)
    lib().orc_slab_bc_rhs(nx, ny, nz, h, _p(origin), float(Q), float(pz), _p(out))
    return out


def poisson(rho, grid, tol=1e-12, max_iter=100000, V0=None, bc="isolated"):
    """Per-orbital Poisson solves -Delta_h V_i = 4 pi rho_i (Sec. II.A); rho
    is [n, G].  Boundary by bc: "isolated" = multipole (l <= 2) Dirichlet
    values on the 6-layer ghost shell; "periodic" = -Delta_h V = 4 pi (rho -
    mean rho) with zero-mean V; "slab" = periodic along x, y and the
    dipole-corrected ghost planes of slab_bc_rhs along z.  Returns
    (V [n, G], iterations [n]); iterations -1 = not converged."""
    nx, ny, nz, h, origin = _grid(grid)
    rho = _f64(np.atleast_2d(rho))
    V = np.zeros_like(rho) if V0 is None else _f64(np.array(V0, dtype=np.float64).reshape(rho.shape))
    it = np.zeros(rho.shape[0], dtype=np.int32)
    if bc == "isolated":
        lib().orc_poisson_batch(rho.shape[0], nx, ny, nz, h, _p(origin), _p(rho), _p(V),
                                tol, max_iter, it.ctypes.data_as(_I))
        return V, it
    if bc == "periodic":
        b = 4.0 * np.pi * (rho - rho.mean(axis=1, keepdims=True))
        if V0 is not None:
            V -= V.mean(axis=1, keepdims=True)
    elif bc == "slab":
        Q, pz = slab_moments(rho, grid)
        b = 4.0 * np.pi * rho + np.stack([slab_bc_rhs(Q[i], pz[i], grid) for i in range(rho.shape[0])])
    else:
        raise ValueError("unknown boundary %r" % (bc,))
    b = _f64(b)
    lib().orc_cg_batch_bc(rho.shape[0], nx, ny, nz, h, BC_MASK[bc], _p(b), _p(V), tol, max_iter,
                          it.ctypes.data_as(_I))
    return V, it


def interp(u, grid, a, bc="isolated"):
    """Tricubic Lagrange interpolation (Sec. II.B, 'cubic interpolation') of
    the rows of u at point a: values [nf] and exact interpolant gradients
    [nf, 3].  Nodes wrap along the periodic directions of bc."""
    nx, ny, nz, h, origin = _grid(grid)
    u = _f64(np.atleast_2d(u))
    nf = u.shape[0]
    val = np.zeros(nf)
    grad = np.zeros((nf, 3))
    lib().orc_interp_bc(nx, ny, nz, h, _p(origin), BC_MASK[bc], nf, _p(u), _p(_f64(a)), _p(val), _p(grad))
    return val, grad


def interp_scatter(grid, a, coef, out, bc="isolated"):
    """out += coef * (interpolation weights of point a): adjoint of interp."""
    nx, ny, nz, h, origin = _grid(grid)
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    lib().orc_interp_scatter_bc(nx, ny, nz, h, _p(origin), BC_MASK[bc], _p(_f64(a)), float(coef), _p(out))


def grad_central(u, grid):
    """Grid gradient of the paper's force scheme (Sec. II.B): [3, G]."""
    nx, ny, nz, h, _ = _grid(grid)
    u = _f64(u)
    out = np.zeros((3, u.size))
    lib().orc_grad_central(nx, ny, nz, h, _p(u), _p(out))
    return out


def pw92_ferro(rs):
    ec, dec = ctypes.c_double(), ctypes.c_double()
    lib().orc_pw92_ferro(float(rs), ctypes.byref(ec), ctypes.byref(dec))
    return ec.value, dec.value


def lsda_pol(n, rho_min=1e-30):
    """Fully polarised LSDA (Slater exchange + PW92 correlation at zeta = 1)
    per point: (eps_xc, v_xc) for spin densities (n, 0)."""
    n = _f64(n)
    eps = np.empty_like(n)
    v = np.empty_like(n)
    lib().orc_lsda_pol_grid(n.size, _p(n), float(rho_min), _p(eps), _p(v))
    return eps, v


# ---------------------------------------------------------------------------
# Fermi-Loewdin orbitals (Sec. I.B, Eqs. 6-8; Sec. II.B)
# ---------------------------------------------------------------------------

def eigh_sym(S):
    """Eigen-decomposition of a symmetric matrix (LAPACK through numpy)."""
    lam, U = np.linalg.eigh(S)
    return lam, U


def _interp_all(psi, grid, fods, bc="isolated"):
    N = fods.shape[0]
    vals = np.zeros((N, psi.shape[0]))       # vals[i, a] = psi_a(a_i)
    grads = np.zeros((N, psi.shape[0], 3))   # grads[i, a] = grad psi_a(a_i)
    for i in range(N):
        vals[i], grads[i] = interp(psi, grid, fods[i], bc)
    return vals, grads


def build_flos(psi, fods, grid, illcond=1e-10, bc="isolated"):
    """One spin block: psi [N, G] (KS orbitals), fods [N, 3].

    rho(a_i) = sum_a psi_a(a_i)^2 (unit occupations, Sec. II.B);
    T_ia = psi_a(a_i)/sqrt(rho(a_i)) (Eq. 8); F = T psi (Eq. 7);
    S = dV F F^T summed over the grid; phi = S^{-1/2} F (symmetric Loewdin).
    Raises ValueError when lambda_min(S) < illcond * lambda_max(S)."""
    psi = _f64(psi)
    fods = _f64(fods).reshape(-1, 3)
    h = float(grid[3])
    dV = h ** 3
    vals, grads = _interp_all(psi, grid, fods, bc)
    rho_a = np.sum(vals ** 2, axis=1)
    T = vals / np.sqrt(rho_a)[:, None]
    F = T @ psi
    S = dV * (F @ F.T)
    lam, U = eigh_sym(S)
    if lam[0] < illcond * lam[-1]:
        raise ValueError("ill-conditioned Fermi-orbital overlap: lambda_min/lambda_max = %g" % (lam[0] / lam[-1]))
    Q = (U / np.sqrt(lam)) @ U.T
    phi = Q @ F
    return dict(vals=vals, grads=grads, rho_a=rho_a, T=T, F=F, S=S, lam=lam, evec=U, Q=Q, phi=phi)


# ---------------------------------------------------------------------------
# Energy and averaged potential (Eqs. 1, 5, 13)
# ---------------------------------------------------------------------------

def sic_forward(psi_blocks, fod_blocks, grid, scale=1.0, rho_min=1e-30, tol=1e-12,
                max_iter=100000, illcond=1e-10, V0_blocks=None, bc="isolated"):
    """One system.  psi_blocks / fod_blocks: one [N, G] / [N, 3] array per
    spin.  Returns a dict with per-spin lists and the scalar E_sic."""
    h = float(grid[3])
    dV = h ** 3
    out = dict(blocks=[], E_sic=0.0)
    for s, (psi, fods) in enumerate(zip(psi_blocks, fod_blocks)):
        psi = _f64(psi)
        fl = build_flos(psi, fods, grid, illcond, bc)
        phi = fl["phi"]
        rho = phi ** 2                                  # orbital densities
        V, it = poisson(rho, grid, tol, max_iter, None if V0_blocks is None else V0_blocks[s], bc)
        eps, vxc = lsda_pol(rho, rho_min)
        U = 0.5 * dV * np.sum(rho * V, axis=1)         # self-Hartree U[rho_i]
        Exc = dV * np.sum(rho * eps, axis=1)           # E_xc[rho_i, 0]
        Vsic = -(V + vxc)                              # orbital SIC potential
        rho_s = np.sum(psi ** 2, axis=0)               # spin density
        num = scale * np.sum(rho * Vsic, axis=0)
        Vavg = np.where(rho_s > rho_min, num / np.where(rho_s > rho_min, rho_s, 1.0), 0.0)
        out["E_sic"] += -float(np.sum(U + Exc))
        fl.update(rho=rho, V=V, iters=it, eps=eps, vxc=vxc, U=U, Exc=Exc, Vsic=Vsic,
                  rho_s=rho_s, Vavg=Vavg, psi=psi, fods=_f64(fods).reshape(-1, 3))
        out["blocks"].append(fl)
    return out


def _dk_kernel(lam):
    """K_ij = (f(l_i) - f(l_j))/(l_i - l_j) for f = l^{-1/2}, in the form
    -1/(a_i a_j (a_i + a_j)), a = sqrt(l); diagonal f'(l) = -l^{-3/2}/2."""
    a = np.sqrt(lam)
    return -1.0 / (a[:, None] * a[None, :] * (a[:, None] + a[None, :]))


def _exact_hartree_gradient(blk, grid, tol, max_iter):
    """d U_i / d rho_i = (dV/2)(G + G^T) rho_i for V = G rho, where the
    multipole boundary makes G non-symmetric: G^T rho = 4 pi W + K^T W with
    W = A^{-1} rho (zero-boundary solve) and K the boundary map rho -> bc."""
    rho = blk["rho"]
    W, _ = cg_zero_bc(rho, grid, tol, max_iter)
    GT = np.empty_like(rho)
    for i in range(rho.shape[0]):
        GT[i] = 4.0 * np.pi * W[i] + bc_rhs_adjoint(W[i], grid)
    return 0.5 * (blk["V"] + GT)


def sic_backward(fwd, grid, gE=1.0, adjoint="reuse_v", grad_mode="interp_exact",
                 tol=1e-12, max_iter=100000, bc="isolated"):
    """Reverse mode of sic_forward for E_sic (times the upstream gE).

    adjoint='reuse_v': dU_i/drho_i = dV V_i (the potential itself);
    adjoint='exact'  : the symmetrised (G + G^T)/2 form.
    grad_mode='interp_exact': grad psi(a) is the derivative of the cubic
    interpolant; 'paper_central': central-difference grid gradient then the
    same cubic interpolation (Sec. II.B).
    Extended systems (bc != "isolated") take adjoint='reuse_v' and
    grad_mode='interp_exact' only.
    Returns (dE_dpsi per spin [N, G], dE_dfod per spin [N, 3])."""
    if bc != "isolated" and (adjoint != "reuse_v" or grad_mode != "interp_exact"):
        raise ValueError("extended systems: adjoint='reuse_v' and grad_mode='interp_exact' only")
    h = float(grid[3])
    dV = h ** 3
    dpsi, dfod = [], []
    for blk in fwd["blocks"]:
        psi, phi, F, T, Q, U, lam = (blk[k] for k in ("psi", "phi", "F", "T", "Q", "evec", "lam"))
        vals, grads, rho_a, fods = blk["vals"], blk["grads"], blk["rho_a"], blk["fods"]
        Veff = blk["V"] if adjoint == "reuse_v" else _exact_hartree_gradient(blk, grid, tol, max_iter)
        Vsic = -(Veff + blk["vxc"])
        Phib = gE * 2.0 * dV * Vsic * phi              # dE/dphi on the grid
        Fb = Q.T @ Phib                                # through phi = Q F
        Qb = Phib @ F.T
        Sb = U @ ((U.T @ Qb @ U) * _dk_kernel(lam)) @ U.T   # Daleckii-Krein
        Fb = Fb + dV * (Sb + Sb.T) @ F                 # through S = dV F F^T
        psib = T.T @ Fb                                # through F = T psi
        Tb = Fb @ psi.T
        # through T_ia = v_ia / sqrt(rho_i), v_ia = psi_a(a_i) (product form of Eq. 11)
        sq = np.sqrt(rho_a)
        vb = Tb / sq[:, None] - vals * (np.sum(Tb * vals, axis=1) / (rho_a * sq))[:, None]
        N = fods.shape[0]
        force = np.zeros((N, 3))
        if grad_mode == "paper_central":
            cgrad = np.stack([grad_central(psi[a], grid) for a in range(psi.shape[0])])  # [Na,3,G]
        for i in range(N):
            for a in range(psi.shape[0]):
                interp_scatter(grid, fods[i], vb[i, a], psib[a], bc)
            if grad_mode == "interp_exact":
                force[i] = vb[i] @ grads[i]
            else:
                g3 = np.zeros((psi.shape[0], 3))
                for d in range(3):
                    g3[:, d], _ = interp(cgrad[:, d, :], grid, fods[i])
                force[i] = vb[i] @ g3
        dpsi.append(psib)
        dfod.append(force)
    return dpsi, dfod


def pederson_fod_gradient(fwd, grid, adjoint="reuse_v", tol=1e-12, max_iter=100000):
    """FOD gradient by Eq. 9: dE/da_m = sum_kl eps_kl (<dphi_k/da_m|phi_l> -
    <dphi_l/da_m|phi_k>), eps_kl = <phi_l|V_k^SIC|phi_k>.  dF/da follows
    Eqs. 10-11 in product form (no division by psi_a(a_i)); the derivative of
    S^{-1/2} is the forward Daleckii-Krein formula.  An independent route to
    sic_backward's FOD gradient (psi held fixed)."""
    h = float(grid[3])
    dV = h ** 3
    res = []
    for blk in fwd["blocks"]:
        psi, phi, F, Q, U, lam = (blk[k] for k in ("psi", "phi", "F", "Q", "evec", "lam"))
        vals, grads, rho_a = blk["vals"], blk["grads"], blk["rho_a"]
        Veff = blk["V"] if adjoint == "reuse_v" else _exact_hartree_gradient(blk, grid, tol, max_iter)
        Vsic = -(Veff + blk["vxc"])
        eps = dV * (phi * Vsic) @ phi.T                # eps[k, l] = <phi_l|V_k|phi_k>
        K = _dk_kernel(lam)
        N = phi.shape[0]
        force = np.zeros((N, 3))
        for m in range(N):
            sq = np.sqrt(rho_a[m])
            grho = 2.0 * vals[m] @ grads[m]            # grad rho(a_m), [3]
            for d in range(3):
                dT = grads[m][:, d] / sq - vals[m] * grho[d] / (2.0 * rho_a[m] * sq)
                dF = np.zeros_like(F)
                dF[m] = dT @ psi
                dS = dV * (dF @ F.T + F @ dF.T)
                dQ = U @ ((U.T @ dS @ U) * K) @ U.T
                dphi = dQ @ F + Q @ dF
                A = dV * dphi @ phi.T                  # A[k, l] = <dphi_k|phi_l>
                force[m, d] = np.sum(eps * (A - A.T))
        res.append(force)
    return res
