"""Pins of the oracle's extended-system boundaries (Sec. II.A: periodic
conditions along extended directions; Dirichlet values from a dipole
correction for surfaces), each against something other than the oracle:
the Fourier symbol of the periodic stencil, shift invariance, the closed-form
potential of a Gaussian charge sheet, interpolation on an explicitly tiled
grid, and central differences of the energy."""
import math

import numpy as np
import pytest

from paper_2108_01186_gb300 import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build_library()
    return oracle


def _symbol(w, theta):
    """Fourier symbol of the centred second difference: w0 + 2 sum w_m cos(m theta)."""
    return w[0] + 2.0 * sum(w[m] * np.cos(m * theta) for m in range(1, len(w)))


def _wave(n, k, phase):
    x = np.arange(n)
    return np.cos(2 * np.pi * k * x / n + phase)


def test_periodic_laplacian_is_diagonal_on_plane_waves(orc):
    nx, ny, nz, h = 13, 14, 16, 0.37
    grid = (nx, ny, nz, h, np.zeros(3))
    w = orc.fd_weights()
    for kx, ky, kz in ((1, 0, 0), (2, 3, 5), (6, 7, 8)):
        u = (_wave(nz, kz, 0.3)[:, None, None] * _wave(ny, ky, -0.7)[None, :, None]
             * _wave(nx, kx, 1.1)[None, None, :]).ravel()
        lam = sum(_symbol(w, 2 * np.pi * k / n) for k, n in ((kx, nx), (ky, ny), (kz, nz))) / h ** 2
        assert np.max(np.abs(orc.laplacian(u, grid, "periodic") - lam * u)) < 1e-11 * abs(lam)


def test_periodic_laplacian_commutes_with_cyclic_shifts(orc):
    nx, ny, nz, h = 13, 15, 14, 0.3
    grid = (nx, ny, nz, h, np.zeros(3))
    u = np.random.default_rng(1).normal(size=(nz, ny, nx))
    Lu = orc.laplacian(u.ravel(), grid, "periodic").reshape(nz, ny, nx)
    for ax, sh in ((0, 5), (1, -3), (2, 7)):
        Ls = orc.laplacian(np.roll(u, sh, axis=ax).ravel(), grid, "periodic").reshape(nz, ny, nx)
        assert np.max(np.abs(Ls - np.roll(Lu, sh, axis=ax))) < 1e-10
    # the slab operator commutes with shifts along x and y only
    Lu = orc.laplacian(u.ravel(), grid, "slab").reshape(nz, ny, nx)
    Ls = orc.laplacian(np.roll(u, 4, axis=2).ravel(), grid, "slab").reshape(nz, ny, nx)
    assert np.max(np.abs(Ls - np.roll(Lu, 4, axis=2))) < 1e-10
    Ls = orc.laplacian(np.roll(u, 4, axis=0).ravel(), grid, "slab").reshape(nz, ny, nx)
    assert np.max(np.abs(Ls - np.roll(Lu, 4, axis=0))) > 1.0


def test_slab_laplacian_separates(orc):
    # u = cos(theta x) f(z): Delta_h u = (symbol_x / h^2) u + cos(theta x) D_z f
    # with D_z the zero-outside 1-D operator (the isolated operator on a
    # 1 x 1 x nz grid minus the two absent directions' centre terms)
    nx, ny, nz, h = 14, 13, 17, 0.4
    grid = (nx, ny, nz, h, np.zeros(3))
    w = orc.fd_weights()
    f = np.random.default_rng(2).normal(size=nz)
    cx = _wave(nx, 3, 0.4)
    u = (f[:, None, None] * np.ones(ny)[None, :, None] * cx[None, None, :]).ravel()
    Dz = orc.laplacian(f, (1, 1, nz, h, np.zeros(3))) - 2 * w[0] * f / h ** 2
    ref = (_symbol(w, 2 * np.pi * 3 / nx) / h ** 2) * u + (Dz[:, None, None] * np.ones(ny)[None, :, None]
                                                          * cx[None, None, :]).ravel()
    assert np.max(np.abs(orc.laplacian(u, grid, "slab") - ref)) < 1e-10


def test_periodic_poisson_of_a_plane_wave(orc):
    nx, ny, nz, h = 14, 13, 15, 0.35
    grid = (nx, ny, nz, h, np.zeros(3))
    w = orc.fd_weights()
    wave = (_wave(nz, 2, 0.0)[:, None, None] * _wave(ny, 1, 0.5)[None, :, None]
            * _wave(nx, 3, -0.2)[None, None, :]).ravel()
    rho = 0.7 + 0.2 * wave
    V, it = orc.poisson(rho[None], grid, tol=1e-13, bc="periodic")
    assert it[0] > 0
    # -Delta_h V = 4 pi (rho - mean rho): the background removes the constant
    lam = -sum(_symbol(w, 2 * np.pi * k / n) for k, n in ((3, nx), (1, ny), (2, nz))) / h ** 2
    ref = 4 * np.pi * 0.2 * wave / lam
    assert abs(V[0].mean()) < 1e-12
    assert np.max(np.abs(V[0] - ref)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("z0", [0.0, 1.7, -2.3])
def test_slab_potential_of_a_gaussian_sheet(orc, z0):
    # a charge sheet uniform in x, y with a Gaussian profile in z at z0 (off
    # the centre: a dipole about the box centre).  Continuum: V(z) = -(2 pi Q /
    # A) E|z - Z|, Z ~ N(z0, s^2), i.e. (z - z0) erf((z - z0)/(s sqrt 2)) +
    # s sqrt(2/pi) exp(-(z - z0)^2 / 2 s^2).  The 12th-order discrete problem
    # with the dipole-corrected ghost planes reproduces it to its
    # discretisation error; a wrong sign or weight of the dipole term is off
    # by O(1).
    nx, ny, nz, h, s = 13, 14, 120, 0.2, 1.3
    origin = np.array([0.1, -0.3, -0.5 * h * (nz - 1)])
    grid = (nx, ny, nz, h, origin)
    z = origin[2] + h * np.arange(nz)
    prof = np.exp(-(z - z0) ** 2 / (2 * s * s))
    rho = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).ravel().copy()
    rho /= h ** 3 * rho.sum()                                  # Q = 1
    V, it = orc.poisson(rho[None], grid, tol=1e-13, bc="slab")
    assert it[0] > 0
    A = nx * ny * h * h
    d = z - z0
    Vz = -(2 * np.pi / A) * (d * np.array([math.erf(t) for t in d / (s * math.sqrt(2))])
                             + s * math.sqrt(2 / math.pi) * np.exp(-d * d / (2 * s * s)))
    Vg = V[0].reshape(nz, ny, nx)
    assert np.max(np.abs(Vg - Vg[:, :1, :1])) < 1e-12 * np.max(np.abs(Vg))   # uniform in x, y
    assert np.max(np.abs(Vg[:, 0, 0] - Vz)) < 1e-7 * np.max(np.abs(Vz))
    Q, pz = orc.slab_moments(rho[None], grid)
    assert abs(Q[0] - 1.0) < 1e-12 and abs(pz[0] - z0) < 1e-9


def test_periodic_interpolation_equals_a_tiled_grid(orc):
    nx, ny, nz, h = 13, 14, 15, 0.45
    origin = np.array([0.2, -1.0, 0.5])
    u = np.random.default_rng(3).normal(size=(2, nz, ny, nx))
    big = np.tile(u, (1, 3, 3, 3))                         # cells -1, 0, 1 along each axis
    L = h * np.array([nx, ny, nz])
    gbig = (3 * nx, 3 * ny, 3 * nz, h, origin - L)
    g = (nx, ny, nz, h, origin)
    # (points off the node planes: the interpolant is only continuous across cells)
    for a in (origin + L - 0.3 * h, origin + np.array([-0.2, 0.1, 0.7]) * h, origin + 0.37 * L,
              origin + L + np.array([0.7, 1.3, 0.1]) * h):
        v, gr = orc.interp(u.reshape(2, -1), g, a, "periodic")
        ab = a - L * np.floor((a - origin) / L)                # the same point inside cell 0
        vb, grb = orc.interp(big.reshape(2, -1), gbig, ab, "isolated")
        assert np.max(np.abs(v - vb)) < 1e-13 and np.max(np.abs(gr - grb)) < 1e-12
    # slab: x, y wrap, z does not
    a = origin + np.array([nx - 0.5, -0.4, 2.3]) * h
    v, _ = orc.interp(u.reshape(2, -1), g, a, "slab")
    vz, _ = orc.interp(np.tile(u, (1, 1, 3, 3)).reshape(2, -1), (3 * nx, 3 * ny, nz, h, origin - L * [1, 1, 0]),
                       a, "isolated")
    assert np.max(np.abs(v - vz)) < 1e-13


def test_periodic_scatter_is_the_adjoint_of_interpolation(orc):
    nx, ny, nz, h = 13, 13, 14, 0.5
    g = (nx, ny, nz, h, np.zeros(3))
    u = np.random.default_rng(4).normal(size=nx * ny * nz)
    a = np.array([nx - 0.6, 0.3, nz - 1.2]) * h
    for bc in ("periodic", "slab"):
        out = np.zeros(nx * ny * nz)
        orc.interp_scatter(g, a, 1.7, out, bc)
        v, _ = orc.interp(u, g, a, bc)
        assert abs(out @ u - 1.7 * v[0]) < 1e-12


def test_periodic_fod_gradient_matches_central_differences(orc):
    # with a uniform background the Hartree map is symmetric, so the reverse
    # mode that reuses V is exact; orbitals and FODs cross the cell faces
    s = synth.make_extended_system(16, 0.5, 2, [3], seed=11, bc="periodic")
    f = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-13, bc="periodic")
    _, g = orc.sic_backward(f, s.grid, bc="periodic")
    eps = 1e-4
    for i, d in ((0, 0), (1, 2), (2, 1)):
        fp = s.fods[0].copy(); fp[i, d] += eps
        fm = s.fods[0].copy(); fm[i, d] -= eps
        Ep = orc.sic_forward(s.psi, [fp], s.grid, tol=1e-13, bc="periodic")["E_sic"]
        Em = orc.sic_forward(s.psi, [fm], s.grid, tol=1e-13, bc="periodic")["E_sic"]
        assert abs((Ep - Em) / (2 * eps) - g[0][i, d]) < 1e-6


def test_periodic_energy_is_invariant_under_cell_translation(orc):
    # rolling the orbitals by whole grid steps and moving the FODs with them
    # leaves every energy unchanged (no boundary in a periodic cell)
    s = synth.make_extended_system(16, 0.5, 2, [2], seed=12, bc="periodic")
    f0 = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-13, bc="periodic")
    psi = [np.roll(p.reshape(-1, 16, 16, 16), (3, -5, 7), axis=(1, 2, 3)).reshape(p.shape[0], -1) for p in s.psi]
    fods = [f + s.h * np.array([7, -5, 3]) for f in s.fods]
    f1 = orc.sic_forward(psi, fods, s.grid, tol=1e-13, bc="periodic")
    assert abs(f1["E_sic"] - f0["E_sic"]) < 1e-11
