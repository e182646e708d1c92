"""Pins of the oracle's SC_AvgSIC Hamiltonian apply (Sec. II.C, Eq. 13):
the kinetic part against the analytic -1/2 Laplacian of a Gaussian, the
operator's symmetry and the potential term (no GPU)."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build_library()


def _grid(n, h):
    o = -0.5 * h * (n - 1)
    return (n, n, n, h, np.array([o, o, o]))


def _coords(grid):
    n, _, _, h, o = grid
    x = o[0] + h * np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def test_kinetic_part_of_a_gaussian():
    # -1/2 Laplacian of exp(-a r^2) is a (3 - 2 a r^2) exp(-a r^2); the error
    # of the 12th-order operator falls like h^12 (box edge 10 bohr, a = 0.8)
    a = 0.8
    err = []
    for n, h in ((40, 0.25), (50, 0.2)):
        g = _grid(n, h)
        X, Y, Z = _coords(g)
        r2 = (X ** 2 + Y ** 2 + Z ** 2).ravel()
        psi = np.exp(-a * r2)
        H = oracle.hamiltonian_apply(psi, g)[0]
        exact = a * (3.0 - 2.0 * a * r2) * psi
        err.append(np.max(np.abs(H - exact)) / np.max(np.abs(exact)))
    assert err[0] < 1e-6 and err[1] < 1e-7
    assert err[0] / err[1] > 0.6 * (0.25 / 0.2) ** 12


def test_symmetric_and_potential_term():
    g = _grid(14, 0.4)
    rng = np.random.default_rng(3)
    G = 14 ** 3
    u, w, v = rng.normal(size=(3, G))
    vavg = rng.normal(size=G)
    Hu = oracle.hamiltonian_apply(u, g, v, vavg)[0]
    Hw = oracle.hamiltonian_apply(w, g, v, vavg)[0]
    assert abs(w @ Hu - u @ Hw) < 1e-10 * np.abs(w @ Hu)
    # the potential term is pointwise: H(u; v + c) - H(u; v) = c u
    Hc = oracle.hamiltonian_apply(u, g, v + 0.7, vavg)[0]
    assert np.max(np.abs(Hc - Hu - 0.7 * u)) < 1e-12
    # without potentials, <u|H|u> = 1/2 of the discrete Dirichlet energy > 0
    H0 = oracle.hamiltonian_apply(u, g)[0]
    assert u @ H0 > 0
