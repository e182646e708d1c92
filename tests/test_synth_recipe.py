"""CPU checks of the seeded input recipe (the stand-ins for the paper's
molecules): every stated property of the generator holds on the generated
systems, and equal seeds give identical inputs."""
import numpy as np
import pytest

from paper_2108_01186_gb300 import synth


@pytest.fixture(scope="module", params=[(40, 0.4, 3, [5, 3], 17), (36, 0.45, 4, [7], 5)])
def system(request):
    n, h, natoms, norb, seed = request.param
    return synth.make_system(n, h, natoms, norb, seed)


def test_atoms_are_padded_and_separated(system):
    s = system
    L = s.n * s.h
    half = L / 2 - min(6.0, 0.4 * L)
    assert np.all(np.abs(s.atoms) <= half + 1e-12)
    d = np.linalg.norm(s.atoms[:, None, :] - s.atoms[None, :, :], axis=-1)
    assert np.all(d[np.triu_indices(len(s.atoms), 1)] >= 2.0)


def test_orbitals_are_orthonormal_on_the_grid(system):
    s = system
    dV = s.h ** 3
    for psi, N in zip(s.psi, s.norb):
        assert psi.shape == (N, s.G) and psi.dtype == np.float64 and psi.flags.c_contiguous
        assert np.allclose(dV * psi @ psi.T, np.eye(N), atol=1e-12)


def test_fods_follow_the_placement_rules(system):
    s = system
    for f, N in zip(s.fods, s.norb):
        assert f.shape == (N, 3)
        for i in range(N):
            assert np.linalg.norm(f[i] - s.atoms[i % len(s.atoms)]) <= 0.5 + 1e-12
            u = (f[i] - s.origin) / s.h
            assert np.all(np.abs(u - np.round(u)) >= 1e-3)
        d = np.linalg.norm(f[:, None, :] - f[None, :, :], axis=-1)
        assert np.all(d[np.triu_indices(N, 1)] >= 0.3)


def test_seeds_are_deterministic_and_distinct():
    a = synth.make_system(16, 0.5, 2, [3, 2], seed=123)
    b = synth.make_system(16, 0.5, 2, [3, 2], seed=123)
    c = synth.make_system(16, 0.5, 2, [3, 2], seed=124)
    for k in range(2):
        assert np.array_equal(a.psi[k], b.psi[k]) and np.array_equal(a.fods[k], b.fods[k])
    assert not np.array_equal(a.psi[0], c.psi[0])
    # the two spins draw from their own streams
    assert not np.allclose(a.psi[0][:2], a.psi[1][:2])


def test_grid_convention():
    s = synth.make_system(10, 0.5, 1, [1], seed=1)
    nx, ny, nz, h, origin = s.grid
    assert (nx, ny, nz, h) == (10, 10, 10, 0.5)
    # the box is centred at 0: the first and last points are symmetric
    assert np.allclose(origin, -0.5 * h * (s.n - 1))
    assert s.G == 1000 and s.nspin == 1


def test_periodic_cell_images_keep_orbitals_periodic():
    # a basis summed over its images varies smoothly across the cell faces:
    # the wrap-around neighbour of the last plane is about as close in value
    # as an interior neighbour
    s = synth.make_extended_system(24, 0.45, 2, [3], seed=23, bc="periodic")
    psi = s.psi[0].reshape(3, s.n, s.n, s.n)
    wrap = np.max(np.abs(psi[:, :, :, -1] - psi[:, :, :, 0]))
    inner = np.max(np.abs(np.diff(psi, axis=3)))
    assert wrap <= 1.5 * inner
    d = s.atoms[:, None, :] - s.atoms[None, :, :]
    L = s.n * s.h
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=-1)
    assert np.all(r[np.triu_indices(len(s.atoms), 1)] >= 2.0)
