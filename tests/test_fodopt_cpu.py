"""FIRE minimiser of the FOD relaxation, on CPU: the library's batched
torch version and the oracle's NumPy version, pinned to closed-form minima
and to each other (no GPU; the energies here are analytic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fodopt as ofire  # noqa: E402
from paper_2108_01186_gb300 import fodopt  # noqa: E402


def quad(x, k, c, B):
    """E = 1/2 (x-c)^T K (x-c) with K = diag(k) + B B^T (SPD), its gradient."""
    d = x - c
    Kd = k * d + B @ (B.T @ d)
    return 0.5 * float(d @ Kd), Kd


def lj_cluster(x, n):
    """Lennard-Jones energy (eps = sigma = 1) of n atoms, gradient."""
    p = x.reshape(n, 3)
    E = 0.0
    g = np.zeros_like(p)
    for i in range(n):
        for j in range(i + 1, n):
            r = p[i] - p[j]
            r2 = float(r @ r)
            s6 = 1.0 / r2 ** 3
            E += 4.0 * (s6 * s6 - s6)
            f = (-48.0 * s6 * s6 + 24.0 * s6) / r2   # dE/dr * 1/r
            g[i] += f * r
            g[j] -= f * r
    return E, g.ravel()


def torch_fun(fun):
    def eg(x):
        E, g = fun(x.numpy())
        return torch.tensor([E], dtype=torch.float64), torch.tensor(g, dtype=torch.float64)
    return eg


def test_quadratic_minimum_and_identical_trajectories():
    rng = np.random.default_rng(5)
    n = 12
    k = rng.uniform(0.2, 3.0, n)
    B = 0.3 * rng.normal(size=(n, 2))
    c = rng.normal(size=n)
    x0 = c + rng.normal(size=n)
    fun = lambda x: quad(x, k, c, B)  # noqa: E731
    xo, Eo, fmo, so, hist = ofire.fire(fun, x0, fmax=1e-8, max_steps=5000)
    assert fmo < 1e-8 and np.max(np.abs(xo - c)) < 1e-7 and Eo < 1e-15
    seg = torch.zeros(n, dtype=torch.int64)
    xt, Et, fmt, st = fodopt.fire_minimize(torch_fun(fun), torch.tensor(x0), seg, 1, fmax=1e-8, max_steps=5000)
    assert int(st[0]) == so
    assert np.max(np.abs(xt.numpy() - xo)) < 1e-12


def test_lennard_jones_dimer_and_triangle():
    # dimer: r = 2^(1/6), E = -1; triangle: equilateral at r = 2^(1/6), E = -3
    for n, e_min in ((2, -1.0), (3, -3.0)):
        rng = np.random.default_rng(n)
        x0 = (np.eye(3)[:n] * 1.3 + 0.05 * rng.normal(size=(n, 3))).ravel()
        fun = lambda x: lj_cluster(x, n)  # noqa: E731
        x, E, fm, steps, _ = ofire.fire(fun, x0, fmax=1e-7, max_steps=20000, dt0=0.01, dt_max=0.05)
        assert fm < 1e-7 and abs(E - e_min) < 1e-10
        p = x.reshape(n, 3)
        for i in range(n):
            for j in range(i + 1, n):
                assert abs(np.linalg.norm(p[i] - p[j]) - 2 ** (1 / 6)) < 1e-6
        seg = torch.zeros(3 * n, dtype=torch.int64)
        par = fodopt.FireParams(dt0=0.01, dt_max=0.05)
        xt, Et, fmt, st = fodopt.fire_minimize(torch_fun(fun), torch.tensor(x0), seg, 1, 1e-7, 20000, par)
        assert np.max(np.abs(xt.numpy() - x)) < 1e-9


def test_batched_systems_are_independent():
    rng = np.random.default_rng(9)
    sizes = [6, 9]
    probs = []
    for n in sizes:
        k = rng.uniform(0.5, 2.0, n)
        B = 0.2 * rng.normal(size=(n, 1))
        c = rng.normal(size=n)
        probs.append((k, B, c, c + rng.normal(size=n)))

    def eg(x):
        xs = x.numpy()
        Es, gs, o = [], [], 0
        for (k, B, c, _), n in zip(probs, sizes):
            E, g = quad(xs[o:o + n], k, c, B)
            Es.append(E)
            gs.append(g)
            o += n
        return torch.tensor(Es, dtype=torch.float64), torch.tensor(np.concatenate(gs))

    x0 = torch.tensor(np.concatenate([p[3] for p in probs]))
    seg = torch.cat([torch.full((n,), i, dtype=torch.int64) for i, n in enumerate(sizes)])
    xb, Eb, fmb, sb = fodopt.fire_minimize(eg, x0, seg, 2, fmax=1e-6, max_steps=3000)
    o = 0
    for i, ((k, B, c, xi), n) in enumerate(zip(probs, sizes)):
        xo, Eo, fmo, so, _ = ofire.fire(lambda x: quad(x, k, c, B), xi, fmax=1e-6, max_steps=3000)
        assert int(sb[i]) == so
        assert np.max(np.abs(xb.numpy()[o:o + n] - xo)) < 1e-12
        o += n
