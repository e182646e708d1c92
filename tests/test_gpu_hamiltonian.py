"""SC_AvgSIC Hamiltonian apply (Sec. II.C, Eq. 13) on the GPU against the
oracle: every orbital at the 40^3 and uneven sizes (float64 and mixed
precision), sampled orbitals at 128^3, argument errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2108_01186_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01186_gb300 import build
    build.build()
    from paper_2108_01186_gb300 import flosic
    return flosic


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build_library()
    return oracle


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def _check(F, orc, systems, prec, rtol, rng):
    ctx = F.Context(systems, precision=prec, cg_tol=1e-10)
    psi = _dev(np.concatenate([p.ravel() for s in systems for p in s.psi]))
    vloc = [rng.normal(size=s.G) * 0.3 - 1.0 for s in systems]
    vavg = [rng.normal(size=s.G) * 0.1 for s in systems for _ in s.norb]
    H = ctx.hamiltonian_apply(psi, _dev(np.concatenate(vloc)), _dev(np.concatenate(vavg))).cpu().numpy()
    H0 = ctx.hamiltonian_apply(psi).cpu().numpy()
    off, blk = 0, 0
    for si, s in enumerate(systems):
        for sp, N in enumerate(s.norb):
            ref = orc.hamiltonian_apply(s.psi[sp], s.grid, vloc[si], vavg[blk])
            ref0 = orc.hamiltonian_apply(s.psi[sp], s.grid)
            got = H[off:off + N * s.G].reshape(N, s.G)
            got0 = H0[off:off + N * s.G].reshape(N, s.G)
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(got - ref)) < rtol * scale, (si, sp, np.max(np.abs(got - ref)) / scale)
            assert np.max(np.abs(got0 - ref0)) < rtol * np.max(np.abs(ref0))
            off += N * s.G
            blk += 1


@pytest.mark.parametrize("prec,rtol", [(0, 1e-13), (1, 1e-12)])
def test_hamiltonian_matches_oracle(F, orc, prec, rtol):
    rng = np.random.default_rng(7)
    systems = [synth.make_config(0), synth.make_system(23, 0.35, 2, [4, 2], seed=42),
               synth.make_system(15, 0.5, 1, [1], seed=43)]
    _check(F, orc, systems, prec, rtol, rng)


def test_hamiltonian_full_size_sampled(F, orc):
    s = synth.make_config(3)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10)
    psi = _dev(np.concatenate([p.ravel() for p in s.psi]))
    rng = np.random.default_rng(11)
    vavg = [rng.normal(size=s.G) * 0.1 for _ in s.norb]
    H = ctx.hamiltonian_apply(psi, None, _dev(np.concatenate(vavg))).cpu().numpy()
    G, N = s.G, s.norb[0]
    for sp, a in ((0, 0), (0, N - 1), (1, 5)):
        ref = orc.hamiltonian_apply(s.psi[sp][a], s.grid, None, vavg[sp])[0]
        got = H[(sp * N + a) * G:(sp * N + a + 1) * G]
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hamiltonian_argument_errors(F):
    s = synth.make_system(12, 0.5, 1, [2], seed=5)
    ctx = F.Context([s])
    psi = _dev(np.concatenate([p.ravel() for p in s.psi]))
    L = F.load_library()
    assert L.flosic_hamiltonian_apply(ctx._h, F._ptr(psi), None, None, F._ptr(psi), F._stream()) == F.FLOSIC_ERR_ARG
    assert L.flosic_hamiltonian_apply(ctx._h, None, None, None, F._ptr(psi), F._stream()) == F.FLOSIC_ERR_ARG
    assert L.flosic_hamiltonian_apply(None, F._ptr(psi), None, None, F._ptr(psi), F._stream()) == F.FLOSIC_ERR_ARG
