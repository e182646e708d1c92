"""The Alternating Anderson-Richardson inner solver (the electrostatics
iteration of Sec. II.A) against the FP64 oracle and against the CG path.

AAR replaces only the float32 inner solve of the mixed refinement; the
float-float outer loop still stops at ||b - A V|| <= tol ||b||, so the
tolerances are those of the mixed CG path: 1e-8 of max|V| at tol 1e-10
on the Poisson solutions, 1e-6 Ha per orbital on the energies.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2108_01186_gb300 import synth  # noqa: E402


def _flat(arrs):
    return torch.tensor(np.concatenate([a.ravel() for a in arrs]), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


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


def _poisson_refs(orc, s):
    fl = [orc.build_flos(s.psi[sp], s.fods[sp], s.grid) for sp in range(len(s.psi))]
    Vref = [orc.poisson(f["phi"] ** 2, s.grid, tol=1e-13)[0] for f in fl]
    return _flat([f["phi"] for f in fl]), Vref


def _check_V(V, Vref, s, vtol):
    off = 0
    Vn = _np(V)
    for sp, N in enumerate(s.norb):
        Vb = Vn[off * s.G:(off + N) * s.G].reshape(N, s.G)
        assert np.max(np.abs(Vb - Vref[sp])) < vtol * np.max(np.abs(Vref[sp]))
        off += N


@pytest.mark.parametrize("pc", [0, 1])
def test_aar_poisson_parity_ragged(F, orc, pc):
    # ragged grid (21^3, not a multiple of any tile), two spins of unequal size
    s = synth.make_system(21, 0.42, 2, [3, 2], seed=31)
    phi, Vref = _poisson_refs(orc, s)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, preconditioner=pc, solver=F.SOLVER_AAR)
    V, iters, conv = ctx.orbital_poisson(phi)
    assert np.all(_np(conv) == 1)
    _check_V(V, Vref, s, 1e-8)


@pytest.mark.parametrize("m,p,omega,beta", [(7, 6, 0.6, 0.6), (1, 2, 1.0, 1.0), (8, 3, 0.8, 0.5)])
def test_aar_parameters_converge_to_the_same_solution(F, orc, m, p, omega, beta):
    # 40^3 grid: several multigrid levels and several level-0 tiles per orbital
    s = synth.make_system(40, 0.3, 3, [5], seed=7)
    phi, Vref = _poisson_refs(orc, s)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, preconditioner=F.PC_MG, solver=F.SOLVER_AAR,
                    aar_m=m, aar_p=p, aar_omega=omega, aar_beta=beta)
    V, iters, conv = ctx.orbital_poisson(phi)
    assert np.all(_np(conv) == 1)
    _check_V(V, Vref, s, 1e-8)


def test_aar_multigrid_against_cg_and_jacobi(F, orc):
    s = synth.make_system(40, 0.3, 3, [5], seed=7)
    phi, Vref = _poisson_refs(orc, s)
    its = {}
    for name, kw in (("cg", dict(solver=F.SOLVER_PCG, preconditioner=F.PC_MG)),
                     ("aar_mg", dict(solver=F.SOLVER_AAR, preconditioner=F.PC_MG)),
                     ("aar_jacobi", dict(solver=F.SOLVER_AAR, preconditioner=F.PC_NONE))):
        ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, **kw)
        V, it, conv = ctx.orbital_poisson(phi)
        assert np.all(_np(conv) == 1), name
        _check_V(V, Vref, s, 1e-8)
        its[name] = _np(it).max()
    # the V-cycle makes AAR grid-independent; Jacobi-preconditioned AAR is
    # much slower on a 40^3 grid
    assert its["aar_mg"] * 5 < its["aar_jacobi"], its


def test_aar_warm_start_and_forward_energies(F, orc):
    s = synth.make_config(0)
    ref = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-12)
    psi, fods = _flat(s.psi), _flat(s.fods)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, preconditioner=F.PC_MG, solver=F.SOLVER_AAR)
    out = ctx.forward(psi, fods)
    assert np.all(_np(out["conv"]) == 1)
    assert np.max(np.abs(_np(out["U"]) - ref["blocks"][0]["U"])) < 1e-6
    assert np.max(np.abs(_np(out["Exc"]) - ref["blocks"][0]["Exc"])) < 1e-6
    assert abs(_np(out["E_sic"])[0] - ref["E_sic"]) < 1e-6
    assert np.max(np.abs(_np(out["V"]).reshape(5, -1) - ref["blocks"][0]["V"])) < 1e-6
    # a warm start from the converged potentials needs (almost) no work
    phi = out["phi"]
    V0, it0, _ = ctx.orbital_poisson(phi)
    V1, it1, conv = ctx.orbital_poisson(phi, V0.clone())
    assert np.all(_np(conv) == 1)
    assert _np(it1).max() < _np(it0).min()


def test_aar_uneven_batch(F, orc):
    systems = [synth.make_system(18, 0.45, 2, [3], seed=41),
               synth.make_system(23, 0.35, 2, [4, 2], seed=42),
               synth.make_system(5, 0.9, 1, [1], seed=44),
               synth.make_system(24, 0.5, 2, [5], seed=46)]
    ctx = F.Context(systems, precision=F.MIXED, cg_tol=1e-11, preconditioner=F.PC_MG, solver=F.SOLVER_AAR)
    psi = _flat([p for s in systems for p in s.psi])
    fods = _flat([f for s in systems for f in s.fods])
    out = ctx.forward(psi, fods, scale=0.5)
    assert np.all(_np(out["conv"]) == 1)
    E = _np(out["E_sic"])
    for k, s in enumerate(systems):
        ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-12)
        assert abs(E[k] - ref["E_sic"]) < 1e-6 * len(s.psi[0])
