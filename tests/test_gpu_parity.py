"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (derived from the arithmetic):
* FP64 path, solves to 1e-12: potentials agree to ~1e-10 of max|V|; FLOs,
  overlaps and gradients to ~1e-10 (different but exact-in-FP64 orderings
  and eigen-solvers).
* MIXED path, solves to 1e-10: potentials and per-orbital energies within
  1e-6 Ha, FOD gradients within 1e-5 Ha/bohr (the accuracy targets of the
  mixed path).
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


def _blocks(t, systems):
    """Split a packed orbital array into per (system, spin) [N, G] arrays."""
    out, off = [], 0
    for s in systems:
        per = []
        for N in s.norb:
            per.append(t[off:off + N * s.G].reshape(N, s.G))
            off += N * s.G
        out.append(per)
    return out


# ragged grid (G not a multiple of the chunk), two spins of unequal size
@pytest.fixture(scope="module")
def ragged():
    s = synth.make_system(21, 0.42, 2, [3, 2], seed=31)
    return s


@pytest.mark.parametrize("prec", [0, 1])
def test_build_flos_parity(F, orc, ragged, prec):
    s = ragged
    ctx = F.Context([s], precision=prec)
    phi, S, Q = ctx.build_flos(_flat(s.psi), _flat(s.fods))
    phi_b = _blocks(_np(phi), [s])[0]
    # FP64: float64 throughout; MIXED: grid products in float32 with float64
    # sums over 16-point tiles (relative error ~1e-7)
    tphi, tS = (1e-11, 1e-12) if prec == 0 else (2e-6, 1e-6)
    off = 0
    for sp in range(2):
        fl = orc.build_flos(s.psi[sp], s.fods[sp], s.grid)
        N = s.norb[sp]
        assert np.max(np.abs(phi_b[sp] - fl["phi"])) < tphi * np.max(np.abs(fl["phi"]))
        assert np.max(np.abs(_np(S)[off:off + N * N].reshape(N, N) - fl["S"])) < tS
        assert np.max(np.abs(_np(Q)[off:off + N * N].reshape(N, N) - fl["Q"])) < 10 * tS
        off += N * N


@pytest.mark.parametrize("pc", [0, 1])
@pytest.mark.parametrize("prec,tol,vtol", [(0, 1e-12, 1e-10), (1, 1e-10, 1e-8)])
def test_poisson_parity(F, orc, ragged, prec, tol, vtol, pc):
    s = ragged
    fl = [orc.build_flos(s.psi[sp], s.fods[sp], s.grid) for sp in range(2)]
    phi = _flat([f["phi"] for f in fl])
    ctx = F.Context([s], precision=prec, cg_tol=tol, preconditioner=pc)
    V, iters, conv = ctx.orbital_poisson(phi)
    assert np.all(_np(conv) == 1)
    Vb = _blocks(_np(V), [s])[0]
    for sp in range(2):
        Vref, _ = orc.poisson(fl[sp]["phi"] ** 2, s.grid, tol=1e-13)
        assert np.max(np.abs(Vb[sp] - Vref)) < vtol * np.max(np.abs(Vref))


def test_poisson_warm_start_converges_immediately(F, orc, ragged):
    s = ragged
    fl = [orc.build_flos(s.psi[sp], s.fods[sp], s.grid) for sp in range(2)]
    phi = _flat([f["phi"] for f in fl])
    ctx = F.Context([s], precision=0, cg_tol=1e-10, preconditioner=0)
    V, it0, _ = ctx.orbital_poisson(phi)
    V2, it1, conv = ctx.orbital_poisson(phi, V.clone())
    assert np.all(_np(conv) == 1)
    assert _np(it1).max() < _np(it0).min()


@pytest.mark.parametrize("scale", [1.0, 0.5])
def test_energy_potential_parity(F, orc, ragged, scale):
    s = ragged
    ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=scale, tol=1e-13)
    ctx = F.Context([s], precision=0)
    psi = _flat(s.psi)
    phi = _flat([b["phi"] for b in ref["blocks"]])
    V = _flat([b["V"] for b in ref["blocks"]])
    E, Vavg, U, Exc = ctx.sic_energy_potential(psi, phi, V, scale)
    assert abs(_np(E)[0] - ref["E_sic"]) < 1e-12
    assert np.max(np.abs(_np(U) - np.concatenate([b["U"] for b in ref["blocks"]]))) < 1e-13
    assert np.max(np.abs(_np(Exc) - np.concatenate([b["Exc"] for b in ref["blocks"]]))) < 1e-13
    Va = _np(Vavg).reshape(2, s.G)
    for sp in range(2):
        assert np.max(np.abs(Va[sp] - ref["blocks"][sp]["Vavg"])) < 1e-11


@pytest.mark.parametrize("adjoint,grad_mode", [(0, 0), (1, 0), (0, 1)])
def test_backward_parity(F, orc, ragged, adjoint, grad_mode):
    s = ragged
    ref = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-13)
    dpsi_ref, dfod_ref = orc.sic_backward(ref, s.grid, gE=1.7,
                                          adjoint=("reuse_v", "exact")[adjoint],
                                          grad_mode=("interp_exact", "paper_central")[grad_mode], tol=1e-13)
    ctx = F.Context([s], precision=0, cg_tol=1e-13, adjoint_mode=adjoint, fod_grad_mode=grad_mode,
                    preconditioner=0)
    psi, fods = _flat(s.psi), _flat(s.fods)
    phi, _, _ = ctx.build_flos(psi, fods)
    V = _flat([b["V"] for b in ref["blocks"]])
    gE = torch.tensor([1.7], dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi, fods, phi, V, gE)
    g = _np(dfod).reshape(-1, 3)
    gr = np.concatenate(dfod_ref)
    assert np.max(np.abs(g - gr)) < 1e-9 * max(1.0, np.max(np.abs(gr)))
    dp = np.concatenate([d.ravel() for d in dpsi_ref])
    assert np.max(np.abs(_np(dpsi) - dp)) < 1e-9 * np.max(np.abs(dp))


@pytest.mark.parametrize("pc", [0, 1])
def test_forward_config0_fp64_and_mixed(F, orc, pc):
    s = synth.make_config(0)
    ref = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-12)
    psi, fods = _flat(s.psi), _flat(s.fods)
    for prec in (0, 1):
        ctx = F.Context([s], precision=prec, cg_tol=1e-10, preconditioner=pc)
        out = ctx.forward(psi, fods)
        assert np.all(_np(out["conv"]) == 1)
        Uref = ref["blocks"][0]["U"]
        # FP64: everything in float64; MIXED: float32 CG + float64 refinement
        # and float32 pointwise xc summed in float64 (1e-6 Ha per orbital)
        etol = 1e-9 if prec == 0 else 1e-6
        assert np.max(np.abs(_np(out["U"]) - Uref)) < max(etol, 1e-7)
        assert np.max(np.abs(_np(out["Exc"]) - ref["blocks"][0]["Exc"])) < etol
        assert abs(_np(out["E_sic"])[0] - ref["E_sic"]) < 1e-6
        assert np.max(np.abs(_np(out["V"]).reshape(5, -1) - ref["blocks"][0]["V"])) < 1e-6


@pytest.mark.parametrize("pc", [0, 1])
def test_uneven_batch_matches_per_system_oracle(F, orc, pc):
    # different grids give different multigrid depths (5 is a single level)
    # aligned rows (nx % 4 == 0: copy-engine stencil) and unaligned ones
    # (plain-load stencil) in the same batch
    systems = [synth.make_system(18, 0.45, 2, [3], seed=41),
               synth.make_system(23, 0.35, 2, [4, 2], seed=42),
               synth.make_system(15, 0.5, 1, [1], seed=43),
               synth.make_system(5, 0.9, 1, [1], seed=44),
               synth.make_system(20, 0.45, 1, [3, 3], seed=45),
               synth.make_system(24, 0.5, 2, [5], seed=46)]
    ctx = F.Context(systems, precision=1, cg_tol=1e-11, preconditioner=pc)
    psi = _flat([p for s in systems for p in s.psi])
    fods = _flat([f for s in systems for f in s.fods])
    out = ctx.forward(psi, fods, scale=0.5)
    E = _np(out["E_sic"])
    for k, s in enumerate(systems):
        ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-12)
        assert abs(E[k] - ref["E_sic"]) < 1e-6 * len(s.psi[0])


def test_single_orbital_fod_gradient_vanishes(F):
    s = synth.make_system(16, 0.5, 1, [1], seed=8)
    ctx = F.Context([s], precision=0, cg_tol=1e-12, preconditioner=0)
    psi, fods = _flat(s.psi), _flat(s.fods)
    out = ctx.forward(psi, fods)
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    _, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    assert np.max(np.abs(_np(dfod))) < 1e-12


def test_error_paths(F):
    s = synth.make_system(16, 0.5, 2, [3], seed=9)
    psi, fods = _flat(s.psi), _flat(s.fods)
    ctx = F.Context([s], precision=1)
    f2 = fods.clone().reshape(-1, 3)
    f2[1] = f2[0]
    with pytest.raises(F.FlosicError) as e:
        ctx.build_flos(psi, f2.reshape(-1))
    assert e.value.code == F.FLOSIC_ERR_ILLCOND
    p2 = psi.clone()
    p2[5] = float("nan")
    with pytest.raises(F.FlosicError) as e:
        ctx.build_flos(p2, fods)
    assert e.value.code == F.FLOSIC_ERR_NONFINITE
    ctx2 = F.Context([s], precision=0, max_iter=3, preconditioner=0)
    phi, _, _ = ctx2.build_flos(psi, fods)
    with pytest.raises(F.FlosicError) as e:
        ctx2.orbital_poisson(phi)
    assert e.value.code == F.FLOSIC_ERR_NOCONV
    V, iters, conv = ctx2.orbital_poisson(phi, check=False)
    assert np.all(_np(conv) == 0) and np.all(_np(iters) <= 3)
    with pytest.raises(F.FlosicError) as e:
        F.Context([s]).sic_backward(psi, fods, phi, V, torch.ones(1, dtype=torch.float64, device="cuda"))
    assert e.value.code == F.FLOSIC_ERR_ARG


def test_autograd_function(F, orc):
    s = synth.make_system(20, 0.45, 2, [3], seed=12)
    ctx = F.Context([s], precision=1, cg_tol=1e-11, preconditioner=0)
    psi = _flat(s.psi).requires_grad_(True)
    fods = _flat(s.fods).requires_grad_(True)
    E, Vavg, U, Exc = F.FlosicStep.apply(ctx, psi, fods, 1.0)
    (2.0 * E.sum()).backward()
    ref = orc.sic_forward(s.psi, s.fods, s.grid, tol=1e-12)
    _, g = orc.sic_backward(ref, s.grid, gE=2.0)
    assert np.max(np.abs(_np(fods.grad).reshape(-1, 3) - g[0])) < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_multigrid_cuts_iterations(F, orc, prec):
    s = synth.make_system(40, 0.3, 3, [5], seed=7)
    fl = orc.build_flos(s.psi[0], s.fods[0], s.grid)
    phi = _flat([fl["phi"]])
    its = {}
    Vs = {}
    for pc in (0, 1):
        ctx = F.Context([s], precision=prec, cg_tol=1e-10, preconditioner=pc)
        V, it, conv = ctx.orbital_poisson(phi)
        assert np.all(_np(conv) == 1)
        its[pc] = _np(it).max()
        Vs[pc] = _np(V)
    assert its[1] * 5 < its[0]
    assert np.max(np.abs(Vs[1] - Vs[0])) < 1e-8 * np.max(np.abs(Vs[0]))
