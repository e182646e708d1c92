"""The orbital-unit partition on one GPU: a step run with two complementary
orbital masks (the shares of two ranks, as paper_2108_01186_gb300.dist
assigns them) sums to the unmasked step, FP64 and mixed precision.  E_SIC,
U and E_xc sum over orbitals (Eq. 1), V_avg's numerator sums over orbitals
(Eq. 13), and the FOD gradient and dE/dpsi are linear in the per-orbital
adjoint seeds (Eqs. 9-11)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2108_01186_gb300 import dist as D  # noqa: E402
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


def _step(ctx, psi, fods, gE):
    out = ctx.forward(psi, fods, scale=0.5)
    dpsi, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    return {k: _np(v) for k, v in out.items() if k in ("V", "iters", "conv", "E_sic", "V_avg", "U", "Exc")} | \
        dict(dpsi=_np(dpsi), dfod=_np(dfod))


@pytest.mark.parametrize("prec", [0, 1])
def test_complementary_masks_sum_to_the_unmasked_step(F, prec):
    s = synth.make_system(40, 0.3, 3, [3, 2], seed=5)
    ctx = F.Context([s], precision=prec, cg_tol=1e-12 if prec == 0 else 1e-10,
                    solver=F.SOLVER_PCG if prec == 0 else F.SOLVER_KRON)
    psi, fods = _flat(s.psi), _flat(s.fods)
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    full = _step(ctx, psi, fods, gE)
    parts = []
    for rank in range(2):
        mask = D.orbital_mask(ctx.norb, rank, 2)
        ctx.set_orbital_mask(mask)
        p = _step(ctx, psi, fods, gE)
        m = np.array(mask)
        # masked orbitals: V = 0, 0 iterations, reported converged
        V = p["V"].reshape(ctx.norb, -1)
        assert np.all(V[m == 0] == 0) and np.all(p["iters"][m == 0] == 0) and np.all(p["conv"] == 1)
        assert np.all(p["U"][m == 0] == 0) and np.all(p["Exc"][m == 0] == 0)
        parts.append(p)
    ctx.set_orbital_mask(None)
    again = _step(ctx, psi, fods, gE)             # back to every orbital
    assert np.array_equal(again["E_sic"], full["E_sic"])
    rel = 1e-12 if prec == 0 else 2e-6
    Vfull = full["V"].reshape(ctx.norb, -1)
    Vsum = parts[0]["V"].reshape(ctx.norb, -1) + parts[1]["V"].reshape(ctx.norb, -1)
    assert np.max(np.abs(Vsum - Vfull)) <= rel * np.max(np.abs(Vfull))
    for k in ("E_sic", "U", "Exc", "V_avg", "dfod", "dpsi"):
        tot = parts[0][k] + parts[1][k]
        assert np.max(np.abs(tot - full[k])) <= rel * max(1.0, np.max(np.abs(full[k]))), k


def test_mask_rejects_bad_entries(F):
    s = synth.make_system(21, 0.42, 2, [3], seed=31)
    ctx = F.Context([s], precision=0)
    with pytest.raises(F.FlosicError):
        ctx.set_orbital_mask([1, 2, 0])
    ctx64x = F.Context([s], precision=0, adjoint_mode=F.ADJ_EXACT)
    with pytest.raises(F.FlosicError):
        ctx64x.set_orbital_mask([1, 0, 0])
    ctx64x.set_orbital_mask([1, 1, 1])            # a full mask is always allowed
