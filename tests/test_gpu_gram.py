"""Tensor-core overlap (split-BF16 tcgen05 Gram, mixed precision) for wide
spin blocks, against the oracle's FLO build: 70 and 120 orbitals exercise
the 96- and 128-column accumulators (fewer orbitals are covered by the
other parity tests); a 40-orbital block covers the mixed-precision adjoint's
wide tile shapes."""
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


@pytest.mark.parametrize("N,natoms", [(70, 18), (120, 30)])
def test_wide_block_overlap_and_flos(F, orc, N, natoms):
    s = synth.make_system(40, 0.5, natoms, [N], seed=900 + N)
    psi = torch.tensor(s.psi[0].ravel(), device="cuda")
    fods = torch.tensor(s.fods[0].ravel(), device="cuda")
    fl = orc.build_flos(s.psi[0], s.fods[0], s.grid)
    lam = np.linalg.eigvalsh(fl["S"])
    for prec, stol in ((F.MIXED, 1e-6), (F.FP64, 1e-11)):
        ctx = F.Context([s], precision=prec, cg_tol=1e-10)
        phi, S, Q = ctx.build_flos(psi, fods)
        S = S.cpu().numpy().reshape(N, N)
        phi = phi.cpu().numpy().reshape(N, -1)
        err = np.max(np.abs(S - fl["S"]))
        assert err < stol, (prec, err)
        # phi = S^{-1/2} F amplifies an error in S by up to 1/lambda_min
        ptol = 4.0 * stol / lam[0] + (2e-6 if prec == F.MIXED else 1e-12)
        perr = np.max(np.abs(phi - fl["phi"])) / np.max(np.abs(fl["phi"]))
        assert perr < ptol, (prec, perr, ptol, lam[0])


def test_wide_block_mixed_adjoint(F, orc):
    # 40 orbitals: the adjoint contraction's 64-wide tile shape and the general
    # small-matrix product for psibar (blocks of more than 32 orbitals), mixed
    # precision, against the oracle's adjoint on the GPU's own phi and V
    s = synth.make_system(40, 0.5, 10, [40], seed=946)
    N, G = 40, s.G
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10)
    psi = torch.tensor(s.psi[0].ravel(), device="cuda")
    fods = torch.tensor(s.fods[0].ravel(), device="cuda")
    out = ctx.forward(psi, fods)
    assert np.all(out["conv"].cpu().numpy() == 1)
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    ph = out["phi"].cpu().numpy().reshape(N, G)
    Vb = out["V"].cpu().numpy().reshape(N, G)
    fl = orc.build_flos(s.psi[0], s.fods[0], s.grid)
    rho = ph ** 2
    eps, vxc = orc.lsda_pol(rho)
    fl.update(rho=rho, V=Vb, eps=eps, vxc=vxc, psi=s.psi[0], fods=s.fods[0])
    dpsi_ref, dfod_ref = orc.sic_backward(dict(blocks=[fl], E_sic=0.0), s.grid)
    assert np.max(np.abs(dfod.cpu().numpy().reshape(-1, 3) - dfod_ref[0])) < 2e-6
    dp = dpsi_ref[0].ravel()
    assert np.max(np.abs(dpsi.cpu().numpy() - dp)) / np.max(np.abs(dp)) < 4e-6
