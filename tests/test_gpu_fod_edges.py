"""GPU parity with FODs where the tricubic interpolation (Sec. II.B) meets
its edge cases: a FOD in the outermost cell of the box, so that some of its
64 nodes lie outside the grid (they read as zero), and a FOD within 1e-3 h
of a node plane along one direction and exactly on a node plane along
another (the cell with t = 0 is taken).  Forward (FLOs, energies, V_avg) and
adjoint (FOD gradient, dE/dpsi) are compared with the oracle element by
element, FP64 and mixed precision.
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


@pytest.fixture(scope="module")
def edge_system():
    s = synth.make_system(21, 0.42, 2, [3, 2], seed=31)
    nx, ny, nz, h, o = s.grid
    f = [x.copy() for x in s.fods]
    # FOD 0 of spin 0: the outermost cell along x (node -1 outside) and along y (node ny outside)
    f[0][0] = [o[0] + 0.37 * h, o[1] + (ny - 1.6) * h, f[0][0][2]]
    # FOD 1 of spin 0: 4e-4 h past a node plane along x, exactly on a node plane along z
    i = int(round((f[0][1][0] - o[0]) / h))
    k = int(round((f[0][1][2] - o[2]) / h))
    f[0][1] = [o[0] + (i + 4e-4) * h, f[0][1][1], o[2] + k * h]
    # FOD 1 of spin 1: the last cell along z (node nz outside)
    f[1][1] = [f[1][1][0], f[1][1][1], o[2] + (nz - 1.25) * h]
    s.fods = f
    return s


@pytest.mark.parametrize("prec", [0, 1])
def test_edge_fods_forward_and_adjoint(F, orc, edge_system, prec):
    s = edge_system
    ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-13)
    dpsi_ref, dfod_ref = orc.sic_backward(ref, s.grid, tol=1e-13)
    ctx = F.Context([s], precision=prec, cg_tol=1e-12 if prec == 0 else 1e-10, preconditioner=F.PC_MG,
                    solver=F.SOLVER_PCG if prec == 0 else F.SOLVER_KRON)
    psi, fods = _flat(s.psi), _flat(s.fods)
    out = ctx.forward(psi, fods, scale=0.5)
    assert np.all(_np(out["conv"]) == 1)
    phi = _np(out["phi"])
    G = s.G
    off = 0
    for sp, N in enumerate(s.norb):
        pr = ref["blocks"][sp]["phi"]
        tol = 1e-11 if prec == 0 else 2e-6
        assert np.max(np.abs(phi[off * G:(off + N) * G].reshape(N, G) - pr)) < tol * np.max(np.abs(pr))
        off += N
    # mixed: the per-orbital energy bar of the mixed path (measured U error 2e-7 Ha here)
    etol = 1e-10 if prec == 0 else 1e-6
    assert np.max(np.abs(_np(out["U"]) - np.concatenate([b["U"] for b in ref["blocks"]]))) < etol
    assert np.max(np.abs(_np(out["Exc"]) - np.concatenate([b["Exc"] for b in ref["blocks"]]))) < etol
    assert abs(_np(out["E_sic"])[0] - ref["E_sic"]) < etol * sum(s.norb)
    Va = _np(out["V_avg"]).reshape(2, G)
    for sp in range(2):
        rho_s = np.sum(s.psi[sp] ** 2, axis=0)
        m = rho_s > 1e-12
        assert np.max(np.abs(Va[sp][m] - ref["blocks"][sp]["Vavg"][m])) < (1e-9 if prec == 0 else 1e-6)
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    g = _np(dfod).reshape(-1, 3)
    gr = np.concatenate(dfod_ref)
    assert np.max(np.abs(g - gr)) < (1e-9 if prec == 0 else 1e-5)
    dp = np.concatenate([d.ravel() for d in dpsi_ref])
    assert np.max(np.abs(_np(dpsi) - dp)) < (1e-9 if prec == 0 else 1e-5) * np.max(np.abs(dp))
