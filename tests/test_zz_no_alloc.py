"""The allocation-free Poisson entry point against the regular one.

flosic_orbital_poisson_noalloc serves callers that cannot allocate device
memory while they run (a framework's memory arena, a hard memory cap, a
latency-critical loop that must not take cudaMalloc/cudaFree).  Called
through the C ABI, twice in a row, it must give the potentials that
flosic_orbital_poisson gives for the same orbitals, within the FP64 Poisson
parity tolerance of the other GPU tests, and the oracle's potentials too.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2108_01186_gb300 import synth  # noqa: E402


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_01186_gb300 import build
    build.build()
    from paper_2108_01186_gb300 import flosic as F
    s = synth.make_system(21, 0.42, 2, [3], seed=31)      # ragged: G = 9261, several chunks
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi]), dtype=torch.float64, device="cuda")
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods]), dtype=torch.float64, device="cuda")
    ctx = F.Context([s], precision=F.FP64, cg_tol=1e-12, preconditioner=F.PC_NONE)
    phi, _, _ = ctx.build_flos(psi, fods)
    return F, s, ctx, phi


def test_noalloc_matches_regular_solve_twice(orc):
    F, s, ctx, phi = _setup()
    V_ref, it_ref, conv_ref = ctx.orbital_poisson(phi)
    assert np.all(conv_ref.cpu().numpy() == 1)
    ref = V_ref.cpu().numpy()
    it_ref = it_ref.cpu().numpy()
    scale = np.max(np.abs(ref))
    # the oracle's own solve of the same densities (the GPU's phi as input)
    V_orc, _ = orc.poisson(phi.cpu().numpy().reshape(3, -1) ** 2, s.grid, tol=1e-13)
    for call in range(2):
        V = torch.full_like(phi, float("nan"))
        iters = torch.zeros(3, dtype=torch.int32, device="cuda")
        conv = torch.zeros(3, dtype=torch.int32, device="cuda")
        rc = F.orbital_poisson_noalloc(s.grid, phi, V, cg_tol=1e-12, max_iter=20000, iters=iters, conv=conv)
        assert rc == F.FLOSIC_OK, F.load_library().flosic_noalloc_last_error()
        torch.cuda.synchronize()
        assert np.all(conv.cpu().numpy() == 1)
        # the same plain CG as the regular FP64 path: the same iteration counts, to a step or two
        assert np.all(np.abs(iters.cpu().numpy() - it_ref) <= 2), (iters.cpu().numpy(), it_ref)
        Vn = V.cpu().numpy()
        assert np.max(np.abs(Vn - ref)) < 1e-10 * scale, call
        assert np.max(np.abs(Vn - V_orc.ravel())) < 1e-10 * scale, call
    # without the optional outputs
    V = torch.full_like(phi, float("nan"))
    rc = F.orbital_poisson_noalloc(s.grid, phi, V, cg_tol=1e-12, max_iter=20000)
    assert rc == F.FLOSIC_OK, F.load_library().flosic_noalloc_last_error()
    torch.cuda.synchronize()
    assert np.max(np.abs(V.cpu().numpy() - ref)) < 1e-10 * scale


def test_noalloc_reports_noconv_and_refuses_oversize():
    F, s, ctx, phi = _setup()
    # three iterations cannot reach 1e-12: NOCONV, every flag 0, finite V
    V = torch.full_like(phi, float("nan"))
    iters = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    conv = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    rc = F.orbital_poisson_noalloc(s.grid, phi, V, cg_tol=1e-12, max_iter=3, iters=iters, conv=conv)
    torch.cuda.synchronize()
    assert rc == F.FLOSIC_ERR_NOCONV
    assert np.all(conv.cpu().numpy() == 0)
    assert np.all(iters.cpu().numpy() == 3)
    assert np.all(np.isfinite(V.cpu().numpy()))
    assert b"max_iter" in F.load_library().flosic_noalloc_last_error()
    # sizes beyond the static scratch are refused before any work is queued
    big = (128, 128, 128, 0.2, np.zeros(3))
    phi_big = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert F.orbital_poisson_noalloc(big, phi_big.expand(128 ** 3).contiguous(), phi_big.expand(128 ** 3).contiguous()) \
        == F.FLOSIC_ERR_ARG
    # and a later call still works
    V = torch.full_like(phi, float("nan"))
    assert F.orbital_poisson_noalloc(s.grid, phi, V, cg_tol=1e-12, max_iter=20000) == F.FLOSIC_OK
