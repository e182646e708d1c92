"""flosic_step_host: one whole step (FLO build, Poisson, energies, V_avg,
adjoint) with host arrays in and out.  It runs the same kernels as the four
device-pointer calls, so its outputs equal theirs; inputs handed over in
advance (psi_next, fods_next) are used on the next call that passes them."""
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


def _host(ctx, pinned=True):
    mk = (lambda n, dt=torch.float64: torch.empty(n, dtype=dt).pin_memory()) if pinned else \
        (lambda n, dt=torch.float64: torch.empty(n, dtype=dt))
    return dict(E_sic=mk(ctx.nsys), U=mk(ctx.norb), Exc=mk(ctx.norb), V_avg=mk(ctx.vavg_elems),
                dE_dpsi=mk(ctx.orb_elems), dE_dfod=mk(3 * ctx.norb), conv=mk(ctx.norb, torch.int32))


def _device_step(ctx, psi, fods, scale, gE):
    out = ctx.forward(psi.cuda(), fods.cuda(), scale=scale)
    g = torch.full((ctx.nsys,), gE, dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi.cuda(), fods.cuda(), out["phi"], out["V"], g)
    return dict(E_sic=out["E_sic"].cpu(), U=out["U"].cpu(), Exc=out["Exc"].cpu(), V_avg=out["V_avg"].cpu(),
                dE_dpsi=dpsi.cpu(), dE_dfod=dfod.cpu(), conv=out["conv"].cpu())


@pytest.mark.parametrize("prec", [0, 1])
def test_host_step_equals_the_device_calls(F, prec):
    s = synth.make_system(24, 0.4, 2, [3, 2], seed=8)
    ctx = F.Context([s], precision=prec, cg_tol=1e-12 if prec == 0 else 1e-10,
                    solver=F.SOLVER_PCG if prec == 0 else F.SOLVER_KRON)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi])).pin_memory()
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods])).pin_memory()
    ref = _device_step(ctx, psi, fods, 0.5, 1.3)
    out = _host(ctx)
    assert ctx.step_host(psi, fods, 0.5, 1.3, **out) == F.FLOSIC_OK
    for k, v in ref.items():
        assert torch.equal(out[k], v.to(out[k].dtype)), k


def test_host_step_prefetch_and_pageable_memory(F):
    s = synth.make_system(24, 0.4, 2, [3, 2], seed=8)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, solver=F.SOLVER_KRON)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi])).pin_memory()
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods])).pin_memory()
    fods2 = (fods + 0.01).pin_memory()                   # a second input set: moved FODs
    a, b = _host(ctx), _host(ctx)
    # call 1 copies the second set while it computes; call 2 uses that copy
    assert ctx.step_host(psi, fods, dE_dfod=a["dE_dfod"], E_sic=a["E_sic"], psi_next=psi, fods_next=fods2) == 0
    assert ctx.step_host(psi, fods2, E_sic=b["E_sic"], dE_dfod=b["dE_dfod"]) == 0
    ref1, ref2 = _device_step(ctx, psi, fods, 1.0, 1.0), _device_step(ctx, psi, fods2, 1.0, 1.0)
    assert torch.equal(a["E_sic"], ref1["E_sic"]) and torch.equal(a["dE_dfod"], ref1["dE_dfod"])
    assert torch.equal(b["E_sic"], ref2["E_sic"]) and torch.equal(b["dE_dfod"], ref2["dE_dfod"])
    assert not torch.equal(a["E_sic"], b["E_sic"])
    # pageable host arrays work too (copied synchronously); a prefetch that is not used is ignored
    pg = _host(ctx, pinned=False)
    assert ctx.step_host(psi.clone(), fods.clone(), psi_next=psi, fods_next=fods2, E_sic=pg["E_sic"]) == 0
    assert ctx.step_host(psi, fods, E_sic=pg["E_sic"]) == 0
    assert torch.equal(pg["E_sic"], ref1["E_sic"])


def test_host_step_pipelined_next_step_equals_the_device_calls(F):
    """With psi_next/fods_next the call starts the next step's FLO build and
    Poisson solve; the next call (its own scale and gE) must return exactly
    what the device calls return, over a chain of calls."""
    s = synth.make_system(24, 0.4, 2, [3, 2], seed=8)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, solver=F.SOLVER_KRON)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi])).pin_memory()
    fods = [torch.tensor(np.concatenate([f.ravel() for f in s.fods])).pin_memory()]
    fods += [(fods[0] + 0.01 * k).pin_memory() for k in (1, 2, 3)]
    params = [(1.0, 1.0), (0.5, 2.0), (0.75, -1.5), (1.0, 0.25)]
    outs = [_host(ctx) for _ in fods]
    for k in range(len(fods)):
        nxt = dict(psi_next=psi, fods_next=fods[k + 1]) if k + 1 < len(fods) else {}
        rc = ctx.step_host(psi, fods[k], params[k][0], params[k][1], **outs[k], **nxt)
        assert rc == F.FLOSIC_OK
    for k in range(len(fods)):
        ref = _device_step(ctx, psi, fods[k], *params[k])
        for name, v in ref.items():
            assert torch.equal(outs[k][name], v.to(outs[k][name].dtype)), (k, name)


def test_host_step_started_next_step_is_dropped_by_other_calls(F):
    """A device-pointer call between two host steps changes the workspace:
    the started next step must not be used (the next call recomputes)."""
    s = synth.make_system(24, 0.4, 2, [3, 2], seed=8)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, solver=F.SOLVER_KRON)
    psi = torch.tensor(np.concatenate([p.ravel() for p in s.psi])).pin_memory()
    fods = torch.tensor(np.concatenate([f.ravel() for f in s.fods])).pin_memory()
    fods2 = (fods + 0.02).pin_memory()
    a, b = _host(ctx), _host(ctx)
    assert ctx.step_host(psi, fods, **a, psi_next=psi, fods_next=fods2) == F.FLOSIC_OK
    # another system state through the device calls (moved FODs)
    ctx.forward(psi.cuda(), (fods - 0.03).cuda())
    assert ctx.step_host(psi, fods2, **b) == F.FLOSIC_OK
    ref = _device_step(ctx, psi, fods2, 1.0, 1.0)
    for name, v in ref.items():
        assert torch.equal(b[name], v.to(b[name].dtype)), name
