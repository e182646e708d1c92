"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects bad descriptors before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flosic.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2108_01186_gb300 import build
    build.build()
    from paper_2108_01186_gb300 import flosic as F
    return F.load_library()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(flosic_\w+)\s*\(", text, re.M)))


def test_header_declares_the_step_calls():
    names = _declared()
    for n in ("flosic_build_flos", "flosic_orbital_poisson", "flosic_sic_energy_potential",
              "flosic_sic_backward", "flosic_create", "flosic_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_default_options(lib):
    from paper_2108_01186_gb300 import flosic as F
    o = F.FlosicOptions()
    assert lib.flosic_default_options(ctypes.byref(o)) == 0
    assert o.precision == F.MIXED and o.cg_tol == 1e-10 and o.preconditioner == F.PC_MG
    assert o.solver == F.SOLVER_PCG and (o.aar_omega, o.aar_beta, o.aar_m, o.aar_p) == (0.6, 0.6, 7, 6)
    assert o.kron_tensor_cores == 1
    assert o.autotune == 1
    assert lib.flosic_default_options(None) == F.FLOSIC_ERR_ARG


def _sys(**kw):
    from paper_2108_01186_gb300 import flosic as F
    s = F.FlosicSystem()
    s.nx = s.ny = s.nz = 8
    s.h = 0.5
    s.nspin = 1
    s.norb[0] = 2
    for k, v in kw.items():
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("bad", [dict(nx=0), dict(h=-1.0), dict(nspin=3)])
def test_create_rejects_bad_systems(lib, bad):
    from paper_2108_01186_gb300 import flosic as F
    h = ctypes.c_void_p()
    s = _sys(**bad)
    rc = lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, None)
    assert rc == F.FLOSIC_ERR_ARG
    assert not h.value
    assert len(lib.flosic_last_error(None)) > 0


def test_create_rejects_bad_options(lib):
    from paper_2108_01186_gb300 import flosic as F
    o = F.default_options(cg_tol=0.0)
    h = ctypes.c_void_p()
    s = _sys()
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, ctypes.byref(o)) == F.FLOSIC_ERR_ARG
    o = F.default_options(precision=7)
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, ctypes.byref(o)) == F.FLOSIC_ERR_ARG


@pytest.mark.parametrize("bad", [dict(solver=3), dict(solver=1, precision=0), dict(solver=1, aar_m=0),
                                 dict(solver=1, aar_m=9), dict(solver=1, aar_p=1), dict(solver=1, aar_omega=0.0),
                                 dict(solver=1, aar_beta=2.0)])
def test_create_rejects_bad_aar_options(lib, bad):
    # validated before any device work: the AAR solver runs only as the
    # float32 inner solver of the mixed path, history 1..8, p >= 2
    from paper_2108_01186_gb300 import flosic as F
    o = F.default_options(**bad)
    h = ctypes.c_void_p()
    s = _sys()
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, ctypes.byref(o)) == F.FLOSIC_ERR_ARG
    assert not h.value


def test_too_many_orbitals_rejected(lib):
    from paper_2108_01186_gb300 import flosic as F
    h = ctypes.c_void_p()
    s = _sys()
    s.norb[0] = 129
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, None) == F.FLOSIC_ERR_ARG


def test_null_context_calls_are_rejected(lib):
    from paper_2108_01186_gb300 import flosic as F
    assert lib.flosic_build_flos(None, None, None, None, None, None, None) == F.FLOSIC_ERR_ARG
    assert lib.flosic_destroy(None) == F.FLOSIC_OK
    out = (ctypes.c_int64 * 6)()
    assert lib.flosic_layout(None, out) == F.FLOSIC_ERR_ARG


@pytest.mark.parametrize("bad", [dict(solver=2, precision=0), dict(boundary=3), dict(boundary=1),
                                 dict(boundary=2, solver=1),
                                 dict(boundary=1, solver=2, adjoint_mode=1),
                                 dict(boundary=2, solver=2, fod_grad_mode=1)])
def test_create_rejects_bad_boundary_options(lib, bad):
    # extended boundaries run on the Kronecker solver only (mixed precision),
    # with the V-reusing adjoint and the interpolant's FOD gradient
    from paper_2108_01186_gb300 import flosic as F
    o = F.default_options(**bad)
    h = ctypes.c_void_p()
    s = _sys(nx=16, ny=16, nz=16)
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, ctypes.byref(o)) == F.FLOSIC_ERR_ARG
    assert not h.value


@pytest.mark.parametrize("dims,opts", [((12, 16, 16), dict(boundary=1, solver=2)),
                                       ((16, 12, 16), dict(boundary=2, solver=2)),
                                       ((16, 16, 257), dict(solver=2))])
def test_create_rejects_bad_extended_grids(lib, dims, opts):
    # periodic sides need 13 points (the stencil's taps stay distinct); the
    # Kronecker solver keeps its matrices in shared memory (n <= 256)
    from paper_2108_01186_gb300 import flosic as F
    o = F.default_options(**opts)
    h = ctypes.c_void_p()
    s = _sys(nx=dims[0], ny=dims[1], nz=dims[2])
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, ctypes.byref(o)) == F.FLOSIC_ERR_ARG
    assert b"13" in lib.flosic_last_error(None) or b"256" in lib.flosic_last_error(None)


def test_create_rejects_grids_beyond_32bit_point_indices(lib):
    # block-local point indices are 32-bit: nx*ny*nz must stay below 2^31
    from paper_2108_01186_gb300 import flosic as F
    h = ctypes.c_void_p()
    s = _sys(nx=1291, ny=1291, nz=1291)
    assert lib.flosic_create(ctypes.byref(h), ctypes.byref(s), 1, None) == F.FLOSIC_ERR_ARG
    assert not h.value
    assert b"grid points" in lib.flosic_last_error(None)
