"""The Kronecker-product solver and the extended-system boundaries (Sec.
II.A: the Kronecker form of the Laplacian; periodic conditions along
extended directions; dipole-corrected Dirichlet values for surfaces) on the
GPU against the FP64 oracle.

The KRON solver replaces only the float32 inner solve of the mixed
refinement (the float-float residual still stops at ||b - A V|| <= tol ||b||),
so the tolerances are those of the mixed CG path: 1e-8 of max|V| at tol
1e-10 on the Poisson solutions, 1e-6 Ha per orbital on energies and
potentials, 1e-5 Ha/bohr on FOD gradients.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2108_01186_gb300 import synth  # noqa: E402

BC_NAMES = {0: "isolated", 1: "periodic", 2: "slab"}


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


def _ctx(F, systems, bc, tol=1e-10):
    return F.Context(systems, precision=F.MIXED, cg_tol=tol, solver=F.SOLVER_KRON, boundary=bc)


def _check_poisson(F, orc, s, bc, vtol=1e-8):
    name = BC_NAMES[bc]
    fl = [orc.build_flos(s.psi[sp], s.fods[sp], s.grid, bc=name) for sp in range(len(s.psi))]
    ctx = _ctx(F, [s], bc)
    V, iters, conv = ctx.orbital_poisson(_flat([f["phi"] for f in fl]))
    assert np.all(_np(conv) == 1)
    Vn = _np(V)
    off = 0
    for sp, N in enumerate(s.norb):
        Vref, _ = orc.poisson(fl[sp]["phi"] ** 2, s.grid, tol=1e-13, bc=name)
        got = Vn[off * s.G:(off + N) * s.G].reshape(N, s.G)
        assert np.max(np.abs(got - Vref)) < vtol * np.max(np.abs(Vref)), (name, sp)
        off += N
    return _np(iters)


def test_kron_isolated_poisson_parity(F, orc):
    # ragged grid (21^3), two spins of unequal size; a 40^3 grid
    its = _check_poisson(F, orc, synth.make_system(21, 0.42, 2, [3, 2], seed=31), 0)
    assert its.max() <= 6
    its = _check_poisson(F, orc, synth.make_system(40, 0.3, 3, [5], seed=7), 0)
    assert its.max() <= 6


def test_kron_cold_start_zero_orbital_and_repeat(F, orc):
    # A cold start of the Kronecker refinement stores neither x = 0 nor d = 0:
    # an orbital with phi = 0 needs no solve and must come out V = 0 exactly,
    # and a second cold solve on the same context (workspace holding the first
    # one's x and d) must give the same potentials bit for bit.
    s = synth.make_system(24, 0.4, 2, [3, 2], seed=33)
    fl = [orc.build_flos(s.psi[sp], s.fods[sp], s.grid) for sp in range(2)]
    phis = [fl[0]["phi"].copy(), fl[1]["phi"].copy()]
    phis[0][1] = 0.0
    ctx = _ctx(F, [s], 0)
    phi = _flat(phis)
    V1, _, conv1 = ctx.orbital_poisson(phi)
    V1 = _np(V1).copy()
    assert np.all(_np(conv1) == 1)
    assert np.all(V1[s.G:2 * s.G] == 0.0)
    off = 0
    for sp, N in enumerate(s.norb):
        Vref, _ = orc.poisson(phis[sp] ** 2, s.grid, tol=1e-13)
        got = V1[off * s.G:(off + N) * s.G].reshape(N, s.G)
        assert np.max(np.abs(got - Vref)) < 1e-8 * np.max(np.abs(Vref)), sp
        off += N
    V2, _, _ = ctx.orbital_poisson(phi)
    assert np.array_equal(_np(V2), V1)


@pytest.mark.parametrize("bc", [1, 2])
def test_extended_poisson_parity(F, orc, bc):
    name = BC_NAMES[bc]
    _check_poisson(F, orc, synth.make_extended_system(16, 0.5, 2, [3, 2], seed=21, bc=name), bc)
    _check_poisson(F, orc, synth.make_extended_system(30, 0.4, 3, [4], seed=22, bc=name), bc)


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_extended_forward_backward_parity(F, orc, bc):
    name = BC_NAMES[bc]
    s = (synth.make_system(24, 0.45, 2, [3, 2], seed=23) if bc == 0 else
         synth.make_extended_system(24, 0.45, 2, [3, 2], seed=23, bc=name))
    ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-13, bc=name)
    dpsi_ref, dfod_ref = orc.sic_backward(ref, s.grid, gE=1.3, bc=name)
    ctx = _ctx(F, [s], bc)
    psi, fods = _flat(s.psi), _flat(s.fods)
    out = ctx.forward(psi, fods, scale=0.5)
    assert np.all(_np(out["conv"]) == 1)
    assert abs(_np(out["E_sic"])[0] - ref["E_sic"]) < 1e-6
    U = np.concatenate([b["U"] for b in ref["blocks"]])
    Exc = np.concatenate([b["Exc"] for b in ref["blocks"]])
    assert np.max(np.abs(_np(out["U"]) - U)) < 1e-6
    assert np.max(np.abs(_np(out["Exc"]) - Exc)) < 1e-6
    Va = _np(out["V_avg"]).reshape(len(s.psi), s.G)
    for sp, b in enumerate(ref["blocks"]):
        assert np.max(np.abs(Va[sp] - b["Vavg"])) < 1e-6
    gE = torch.tensor([1.3], dtype=torch.float64, device="cuda")
    dpsi, dfod = ctx.sic_backward(psi, fods, out["phi"], out["V"], gE)
    assert np.max(np.abs(_np(dfod).reshape(-1, 3) - np.concatenate(dfod_ref))) < 1e-5
    dp = np.concatenate([d.ravel() for d in dpsi_ref])
    assert np.max(np.abs(_np(dpsi) - dp)) < 1e-5 * np.max(np.abs(dp))


@pytest.mark.parametrize("bc", [1, 2])
def test_extended_hamiltonian_parity(F, orc, bc):
    name = BC_NAMES[bc]
    s = synth.make_extended_system(20, 0.45, 2, [3, 2], seed=24, bc=name)
    rng = np.random.default_rng(5)
    vavg = [rng.normal(size=s.G) * 0.1 for _ in s.norb]
    ctx = _ctx(F, [s], bc)
    H = _np(ctx.hamiltonian_apply(_flat(s.psi), None, _flat(vavg)))
    off = 0
    for sp, N in enumerate(s.norb):
        ref = orc.hamiltonian_apply(s.psi[sp], s.grid, None, vavg[sp], bc=name)
        got = H[off * s.G:(off + N) * s.G].reshape(N, s.G)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
        off += N


def test_kron_uneven_batch(F, orc):
    systems = [synth.make_system(18, 0.45, 2, [3], seed=41),
               synth.make_system(23, 0.35, 2, [4, 2], seed=42),
               synth.make_system(5, 0.9, 1, [1], seed=44),
               synth.make_system(24, 0.5, 2, [5], seed=46)]
    ctx = F.Context(systems, precision=F.MIXED, cg_tol=1e-11, solver=F.SOLVER_KRON)
    psi = _flat([p for s in systems for p in s.psi])
    fods = _flat([f for s in systems for f in s.fods])
    out = ctx.forward(psi, fods, scale=0.5)
    assert np.all(_np(out["conv"]) == 1)
    E = _np(out["E_sic"])
    for k, s in enumerate(systems):
        ref = orc.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-12)
        assert abs(E[k] - ref["E_sic"]) < 1e-6 * len(s.psi[0])


def test_kron_full_size_discrete_residual(F, orc):
    # the 128^3 workload: the discrete Poisson problem of sampled orbitals,
    # evaluated by the oracle's operators in float64
    s = synth.make_config(3)
    ctx = F.Context([s], precision=F.MIXED, cg_tol=1e-10, solver=F.SOLVER_KRON)
    psi, fods = _flat(s.psi), _flat(s.fods)
    out = ctx.forward(psi, fods)
    assert np.all(_np(out["conv"]) == 1)
    assert _np(out["iters"]).max() <= 6
    phi, V = _np(out["phi"]), _np(out["V"])
    G = s.G
    for o in (0, 33, 63):
        rho = phi[o * G:(o + 1) * G] ** 2
        b = 4 * np.pi * rho + orc.bc_rhs(orc.multipole_moments(rho, s.grid), s.grid)
        res = b + orc.laplacian(V[o * G:(o + 1) * G], s.grid)
        assert np.linalg.norm(res) / np.linalg.norm(b) <= 2e-10


def _gauss_orbitals(grid, norb, seed):
    """Normalised Gaussian orbitals on a (possibly non-cubic) grid, seeded
    centres within the central half of the box and widths 0.6-1.2 bohr."""
    nx, ny, nz, h, o = grid
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(o[2] + h * np.arange(nz), o[1] + h * np.arange(ny), o[0] + h * np.arange(nx), indexing="ij")
    L = np.array([nx, ny, nz]) * h
    out = []
    for _ in range(norb):
        c = o + L * (0.25 + 0.5 * rng.random(3))
        sg = 0.6 + 0.6 * rng.random()
        f = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * sg * sg)).ravel()
        out.append(f / np.sqrt(np.sum(f * f) * h ** 3))
    return np.array(out)


def _grid_dict(nx, ny, nz, h, norb):
    o = -0.5 * h * (np.array([nx, ny, nz]) - 1)
    return dict(nx=nx, ny=ny, nz=nz, h=h, origin=list(o), norb=[norb]), (nx, ny, nz, h, o)


@pytest.mark.parametrize("dims", [(48, 40, 56), (128, 16, 8)])
def test_kron_tensor_cores_match_cuda_cores_and_oracle(F, orc, dims):
    # non-cubic grids: each direction has its own operator, and the passes
    # rotate the layout through all three
    sysd, grid = _grid_dict(*dims, 0.3, 3)
    phi = _gauss_orbitals(grid, 3, seed=sum(dims))
    Vref, _ = orc.poisson(phi ** 2, grid, tol=1e-13)
    out = {}
    for tc in (1, 0):
        ctx = F.Context([sysd], precision=F.MIXED, cg_tol=1e-11, solver=F.SOLVER_KRON, kron_tensor_cores=tc)
        V, iters, conv = ctx.orbital_poisson(_flat([phi]))
        assert np.all(_np(conv) == 1)
        out[tc] = (_np(V).reshape(3, -1), _np(iters))
    scale = np.max(np.abs(Vref))
    for tc in (1, 0):
        assert np.max(np.abs(out[tc][0] - Vref)) < 1e-9 * scale, tc
    # the tensor-core transforms need no more refinement rounds than the CUDA-core ones
    assert np.all(out[1][1] <= out[0][1] + 1), (out[1][1], out[0][1])


def test_kron_batch_mixing_tensor_core_and_cuda_core_blocks(F, orc):
    # 40^3 and 32x24x16 qualify for the tensor cores; 21^3 (sides not a
    # multiple of 8) keeps the CUDA-core transforms; every pass launches both
    specs = [(40, 40, 40, 0.3, 2, 11), (21, 21, 21, 0.42, 4, 12), (32, 24, 16, 0.35, 3, 13)]
    sysds, grids, phis = [], [], []
    for nx, ny, nz, h, norb, seed in specs:
        sd, g = _grid_dict(nx, ny, nz, h, norb)
        sysds.append(sd)
        grids.append(g)
        phis.append(_gauss_orbitals(g, norb, seed))
    ctx = F.Context(sysds, precision=F.MIXED, cg_tol=1e-11, solver=F.SOLVER_KRON)
    V, iters, conv = ctx.orbital_poisson(_flat(phis))
    assert np.all(_np(conv) == 1)
    Vn = _np(V)
    off = 0
    for g, ph in zip(grids, phis):
        G = g[0] * g[1] * g[2]
        Vref, _ = orc.poisson(ph ** 2, g, tol=1e-13)
        got = Vn[off:off + len(ph) * G].reshape(len(ph), G)
        assert np.max(np.abs(got - Vref)) < 1e-9 * np.max(np.abs(Vref))
        off += len(ph) * G


def test_autotuner_picks_a_path_per_shape_and_keeps_parity(F, orc):
    """The autotuner (default) times each qualifying block shape on the tensor
    cores and on the CUDA cores and keeps the faster: a block is reported on
    the tensor cores only if it qualifies, without the tuner every qualifying
    block is, and the tuned context's potentials match the oracle."""
    specs = [(40, 40, 40, 0.3, 2, 11), (21, 21, 21, 0.42, 4, 12), (32, 24, 16, 0.35, 3, 13), (8, 8, 8, 0.5, 2, 14)]
    sysds, grids, phis = [], [], []
    for nx, ny, nz, h, norb, seed in specs:
        sd, g = _grid_dict(nx, ny, nz, h, norb)
        sysds.append(sd)
        grids.append(g)
        phis.append(_gauss_orbitals(g, norb, seed))
    off, eligible = 0, []
    for nx, ny, nz, h, norb, seed in specs:
        eligible.append(all(n % 8 == 0 and n <= 128 for n in (nx, ny, nz)) and off % 4 == 0)
        off += norb * nx * ny * nz
    tuned = F.Context(sysds, precision=F.MIXED, cg_tol=1e-11, solver=F.SOLVER_KRON)
    plain = F.Context(sysds, precision=F.MIXED, cg_tol=1e-11, solver=F.SOLVER_KRON, autotune=0)
    for p, q, el in zip(tuned.block_paths(), plain.block_paths(), eligible):
        assert q["tensor_core_transforms"] == el
        assert (not p["tensor_core_transforms"]) or el
    V, iters, conv = tuned.orbital_poisson(_flat(phis))
    assert np.all(_np(conv) == 1)
    Vn = _np(V)
    off = 0
    for g, ph in zip(grids, phis):
        G = g[0] * g[1] * g[2]
        Vref, _ = orc.poisson(ph ** 2, g, tol=1e-13)
        got = Vn[off:off + len(ph) * G].reshape(len(ph), G)
        assert np.max(np.abs(got - Vref)) < 1e-9 * np.max(np.abs(Vref))
        off += len(ph) * G
