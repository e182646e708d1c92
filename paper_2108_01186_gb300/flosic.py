"""Thin Python binding of the C ABI in include/flosic.h (ctypes).

Argument marshalling only: every step of the FLO-SIC path runs in the CUDA
kernels of libflosic.so.  Tensors are torch CUDA float64 tensors laid out as
the header describes (per spin block [N][G] arrays packed back to back).
There is no CPU fallback: if the library or a GPU is missing, calls raise.
"""
import ctypes
import functools
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflosic.so")

FLOSIC_OK, FLOSIC_ERR_ARG, FLOSIC_ERR_CUDA, FLOSIC_ERR_ILLCOND, FLOSIC_ERR_NOCONV, FLOSIC_ERR_NONFINITE = range(6)
FP64, MIXED = 0, 1
GRAD_INTERP, GRAD_PAPER = 0, 1
ADJ_REUSE_V, ADJ_EXACT = 0, 1
PC_NONE, PC_MG = 0, 1
SOLVER_PCG, SOLVER_AAR, SOLVER_KRON = 0, 1, 2
BC_ISOLATED, BC_PERIODIC, BC_SLAB = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "ARG", 2: "CUDA", 3: "ILLCOND", 4: "NOCONV", 5: "NONFINITE"}

ABI_FUNCTIONS = ("flosic_default_options", "flosic_create", "flosic_destroy", "flosic_last_error",
                 "flosic_layout", "flosic_build_flos", "flosic_orbital_poisson",
                 "flosic_sic_energy_potential", "flosic_sic_backward", "flosic_profile",
                 "flosic_profile_read", "flosic_orbital_poisson_noalloc", "flosic_noalloc_last_error",
                 "flosic_hamiltonian_apply", "flosic_profile_read_overlap", "flosic_set_orbital_mask",
                 "flosic_step_host", "flosic_block_paths")


class FlosicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("flosic %s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


class FlosicSystem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("nspin", ctypes.c_int), ("norb", ctypes.c_int * 2)]


class FlosicOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cg_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("fod_grad_mode", ctypes.c_int), ("adjoint_mode", ctypes.c_int),
                ("rho_min", ctypes.c_double), ("illcond_tol", ctypes.c_double),
                ("preconditioner", ctypes.c_int), ("solver", ctypes.c_int),
                ("aar_omega", ctypes.c_double), ("aar_beta", ctypes.c_double),
                ("aar_m", ctypes.c_int), ("aar_p", ctypes.c_int), ("boundary", ctypes.c_int),
                ("kron_tensor_cores", ctypes.c_int), ("autotune", ctypes.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Loads libflosic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FlosicError(FLOSIC_ERR_CUDA, "libflosic.so not built (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.flosic_default_options.argtypes = [ctypes.POINTER(FlosicOptions)]
    L.flosic_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(FlosicSystem), i, ctypes.POINTER(FlosicOptions)]
    L.flosic_destroy.argtypes = [vp]
    L.flosic_last_error.argtypes = [vp]
    L.flosic_last_error.restype = ctypes.c_char_p
    L.flosic_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.flosic_build_flos.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.flosic_orbital_poisson.argtypes = [vp, vp, vp, i, vp, vp, vp]
    L.flosic_sic_energy_potential.argtypes = [vp, vp, vp, vp, d, vp, vp, vp, vp, vp]
    L.flosic_sic_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.flosic_hamiltonian_apply.argtypes = [vp, vp, vp, vp, vp, vp]
    L.flosic_set_orbital_mask.argtypes = [vp, vp]
    L.flosic_block_paths.argtypes = [vp, vp]
    L.flosic_step_host.argtypes = [vp, vp, vp, d, d, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.flosic_profile.argtypes = [vp, i]
    L.flosic_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i]
    L.flosic_profile_read_overlap.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i]
    L.flosic_orbital_poisson_noalloc.argtypes = [i, i, i, d, ctypes.POINTER(d), i, vp, vp, d, i, vp, vp, vp]
    L.flosic_noalloc_last_error.argtypes = []
    L.flosic_noalloc_last_error.restype = ctypes.c_char_p
    for f in ABI_FUNCTIONS:
        if f not in ("flosic_last_error", "flosic_noalloc_last_error"):
            getattr(L, f).restype = i
    _lib = L
    return L


def default_options(**overrides):
    L = load_library()
    o = FlosicOptions()
    L.flosic_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _on_device(fn):
    """Runs a Context method with the context's device current (the library
    launches on the current device, on its current stream)."""
    @functools.wraps(fn)
    def wrapper(self, *args, **kwargs):
        with torch.cuda.device(self.device):
            return fn(self, *args, **kwargs)
    return wrapper


class Context:
    """A batch of systems on the current CUDA device (owns the workspace).

    systems: sequence of dicts or objects with n (or nx, ny, nz), h, origin
    and norb (list of 1 or 2 orbital counts)."""

    def __init__(self, systems, **options):
        if not torch.cuda.is_available():
            raise FlosicError(FLOSIC_ERR_CUDA, "no CUDA device")
        self._L = load_library()
        arr = (FlosicSystem * len(systems))()
        self.systems = []
        for k, s in enumerate(systems):
            g = _sysdict(s)
            arr[k].nx, arr[k].ny, arr[k].nz = g["nx"], g["ny"], g["nz"]
            arr[k].h = g["h"]
            for d in range(3):
                arr[k].origin[d] = g["origin"][d]
            arr[k].nspin = len(g["norb"])
            for sp, n in enumerate(g["norb"]):
                arr[k].norb[sp] = n
            self.systems.append(g)
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        rc = self._L.flosic_create(ctypes.byref(h), arr, len(systems), ctypes.byref(self.options))
        if rc != FLOSIC_OK:
            raise FlosicError(rc, self._L.flosic_last_error(None).decode())
        self._h = h
        lay = (ctypes.c_int64 * 6)()
        self._check(self._L.flosic_layout(h, lay))
        self.norb, self.orb_elems, self.vavg_elems, self.mat_elems, self.nblk, self.nsys = [int(x) for x in lay]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def _check(self, rc):
        if rc != FLOSIC_OK:
            raise FlosicError(rc, self._L.flosic_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._L is not None:
            self._L.flosic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n, dtype=torch.float64):
        return torch.empty(n, dtype=dtype, device=self.device)

    def _req(self, t, n, name, dtype=torch.float64):
        """Every array handed to the library: a contiguous tensor of the
        expected type and size on the context's device (the C ABI takes bare
        pointers and cannot check them)."""
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == self.device and t.dtype == dtype
                and t.is_contiguous() and t.numel() == n):
            raise FlosicError(FLOSIC_ERR_ARG, "%s must be a contiguous %s tensor of %d elements on %s"
                              % (name, dtype, n, self.device))

    # ---- the four calls of the step --------------------------------------
    @_on_device
    def build_flos(self, psi, fods, want_matrices=True):
        self._req(psi, self.orb_elems, "psi")
        self._req(fods, 3 * self.norb, "fods")
        phi = self._empty(self.orb_elems)
        S = self._empty(self.mat_elems) if want_matrices else None
        Q = self._empty(self.mat_elems) if want_matrices else None
        self._check(self._L.flosic_build_flos(self._h, _ptr(psi), _ptr(fods), _ptr(phi), _ptr(S), _ptr(Q), _stream()))
        return phi, S, Q

    @_on_device
    def orbital_poisson(self, phi, V=None, check=True):
        self._req(phi, self.orb_elems, "phi")
        warm = V is not None
        if V is None:
            V = self._empty(self.orb_elems)
        else:
            self._req(V, self.orb_elems, "V")
        iters = self._empty(self.norb, torch.int32)
        conv = self._empty(self.norb, torch.int32)
        rc = self._L.flosic_orbital_poisson(self._h, _ptr(phi), _ptr(V), int(warm), _ptr(iters), _ptr(conv), _stream())
        if check or rc not in (FLOSIC_OK, FLOSIC_ERR_NOCONV):
            self._check(rc)
        return V, iters, conv

    @_on_device
    def sic_energy_potential(self, psi, phi, V, scale=1.0):
        for t, nm in ((psi, "psi"), (phi, "phi"), (V, "V")):
            self._req(t, self.orb_elems, nm)
        U = self._empty(self.norb)
        Exc = self._empty(self.norb)
        E = self._empty(self.nsys)
        Vavg = self._empty(self.vavg_elems)
        self._check(self._L.flosic_sic_energy_potential(self._h, _ptr(psi), _ptr(phi), _ptr(V), float(scale),
                                                        _ptr(U), _ptr(Exc), _ptr(E), _ptr(Vavg), _stream()))
        return E, Vavg, U, Exc

    @_on_device
    def sic_backward(self, psi, fods, phi, V, gE, want_dpsi=True):
        for t, nm in ((psi, "psi"), (phi, "phi"), (V, "V")):
            self._req(t, self.orb_elems, nm)
        self._req(fods, 3 * self.norb, "fods")
        self._req(gE, self.nsys, "gE")
        dpsi = self._empty(self.orb_elems) if want_dpsi else None
        dfod = self._empty(3 * self.norb)
        self._check(self._L.flosic_sic_backward(self._h, _ptr(psi), _ptr(fods), _ptr(phi), _ptr(V), _ptr(gE),
                                                _ptr(dpsi), _ptr(dfod), _stream()))
        return dpsi, dfod

    @_on_device
    def step_host(self, psi, fods, scale=1.0, gE=1.0, E_sic=None, U=None, Exc=None, V_avg=None, dE_dpsi=None,
                  dE_dfod=None, conv=None, psi_next=None, fods_next=None):
        """Calls flosic_step_host: one forward + adjoint step with every array in
        host memory (contiguous CPU tensors, float64 / int32 for conv; pinned
        for full-speed copies).  Outputs are filled in place; returns the
        status (OK or NOCONV).  With psi_next/fods_next the library copies
        them during this step and starts their FLO build and Poisson solve
        while this step's outputs are copied out; the next call with exactly
        those tensors picks that work up."""
        def host(t, n, dtype, name):
            if t is None:
                return None
            if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == dtype
                    and t.is_contiguous() and t.numel() == n):
                raise FlosicError(FLOSIC_ERR_ARG, "%s: contiguous CPU %s tensor of %d elements" % (name, dtype, n))
            return ctypes.c_void_p(t.data_ptr())
        f64 = torch.float64
        args = [host(psi, self.orb_elems, f64, "psi"), host(fods, 3 * self.norb, f64, "fods")]
        if args[0] is None or args[1] is None:
            raise FlosicError(FLOSIC_ERR_ARG, "psi and fods are required")
        outs = [host(E_sic, self.nsys, f64, "E_sic"), host(U, self.norb, f64, "U"), host(Exc, self.norb, f64, "Exc"),
                host(V_avg, self.vavg_elems, f64, "V_avg"), host(dE_dpsi, self.orb_elems, f64, "dE_dpsi"),
                host(dE_dfod, 3 * self.norb, f64, "dE_dfod"), host(conv, self.norb, torch.int32, "conv")]
        nxt = [host(psi_next, self.orb_elems, f64, "psi_next"), host(fods_next, 3 * self.norb, f64, "fods_next")]
        rc = self._L.flosic_step_host(self._h, args[0], args[1], float(scale), float(gE), *outs, *nxt, _stream())
        if rc not in (FLOSIC_OK, FLOSIC_ERR_NOCONV):
            self._check(rc)
        return rc

    def block_paths(self):
        """Calls flosic_block_paths: per spin block (packed order) a dict of the
        kernel paths the context took (tensor-core transforms, copy-engine
        refinement update, asynchronous-copy overlap Gram)."""
        out = (ctypes.c_int * self.nblk)()
        self._check(self._L.flosic_block_paths(self._h, ctypes.cast(out, ctypes.c_void_p)))
        return [dict(tensor_core_transforms=bool(v & 1), tma_update=bool(v & 2), async_gram=bool(v & 4))
                for v in out]

    @_on_device
    def set_orbital_mask(self, mask=None):
        """Calls flosic_set_orbital_mask: mask = a sequence of 0/1 per orbital
        (context order) or None for every orbital."""
        if mask is None:
            self._check(self._L.flosic_set_orbital_mask(self._h, None))
            return
        m = [int(v) for v in mask]
        if len(m) != self.norb:
            raise FlosicError(FLOSIC_ERR_ARG, "mask needs one entry per orbital (%d)" % self.norb)
        arr = (ctypes.c_int * len(m))(*m)
        self._check(self._L.flosic_set_orbital_mask(self._h, ctypes.cast(arr, ctypes.c_void_p)))

    @_on_device
    def hamiltonian_apply(self, psi, vloc=None, V_avg=None, out=None):
        """H psi = -1/2 Delta_h psi + (vloc + V_avg) psi per orbital (the
        SC_AvgSIC Hamiltonian); vloc one field per system, V_avg one per spin
        block (as returned by sic_energy_potential), either may be None."""
        self._req(psi, self.orb_elems, "psi")
        if vloc is not None:
            total = sum(g["nx"] * g["ny"] * g["nz"] for g in self.systems)
            self._req(vloc, total, "vloc")
        if V_avg is not None:
            self._req(V_avg, self.vavg_elems, "V_avg")
        if out is not None:
            self._req(out, self.orb_elems, "out")
        hpsi = self._empty(self.orb_elems) if out is None else out
        self._check(self._L.flosic_hamiltonian_apply(self._h, _ptr(psi), _ptr(vloc), _ptr(V_avg), _ptr(hpsi),
                                                     _stream()))
        return hpsi

    @_on_device
    def profile(self, enable=True):
        self._check(self._L.flosic_profile(self._h, int(enable)))

    @_on_device
    def profile_read(self, reset=True):
        out = (ctypes.c_double * 4)()
        self._check(self._L.flosic_profile_read(self._h, out, int(reset)))
        return dict(kernel_ms=out[0], kernel_launches=int(out[1]), launches=int(out[2]), kernel_bytes=out[3])

    @_on_device
    def profile_read_overlap(self, reset=True):
        """Timed launches of the mixed path's tensor-core overlap kernel:
        summed ms, launch count and algorithmic flops (2 N^2 G per block)."""
        out = (ctypes.c_double * 3)()
        self._check(self._L.flosic_profile_read_overlap(self._h, out, int(reset)))
        return dict(kernel_ms=out[0], kernel_launches=int(out[1]), flops=out[2])

    @_on_device
    def forward(self, psi, fods, scale=1.0, V0=None):
        phi, S, Q = self.build_flos(psi, fods)
        V, iters, conv = self.orbital_poisson(phi, V0)
        E, Vavg, U, Exc = self.sic_energy_potential(psi, phi, V, scale)
        return dict(phi=phi, S=S, S_mhalf=Q, V=V, iters=iters, conv=conv, E_sic=E, V_avg=Vavg, U=U, Exc=Exc)


def orbital_poisson_noalloc(grid, phi, V, cg_tol=1e-10, max_iter=20000, iters=None, conv=None):
    """Calls flosic_orbital_poisson_noalloc: one grid (nx, ny, nz, h, origin),
    phi and V [norb*G] CUDA float64 tensors on one device (iters, conv:
    optional [norb] int32 tensors there); returns the status code."""
    L = load_library()
    nx, ny, nz, h, origin = grid
    G = nx * ny * nz
    norb = phi.numel() // G if isinstance(phi, torch.Tensor) and G > 0 else 0

    def ok(t, n, dtype):
        return (isinstance(t, torch.Tensor) and t.is_cuda and t.device == phi.device and t.dtype == dtype
                and t.is_contiguous() and t.numel() == n)

    if not (norb > 0 and ok(phi, norb * G, torch.float64) and ok(V, norb * G, torch.float64)
            and all(t is None or ok(t, norb, torch.int32) for t in (iters, conv))):
        raise FlosicError(FLOSIC_ERR_ARG, "phi and V: contiguous CUDA float64 tensors of norb*G elements on one "
                                          "device; iters, conv: None or int32 tensors of norb elements there")
    org = (ctypes.c_double * 3)(*[float(x) for x in origin])
    with torch.cuda.device(phi.device):
        return L.flosic_orbital_poisson_noalloc(int(nx), int(ny), int(nz), float(h), org, int(norb), _ptr(phi), _ptr(V),
                                            float(cg_tol), int(max_iter), _ptr(iters), _ptr(conv), _stream())


def _sysdict(s):
    g = s if isinstance(s, dict) else {k: getattr(s, k) for k in ("n", "h", "origin", "norb") if hasattr(s, k)}
    g = dict(g)
    if "n" in g:
        g.setdefault("nx", g["n"])
        g.setdefault("ny", g["n"])
        g.setdefault("nz", g["n"])
    g["origin"] = [float(x) for x in g["origin"]]
    g["norb"] = [int(x) for x in g["norb"]]
    return g


class FlosicStep(torch.autograd.Function):
    """(psi, fods) -> (E_sic [nsys], V_avg, U, Exc) with a hand-written
    backward for E_sic (dE/dpsi and the FOD gradient); V_avg, U and Exc
    carry no gradient."""

    @staticmethod
    def forward(ctx, context, psi, fods, scale):
        out = context.forward(psi.detach(), fods.detach(), scale)
        ctx.context = context
        ctx.save_for_backward(psi, fods, out["phi"], out["V"])
        ctx.mark_non_differentiable(out["V_avg"], out["U"], out["Exc"])
        return out["E_sic"], out["V_avg"], out["U"], out["Exc"]

    @staticmethod
    def backward(ctx, gE, gV, gU, gX):
        psi, fods, phi, V = ctx.saved_tensors
        if gE is None:
            return None, None, None, None
        dpsi, dfod = ctx.context.sic_backward(psi.detach(), fods.detach(), phi, V, gE.contiguous().to(torch.float64),
                                              want_dpsi=ctx.needs_input_grad[1])
        return None, dpsi, dfod, None
