/*
 * flosic.h -- C ABI of the GB300 (sm_103a) real-space FLO-SIC orbital-SIC step.
 *
 * Method: Diaz, Suryanarayana, Xu, Baruah, Pask, Zope, "Implementation of
 * Perdew-Zunger self-interaction correction in real space using
 * Fermi-Loewdin orbitals" (arXiv 2108.01186).  One step takes Kohn-Sham
 * orbitals psi on a uniform grid and Fermi-orbital descriptor (FOD)
 * positions a_i, and returns the PZ-SIC energy (Eq. 1), the scaled averaged
 * SIC potential (Eq. 13) and, in reverse mode, dE_SIC/dpsi and the FOD
 * gradient dE_SIC/da (Eqs. 9-11).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller, except the
 *    options/system descriptors and the pointers marked "host".
 *  - A batch holds nsys independent systems.  System s has an nx*ny*nz
 *    interior grid with spacing h (bohr); point (i,j,k) sits at
 *    origin + h*(i,j,k) and has flat index (k*ny + j)*nx + i (x fastest).
 *    G = nx*ny*nz.  Orbitals vanish outside the interior (zero Dirichlet),
 *    except along the periodic directions of flosic_options.boundary, where
 *    they wrap around the cell.
 *  - A "spin block" is one spin of one system with N = norb[spin] orbitals.
 *    Blocks are ordered system-major, then spin.  Orbital-sized arrays
 *    (psi, phi, V, dE_dpsi) are the blocks' [N][G] float64 arrays packed
 *    back to back; FOD arrays are [N][3] float64 per block packed the same
 *    way; N x N matrices (S, S_mhalf) are row-major per block, packed;
 *    per-orbital scalars (U, Exc, iters, conv_flags) are packed per block;
 *    V_avg is one [G] array per block; E_sic and gE hold one value per
 *    system.  flosic_layout() returns every packed size.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, passed as
 *    void*), except that calls whose result can fail on the device
 *    (flosic_build_flos: ILLCOND/NONFINITE, flosic_orbital_poisson: NOCONV)
 *    wait for the stream before they return the status.
 *  - Every call returns an int status (flosic_status); nothing throws across
 *    the ABI.  flosic_last_error() returns a message for the last failure.
 *  - The context owns its device workspace (allocated in flosic_create,
 *    freed in flosic_destroy).  A context must not be used by two streams
 *    at once.
 */
#ifndef FLOSIC_H
#define FLOSIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLOSIC_OK = 0,
    FLOSIC_ERR_ARG = 1,        /* bad argument or descriptor */
    FLOSIC_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    FLOSIC_ERR_ILLCOND = 3,    /* FO overlap near singular (FODs too close) */
    FLOSIC_ERR_NOCONV = 4,     /* a Poisson solve hit max_iter */
    FLOSIC_ERR_NONFINITE = 5   /* NaN/Inf met in an input or result */
} flosic_status;

enum { FLOSIC_FP64 = 0, FLOSIC_MIXED = 1 };                 /* precision */
enum { FLOSIC_GRAD_INTERP = 0, FLOSIC_GRAD_PAPER = 1 };     /* fod_grad_mode */
enum { FLOSIC_ADJ_REUSE_V = 0, FLOSIC_ADJ_EXACT = 1 };      /* adjoint_mode */
enum { FLOSIC_PC_NONE = 0, FLOSIC_PC_MG = 1 };              /* preconditioner */
/* inner solver of the mixed path: conjugate gradients (this library's
 * default), Alternating Anderson-Richardson (the iteration Sec. II.A's code
 * uses for its electrostatics), or the Kronecker-product solver: Sec. II.A
 * writes the Laplacian as a Kronecker sum A = T_x (+) T_y (+) T_z of 1-D
 * operators; with the eigen-decompositions T_d = Q_d L_d Q_d^T the inverse
 * is (Q_x x Q_y x Q_z) (L_x (+) L_y (+) L_z)^{-1} (Q_x x Q_y x Q_z)^T,
 * applied in float32 as six dense 1-D transforms per orbital (one "iteration"
 * per application; the float-float refinement around it reaches cg_tol) */
enum { FLOSIC_SOLVER_PCG = 0, FLOSIC_SOLVER_AAR = 1, FLOSIC_SOLVER_KRON = 2 };
/* boundary conditions of the orbital Poisson problems (Sec. II.A: Dirichlet
 * values from a multipole expansion for isolated systems, periodic conditions
 * along extended directions, a dipole correction for surfaces):
 *   ISOLATED: multipole (l <= 2) values on the ghost shell;
 *   PERIODIC: every direction periodic; each orbital density is neutralised
 *             by a uniform background and V_i has zero mean;
 *   SLAB:     periodic along x and y; along z the ghost planes carry the
 *             planar-average potential -(2 pi/A)(Q |z - c_z| - sgn(z - c_z) p_z)
 *             of the orbital's charge Q and dipole p_z (A = nx ny h^2).
 * Along periodic directions the stencil, the FOD interpolation nodes and the
 * FOD coordinates wrap around the cell.  PERIODIC and SLAB require the KRON
 * solver, ADJ_REUSE_V, GRAD_INTERP and periodic sides of at least 13. */
enum { FLOSIC_BC_ISOLATED = 0, FLOSIC_BC_PERIODIC = 1, FLOSIC_BC_SLAB = 2 };

typedef struct {
    int nx, ny, nz;       /* interior grid points per direction (>= 1;
                             nx*ny*nz < 2^31) */
    double h;             /* grid spacing, bohr (> 0) */
    double origin[3];     /* position of point (0,0,0), bohr */
    int nspin;            /* 1 or 2 */
    int norb[2];          /* occupied orbitals = FODs per spin (>= 1) */
} flosic_system;

typedef struct {
    int precision;        /* FLOSIC_FP64: every step in float64.
                             FLOSIC_MIXED: float32 inner Poisson solves
                             inside a float-float residual refinement, the
                             overlap on the tensor cores (split bf16); the
                             rest float64. */
    double cg_tol;        /* relative residual ||b - A V|| / ||b|| per solve */
    int max_iter;         /* CG iteration cap per solve (all refinement
                             sweeps together) */
    int fod_grad_mode;    /* grad psi at the FODs: FLOSIC_GRAD_INTERP = exact
                             derivative of the cubic interpolant (consistent
                             with the energy); FLOSIC_GRAD_PAPER = central-
                             difference grid gradient then cubic
                             interpolation (Sec. II.B) */
    int adjoint_mode;     /* dU/drho: FLOSIC_ADJ_REUSE_V uses V itself;
                             FLOSIC_ADJ_EXACT adds the transpose of the
                             multipole boundary map (one extra zero-boundary
                             solve per orbital) */
    double rho_min;       /* density cutoff of xc and of V_avg */
    double illcond_tol;   /* ILLCOND when lambda_min(S) < tol*lambda_max(S) */
    int preconditioner;   /* FLOSIC_PC_NONE or FLOSIC_PC_MG (multigrid
                             V-cycle on the 7-point Laplacian) */
    int solver;           /* FLOSIC_SOLVER_PCG (default), FLOSIC_SOLVER_AAR
                             or FLOSIC_SOLVER_KRON: the float32 inner solver
                             of the MIXED path (AAR and KRON require MIXED;
                             FP64 runs PCG) */
    double aar_omega;     /* AAR Richardson relaxation (default 0.6) */
    double aar_beta;      /* AAR Anderson mixing (default 0.6) */
    int aar_m;            /* AAR history length, 1..8 (default 7) */
    int aar_p;            /* AAR: every p-th step is an Anderson step, >= 2
                             (default 6) */
    int boundary;         /* FLOSIC_BC_ISOLATED (default), _PERIODIC, _SLAB */
    int kron_tensor_cores; /* KRON solver: 1 (default) runs the 1-D transforms
                             of every spin block whose sides are multiples of
                             8 and at most 128 on the tensor cores (split
                             bf16, float32 accumulation); 0 keeps them all on
                             the CUDA cores (float32) */
    int autotune;         /* KRON solver with kron_tensor_cores 1: 1 (default)
                             times, at context creation, one inner solve of
                             each distinct block shape (nx, ny, nz, N) that
                             qualifies for the tensor cores with the tensor-
                             core and with the CUDA-core transforms, and keeps
                             the faster per shape (flosic_block_paths reports
                             the choice); 0 takes the tensor cores wherever
                             they qualify */
} flosic_options;

typedef struct flosic_ctx flosic_ctx;

/* Fills *opt with the defaults: MIXED, cg_tol 1e-10, max_iter 20000,
 * GRAD_INTERP, ADJ_REUSE_V, rho_min 1e-30, illcond_tol 1e-10, PC_MG,
 * SOLVER_PCG (AAR parameters 0.6, 0.6, 7, 6), BC_ISOLATED,
 * kron_tensor_cores 1, autotune 1.  The KRON solver
 * requires MIXED and every side <= 256.
 * Returns FLOSIC_ERR_ARG if opt is NULL. */
int flosic_default_options(flosic_options* opt);

/* Creates a context for nsys systems (host array sys[nsys]) and allocates
 * its device workspace on the current device.  opt may be NULL (defaults).
 * Errors: ARG (bad descriptor), CUDA (allocation failed).  On error *ctx is
 * NULL and the message is available from flosic_last_error(NULL). */
int flosic_create(flosic_ctx** ctx, const flosic_system* sys, int nsys,
                  const flosic_options* opt);

/* Frees the context and its workspace.  NULL is a no-op. */
int flosic_destroy(flosic_ctx* ctx);

/* Message of the last failing call on ctx (or of the calling thread's last
 * failed flosic_create when ctx is NULL).  Owned by the library. */
const char* flosic_last_error(const flosic_ctx* ctx);

/* Packed sizes (host array out[6]): [0] orbitals in the batch, [1] elements
 * of an orbital-sized array (sum N*G), [2] elements of V_avg (sum of G over
 * blocks), [3] elements of the N x N matrix arrays (sum N*N), [4] spin
 * blocks, [5] systems. */
int flosic_layout(const flosic_ctx* ctx, int64_t* out);

/* The kernel paths of every spin block (host array out[blocks], blocks in
 * the packed order), no counterpart in the paper: bit 0 = its Kronecker
 * transforms run on the tensor cores (KRON solver; the autotuner's pick
 * when autotune is 1), bit 1 = its refinement update is staged by the copy
 * engine, bit 2 = its overlap Gram stages psi with asynchronous copies
 * (MIXED).  Errors: ARG. */
int flosic_block_paths(const flosic_ctx* ctx, int* out);

/* Steps a1-a5 (Sec. II.B, Eqs. 6-8, Loewdin of Sec. I.B):
 *   psi_a(a_i), grad psi_a(a_i) by tricubic Lagrange interpolation,
 *   rho(a_i) = sum_a psi_a(a_i)^2, T_ia = psi_a(a_i)/sqrt(rho(a_i)),
 *   F = T psi, S = dV F F^T (summed over the grid), S = U L U^T,
 *   S^{-1/2} = U L^{-1/2} U^T, phi = S^{-1/2} F.
 * In:  psi [sum N*G] float64, fods [sum N*3] float64 (bohr).
 * Out: phi [sum N*G] float64 (the FLOs), S and S_mhalf [sum N*N] float64.
 *      S and S_mhalf may be NULL (not returned).
 * The context keeps T, the eigen-pairs and the interpolation data for
 * flosic_sic_backward.  Errors: ARG, CUDA, ILLCOND (some block's overlap is
 * near singular; phi is then undefined), NONFINITE (NaN/Inf in psi or at a
 * FOD).  Waits for `stream` before returning. */
int flosic_build_flos(flosic_ctx* ctx, const double* psi, const double* fods,
                      double* phi, double* S, double* S_mhalf, void* stream);

/* Orbital mask for sharding the orbital units of one system over several
 * GPUs (Sec. II.A solves one Poisson problem per orbital; Eq. 1 sums E_SIC
 * over orbitals and Eq. 13 sums V_avg's numerator over orbitals, so sums
 * over disjoint orbital subsets add up to the whole).  mask: host array of
 * one int per orbital (0 or 1, in the context's orbital order) or NULL
 * (every orbital).  Afterwards flosic_orbital_poisson solves only orbitals
 * with mask 1 (the others get V = 0, iters 0, conv 1);
 * flosic_sic_energy_potential gives U = E_xc = 0 to masked orbitals, leaves
 * them out of E_SIC and of V_avg's numerator (the denominator rho_sigma
 * still sums every psi of the spin), and caches V^SIC = 0 for them, so
 * flosic_sic_backward's gradients are those of the unmasked orbitals'
 * energy terms alone.  Summing V_avg, U, E_xc, E_SIC, dE/dpsi and dE/da
 * over ranks whose masks partition the orbitals gives the unmasked values.
 * flosic_build_flos is not masked (every rank builds all FLOs of a spin).
 * Synchronous.  Errors: ARG (NULL ctx, an entry other than 0 or 1, or a
 * partial mask with ADJ_EXACT), CUDA. */
int flosic_set_orbital_mask(flosic_ctx* ctx, const int* mask);

/* Steps a6-a7 (Sec. II.A): per orbital, -Delta_h V_i = 4 pi phi_i^2 with the
 * 12th-order centred Laplacian and, by flosic_options.boundary, Dirichlet
 * values from the l <= 2 multipole expansion of phi_i^2 about the box centre
 * on the 6-layer ghost shell (isolated), a neutralising background with
 * zero-mean V (periodic), or the dipole-corrected planar potential on the
 * z ghost planes (slab); solved to ||b - A V|| <= cg_tol ||b|| by the
 * options' solver (FP64: float64 CG; MIXED: float32 inner solves -- CG, AAR
 * or the Kronecker-product inverse -- inside a float-float refinement).
 * In:  phi [sum N*G] float64.  In/out: V [sum N*G] float64 (in: warm start
 * if warm_start != 0, ignored otherwise; out: the potentials).
 * Out (may be NULL): iters [orbitals] int32 (inner iterations per orbital,
 * all refinement rounds summed; one per Kronecker application),
 * conv_flags [orbitals] int32 (1 = converged).
 * Errors: ARG, CUDA, NOCONV (some orbital hit max_iter; V holds the last
 * iterate).  Waits for `stream` before returning. */
int flosic_orbital_poisson(flosic_ctx* ctx, const double* phi, double* V,
                           int warm_start, int* iters, int* conv_flags,
                           void* stream);

/* Steps a8-a9 (Eq. 1, the bracketed term of Eq. 5, Eq. 13):
 *   rho_i = phi_i^2, U_i = (dV/2) sum rho_i V_i,
 *   E_xc,i = dV sum rho_i eps_xc(rho_i, 0) (LSDA exchange + PW92 at zeta=1),
 *   E_sic = -sum_{i,spin} (U_i + E_xc,i) per system,
 *   V_i^SIC = -(V_i + v_xc(rho_i)),
 *   V_avg = scale * sum_i rho_i V_i^SIC / rho_spin with rho_spin =
 *   sum_a psi_a^2 (0 where rho_spin < rho_min).
 * In:  psi, phi, V [sum N*G] float64; scale (host scalar).
 * Out (any may be NULL): U, Exc [orbitals], E_sic [nsys], V_avg [sum G].
 * Errors: ARG, CUDA. */
int flosic_sic_energy_potential(flosic_ctx* ctx, const double* psi,
                                const double* phi, const double* V, double scale,
                                double* U, double* Exc, double* E_sic,
                                double* V_avg, void* stream);

/* Step a10 (Eqs. 9-11, by reverse mode): gradients of sum_s gE[s]*E_sic[s]
 * with respect to the grid values of psi and to the FOD positions.  Uses the
 * data kept by the last flosic_build_flos on this context; psi, fods, phi
 * and V must be the arrays of that forward step.
 * In:  psi, phi, V [sum N*G], fods [sum N*3], gE [nsys] float64.
 * Out: dE_dpsi [sum N*G] float64 (partial derivative with respect to each
 *      grid value, i.e. the functional derivative times dV) and dE_dfod
 *      [sum N*3] float64 (hartree/bohr); either may be NULL.
 * Errors: ARG (no forward step recorded), CUDA, NOCONV (adjoint_mode EXACT
 * and an extra solve hit max_iter). */
int flosic_sic_backward(flosic_ctx* ctx, const double* psi, const double* fods,
                        const double* phi, const double* V, const double* gE,
                        double* dE_dpsi, double* dE_dfod, void* stream);

/* SC_AvgSIC Hamiltonian apply (Sec. II.C, Eq. 13): the averaged SIC
 * potential enters one Kohn-Sham Hamiltonian per spin.  For every orbital a
 * of every spin block:
 *   Hpsi_a = -1/2 Delta_h psi_a + (vloc + V_avg) psi_a
 * with the 12th-order Laplacian of the Poisson solves and zero values
 * outside the box (orbitals vanish there).
 * In:  psi [sum N*G] float64, the orbitals H is applied to;
 *      vloc [sum over systems of G] float64 or NULL: the other local terms
 *      of Eq. 13 (external, Hartree, exchange-correlation), one field per
 *      system;
 *      V_avg [sum G over spin blocks] float64 or NULL: the averaged SIC
 *      potential as written by flosic_sic_energy_potential (scaled by s).
 * Out: Hpsi [sum N*G] float64 (must not overlap psi).
 * Precision follows the context: FP64 in float64; MIXED with the Laplacian
 * and the potential term in float-float pairs (~48 bits), no float64
 * arithmetic per point but the final sum.
 * Errors: ARG (NULL ctx, psi or Hpsi, or Hpsi == psi), CUDA.  Asynchronous
 * on `stream`. */
int flosic_hamiltonian_apply(flosic_ctx* ctx, const double* psi, const double* vloc,
                             const double* V_avg, double* Hpsi, void* stream);

/* One whole step (steps a1-a10) with inputs and outputs in HOST memory:
 * flosic_build_flos, flosic_orbital_poisson (cold start),
 * flosic_sic_energy_potential and flosic_sic_backward on device copies
 * that the context owns (allocated at the first call: two input sets and
 * the intermediate and output arrays, about 5 orbital-sized float64 arrays).
 * No counterpart in the paper; it exists so that the host<->device copies
 * of a step are issued by the library.
 * In (host): psi [sum N*G], fods [sum N*3] float64; scale (V_avg factor);
 *   gE (the same upstream factor for every system's E_sic).
 * Out (host, any may be NULL): E_sic [nsys], U, Exc [orbitals],
 *   V_avg [sum G], dE_dpsi [sum N*G], dE_dfod [sum N*3] float64,
 *   conv_flags [orbitals] int32.
 * psi_next, fods_next (host, both or neither): the inputs of the next
 *   call; they are copied to the context's second input set on a separate
 *   stream while this step computes, and the next call that passes exactly
 *   these pointers uses them without copying again (the caller must not
 *   change their contents in between).  With them, the call also starts
 *   the next step's FLO build and Poisson solve on `stream` once this
 *   step's outputs are final, while those outputs travel to the host on a
 *   second stream; the next call that passes exactly these pointers finds
 *   that work done and only adds the energies and the adjoint (with its own
 *   scale and gE).  Any other call on the context in between discards it
 *   (the next step is then computed in full).  Work of the next step may
 *   still be running on `stream` when this call returns.  A failure of the
 *   started FLO build or solve is reported by the next call, which repeats
 *   them; only a CUDA error is returned at once.
 * Host arrays should be page-locked (cudaHostAlloc / pinned) for the copies
 * to run asynchronously at full speed.  The outputs are in host memory on
 * return.  Errors: as the four step calls; NOCONV is returned after the
 * outputs are copied. */
int flosic_step_host(flosic_ctx* ctx, const double* psi, const double* fods, double scale, double gE,
                     double* E_sic, double* U, double* Exc, double* V_avg, double* dE_dpsi,
                     double* dE_dfod, int* conv_flags, const double* psi_next,
                     const double* fods_next, void* stream);

/* Instrumentation (no counterpart in the paper): enable != 0 records a CUDA
 * event pair, on the stream the work runs on, around every launch of the
 * dominant kernel of the context's Poisson solver: the stencil apply of CG
 * (FLOSIC_SOLVER_PCG), the residual update of AAR (FLOSIC_SOLVER_AAR), or
 * one whole inner solve of the Kronecker-product solver, i.e. its
 * transform passes (FLOSIC_SOLVER_KRON).  Errors: ARG, CUDA. */
int flosic_profile(flosic_ctx* ctx, int enable);

/* Host array out[4]: [0] summed duration (ms) of the timed launches (or
 * inner solves), [1] their number, [2] kernels launched by ctx (all
 * kinds), [3] the algorithmic work of the timed launches, counted on the
 * device: for CG and AAR the bytes their stencil sweep must move (CG: per
 * active orbital and launch, read z, p_old, q_old and write p, q; 3 arrays
 * on the first iteration of a solve), for the Kronecker-product solver the
 * flops of its transforms (2 (n_s^2 + n_a^2) per line and pass, n_s and n_a
 * the even and odd half sizes of the line).  Waits for the device.
 * reset != 0 zeroes the counters. */
int flosic_profile_read(flosic_ctx* ctx, double* out, int reset);

/* Instrumentation (no counterpart in the paper), the tensor-core overlap of
 * the mixed path (timed while flosic_profile is enabled): host array out[3]:
 * [0] summed duration (ms) of the overlap-kernel launches, [1] their number,
 * [2] their algorithmic flops (2 N^2 G per spin block and launch; the split
 * products and padding the tensor cores also execute are not counted).
 * Waits for the device.  reset != 0 zeroes the counters.  Errors: ARG, CUDA. */
int flosic_profile_read_overlap(flosic_ctx* ctx, double* out, int reset);

/* Allocation-free Poisson solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they
 * run -- code inside another framework's memory arena or under a hard
 * memory cap, and latency-critical loops that must not call
 * cudaMalloc/cudaFree (those can synchronise the whole device and fail when
 * memory is tight).  It computes what flosic_orbital_poisson computes for
 * one grid (float64 conjugate gradients, no preconditioner, the same
 * 12th-order Laplacian and l <= 2 multipole boundary values) without a
 * context and without allocating anything: no cudaMalloc, no cudaFree, no
 * host heap.  Its scratch is one static device array of about 32 MiB that
 * every GPU loading this library holds until the process exits.
 *   nx, ny, nz, h, origin (host [3]): the grid, as in flosic_system.
 *   phi [norb][G] float64 (device): orbitals; rho = phi^2.
 *   V   [norb][G] float64 (device): out, the potentials (no warm start).
 *   cg_tol, max_iter: as in flosic_options.
 *   iters, conv_flags [norb] int32 (device, may be NULL): as in
 *   flosic_orbital_poisson.
 * Limits: 1 <= norb <= 128 and norb*nx*ny*nz <= 1048576; larger problems
 * are rejected with FLOSIC_ERR_ARG before any work is queued.
 * The first call on a device sets that device up (looks up the device
 * address of the scratch array and uploads the stencil weights); make that
 * first call before any stream capture.  That set-up is kept until the
 * process exits: resetting the device (cudaDeviceReset) after the first
 * call is not supported.  All calls share the one scratch array, so calls
 * that overlap on the GPU (from two host threads or on two streams) race
 * and must be serialised by the caller.  Every call synchronises `stream`:
 * it reads the number of unconverged orbitals back to the host every 8
 * iterations and the convergence flags at the end.
 * Errors: ARG, CUDA, NOCONV; the message is in flosic_noalloc_last_error(). */
int flosic_orbital_poisson_noalloc(int nx, int ny, int nz, double h, const double* origin,
                                   int norb, const double* phi, double* V, double cg_tol,
                                   int max_iter, int* iters, int* conv_flags, void* stream);

/* Message of the last failing flosic_orbital_poisson_noalloc call made
 * from the calling host thread (one buffer per host thread). */
const char* flosic_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLOSIC_H */
