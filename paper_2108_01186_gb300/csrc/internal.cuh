// Internal declarations of the sm_103a FLO-SIC library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/flosic.h"

namespace flosic {

constexpr int kHalf = 6;          // half-width of the 12th-order stencil
constexpr int kChunk = 1024;      // grid points per chunk of a chunked kernel
constexpr int kChunkThreads = 256;
constexpr int kMaxN = 128;        // orbitals per spin block supported
constexpr long long kMaxGridPoints = 2147483647LL;   // nx*ny*nz per system (32-bit point indices)
constexpr double kPi = 3.14159265358979323846;

// One spin block of one system, as seen by the kernels.
struct BlkDesc {
    int nx, ny, nz, N;
    double h, dV, ox, oy, oz;   // spacing, volume element, origin
    double cx, cy, cz;          // multipole centre (box centre)
    long long G;                // grid points
    long long off;              // offset of orbital 0 in orbital-sized arrays
    long long moff;             // offset in N x N arrays
    long long voff;             // offset in V_avg
    long long soff;             // offset of this block's system in per-system grid arrays
    long long fod_off;          // offset (in FODs) of FOD 0
    int orb0;                   // global index of orbital 0
    int sys, spin;
    long long chunk0;           // first global chunk of orbital 0
    int nchunk;                 // chunks per orbital
    long long bnd0;             // first entry in the boundary-point list
    int nbnd;                   // points within 6 of a Dirichlet face (they have ghost taps)
    int per;                    // periodic directions (bit 0 x, 1 y, 2 z)
    long long kq[3];            // Kronecker solver: offsets of Q_d (then Q_d^T) in the matrix table
    long long kl[3];            // and of the eigenvalues of T_d
    long long kt[3];            // tensor-core transforms: offsets of the split bf16 matrices
    int tc;                     // 1: this block's transforms run on the tensor cores
    int gtma;                   // 1: the overlap Gram's psi tiles are staged by the copy engine
};

// periodic-direction mask of a boundary mode
inline int boundary_mask(int boundary) {
    return boundary == FLOSIC_BC_PERIODIC ? 7 : (boundary == FLOSIC_BC_SLAB ? 3 : 0);
}
// wraps a coordinate of a periodic direction that is at most n outside [0, n)
__host__ __device__ __forceinline__ int wrap_coord(int q, int n) { return q < 0 ? q + n : (q >= n ? q - n : q); }

// One multigrid level of one spin block (level 0 = the fine grid).
constexpr int kMaxLevels = 10;
constexpr int kTileX = 32, kTileY = 16, kTileZ = 32;   // 3-D tiles of the sweeps (threads 32 x 8)
constexpr int kTileZc = 4;   // tile z-depth on the coarse multigrid levels (enough CTAs to fill the GPU)
constexpr int kCoarseSweeps = 40;      // damped-Jacobi sweeps on the coarsest level
constexpr int kCoarseMax = 2000;       // largest coarsest level (points) kept in shared memory
// planes of a tile staged with the 6-point x/y halo by the z-marching sweeps
constexpr int kPX = kTileX + 2 * kHalf;   // staged plane width
constexpr int kPY = kTileY + 2 * kHalf;   // staged plane height
constexpr int kSlots = (kPX * kPY + kTileX * (kTileY / 2) - 1) / (kTileX * (kTileY / 2));   // per thread
struct LvlDesc {
    int nx, ny, nz;
    int coarsest;          // 1 if this is the block's last level
    double h;              // 2^l h
    long long G;           // points (0: the block has no such level)
    long long off;         // offset of orbital 0 in this level's arrays
    long long chunk0;      // first chunk of orbital 0 in this level's chunk table
    int nchunk;            // chunks per orbital
    long long tile0;       // first tile of orbital 0 in this level's tile table
    int ntile;             // tiles per orbital
    int tma;               // level 0: 1 if the stencil operands of this block are TMA-staged
    int utma;              // level 0: 1 if the refinement update's operands are TMA-staged
    int per;               // level 0: periodic directions (bit 0 x, 1 y, 2 z); 0 on coarse levels
    int tz;                // z-depth of this level's tiles (kTileZ on level 0, kTileZc below)
    // Diagonal weight (units 1/h_l^2) of the 7-point operator at the last
    // point of each dimension, 2 elsewhere; differs from 2 on levels whose
    // parent had an even side (see multigrid.cu).  corr = any of them != 2.
    float cl[3];
    int corr;
    // 1/dd by which dimensions the point is last in (bit 0 x, 1 y, 2 z),
    // dd = 6 + sum over those dimensions of (cl - 2)
    float idd[8];
};

// Per-level buffers as the kernels see them (passed by value).
template <class T>
struct MgPtrs {
    T* r[kMaxLevels];      // level right-hand side (level 0: the CG residual)
    T* e[kMaxLevels];      // level correction (level 0: z = M r)
    T* t[kMaxLevels];      // scratch (level 0: the CG q buffer, idle during the V-cycle)
    const LvlDesc* lvl[kMaxLevels];
    const int* coarsest_level;   // [nblk]
};

// Per-orbital state of the batched conjugate-gradient solver.
struct CgState {
    double* rr;        // [norb] r.r (or r.z) of the current iterate
    double* pq;        // [norb] p.Ap
    double* bb;        // [norb] ||b||^2 of the current linear system
    double* thr;       // [norb] stop when rr <= thr
    double* beta;      // [norb] rr_new / rr_old (or rz_new / rz_old)
    double* rz;        // [norb] r.z of the preconditioned solver
    double* part;      // [max(chunks, tiles)] per-CTA partial sums
    double* part2;     // [max(chunks, tiles)] a second set of partial sums
    unsigned* count;   // [norb] last-block counters
    int* active;       // [norb] 1 = CG still iterating
    int* oactive;      // [norb] 1 = still refining (mixed precision)
    int* iters;        // [norb] iterations done (all precisions)
    int* n_active;     // [1] number of orbitals with active = 1
    int* n_oactive;    // [1] number of orbitals with oactive = 1
    int* conv;         // [norb] 1 = converged
    double* prof_bytes;  // [1] algorithmic bytes moved by the stencil-apply launches
    unsigned* dmax;      // [norb] float bits of max |d| of the current correction (refinement update)
    int* xz;             // [norb] 1 = the refinement's x is zero and not stored (cold Kronecker start)
    const int* mask;     // [norb] 1 = this context solves the orbital (see flosic_set_orbital_mask)
};

struct Workspace {
    // FLO build (N x N per block, packed like S)
    double *vals, *grads, *rho_a, *T, *M, *S, *Q, *C, *U, *lam, *P;
    double *vbar;          // [sum N*N] adjoint of psi at the FODs
    int* node_idx;         // [norb][64] grid index of each FOD's interpolation nodes (-1: outside)
    double* node_wt;       // [norb][64] their tricubic weights
    double* tmp;           // [4][sum N*N] scratch of the small kernels
    double* E2;            // [sum 2 N*N] [C^T | D] of the reverse apply
    long long mat_elems;   // sum N*N
    double* mat_part;      // partial N x N sums [kparts][sum N*N]
    float* gram_part;      // mixed path: tensor-core Gram partials [per block: chunks][N][N]
    // AAR inner solver (mixed path): previous f, history rings of m slots
    // (dx, df), per-tile dot partials, per-orbital weights
    float *aar_fprev, *aar_X, *aar_F;
    double *aar_part, *aar_gamma;
    long long* gram_off;   // [nblk] offsets into gram_part
    double* mom;           // [norb][10]
    double* mom_part;      // [nchunk_total][10]
    double* e_part;        // [nchunk_total][2] energies partials
    double* e_orb;         // [norb][2] U_i, E_xc,i
    int* status;           // [4] device status words
    int* mask;             // [norb] orbital mask (1 = computed here), all ones by default
    // Poisson
    double *b64, *r64, *p64, *q64;   // FP64 CG vectors / refinement
    float *d32, *r32, *p32, *q32;    // FP32 inner CG vectors
    double* veff;                    // exact adjoint: zero-boundary solve, then its V^SIC
    double* vsic;                    // V_i^SIC = -(V_i + v_xc,i) of the last energy pass (float64
                                     // path, or the exact adjoint's input)
    float* wbar;                     // mixed path, V reused in the adjoint: V_i^SIC phi_i as float
    double *z64, *p64b;              // multigrid PCG (FP64): z = M r, V-cycle scratch
    float *z32, *p32b;               // multigrid PCG (FP32)
    CgState cg;
};

struct Multigrid {
    bool enabled = false;
    int nlev = 0;                              // levels of the deepest block
    LvlDesc* d_lvl[kMaxLevels] = {};           // [nblk] per level (device)
    std::vector<LvlDesc> h_lvl[kMaxLevels];
    long long nchunk[kMaxLevels] = {};         // chunks per level (all orbitals)
    long long elems[kMaxLevels] = {};          // elements per level (all orbitals)
    int* d_coarsest_level = nullptr;           // [nblk]
    int4* d_tiles[kMaxLevels] = {};            // tile -> (orbital, x0, y0, z0) per level
    long long ntiles[kMaxLevels] = {};
    long long coarsest_max = 0;
    void* r[kMaxLevels] = {};                  // levels >= 1 (T = float or double)
    void* e[kMaxLevels] = {};
    void* t[kMaxLevels] = {};
};

}  // namespace flosic

namespace flosic {
// Kronecker-product solver: transform matrices, eigenvalues and the launch
// shape of its three passes (x, y, z lines).
struct KronPlan {
    float* mat = nullptr;          // per distinct 1-D operator: Q (n x n), then Q^T
    float* lam = nullptr;          // per distinct 1-D operator: eigenvalues (n)
    long long* items = nullptr;    // [3][nblk + 1] first tile of each block per pass (CUDA-core kernel)
    long long total[3] = {0, 0, 0};
    int threads[3] = {0, 0, 0};
    size_t smem[3] = {0, 0, 0};
    int grid[3] = {0, 0, 0};
    int n_simt = 0, n_tc = 0;      // blocks on the CUDA-core and on the tensor-core transforms
    uint16_t* tc_mat = nullptr;    // per distinct operator of a tensor-core block: split bf16 matrices
    long long* tc_items = nullptr; // [6][nblk + 1] first tile of each block per pass (tensor-core kernel)
    std::vector<int> tc_force;     // [nblk] host: 0 = CUDA-core transforms even if eligible (autotuner)
    void* tc_maps = nullptr;       // [6][nblk] CUtensorMap of each pass's input rows
    void* tc_omaps = nullptr;      // [6][nblk] CUtensorMap of each pass's output lines
    long long tc_total[6] = {0, 0, 0, 0, 0, 0};
    int tc_grid[6] = {0, 0, 0, 0, 0, 0};
};
}  // namespace flosic

struct flosic_ctx {
    flosic_options opt;
    std::vector<flosic_system> sys;
    std::vector<flosic::BlkDesc> blk;       // host copy
    flosic::BlkDesc* d_blk = nullptr;       // device copy
    int nblk = 0, norb = 0;
    long long orb_elems = 0, vavg_elems = 0, mat_elems = 0, nchunk_total = 0;
    long long sgrid_elems = 0;   // sum over systems of the grid points (per-system fields)
    int kparts = 0;                         // K-splits of the grid contractions
    int num_sms = 152;                      // multiprocessors of the context's device
    std::vector<int> h_orb_blk;
    int* d_orb_blk = nullptr;               // [norb] block of each orbital
    int* d_chunk_orb = nullptr;             // [nchunk_total] orbital of each chunk
    int* d_sys_orb0 = nullptr;              // [nsys+1] first orbital of each system
    int* d_bidx = nullptr;                  // boundary points (flat index) of every block
    double* d_bcoef = nullptr;              // [sum nbnd][10] boundary-map coefficients
    flosic::Workspace ws{};
    flosic::Multigrid mg;
    flosic::KronPlan kron;
    int n_unmasked = 0;                     // orbitals with mask 1
    bool have_forward = false;
    bool have_energy = false;
    std::string err;
    int* h_pinned = nullptr;                // small pinned host buffer
    int* h_pinned_dev = nullptr;            // its device view (mapped), or null
    mutable long long launches = 0;         // kernels launched by this context
    int n_tma_blocks = 0;                   // blocks whose stencil operands the copy engine stages
    void* d_tmaps = nullptr;                // per-block tensor maps of the z buffer (CUtensorMap)
    int n_utma_blocks = 0;                  // blocks whose refinement-update operands the copy engine stages
    void* d_umaps = nullptr;                // per-block tensor maps of d, r and x for the update (CUtensorMap)
    // optional CUDA-event timing of the dominant kernel (the CG stencil apply)
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;       // start/stop pairs, recorded in order
    int prof_used = 0;                      // pairs recorded and not yet summed
    double prof_ms = 0.0;                   // summed duration of timed launches
    long long prof_launches = 0;
    // the same for the tensor-core overlap launches (mixed path)
    std::vector<cudaEvent_t> ov_ev;
    int ov_used = 0;
    double ov_ms = 0.0, ov_flops = 0.0;   // timed duration, algorithmic flops (2 N^2 G per block)
    long long ov_launches = 0;
    std::vector<void*> allocations;
    // flosic_step_host: device copies of the step's inputs (two sets, so
    // the next step's can arrive while this one computes) and outputs,
    // allocated at the first call
    struct HostStep {
        bool ready = false;
        double* psi[2] = {nullptr, nullptr};
        double* fods[2] = {nullptr, nullptr};
        const double* pre_psi = nullptr;    // host arrays already copied into set `pre`
        const double* pre_fods = nullptr;
        int pre = -1;
        double *phi = nullptr, *V = nullptr, *Vavg = nullptr, *dpsi = nullptr, *dfod = nullptr;
        double *E = nullptr, *U = nullptr, *Exc = nullptr, *gE = nullptr;
        int* conv[2] = {nullptr, nullptr};  // convergence flags of the step computed in set k
        cudaStream_t copy = nullptr;        // host -> device copies of the next step's inputs
        cudaStream_t copy_out = nullptr;    // device -> host copies of a step's outputs
        cudaEvent_t copied[2] = {nullptr, nullptr};
        cudaEvent_t done = nullptr;         // a step's outputs are final
        // the next step's FLO build and Poisson solve, started by the previous
        // call on its prefetched inputs (valid until another call uses the context)
        bool fwd_valid = false;
        const double* fwd_psi = nullptr;
        const double* fwd_fods = nullptr;
        int fwd_rc = 0;                     // the solve's return code (OK or NOCONV)
        int fwd_conv = 0;                   // its flags' set
    } hs;
};

namespace flosic {

// Mixed precision with V reused in the adjoint: the energy pass stores
// wbar_i = V_i^SIC phi_i (float32), all the adjoint reads per point besides
// psi; otherwise V_i^SIC itself (float64).
// Copies n status words from device memory to the context's pinned host
// buffer on stream s: through its mapping by a one-warp kernel when the
// buffer is mapped (no copy engine, so the read does not queue behind a large
// transfer another stream has in flight), else by cudaMemcpyAsync.
cudaError_t fetch_words(const flosic_ctx* c, const int* src, int n, cudaStream_t s);
// Fills n doubles of device memory with v on stream s (a one-warp kernel).
void fill_doubles(const flosic_ctx* c, double* dst, int n, double v, cudaStream_t s);

inline bool uses_wbar(const flosic_ctx* c) {
    return c->opt.precision == FLOSIC_MIXED && c->opt.adjoint_mode == FLOSIC_ADJ_REUSE_V;
}

// ---- launchers implemented in the .cu files ----------------------------
// FLO build (flo_build.cu)
void launch_interp_fod(const flosic_ctx* c, const double* psi, const double* fods, cudaStream_t s);
void launch_gram(const flosic_ctx* c, const double* psi, cudaStream_t s);
void launch_lowdin(const flosic_ctx* c, double* S_out, double* Q_out, cudaStream_t s);
size_t lowdin_smem(const flosic_ctx* c);   // dynamic shared memory of the Loewdin kernel
// raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (never lowers it; thread-safe)
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes);
void launch_flo_apply(const flosic_ctx* c, const double* psi, double* phi, cudaStream_t s);
void launch_backward_contract(const flosic_ctx* c, const double* psi, const double* phi,
                              const double* Vsrc, const double* gE, cudaStream_t s);
void launch_backward_small(const flosic_ctx* c, double* dE_dfod, cudaStream_t s);
void launch_psibar(const flosic_ctx* c, const double* psi, const double* phi, const double* Vsrc,
                   const double* gE, const double* fods, double* dpsi, cudaStream_t s);
// Poisson (poisson.cu)
void launch_rhs(flosic_ctx* c, const double* phi, bool with_bc, double* b, cudaStream_t s);
cudaError_t upload_boundary_constants();
cudaError_t setup_boundary(flosic_ctx* c);
int run_poisson(flosic_ctx* c, double* b, double* V, bool warm, cudaStream_t s);
void finish_poisson(flosic_ctx* c, int* iters, int* conv, cudaStream_t s);
cudaError_t upload_stencil_constants();
void launch_bc_adjoint(flosic_ctx* c, const double* W, const double* V, double* out, cudaStream_t s);
// xc / energies (xc.cu)
void launch_xc_energy(const flosic_ctx* c, const double* psi, const double* phi, const double* V,
                      double scale, double* Vavg, cudaStream_t s);
void launch_energy_reduce(const flosic_ctx* c, double* U, double* Exc, double* E_sic,
                          cudaStream_t s);

// Kronecker-product inner solver (mixed precision)
int kron_max_n();
cudaError_t setup_kron(flosic_ctx* c);
void launch_kron_solve(flosic_ctx* c, const float* r, float* d, float* t1, float* t2, cudaStream_t s);
// its transforms on the tensor cores (kron_tc.cu)
bool kron_tc_eligible(const BlkDesc& B);
// times the tensor-core and CUDA-core transforms per distinct eligible block
// shape and re-plans the solver with the faster per shape (kron.cu)
cudaError_t kron_autotune(flosic_ctx* c);
void kron_tc_pack(int n, const std::vector<double>& Vs, const std::vector<double>& Va, std::vector<uint16_t>& out);
size_t kron_tc_smem();
const void* kron_tc_symbol();
bool kron_tc_map(void* encode_fn, CUtensorMap* map, const BlkDesc& B, int axis, const float* buf);
bool kron_tc_map_out(void* encode_fn, CUtensorMap* map, const BlkDesc& B, int axis, float* buf);
long long kron_tc_tiles(const BlkDesc& B, int axis);
void launch_kron_tc_pass(flosic_ctx* c, int step, float* out, cudaStream_t s);
// Alternating Anderson-Richardson inner solver (mixed precision)
template <class T>
void launch_aar_step(flosic_ctx* c, T* x, T* r, T* f, int k, bool anderson, cudaStream_t s,
                     void (*precondition)(flosic_ctx*, T*, T*, cudaStream_t));
long long aar_part_elems(long long ntiles0);
int aar_max_m();
// tensor-core overlap Gram (mixed precision)
long long gram_tc_part_elems(const flosic_ctx* c, std::vector<long long>& off);
cudaError_t setup_gram_tc();
bool gram_async_eligible(const BlkDesc& B);   // the overlap Gram's asynchronous-copy kernel takes B
void launch_gram_tc(const flosic_ctx* c, const double* psi, cudaStream_t s);
// SC_AvgSIC Hamiltonian apply: H psi = -1/2 Delta_h psi + (v_loc + V_avg) psi
void launch_hamiltonian(const flosic_ctx* c, const double* psi, const double* vloc, const double* vavg,
                        double* hpsi, cudaStream_t s);
cudaError_t upload_hamiltonian_constants();
template <class T>
void launch_vcycle(const flosic_ctx* c, const MgPtrs<T>& mp, const int* active, cudaStream_t s);
template <class T>
void launch_apply12_pcg(flosic_ctx* c, const T* z, T* p, T* q, cudaStream_t s);
template <class T>
void launch_residual12_aar(flosic_ctx* c, const T* dx, T* r, cudaStream_t s);
size_t apply12_tma_smem(size_t elem);
const void* apply12_tma_symbol(bool f32);
void launch_residual12(flosic_ctx* c, const double* b, const double* x, double* r, double tol2, int max_iter,
                       int* flag, int* counter, int want_bb, cudaStream_t s);
cudaError_t upload_ff_weights();
int setup_update_maps(flosic_ctx* c);   // refinement update's tensor maps (refine.cu); blocks on that path
// mixed precision: float-float refinement around the float32 inner solves
// (b holds float-float pairs, written so by launch_rhs; x the solution's)
void launch_ff_init(flosic_ctx* c, const double* b, const double* V, bool warm, bool keep_zero, float2* x,
                    float* p32, double tol2, double inner_tol2, cudaStream_t s);
void launch_residual_ff(flosic_ctx* c, const double* b, const float2* x, float* p32, double tol2,
                        double inner_tol2, bool store_r, cudaStream_t s);
void launch_correct_ff(flosic_ctx* c, float2* x, cudaStream_t s);
// Kronecker inner solver: x += d and r -= A d in one sweep (r in pairs over b)
void launch_update_ff(flosic_ctx* c, double* r, float2* x, bool x_zero, double tol2, double inner_tol2,
                      cudaStream_t s);
void launch_join_ff(flosic_ctx* c, const float2* x, double* V, cudaStream_t s);
void stencil_weights(double* w);   // 12th-order weights w_0..w_6
const void* k_lowdin_symbol();
int check_cuda(flosic_ctx* c, cudaError_t e, const char* what);
inline void note_launch(const flosic_ctx* c) { ++c->launches; }
// Event pair around one launch of the dominant kernel (no-op unless profiling).
void prof_begin(flosic_ctx* c, cudaStream_t s);
void prof_end(flosic_ctx* c, cudaStream_t s);
void prof_collect(flosic_ctx* c);   // after a stream sync: sum recorded pairs
void ov_collect(flosic_ctx* c);     // the same for the overlap timer


}  // namespace flosic

// ---- device helpers ------------------------------------------------------
namespace flosic {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int linear_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

// Block-wide sum of one double (fixed order: warps then lanes).  All threads
// get the result.  scratch must hold 32 doubles.  Any block shape.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int tid = linear_tid();
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = (tid < nw) ? scratch[tid] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (tid == 0) scratch[0] = t;
    __syncthreads();
    double r = scratch[0];
    __syncthreads();
    return r;
}

// Block-wide sum of float partials: warps reduce in float, the warp sums
// are combined in float64 (fixed order).  Returns the sum to every thread.
__device__ __forceinline__ double block_sum(float v, double* scratch) {
    const int tid = linear_tid();
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = (double)v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += scratch[w];
        scratch[0] = t;
    }
    __syncthreads();
    const double r = scratch[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// float64 <-> float32 conversions from integer operations.  GB300 issues
// every float64 operation, conversions included, at about 1/70 of its
// float32 rate (measured: ~0.5 Top/s against ~35 Top/s), so a kernel that
// streams float64 data can afford well under one such operation per value it
// loads.  These keep per-point work on the integer and float32 pipes.
// Normal float32 range: magnitudes below 2^-126 become 0, magnitudes beyond
// the float32 range become infinite (non-finite values stay non-finite).
// ---------------------------------------------------------------------------
// round to nearest (ties away from zero)
__device__ __forceinline__ float d2f(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v) + (1ull << 28);
    const unsigned hi = (unsigned)(u >> 32);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned sign = hi & 0x80000000u;
    const unsigned m = (unsigned)(u >> 29) & 0x7fffffu;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | m);
}
// exact (float32 subnormals flushed to 0)
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (e == 0) return __hiloint2double((int)sign, 0);
    const unsigned e11 = (e == 255u) ? 2047u : e + 896u;
    return __hiloint2double((int)(sign | (e11 << 20) | (m >> 3)), (int)(m << 29));
}
// v = hi + lo, hi = d2f(v), lo = v - hi rounded to float (~48 significant bits).
// The 29 bits d2f drops, sign-extended from their top bit, are v - hi in
// units of 2^(e - 1075) (negative when hi was rounded up); one integer-to-float
// conversion and a scale by that power of two (with v's sign) give lo.
__device__ __forceinline__ float2 d2ff(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const float h = d2f(v);
    const int ev = (int)((u >> 52) & 0x7ffu);
    const int rem = (int)((unsigned)u << 3) >> 3;                 // the 29 dropped bits, signed
    const unsigned pe = (unsigned)(ev - 1075 + 127);              // 2^(ev - 1075) as a float exponent
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const float lo = (pe - 1u < 254u) ? __int2float_rn(rem) * __uint_as_float((pe << 23) | sign) : 0.f;
    return make_float2(h, lo);
}
// hi + lo in float64 (one float64 addition)
__device__ __forceinline__ double ff2d(float2 p) { return f2d(p.x) + f2d(p.y); }

// ---------------------------------------------------------------------------
// Float-float arithmetic: unevaluated pairs (h, l) of float32 numbers with
// |l| <= ulp(h)/2, about 48 significant bits.  Knuth's error-free two-sum
// for additions, an FMA-based exact two-product for products.
// ---------------------------------------------------------------------------
struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = ff_two_sum(x.h, y.h);
    const ff t = ff_two_sum(x.l, y.l);
    s.l += t.h;
    s = ff_quick(s.h, s.l);
    s.l += t.l;
    return ff_quick(s.h, s.l);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    return ff_quick(p, e);
}
// Sum of six pairs: exact two-sums on the high parts, the low parts and the
// rounding errors added in float (error ~ 6 eps^2 of the largest term).
__device__ __forceinline__ ff ff_sum6(ff a, ff b, ff c, ff d, ff e, ff f) {
    ff s = ff_two_sum(a.h, b.h);
    float err = s.l;
    s = ff_two_sum(s.h, c.h); err += s.l;
    s = ff_two_sum(s.h, d.h); err += s.l;
    s = ff_two_sum(s.h, e.h); err += s.l;
    s = ff_two_sum(s.h, f.h); err += s.l;
    err += ((a.l + b.l) + (c.l + d.l)) + (e.l + f.l);
    return ff_quick(s.h, err);
}
// a + b with b a plain float (two-sum, then renormalise)
__device__ __forceinline__ ff ff_addf(ff a, float b) {
    const ff s = ff_two_sum(a.h, b);
    return ff_quick(s.h, s.l + a.l);
}
// Running sum of pairs (th, tl) with |tl| small against |th|: exact
// two-sum of the high parts, the low parts and its rounding error gathered in
// a.l without renormalising; after n terms the error is ~n 2^-48 sum |terms|
// (relative to the sum itself when the terms share a sign).  Renormalise with
// ff_quick at the end.
__device__ __forceinline__ ff ff_acc(ff a, float th, float tl) {
    const ff s = ff_two_sum(a.h, th);
    return {s.h, a.l + (s.l + tl)};
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {   // pair times float
    const float p = a.h * b;
    return ff_quick(p, fmaf(a.h, b, -p) + a.l * b);
}
__device__ __forceinline__ ff to_ff(float2 p) { return {p.x, p.y}; }
__device__ __forceinline__ double ff_to_double(ff a) { return f2d(a.h) + f2d(a.l); }
// warp-wide pair sum (every lane gets it)
__device__ __forceinline__ ff warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ff w = {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = ff_add(v, w);
    }
    return v;
}

__device__ __forceinline__ int find_block(const BlkDesc* blk, int nblk, int orb) {
    int b = 0;
    while (b + 1 < nblk && blk[b + 1].orb0 <= orb) ++b;
    return b;
}

// ---- 3-D tiles of one orbital (x0, y0, z0; kTileX x kTileY x kTileZ) ----
struct TilePos {
    int o, b, x0, y0, z0, z1;
    long long base;    // offset of the orbital in the level's arrays
    long long first;   // global tile index of the orbital's first tile
};

__device__ __forceinline__ TilePos tile_pos(const BlkDesc* blk, const LvlDesc* L, const int4* tiles,
                                            const int* orb_blk, int t) {
    const int4 tl = tiles[t];
    TilePos p;
    p.o = tl.x;
    p.b = orb_blk[p.o];
    const LvlDesc& D = L[p.b];
    const int i = p.o - blk[p.b].orb0;
    p.x0 = tl.y;
    p.y0 = tl.z;
    p.z0 = tl.w;
    p.z1 = min(p.z0 + D.tz, D.nz);
    p.base = D.off + (long long)i * D.G;
    p.first = D.tile0 + (long long)i * D.ntile;
    return p;
}

// Stores this CTA's partial and returns true in the CTA that arrives last
// among the ntile CTAs of one orbital.
template <class P>
__device__ __forceinline__ bool tile_arrive(P partial, double* part, int t, unsigned* counter, int ntile,
                                            double* scratch) {
    __shared__ bool last;
    const double s = block_sum(partial, scratch);
    if (linear_tid() == 0) {
        part[t] = s;
        __threadfence();
        last = (atomicAdd(counter, 1u) == (unsigned)(ntile - 1));
    }
    __syncthreads();
    return last;
}

// Fixed-order sum of part[first .. first + n) read through L2.
__device__ __forceinline__ double tile_gather(const double* part, long long first, int n, double* scratch) {
    double v = 0.0;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int k = linear_tid(); k < n; k += nt) v += __ldcg(part + first + k);
    return block_sum(v, scratch);
}

template <class T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

// Elementwise sweep over one tile, vectorised along x when the rows are
// aligned (nx a multiple of the vector width); body(g, n) handles n
// consecutive points starting at flat index g (n = vector width, or 1).
template <class T, class Body>
__device__ __forceinline__ void tile_elementwise(const LvlDesc& D, const TilePos& P, Body body) {
    constexpr int V = Vec<T>::n;
    constexpr int XG = kTileX / V;               // vector groups per row
    constexpr int RPI = 256 / XG;                // rows per pass
    const int tid = linear_tid();
    const int xg = tid % XG, r0 = tid / XG;
    const int nz = P.z1 - P.z0;
    const int nrows = kTileY * nz;
    const bool vec = (D.nx % V == 0) && (P.base % V == 0);
    const int x = P.x0 + xg * V;
#pragma unroll 4
    for (int row = r0; row < nrows; row += RPI) {
        const int y = P.y0 + row % kTileY, z = P.z0 + row / kTileY;
        if (y >= D.ny || x >= D.nx) continue;
        const long long g = P.base + ((long long)z * D.ny + y) * D.nx + x;
        if (vec) {
            body(g, V);
        } else {
            for (int k = 0; k < V && x + k < D.nx; ++k) body(g + k, 1);
        }
    }
}



// Same sweep, passing the coordinates of the first point: body(x, y, z, g, n).
template <class T, class Body>
__device__ __forceinline__ void tile_rows(const LvlDesc& D, const TilePos& P, Body body) {
    constexpr int V = Vec<T>::n;
    constexpr int XG = kTileX / V;
    constexpr int RPI = 256 / XG;
    const int tid = linear_tid();
    const int xg = tid % XG, r0 = tid / XG;
    const int nz = P.z1 - P.z0;
    const int nrows = kTileY * nz;
    const bool vec = (D.nx % V == 0) && (P.base % V == 0);
    const int x = P.x0 + xg * V;
#pragma unroll 2
    for (int row = r0; row < nrows; row += RPI) {
        const int y = P.y0 + row % kTileY, z = P.z0 + row / kTileY;
        if (y >= D.ny || x >= D.nx) continue;
        const long long g = P.base + ((long long)z * D.ny + y) * D.nx + x;
        if (vec) {
            body(x, y, z, g, V);
        } else {
            for (int k = 0; k < V && x + k < D.nx; ++k) body(x + k, y, z, g + k, 1);
        }
    }
}

}  // namespace flosic
