// Per-orbital Poisson solves (Sec. II.A): -Delta_h V_i = 4 pi rho_i with the
// 12th-order centred Laplacian, Dirichlet values from the l <= 2 multipole
// expansion of rho_i on the 6-layer ghost shell, and batched conjugate
// gradients over every orbital of every system in one launch per step.
//
// The ghost values are known, so they move to the right-hand side:
//   A V = 4 pi rho + bc,  A = -Delta_h with zero ghosts (SPD),
//   bc(g) = (1/h^2) sum over the taps of g that leave the interior of w_m V_b.
//
// Precision: FP64 runs CG in float64.  MIXED runs CG in float32 on the
// correction equation A d = r and refines x += d against a float64 residual
// r = b - A x until ||r|| <= tol ||b||.
#include <cstdio>

#include "internal.cuh"

namespace flosic {

__constant__ double c_w[kHalf + 1];
__constant__ float c_wf[kHalf + 1];

// Centred second-derivative weights of order 12 on a unit grid:
//   w_k = 2 (-1)^{k+1} (6!)^2 / (k^2 (6-k)! (6+k)!), w_0 = -2 sum_k 1/k^2.
void stencil_weights(double* w) {
    auto fact = [](int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; };
    const double m6 = fact(kHalf);
    w[0] = 0.0;
    for (int k = 1; k <= kHalf; ++k) {
        w[k] = ((k & 1) ? 2.0 : -2.0) * m6 * m6 / (double(k) * k * fact(kHalf - k) * fact(kHalf + k));
        w[0] -= 2.0 / (double(k) * k);
    }
}

cudaError_t upload_stencil_constants() {
    double w[kHalf + 1];
    float wf[kHalf + 1];
    stencil_weights(w);
    for (int k = 0; k <= kHalf; ++k) wf[k] = (float)w[k];
    cudaError_t e = cudaMemcpyToSymbol(c_w, w, sizeof(w));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_wf, wf, sizeof(wf));
}

// ---------------------------------------------------------------------------
// chunk bookkeeping and deterministic per-orbital reductions
// ---------------------------------------------------------------------------
struct ChunkPos {
    int o, b, i;
    long long base, g0;
    int npts;
    long long first;   // global chunk index of chunk 0 of this orbital
};

__device__ __forceinline__ ChunkPos decode_chunk(const BlkDesc* blk, const int* chunk_orb,
                                                 const int* orb_blk, long long t) {
    ChunkPos p;
    p.o = chunk_orb[t];
    p.b = orb_blk[p.o];
    const BlkDesc& B = blk[p.b];
    p.i = p.o - B.orb0;
    p.first = B.chunk0 + (long long)p.i * B.nchunk;
    const long long c = t - p.first;
    p.base = B.off + (long long)p.i * B.G;
    p.g0 = c * kChunk;
    const long long rem = B.G - p.g0;
    p.npts = rem < kChunk ? (int)rem : kChunk;
    return p;
}

// Writes this CTA's partial and returns true in the CTA that arrives last
// among the nchunk CTAs of one orbital.
__device__ __forceinline__ bool arrive(double partial, double* part, long long t, unsigned* counter,
                                       int nchunk, double* scratch) {
    __shared__ bool last;
    const double s = block_sum(partial, scratch);
    if (threadIdx.x == 0) {
        part[t] = s;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)(nchunk - 1));
    }
    __syncthreads();
    return last;
}

// Sum of part[first .. first+n) in a fixed order (strided per thread, then
// block_sum), read through L2.
__device__ __forceinline__ double gather_sum(const double* part, long long first, int n,
                                             double* scratch) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += __ldcg(part + first + k);
    return block_sum(v, scratch);
}

// (-Delta_h u)(g) with u = 0 outside the interior (zero ghost values).
template <class T>
__device__ __forceinline__ T apply_A(const T* __restrict__ u, long long g, int x, int y, int z,
                                     int nx, int ny, int nz, T ih2);

template <>
__device__ __forceinline__ double apply_A<double>(const double* __restrict__ u, long long g, int x,
                                                  int y, int z, int nx, int ny, int nz, double ih2) {
    const long long sy = nx, sz = (long long)nx * ny;
    double acc = 3.0 * c_w[0] * u[g];
#pragma unroll
    for (int m = 1; m <= kHalf; ++m) {
        double s = 0.0;
        if (x - m >= 0) s += u[g - m];
        if (x + m < nx) s += u[g + m];
        if (y - m >= 0) s += u[g - m * sy];
        if (y + m < ny) s += u[g + m * sy];
        if (z - m >= 0) s += u[g - m * sz];
        if (z + m < nz) s += u[g + m * sz];
        acc += c_w[m] * s;
    }
    return -acc * ih2;
}

template <>
__device__ __forceinline__ float apply_A<float>(const float* __restrict__ u, long long g, int x,
                                                int y, int z, int nx, int ny, int nz, float ih2) {
    const long long sy = nx, sz = (long long)nx * ny;
    float acc = 3.0f * c_wf[0] * u[g];
#pragma unroll
    for (int m = 1; m <= kHalf; ++m) {
        float s = 0.0f;
        if (x - m >= 0) s += u[g - m];
        if (x + m < nx) s += u[g + m];
        if (y - m >= 0) s += u[g - m * sy];
        if (y + m < ny) s += u[g + m * sy];
        if (z - m >= 0) s += u[g - m * sz];
        if (z + m < nz) s += u[g + m * sz];
        acc += c_wf[m] * s;
    }
    return -acc * ih2;
}

__device__ __forceinline__ void xyz_of(long long g, int nx, int ny, int& x, int& y, int& z) {
    const long long pl = (long long)nx * ny;
    z = (int)(g / pl);
    const long long r = g - (long long)z * pl;
    y = (int)(r / nx);
    x = (int)(r - (long long)y * nx);
}

// ---------------------------------------------------------------------------
// multipole moments (l <= 2) of rho_i about the box centre
// ---------------------------------------------------------------------------
__global__ void k_moments(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                          const int* __restrict__ orb_blk, const double* __restrict__ src,
                          int square, double* __restrict__ mom_part) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    const BlkDesc& B = blk[P.b];
    double m[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) m[q] = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x, y, z;
        xyz_of(g, B.nx, B.ny, x, y, z);
        const double v = src[P.base + g];
        const double rho = square ? v * v : v;
        const double Rx = B.ox + B.h * x - B.cx, Ry = B.oy + B.h * y - B.cy, Rz = B.oz + B.h * z - B.cz;
        const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
        m[0] += rho;
        m[1] += rho * Rx;
        m[2] += rho * Ry;
        m[3] += rho * Rz;
        m[4] += rho * (3.0 * Rx * Rx - r2);
        m[5] += rho * (3.0 * Ry * Ry - r2);
        m[6] += rho * (3.0 * Rz * Rz - r2);
        m[7] += rho * 3.0 * Rx * Ry;
        m[8] += rho * 3.0 * Rx * Rz;
        m[9] += rho * 3.0 * Ry * Rz;
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const double s = block_sum(m[q], scratch);
        if (threadIdx.x == 0) mom_part[t * 10 + q] = s;
    }
}

// One warp per orbital: mom[o][q] = dV * sum over its chunks (fixed order).
__global__ void k_sum_chunks10(const BlkDesc* __restrict__ blk, const int* __restrict__ orb_blk,
                               int norb, const double* __restrict__ part, double* __restrict__ out,
                               int scale_dV) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= norb) return;
    const BlkDesc& B = blk[orb_blk[o]];
    const long long first = B.chunk0 + (long long)(o - B.orb0) * B.nchunk;
    for (int q = 0; q < 10; ++q) {
        double v = 0.0;
        for (int c = lane; c < B.nchunk; c += 32) v += part[(first + c) * 10 + q];
        v = warp_sum(v);
        if (lane == 0) out[o * 10 + q] = scale_dV ? v * B.dV : v;
    }
}

void launch_moments(const flosic_ctx* c, const double* src, bool square, cudaStream_t s) {
    k_moments<<<(unsigned)c->nchunk_total, kChunkThreads, 0, s>>>(c->d_blk, c->d_chunk_orb,
                                                                  c->d_orb_blk, src, square ? 1 : 0,
                                                                  c->ws.mom_part); note_launch(c);
    k_sum_chunks10<<<(c->norb * 32 + 255) / 256, 256, 0, s>>>(c->d_blk, c->d_orb_blk, c->norb,
                                                              c->ws.mom_part, c->ws.mom, 1); note_launch(c);
}

// Multipole potential at offset R from the centre (moments mom[10]).
__device__ __forceinline__ double multipole_value(const double* mom, double Rx, double Ry, double Rz) {
    const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const double ir = rsqrt(r2);
    const double ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    double v = mom[0] * ir + (mom[1] * Rx + mom[2] * Ry + mom[3] * Rz) * ir3;
    const double quad = mom[4] * Rx * Rx + mom[5] * Ry * Ry + mom[6] * Rz * Rz +
                        2.0 * (mom[7] * Rx * Ry + mom[8] * Rx * Rz + mom[9] * Ry * Rz);
    return v + 0.5 * quad * ir5;
}

// ---------------------------------------------------------------------------
// right-hand side: b = 4 pi phi^2 + bc (mode 0) or b = phi^2 (mode 1, zero
// boundary, for the exact adjoint); also ||b||^2 per orbital.
// ---------------------------------------------------------------------------
__global__ void k_rhs(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                      const int* __restrict__ orb_blk, const double* __restrict__ phi,
                      const double* __restrict__ mom_all, int mode, double* __restrict__ b,
                      CgState st) {
    __shared__ double scratch[32];
    __shared__ double mom[10];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    const BlkDesc& B = blk[P.b];
    if (threadIdx.x < 10) mom[threadIdx.x] = mom_all[P.o * 10 + threadIdx.x];
    __syncthreads();
    const double ih2 = 1.0 / (B.h * B.h);
    double bb = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        const double v = phi[P.base + g];
        double val = (mode == 0 ? 4.0 * kPi : 1.0) * v * v;
        if (mode == 0) {
            int x, y, z;
            xyz_of(g, B.nx, B.ny, x, y, z);
            const int p[3] = {x, y, z};
            const int n[3] = {B.nx, B.ny, B.nz};
            double acc = 0.0;
            for (int d = 0; d < 3; ++d) {
                if (p[d] >= kHalf && p[d] < n[d] - kHalf) continue;
                for (int m = 1; m <= kHalf; ++m) {
                    for (int sg = -1; sg <= 1; sg += 2) {
                        const int qd = p[d] + sg * m;
                        if (qd >= 0 && qd < n[d]) continue;
                        int q[3] = {x, y, z};
                        q[d] = qd;
                        const double Rx = B.ox + B.h * q[0] - B.cx;
                        const double Ry = B.oy + B.h * q[1] - B.cy;
                        const double Rz = B.oz + B.h * q[2] - B.cz;
                        acc += c_w[m] * multipole_value(mom, Rx, Ry, Rz);
                    }
                }
            }
            val += acc * ih2;
        }
        b[P.base + g] = val;
        bb += val * val;
    }
    const BlkDesc& Bb = B;
    if (arrive(bb, st.part, t, st.count + P.o, Bb.nchunk, scratch)) {
        const double s = gather_sum(st.part, P.first, Bb.nchunk, scratch);
        if (threadIdx.x == 0) {
            st.bb[P.o] = s;
            st.count[P.o] = 0;
        }
    }
}

void launch_rhs(const flosic_ctx* c, const double* phi, bool with_bc, double* b, cudaStream_t s) {
    k_rhs<<<(unsigned)c->nchunk_total, kChunkThreads, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk,
                                                              phi, c->ws.mom, with_bc ? 0 : 1, b,
                                                              c->ws.cg); note_launch(c);
}

// ---------------------------------------------------------------------------
// conjugate gradients, batched over orbitals (one CTA per chunk of points)
// ---------------------------------------------------------------------------
__global__ void k_cg_reset(int norb, CgState st) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o == 0) {
        *st.n_active = norb;
        *st.n_oactive = norb;
    }
    if (o >= norb) return;
    st.active[o] = 1;
    st.oactive[o] = 1;
    st.iters[o] = 0;
    st.conv[o] = 0;
    st.count[o] = 0;
}

// r = b - A x (float64), rr = r.r; if the orbital already meets the target
// it stops (converged).  When init_p, p = r (the FP64 CG start).
__global__ void k_residual64(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                             const int* __restrict__ orb_blk, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r,
                             double* __restrict__ p, int init_p, double tol2, int max_iter,
                             int* __restrict__ flag, int* __restrict__ counter, CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!flag[P.o]) return;
    const BlkDesc& B = blk[P.b];
    const double ih2 = 1.0 / (B.h * B.h);
    double rr = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x_, y_, z_;
        xyz_of(g, B.nx, B.ny, x_, y_, z_);
        const double rv = b[P.base + g] - apply_A<double>(x + P.base, g, x_, y_, z_, B.nx, B.ny, B.nz, ih2);
        r[P.base + g] = rv;
        if (init_p) p[P.base + g] = rv;
        rr += rv * rv;
    }
    if (arrive(rr, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double s = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            st.count[P.o] = 0;
            st.rr[P.o] = s;
            st.thr[P.o] = tol2 * st.bb[P.o];
            if (!(s > st.thr[P.o])) {          // converged (also b = 0)
                flag[P.o] = 0;
                st.conv[P.o] = 1;
                atomicSub(counter, 1);
            } else if (st.iters[P.o] >= max_iter || !isfinite(s)) {
                flag[P.o] = 0;
                atomicSub(counter, 1);
            }
        }
    }
}

// q = A p, pq = p.q
template <class T>
__global__ void k_cg_apply(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                           const int* __restrict__ orb_blk, const T* __restrict__ p,
                           T* __restrict__ q, CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.active[P.o]) return;
    const BlkDesc& B = blk[P.b];
    const T ih2 = (T)(1.0 / (B.h * B.h));
    double pq = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x, y, z;
        xyz_of(g, B.nx, B.ny, x, y, z);
        const T qv = apply_A<T>(p + P.base, g, x, y, z, B.nx, B.ny, B.nz, ih2);
        q[P.base + g] = qv;
        pq += (double)p[P.base + g] * (double)qv;
    }
    if (arrive(pq, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double s = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            st.count[P.o] = 0;
            st.pq[P.o] = s;
        }
    }
}

// x += alpha p, r -= alpha q, rr = r.r, beta = rr_new/rr_old; convergence
// when rr <= thr[o].  set_conv marks converged orbitals (FP64 solve);
// the inner float32 solve leaves that to the float64 residual.
template <class T>
__global__ void k_cg_update(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                            const int* __restrict__ orb_blk, T* __restrict__ x, T* __restrict__ r,
                            const T* __restrict__ p, const T* __restrict__ q, int max_iter,
                            int set_conv, CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.active[P.o]) return;
    const BlkDesc& B = blk[P.b];
    const double pqv = st.pq[P.o];
    const T alpha = (pqv > 0.0) ? (T)(st.rr[P.o] / pqv) : (T)0;
    double rr = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.base + P.g0 + k;
        x[g] += alpha * p[g];
        const T rv = r[g] - alpha * q[g];
        r[g] = rv;
        rr += (double)rv * (double)rv;
    }
    if (arrive(rr, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double s = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            const int o = P.o;
            st.count[o] = 0;
            const double old = st.rr[o];
            st.rr[o] = s;
            st.beta[o] = s / old;
            const int it = ++st.iters[o];
            if (!(s > st.thr[o])) {
                st.active[o] = 0;
                if (set_conv) st.conv[o] = 1;
                atomicSub(st.n_active, 1);
            } else if (it >= max_iter || !isfinite(s) || !(pqv > 0.0)) {
                st.active[o] = 0;
                atomicSub(st.n_active, 1);
            }
        }
    }
}

// p = r + beta p
template <class T>
__global__ void k_cg_pupdate(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                             const int* __restrict__ orb_blk, const T* __restrict__ r,
                             T* __restrict__ p, CgState st) {
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.active[P.o]) return;
    const T beta = (T)st.beta[P.o];
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.base + P.g0 + k;
        p[g] = r[g] + beta * p[g];
    }
}

// Start of an inner float32 solve of A d = r64 for orbitals still refining:
// r32 = p32 = float(r64), d32 = 0, rr = r32.r32; inner target
// thr = max(inner_tol^2 rr, (tol^2/4) bb).
__global__ void k_inner_init(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                             const int* __restrict__ orb_blk, const double* __restrict__ r64,
                             float* __restrict__ r32, float* __restrict__ p32, float* __restrict__ d32,
                             double inner_tol2, double tol2, CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.oactive[P.o]) return;
    const BlkDesc& B = blk[P.b];
    double rr = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.base + P.g0 + k;
        const float v = (float)r64[g];
        r32[g] = v;
        p32[g] = v;
        d32[g] = 0.0f;
        rr += (double)v * (double)v;
    }
    if (arrive(rr, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double s = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            const int o = P.o;
            st.count[o] = 0;
            st.rr[o] = s;
            const double a = inner_tol2 * s, c = 0.25 * tol2 * st.bb[o];
            st.thr[o] = a > c ? a : c;
            if (s > st.thr[o]) {
                st.active[o] = 1;
                atomicAdd(st.n_active, 1);
            } else {
                st.active[o] = 0;
            }
        }
    }
}

// x64 += d32 for orbitals still refining.
__global__ void k_correct(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                          const int* __restrict__ orb_blk, const float* __restrict__ d32,
                          double* __restrict__ x, CgState st) {
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.oactive[P.o]) return;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.base + P.g0 + k;
        x[g] += (double)d32[g];
    }
}

__global__ void k_cg_finish(int norb, CgState st, int* out_iters, int* out_conv, int* status) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= norb) return;
    if (out_iters) out_iters[o] = st.iters[o];
    if (out_conv) out_conv[o] = st.conv[o];
    if (!st.conv[o]) atomicOr(status + 1, 1);
}

static int read_count(flosic_ctx* c, const int* dptr, cudaStream_t s) {
    if (check_cuda(c, cudaMemcpyAsync(c->h_pinned, dptr, sizeof(int), cudaMemcpyDeviceToHost, s),
                   "cudaMemcpyAsync") != FLOSIC_OK)
        return -1;
    if (check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize") != FLOSIC_OK) return -1;
    prof_collect(c);
    return c->h_pinned[0];
}

// Solves A V = b for every orbital (b from launch_rhs, ||b||^2 in cg.bb).
// Returns a flosic status; iteration counts and convergence flags stay in the
// CG state (copied out by finish_poisson).
int run_poisson(flosic_ctx* c, const double* b, double* V, bool warm, cudaStream_t s) {
    Workspace& w = c->ws;
    CgState& st = w.cg;
    const unsigned nb = (unsigned)c->nchunk_total;
    const int T = kChunkThreads;
    const double tol2 = c->opt.cg_tol * c->opt.cg_tol;
    const int max_iter = c->opt.max_iter;
    const int check_every = 8;
    if (!warm && check_cuda(c, cudaMemsetAsync(V, 0, sizeof(double) * c->orb_elems, s), "memset V"))
        return FLOSIC_ERR_CUDA;
    k_cg_reset<<<(c->norb + 255) / 256, 256, 0, s>>>(c->norb, st); note_launch(c);
    if (c->opt.precision == FLOSIC_FP64) {
        k_residual64<<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, b, V, w.r64, w.p64, 1,
                                      tol2, max_iter, st.active, st.n_active, st); note_launch(c);
        for (int it = 0; it < max_iter; ++it) {
            if (it % check_every == 0) {
                const int na = read_count(c, st.n_active, s);
                if (na < 0) return FLOSIC_ERR_CUDA;
                if (na == 0) break;
            }
            prof_begin(c, s);
            k_cg_apply<double><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.p64, w.q64, st); note_launch(c);
            prof_end(c, s);
            k_cg_update<double><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, V, w.r64, w.p64,
                                                 w.q64, max_iter, 1, st); note_launch(c);
            k_cg_pupdate<double><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.r64, w.p64, st); note_launch(c);
        }
    } else {
        const double inner_tol2 = 1e-10;   // each float32 solve gains ~5 digits
        for (int outer = 0; outer < 40; ++outer) {
            k_residual64<<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, b, V, w.r64, nullptr,
                                          0, tol2, max_iter, st.oactive, st.n_oactive, st); note_launch(c);
            const int na = read_count(c, st.n_oactive, s);
            if (na < 0) return FLOSIC_ERR_CUDA;
            if (na == 0) break;
            if (check_cuda(c, cudaMemsetAsync(st.n_active, 0, sizeof(int), s), "memset"))
                return FLOSIC_ERR_CUDA;
            k_inner_init<<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.r64, w.r32, w.p32,
                                          w.d32, inner_tol2, tol2, st); note_launch(c);
            for (int it = 0; it < max_iter; ++it) {
                if (it % check_every == 0) {
                    const int ni = read_count(c, st.n_active, s);
                    if (ni < 0) return FLOSIC_ERR_CUDA;
                    if (ni == 0) break;
                }
                prof_begin(c, s);
                k_cg_apply<float><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.p32, w.q32, st); note_launch(c);
                prof_end(c, s);
                k_cg_update<float><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.d32, w.r32,
                                                    w.p32, w.q32, max_iter, 0, st); note_launch(c);
                k_cg_pupdate<float><<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.r32, w.p32, st); note_launch(c);
            }
            k_correct<<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, w.d32, V, st); note_launch(c);
        }
    }
    return check_cuda(c, cudaGetLastError(), "poisson kernels");
}

void finish_poisson(flosic_ctx* c, int* iters, int* conv, cudaStream_t s) {
    k_cg_finish<<<(c->norb + 255) / 256, 256, 0, s>>>(c->norb, c->ws.cg, iters, conv, c->ws.status); note_launch(c);
}

// ---------------------------------------------------------------------------
// exact Poisson adjoint: transpose of the boundary map
// ---------------------------------------------------------------------------
// Coefficients c_m = sum_g W_g (1/h^2) sum_{ghost taps} w_m dV_b/dmom_m(R_tap).
__global__ void k_bcadj_coef(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                             const int* __restrict__ orb_blk, const double* __restrict__ W,
                             double* __restrict__ part) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    const BlkDesc& B = blk[P.b];
    const double ih2 = 1.0 / (B.h * B.h);
    double cf[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) cf[q] = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x, y, z;
        xyz_of(g, B.nx, B.ny, x, y, z);
        const int p[3] = {x, y, z};
        const int n[3] = {B.nx, B.ny, B.nz};
        bool near = false;
        for (int d = 0; d < 3; ++d) near |= (p[d] < kHalf || p[d] >= n[d] - kHalf);
        if (!near) continue;
        const double wg = W[P.base + g] * ih2;
        for (int d = 0; d < 3; ++d) {
            for (int m = 1; m <= kHalf; ++m) {
                for (int sg = -1; sg <= 1; sg += 2) {
                    const int qd = p[d] + sg * m;
                    if (qd >= 0 && qd < n[d]) continue;
                    int q[3] = {x, y, z};
                    q[d] = qd;
                    const double Rx = B.ox + B.h * q[0] - B.cx;
                    const double Ry = B.oy + B.h * q[1] - B.cy;
                    const double Rz = B.oz + B.h * q[2] - B.cz;
                    const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
                    const double ir = rsqrt(r2), ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
                    const double f = wg * c_w[m];
                    cf[0] += f * ir;
                    cf[1] += f * Rx * ir3;
                    cf[2] += f * Ry * ir3;
                    cf[3] += f * Rz * ir3;
                    cf[4] += f * 0.5 * Rx * Rx * ir5;
                    cf[5] += f * 0.5 * Ry * Ry * ir5;
                    cf[6] += f * 0.5 * Rz * Rz * ir5;
                    cf[7] += f * Rx * Ry * ir5;
                    cf[8] += f * Rx * Rz * ir5;
                    cf[9] += f * Ry * Rz * ir5;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const double s = block_sum(cf[q], scratch);
        if (threadIdx.x == 0) part[t * 10 + q] = s;
    }
}

// veff = (V + G^T rho)/2 with G^T rho = 4 pi W + dV sum_m c_m basis_m(R).
__global__ void k_veff(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                       const int* __restrict__ orb_blk, const double* __restrict__ W,
                       const double* __restrict__ V, const double* __restrict__ coef,
                       double* __restrict__ veff) {
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    const BlkDesc& B = blk[P.b];
    double c[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) c[q] = coef[P.o * 10 + q];
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x, y, z;
        xyz_of(g, B.nx, B.ny, x, y, z);
        const double Rx = B.ox + B.h * x - B.cx, Ry = B.oy + B.h * y - B.cy, Rz = B.oz + B.h * z - B.cz;
        const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
        const double kt = c[0] + c[1] * Rx + c[2] * Ry + c[3] * Rz + c[4] * (3 * Rx * Rx - r2) +
                          c[5] * (3 * Ry * Ry - r2) + c[6] * (3 * Rz * Rz - r2) + c[7] * 3 * Rx * Ry +
                          c[8] * 3 * Rx * Rz + c[9] * 3 * Ry * Rz;
        const long long gi = P.base + g;
        veff[gi] = 0.5 * (V[gi] + 4.0 * kPi * W[gi] + B.dV * kt);
    }
}

void launch_bc_adjoint(const flosic_ctx* c, const double* W, const double* V, double* veff,
                       cudaStream_t s) {
    k_bcadj_coef<<<(unsigned)c->nchunk_total, kChunkThreads, 0, s>>>(c->d_blk, c->d_chunk_orb,
                                                                     c->d_orb_blk, W, c->ws.mom_part); note_launch(c);
    k_sum_chunks10<<<(c->norb * 32 + 255) / 256, 256, 0, s>>>(c->d_blk, c->d_orb_blk, c->norb,
                                                              c->ws.mom_part, c->ws.mom, 0); note_launch(c);
    k_veff<<<(unsigned)c->nchunk_total, kChunkThreads, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk,
                                                               W, V, c->ws.mom, veff); note_launch(c);
}

}  // namespace flosic
