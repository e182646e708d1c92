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

template <class T> __device__ __forceinline__ T c_wf_or_w(int m);
template <> __device__ __forceinline__ float c_wf_or_w<float>(int m) { return c_wf[m]; }
template <> __device__ __forceinline__ double c_wf_or_w<double>(int m) { return c_w[m]; }

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

cudaError_t upload_stencil12_constants();

cudaError_t upload_stencil_constants() {
    {
        cudaError_t e = upload_stencil12_constants();
        if (e == cudaSuccess) e = upload_hamiltonian_constants();
        if (e != cudaSuccess) return e;
    }
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
// conjugate gradients, batched over orbitals (one CTA per chunk of points)
// ---------------------------------------------------------------------------
// Masked orbitals (mask 0) take no part: inactive from the start, reported
// converged after 0 iterations; nact = the number of unmasked orbitals.
__global__ void k_cg_reset(int norb, int nact, CgState st) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o == 0) {
        *st.n_active = nact;
        *st.n_oactive = nact;
    }
    if (o >= norb) return;
    const int on = st.mask[o] != 0;
    st.active[o] = on;
    st.oactive[o] = on;
    st.iters[o] = 0;
    st.conv[o] = 1 - on;
    st.count[o] = 0;
    st.rz[o] = 0.0;
    st.beta[o] = 0.0;
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

// Preconditioned CG, fused: p = z + beta p_old (p = z on the first
// iteration, beta = 0), q = A p, pq = p.q.  The taps read z and p_old.
template <class T>
__global__ void k_pcg_apply(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                            const int* __restrict__ orb_blk, const T* __restrict__ z,
                            const T* __restrict__ pold, T* __restrict__ pnew, T* __restrict__ q, CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.active[P.o]) return;
    const BlkDesc& B = blk[P.b];
    const double bd = st.beta[P.o];
    const bool first = (bd == 0.0);
    const T beta = (T)bd;
    const T ih2 = (T)(1.0 / (B.h * B.h));
    const T* zb = z + P.base;
    const T* pb = pold + P.base;
    const long long sy = B.nx, sz = (long long)B.nx * B.ny;
    double pq = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.g0 + k;
        int x, y, zz;
        xyz_of(g, B.nx, B.ny, x, y, zz);
        auto pv = [&](long long h) -> T { return first ? zb[h] : zb[h] + beta * pb[h]; };
        const T pc = pv(g);
        T acc = T(3) * c_wf_or_w<T>(0) * pc;
#pragma unroll
        for (int m = 1; m <= kHalf; ++m) {
            T sm = 0;
            if (x - m >= 0) sm += pv(g - m);
            if (x + m < B.nx) sm += pv(g + m);
            if (y - m >= 0) sm += pv(g - m * sy);
            if (y + m < B.ny) sm += pv(g + m * sy);
            if (zz - m >= 0) sm += pv(g - m * sz);
            if (zz + m < B.nz) sm += pv(g + m * sz);
            acc += (T)c_wf_or_w<T>(m) * sm;
        }
        const T qv = -acc * ih2;
        pnew[P.base + g] = pc;
        q[P.base + g] = qv;
        pq += (double)pc * (double)qv;
    }
    if (arrive(pq, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double sum = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            st.count[P.o] = 0;
            st.pq[P.o] = sum;
        }
    }
}

// x += alpha p, r -= alpha q with alpha = rz/pq; rr = r.r decides convergence.
template <class T>
__global__ void k_pcg_update(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                             const int* __restrict__ orb_blk, T* __restrict__ x, T* __restrict__ r,
                             const T* __restrict__ p, const T* __restrict__ q, int max_iter, int set_conv,
                             CgState st) {
    __shared__ double scratch[32];
    const long long t = blockIdx.x;
    const ChunkPos P = decode_chunk(blk, chunk_orb, orb_blk, t);
    if (!st.active[P.o]) return;
    const BlkDesc& B = blk[P.b];
    const double pqv = st.pq[P.o];
    const T alpha = (pqv > 0.0) ? (T)(st.rz[P.o] / pqv) : (T)0;
    double rr = 0.0;
    for (int k = threadIdx.x; k < P.npts; k += blockDim.x) {
        const long long g = P.base + P.g0 + k;
        x[g] += alpha * p[g];
        const T rv = r[g] - alpha * q[g];
        r[g] = rv;
        rr += (double)rv * (double)rv;
    }
    if (arrive(rr, st.part, t, st.count + P.o, B.nchunk, scratch)) {
        const double sum = gather_sum(st.part, P.first, B.nchunk, scratch);
        if (threadIdx.x == 0) {
            const int o = P.o;
            st.count[o] = 0;
            st.rr[o] = sum;
            const int it = ++st.iters[o];
            if (!(sum > st.thr[o])) {
                st.active[o] = 0;
                if (set_conv) st.conv[o] = 1;
                atomicSub(st.n_active, 1);
            } else if (it >= max_iter || !isfinite(sum) || !(pqv > 0.0)) {
                st.active[o] = 0;
                atomicSub(st.n_active, 1);
            }
        }
    }
}

// x += alpha p, r -= alpha q with alpha = rz/pq; rr = r.r decides
// convergence (tile version, vectorised).
template <class T>
__global__ void __launch_bounds__(256) k_pcg_update_t(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                      const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                      T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                      const T* __restrict__ q, int max_iter, int set_conv, CgState st) {
    using VT = typename Vec<T>::type;
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const double pqv = st.pq[P.o];
    const T alpha = (pqv > 0.0) ? (T)(st.rz[P.o] / pqv) : (T)0;
    T rr = T(0);   // per-thread partial in the working precision; tile sums in float64
    tile_elementwise<T>(D, P, [&](long long g, int n) {
        if (n > 1) {
            VT xv = *reinterpret_cast<VT*>(x + g);
            VT rv = *reinterpret_cast<VT*>(r + g);
            const VT pv = *reinterpret_cast<const VT*>(p + g);
            const VT qv = *reinterpret_cast<const VT*>(q + g);
            T* xs = reinterpret_cast<T*>(&xv);
            T* rs = reinterpret_cast<T*>(&rv);
            const T* ps = reinterpret_cast<const T*>(&pv);
            const T* qs = reinterpret_cast<const T*>(&qv);
#pragma unroll
            for (int k = 0; k < Vec<T>::n; ++k) {
                xs[k] += alpha * ps[k];
                rs[k] -= alpha * qs[k];
                rr += rs[k] * rs[k];
            }
            *reinterpret_cast<VT*>(x + g) = xv;
            *reinterpret_cast<VT*>(r + g) = rv;
        } else {
            x[g] += alpha * p[g];
            const T rv = r[g] - alpha * q[g];
            r[g] = rv;
            rr += rv * rv;
        }
    });
    if (tile_arrive(rr, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            const int o = P.o;
            st.count[o] = 0;
            st.rr[o] = sum;
            const int it = ++st.iters[o];
            if (!(sum > st.thr[o])) {
                st.active[o] = 0;
                if (set_conv) st.conv[o] = 1;
                atomicSub(st.n_active, 1);
            } else if (it >= max_iter || !isfinite(sum) || !(pqv > 0.0)) {
                st.active[o] = 0;
                atomicSub(st.n_active, 1);
            }
        }
    }
}

// Residual of a zero start vector: r = b, rr = bb = b.b; same stopping
// logic as the stencil residual kernel.
__global__ void __launch_bounds__(256) k_residual_zero(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                       const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                       const double* __restrict__ b, double* __restrict__ r,
                                                       double tol2, int* __restrict__ flag, int* __restrict__ counter,
                                                       CgState st) {
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!flag[P.o]) return;
    const LvlDesc& D = L[P.b];
    double bb = 0.0;
    tile_elementwise<double>(D, P, [&](long long g, int n) {
        for (int k = 0; k < n; ++k) {
            const double v = b[g + k];
            r[g + k] = v;
            bb += v * v;
        }
    });
    if (tile_arrive(bb, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            const int o = P.o;
            st.count[o] = 0;
            st.rr[o] = sum;
            st.bb[o] = sum;
            st.thr[o] = tol2 * sum;
            if (!(sum > st.thr[o])) {
                flag[o] = 0;
                st.conv[o] = 1;
                atomicSub(counter, 1);
            }
        }
    }
}

// V = 0 on every orbital the mask leaves out (one CTA per chunk of points).
__global__ void k_zero_masked(const BlkDesc* __restrict__ blk, const int* __restrict__ chunk_orb,
                              const int* __restrict__ orb_blk, const int* __restrict__ mask, double* __restrict__ V) {
    const int o = chunk_orb[blockIdx.x];
    if (mask[o]) return;
    const BlkDesc& B = blk[orb_blk[o]];
    const long long c = (long long)blockIdx.x - (B.chunk0 + (long long)(o - B.orb0) * B.nchunk);
    const long long base = B.off + (long long)(o - B.orb0) * B.G;
    for (int k = threadIdx.x; k < kChunk; k += blockDim.x) {
        const long long g = c * kChunk + k;
        if (g < B.G) V[base + g] = 0.0;
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
    if (check_cuda(c, fetch_words(c, dptr, 1, s), "count read") != FLOSIC_OK) return -1;
    if (check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize") != FLOSIC_OK) return -1;
    prof_collect(c);
    return reinterpret_cast<volatile int*>(c->h_pinned)[0];
}

static void launch_residual_zero(flosic_ctx* c, const double* b, double* r, double tol2, int* flag, int* counter,
                                 cudaStream_t s) {
    k_residual_zero<<<(unsigned)c->mg.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
        c->d_blk, c->mg.d_lvl[0], c->mg.d_tiles[0], c->d_orb_blk, b, r, tol2, flag, counter, c->ws.cg); note_launch(c);
}

template <class T>
static MgPtrs<T> mg_ptrs(const flosic_ctx* c, T* r, T* z, T* q) {
    MgPtrs<T> mp{};
    for (int l = 0; l < kMaxLevels; ++l) {
        mp.r[l] = (T*)c->mg.r[l];
        mp.e[l] = (T*)c->mg.e[l];
        mp.t[l] = (T*)c->mg.t[l];
        mp.lvl[l] = c->mg.d_lvl[l];
    }
    mp.r[0] = r;
    mp.e[0] = z;
    mp.t[0] = q;
    mp.coarsest_level = c->mg.d_coarsest_level;
    return mp;
}

// Multigrid-preconditioned CG on A x = r0 for the active orbitals (r holds
// the starting residual, rr/thr/active/n_active are set, rz = beta = 0).
// The direction image uses the recurrence q = A z + beta q, so the stencil
// reads one array (z); tbuf is the level-0 scratch of the V-cycle.
template <class T>
static int pcg_mg(flosic_ctx* c, T* x, T* r, T* z, T* p, T* tbuf, T* q, int set_conv, cudaStream_t s) {
    CgState& st = c->ws.cg;
    const int max_iter = c->opt.max_iter;
    const MgPtrs<T> mp = mg_ptrs<T>(c, r, z, tbuf);
    for (int it = 0; it < max_iter; ++it) {
        if (it % 4 == 0) {
            const int na = read_count(c, st.n_active, s);
            if (na < 0) return FLOSIC_ERR_CUDA;
            if (na == 0) break;
        }
        launch_vcycle<T>(c, mp, st.active, s);
        launch_apply12_pcg<T>(c, z, p, q, s);
        k_pcg_update_t<T><<<(unsigned)c->mg.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
            c->d_blk, c->mg.d_lvl[0], c->mg.d_tiles[0], c->d_orb_blk, x, r, p, q, max_iter, set_conv, st); note_launch(c);
    }
    return FLOSIC_OK;
}

// The multigrid preconditioner of the AAR steps: f = M r.
static void aar_vcycle(flosic_ctx* c, float* r, float* f, cudaStream_t s) {
    launch_vcycle<float>(c, mg_ptrs<float>(c, r, f, c->ws.p32b), c->ws.cg.active, s);
}

// Float32 AAR on A d = r32 for the active orbitals (d32 = 0, r32 = the
// starting residual, thr/active/n_active set by the refinement round).
static int aar_inner(flosic_ctx* c, cudaStream_t s) {
    Workspace& w = c->ws;
    const int p = c->opt.aar_p;
    for (int k = 0; k < c->opt.max_iter; ++k) {
        if (k % 4 == 0) {
            const int na = read_count(c, w.cg.n_active, s);
            if (na < 0) return FLOSIC_ERR_CUDA;
            if (na == 0) break;
        }
        launch_aar_step<float>(c, w.d32, w.r32, w.z32, k, k >= 1 && (k + 1) % p == 0, s, aar_vcycle);
    }
    return FLOSIC_OK;
}

// Solves A V = b for every orbital (b from launch_rhs, ||b||^2 in cg.bb).
// Returns a flosic status; iteration counts and convergence flags stay in the
// CG state (copied out by finish_poisson).
int run_poisson(flosic_ctx* c, double* b, double* V, bool warm, cudaStream_t s) {
    Workspace& w = c->ws;
    CgState& st = w.cg;
    const unsigned nb = (unsigned)c->nchunk_total;
    const int T = kChunkThreads;
    const double tol2 = c->opt.cg_tol * c->opt.cg_tol;
    const int max_iter = c->opt.max_iter;
    const int check_every = 8;
    const bool mg = c->mg.enabled;
    if (!warm && c->opt.precision == FLOSIC_FP64 &&
        check_cuda(c, cudaMemsetAsync(V, 0, sizeof(double) * c->orb_elems, s), "memset V"))
        return FLOSIC_ERR_CUDA;
    k_cg_reset<<<(c->norb + 255) / 256, 256, 0, s>>>(c->norb, c->n_unmasked, st); note_launch(c);
    if (c->opt.precision == FLOSIC_FP64) {
        if (warm)
            launch_residual12(c, b, V, w.r64, tol2, max_iter, st.active, st.n_active, 1, s);
        else
            launch_residual_zero(c, b, w.r64, tol2, st.active, st.n_active, s);
        if (!mg && check_cuda(c, cudaMemcpyAsync(w.p64, w.r64, sizeof(double) * c->orb_elems,
                                                 cudaMemcpyDeviceToDevice, s), "copy p"))
            return FLOSIC_ERR_CUDA;
        if (mg) {
            int rc = pcg_mg<double>(c, V, w.r64, w.z64, w.p64, w.p64b, w.q64, 1, s);
            if (rc) return rc;
        } else {
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
        }
    } else {
        // float32 inner solves inside a float-float refinement (refine.cu);
        // b becomes its pairs, the idle float64 residual buffer holds x
        const double inner_tol2 = 1e-12;   // each float32 solve gains ~6 digits
        float2* x = reinterpret_cast<float2*>(w.r64);
        float* p32 = (mg || c->opt.solver != FLOSIC_SOLVER_PCG) ? nullptr : w.p32;
        if (check_cuda(c, cudaMemsetAsync(st.n_active, 0, sizeof(int), s), "memset")) return FLOSIC_ERR_CUDA;
        // with the Kronecker solve (which overwrites d), each round ends with one
        // sweep: x += d and the residual updated from d, r -= A d (b holds r);
        // a cold start then stores neither x = 0 nor d = 0
        const bool fused = c->opt.solver == FLOSIC_SOLVER_KRON;
        launch_ff_init(c, b, V, warm, fused && !warm, x, p32, tol2, inner_tol2, s);
        for (int round = 0; round < 40; ++round) {
            if ((round > 0 && !fused) || (round == 0 && warm)) {
                if (check_cuda(c, cudaMemsetAsync(st.n_active, 0, sizeof(int), s), "memset"))
                    return FLOSIC_ERR_CUDA;
                launch_residual_ff(c, b, x, p32, tol2, inner_tol2, fused, s);
            }
            const int na = read_count(c, st.n_oactive, s);
            if (na < 0) return FLOSIC_ERR_CUDA;
            if (na == 0) break;
            if (c->opt.solver == FLOSIC_SOLVER_KRON) {
                launch_kron_solve(c, w.r32, w.d32, w.p32, w.q32, s);
            } else if (c->opt.solver == FLOSIC_SOLVER_AAR) {
                int rc = aar_inner(c, s);
                if (rc) return rc;
            } else if (mg) {
                int rc = pcg_mg<float>(c, w.d32, w.r32, w.z32, w.p32, w.p32b, w.q32, 0, s);
                if (rc) return rc;
            } else {
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
            }
            if (fused) {
                if (check_cuda(c, cudaMemsetAsync(st.n_active, 0, sizeof(int), s), "memset"))
                    return FLOSIC_ERR_CUDA;
                launch_update_ff(c, b, x, round == 0 && !warm, tol2, inner_tol2, s);
            } else {
                launch_correct_ff(c, x, s);
            }
        }
        launch_join_ff(c, x, V, s);
    }
    if (c->n_unmasked < c->norb) {
        k_zero_masked<<<nb, T, 0, s>>>(c->d_blk, c->d_chunk_orb, c->d_orb_blk, st.mask, V);
        note_launch(c);
    }
    return check_cuda(c, cudaGetLastError(), "poisson kernels");
}

void finish_poisson(flosic_ctx* c, int* iters, int* conv, cudaStream_t s) {
    k_cg_finish<<<(c->norb + 255) / 256, 256, 0, s>>>(c->norb, c->ws.cg, iters, conv, c->ws.status); note_launch(c);
}

}  // namespace flosic
