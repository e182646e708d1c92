// Allocation-free variant of the per-orbital Poisson solve.
//
// Some callers cannot allocate device memory while they run: code that lives
// inside another framework's memory arena or under a hard memory cap, and
// latency-critical loops that must not take cudaMalloc/cudaFree (which can
// synchronise the whole device and can fail when memory is tight).  For them
// flosic_orbital_poisson_noalloc solves the same problem as
// flosic_orbital_poisson (one grid, float64 conjugate gradients, no
// preconditioner) using only the caller's input/output arrays and one
// statically sized scratch array in device memory, declared below.
//
// The scratch array belongs to every GPU that loads this library and stays
// allocated until the process exits.  Every call shares it, so calls whose
// work overlaps on a GPU (two host threads, or two streams) race on it and
// must be serialised by the caller.  The array keeps whatever the last call
// left; each call initialises every word it reads before reading it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace flosic {
namespace {

constexpr long long kNaMaxElems = 1LL << 20;   // orbitals x grid points per call
constexpr int kNaMaxOrb = kMaxN;               // orbitals per call
constexpr int kNaChunk = 1024;                 // points per CTA
constexpr long long kNaMaxChunks = kNaMaxElems / kNaChunk + kNaMaxOrb;
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// scratch layout (doubles): b, r, p, q [kNaMaxElems] each, then per chunk
// partial sums (pq, rr, bb: 1 each; moments: 10), then per orbital scalars.
constexpr long long kNaOffB = 0;
constexpr long long kNaOffR = kNaOffB + kNaMaxElems;
constexpr long long kNaOffP = kNaOffR + kNaMaxElems;
constexpr long long kNaOffQ = kNaOffP + kNaMaxElems;
constexpr long long kNaOffPart = kNaOffQ + kNaMaxElems;               // 3 x chunks
constexpr long long kNaOffMomPart = kNaOffPart + 3 * kNaMaxChunks;   // 10 x chunks
constexpr long long kNaOffOrb = kNaOffMomPart + 10 * kNaMaxChunks;   // per-orbital block
constexpr int kNaOrbDoubles = 8;   // rr, alpha, beta, bb, and 4 int slots packed below
constexpr long long kNaScratchDoubles = kNaOffOrb + (long long)kNaOrbDoubles * kNaMaxOrb + 64;

// about 32 MiB of device memory on every GPU that loads the library
static __device__ __align__(256) double g_na_scratch[kNaScratchDoubles];

__constant__ double c_na_w[kHalf + 1];

struct NaGrid {
    int nx, ny, nz, norb, nchunk;
    long long G;
    double h, ih2, dV, ox, oy, oz, cx, cy, cz;
};

struct NaOrb {            // per-orbital scalars inside the scratch array
    double *rr, *alpha, *beta, *bb;
    int *active, *iters, *conv, *n_active;
};

__device__ __forceinline__ NaOrb na_orb(double* base) {
    NaOrb o;
    o.rr = base;
    o.alpha = base + kNaMaxOrb;
    o.beta = base + 2 * kNaMaxOrb;
    o.bb = base + 3 * kNaMaxOrb;
    int* ib = (int*)(base + 4 * kNaMaxOrb);
    o.active = ib;
    o.iters = ib + kNaMaxOrb;
    o.conv = ib + 2 * kNaMaxOrb;
    o.n_active = ib + 3 * kNaMaxOrb;
    return o;
}

__device__ __forceinline__ void na_xyz(const NaGrid& g, long long i, int& x, int& y, int& z) {
    const long long pl = (long long)g.nx * g.ny;
    z = (int)(i / pl);
    const long long r = i - (long long)z * pl;
    y = (int)(r / g.nx);
    x = (int)(r - (long long)y * g.nx);
}

__device__ __forceinline__ double na_apply(const NaGrid& g, const double* u, long long i, int x, int y, int z) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    double acc = 3.0 * c_na_w[0] * u[i];
    for (int m = 1; m <= kHalf; ++m) {
        double s = 0.0;
        if (x - m >= 0) s += u[i - m];
        if (x + m < g.nx) s += u[i + m];
        if (y - m >= 0) s += u[i - m * sy];
        if (y + m < g.ny) s += u[i + m * sy];
        if (z - m >= 0) s += u[i - m * sz];
        if (z + m < g.nz) s += u[i + m * sz];
        acc += c_na_w[m] * s;
    }
    return -acc * g.ih2;
}

__device__ __forceinline__ double na_multipole(const double* m, double Rx, double Ry, double Rz) {
    const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const double ir = rsqrt(r2), ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
    const double quad = m[4] * Rx * Rx + m[5] * Ry * Ry + m[6] * Rz * Rz +
                        2.0 * (m[7] * Rx * Ry + m[8] * Rx * Rz + m[9] * Ry * Rz);
    return m[0] * ir + (m[1] * Rx + m[2] * Ry + m[3] * Rz) * ir3 + 0.5 * quad * ir5;
}

// moments of phi^2 per (chunk, orbital)
__global__ void k_na_moments(NaGrid g, const double* __restrict__ phi, double* __restrict__ mom_part) {
    __shared__ double scratch[32];
    const int c = blockIdx.x, o = blockIdx.y;
    double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < kNaChunk; k += blockDim.x) {
        const long long i = (long long)c * kNaChunk + k;
        if (i >= g.G) break;
        int x, y, z;
        na_xyz(g, i, x, y, z);
        const double v = phi[o * g.G + i], rho = v * v;
        const double Rx = g.ox + g.h * x - g.cx, Ry = g.oy + g.h * y - g.cy, Rz = g.oz + g.h * z - g.cz;
        const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
        m[0] += rho; m[1] += rho * Rx; m[2] += rho * Ry; m[3] += rho * Rz;
        m[4] += rho * (3 * Rx * Rx - r2); m[5] += rho * (3 * Ry * Ry - r2); m[6] += rho * (3 * Rz * Rz - r2);
        m[7] += rho * 3 * Rx * Ry; m[8] += rho * 3 * Rx * Rz; m[9] += rho * 3 * Ry * Rz;
    }
    for (int q = 0; q < 10; ++q) {
        const double s = block_sum(m[q], scratch);
        if (threadIdx.x == 0) mom_part[((long long)o * g.nchunk + c) * 10 + q] = s;
    }
}

// b = 4 pi phi^2 + boundary terms; r = p = b; x = 0; per-chunk ||b||^2
__global__ void k_na_rhs(NaGrid g, const double* __restrict__ phi, const double* __restrict__ mom_part,
                         double* __restrict__ b, double* __restrict__ r, double* __restrict__ p,
                         double* __restrict__ x, double* __restrict__ bb_part) {
    __shared__ double scratch[32];
    __shared__ double mom[10];
    const int c = blockIdx.x, o = blockIdx.y;
    if (threadIdx.x < 10) {
        double s = 0.0;
        for (int k = 0; k < g.nchunk; ++k) s += mom_part[((long long)o * g.nchunk + k) * 10 + threadIdx.x];
        mom[threadIdx.x] = s * g.dV;
    }
    __syncthreads();
    double bb = 0.0;
    for (int k = threadIdx.x; k < kNaChunk; k += blockDim.x) {
        const long long i = (long long)c * kNaChunk + k;
        if (i >= g.G) break;
        int xi, yi, zi;
        na_xyz(g, i, xi, yi, zi);
        const int pp[3] = {xi, yi, zi}, n[3] = {g.nx, g.ny, g.nz};
        const double v = phi[o * g.G + i];
        double acc = 0.0;
        for (int d = 0; d < 3; ++d)
            for (int m = 1; m <= kHalf; ++m)
                for (int sg = -1; sg <= 1; sg += 2) {
                    const int qd = pp[d] + sg * m;
                    if (qd >= 0 && qd < n[d]) continue;
                    int q[3] = {xi, yi, zi};
                    q[d] = qd;
                    acc += c_na_w[m] * na_multipole(mom, g.ox + g.h * q[0] - g.cx, g.oy + g.h * q[1] - g.cy,
                                                    g.oz + g.h * q[2] - g.cz);
                }
        const double bv = 4.0 * kPi * v * v + acc * g.ih2;
        const long long j = o * g.G + i;
        b[j] = bv;
        r[j] = bv;
        p[j] = bv;
        x[j] = 0.0;
        bb += bv * bv;
    }
    const double s = block_sum(bb, scratch);
    if (threadIdx.x == 0) bb_part[(long long)o * g.nchunk + c] = s;
}

// one CTA per orbital: sum of its chunk partials, fixed order
__device__ __forceinline__ double na_sum(const NaGrid& g, const double* part, int o, double* scratch) {
    double v = 0.0;
    for (int k = threadIdx.x; k < g.nchunk; k += blockDim.x) v += part[(long long)o * g.nchunk + k];
    return block_sum(v, scratch);
}

__global__ void k_na_init(NaGrid g, const double* __restrict__ bb_part, double* orbbase, int max_iter) {
    __shared__ double scratch[32];
    const int o = blockIdx.x;
    NaOrb S = na_orb(orbbase);
    const double bb = na_sum(g, bb_part, o, scratch);
    if (threadIdx.x == 0) {
        S.bb[o] = bb;
        S.rr[o] = bb;
        S.iters[o] = 0;
        S.conv[o] = (bb == 0.0) ? 1 : 0;
        S.active[o] = (bb > 0.0 && max_iter > 0) ? 1 : 0;
    }
}

__global__ void k_na_apply(NaGrid g, const double* __restrict__ p, double* __restrict__ q,
                           double* __restrict__ pq_part, const double* orbbase) {
    __shared__ double scratch[32];
    const int c = blockIdx.x, o = blockIdx.y;
    NaOrb S = na_orb((double*)orbbase);
    if (!S.active[o]) return;
    double pq = 0.0;
    for (int k = threadIdx.x; k < kNaChunk; k += blockDim.x) {
        const long long i = (long long)c * kNaChunk + k;
        if (i >= g.G) break;
        int x, y, z;
        na_xyz(g, i, x, y, z);
        const double qv = na_apply(g, p + o * g.G, i, x, y, z);
        q[o * g.G + i] = qv;
        pq += p[o * g.G + i] * qv;
    }
    const double s = block_sum(pq, scratch);
    if (threadIdx.x == 0) pq_part[(long long)o * g.nchunk + c] = s;
}

__global__ void k_na_alpha(NaGrid g, const double* __restrict__ pq_part, double* orbbase) {
    __shared__ double scratch[32];
    const int o = blockIdx.x;
    NaOrb S = na_orb(orbbase);
    if (!S.active[o]) return;
    const double pq = na_sum(g, pq_part, o, scratch);
    if (threadIdx.x == 0) {
        if (pq > 0.0) {
            S.alpha[o] = S.rr[o] / pq;
        } else {
            S.alpha[o] = 0.0;
            S.active[o] = 0;   // breakdown: stop (not converged)
        }
    }
}

__global__ void k_na_update(NaGrid g, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ rr_part, const double* orbbase) {
    __shared__ double scratch[32];
    const int c = blockIdx.x, o = blockIdx.y;
    NaOrb S = na_orb((double*)orbbase);
    if (!S.active[o]) return;
    const double a = S.alpha[o];
    double rr = 0.0;
    for (int k = threadIdx.x; k < kNaChunk; k += blockDim.x) {
        const long long i = (long long)c * kNaChunk + k;
        if (i >= g.G) break;
        const long long j = o * g.G + i;
        x[j] += a * p[j];
        const double rv = r[j] - a * q[j];
        r[j] = rv;
        rr += rv * rv;
    }
    const double s = block_sum(rr, scratch);
    if (threadIdx.x == 0) rr_part[(long long)o * g.nchunk + c] = s;
}

__global__ void k_na_beta(NaGrid g, const double* __restrict__ rr_part, double* orbbase, double tol2,
                          int max_iter) {
    __shared__ double scratch[32];
    const int o = blockIdx.x;
    NaOrb S = na_orb(orbbase);
    if (!S.active[o]) return;
    const double rr = na_sum(g, rr_part, o, scratch);
    if (threadIdx.x == 0) {
        S.beta[o] = rr / S.rr[o];
        S.rr[o] = rr;
        const int it = ++S.iters[o];
        if (!(rr > tol2 * S.bb[o])) {
            S.active[o] = 0;
            S.conv[o] = 1;
        } else if (it >= max_iter || !isfinite(rr)) {
            S.active[o] = 0;
        }
    }
}

__global__ void k_na_pupdate(NaGrid g, const double* __restrict__ r, double* __restrict__ p,
                             const double* orbbase) {
    const int c = blockIdx.x, o = blockIdx.y;
    NaOrb S = na_orb((double*)orbbase);
    if (!S.active[o]) return;
    const double be = S.beta[o];
    for (int k = threadIdx.x; k < kNaChunk; k += blockDim.x) {
        const long long i = (long long)c * kNaChunk + k;
        if (i >= g.G) break;
        const long long j = o * g.G + i;
        p[j] = r[j] + be * p[j];
    }
}

__global__ void k_na_count(int norb, double* orbbase) {
    NaOrb S = na_orb(orbbase);
    if (threadIdx.x == 0) {
        int n = 0;
        for (int o = 0; o < norb; ++o) n += S.active[o];
        *S.n_active = n;
    }
}

__global__ void k_na_finish(int norb, const double* orbbase, int* iters, int* conv) {
    NaOrb S = na_orb((double*)orbbase);
    const int o = threadIdx.x + blockIdx.x * blockDim.x;
    if (o >= norb) return;
    if (iters) iters[o] = S.iters[o];
    if (conv) conv[o] = S.conv[o];
}

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {nullptr};

// Message of the last failure on this host thread: a fixed buffer per
// thread, so that no call allocates and calls from different host threads
// (each driving its own GPU) never write the same buffer.
thread_local char g_na_error[256] = "";

void na_fail(const char* what, const char* detail) {
    snprintf(g_na_error, sizeof g_na_error, "%s%s%s", what, detail ? ": " : "", detail ? detail : "");
}

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the stencil
// weights in this file's constant bank.  The result is kept for the life of
// the process, so it is not redone if the device's primary context is torn
// down (cudaDeviceReset) after the first call; that is not supported.
int na_setup(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { na_fail("cudaGetDevice", cudaGetErrorString(e)); return FLOSIC_ERR_CUDA; }
    if (dev < 0 || dev >= kNaMaxDevices) { na_fail("device ordinal out of range", nullptr); return FLOSIC_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_na_scratch);
        if (e != cudaSuccess) { na_fail("cudaGetSymbolAddress", cudaGetErrorString(e)); return FLOSIC_ERR_CUDA; }
        double w[kHalf + 1];
        stencil_weights(w);
        e = cudaMemcpyToSymbol(c_na_w, w, sizeof(w));
        if (e != cudaSuccess) { na_fail("cudaMemcpyToSymbol", cudaGetErrorString(e)); return FLOSIC_ERR_CUDA; }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return FLOSIC_OK;
}

}  // namespace
}  // namespace flosic

using namespace flosic;

extern "C" const char* flosic_noalloc_last_error(void) { return g_na_error; }

extern "C" int flosic_orbital_poisson_noalloc(int nx, int ny, int nz, double h, const double* origin, int norb,
                                              const double* phi, double* V, double cg_tol, int max_iter,
                                              int* iters, int* conv_flags, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !origin || norb < 1 || !phi || !V || !(cg_tol > 0.0) ||
        max_iter < 1) {
        na_fail("bad argument", nullptr);
        return FLOSIC_ERR_ARG;
    }
    const long long G = (long long)nx * ny * nz;
    if (norb > kNaMaxOrb || G * norb > kNaMaxElems) {
        na_fail("problem too large for the static scratch: need norb <= 128 and norb*nx*ny*nz <= 1048576", nullptr);
        return FLOSIC_ERR_ARG;
    }
    double* base = nullptr;
    int rc = na_setup(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    NaGrid g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.norb = norb; g.G = G;
    g.nchunk = (int)((G + kNaChunk - 1) / kNaChunk);
    g.h = h; g.ih2 = 1.0 / (h * h); g.dV = h * h * h;
    g.ox = origin[0]; g.oy = origin[1]; g.oz = origin[2];
    g.cx = origin[0] + 0.5 * h * (nx - 1);
    g.cy = origin[1] + 0.5 * h * (ny - 1);
    g.cz = origin[2] + 0.5 * h * (nz - 1);
    double *b = base + kNaOffB, *r = base + kNaOffR, *p = base + kNaOffP, *q = base + kNaOffQ;
    double* pq_part = base + kNaOffPart;
    double* rr_part = pq_part + kNaMaxChunks;
    double* bb_part = rr_part + kNaMaxChunks;
    double* mom_part = base + kNaOffMomPart;
    double* orbbase = base + kNaOffOrb;
    int* n_active_dev = (int*)(orbbase + 4 * kNaMaxOrb) + 3 * kNaMaxOrb;
    const dim3 grid(g.nchunk, norb);
    const double tol2 = cg_tol * cg_tol;
    k_na_moments<<<grid, kNaThreads, 0, s>>>(g, phi, mom_part);
    k_na_rhs<<<grid, kNaThreads, 0, s>>>(g, phi, mom_part, b, r, p, V, bb_part);
    k_na_init<<<norb, kNaThreads, 0, s>>>(g, bb_part, orbbase, max_iter);
    const int check_every = 8;
    for (int it = 0; it < max_iter; ++it) {
        if (it % check_every == 0) {
            k_na_count<<<1, 32, 0, s>>>(norb, orbbase);
            int n_active = 0;
            cudaError_t e = cudaMemcpyAsync(&n_active, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { na_fail("CUDA", cudaGetErrorString(e)); return FLOSIC_ERR_CUDA; }
            if (n_active == 0) break;
        }
        k_na_apply<<<grid, kNaThreads, 0, s>>>(g, p, q, pq_part, orbbase);
        k_na_alpha<<<norb, kNaThreads, 0, s>>>(g, pq_part, orbbase);
        k_na_update<<<grid, kNaThreads, 0, s>>>(g, V, r, p, q, rr_part, orbbase);
        k_na_beta<<<norb, kNaThreads, 0, s>>>(g, rr_part, orbbase, tol2, max_iter);
        k_na_pupdate<<<grid, kNaThreads, 0, s>>>(g, r, p, orbbase);
    }
    k_na_finish<<<(norb + 127) / 128, 128, 0, s>>>(norb, orbbase, iters, conv_flags);
    // report convergence from the scratch flags
    int conv_host[kNaMaxOrb];
    const int* conv_dev = (const int*)(orbbase + 4 * kNaMaxOrb) + 2 * kNaMaxOrb;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(conv_host, conv_dev, sizeof(int) * norb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { na_fail("CUDA", cudaGetErrorString(e)); return FLOSIC_ERR_CUDA; }
    for (int o = 0; o < norb; ++o)
        if (!conv_host[o]) { na_fail("a Poisson solve reached max_iter", nullptr); return FLOSIC_ERR_NOCONV; }
    return FLOSIC_OK;
}
