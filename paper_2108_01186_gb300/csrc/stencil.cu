// The 12th-order Laplacian on 3-D tiles (Sec. II.A: high-order centred
// finite differences), the hot kernel of the Poisson solves.
//
// A CTA owns a 32 x 16 (x, y) column tile of one orbital and marches along z
// through 32 planes.  Per plane it stages the tile plus a 6-point halo in x
// and y in shared memory (x/y taps), while each thread keeps the 13 values of
// its two columns between z-6 and z+6 in registers (z taps).  Every input
// value therefore comes from DRAM about once; halos come from L2.  Points
// outside the interior read as zero (zero ghost values of the correction
// equation).  Threads: 32 x 8, two y rows each.
#include <cuda.h>

#include "internal.cuh"

namespace flosic {

// this file's copy of the 12th-order weights (constant banks are per file)
__constant__ double c_w12[kHalf + 1];
__constant__ float c_w12f[kHalf + 1];

cudaError_t upload_stencil12_constants() {
    double w[kHalf + 1];
    float wf[kHalf + 1];
    stencil_weights(w);
    for (int k = 0; k <= kHalf; ++k) wf[k] = (float)w[k];
    cudaError_t e = cudaMemcpyToSymbol(c_w12, w, sizeof(w));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_w12f, wf, sizeof(wf));
}

template <class T> __device__ __forceinline__ T wgt(int m);
template <> __device__ __forceinline__ float wgt<float>(int m) { return c_w12f[m]; }
template <> __device__ __forceinline__ double wgt<double>(int m) { return c_w12[m]; }

constexpr int kPX = kTileX + 2 * kHalf;   // staged plane width
constexpr int kPY = kTileY + 2 * kHalf;   // staged plane height

// Value source of the stencil: the fused PCG direction p = z + beta p_old
// (first iteration: p = z) or a plain array.
template <class T>
struct SrcPcg {
    const T* z;
    const T* p;
    T beta;
    bool first;
    __device__ __forceinline__ T operator()(long long g) const { return first ? z[g] : z[g] + beta * p[g]; }
};
template <class T>
struct SrcPlain {
    const T* u;
    __device__ __forceinline__ T operator()(long long g) const { return u[g]; }
};

// Core of the tiled sweep: for each plane z of the tile calls
// epi(g, k, center, A_center) for the thread's two points (k = 0, 1), where
// A_center = (-Delta_h u) at that point.  The staged plane of z+1 is loaded
// into registers while plane z is computed, so each thread keeps about a
// dozen loads in flight.
constexpr int kSlots = (kPX * kPY + kTileX * (kTileY / 2) - 1) / (kTileX * (kTileY / 2));

template <class T, class Src, class Epi>
__device__ __forceinline__ void sweep12(const LvlDesc& D, const TilePos& P, const Src& src, T ih2, Epi epi,
                                        T (*plane)[kPX]) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTileX + tx;
    const int nthr = kTileX * (kTileY / 2);
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const int gx = P.x0 + tx;
    const int gy0 = P.y0 + ty, gy1 = P.y0 + ty + kTileY / 2;
    const bool in0 = gx < D.nx && gy0 < D.ny, in1 = gx < D.nx && gy1 < D.ny;
    const long long c0 = gy0 * sy + gx, c1 = gy1 * sy + gx;
    // this thread's slots of the staged plane: in-plane offset, or -1
    long long soff[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        const int e = tid + j * nthr;
        soff[j] = -1;
        if (e < kPX * kPY) {
            const int yy = e / kPX, xx = e - yy * kPX;
            const int px = P.x0 - kHalf + xx, py = P.y0 - kHalf + yy;
            if (px >= 0 && px < D.nx && py >= 0 && py < D.ny) soff[j] = py * sy + px;
        }
    }
    // column queues: q0/q1[j] = u at (gx, gy, z - 6 + j)
    T q0[2 * kHalf + 1], q1[2 * kHalf + 1];
#pragma unroll
    for (int j = 0; j < 2 * kHalf; ++j) {
        const int zz = P.z0 - kHalf + j;
        const bool okz = zz >= 0 && zz < D.nz;
        q0[j] = (in0 && okz) ? src(P.base + zz * sz + c0) : T(0);
        q1[j] = (in1 && okz) ? src(P.base + zz * sz + c1) : T(0);
    }
    T pre[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? src(P.base + P.z0 * sz + soff[j]) : T(0);
    const T w0 = T(3) * wgt<T>(0);
    T* flat = &plane[0][0];
    for (int z = P.z0; z < P.z1; ++z) {
#pragma unroll
        for (int j = 0; j < kSlots; ++j) {
            const int e = tid + j * nthr;
            if (e < kPX * kPY) flat[e] = pre[j];
        }
        {
            const int zz = z + kHalf;
            q0[2 * kHalf] = (in0 && zz < D.nz) ? src(P.base + zz * sz + c0) : T(0);
            q1[2 * kHalf] = (in1 && zz < D.nz) ? src(P.base + zz * sz + c1) : T(0);
        }
        __syncthreads();
        if (z + 1 < P.z1) {
            const long long pz = P.base + (z + 1) * sz;
#pragma unroll
            for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? src(pz + soff[j]) : T(0);
        }
        const int lx = tx + kHalf;
        const int ly0 = ty + kHalf, ly1 = ty + kTileY / 2 + kHalf;
        T a0 = w0 * q0[kHalf], a1 = w0 * q1[kHalf];
#pragma unroll
        for (int m = 1; m <= kHalf; ++m) {
            const T wm = wgt<T>(m);
            a0 += wm * (plane[ly0][lx - m] + plane[ly0][lx + m] + plane[ly0 - m][lx] + plane[ly0 + m][lx] +
                        q0[kHalf - m] + q0[kHalf + m]);
            a1 += wm * (plane[ly1][lx - m] + plane[ly1][lx + m] + plane[ly1 - m][lx] + plane[ly1 + m][lx] +
                        q1[kHalf - m] + q1[kHalf + m]);
        }
        if (in0) epi(P.base + z * sz + c0, 0, q0[kHalf], -a0 * ih2);
        if (in1) epi(P.base + z * sz + c1, 1, q1[kHalf], -a1 * ih2);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 2 * kHalf; ++j) {
            q0[j] = q0[j + 1];
            q1[j] = q1[j + 1];
        }
    }
}

// PCG direction and its image with one stencil sweep of z (the
// preconditioned residual): p = z + beta p, q = A z + beta q (first
// iteration, beta = 0: p = z, q = A z); pq = p.q per orbital.  Plain-load
// variant for grids whose rows are not 16-byte aligned.
template <class T>
__global__ void __launch_bounds__(256) k_apply12_pcg(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     const T* __restrict__ z, T* __restrict__ p, T* __restrict__ q,
                                                     CgState st) {
    __shared__ T plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const double bd = st.beta[P.o];
    const bool first = (bd == 0.0);
    const T beta = (T)bd;
    SrcPlain<T> src{z};
    const T ih2 = (T)(1.0 / (D.h * D.h));
    double pq = 0.0;
    sweep12<T>(D, P, src, ih2, [&](long long g, int, T zc, T az) {
        const T pn = first ? zc : zc + beta * p[g];
        const T qn = first ? az : az + beta * q[g];
        p[g] = pn;
        q[g] = qn;
        pq += (double)pn * (double)qn;
    }, plane);
    const int o = P.o;
    if (tile_arrive(pq, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[o] = 0;
            st.pq[o] = sum;
        }
    }
}

// ---------------------------------------------------------------------------
// TMA variant: the staged planes (tile plus halo, 48 x 28) arrive by
// cp.async.bulk.tensor into a ring of kRing shared-memory stages, completed
// on mbarriers; out-of-range rows, columns and planes are zero-filled by the
// copy engine, which is exactly the zero ghost value of the correction
// equation.  Ring: the plane of the output step (x/y taps), the six above it
// (the head of the register z-queue comes from the plane six steps ahead),
// and three more planes in flight.
// ---------------------------------------------------------------------------
constexpr int kSX = 48;        // staged width: x0 - 8 .. x0 + 39 (x0 - 8 keeps the copy 16-byte aligned)
constexpr int kSY = kTileY + 2 * kHalf;   // 28: y0 - 6 .. y0 + 21
constexpr int kRing = 10;
constexpr long long kWaitLimit = 1LL << 22;   // bounded mbarrier wait (far beyond any real copy latency)

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Waits for the phase with the given parity; gives up after kWaitLimit
// polls and reports it through *err (never hangs the GPU).
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* err) {
    const unsigned a = smem_addr(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return;
    }
    atomicOr(err, 1);
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

template <class T>
__global__ void __launch_bounds__(256) k_apply12_tma(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     const CUtensorMap* __restrict__ maps, T* __restrict__ p,
                                                     T* __restrict__ q, CgState st, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the copy engine wants 128-byte aligned stages: align the base explicitly
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    T* ring = reinterpret_cast<T*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(T) * kRing * kSY * kSX);
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const CUtensorMap* map = maps + P.b;
    const int oi = P.o - blk[P.b].orb0;
    const int tid = linear_tid();
    const int nzt = P.z1 - P.z0;
    const int np = nzt + 2 * kHalf;           // planes z0-6 .. z1+5
    const unsigned bytes = sizeof(T) * kSY * kSX;
    auto slot = [&](int k) { return ring + (size_t)(k % kRing) * kSY * kSX; };
    auto issue = [&](int k) {
        uint64_t* b = bar + (k % kRing);
        mbar_expect_tx(b, bytes);
        tma_load_4d(slot(k), map, P.x0 - 8, P.y0 - kHalf, P.z0 - kHalf + k, oi, b);
    };
    if (tid == 0) {
        for (int r = 0; r < kRing; ++r) mbar_init(bar + r, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < kRing && k < np; ++k) issue(k);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lx = tx + 8, ly0 = ty + kHalf, ly1 = ty + kTileY / 2 + kHalf;
    const int gx = P.x0 + tx, gy0 = P.y0 + ty, gy1 = P.y0 + ty + kTileY / 2;
    const bool in0 = gx < D.nx && gy0 < D.ny, in1 = gx < D.nx && gy1 < D.ny;
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const long long c0 = gy0 * sy + gx, c1 = gy1 * sy + gx;
    T q0[2 * kHalf + 1], q1[2 * kHalf + 1];
    // prologue: queue entries from planes 0..11; planes 0..5 are then done
    // with and their stages are refilled (planes kRing .. kRing + 5)
#pragma unroll
    for (int k = 0; k < 2 * kHalf; ++k) {
        mbar_wait(bar + (k % kRing), (k / kRing) & 1, err);
        const T* sl = slot(k);
        q0[k] = sl[ly0 * kSX + lx];
        q1[k] = sl[ly1 * kSX + lx];
        if (k < kHalf) {
            __syncthreads();
            if (tid == 0 && k + kRing < np) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + kRing);
            }
        }
    }
    const double bd = st.beta[P.o];
    const bool first = (bd == 0.0);
    const T beta = (T)bd;
    const T ih2 = (T)(1.0 / (D.h * D.h));
    const T w0 = T(3) * wgt<T>(0);
    double pq = 0.0;
    // p_old and q_old of the thread's two points, loaded one plane ahead
    T pp0 = 0, pp1 = 0, qq0 = 0, qq1 = 0;
    if (!first) {
        const long long zo = P.base + P.z0 * sz;
        if (in0) { pp0 = p[zo + c0]; qq0 = q[zo + c0]; }
        if (in1) { pp1 = p[zo + c1]; qq1 = q[zo + c1]; }
    }
    for (int s = 0; s < nzt; ++s) {
        T np0 = 0, np1 = 0, nq0 = 0, nq1 = 0;
        if (!first && s + 1 < nzt) {
            const long long zn = P.base + (P.z0 + s + 1) * sz;
            if (in0) { np0 = p[zn + c0]; nq0 = q[zn + c0]; }
            if (in1) { np1 = p[zn + c1]; nq1 = q[zn + c1]; }
        }
        const int kh = s + 2 * kHalf;      // head plane z + 6
        mbar_wait(bar + (kh % kRing), (kh / kRing) & 1, err);
        const T* hs = slot(kh);
        q0[2 * kHalf] = hs[ly0 * kSX + lx];
        q1[2 * kHalf] = hs[ly1 * kSX + lx];
        const T* pl = slot(s + kHalf);     // plane z
        T a0 = w0 * q0[kHalf], a1 = w0 * q1[kHalf];
#pragma unroll
        for (int m = 1; m <= kHalf; ++m) {
            const T wm = wgt<T>(m);
            a0 += wm * (pl[ly0 * kSX + lx - m] + pl[ly0 * kSX + lx + m] + pl[(ly0 - m) * kSX + lx] +
                        pl[(ly0 + m) * kSX + lx] + q0[kHalf - m] + q0[kHalf + m]);
            a1 += wm * (pl[ly1 * kSX + lx - m] + pl[ly1 * kSX + lx + m] + pl[(ly1 - m) * kSX + lx] +
                        pl[(ly1 + m) * kSX + lx] + q1[kHalf - m] + q1[kHalf + m]);
        }
        const long long zo = P.base + (P.z0 + s) * sz;
        if (in0) {
            const long long g = zo + c0;
            const T pn = q0[kHalf] + beta * pp0;
            const T qn = -a0 * ih2 + beta * qq0;
            p[g] = pn;
            q[g] = qn;
            pq += (double)pn * (double)qn;
        }
        if (in1) {
            const long long g = zo + c1;
            const T pn = q1[kHalf] + beta * pp1;
            const T qn = -a1 * ih2 + beta * qq1;
            p[g] = pn;
            q[g] = qn;
            pq += (double)pn * (double)qn;
        }
        pp0 = np0; pp1 = np1; qq0 = nq0; qq1 = nq1;
        __syncthreads();                   // stage of plane z is free
        if (tid == 0 && s + kHalf + kRing < np) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(s + kHalf + kRing);
        }
#pragma unroll
        for (int j = 0; j < 2 * kHalf; ++j) {
            q0[j] = q0[j + 1];
            q1[j] = q1[j + 1];
        }
    }
    const int o = P.o;
    if (tile_arrive(pq, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[o] = 0;
            st.pq[o] = sum;
        }
    }
}

size_t apply12_tma_smem(size_t elem) { return elem * kRing * kSY * kSX + sizeof(uint64_t) * kRing + 128; }

const void* apply12_tma_symbol(bool f32) {
    return f32 ? (const void*)k_apply12_tma<float> : (const void*)k_apply12_tma<double>;
}

// r = b - A x in float64, rr = r.r; orbitals whose rr <= tol2 * bb stop
// (flag 0, converged), as do orbitals past max_iter or with a non-finite rr.
__global__ void __launch_bounds__(256) k_residual12(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                    const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                    const double* __restrict__ b, const double* __restrict__ x,
                                                    double* __restrict__ r, double tol2, int max_iter,
                                                    int* __restrict__ flag, int* __restrict__ counter, int want_bb,
                                                    CgState st) {
    __shared__ double plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!flag[P.o]) return;
    const LvlDesc& D = L[P.b];
    SrcPlain<double> src{x};
    const double ih2 = 1.0 / (D.h * D.h);
    double rr = 0.0, bb = 0.0;
    sweep12<double>(D, P, src, ih2, [&](long long g, int, double, double ax) {
        const double bv = b[g];
        const double rv = bv - ax;
        r[g] = rv;
        rr += rv * rv;
        bb += bv * bv;
    }, plane);
    const int o = P.o;
    double bbs = 0.0;
    if (want_bb) {
        bbs = block_sum(bb, scratch);
        if (linear_tid() == 0) st.part2[blockIdx.x] = bbs;
    }
    if (tile_arrive(rr, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double s = tile_gather(st.part, P.first, D.ntile, scratch);
        if (want_bb) {
            const double sb = tile_gather(st.part2, P.first, D.ntile, scratch);
            if (linear_tid() == 0) st.bb[o] = sb;
        }
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            st.count[o] = 0;
            st.rr[o] = s;
            st.thr[o] = tol2 * st.bb[o];
            if (!(s > st.thr[o])) {
                flag[o] = 0;
                st.conv[o] = 1;
                atomicSub(counter, 1);
            } else if (st.iters[o] >= max_iter || !isfinite(s)) {
                flag[o] = 0;
                atomicSub(counter, 1);
            }
        }
    }
}

template <class T>
void launch_apply12_pcg(flosic_ctx* c, const T* z, T* p, T* q, cudaStream_t s) {
    const Multigrid& M = c->mg;
    prof_begin(c, s);
    if (c->tma_ok) {
        k_apply12_tma<T><<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), apply12_tma_smem(sizeof(T)), s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, (const CUtensorMap*)c->d_tmaps, p, q, c->ws.cg,
            c->ws.status + 3);
    } else {
        k_apply12_pcg<T><<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, z, p, q, c->ws.cg);
    }
    note_launch(c);
    prof_end(c, s);
}
template void launch_apply12_pcg<float>(flosic_ctx*, const float*, float*, float*, cudaStream_t);
template void launch_apply12_pcg<double>(flosic_ctx*, const double*, double*, double*, cudaStream_t);

void launch_residual12(flosic_ctx* c, const double* b, const double* x, double* r, double tol2, int max_iter,
                       int* flag, int* counter, int want_bb, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_residual12<<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, b, x, r, tol2, max_iter, flag, counter, want_bb,
        c->ws.cg); note_launch(c);
}

}  // namespace flosic
