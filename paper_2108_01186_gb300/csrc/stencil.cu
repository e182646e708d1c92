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
    {
        cudaError_t e = upload_ff_weights();
        if (e != cudaSuccess) return e;
    }
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
    if (!st.active[P.o] || L[P.b].tma) return;
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
            atomicAdd(st.prof_bytes, (double)D.G * sizeof(T) * (first ? 3 : 5));
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

template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Ring stage: the staged plane z with halo (48 x 28), and three 32 x 16
// centre tiles: z at plane z+6 (head of the register z-queue), p_old and
// q_old at plane z.  Threads 16 x 8; each owns the 2 x 2 points
// (x0 + 2tx + a, y0 + 2ty + b).
constexpr int kStagePlane = kSX * kSY;
constexpr int kStageCtr = kTileX * kTileY;
constexpr int kStageElems = kStagePlane + 3 * kStageCtr;
constexpr int kRing2 = 4;

template <class T>
__global__ void __launch_bounds__(128) k_apply12_tma(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     const CUtensorMap* __restrict__ maps, const T* __restrict__ z,
                                                     T* __restrict__ p, T* __restrict__ q, CgState st,
                                                     int* __restrict__ err) {
    using V2 = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    T* ring = reinterpret_cast<T*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + sizeof(T) * kRing2 * kStageElems);
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o] || !L[P.b].tma) return;
    const LvlDesc& D = L[P.b];
    const CUtensorMap* mp = maps + 4 * P.b;    // z with halo, z centre, p centre, q centre
    const int oi = P.o - blk[P.b].orb0;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nzt = P.z1 - P.z0;
    const double bd = st.beta[P.o];
    const bool first = (bd == 0.0);
    const unsigned bytes = sizeof(T) * (first ? kStagePlane + kStageCtr : kStageElems);
    auto stage = [&](int s) { return ring + (size_t)(s % kRing2) * kStageElems; };
    auto issue = [&](int s) {
        uint64_t* b = bar + (s % kRing2);
        T* st_ = stage(s);
        const int zz = P.z0 + s;
        mbar_expect_tx(b, bytes);
        tma_load_4d(st_, mp + 0, P.x0 - 8, P.y0 - kHalf, zz, oi, b);
        tma_load_4d(st_ + kStagePlane, mp + 1, P.x0, P.y0, zz + kHalf, oi, b);
        if (!first) {
            tma_load_4d(st_ + kStagePlane + kStageCtr, mp + 2, P.x0, P.y0, zz, oi, b);
            tma_load_4d(st_ + kStagePlane + 2 * kStageCtr, mp + 3, P.x0, P.y0, zz, oi, b);
        }
    };
    if (tid == 0) {
        for (int r = 0; r < kRing2; ++r) mbar_init(bar + r, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < kRing2 && k < nzt; ++k) issue(k);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = P.x0 + 2 * tx;
    const int gy0 = P.y0 + 2 * ty;
    const bool inx = gx < D.nx;
    const bool iny[2] = {gy0 < D.ny, gy0 + 1 < D.ny};
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    // register z-queues of the four points: qz[b][a][j], planes z-6 .. z+6
    T qz[2][2][2 * kHalf + 1];
#pragma unroll
    for (int j = 0; j < 2 * kHalf; ++j) {
        const int zz = P.z0 - kHalf + j;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            V2 v;
            v.x = T(0);
            v.y = T(0);
            if (inx && iny[b] && zz >= 0 && zz < D.nz)
                v = *reinterpret_cast<const V2*>(z + P.base + zz * sz + (gy0 + b) * sy + gx);
            qz[b][0][j] = v.x;
            qz[b][1][j] = v.y;
        }
    }
    const T beta = (T)bd;
    const T ih2 = (T)(1.0 / (D.h * D.h));
    T wm[kHalf + 1];
#pragma unroll
    for (int m = 0; m <= kHalf; ++m) wm[m] = wgt<T>(m);
    const T w0 = T(3) * wm[0];
    T pqf = T(0);
    const int lx = 2 * tx + 8, ly0 = 2 * ty + kHalf;
    for (int s = 0; s < nzt; ++s) {
        mbar_wait(bar + (s % kRing2), (s / kRing2) & 1, err);
        const T* pl = stage(s);
        const T* hd = pl + kStagePlane;
        const T* po = pl + kStagePlane + kStageCtr;
        const T* qo = pl + kStagePlane + 2 * kStageCtr;
        // queue heads (plane z + 6) and the y-window of the column pair
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const V2 h = *reinterpret_cast<const V2*>(hd + (2 * ty + b) * kTileX + 2 * tx);
            qz[b][0][2 * kHalf] = h.x;
            qz[b][1][2 * kHalf] = h.y;
        }
        T yw[2][2 * kHalf + 2];     // [a][k], rows 2ty .. 2ty+13
#pragma unroll
        for (int k = 0; k < 2 * kHalf + 2; ++k) {
            const V2 v = *reinterpret_cast<const V2*>(pl + (2 * ty + k) * kSX + lx);
            yw[0][k] = v.x;
            yw[1][k] = v.y;
        }
        T out[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            T xw[2 * kHalf + 2];    // cols lx-6 .. lx+7 of row ly0+b
#pragma unroll
            for (int k = 0; k < kHalf + 1; ++k) {
                const V2 v = *reinterpret_cast<const V2*>(pl + (ly0 + b) * kSX + lx - kHalf + 2 * k);
                xw[2 * k] = v.x;
                xw[2 * k + 1] = v.y;
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                T acc = w0 * yw[a][kHalf + b];
#pragma unroll
                for (int m = 1; m <= kHalf; ++m)
                    acc += wm[m] * (xw[kHalf + a - m] + xw[kHalf + a + m] + yw[a][kHalf + b - m] +
                                    yw[a][kHalf + b + m] + qz[b][a][kHalf - m] + qz[b][a][kHalf + m]);
                out[b][a] = -acc * ih2;
            }
        }
        const long long zo = P.base + (P.z0 + s) * sz;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!(inx && iny[b])) continue;
            V2 pn, qn;
            pn.x = yw[0][kHalf + b];
            pn.y = yw[1][kHalf + b];
            qn.x = out[b][0];
            qn.y = out[b][1];
            if (!first) {
                const V2 pv = *reinterpret_cast<const V2*>(po + (2 * ty + b) * kTileX + 2 * tx);
                const V2 qv = *reinterpret_cast<const V2*>(qo + (2 * ty + b) * kTileX + 2 * tx);
                pn.x += beta * pv.x;
                pn.y += beta * pv.y;
                qn.x += beta * qv.x;
                qn.y += beta * qv.y;
            }
            const long long g = zo + (gy0 + b) * sy + gx;
            *reinterpret_cast<V2*>(p + g) = pn;
            *reinterpret_cast<V2*>(q + g) = qn;
            pqf += pn.x * qn.x + pn.y * qn.y;
        }
        __syncthreads();                   // stage s is free
        if (tid == 0 && s + kRing2 < nzt) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(s + kRing2);
        }
#pragma unroll
        for (int j = 0; j < 2 * kHalf; ++j) {
            qz[0][0][j] = qz[0][0][j + 1];
            qz[0][1][j] = qz[0][1][j + 1];
            qz[1][0][j] = qz[1][0][j + 1];
            qz[1][1][j] = qz[1][1][j + 1];
        }
    }
    const int o = P.o;
    if (tile_arrive(pqf, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[o] = 0;
            st.pq[o] = sum;
            // algorithmic bytes of this orbital: read z (+ p_old, q_old), write p, q
            atomicAdd(st.prof_bytes, (double)D.G * sizeof(T) * (first ? 3 : 5));
        }
    }
}

size_t apply12_tma_smem(size_t elem) { return elem * kRing2 * kStageElems + sizeof(uint64_t) * kRing2 + 128; }

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

// The residual of an Alternating Anderson-Richardson step, updated with the
// last step dx: r -= A dx with one staged sweep of dx, rr = r.r per orbital.
// (Recomputing b - A x in float32 would stall near eps times the condition
// number of A; the update carries the rounding of dx only, as CG's
// recursive residual does, and the float-float refinement around the solve
// recomputes the true residual.)  The last tile of an orbital counts the
// step and applies the stop tests (target thr, max_iter, non-finite).
// Reads dx and r, writes r.
template <class T>
__global__ void __launch_bounds__(256) k_residual12_aar(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                        const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                        const T* __restrict__ dx, T* __restrict__ r, int max_iter,
                                                        CgState st) {
    __shared__ T plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    SrcPlain<T> src{dx};
    const T ih2 = (T)(1.0 / (D.h * D.h));
    T rr = T(0);
    sweep12<T>(D, P, src, ih2, [&](long long g, int, T, T adx) {
        const T rv = r[g] - adx;
        r[g] = rv;
        rr += rv * rv;
    }, plane);
    const int o = P.o;
    if (tile_arrive(rr, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[o] = 0;
            st.rr[o] = sum;
            const int it = ++st.iters[o];
            if (!(sum > st.thr[o]) || it >= max_iter || !isfinite(sum)) {
                st.active[o] = 0;
                atomicSub(st.n_active, 1);
            }
            atomicAdd(st.prof_bytes, (double)D.G * sizeof(T) * 3);
        }
    }
}

template <class T>
void launch_residual12_aar(flosic_ctx* c, const T* dx, T* r, cudaStream_t s) {
    const Multigrid& M = c->mg;
    prof_begin(c, s);
    k_residual12_aar<T><<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, dx, r, c->opt.max_iter, c->ws.cg);
    note_launch(c);
    prof_end(c, s);
}
template void launch_residual12_aar<float>(flosic_ctx*, const float*, float*, cudaStream_t);

template <class T>
void launch_apply12_pcg(flosic_ctx* c, const T* z, T* p, T* q, cudaStream_t s) {
    const Multigrid& M = c->mg;
    prof_begin(c, s);
    if (c->n_tma_blocks > 0) {       // blocks whose operands the copy engine stages
        k_apply12_tma<T><<<(unsigned)M.ntiles[0], dim3(kTileX / 2, kTileY / 2), apply12_tma_smem(sizeof(T)), s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, (const CUtensorMap*)c->d_tmaps, z, p, q, c->ws.cg,
            c->ws.status + 3);
        note_launch(c);
    }
    if (c->n_tma_blocks < c->nblk) {  // the rest: the same sweep with plain loads
        k_apply12_pcg<T><<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, z, p, q, c->ws.cg);
        note_launch(c);
    }
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
