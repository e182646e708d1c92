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

// p = z + beta p_old, q = A p, pq = p.q (per orbital, deterministic).
template <class T>
__global__ void __launch_bounds__(256) k_apply12_pcg(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     const T* __restrict__ z, const T* __restrict__ pold,
                                                     T* __restrict__ pnew, T* __restrict__ q, CgState st) {
    __shared__ T plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const double bd = st.beta[P.o];
    SrcPcg<T> src{z, pold, (T)bd, bd == 0.0};
    const T ih2 = (T)(1.0 / (D.h * D.h));
    double pq = 0.0;
    sweep12<T>(D, P, src, ih2, [&](long long g, int, T pc, T qv) {
        pnew[g] = pc;
        q[g] = qv;
        pq += (double)pc * (double)qv;
    }, plane);
    const int o = P.o;
    if (tile_arrive(pq, st.part, blockIdx.x, st.count + o, D.ntile, scratch)) {
        const double s = tile_gather(st.part, P.first, D.ntile, scratch);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            st.count[o] = 0;
            st.pq[o] = s;
        }
    }
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
void launch_apply12_pcg(flosic_ctx* c, const T* z, const T* pold, T* pnew, T* q, cudaStream_t s) {
    const Multigrid& M = c->mg;
    prof_begin(c, s);
    k_apply12_pcg<T><<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, z, pold, pnew, q, c->ws.cg); note_launch(c);
    prof_end(c, s);
}
template void launch_apply12_pcg<float>(flosic_ctx*, const float*, const float*, float*, float*, cudaStream_t);
template void launch_apply12_pcg<double>(flosic_ctx*, const double*, const double*, double*, double*, cudaStream_t);

void launch_residual12(flosic_ctx* c, const double* b, const double* x, double* r, double tol2, int max_iter,
                       int* flag, int* counter, int want_bb, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_residual12<<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, b, x, r, tol2, max_iter, flag, counter, want_bb,
        c->ws.cg); note_launch(c);
}

}  // namespace flosic
