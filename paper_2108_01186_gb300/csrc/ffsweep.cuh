// 12th-order Laplacian in float-float arithmetic on one 3-D tile (Sec. II.A:
// high-order centred finite differences), shared by the refinement residual
// and the mixed-precision Hamiltonian apply.
//
// A CTA (32 x 8 threads) owns a 32 x 16 column tile of one orbital and
// marches along z: per plane the tile plus its 6-point x/y halo is staged in
// shared memory as pairs, each thread keeps the 13 z-values of its two
// columns in registers, and the next plane's slots are loaded while the
// current one is computed.  Values outside the interior read as zero, or,
// along the periodic directions of the level (D.per), wrap around the box.
#pragma once
#include "internal.cuh"

namespace flosic {

// weights 3 w_0, w_1 .. w_6 of the Laplacian as (hi, lo) pairs (one copy per
// translation unit that includes this header; upload_ffsweep_weights fills it)
static __constant__ float c_wff[2 * (kHalf + 1)];

static inline cudaError_t upload_ffsweep_weights() {
    double w[kHalf + 1];
    stencil_weights(w);
    float f[2 * (kHalf + 1)];
    for (int m = 0; m <= kHalf; ++m) {
        const double ww = (m == 0) ? 3.0 * w[0] : w[m];
        f[2 * m] = (float)ww;
        f[2 * m + 1] = (float)(ww - (double)f[2 * m]);
    }
    return cudaMemcpyToSymbol(c_wff, f, sizeof(f));
}

// load(g) -> float2 pair of the operand at flat index g (only called for
// points inside the grid); epi(g, centre, lap) with lap = h^2 Delta_h u at g
// as a pair, called for every point of the tile inside the grid.
// kSloppy: the seven weighted terms are accumulated with the two-sum of the
// high parts and a plain sum of the low parts (error ~ eps^2 times the sum
// of the terms' magnitudes, ~1e-12 of the result for the smooth potentials
// of the refinement residual) instead of the renormalised pair addition
// (error ~ eps^2 of the result, kept for the Hamiltonian apply).
template <bool kSloppy = false, class Load, class Epi>
__device__ __forceinline__ void ff_sweep12(const LvlDesc& D, const TilePos& P, Load load, Epi epi,
                                           ff (*plane)[kPX]) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTileX + tx;
    const int nthr = kTileX * (kTileY / 2);
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const int gx = P.x0 + tx;
    const int gy0 = P.y0 + ty, gy1 = P.y0 + ty + kTileY / 2;
    const bool in0 = gx < D.nx && gy0 < D.ny, in1 = gx < D.nx && gy1 < D.ny;
    const long long c0 = gy0 * sy + gx, c1 = gy1 * sy + gx;
    long long soff[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        const int e = tid + j * nthr;
        soff[j] = -1;
        if (e < kPX * kPY) {
            const int yy = e / kPX, xx = e - yy * kPX;
            int px = P.x0 - kHalf + xx, py = P.y0 - kHalf + yy;
            if (D.per & 1) px = wrap_coord(px, D.nx);
            if (D.per & 2) py = wrap_coord(py, D.ny);
            if (px >= 0 && px < D.nx && py >= 0 && py < D.ny) soff[j] = py * sy + px;
        }
    }
    const float2 zero2 = make_float2(0.f, 0.f);
    ff q0[2 * kHalf + 1], q1[2 * kHalf + 1];
    const bool perz = (D.per & 4) != 0;
#pragma unroll
    for (int j = 0; j < 2 * kHalf; ++j) {
        int zz = P.z0 - kHalf + j;
        if (perz) zz = wrap_coord(zz, D.nz);
        const bool okz = zz >= 0 && zz < D.nz;
        q0[j] = to_ff((in0 && okz) ? load(P.base + zz * sz + c0) : zero2);
        q1[j] = to_ff((in1 && okz) ? load(P.base + zz * sz + c1) : zero2);
    }
    float2 pre[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? load(P.base + P.z0 * sz + soff[j]) : zero2;
    ff w[kHalf + 1];
#pragma unroll
    for (int m = 0; m <= kHalf; ++m) w[m] = {c_wff[2 * m], c_wff[2 * m + 1]};
    ff* flat = &plane[0][0];
    for (int z = P.z0; z < P.z1; ++z) {
#pragma unroll
        for (int j = 0; j < kSlots; ++j) {
            const int e = tid + j * nthr;
            if (e < kPX * kPY) flat[e] = to_ff(pre[j]);
        }
        {
            int zz = z + kHalf;
            if (perz) zz = wrap_coord(zz, D.nz);
            q0[2 * kHalf] = to_ff((in0 && zz < D.nz) ? load(P.base + zz * sz + c0) : zero2);
            q1[2 * kHalf] = to_ff((in1 && zz < D.nz) ? load(P.base + zz * sz + c1) : zero2);
        }
        __syncthreads();
        if (z + 1 < P.z1) {
            const long long pz = P.base + (z + 1) * sz;
#pragma unroll
            for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? load(pz + soff[j]) : zero2;
        }
        const int lx = tx + kHalf;
        const int ly[2] = {ty + kHalf, ty + kTileY / 2 + kHalf};
        const bool in[2] = {in0, in1};
        const long long cc[2] = {c0, c1};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const ff* qk = (k == 0) ? q0 : q1;
            ff acc = ff_mul(w[0], qk[kHalf]);
#pragma unroll
            for (int m = 1; m <= kHalf; ++m) {
                const ff sm = ff_sum6(plane[ly[k]][lx - m], plane[ly[k]][lx + m], plane[ly[k] - m][lx],
                                      plane[ly[k] + m][lx], qk[kHalf - m], qk[kHalf + m]);
                const ff tm = ff_mul(w[m], sm);
                if constexpr (kSloppy) {
                    const ff s2 = ff_two_sum(acc.h, tm.h);
                    acc = ff_quick(s2.h, s2.l + (acc.l + tm.l));
                } else {
                    acc = ff_add(acc, tm);
                }
            }
            if (in[k]) epi(P.base + z * sz + cc[k], qk[kHalf], acc);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 2 * kHalf; ++j) {
            q0[j] = q0[j + 1];
            q1[j] = q1[j + 1];
        }
    }
}

}  // namespace flosic
