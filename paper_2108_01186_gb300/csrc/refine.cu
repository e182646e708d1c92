// Mixed-precision refinement of the per-orbital Poisson solves (Sec. II.A
// solves them iteratively; splitting the precision is this library's).
//
// The float32 multigrid-preconditioned CG computes corrections d of
// A d = r.  The solution x, the right-hand side b and the residual
// r = b - A x live in unevaluated float-float pairs (hi, lo), about 48
// significant bits: Knuth's error-free two-sum for additions and an
// FMA-based exact two-product.  GB300 runs float64 at a small fraction of
// its float32 rate, so inside the refinement loop no float64 operation runs
// per grid point; float64 appears only where x is joined into the float64
// result (one addition per point).  b arrives in pairs from the
// right-hand-side pass; a warm start is split with integer operations.
//
// Round structure per orbital:  r = b - A x (pairs) -> stop if
// r.r <= tol^2 b.b, else a float32 solve of A d = float(r) to
// max(inner_tol^2 r.r, tol^2 b.b / 4) -> x += d (pairs).
#include <cmath>
#include <vector>

#include <cudaTypedefs.h>

#include "ffsweep.cuh"
#include "tcgen05.cuh"

namespace flosic {


bool ix_weights_match();

// the float-float weights, after checking the update's integer weights
// against the float64 ones (a mismatch fails the context's creation)
cudaError_t upload_ff_weights() {
    if (!ix_weights_match()) return cudaErrorInvalidValue;
    return upload_ffsweep_weights();
}

// Last CTA of an orbital, once r.r is known: the outer stop test, else the
// start of the next float32 solve (its target, active flag and counters).
__device__ __forceinline__ void start_round(CgState& st, int o, double rr, double tol2, double inner_tol2,
                                            int max_iter) {
    st.rr[o] = rr;
    st.active[o] = 0;
    if (!(rr > tol2 * st.bb[o])) {
        st.oactive[o] = 0;
        st.conv[o] = 1;
        atomicSub(st.n_oactive, 1);
        return;
    }
    if (st.iters[o] >= max_iter || !isfinite(rr)) {
        st.oactive[o] = 0;
        atomicSub(st.n_oactive, 1);
        return;
    }
    const double a = inner_tol2 * rr, c = 0.25 * tol2 * st.bb[o];
    st.thr[o] = a > c ? a : c;
    st.rz[o] = 0.0;
    st.beta[o] = 0.0;
    st.active[o] = 1;
    atomicAdd(st.n_active, 1);
}

// Start of the refinement: b arrives in pairs (from the right-hand-side
// pass), x = warm start (pairs) or 0; b.b per orbital.  Without a warm start
// the residual is b itself: r32 = float(b), d32 = 0 (p32 = r32 when given)
// and the first float32 solve starts here.  keep_zero (cold start of a solver
// that overwrites d, the Kronecker solve): neither x nor d is stored; xz marks
// x as zero until the first update writes it.
__global__ void __launch_bounds__(256) k_ff_init(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                 const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                 const float2* __restrict__ b, const double* __restrict__ V,
                                                 float2* __restrict__ x, float* __restrict__ r32,
                                                 float* __restrict__ p32, float* __restrict__ d32, int warm,
                                                 int keep_zero, double tol2, double inner_tol2, int max_iter,
                                                 CgState st) {
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o]) return;
    const LvlDesc& D = L[P.b];
    float bb = 0.f;
    tile_elementwise<float>(D, P, [&](long long g, int n) {
        if (n == 4) {   // aligned group of four points: 16-byte accesses
            const float4 b01 = *reinterpret_cast<const float4*>(b + g);       // pairs g, g+1
            const float4 b23 = *reinterpret_cast<const float4*>(b + g + 2);   // pairs g+2, g+3
            const float4 bh = make_float4(b01.x, b01.z, b23.x, b23.z);
            bb += bh.x * bh.x + bh.y * bh.y + bh.z * bh.z + bh.w * bh.w;
            if (warm) {
                const double2 v01 = *reinterpret_cast<const double2*>(V + g);
                const double2 v23 = *reinterpret_cast<const double2*>(V + g + 2);
                const float2 a = d2ff(v01.x), c = d2ff(v01.y), e = d2ff(v23.x), f = d2ff(v23.y);
                *reinterpret_cast<float4*>(x + g) = make_float4(a.x, a.y, c.x, c.y);
                *reinterpret_cast<float4*>(x + g + 2) = make_float4(e.x, e.y, f.x, f.y);
            } else {
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!keep_zero) {
                    *reinterpret_cast<float4*>(x + g) = z4;
                    *reinterpret_cast<float4*>(x + g + 2) = z4;
                    *reinterpret_cast<float4*>(d32 + g) = z4;
                }
                *reinterpret_cast<float4*>(r32 + g) = bh;
                if (p32) *reinterpret_cast<float4*>(p32 + g) = bh;
            }
            return;
        }
        for (int k = 0; k < n; ++k) {
            const float bh = b[g + k].x;
            bb += bh * bh;
            if (warm) {
                x[g + k] = d2ff(V[g + k]);
            } else {
                if (!keep_zero) {
                    x[g + k] = make_float2(0.f, 0.f);
                    d32[g + k] = 0.f;
                }
                r32[g + k] = bh;
                if (p32) p32[g + k] = bh;
            }
        }
    });
    if (tile_arrive(bb, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[P.o] = 0;
            st.bb[P.o] = sum;
            st.xz[P.o] = (!warm && keep_zero) ? 1 : 0;
            if (!warm) start_round(st, P.o, sum, tol2, inner_tol2, max_iter);
        }
    }
}

// r = b - A x in pairs on the tiles of the float-float sweep.  Writes
// r32 = float(r), d32 = 0 (p32 = r32 when given) and starts the next round;
// with store_r also r itself as pairs over b (each point's r needs only its
// own b), for the rounds that then update r from the corrections.
__global__ void __launch_bounds__(256) k_residual12_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                       const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                       float2* __restrict__ b, const float2* __restrict__ x,
                                                       float* __restrict__ r32, float* __restrict__ p32,
                                                       float* __restrict__ d32, double tol2, double inner_tol2,
                                                       int max_iter, int store_r, CgState st) {
    __shared__ ff plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o]) return;
    const LvlDesc& D = L[P.b];
    const ff ih2 = to_ff(d2ff(1.0 / (D.h * D.h)));   // once per CTA
    float rrf = 0.f;
    ff_sweep12<true>(
        D, P, [&](long long g) { return x[g]; },
        [&](long long g, ff, ff acc) {
            // acc = h^2 Delta_h x, so r = b - A x = b + acc / h^2
            const ff r = ff_add(to_ff(b[g]), ff_mul(acc, ih2));
            const float rv = r.h;
            if (store_r) b[g] = make_float2(r.h, r.l);
            r32[g] = rv;
            d32[g] = 0.f;
            if (p32) p32[g] = rv;
            rrf += rv * rv;
        },
        plane);
    if (tile_arrive(rrf, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[P.o] = 0;
            start_round(st, P.o, sum, tol2, inner_tol2, max_iter);
        }
    }
}

// ---------------------------------------------------------------------------
// Exact stencil sums for the refinement update.  The 12th-order weights of
// the second derivative (Sec. II.A: centred differences, w_m =
// 2 (-1)^(m+1) (6!)^2 / (m^2 (6-m)! (6+m)!), w_0 = -2 sum w_m) are rationals
// whose common denominator is 831600, so W_m = 831600 w_m are integers and
// h^2 Delta_h u = (1 / 831600) sum_m W_m (sum of the six neighbours at
// distance m).  A float32 field d whose magnitude is below 2^e splits
// exactly into y = d 2^(28-e) = hi + lo with hi = rint(y) an integer
// (|hi| <= 2^28) and |lo| <= 1/2: the hi parts are summed and weighted in
// integers (six of them stay below 2^31, the weighted sum below 2^53), so
// that part is exact, and the lo parts in float32, an error of a few units
// of 2^(e-28) / 831600 in h^2 Delta_h d per point -- about 1e-14 of
// max |d| / h^2, below the float-float sweep's error on smooth fields.
// ---------------------------------------------------------------------------
constexpr long long kW12Den = 831600;

__host__ __device__ constexpr long long w12_fact(int n) { return n <= 1 ? 1 : n * w12_fact(n - 1); }
__host__ __device__ constexpr long long w12_num(int m) {   // 2 (6!)^2 831600, signed
    return (m % 2 == 1 ? 2 : -2) * w12_fact(6) * w12_fact(6) * kW12Den;
}
__host__ __device__ constexpr long long w12_den(int m) { return (long long)m * m * w12_fact(6 - m) * w12_fact(6 + m); }
// W_m for m >= 1; W_0 of the three-dimensional centre is 3 (-2 sum_m W_m)
__host__ __device__ constexpr long long w12_int(int m) { return w12_num(m) / w12_den(m); }
__host__ __device__ constexpr long long w12_centre3() {
    return -6 * (w12_int(1) + w12_int(2) + w12_int(3) + w12_int(4) + w12_int(5) + w12_int(6));
}
static_assert(w12_num(1) % w12_den(1) == 0 && w12_num(2) % w12_den(2) == 0 && w12_num(3) % w12_den(3) == 0 &&
                  w12_num(4) % w12_den(4) == 0 && w12_num(5) % w12_den(5) == 0 && w12_num(6) % w12_den(6) == 0,
              "831600 is a common denominator of the 12th-order weights");
static_assert(w12_centre3() > -(1LL << 24) && w12_int(1) < (1LL << 24), "weights exact in float32");

// Host check of the integer weights against the float64 ones the other
// stencils use (|W_m / 831600 - w_m| at rounding level).
bool ix_weights_match() {
    double w[kHalf + 1];
    stencil_weights(w);
    for (int m = 1; m <= kHalf; ++m)
        if (std::fabs((double)w12_int(m) / (double)kW12Den - w[m]) > 1e-15 * std::fabs(w[m])) return false;
    return std::fabs((double)w12_centre3() / (double)kW12Den - 3.0 * w[0]) <= 1e-15 * std::fabs(3.0 * w[0]);
}

struct __align__(8) IxPt {
    int h;     // rint(y)
    float l;   // y - rint(y), or y itself when it is not finite
};

// y = d 2^es (exact) split into hi + lo; a non-finite y keeps hi = 0 and
// carries inf / NaN in lo, so it reaches the residual.
__device__ __forceinline__ IxPt ix_split(float d, float s) {
    const float y = d * s;
    const float r = rintf(y);
    const bool fin = fabsf(y) < 536870912.f;   // 2^29
    return {fin ? __float2int_rn(r) : 0, fin ? y - r : y};
}

// I + Lo as a float-float pair (|I| < 2^53): |I| in three pieces of at most 23
// bits, each turned into a float exactly by the 2^23 bias (integer and float
// additions only -- no 64-bit conversion, which would run on the float64
// pipe), summed with a two-sum; Lo is added to the low part (one rounding).
__device__ __forceinline__ ff ix_to_ff(long long I, float Lo) {
    const unsigned long long M = I < 0 ? 0ull - (unsigned long long)I : (unsigned long long)I;
    const float f0 = __uint_as_float(0x4B000000u | ((unsigned)M & 0x7fffffu)) - 8388608.f;
    const float f1 = (__uint_as_float(0x4B000000u | ((unsigned)(M >> 23) & 0x7fffffu)) - 8388608.f) * 8388608.f;
    const float f2 = (__uint_as_float(0x4B000000u | (unsigned)(M >> 46)) - 8388608.f) * 70368744177664.f;
    ff v = ff_two_sum(f2, f1);
    const float sg = I < 0 ? -1.f : 1.f;
    v = ff_two_sum(sg * v.h, sg * (v.l + f0) + Lo);
    return v;
}

// ix_split without the finiteness test, for sums taken in unsigned (wrapping)
// integers: a non-finite y still carries inf / NaN in lo, and its saturated
// integer part only wraps the integer sum, which lo then overrides.
__device__ __forceinline__ IxPt ix_split_w(float d, float s) {
    const float y = d * s;
    const float r = rintf(y);
    return {__float2int_rn(r), y - r};
}

// ix_to_ff for |I| < 2^53 from I + 2^53 (non-negative): the pieces of 23, 23
// and 8 bits each exact as floats, the bias removed from the top piece.
__device__ __forceinline__ ff ix_to_ff_b(long long I, float Lo) {
    const unsigned long long M = (unsigned long long)I + (1ull << 53);
    const float f0 = __uint_as_float(0x4B000000u | ((unsigned)M & 0x7fffffu)) - 8388608.f;
    const float f1 = (__uint_as_float(0x4B000000u | ((unsigned)(M >> 23) & 0x7fffffu)) - 8388608.f) * 8388608.f;
    const float f2 = (__uint_as_float(0x4B000000u | (unsigned)(M >> 46)) - 8388736.f) * 70368744177664.f;
    const ff v = ff_two_sum(f2, f1);
    return ff_two_sum(v.h, (v.l + f0) + Lo);
}

// Per orbital, max |d| over its grid (float bits in st.dmax, atomicMax on
// the bit patterns of non-negative floats); the update's last CTA of the
// orbital resets it.  NaN values are skipped here and reach the residual
// through the split.
__global__ void __launch_bounds__(256) k_dmax(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                              const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                              const float* __restrict__ d32, CgState st) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o]) return;
    const LvlDesc& D = L[P.b];
    float m = 0.f;
    tile_elementwise<float>(D, P, [&](long long g, int n) {
        if (n == 4) {
            const float4 v = *reinterpret_cast<const float4*>(d32 + g);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            return;
        }
        for (int k = 0; k < n; ++k) m = fmaxf(m, fabsf(d32[g + k]));
    });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((linear_tid() & 31) == 0 && m > 0.f) atomicMax(st.dmax + P.o, __float_as_uint(m));
}

// One refinement round's update from the float32 correction d of the inner
// solve: r -= A d (r in pairs, in place: r_{k+1} = b - A x_{k+1} =
// r_k - A d_k), x += d (pairs), r32 = float(r), and the next round's start.
// A d comes from the exact integer sums above, on the tiles of the other
// 12th-order sweeps (a CTA of 32 x 8 threads owns a 32 x 16 column tile and
// marches along z: the plane with its 6-point x/y halo staged in shared
// memory as split values, the 13 z-values of each of its two columns in
// registers).  d is left as it is (neighbouring tiles read it as halo): this
// serves inner solvers that overwrite d (the Kronecker-product solve), not
// those that start from d = 0.
// kXZ: the first update after a cold start that stored no x (x = 0, not read)
template <bool kXZ>
__global__ void __launch_bounds__(256, 2) k_update12_ix(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     float2* __restrict__ r, float2* __restrict__ x,
                                                     float* __restrict__ r32, const float* __restrict__ d32,
                                                     double tol2, double inner_tol2, int max_iter, CgState st) {
    __shared__ IxPt plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o] || L[P.b].utma) return;
    const LvlDesc& D = L[P.b];
    // |d| < 2^(E - 126) with E the biased exponent of max |d|: scale by
    // 2^es, es = 154 - E (so |y| < 2^28), kept within the normal range
    const int E = (int)((st.dmax[P.o] >> 23) & 0xffu);
    const int es = max(-126, min(126, 154 - E));
    const float s = __uint_as_float((unsigned)(es + 127) << 23);    // 2^es
    const float is = __uint_as_float((unsigned)(127 - es) << 23);   // 2^-es
    const ff cf = to_ff(d2ff(ldexp(1.0 / ((double)kW12Den * D.h * D.h), -es)));   // units -> Delta_h d
    constexpr int kWc = (int)w12_centre3();
    constexpr int kW1 = (int)w12_int(1), kW2 = (int)w12_int(2), kW3 = (int)w12_int(3);
    constexpr int kW4 = (int)w12_int(4), kW5 = (int)w12_int(5), kW6 = (int)w12_int(6);
    const int kW[kHalf + 1] = {kWc, kW1, kW2, kW3, kW4, kW5, kW6};

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTileX + tx;
    const int nthr = kTileX * (kTileY / 2);
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const int gx = P.x0 + tx;
    const int gy0 = P.y0 + ty, gy1 = P.y0 + ty + kTileY / 2;
    const bool in0 = gx < D.nx && gy0 < D.ny, in1 = gx < D.nx && gy1 < D.ny;
    const long long c0 = gy0 * sy + gx, c1 = gy1 * sy + gx;
    int soff[kSlots];   // in-plane offsets of this thread's staged points (-1: outside)
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        const int e = tid + j * nthr;
        soff[j] = -1;
        if (e < kPX * kPY) {
            const int yy = e / kPX, xx = e - yy * kPX;
            int px = P.x0 - kHalf + xx, py = P.y0 - kHalf + yy;
            if (D.per & 1) px = wrap_coord(px, D.nx);
            if (D.per & 2) py = wrap_coord(py, D.ny);
            if (px >= 0 && px < D.nx && py >= 0 && py < D.ny) soff[j] = py * D.nx + px;
        }
    }
    IxPt q0[2 * kHalf + 1], q1[2 * kHalf + 1];
    const bool perz = (D.per & 4) != 0;
#pragma unroll
    for (int j = 0; j < 2 * kHalf; ++j) {
        int zz = P.z0 - kHalf + j;
        if (perz) zz = wrap_coord(zz, D.nz);
        const bool okz = zz >= 0 && zz < D.nz;
        q0[j] = ix_split((in0 && okz) ? d32[P.base + zz * sz + c0] : 0.f, s);
        q1[j] = ix_split((in1 && okz) ? d32[P.base + zz * sz + c1] : 0.f, s);
    }
    float pre[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? d32[P.base + P.z0 * sz + soff[j]] : 0.f;
    // r and x of this thread's two points, one plane ahead of their use
    constexpr bool xz = kXZ;
    const float2 f0 = make_float2(0.f, 0.f);
    float4 rx0 = make_float4(0.f, 0.f, 0.f, 0.f), rx1 = rx0;   // (r.h, r.l, x.h, x.l)
    if (in0) {
        const float2 rv = r[P.base + P.z0 * sz + c0], xv = xz ? f0 : x[P.base + P.z0 * sz + c0];
        rx0 = make_float4(rv.x, rv.y, xv.x, xv.y);
    }
    if (in1) {
        const float2 rv = r[P.base + P.z0 * sz + c1], xv = xz ? f0 : x[P.base + P.z0 * sz + c1];
        rx1 = make_float4(rv.x, rv.y, xv.x, xv.y);
    }
    IxPt* flat = &plane[0][0];
    float rrf = 0.f;
    for (int z = P.z0; z < P.z1; ++z) {
#pragma unroll
        for (int j = 0; j < kSlots; ++j) {
            const int e = tid + j * nthr;
            if (e < kPX * kPY) flat[e] = ix_split(pre[j], s);
        }
        {
            int zz = z + kHalf;
            if (perz) zz = wrap_coord(zz, D.nz);
            q0[2 * kHalf] = ix_split((in0 && zz < D.nz) ? d32[P.base + zz * sz + c0] : 0.f, s);
            q1[2 * kHalf] = ix_split((in1 && zz < D.nz) ? d32[P.base + zz * sz + c1] : 0.f, s);
        }
        __syncthreads();
        float4 nx0 = rx0, nx1 = rx1;
        if (z + 1 < P.z1) {
            const long long pz = P.base + (z + 1) * sz;
#pragma unroll
            for (int j = 0; j < kSlots; ++j) pre[j] = (soff[j] >= 0) ? d32[pz + soff[j]] : 0.f;
            if (in0) {
                const float2 rv = r[pz + c0], xv = xz ? f0 : x[pz + c0];
                nx0 = make_float4(rv.x, rv.y, xv.x, xv.y);
            }
            if (in1) {
                const float2 rv = r[pz + c1], xv = xz ? f0 : x[pz + c1];
                nx1 = make_float4(rv.x, rv.y, xv.x, xv.y);
            }
        }
        const int lx = tx + kHalf;
        const int ly[2] = {ty + kHalf, ty + kTileY / 2 + kHalf};
        const bool in[2] = {in0, in1};
        const long long cc[2] = {c0, c1};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const IxPt* qk = (k == 0) ? q0 : q1;
            long long I = (long long)kW[0] * qk[kHalf].h;
            float Lo = (float)kW[0] * qk[kHalf].l;
#pragma unroll
            for (int m = 1; m <= kHalf; ++m) {
                const IxPt a = plane[ly[k]][lx - m], b = plane[ly[k]][lx + m];
                const IxPt c = plane[ly[k] - m][lx], d = plane[ly[k] + m][lx];
                const IxPt e = qk[kHalf - m], f = qk[kHalf + m];
                const int hs = ((a.h + b.h) + (c.h + d.h)) + (e.h + f.h);
                const float ls = ((a.l + b.l) + (c.l + d.l)) + (e.l + f.l);
                I += (long long)kW[m] * hs;
                Lo = fmaf((float)kW[m], ls, Lo);
            }
            if (in[k]) {
                const long long g = P.base + z * sz + cc[k];
                // I + Lo in float-float (I's two leading float parts), times 2^-es / (831600 h^2)
                const ff ad = ff_mul(ix_to_ff(I, Lo), cf);   // Delta_h d, so r - A d = r + ad
                const float4 rx = (k == 0) ? rx0 : rx1;
                const ff rn = ff_add(ff{rx.x, rx.y}, ad);
                const float dc = (__int2float_rn(qk[kHalf].h) + qk[kHalf].l) * is;   // d at the point (exact)
                const ff xs = ff_two_sum(rx.z, dc);
                const ff xn = ff_quick(xs.h, xs.l + rx.w);
                r[g] = make_float2(rn.h, rn.l);
                x[g] = make_float2(xn.h, xn.l);
                r32[g] = rn.h;
                rrf += rn.h * rn.h;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 2 * kHalf; ++j) {
            q0[j] = q0[j + 1];
            q1[j] = q1[j + 1];
        }
        rx0 = nx0;
        rx1 = nx1;
    }
    if (tile_arrive(rrf, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[P.o] = 0;
            st.dmax[P.o] = 0u;   // every CTA of the orbital has read it (and xz)
            st.xz[P.o] = 0;      // x is stored now
            start_round(st, P.o, sum, tol2, inner_tol2, max_iter);
        }
    }
}

// The same update with its operands staged by the copy engine (blocks
// whose rows and offset are 16-byte aligned and that have no periodic
// direction: the zero fill of the copies is the zero ghost value).  A ring
// of kURing stages runs ahead of the z-march, each holding the plane z of d
// with its halo (48 x 28: x0 - 8 keeps the copy 16-byte aligned), d at
// plane z + 6 (32 x 16, the head of the register z-queues) and r and x at
// plane z (32 x 16 pairs).  Each plane's d is split once into shared memory
// (hi, lo; two buffers, so one barrier per plane serves both the split plane
// and the stage of the plane before); a thread owns the two points (x0 + 2 tx + a, y0 + ty), reads
// their x-window (14 values) and y-windows as 16-byte pairs and keeps their
// z-windows in registers.
constexpr int kUX = 48;                              // staged width: x0 - 8 .. x0 + 39
constexpr int kUY = kTileY + 2 * kHalf;              // 28: y0 - 6 .. y0 + 21
constexpr int kUPlane = kUX * kUY;                   // floats of the halo plane
constexpr int kUCtr = kTileX * kTileY;               // points of a centre tile
constexpr int kUStage = kUPlane + 5 * kUCtr;         // floats: plane, d head, r pairs, x pairs
constexpr int kURing = 5;
constexpr unsigned kUStageBytes = 4u * kUStage;

// the stages, two split planes (one barrier per plane), the stages' mbarriers
size_t update_tma_smem() { return 4 * (size_t)kURing * kUStage + 2 * sizeof(IxPt) * kUPlane + 8 * kURing + 128; }

template <bool kXZ>
__global__ void __launch_bounds__(256, 2) k_update12_tma(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                         const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                         const CUtensorMap* __restrict__ maps,
                                                         const float* __restrict__ d32, float2* __restrict__ r,
                                                         float2* __restrict__ x, float* __restrict__ r32,
                                                         double tol2, double inner_tol2, int max_iter, CgState st,
                                                         int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char us_raw[];
    unsigned char* smem = us_raw + ((128 - (tc_smem_addr(us_raw) & 127)) & 127);
    float* ring = reinterpret_cast<float*>(smem);
    IxPt* spb = reinterpret_cast<IxPt*>(smem + 4 * (size_t)kURing * kUStage);   // two split planes
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 4 * (size_t)kURing * kUStage + 2 * sizeof(IxPt) * kUPlane);
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o] || !L[P.b].utma) return;
    const LvlDesc& D = L[P.b];
    const CUtensorMap* mp = maps + 4 * P.b;   // d with halo, d centre, r pairs, x pairs
    const int oi = P.o - blk[P.b].orb0;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nzt = P.z1 - P.z0;
    constexpr bool xz = kXZ;   // x is zero and not stored yet: its tiles are not copied
    const int E = (int)((st.dmax[P.o] >> 23) & 0xffu);
    const int es = max(-126, min(126, 154 - E));
    const float sc = __uint_as_float((unsigned)(es + 127) << 23);   // 2^es
    const float is = __uint_as_float((unsigned)(127 - es) << 23);   // 2^-es
    const ff cf = to_ff(d2ff(ldexp(1.0 / ((double)kW12Den * D.h * D.h), -es)));
    constexpr int kWc = (int)w12_centre3();
    constexpr int kW1 = (int)w12_int(1), kW2 = (int)w12_int(2), kW3 = (int)w12_int(3);
    constexpr int kW4 = (int)w12_int(4), kW5 = (int)w12_int(5), kW6 = (int)w12_int(6);
    const int kW[kHalf + 1] = {kWc, kW1, kW2, kW3, kW4, kW5, kW6};
    auto issue = [&](int k) {
        uint64_t* b = bar + (k % kURing);
        float* sg = ring + (size_t)(k % kURing) * kUStage;
        const int zz = P.z0 + k;
        tc_mbar_expect_tx(b, xz ? kUStageBytes - 8u * kUCtr : kUStageBytes);
        tc_tma_load_4d(sg, mp + 0, P.x0 - 8, P.y0 - kHalf, zz, oi, b);
        tc_tma_load_4d(sg + kUPlane, mp + 1, P.x0, P.y0, zz + kHalf, oi, b);
        tc_tma_load_4d(sg + kUPlane + kUCtr, mp + 2, 2 * P.x0, P.y0, zz, oi, b);
        if (!xz) tc_tma_load_4d(sg + kUPlane + 3 * kUCtr, mp + 3, 2 * P.x0, P.y0, zz, oi, b);
    };
    if (tid == 0) {
        for (int k = 0; k < kURing; ++k) tc_mbar_init(bar + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < kURing && k < nzt; ++k) issue(k);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;   // 16 x 16
    const int gx = P.x0 + 2 * tx, gy = P.y0 + ty;
    const bool in = gx < D.nx && gy < D.ny;           // nx is a multiple of 4: gx + 1 < nx as well
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const long long col = gy * sy + gx;
    // z-windows of the two points as rings of 13 registers: plane z - 6 + j of
    // step k sits in slot (k + j) mod 13, so nothing moves between planes (the
    // z-loop is unrolled by 13 to make every slot index a constant)
    constexpr int kQ = 2 * kHalf + 1;
    IxPt q0[kQ], q1[kQ];
#pragma unroll
    for (int j = 0; j < 2 * kHalf; ++j) {
        const int zz = P.z0 - kHalf + j;
        float2 v = make_float2(0.f, 0.f);
        if (in && zz >= 0 && zz < D.nz) v = *reinterpret_cast<const float2*>(d32 + P.base + zz * sz + col);
        q0[j] = ix_split_w(v.x, sc);
        q1[j] = ix_split_w(v.y, sc);
    }
    float rrf = 0.f;
    const int ly = ty + kHalf, cx = 2 * tx + 8;       // the points' row and first column in the staged plane
    for (int k0 = 0; k0 < nzt; k0 += kQ) {
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
            const int k = k0 + u;
            if (k >= nzt) break;
            if (!tc_mbar_wait(bar + (k % kURing), (uint32_t)((k / kURing) & 1))) atomicOr(status + 3, 8);
            const float* sg = ring + (size_t)(k % kURing) * kUStage;
            IxPt* const sp = spb + (k & 1) * kUPlane;
            for (int e = tid; e < kUPlane; e += 256) sp[e] = ix_split_w(sg[e], sc);
            {
                const float2 hv = *reinterpret_cast<const float2*>(sg + kUPlane + ty * kTileX + 2 * tx);
                q0[(u + 2 * kHalf) % kQ] = ix_split_w(hv.x, sc);
                q1[(u + 2 * kHalf) % kQ] = ix_split_w(hv.y, sc);
            }
            // the split plane is written, and every thread has finished plane k - 1: its
            // stage takes plane k - 1 + kURing (the other split plane is free for plane k + 1)
            __syncthreads();
            if (tid == 0 && k >= 1 && k - 1 + kURing < nzt) {
                tc_fence_proxy_async();
                issue(k - 1 + kURing);
            }
            // x-window of row ly, columns cx - 6 .. cx + 7, as 7 pairs
            IxPt xw[2 * kHalf + 2];
#pragma unroll
            for (int k2 = 0; k2 < kHalf + 1; ++k2) {
                const int4 v = *reinterpret_cast<const int4*>(sp + ly * kUX + cx - kHalf + 2 * k2);
                xw[2 * k2] = {v.x, __int_as_float(v.y)};
                xw[2 * k2 + 1] = {v.z, __int_as_float(v.w)};
            }
            const IxPt c0 = q0[(u + kHalf) % kQ], c1 = q1[(u + kHalf) % kQ];
            long long I0 = (long long)kW[0] * c0.h, I1 = (long long)kW[0] * c1.h;
            float L0 = (float)kW[0] * c0.l, L1 = (float)kW[0] * c1.l;
#pragma unroll
            for (int m = 1; m <= kHalf; ++m) {
                const int4 uu = *reinterpret_cast<const int4*>(sp + (ly - m) * kUX + cx);   // rows ly -+ m
                const int4 ww = *reinterpret_cast<const int4*>(sp + (ly + m) * kUX + cx);
                const IxPt a0 = q0[(u + kHalf - m) % kQ], b0 = q0[(u + kHalf + m) % kQ];
                const IxPt a1 = q1[(u + kHalf - m) % kQ], b1 = q1[(u + kHalf + m) % kQ];
                const unsigned h0 = (((unsigned)xw[kHalf - m].h + (unsigned)xw[kHalf + m].h) +
                                     ((unsigned)uu.x + (unsigned)ww.x)) + ((unsigned)a0.h + (unsigned)b0.h);
                const unsigned h1 = (((unsigned)xw[kHalf + 1 - m].h + (unsigned)xw[kHalf + 1 + m].h) +
                                     ((unsigned)uu.z + (unsigned)ww.z)) + ((unsigned)a1.h + (unsigned)b1.h);
                const float l0 = ((xw[kHalf - m].l + xw[kHalf + m].l) +
                                  (__int_as_float(uu.y) + __int_as_float(ww.y))) + (a0.l + b0.l);
                const float l1 = ((xw[kHalf + 1 - m].l + xw[kHalf + 1 + m].l) +
                                  (__int_as_float(uu.w) + __int_as_float(ww.w))) + (a1.l + b1.l);
                I0 += (long long)kW[m] * (int)h0;
                I1 += (long long)kW[m] * (int)h1;
                L0 = fmaf((float)kW[m], l0, L0);
                L1 = fmaf((float)kW[m], l1, L1);
            }
            if (in) {
                const float4 rv = *reinterpret_cast<const float4*>(sg + kUPlane + kUCtr + ty * 2 * kTileX + 4 * tx);
                const float4 xv = xz ? make_float4(0.f, 0.f, 0.f, 0.f)
                                     : *reinterpret_cast<const float4*>(sg + kUPlane + 3 * kUCtr + ty * 2 * kTileX + 4 * tx);
                const long long g = P.base + (P.z0 + k) * sz + col;
                ff rn[2], xn[2];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const long long I = a == 0 ? I0 : I1;
                    const float Lo = a == 0 ? L0 : L1;
                    const IxPt qc = a == 0 ? c0 : c1;
                    const ff ad = ff_mul(ix_to_ff_b(I, Lo), cf);
                    rn[a] = ff_add(a == 0 ? ff{rv.x, rv.y} : ff{rv.z, rv.w}, ad);
                    const float dc = (__int2float_rn(qc.h) + qc.l) * is;
                    const ff xs = ff_two_sum(a == 0 ? xv.x : xv.z, dc);
                    xn[a] = ff_quick(xs.h, xs.l + (a == 0 ? xv.y : xv.w));
                    rrf += rn[a].h * rn[a].h;
                }
                *reinterpret_cast<float4*>(r + g) = make_float4(rn[0].h, rn[0].l, rn[1].h, rn[1].l);
                *reinterpret_cast<float4*>(x + g) = make_float4(xn[0].h, xn[0].l, xn[1].h, xn[1].l);
                *reinterpret_cast<float2*>(r32 + g) = make_float2(rn[0].h, rn[1].h);
            }
        }
    }
    if (tile_arrive(rrf, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[P.o] = 0;
            st.dmax[P.o] = 0u;
            st.xz[P.o] = 0;
            start_round(st, P.o, sum, tol2, inner_tol2, max_iter);
        }
    }
}

// Tensor maps of the update's operands, four per block, each a 4-D view
// (x, y, z, orbital): d with 48 x 28 boxes and 32 x 16 boxes, and the pair
// arrays r (b) and x as float32 rows of 2 nx values with 64 x 16 boxes.
// Blocks with a periodic direction, or whose rows or offset are not
// 16-byte aligned, keep k_update12_ix (flag utma = 0).  Returns the number
// of blocks on the copy-engine path.
int setup_update_maps(flosic_ctx* c) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return 0;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    std::vector<CUtensorMap> maps(4 * (size_t)c->nblk);
    std::vector<LvlDesc>& L0 = c->mg.h_lvl[0];
    int n_ok = 0;
    for (int b = 0; b < c->nblk; ++b) {
        const BlkDesc& B = c->blk[b];
        L0[b].utma = 0;
        if (B.nx % 4 != 0 || B.off % 4 != 0 || B.per != 0) continue;
        const cuuint64_t dims[4] = {(cuuint64_t)B.nx, (cuuint64_t)B.ny, (cuuint64_t)B.nz, (cuuint64_t)B.N};
        const cuuint64_t strides[3] = {(cuuint64_t)B.nx * 4, (cuuint64_t)B.nx * B.ny * 4, (cuuint64_t)B.G * 4};
        const cuuint64_t dims2[4] = {2 * (cuuint64_t)B.nx, (cuuint64_t)B.ny, (cuuint64_t)B.nz, (cuuint64_t)B.N};
        const cuuint64_t strides2[3] = {(cuuint64_t)B.nx * 8, (cuuint64_t)B.nx * B.ny * 8, (cuuint64_t)B.G * 8};
        const cuuint32_t box_halo[4] = {(cuuint32_t)kUX, (cuuint32_t)kUY, 1, 1};
        const cuuint32_t box_ctr[4] = {(cuuint32_t)kTileX, (cuuint32_t)kTileY, 1, 1};
        const cuuint32_t box_pair[4] = {2 * (cuuint32_t)kTileX, (cuuint32_t)kTileY, 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        float* d = c->ws.d32 + B.off;
        float* rb = reinterpret_cast<float*>(c->ws.b64 + B.off);
        float* xb = reinterpret_cast<float*>(c->ws.r64 + B.off);
        bool ok = true;
        auto enc = [&](CUtensorMap* m, void* base, const cuuint64_t* dm, const cuuint64_t* sd, const cuuint32_t* bx) {
            return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dm, sd, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        ok = enc(&maps[4 * b + 0], d, dims, strides, box_halo) && enc(&maps[4 * b + 1], d, dims, strides, box_ctr) &&
             enc(&maps[4 * b + 2], rb, dims2, strides2, box_pair) && enc(&maps[4 * b + 3], xb, dims2, strides2, box_pair);
        if (!ok) continue;
        L0[b].utma = 1;
        ++n_ok;
    }
    if (n_ok == 0) return 0;
    void* dm = nullptr;
    if (cudaMalloc(&dm, sizeof(CUtensorMap) * maps.size()) != cudaSuccess) return 0;
    c->allocations.push_back(dm);
    if (cudaMemcpy(dm, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_update12_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_tma_smem()) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_update12_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)update_tma_smem()) != cudaSuccess ||
        cudaMemcpy(c->mg.d_lvl[0], L0.data(), sizeof(LvlDesc) * c->nblk, cudaMemcpyHostToDevice) != cudaSuccess) {
        for (auto& D : L0) D.utma = 0;
        cudaMemcpy(c->mg.d_lvl[0], L0.data(), sizeof(LvlDesc) * c->nblk, cudaMemcpyHostToDevice);
        return 0;
    }
    c->d_umaps = dm;
    return n_ok;
}

// x += d32 in pairs for the orbitals still refining.
__global__ void __launch_bounds__(256) k_correct_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                    const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                    const float* __restrict__ d32, float2* __restrict__ x,
                                                    CgState st) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o]) return;
    const LvlDesc& D = L[P.b];
    tile_elementwise<float>(D, P, [&](long long g, int n) {
        if (n == 4) {
            const float4 d = *reinterpret_cast<const float4*>(d32 + g);
            float4 a = *reinterpret_cast<float4*>(x + g);       // pairs g, g+1
            float4 c = *reinterpret_cast<float4*>(x + g + 2);   // pairs g+2, g+3
            ff s;
            s = ff_two_sum(a.x, d.x); s = ff_quick(s.h, s.l + a.y); a.x = s.h; a.y = s.l;
            s = ff_two_sum(a.z, d.y); s = ff_quick(s.h, s.l + a.w); a.z = s.h; a.w = s.l;
            s = ff_two_sum(c.x, d.z); s = ff_quick(s.h, s.l + c.y); c.x = s.h; c.y = s.l;
            s = ff_two_sum(c.z, d.w); s = ff_quick(s.h, s.l + c.w); c.z = s.h; c.w = s.l;
            *reinterpret_cast<float4*>(x + g) = a;
            *reinterpret_cast<float4*>(x + g + 2) = c;
        } else {
            const float2 v = x[g];
            ff s = ff_two_sum(v.x, d32[g]);
            s = ff_quick(s.h, s.l + v.y);
            x[g] = make_float2(s.h, s.l);
        }
    });
}

// V = x (pairs joined into float64), every orbital.
__global__ void __launch_bounds__(256) k_join_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                 const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                 const float2* __restrict__ x, const int* __restrict__ xz,
                                                 double* __restrict__ V) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    if (xz[P.o]) {   // never updated (no solve needed): V = 0
        tile_elementwise<float>(D, P, [&](long long g, int n) {
            for (int k = 0; k < n; ++k) V[g + k] = 0.0;
        });
        return;
    }
    tile_elementwise<float>(D, P, [&](long long g, int n) {
        if (n == 4) {   // aligned group of four points: 16-byte accesses
            const float4 a = *reinterpret_cast<const float4*>(x + g);
            const float4 c = *reinterpret_cast<const float4*>(x + g + 2);
            *reinterpret_cast<double2*>(V + g) = make_double2(ff2d(make_float2(a.x, a.y)), ff2d(make_float2(a.z, a.w)));
            *reinterpret_cast<double2*>(V + g + 2) =
                make_double2(ff2d(make_float2(c.x, c.y)), ff2d(make_float2(c.z, c.w)));
            return;
        }
        for (int k = 0; k < n; ++k) V[g + k] = ff2d(x[g + k]);
    });
}

static dim3 tile_threads() { return dim3(kTileX, kTileY / 2); }

// x is the solution in pairs (float2 per point), p32 may be null.
void launch_ff_init(flosic_ctx* c, const double* b, const double* V, bool warm, bool keep_zero, float2* x,
                    float* p32, double tol2, double inner_tol2, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_ff_init<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, reinterpret_cast<const float2*>(b), V, x, c->ws.r32, p32,
        c->ws.d32, warm ? 1 : 0, keep_zero ? 1 : 0, tol2, inner_tol2, c->opt.max_iter, c->ws.cg);
    note_launch(c);
}

void launch_residual_ff(flosic_ctx* c, const double* b, const float2* x, float* p32, double tol2,
                        double inner_tol2, bool store_r, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_residual12_ff<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, reinterpret_cast<float2*>(const_cast<double*>(b)), x,
        c->ws.r32, p32, c->ws.d32, tol2, inner_tol2, c->opt.max_iter, store_r ? 1 : 0, c->ws.cg);
    note_launch(c);
}

// x_zero: the first update after a cold start that stored no x
void launch_update_ff(flosic_ctx* c, double* r, float2* x, bool x_zero, double tol2, double inner_tol2,
                      cudaStream_t s) {
    const Multigrid& M = c->mg;
    if (c->kron.n_simt > 0) {   // the tensor-core passes record max |d| themselves
        k_dmax<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk,
                                                                c->ws.d32, c->ws.cg);
        note_launch(c);
    }
    if (c->n_utma_blocks > 0) {   // blocks whose operands the copy engine stages
        auto kern = x_zero ? k_update12_tma<true> : k_update12_tma<false>;
        kern<<<(unsigned)M.ntiles[0], dim3(kTileX / 2, kTileY), update_tma_smem(), s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, (const CUtensorMap*)c->d_umaps, c->ws.d32,
            reinterpret_cast<float2*>(r), x, c->ws.r32, tol2, inner_tol2, c->opt.max_iter, c->ws.cg, c->ws.status);
        note_launch(c);
    }
    if (c->n_utma_blocks < c->nblk) {   // the rest: plain loads
        auto kern = x_zero ? k_update12_ix<true> : k_update12_ix<false>;
        kern<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(
            c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, reinterpret_cast<float2*>(r), x, c->ws.r32, c->ws.d32,
            tol2, inner_tol2, c->opt.max_iter, c->ws.cg);
        note_launch(c);
    }
}

void launch_correct_ff(flosic_ctx* c, float2* x, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_correct_ff<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk,
                                                                  c->ws.d32, x, c->ws.cg);
    note_launch(c);
}

void launch_join_ff(flosic_ctx* c, const float2* x, double* V, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_join_ff<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, x,
                                                               c->ws.cg.xz, V);
    note_launch(c);
}

}  // namespace flosic
