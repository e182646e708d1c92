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
#include "ffsweep.cuh"

namespace flosic {


cudaError_t upload_ff_weights() { return upload_ffsweep_weights(); }

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
// and the first float32 solve starts here.
__global__ void __launch_bounds__(256) k_ff_init(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                 const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                 const float2* __restrict__ b, const double* __restrict__ V,
                                                 float2* __restrict__ x, float* __restrict__ r32,
                                                 float* __restrict__ p32, float* __restrict__ d32, int warm,
                                                 double tol2, double inner_tol2, int max_iter, CgState st) {
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
                *reinterpret_cast<float4*>(x + g) = z4;
                *reinterpret_cast<float4*>(x + g + 2) = z4;
                *reinterpret_cast<float4*>(r32 + g) = bh;
                *reinterpret_cast<float4*>(d32 + g) = z4;
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
                x[g + k] = make_float2(0.f, 0.f);
                r32[g + k] = bh;
                d32[g + k] = 0.f;
                if (p32) p32[g + k] = bh;
            }
        }
    });
    if (tile_arrive(bb, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
        const double sum = tile_gather(st.part, P.first, D.ntile, scratch);
        if (linear_tid() == 0) {
            st.count[P.o] = 0;
            st.bb[P.o] = sum;
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

// One refinement round's update from the float32 correction d of the inner
// solve: r -= A d (r in pairs, in place: r_{k+1} = b - A x_{k+1} =
// r_k - A d_k), x += d (pairs), r32 = float(r), and the next round's start.
// The operand of the sweep is d itself, a float32 field, so the stencil sums
// run on plain floats.  d is left as it is (neighbouring tiles read it as
// halo): this serves inner solvers that overwrite d (the Kronecker-product
// solve), not those that start from d = 0.
__global__ void __launch_bounds__(256) k_update12_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     float2* __restrict__ r, float2* __restrict__ x,
                                                     float* __restrict__ r32, const float* __restrict__ d32,
                                                     double tol2, double inner_tol2, int max_iter, CgState st) {
    __shared__ float plane[kPY][kPX];
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.oactive[P.o]) return;
    const LvlDesc& D = L[P.b];
    const ff ih2 = to_ff(d2ff(1.0 / (D.h * D.h)));   // once per CTA
    float rrf = 0.f;
    ff_sweep12_f(
        D, P, [&](long long g) { return d32[g]; },
        [&](long long g, float dc, ff acc) {
            // acc = h^2 Delta_h d, so r - A d = r + acc / h^2
            const ff rn = ff_add(to_ff(r[g]), ff_mul(acc, ih2));
            const float2 xv = x[g];
            const ff xs = ff_two_sum(xv.x, dc);
            const ff xn = ff_quick(xs.h, xs.l + xv.y);
            r[g] = make_float2(rn.h, rn.l);
            x[g] = make_float2(xn.h, xn.l);
            r32[g] = rn.h;
            rrf += rn.h * rn.h;
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
                                                 const float2* __restrict__ x, double* __restrict__ V) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
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
void launch_ff_init(flosic_ctx* c, const double* b, const double* V, bool warm, float2* x, float* p32,
                    double tol2, double inner_tol2, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_ff_init<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk,
                                                               reinterpret_cast<const float2*>(b), V, x, c->ws.r32, p32, c->ws.d32, warm ? 1 : 0, tol2,
                                                               inner_tol2, c->opt.max_iter, c->ws.cg);
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

void launch_update_ff(flosic_ctx* c, double* r, float2* x, double tol2, double inner_tol2, cudaStream_t s) {
    const Multigrid& M = c->mg;
    k_update12_ff<<<(unsigned)M.ntiles[0], tile_threads(), 0, s>>>(
        c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, reinterpret_cast<float2*>(r), x, c->ws.r32, c->ws.d32,
        tol2, inner_tol2, c->opt.max_iter, c->ws.cg);
    note_launch(c);
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
                                                               V);
    note_launch(c);
}

}  // namespace flosic
