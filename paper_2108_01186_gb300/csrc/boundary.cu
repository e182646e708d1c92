// Right-hand side of the per-orbital Poisson problems (Sec. II.A: Dirichlet
// values of the potential from a multipole expansion, isolated systems; a
// dipole correction for slabs; periodic cells take a neutralising
// background instead of ghost values).
//
// With the ghost values known, -Delta_h V = 4 pi rho becomes
//   A V = 4 pi rho + bc,  bc(g) = (1/h^2) sum_{taps of g outside} w_m V_b(R_tap),
//   V_b(R) = sum_k mom_k beta_k(R),
//   beta = {1/R, R_x/R^3, R_y/R^3, R_z/R^3, R_x^2/2R^5, R_y^2/2R^5, R_z^2/2R^5,
//           R_x R_y/R^5, R_x R_z/R^5, R_y R_z/R^5}
// for the moments mom = {Q, p, Theta_xx, Theta_yy, Theta_zz, Theta_xy,
// Theta_xz, Theta_yz} of rho about the box centre.  bc is linear in the
// moments with coefficients that depend only on the grid:
//   bc(g) = sum_k mom_k B_k(g),  B_k(g) = (1/h^2) sum_taps w_m beta_k(R_tap).
// B is computed once per context for the points within 6 of a face (the only
// points with ghost taps); a step then needs one pass for 4 pi rho and the
// moments, and 10 multiply-adds per boundary point and orbital.  The exact
// Poisson adjoint uses the same B: its transpose gives sum_g W_g B_k(g).
#include "internal.cuh"

namespace flosic {

__constant__ double c_wb[kHalf + 1];

cudaError_t upload_boundary_constants() {
    double w[kHalf + 1];
    stencil_weights(w);
    return cudaMemcpyToSymbol(c_wb, w, sizeof(w));
}

// One thread per boundary point of one block: B[j][0..9].
__global__ void k_bnd_coef(const BlkDesc* __restrict__ blk, int b, const int* __restrict__ bidx,
                           double* __restrict__ bcoef) {
    const BlkDesc& B = blk[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.nbnd) return;
    const int g = bidx[B.bnd0 + j];
    const int pl = B.nx * B.ny;
    const int z = g / pl, rem = g - z * pl, y = rem / B.nx, x = rem - y * B.nx;
    const int p[3] = {x, y, z};
    const int n[3] = {B.nx, B.ny, B.nz};
    const double ih2 = 1.0 / (B.h * B.h);
    double cf[10];
    for (int k = 0; k < 10; ++k) cf[k] = 0.0;
    // slab: periodic along x and y, ghost planes along z hold
    // V_b(Z) = -(2 pi/A)(Q |Z| - sgn(Z) p_z), linear in mom[0] = Q and mom[3] = p_z
    const bool slab = (B.per == 3);
    const double area = (double)B.nx * B.ny * B.h * B.h;
    for (int d = 0; d < 3; ++d)
        for (int m = 1; m <= kHalf; ++m)
            for (int sg = -1; sg <= 1; sg += 2) {
                if ((B.per >> d) & 1) continue;   // periodic direction: the tap wraps, no ghost value
                const int qd = p[d] + sg * m;
                if (qd >= 0 && qd < n[d]) continue;
                if (slab) {
                    const double Z = B.oz + B.h * qd - B.cz;
                    const double f = c_wb[m] * ih2 * (2.0 * kPi / area);
                    cf[0] -= f * fabs(Z);
                    cf[3] += f * (Z > 0.0 ? 1.0 : -1.0);
                    continue;
                }
                int q[3] = {x, y, z};
                q[d] = qd;
                const double Rx = B.ox + B.h * q[0] - B.cx, Ry = B.oy + B.h * q[1] - B.cy,
                             Rz = B.oz + B.h * q[2] - B.cz;
                const double ir = rsqrt(Rx * Rx + Ry * Ry + Rz * Rz);
                const double ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
                const double f = c_wb[m] * ih2;
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
    double* out = bcoef + (B.bnd0 + (long long)j) * 10;
    for (int k = 0; k < 10; ++k) out[k] = cf[k];
}

cudaError_t setup_boundary(flosic_ctx* c) {
    for (int b = 0; b < c->nblk; ++b) {
        const int nb = c->blk[b].nbnd;
        if (nb == 0) continue;
        k_bnd_coef<<<(nb + 255) / 256, 256>>>(c->d_blk, b, c->d_bidx, c->d_bcoef);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

// Last tile of an orbital: the ten moments from the per-tile partials
// (fixed order), times dV.
__device__ __forceinline__ void gather_moments(const TilePos& P, const LvlDesc& D, const BlkDesc& B,
                                               const double* __restrict__ mom_part, double* __restrict__ mom,
                                               unsigned* __restrict__ count, double* scratch) {
    __shared__ bool last;
    if (linear_tid() == 0) {
        __threadfence();
        last = (atomicAdd(count + P.o, 1u) == (unsigned)(D.ntile - 1));
    }
    __syncthreads();
    if (last) {
        for (int k = 0; k < 10; ++k) {
            double v = 0.0;
            for (int t = linear_tid(); t < D.ntile; t += blockDim.x * blockDim.y)
                v += __ldcg(mom_part + (P.first + t) * 10 + k);
            v = block_sum(v, scratch);
            if (linear_tid() == 0) mom[P.o * 10 + k] = v * B.dV;
        }
        if (linear_tid() == 0) count[P.o] = 0;
    }
}

// packed two-lane a - b and -a (exact: a product with -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

// Pass 1 over the tiles: b = scale * phi^2 and (for the multipole boundary)
// the l <= 2 moments of phi^2 per orbital.  Per column (x, y) the z-sums
// S0 = sum rho, S1 = sum rho Z, S2 = sum rho Z^2 give all ten moments.
__global__ void __launch_bounds__(256) k_rhs_bulk(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                  const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                  const double* __restrict__ phi, double scale, int want_mom,
                                                  double* __restrict__ b, double* __restrict__ mom_part,
                                                  double* __restrict__ mom, unsigned* __restrict__ count,
                                                  const int* __restrict__ mask) {
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!mask[P.o]) return;   // an orbital this context does not solve (every CTA of it returns)
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    const int x = P.x0 + threadIdx.x;
    for (int k = 0; k < 2; ++k) {
        const int y = P.y0 + threadIdx.y + k * (kTileY / 2);
        if (x >= D.nx || y >= D.ny) continue;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int z = P.z0; z < P.z1; ++z) {
            const long long g = P.base + ((long long)z * D.ny + y) * D.nx + x;
            const double v = phi[g];
            const double rho = v * v;
            b[g] = scale * rho;
            const double Z = B.oz + B.h * z - B.cz;
            s0 += rho;
            s1 += rho * Z;
            s2 += rho * Z * Z;
        }
        const double X = B.ox + B.h * x - B.cx, Y = B.oy + B.h * y - B.cy;
        const double sxx = X * X * s0, syy = Y * Y * s0, r2 = sxx + syy + s2;
        m[0] += s0;
        m[1] += X * s0;
        m[2] += Y * s0;
        m[3] += s1;
        m[4] += 3.0 * sxx - r2;
        m[5] += 3.0 * syy - r2;
        m[6] += 3.0 * s2 - r2;
        m[7] += 3.0 * X * Y * s0;
        m[8] += 3.0 * X * s1;
        m[9] += 3.0 * Y * s1;
    }
    if (!want_mom) return;
    for (int k = 0; k < 10; ++k) {
        const double s = block_sum(m[k], scratch);
        if (linear_tid() == 0) mom_part[(long long)blockIdx.x * 10 + k] = s;
    }
    gather_moments(P, D, B, mom_part, mom, count, scratch);
}

// The same pass for the mixed-precision path: b is written as float-float
// pairs (rho = phi^2 to ~48 bits) and the moments are accumulated as pairs,
// so they match the float64 pass to ~1e-13 while no float64 operation runs
// per grid point.
__global__ void __launch_bounds__(256, 2) k_rhs_bulk_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                     const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                     const double* __restrict__ phi, double scale, int want_mom,
                                                     float2* __restrict__ b, double* __restrict__ mom_part,
                                                     double* __restrict__ mom, unsigned* __restrict__ count,
                                                     const int* __restrict__ mask) {
    __shared__ double scratch[32];
    __shared__ float2 red[10][256];   // per-thread moment pairs
    __shared__ float2 red2[10][16];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!mask[P.o]) return;   // an orbital this context does not solve (every CTA of it returns)
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    ff m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = {0.f, 0.f};
    const ff sc = to_ff(d2ff(scale)), hz = to_ff(d2ff(B.h));
    const int x = P.x0 + threadIdx.x;
    const long long plane = (long long)D.ny * D.nx;
    constexpr int kZU = 4;   // z loads per column a thread has in flight before their products
    // The thread's two columns (x, y_0) and (x, y_0 + 8) side by side: lane a
    // of every float2 is column a, and each float operation of the pair
    // arithmetic runs on both columns at once (packed two-lane instructions,
    // the same IEEE operations per lane as the one-column form).
    // q_n = sum rho k^n over a column's points, k = z - z0 = 0, 1, ...
    // (non-negative terms, so the pairs need no renormalisation per point);
    // the z-moments about the centre follow once per column below.
    const int yc[2] = {P.y0 + (int)threadIdx.y, P.y0 + (int)threadIdx.y + kTileY / 2};
    const bool inc[2] = {x < D.nx && yc[0] < D.ny, x < D.nx && yc[1] < D.ny};
    float2 q0h = make_float2(0.f, 0.f), q0l = q0h, q1h = q0h, q1l = q0h, q2h = q0h, q2l = q0h;
    if (inc[0] || inc[1]) {
        const float2 sch = make_float2(sc.h, sc.h), scl = make_float2(sc.l, sc.l), two = make_float2(2.f, 2.f);
        const long long dy = (long long)(kTileY / 2) * D.nx;   // column 1 lies 8 rows after column 0
        float2 kf = make_float2(0.f, 0.f);
        const float2 one = make_float2(1.f, 1.f);
        long long g = P.base + ((long long)P.z0 * D.ny + yc[0]) * D.nx + x;
        for (int z = P.z0; z < P.z1; z += kZU, g += kZU * plane) {
            double pv0[kZU], pv1[kZU];
#pragma unroll
            for (int u = 0; u < kZU; ++u) {
                pv0[u] = (inc[0] && z + u < P.z1) ? __ldcs(phi + g + u * plane) : 0.0;
                pv1[u] = (inc[1] && z + u < P.z1) ? __ldcs(phi + g + dy + u * plane) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kZU; ++u) {
                if (z + u >= P.z1) break;
                const float2 f0 = d2ff(pv0[u]), f1 = d2ff(pv1[u]);
                const float2 fx = make_float2(f0.x, f1.x), fy = make_float2(f0.y, f1.y);
                // rho = phi^2 as pairs
                const float2 ph = __fmul2_rn(fx, fx);
                const float2 pe = __fadd2_rn(__ffma2_rn(fx, fx, neg2(ph)), __fmul2_rn(__fmul2_rn(two, fx), fy));
                const float2 rh = __fadd2_rn(ph, pe);
                const float2 rl = sub2(pe, sub2(rh, ph));
                // b = sc rho
                const float2 bp = __fmul2_rn(sch, rh);
                float2 be = __ffma2_rn(sch, rh, neg2(bp));
                be = __ffma2_rn(sch, rl, be);
                be = __ffma2_rn(scl, rh, be);
                const float2 bh = __fadd2_rn(bp, be);
                const float2 bl = sub2(be, sub2(bh, bp));
                if (inc[0]) __stcs(b + g + u * plane, make_float2(bh.x, bl.x));
                if (inc[1]) __stcs(b + g + dy + u * plane, make_float2(bh.y, bl.y));
                // rho k and rho k^2 as unnormalised pairs
                const float2 t1 = __fmul2_rn(rh, kf);
                const float2 e1 = __ffma2_rn(rl, kf, __ffma2_rn(rh, kf, neg2(t1)));
                const float2 t2 = __fmul2_rn(t1, kf);
                const float2 e2 = __ffma2_rn(e1, kf, __ffma2_rn(t1, kf, neg2(t2)));
                // q += term: exact two-sum of the high parts, the rest gathered in the low part
                auto acc = [&](float2& qh, float2& ql, float2 th, float2 tl) {
                    const float2 sh = __fadd2_rn(qh, th);
                    const float2 bb = sub2(sh, qh);
                    const float2 er = __fadd2_rn(sub2(qh, sub2(sh, bb)), sub2(th, bb));
                    ql = __fadd2_rn(ql, __fadd2_rn(er, tl));
                    qh = sh;
                };
                acc(q0h, q0l, rh, rl);
                acc(q1h, q1l, t1, e1);
                acc(q2h, q2l, t2, e2);
                kf = __fadd2_rn(kf, one);
            }
        }
    }
    const ff Z0 = to_ff(d2ff(B.oz + B.h * P.z0 - B.cz));
    for (int k = 0; k < 2; ++k) {
        if (!inc[k]) continue;
        const int y = yc[k];
        // Z = Z0 + h k:  S0 = q0, S1 = Z0 q0 + h q1, S2 = Z0 (Z0 q0 + 2 h q1) + h^2 q2
        const ff q0 = ff_quick(k ? q0h.y : q0h.x, k ? q0l.y : q0l.x);
        const ff q1 = ff_quick(k ? q1h.y : q1h.x, k ? q1l.y : q1l.x);
        const ff q2 = ff_quick(k ? q2h.y : q2h.x, k ? q2l.y : q2l.x);
        const ff hq1 = ff_mul(hz, q1), z0q0 = ff_mul(Z0, q0);
        const ff s0 = q0;
        const ff s1 = ff_add(z0q0, hq1);
        const ff s2 = ff_add(ff_mul(Z0, ff_add(z0q0, ff_mulf(hq1, 2.f))), ff_mul(ff_mul(hz, hz), q2));
        const ff X = to_ff(d2ff(B.ox + B.h * x - B.cx)), Y = to_ff(d2ff(B.oy + B.h * y - B.cy));
        const ff sxx = ff_mul(ff_mul(X, X), s0), syy = ff_mul(ff_mul(Y, Y), s0);
        const ff r2 = ff_add(ff_add(sxx, syy), s2);
        const ff mr2 = {-r2.h, -r2.l};
        m[0] = ff_add(m[0], s0);
        m[1] = ff_add(m[1], ff_mul(X, s0));
        m[2] = ff_add(m[2], ff_mul(Y, s0));
        m[3] = ff_add(m[3], s1);
        m[4] = ff_add(m[4], ff_add(ff_mulf(sxx, 3.f), mr2));
        m[5] = ff_add(m[5], ff_add(ff_mulf(syy, 3.f), mr2));
        m[6] = ff_add(m[6], ff_add(ff_mulf(s2, 3.f), mr2));
        m[7] = ff_add(m[7], ff_mulf(ff_mul(ff_mul(X, Y), s0), 3.f));
        m[8] = ff_add(m[8], ff_mulf(ff_mul(X, s1), 3.f));
        m[9] = ff_add(m[9], ff_mulf(ff_mul(Y, s1), 3.f));
    }
    if (!want_mom) return;
    // CTA sums of the ten pairs in a fixed order: 16 threads per moment add
    // 16 values each, then one thread per moment adds their 16 partials
    const int tid = linear_tid();
#pragma unroll
    for (int k = 0; k < 10; ++k) red[k][tid] = make_float2(m[k].h, m[k].l);
    __syncthreads();
    if (tid < 160) {
        const int k = tid >> 4, p = tid & 15;
        ff v = to_ff(red[k][p]);
        for (int q = 1; q < 16; ++q) v = ff_add(v, to_ff(red[k][p + 16 * q]));
        red2[k][p] = make_float2(v.h, v.l);
    }
    __syncthreads();
    if (tid < 10) {
        ff v = to_ff(red2[tid][0]);
        for (int q = 1; q < 16; ++q) v = ff_add(v, to_ff(red2[tid][q]));
        mom_part[(long long)blockIdx.x * 10 + tid] = ff_to_double(v);
    }
    __syncthreads();
    gather_moments(P, D, B, mom_part, mom, count, scratch);
}

// Pass 2: b[g_j] += sum_k mom_k B_k(g_j) for every boundary point of every
// orbital (thread per boundary point, looping over the block's orbitals).
// kFF: b holds float-float pairs and the boundary term is formed in pairs
// (it carries most of ||b||, so it needs the full ~48 bits).
template <bool kFF>
__global__ void k_rhs_bc(const BlkDesc* __restrict__ blk, int b, const int* __restrict__ bidx,
                         const double* __restrict__ bcoef, const double* __restrict__ mom,
                         double* __restrict__ rhs) {
    const BlkDesc& B = blk[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (kFF) {   // the block's moments as pairs, converted once per CTA
        extern __shared__ float2 mom_ff[];
        for (int e = threadIdx.x; e < 10 * B.N; e += blockDim.x) mom_ff[e] = d2ff(mom[B.orb0 * 10 + e]);
        __syncthreads();
        if (j >= B.nbnd) return;
        const int g = bidx[B.bnd0 + j];
        const double* src = bcoef + (B.bnd0 + (long long)j) * 10;
        ff cf[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) cf[k] = to_ff(d2ff(src[k]));
        float2* rp = reinterpret_cast<float2*>(rhs);
        for (int i = 0; i < B.N; ++i) {
            const float2* mo = mom_ff + i * 10;
            ff acc = {0.f, 0.f};   // unnormalised products gathered by ff_acc (error ~2^-44 sum |terms|)
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                const float2 m = mo[k];
                const float p = m.x * cf[k].h;
                acc = ff_acc(acc, p, fmaf(m.x, cf[k].l, fmaf(m.y, cf[k].h, fmaf(m.x, cf[k].h, -p))));
            }
            const long long idx = B.off + (long long)i * B.G + g;
            const ff v = ff_add(to_ff(rp[idx]), ff_quick(acc.h, acc.l));
            rp[idx] = make_float2(v.h, v.l);
        }
    } else {
        if (j >= B.nbnd) return;
        const int g = bidx[B.bnd0 + j];
        const double* src = bcoef + (B.bnd0 + (long long)j) * 10;
        double cf[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) cf[k] = src[k];
        for (int i = 0; i < B.N; ++i) {
            const double* mo = mom + (B.orb0 + i) * 10;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 10; ++k) acc += mo[k] * cf[k];
            rhs[B.off + (long long)i * B.G + g] += acc;
        }
    }
}

// Periodic cells: b -= 4 pi Q / (G dV), the uniform background that
// neutralises each orbital density (b in pairs, Q = mom[0]).
__global__ void __launch_bounds__(256) k_rhs_neutralise_ff(const BlkDesc* __restrict__ blk,
                                                           const LvlDesc* __restrict__ L,
                                                           const int4* __restrict__ tiles,
                                                           const int* __restrict__ orb_blk,
                                                           const double* __restrict__ mom, float2* __restrict__ b) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    const ff sh = to_ff(d2ff(-4.0 * kPi * mom[P.o * 10] / ((double)B.G * B.dV)));   // once per CTA
    tile_elementwise<float>(D, P, [&](long long g, int n) {
        for (int k = 0; k < n; ++k) {
            const ff v = ff_add(to_ff(b[g + k]), sh);
            b[g + k] = make_float2(v.h, v.l);
        }
    });
}

void launch_rhs(flosic_ctx* c, const double* phi, bool with_bc, double* b, cudaStream_t s) {
    const Multigrid& M = c->mg;
    const bool ff = (c->opt.precision == FLOSIC_MIXED);
    const double scale = with_bc ? 4.0 * kPi : 1.0;
    const dim3 tb(kTileX, kTileY / 2);
    if (ff)
        k_rhs_bulk_ff<<<(unsigned)M.ntiles[0], tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, phi,
                                                           scale, with_bc ? 1 : 0, reinterpret_cast<float2*>(b),
                                                           c->ws.mom_part, c->ws.mom, c->ws.cg.count, c->ws.mask);
    else
        k_rhs_bulk<<<(unsigned)M.ntiles[0], tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, phi, scale,
                                                        with_bc ? 1 : 0, b, c->ws.mom_part, c->ws.mom, c->ws.cg.count,
                                                        c->ws.mask);
    note_launch(c);
    if (!with_bc) return;
    if (c->opt.boundary == FLOSIC_BC_PERIODIC) {   // mixed precision only (validated)
        k_rhs_neutralise_ff<<<(unsigned)M.ntiles[0], tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk,
                                                                 c->ws.mom, reinterpret_cast<float2*>(b));
        note_launch(c);
        return;
    }
    for (int k = 0; k < c->nblk; ++k) {
        const int nb = c->blk[k].nbnd;
        if (nb == 0) continue;
        if (ff)
            k_rhs_bc<true><<<(nb + 127) / 128, 128, sizeof(float2) * 10 * c->blk[k].N, s>>>(c->d_blk, k, c->d_bidx,
                                                                                       c->d_bcoef, c->ws.mom, b);
        else
            k_rhs_bc<false><<<(nb + 127) / 128, 128, 0, s>>>(c->d_blk, k, c->d_bidx, c->d_bcoef, c->ws.mom, b);
        note_launch(c);
    }
}

// Exact Poisson adjoint: c_k = sum_g W_g B_k(g) per orbital (K^T of the
// boundary map, before spreading with the moment weights).
__global__ void k_bcadj_coef(const BlkDesc* __restrict__ blk, int b, const int* __restrict__ bidx,
                             const double* __restrict__ bcoef, const double* __restrict__ W,
                             double* __restrict__ coef) {
    __shared__ double scratch[32];
    const BlkDesc& B = blk[b];
    const int i = blockIdx.x;   // orbital within the block
    double acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    const double* w = W + B.off + (long long)i * B.G;
    for (int j = threadIdx.x; j < B.nbnd; j += blockDim.x) {
        const double wv = w[bidx[B.bnd0 + j]];
        const double* cf = bcoef + (B.bnd0 + (long long)j) * 10;
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] += wv * cf[k];
    }
    for (int k = 0; k < 10; ++k) {
        const double v = block_sum(acc[k], scratch);
        if (threadIdx.x == 0) coef[(B.orb0 + i) * 10 + k] = v;
    }
}

// veff = (V + G^T rho)/2, G^T rho = 4 pi W + dV sum_k c_k mbasis_k(R), with the
// moment weights mbasis = {1, R, 3RR - R^2 I (xx, yy, zz), 3 R_x R_y, ...};
// writes V^SIC of the exact adjoint, -(veff + v_xc) = vsic + V - veff.
__global__ void __launch_bounds__(256) k_veff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                              const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                              const double* __restrict__ W, const double* __restrict__ V,
                                              const double* __restrict__ coef, const double* __restrict__ vsic,
                                              double* __restrict__ out) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    double c[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) c[k] = coef[P.o * 10 + k];
    const int x = P.x0 + threadIdx.x;
    for (int k = 0; k < 2; ++k) {
        const int y = P.y0 + threadIdx.y + k * (kTileY / 2);
        if (x >= D.nx || y >= D.ny) continue;
        const double Rx = B.ox + B.h * x - B.cx, Ry = B.oy + B.h * y - B.cy;
        for (int z = P.z0; z < P.z1; ++z) {
            const double Rz = B.oz + B.h * z - B.cz;
            const double r2 = Rx * Rx + Ry * Ry + Rz * Rz;
            const double kt = c[0] + c[1] * Rx + c[2] * Ry + c[3] * Rz + c[4] * (3 * Rx * Rx - r2) +
                              c[5] * (3 * Ry * Ry - r2) + c[6] * (3 * Rz * Rz - r2) + c[7] * 3 * Rx * Ry +
                              c[8] * 3 * Rx * Rz + c[9] * 3 * Ry * Rz;
            const long long g = P.base + ((long long)z * D.ny + y) * D.nx + x;
            const double veff = 0.5 * (V[g] + 4.0 * kPi * W[g] + B.dV * kt);
            out[g] = vsic[g] + V[g] - veff;
        }
    }
}

void launch_bc_adjoint(flosic_ctx* c, const double* W, const double* V, double* out, cudaStream_t s) {
    for (int k = 0; k < c->nblk; ++k) {
        k_bcadj_coef<<<c->blk[k].N, 256, 0, s>>>(c->d_blk, k, c->d_bidx, c->d_bcoef, W, c->ws.mom); note_launch(c);
    }
    const Multigrid& M = c->mg;
    k_veff<<<(unsigned)M.ntiles[0], dim3(kTileX, kTileY / 2), 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk,
                                                                       W, V, c->ws.mom, c->ws.vsic, out); note_launch(c);
}

}  // namespace flosic
