// Fermi-Loewdin orbitals (Sec. I.B, Eqs. 6-8; Sec. II.B) and the reverse
// mode of that map for the FOD gradient (Eqs. 9-11).
//
// Forward, per spin block with N orbitals on G points:
//   interpolation: v_ia = psi_a(a_i) and grad psi_a(a_i) (tricubic Lagrange)
//   Gram:          M = dV psi psi^T            (grid contraction, K = G)
//   small:         rho_i = sum_a v_ia^2, T = v / sqrt(rho), S = T M T^T
//                  (= dV F F^T with F = T psi), S = U L U^T (Jacobi),
//                  Q = S^{-1/2} = U L^{-1/2} U^T, C = Q T
//   apply:         phi = C psi                 (N x N times N x G)
// F itself is never stored: phi = Q F = (Q T) psi.
//
// Reverse, with Phibar_i = dE/dphi_i = 2 dV V_i^SIC phi_i (times gE; V^SIC
// as stored by the energy pass):
//   P = Phibar psi^T (grid contraction), Qbar = P T^T, Daleckii-Krein
//   Sbar = U[(U^T Qbar U) o K]U^T with K_ij = -1/(a_i a_j (a_i + a_j)),
//   a = sqrt(lambda); Tbar = Q P + (Sbar + Sbar^T) T M;
//   vbar = Tbar/sqrt(rho) - v (Tbar.v)/rho^{3/2} (product form of Eq. 11);
//   dE/da_i = sum_a vbar_ia grad psi_a(a_i);
//   psibar = C^T Phibar + dV T^T (Sbar + Sbar^T) T psi + interpolation adjoint.
#include <type_traits>

#include "internal.cuh"
#include "xc_device.cuh"

namespace flosic {

// ---------------------------------------------------------------------------
// tricubic Lagrange interpolation at the FODs
// ---------------------------------------------------------------------------
// 4-point Lagrange basis on nodes -1, 0, 1, 2 at t and its derivative.
__device__ __forceinline__ void lagrange4(double t, double* L, double* dL) {
    const double tp = t + 1.0, tm = t - 1.0, t2 = t - 2.0;
    L[0] = -t * tm * t2 * (1.0 / 6.0);
    L[1] = tp * tm * t2 * 0.5;
    L[2] = -tp * t * t2 * 0.5;
    L[3] = tp * t * tm * (1.0 / 6.0);
    dL[0] = -(3.0 * t * t - 6.0 * t + 2.0) * (1.0 / 6.0);
    dL[1] = (3.0 * t * t - 4.0 * t - 1.0) * 0.5;
    dL[2] = -(3.0 * t * t - 2.0 * t - 2.0) * 0.5;
    dL[3] = (3.0 * t * t - 1.0) * (1.0 / 6.0);
}

struct Cell {
    int i0[3];
    double L[3][4], dL[3][4];
};

// Along a periodic direction of n points the coordinate is first reduced
// to [0, n) grid units (the FOD's image inside the cell).
__device__ __forceinline__ Cell cell_of(const BlkDesc& B, const double* a) {
    Cell c;
    const double o[3] = {B.ox, B.oy, B.oz};
    const int n[3] = {B.nx, B.ny, B.nz};
    for (int d = 0; d < 3; ++d) {
        double u = (a[d] - o[d]) / B.h;
        if ((B.per >> d) & 1) u -= n[d] * floor(u / n[d]);
        const double f = floor(u);
        c.i0[d] = (int)f;
        lagrange4(u - f, c.L[d], c.dL[d]);
    }
    return c;
}

// interpolation nodes along periodic directions wrap around the cell (the
// nodes of one cell lie at most 2 points outside it)
__device__ __forceinline__ void wrap_node(const BlkDesc& B, int& qx, int& qy, int& qz) {
    if (B.per & 1) qx = wrap_coord(qx, B.nx);
    if (B.per & 2) qy = wrap_coord(qy, B.ny);
    if (B.per & 4) qz = wrap_coord(qz, B.nz);
}

// one of the paper's grid-gradient components at an interior node: central
// difference inside, one-sided at the first and last point of the line
__device__ __forceinline__ double grid_grad(const double* u, const BlkDesc& B, int x, int y, int z,
                                            int d) {
    const int p[3] = {x, y, z};
    const int n[3] = {B.nx, B.ny, B.nz};
    const long long st[3] = {1, B.nx, (long long)B.nx * B.ny};
    const long long g = ((long long)z * B.ny + y) * B.nx + x;
    if (n[d] == 1) return 0.0;
    if (p[d] == 0) return (u[g + st[d]] - u[g]) / B.h;
    if (p[d] == n[d] - 1) return (u[g] - u[g - st[d]]) / B.h;
    return (u[g + st[d]] - u[g - st[d]]) / (2.0 * B.h);
}

// One warp per (block, FOD i, orbital a): vals[moff + i N + a] = psi_a(a_i)
// and grads[3 (moff + i N + a) + d].
__global__ void k_interp_fod(const BlkDesc* __restrict__ blk, int nblk, long long total,
                             const double* __restrict__ psi, const double* __restrict__ fods,
                             int mode, double* __restrict__ vals, double* __restrict__ grads,
                             int* __restrict__ status) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= total) return;
    int b = 0;
    while (b + 1 < nblk && blk[b + 1].moff <= w) ++b;
    const BlkDesc& B = blk[b];
    const long long r = w - B.moff;
    const int i = (int)(r / B.N), a = (int)(r % B.N);
    const double* f = fods + (B.fod_off + i) * 3;
    const double fa[3] = {f[0], f[1], f[2]};
    const Cell c = cell_of(B, fa);
    const double* u = psi + B.off + (long long)a * B.G;
    double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int node = lane; node < 64; node += 32) {
        const int e = node & 3, bb = (node >> 2) & 3, cc = node >> 4;
        int qx = c.i0[0] - 1 + e, qy = c.i0[1] - 1 + bb, qz = c.i0[2] - 1 + cc;
        if (B.per) wrap_node(B, qx, qy, qz);
        if (qx < 0 || qx >= B.nx || qy < 0 || qy >= B.ny || qz < 0 || qz >= B.nz) continue;
        const double uv = u[((long long)qz * B.ny + qy) * B.nx + qx];
        const double wgt = c.L[0][e] * c.L[1][bb] * c.L[2][cc];
        v += wgt * uv;
        if (mode == FLOSIC_GRAD_INTERP) {
            g0 += c.dL[0][e] * c.L[1][bb] * c.L[2][cc] * uv;
            g1 += c.L[0][e] * c.dL[1][bb] * c.L[2][cc] * uv;
            g2 += c.L[0][e] * c.L[1][bb] * c.dL[2][cc] * uv;
        } else {
            g0 += wgt * grid_grad(u, B, qx, qy, qz, 0);
            g1 += wgt * grid_grad(u, B, qx, qy, qz, 1);
            g2 += wgt * grid_grad(u, B, qx, qy, qz, 2);
        }
    }
    v = warp_sum(v);
    g0 = warp_sum(g0);
    g1 = warp_sum(g1);
    g2 = warp_sum(g2);
    if (lane == 0) {
        const double sc = (mode == FLOSIC_GRAD_INTERP) ? 1.0 / B.h : 1.0;
        vals[w] = v;
        grads[3 * w + 0] = g0 * sc;
        grads[3 * w + 1] = g1 * sc;
        grads[3 * w + 2] = g2 * sc;
        if (!isfinite(v) || !isfinite(fa[0] + fa[1] + fa[2])) atomicOr(status + 0, 1);
    }
}

void launch_interp_fod(const flosic_ctx* c, const double* psi, const double* fods, cudaStream_t s) {
    const long long total = c->mat_elems;
    const unsigned blocks = (unsigned)((total * 32 + 255) / 256);
    k_interp_fod<<<blocks, 256, 0, s>>>(c->d_blk, c->nblk, total, psi, fods, c->opt.fod_grad_mode,
                                        c->ws.vals, c->ws.grads, c->ws.status); note_launch(c);
}

// ---------------------------------------------------------------------------
// grid contractions C_ij = sum_g A_i(g) B_j(g) per block (K-split partials)
// ---------------------------------------------------------------------------
// Operand loaders: operator() gives the float64 value; bindf(B) gives a
// loader bound to one block that forms the value in float32 from the float64
// data with integer-op conversions (no float64 operation per element).
struct LoadPsi {
    const double* p;
    __device__ __forceinline__ double operator()(const BlkDesc& B, int i, long long g) const {
        return p[B.off + (long long)i * B.G + g];
    }
    struct F {
        const double* p;
        long long G;
        __device__ __forceinline__ float operator()(int i, long long g) const { return d2f(p[(long long)i * G + g]); }
        // split form: the float64 load alone (kept in flight), then the conversion
        using Raw = double;
        __device__ __forceinline__ Raw raw(int i, long long g) const { return __ldcs(p + (long long)i * G + g); }
        __device__ __forceinline__ static Raw zero() { return 0.0; }
        __device__ __forceinline__ float cvt(Raw r) const { return d2f(r); }
    };
    __device__ __forceinline__ F bindf(const BlkDesc& B) const { return F{p + B.off, B.G}; }
};

// Phibar_i(g) = gE * 2 dV * V_i^SIC(g) * phi_i(g) with V^SIC = -(V + v_xc)
// as stored by the energy pass (or its exact-adjoint variant).
struct LoadPhibar {
    const double* phi;
    const double* vsic;
    const double* gE;
    __device__ __forceinline__ double operator()(const BlkDesc& B, int i, long long g) const {
        const long long k = B.off + (long long)i * B.G + g;
        return gE[B.sys] * 2.0 * B.dV * vsic[k] * phi[k];
    }
    struct F {
        const double* phi;
        const double* vsic;
        long long G;
        float coef;
        __device__ __forceinline__ float operator()(int i, long long g) const {
            const long long k = (long long)i * G + g;
            return coef * d2f(vsic[k]) * d2f(phi[k]);
        }
        using Raw = double2;   // (phi, V^SIC)
        __device__ __forceinline__ Raw raw(int i, long long g) const {
            const long long k = (long long)i * G + g;
            return make_double2(__ldcs(phi + k), __ldcs(vsic + k));
        }
        __device__ __forceinline__ static Raw zero() { return make_double2(0.0, 0.0); }
        __device__ __forceinline__ float cvt(Raw r) const { return coef * d2f(r.y) * d2f(r.x); }
    };
    __device__ __forceinline__ F bindf(const BlkDesc& B) const {
        return F{phi + B.off, vsic + B.off, B.G, (float)(gE[B.sys] * 2.0 * B.dV)};
    }
};

// The same Phibar from wbar_i = V_i^SIC phi_i, which the mixed-precision
// energy pass stores as float32 when the adjoint reuses V (4 bytes a point
// instead of phi and V^SIC, 16).
struct LoadWbar {
    const float* w;
    const double* gE;
    __device__ __forceinline__ double operator()(const BlkDesc& B, int i, long long g) const {
        return gE[B.sys] * 2.0 * B.dV * (double)w[B.off + (long long)i * B.G + g];
    }
    struct F {
        const float* w;
        long long G;
        float coef;
        __device__ __forceinline__ float operator()(int i, long long g) const { return coef * w[(long long)i * G + g]; }
        using Raw = float;
        __device__ __forceinline__ Raw raw(int i, long long g) const { return __ldcs(w + (long long)i * G + g); }
        __device__ __forceinline__ static Raw zero() { return 0.f; }
        __device__ __forceinline__ float cvt(Raw r) const { return coef * r; }
    };
    __device__ __forceinline__ F bindf(const BlkDesc& B) const {
        return F{w + B.off, B.G, (float)(gE[B.sys] * 2.0 * B.dV)};
    }
};

// TC: arithmetic of the products and of the sum within one 16-point k tile.
// float (mixed precision): float32 operands from the bound loaders, tile sums
// accumulated as float-float pairs, one float64 addition per matrix element
// at the end; double: float64 throughout.
template <int RM, class TC, class LA, class LB>
__global__ void __launch_bounds__(256) k_contract(const BlkDesc* __restrict__ blk, int kparts, LA la,
                                                  LB lb, double* __restrict__ part, long long mat_elems) {
    constexpr int KT = 16;
    constexpr int NP = 16 * RM;
    __shared__ TC As[KT][NP + 1];
    __shared__ TC Bs[KT][NP + 1];
    const BlkDesc& B = blk[blockIdx.y];
    const int N = B.N;
    const long long G = B.G;
    const int kp = blockIdx.x;
    const long long kb = G * kp / kparts, ke = G * (kp + 1) / kparts;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    constexpr bool kF = std::is_same<TC, float>::value;
    const auto fa = la.bindf(B);
    const auto fb = lb.bindf(B);
    TC acc[RM][RM], acl[RM][RM];   // (sum, low part) pairs when kF
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int q = 0; q < RM; ++q) acc[r][q] = acl[r][q] = TC(0);
    for (long long k0 = kb; k0 < ke; k0 += KT) {
        for (int idx = threadIdx.x; idx < KT * NP; idx += 256) {
            const int i = idx / KT, kk = idx % KT;
            const long long g = k0 + kk;
            const bool ok = (i < N) && (g < ke);
            if constexpr (kF) {
                As[kk][i] = ok ? fa(i, g) : 0.f;
                Bs[kk][i] = ok ? fb(i, g) : 0.f;
            } else {
                As[kk][i] = ok ? la(B, i, g) : 0.0;
                Bs[kk][i] = ok ? lb(B, i, g) : 0.0;
            }
        }
        __syncthreads();
        TC tacc[RM][RM];
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int q = 0; q < RM; ++q) tacc[r][q] = TC(0);
#pragma unroll 4
        for (int kk = 0; kk < KT; ++kk) {
            TC a[RM], bv[RM];
#pragma unroll
            for (int r = 0; r < RM; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < RM; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int q = 0; q < RM; ++q) tacc[r][q] += a[r] * bv[q];
        }
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                if constexpr (kF) {   // two-sum into the pair
                    const float a = acc[r][q], b = tacc[r][q];
                    const float s2 = a + b, bb = s2 - a;
                    acl[r][q] += (a - (s2 - bb)) + (b - bb);
                    acc[r][q] = s2;
                } else {
                    acc[r][q] += tacc[r][q];
                }
            }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
            const int i = ty + 16 * r, j = tx + 16 * q;
            double v;
            if constexpr (kF) v = f2d(acc[r][q]) + f2d(acl[r][q]);
            else v = acc[r][q];
            if (i < N && j < N) part[(long long)kp * mat_elems + B.moff + (long long)i * N + j] = v;
        }
}

// Mixed-precision variant of k_contract for N <= 16 RM: 64-point steps whose
// operand values (float32 from the bound loaders) are fetched into registers
// while the previous step is multiplied.  The step's A and B tiles are staged
// as [point][orbital] rows of float4 groups (group index XOR-swizzled by the
// point so the 16-byte stores of consecutive points hit distinct banks).
// Output tiles of 4 x 4 per thread: the CTA's 256 threads form KG = 256 /
// (NP/4)^2 groups, each holding the whole NP x NP product for every KG-th
// point of a step, so a point costs each thread two 16-byte shared loads for
// 16 FMAs (8 packed two-lane instructions).  Float sums of up to 16 points are
// two-summed into (sum, low)
// pairs; the groups' pairs are added at the end in a fixed order.
template <int RM, class LA, class LB>
__global__ void __launch_bounds__(256, RM <= 2 ? 2 : 1) k_contract_f(const BlkDesc* __restrict__ blk, int kparts, LA la, LB lb,
                                                       double* __restrict__ part, long long mat_elems) {
    constexpr int KT = 64;
    constexpr int NP = 16 * RM;
    constexpr int C4 = NP / 4;                 // float4 groups per staged row
    constexpr int L = C4 * C4;                 // threads per group (one 4 x 4 output tile each)
    constexpr int KG = 256 / L;                // groups
    constexpr int KPG = KT / KG;               // points per group and step
    constexpr int SUB = KPG < 16 ? KPG : 16;   // points per float sub-sum
    constexpr int PC = C4 / 4;                 // float4 groups a thread stages per operand
    static_assert(L * KG == 256 && PC >= 1, "tile shape");
    constexpr int kStage = 2 * KT * NP;                  // floats of the A and B tiles
    constexpr int kRed = (KG > 1 ? (KG / 2) : 0) * L * 32;   // floats of the group reduction
    __shared__ __align__(16) float sm[kStage > kRed ? kStage : kRed];
    float4* As4 = reinterpret_cast<float4*>(sm);
    float4* Bs4 = As4 + KT * C4;
    const BlkDesc& B = blk[blockIdx.y];
    const int N = B.N;
    const long long G = B.G;
    const int kp = blockIdx.x;
    const long long kb = G * kp / kparts, ke = G * (kp + 1) / kparts;
    const int tid = threadIdx.x;
    const auto fa = la.bindf(B);
    const auto fb = lb.bindf(B);
    using FA = std::remove_const_t<decltype(fa)>;
    using FB = std::remove_const_t<decltype(fb)>;
    // staging: point kk0 of the step, float4 groups c0 + 4 m (orbitals 4 (c0 + 4 m) + j)
    const int kk0 = tid & (KT - 1), c0 = tid >> 6;
    typename FA::Raw pa[PC][4];
    typename FB::Raw pb[PC][4];
    auto fetch = [&](long long k0) {
        const long long g = k0 + kk0;
        const bool gin = g < ke;
#pragma unroll
        for (int m = 0; m < PC; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = 4 * (c0 + 4 * m) + j;
                const bool ok = gin && i < N;
                pa[m][j] = ok ? fa.raw(i, g) : FA::zero();
                pb[m][j] = ok ? fb.raw(i, g) : FB::zero();
            }
    };
    // compute: group kg takes points kg + KG t of each step; tile rows 4 rg.., columns 4 cg..
    const int kg = tid / L, li = tid % L, rg = li % C4, cg = li / C4;
    float acc[4][4], acl[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = acl[r][q] = 0.f;
    if (kb < ke) fetch(kb);
    for (long long k0 = kb; k0 < ke; k0 += KT) {
        __syncthreads();   // the previous step's tiles are read
#pragma unroll
        for (int m = 0; m < PC; ++m) {
            const int c = c0 + 4 * m, cs = c ^ (kk0 & (C4 - 1));
            As4[kk0 * C4 + cs] = make_float4(fa.cvt(pa[m][0]), fa.cvt(pa[m][1]), fa.cvt(pa[m][2]), fa.cvt(pa[m][3]));
            Bs4[kk0 * C4 + cs] = make_float4(fb.cvt(pb[m][0]), fb.cvt(pb[m][1]), fb.cvt(pb[m][2]), fb.cvt(pb[m][3]));
        }
        __syncthreads();
        if (k0 + KT < ke) fetch(k0 + KT);
#pragma unroll
        for (int s0 = 0; s0 < KPG; s0 += SUB) {
            float2 t[4][2];   // columns (0, 1) and (2, 3) of each row: packed FMAs
#pragma unroll
            for (int r = 0; r < 4; ++r) t[r][0] = t[r][1] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int u = s0; u < s0 + SUB; ++u) {
                const int kk = kg + KG * u;
                const float4 a = As4[kk * C4 + (rg ^ (kk & (C4 - 1)))];
                const float4 b = Bs4[kk * C4 + (cg ^ (kk & (C4 - 1)))];
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float2 b01 = make_float2(b.x, b.y), b23 = make_float2(b.z, b.w);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 ar = make_float2(av[r], av[r]);
                    t[r][0] = __ffma2_rn(ar, b01, t[r][0]);
                    t[r][1] = __ffma2_rn(ar, b23, t[r][1]);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {   // two-sum into the pair
                    const float x = acc[r][q], y = (q & 1) ? t[r][q >> 1].y : t[r][q >> 1].x;
                    const float s2 = x + y, bb = s2 - x;
                    acl[r][q] += (x - (s2 - bb)) + (y - bb);
                    acc[r][q] = s2;
                }
        }
    }
    // groups KG/2.. hand their pairs to groups 0..KG/2-1, and so on (fixed order)
    float2* red = reinterpret_cast<float2*>(sm);
#pragma unroll 1
    for (int half = KG / 2; half >= 1; half /= 2) {
        __syncthreads();
        if (kg >= half && kg < 2 * half) {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                red[(e * half + kg - half) * L + li] = make_float2(acc[e >> 2][e & 3], acl[e >> 2][e & 3]);
        }
        __syncthreads();
        if (kg < half) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float2 o = red[(e * half + kg) * L + li];
                const ff s = ff_add(ff{acc[e >> 2][e & 3], acl[e >> 2][e & 3]}, ff{o.x, o.y});
                acc[e >> 2][e & 3] = s.h;
                acl[e >> 2][e & 3] = s.l;
            }
        }
    }
    if (kg == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * rg + r, j = 4 * cg + q;
                if (i < N && j < N)
                    part[(long long)kp * mat_elems + B.moff + (long long)i * N + j] = f2d(acc[r][q]) + f2d(acl[r][q]);
            }
    }
}

// out[e] = sum_kp part[kp][e] in a fixed order
__global__ void k_sum_parts(const double* __restrict__ part, int kparts, long long n,
                            double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int k = 0; k < kparts; ++k) s += part[(long long)k * n + e];
    out[e] = s;
}

static int max_block_n(const flosic_ctx* c) {
    int m = 0;
    for (const auto& b : c->blk) m = b.N > m ? b.N : m;
    return m;
}

template <class LA, class LB>
static void contract(const flosic_ctx* c, LA la, LB lb, double* out, cudaStream_t s) {
    const int nmax = max_block_n(c);
    const bool f32 = (c->opt.precision == FLOSIC_MIXED);
    int kparts = c->kparts;   // one wave: 4 CTAs per SM, 2 for the float kernels (1 at N > 32)
    if (f32 && nmax <= 64) {
        const int per_sm = nmax <= 32 ? 2 : 1;
        const int k2 = (per_sm * c->num_sms + c->nblk - 1) / c->nblk;
        kparts = k2 < 1 ? 1 : (k2 < kparts ? k2 : kparts);
    }
    const dim3 grid(kparts, c->nblk);
    double* part = c->ws.mat_part;
    if (f32) {
        if (nmax <= 16) k_contract_f<1><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else if (nmax <= 32) k_contract_f<2><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else if (nmax <= 64) k_contract_f<4><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else k_contract<8, float><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
    } else {
        if (nmax <= 16) k_contract<1, double><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else if (nmax <= 32) k_contract<2, double><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else if (nmax <= 64) k_contract<4, double><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
        else k_contract<8, double><<<grid, 256, 0, s>>>(c->d_blk, kparts, la, lb, part, c->mat_elems);
    }
    note_launch(c);
    k_sum_parts<<<(unsigned)((c->mat_elems + 255) / 256), 256, 0, s>>>(part, kparts, c->mat_elems, out); note_launch(c);
}

// Raw Gram psi psi^T per block: tensor cores (split-BF16) in mixed precision,
// the float64 contraction otherwise.
void launch_gram(const flosic_ctx* c, const double* psi, cudaStream_t s) {
    if (c->opt.precision == FLOSIC_MIXED)
        launch_gram_tc(c, psi, s);
    else
        contract(c, LoadPsi{psi}, LoadPsi{psi}, c->ws.M, s);
}

// Vsrc: V^SIC in float64, or null when the energy pass stored wbar instead
void launch_backward_contract(const flosic_ctx* c, const double* psi, const double* phi,
                              const double* vsic, const double* gE, cudaStream_t s) {
    if (!vsic) contract(c, LoadWbar{c->ws.wbar, gE}, LoadPsi{psi}, c->ws.P, s);
    else contract(c, LoadPhibar{phi, vsic, gE}, LoadPsi{psi}, c->ws.P, s);
}

// ---------------------------------------------------------------------------
// small dense algebra, one CTA per spin block
// ---------------------------------------------------------------------------
// Y = op(A) op(B) for row-major N x N matrices in global memory (ta/tb:
// transpose).  All threads of the CTA take part; ends with __syncthreads.
__device__ void mm(int N, const double* A, bool ta, const double* Bm, bool tb, double* Y) {
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e / N, j = e % N;
        double s = 0.0;
        for (int k = 0; k < N; ++k) {
            const double a = ta ? A[k * N + i] : A[i * N + k];
            const double b = tb ? Bm[j * N + k] : Bm[k * N + j];
            s += a * b;
        }
        Y[e] = s;
    }
    __syncthreads();
}

// Cyclic Jacobi eigen-decomposition of the symmetric matrix S (N x N,
// row-major with row stride ld, shared memory), round-robin ordering so that
// the N/2 rotations of a round are disjoint and run in parallel.  On exit S
// is diagonal (the eigenvalues) and U (stride ld) holds the eigenvectors as
// columns.  Stops when the squared off-diagonal norm is at most tol times
// the squared diagonal one, or after max_sweeps sweeps.  T = float runs the
// rounds in float32.  A row stride of N + 1 keeps the column updates (lanes
// over rows) free of shared-memory bank conflicts.
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class T, bool kFloatAngle = false>
__device__ void jacobi_eig_t(int N, int ld, T* S, T* U, double tol, int max_sweeps) {
    __shared__ int rp[kMaxN / 2], rq[kMaxN / 2];
    __shared__ T rc[kMaxN / 2], rs[kMaxN / 2];
    __shared__ double scratch[32];
    const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-300);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < N; i += nw)
        for (int k = lane; k < N; k += 32) U[i * ld + k] = (i == k) ? T(1) : T(0);
    __syncthreads();
    const int N2 = N + (N & 1);
    const int m = N2 - 1;
    const int np = N2 / 2;
    for (int sweep = 0; sweep < max_sweeps && N > 1; ++sweep) {
        T off = T(0), dg = T(0);
        for (int i = warp; i < N; i += nw)
            for (int k = lane; k < N; k += 32) {
                const T v = S[i * ld + k];
                if (i == k) dg += v * v; else off += v * v;
            }
        const double offs = block_sum(off, scratch);
        const double dgs = block_sum(dg, scratch);
        if (offs <= tol * dgs) break;
        for (int round = 0; round < m; ++round) {
            if (threadIdx.x < np) {
                const int t = threadIdx.x;
                int p, q;   // the round-robin pairing of round `round` (round + t < 2m, no division)
                if (t == 0) {
                    p = 0;
                    q = round + 1;
                } else {
                    p = round + t;
                    if (p >= m) p -= m;
                    ++p;
                    q = round - t + m;
                    if (q >= m) q -= m;
                    ++q;
                }
                if (p > q) { const int tmp = p; p = q; q = tmp; }
                T c = T(1), sn = T(0);
                if (q < N) {
                    const T apq = S[p * ld + q];
                    if constexpr (kFloatAngle) {
                        // a nearly diagonal float64 matrix: the angle in float32 (relative error
                        // ~1e-7 leaves ~1e-7 of S_pq, removed by the next sweep), c and s from it in
                        // float64, so the rotation is orthogonal to float64 rounding
                        const float apf = (float)apq, dqf = (float)(S[q * ld + q] - S[p * ld + p]);
                        if (fabsf(apf) > 1e-30f) {
                            const float th = dqf / (2.f * apf), at = fabsf(th);
                            float tf = at > 1e15f ? 0.5f / at : 1.f / (at + sqrtf(th * th + 1.f));
                            if (th < 0.f) tf = -tf;
                            const T tt = (T)tf;
                            c = rsq(tt * tt + T(1));
                            sn = tt * c;
                        }
                    } else if (fabs(apq) > tiny) {
                        const T th = (S[q * ld + q] - S[p * ld + p]) / (T(2) * apq);
                        const T tt = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                        c = rsq(tt * tt + T(1));
                        sn = tt * c;
                    }
                }
                rp[t] = p;
                rq[t] = q < N ? q : p;   // dummy partner: identity rotation
                rc[t] = c;
                rs[t] = (q < N) ? sn : T(0);
            }
            __syncthreads();
            for (int t = warp; t < np; t += nw) {   // rows p, q
                const int p = rp[t], q = rq[t];
                if (p == q) continue;
                const T c = rc[t], sn = rs[t];
                for (int k = lane; k < N; k += 32) {
                    const T a = S[p * ld + k], b = S[q * ld + k];
                    S[p * ld + k] = c * a - sn * b;
                    S[q * ld + k] = sn * a + c * b;
                }
            }
            __syncthreads();
            for (int t = warp; t < np; t += nw) {   // columns p, q
                const int p = rp[t], q = rq[t];
                if (p == q) continue;
                const T c = rc[t], sn = rs[t];
                for (int k = lane; k < N; k += 32) {
                    T a = S[k * ld + p], b = S[k * ld + q];
                    S[k * ld + p] = c * a - sn * b;
                    S[k * ld + q] = sn * a + c * b;
                    a = U[k * ld + p];
                    b = U[k * ld + q];
                    U[k * ld + p] = c * a - sn * b;
                    U[k * ld + q] = sn * a + c * b;
                }
            }
            __syncthreads();
        }
    }
}

__device__ void jacobi_eig(int N, double* S, double* U) { jacobi_eig_t<double>(N, N, S, U, 1e-30, 40); }

// Blocks of up to this many orbitals take the two-stage eigen-solver in the
// mixed path (its four N x N work matrices fit in shared memory).
constexpr int kLowdinTwoStageMax = 64;

// Per block: T, S, eigen-pairs, Q = S^{-1/2}, C = Q T; ILLCOND / NONFINITE.
//
// two_stage (mixed path, every block N <= kLowdinTwoStageMax): float32 Jacobi
// sweeps to an off-diagonal norm of ~3e-6, two float64 Newton-Schulz steps
// U <- U (3I - U^T U) / 2 that make U orthogonal to float64 rounding, then
// float64 Jacobi on the nearly diagonal U^T S U (two sweeps) and U <- U V.
// The float64 sweeps, each a chain of barrier-separated rounds on one SM's
// float64 pipe, drop from ~8 to ~2; the eigenpairs are those of the float64
// decomposition to rounding.  Otherwise float64 Jacobi from the start.
__global__ void __launch_bounds__(512) k_lowdin(const BlkDesc* __restrict__ blk, Workspace w,
                                                double illcond, double* S_out, double* Q_out,
                                                int two_stage) {
    extern __shared__ double Ssh[];
    __shared__ double scratch[32];
    __shared__ double il[kMaxN];
    const BlkDesc& B = blk[blockIdx.x];
    const int N = B.N;
    const long long mo = B.moff;
    const double* vals = w.vals + mo;
    double* T = w.T + mo;
    double* M = w.M + mo;
    double* X = w.tmp + mo;
    double* U = w.U + mo;
    double* Q = w.Q + mo;
    // M = dV * (raw Gram), finiteness of psi
    double bad = 0.0;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        M[e] *= B.dV;
        if (!isfinite(M[e]) || !isfinite(vals[e])) bad = 1.0;
    }
    bad = block_sum(bad, scratch);
    if (bad > 0.0) {
        if (threadIdx.x == 0) atomicOr(w.status + 0, 1);
        return;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double r = 0.0;
        for (int a = 0; a < N; ++a) r += vals[i * N + a] * vals[i * N + a];
        w.rho_a[B.orb0 + i] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) T[e] = vals[e] * rsqrt(w.rho_a[B.orb0 + e / N]);
    __syncthreads();
    mm(N, T, false, M, false, X);          // X = T M
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // S = X T^T
        const int i = e / N, j = e % N;
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += X[i * N + k] * T[j * N + k];
        Ssh[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // exact symmetry
        const int i = e / N, j = e % N;
        if (i < j) {
            const double v = 0.5 * (Ssh[e] + Ssh[j * N + i]);
            Ssh[e] = v;
            Ssh[j * N + i] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        w.S[mo + e] = Ssh[e];
        if (S_out) S_out[mo + e] = Ssh[e];
    }
    __syncthreads();
    const int ldp = N + 1;   // padded row stride of the Jacobi matrices
    double* Sd = Ssh;        // the diagonalised S (eigenvalues on its diagonal), row stride ldS
    int ldS = N;
    if (two_stage) {
        double* U64 = Ssh + N * N;   // shared: U (float64), V (float64, padded), then S and U
        double* V64 = U64 + N * N;   // in float32 (padded), whose space later holds S (float64, padded)
        double* Sp = V64 + N * ldp;
        float* S32 = reinterpret_cast<float*>(Sp);
        float* U32 = S32 + N * ldp;
        double* Y = w.tmp + w.mat_elems + mo;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) S32[(e / N) * ldp + e % N] = d2f(Ssh[e]);
        __syncthreads();
        jacobi_eig_t<float>(N, ldp, S32, U32, 1e-11, 12);
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) U64[e] = f2d(U32[(e / N) * ldp + e % N]);
        __syncthreads();
        for (int it = 0; it < 2; ++it) {   // U <- U (3I - U^T U) / 2
            mm(N, U64, true, U64, false, X);
            for (int e = threadIdx.x; e < N * N; e += blockDim.x)
                X[e] = ((e / N == e % N) ? 1.5 : 0.0) - 0.5 * X[e];
            __syncthreads();
            mm(N, U64, false, X, false, Y);
            for (int e = threadIdx.x; e < N * N; e += blockDim.x) U64[e] = Y[e];
            __syncthreads();
        }
        mm(N, Ssh, false, U64, false, X);   // X = S U
        mm(N, U64, true, X, false, Y);      // Y = U^T S U
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // exact symmetry
            const int i = e / N, j = e % N;
            Sp[i * ldp + j] = (i == j) ? Y[e] : 0.5 * (Y[e] + Y[j * N + i]);
        }
        __syncthreads();
        jacobi_eig_t<double, true>(N, ldp, Sp, V64, 1e-30, 40);
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // U = U V
            const int i = e / N, j = e % N;
            double sum = 0.0;
            for (int k = 0; k < N; ++k) sum += U64[i * N + k] * V64[k * ldp + j];
            U[e] = sum;
        }
        __syncthreads();
        Sd = Sp;
        ldS = ldp;
    } else {
        jacobi_eig(N, Ssh, U);
    }
    double* lam = w.lam + B.orb0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        lam[i] = Sd[i * ldS + i];
        il[i] = rsqrt(fmax(Sd[i * ldS + i], 1e-300));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double lmin = lam[0], lmax = lam[0];
        for (int i = 1; i < N; ++i) {
            lmin = fmin(lmin, lam[i]);
            lmax = fmax(lmax, lam[i]);
        }
        if (!(lmin > illcond * lmax) || !(lmin > 0.0)) atomicOr(w.status + 2, 1);
    }
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // Q = U L^{-1/2} U^T
        const int i = e / N, j = e % N;
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += U[i * N + k] * U[j * N + k] * il[k];
        Q[e] = s;
        if (Q_out) Q_out[mo + e] = s;
    }
    __syncthreads();
    mm(N, Q, false, T, false, w.C + mo);   // C = Q T
}

static bool lowdin_two_stage(const flosic_ctx* c) {
    return c->opt.precision == FLOSIC_MIXED && max_block_n(c) <= kLowdinTwoStageMax;
}

size_t lowdin_smem(const flosic_ctx* c) {
    const size_t n2 = (size_t)max_block_n(c) * max_block_n(c);
    const size_t np = (size_t)max_block_n(c) * (max_block_n(c) + 1);   // a padded matrix
    return lowdin_two_stage(c) ? 2 * n2 * sizeof(double) + 2 * np * sizeof(double) : n2 * sizeof(double);
}

void launch_lowdin(const flosic_ctx* c, double* S_out, double* Q_out, cudaStream_t s) {
    k_lowdin<<<c->nblk, 512, lowdin_smem(c), s>>>(c->d_blk, c->ws, c->opt.illcond_tol, S_out, Q_out,
                                                   lowdin_two_stage(c) ? 1 : 0);
    note_launch(c);
}

// ---------------------------------------------------------------------------
// out_j(g) = sum_k E_jk X_k(g): small matrix times a tall operand, per block
// ---------------------------------------------------------------------------
template <class PB>
struct LoadPhibarPsi {   // rows 0..N-1: Phibar (PB: LoadPhibar or LoadWbar); rows N..2N-1: psi
    PB pb;
    const double* psi;
    __device__ __forceinline__ double operator()(const BlkDesc& B, int k, long long g) const {
        if (k < B.N) return pb(B, k, g);
        return psi[B.off + (long long)(k - B.N) * B.G + g];
    }
    struct F {
        typename PB::F pb;
        const double* psi;
        long long G;
        int N;
        __device__ __forceinline__ float operator()(int k, long long g) const {
            return (k < N) ? pb(k, g) : d2f(psi[(long long)(k - N) * G + g]);
        }
    };
    __device__ __forceinline__ F bindf(const BlkDesc& B) const { return F{pb.bindf(B), psi + B.off, B.G, B.N}; }
};

// TC: arithmetic of the products and sums (float in mixed precision, with
// operands and results converted by integer operations).  A CTA takes tiles
// of 32 PTS points (lane l: points l + 32 q, q < PTS), so each chunk of E
// staged in shared memory serves PTS x 32 points.
template <int RJ, int PTS, class TC, class LX>
__global__ void __launch_bounds__(256) k_smallmat(const BlkDesc* __restrict__ blk,
                                                  const double* __restrict__ E, int mult, LX lx,
                                                  double* __restrict__ out) {
    constexpr int TG = 32 * PTS, KC = 32;
    __shared__ TC Es[8 * RJ][KC + 1];
    __shared__ TC Xs[KC][TG];
    const BlkDesc& B = blk[blockIdx.y];
    const int N = B.N, K = mult * N;
    const double* Eb = E + mult * B.moff;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    constexpr bool kF = std::is_same<TC, float>::value;
    const auto fx = lx.bindf(B);
    for (long long tile = blockIdx.x; tile * TG < B.G; tile += gridDim.x) {
        TC acc[RJ][PTS];
#pragma unroll
        for (int r = 0; r < RJ; ++r)
#pragma unroll
            for (int q = 0; q < PTS; ++q) acc[r][q] = TC(0);
        for (int kc = 0; kc < K; kc += KC) {
            for (int e = threadIdx.x; e < 8 * RJ * KC; e += 256) {
                const int j = e / KC, kk = e % KC;
                const bool ok = j < N && kc + kk < K;
                if constexpr (kF) Es[j][kk] = ok ? d2f(Eb[(long long)j * K + kc + kk]) : 0.f;
                else Es[j][kk] = ok ? Eb[(long long)j * K + kc + kk] : 0.0;
            }
            for (int kk = wq; kk < KC; kk += 8) {
#pragma unroll
                for (int q = 0; q < PTS; ++q) {
                    const long long g = tile * TG + lane + 32 * q;
                    const bool ok = kc + kk < K && g < B.G;
                    if constexpr (kF) Xs[kk][lane + 32 * q] = ok ? fx(kc + kk, g) : 0.f;
                    else Xs[kk][lane + 32 * q] = ok ? lx(B, kc + kk, g) : 0.0;
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < KC; ++kk) {
                TC x[PTS];
#pragma unroll
                for (int q = 0; q < PTS; ++q) x[q] = Xs[kk][lane + 32 * q];
#pragma unroll
                for (int r = 0; r < RJ; ++r) {
                    const TC ev = Es[wq + 8 * r][kk];
#pragma unroll
                    for (int q = 0; q < PTS; ++q) acc[r][q] += ev * x[q];
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < PTS; ++q) {
            const long long g = tile * TG + lane + 32 * q;
            if (g >= B.G) continue;
#pragma unroll
            for (int r = 0; r < RJ; ++r) {
                const int j = wq + 8 * r;
                if (j < N) {
                    if constexpr (kF) out[B.off + (long long)j * B.G + g] = f2d(acc[r][q]);
                    else out[B.off + (long long)j * B.G + g] = acc[r][q];
                }
            }
        }
    }
}

// Row loaders of the row-tile kernel below, one per segment of rows of X
// (rows() of them per block): load() issues the float64 (or float32) load of
// X_k(g) and returns it untouched, so the next group of k can be in flight
// while the current one is multiplied; cvt() forms the float32 value with
// integer-op conversions.
template <int KU>
struct RowsPsi {   // psi_k
    static constexpr int kGroup = KU;   // k values fetched ahead
    using Raw = double;
    const double* p;
    struct Bound {
        const double* p;
        long long G;
        int n;
        __device__ __forceinline__ int rows() const { return n; }
        __device__ __forceinline__ Raw load(int k, long long g) const { return __ldcs(p + (long long)k * G + g); }
        __device__ __forceinline__ float cvt(Raw r) const { return d2f(r); }
    };
    __device__ __forceinline__ static Raw zero() { return 0.0; }
    __device__ __forceinline__ Bound bind(const BlkDesc& B) const { return Bound{p + B.off, B.G, B.N}; }
};

// Phibar_k = coef V_k^SIC phi_k from float64 phi and V^SIC (two loads)
struct RowsPhibar {
    static constexpr int kGroup = 4;
    using Raw = double2;
    const double* phi;
    const double* vsic;
    const double* gE;
    struct Bound {
        const double *phi, *vsic;
        long long G;
        int n;
        float coef;
        __device__ __forceinline__ int rows() const { return n; }
        __device__ __forceinline__ Raw load(int k, long long g) const {
            const long long e = (long long)k * G + g;
            return make_double2(__ldcs(phi + e), __ldcs(vsic + e));
        }
        __device__ __forceinline__ float cvt(Raw r) const { return coef * d2f(r.y) * d2f(r.x); }
    };
    __device__ __forceinline__ static Raw zero() { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ Bound bind(const BlkDesc& B) const {
        return Bound{phi + B.off, vsic + B.off, B.G, B.N, (float)(gE[B.sys] * 2.0 * B.dV)};
    }
};

// Phibar_k = coef wbar_k (wbar = V^SIC phi stored as float32 by the energy pass)
struct RowsWbar {
    static constexpr int kGroup = 8;
    using Raw = float;
    const float* w;
    const double* gE;
    struct Bound {
        const float* w;
        long long G;
        int n;
        float coef;
        __device__ __forceinline__ int rows() const { return n; }
        __device__ __forceinline__ Raw load(int k, long long g) const { return __ldcs(w + (long long)k * G + g); }
        __device__ __forceinline__ float cvt(Raw r) const { return coef * r; }
    };
    __device__ __forceinline__ static Raw zero() { return 0.f; }
    __device__ __forceinline__ Bound bind(const BlkDesc& B) const {
        return Bound{w + B.off, B.G, B.N, (float)(gE[B.sys] * 2.0 * B.dV)};
    }
};

// no rows (a single-segment product)
struct RowsNone {
    static constexpr int kGroup = 1;
    using Raw = float;
    struct Bound {
        __device__ __forceinline__ int rows() const { return 0; }
        __device__ __forceinline__ Raw load(int, long long) const { return 0.f; }
        __device__ __forceinline__ float cvt(Raw r) const { return r; }
    };
    __device__ __forceinline__ static Raw zero() { return 0.f; }
    __device__ __forceinline__ Bound bind(const BlkDesc&) const { return Bound{}; }
};

constexpr int kRowTile = 256;     // points per tile of the row-tile kernel (one per thread)
constexpr int kRowMaxK = 64;      // K = mult N it takes (N <= 32, mult <= 2)

// out_j(g) = sum_k E_jk X_k(g) for blocks with N <= NJ <= 32 (mixed
// precision): one point per thread with all N outputs in registers, E (as
// float, transposed) in shared memory for the whole block, so a k step is
// NJ/4 broadcast 16-byte shared loads and NJ FMAs per point (NJ/2 packed
// two-lane instructions).  The rows of X come in two segments (R1: k < K1,
// R2: the K2 rows after them; R2 may be empty), each fetched in groups of its
// own kGroup with its own load type, so no group mixes two kinds of rows.  Persistent CTAs walk a contiguous range
// of the (block, 256-point tile) items; the loads of the next group (of the
// same segment, the other segment or the next tile) are issued before the
// current group is multiplied.
template <int NJ, class R1, class R2>
__global__ void __launch_bounds__(kRowTile, 2) k_smallmat_rows(const BlkDesc* __restrict__ blk, int nblk,
                                                               long long total, const double* __restrict__ E,
                                                               int mult, R1 r1, R2 r2, double* __restrict__ out) {
    constexpr int KU1 = R1::kGroup, KU2 = R2::kGroup;
    constexpr bool kTwo = !std::is_same<R2, RowsNone>::value;
    constexpr int kRows = kRowMaxK + KU1 + KU2;   // staged rows of E: both segments, each padded to its groups
    __shared__ float4 es4[kRows * (NJ / 4)];      // [row][j], zero past a segment's rows
    float* es = reinterpret_cast<float*>(es4);
    const long long per_cta = (total + gridDim.x - 1) / gridDim.x;
    const long long it0 = (long long)blockIdx.x * per_cta;
    const long long it1 = it0 + per_cta < total ? it0 + per_cta : total;
    if (it0 >= it1) return;   // uniform over the CTA
    // block of the first item
    int b = 0;
    long long base = 0;
    for (;;) {
        const long long nt = (blk[b].G + kRowTile - 1) / kRowTile;
        if (it0 < base + nt || b + 1 >= nblk) break;
        base += nt;
        ++b;
    }
    const int tid = threadIdx.x;
    long long item = it0;
    while (item < it1) {
        const BlkDesc& B = blk[b];
        const auto f1 = r1.bind(B);
        const auto f2 = r2.bind(B);
        const int K1 = f1.rows(), K2 = f2.rows(), K = mult * B.N;   // K1 + K2 = K
        const int ng1 = (K1 + KU1 - 1) / KU1, ng2 = kTwo ? (K2 + KU2 - 1) / KU2 : 0;
        const int s2 = ng1 * KU1;   // first staged row of segment 2
        const long long ntile = (B.G + kRowTile - 1) / kRowTile;
        const long long item_end = (base + ntile < it1) ? base + ntile : it1;
        {   // E of this block, transposed, as float
            const double* Eb = E + (long long)mult * B.moff;
            __syncthreads();   // the previous block's products are done with es
            for (int e = tid; e < (s2 + ng2 * KU2) * NJ; e += kRowTile) {
                const int row = e / NJ, j = e - row * NJ;
                const int k = row < s2 ? row : K1 + (row - s2);           // column of E
                const bool ok = j < B.N && (row < s2 ? row < K1 : row - s2 < K2);
                es[e] = ok ? d2f(Eb[(long long)j * K + k]) : 0.f;
            }
            __syncthreads();
        }
        typename R1::Raw raw1[KU1];
        typename R2::Raw raw2[KU2];
        auto fetch1 = [&](long long tl, int grp) {
            const long long g = tl * kRowTile + tid;
#pragma unroll
            for (int u = 0; u < KU1; ++u) {
                const int k = grp * KU1 + u;
                raw1[u] = (g < B.G && k < K1) ? f1.load(k, g) : R1::zero();
            }
        };
        auto fetch2 = [&](long long tl, int grp) {
            const long long g = tl * kRowTile + tid;
#pragma unroll
            for (int u = 0; u < KU2; ++u) {
                const int k = grp * KU2 + u;
                raw2[u] = (g < B.G && k < K2) ? f2.load(k, g) : R2::zero();
            }
        };
        if (ng1 > 0) fetch1(item - base, 0);
        else if (ng2 > 0) fetch2(item - base, 0);
        for (; item < item_end; ++item) {
            const long long tl = item - base, g = tl * kRowTile + tid;
            const bool more = item + 1 < item_end;
            float2 acc[NJ / 2];   // outputs (2j, 2j + 1): two FMAs per packed instruction
#pragma unroll
            for (int j = 0; j < NJ / 2; ++j) acc[j] = make_float2(0.f, 0.f);
            for (int grp = 0; grp < ng1; ++grp) {
                float x[KU1];
#pragma unroll
                for (int u = 0; u < KU1; ++u) x[u] = f1.cvt(raw1[u]);
                const bool same = grp + 1 < ng1;   // next: this segment, the other one or the next tile
                if (same || (ng2 == 0 && more)) fetch1(same ? tl : tl + 1, same ? grp + 1 : 0);
                else if (ng2 > 0) fetch2(tl, 0);
#pragma unroll
                for (int u = 0; u < KU1; ++u) {
                    const float4* er = es4 + (long long)(grp * KU1 + u) * (NJ / 4);
                    const float2 xu = make_float2(x[u], x[u]);
#pragma unroll
                    for (int q = 0; q < NJ / 4; ++q) {
                        const float4 ev = er[q];
                        acc[2 * q] = __ffma2_rn(make_float2(ev.x, ev.y), xu, acc[2 * q]);
                        acc[2 * q + 1] = __ffma2_rn(make_float2(ev.z, ev.w), xu, acc[2 * q + 1]);
                    }
                }
            }
            for (int grp = 0; kTwo && grp < ng2; ++grp) {
                float x[KU2];
#pragma unroll
                for (int u = 0; u < KU2; ++u) x[u] = f2.cvt(raw2[u]);
                const bool same = grp + 1 < ng2;
                if (same || (ng1 == 0 && more)) fetch2(same ? tl : tl + 1, same ? grp + 1 : 0);
                else if (more) fetch1(tl + 1, 0);
#pragma unroll
                for (int u = 0; u < KU2; ++u) {
                    const float4* er = es4 + (long long)(s2 + grp * KU2 + u) * (NJ / 4);
                    const float2 xu = make_float2(x[u], x[u]);
#pragma unroll
                    for (int q = 0; q < NJ / 4; ++q) {
                        const float4 ev = er[q];
                        acc[2 * q] = __ffma2_rn(make_float2(ev.x, ev.y), xu, acc[2 * q]);
                        acc[2 * q + 1] = __ffma2_rn(make_float2(ev.z, ev.w), xu, acc[2 * q + 1]);
                    }
                }
            }
            if (g < B.G) {
                double* o = out + B.off + g;
#pragma unroll
                for (int j = 0; j < NJ; ++j)
                    if (j < B.N) __stcs(o + (long long)j * B.G, f2d((j & 1) ? acc[j >> 1].y : acc[j >> 1].x));
            }
        }
        base += ntile;
        ++b;
    }
}

// R2 = RowsNone: a single segment (K2 = 0)
template <class R1, class R2>
static bool smallmat_rows(const flosic_ctx* c, const double* E, int mult, R1 r1, R2 r2, double* out,
                          cudaStream_t s) {
    const int nmax = max_block_n(c);
    if (c->opt.precision != FLOSIC_MIXED || nmax > 32 || mult * nmax > kRowMaxK) return false;
    long long total = 0;
    for (const auto& b : c->blk) total += (b.G + kRowTile - 1) / kRowTile;
    const long long wave = 2LL * c->num_sms;   // one wave of 2 CTAs per SM
    const unsigned grid = (unsigned)(total < wave ? total : wave);
    if (nmax <= 8) k_smallmat_rows<8><<<grid, kRowTile, 0, s>>>(c->d_blk, c->nblk, total, E, mult, r1, r2, out);
    else if (nmax <= 16) k_smallmat_rows<16><<<grid, kRowTile, 0, s>>>(c->d_blk, c->nblk, total, E, mult, r1, r2, out);
    else k_smallmat_rows<32><<<grid, kRowTile, 0, s>>>(c->d_blk, c->nblk, total, E, mult, r1, r2, out);
    note_launch(c);
    return true;
}

template <class LX>
static void smallmat(const flosic_ctx* c, const double* E, int mult, LX lx, double* out, cudaStream_t s) {
    const int nmax = max_block_n(c);
    long long gmax = 0;
    for (const auto& b : c->blk) gmax = b.G > gmax ? b.G : gmax;
    if (c->opt.precision == FLOSIC_MIXED) {   // 32-point tiles (128-point tiles measured no faster)
        const unsigned gx = (unsigned)((gmax + 31) / 32 < 65535 ? (gmax + 31) / 32 : 65535);
        const dim3 grid(gx, c->nblk);
        if (nmax <= 16) k_smallmat<2, 1, float><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else if (nmax <= 32) k_smallmat<4, 1, float><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else if (nmax <= 64) k_smallmat<8, 1, float><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else k_smallmat<16, 1, float><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
    } else {                                   // 32-point tiles
        const unsigned gx = (unsigned)((gmax + 31) / 32 < 65535 ? (gmax + 31) / 32 : 65535);
        const dim3 grid(gx, c->nblk);
        if (nmax <= 16) k_smallmat<2, 1, double><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else if (nmax <= 32) k_smallmat<4, 1, double><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else if (nmax <= 64) k_smallmat<8, 1, double><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
        else k_smallmat<16, 1, double><<<grid, 256, 0, s>>>(c->d_blk, E, mult, lx, out);
    }
    note_launch(c);
}

void launch_flo_apply(const flosic_ctx* c, const double* psi, double* phi, cudaStream_t s) {
    if (!smallmat_rows(c, c->ws.C, 1, RowsPsi<16>{psi}, RowsNone{}, phi, s)) smallmat(c, c->ws.C, 1, LoadPsi{psi}, phi, s);
}

// ---------------------------------------------------------------------------
// reverse mode, small part (one CTA per block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_backward_small(const BlkDesc* __restrict__ blk, Workspace w,
                                                        double* dE_dfod) {
    const BlkDesc& B = blk[blockIdx.x];
    const int N = B.N;
    const long long mo = B.moff;
    const double *P = w.P + mo, *T = w.T + mo, *Q = w.Q + mo, *U = w.U + mo, *M = w.M + mo;
    const double* lam = w.lam + B.orb0;
    const double* vals = w.vals + mo;
    const double* rho = w.rho_a + B.orb0;
    const long long me = w.mat_elems;
    double* A1 = w.tmp + mo;
    double* A2 = w.tmp + me + mo;
    double* A3 = w.tmp + 2 * me + mo;
    double* Ss = w.tmp + 3 * me + mo;   // Sbar + Sbar^T
    double* vbar = w.vbar + mo;
    double* E2 = w.E2 + 2 * mo;         // [N][2N] = [C^T | D]
    mm(N, P, false, T, true, A1);       // Qbar = P T^T
    mm(N, U, true, A1, false, A2);      // U^T Qbar
    mm(N, A2, false, U, false, A3);     // U^T Qbar U
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {   // o K
        const double ai = sqrt(lam[e / N]), aj = sqrt(lam[e % N]);
        A3[e] *= -1.0 / (ai * aj * (ai + aj));
    }
    __syncthreads();
    mm(N, U, false, A3, false, A2);     // U X
    mm(N, A2, false, U, true, A1);      // Sbar = U X U^T
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) Ss[e] = A1[e] + A1[(e % N) * N + e / N];
    __syncthreads();
    mm(N, Q, false, P, false, A1);      // Q P
    mm(N, Ss, false, T, false, A2);     // Ss T
    mm(N, A2, false, M, false, A3);     // Ss T M
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) A1[e] += A3[e];   // Tbar
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {          // vbar (product form)
        double tv = 0.0;
        for (int a = 0; a < N; ++a) tv += A1[i * N + a] * vals[i * N + a];
        const double sq = sqrt(rho[i]);
        for (int a = 0; a < N; ++a)
            vbar[i * N + a] = A1[i * N + a] / sq - vals[i * N + a] * tv / (rho[i] * sq);
    }
    __syncthreads();
    if (dE_dfod) {
        for (int e = threadIdx.x; e < 3 * N; e += blockDim.x) {
            const int i = e / 3, d = e % 3;
            double s = 0.0;
            for (int a = 0; a < N; ++a) s += vbar[i * N + a] * w.grads[3 * (mo + i * N + a) + d];
            dE_dfod[(B.fod_off + i) * 3 + d] = s;
        }
    }
    mm(N, T, true, Ss, false, A2);      // T^T Ss
    mm(N, A2, false, T, false, A3);     // T^T Ss T
    for (int e = threadIdx.x; e < 2 * N * N; e += blockDim.x) {
        const int j = e / (2 * N), k = e % (2 * N);
        E2[e] = (k < N) ? w.C[mo + k * N + j] : B.dV * A3[j * N + (k - N)];
    }
}

void launch_backward_small(const flosic_ctx* c, double* dE_dfod, cudaStream_t s) {
    k_backward_small<<<c->nblk, 512, 0, s>>>(c->d_blk, c->ws, dE_dfod); note_launch(c);
}

// The 64 tricubic interpolation nodes of every FOD (one thread per FOD and
// node): grid index within the orbital (-1 outside a Dirichlet box) and
// weight L_x L_y L_z.
__global__ void k_interp_nodes(const BlkDesc* __restrict__ blk, const int* __restrict__ orb_blk, int norb,
                               const double* __restrict__ fods, int* __restrict__ node_idx,
                               double* __restrict__ node_wt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 64LL * norb) return;
    const int f = (int)(t >> 6), node = (int)(t & 63);
    const BlkDesc& B = blk[orb_blk[f]];
    const double* fp = fods + (B.fod_off + (f - B.orb0)) * 3;
    const double fa[3] = {fp[0], fp[1], fp[2]};
    const Cell c = cell_of(B, fa);
    const int e = node & 3, bb = (node >> 2) & 3, cc = node >> 4;
    int qx = c.i0[0] - 1 + e, qy = c.i0[1] - 1 + bb, qz = c.i0[2] - 1 + cc;
    if (B.per) wrap_node(B, qx, qy, qz);
    const bool in = !(qx < 0 || qx >= B.nx || qy < 0 || qy >= B.ny || qz < 0 || qz >= B.nz);
    node_idx[t] = in ? (qz * B.ny + qy) * B.nx + qx : -1;
    node_wt[t] = c.L[0][e] * c.L[1][bb] * c.L[2][cc];
}

// psibar_a(node) += sum_i vbar_ia L(a_i, node): one warp per orbital a,
// FODs in sequence (deterministic); the next FOD's nodes, weights and
// coefficient are loaded before this FOD's read-modify-writes.
__global__ void k_interp_scatter(const BlkDesc* __restrict__ blk, const int* __restrict__ orb_blk,
                                 int norb, const double* __restrict__ vbar,
                                 const int* __restrict__ node_idx, const double* __restrict__ node_wt,
                                 double* __restrict__ dpsi) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= norb) return;
    const BlkDesc& B = blk[orb_blk[o]];
    const int a = o - B.orb0;
    double* u = dpsi + B.off + (long long)a * B.G;
    int ix0 = 0, ix1 = 0;
    double w0 = 0.0, w1 = 0.0, coef = 0.0;
    auto load = [&](int i) {
        const long long t = 64LL * (B.orb0 + i);
        ix0 = node_idx[t + lane];
        ix1 = node_idx[t + 32 + lane];
        w0 = node_wt[t + lane];
        w1 = node_wt[t + 32 + lane];
        coef = vbar[B.moff + i * B.N + a];
    };
    if (B.N > 0) load(0);
    for (int i = 0; i < B.N; ++i) {
        const int j0 = ix0, j1 = ix1;
        const double v0 = coef * w0, v1 = coef * w1;
        if (i + 1 < B.N) load(i + 1);
        if (j0 >= 0) u[j0] += v0;
        if (j1 >= 0) u[j1] += v1;
        __syncwarp();
    }
}

void launch_psibar(const flosic_ctx* c, const double* psi, const double* phi, const double* vsic,
                   const double* gE, const double* fods, double* dpsi, cudaStream_t s) {
    if (!vsic) {   // the energy pass stored wbar = V^SIC phi (mixed precision)
        if (!smallmat_rows(c, c->ws.E2, 2, RowsWbar{c->ws.wbar, gE}, RowsPsi<8>{psi}, dpsi, s))
            smallmat(c, c->ws.E2, 2, LoadPhibarPsi<LoadWbar>{LoadWbar{c->ws.wbar, gE}, psi}, dpsi, s);
    } else if (!smallmat_rows(c, c->ws.E2, 2, RowsPhibar{phi, vsic, gE}, RowsPsi<8>{psi}, dpsi, s)) {
        smallmat(c, c->ws.E2, 2, LoadPhibarPsi<LoadPhibar>{LoadPhibar{phi, vsic, gE}, psi}, dpsi, s);
    }
    k_interp_nodes<<<(unsigned)((64LL * c->norb + 255) / 256), 256, 0, s>>>(c->d_blk, c->d_orb_blk, c->norb, fods,
                                                                            c->ws.node_idx, c->ws.node_wt);
    note_launch(c);
    k_interp_scatter<<<(c->norb * 32 + 255) / 256, 256, 0, s>>>(c->d_blk, c->d_orb_blk, c->norb, c->ws.vbar,
                                                                 c->ws.node_idx, c->ws.node_wt, dpsi);
    note_launch(c);
}

}  // namespace flosic

namespace flosic {
const void* k_lowdin_symbol() { return (const void*)k_lowdin; }
}  // namespace flosic
