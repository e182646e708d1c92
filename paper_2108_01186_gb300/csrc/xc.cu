// PZ-SIC energy (Eq. 1) and the averaged SIC potential (Eq. 13).
//
// Per spin block, one pass over the grid with every orbital of the block:
//   rho_i = phi_i^2, (eps_i, v_xc,i) = fully polarised LSDA of rho_i,
//   partial sums of rho_i V_i and rho_i eps_i per orbital (-> U_i, E_xc,i),
//   V_avg = scale * sum_i rho_i V_i^SIC / rho_spin, V_i^SIC = -(V_i + v_xc,i),
//   rho_spin = sum_a psi_a^2 (V_avg = 0 where rho_spin <= rho_min).
#include <type_traits>

#include "internal.cuh"
#include "xc_device.cuh"

namespace flosic {

// 256 threads per chunk, 4 points each (64 threads with 16 points each, which
// shares the per-orbital warp sums among more points, measured 1.9x slower)
constexpr int kXcThreads = kChunkThreads;
constexpr int kXcPts = kChunk / kXcThreads;   // points per thread

// Warp sum of float partials carried as a float-float pair (two-sum per
// level), returned in float64.
__device__ __forceinline__ double warp_sum_ff(float v) {
    float h = v, l = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        const float s = h + oh, bb = s - h;
        const float e = (h - (s - bb)) + (oh - bb) + (l + ol);
        h = s + e;
        l = e - (h - s);
    }
    return f2d(h) + f2d(l);
}

// kF32 (mixed precision): no float64 operation per point.  The float64
// inputs are converted with integer operations; rho V (for U_i) is formed and
// summed as float-float pairs, the functional, V^SIC and V_avg in float32;
// per-orbital sums are float-float within a warp, float64 across warps.
// Otherwise float64 throughout.
// Also stores, for the reverse mode, V_i^SIC = -(V_i + v_xc,i) (vsic, float64)
// or wbar_i = V_i^SIC phi_i (wbar, float32; kF32 only); either may be null.
template <bool kF32>
__global__ void __launch_bounds__(kXcThreads)
k_xc_energy(const BlkDesc* __restrict__ blk, const double* __restrict__ psi,
            const double* __restrict__ phi, const double* __restrict__ V, double scale,
            double rho_min, double* __restrict__ Vavg, double* __restrict__ e_part,
            double* __restrict__ vsic, float* __restrict__ wbar, const int* __restrict__ mask) {
    using R = typename std::conditional<kF32, float, double>::type;
    __shared__ double red[kXcThreads / 32][kMaxN][2];
    const BlkDesc& B = blk[blockIdx.y];
    const int c = blockIdx.x;
    if (c >= B.nchunk) return;
    const long long g0 = (long long)c * kChunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const R rmin = (R)rho_min;
    R num[kXcPts], rs[kXcPts];
#pragma unroll
    for (int k = 0; k < kXcPts; ++k) num[k] = rs[k] = R(0);
    for (int i = 0; i < B.N; ++i) {
        const long long base = B.off + (long long)i * B.G;
        const bool on = mask[B.orb0 + i] != 0;   // masked: only its psi^2 enters (rho_sigma)
        R u = R(0), ex = R(0);
        ff uff = {0.f, 0.f};   // kF32: rho V as pairs (U to ~1e-13 relative)
#pragma unroll
        for (int k = 0; k < kXcPts; ++k) {
            const long long g = g0 + threadIdx.x + k * kXcThreads;
            if (g >= B.G) continue;
            if (!on) {
                const R p = kF32 ? (R)d2f(psi[base + g]) : (R)psi[base + g];
                rs[k] += p * p;
                if (vsic) vsic[base + g] = 0.0;
                if (kF32 && wbar) wbar[base + g] = 0.f;
                continue;
            }
            R f, v, p, eps, vxc;
            if (kF32) {
                const float2 f2 = d2ff(phi[base + g]), v2 = d2ff(V[base + g]);
                f = f2.x;
                v = v2.x;
                p = d2f(psi[base + g]);
                const float ph = f2.x * f2.x;
                const ff rho2 = ff_quick(ph, fmaf(f2.x, f2.x, -ph) + 2.f * f2.x * f2.y);
                const float pv = rho2.h * v2.x;   // rho V as an unnormalised pair
                uff = ff_acc(uff, pv, fmaf(rho2.h, v2.y, fmaf(rho2.l, v2.x, fmaf(rho2.h, v2.x, -pv))));
                float ef, vf;
                lsda_pol_f(f * f, (float)rmin, ef, vf);
                eps = ef;
                vxc = vf;
            } else {
                f = phi[base + g];
                v = V[base + g];
                p = psi[base + g];
                double ed, vd;
                lsda_pol(f * f, rho_min, ed, vd);
                eps = (R)ed;
                vxc = (R)vd;
            }
            const R rho = f * f;
            u += rho * v;
            ex += rho * eps;
            const R vs = -(v + vxc);
            if (kF32) {
                if (vsic) vsic[base + g] = f2d((float)vs);
                if (wbar) __stcs(wbar + base + g, (float)vs * (float)f);
            } else {
                vsic[base + g] = (double)vs;
            }
            num[k] += rho * vs;
            rs[k] += p * p;
        }
        double us, es;
        if (kF32) {
            us = ff_to_double(warp_sum(ff_quick(uff.h, uff.l)));
            es = warp_sum_ff((float)ex);
        } else {
            us = warp_sum((double)u);
            es = warp_sum((double)ex);
        }
        if (lane == 0) {
            red[wid][i][0] = us;
            red[wid][i][1] = es;
        }
    }
    if (Vavg) {
#pragma unroll
        for (int k = 0; k < kXcPts; ++k) {
            const long long g = g0 + threadIdx.x + k * kXcThreads;
            if (g >= B.G) continue;
            if (kF32)
                Vavg[B.voff + g] = (rs[k] > rmin) ? f2d((float)scale * ((float)num[k] / (float)rs[k])) : 0.0;
            else
                Vavg[B.voff + g] = (rs[k] > rmin) ? scale * (double)num[k] / (double)rs[k] : 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * B.N; e += blockDim.x) {
        const int i = e >> 1, q = e & 1;
        double s = 0.0;
        for (int w = 0; w < kXcThreads / 32; ++w) s += red[w][i][q];
        e_part[(B.chunk0 + (long long)i * B.nchunk + c) * 2 + q] = s;
    }
}

void launch_xc_energy(const flosic_ctx* c, const double* psi, const double* phi, const double* V,
                      double scale, double* Vavg, cudaStream_t s) {
    int cmax = 0;
    for (const auto& b : c->blk) cmax = b.nchunk > cmax ? b.nchunk : cmax;
    const dim3 grid(cmax, c->nblk);
    if (c->opt.precision == FLOSIC_MIXED)
        k_xc_energy<true><<<grid, kXcThreads, 0, s>>>(c->d_blk, psi, phi, V, scale, c->opt.rho_min, Vavg,
                                                         c->ws.e_part, c->ws.vsic, c->ws.wbar, c->ws.mask);
    else
        k_xc_energy<false><<<grid, kXcThreads, 0, s>>>(c->d_blk, psi, phi, V, scale, c->opt.rho_min, Vavg,
                                                          c->ws.e_part, c->ws.vsic, nullptr, c->ws.mask);
    note_launch(c);
}

// One warp per orbital: U_i = (dV/2) sum rho V, E_xc,i = dV sum rho eps.
__global__ void k_energy_orb(const BlkDesc* __restrict__ blk, const int* __restrict__ orb_blk, int norb,
                             const double* __restrict__ e_part, double* __restrict__ e_orb,
                             double* U, double* Exc) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= norb) return;
    const BlkDesc& B = blk[orb_blk[o]];
    const long long first = B.chunk0 + (long long)(o - B.orb0) * B.nchunk;
    double u = 0.0, ex = 0.0;
    for (int k = lane; k < B.nchunk; k += 32) {
        u += e_part[(first + k) * 2 + 0];
        ex += e_part[(first + k) * 2 + 1];
    }
    u = warp_sum(u) * 0.5 * B.dV;
    ex = warp_sum(ex) * B.dV;
    if (lane == 0) {
        e_orb[2 * o] = u;
        e_orb[2 * o + 1] = ex;
        if (U) U[o] = u;
        if (Exc) Exc[o] = ex;
    }
}

// E_sic[s] = -sum over the orbitals of system s of (U + E_xc), in order.
__global__ void k_energy_sys(int nsys, const int* __restrict__ sys_orb0, const double* __restrict__ e_orb,
                             double* E_sic) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    double e = 0.0;
    for (int o = sys_orb0[s]; o < sys_orb0[s + 1]; ++o) e -= e_orb[2 * o] + e_orb[2 * o + 1];
    E_sic[s] = e;
}

void launch_energy_reduce(const flosic_ctx* c, double* U, double* Exc, double* E_sic, cudaStream_t s) {
    k_energy_orb<<<(c->norb * 32 + 255) / 256, 256, 0, s>>>(c->d_blk, c->d_orb_blk, c->norb, c->ws.e_part,
                                                            c->ws.e_orb, U, Exc); note_launch(c);
    if (E_sic) {
        const int nsys = (int)c->sys.size();
        k_energy_sys<<<(nsys + 127) / 128, 128, 0, s>>>(nsys, c->d_sys_orb0, c->ws.e_orb, E_sic); note_launch(c);
    }
}

}  // namespace flosic
