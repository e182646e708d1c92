// PZ-SIC energy (Eq. 1) and the averaged SIC potential (Eq. 13).
//
// Per spin block, one pass over the grid with every orbital of the block:
//   rho_i = phi_i^2, (eps_i, v_xc,i) = fully polarised LSDA of rho_i,
//   partial sums of rho_i V_i and rho_i eps_i per orbital (-> U_i, E_xc,i),
//   V_avg = scale * sum_i rho_i V_i^SIC / rho_spin, V_i^SIC = -(V_i + v_xc,i),
//   rho_spin = sum_a psi_a^2 (V_avg = 0 where rho_spin <= rho_min).
#include "internal.cuh"
#include "xc_device.cuh"

namespace flosic {

constexpr int kXcPts = kChunk / kChunkThreads;   // points per thread

// kF32: pointwise functional in float32 (mixed precision); sums in float64.
// Also stores V_i^SIC = -(V_i + v_xc,i) for the reverse mode.
template <bool kF32>
__global__ void __launch_bounds__(kChunkThreads)
k_xc_energy(const BlkDesc* __restrict__ blk, const double* __restrict__ psi,
            const double* __restrict__ phi, const double* __restrict__ V, double scale,
            double rho_min, double* __restrict__ Vavg, double* __restrict__ e_part,
            double* __restrict__ vsic) {
    __shared__ double red[kChunkThreads / 32][kMaxN][2];
    const BlkDesc& B = blk[blockIdx.y];
    const int c = blockIdx.x;
    if (c >= B.nchunk) return;
    const long long g0 = (long long)c * kChunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double num[kXcPts], rs[kXcPts];
#pragma unroll
    for (int k = 0; k < kXcPts; ++k) num[k] = rs[k] = 0.0;
    for (int i = 0; i < B.N; ++i) {
        const long long base = B.off + (long long)i * B.G;
        double u = 0.0, ex = 0.0;
#pragma unroll
        for (int k = 0; k < kXcPts; ++k) {
            const long long g = g0 + threadIdx.x + k * kChunkThreads;
            if (g >= B.G) continue;
            const double f = phi[base + g], v = V[base + g], p = psi[base + g];
            const double rho = f * f;
            double eps, vxc;
            if (kF32) {
                float ef, vf;
                lsda_pol_f((float)rho, (float)rho_min, ef, vf);
                eps = ef;
                vxc = vf;
            } else {
                lsda_pol(rho, rho_min, eps, vxc);
            }
            u += rho * v;
            ex += rho * eps;
            const double vs = -(v + vxc);
            vsic[base + g] = vs;
            num[k] += rho * vs;
            rs[k] += p * p;
        }
        u = warp_sum(u);
        ex = warp_sum(ex);
        if (lane == 0) {
            red[wid][i][0] = u;
            red[wid][i][1] = ex;
        }
    }
    if (Vavg) {
#pragma unroll
        for (int k = 0; k < kXcPts; ++k) {
            const long long g = g0 + threadIdx.x + k * kChunkThreads;
            if (g < B.G) Vavg[B.voff + g] = (rs[k] > rho_min) ? scale * num[k] / rs[k] : 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * B.N; e += blockDim.x) {
        const int i = e >> 1, q = e & 1;
        double s = 0.0;
        for (int w = 0; w < kChunkThreads / 32; ++w) s += red[w][i][q];
        e_part[(B.chunk0 + (long long)i * B.nchunk + c) * 2 + q] = s;
    }
}

void launch_xc_energy(const flosic_ctx* c, const double* psi, const double* phi, const double* V,
                      double scale, double* Vavg, cudaStream_t s) {
    int cmax = 0;
    for (const auto& b : c->blk) cmax = b.nchunk > cmax ? b.nchunk : cmax;
    const dim3 grid(cmax, c->nblk);
    if (c->opt.precision == FLOSIC_MIXED)
        k_xc_energy<true><<<grid, kChunkThreads, 0, s>>>(c->d_blk, psi, phi, V, scale, c->opt.rho_min, Vavg,
                                                         c->ws.e_part, c->ws.vsic);
    else
        k_xc_energy<false><<<grid, kChunkThreads, 0, s>>>(c->d_blk, psi, phi, V, scale, c->opt.rho_min, Vavg,
                                                          c->ws.e_part, c->ws.vsic);
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
