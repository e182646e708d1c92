// SC_AvgSIC Hamiltonian apply (Sec. II.C, Eq. 13): the averaged SIC
// potential enters one Kohn-Sham Hamiltonian per spin,
//   H psi_a = -1/2 Delta_h psi_a + (v_loc + V_avg,sigma) psi_a,
// with the same 12th-order Laplacian and zero Dirichlet boundary as the
// Poisson solves (orbitals vanish outside the box).  v_loc stands for the
// remaining local terms of Eq. 13 (external, Hartree, v_xc), one field per
// system; V_avg is the averaged SIC potential of the energy pass (already
// scaled by s), one field per spin block.  Either may be absent.
#include "ffsweep.cuh"

namespace flosic {

__constant__ double c_w64[kHalf + 1];   // this file's copy of the 12th-order weights

// Mixed precision: the Laplacian in float-float pairs on the staged sweep
// (psi split by integer operations), the potential term in pairs, one
// float64 addition per point for the float64 result.
__global__ void __launch_bounds__(256) k_hamiltonian_ff(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                        const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                        const double* __restrict__ psi, const double* __restrict__ vloc,
                                                        const double* __restrict__ vavg, double* __restrict__ hpsi) {
    __shared__ ff plane[kPY][kPX];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    const ff mh = to_ff(d2ff(-0.5 / (D.h * D.h)));
    ff_sweep12(
        D, P, [&](long long g) { return d2ff(psi[g]); },
        [&](long long g, ff u, ff acc) {
            const long long q = g - P.base;   // grid point within the orbital
            ff v = {0.f, 0.f};
            if (vloc) v = to_ff(d2ff(vloc[B.soff + q]));
            if (vavg) v = ff_add(v, to_ff(d2ff(vavg[B.voff + q])));
            const ff hv = ff_add(ff_mul(acc, mh), ff_mul(v, u));
            hpsi[g] = ff_to_double(hv);
        },
        plane);
}

// float64: plain loads of the 37 taps (through L1), float64 arithmetic.
__global__ void __launch_bounds__(256) k_hamiltonian64(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                       const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                       const double* __restrict__ psi, const double* __restrict__ vloc,
                                                       const double* __restrict__ vavg, double* __restrict__ hpsi) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    const BlkDesc& B = blk[P.b];
    double w[kHalf + 1];
#pragma unroll
    for (int m = 0; m <= kHalf; ++m) w[m] = c_w64[m];
    const double mh = -0.5 / (D.h * D.h);
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    const int x = P.x0 + threadIdx.x;
    if (x >= D.nx) return;
    for (int k = 0; k < 2; ++k) {
        const int y = P.y0 + threadIdx.y + k * (kTileY / 2);
        if (y >= D.ny) continue;
        for (int z = P.z0; z < P.z1; ++z) {
            const long long q = (long long)z * sz + y * sy + x;
            const long long g = P.base + q;
            const double u = psi[g];
            double acc = 3.0 * w[0] * u;
            for (int m = 1; m <= kHalf; ++m) {
                double s = 0.0;
                if (x - m >= 0) s += psi[g - m];
                if (x + m < D.nx) s += psi[g + m];
                if (y - m >= 0) s += psi[g - m * sy];
                if (y + m < D.ny) s += psi[g + m * sy];
                if (z - m >= 0) s += psi[g - m * sz];
                if (z + m < D.nz) s += psi[g + m * sz];
                acc += w[m] * s;
            }
            double v = 0.0;
            if (vloc) v += vloc[B.soff + q];
            if (vavg) v += vavg[B.voff + q];
            hpsi[g] = mh * acc + v * u;
        }
    }
}

void launch_hamiltonian(const flosic_ctx* c, const double* psi, const double* vloc, const double* vavg,
                        double* hpsi, cudaStream_t s) {
    const Multigrid& M = c->mg;
    const dim3 tb(kTileX, kTileY / 2);
    if (c->opt.precision == FLOSIC_MIXED)
        k_hamiltonian_ff<<<(unsigned)M.ntiles[0], tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, psi,
                                                               vloc, vavg, hpsi);
    else
        k_hamiltonian64<<<(unsigned)M.ntiles[0], tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, psi,
                                                              vloc, vavg, hpsi);
    note_launch((flosic_ctx*)c);
}

cudaError_t upload_hamiltonian_constants() {
    double w[kHalf + 1];
    stencil_weights(w);
    const cudaError_t e = cudaMemcpyToSymbol(c_w64, w, sizeof(w));
    if (e != cudaSuccess) return e;
    return upload_ffsweep_weights();
}

}  // namespace flosic
