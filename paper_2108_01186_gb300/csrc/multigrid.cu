// Multigrid preconditioner of the Poisson CG (Sec. II.A solves the
// electrostatics iteratively; the solver here is preconditioned CG).
//
// M ~ A2^{-1}, one V-cycle on the 7-point Laplacian A2 (spacing 2^l h on
// level l, zero outside the interior).  A2 and the 12th-order operator A
// satisfy 1 <= x^T A x / x^T A2 x <= 1.77 for every grid function vanishing
// outside the interior (the ratio of their Fourier symbols), so CG on A with
// this preconditioner converges in a few tens of iterations at any grid
// size instead of O(n).
//
// Vertex-centred coarsening: coarse point I sits on fine point 2I+1,
// n_c = floor(n/2); coarsen while every side is >= 6.  Restriction is full
// weighting (1/4, 1/2, 1/4 per direction) = (1/8) P^T with P trilinear
// interpolation.  Smoother: one damped-Jacobi sweep before and after
// (omega = 0.8); coarsest level: 40 damped-Jacobi sweeps from zero in shared
// memory.  Every piece is symmetric and the smoother converges in the A2
// norm, so the V-cycle is a symmetric positive definite operator.
//
// Kernels work on per-level tables of 3-D tiles (one CTA per 32 x 16 x 32
// tile of one orbital) so that all orbitals of all systems run in one launch
// per level.
#include "internal.cuh"

namespace flosic {

// Each CTA (32 x 8 threads) owns a 32 x 16 x 32 tile of one orbital on one
// level: thread (tx, ty) handles the points (x0+tx, y0+ty+8k, z), k = 0, 1,
// for every plane z of the tile.  Neighbours come through L1.
template <class Body>
__device__ __forceinline__ void for_tile_points(const LvlDesc& D, const TilePos& P, Body body) {
    const int x = P.x0 + threadIdx.x;
    if (x >= D.nx) return;
    for (int k = 0; k < 2; ++k) {
        const int y = P.y0 + threadIdx.y + k * (kTileY / 2);
        if (y >= D.ny) continue;
        for (int z = P.z0; z < P.z1; ++z) body(x, y, z, ((long long)z * D.ny + y) * D.nx + x);
    }
}

// sum of the six neighbours (zero outside)
template <class T>
__device__ __forceinline__ T nbr6(const T* __restrict__ u, long long g, int x, int y, int z, const LvlDesc& D) {
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    T s = 0;
    if (x > 0) s += u[g - 1];
    if (x < D.nx - 1) s += u[g + 1];
    if (y > 0) s += u[g - sy];
    if (y < D.ny - 1) s += u[g + sy];
    if (z > 0) s += u[g - sz];
    if (z < D.nz - 1) s += u[g + sz];
    return s;
}

// s = r - A2 (omega D^-1 r) = (1 - omega) r + (omega/6) sum_nbr r
template <class T>
__global__ void __launch_bounds__(256) k_mg_resid_smooth(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                         const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                         const int* __restrict__ active, const T* __restrict__ r,
                                                         T* __restrict__ s, T omega) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    if (!active[P.o] || D.coarsest) return;
    const T* rb = r + P.base;
    T* sb = s + P.base;
    for_tile_points(D, P, [&](int x, int y, int z, long long g) {
        sb[g] = (T(1) - omega) * rb[g] + omega * T(1.0 / 6.0) * nbr6(rb, g, x, y, z, D);
    });
}

// r_c(I) = sum over the 27 fine neighbours of 2I+1 of (1/4,1/2,1/4)^3 s_f
template <class T>
__global__ void __launch_bounds__(256) k_mg_restrict(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ Lc,
                                                     const LvlDesc* __restrict__ Lf, const int4* __restrict__ tiles_c,
                                                     const int* __restrict__ orb_blk, const int* __restrict__ active,
                                                     const T* __restrict__ sf, T* __restrict__ rc) {
    const TilePos P = tile_pos(blk, Lc, tiles_c, orb_blk, blockIdx.x);
    if (!active[P.o]) return;
    const LvlDesc& C = Lc[P.b];
    const LvlDesc& F = Lf[P.b];
    const T* fb = sf + F.off + (long long)(P.o - blk[P.b].orb0) * F.G;
    T* cb = rc + P.base;
    const long long fy = F.nx, fz = (long long)F.nx * F.ny;
    for_tile_points(C, P, [&](int X, int Y, int Z, long long g) {
        T acc = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int zf = 2 * Z + c;
            if (zf >= F.nz) continue;
            const T wc = (c == 1) ? T(0.5) : T(0.25);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int yf = 2 * Y + b;
                if (yf >= F.ny) continue;
                const T wb = (b == 1) ? T(0.5) : T(0.25);
                const T* row = fb + zf * fz + yf * fy + 2 * X;
                T rsum = T(0.25) * row[0] + T(0.5) * row[1];
                if (2 * X + 2 < F.nx) rsum += T(0.25) * row[2];
                acc += wc * wb * rsum;
            }
        }
        cb[g] = acc;
    });
}

// trilinear prolongation of the coarse correction at fine point (x, y, z)
template <class T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ ec, const LvlDesc& C, int x, int y, int z) {
    int I0[3], I1[3];
    T w0[3], w1[3];
    const int p[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (p[d] & 1) {              // on a coarse point
            I0[d] = (p[d] - 1) >> 1; w0[d] = T(1);
            I1[d] = -1;              w1[d] = T(0);
        } else {                     // halfway between two coarse points
            I0[d] = (p[d] >> 1) - 1; w0[d] = T(0.5);
            I1[d] = p[d] >> 1;       w1[d] = T(0.5);
        }
    }
    const int n[3] = {C.nx, C.ny, C.nz};
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int Z = c ? I1[2] : I0[2];
        const T wz = c ? w1[2] : w0[2];
        if (Z < 0 || Z >= n[2] || wz == T(0)) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int Y = b ? I1[1] : I0[1];
            const T wy = b ? w1[1] : w0[1];
            if (Y < 0 || Y >= n[1] || wy == T(0)) continue;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int X = a ? I1[0] : I0[0];
                const T wx = a ? w1[0] : w0[0];
                if (X < 0 || X >= n[0] || wx == T(0)) continue;
                acc += wz * wy * wx * ec[((long long)Z * n[1] + Y) * n[0] + X];
            }
        }
    }
    return acc;
}

// t = omega D^-1 r + P e_c   (pre-smoothed part plus the coarse correction)
template <class T>
__global__ void __launch_bounds__(256) k_mg_prolong(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ Lf,
                                                    const LvlDesc* __restrict__ Lc, const int4* __restrict__ tiles_f,
                                                    const int* __restrict__ orb_blk, const int* __restrict__ active,
                                                    const T* __restrict__ r, const T* __restrict__ ec,
                                                    T* __restrict__ t, T omega) {
    const TilePos P = tile_pos(blk, Lf, tiles_f, orb_blk, blockIdx.x);
    const LvlDesc& F = Lf[P.b];
    if (!active[P.o] || F.coarsest) return;
    const LvlDesc& C = Lc[P.b];
    const T* eb = ec + C.off + (long long)(P.o - blk[P.b].orb0) * C.G;
    const T* rb = r + P.base;
    T* tb = t + P.base;
    const T dinv = omega * T(F.h * F.h / 6.0);
    for_tile_points(F, P, [&](int x, int y, int z, long long g) { tb[g] = dinv * rb[g] + prolong_at(eb, C, x, y, z); });
}

// e = t + omega D^-1 (r - A2 t) = (1 - omega) t + (omega/6)(h^2 r + sum_nbr t);
// on level 0 also z.r per orbital -> rz, beta = rz / rz_old.
template <class T, bool kLevel0>
__global__ void __launch_bounds__(256) k_mg_postsmooth(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                       const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                       const int* __restrict__ active, const T* __restrict__ r,
                                                       const T* __restrict__ t, T* __restrict__ e, T omega,
                                                       CgState st) {
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    if (!active[P.o] || D.coarsest) return;
    const T* tb = t + P.base;
    const T* rb = r + P.base;
    T* eb = e + P.base;
    const T h2 = T(D.h * D.h);
    double rz = 0.0;
    for_tile_points(D, P, [&](int x, int y, int z, long long g) {
        const T rv = rb[g];
        const T ev = (T(1) - omega) * tb[g] + omega * T(1.0 / 6.0) * (h2 * rv + nbr6(tb, g, x, y, z, D));
        eb[g] = ev;
        if (kLevel0) rz += (double)rv * (double)ev;
    });
    if (kLevel0) {
        if (tile_arrive(rz, st.part, blockIdx.x, st.count + P.o, D.ntile, scratch)) {
            const double v = tile_gather(st.part, P.first, D.ntile, scratch);
            if (linear_tid() == 0) {
                st.count[P.o] = 0;
                const double old = st.rz[P.o];
                st.beta[P.o] = (old != 0.0) ? v / old : 0.0;
                st.rz[P.o] = v;
            }
        }
    }
}

// Coarsest level of each block: damped Jacobi from zero, in shared memory,
// one CTA per orbital.  When the coarsest level is level 0 this is the whole
// preconditioner and the CTA also forms rz and beta.
template <class T>
__global__ void k_mg_coarsest(const BlkDesc* __restrict__ blk, MgPtrs<T> mp, const int* __restrict__ orb_blk,
                              int norb, const int* __restrict__ active, T omega, int nsweep, CgState st) {
    extern __shared__ unsigned char smem_raw[];
    T* sh = reinterpret_cast<T*>(smem_raw);
    __shared__ double scratch[32];
    const int o = blockIdx.x;
    if (o >= norb || !active[o]) return;
    const int b = orb_blk[o];
    const int lev = mp.coarsest_level[b];
    const LvlDesc& D = mp.lvl[lev][b];
    const int i = o - blk[b].orb0;
    const int G = (int)D.G;
    const long long base = D.off + (long long)i * D.G;
    const T* r = mp.r[lev] + base;
    T* e = mp.e[lev] + base;
    T* rs = sh;
    T* ea = sh + G;
    T* eb = sh + 2 * G;
    const T h2 = T(D.h * D.h);
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        rs[k] = r[k];
        ea[k] = omega * h2 * T(1.0 / 6.0) * rs[k];
    }
    __syncthreads();
    const int pl = D.nx * D.ny;
    for (int sw = 1; sw < nsweep; ++sw) {
        for (int k = threadIdx.x; k < G; k += blockDim.x) {
            const int z = k / pl, rem = k - z * pl, y = rem / D.nx, x = rem - y * D.nx;
            eb[k] = (T(1) - omega) * ea[k] + omega * T(1.0 / 6.0) * (h2 * rs[k] + nbr6(ea, k, x, y, z, D));
        }
        __syncthreads();
        T* tmp = ea; ea = eb; eb = tmp;
    }
    double rz = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        e[k] = ea[k];
        rz += (double)rs[k] * (double)ea[k];
    }
    if (lev == 0) {
        rz = block_sum(rz, scratch);
        if (threadIdx.x == 0) {
            const double old = st.rz[o];
            st.beta[o] = (old != 0.0) ? rz / old : 0.0;
            st.rz[o] = rz;
        }
    }
}

template <class T>
void launch_vcycle(const flosic_ctx* c, const MgPtrs<T>& mp, const int* active, cudaStream_t s) {
    const Multigrid& M = c->mg;
    const T omega = T(0.8);
    const int thr = kChunkThreads;
    const dim3 tb(kTileX, kTileY / 2);
    for (int l = 0; l + 1 < M.nlev; ++l) {
        if (M.ntiles[l] > 0) {
            k_mg_resid_smooth<T><<<(unsigned)M.ntiles[l], tb, 0, s>>>(c->d_blk, M.d_lvl[l], M.d_tiles[l],
                                                                     c->d_orb_blk, active, mp.r[l], mp.t[l],
                                                                     omega); note_launch(c);
        }
        if (M.ntiles[l + 1] > 0) {
            k_mg_restrict<T><<<(unsigned)M.ntiles[l + 1], tb, 0, s>>>(c->d_blk, M.d_lvl[l + 1], M.d_lvl[l],
                                                                     M.d_tiles[l + 1], c->d_orb_blk, active,
                                                                     mp.t[l], mp.r[l + 1]); note_launch(c);
        }
    }
    const size_t shm = 3 * sizeof(T) * (size_t)M.coarsest_max;
    k_mg_coarsest<T><<<c->norb, thr, shm, s>>>(c->d_blk, mp, c->d_orb_blk, c->norb, active, omega,
                                               kCoarseSweeps, c->ws.cg); note_launch(c);
    for (int l = M.nlev - 2; l >= 0; --l) {
        if (M.ntiles[l] == 0) continue;
        k_mg_prolong<T><<<(unsigned)M.ntiles[l], tb, 0, s>>>(c->d_blk, M.d_lvl[l], M.d_lvl[l + 1],
                                                            M.d_tiles[l], c->d_orb_blk, active, mp.r[l],
                                                            mp.e[l + 1], mp.t[l], omega); note_launch(c);
        if (l == 0)
            k_mg_postsmooth<T, true><<<(unsigned)M.ntiles[0], tb, 0, s>>>(
                c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, active, mp.r[0], mp.t[0], mp.e[0], omega,
                c->ws.cg);
        else
            k_mg_postsmooth<T, false><<<(unsigned)M.ntiles[l], tb, 0, s>>>(
                c->d_blk, M.d_lvl[l], M.d_tiles[l], c->d_orb_blk, active, mp.r[l], mp.t[l], mp.e[l], omega,
                c->ws.cg);
        note_launch(c);
    }
}

template void launch_vcycle<float>(const flosic_ctx*, const MgPtrs<float>&, const int*, cudaStream_t);
template void launch_vcycle<double>(const flosic_ctx*, const MgPtrs<double>&, const int*, cudaStream_t);

}  // namespace flosic
