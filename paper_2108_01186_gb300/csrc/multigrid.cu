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
// n_c = floor(n/2); coarsen while every side is >= 6.  On an even side the
// last coarse point is the last fine point, so the coarse grid's zero
// boundary would sit one coarse spacing out while the true one is closer:
// the 7-point operator of such a level keeps the off-diagonal -1/h_l^2 but
// takes at the last point of that dimension the diagonal weight of the 1-D
// Galerkin operator P^T A P / 2 (c' = 2c - 1 for an even parent side,
// 1 + c/2 for an odd one, c = 2 on the fine grid).  Without it the V-cycle
// loses most of its strength on grids such as 128^3.  Restriction is full
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

// 1 / (sum of the diagonal weights) at (x, y, z) of a level: 1/6 away from
// the last point of every dimension.
template <class T>
__device__ __forceinline__ T inv_diag(const LvlDesc& D, int x, int y, int z) {
    const int m = (x == D.nx - 1 ? 1 : 0) | (y == D.ny - 1 ? 2 : 0) | (z == D.nz - 1 ? 4 : 0);
    return T(D.idd[m]);
}

template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Gathers, for n consecutive points starting at (x, y, z) (n = vector width
// or 1), the centre values and the sum of the six neighbours (zero outside).
template <class T, int V>
__device__ __forceinline__ void centre_nbr(const T* __restrict__ u, const LvlDesc& D, int x, int y, int z,
                                           long long g, int n, T* c, T* nb) {
    using VT = typename Vec<T>::type;
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    if (n == V) {
        const VT cv = *reinterpret_cast<const VT*>(u + g);
        VT ym, yp, zm, zp;
        const T* cs = reinterpret_cast<const T*>(&cv);
        T zero[V];
#pragma unroll
        for (int k = 0; k < V; ++k) zero[k] = T(0);
        ym = (y > 0) ? *reinterpret_cast<const VT*>(u + g - sy) : *reinterpret_cast<const VT*>(zero);
        yp = (y < D.ny - 1) ? *reinterpret_cast<const VT*>(u + g + sy) : *reinterpret_cast<const VT*>(zero);
        zm = (z > 0) ? *reinterpret_cast<const VT*>(u + g - sz) : *reinterpret_cast<const VT*>(zero);
        zp = (z < D.nz - 1) ? *reinterpret_cast<const VT*>(u + g + sz) : *reinterpret_cast<const VT*>(zero);
        const T xl = (x > 0) ? u[g - 1] : T(0);
        const T xr = (x + V < D.nx) ? u[g + V] : T(0);
        const T* a = reinterpret_cast<const T*>(&ym);
        const T* b = reinterpret_cast<const T*>(&yp);
        const T* cz = reinterpret_cast<const T*>(&zm);
        const T* d = reinterpret_cast<const T*>(&zp);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            c[k] = cs[k];
            const T left = (k == 0) ? xl : cs[k - 1];
            const T right = (k == V - 1) ? xr : cs[k + 1];
            nb[k] = left + right + a[k] + b[k] + cz[k] + d[k];
        }
    } else {
        c[0] = u[g];
        T sum = 0;
        if (x > 0) sum += u[g - 1];
        if (x < D.nx - 1) sum += u[g + 1];
        if (y > 0) sum += u[g - sy];
        if (y < D.ny - 1) sum += u[g + sy];
        if (z > 0) sum += u[g - sz];
        if (z < D.nz - 1) sum += u[g + sz];
        nb[0] = sum;
    }
}

template <class T, int V>
__device__ __forceinline__ void store_n(T* dst, const T* v, int n) {
    using VT = typename Vec<T>::type;
    if (n == V) *reinterpret_cast<VT*>(dst) = *reinterpret_cast<const VT*>(v);
    else dst[0] = v[0];
}

// s = r - A2 (omega D^-1 r) = (1 - omega) r + omega sum_nbr r / dd(nbr),
// dd = 6 except on the last points of a level with corrected weights.
template <class T>
__global__ void __launch_bounds__(256) k_mg_resid_smooth(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                         const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                         const int* __restrict__ active, const T* __restrict__ r,
                                                         T* __restrict__ s, T omega) {
    constexpr int V = Vec<T>::n;
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    if (!active[P.o] || D.coarsest) return;
    const long long sy = D.nx, sz = (long long)D.nx * D.ny;
    tile_rows<T>(D, P, [&](int x, int y, int z, long long g, int n) {
        if (D.corr && (x + n >= D.nx - 1 || y >= D.ny - 2 || z >= D.nz - 2)) {
            // a neighbour may lie on a last point: weight each one
            for (int k = 0; k < n; ++k) {
                const int xk = x + k;
                const long long gk = g + k;
                T sum = T(0);
                if (xk > 0) sum += r[gk - 1] * inv_diag<T>(D, xk - 1, y, z);
                if (xk < D.nx - 1) sum += r[gk + 1] * inv_diag<T>(D, xk + 1, y, z);
                if (y > 0) sum += r[gk - sy] * inv_diag<T>(D, xk, y - 1, z);
                if (y < D.ny - 1) sum += r[gk + sy] * inv_diag<T>(D, xk, y + 1, z);
                if (z > 0) sum += r[gk - sz] * inv_diag<T>(D, xk, y, z - 1);
                if (z < D.nz - 1) sum += r[gk + sz] * inv_diag<T>(D, xk, y, z + 1);
                s[gk] = (T(1) - omega) * r[gk] + omega * sum;
            }
            return;
        }
        T c[V], nb[V], out[V];
        centre_nbr<T, V>(r, D, x, y, z, g, n, c, nb);
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = (T(1) - omega) * c[k] + omega * T(1.0 / 6.0) * nb[k];
        store_n<T, V>(s + g, out, n);
    });
}

// r_c(I) = sum over the 27 fine neighbours of 2I+1 of (1/4,1/2,1/4)^3 s_f;
// V consecutive coarse points per thread, fine rows read with vector loads
// when they are aligned.
template <class T>
__global__ void __launch_bounds__(256) k_mg_restrict(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ Lc,
                                                     const LvlDesc* __restrict__ Lf, const int4* __restrict__ tiles_c,
                                                     const int* __restrict__ orb_blk, const int* __restrict__ active,
                                                     const T* __restrict__ sf, T* __restrict__ rc) {
    constexpr int V = Vec<T>::n;
    using VT = typename Vec<T>::type;
    const TilePos P = tile_pos(blk, Lc, tiles_c, orb_blk, blockIdx.x);
    if (!active[P.o]) return;
    const LvlDesc& C = Lc[P.b];
    const LvlDesc& F = Lf[P.b];
    const long long fbase = F.off + (long long)(P.o - blk[P.b].orb0) * F.G;
    const T* fb = sf + fbase;
    const long long fy = F.nx, fz = (long long)F.nx * F.ny;
    const bool fvec = (F.nx % (2 * V) == 0) && (fbase % (2 * V) == 0);
    tile_rows<T>(C, P, [&](int X, int Y, int Z, long long g, int n) {
        T acc[V];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = T(0);
        const int xf0 = 2 * X;
        for (int c = 0; c < 3; ++c) {
            const int zf = 2 * Z + c;
            if (zf >= F.nz) continue;
            const T wc = (c == 1) ? T(0.5) : T(0.25);
            for (int b = 0; b < 3; ++b) {
                const int yf = 2 * Y + b;
                if (yf >= F.ny) continue;
                const T w = wc * ((b == 1) ? T(0.5) : T(0.25));
                const T* row = fb + zf * fz + yf * fy;
                T f[2 * V + 1];
                if (n == V && fvec) {
                    const VT a0 = *reinterpret_cast<const VT*>(row + xf0);
                    const VT a1 = *reinterpret_cast<const VT*>(row + xf0 + V);
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        f[k] = reinterpret_cast<const T*>(&a0)[k];
                        f[V + k] = reinterpret_cast<const T*>(&a1)[k];
                    }
                    f[2 * V] = (xf0 + 2 * V < F.nx) ? row[xf0 + 2 * V] : T(0);
                } else {
#pragma unroll
                    for (int k = 0; k < 2 * V + 1; ++k) f[k] = (xf0 + k < F.nx) ? row[xf0 + k] : T(0);
                }
#pragma unroll
                for (int k = 0; k < V; ++k)
                    acc[k] += w * (T(0.25) * f[2 * k] + T(0.5) * f[2 * k + 1] + T(0.25) * f[2 * k + 2]);
            }
        }
        store_n<T, V>(rc + g, acc, n);
    });
}

// trilinear prolongation at fine x from one coarse row (OOB zero)
template <class T>
__device__ __forceinline__ T prolong_x(const T* __restrict__ row, int ncx, int x) {
    if (x & 1) {
        const int I = (x - 1) >> 1;
        return (I < ncx) ? row[I] : T(0);
    }
    const int I0 = (x >> 1) - 1, I1 = x >> 1;
    T v = 0;
    if (I0 >= 0) v += row[I0];
    if (I1 < ncx) v += row[I1];
    return T(0.5) * v;
}

// Coarse rows of a fine row along y (or z): odd y sits on coarse (y-1)/2,
// even y halfway between y/2-1 and y/2 (rows outside the coarse grid drop).
template <class T>
__device__ __forceinline__ int coarse_rows(int y, int nc, int* J, T* w) {
    if (y & 1) {
        J[0] = (y - 1) >> 1;
        w[0] = T(1);
        return 1;
    }
    const int lo = (y >> 1) - 1, hi = y >> 1;
    const bool vlo = lo >= 0, vhi = hi < nc;
    J[0] = vlo ? lo : hi;
    J[1] = hi;
    w[0] = w[1] = T(0.5);
    return (vlo && vhi) ? 2 : 1;
}

// t = omega D^-1 r + P e_c (pre-smoothed part plus the coarse correction)
// for the V consecutive fine points (x .. x+n-1) of one row: their trilinear
// values come from the 1, 2 or 4 coarse rows around the row.
template <class T>
__device__ __forceinline__ void prolong_row(const LvlDesc& F, const LvlDesc& C, const T* __restrict__ eb,
                                            const T* __restrict__ r, T* __restrict__ t, T oh2, int x, int y, int z,
                                            long long g, int n) {
    constexpr int V = Vec<T>::n;
    using VT = typename Vec<T>::type;
    int Jr[2], Kr[2];
    T wy[2], wz[2];
    const int nj = coarse_rows<T>(y, C.ny, Jr, wy);
    const int nk = coarse_rows<T>(z, C.nz, Kr, wz);
    T u[V];
#pragma unroll
    for (int k = 0; k < V; ++k) u[k] = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if (b >= nk) continue;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a >= nj) continue;
            const T* row = eb + ((long long)Kr[b] * C.ny + Jr[a]) * C.nx;
            const T w = wy[a] * wz[b];
            if (n == V) {
                // x is a multiple of V and F.nx of V, so C.nx = F.nx / 2
                const int I = x >> 1;
                const T e0 = (I >= 1) ? row[I - 1] : T(0);
                const T e1 = row[I];
                if (V == 4) {
                    const T e2 = row[I + 1];
                    u[0] += w * T(0.5) * (e0 + e1);
                    u[1] += w * e1;
                    u[2] += w * T(0.5) * (e1 + e2);
                    u[3] += w * e2;
                } else {
                    u[0] += w * T(0.5) * (e0 + e1);
                    u[1] += w * e1;
                }
            } else {
                u[0] += w * prolong_x(row, C.nx, x);
            }
        }
    }
    T rv[V], out[V];
    if (n == V) {
        const VT v = *reinterpret_cast<const VT*>(r + g);
#pragma unroll
        for (int k = 0; k < V; ++k) rv[k] = reinterpret_cast<const T*>(&v)[k];
    } else {
        rv[0] = r[g];
    }
    const bool edge = F.corr && (x + n >= F.nx || y == F.ny - 1 || z == F.nz - 1);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const T d = oh2 * (edge ? inv_diag<T>(F, x + k, y, z) : T(1.0 / 6.0));
        out[k] = d * rv[k] + u[k];
    }
    store_n<T, V>(t + g, out, n);
}

// Prolongation kernel.  float32 rows aligned to 4 go four rows at a time: the
// fine rows (y, y+1) x (z, z+1), y and z even, share the coarse rows J-1, J
// and K-1, K (J = y/2, K = z/2), so one thread loads those four coarse rows
// (three values each, zero outside the coarse grid) and all four fine rows
// at once.  Everything else goes row by row.
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
    const T oh2 = omega * T(F.h * F.h);
    constexpr bool kQuad = sizeof(T) == sizeof(float);
    if (!kQuad || F.corr || (F.nx % 4) != 0 || (P.base % 4) != 0) {
        tile_rows<T>(F, P, [&](int x, int y, int z, long long g, int n) {
            prolong_row<T>(F, C, eb, r, t, oh2, x, y, z, g, n);
        });
        return;
    }
    const long long sy = F.nx, sz = (long long)F.nx * F.ny;
    const T d = oh2 * T(1.0 / 6.0);
    const int nzp = (P.z1 - P.z0 + 1) >> 1;                 // z pairs in the tile
    for (int w = linear_tid(); w < 8 * (kTileY / 2) * nzp; w += 256) {
        const int xg = w & 7, rest = w >> 3;
        const int yp = rest % (kTileY / 2), zp = rest / (kTileY / 2);
        const int x = P.x0 + 4 * xg, y = P.y0 + 2 * yp, z = P.z0 + 2 * zp;
        if (x >= F.nx || y >= F.ny) continue;
        if (y + 1 >= F.ny || z + 1 >= P.z1) {               // ragged edge: row by row
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                    if (y + b < F.ny && z + c < P.z1)
                        prolong_row<T>(F, C, eb, r, t, oh2, x, y + b, z + c,
                                       P.base + (z + c) * sz + (y + b) * sy + x, 4);
            continue;
        }
        const int I = x >> 1, J = y >> 1, K = z >> 1;
        // coarse rows (J-1+a, K-1+c), a, c in {0, 1}: values I-1, I, I+1
        T E[2][2][3];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int JJ = J - 1 + a, KK = K - 1 + c;
                const bool ok = JJ >= 0 && JJ < C.ny && KK >= 0 && KK < C.nz;
                const T* row = eb + ((long long)(ok ? KK : 0) * C.ny + (ok ? JJ : 0)) * C.nx;
                E[c][a][0] = (ok && I >= 1) ? row[I - 1] : T(0);
                E[c][a][1] = ok ? row[I] : T(0);
                E[c][a][2] = ok ? row[I + 1] : T(0);
            }
        float4 rv[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
                rv[c][b] = *reinterpret_cast<const float4*>(r + P.base + (z + c) * sz + (y + b) * sy + x);
        // x-interpolated coarse rows
        T X[2][2][4];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                X[c][a][0] = T(0.5) * (E[c][a][0] + E[c][a][1]);
                X[c][a][1] = E[c][a][1];
                X[c][a][2] = T(0.5) * (E[c][a][1] + E[c][a][2]);
                X[c][a][3] = E[c][a][2];
            }
        // even fine index: 1/2 of coarse index - 1 and 1/2 of it; odd: the coarse index
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                T u[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const T y0 = b ? X[0][1][k] : T(0.5) * (X[0][0][k] + X[0][1][k]);   // plane K-1
                    const T y1 = b ? X[1][1][k] : T(0.5) * (X[1][0][k] + X[1][1][k]);   // plane K
                    u[k] = c ? y1 : T(0.5) * (y0 + y1);
                }
                const float4 v = rv[c][b];
                float4 o;
                o.x = d * v.x + u[0];
                o.y = d * v.y + u[1];
                o.z = d * v.z + u[2];
                o.w = d * v.w + u[3];
                *reinterpret_cast<float4*>(t + P.base + (z + c) * sz + (y + b) * sy + x) = o;
            }
    }
}

// e = t + omega D^-1 (r - A2 t) = (1 - omega) t + (omega/dd)(h^2 r + sum_nbr t);
// on level 0 also z.r per orbital -> rz, beta = rz / rz_old.
template <class T, bool kLevel0>
__global__ void __launch_bounds__(256) k_mg_postsmooth(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                       const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                       const int* __restrict__ active, const T* __restrict__ r,
                                                       const T* __restrict__ t, T* __restrict__ e, T omega,
                                                       CgState st) {
    constexpr int V = Vec<T>::n;
    using VT = typename Vec<T>::type;
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    const LvlDesc& D = L[P.b];
    if (!active[P.o] || D.coarsest) return;
    const T h2 = T(D.h * D.h);
    T rz = T(0);   // per-thread partial in the working precision; tile sums in float64
    tile_rows<T>(D, P, [&](int x, int y, int z, long long g, int n) {
        T c[V], nb[V], rv[V], out[V];
        centre_nbr<T, V>(t, D, x, y, z, g, n, c, nb);
        if (n == V) {
            const VT v = *reinterpret_cast<const VT*>(r + g);
#pragma unroll
            for (int k = 0; k < V; ++k) rv[k] = reinterpret_cast<const T*>(&v)[k];
        } else {
            rv[0] = r[g];
        }
        const bool edge = !kLevel0 && D.corr && (x + n >= D.nx || y == D.ny - 1 || z == D.nz - 1);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T w = edge ? inv_diag<T>(D, x + k, y, z) : T(1.0 / 6.0);
            out[k] = (T(1) - omega) * c[k] + omega * w * (h2 * rv[k] + nb[k]);
            if (kLevel0 && k < n) rz += rv[k] * out[k];
        }
        store_n<T, V>(e + g, out, n);
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
    const int pl = D.nx * D.ny;
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        const int z = k / pl, rem = k - z * pl, y = rem / D.nx, x = rem - y * D.nx;
        rs[k] = r[k];
        ea[k] = omega * h2 * inv_diag<T>(D, x, y, z) * rs[k];
    }
    __syncthreads();
    for (int sw = 1; sw < nsweep; ++sw) {
        for (int k = threadIdx.x; k < G; k += blockDim.x) {
            const int z = k / pl, rem = k - z * pl, y = rem / D.nx, x = rem - y * D.nx;
            eb[k] = (T(1) - omega) * ea[k] +
                    omega * inv_diag<T>(D, x, y, z) * (h2 * rs[k] + nbr6(ea, k, x, y, z, D));
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
