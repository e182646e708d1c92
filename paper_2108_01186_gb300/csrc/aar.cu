// Alternating Anderson-Richardson (AAR) for the per-orbital Poisson solves:
// the iteration the paper's code uses for its electrostatics (Sec. II.A),
// offered beside preconditioned CG as the float32 inner solver of the
// mixed-precision refinement.  Written from the method's definition
// (Suryanarayana, Pratapa, Pask, Comput. Phys. Commun. 234, 278 (2019)):
//
//   r_k = b - A x_k,  f_k = M r_k             (M: the multigrid V-cycle,
//                                               or Jacobi without it;
//                                               r_k = r_{k-1} - A dx_{k-1})
//   k+1 not a multiple of p:  x_{k+1} = x_k + omega f_k          (Richardson)
//   otherwise:                x_{k+1} = x_k + beta f_k - (X_k + beta F_k) g_k
//   with g_k = argmin |f_k - F_k g|, X_k = [dx_{k-m} .. dx_{k-1}],
//   F_k = [df_{k-m} .. df_{k-1}], dx_i = x_{i+1} - x_i, df_i = f_{i+1} - f_i.
//
// All orbitals of all systems iterate together (one launch per step);
// converged ones drop out through the active flags.  The history lives in
// ring buffers of m slots; at an Anderson step one pass forms F^T F and
// F^T f per orbital (per-tile partials, float64 across tiles) and one thread
// per orbital solves the m x m normal equations in float64.
#include "internal.cuh"

namespace flosic {

// Without the multigrid preconditioner: Jacobi, f = r / diag(A).
// w0 is the centre weight of the 12th-order second derivative (negative).
template <class T>
__global__ void __launch_bounds__(256) k_aar_jacobi(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                    const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                    const T* __restrict__ r, T* __restrict__ f, double w0,
                                                    CgState st) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const T s = (T)(D.h * D.h / (-3.0 * w0));
    tile_elementwise<T>(D, P, [&](long long g, int n) {
        for (int k = 0; k < n; ++k) f[g + k] = s * r[g + k];
    });
}

// Richardson step k: push df_{k-1} = f - f_prev (k >= 1), f_prev = f,
// dx_k = omega f into slot k mod m, x += dx_k.
template <class T>
__global__ void __launch_bounds__(256) k_aar_richardson(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                        const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                        const T* __restrict__ f, T* __restrict__ fprev,
                                                        T* __restrict__ X, T* __restrict__ F, long long stride,
                                                        T* __restrict__ x, int k, int m, T omega, CgState st) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    T* Xk = X + (long long)(k % m) * stride;
    T* Fp = F + (long long)((k + m - 1) % m) * stride;
    tile_elementwise<T>(D, P, [&](long long g, int n) {
        for (int q = 0; q < n; ++q) {
            const long long e = g + q;
            const T fv = f[e];
            if (k >= 1) Fp[e] = fv - fprev[e];
            fprev[e] = fv;
            const T dx = omega * fv;
            Xk[e] = dx;
            x[e] += dx;
        }
    });
}

constexpr int kAarMaxM = 8;
constexpr int kAarDots = kAarMaxM * (kAarMaxM + 1) / 2 + kAarMaxM;   // F^T F (upper) and F^T f

// Anderson step k, part 1: push df_{k-1}, f_prev = f, and per-tile partial
// sums of F_i . F_j (i <= j) and F_i . f over the mk = min(k, m) valid slots
// (slot of pair i: i mod m, pairs k-mk .. k-1).
template <class T>
__global__ void __launch_bounds__(256) k_aar_dots(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                  const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                  const T* __restrict__ f, T* __restrict__ fprev,
                                                  T* __restrict__ F, long long stride, int k, int m,
                                                  double* __restrict__ part, CgState st) {
    __shared__ double scratch[32];
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const int mk = k < m ? k : m;
    T* Fp = F + (long long)((k + m - 1) % m) * stride;
    float acc[kAarDots];
#pragma unroll
    for (int q = 0; q < kAarDots; ++q) acc[q] = 0.f;
    tile_elementwise<T>(D, P, [&](long long g, int n) {
        for (int q = 0; q < n; ++q) {
            const long long e = g + q;
            const T fv = f[e];
            Fp[e] = fv - fprev[e];
            fprev[e] = fv;
            float Fv[kAarMaxM];
#pragma unroll
            for (int i = 0; i < kAarMaxM; ++i)
                Fv[i] = (i < mk) ? (float)F[(long long)((k - mk + i) % m) * stride + e] : 0.f;
            int t = 0;
#pragma unroll
            for (int i = 0; i < kAarMaxM; ++i) {
#pragma unroll
                for (int j = i; j < kAarMaxM; ++j) acc[t++] += Fv[i] * Fv[j];
            }
#pragma unroll
            for (int i = 0; i < kAarMaxM; ++i) acc[t++] += Fv[i] * (float)fv;
        }
    });
#pragma unroll
    for (int q = 0; q < kAarDots; ++q) {
        const double s = block_sum(acc[q], scratch);
        if (linear_tid() == 0) part[(long long)blockIdx.x * kAarDots + q] = s;
    }
}

// Anderson step k, part 2 (one thread per active orbital): sum the tile
// partials in tile order, solve (F^T F) g = F^T f by Gaussian elimination
// with partial pivoting in float64 (a relative 1e-12 ridge keeps it
// defined when the history is nearly dependent).
__global__ void k_aar_gamma(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L, const int* __restrict__ orb_blk,
                            int norb, const double* __restrict__ part, int k, int m, double* __restrict__ gamma,
                            CgState st) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= norb || !st.active[o]) return;
    const int b = orb_blk[o];
    const LvlDesc& D = L[b];
    const long long first = D.tile0 + (long long)(o - blk[b].orb0) * D.ntile;
    const int mk = k < m ? k : m;
    double S[kAarDots];
    for (int q = 0; q < kAarDots; ++q) S[q] = 0.0;
    for (int t = 0; t < D.ntile; ++t)
        for (int q = 0; q < kAarDots; ++q) S[q] += part[(first + t) * kAarDots + q];
    double A[kAarMaxM][kAarMaxM + 1];
    int t = 0;
    for (int i = 0; i < kAarMaxM; ++i)
        for (int j = i; j < kAarMaxM; ++j) {
            A[i][j] = A[j][i] = S[t];
            ++t;
        }
    double tr = 0.0;
    for (int i = 0; i < mk; ++i) tr += A[i][i];
    for (int i = 0; i < kAarMaxM; ++i) {
        A[i][kAarMaxM] = S[t++];
        if (i < mk) A[i][i] += 1e-12 * tr + 1e-300;
    }
    for (int c = 0; c < mk; ++c) {   // elimination with partial pivoting
        int piv = c;
        for (int i = c + 1; i < mk; ++i)
            if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
        if (piv != c)
            for (int j = 0; j <= kAarMaxM; ++j) {
                const double tmp = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = tmp;
            }
        for (int i = c + 1; i < mk; ++i) {
            const double fct = A[i][c] / A[c][c];
            for (int j = c; j < mk; ++j) A[i][j] -= fct * A[c][j];
            A[i][kAarMaxM] -= fct * A[c][kAarMaxM];
        }
    }
    double g[kAarMaxM];
    for (int i = kAarMaxM - 1; i >= 0; --i) {
        if (i >= mk) { g[i] = 0.0; continue; }
        double v = A[i][kAarMaxM];
        for (int j = i + 1; j < mk; ++j) v -= A[i][j] * g[j];
        g[i] = v / A[i][i];
    }
    for (int i = 0; i < kAarMaxM; ++i) gamma[(long long)o * kAarMaxM + i] = isfinite(g[i]) ? g[i] : 0.0;
}

// Anderson step k, part 3: dx_k = beta f - sum_i g_i (X_i + beta F_i),
// x += dx_k, dx_k into slot k mod m (read before it is overwritten).
template <class T>
__global__ void __launch_bounds__(256) k_aar_anderson(const BlkDesc* __restrict__ blk, const LvlDesc* __restrict__ L,
                                                      const int4* __restrict__ tiles, const int* __restrict__ orb_blk,
                                                      const T* __restrict__ f, T* __restrict__ X,
                                                      const T* __restrict__ F, long long stride, T* __restrict__ x,
                                                      int k, int m, T beta, const double* __restrict__ gamma,
                                                      CgState st) {
    const TilePos P = tile_pos(blk, L, tiles, orb_blk, blockIdx.x);
    if (!st.active[P.o]) return;
    const LvlDesc& D = L[P.b];
    const int mk = k < m ? k : m;
    T gm[kAarMaxM];
#pragma unroll
    for (int i = 0; i < kAarMaxM; ++i) gm[i] = (T)gamma[(long long)P.o * kAarMaxM + i];
    T* Xk = X + (long long)(k % m) * stride;
    tile_elementwise<T>(D, P, [&](long long g, int n) {
        for (int q = 0; q < n; ++q) {
            const long long e = g + q;
            const T fv = f[e];
            T dx = beta * fv;
#pragma unroll
            for (int i = 0; i < kAarMaxM; ++i) {
                if (i >= mk) break;
                const long long so = (long long)((k - mk + i) % m) * stride + e;
                dx -= gm[i] * (X[so] + beta * F[so]);
            }
            Xk[e] = dx;
            x[e] += dx;
        }
    });
}

template <class T>
void launch_aar_step(flosic_ctx* c, T* x, T* r, T* f, int k, bool anderson, cudaStream_t s,
                     void (*precondition)(flosic_ctx*, T*, T*, cudaStream_t)) {
    const Multigrid& M = c->mg;
    const unsigned nt = (unsigned)M.ntiles[0];
    const dim3 tb(kTileX, kTileY / 2);
    CgState& st = c->ws.cg;
    Workspace& w = c->ws;
    const int m = c->opt.aar_m;
    T* X = (T*)w.aar_X;
    T* F = (T*)w.aar_F;
    T* fprev = (T*)w.aar_fprev;
    const long long stride = c->orb_elems;
    // r_k = r_{k-1} - A dx_{k-1} (at k = 0, x = 0 and r is the right-hand side)
    if (k > 0) launch_residual12_aar<T>(c, X + (long long)((k - 1) % m) * stride, r, s);
    if (M.enabled) {
        precondition(c, r, f, s);
    } else {
        double w[kHalf + 1];
        stencil_weights(w);
        k_aar_jacobi<T><<<nt, tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, r, f, w[0], st);
        note_launch(c);
    }
    if (!anderson) {
        k_aar_richardson<T><<<nt, tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, f, fprev, X, F, stride,
                                              x, k, m, (T)c->opt.aar_omega, st); note_launch(c);
        return;
    }
    k_aar_dots<T><<<nt, tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, f, fprev, F, stride, k, m,
                                    w.aar_part, st); note_launch(c);
    k_aar_gamma<<<(c->norb + 127) / 128, 128, 0, s>>>(c->d_blk, M.d_lvl[0], c->d_orb_blk, c->norb, w.aar_part, k, m,
                                                      w.aar_gamma, st); note_launch(c);
    k_aar_anderson<T><<<nt, tb, 0, s>>>(c->d_blk, M.d_lvl[0], M.d_tiles[0], c->d_orb_blk, f, X, F, stride, x, k, m,
                                        (T)c->opt.aar_beta, w.aar_gamma, st); note_launch(c);
}

template void launch_aar_step<float>(flosic_ctx*, float*, float*, float*, int, bool, cudaStream_t,
                                     void (*)(flosic_ctx*, float*, float*, cudaStream_t));

long long aar_part_elems(long long ntiles0) { return ntiles0 * kAarDots; }
int aar_max_m() { return kAarMaxM; }

}  // namespace flosic
