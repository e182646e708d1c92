// Kronecker-product solver of the per-orbital Poisson problems.
//
// Sec. II.A writes the finite-difference Laplacian in Kronecker-product
// form: with zero ghost values (the Dirichlet data sit in the right-hand
// side) or periodic wrap-around along each direction,
//   A = -Delta_h = T_x (+) T_y (+) T_z,   T_d = -(1/h^2) D2_d,
// where D2_d is the 1-D 12th-order second difference of direction d.  Each
// T_d is symmetric; with T_d = Q_d L_d Q_d^T (computed once per context in
// float64 on the host by cyclic Jacobi) the inverse is
//   A^{-1} = (Q_x x Q_y x Q_z) diag(1 / (l_i + l_j + l_k)) (Q_x x Q_y x Q_z)^T.
// In a periodic cell the constant mode (l = 0 in every direction) is the
// null space of A; its coefficient is set to zero (zero-mean potential).
//
// On the device the inverse is six dense 1-D transforms per orbital (three
// forward with Q_d, three back with Q_d^T, the diagonal scaling folded into
// the forward z pass), each a float32 matrix product over one direction's
// lines.  T_d commutes with the reflection j -> n-1-j (it is persymmetric),
// so its eigenvectors are even or odd and each transform is two half-size
// products on the even and odd parts of the line (half the flops).  A
// persistent CTA keeps the two half-size matrices of its block in shared
// memory and streams 64-line tiles through them: the next tile is fetched
// into registers (coalesced) while the current one is multiplied (8 x 4
// outputs per thread, about 2n threads).  The
// mixed refinement calls it as its float32 inner solve; the float-float
// residual around it carries the accuracy to the requested tolerance.
#include <cmath>
#include <cstring>
#include <array>
#include <map>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace flosic {
namespace {

constexpr int kKronCols = 64;                  // lines per tile
constexpr int kKronLd = kKronCols + 4;         // shared row stride of a tile (16-byte rows)
constexpr int kKronMaxN = 256;                 // 2 (128^2) + 256 * 68 floats fit in 227 KB
constexpr int kKronPre = kKronCols / 2;        // tile values per thread (2 n8 threads, n8 x 64 values)

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row
// major, destroyed): on return A's diagonal holds the eigenvalues and the
// columns of V the eigenvectors.  Each rotation annihilates a_pq
// (tau = (a_qq - a_pp) / 2 a_pq, t = sgn(tau) / (|tau| + sqrt(1 + tau^2))).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double a : A) fro += a * a;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-32 * fro) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < n; ++k) {   // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
}

// T_d of one direction: n points, spacing h, periodic or zero outside.
std::vector<double> axis_operator(int n, double h, bool periodic) {
    double w[kHalf + 1];
    stencil_weights(w);
    std::vector<double> T((size_t)n * n, 0.0);
    const double ih2 = 1.0 / (h * h);
    for (int j = 0; j < n; ++j)
        for (int m = -kHalf; m <= kHalf; ++m) {
            int q = j + m;
            if (q < 0 || q >= n) {
                if (!periodic) continue;
                q = ((q % n) + n) % n;
            }
            T[(size_t)j * n + q] -= w[m < 0 ? -m : m] * ih2;
        }
    return T;
}

__host__ __device__ inline int round8(int n) { return (n + 7) & ~7; }

// device array owned by the context (freed with it)
template <class T>
cudaError_t ctx_alloc(flosic_ctx* c, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (n > 0 ? n : 1));
    if (e == cudaSuccess) {
        c->allocations.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}

struct KronArgs {
    const BlkDesc* blk;
    int nblk;
    const long long* item0;   // [nblk + 1] first tile item of each block in this pass
    const float* mat;         // transform matrices (Q_d and Q_d^T per distinct operator)
    const float* lam;         // eigenvalues per distinct operator
    const float* in;
    float* out;
    const int* active;
    double* flops;            // algorithmic flop counter (profiling)
    int axis;                 // 0 x, 1 y, 2 z
    int inverse;              // 0: coefficients = Q^T v; 1: values = Q c
    int scale;                // forward z pass: divide by l_i + l_j + l_k
};

// Item -> (block, orbital, tile): tiles of kKronCols lines along the pass direction.
//   x: lines are grid rows (y, z), tile q = rows q*C .. q*C+C-1 (a contiguous run of C*nx values)
//   y: lines are (x, z) columns at fixed z, tile q = (z, x-group)
//   z: lines are xy points, tile q = xy points q*C .. q*C+C-1
__device__ __forceinline__ int pass_groups(const BlkDesc& B, int axis) {
    if (axis == 0) return (B.ny * B.nz + kKronCols - 1) / kKronCols;
    if (axis == 1) return B.nz * ((B.nx + kKronCols - 1) / kKronCols);
    return (B.nx * B.ny + kKronCols - 1) / kKronCols;
}

// Addressing of one tile: element (j, c) = position j along line c lies at
// cbase + c * cstride + j * jstride; ncol lines are valid.
struct Tile {
    long long cbase, cstride, jstride;
    int ncol, q;
};

__device__ __forceinline__ Tile tile_of(const BlkDesc& B, int axis, int i_orb, int q) {
    Tile t;
    const long long base = B.off + (long long)i_orb * B.G;
    const long long sxy = (long long)B.nx * B.ny;
    t.q = q;
    if (axis == 0) {
        t.cbase = base + (long long)q * kKronCols * B.nx;
        t.cstride = B.nx;
        t.jstride = 1;
        t.ncol = min(kKronCols, B.ny * B.nz - q * kKronCols);
    } else if (axis == 1) {
        const int gx = (B.nx + kKronCols - 1) / kKronCols;
        const int zi = q / gx, xg = q - zi * gx;
        t.cbase = base + (long long)zi * sxy + (long long)xg * kKronCols;
        t.cstride = 1;
        t.jstride = B.nx;
        t.ncol = min(kKronCols, B.nx - xg * kKronCols);
    } else {
        t.cbase = base + (long long)q * kKronCols;
        t.cstride = 1;
        t.jstride = sxy;
        t.ncol = (int)min((long long)kKronCols, sxy - (long long)q * kKronCols);
    }
    return t;
}

// The thread's kKronPre elements of a tile of R rows (R a multiple of 32,
// the CTA's 2 Rmax threads): element k is (j0 + k jstep, c0 + k cstep),
// coalesced along the contiguous direction.  x lines (j contiguous): lanes
// take consecutive j, warp g covers line g / (R/32) + 2k, rows
// 32 (g mod R/32) ..; y, z lines (c contiguous): lanes take consecutive c.
struct TileMap {
    int j0, jstep, c0, cstep;
    bool on;
};

__device__ __forceinline__ TileMap tile_map(int axis, int tid, int nthr, int R) {
    TileMap m;
    if (axis == 0) {
        const int rb = R >> 5, g0 = tid >> 5;
        m.on = g0 < 2 * rb;
        m.c0 = m.on ? g0 / rb : 0;
        m.cstep = 2;
        m.j0 = (tid & 31) + 32 * (m.on ? g0 % rb : 0);
        m.jstep = 0;
    } else {
        m.on = true;
        m.c0 = tid & (kKronCols - 1);
        m.cstep = 0;
        m.j0 = tid >> 6;
        m.jstep = nthr >> 6;
    }
    return m;
}

__device__ __forceinline__ void tile_fetch(const float* __restrict__ in, const Tile& t, const TileMap& mp, int n,
                                           float* pre) {
#pragma unroll
    for (int k = 0; k < kKronPre; ++k) {
        const int j = mp.j0 + k * mp.jstep, c = mp.c0 + k * mp.cstep;
        pre[k] = (mp.on && c < t.ncol && j < n)
                     ? __ldcs(in + t.cbase + (long long)c * t.cstride + (long long)j * t.jstride)
                     : 0.f;
    }
}

// rows of the two halves in shared memory: the even part padded to 8, the
// whole tile to 32 (the odd part takes the rest)
__host__ __device__ __forceinline__ int kron_rows(int n) { return ((round8((n + 1) / 2) + round8(n / 2)) + 31) & ~31; }

// next item at or after it whose orbital is active (it1 if none)
__device__ __forceinline__ long long next_active(const KronArgs& a, long long it, long long it1, int& b) {
    for (; it < it1; ++it) {
        while (b + 1 < a.nblk && it >= a.item0[b + 1]) ++b;
        const BlkDesc& B = a.blk[b];
        const int groups = pass_groups(B, a.axis);
        const int i_orb = (int)((it - a.item0[b]) / groups);
        if (a.active[B.orb0 + i_orb]) return it;
    }
    return it1;
}

__device__ __forceinline__ int axis_n(const BlkDesc& B, int axis) {
    return axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
}

// One pass over every tile of the CTA's contiguous item range.
//
// Even/odd split: T_d commutes with the reflection j -> n-1-j, so its
// eigenvectors are symmetric or antisymmetric and the transform splits into
// two half-size products.  Forward: s_k = v_k + v_{n-1-k} (k < ns, the middle
// point doubled), a_k = v_k - v_{n-1-k} (k < na); coefficients
// c_s = Fs^T s, c_a = Fa^T a, stored as [c_s | c_a] along the line.
// Inverse: S = Is c_s, A = Ia c_a; v_k = S_k + A_k, v_{n-1-k} = S_k - A_k,
// v_mid = S_mid.  (Fs, Fa, Is, Ia carry the 1/sqrt 2 of the even/odd basis.)
//
// Thread (ib, cq) owns output rows 8 ib .. 8 ib + 7 (the symmetric half in
// rows [0, ns8), the antisymmetric half in [ns8, ns8 + na8)) and columns
// 4 cq .. 4 cq + 3; the next tile is fetched into registers while the
// current one is multiplied.
__global__ void __launch_bounds__(2 * kKronMaxN) k_kron_pass(KronArgs a, long long total) {
    extern __shared__ __align__(16) float kron_smem[];
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const long long per_cta = (total + gridDim.x - 1) / gridDim.x;
    const long long it0 = (long long)blockIdx.x * per_cta;
    const long long it1 = it0 + per_cta < total ? it0 + per_cta : total;
    if (it0 >= it1) return;
    int bs = 0;   // block of the item being fetched
    long long item = next_active(a, it0, it1, bs);
    if (item >= it1) return;
    float pre[kKronPre];
    {
        const BlkDesc& B = a.blk[bs];
        const int nn = axis_n(B, a.axis);
        const int groups = pass_groups(B, a.axis);
        const long long r = item - a.item0[bs];
        tile_fetch(a.in, tile_of(B, a.axis, (int)(r / groups), (int)(r % groups)),
                   tile_map(a.axis, tid, nthr, kron_rows(nn)), nn, pre);
    }
    float* Ps = kron_smem;
    float* Pa = nullptr;
    float* S = nullptr;
    int cur = -1, n = 0, ns = 0, na = 0, ns8 = 0, na8 = 0, R = 0;
    TileMap mp{};
    const int cq = tid % (kKronCols / 4), ib = tid / (kKronCols / 4);
    const int r0 = ib * 8, c0 = cq * 4;
    while (item < it1) {
        const int b = bs;
        const BlkDesc& B = a.blk[b];
        const int groups = pass_groups(B, a.axis);
        const long long rr = item - a.item0[b];
        const Tile t = tile_of(B, a.axis, (int)(rr / groups), (int)(rr % groups));
        __syncthreads();   // the previous tile is finished with S (and the matrices)
        if (b != cur) {
            n = axis_n(B, a.axis);
            ns = (n + 1) / 2;
            na = n / 2;
            ns8 = round8(ns);
            R = kron_rows(n);
            na8 = R - ns8;
            mp = tile_map(a.axis, tid, nthr, R);
            Pa = Ps + ns8 * ns8;
            S = Pa + na8 * na8;
            const float* src = a.mat + B.kq[a.axis] + (a.inverse ? (long long)ns * ns + (long long)na * na : 0);
            for (int e = tid; e < ns8 * ns8; e += nthr) {
                const int jj = e / ns8, ii = e - jj * ns8;
                Ps[e] = (jj < ns && ii < ns) ? src[jj * ns + ii] : 0.f;
            }
            const float* srca = src + (long long)ns * ns;
            for (int e = tid; e < na8 * na8; e += nthr) {
                const int jj = e / na8, ii = e - jj * na8;
                Pa[e] = (jj < na && ii < na) ? srca[jj * na + ii] : 0.f;
            }
            cur = b;
        }
#pragma unroll
        for (int k = 0; k < kKronPre; ++k) {
            const int j = mp.j0 + k * mp.jstep, c = mp.c0 + k * mp.cstep;
            if (mp.on && j < R) S[j * kKronLd + c] = pre[k];   // (a smaller block leaves extra slots)
        }
        __syncthreads();
        if (!a.inverse) {   // fold each line into its even and odd parts
            for (int e = tid; e < na * kKronCols; e += nthr) {
                const int k = e >> 6, c = e & (kKronCols - 1);
                const float u = S[k * kKronLd + c], w = S[(n - 1 - k) * kKronLd + c];
                S[k * kKronLd + c] = u + w;
                S[(n - 1 - k) * kKronLd + c] = u - w;
            }
            if (n & 1)
                for (int c = tid; c < kKronCols; c += nthr) S[na * kKronLd + c] *= 2.f;
            __syncthreads();
        }
        // fetch the next active tile while this one is multiplied
        long long nxt = next_active(a, item + 1, it1, bs);
        if (nxt < it1) {
            const BlkDesc& Bn = a.blk[bs];
            const int nn = axis_n(Bn, a.axis);
            const int gn = pass_groups(Bn, a.axis);
            const long long rn = nxt - a.item0[bs];
            tile_fetch(a.in, tile_of(Bn, a.axis, (int)(rn / gn), (int)(rn % gn)),
                       tile_map(a.axis, tid, nthr, kron_rows(nn)), nn, pre);
        }
        const bool sym = r0 < ns8;
        const int m0 = sym ? r0 : r0 - ns8;             // first mode (or position) of this thread
        const int K = sym ? ns : na;
        const int pld = sym ? ns8 : na8;
        const float* P = sym ? Ps : Pa;
        // input row of the k-th term: forward s_k = row k, a_k = row n-1-k;
        // inverse c_s[k] = row k, c_a[k] = row ns + k
        const int rbase = sym ? 0 : (a.inverse ? ns : n - 1);
        const int rstep = (!sym && !a.inverse) ? -1 : 1;
        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        const bool comp = r0 < R;
        if (comp) {
            const float* srow = S + rbase * kKronLd + c0;
            const int sstep = rstep * kKronLd;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                const float4 p0 = *reinterpret_cast<const float4*>(P + k * pld + m0);
                const float4 p1 = *reinterpret_cast<const float4*>(P + k * pld + m0 + 4);
                const float4 sv = *reinterpret_cast<const float4*>(srow + k * sstep);
                const float pr[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                const float sc[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(pr[u], sc[v], acc[u][v]);
            }
        }
        const int nmode = sym ? ns : na;                 // valid outputs of this half
        const int pos0 = sym ? 0 : ns;                   // their place along the line
        if (!a.inverse) {
            if (comp) {
                if (a.scale) {   // forward z pass: column c is the xy mode (t % nx, t / nx)
                    const long long sxy = (long long)B.nx * B.ny;
                    const float* lx = a.lam + B.kl[0];
                    const float* ly = a.lam + B.kl[1];
                    const float* lz = a.lam + B.kl[2];
                    float lxy[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const long long tt = (long long)t.q * kKronCols + c0 + v;
                        const int ti = (int)(tt < sxy ? tt : 0);
                        const int yi = ti / B.nx, xi = ti - yi * B.nx;
                        lxy[v] = lx[xi] + ly[yi];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int m = m0 + u;
                        const float l3 = lz[m < nmode ? pos0 + m : 0];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {   // (fast division: 2 ulp, far below the solve's accuracy)
                            const float sm = lxy[v] + l3;
                            acc[u][v] = (sm > 0.f) ? __fdividef(acc[u][v], sm) : 0.f;
                        }
                    }
                }
                if (a.axis == 0) {   // per line c: 8 consecutive positions (two 16-byte stores when aligned)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int c = c0 + v;
                        if (c >= t.ncol) break;
                        const long long off = t.cbase + (long long)c * t.cstride + pos0 + m0;
                        if (m0 + 7 < nmode && (off & 3) == 0) {
                            __stcs(reinterpret_cast<float4*>(a.out + off),
                                   make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]));
                            __stcs(reinterpret_cast<float4*>(a.out + off + 4),
                                   make_float4(acc[4][v], acc[5][v], acc[6][v], acc[7][v]));
                        } else {
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (m0 + u < nmode) __stcs(a.out + off + u, acc[u][v]);
                        }
                    }
                } else {             // per position: 4 consecutive lines (one 16-byte store when aligned)
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int m = m0 + u;
                        if (m >= nmode) break;
                        const long long off = t.cbase + (long long)(pos0 + m) * t.jstride + c0;
                        if (c0 + 3 < t.ncol && (off & 3) == 0) {
                            __stcs(reinterpret_cast<float4*>(a.out + off),
                                   make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]));
                        } else {
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                if (c0 + v < t.ncol) __stcs(a.out + off + v, acc[u][v]);
                        }
                    }
                }
            }
        } else {
            __syncthreads();   // every product has read its coefficients
            if (comp) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int m = m0 + u;
                    if (m < nmode)
                        *reinterpret_cast<float4*>(S + (pos0 + m) * kKronLd + c0) =
                            make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                }
            }
            __syncthreads();
            // v_k = S_k + A_k, v_{n-1-k} = S_k - A_k, v_mid = S_mid (rows: S at k, A at ns + k)
#pragma unroll 4
            for (int k = 0; k < kKronPre; ++k) {
                const int j = mp.j0 + k * mp.jstep, c = mp.c0 + k * mp.cstep;
                if (!mp.on || j >= n || c >= t.ncol) continue;
                float v;
                if (j < na) v = S[j * kKronLd + c] + S[(ns + j) * kKronLd + c];
                else if (j >= ns) v = S[(n - 1 - j) * kKronLd + c] - S[(ns + n - 1 - j) * kKronLd + c];
                else v = S[j * kKronLd + c];
                __stcs(a.out + t.cbase + (long long)c * t.cstride + (long long)j * t.jstride, v);
            }
        }
        if (a.flops && tid == 0) atomicAdd(a.flops, 2.0 * ((double)ns * ns + (double)na * na) * t.ncol);
        item = nxt;
    }
}

// Orbitals solved this round: leave the inner solve, count one application.
__global__ void k_kron_done(int norb, CgState st) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < norb && st.active[o]) {
        st.active[o] = 0;
        ++st.iters[o];
    }
}

}  // namespace

int kron_max_n() { return kKronMaxN; }

// Tensor-core transforms: the split bf16 matrices, per pass the tile table
// and the input tensor maps of every tensor-core block (the pass reads the
// workspace arrays r32, p32, q32 in the order of launch_kron_solve), the
// kernel's shared-memory limit and one CTA per SM.
cudaError_t setup_kron_tc(flosic_ctx* c, const std::vector<uint16_t>& tcmat, int sms) {
    KronPlan& K = c->kron;
    cudaError_t e = ctx_alloc(c, &K.tc_mat, tcmat.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(K.tc_mat, tcmat.data(), sizeof(uint16_t) * tcmat.size(), cudaMemcpyHostToDevice);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (e == cudaSuccess &&
        (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
         q != cudaDriverEntryPointSuccess || !fn))
        e = cudaErrorNotSupported;
    // the buffers of launch_kron_solve's passes as the refinement calls it
    // (r = r32, d = d32, scratch p32 and q32)
    const float* in_buf[6] = {c->ws.r32, c->ws.p32, c->ws.q32, c->ws.p32, c->ws.q32, c->ws.p32};
    float* out_buf[6] = {c->ws.p32, c->ws.q32, c->ws.p32, c->ws.q32, c->ws.p32, c->ws.d32};
    std::vector<CUtensorMap> maps(12 * (size_t)c->nblk);   // inputs, then outputs
    std::vector<long long> items(6 * (size_t)(c->nblk + 1));
    std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    for (int st = 0; st < 6 && e == cudaSuccess; ++st) {
        long long acc = 0;
        for (int b = 0; b < c->nblk; ++b) {
            const BlkDesc& B = c->blk[b];
            items[(size_t)st * (c->nblk + 1) + b] = acc;
            if (!B.tc) continue;
            acc += kron_tc_tiles(B, st % 3);
            if (!kron_tc_map(fn, &maps[(size_t)st * c->nblk + b], B, st % 3, in_buf[st]) ||
                !kron_tc_map_out(fn, &maps[(size_t)(6 + st) * c->nblk + b], B, st % 3, out_buf[st]))
                e = cudaErrorInvalidValue;
        }
        items[(size_t)st * (c->nblk + 1) + c->nblk] = acc;
        K.tc_total[st] = acc;
        K.tc_grid[st] = (int)(acc < sms ? (acc > 0 ? acc : 1) : sms);
    }
    void* dm = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(CUtensorMap) * maps.size());
    if (e == cudaSuccess) {
        c->allocations.push_back(dm);
        K.tc_maps = dm;
        K.tc_omaps = reinterpret_cast<CUtensorMap*>(dm) + 6 * (size_t)c->nblk;
        e = cudaMemcpy(dm, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = ctx_alloc(c, &K.tc_items, items.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(K.tc_items, items.data(), sizeof(long long) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ensure_dyn_smem(kron_tc_symbol(), kron_tc_smem());
    return e;
}

// Host set-up: for every distinct 1-D operator (n, h, periodic) the
// eigen-decompositions of its even and odd blocks, the forward and inverse
// half-size matrices in float32, the eigenvalues (the periodic constant mode
// set to exactly zero), per-block offsets and the tile counts of the passes.
cudaError_t setup_kron(flosic_ctx* c) {
    std::map<std::tuple<int, double, int>, std::pair<long long, long long>> seen;
    std::map<std::tuple<int, double, int>, std::pair<std::vector<double>, std::vector<double>>> vecs;
    std::map<std::tuple<int, double, int>, long long> tc_seen;
    std::vector<float> mat, lam;
    std::vector<uint16_t> tcmat;
    KronPlan& K = c->kron;
    K.n_simt = K.n_tc = 0;
    for (BlkDesc& B : c->blk) {
        const int bi = (int)(&B - c->blk.data());
        const bool forced_off = !K.tc_force.empty() && K.tc_force[bi] == 0;
        B.tc = (c->opt.kron_tensor_cores && kron_tc_eligible(B) && !forced_off) ? 1 : 0;
        ++(B.tc ? K.n_tc : K.n_simt);
        const int nd[3] = {B.nx, B.ny, B.nz};
        for (int d = 0; d < 3; ++d) {
            const int n = nd[d];
            const int periodic = (B.per >> d) & 1;
            const auto key = std::make_tuple(n, B.h, periodic);
            auto it = seen.find(key);
            if (it == seen.end()) {
                const std::vector<double> T = axis_operator(n, B.h, periodic != 0);
                const int ns = (n + 1) / 2, na = n / 2;
                // even/odd basis: e_k = (d_k + d_{n-1-k}) / sqrt 2 (k < na), e_mid = d_mid;
                // o_k = (d_k - d_{n-1-k}) / sqrt 2; T is persymmetric, so U^T T U is block diagonal
                const double r2 = std::sqrt(0.5);
                std::vector<double> Ts((size_t)ns * ns), Ta((size_t)na * na), Vs, Va;
                // support of e_k / o_k: points k and n-1-k with weights (w, w) / (w, -w)
                auto proj = [&](int k, int l, bool odd) {
                    const int pk[2] = {k, n - 1 - k}, pl[2] = {l, n - 1 - l};
                    const double wk = (!odd && k == n - 1 - k) ? 1.0 : r2;
                    const double wl = (!odd && l == n - 1 - l) ? 1.0 : r2;
                    const int mk = (pk[0] == pk[1]) ? 1 : 2, ml = (pl[0] == pl[1]) ? 1 : 2;
                    double v = 0.0;
                    for (int a = 0; a < mk; ++a)
                        for (int b = 0; b < ml; ++b) {
                            const double sa = (odd && a == 1) ? -1.0 : 1.0, sb = (odd && b == 1) ? -1.0 : 1.0;
                            v += sa * wk * T[(size_t)pk[a] * n + pl[b]] * sb * wl;
                        }
                    return v;
                };
                for (int k = 0; k < ns; ++k)
                    for (int l = 0; l < ns; ++l) Ts[(size_t)k * ns + l] = proj(k, l, false);
                for (int k = 0; k < na; ++k)
                    for (int l = 0; l < na; ++l) Ta[(size_t)k * na + l] = proj(k, l, true);
                jacobi_eigen(ns, Ts, Vs);
                if (na > 0) jacobi_eigen(na, Ta, Va);
                // forward Fs[k][m] = Vs[k][m] fs_k (fs = 1/sqrt 2, 1/2 at the middle: s_mid = 2 v_mid),
                // Fa = Va / sqrt 2; inverse in the kernel's transposed form Is[m][k] = Vs[k][m] gs_k
                // (gs = 1/sqrt 2, 1 at the middle), Ia[m][k] = Va[k][m] / sqrt 2
                const long long qo = (long long)mat.size(), lo = (long long)lam.size();
                mat.resize(mat.size() + 2 * ((size_t)ns * ns + (size_t)na * na));
                float* Fs = mat.data() + qo;
                float* Fa = Fs + (size_t)ns * ns;
                float* Is = Fa + (size_t)na * na;
                float* Ia = Is + (size_t)ns * ns;
                for (int k = 0; k < ns; ++k)
                    for (int m = 0; m < ns; ++m) {
                        const double v = Vs[(size_t)k * ns + m];
                        Fs[(size_t)k * ns + m] = (float)(v * (k < na ? r2 : 0.5));
                        Is[(size_t)m * ns + k] = (float)(v * (k < na ? r2 : 1.0));
                    }
                for (int k = 0; k < na; ++k)
                    for (int m = 0; m < na; ++m) {
                        const double v = Va[(size_t)k * na + m] * r2;
                        Fa[(size_t)k * na + m] = (float)v;
                        Ia[(size_t)m * na + k] = (float)v;
                    }
                int kmin = 0;   // the periodic constant mode is symmetric
                for (int k = 0; k < ns; ++k) {
                    lam.push_back((float)Ts[(size_t)k * ns + k]);
                    if (std::fabs(Ts[(size_t)k * ns + k]) < std::fabs(Ts[(size_t)kmin * ns + kmin])) kmin = k;
                }
                for (int k = 0; k < na; ++k) lam.push_back((float)Ta[(size_t)k * na + k]);
                if (periodic) lam[lo + kmin] = 0.f;
                it = seen.emplace(key, std::make_pair(qo, lo)).first;
                vecs.emplace(key, std::make_pair(std::move(Vs), std::move(Va)));
            }
            B.kq[d] = it->second.first;
            B.kl[d] = it->second.second;
            B.kt[d] = 0;
            if (B.tc) {
                auto jt = tc_seen.find(key);
                if (jt == tc_seen.end()) {
                    const auto& V = vecs.at(key);
                    const long long to = (long long)tcmat.size();
                    kron_tc_pack(n, V.first, V.second, tcmat);
                    jt = tc_seen.emplace(key, to).first;
                }
                B.kt[d] = jt->second;
            }
        }
    }
    cudaError_t e = ctx_alloc(c, &K.mat, mat.size());
    if (e == cudaSuccess) e = ctx_alloc(c, &K.lam, lam.size());
    if (e == cudaSuccess) e = cudaMemcpy(K.mat, mat.data(), sizeof(float) * mat.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(K.lam, lam.data(), sizeof(float) * lam.size(), cudaMemcpyHostToDevice);
    // tile items per pass and block
    std::vector<long long> items(3 * (size_t)(c->nblk + 1));
    for (int d = 0; d < 3; ++d) {
        long long acc = 0;
        int nmax = 8;
        size_t smem = 0;   // the largest block's need (not monotone in n: the odd half fills the rows up to 32)
        for (int b = 0; b < c->nblk; ++b) {
            const BlkDesc& B = c->blk[b];
            items[(size_t)d * (c->nblk + 1) + b] = acc;
            long long g;
            if (d == 0) g = (B.ny * (long long)B.nz + kKronCols - 1) / kKronCols;
            else if (d == 1) g = (long long)B.nz * ((B.nx + kKronCols - 1) / kKronCols);
            else g = ((long long)B.nx * B.ny + kKronCols - 1) / kKronCols;
            if (!B.tc) acc += g * B.N;   // tensor-core blocks take no tiles of this kernel
            const int n = d == 0 ? B.nx : (d == 1 ? B.ny : B.nz);
            nmax = n > nmax ? n : nmax;
            const int Rb = kron_rows(n), s8 = round8((n + 1) / 2), a8 = Rb - s8;
            const size_t need = (size_t)(s8 * s8 + a8 * a8 + Rb * kKronLd) * sizeof(float);
            smem = need > smem ? need : smem;
        }
        items[(size_t)d * (c->nblk + 1) + c->nblk] = acc;
        K.total[d] = acc;
        K.threads[d] = 2 * kron_rows(nmax);   // kron_rows is monotone in n
        K.smem[d] = smem;
    }
    if (e == cudaSuccess) e = ctx_alloc(c, &K.items, items.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(K.items, items.data(), sizeof(long long) * items.size(), cudaMemcpyHostToDevice);
    size_t smax = 0;
    for (int d = 0; d < 3; ++d) smax = K.smem[d] > smax ? K.smem[d] : smax;
    if (e == cudaSuccess)
        e = ensure_dyn_smem((const void*)k_kron_pass, smax);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kron_pass, K.threads[d], K.smem[d]);
        long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
        K.grid[d] = (int)(grid < K.total[d] ? grid : (K.total[d] > 0 ? K.total[d] : 1));
    }
    if (e == cudaSuccess && K.n_tc > 0) e = setup_kron_tc(c, tcmat, sms);
    return e;
}

// Autotuner of the transforms: per distinct shape (nx, ny, nz, N, periodic
// sides) of the blocks that qualify for the tensor cores, one inner solve of
// one block of that shape is timed (CUDA events, after a warm-up solve, three
// solves averaged, zero input: the transforms' cost does not depend on the
// values) with every qualifying block on the tensor cores and again with
// every block on the CUDA cores; each shape keeps the faster, and the solver
// is planned once more with those choices.  Runs once, at context creation.
cudaError_t kron_autotune(flosic_ctx* c) {
    KronPlan& K = c->kron;
    std::map<std::array<long long, 5>, std::vector<int>> groups;
    for (int b = 0; b < c->nblk; ++b) {
        const BlkDesc& B = c->blk[b];
        if (kron_tc_eligible(B)) groups[{B.nx, B.ny, B.nz, B.N, B.per}].push_back(b);
    }
    if (groups.empty()) return cudaSuccess;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int* dflags = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&dflags, sizeof(int) * (size_t)c->norb * groups.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws.r32, 0, sizeof(float) * (size_t)c->orb_elems, s);
    // per group: only the first block's orbitals active
    std::vector<int> hflags((size_t)c->norb * groups.size(), 0);
    {
        size_t gi = 0;
        for (const auto& g : groups) {
            const BlkDesc& B = c->blk[g.second[0]];
            for (int o = 0; o < B.N; ++o) hflags[gi * c->norb + B.orb0 + o] = 1;
            ++gi;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(dflags, hflags.data(), sizeof(int) * hflags.size(), cudaMemcpyHostToDevice);
    std::vector<float> t_tc(groups.size(), 0.f), t_cc(groups.size(), 0.f);
    auto plan = [&](int force) {   // force 1: every qualifying block on the tensor cores; 0: none
        K.tc_force.assign((size_t)c->nblk, force);
        cudaError_t r = setup_kron(c);
        if (r == cudaSuccess)
            r = cudaMemcpy(c->d_blk, c->blk.data(), sizeof(BlkDesc) * c->nblk, cudaMemcpyHostToDevice);
        return r;
    };
    auto time_groups = [&](std::vector<float>& t) {
        cudaError_t r = cudaSuccess;
        for (size_t gi = 0; gi < groups.size() && r == cudaSuccess; ++gi) {
            for (int rep = 0; rep < 4 && r == cudaSuccess; ++rep) {
                if (rep == 1) r = cudaEventRecord(e0, s);
                if (r == cudaSuccess)
                    r = cudaMemcpyAsync(c->ws.cg.active, dflags + gi * c->norb, sizeof(int) * c->norb,
                                        cudaMemcpyDeviceToDevice, s);
                if (r == cudaSuccess) launch_kron_solve(c, c->ws.r32, c->ws.d32, c->ws.p32, c->ws.q32, s);
            }
            if (r == cudaSuccess) r = cudaEventRecord(e1, s);
            if (r == cudaSuccess) r = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
            t[gi] = ms / 3.f;
        }
        return r;
    };
    if (e == cudaSuccess) e = plan(1);
    if (e == cudaSuccess) e = time_groups(t_tc);
    if (e == cudaSuccess) e = plan(0);
    if (e == cudaSuccess) e = time_groups(t_cc);
    // the choices, then the final plan
    std::vector<int> force((size_t)c->nblk, 1);
    {
        size_t gi = 0;
        for (const auto& g : groups) {
            const int keep_tc = (e != cudaSuccess || t_tc[gi] <= t_cc[gi]) ? 1 : 0;
            for (int b : g.second) force[(size_t)b] = keep_tc;
            ++gi;
        }
    }
    if (s) cudaStreamSynchronize(s);
    cudaGetLastError();
    K.tc_force = force;
    cudaError_t f = setup_kron(c);
    if (f == cudaSuccess) f = cudaMemcpy(c->d_blk, c->blk.data(), sizeof(BlkDesc) * c->nblk, cudaMemcpyHostToDevice);
    if (f == cudaSuccess) f = cudaMemset(c->ws.cg.dmax, 0, sizeof(unsigned) * c->norb);
    if (dflags) cudaFree(dflags);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return f;   // a failed timing keeps the tensor cores; only the final plan's failure is an error
}

// d = A^{-1} r for the active orbitals (float32); t1, t2 are scratch arrays
// of the orbital size.  Marks the orbitals done and counts one iteration.
void launch_kron_solve(flosic_ctx* c, const float* r, float* d, float* t1, float* t2, cudaStream_t s) {
    const KronPlan& K = c->kron;
    KronArgs a{};
    a.blk = c->d_blk;
    a.nblk = c->nblk;
    a.mat = K.mat;
    a.lam = K.lam;
    a.active = c->ws.cg.active;
    a.flops = c->profiling ? c->ws.cg.prof_bytes : nullptr;
    // Pass i of the CUDA-core kernel (standard layout throughout: x, y, z
    // forward, z, y, x inverse) and pass i of the tensor-core kernel (x, y,
    // z forward, x, y, z inverse with rotating layouts) read and write the
    // same arrays, each on its own blocks.
    struct Step { int axis, inverse, scale; const float* in; float* out; };
    const Step steps[6] = {{0, 0, 0, r, t1}, {1, 0, 0, t1, t2}, {2, 0, 1, t2, t1},
                           {2, 1, 0, t1, t2}, {1, 1, 0, t2, t1}, {0, 1, 0, t1, d}};
    prof_begin(c, s);
    for (int i = 0; i < 6; ++i) {
        const Step& st = steps[i];
        if (K.n_simt > 0) {
            a.axis = st.axis;
            a.inverse = st.inverse;
            a.scale = st.scale;
            a.in = st.in;
            a.out = st.out;
            a.item0 = K.items + (size_t)st.axis * (c->nblk + 1);
            k_kron_pass<<<K.grid[st.axis], K.threads[st.axis], K.smem[st.axis], s>>>(a, K.total[st.axis]);
            note_launch(c);
        }
        if (K.n_tc > 0) launch_kron_tc_pass(c, i, st.out, s);
    }
    prof_end(c, s);
    k_kron_done<<<(c->norb + 255) / 256, 256, 0, s>>>(c->norb, c->ws.cg);
    note_launch(c);
}

}  // namespace flosic
