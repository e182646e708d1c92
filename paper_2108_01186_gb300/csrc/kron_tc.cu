// The Kronecker-product transforms of the mixed-precision inner Poisson
// solve on the fifth-generation tensor cores (tcgen05).
//
// Sec. II.A writes the finite-difference Laplacian as a Kronecker sum; its
// inverse is three forward 1-D transforms, a diagonal scaling and three
// inverse transforms (kron.cu has the algebra and the CUDA-core kernel).
// Each transform multiplies every line of one direction by a dense matrix:
// a GEMM with K = the line length, so it belongs on the tensor cores.
//
// Layout.  A pass reads its input as rows (one row = one line, its n points
// contiguous) and writes its output transposed: out[orb][k][row], k the
// position (or mode) along the line.  The three directions therefore rotate
// through the passes: the standard [z][y][x] input r becomes [mx][z][y]
// after the x pass, [my][mx][z] after the y pass, [mz][my][mx] after the z
// pass (with the scaling), [x][mz][my], [y][x][mz] and finally the standard
// [z][y][x] after the inverse x, y and z passes.  Every input row is a
// contiguous run that one tiled bulk copy (TMA, 128-byte swizzle) brings to
// shared memory; every output store is coalesced (the 32 lanes of a warp
// own 32 consecutive rows).
//
// One CTA per SM (13 warps) streams tiles of 128 rows.  The copy engine
// delivers a tile's rows (float32) into one of two staging buffers, so the
// next tile's rows are on their way while this one is converted.  Eight
// converter warps fold each row into its even and odd halves (s_k = v_k +
// v_{n-1-k}, a_k = v_k - v_{n-1-k}: T_d commutes with the reflection, so the
// transform splits into two half-size products) and write each half as
// three bf16 terms (v = v1 + v2 + v3, ~24 significant bits) straight into
// tensor memory, the MMAs' A operand (row i in lane i); the split matrices
// stay in shared memory (B operand, K-major, 128-byte swizzle).  A control
// thread issues the copies and the MMAs (M = 128 rows, N = 64 modes, K = 16
// per instruction): the six split products v_i w_j with i + j <= 2 of each
// half, the v1 w1 product into its own accumulator and the five smaller ones
// into a second.  Four epilogue warps read the accumulators back
// (tcgen05.ld), add them, apply the scaling (forward z) or the even/odd
// recombination (inverse), write 16 output lines of 32 rows at a time to
// shared memory and hand them to the copy engine (tiled bulk stores).
// Operands in tensor memory leave shared memory only the copies, the
// matrices and the output staging to carry.
//
// Accuracy: keeping the dominant product in its own short accumulation
// chain (4 instructions of K = 16 per half) holds the tensor cores'
// float32 accumulation error to the level of a float32 CUDA-core product,
// so two refinement rounds still reach 1e-10 at 128^3.
//
// Blocks qualify when every side is a multiple of 8 and at most 128 and
// their offset keeps rows 16-byte aligned; other blocks keep the CUDA-core
// kernel (kron.cu).  Every mbarrier wait is bounded; a timeout sets bit 4 of
// status word 3, lets the CTA wait (bounded) for its copies and MMAs in
// flight, frees its tensor memory and return.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace flosic {
namespace {

constexpr int kTcRows = 128;                      // rows (lines) per tile: MMA M
constexpr int kTcHalf = 64;                       // half-line length (K) and modes per half (N), padded
constexpr int kTcConv = 256;                      // converter threads (warps 1-8: two per row)
constexpr int kTcEpi = 128;                       // epilogue threads (warps 9-12: one per row)
constexpr int kTcThreads = 32 + kTcConv + kTcEpi; // + the control warp: 13 warps, 128 registers each
constexpr int kTcBTile = kTcHalf * kTcHalf * 2;   // one split of one half-matrix (bf16): 8 KB
constexpr int kTcBox = kTcRows * 32 * 4;          // one copy: 128 rows x 32 points (float32): 16 KB
constexpr int kTcRaw = 4 * kTcBox;                // one tile's rows (up to 128 points): 64 KB
constexpr int kTcLines = 16;                      // output lines per bulk store
constexpr int kTcStage = kTcLines * 32 * 4;       // one bulk store: 16 lines x 32 rows (float32): 2 KB
constexpr int kTcOffB = 0;                        // 6 half-matrix tiles (2 halves x 3 splits)
constexpr int kTcOffRaw = kTcOffB + 6 * kTcBTile; // two tile buffers of staged rows
constexpr int kTcOffOut = kTcOffRaw + 2 * kTcRaw; // per epilogue warp: 2 buffers x 2 stores
constexpr int kTcSmem = kTcOffOut + 4 * 4 * kTcStage + 1024;   // + 1024-byte alignment slack
constexpr uint32_t kTcCols = 512;                 // tensor-memory columns
constexpr uint32_t kTcColA = 256;                 // A operands: half h, split s at 256 + 32 (3 h + s)
constexpr int kTcMatElems = 64 * 64;              // one padded half-matrix
constexpr int kTcOpElems = 12 * kTcMatElems;      // per operator: 2 directions x 2 halves x 3 splits

__constant__ int c_tc_pa[6] = {0, 0, 1, 0, 2, 1};   // split of the data operand (A) of product p
__constant__ int c_tc_pb[6] = {0, 1, 0, 2, 0, 1};   // split of the matrix operand (B)

struct KronTcArgs {
    const BlkDesc* blk;
    int nblk;
    const long long* item0;   // [nblk + 1] first tile of each block in this pass
    const CUtensorMap* maps;  // [nblk] the pass's input rows of each block
    const CUtensorMap* omaps; // [nblk] the pass's output lines of each block (16 lines x 32 rows)
    const uint16_t* mat;      // bf16 split matrices (kTcOpElems per operator)
    const float* lam;         // eigenvalues per distinct operator
    float* out;
    const int* active;
    double* flops;            // algorithmic flop counter (profiling) or null
    unsigned* dmax;           // [norb] max |output| per orbital (float bits, atomicMax) or null
    int* status;
    int axis, inverse, scale;
};

struct TcTile {
    int b, o, q;   // block, orbital within the block, tile within the orbital
};

// What a warp needs of its tile's block, read once per block change.
struct TcBlk {
    int b = -1, n, ns, nx;
    long long G, R, off;
    long long kt, kl0, kl1, kl2;
};

__device__ __forceinline__ void tc_blk_load(TcBlk& k, const BlkDesc* blk, int b, int axis) {
    if (k.b == b) return;
    const BlkDesc& B = blk[b];
    k.b = b;
    k.n = axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
    k.ns = k.n >> 1;
    k.nx = B.nx;
    k.G = B.G;
    k.R = B.G / k.n;
    k.off = B.off;
    k.kt = B.kt[axis];
    k.kl0 = B.kl[0];
    k.kl1 = B.kl[1];
    k.kl2 = B.kl[2];
}

__device__ __forceinline__ int tc_side(const BlkDesc& B, int axis) { return axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz); }

__device__ __forceinline__ int tc_tiles_per_orb(const BlkDesc& B, int axis) {
    const long long R = B.G / tc_side(B, axis);
    return (int)((R + kTcRows - 1) / kTcRows);
}

// next item at or after it whose orbital is active (it1 if none); b tracks the block
__device__ __forceinline__ long long tc_next(const KronTcArgs& a, long long it, long long it1, int& b, TcTile& t) {
    for (; it < it1; ++it) {
        while (b + 1 < a.nblk && it >= a.item0[b + 1]) ++b;
        const BlkDesc& B = a.blk[b];
        const int tpo = tc_tiles_per_orb(B, a.axis);
        const long long r = it - a.item0[b];
        const int o = (int)(r / tpo);
        if (a.active[B.orb0 + o]) {
            t.b = b;
            t.o = o;
            t.q = (int)(r - (long long)o * tpo);
            return it;
        }
    }
    return it1;
}

// Three bf16 terms of a pair of floats (f0, f1), each packed as bf16x2 (f0 in
// the low half): v = v1 + v2 + v3 with v1 = bf16(v), v2 = bf16(v - v1),
// v3 = bf16(v - v1 - v2) (the differences are exact in float32).
__device__ __forceinline__ void tc_split2(float f0, float f1, uint32_t& w1, uint32_t& w2, uint32_t& w3) {
    const __nv_bfloat162 b1 = __floats2bfloat162_rn(f0, f1);
    w1 = *reinterpret_cast<const uint32_t*>(&b1);
    const float r0 = f0 - __uint_as_float(w1 << 16), r1 = f1 - __uint_as_float(w1 & 0xffff0000u);
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0, r1);
    w2 = *reinterpret_cast<const uint32_t*>(&b2);
    const float q0 = r0 - __uint_as_float(w2 << 16), q1 = r1 - __uint_as_float(w2 & 0xffff0000u);
    const __nv_bfloat162 b3 = __floats2bfloat162_rn(q0, q1);
    w3 = *reinterpret_cast<const uint32_t*>(&b3);
}

// four consecutive points pos..pos+3 (pos a multiple of 4) of row r of the staged copy
__device__ __forceinline__ float4 tc_raw4(const unsigned char* sR, int r, int pos) {
    return *reinterpret_cast<const float4*>(sR + (pos >> 5) * kTcBox + r * 128 + ((((pos & 31) >> 2) ^ (r & 7)) << 4));
}

// Warp roles: warp 0 issues the copies and the MMAs (one lane), warps 1-8
// convert (two threads per row: warp w owns tensor-memory lanes
// 32 (w mod 4) .. + 31, K values 32 kp .. + 31 with kp = (w - 1) / 4),
// warps 9-12 drain the accumulators and store (one thread per row).  They
// meet only at mbarriers:
//   bar_tma[b]   rows of the tile in staging buffer b have arrived  (copy engine)
//   bar_raw[b]   every converter has read buffer b                   (8 warp arrivals)
//   bar_conv[h]  half h's operand splits are in tensor memory        (8 warp arrivals)
//   bar_half[h]  half h's MMAs have completed                        (MMA commit)
//   bar_mma      the tile's MMAs have completed                      (MMA commit)
//   bar_empty    the epilogue has read the accumulators              (4 warp arrivals)
// Tile t's rows land in buffer t mod 2, and the copy of tile t + 2 is issued
// as soon as tile t's rows are read, so a copy has two tiles' time to land;
// the even half's MMAs run while the odd half is converted, and the
// accumulators are read before the next tile's MMAs overwrite them.  Every
// wait sleeps on its mbarrier, gives up after about two seconds or as soon
// as another warp has given up (s_abort), and the decision is warp-uniform.
__global__ void __launch_bounds__(kTcThreads, 1) k_kron_tc(KronTcArgs a, long long total) {
    extern __shared__ unsigned char kt_smem_raw[];
    __shared__ uint64_t bar_tma[2], bar_raw[2], bar_conv[2], bar_half[2], bar_mma, bar_empty;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_abort;
    __shared__ int s_tma_issued[2], s_mma_issued;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long per_cta = (total + gridDim.x - 1) / gridDim.x;
    const long long it0 = (long long)blockIdx.x * per_cta;
    const long long it1 = it0 + per_cta < total ? it0 + per_cta : total;
    if (it0 >= it1) return;
    int bsearch = 0;
    TcTile first{};
    const long long item0 = tc_next(a, it0, it1, bsearch, first);
    if (item0 >= it1) return;   // uniform: every thread walks the same items

    unsigned char* sm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(kt_smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sB = sm + kTcOffB;
    unsigned char* sR = sm + kTcOffRaw;
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc_mbar_init(&bar_tma[b], 1);
            tc_mbar_init(&bar_raw[b], kTcConv / 32);
            tc_mbar_init(&bar_conv[b], kTcConv / 32);
            tc_mbar_init(&bar_half[b], 1);
            s_tma_issued[b] = 0;
        }
        tc_mbar_init(&bar_mma, 1);
        tc_mbar_init(&bar_empty, kTcEpi / 32);
        s_abort = 0;
        s_mma_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, kTcCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- control: copies and MMAs (lane 0) --------------------------------
        if (lane == 0) {
            TcBlk kc;
            auto issue_copy = [&](const TcTile& t, int buf) {
                tc_blk_load(kc, a.blk, t.b, a.axis);
                const int nbox = (kc.n + 31) >> 5;
                const int row0 = (int)((long long)t.o * kc.R + (long long)t.q * kTcRows);
                unsigned char* dst = sR + buf * kTcRaw;
                tc_mbar_expect_tx(&bar_tma[buf], (uint32_t)(nbox * kTcBox));
                for (int bx = 0; bx < nbox; ++bx)
                    tc_tma_load_2d(dst + bx * kTcBox, a.maps + t.b, 32 * bx, row0, &bar_tma[buf]);
                ++s_tma_issued[buf];
            };
            const uint32_t idesc = umma_idesc_bf16(kTcRows, kTcHalf);
            const uint32_t b0 = tc_smem_addr(sB);
            // copies run two tiles ahead: tile t (cur), t + 1 (t1, item n1), t + 2 (t2, item n2)
            int bs = bsearch;
            TcTile cur = first, t1{}, t2{};
            long long n1 = tc_next(a, item0 + 1, it1, bs, t1);
            long long n2 = n1 < it1 ? tc_next(a, n1 + 1, it1, bs, t2) : it1;
            issue_copy(first, 0);
            if (n1 < it1) issue_copy(t1, 1);
            for (int t = 0;; ++t) {
                // tile t's rows are read: the copy of tile t + 2 may land in their buffer
                if (!tc_mbar_sleep_or_abort(&bar_raw[t & 1], (uint32_t)((t >> 1) & 1), &s_abort)) break;
                if (n2 < it1) issue_copy(t2, t & 1);
                bool ok = true;
                for (int h = 0; h < 2 && ok; ++h) {
                    ok = tc_mbar_sleep_or_abort(&bar_conv[h], (uint32_t)(t & 1), &s_abort);
                    // the accumulators were read by the epilogue of tile t - 1
                    if (ok && h == 0 && t >= 1)
                        ok = tc_mbar_sleep_or_abort(&bar_empty, (uint32_t)((t - 1) & 1), &s_abort);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t dm = tmem + (uint32_t)(h * 128);
                    const uint32_t am = tmem + kTcColA + (uint32_t)(h * 96);
#pragma unroll 1
                    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                        for (int p = 0; p < 6; ++p) {
                            const uint32_t ta = am + (uint32_t)(32 * c_tc_pa[p] + 8 * kk);
                            const uint64_t db = umma_desc_sw128(b0 + (h * 3 + c_tc_pb[p]) * kTcBTile + kk * 32);
                            if (p == 0) umma_bf16_ts(dm, ta, db, idesc, kk != 0);
                            else umma_bf16_ts(dm + 64, ta, db, idesc, (kk | (p - 1)) != 0);
                        }
                    }
                    umma_commit(&bar_half[h]);
                }
                if (!ok) break;
                umma_commit(&bar_mma);
                ++s_mma_issued;
                if (a.flops) {
                    const BlkDesc& B = a.blk[cur.b];
                    const int n = tc_side(B, a.axis), ns = n >> 1;
                    const long long rows = B.G / n - (long long)cur.q * kTcRows;
                    atomicAdd(a.flops, 4.0 * (double)ns * ns * (double)(rows < kTcRows ? rows : kTcRows));
                }
                if (n1 >= it1) break;
                cur = t1;
                t1 = t2;
                n1 = n2;
                n2 = n1 < it1 ? tc_next(a, n1 + 1, it1, bs, t2) : it1;
            }
        }
        __syncwarp();
    } else if (warp <= kTcConv / 32) {
        // ---- converters: rows in, fold, split, operand splits in tensor memory --
        const int qd = warp & 3;                         // tensor-memory lane quadrant
        const int r = 32 * qd + lane;                    // row of the tile
        const int kp = (warp - 1) >> 2;                  // K values 32 kp .. 32 kp + 31
        const uint32_t ta_row = tmem + ((uint32_t)(32 * qd) << 16) + kTcColA + (uint32_t)(16 * kp);
        TcTile cur = first;
        long long item = item0;
        int bs = bsearch, loaded_b = -1;
        TcBlk kb;
        for (int t = 0;; ++t) {
            bool ok = tc_mbar_sleep_or_abort(&bar_tma[t & 1], (uint32_t)((t >> 1) & 1), &s_abort);
            if (!__all_sync(0xffffffffu, ok)) { s_abort = 1; break; }
            tc_blk_load(kb, a.blk, cur.b, a.axis);
            const int n = kb.n, ns = kb.ns;
            const unsigned char* raw = sR + (t & 1) * kTcRaw;
            float4 fr[8], bk[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int k = 32 * kp + 4 * g;
                fr[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                bk[g] = fr[g];
                if (k < ns) {
                    fr[g] = tc_raw4(raw, r, k);
                    bk[g] = tc_raw4(raw, r, a.inverse ? ns + k : n - 4 - k);
                }
            }
            __syncwarp();
            if (lane == 0) tc_mbar_arrive(&bar_raw[t & 1]);   // the staged rows may be overwritten
            bool wrote_b = false;
            if (cur.b != loaded_b) {   // this block's matrices, once the last tile's MMAs have completed
                ok = t < 1 || tc_mbar_sleep_or_abort(&bar_half[1], (uint32_t)((t - 1) & 1), &s_abort);
                if (!__all_sync(0xffffffffu, ok)) { s_abort = 1; break; }
                const uint16_t* src = a.mat + kb.kt + (a.inverse ? 6 * kTcMatElems : 0);
                for (int i = tid - 32; i < 6 * 64 * 8; i += kTcConv) {
                    const int mt = i >> 9, m = (i >> 3) & 63, c = i & 7;
                    const uint4 v = *reinterpret_cast<const uint4*>(src + mt * kTcMatElems + m * 64 + c * 8);
                    *reinterpret_cast<uint4*>(sB + mt * kTcBTile + m * 128 + ((c ^ (m & 7)) << 4)) = v;
                }
                loaded_b = cur.b;
                wrote_b = true;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // the last tile's MMAs of this half have read its operand splits
                ok = t < 1 || tc_mbar_sleep_or_abort(&bar_half[h], (uint32_t)((t - 1) & 1), &s_abort);
                if (!__all_sync(0xffffffffu, ok)) {
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t th = ta_row + (uint32_t)(h * 96);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {   // K = 32 kp + 8 cc .. + 7: columns 16 kp + 4 cc .. + 3
                    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float4 x = fr[2 * cc + e], y = bk[2 * cc + e];
                        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
                        float v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (a.inverse) v[i] = h == 0 ? xs[i] : ys[i];
                            else v[i] = h == 0 ? xs[i] + ys[3 - i] : xs[i] - ys[3 - i];
                        }
                        tc_split2(v[0], v[1], w1[2 * e], w2[2 * e], w3[2 * e]);
                        tc_split2(v[2], v[3], w1[2 * e + 1], w2[2 * e + 1], w3[2 * e + 1]);
                    }
                    tmem_st4(th + (uint32_t)(4 * cc), w1[0], w1[1], w1[2], w1[3]);
                    tmem_st4(th + (uint32_t)(32 + 4 * cc), w2[0], w2[1], w2[2], w2[3]);
                    tmem_st4(th + (uint32_t)(64 + 4 * cc), w3[0], w3[1], w3[2], w3[3]);
                }
                tmem_wait_st();
                if (h == 0 && wrote_b) tc_fence_proxy_async();   // the matrices, for the MMAs' reads
                tc_fence_before();
                __syncwarp();
                if (lane == 0) tc_mbar_arrive(&bar_conv[h]);
            }
            if (s_abort) break;
            TcTile nxt_t{};
            const long long nxt = tc_next(a, item + 1, it1, bs, nxt_t);
            if (nxt >= it1) break;
            cur = nxt_t;
            item = nxt;
        }
    } else {
        // ---- epilogue: accumulators -> scaling / recombination -> stores -------
        const int g4 = warp & 3;                                  // TMEM lanes 32 g4 .. = tile rows
        const int r = 32 * g4 + lane;                             // one row per thread
        float* const stage = reinterpret_cast<float*>(sm + kTcOffOut + (warp - 1 - kTcConv / 32) * 4 * kTcStage);
        TcTile cur = first;
        long long item = item0;
        int bs = bsearch, u = 0;   // u: bulk-stored line groups so far (staging buffer u mod 2)
        TcBlk kb;
        for (int t = 0;; ++t) {
            const bool ok = tc_mbar_sleep_or_abort(&bar_mma, (uint32_t)(t & 1), &s_abort);
            if (!__all_sync(0xffffffffu, ok)) { s_abort = 1; break; }
            tc_fence_after();
            tc_blk_load(kb, a.blk, cur.b, a.axis);
            const int n = kb.n, ns = kb.ns;
            const long long R = kb.R;
            const long long l = (long long)cur.q * kTcRows + r;   // row within the orbital
            const int x0 = cur.q * kTcRows + 32 * g4;               // first row of this warp's lines
            float lxy = 0.f;
            if (a.scale && l < R) {   // forward z: rows are (my, mx), mx fastest
                const int li = (int)l, my = li / kb.nx, mx = li - my * kb.nx;
                lxy = a.lam[kb.kl0 + mx] + a.lam[kb.kl1 + my];
            }
            const float* lz = a.lam + kb.kl2;
            const uint32_t ta = tmem + ((uint32_t)(32 * g4) << 16);
            float amax = 0.f;   // max |output| of this row (for a.dmax)
            float* const dst = a.out + kb.off + (long long)cur.o * kb.G + (l < R ? l : 0);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float e0[16], e1[16], o0[16], o1[16];
                tmem_ld16(ta + 16 * c, e0);
                tmem_ld16(ta + 16 * c + 64, e1);
                tmem_ld16(ta + 16 * c + 128, o0);
                tmem_ld16(ta + 16 * c + 192, o1);
                tmem_wait_ld();
                if (c == 3) {   // the accumulators are read: the next tile's MMAs may overwrite them
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc_mbar_arrive(&bar_empty);
                }
                const int m0 = 16 * c;
                if (m0 >= ns) continue;
                // lines of output position p1 = m (forward: even mode m; inverse: point m) and
                // p2 (forward: odd mode ns + m; inverse: point n - 1 - m)
                float v1[16], v2[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float ve = e0[j] + e1[j], vo = o0[j] + o1[j];
                    if (!a.inverse) {
                        if (a.scale) {   // (fast division: 2 ulp, far below the solve's accuracy)
                            const float se = lxy + lz[m0 + j], so = lxy + lz[ns + m0 + j];
                            ve = se > 0.f ? __fdividef(ve, se) : 0.f;
                            vo = so > 0.f ? __fdividef(vo, so) : 0.f;
                        }
                        v1[j] = ve;
                        v2[j] = vo;
                    } else {
                        v1[j] = ve + vo;
                        v2[j] = ve - vo;
                    }
                }
                if (a.dmax) {   // (last inverse pass only) a tree of maxima, not a chain
                    float mj[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float u0 = m0 + j < ns ? fmaxf(fabsf(v1[j]), fabsf(v2[j])) : 0.f;
                        const float u1 = m0 + j + 8 < ns ? fmaxf(fabsf(v1[j + 8]), fabsf(v2[j + 8])) : 0.f;
                        mj[j] = fmaxf(u0, u1);
                    }
                    amax = fmaxf(amax, fmaxf(fmaxf(fmaxf(mj[0], mj[1]), fmaxf(mj[2], mj[3])),
                                             fmaxf(fmaxf(mj[4], mj[5]), fmaxf(mj[6], mj[7]))));
                }
                if (m0 + kTcLines <= ns) {
                    // 16 whole lines: stage them (line j of 32 rows) and store in bulk
                    float* const sb = stage + (u & 1) * 2 * (kTcStage / 4);
                    if (lane == 0) tc_bulk_wait_read1();   // the store from this buffer two groups ago has read it
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        sb[j * 32 + lane] = v1[j];
                        sb[kTcStage / 4 + (a.inverse ? 15 - j : j) * 32 + lane] = v2[j];
                    }
                    tc_fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        if (x0 < R) {
                            const int y0 = cur.o * n;
                            tc_tma_store_2d(a.omaps + cur.b, x0, y0 + m0, sb);
                            tc_tma_store_2d(a.omaps + cur.b, x0, y0 + (a.inverse ? n - kTcLines - m0 : ns + m0),
                                            sb + kTcStage / 4);
                        }
                        tc_bulk_commit();
                    }
                    ++u;
                } else if (l < R) {
                    // a partial group of lines (ns not a multiple of 16): plain stores
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (m0 + j < ns) {
                            const int k1 = m0 + j, k2 = a.inverse ? n - 1 - m0 - j : ns + m0 + j;
                            __stcs(dst + (long long)k1 * R, v1[j]);
                            __stcs(dst + (long long)k2 * R, v2[j]);
                        }
                    }
                }
            }
            if (a.dmax) {   // rows past the orbital's last one hold no output
                float m = l < R ? amax : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0 && m > 0.f) atomicMax(a.dmax + a.blk[cur.b].orb0 + cur.o, __float_as_uint(m));
            }
            TcTile nxt_t{};
            const long long nxt = tc_next(a, item + 1, it1, bs, nxt_t);
            if (nxt >= it1) break;
            cur = nxt_t;
            item = nxt;
        }
        if (lane == 0) tc_bulk_wait_all();   // the bulk stores have completed
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0) {
        atomicOr(a.status + 3, 4);
        // let the copies and the MMAs this CTA has in flight finish (bounded)
        for (int b = 0; b < 2; ++b)
            if (s_tma_issued[b] > 0) tc_mbar_wait(&bar_tma[b], (uint32_t)((s_tma_issued[b] - 1) & 1));
        if (s_mma_issued > 0) tc_mbar_wait(&bar_mma, (uint32_t)((s_mma_issued - 1) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTcCols);
    }
}

uint16_t host_bf16(float f) {   // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double host_bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

}  // namespace

bool kron_tc_eligible(const BlkDesc& B) {
    const int nd[3] = {B.nx, B.ny, B.nz};
    for (int d = 0; d < 3; ++d)
        if (nd[d] < 8 || nd[d] > 2 * kTcHalf || nd[d] % 8 != 0) return false;
    return B.off % 4 == 0;
}

// The operator's four half-matrices in the transform kernel's operand form
// (rows = outputs, K = inputs, padded to 64 x 64), each as three bf16
// splits of the float64 value: [direction][half][split][64][64].
//   forward: c_s[m] = sum_k s_k Vs[k][m] / sqrt 2, c_a[m] = sum_k a_k Va[k][m] / sqrt 2
//   inverse: S_k = sum_m c_s[m] Vs[k][m] / sqrt 2, A_k = sum_m c_a[m] Va[k][m] / sqrt 2
// (n even, so every even/odd basis vector carries 1/sqrt 2).
void kron_tc_pack(int n, const std::vector<double>& Vs, const std::vector<double>& Va, std::vector<uint16_t>& out) {
    const int h = n / 2;
    const double r2 = std::sqrt(0.5);
    const size_t o0 = out.size();
    out.resize(o0 + kTcOpElems, 0);
    for (int dir = 0; dir < 2; ++dir)
        for (int half = 0; half < 2; ++half) {
            const std::vector<double>& V = half == 0 ? Vs : Va;
            for (int row = 0; row < h; ++row)
                for (int k = 0; k < h; ++k) {
                    // forward: row = mode m, k = point; inverse: row = point, k = mode
                    const double v = (dir == 0 ? V[(size_t)k * h + row] : V[(size_t)row * h + k]) * r2;
                    const uint16_t b1 = host_bf16((float)v);
                    const double q1 = v - host_bf16_value(b1);
                    const uint16_t b2 = host_bf16((float)q1);
                    const double q2 = q1 - host_bf16_value(b2);
                    const uint16_t b3 = host_bf16((float)q2);
                    const uint16_t bs[3] = {b1, b2, b3};
                    for (int s = 0; s < 3; ++s)
                        out[o0 + (size_t)((dir * 2 + half) * 3 + s) * kTcMatElems + (size_t)row * 64 + k] = bs[s];
                }
        }
}

size_t kron_tc_smem() { return (size_t)kTcSmem; }
const void* kron_tc_symbol() { return (const void*)k_kron_tc; }

// Input rows of pass `step` (axis step mod 3) of block B as a 2-D tensor map:
// n points per row (contiguous), N G / n rows, boxes of 32 points x 128 rows.
bool kron_tc_map(void* encode_fn, CUtensorMap* map, const BlkDesc& B, int axis, const float* buf) {
    auto encode = reinterpret_cast<CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                                CUtensorMapInterleave, CUtensorMapSwizzle,
                                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill)>(encode_fn);
    const int n = axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)(B.G / n) * (cuuint64_t)B.N};
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};
    const cuuint32_t box[2] = {32, (cuuint32_t)kTcRows};
    const cuuint32_t estr[2] = {1, 1};
    void* base = const_cast<float*>(buf) + B.off;
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output lines of pass `step` of block B as a 2-D tensor map: the output is
// out[orb][k][row], so R = G / n rows per line (contiguous) and N n lines;
// boxes of 32 rows x 16 lines, no swizzle (the epilogue stages line-major).
bool kron_tc_map_out(void* encode_fn, CUtensorMap* map, const BlkDesc& B, int axis, float* buf) {
    auto encode = reinterpret_cast<CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                                CUtensorMapInterleave, CUtensorMapSwizzle,
                                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill)>(encode_fn);
    const int n = axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
    const long long R = B.G / n;
    const cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)n * (cuuint64_t)B.N};
    const cuuint64_t strides[1] = {(cuuint64_t)R * sizeof(float)};
    const cuuint32_t box[2] = {32, (cuuint32_t)kTcLines};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, buf + B.off, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long long kron_tc_tiles(const BlkDesc& B, int axis) {
    const int n = axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
    const long long R = B.G / n;
    return (long long)B.N * ((R + kTcRows - 1) / kTcRows);
}

void launch_kron_tc_pass(flosic_ctx* c, int step, float* out, cudaStream_t s) {
    const KronPlan& K = c->kron;
    KronTcArgs a{};
    a.blk = c->d_blk;
    a.nblk = c->nblk;
    a.item0 = K.tc_items + (size_t)step * (c->nblk + 1);
    a.maps = reinterpret_cast<const CUtensorMap*>(K.tc_maps) + (size_t)step * c->nblk;
    a.omaps = reinterpret_cast<const CUtensorMap*>(K.tc_omaps) + (size_t)step * c->nblk;
    a.mat = K.tc_mat;
    a.lam = K.lam;
    a.out = out;
    a.active = c->ws.cg.active;
    a.flops = c->profiling ? c->ws.cg.prof_bytes : nullptr;
    a.dmax = step == 5 ? c->ws.cg.dmax : nullptr;   // the correction d: its scale for the refinement update
    a.status = c->ws.status;
    a.axis = step % 3;
    a.inverse = step >= 3;
    a.scale = step == 2;
    k_kron_tc<<<K.tc_grid[step], kTcThreads, kTcSmem, s>>>(a, K.tc_total[step]);
    note_launch(c);
}

}  // namespace flosic
