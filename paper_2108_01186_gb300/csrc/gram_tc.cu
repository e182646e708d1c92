// Grid-summed overlap Gram M_ab = sum_g psi_a(g) psi_b(g) on the fifth-
// generation tensor cores (the overlap of the Fermi orbitals, S = dV F F^T =
// dV T M T^T, Sec. II, Eqs. 6-8), mixed-precision path.
//
// Split-BF16: each float64 value is taken to float32 (integer operations) and
// written as three bfloat16 terms v = v1 + v2 + v3 (~24 significant bits).
// The products v1w1 + v1w2 + v2w1 + v1w3 + v3w1 + v2w2 keep float32-level
// accuracy; they are six tcgen05.mma (kind::f16, bf16 inputs, float32
// accumulation in tensor memory) per 16-point K slice, M = 128 (orbital rows
// padded), N = the orbital count rounded up to 32.  One CTA sums a chunk of
// 2048 grid points of one spin block, writes the float32 partial, and a
// second kernel adds the partials in float64 in a fixed order.
//
// Per 64-point stage the CTA's 128 threads load the N x 64 float64 block,
// split it and store the three bf16 tiles K-major with the 128-byte swizzle
// (row r, 16-byte chunk c at chunk c ^ (r mod 8)); thread 0 issues the MMAs
// and commits them to the stage's mbarrier.  Two stages alternate; every
// mbarrier wait is bounded and a timeout sets the status word.
//
// The tensor cores' float32 accumulation drifts with the length of the
// accumulation chain (measured: S off by ~1e-5 after 2048 points, ~2e-6
// after 256).  So the hi x hi products, which carry almost all of the sum,
// go to a TMEM accumulator that restarts every 64-point stage (two of them,
// alternating); each finished stage is read back (tcgen05.ld) and added in
// float32 registers with round-to-nearest.  The five cross products
// (<= 2^-8 of the total) stay in one accumulator for the whole chunk.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace flosic {

constexpr int kGK = 64;                      // grid points per stage (128 bytes of bf16 per row)
constexpr int kGChunk = 2048;                // grid points per CTA
constexpr int kGRows = 128;                  // MMA M: orbital rows, padded
constexpr int kGTile = kGRows * kGK * 2;     // one bf16 tile: 16 KB
constexpr int kGStages = 2;
constexpr int kGSmem = kGStages * 3 * kGTile + 1024;   // + 1024-byte alignment slack

// the six split pairs (i, j) with i + j <= 2 (0-based), A split i with B split j
__constant__ int c_pair_a[6] = {0, 0, 1, 0, 2, 1};
__constant__ int c_pair_b[6] = {0, 1, 0, 2, 0, 1};

// Three bf16 terms of a pair of floats (f0, f1), each packed as bf16x2 (f0 in
// the low half): v = v1 + v2 + v3 with v1 = bf16(v), v2 = bf16(v - v1),
// v3 = bf16(v - v1 - v2) (the differences are exact in float32).
__device__ __forceinline__ void gram_split2(float f0, float f1, uint32_t& w1, uint32_t& w2, uint32_t& w3) {
    const __nv_bfloat162 b1 = __floats2bfloat162_rn(f0, f1);
    w1 = *reinterpret_cast<const uint32_t*>(&b1);
    const float r0 = f0 - __uint_as_float(w1 << 16), r1 = f1 - __uint_as_float(w1 & 0xffff0000u);
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0, r1);
    w2 = *reinterpret_cast<const uint32_t*>(&b2);
    const float q0 = r0 - __uint_as_float(w2 << 16), q1 = r1 - __uint_as_float(w2 & 0xffff0000u);
    const __nv_bfloat162 b3 = __floats2bfloat162_rn(q0, q1);
    w3 = *reinterpret_cast<const uint32_t*>(&b3);
}

// Reads 32 columns of this warp's 32 TMEM lanes and adds them to acc.
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float* acc) {
    float v[32];
    tmem_ld32(taddr, v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] += v[j];
}

// Orbital rows are padded to NN = 32 NB per sub-chunk; with NN <= 64 several
// point sub-chunks share the 128 MMA rows (P = 128 / NN of them: row q NN + a
// holds orbital a over the points of sub-chunk q), so no MMA row is padding
// when N is a multiple of 32 and a stage moves P times as many points.  The
// MMA then runs N = P NN columns, and only the diagonal blocks (sub-chunk q
// with itself) are read back: warp w holds rows 32 w .. 32 w + 31, i.e. part
// of sub-chunk q = 32 w / NN, and reads its block's NN columns from q NN.
template <int NB>
__host__ __device__ constexpr int gram_pack() { return (32 * NB <= 64) ? 128 / (32 * NB) : 1; }

template <int NB>   // NB = orbital rows per sub-chunk / 32 (1 .. 4)
__global__ void __launch_bounds__(256, NB <= 2 ? 2 : 1) k_gram_tc(const BlkDesc* __restrict__ blk, const double* __restrict__ psi,
                                                    float* __restrict__ part, const long long* __restrict__ part_off,
                                                    int* __restrict__ status) {
    extern __shared__ unsigned char g_smem_raw[];
    __shared__ uint64_t mbar[kGStages];
    __shared__ uint32_t tmem_base;
    constexpr int NN = 32 * NB;                      // orbital rows per sub-chunk
    constexpr int P = gram_pack<NB>();               // sub-chunks sharing the 128 rows
    constexpr int MN = P * NN;                       // MMA N (columns of one accumulator)
    constexpr int kSub = kGChunk / P;                // points per sub-chunk
    constexpr uint32_t kCols = (2 * MN <= 128) ? 128 : 256;
    const BlkDesc& B = blk[blockIdx.y];
    if (B.gtma) return;                              // k_gram_tma's block
    const int N = B.N;
    const long long g_begin = (long long)blockIdx.x * kGChunk;
    if (g_begin >= B.G) return;                      // whole CTA
    const long long g_end = min(g_begin + (long long)kGChunk, B.G);
    const int nst = kSub / kGK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(g_smem_raw) + 1023) & ~(uintptr_t)1023);
    // zero every tile once: padding rows and points past the chunk stay zero
    for (int i = tid; i < kGStages * 3 * kGTile / 16; i += 256)
        reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        tc_mbar_init(&mbar[0], 1);
        tc_mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;                 // columns: [0,MN) hi x hi of a stage, [MN,2MN) cross
    // warps 0-3 read the accumulator lanes that hold sub-chunk rows (with
    // P NN < 128, as for NN = 96, the last rows are padding: not read)
    const bool reader = warp < 4 && 32 * warp < P * NN;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const int q_own = (32 * (warp & 3)) / NN;        // the reading warp's sub-chunk
    const uint32_t col0 = (uint32_t)(q_own * NN);    // its diagonal block
    const uint32_t idesc = umma_idesc_bf16(kGRows, MN);
    bool ok = true;
    float acc[NN];                                   // row 32 warp + lane of its sub-chunk's sums
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[j] = 0.f;
    const double* pb = psi + B.off;
    const int k = tid & 63;                          // this thread's point within a stage
    constexpr int kRows = P * NN;                    // rows (q, a) of a stage
    constexpr int kGroup = 16;                       // loads in flight per thread before converting
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;                      // (the MMAs of stage st - 2 completed at stage st - 1)
        unsigned char* tile = base + buf * 3 * kGTile;
        // thread: point k of every sub-chunk, rows (q, a) = tid / 64 + 4 i
#pragma unroll 1
        for (int r0 = tid >> 6; r0 < kRows; r0 += 4 * kGroup) {
            double v[kGroup];
#pragma unroll
            for (int i = 0; i < kGroup; ++i) {
                const int row = r0 + 4 * i;
                const int q = row / NN, a = row - q * NN;
                const long long g = g_begin + (long long)q * kSub + (long long)st * kGK + k;
                v[i] = (row < kRows && a < N && g < g_end) ? pb[(long long)a * B.G + g] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < kGroup; ++i) {
                const int row = r0 + 4 * i;
                const int q = row / NN, a = row - q * NN;
                if (row >= kRows || a >= N) continue;
                const float f = d2f(v[i]);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(f);
                const float r1 = f - __bfloat162float(b1);
                const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
                const __nv_bfloat16 b3 = __float2bfloat16_rn(r1 - __bfloat162float(b2));
                const int off = row * 128 + ((((k >> 3) ^ (row & 7))) << 4) + ((k & 7) << 1);
                *reinterpret_cast<__nv_bfloat16*>(tile + off) = b1;
                *reinterpret_cast<__nv_bfloat16*>(tile + kGTile + off) = b2;
                *reinterpret_cast<__nv_bfloat16*>(tile + 2 * kGTile + off) = b3;
            }
        }
        if (st >= 1) {   // the previous stage's hi x hi sums (read before this stage's MMAs restart them)
            const int pb2 = (st - 1) & 1;
            ok = tc_mbar_wait(&mbar[pb2], (uint32_t)(((st - 1) >> 1) & 1)) && ok;
            ok = __all_sync(0xffffffffu, ok);        // tcgen05.ld is warp-collective
            tc_fence_after();
            if (ok && reader) {
#pragma unroll
                for (int c = 0; c < NB; ++c) tmem_add32(tmem + lane_off + col0 + 32 * c, acc + 32 * c);
            }
        }
        tc_fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t s0 = tc_smem_addr(tile);
            const uint32_t dhi = tmem, dx = tmem + (uint32_t)MN;
#pragma unroll
            for (int kk = 0; kk < kGK / 16; ++kk) {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t da = umma_desc_sw128(s0 + c_pair_a[p] * kGTile + kk * 32);
                    const uint64_t db = umma_desc_sw128(s0 + c_pair_b[p] * kGTile + kk * 32);
                    if (p == 0) umma_bf16(dhi, da, db, idesc, kk != 0);          // restarts every stage
                    else umma_bf16(dx, da, db, idesc, (st | kk | (p - 1)) != 0);
                }
            }
            umma_commit(&mbar[buf]);
        }
    }
    // the last stage (its commit covers every MMA of the CTA): its hi x hi
    // sums, then the cross products
    ok = tc_mbar_wait(&mbar[(nst - 1) & 1], (uint32_t)(((nst - 1) >> 1) & 1)) && ok;
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (ok && reader) {
#pragma unroll
        for (int c = 0; c < NB; ++c) tmem_add32(tmem + lane_off + col0 + 32 * c, acc + 32 * c);
#pragma unroll
        for (int c = 0; c < NB; ++c) tmem_add32(tmem + lane_off + (uint32_t)MN + col0 + 32 * c, acc + 32 * c);
        const int a = warp * 32 + lane - q_own * NN;  // orbital of this row in its sub-chunk
        float* out = part + part_off[blockIdx.y] + ((long long)blockIdx.x * P + q_own) * N * N;
        if (a < N) {
#pragma unroll
            for (int j = 0; j < NN; ++j)
                if (j < N) out[(long long)a * N + j] = acc[j];
        }
    } else if (!ok && tid == 0) {
        atomicOr(status + 3, 2);                     // an MMA completion did not arrive in time
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// The same sums with the float64 psi tiles brought to shared memory by
// asynchronous copies (cp.async, 16 bytes each; blocks whose G and offset are
// even, so every piece is 16-byte aligned): a ring of kGRing stages, the copies
// of stage st + 1 in flight while stage st is converted and multiplied, rows
// past N and points past G zero-filled by the copy.  The warps convert rows
// from shared memory (lane l: points 2l, 2l + 1 of one row) into the same
// K-major swizzled bf16 tiles, so no thread waits on a global load.  MMAs,
// read-back and partials as in k_gram_tc.
constexpr int kGRing = 2;
constexpr int kGStage = kGRows * kGK * 8;                    // float64 rows of a stage: 64 KB
constexpr int kGAsyncSmem = kGRing * kGStage + kGStages * 3 * kGTile + 1024;

__device__ __forceinline__ void gram_cp16(void* dst, const void* src, int bytes) {   // bytes 0 or 16
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc_smem_addr(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void gram_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void gram_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

template <int NB>
__global__ void __launch_bounds__(288, 1) k_gram_async(const BlkDesc* __restrict__ blk, const double* __restrict__ psi,
                                                       float* __restrict__ part,
                                                       const long long* __restrict__ part_off,
                                                       int* __restrict__ status) {
    extern __shared__ unsigned char g_smem_raw[];
    // conv_full[b]: bf16 tile b written (8 converter warps); mma_done[b]: the MMAs
    // of the stage in tile b / per-stage accumulator b completed (commit);
    // hi_free[b]: accumulator b read back (4 reader warps)
    __shared__ uint64_t conv_full[2], mma_done[2], hi_free[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_abort;
    __shared__ int s_mma_issued;
    constexpr int NN = 32 * NB;
    constexpr int P = gram_pack<NB>();
    constexpr int MN = P * NN;
    constexpr int kSub = kGChunk / P;
    constexpr uint32_t kCols = 512;                  // two per-stage accumulators + the cross one
    constexpr int kRows = P * NN;                    // rows (q, a) of a stage
    const BlkDesc& B = blk[blockIdx.y];
    if (!B.gtma) return;                             // k_gram_tc's block
    const int N = B.N;
    const long long g_begin = (long long)blockIdx.x * kGChunk;
    if (g_begin >= B.G) return;
    const int nst = kSub / kGK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(g_smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* tiles = base;                                  // kGStages x 3 bf16 tiles
    double* ring = reinterpret_cast<double*>(base + kGStages * 3 * kGTile);
    const double* pb = psi + B.off;
    // stage st: 16-byte piece `lane` (points 2 lane, 2 lane + 1) of rows warp, warp + 8, ...
    auto issue = [&](int st) {
        double* dst = ring + (size_t)(st % kGRing) * kRows * kGK;
#pragma unroll 4
        for (int row = warp; row < kRows; row += 8) {
            const int q = row / NN, a = row - q * NN;
            const long long g = g_begin + (long long)q * kSub + (long long)st * kGK + 2 * lane;
            const bool in = a < N && g < B.G;   // G even: the pair g, g + 1 is inside or outside together
            gram_cp16(dst + (size_t)row * kGK + 2 * lane, in ? pb + (long long)a * B.G + g : pb, in ? 16 : 0);
        }
    };
    for (int i = tid; i < kGStages * 3 * kGTile / 16; i += blockDim.x)   // padding rows stay zero
        reinterpret_cast<uint4*>(tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp < 8) {
        issue(0);
        gram_cp_commit();
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            tc_mbar_init(&conv_full[k], 8);
            tc_mbar_init(&mma_done[k], 1);
            tc_mbar_init(&hi_free[k], 4);
        }
        s_abort = 0;
        s_mma_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t dcross = tmem + (uint32_t)(2 * MN);
    bool ok = true;
    if (warp == 8) {
        // ---- MMA issue (lane 0): per stage, six split products per 16-point K step
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(kGRows, MN);
            for (int st = 0; st < nst && ok; ++st) {
                const int b = st & 1;
                ok = tc_mbar_sleep_or_abort(&conv_full[b], (uint32_t)((st >> 1) & 1), &s_abort);
                // per-stage accumulator b was read back (stage st - 2)
                if (ok && st >= 2) ok = tc_mbar_sleep_or_abort(&hi_free[b], (uint32_t)(((st - 2) >> 1) & 1), &s_abort);
                if (!ok) break;
                tc_fence_after();
                const uint32_t s0 = tc_smem_addr(tiles + b * 3 * kGTile);
                const uint32_t dhi = tmem + (uint32_t)(b * MN);
#pragma unroll
                for (int kk = 0; kk < kGK / 16; ++kk) {
#pragma unroll
                    for (int p = 0; p < 6; ++p) {
                        const uint64_t da = umma_desc_sw128(s0 + c_pair_a[p] * kGTile + kk * 32);
                        const uint64_t db = umma_desc_sw128(s0 + c_pair_b[p] * kGTile + kk * 32);
                        if (p == 0) umma_bf16(dhi, da, db, idesc, kk != 0);   // restarts every stage
                        else umma_bf16(dcross, da, db, idesc, (st | kk | (p - 1)) != 0);
                    }
                }
                umma_commit(&mma_done[b]);
                ++s_mma_issued;
            }
            if (!ok) s_abort = 1;
        }
        __syncwarp();
    } else {
        // ---- converters (warps 0-7); warps 0-3 also read the accumulators back
        const bool reader = warp < 4 && 32 * warp < P * NN;
        const bool rwarp = warp < 4;
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const int q_own = (32 * (warp & 3)) / NN;
        const uint32_t col0 = (uint32_t)(q_own * NN);
        float acc[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) acc[j] = 0.f;
        auto read_back = [&](int st) {   // stage st's per-stage sums into acc, then release them
            const int b = st & 1;
            bool r = tc_mbar_sleep_or_abort(&mma_done[b], (uint32_t)((st >> 1) & 1), &s_abort);
            r = __all_sync(0xffffffffu, r);
            tc_fence_after();
            if (r && reader) {
#pragma unroll
                for (int c = 0; c < NB; ++c) tmem_add32(tmem + lane_off + (uint32_t)(b * MN) + col0 + 32 * c, acc + 32 * c);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) tc_mbar_arrive(&hi_free[b]);
            return r;
        };
        // Every converter warp runs every iteration and every named barrier (a warp
        // that finds s_abort set only skips the work), so no barrier can hang.
        for (int st = 0; st < nst; ++st) {
            const int b = st & 1;
            tc_named_sync(1, 256);   // every converter is done with stage st - 1: its ring slot is free
            if (st + 1 < nst) issue(st + 1);
            gram_cp_commit();
            gram_cp_wait<1>();       // this thread's copies of stage st have landed
            tc_named_sync(1, 256);   // everyone's
            if (s_abort) continue;
            // tile b was last read by the MMAs of stage st - 2
            bool w = st < 2 || tc_mbar_sleep_or_abort(&mma_done[b], (uint32_t)(((st - 2) >> 1) & 1), &s_abort);
            if (!__all_sync(0xffffffffu, w)) { s_abort = 1; continue; }
            tc_fence_after();
            unsigned char* tile = tiles + b * 3 * kGTile;
            const double* rows = ring + (size_t)(st % kGRing) * kRows * kGK;
#pragma unroll 4
            for (int row = warp; row < kRows; row += 8) {
                const double2 v = *reinterpret_cast<const double2*>(rows + (size_t)row * kGK + 2 * lane);
                uint32_t w1, w2, w3;
                gram_split2(d2f(v.x), d2f(v.y), w1, w2, w3);
                const int off = row * 128 + (((lane >> 2) ^ (row & 7)) << 4) + ((lane & 3) << 2);
                *reinterpret_cast<uint32_t*>(tile + off) = w1;
                *reinterpret_cast<uint32_t*>(tile + kGTile + off) = w2;
                *reinterpret_cast<uint32_t*>(tile + 2 * kGTile + off) = w3;
            }
            tc_fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc_mbar_arrive(&conv_full[b]);
            if (rwarp && st >= 1 && !read_back(st - 1)) s_abort = 1;
        }
        gram_cp_wait<0>();
        ok = !s_abort;
        if (ok && rwarp) {
            ok = read_back(nst - 1);   // the last stage: its commit covers every MMA of the CTA
            if (ok && reader) {
#pragma unroll
                for (int c = 0; c < NB; ++c) tmem_add32(dcross + lane_off + col0 + 32 * c, acc + 32 * c);
                const int a = warp * 32 + lane - q_own * NN;
                float* out = part + part_off[blockIdx.y] + ((long long)blockIdx.x * P + q_own) * N * N;
                if (a < N) {
#pragma unroll
                    for (int j = 0; j < NN; ++j)
                        if (j < N) out[(long long)a * N + j] = acc[j];
                }
            }
        }
        if (!ok && tid == 0) atomicOr(status + 3, 2);   // an MMA completion did not arrive in time
    }
    tc_fence_before();
    __syncthreads();
    if (s_abort && tid == 0 && s_mma_issued > 0) {   // let the MMAs in flight finish (bounded)
        const int last = s_mma_issued - 1;
        tc_mbar_wait(&mma_done[last & 1], (uint32_t)((last >> 1) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// M[block][e] = sum over the block's partials (pk per chunk, pk = the
// launch's sub-chunk count, set by its widest block) in float64: a CTA takes
// 32 elements; its 8 warps sum every 8th partial each, and the 8 sums are
// added in a fixed order.
__global__ void __launch_bounds__(256) k_gram_sum(const BlkDesc* __restrict__ blk, const float* __restrict__ part,
                                                  const long long* __restrict__ part_off, double* __restrict__ M,
                                                  int pk) {
    __shared__ double red[8][32];
    const BlkDesc& B = blk[blockIdx.y];
    const int NN2 = B.N * B.N;
    const int e = blockIdx.x * 32 + (threadIdx.x & 31), w = threadIdx.x >> 5;
    const long long nparts = ((B.G + kGChunk - 1) / kGChunk) * pk;
    double s = 0.0;
    if (e < NN2) {
        const float* p = part + part_off[blockIdx.y] + e;
#pragma unroll 8
        for (long long q = w; q < nparts; q += 8) s += (double)p[q * NN2];
    }
    red[w][threadIdx.x & 31] = s;
    __syncthreads();
    if (w == 0 && e < NN2) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        M[B.moff + e] = t;
    }
}

// sub-chunk partials per chunk of every block: set by the widest block, whose
// row width the one launch of the kernel takes for all blocks
static int gram_launch_pack(const flosic_ctx* c) {
    int nmax = 0;
    for (const auto& b : c->blk) nmax = b.N > nmax ? b.N : nmax;
    const int nb = (nmax + 31) / 32;
    return nb <= 1 ? gram_pack<1>() : nb == 2 ? gram_pack<2>() : 1;
}

long long gram_tc_part_elems(const flosic_ctx* c, std::vector<long long>& off) {
    long long total = 0;
    off.clear();
    const int pk = gram_launch_pack(c);
    for (const auto& b : c->blk) {
        off.push_back(total);
        total += ((b.G + kGChunk - 1) / kGChunk) * pk * (long long)b.N * b.N;
    }
    return total;
}

cudaError_t setup_gram_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)k_gram_async<1>, kGAsyncSmem);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)k_gram_async<2>, kGAsyncSmem);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)k_gram_async<3>, kGAsyncSmem);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)k_gram_async<4>, kGAsyncSmem);
    return e;
}

// blocks whose psi rows the asynchronous-copy kernel can take (16-byte pieces)
bool gram_async_eligible(const BlkDesc& B) { return B.G % 2 == 0 && B.off % 2 == 0; }

void launch_gram_tc(const flosic_ctx* c, const double* psi, cudaStream_t s) {
    long long gmax = 0;
    int nmax = 0;
    for (const auto& b : c->blk) {
        gmax = b.G > gmax ? b.G : gmax;
        nmax = b.N > nmax ? b.N : nmax;
    }
    const dim3 grid((unsigned)((gmax + kGChunk - 1) / kGChunk), (unsigned)c->nblk);
    const int nb = (nmax + 31) / 32;   // accumulator width for the widest block
    float* part = c->ws.gram_part;
    const long long* off = c->ws.gram_off;
    flosic_ctx* cm = const_cast<flosic_ctx*>(c);
    const bool timed = cm->profiling && !cm->ov_ev.empty();
    if (timed) {
        if (2 * (cm->ov_used + 1) > (int)cm->ov_ev.size()) {   // pool full: wait and sum
            cudaEventSynchronize(cm->ov_ev[2 * cm->ov_used - 1]);
            ov_collect(cm);
        }
        cudaEventRecord(cm->ov_ev[2 * cm->ov_used], s);
        for (const auto& b : c->blk) cm->ov_flops += 2.0 * b.N * b.N * (double)b.G;
    }
    int n_async = 0;
    for (const auto& b : c->blk) n_async += b.gtma;
    if (n_async > 0) {   // blocks with 16-byte aligned rows: copies staged asynchronously
        if (nb <= 1) k_gram_async<1><<<grid, 288, kGAsyncSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else if (nb == 2) k_gram_async<2><<<grid, 288, kGAsyncSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else if (nb == 3) k_gram_async<3><<<grid, 288, kGAsyncSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else k_gram_async<4><<<grid, 288, kGAsyncSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        note_launch(cm);
    }
    if (n_async < c->nblk) {   // the others: thread loads
        if (nb <= 1) k_gram_tc<1><<<grid, 256, kGSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else if (nb == 2) k_gram_tc<2><<<grid, 256, kGSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else if (nb == 3) k_gram_tc<3><<<grid, 256, kGSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        else k_gram_tc<4><<<grid, 256, kGSmem, s>>>(c->d_blk, psi, part, off, c->ws.status);
        note_launch(cm);
    }
    if (timed) {
        cudaEventRecord(cm->ov_ev[2 * cm->ov_used + 1], s);
        ++cm->ov_used;
    }
    const dim3 g2((unsigned)((nmax * nmax + 31) / 32), (unsigned)c->nblk);
    k_gram_sum<<<g2, 256, 0, s>>>(c->d_blk, part, off, c->ws.M, gram_launch_pack(c));
    note_launch((flosic_ctx*)c);
}

}  // namespace flosic
