// C ABI of the FLO-SIC step: context, workspace and the four step calls.
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

using namespace flosic;

namespace {
thread_local std::string g_create_error;   // message of this thread's last failed flosic_create

int fail(flosic_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

template <class T>
cudaError_t alloc(flosic_ctx* c, T** p, long long n) {
    *p = nullptr;
    if (n <= 0) n = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)n);
    if (e == cudaSuccess) {
        c->allocations.push_back(q);
        *p = (T*)q;
    }
    return e;
}

void release(flosic_ctx* c) {
    if (c->hs.copy) cudaStreamDestroy(c->hs.copy);
    if (c->hs.copy_out) cudaStreamDestroy(c->hs.copy_out);
    for (cudaEvent_t e : c->hs.copied)
        if (e) cudaEventDestroy(e);
    if (c->hs.done) cudaEventDestroy(c->hs.done);
    c->hs = flosic_ctx::HostStep{};
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    for (cudaEvent_t e : c->ov_ev) cudaEventDestroy(e);
    c->ov_ev.clear();
    for (void* p : c->allocations) cudaFree(p);
    c->allocations.clear();
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    c->h_pinned = nullptr;
    c->h_pinned_dev = nullptr;
}

int validate_options(const flosic_options& o, std::string& why) {
    if (o.precision != FLOSIC_FP64 && o.precision != FLOSIC_MIXED) why = "precision must be FP64 or MIXED";
    else if (!(o.cg_tol > 0.0) || !(o.cg_tol < 1.0)) why = "cg_tol must be in (0, 1)";
    else if (o.max_iter < 1) why = "max_iter must be >= 1";
    else if (o.fod_grad_mode != FLOSIC_GRAD_INTERP && o.fod_grad_mode != FLOSIC_GRAD_PAPER) why = "bad fod_grad_mode";
    else if (o.adjoint_mode != FLOSIC_ADJ_REUSE_V && o.adjoint_mode != FLOSIC_ADJ_EXACT) why = "bad adjoint_mode";
    else if (!(o.rho_min >= 0.0)) why = "rho_min must be >= 0";
    else if (!(o.illcond_tol >= 0.0) || !(o.illcond_tol < 1.0)) why = "illcond_tol must be in [0, 1)";
    else if (o.preconditioner != FLOSIC_PC_NONE && o.preconditioner != FLOSIC_PC_MG) why = "bad preconditioner";
    else if (o.solver != FLOSIC_SOLVER_PCG && o.solver != FLOSIC_SOLVER_AAR && o.solver != FLOSIC_SOLVER_KRON)
        why = "bad solver";
    else if (o.solver != FLOSIC_SOLVER_PCG && o.precision != FLOSIC_MIXED)
        why = "the AAR and KRON solvers require MIXED precision";
    else if (o.boundary != FLOSIC_BC_ISOLATED && o.boundary != FLOSIC_BC_PERIODIC && o.boundary != FLOSIC_BC_SLAB)
        why = "bad boundary";
    else if (o.kron_tensor_cores != 0 && o.kron_tensor_cores != 1) why = "kron_tensor_cores must be 0 or 1";
    else if (o.autotune != 0 && o.autotune != 1) why = "autotune must be 0 or 1";
    else if (o.boundary != FLOSIC_BC_ISOLATED &&
             (o.solver != FLOSIC_SOLVER_KRON || o.adjoint_mode != FLOSIC_ADJ_REUSE_V ||
              o.fod_grad_mode != FLOSIC_GRAD_INTERP))
        why = "PERIODIC and SLAB boundaries require the KRON solver, ADJ_REUSE_V and GRAD_INTERP";
    else if (o.solver == FLOSIC_SOLVER_AAR && (o.aar_m < 1 || o.aar_m > aar_max_m() || o.aar_p < 2 ||
                                               !(o.aar_omega > 0.0 && o.aar_omega < 2.0) ||
                                               !(o.aar_beta > 0.0 && o.aar_beta < 2.0)))
        why = "AAR parameters out of range (1 <= m <= 8, p >= 2, 0 < omega, beta < 2)";
    else return 0;
    return 1;
}

// Tensor maps of the stencil's operands, four per block, each a 4-D view
// (x, y, z, orbital): z with 48 x 28 boxes (tile plus halo), and z, p, q with
// 32 x 16 centre boxes.  Blocks whose rows or offset are not 16-byte aligned
// keep the plain-load stencil (flag tma = 0 in their level-0 descriptor).
// Returns the number of blocks on the copy-engine path.
int setup_tensor_maps(flosic_ctx* c, const void* zbuf, const void* pbuf, const void* qbuf, size_t elem) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return 0;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    std::vector<CUtensorMap> maps(4 * (size_t)c->nblk);
    std::vector<LvlDesc>& L0 = c->mg.h_lvl[0];
    int n_ok = 0;
    for (int b = 0; b < c->nblk; ++b) {
        const BlkDesc& B = c->blk[b];
        L0[b].tma = 0;
        if ((B.nx * elem) % 16 != 0 || (B.off * (long long)elem) % 16 != 0) continue;
        const cuuint64_t dims[4] = {(cuuint64_t)B.nx, (cuuint64_t)B.ny, (cuuint64_t)B.nz, (cuuint64_t)B.N};
        const cuuint64_t strides[3] = {(cuuint64_t)B.nx * elem, (cuuint64_t)B.nx * B.ny * elem,
                                       (cuuint64_t)B.G * elem};
        const cuuint32_t box_halo[4] = {48, (cuuint32_t)(kTileY + 2 * kHalf), 1, 1};
        const cuuint32_t box_ctr[4] = {(cuuint32_t)kTileX, (cuuint32_t)kTileY, 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const void* bufs[4] = {zbuf, zbuf, pbuf, qbuf};
        bool ok = true;
        for (int k = 0; k < 4 && ok; ++k) {
            void* base = (unsigned char*)bufs[k] + B.off * (long long)elem;
            ok = encode(&maps[4 * b + k], elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                        base, dims, strides, k == 0 ? box_halo : box_ctr, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        if (!ok) continue;
        L0[b].tma = 1;
        ++n_ok;
    }
    if (n_ok == 0) return 0;
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(CUtensorMap) * maps.size()) != cudaSuccess) return 0;
    c->allocations.push_back(d);
    if (cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaFuncSetAttribute(apply12_tma_symbol(elem == 4), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)apply12_tma_smem(elem)) != cudaSuccess ||
        cudaMemcpy(c->mg.d_lvl[0], L0.data(), sizeof(LvlDesc) * c->nblk, cudaMemcpyHostToDevice) != cudaSuccess) {
        for (auto& D : L0) D.tma = 0;
        cudaMemcpy(c->mg.d_lvl[0], L0.data(), sizeof(LvlDesc) * c->nblk, cudaMemcpyHostToDevice);
        return 0;
    }
    c->d_tmaps = d;
    return n_ok;
}

// Waits for the stream and returns the device status words.
int read_status(flosic_ctx* c, cudaStream_t s, int* st4) {
    int rc = check_cuda(c, cudaGetLastError(), "kernel launch");
    if (rc) return rc;
    rc = check_cuda(c, fetch_words(c, c->ws.status, 4, s), "status read");
    if (rc) return rc;
    rc = check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) st4[k] = reinterpret_cast<volatile int*>(c->h_pinned)[k];
    prof_collect(c);
    return FLOSIC_OK;
}
}  // namespace

namespace flosic {

__global__ void k_put_words(const int* __restrict__ src, int n, int* dst) {
    if ((int)threadIdx.x < n) reinterpret_cast<volatile int*>(dst)[threadIdx.x] = src[threadIdx.x];
    __threadfence_system();
}

cudaError_t fetch_words(const flosic_ctx* c, const int* src, int n, cudaStream_t s) {
    if (!c->h_pinned_dev) return cudaMemcpyAsync(c->h_pinned, src, sizeof(int) * n, cudaMemcpyDeviceToHost, s);
    k_put_words<<<1, 32, 0, s>>>(src, n, c->h_pinned_dev);
    note_launch(c);
    return cudaGetLastError();
}

__global__ void k_fill_doubles(double* dst, int n, double v) {
    for (int i = threadIdx.x; i < n; i += 32) dst[i] = v;
}

void fill_doubles(const flosic_ctx* c, double* dst, int n, double v, cudaStream_t s) {
    k_fill_doubles<<<1, 32, 0, s>>>(dst, n, v);
    note_launch(c);
}
void prof_collect(flosic_ctx* c) {
    for (int k = 0; k < c->prof_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]) == cudaSuccess) {
            c->prof_ms += ms;
            ++c->prof_launches;
        }
    }
    c->prof_used = 0;
}

void ov_collect(flosic_ctx* c) {
    for (int k = 0; k < c->ov_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ov_ev[2 * k], c->ov_ev[2 * k + 1]) == cudaSuccess) {
            c->ov_ms += ms;
            ++c->ov_launches;
        }
    }
    c->ov_used = 0;
}

void prof_begin(flosic_ctx* c, cudaStream_t s) {
    if (!c->profiling) return;
    if (2 * (c->prof_used + 1) > (int)c->prof_ev.size()) {   // pool full: wait and sum
        cudaEventSynchronize(c->prof_ev[2 * c->prof_used - 1]);
        prof_collect(c);
    }
    cudaEventRecord(c->prof_ev[2 * c->prof_used], s);
}

void prof_end(flosic_ctx* c, cudaStream_t s) {
    if (!c->profiling) return;
    cudaEventRecord(c->prof_ev[2 * c->prof_used + 1], s);
    ++c->prof_used;
}

// The dynamic shared-memory limit is a property of the kernel on a device,
// not of a context: raise it to the largest size any context has needed, and
// never lower it (a later context with smaller blocks must not break the
// launches of an earlier one).
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = granted[std::make_pair(fn, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int check_cuda(flosic_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FLOSIC_OK;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return FLOSIC_ERR_CUDA;
}
}  // namespace flosic

extern "C" {

int flosic_default_options(flosic_options* opt) {
    if (!opt) return FLOSIC_ERR_ARG;
    opt->precision = FLOSIC_MIXED;
    opt->cg_tol = 1e-10;
    opt->max_iter = 20000;
    opt->fod_grad_mode = FLOSIC_GRAD_INTERP;
    opt->adjoint_mode = FLOSIC_ADJ_REUSE_V;
    opt->rho_min = 1e-30;
    opt->illcond_tol = 1e-10;
    opt->preconditioner = FLOSIC_PC_MG;
    opt->solver = FLOSIC_SOLVER_PCG;
    opt->aar_omega = 0.6;
    opt->aar_beta = 0.6;
    opt->aar_m = 7;
    opt->aar_p = 6;
    opt->boundary = FLOSIC_BC_ISOLATED;
    opt->kron_tensor_cores = 1;
    opt->autotune = 1;
    return FLOSIC_OK;
}

const char* flosic_last_error(const flosic_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int flosic_create(flosic_ctx** out, const flosic_system* sys, int nsys, const flosic_options* opt) {
    if (!out) { g_create_error = "ctx pointer is NULL"; return FLOSIC_ERR_ARG; }
    *out = nullptr;
    if (!sys || nsys < 1) { g_create_error = "need at least one system"; return FLOSIC_ERR_ARG; }
    flosic_options o;
    if (opt) o = *opt; else flosic_default_options(&o);
    std::string why;
    if (validate_options(o, why)) { g_create_error = why; return FLOSIC_ERR_ARG; }
    for (int s = 0; s < nsys; ++s) {
        const flosic_system& y = sys[s];
        char buf[160];
        if (y.nx < 1 || y.ny < 1 || y.nz < 1 || !(y.h > 0.0) || !std::isfinite(y.h) ||
            !std::isfinite(y.origin[0]) || !std::isfinite(y.origin[1]) || !std::isfinite(y.origin[2])) {
            snprintf(buf, sizeof buf, "system %d: bad grid", s);
            g_create_error = buf;
            return FLOSIC_ERR_ARG;
        }
        if ((long long)y.nx * y.ny * y.nz > kMaxGridPoints) {   // block-local point indices are 32-bit
            snprintf(buf, sizeof buf, "system %d: more than %lld grid points", s, kMaxGridPoints);
            g_create_error = buf;
            return FLOSIC_ERR_ARG;
        }
        if (y.nspin != 1 && y.nspin != 2) {
            snprintf(buf, sizeof buf, "system %d: nspin must be 1 or 2", s);
            g_create_error = buf;
            return FLOSIC_ERR_ARG;
        }
        for (int sp = 0; sp < y.nspin; ++sp)
            if (y.norb[sp] < 1 || y.norb[sp] > kMaxN) {
                snprintf(buf, sizeof buf, "system %d spin %d: norb must be in [1, %d]", s, sp, kMaxN);
                g_create_error = buf;
                return FLOSIC_ERR_ARG;
            }
        const int per = boundary_mask(o.boundary);
        const int n3[3] = {y.nx, y.ny, y.nz};
        for (int d = 0; d < 3; ++d) {
            if (((per >> d) & 1) && n3[d] < 2 * kHalf + 1) {
                snprintf(buf, sizeof buf, "system %d: periodic sides need >= %d points", s, 2 * kHalf + 1);
                g_create_error = buf;
                return FLOSIC_ERR_ARG;
            }
            if (o.solver == FLOSIC_SOLVER_KRON && n3[d] > kron_max_n()) {
                snprintf(buf, sizeof buf, "system %d: the KRON solver takes sides <= %d", s, kron_max_n());
                g_create_error = buf;
                return FLOSIC_ERR_ARG;
            }
        }
    }
    flosic_ctx* c = new (std::nothrow) flosic_ctx();
    if (!c) { g_create_error = "out of host memory"; return FLOSIC_ERR_ARG; }
    c->opt = o;
    c->sys.assign(sys, sys + nsys);
    // spin blocks, packed offsets, chunk table
    long long off = 0, moff = 0, voff = 0, fod = 0, chunk = 0, soff = 0;
    int orb = 0;
    std::vector<int> sys_orb0(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        const flosic_system& y = sys[s];
        sys_orb0[s] = orb;
        for (int sp = 0; sp < y.nspin; ++sp) {
            BlkDesc b{};
            b.nx = y.nx; b.ny = y.ny; b.nz = y.nz; b.N = y.norb[sp];
            b.h = y.h; b.dV = y.h * y.h * y.h;
            b.ox = y.origin[0]; b.oy = y.origin[1]; b.oz = y.origin[2];
            b.cx = y.origin[0] + 0.5 * y.h * (y.nx - 1);
            b.cy = y.origin[1] + 0.5 * y.h * (y.ny - 1);
            b.cz = y.origin[2] + 0.5 * y.h * (y.nz - 1);
            b.G = (long long)y.nx * y.ny * y.nz;
            b.off = off; b.moff = moff; b.voff = voff; b.fod_off = fod; b.soff = soff;
            b.orb0 = orb; b.sys = s; b.spin = sp;
            b.per = boundary_mask(o.boundary);
            b.nchunk = (int)((b.G + kChunk - 1) / kChunk);
            b.chunk0 = chunk;
            c->blk.push_back(b);
            for (int i = 0; i < b.N; ++i) c->h_orb_blk.push_back((int)c->blk.size() - 1);
            off += b.N * b.G; moff += (long long)b.N * b.N; voff += b.G; fod += b.N;
            chunk += (long long)b.N * b.nchunk; orb += b.N;
        }
        soff += (long long)y.nx * y.ny * y.nz;
    }
    c->sgrid_elems = soff;
    sys_orb0[nsys] = orb;
    c->nblk = (int)c->blk.size();
    c->norb = orb;
    c->orb_elems = off;
    c->vavg_elems = voff;
    c->mat_elems = moff;
    c->nchunk_total = chunk;
    // points within 6 of a non-periodic face, per block (they carry the
    // ghost taps of the Dirichlet values)
    std::vector<int> bidx;
    for (BlkDesc& b : c->blk) {
        b.bnd0 = (long long)bidx.size();
        const bool fx = !(b.per & 1), fy = !(b.per & 2), fz = !(b.per & 4);
        for (int z = 0; z < b.nz; ++z)
            for (int y = 0; y < b.ny; ++y)
                for (int x = 0; x < b.nx; ++x)
                    if ((fx && (x < kHalf || x >= b.nx - kHalf)) || (fy && (y < kHalf || y >= b.ny - kHalf)) ||
                        (fz && (z < kHalf || z >= b.nz - kHalf)))
                        bidx.push_back((z * b.ny + y) * b.nx + x);
        b.nbnd = (int)((long long)bidx.size() - b.bnd0);
    }
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 152;
        cudaGetLastError();   // a failure here surfaces at the first allocation
        c->num_sms = sms;
    }
    int kp = (4 * c->num_sms + c->nblk - 1) / c->nblk;   // one wave of four 256-thread CTAs per SM
    c->kparts = kp < 1 ? 1 : (kp > 1024 ? 1024 : kp);
    std::vector<int> chunk_orb((size_t)chunk);
    for (const BlkDesc& b : c->blk)
        for (int i = 0; i < b.N; ++i)
            for (int k = 0; k < b.nchunk; ++k) chunk_orb[(size_t)(b.chunk0 + (long long)i * b.nchunk + k)] = b.orb0 + i;

    Workspace& w = c->ws;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, long long n) { if (e == cudaSuccess) e = alloc(c, p, n); };
    A(&c->d_blk, c->nblk);
    A(&c->d_orb_blk, c->norb);
    A(&c->d_chunk_orb, chunk);
    A(&c->d_sys_orb0, nsys + 1);
    const long long me = moff;
    w.mat_elems = me;
    A(&w.vals, me); A(&w.grads, 3 * me); A(&w.rho_a, orb); A(&w.T, me); A(&w.M, me);
    A(&w.S, me); A(&w.Q, me); A(&w.C, me); A(&w.U, me); A(&w.lam, orb); A(&w.P, me);
    A(&w.vbar, me); A(&w.tmp, 4 * me); A(&w.E2, 2 * me);
    A(&w.node_idx, 64LL * orb); A(&w.node_wt, 64LL * orb);
    A(&w.mat_part, (long long)c->kparts * me);
    if (o.solver == FLOSIC_SOLVER_AAR) {
        float *fp = nullptr, *X = nullptr, *F = nullptr;
        A(&fp, off); A(&X, (long long)o.aar_m * off); A(&F, (long long)o.aar_m * off);
        w.aar_fprev = fp; w.aar_X = X; w.aar_F = F;
        A(&w.aar_gamma, (long long)orb * aar_max_m());
    }
    std::vector<long long> goff;
    if (o.precision == FLOSIC_MIXED) {
        A(&w.gram_part, gram_tc_part_elems(c, goff));
        A(&w.gram_off, c->nblk);
        if (e == cudaSuccess)
            e = cudaMemcpy(w.gram_off, goff.data(), sizeof(long long) * c->nblk, cudaMemcpyHostToDevice);
    }
    A(&w.mom, 10LL * orb);
    A(&c->d_bidx, (long long)bidx.size()); A(&c->d_bcoef, 10LL * (long long)bidx.size());
    A(&w.e_part, 2 * chunk); A(&w.e_orb, 2LL * orb);
    A(&w.status, 4);
    A(&w.mask, orb);
    A(&w.b64, off); A(&w.r64, off);
    if (o.precision == FLOSIC_FP64) {
        A(&w.p64, off); A(&w.q64, off);
    } else {
        A(&w.d32, off); A(&w.r32, off); A(&w.p32, off); A(&w.q32, off);
    }
    if (o.adjoint_mode == FLOSIC_ADJ_EXACT) A(&w.veff, off);
    if (uses_wbar(c)) A(&w.wbar, off);   // the only per-point adjoint input the mixed path needs
    else A(&w.vsic, off);
    // level 0 (the fine grid) always, coarser multigrid levels when asked for:
    // coarsen each block while every side is >= 6
    Multigrid& M = c->mg;
    {
        const bool want_mg = (o.preconditioner == FLOSIC_PC_MG && o.solver != FLOSIC_SOLVER_KRON);
        std::vector<int> nl(c->nblk);
        std::vector<int> coarsest(c->nblk);
        M.nlev = 0;
        M.coarsest_max = 0;
        for (int b = 0; b < c->nblk; ++b) {
            int d[3] = {c->blk[b].nx, c->blk[b].ny, c->blk[b].nz};
            int L = 1;
            while (want_mg && L < kMaxLevels && d[0] >= 6 && d[1] >= 6 && d[2] >= 6) {
                for (int k = 0; k < 3; ++k) d[k] /= 2;
                ++L;
            }
            nl[b] = L;
            coarsest[b] = L - 1;
            M.nlev = L > M.nlev ? L : M.nlev;
            const long long Gc = (long long)d[0] * d[1] * d[2];
            M.coarsest_max = Gc > M.coarsest_max ? Gc : M.coarsest_max;
        }
        M.enabled = want_mg && M.coarsest_max <= kCoarseMax;
        if (!M.enabled) {
            M.nlev = 1;
            for (int b = 0; b < c->nblk; ++b) { nl[b] = 1; coarsest[b] = 0; }
        }
        const size_t tsz = (o.precision == FLOSIC_FP64) ? sizeof(double) : sizeof(float);
        // last-point diagonal weights per block and dimension, level by level
        std::vector<std::array<double, 3>> cl(c->nblk, std::array<double, 3>{2.0, 2.0, 2.0});
        for (int l = 0; l < M.nlev; ++l) {
            long long offl = 0, chl = 0, tl = 0;
            std::vector<int4> tiles;
            for (int b = 0; b < c->nblk; ++b) {
                const BlkDesc& B = c->blk[b];
                LvlDesc D{};
                D.off = offl;
                D.chunk0 = chl;
                D.tile0 = tl;
                if (l < nl[b]) {
                    D.nx = B.nx >> l; D.ny = B.ny >> l; D.nz = B.nz >> l;
                    D.h = B.h * (double)(1 << l);
                    D.G = (long long)D.nx * D.ny * D.nz;
                    D.nchunk = (int)((D.G + kChunk - 1) / kChunk);
                    D.coarsest = (l == nl[b] - 1) ? 1 : 0;
                    const int sides[3] = {D.nx, D.ny, D.nz};
                    D.corr = 0;
                    for (int k = 0; k < 3; ++k) {
                        D.cl[k] = (float)cl[b][k];
                        D.corr |= (cl[b][k] != 2.0) ? 1 : 0;
                        // the coarse level inherits the Galerkin weight
                        cl[b][k] = (sides[k] % 2 == 0) ? 2.0 * cl[b][k] - 1.0 : 1.0 + 0.5 * cl[b][k];
                    }
                    for (int m = 0; m < 8; ++m) {
                        double dd = 6.0;
                        for (int k = 0; k < 3; ++k)
                            if (m & (1 << k)) dd += (double)D.cl[k] - 2.0;
                        D.idd[m] = (float)(1.0 / dd);
                    }
                    D.tz = (l == 0) ? kTileZ : kTileZc;
                    D.per = (l == 0) ? B.per : 0;
                    const int tx = (D.nx + kTileX - 1) / kTileX, ty = (D.ny + kTileY - 1) / kTileY,
                              tz = (D.nz + D.tz - 1) / D.tz;
                    D.ntile = tx * ty * tz;
                    for (int i = 0; i < B.N; ++i)
                        for (int kz = 0; kz < tz; ++kz)
                            for (int ky = 0; ky < ty; ++ky)
                                for (int kx = 0; kx < tx; ++kx)
                                    tiles.push_back(make_int4(B.orb0 + i, kx * kTileX, ky * kTileY, kz * D.tz));
                    offl += (long long)B.N * D.G;
                    chl += (long long)B.N * D.nchunk;
                    tl += (long long)B.N * D.ntile;
                }
                M.h_lvl[l].push_back(D);
            }
            M.elems[l] = offl;
            M.nchunk[l] = chl;
            M.ntiles[l] = tl;
            A(&M.d_lvl[l], c->nblk);
            if (e == cudaSuccess)
                e = cudaMemcpy(M.d_lvl[l], M.h_lvl[l].data(), sizeof(LvlDesc) * c->nblk, cudaMemcpyHostToDevice);
            A(&M.d_tiles[l], tl);
            if (e == cudaSuccess && tl > 0)
                e = cudaMemcpy(M.d_tiles[l], tiles.data(), sizeof(int4) * tl, cudaMemcpyHostToDevice);
            if (l > 0) {
                unsigned char *pr = nullptr, *pe = nullptr, *pt = nullptr;
                A(&pr, (long long)tsz * offl); A(&pe, (long long)tsz * offl); A(&pt, (long long)tsz * offl);
                M.r[l] = pr; M.e[l] = pe; M.t[l] = pt;
            }
        }
        A(&M.d_coarsest_level, c->nblk);
        if (e == cudaSuccess)
            e = cudaMemcpy(M.d_coarsest_level, coarsest.data(), sizeof(int) * c->nblk, cudaMemcpyHostToDevice);
        if (o.precision == FLOSIC_FP64) {
            if (M.enabled) { A(&w.z64, off); A(&w.p64b, off); }
        } else if (M.enabled || o.solver == FLOSIC_SOLVER_AAR) {
            A(&w.z32, off); A(&w.p32b, off);   // z32: the AAR's f = M r as well
        }
    }
    CgState& g = w.cg;
    A(&g.rr, orb); A(&g.pq, orb); A(&g.bb, orb); A(&g.thr, orb); A(&g.beta, orb); A(&g.rz, orb);
    const long long nparts = chunk > M.ntiles[0] ? chunk : M.ntiles[0];
    if (o.solver == FLOSIC_SOLVER_AAR) A(&w.aar_part, aar_part_elems(M.ntiles[0]));
    A(&w.mom_part, 10 * nparts);
    A(&g.part, nparts); A(&g.part2, nparts); A(&g.count, orb); A(&g.active, orb); A(&g.oactive, orb);
    A(&g.iters, orb); A(&g.n_active, 1); A(&g.n_oactive, 1); A(&g.conv, orb); A(&g.prof_bytes, 1);
    A(&g.dmax, orb); A(&g.xz, orb);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pinned, 16 * sizeof(int));
    if (e == cudaSuccess && cudaHostGetDevicePointer((void**)&c->h_pinned_dev, c->h_pinned, 0) != cudaSuccess) {
        c->h_pinned_dev = nullptr;   // not mapped: status reads take cudaMemcpyAsync
        cudaGetLastError();
    }
    if (e == cudaSuccess && o.solver == FLOSIC_SOLVER_KRON) e = setup_kron(c);   // sets the blocks' kq, kl
    for (BlkDesc& B : c->blk) B.gtma = (o.precision == FLOSIC_MIXED && gram_async_eligible(B)) ? 1 : 0;
    if (e == cudaSuccess) e = cudaMemcpy(c->d_blk, c->blk.data(), sizeof(BlkDesc) * c->nblk, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_orb_blk, c->h_orb_blk.data(), sizeof(int) * c->norb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_chunk_orb, chunk_orb.data(), sizeof(int) * chunk, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_sys_orb0, sys_orb0.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(g.count, 0, sizeof(unsigned) * orb);
    if (e == cudaSuccess) e = cudaMemset(g.dmax, 0, sizeof(unsigned) * orb);
    if (e == cudaSuccess) e = cudaMemset(g.xz, 0, sizeof(int) * orb);
    if (e == cudaSuccess) {   // every orbital computed here until flosic_set_orbital_mask says otherwise
        const std::vector<int> ones((size_t)orb, 1);
        e = cudaMemcpy(w.mask, ones.data(), sizeof(int) * orb, cudaMemcpyHostToDevice);
        g.mask = w.mask;
        c->n_unmasked = (int)orb;
    }
    if (e == cudaSuccess) e = cudaMemset(g.prof_bytes, 0, sizeof(double));
    if (e == cudaSuccess) e = upload_stencil_constants();
    if (e == cudaSuccess) e = upload_boundary_constants();
    if (e == cudaSuccess && !bidx.empty())
        e = cudaMemcpy(c->d_bidx, bidx.data(), sizeof(int) * bidx.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !bidx.empty()) e = setup_boundary(c);
    if (e == cudaSuccess)
        e = ensure_dyn_smem(k_lowdin_symbol(), lowdin_smem(c));
    if (e == cudaSuccess && o.precision == FLOSIC_MIXED) e = setup_gram_tc();
    if (e == cudaSuccess && M.enabled) {
        const bool f32 = (o.precision == FLOSIC_MIXED);
        c->n_tma_blocks = f32 ? setup_tensor_maps(c, w.z32, w.p32, w.q32, 4) : setup_tensor_maps(c, w.z64, w.p64, w.q64, 8);
        cudaGetLastError();   // a refused attribute or entry point only disables the copy-engine path
    }
    if (e == cudaSuccess && o.solver == FLOSIC_SOLVER_KRON) {
        c->n_utma_blocks = setup_update_maps(c);
        cudaGetLastError();   // as above: the update then runs with plain loads
    }
    if (e == cudaSuccess && o.solver == FLOSIC_SOLVER_KRON && o.kron_tensor_cores && o.autotune)
        e = kron_autotune(c);
    if (e != cudaSuccess) {
        g_create_error = std::string("workspace set-up: ") + cudaGetErrorString(e);
        release(c);
        delete c;
        return FLOSIC_ERR_CUDA;
    }
    *out = c;
    return FLOSIC_OK;
}

int flosic_destroy(flosic_ctx* ctx) {
    if (!ctx) return FLOSIC_OK;
    release(ctx);
    delete ctx;
    return FLOSIC_OK;
}

int flosic_layout(const flosic_ctx* c, int64_t* out) {
    if (!c || !out) return FLOSIC_ERR_ARG;
    out[0] = c->norb;
    out[1] = c->orb_elems;
    out[2] = c->vavg_elems;
    out[3] = c->mat_elems;
    out[4] = c->nblk;
    out[5] = (int64_t)c->sys.size();
    return FLOSIC_OK;
}

int flosic_block_paths(const flosic_ctx* c, int* out) {
    if (!c || !out) return FLOSIC_ERR_ARG;
    const std::vector<LvlDesc>& L0 = c->mg.h_lvl[0];
    for (int b = 0; b < c->nblk; ++b) {
        const BlkDesc& B = c->blk[b];
        const bool kron = c->opt.solver == FLOSIC_SOLVER_KRON;
        out[b] = (kron && B.tc ? 1 : 0) | (kron && (int)L0.size() > b && L0[b].utma ? 2 : 0) | (B.gtma ? 4 : 0);
    }
    return FLOSIC_OK;
}

int flosic_build_flos(flosic_ctx* c, const double* psi, const double* fods, double* phi, double* S,
                      double* S_mhalf, void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    if (!psi || !fods || !phi) return fail(c, FLOSIC_ERR_ARG, "psi, fods and phi are required");
    cudaStream_t s = (cudaStream_t)stream;
    c->have_forward = false;
    c->have_energy = false;
    int rc = check_cuda(c, cudaMemsetAsync(c->ws.status, 0, 4 * sizeof(int), s), "memset status");
    if (rc) return rc;
    launch_interp_fod(c, psi, fods, s);
    launch_gram(c, psi, s);
    launch_lowdin(c, S, S_mhalf, s);
    launch_flo_apply(c, psi, phi, s);
    int st[4];
    rc = read_status(c, s, st);
    if (rc) return rc;
    if (st[0]) return fail(c, FLOSIC_ERR_NONFINITE, "non-finite value in psi or at a FOD");
    if (st[2]) return fail(c, FLOSIC_ERR_ILLCOND, "Fermi-orbital overlap is near singular (FODs too close?)");
    c->have_forward = true;
    return FLOSIC_OK;
}

int flosic_orbital_poisson(flosic_ctx* c, const double* phi, double* V, int warm_start, int* iters,
                           int* conv_flags, void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    if (!phi || !V) return fail(c, FLOSIC_ERR_ARG, "phi and V are required");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_cuda(c, cudaMemsetAsync(c->ws.status, 0, 4 * sizeof(int), s), "memset status");
    if (rc) return rc;
    launch_rhs(c, phi, true, c->ws.b64, s);
    rc = run_poisson(c, c->ws.b64, V, warm_start != 0, s);
    if (rc) return rc;
    finish_poisson(c, iters, conv_flags, s);
    int st[4];
    rc = read_status(c, s, st);
    if (rc) return rc;
    if (st[3])
        return fail(c, FLOSIC_ERR_CUDA,
                    "a bulk copy or a tensor-core completion of the Poisson kernels did not arrive (bounded wait expired)");
    if (st[1]) return fail(c, FLOSIC_ERR_NOCONV, "a Poisson solve reached max_iter");
    return FLOSIC_OK;
}

int flosic_sic_energy_potential(flosic_ctx* c, const double* psi, const double* phi, const double* V,
                                double scale, double* U, double* Exc, double* E_sic, double* V_avg,
                                void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    if (!psi || !phi || !V) return fail(c, FLOSIC_ERR_ARG, "psi, phi and V are required");
    if (!std::isfinite(scale)) return fail(c, FLOSIC_ERR_ARG, "scale must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    launch_xc_energy(c, psi, phi, V, scale, V_avg, s);
    launch_energy_reduce(c, U, Exc, E_sic, s);
    c->have_energy = true;
    return check_cuda(c, cudaGetLastError(), "energy kernels");
}

int flosic_set_orbital_mask(flosic_ctx* c, const int* mask) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    std::vector<int> m((size_t)c->norb, 1);
    int on = c->norb;
    if (mask) {
        on = 0;
        for (int o = 0; o < c->norb; ++o) {
            if (mask[o] != 0 && mask[o] != 1) return fail(c, FLOSIC_ERR_ARG, "mask entries must be 0 or 1");
            m[(size_t)o] = mask[o];
            on += mask[o];
        }
        if (on < c->norb && c->opt.adjoint_mode == FLOSIC_ADJ_EXACT)
            return fail(c, FLOSIC_ERR_ARG, "an orbital mask requires ADJ_REUSE_V");
    }
    int rc = check_cuda(c, cudaMemcpy(c->ws.mask, m.data(), sizeof(int) * c->norb, cudaMemcpyHostToDevice),
                        "cudaMemcpy(mask)");
    if (rc) return rc;
    c->n_unmasked = on;
    c->have_energy = false;   // the cached V^SIC belongs to the previous mask
    return FLOSIC_OK;
}

int flosic_hamiltonian_apply(flosic_ctx* c, const double* psi, const double* vloc, const double* V_avg,
                             double* Hpsi, void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    if (!psi || !Hpsi) return fail(c, FLOSIC_ERR_ARG, "psi and Hpsi are required");
    if (Hpsi == psi) return fail(c, FLOSIC_ERR_ARG, "Hpsi must not overlap psi");
    launch_hamiltonian(c, psi, vloc, V_avg, Hpsi, (cudaStream_t)stream);
    return check_cuda(c, cudaGetLastError(), "hamiltonian kernel");
}

int flosic_sic_backward(flosic_ctx* c, const double* psi, const double* fods, const double* phi,
                        const double* V, const double* gE, double* dE_dpsi, double* dE_dfod,
                        void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    c->hs.fwd_valid = false;   // the workspace changes: a started next step is void
    if (!psi || !fods || !phi || !V || !gE) return fail(c, FLOSIC_ERR_ARG, "psi, fods, phi, V, gE are required");
    if (!c->have_forward) return fail(c, FLOSIC_ERR_ARG, "no forward step recorded on this context");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_energy) launch_xc_energy(c, psi, phi, V, 1.0, nullptr, s);   // V^SIC only
    const double* Vsrc = c->ws.vsic;   // null on the mixed path with V reused: wbar holds V^SIC phi
    if (c->opt.adjoint_mode == FLOSIC_ADJ_EXACT) {
        int rc = check_cuda(c, cudaMemsetAsync(c->ws.status, 0, 4 * sizeof(int), s), "memset status");
        if (rc) return rc;
        launch_rhs(c, phi, false, c->ws.b64, s);                 // A W = rho (zero boundary)
        rc = run_poisson(c, c->ws.b64, c->ws.veff, false, s);
        if (rc) return rc;
        finish_poisson(c, nullptr, nullptr, s);
        launch_bc_adjoint(c, c->ws.veff, V, c->ws.veff, s);    // V^SIC of veff = (V + G^T rho)/2
        Vsrc = c->ws.veff;
    }
    launch_backward_contract(c, psi, phi, Vsrc, gE, s);
    launch_backward_small(c, dE_dfod, s);
    if (dE_dpsi) launch_psibar(c, psi, phi, Vsrc, gE, fods, dE_dpsi, s);
    if (c->opt.adjoint_mode == FLOSIC_ADJ_EXACT) {
        int st[4];
        int rc = read_status(c, s, st);
        if (rc) return rc;
        if (st[1]) return fail(c, FLOSIC_ERR_NOCONV, "adjoint Poisson solve reached max_iter");
        return FLOSIC_OK;
    }
    return check_cuda(c, cudaGetLastError(), "backward kernels");
}

int flosic_step_host(flosic_ctx* c, const double* psi_h, const double* fods_h, double scale, double gE,
                     double* E_sic, double* U, double* Exc, double* V_avg, double* dE_dpsi, double* dE_dfod,
                     int* conv_flags, const double* psi_next, const double* fods_next, void* stream) {
    if (!c) return FLOSIC_ERR_ARG;
    if (!psi_h || !fods_h) return fail(c, FLOSIC_ERR_ARG, "psi and fods are required");
    if ((psi_next == nullptr) != (fods_next == nullptr))
        return fail(c, FLOSIC_ERR_ARG, "psi_next and fods_next go together");
    if (!std::isfinite(scale) || !std::isfinite(gE)) return fail(c, FLOSIC_ERR_ARG, "scale and gE must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    auto& H = c->hs;
    const long long orb = c->orb_elems, nf = 3LL * c->norb;
    if (!H.ready) {
        cudaError_t e = cudaSuccess;
        auto A = [&](auto** p, long long n) { if (e == cudaSuccess) e = alloc(c, p, n); };
        A(&H.psi[0], orb); A(&H.psi[1], orb); A(&H.fods[0], nf); A(&H.fods[1], nf);
        A(&H.phi, orb); A(&H.V, orb); A(&H.Vavg, c->vavg_elems); A(&H.dpsi, orb); A(&H.dfod, nf);
        A(&H.E, (long long)c->sys.size()); A(&H.U, c->norb); A(&H.Exc, c->norb); A(&H.gE, (long long)c->sys.size());
        A(&H.conv[0], c->norb); A(&H.conv[1], c->norb);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H.copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H.copy_out, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&H.copied[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return check_cuda(c, e, "host-step buffers");
        H.ready = true;
    }
    const size_t bpsi = sizeof(double) * (size_t)orb, bfod = sizeof(double) * (size_t)nf;
    int rc;
    // this step's inputs: already on the device when the previous call prefetched
    // them, and its FLO build and Poisson solve already done when that call
    // started them (same host arrays, nothing else run on the context since)
    int cur;
    const bool prefetched = H.pre >= 0 && H.pre_psi == psi_h && H.pre_fods == fods_h;
    const bool have_fwd = prefetched && H.fwd_valid && H.fwd_psi == psi_h && H.fwd_fods == fods_h;
    H.fwd_valid = false;
    if (prefetched) {
        cur = H.pre;
        rc = check_cuda(c, cudaStreamWaitEvent(s, H.copied[cur], 0), "cudaStreamWaitEvent");
        if (rc) return rc;
    } else {
        cur = (H.pre >= 0) ? 1 - H.pre : 0;
        rc = check_cuda(c, cudaMemcpyAsync(H.psi[cur], psi_h, bpsi, cudaMemcpyHostToDevice, s), "copy psi");
        if (!rc) rc = check_cuda(c, cudaMemcpyAsync(H.fods[cur], fods_h, bfod, cudaMemcpyHostToDevice, s), "copy fods");
        if (rc) return rc;
    }
    H.pre = -1;
    // the next step's inputs, copied on the copy stream while this step computes
    const int nxt = 1 - cur;
    if (psi_next) {
        rc = check_cuda(c, cudaMemcpyAsync(H.psi[nxt], psi_next, bpsi, cudaMemcpyHostToDevice, H.copy), "prefetch psi");
        if (!rc)
            rc = check_cuda(c, cudaMemcpyAsync(H.fods[nxt], fods_next, bfod, cudaMemcpyHostToDevice, H.copy),
                            "prefetch fods");
        if (!rc) rc = check_cuda(c, cudaEventRecord(H.copied[nxt], H.copy), "cudaEventRecord");
        if (rc) return rc;
        H.pre = nxt;
        H.pre_psi = psi_next;
        H.pre_fods = fods_next;
    }
    const int nsys = (int)c->sys.size();
    // gE for every system by a kernel (a host copy could queue behind the
    // prefetch on the copy engine)
    fill_doubles(c, H.gE, nsys, gE, s);
    rc = check_cuda(c, cudaGetLastError(), "gE fill");
    if (rc) return rc;
    int prc, ci;
    if (have_fwd) {
        prc = H.fwd_rc;
        ci = H.fwd_conv;
    } else {
        ci = 0;
        rc = flosic_build_flos(c, H.psi[cur], H.fods[cur], H.phi, nullptr, nullptr, s);
        if (rc) return rc;
        rc = flosic_orbital_poisson(c, H.phi, H.V, 0, nullptr, H.conv[ci], s);
        if (rc && rc != FLOSIC_ERR_NOCONV) return rc;
        prc = rc;
    }
    rc = flosic_sic_energy_potential(c, H.psi[cur], H.phi, H.V, scale, H.U, H.Exc, H.E, H.Vavg, s);
    if (rc) return rc;
    rc = flosic_sic_backward(c, H.psi[cur], H.fods[cur], H.phi, H.V, H.gE, dE_dpsi ? H.dpsi : nullptr,
                             dE_dfod ? H.dfod : nullptr, s);
    if (rc) return rc;
    // the outputs go to the host on their own stream, once the next step's
    // inputs have arrived (the next FLO build waits for those; the outputs
    // have the whole next forward step to travel) ...
    rc = check_cuda(c, cudaEventRecord(H.done, s), "cudaEventRecord");
    if (!rc) rc = check_cuda(c, cudaStreamWaitEvent(H.copy_out, H.done, 0), "cudaStreamWaitEvent");
    if (!rc && psi_next) rc = check_cuda(c, cudaStreamWaitEvent(H.copy_out, H.copied[nxt], 0), "cudaStreamWaitEvent");
    if (rc) return rc;
    struct Out { void* h; const void* d; size_t n; };
    const Out outs[] = {{E_sic, H.E, sizeof(double) * nsys}, {U, H.U, sizeof(double) * c->norb},
                        {Exc, H.Exc, sizeof(double) * c->norb}, {V_avg, H.Vavg, sizeof(double) * c->vavg_elems},
                        {dE_dfod, H.dfod, bfod}, {conv_flags, H.conv[ci], sizeof(int) * c->norb},
                        {dE_dpsi, H.dpsi, bpsi}};
    for (const Out& o : outs)
        if (o.h && !rc) rc = check_cuda(c, cudaMemcpyAsync(o.h, o.d, o.n, cudaMemcpyDeviceToHost, H.copy_out), "copy out");
    if (rc) return rc;
    // ... while the compute stream starts the next step's FLO build and Poisson
    // solve on its prefetched inputs (they read neither this step's outputs nor
    // its input set, and write the other convergence-flag set)
    if (psi_next) {
        rc = check_cuda(c, cudaStreamWaitEvent(s, H.copied[nxt], 0), "cudaStreamWaitEvent");
        if (rc) return rc;
        int frc = flosic_build_flos(c, H.psi[nxt], H.fods[nxt], H.phi, nullptr, nullptr, s);
        if (!frc) frc = flosic_orbital_poisson(c, H.phi, H.V, 0, nullptr, H.conv[1 - ci], s);
        if (frc == FLOSIC_ERR_CUDA) return frc;
        if (!frc || frc == FLOSIC_ERR_NOCONV) {   // otherwise the next call repeats it and reports
            H.fwd_valid = true;
            H.fwd_psi = psi_next;
            H.fwd_fods = fods_next;
            H.fwd_rc = frc;
            H.fwd_conv = 1 - ci;
        }
    }
    rc = check_cuda(c, cudaStreamSynchronize(H.copy_out), "cudaStreamSynchronize");
    return rc ? rc : prc;
}

int flosic_profile(flosic_ctx* c, int enable) {
    if (!c) return FLOSIC_ERR_ARG;
    if (enable && c->prof_ev.empty()) {
        // both pools or neither: a partial pool is destroyed again
        auto make = [&](std::vector<cudaEvent_t>& pool, int n) {
            for (int k = 0; k < n; ++k) {
                cudaEvent_t e = nullptr;
                int rc = check_cuda(c, cudaEventCreate(&e), "cudaEventCreate");
                if (rc) return rc;
                pool.push_back(e);
            }
            return (int)FLOSIC_OK;
        };
        int rc = make(c->prof_ev, 2 * 1024);
        if (!rc) rc = make(c->ov_ev, 2 * 64);
        if (rc) {
            for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
            for (cudaEvent_t e : c->ov_ev) cudaEventDestroy(e);
            c->prof_ev.clear();
            c->ov_ev.clear();
            return rc;
        }
    }
    c->profiling = enable != 0;
    return FLOSIC_OK;
}

int flosic_profile_read(flosic_ctx* c, double* out, int reset) {
    if (!c || !out) return FLOSIC_ERR_ARG;
    if (c->prof_used > 0) {
        int rc = check_cuda(c, cudaEventSynchronize(c->prof_ev[2 * c->prof_used - 1]), "cudaEventSynchronize");
        if (rc) return rc;
        prof_collect(c);
    }
    double bytes = 0.0;
    int rc = check_cuda(c, cudaMemcpy(&bytes, c->ws.cg.prof_bytes, sizeof(double), cudaMemcpyDeviceToHost),
                        "cudaMemcpy(prof_bytes)");
    if (rc) return rc;
    out[0] = c->prof_ms;
    out[1] = (double)c->prof_launches;
    out[2] = (double)c->launches;
    out[3] = bytes;
    if (reset) {
        c->prof_ms = 0.0;
        c->prof_launches = 0;
        c->launches = 0;
        rc = check_cuda(c, cudaMemset(c->ws.cg.prof_bytes, 0, sizeof(double)), "cudaMemset(prof_bytes)");
        if (rc) return rc;
    }
    return FLOSIC_OK;
}

int flosic_profile_read_overlap(flosic_ctx* c, double* out, int reset) {
    if (!c || !out) return FLOSIC_ERR_ARG;
    if (c->ov_used > 0) {
        int rc = check_cuda(c, cudaEventSynchronize(c->ov_ev[2 * c->ov_used - 1]), "cudaEventSynchronize");
        if (rc) return rc;
        ov_collect(c);
    }
    out[0] = c->ov_ms;
    out[1] = (double)c->ov_launches;
    out[2] = c->ov_flops;
    if (reset) {
        c->ov_ms = 0.0;
        c->ov_launches = 0;
        c->ov_flops = 0.0;
    }
    return FLOSIC_OK;
}

}  // extern "C"
