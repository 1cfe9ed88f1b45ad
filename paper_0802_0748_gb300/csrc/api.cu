// C ABI of the shifted-COCG library (declared in include/scocg.h): handle
// life cycle, argument checks, workspace management and the solve driver
// that launches the persistent kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "api_internal.h"

using namespace scocg;

// ---------------------------------------------------------------- helpers
namespace scocg {

unsigned long long next_generation() {
    static std::atomic<unsigned long long> g{1};
    return g.fetch_add(1);
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SCOCG_OK;
    if (e == cudaErrorMemoryAllocation) return SCOCG_ERR_OOM;
    return SCOCG_ERR_CUDA;
}

void* Workspace::get(size_t bytes) {
    const size_t need = off + ((bytes + 255) / 256) * 256;
    if (need > cap) return nullptr;
    void* p = static_cast<char*>(base) + off;
    off = need;
    return p;
}

cudaError_t Workspace::reserve(size_t bytes) {
    off = 0;
    if (bytes <= cap) return cudaSuccess;
    if (base) cudaFree(base);
    base = nullptr; cap = 0;
    if (gen) *gen = next_generation();
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) { base = nullptr; return e; }
    cap = bytes;
    return cudaSuccess;
}

cudaError_t Workspace::reserve_keep(size_t bytes, size_t keep, cudaStream_t s) {
    off = 0;
    if (bytes <= cap) return cudaSuccess;
    void* nb = nullptr;
    cudaError_t e = cudaMalloc(&nb, bytes);
    if (e != cudaSuccess) return e;
    if (base && keep > 0) e = cudaMemcpyAsync(nb, base, std::min(keep, cap), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaFree(nb); return e; }
    if (base) cudaFree(base);
    if (gen) *gen = next_generation();
    base = nb;
    cap = bytes;
    return cudaSuccess;
}

void Workspace::release() {
    if (base) cudaFree(base);
    base = nullptr; cap = 0; off = 0;
}

void fill_opts(scocg_opts& o, const scocg_opts* in) {
    std::memset(&o, 0, sizeof(o));
    if (in) o = *in;
    if (o.max_iter <= 0) o.max_iter = 100000;
    if (o.replace_every < 0) o.replace_every = 0;
    if (o.timeout_ms <= 0) o.timeout_ms = 10000.0;
    if (o.precision != SCOCG_FP64 && o.precision != SCOCG_MIXED && o.precision != SCOCG_MIXED_DF) o.precision = -1;
    if (o.layout != 0 && o.layout != 1) o.precision = -1;
    if (o.rhs_tile != 0 && o.rhs_tile != 1 && o.rhs_tile != 8 && o.rhs_tile != 16 && o.rhs_tile != 32)
        o.precision = -1;
}

// The seed rule (the method leaves the choice open): smallest Im z, then Re z
// nearest the median of Re z, then the lowest index.
int default_seed(const scocg_c128* z, int K) {
    std::vector<double> re(K);
    for (int k = 0; k < K; ++k) re[k] = z[k].re;
    std::sort(re.begin(), re.end());
    const double med = (K % 2) ? re[K / 2] : 0.5 * (re[K / 2 - 1] + re[K / 2]);
    int best = 0;
    for (int k = 1; k < K; ++k) {
        if (z[k].im < z[best].im) { best = k; continue; }
        if (z[k].im == z[best].im && std::fabs(z[k].re - med) < std::fabs(z[best].re - med)) best = k;
    }
    return best;
}

}  // namespace scocg

extern "C" const char* scocg_strerror(int code) {
    switch (code) {
        case SCOCG_OK: return "ok";
        case SCOCG_NOT_CONVERGED: return "not converged within max_iter (outputs valid)";
        case SCOCG_ERR_INVALID: return "invalid argument";
        case SCOCG_ERR_CUDA: return "CUDA runtime error";
        case SCOCG_ERR_OOM: return "device out of memory";
        case SCOCG_ERR_BREAKDOWN: return "COCG breakdown (zero or non-finite r^T r, r^T A p or pi)";
        case SCOCG_ERR_TIMEOUT: return "device barrier timed out";
        case SCOCG_ERR_UNSYMMETRIC: return "matrix is not symmetric";
        case SCOCG_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the no-allocation solve";
    }
    return "unknown status";
}

// ---------------------------------------------------------------- create / destroy
int scocg::init_ctx(scocg_ctx* h, const scocg_opts* opts, void* stream) {
    fill_opts(h->opts, opts);
    if (h->opts.precision < 0) return SCOCG_ERR_INVALID;
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (e != cudaSuccess) return cuda_status(e);
    if (!coop) return SCOCG_ERR_CUDA;
    e = cudaMalloc(&h->d_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) return cuda_status(e);
    h->ws_gen = next_generation();
    h->ws.gen = &h->ws_gen;
    return SCOCG_OK;
}

void scocg_ctx::free_all() {
    void* ptrs[] = {d_rowptr, d_col, d_val64, d_val32, d_unit_off, d_bcol, d_bval64, d_bval32, d_bval32c, d_ctrl,
                    hub.d_states, hub.d_hop_target, hub.d_hop_sign, hub.d_hop_packed, hub.d_hop2, hub.d_orb2,
                    hub.d_nib2, hub.d_self2, hub.d_self2f, hub.d_amp2, hub.d_amp2f, hub.d_cross2, hub.d_cross2f,
                    hub.d_bonds2, hub.d_diagf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ws.release();
}

extern "C" void scocg_destroy(scocg_handle h) {
    if (!h) return;
    multi_forget(h);
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    h->free_all();
    delete h;
}

extern "C" int scocg_dim(scocg_handle h, int64_t* n) {
    if (!h || !n) return SCOCG_ERR_INVALID;
    *n = h->n;
    return SCOCG_OK;
}

extern "C" int scocg_set_opts(scocg_handle h, const scocg_opts* opts) {
    if (!h) return SCOCG_ERR_INVALID;
    scocg_opts o;
    fill_opts(o, opts);
    if (o.precision < 0) return SCOCG_ERR_INVALID;
    h->opts = o;
    return SCOCG_OK;
}

extern "C" int scocg_create_csr(scocg_handle* out, int64_t n, int64_t nnz, const int64_t* rowptr,
                                const int32_t* col, const double* val, int ptr_on_device,
                                const scocg_opts* opts, void* cuda_stream) {
    if (!out) return SCOCG_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31) || nnz < 0 || nnz >= (int64_t(1) << 31) || !rowptr ||
        (nnz > 0 && (!col || !val)))
        return SCOCG_ERR_INVALID;
    scocg_ctx* h = new (std::nothrow) scocg_ctx();
    if (!h) return SCOCG_ERR_OOM;
    int st = init_ctx(h, opts, cuda_stream);
    if (st != SCOCG_OK) { h->free_all(); delete h; return st; }
    h->kind = HandleKind::kCsr;
    h->n = n;
    h->nnz = nnz;
    cudaStream_t s = h->stream;

    // device copies of the caller's arrays when they are host memory
    const int64_t* d_rp = rowptr;
    const int32_t* d_c = col;
    const double* d_v = val;
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t nnz_a = (size_t)std::max<int64_t>(nnz, 1);
    if (!ptr_on_device) {
        const size_t bytes = 256 * 4 + sizeof(int64_t) * (n + 1) + (sizeof(int32_t) + sizeof(double)) * nnz_a;
        e = cudaMalloc(&tmp, bytes);
        if (e == cudaSuccess) {
            char* p = static_cast<char*>(tmp);
            int64_t* rp = reinterpret_cast<int64_t*>(p);
            p += ((sizeof(int64_t) * (n + 1) + 255) / 256) * 256;
            double* vv = reinterpret_cast<double*>(p);
            p += ((sizeof(double) * nnz_a + 255) / 256) * 256;
            int32_t* cc = reinterpret_cast<int32_t*>(p);
            e = cudaMemcpyAsync(rp, rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(cc, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(vv, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s);
            d_rp = rp; d_c = cc; d_v = vv;
        }
    }
    unsigned* d_flags = nullptr;
    unsigned flags = 0;
    if (e == cudaSuccess) e = cudaMalloc(&d_flags, sizeof(unsigned));
    if (e == cudaSuccess) e = validate_csr(n, nnz, d_rp, d_c, d_v, d_flags, &flags, s);
    if (e == cudaSuccess) {
        if (flags & (kFlagBadPtr | kFlagBadCol | kFlagBadVal)) st = SCOCG_ERR_INVALID;
        else if (flags & kFlagUnsym) st = SCOCG_ERR_UNSYMMETRIC;
    } else {
        st = cuda_status(e);
    }
    h->fp32_exact = !(flags & kFlagNotFp32);
    // int32 CSR with FP64 and FP32 values
    if (st == SCOCG_OK) {
        e = cudaMalloc(&h->d_rowptr, sizeof(int) * (n + 1));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_col, sizeof(int) * nnz_a);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_val64, sizeof(double) * nnz_a);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_val32, sizeof(float) * nnz_a);
        if (e == cudaSuccess)
            e = convert_csr32(n, nnz, d_rp, d_c, d_v, h->d_rowptr, h->d_col, h->d_val64, h->d_val32, s);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    // 4x4-blocked sliced ELL when the pattern allows it
    h->bsr_ok = st == SCOCG_OK && !(flags & kFlagNotBsr4) && nnz > 0;
    if (h->bsr_ok) {
        std::vector<int64_t> rp(n + 1);
        e = cudaMemcpyAsync(rp.data(), d_rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        const int64_t nbr = n / 4, nunits = (nbr + 7) / 8;
        std::vector<int> uoff(nunits + 1, 0);
        if (e == cudaSuccess) {
            int64_t slots = 0;
            for (int64_t u = 0; u < nunits; ++u) {
                int64_t mx = 0;
                for (int64_t B = u * 8; B < std::min<int64_t>(nbr, u * 8 + 8); ++B)
                    mx = std::max<int64_t>(mx, (rp[4 * B + 1] - rp[4 * B]) / 4);
                uoff[u] = (int)slots;
                slots += mx;
            }
            uoff[nunits] = (int)slots;
            h->nunits_bsr = nunits;
            h->nslots = slots;
            e = cudaMalloc(&h->d_unit_off, sizeof(int) * (nunits + 1));
            if (e == cudaSuccess) e = cudaMalloc(&h->d_bcol, sizeof(int) * 8 * std::max<int64_t>(slots, 1));
            if (e == cudaSuccess) e = cudaMalloc(&h->d_bval64, sizeof(double) * 128 * std::max<int64_t>(slots, 1));
            if (e == cudaSuccess) e = cudaMalloc(&h->d_bval32, sizeof(float) * 128 * std::max<int64_t>(slots, 1));
            if (e == cudaSuccess) e = cudaMalloc(&h->d_bval32c, sizeof(float) * 128 * std::max<int64_t>(slots, 1));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->d_unit_off, uoff.data(), sizeof(int) * (nunits + 1), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = convert_bsr4(n, nunits, d_rp, d_c, d_v, h->d_unit_off, h->d_bcol, h->d_bval64, h->d_bval32,
                                 h->d_bval32c, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) st = cuda_status(e);
    }
    if (st == SCOCG_OK) {
        const double avg = (double)nnz / (double)n;
        h->csr_kind = avg <= 4.0 ? LayoutKind::kCsr1 : (avg <= 24.0 ? LayoutKind::kCsr4 : LayoutKind::kCsr16);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    if (d_flags) cudaFree(d_flags);
    if (tmp) { cudaStreamSynchronize(s); cudaFree(tmp); }
    if (st != SCOCG_OK) { h->free_all(); delete h; return st; }
    *out = h;
    return SCOCG_OK;
}

Layout scocg_ctx::layout(bool prefer_csr) const {
    Layout L{};
    prefer_csr = prefer_csr || opts.layout == 1;
    L.kind = (bsr_ok && !prefer_csr) ? LayoutKind::kBsr4 : csr_kind;
    if (force_kind >= 0) L.kind = static_cast<LayoutKind>(force_kind);
    if (L.kind == LayoutKind::kBsr4 && !bsr_ok) L.kind = csr_kind;
    L.n = n; L.nnz = nnz;
    L.rowptr = d_rowptr; L.col = d_col; L.val64 = d_val64; L.val32 = d_val32;
    L.nunits_bsr = nunits_bsr; L.nslots = nslots;
    L.unit_off = d_unit_off; L.bcol = d_bcol; L.bval64 = d_bval64; L.bval32 = d_bval32; L.bval32c = d_bval32c;
    return L;
}

// ---------------------------------------------------------------- apply
extern "C" int scocg_apply(scocg_handle h, scocg_c128 z, const void* x, void* y, int precision) {
    if (!h || !x || !y || (precision != SCOCG_FP64 && precision != SCOCG_MIXED && precision != SCOCG_MIXED_DF))
        return SCOCG_ERR_INVALID;
    cudaError_t e;
    if (h->kind == HandleKind::kHubbard) {
        e = hubbard_apply(h->hub, precision, c2(z.re, z.im), x, y, h->stream);
    } else {
        e = launch_apply(h->layout(false), precision, c2(z.re, z.im), x, y, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

// ---------------------------------------------------------------- solve
namespace scocg {

#ifdef SCOCG_CHECKED
static int* g_trace = nullptr;   // host-mapped flight recorder of the checked build
static int g_trace_n = 0;
#endif

template <typename R>
static int solve_one_rhs(scocg_ctx* h, const double2* d_z, int K, int seed, const double2* b,
                         const int64_t* d_cidx, const void* cvec, int M, double tol, double2* G,
                         int grid, ShiftState S, double* partA, double* partB, double* partC, int strideB,
                         typename Vec<R>::T* r, typename Vec<R>::T* q, typename Vec<R>::T* pseed,
                         typename Vec<R>::T* xhi, typename Vec<R>::T* xlo, double2* xd, const Layout& L,
                         ResumeState* rstate, int resume, double2* Xf = nullptr, double2* Pf = nullptr) {
    SolveArgs<R> a{};
    a.Xf = Xf;
    a.Pf = Pf;
    a.rstate = rstate;
    a.resume = resume;
    a.n = h->n;
    a.rows_per_unit = h->kind == HandleKind::kHubbard ? 32 : rows_per_unit(L.kind);
    a.nunits = h->kind == HandleKind::kHubbard ? h->hub.nunits : (h->n + a.rows_per_unit - 1) / a.rows_per_unit;
    a.r = r; a.q = q; a.b = b;
    a.cvec = static_cast<const typename Vec<R>::T*>(cvec);
    a.cidx = d_cidx;
    a.nproj = M;
    a.p_seed = pseed; a.x_hi = xhi; a.x_lo = xlo; a.xd = xd;
    a.replace_every = h->opts.replace_every;
    a.K = K; a.z = d_z; a.seed = seed;
    a.allow_switch = !h->opts.no_switch;
    a.tol = tol;
    a.max_iter = h->opts.max_iter;
    a.S = S;
    a.partA = partA; a.partB = partB; a.partC = partC; a.strideB = strideB;
    a.sync.count = &h->d_ctrl->count;
    a.sync.status = &h->d_ctrl->status;
    a.sync.timeout_ns = (uint64_t)(h->opts.timeout_ms * 1e6);
    a.sync.nctas = grid;
    a.stats = &h->d_ctrl->stats;
    a.G = G;
    a.debug_inject = h->opts.debug_inject;
    a.dbg = h->d_ctrl->dbg;
    a.trace = nullptr;
    a.phase_ns = nullptr;
#ifdef SCOCG_PHASE_TIMERS
    // phase timers: [grid][8] ns in host-mapped memory, summed over CTAs and printed
    static unsigned long long* h_ns = nullptr;
    static int h_ns_n = 0;
    if (h_ns_n < grid) {
        if (h_ns) cudaFreeHost(h_ns);
        h_ns = nullptr; h_ns_n = 0;
        if (cudaHostAlloc((void**)&h_ns, sizeof(unsigned long long) * 8 * grid, cudaHostAllocMapped) == cudaSuccess)
            h_ns_n = grid;
    }
    if (h_ns) {
        std::memset(h_ns, 0, sizeof(unsigned long long) * 8 * grid);
        cudaHostGetDevicePointer((void**)&a.phase_ns, h_ns, 0);
    }
#endif
#ifdef SCOCG_CHECKED
    // flight recorder: per CTA (iteration, phase) in host-mapped memory, printed
    // after the solve whatever its outcome
    if (g_trace_n < grid) {
        if (g_trace) cudaFreeHost(g_trace);
        g_trace = nullptr;
        g_trace_n = 0;
        if (cudaHostAlloc((void**)&g_trace, sizeof(int) * 2 * grid, cudaHostAllocMapped) == cudaSuccess)
            g_trace_n = grid;
    }
    if (g_trace) {
        for (int i = 0; i < 2 * grid; ++i) g_trace[i] = -1;
        int* d_trace = nullptr;
        if (cudaHostGetDevicePointer((void**)&d_trace, g_trace, 0) == cudaSuccess) a.trace = d_trace;
    }
#endif
    cudaError_t e = cudaMemsetAsync(h->d_ctrl, 0, sizeof(Ctrl), h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (h->kind == HandleKind::kHubbard) e = hubbard_launch_solve(a, h->hub, grid, h->stream);
    else e = launch_solve<R>(a, L, grid, h->stream);
#ifdef SCOCG_PHASE_TIMERS
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (h_ns) {
        double tot[8] = {0};
        for (int c = 0; c < grid; ++c)
            for (int k = 0; k < 8; ++k) tot[k] += (double)((volatile unsigned long long*)h_ns)[8 * c + k];
        std::fprintf(stderr,
                     "scocg phase ms (CTA average): A %.3f bar1 %.3f red1 %.3f B %.3f bar2 %.3f red2 %.3f C %.3f "
                     "tail %.3f\n",
                     tot[0] / grid * 1e-6, tot[1] / grid * 1e-6, tot[6] / grid * 1e-6, tot[2] / grid * 1e-6,
                     tot[3] / grid * 1e-6, tot[5] / grid * 1e-6, tot[4] / grid * 1e-6, tot[7] / grid * 1e-6);
    }
#endif
#ifdef SCOCG_CHECKED
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (a.trace) {
        std::fprintf(stderr, "scocg trace (%s):", cudaGetErrorString(e));
        for (int c = 0; c < grid && c < 16; ++c)
            std::fprintf(stderr, " [%d:%d]", ((volatile int*)g_trace)[2 * c], ((volatile int*)g_trace)[2 * c + 1]);
        std::fprintf(stderr, "\n");
    }
#endif
    return cuda_status(e);
}

__global__ void k_to_c64(int64_t n, const double2* in, float2* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void k_to_df(int64_t n, const double2* in, float4* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = df_from(in[i]);
}

}  // namespace scocg

extern "C" int scocg_solve(scocg_handle h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
                           const int64_t* proj_idx, const void* proj_vec, int nproj, double tol,
                           scocg_c128* G_out, scocg_info* info) {
    if (!h) return SCOCG_ERR_INVALID;
    return solve_impl(h, shifts, nshift, rhs, nrhs, proj_idx, proj_vec, nproj, tol, G_out, info,
                      h->opts.precision, nullptr, nullptr);
}

extern "C" int scocg_solve_resume(scocg_handle h, const scocg_c128* shifts, int nshift, const void* rhs,
                                  const int64_t* proj_idx, const void* proj_vec, int nproj, double tol,
                                  scocg_c128* G_out, scocg_info* info) {
    if (!h) return SCOCG_ERR_INVALID;
    return solve_impl(h, shifts, nshift, rhs, 1, proj_idx, proj_vec, nproj, tol, G_out, info, h->opts.precision,
                      nullptr, nullptr, true);
}

namespace {
// Header of a saved continuation state; the shifts, the unit projection
// indices and the workspace bytes follow it.
struct StateHeader {
    uint64_t magic;
    int32_t version, prec, K, M, dense, kind;
    int64_t n, nnz;          // of the handle's H (a partial check that the loading handle holds the same H)
    uint64_t state_bytes;
};
constexpr uint64_t kStateMagic = 0x31747367636f6373ull;   // "scocgst1" little-endian

size_t state_total(const scocg_ctx* h) {
    return sizeof(StateHeader) + sizeof(scocg_c128) * (size_t)h->rs.K + sizeof(int64_t) * (size_t)h->rs.M +
           h->rs.state_bytes;
}
}  // namespace

extern "C" int scocg_state_size(scocg_handle h, size_t* bytes) {
    if (!h || !bytes) return SCOCG_ERR_INVALID;
    *bytes = 0;
    if (!h->rs.ok) return SCOCG_ERR_INVALID;
    *bytes = state_total(h);
    return SCOCG_OK;
}

extern "C" int scocg_state_save(scocg_handle h, void* buf, size_t bytes) {
    if (!h || !buf || !h->rs.ok || bytes < state_total(h)) return SCOCG_ERR_INVALID;
    StateHeader hd{kStateMagic, 1, h->rs.prec, h->rs.K, h->rs.M, h->rs.dense ? 1 : 0, (int32_t)h->kind, h->n,
                   h->nnz, h->rs.state_bytes};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    std::memcpy(p, h->rs.z.data(), sizeof(scocg_c128) * (size_t)hd.K);
    p += sizeof(scocg_c128) * (size_t)hd.K;
    std::memcpy(p, h->rs.cidx.data(), sizeof(int64_t) * (size_t)hd.M);
    p += sizeof(int64_t) * (size_t)hd.M;
    cudaError_t e = cudaMemcpyAsync(p, h->ws.base, h->rs.state_bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
}

extern "C" int scocg_state_load(scocg_handle h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < sizeof(StateHeader)) return SCOCG_ERR_INVALID;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != 1 || hd.n != h->n || hd.nnz != h->nnz ||
        hd.kind != (int32_t)h->kind || hd.K < 1 || hd.K > 4096 || hd.M < 1 ||
        hd.M > kMaxProj || (hd.prec != SCOCG_FP64 && hd.prec != SCOCG_MIXED && hd.prec != SCOCG_MIXED_DF))
        return SCOCG_ERR_INVALID;
    const size_t need = sizeof(hd) + sizeof(scocg_c128) * (size_t)hd.K + sizeof(int64_t) * (size_t)hd.M +
                        hd.state_bytes;
    if (bytes < need) return SCOCG_ERR_INVALID;
    const char* p = static_cast<const char*>(buf) + sizeof(hd);
    h->rs.ok = false;
    cudaError_t e = h->ws.reserve(hd.state_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws.base, p + sizeof(scocg_c128) * (size_t)hd.K + sizeof(int64_t) * (size_t)hd.M,
                            hd.state_bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    h->rs.prec = hd.prec; h->rs.K = hd.K; h->rs.M = hd.M; h->rs.dense = hd.dense != 0;
    const scocg_c128* z = reinterpret_cast<const scocg_c128*>(p);
    h->rs.z.assign(z, z + hd.K);
    const int64_t* ci = reinterpret_cast<const int64_t*>(p + sizeof(scocg_c128) * (size_t)hd.K);
    h->rs.cidx.assign(ci, ci + hd.M);
    h->rs.state_bytes = hd.state_bytes;
    h->rs.ok = true;
    return SCOCG_OK;
}

// The solve driver.  prec selects the vector precision; Xf/Pf (device
// complex128 [nshift][N] each, FP64 only, one right-hand side) switch on the
// full-vector mode that forms every shift's solution x_k.
int scocg::solve_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
                      const int64_t* proj_idx, const void* proj_vec, int nproj, double tol, scocg_c128* G_out,
                      scocg_info* info, int prec, double2* Xf, double2* Pf, bool resume) {
    if (!h || !shifts || nshift < 1 || nshift > 4096 || !rhs || nrhs < 1 || nproj < 1 ||
        nproj > kMaxProj || !G_out || (proj_idx == nullptr) == (proj_vec == nullptr) || !(tol >= 0.0))
        return SCOCG_ERR_INVALID;
    for (int k = 0; k < nshift; ++k)
        if (!std::isfinite(shifts[k].re) || !std::isfinite(shifts[k].im)) return SCOCG_ERR_INVALID;
    if (proj_idx)
        for (int64_t j = 0; j < (int64_t)nrhs * nproj; ++j)
            if (proj_idx[j] < 0 || proj_idx[j] >= h->n) return SCOCG_ERR_INVALID;
    if (Xf && (prec != SCOCG_FP64 || nrhs != 1 || nshift > kMaxFullShifts || !Pf)) return SCOCG_ERR_INVALID;
    if (resume) {
        // the same inputs as the stopped solve: precision, shifts (bit for
        // bit), projection kind and unit indices, one right-hand side
        const auto& rs = h->rs;
        if (!rs.ok || Xf || nrhs != 1 || prec != rs.prec || nshift != rs.K || nproj != rs.M ||
            (proj_vec != nullptr) != rs.dense ||
            std::memcmp(shifts, rs.z.data(), sizeof(scocg_c128) * (size_t)nshift) != 0 ||
            (proj_idx && std::memcmp(proj_idx, rs.cidx.data(), sizeof(int64_t) * (size_t)nproj) != 0))
            return SCOCG_ERR_INVALID;
    }
    if (!resume) h->rs.ok = false;   // any other solve overwrites the state
    const size_t dyn_smem = Xf ? (size_t)nshift * kFullSmem : 0;
    const bool mixed = prec == SCOCG_MIXED;
    const bool dfm = prec == SCOCG_MIXED_DF;
    // several right-hand sides with unit projections: the block kernel
    if (!Xf && nrhs > 1 && proj_idx && h->kind == HandleKind::kCsr && nproj <= kMaxProjB &&
        !(mixed && h->opts.replace_every > 0) && h->opts.rhs_tile != 1) {
        int T = h->opts.rhs_tile, per_sm = 0;
        if (T == 0) {
            if (h->opts.autotune) {
                const int st = block_autotune(h, shifts, nshift, rhs, nrhs, proj_idx, nproj, tol, G_out, prec, &T,
                                              &per_sm);
                if (st < 0) return st;
            } else {
                T = block_default_tile(nrhs);
            }
        }
        return block_solve(h, shifts, nshift, rhs, nrhs, proj_idx, nproj, tol, G_out, info, prec, T, per_sm);
    }
    const int64_t n = h->n;
    const int K = nshift, M = nproj;
    const int seed = (h->opts.seed >= 0 && h->opts.seed < K) ? h->opts.seed : default_seed(shifts, K);
    cudaStream_t s = h->stream;

    const Layout L = h->kind == HandleKind::kHubbard ? Layout{} : h->layout(false);
    int maxco = h->kind == HandleKind::kHubbard ? hubbard_max_ctas(h->hub, prec, h->num_sms, dyn_smem)
                                                 : max_coresident_ctas(L, prec, h->num_sms, dyn_smem);
    if (maxco <= 0) return SCOCG_ERR_CUDA;
    const int rpu = h->kind == HandleKind::kHubbard ? 32 : rows_per_unit(L.kind);
    const int64_t nunits = h->kind == HandleKind::kHubbard ? h->hub.nunits : (n + rpu - 1) / rpu;
    // one warp per unit of rows and one thread per shift at least; small
    // problems are latency bound and still gain from up to 32 CTAs (4,096-row
    // chain: 24.4 us per iteration at 8 CTAs, 21.1 at 32)
    int64_t want = std::max<int64_t>((nunits + kWarps - 1) / kWarps, (K + kBlock - 1) / kBlock);
    want = std::max<int64_t>(want, std::min<int64_t>(32, nunits));
    if (h->opts.grid > 0) want = h->opts.grid;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxco));
    if ((int64_t)grid * kBlock < K) return SCOCG_ERR_INVALID;
    const int strideB = 3 + 2 * M + 1;

    // workspace layout: the same sequence of pieces is measured, then carved
    const size_t velem = mixed ? sizeof(float2) : (dfm ? sizeof(float4) : sizeof(double2));
    const size_t vbytes = velem * (size_t)n;
    void *r = nullptr, *q = nullptr, *ps = nullptr, *xh = nullptr, *xl = nullptr, *cvec = nullptr;
    double2* xd = nullptr;
    int64_t* d_cidx = nullptr;
    double2* d_z = nullptr;
    ShiftState S{};
    ResumeState* rstate = nullptr;
    size_t state_end = 0;
    double *partA = nullptr, *partB = nullptr, *partC = nullptr;
    auto carve = [&](Carver& c) {
        r = c.take(vbytes);
        q = c.take(vbytes);
        if (mixed) {
            ps = c.take(vbytes); xh = c.take(vbytes); xl = c.take(vbytes);
            xd = (double2*)c.take(sizeof(double2) * n);
        }
        if ((mixed || dfm) && proj_vec) cvec = c.take(velem * (size_t)n * M);
        d_cidx = (int64_t*)c.take(sizeof(int64_t) * M);
        d_z = (double2*)c.take(sizeof(double2) * K);
        S.pi_prev = (double2*)c.take(sizeof(double2) * K);
        S.pi_cur = (double2*)c.take(sizeof(double2) * K);
        S.sigma = (double2*)c.take(sizeof(double2) * K);
        S.alpha_k = (double2*)c.take(sizeof(double2) * K);
        S.inv_cur = (double2*)c.take(sizeof(double2) * K);
        S.P = (double2*)c.take(sizeof(double2) * (size_t)K * M);
        S.X = (double2*)c.take(sizeof(double2) * (size_t)K * M);
        S.frozen = (int*)c.take(sizeof(int) * K);
        S.iters = (int*)c.take(sizeof(int) * K);
        S.resid = (double*)c.take(sizeof(double) * K);
        rstate = (ResumeState*)c.take(sizeof(ResumeState));
        state_end = c.off;
        partA = (double*)c.take(sizeof(double) * grid * 4);
        partB = (double*)c.take(sizeof(double) * grid * strideB);
        partC = (double*)c.take(sizeof(double) * grid * kPartC);
    };
    Carver measure{nullptr, 0};
    carve(measure);
    // a continuation keeps the state bytes when the workspace grows (its
    // partials may be sized for another grid)
    cudaError_t e = resume ? h->ws.reserve_keep(measure.off, h->rs.state_bytes, s) : h->ws.reserve(measure.off);
    if (e != cudaSuccess) return cuda_status(e);
    Carver cut{static_cast<char*>(h->ws.base), 0};
    carve(cut);
    if (resume && state_end != h->rs.state_bytes) return SCOCG_ERR_INVALID;

    e = cudaMemcpyAsync(d_z, shifts, sizeof(double2) * K, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && mixed && proj_vec) {
        const int64_t tot = n * M;
        k_to_c64<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(tot, (const double2*)proj_vec, (float2*)cvec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && dfm && proj_vec) {
        const int64_t tot = n * M;
        k_to_df<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(tot, (const double2*)proj_vec, (float4*)cvec);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_status(e);
    const void* cv = proj_vec ? ((mixed || dfm) ? cvec : proj_vec) : nullptr;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0); cudaEventCreate(&ev1);
    float total_ms = 0.f;
    int worst = SCOCG_OK;
    int iters = 0, nsw = 0, seed_final = seed, nrep = 0;
    long long siters = 0;
    std::vector<int> h_iters(K);
    std::vector<double> h_resid(K);
    for (int j = 0; j < nrhs && worst >= 0; ++j) {
        if (proj_idx) {
            e = cudaMemcpyAsync(d_cidx, proj_idx + (size_t)j * M, sizeof(int64_t) * M, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { worst = cuda_status(e); break; }
        }
        const double2* b = static_cast<const double2*>(rhs) + (size_t)j * n;
        double2* G = reinterpret_cast<double2*>(G_out) + (size_t)j * M * K;
        cudaEventRecord(ev0, s);
        const int64_t* ci = proj_idx ? d_cidx : nullptr;
        ResumeState* rsj = nrhs == 1 && !Xf ? rstate : nullptr;
        const int res = resume ? 1 : 0;
        int st = mixed ? solve_one_rhs<float>(h, d_z, K, seed, b, ci, cv, M, tol, G, grid, S, partA, partB, partC,
                                              strideB, (float2*)r, (float2*)q, (float2*)ps, (float2*)xh,
                                              (float2*)xl, xd, L, rsj, res)
               : dfm ? solve_one_rhs<DF>(h, d_z, K, seed, b, ci, cv, M, tol, G, grid, S, partA, partB, partC,
                                         strideB, (float4*)r, (float4*)q, nullptr, nullptr, nullptr, nullptr, L,
                                         rsj, res)
                     : solve_one_rhs<double>(h, d_z, K, seed, b, ci, cv, M, tol, G, grid, S, partA, partB, partC,
                                             strideB, (double2*)r, (double2*)q, nullptr, nullptr, nullptr, nullptr, L,
                                             rsj, res, Xf, Pf);
        cudaEventRecord(ev1, s);
        if (st != SCOCG_OK) { worst = st; break; }
        Ctrl c;
        e = cudaMemcpyAsync(&c, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_iters.data(), S.iters, sizeof(int) * K, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_resid.data(), S.resid, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { worst = cuda_status(e); break; }
        if (c.dbg[0]) {
            std::fprintf(stderr, "scocg checked build: out-of-range index at site %llu: %lld (limit %lld)\n",
                         c.dbg[1], (long long)c.dbg[2], (long long)c.dbg[3]);
            worst = SCOCG_ERR_INVALID;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        total_ms += ms;
        const int dst = c.status;
        if (dst < 0) worst = dst;
        else if (dst == SCOCG_NOT_CONVERGED && worst == SCOCG_OK) worst = SCOCG_NOT_CONVERGED;
        iters = std::max(iters, c.stats.iters);
        nsw += c.stats.n_switch;
        nrep += c.stats.n_replace;
        seed_final = c.stats.seed;
        siters += c.stats.shift_iters;
        if (info) {
            if (info->freeze_iter) std::memcpy(info->freeze_iter + (size_t)j * K, h_iters.data(), sizeof(int) * K);
            if (info->resid)   // the kernel keeps squared residual estimates
                for (int k = 0; k < K; ++k) info->resid[(size_t)j * K + k] = std::sqrt(h_resid[k]);
        }
    }
    cudaEventDestroy(ev0); cudaEventDestroy(ev1);
    // a single-right-hand-side solve that stopped at max_iter can be continued
    h->rs.ok = nrhs == 1 && !Xf && worst == SCOCG_NOT_CONVERGED;
    if (h->rs.ok) {
        h->rs.prec = prec; h->rs.K = K; h->rs.M = M; h->rs.dense = proj_vec != nullptr;
        h->rs.z.assign(shifts, shifts + K);
        h->rs.cidx.assign(M, 0);
        if (proj_idx) h->rs.cidx.assign(proj_idx, proj_idx + M);
        h->rs.state_bytes = state_end;
    }
    if (info) {
        info->iters = iters;
        info->n_switch = nsw;
        info->seed_final = seed_final;
        info->n_replace = nrep;
        info->shift_iters = siters;
        info->seconds = total_ms * 1e-3;
        info->bytes_per_iter = h->bytes_per_iter(prec, proj_vec != nullptr, M);
    }
    return worst;
}

double scocg_ctx::bytes_per_iter(int prec, bool dense_proj, int M) const {
    const bool mixed = prec == SCOCG_MIXED;
    // Algorithmic bytes of one seed iteration: H once in the device layout,
    // plus every vector pass the kernel makes (phase A: gather r, read and
    // write q; phase B: read r and q, write r, read each dense c_m; MIXED adds
    // the seed p (read, write) and the compensated x (two vectors read, write)).
    const double vb = mixed ? 8.0 : 16.0;   // FP64 and compensated FP32 entries are both 16 bytes
    double hbytes;
    if (kind == HandleKind::kHubbard) {
        hbytes = hub.table_bytes;
    } else {
        const Layout L = layout(false);
        const double rb = prec == SCOCG_FP64 ? 8.0 : 4.0;
        if (L.kind == LayoutKind::kBsr4) hbytes = (double)nslots * 8 * (4 + 16 * rb) + 4.0 * (nunits_bsr + 1);
        else hbytes = (double)nnz * (4 + rb) + 4.0 * (n + 1);
    }
    double passes = 6 + (dense_proj ? M : 0);
    if (mixed && opts.replace_every > 0) passes += 6;
    return hbytes + passes * vb * (double)n;
}

// ---------------------------------------------------------------- not yet built entry points
extern "C" int scocg_solve_full(scocg_handle h, const scocg_c128* shifts, int nshift, const void* rhs, double tol,
                                void* X_out, scocg_info* info) {
    return solve_full_impl(h, shifts, nshift, rhs, tol, X_out, info);
}

extern "C" int scocg_grad(scocg_handle h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
                          const int64_t* proj_idx, const void* proj_vec, int nproj, double tol,
                          const scocg_c128* dL_dG, double* dL_dval, scocg_info* info) {
    return grad_impl(h, shifts, nshift, rhs, nrhs, proj_idx, proj_vec, nproj, tol, dL_dG, dL_dval, info);
}
