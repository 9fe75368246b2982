// C ABI of libgnk: argument checks, host/device staging and the handle's
// lifecycle.  The numerical work is in pairsum.cu, circulant.cu, ops.cu and
// krylov.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>
#include <utility>
#include <vector>

#include "gnk_internal.h"

namespace gnk {

static thread_local char g_err[1024] = "";
static std::atomic<unsigned long long> g_launches{0};

static thread_local bool g_count_off = false;

void count_launches(unsigned long long n) {
    if (!g_count_off) g_launches.fetch_add(n, std::memory_order_relaxed);
}

void count_suppress(bool on) { g_count_off = on; }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of an input array of `count` doubles: the pointer itself when it
// is device memory, else a copy in staging slot `slot` of the handle.
int stage_in(const Boundary& b, const double* p, size_t count, int slot, cudaStream_t st,
             const double** out) {
    if (is_device_ptr(p)) {
        *out = p;
        return GNK_OK;
    }
    double* dst = b.stage + (size_t)slot * 2 * b.N;
    GNK_TRY_CUDA(cudaMemcpyAsync(dst, p, count * sizeof(double), cudaMemcpyHostToDevice, st));
    *out = dst;
    return GNK_OK;
}

struct Out {
    double* user = nullptr;
    double* dev = nullptr;
    size_t count = 0;
    bool host = false;
};

Out stage_out(const Boundary& b, double* p, size_t count, int slot) {
    Out o;
    o.user = p;
    o.count = count;
    o.host = !is_device_ptr(p);
    o.dev = o.host ? b.stage + (size_t)slot * 2 * b.N : p;
    return o;
}

int finish_out(const Out& o, cudaStream_t st) {
    if (!o.host) return GNK_OK;
    GNK_TRY_CUDA(cudaMemcpyAsync(o.user, o.dev, o.count * sizeof(double), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    return GNK_OK;
}

int check_handle(const gnk_boundary* h) {
    if (!h) {
        set_error("NULL boundary handle");
        return GNK_EINVAL;
    }
    return GNK_OK;
}

int check_prec(int prec) {
    if (prec != GNK_PREC_FP64 && prec != GNK_PREC_FP32 && prec != GNK_PREC_DF32 && prec != GNK_PREC_FMM) {
        set_error("precision must be GNK_PREC_FP64, GNK_PREC_FP32, GNK_PREC_DF32 or GNK_PREC_FMM here, "
                  "got %d", prec);
        return GNK_EINVAL;
    }
    return GNK_OK;
}

// Frees the handle's device memory once every stream's work on it is done
// (the device synchronisation that cudaFree would imply), back to the pool.
void release(Boundary& b) {
    void* ptrs[] = {b.arena, b.V, b.kry, b.kstate};
    bool any = b.fmm != nullptr;
    for (void* p : ptrs) any = any || p != nullptr;
    if (!any) return;
    cudaDeviceSynchronize();
    cudaGetLastError();
    release_fmm(b);
    for (void* p : ptrs)
        if (p) pool_free(p, 0);
    b.arena = nullptr;
    b.V = nullptr;
    b.kry = nullptr;
    b.kstate = nullptr;
}

// Carves the handle's fixed-size buffers out of one device allocation
// (256-byte aligned pieces).
struct Arena {
    std::vector<std::pair<void**, size_t>> parts;
    template <class T>
    void add(T** p, size_t count) {
        parts.emplace_back(reinterpret_cast<void**>(p), count * sizeof(T));
    }
    int allocate(void** base, cudaStream_t st) {
        size_t total = 0;
        for (auto& pr : parts) total += (pr.second + 255) / 256 * 256;
        if (pool_alloc(base, total + 256, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of %zu bytes failed", total);
            return GNK_ENOMEM;
        }
        char* c = static_cast<char*>(*base);
        for (auto& pr : parts) {
            *pr.first = c;
            c += (pr.second + 255) / 256 * 256;
        }
        return GNK_OK;
    }
};

int options_from(const gnk_options* in, gnk_options* o) {
    gnk_default_options(o);
    if (in) *o = *in;
    if (o->restart < 1 || o->restart > 1000 || o->maxit < 1 || !(o->tol > 0.0) ||
        (o->precision != GNK_PREC_FP64 && o->precision != GNK_PREC_MIXED &&
         o->precision != GNK_PREC_DF32 && o->precision != GNK_PREC_MIXED_DF &&
         o->precision != GNK_PREC_FMM && o->precision != GNK_PREC_MIXED_FMM) ||
        o->max_refine < 0 || !(o->inner_tol > 0.0) || o->tile_chunks < 0 || o->tile_chunks > 64 ||
        o->tile_variant < 0 || o->tile_variant > 7) {
        set_error("invalid gnk_options (restart 1..1000, maxit >= 1, tol > 0, precision "
                  "FP64|MIXED|DF32|MIXED_DF|FMM|MIXED_FMM, max_refine >= 0, inner_tol > 0, "
                  "tile_chunks 0..64, tile_variant 0..7)");
        return GNK_EINVAL;
    }
    return GNK_OK;
}

// The tile override of one call on a handle (calls on one handle never
// overlap, so the handle carries it for the duration of the call).
struct TileOverride {
    const Boundary& b;
    TileOverride(const Boundary& bb, int chunks) : b(bb) { b.tile_chunks = chunks; }
    ~TileOverride() { b.tile_chunks = 0; }
};

// Phase times of one call (gnk_options.timing): an event on the caller's
// stream at each phase boundary, read once at the end of the call.
struct Phases {
    static constexpr int kMax = 5;
    cudaEvent_t ev[kMax] = {};
    int n = 0;
    bool on = false;
    cudaStream_t st = nullptr;
    Phases(bool enable, cudaStream_t s) : on(enable), st(s) { mark(); }
    void mark() {
        if (!on || n >= kMax) return;
        if (cudaEventCreate(&ev[n]) != cudaSuccess || cudaEventRecord(ev[n], st) != cudaSuccess) {
            cudaGetLastError();
            on = false;
            return;
        }
        ++n;
    }
    // Elapsed ms between consecutive marks into out[0..k).
    void read(double* const* out, int k) {
        if (!on || n < 2) return;
        if (cudaEventSynchronize(ev[n - 1]) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        for (int i = 0; i < k && i + 1 < n; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) *out[i] = ms;
            else cudaGetLastError();
        }
    }
    ~Phases() {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    }
};

// Work of the setup phase that a timed call does up front: for the FMM
// precisions the quadtree and its power table (the work an untimed call does
// at its first product; a deferred Eone stays fused with the right-hand side).
int timed_setup(const Boundary& b, int outer, cudaStream_t st) {
    if (outer == GNK_PREC_FMM) GNK_TRY(ensure_fmm(b, kMaxRHS, st));
    return GNK_OK;
}

int build(Boundary& b, int m1, int n, const double* et, const double* etp, const double* etpp,
          const double* A, const double* Ap, int bounded, int eone_prec, int defer, int plain,
          cudaStream_t st) {
    const size_t N = (size_t)m1 * n;
    b.m1 = m1;
    b.n = n;
    b.N = (int)N;
    b.bounded = bounded ? 1 : 0;
    b.has_adjoint = etpp != nullptr;
    b.plain = plain;
    GNK_TRY_CUDA(cudaGetDevice(&b.device));
    GNK_TRY_CUDA(cudaDeviceGetAttribute(&b.sms, cudaDevAttrMultiProcessorCount, b.device));

    const int tiles32 = (b.N + kSrcTile32 - 1) / kSrcTile32;
    // launch plans (they fix the size of the split-source workspace)
    b.plan64 = make_plan(b.N, b.sms, pair_blocks_per_sm(GNK_PREC_FP64), kThreads64 * kTargets64,
                         kSrcTile64);
    b.plan32 = make_plan(b.N, b.sms, pair_blocks_per_sm(GNK_PREC_FP32), kThreads32 * kTargets32,
                         kSrcTile32);
    b.plandf = make_plan(b.N, b.sms, pair_blocks_per_sm(GNK_PREC_DF32), kThreadsDF * kTargetsDF,
                         kSrcTile32);
    GNK_TRY(pair_workspace_bytes(b, &b.partial_bytes));
    // every fixed-size buffer of the handle lives in one device allocation
    Arena ar;
    ar.add(&b.et, N);
    ar.add(&b.etp, N);
    ar.add(&b.A, N);
    ar.add(&b.q, N);
    ar.add(&b.Eone, N);
    ar.add(&b.b1, N);
    ar.add(&b.d1, N);
    ar.add(&b.e, N);
    ar.add(&b.ref32, (size_t)tiles32);
    ar.add(&b.off32, N);
    ar.add(&b.et32, N);
    ar.add(&b.q32, N);
    ar.add(&b.A32, N);
    ar.add(&b.ref64, (size_t)tiles32);
    ar.add(&b.offdf, N);
    ar.add(&b.twiddle, (size_t)n);
    ar.add(&b.Lcol, (size_t)n);
    ar.add(&b.zbuf, kMaxRHS * N);
    ar.add(&b.r0, N);
    ar.add(&b.r1, N);
    ar.add(&b.r2, N);
    ar.add(&b.r3, N);
    ar.add(&b.r4, N);
    ar.add(&b.r5, N);
    ar.add(&b.r6, N);
    ar.add(&b.ones, N);
    ar.add(&b.means, (size_t)m1);
    ar.add(&b.stage, 4 * 2 * N);
    ar.add(reinterpret_cast<char**>(&b.partial), b.partial_bytes);
    ar.add(&b.flag, 1);
    GNK_TRY(ar.allocate(&b.arena, st));

    // geometry copies (host or device sources; cudaMemcpyDefault infers the direction)
    GNK_TRY_CUDA(cudaMemcpyAsync(b.et, et, N * sizeof(double2), cudaMemcpyDefault, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(b.etp, etp, N * sizeof(double2), cudaMemcpyDefault, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(b.A, A, N * sizeof(double2), cudaMemcpyDefault, st));
    const double* d_etpp = nullptr;
    const double* d_Ap = nullptr;
    if (etpp) {
        double* s0 = b.stage;
        GNK_TRY_CUDA(cudaMemcpyAsync(s0, etpp, N * sizeof(double2), cudaMemcpyDefault, st));
        d_etpp = s0;
        if (Ap) {
            double* s1 = b.stage + 2 * N;
            GNK_TRY_CUDA(cudaMemcpyAsync(s1, Ap, N * sizeof(double2), cudaMemcpyDefault, st));
            d_Ap = s1;
        }
    }
    int* d_flag = b.flag;
    GNK_TRY_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    GNK_TRY_CUDA(cudaMemsetAsync(b.e, 0, N * sizeof(double), st));
    int s = run_prepare_geometry(b, d_etpp, d_Ap, d_flag, st);
    int flag = 0;
    if (s == GNK_OK) {
        cudaError_t e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("geometry preparation failed: %s", cudaGetErrorString(e));
            s = GNK_ECUDA;
        }
    }
    GNK_TRY(s);
    if (flag & 1) {
        set_error("non-finite value in eta, eta', eta'', A or A'");
        return GNK_ENONFINITE;
    }
    if (flag & 2) {
        set_error("A(t) vanishes at a node");
        return GNK_EINVAL;
    }
    b.A_real = (flag & 4) ? 0 : 1;


    b.eone_prec = eone_prec;
    if (plain) {
        // the diagonals came from the geometry preparation; no Cauchy sum is needed
        GNK_TRY_CUDA(cudaMemsetAsync(b.Eone, 0, N * sizeof(double2), st));
        GNK_TRY_CUDA(cudaStreamSynchronize(st));
        return GNK_OK;
    }
    // Eone = E q with diag(B1), diag(D1); with eta'' also E eta' and e (Eq. bve)
    PairJob j;
    j.R = b.has_adjoint ? 2 : 1;
    j.mode = W_COMPLEX;
    j.w[0] = b.q;
    j.w[1] = b.etp;
    j.epi = EPI_EONE;
    j.out_c = b.Eone;
    j.out = b.b1;
    j.out2 = b.d1;
    j.out3 = b.e;
    if (defer) {
        b.eone_pending = 1;  // formed by the first call that needs them
        return GNK_OK;
    }
    GNK_TRY(run_pairsum(b, j, eone_prec, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    return GNK_OK;
}

}  // namespace
}  // namespace gnk

using namespace gnk;

extern "C" {

void gnk_default_options(gnk_options* o) {
    if (!o) return;
    o->restart = 20;
    o->maxit = 50;
    o->tol = 1e-12;
    o->precision = GNK_PREC_FP64;
    o->max_refine = 10;
    o->inner_tol = 1e-5;
    o->tile_chunks = 0;
    o->tile_variant = 0;
    o->timing = 0;
}

int gnk_last_error(char* buf, size_t len) {
    const int l = (int)strlen(g_err);
    if (buf && len > 0) {
        strncpy(buf, g_err, len - 1);
        buf[len - 1] = '\0';
    }
    return l;
}

const char* gnk_version(void) { return "gnk-gb300 0.1 (sm_103a)"; }

unsigned long long gnk_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int gnk_build_boundary(gnk_boundary** out, int m1, int n, const double* et, const double* etp,
                       const double* etpp, const double* A, const double* Ap, int bounded,
                       void* stream) {
    return gnk_build_boundary_ex(out, m1, n, et, etp, etpp, A, Ap, bounded, GNK_PREC_FP64, stream);
}

int gnk_build_boundary_ex(gnk_boundary** out, int m1, int n, const double* et, const double* etp,
                          const double* etpp, const double* A, const double* Ap, int bounded,
                          int precision, void* stream) {
    const int defer = (precision & GNK_BUILD_DEFER) ? 1 : 0;
    const int plain = (precision & GNK_BUILD_PLAIN) ? 1 : 0;
    precision &= ~(GNK_BUILD_DEFER | GNK_BUILD_PLAIN);
    if (precision != GNK_PREC_FP64 && precision != GNK_PREC_DF32 && precision != GNK_PREC_FMM) {
        set_error("gnk_build_boundary_ex: precision must be GNK_PREC_FP64, GNK_PREC_DF32 or "
                  "GNK_PREC_FMM (optionally | GNK_BUILD_DEFER | GNK_BUILD_PLAIN)");
        return GNK_EINVAL;
    }
    if (plain && !etpp) {
        set_error("gnk_build_boundary_ex: GNK_BUILD_PLAIN needs eta'' (the diagonal N(t,t))");
        return GNK_EINVAL;
    }
    if (!out || !et || !etp || !A) {
        set_error("gnk_build_boundary: out, et, etp and A must not be NULL");
        return GNK_EINVAL;
    }
    *out = nullptr;
    if (m1 < 1 || n < 4 || (n % 2) != 0) {
        set_error("gnk_build_boundary: need m1 >= 1 and n even, n >= 4 (got m1=%d n=%d)", m1, n);
        return GNK_EINVAL;
    }
    if ((long long)m1 * n > (1LL << 28)) {
        set_error("gnk_build_boundary: (m+1) n = %lld exceeds 2^28 nodes", (long long)m1 * n);
        return GNK_EINVAL;
    }
    cudaGetLastError();  // a stale, non-sticky error of earlier calls is not ours
    gnk_boundary* h = new (std::nothrow) gnk_boundary();
    if (!h) {
        set_error("host allocation failed");
        return GNK_ENOMEM;
    }
    const int s = build(h->b, m1, n, et, etp, etpp, A, Ap, bounded, precision, defer, plain,
                        (cudaStream_t)stream);
    if (s != GNK_OK) {
        release(h->b);
        delete h;
        return s;
    }
    *out = h;
    return GNK_OK;
}

int gnk_free_boundary(gnk_boundary* h) {
    if (!h) return GNK_OK;
    release(h->b);
    delete h;
    return GNK_OK;
}

int gnk_boundary_size(const gnk_boundary* h, int* m1, int* n) {
    GNK_TRY(check_handle(h));
    if (m1) *m1 = h->b.m1;
    if (n) *n = h->b.n;
    return GNK_OK;
}

int gnk_cauchy_sum(const gnk_boundary* h, const double* w, double* z, int precision, void* stream) {
    GNK_TRY(check_handle(h));
    GNK_TRY(check_prec(precision));
    if (!w || !z) {
        set_error("gnk_cauchy_sum: NULL array");
        return GNK_EINVAL;
    }
    const Boundary& b = h->b;
    cudaStream_t st = (cudaStream_t)stream;
    const double* dw;
    GNK_TRY(stage_in(b, w, 2 * (size_t)b.N, 0, st, &dw));
    Out o = stage_out(b, z, 2 * (size_t)b.N, 1);
    PairJob j;
    j.R = 1;
    j.mode = W_COMPLEX;
    j.w[0] = reinterpret_cast<const double2*>(dw);
    j.epi = EPI_Z;
    j.out_c = reinterpret_cast<double2*>(o.dev);
    GNK_TRY(run_pairsum(b, j, precision, st));
    return finish_out(o, st);
}

typedef int (*unary_op)(const Boundary&, const double*, double*, int, cudaStream_t);

static int apply_unary(const gnk_boundary* h, const double* x, double* y, int prec, void* stream,
                       int which) {
    GNK_TRY(check_handle(h));
    GNK_TRY(check_prec(prec));
    if (!x || !y) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    const Boundary& b = h->b;
    if (which == 2 && !b.has_adjoint) {
        set_error("the adjoint operator needs a handle built with eta''");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (which != 3) GNK_TRY(ensure_eone(b, st));
    const double* dx;
    GNK_TRY(stage_in(b, x, b.N, 0, st, &dx));
    Out o = stage_out(b, y, b.N, 1);
    if (which == 0) GNK_TRY(op_IminusN(b, dx, o.dev, prec, st));
    else if (which == 1) GNK_TRY(op_M(b, dx, o.dev, prec, st));
    else if (which == 2) GNK_TRY(op_adjoint(b, dx, o.dev, prec, st));
    else GNK_TRY(run_circulant(b, dx, o.dev, st));
    return finish_out(o, st);
}

int gnk_apply_IminusN(const gnk_boundary* h, const double* x, double* y, int precision, void* stream) {
    return apply_unary(h, x, y, precision, stream, 0);
}

int gnk_apply_M(const gnk_boundary* h, const double* x, double* y, int precision, void* stream) {
    return apply_unary(h, x, y, precision, stream, 1);
}

int gnk_apply_adjoint(const gnk_boundary* h, const double* x, double* y, int precision, void* stream) {
    return apply_unary(h, x, y, precision, stream, 2);
}

int gnk_apply_circulant(const gnk_boundary* h, const double* x, double* y, void* stream) {
    return apply_unary(h, x, y, GNK_PREC_FP64, stream, 3);
}

static int solve_common(const gnk_boundary* h, const double* gam, double* mu, const gnk_options* opt,
                        gnk_result* info, void* stream, int adjoint) {
    GNK_TRY(check_handle(h));
    cudaGetLastError();
    if (!gam || !mu) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    gnk_options o;
    GNK_TRY(options_from(opt, &o));
    const Boundary& b = h->b;
    if (adjoint && !b.has_adjoint) {
        set_error("gnk_solve_adjoint_ie needs a handle built with eta''");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const TileOverride tile(b, o.tile_chunks);
    Phases ph(o.timing != 0, st);
    if (o.timing) GNK_TRY(timed_setup(b, outer_precision(o.precision), st));
    // the products of the equation are z = E(q x): their near-field cache forms
    // beside the work up to the first product
    if (!adjoint && outer_precision(o.precision) == GNK_PREC_FMM) GNK_TRY(fmm_start_near_cache(b, st));
    GNK_TRY(ensure_eone(b, st));
    ph.mark();
    const double* dg;
    GNK_TRY(stage_in(b, gam, b.N, 0, st, &dg));
    Out o_mu = stage_out(b, mu, b.N, 1);
    const double* rhs = dg;
    if (!adjoint) {
        // right-hand side -y = -(D - diag(D1) + Lhat) gamma (Eqs. sys, y)
        GNK_TRY(op_M(b, dg, b.r4, outer_precision(o.precision), st));
        GNK_TRY(op_negate(b.r4, b.N, st));
        rhs = b.r4;
    }
    ph.mark();
    const int s = solve(b, adjoint, rhs, o_mu.dev, o, info, st);
    if (s != GNK_OK && s != GNK_ENOTCONV && s != GNK_ENONFINITE) return s;
    ph.mark();
    if (info) {
        double* outs[3] = {&info->setup_ms, &info->rhs_ms, &info->solve_ms};
        ph.read(outs, 3);
    }
    GNK_TRY(finish_out(o_mu, st));
    if (s == GNK_ENOTCONV) set_error("GMRES did not reach tol within maxit cycles");
    if (s == GNK_ENONFINITE) set_error("non-finite value in the GMRES iteration");
    return s;
}

int gnk_solve_ie(const gnk_boundary* h, const double* gam, double* mu, const gnk_options* opt,
                 gnk_result* info, void* stream) {
    return solve_common(h, gam, mu, opt, info, stream, 0);
}

int gnk_solve_adjoint_ie(const gnk_boundary* h, const double* gam, double* mu, const gnk_options* opt,
                         gnk_result* info, void* stream) {
    return solve_common(h, gam, mu, opt, info, stream, 1);
}

int gnk_fbie(const gnk_boundary* hd, const double* gam, double* mu, double* hv, double* hk,
             const gnk_options* opt, gnk_result* info, void* stream) {
    GNK_TRY(check_handle(hd));
    if (!gam || !mu || !hv) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    cudaGetLastError();
    gnk_options o;
    GNK_TRY(options_from(opt, &o));
    const Boundary& b = hd->b;
    cudaStream_t st = (cudaStream_t)stream;
    const int outer = outer_precision(o.precision);
    const TileOverride tile(b, o.tile_chunks);
    Phases ph(o.timing != 0, st);
    // a timed call forms the deferred precompute and the tree as their own phase
    if (o.timing) GNK_TRY(timed_setup(b, outer, st));
    // every product of the FBIE is z = E(q x): its near-field cache forms on a
    // stream of its own beside the work up to the first product
    if (outer == GNK_PREC_FMM) GNK_TRY(fmm_start_near_cache(b, st));
    ph.mark();
    const double* dg;
    GNK_TRY(stage_in(b, gam, b.N, 0, st, &dg));
    Out o_mu = stage_out(b, mu, b.N, 1);
    Out o_h = stage_out(b, hv, b.N, 2);
    // -y and f_B(gamma) from one Cauchy sum; a deferred handle forms Eone in the same launch
    if (b.eone_pending && !b.has_adjoint && b.eone_prec == outer) {
        GNK_TRY(op_eone_rhs_fb(b, dg, b.r4, b.r5, b.eone_prec, st));
    } else {
        GNK_TRY(ensure_eone(b, st));
        GNK_TRY(op_rhs_fb(b, dg, b.r4, b.r5, outer, st));
    }
    ph.mark();
    int fc_valid = 0;
    const int s = solve(b, 0, b.r4, o_mu.dev, o, info, st, b.r6, &fc_valid);
    if (s != GNK_OK && s != GNK_ENOTCONV && s != GNK_ENONFINITE) return s;
    ph.mark();
    if (!fc_valid) GNK_TRY(op_M(b, o_mu.dev, b.r6, outer, st));  // f_C(mu)
    GNK_TRY(op_half_diff(b.r6, b.r5, o_h.dev, b.N, st));
    if (hk) {
        Out o_k = stage_out(b, hk, b.m1, 3);
        GNK_TRY(run_component_means(b, o_h.dev, o_k.dev, st));
        GNK_TRY(finish_out(o_k, st));
    }
    ph.mark();
    if (info) {
        double* outs[4] = {&info->setup_ms, &info->rhs_ms, &info->solve_ms, &info->h_ms};
        ph.read(outs, 4);
    }
    GNK_TRY(finish_out(o_mu, st));
    GNK_TRY(finish_out(o_h, st));
    if (s == GNK_ENOTCONV) set_error("GMRES did not reach tol within maxit cycles");
    if (s == GNK_ENONFINITE) set_error("non-finite value in the GMRES iteration");
    return s;
}

int gnk_solve_ie_transpose(const gnk_boundary* hd, const double* rhs, double* x, const gnk_options* opt,
                           gnk_result* info, void* stream) {
    GNK_TRY(check_handle(hd));
    if (!rhs || !x) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    gnk_options o;
    GNK_TRY(options_from(opt, &o));
    const Boundary& b = hd->b;
    cudaStream_t st = (cudaStream_t)stream;
    const TileOverride tile(b, o.tile_chunks);
    GNK_TRY(ensure_eone(b, st));
    const double* dr;
    GNK_TRY(stage_in(b, rhs, b.N, 0, st, &dr));
    Out ox = stage_out(b, x, b.N, 1);
    const int s = solve(b, OP_KT, dr, ox.dev, o, info, st);
    if (s != GNK_OK && s != GNK_ENOTCONV && s != GNK_ENONFINITE) return s;
    GNK_TRY(finish_out(ox, st));
    if (s == GNK_ENOTCONV) set_error("GMRES did not reach tol within maxit cycles");
    return s;
}

namespace {
// A device view of a caller array for the backward pass: the array itself if
// it is device memory, else a temporary device copy (inputs) or buffer
// (outputs) that is released, after copying back, by the destructor's owner.
struct DevArr {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool tmp = false;
};

int dev_view(const void* p, size_t bytes, bool input, cudaStream_t st, DevArr* out) {
    out->user = const_cast<void*>(p);
    out->bytes = bytes;
    if (is_device_ptr(p)) {
        out->dev = const_cast<void*>(p);
        return GNK_OK;
    }
    if (pool_alloc(&out->dev, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("staging allocation failed");
        return GNK_ENOMEM;
    }
    out->tmp = true;
    if (input) GNK_TRY_CUDA(cudaMemcpyAsync(out->dev, p, bytes, cudaMemcpyHostToDevice, st));
    return GNK_OK;
}
}  // namespace

int gnk_fbie_backward(const gnk_boundary* hd, const double* mu, const double* gam, const double* grad_mu,
                      const double* grad_h, const double* grad_hk, double* grad_et, double* grad_etp,
                      double* grad_A, double* grad_gam, const gnk_options* opt, gnk_result* info,
                      void* stream) {
    GNK_TRY(check_handle(hd));
    if (!mu || !gam || !grad_mu || !grad_h || !grad_et || !grad_etp || !grad_A || !grad_gam) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    if (hd->b.plain) {
        set_error("gnk_fbie_backward: the handle holds the form without singularity subtraction");
        return GNK_EINVAL;
    }
    gnk_options o;
    GNK_TRY(options_from(opt, &o));
    const Boundary& b = hd->b;
    cudaStream_t st = (cudaStream_t)stream;
    const TileOverride tile(b, o.tile_chunks);
    GNK_TRY(ensure_eone(b, st));
    const size_t rN = (size_t)b.N * sizeof(double), cN = 2 * rN;
    DevArr v[9];
    const void* src[9] = {mu, gam, grad_mu, grad_h, grad_et, grad_etp, grad_A, grad_gam, grad_hk};
    const size_t sz[9] = {rN, rN, rN, rN, cN, cN, cN, rN, (size_t)b.m1 * sizeof(double)};
    int rc = GNK_OK;
    for (int k = 0; k < 9 && rc == GNK_OK; ++k) {
        if (!src[k]) continue;  // grad_hk is optional
        rc = dev_view(src[k], sz[k], k < 4 || k == 8, st, &v[k]);
    }
    int s = rc;
    if (rc == GNK_OK) {
        s = fbie_backward(b, (const double*)v[0].dev, (const double*)v[1].dev, (const double*)v[2].dev,
                          (const double*)v[3].dev, (const double*)v[8].dev, (double2*)v[4].dev,
                          (double2*)v[5].dev, (double2*)v[6].dev, (double*)v[7].dev, o, info, st);
        if (s == GNK_OK || s == GNK_ENOTCONV) {
            for (int k = 4; k < 8; ++k)
                if (v[k].tmp && cudaMemcpyAsync(v[k].user, v[k].dev, v[k].bytes, cudaMemcpyDeviceToHost,
                                                st) != cudaSuccess) {
                    cudaGetLastError();
                    s = GNK_ECUDA;
                }
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                cudaGetLastError();
                s = GNK_ECUDA;
            }
        }
    }
    for (int k = 0; k < 9; ++k)
        if (v[k].tmp) pool_free(v[k].dev, st);
    return s;
}

int gnk_cauchy_eval(const gnk_boundary* hd, int nz, const double* z, const double* f, const double* finf,
                    double* fz, int precision, void* stream) {
    cudaGetLastError();
    GNK_TRY(check_handle(hd));
    if (precision != GNK_PREC_FP64 && precision != GNK_PREC_DF32) {
        set_error("gnk_cauchy_eval: precision must be GNK_PREC_FP64 or GNK_PREC_DF32, got %d", precision);
        return GNK_EINVAL;
    }
    if (nz < 0) {
        set_error("gnk_cauchy_eval: nz = %d < 0", nz);
        return GNK_EINVAL;
    }
    if (nz == 0) return GNK_OK;
    if (!z || !f || !fz) {
        set_error("gnk_cauchy_eval: NULL array");
        return GNK_EINVAL;
    }
    const Boundary& b = hd->b;
    cudaStream_t st = (cudaStream_t)stream;
    const double2 fi = finf ? make_double2(finf[0], finf[1]) : make_double2(0.0, 0.0);
    DevArr v[3];
    const void* src[3] = {z, f, fz};
    const size_t sz[3] = {2 * sizeof(double) * (size_t)nz, 2 * sizeof(double) * (size_t)b.N,
                          2 * sizeof(double) * (size_t)nz};
    int rc = GNK_OK;
    for (int k = 0; k < 3 && rc == GNK_OK; ++k) rc = dev_view(src[k], sz[k], k < 2, st, &v[k]);
    if (rc == GNK_OK)
        rc = cauchy_eval(b, nz, (const double2*)v[0].dev, (const double2*)v[1].dev, fi, (double2*)v[2].dev,
                         precision, st);
    if (rc == GNK_OK && v[2].tmp) {
        if (cudaMemcpyAsync(v[2].user, v[2].dev, v[2].bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("gnk_cauchy_eval: %s", cudaGetErrorString(cudaGetLastError()));
            rc = GNK_ECUDA;
        }
    }
    if (rc != GNK_OK) cudaStreamSynchronize(st);
    for (int k = 0; k < 3; ++k)
        if (v[k].tmp) pool_free(v[k].dev, st);
    return rc;
}

// Device views of the arrays of one call (host arrays staged through temporary
// device buffers); outputs are copied back by finish().
struct Views {
    DevArr v[8];
    int n = 0;
    int add(const void* p, size_t bytes, bool input, cudaStream_t st, void** dev) {
        const int rc = dev_view(p, bytes, input, st, &v[n]);
        if (rc == GNK_OK) *dev = v[n].dev;
        ++n;
        return rc;
    }
    int finish(int rc, const bool* is_out, cudaStream_t st) {
        if (rc == GNK_OK)
            for (int k = 0; k < n; ++k)
                if (is_out[k] && v[k].tmp &&
                    cudaMemcpyAsync(v[k].user, v[k].dev, v[k].bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
                    set_error("%s", cudaGetErrorString(cudaGetLastError()));
                    rc = GNK_ECUDA;
                }
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == GNK_OK) {
            set_error("%s", cudaGetErrorString(cudaGetLastError()));
            rc = GNK_ECUDA;
        }
        for (int k = 0; k < n; ++k)
            if (v[k].tmp) pool_free(v[k].dev, st);
        return rc;
    }
};

int gnk_slit_map_data(int m1, int n, const double* et, const double* alpha, const double* theta, int bounded,
                      double* A, double* gam, void* stream) {
    cudaGetLastError();
    if (!et || !alpha || !theta || !A || !gam || m1 < 1 || n < 4 || (n % 2) != 0 ||
        (long long)m1 * n > (1LL << 28)) {
        set_error("gnk_slit_map_data: NULL array or m1, n out of range");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)m1 * n;
    Views vw;
    void *det, *dth, *dA, *dg;
    int rc = vw.add(et, 16 * N, true, st, &det);
    if (rc == GNK_OK) rc = vw.add(theta, 8 * (size_t)m1, true, st, &dth);
    if (rc == GNK_OK) rc = vw.add(A, 16 * N, false, st, &dA);
    if (rc == GNK_OK) rc = vw.add(gam, 8 * N, false, st, &dg);
    if (rc == GNK_OK)
        rc = slit_data(m1, n, (const double2*)det, make_double2(alpha[0], alpha[1]), (const double*)dth, bounded,
                       (double2*)dA, (double*)dg, st);
    const bool out[4] = {false, false, true, true};
    return vw.finish(rc, out, st);
}

int gnk_slit_map(const gnk_boundary* hd, const double* alpha, const double* gam, const double* mu,
                 const double* h, const double* hk, double* w, void* stream) {
    cudaGetLastError();
    GNK_TRY(check_handle(hd));
    const Boundary& b = hd->b;
    if (!alpha || !gam || !mu || !h || !hk || !w) {
        set_error("gnk_slit_map: NULL array");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = b.N;
    Views vw;
    void *dg, *dmu, *dh, *dhk, *dw;
    int rc = vw.add(gam, 8 * N, true, st, &dg);
    if (rc == GNK_OK) rc = vw.add(mu, 8 * N, true, st, &dmu);
    if (rc == GNK_OK) rc = vw.add(h, 8 * N, true, st, &dh);
    if (rc == GNK_OK) rc = vw.add(hk, 8 * (size_t)b.m1, true, st, &dhk);
    if (rc == GNK_OK) rc = vw.add(w, 16 * N, false, st, &dw);
    if (rc == GNK_OK) rc = slit_nodes_f(b, (const double*)dg, (const double*)dmu, (const double*)dh, b.zbuf, st);
    if (rc == GNK_OK)
        rc = slit_w(b.et, b.zbuf, b.N, make_double2(alpha[0], alpha[1]), (const double*)dhk, b.bounded,
                    (double2*)dw, st);
    const bool out[5] = {false, false, false, false, true};
    return vw.finish(rc, out, st);
}

int gnk_slit_map_eval(const gnk_boundary* hd, const double* alpha, const double* gam, const double* mu,
                      const double* h, const double* hk, int nz, const double* z, double* wz, int precision,
                      void* stream) {
    cudaGetLastError();
    GNK_TRY(check_handle(hd));
    const Boundary& b = hd->b;
    if (precision != GNK_PREC_FP64 && precision != GNK_PREC_DF32) {
        set_error("gnk_slit_map_eval: precision must be GNK_PREC_FP64 or GNK_PREC_DF32, got %d", precision);
        return GNK_EINVAL;
    }
    if (nz < 0) {
        set_error("gnk_slit_map_eval: nz < 0");
        return GNK_EINVAL;
    }
    if (nz == 0) return GNK_OK;
    if (!alpha || !gam || !mu || !h || !hk || !z || !wz) {
        set_error("gnk_slit_map_eval: NULL array");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = b.N;
    Views vw;
    void *dg, *dmu, *dh, *dhk, *dz, *dw;
    int rc = vw.add(gam, 8 * N, true, st, &dg);
    if (rc == GNK_OK) rc = vw.add(mu, 8 * N, true, st, &dmu);
    if (rc == GNK_OK) rc = vw.add(h, 8 * N, true, st, &dh);
    if (rc == GNK_OK) rc = vw.add(hk, 8 * (size_t)b.m1, true, st, &dhk);
    if (rc == GNK_OK) rc = vw.add(z, 16 * (size_t)nz, true, st, &dz);
    if (rc == GNK_OK) rc = vw.add(wz, 16 * (size_t)nz, false, st, &dw);
    const double2 al = make_double2(alpha[0], alpha[1]);
    if (rc == GNK_OK) rc = slit_nodes_f(b, (const double*)dg, (const double*)dmu, (const double*)dh, b.zbuf, st);
    // f(z) by the Cauchy formula into wz, then w(z) in place
    if (rc == GNK_OK)
        rc = cauchy_eval(b, nz, (const double2*)dz, b.zbuf, make_double2(0.0, 0.0), (double2*)dw, precision, st);
    if (rc == GNK_OK)
        rc = slit_w((const double2*)dz, (const double2*)dw, nz, al, (const double*)dhk, b.bounded, (double2*)dw, st);
    const bool out[6] = {false, false, false, false, false, true};
    return vw.finish(rc, out, st);
}

int gnk_slit_map_adjoint_data(int m1, int n, const double* etp, const double* theta, int bounded, double* Ap,
                              void* stream) {
    cudaGetLastError();
    if (!etp || !theta || !Ap || m1 < 1 || n < 4 || (n % 2) != 0 || (long long)m1 * n > (1LL << 28)) {
        set_error("gnk_slit_map_adjoint_data: NULL array or m1, n out of range");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)m1 * n;
    Views vw;
    void *detp, *dth, *dAp;
    int rc = vw.add(etp, 16 * N, true, st, &detp);
    if (rc == GNK_OK) rc = vw.add(theta, 8 * (size_t)m1, true, st, &dth);
    if (rc == GNK_OK) rc = vw.add(Ap, 16 * N, false, st, &dAp);
    if (rc == GNK_OK)
        rc = slit_dA(m1, n, (const double2*)detp, (const double*)dth, bounded, (double2*)dAp, st);
    const bool out[3] = {false, false, true};
    return vw.finish(rc, out, st);
}

int gnk_slit_map_adjoint(const gnk_boundary* hd, const double* alpha, const double* theta, const gnk_options* opt,
                         double* w, double* omega, double* psi, double* params, gnk_result* info, void* stream) {
    cudaGetLastError();
    GNK_TRY(check_handle(hd));
    const Boundary& b = hd->b;
    if (!alpha || !theta || !w) {
        set_error("gnk_slit_map_adjoint: NULL array");
        return GNK_EINVAL;
    }
    if (!b.has_adjoint) {
        set_error("gnk_slit_map_adjoint needs a handle built with eta'' and A'");
        return GNK_EINVAL;
    }
    gnk_options o;
    GNK_TRY(options_from(opt, &o));
    cudaStream_t st = (cudaStream_t)stream;
    // theta is read on the host: each boundary is a circular (pi/2) or a radial
    // (0) slit, and the outer boundary of bounded G maps to the unit circle
    std::vector<double> th(b.m1);
    if (is_device_ptr(theta)) {
        GNK_TRY_CUDA(cudaMemcpyAsync(th.data(), theta, th.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        GNK_TRY_CUDA(cudaStreamSynchronize(st));
    } else {
        std::memcpy(th.data(), theta, th.size() * sizeof(double));
    }
    for (int k = 0; k < b.m1; ++k) {
        if (th[k] != 0.5 * M_PI && th[k] != 0.0) {
            set_error("gnk_slit_map_adjoint: theta[%d] = %g is neither pi/2 nor 0", k, th[k]);
            return GNK_EINVAL;
        }
    }
    if (b.bounded && th[0] != 0.5 * M_PI) {
        set_error("gnk_slit_map_adjoint: the outer boundary of a bounded domain needs theta = pi/2");
        return GNK_EINVAL;
    }
    const TileOverride tile(b, o.tile_chunks);
    GNK_TRY(ensure_eone(b, st));
    const size_t N = b.N;
    Views vw;
    bool out[5];
    void *dth, *dw, *dom = nullptr, *dpsi = nullptr, *dpar = nullptr;
    int rc = vw.add(theta, 8 * (size_t)b.m1, true, st, &dth);
    out[0] = false;
    if (rc == GNK_OK) rc = vw.add(w, 16 * N, false, st, &dw);
    out[1] = true;
    int k = 2;
    if (rc == GNK_OK && omega) {
        rc = vw.add(omega, 16 * N, false, st, &dom);
        out[k++] = true;
    }
    if (rc == GNK_OK && psi) {
        rc = vw.add(psi, 8 * N, false, st, &dpsi);
        out[k++] = true;
    }
    if (rc == GNK_OK && params) {
        rc = vw.add(params, 8 * ((size_t)b.m1 + 1), false, st, &dpar);
        out[k++] = true;
    }
    int s = rc;
    if (rc == GNK_OK)
        s = slit_map_adjoint(b, make_double2(alpha[0], alpha[1]), (const double*)dth, o, (double2*)dw,
                             (double2*)dom, (double*)dpsi, (double*)dpar, info, st);
    // the outputs of a call whose solves stopped at maxit are still copied back
    const int rcf = (s == GNK_ENOTCONV) ? GNK_OK : s;
    const int fin = vw.finish(rcf, out, st);
    if (fin != rcf) return fin;  // a CUDA failure while copying back
    if (s == GNK_ENOTCONV) set_error("GMRES did not reach tol within maxit cycles in one of the solves");
    if (s == GNK_ENONFINITE) set_error("non-finite value in the GMRES iteration");
    return s;
}

int gnk_slit_map_adjoint_eval(const gnk_boundary* hd, const double* alpha, const double* omega, int nz,
                              const double* z, double* wz, int precision, void* stream) {
    cudaGetLastError();
    GNK_TRY(check_handle(hd));
    const Boundary& b = hd->b;
    if (precision != GNK_PREC_FP64 && precision != GNK_PREC_DF32) {
        set_error("gnk_slit_map_adjoint_eval: precision must be GNK_PREC_FP64 or GNK_PREC_DF32, got %d",
                  precision);
        return GNK_EINVAL;
    }
    if (nz < 0) {
        set_error("gnk_slit_map_adjoint_eval: nz < 0");
        return GNK_EINVAL;
    }
    if (nz == 0) return GNK_OK;
    if (!alpha || !omega || !z || !wz) {
        set_error("gnk_slit_map_adjoint_eval: NULL array");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Views vw;
    void *dom, *dz, *dw;
    int rc = vw.add(omega, 16 * (size_t)b.N, true, st, &dom);
    if (rc == GNK_OK) rc = vw.add(z, 16 * (size_t)nz, true, st, &dz);
    if (rc == GNK_OK) rc = vw.add(wz, 16 * (size_t)nz, false, st, &dw);
    // omega(z) by the Cauchy formula (omega(inf) = 0 for unbounded G) into wz,
    // then w = (z - alpha) exp(omega) in place
    if (rc == GNK_OK)
        rc = cauchy_eval(b, nz, (const double2*)dz, (const double2*)dom, make_double2(0.0, 0.0), (double2*)dw,
                         precision, st);
    if (rc == GNK_OK)
        rc = slit_w((const double2*)dz, (const double2*)dw, nz, make_double2(alpha[0], alpha[1]), nullptr, 0,
                    (double2*)dw, st);
    const bool out[3] = {false, false, true};
    return vw.finish(rc, out, st);
}

int gnk_compute_h(const gnk_boundary* h, const double* mu, const double* gam, double* hv, double* hk,
                  void* stream) {
    GNK_TRY(check_handle(h));
    if (!mu || !gam || !hv) {
        set_error("NULL array");
        return GNK_EINVAL;
    }
    const Boundary& b = h->b;
    cudaStream_t st = (cudaStream_t)stream;
    GNK_TRY(ensure_eone(b, st));
    const double *dmu, *dg;
    GNK_TRY(stage_in(b, mu, b.N, 0, st, &dmu));
    GNK_TRY(stage_in(b, gam, b.N, 1, st, &dg));
    Out o_h = stage_out(b, hv, b.N, 2);
    GNK_TRY(op_h(b, dmu, dg, o_h.dev, st));
    if (hk) {
        Out o_k = stage_out(b, hk, b.m1, 3);
        GNK_TRY(run_component_means(b, o_h.dev, o_k.dev, st));
        GNK_TRY(finish_out(o_k, st));
    }
    return finish_out(o_h, st);
}

}  // extern "C"
