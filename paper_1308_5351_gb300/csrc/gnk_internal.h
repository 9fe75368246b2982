// Internal declarations of libgnk (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/gnk.h"

namespace gnk {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define GNK_TRY_CUDA(call)                                                     \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            ::gnk::set_error("%s failed: %s (%s:%d)", #call,                    \
                             cudaGetErrorString(e_), __FILE__, __LINE__);      \
            return GNK_ECUDA;                                                  \
        }                                                                      \
    } while (0)

#define GNK_TRY(call)                                                          \
    do {                                                                       \
        int s_ = (call);                                                       \
        if (s_ != GNK_OK) return s_;                                           \
    } while (0)

// ---------------------------------------------------------------- launch counter
// Host-side count of kernel launches made by the library (all devices).
void count_launches(unsigned long long n);
// While on (calling thread), launches are not counted: used while a stream is
// captured into a graph, whose replays are counted instead.
void count_suppress(bool on);

// ---------------------------------------------------------------- device memory
// From a per-device stream-ordered pool that keeps freed memory (mem.cu):
// allocation and free are ordered on st and never synchronise the device.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
cudaError_t pool_free(void* p, cudaStream_t st);

// ---------------------------------------------------------------- profiling
// Kinds of instrumented launches (gnk_profile_query's `kind`).
enum ProfKind : int {
    PK_PAIR64 = 0,   // FP64 pair-sum kernel; work = pair evaluations (R N (N-1))
    PK_PAIR32 = 1,   // FP32 pair-sum kernel; work = pair evaluations
    PK_REDUCE = 2,   // chunk reduction + epilogue; work = bytes moved
    PK_CIRC = 3,     // circulant FFT / direct kernel; work = bytes moved
    PK_KRYLOV = 4,   // GMRES vector kernels; work = bytes moved
    PK_OTHER = 5,
    PK_PAIRDF = 6,   // double-float pair-sum kernel; work = pair evaluations
    PK_FMM = 7,      // FMM M2L; work = the R N (N-1) pairs the product stands for
    PK_FMMNEAR = 8,  // FMM near field (double-float); work = near-field pair evaluations
    PK_FMML2P = 9,   // FMM L2P and the sum with the near field
    PK_FMMUP = 10,   // FMM upward pass (P2M and the M2M chain)
    PK_FMML2L = 11,  // FMM L2L per leaf
};
struct ProfToken {
    void* ev = nullptr;
};
// kind >= 0: nothing is recorded while that kind is masked out (gnk_profile_mask)
ProfToken prof_begin(cudaStream_t st, int kind = -1);
// `instr`: algorithmic instructions of the launch on its limiting pipe
// (FP32 pipe for the FP32 and double-float pair kernels, FP64 pipe for the FP64 one).
long prof_end(const ProfToken& t, int kind, double work, cudaStream_t st, double instr = 0.0,
              double bytes = 0.0);
void prof_skip(long idx);
// Collect the record indices of the launches made between begin and end
// (calling thread only), to mark launches that a device flag turned into
// no-ops after the fact.
void prof_collect_begin();
void prof_collect_end(std::vector<long>* out);

// ---------------------------------------------------------------- tiling
// Sources per shared-memory tile of the pair-sum kernels.
constexpr int kSrcTile64 = 128;   // FP64 kernel
constexpr int kSrcTile32 = 256;   // FP32 kernel (also the tile of the FP32 reference points)
constexpr int kThreads64 = 128;   // threads per block, FP64 kernel
constexpr int kTargets64 = 2;     // targets per thread, FP64 kernel
constexpr int kThreads32 = 256;   // threads per block, FP32 kernel
constexpr int kTargets32 = 4;     // targets per thread, FP32 kernel
constexpr int kThreadsDF = 256;   // threads per block, double-float kernel
constexpr int kTargetsDF = 2;     // targets per thread, double-float kernel
constexpr int kMaxRHS = 2;        // right-hand sides per pair-sum launch

// How the sources' complex weights are formed when a source tile is loaded.
enum WeightMode : int {
    W_COMPLEX = 0,   // w_j given (complex)
    W_SCALED = 1,    // w_j = s_j * x_j, s complex, x real
};

// Pointwise epilogues applied after the partial sums are reduced; they
// implement the operators of Secs. 3 and 4 around z = E w.
enum Epilogue : int {
    EPI_Z = 0,        // out_c = z
    EPI_IMINUSN = 1,  // out = 2x + b1 x + (2/n) Im(A z)                 (f_B)
    EPI_M = 2,        // out = -(2/n) Re(A z) - d1 x + Lx               (f_C)
    EPI_ADJ = 3,      // out = e x + (2/n) Im(q z) + mean_k(x)           (g_B)
    EPI_RESID = 4,    // out = rhs - f_B(x)
    EPI_RESID_ADJ = 5,// out = rhs - g_B(x)
    EPI_H = 6,        // out = (f_C(mu) - f_B(gam)) / 2, z = E(q mu), z2 = E(q gam)
    EPI_EONE = 7,     // b1 = -(2/n) Im(A z), d1 = -(2/n) Re(A z); if R=2: e from z2
    EPI_RHS_FB = 8,   // out = -f_C(x) (the right-hand side -y), out2 = f_B(x)
    EPI_RESID_FC = 9, // out = rhs - f_B(x), out2 = f_C(x)
    EPI_IMINUSN_T = 10,  // out = (2I + diag(B1) - B)^T x, z = E(A x)
    EPI_RESID_T = 11,    // out = rhs - (2I + diag(B1) - B)^T x
    EPI_MT = 12,         // out = (D - diag(D1) + Lhat)^T x, z = E(A x), Lx = Lhat x
    EPI_EONE_RHS = 13,   // z0 = E q, z1 = E(q gamma): Eone, diag(B1), diag(D1), -y, f_B(gamma)
};

// Operators a GMRES solve can use.
enum OpId : int {
    OP_K = 0,    // 2I + diag(B1) - B        (discrete I - N, Eq. sys)
    OP_ADJ = 1,  // diag(e) + B^T + Phat     (discrete I + N* + J, Eq. sys*)
    OP_KT = 2,   // (2I + diag(B1) - B)^T    (transposed system of the gradient)
};

struct PairPlan {
    int tiles_tgt = 0;     // target tiles (blocks along x)
    int tiles_src = 0;     // source tiles
    int chunks = 1;        // source chunks (blocks along y)
    int tiles_per_chunk = 0;
};

// Everything a launch of the pair-sum + reduce pipeline needs.
struct PairJob {
    int R = 1;                    // right-hand sides
    int mode = W_SCALED;
    const double2* w[kMaxRHS] = {nullptr, nullptr};   // W_COMPLEX
    const double* x[kMaxRHS] = {nullptr, nullptr};    // W_SCALED
    const double2* s = nullptr;                        // W_SCALED scale (q or A)
    int epi = EPI_Z;
    double2* out_c = nullptr;     // EPI_Z: complex output(s), R x N
    double* out = nullptr;        // real output
    double* out2 = nullptr;       // EPI_EONE: second real output
    double* out3 = nullptr;       // EPI_EONE: third real output (e)
    const double* ex = nullptr;   // epilogue x (the vector the operator acts on)
    const double* ex2 = nullptr;  // EPI_H: gamma
    const double* rhs = nullptr;  // EPI_RESID*
    const double* Lx = nullptr;   // EPI_M / EPI_H: Lhat x
    const double* means = nullptr;// EPI_ADJ: per-component means of x
    const int* done = nullptr;    // skip the whole job if *done != 0
    int comp = 0;                 // set by run_pairsum: 0 both parts, 1 only Im z, 2 only Re z
};

struct FmmTree;  // fmm.cu

// ---------------------------------------------------------------- handle
struct Boundary {
    int m1 = 0, n = 0, N = 0;
    int bounded = 0;
    int has_adjoint = 0;
    int device = 0;
    int sms = 0;

    // FP64 geometry and precomputed diagonals (device)
    double2* et = nullptr;
    double2* etp = nullptr;
    double2* A = nullptr;
    double2* q = nullptr;       // eta'/A
    double2* Eone = nullptr;    // E q
    double* b1 = nullptr;       // diag(B 1)
    double* d1 = nullptr;       // diag(D 1)
    double* e = nullptr;        // adjoint diagonal (nullptr without eta'')

    // FP32 geometry: positions relative to one reference node per source tile
    float4* ref32 = nullptr;    // per source tile: (hi.x, hi.y, lo.x, lo.y) of the reference
    float2* off32 = nullptr;    // per node: eta_j - ref(tile(j)), rounded to FP32
    float4* et32 = nullptr;     // per node: hi/lo split of eta (hi.x, hi.y, lo.x, lo.y)
    float2* q32 = nullptr;
    float2* A32 = nullptr;
    // double-float geometry: FP64 reference node per source tile, df32 offsets
    double2* ref64 = nullptr;   // per source tile
    float4* offdf = nullptr;    // per node: (dx.h, dy.h, dx.l, dy.l)

    // circulant part
    int fft_pow2 = 0;           // n is a power of two
    double2* twiddle = nullptr; // exp(-2 pi i k / n), k < n/2
    double* Lcol = nullptr;     // first column of L (direct product fallback)

    // workspace
    void* partial = nullptr;    // split-source partial sums
    size_t partial_bytes = 0;
    // source-chunk override of the direct pair kernels for the current call
    // (gnk_options.tile_chunks; 0: the plans below) and the larger partial-sum
    // workspace it may need (from the memory pool, kept until the handle is freed)
    mutable int tile_chunks = 0;
    mutable void* partial_x = nullptr;
    mutable size_t partial_x_bytes = 0;
    double2* zbuf = nullptr;    // complex scratch, kMaxRHS x N
    double* r0 = nullptr;       // real scratch vectors (N each)
    double* r1 = nullptr;
    double* r2 = nullptr;
    double* r3 = nullptr;
    double* r4 = nullptr;
    double* r5 = nullptr;
    double* r6 = nullptr;
    double* ones = nullptr;     // N ones (weights q = q * 1)
    int* flag = nullptr;        // input checks of the geometry preparation
    void* arena = nullptr;      // the one allocation that holds the buffers above
    int eone_pending = 0;       // Eone, diag(B1), diag(D1), e not yet formed
    int plain = 0;              // 1: diagonals of the form without singularity subtraction
    int A_real = 0;             // 1: Im A = 0 at every node (then f_B needs only Im E(qx))
    FmmTree* fmm = nullptr;     // quadtree and expansions, built on the first FMM product
    int df_scalar = 0;          // 1: scalar double-float kernel instead of the packed one
    int f32_scalar = 0;         // 1: scalar FP32 kernel instead of the packed one
    double* means = nullptr;    // m1
    double* stage = nullptr;    // host-staging buffers: 4 x 2N doubles
    PairPlan plan64, plan32, plandf;
    int eone_prec = GNK_PREC_FP64;  // arithmetic of the precomputed sums

    // Krylov workspace (allocated on first solve, grown as needed)
    double* V = nullptr;        // (restart+1) x N
    int V_cols = 0;
    double* kry = nullptr;      // small dense state (H, g, cs, sn, y, partials)
    size_t kry_bytes = 0;
    void* kstate = nullptr;     // device KrylovState
};

// ---------------------------------------------------------------- pair sums
PairPlan make_plan(int N, int sms, int blocks_per_sm, int targets_per_block, int src_tile);
int pair_workspace_bytes(const Boundary& b, size_t* bytes);
int run_pairsum64(const Boundary& b, const PairJob& job, cudaStream_t st);
int run_pairsum32(const Boundary& b, const PairJob& job, cudaStream_t st);
int run_pairsumdf(const Boundary& b, const PairJob& job, cudaStream_t st);
int run_pairsum(const Boundary& b, const PairJob& job, int precision, cudaStream_t st);
// 0: both parts of z = E(q x) are read by the job's epilogue; 1: only Im z; 2: only Re z
int pair_component_needed(const Boundary& b, const PairJob& job);
int pair_blocks_per_sm(int precision);

// ---------------------------------------------------------------- circulant / pointwise
int run_circulant(const Boundary& b, const double* x, double* y, cudaStream_t st);
int run_component_means(const Boundary& b, const double* x, double* means, cudaStream_t st);
int run_prepare_geometry(Boundary& b, const double* etpp, const double* Ap, int* d_flag,
                         cudaStream_t st);
int run_prepare_nodes(Boundary& b, const double* etpp, const double* Ap, int* d_flag, cudaStream_t st);
void circulant_tables(int n, std::vector<double2>* tw, std::vector<double>* col);
int run_batch_circulant(const int4* desc, const long long* base, int nblocks, int nmax,
                        const double* x, double* y, const double2* tw, const double* col, cudaStream_t st);

// ---------------------------------------------------------------- operators (ops.cu)
int op_IminusN(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
               const int* done = nullptr);
int op_M(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st);
int op_adjoint(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
               const int* done = nullptr);
int op_resid(const Boundary& b, int op, const double* rhs, const double* x, double* r,
             int prec, cudaStream_t st, double* fc_out = nullptr);
int op_IminusN_T(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
                 const int* done = nullptr);
int op_MT(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st);
int op_rhs_fb(const Boundary& b, const double* gam, double* rhs, double* fb, int prec,
              cudaStream_t st);
int op_half_diff(const double* a, const double* b, double* out, int N, cudaStream_t st);
// Forms Eone, diag(B1), diag(D1) (and e) if the handle deferred them.
int ensure_eone(const Boundary& b, cudaStream_t st);
// Deferred handles: Eone and the first right-hand side in one two-RHS launch.
int op_eone_rhs_fb(const Boundary& b, const double* gam, double* rhs, double* fb, int prec,
                   cudaStream_t st);
int op_h(const Boundary& b, const double* mu, const double* gam, double* h, cudaStream_t st);
int op_negate(double* x, int N, cudaStream_t st);

// ---------------------------------------------------------------- Krylov (krylov.cu)
// Solves with operator `op` (OpId).  When
// fc_out is given, the last true residual also writes f_C(x) of the returned
// x there and *fc_valid is set (f_C(mu) is the first half of h, Eq. bh).
int solve(const Boundary& b, int op, const double* rhs, double* x,
          const gnk_options& opt, gnk_result* info, cudaStream_t st,
          double* fc_out = nullptr, int* fc_valid = nullptr);
// Arithmetic of the outer (refinement) products for a solve precision.
int outer_precision(int solve_precision);
// Test hook behind gnk_debug_barrier_fault.
int debug_barrier_fault(int skip_block, int spin_limit);

// ---------------------------------------------------------------- gradients (grad.cu)
// gh: dL/dh at the nodes; ghk (nullable): dL/dh_k of the component means.
int fbie_backward(const Boundary& b, const double* mu, const double* gam, const double* gm,
                  const double* gh, const double* ghk, double2* g_et, double2* g_etp, double2* g_A,
                  double* g_gam, const gnk_options& opt, gnk_result* info, cudaStream_t st);
int fbie_backward_nodes(Boundary& b, const double* mu, const double* gam, const double* gm,
                        const double* gh, double2* g_et, double2* g_etp, double2* g_A, double* g_gam,
                        const gnk_options& opt, gnk_result* info, cudaStream_t st);

// ---------------------------------------------------------------- FMM (fmm.cu)
int run_fmm(const Boundary& b, const PairJob& job, cudaStream_t st);
int run_fmm_ef(const Boundary& b, const double2* w0, const double2* w1, double2* E, double2* F, cudaStream_t st);
int ensure_fmm(const Boundary& b, int R, cudaStream_t st);
int fmm_start_near_cache(const Boundary& b, cudaStream_t st);
void release_fmm(Boundary& b);
double fmm_instr(const Boundary& b, int R, int which);
double fmm_near_instr(const Boundary& b, int R);
// Device word set by an FMM kernel whose bounded wait gave up (null before the tree).
const int* fmm_fault_word(const Boundary& b);
// the chunk reduction and epilogue of the pair sums, for products formed elsewhere
cudaError_t launch_reduce_public(const Boundary& b, const PairJob& job, int chunks, int ptype,
                                 cudaStream_t st);

// ---------------------------------------------------------------- slit maps (slitmap.cu)
int slit_data(int m1, int n, const double2* et, double2 alpha, const double* theta, int bounded, double2* A,
              double* gam, cudaStream_t st);
int slit_nodes_f(const Boundary& b, const double* gam, const double* mu, const double* h, double2* f,
                 cudaStream_t st);
int slit_w(const double2* z, const double2* f, int M, double2 alpha, const double* hk, int bounded, double2* w,
           cudaStream_t st);
// the adjoint route (slitmap_adj.cu): A' of the slit map's A, and the whole
// route on a handle built with that A and A' (theta on the device, each pi/2 or 0)
int slit_dA(int m1, int n, const double2* etp, const double* theta, int bounded, double2* Ap, cudaStream_t st);
int slit_map_adjoint(const Boundary& b, double2 alpha, const double* theta, const gnk_options& opt, double2* w,
                     double2* omega, double* psi_out, double* params, gnk_result* info, cudaStream_t st);

// ---------------------------------------------------------------- Cauchy formula (cauchy_eval.cu)
int cauchy_eval(const Boundary& b, int M, const double2* z, const double2* f, double2 finf, double2* out,
                int precision, cudaStream_t st);

}  // namespace gnk

struct gnk_boundary {
    gnk::Boundary b;
};
