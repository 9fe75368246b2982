// Restarted GMRES (Sec. 3.5, Eq. ie-gmres; Sec. 4.5, Eq. ie*-gmres) with
// every Arnoldi, Givens and convergence step on the device, and FP64
// iterative refinement around an FP32-operator GMRES for GNK_PREC_MIXED.
//
// Semantics follow MATLAB's gmres(A, b, restart, tol, maxit) as used by the
// paper: x0 = 0, no preconditioner, cycles of at most `restart` Arnoldi
// steps, at most `maxit` cycles, stop when ||b - A x||_2 <= tol ||b||_2 with
// the residual recomputed from x at the start of every cycle.
//
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): each pass
// is one multi-dot and one update over the basis instead of j dependent
// passes.  A whole Arnoldi step (both passes, the norm, the Givens update and
// the scaling of the new basis vector) is one cooperative launch whose blocks
// meet at two bounded grid barriers (the new norm follows from the second
// pass by Pythagoras unless it cancels, then a third): in double-float on the
// FP32 pipe from shared memory (k_arnoldi_df) for every operator precision but
// plain FP64, in FP64 (k_arnoldi) for that one.  The norms at the start of a
// cycle finish in the last block to arrive (atomic ticket + fence, no spinning).
// Partial sums are added in a fixed order, so results are reproducible.
// Inside a cycle every kernel first reads the device flag `done`, so the host
// enqueues a whole cycle without waiting and synchronises once per cycle.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "gnk_internal.h"
#include "pairmath.cuh"
#include "tma.cuh"

namespace gnk {
namespace {

struct KState {
    double bnorm;     // ||b||
    double beta;      // ||r|| at the start of the current cycle
    double tol;       // relative tolerance
    double est;       // Givens residual estimate |g_{k}|
    double hnext;     // h_{j+1,j} of the last step (before rotation)
    int k;            // Arnoldi steps completed in the current cycle
    int last_k;       // steps of the previous cycle
    int done;         // the current cycle has finished
    int nonfinite;    // a NaN/Inf was met
    int restart;
    unsigned counter; // last-block ticket
    int bar_err;      // a grid barrier wait gave up
    int bar_limit;    // polls before a grid barrier wait gives up
    int bar_skip;     // test hook: this block never arrives at a barrier (-1: none)
    // grid barrier of the Arnoldi step: arrivals and generation on cache lines
    // of their own, away from the fields above and from each other
    alignas(128) unsigned bar_count;
    alignas(128) unsigned bar_gen;
    char pad_[124];
};

constexpr int KT = 256;       // threads per block of the vector kernels
constexpr int KB_MAX = 256;   // maximum blocks of the vector kernels

struct KPtrs {
    double* H;     // (restart+1) x restart, column-major, ld = restart+1
    double* g;     // restart+1
    double* cs;    // restart
    double* sn;    // restart
    double* h1;    // restart+1
    double* h2;    // restart+1
    double* y;     // restart
    double* part;  // KB_MAX x ld
    int ld;
};

size_t kry_doubles(int restart) {
    const size_t ld = restart + 1;
    return ld * restart + ld + 2 * (size_t)restart + 2 * ld + restart + 2 * KB_MAX * ld;
}

KPtrs kry_ptrs(double* base, int restart) {
    KPtrs p;
    p.ld = restart + 1;
    p.H = base;
    p.g = p.H + (size_t)p.ld * restart;
    p.cs = p.g + p.ld;
    p.sn = p.cs + restart;
    p.h1 = p.sn + restart;
    p.h2 = p.h1 + p.ld;
    p.y = p.h2 + p.ld;
    p.part = p.y + restart;  // two regions of KB_MAX x ld
    return p;
}

int vec_blocks(int N) {
    const int b = (N + KT - 1) / KT;
    return b < 1 ? 1 : (b > KB_MAX ? KB_MAX : b);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < KT / 32; ++w) s += red[w];
    return s;  // valid in thread 0
}

// sum_{b < nb} part[b * stride] over all threads of the (last) block, in a fixed
// order: thread t adds b = t, t + KT, ...; then the block tree.  Valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part, size_t stride, int nb, double* red) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += KT) t += part[(size_t)b * stride];
    return block_sum(t, red);
}

// True in every thread of the last block to finish writing its partials.
__device__ __forceinline__ bool arrive_last(unsigned* counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return last;
}

// ||x||^2 partials -> last block: mode 0 stores bnorm; mode 1 starts a cycle.
__global__ void __launch_bounds__(KT) k_norm(const double* __restrict__ x, int N, KPtrs p,
                                             KState* s, int mode) {
    __shared__ double red[KT / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * KT + threadIdx.x; i < N; i += gridDim.x * KT) acc = fma(x[i], x[i], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) p.part[blockIdx.x] = acc;
    if (!arrive_last(&s->counter)) return;
    const double t = sum_partials(p.part, 1, gridDim.x, red);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(t);
        if (mode == 0) {
            s->bnorm = nrm;
        } else {
            s->beta = nrm;
            s->est = nrm;
            s->last_k = s->k;
            s->k = 0;
            if (!isfinite(nrm)) s->nonfinite = 1;
            s->done = (!(nrm > s->tol * s->bnorm)) ? 1 : 0;  // also stops on NaN
            p.g[0] = nrm;
            for (int k = 1; k <= s->restart; ++k) p.g[k] = 0.0;
        }
        s->counter = 0;
    }
}

// v0 = r / beta (and its double-float copy when vd0 is given)
__global__ void __launch_bounds__(KT) k_scale_first(const double* __restrict__ r, double* __restrict__ v0,
                                                    float2* __restrict__ vd0, int N, const KState* s) {
    if (s->done) return;
    const double inv = 1.0 / s->beta;
    for (int i = blockIdx.x * KT + threadIdx.x; i < N; i += gridDim.x * KT) {
        const double v = r[i] * inv;
        v0[i] = v;
        if (vd0) {
            const df d = df_split_fast(v);
            vd0[i] = make_float2(d.h, d.l);
        }
    }
}

// dot products per pass over w in the Arnoldi step
constexpr int KD = 16;

// ---- one Arnoldi step in one cooperative launch.  After the product
// w = A v_j: the two CGS passes (multi-dot, update), ||w||, the Givens update
// of column j and v_{j+1} = w / h_{j+1,j}.  Each block takes a contiguous
// range of the vectors; the partial sums meet at grid barriers, after
// which every block adds them in the same fixed order (so all blocks hold
// the same coefficients without another barrier).  Block 0 does the Givens
// step.  The launch is cooperative, so all blocks are resident and every
// barrier is reached; the waits are bounded all the same, and one that gives
// up sets bar_err, which the host reports.
constexpr int kBarSpin = 1 << 20;

// The test hook (bar_skip, set only through gnk_debug_barrier_fault) makes one
// block pass every barrier without arriving, so that the others' bounded
// waits run out: the failure path is exercised without a fault.
__device__ __forceinline__ void grid_barrier(KState* s) {
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x != s->bar_skip) {
        volatile unsigned* gen = &s->bar_gen;
        const unsigned g = *gen;
        const int limit = s->bar_limit;
        __threadfence();
        if (atomicAdd(&s->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&s->bar_count, 0u);
            __threadfence();
            atomicAdd(&s->bar_gen, 1u);
        } else {
            for (int it = 0; *gen == g; ++it) {
                if (it >= limit || *(volatile int*)&s->bar_err) {
                    atomicExch(&s->bar_err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// dots of w with v_0 .. v_{nv-1} over [i0, i1), block sums to out[0 .. nv);
// with_norm: also w . w to out[nv].  The block sums take the fewest FP64
// additions (GB300's FP64 pipe has 2 lanes per SM, so shuffle trees, which
// add on all 32 lanes at every step, cost 5x more): every thread's partials
// go to shared memory (buf, KD x KT doubles), kn x 8 threads each add 32 of
// them (a stride-8 slice), then one thread per dot adds the 8 slices, all in
// a fixed order.
__device__ __forceinline__ void range_dots(const double* __restrict__ V, int N, int nv, const double* w,
                                           int i0, int i1, double* out, double (*red)[KD], double* buf,
                                           bool with_norm) {
    const int nt = nv + (with_norm ? 1 : 0);
    for (int k0 = 0; k0 < nt; k0 += KD) {
        const int kn = min(KD, nt - k0);
        double acc[KD];
#pragma unroll
        for (int q = 0; q < KD; ++q) acc[q] = 0.0;
        for (int i = i0 + threadIdx.x; i < i1; i += KT) {
            const double wi = w[i];
#pragma unroll
            for (int q = 0; q < KD; ++q)
                if (q < kn) acc[q] = fma((k0 + q < nv) ? V[(size_t)(k0 + q) * N + i] : wi, wi, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < KD; ++q)
            if (q < kn) buf[q * KT + threadIdx.x] = acc[q];
        __syncthreads();
        if (threadIdx.x < kn * 8) {
            const int q = threadIdx.x >> 3, part = threadIdx.x & 7;
            double t = 0.0;
#pragma unroll 8
            for (int e = 0; e < KT / 8; ++e) t += buf[q * KT + e * 8 + part];
            red[part][q] = t;
        }
        __syncthreads();
        if (threadIdx.x < kn) {
            double t = 0.0;
            for (int part = 0; part < 8; ++part) t += red[part][threadIdx.x];
            out[k0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// hs[k] = sum_b part[b * ld + k] over the nb blocks, k < nv: lane = coefficient,
// warp w adds its eighth of the blocks in order, then the warps' sums are added
// in warp order; read from L2 (the partials of other blocks)
__device__ __forceinline__ void reduce_coeffs(const double* part, int ld, int nv, int nb, double* hs,
                                              double (*red8)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = KT / 32;
    const int per = (nb + NW - 1) / NW, b0 = min(nb, wid * per), b1 = min(nb, b0 + per);
    for (int k0 = 0; k0 < nv; k0 += 32) {
        const int k = k0 + lane;
        double t = 0.0;
        if (k < nv) {
#pragma unroll 4
            for (int b = b0; b < b1; ++b) t += __ldcg(part + (size_t)b * ld + k);
        }
        red8[wid][lane] = t;
        __syncthreads();
        if (wid == 0 && k < nv) {
            double u = red8[0][lane];
            for (int ww = 1; ww < NW; ++ww) u += red8[ww][lane];
            hs[k] = u;
        }
        __syncthreads();
    }
}

// As reduce_coeffs, with every partial loaded at once (one round of
// independent L2 loads instead of a chain per warp) into `stage` (at least
// nb * nv doubles of shared memory), then summed per coefficient in a fixed
// order: 8 threads per coefficient each add a contiguous eighth of the blocks,
// then the eighths are added in order.  The result is the same in every block.
constexpr int kStage = 4096;  // doubles of the staging area
constexpr int kPool = KD * KT > 1025 + 2 * 1024 ? KD * KT : 1025 + 2 * 1024;
constexpr size_t kArnoldiDyn = (size_t)(kPool + kStage) * sizeof(double);  // dynamic shared bytes

__device__ __forceinline__ void reduce_coeffs_staged(const double* part, int ld, int nv, int nb, double* hs,
                                                     double* stage, double (*red8)[32]) {
    const int tot = nv * nb;
    for (int e = threadIdx.x; e < tot; e += KT) {  // e = b * nv + k
        const int b = e / nv, k = e - b * nv;
        stage[e] = __ldcg(part + (size_t)b * ld + k);
    }
    __syncthreads();
    const int per = (nb + 7) / 8;
    for (int k0 = 0; k0 < nv; k0 += KT / 8) {
        const int k = k0 + (threadIdx.x >> 3), slice = threadIdx.x & 7;
        double t = 0.0;
        if (k < nv) {
            const int b0 = min(nb, slice * per), b1 = min(nb, b0 + per);
            for (int b = b0; b < b1; ++b) t += stage[b * nv + k];
        }
        red8[slice][threadIdx.x >> 3] = t;  // red8 is [8][32]: slices x coefficients of this round
        __syncthreads();
        if (threadIdx.x < KT / 8 && k0 + (int)threadIdx.x < nv) {
            double u = red8[0][threadIdx.x];
            for (int sl = 1; sl < 8; ++sl) u += red8[sl][threadIdx.x];
            hs[k0 + threadIdx.x] = u;
        }
        __syncthreads();
    }
}

// Givens update of column j by block 0: the column h = h1 + h2 (in h1),
// h_{j+1,j} = hn and the previous rotations (staged in shared memory by
// givens_stage while the grid waits at its second barrier), one thread
// applies the rotations, and the column is stored in parallel.  Also
// the residual estimate and the end-of-cycle test (the triangular solve for y
// is k_solve_y's, once per cycle).
__device__ __forceinline__ void givens_stage(int j, double* scs, double* ssn, KPtrs p) {
    for (int k = threadIdx.x; k < j; k += blockDim.x) {
        scs[k] = p.cs[k];
        ssn[k] = p.sn[k];
    }
    if (threadIdx.x == 0) scs[1023] = p.g[j];  // g_j (scs holds at most j <= 1023 rotations before it)
}

__device__ void givens_step(int j, double hn, double* h1, const double* h2, const double* scs, const double* ssn,
                            KPtrs p, KState* s) {
    const int nv = j + 1;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) h1[k] = h1[k] + h2[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double* col = h1;
        col[j + 1] = hn;
        s->hnext = hn;
        for (int k = 0; k < j; ++k) {  // previous rotations
            const double a = col[k], b = col[k + 1];
            col[k] = scs[k] * a + ssn[k] * b;
            col[k + 1] = -ssn[k] * a + scs[k] * b;
        }
        const double a = col[j], b = col[j + 1];
        const double r = hypot(a, b);
        const double c = (r > 0.0) ? a / r : 1.0;
        const double sn = (r > 0.0) ? b / r : 0.0;
        p.cs[j] = c;
        p.sn[j] = sn;
        col[j] = r;
        col[j + 1] = 0.0;
        const double gj = p.g[j];
        p.g[j + 1] = -sn * gj;
        p.g[j] = c * gj;
        const double est = fabs(sn * gj);
        s->est = est;
        s->k = j + 1;
        const bool bad = !isfinite(est) || !isfinite(hn);
        if (bad) s->nonfinite = 1;
        if (bad || est <= s->tol * s->bnorm || j + 1 == s->restart || hn == 0.0) s->done = 1;
    }
    __syncthreads();
    double* colg = p.H + (size_t)j * p.ld;
    for (int k = threadIdx.x; k < j + 2; k += blockDim.x) colg[k] = h1[k];
}

// givens_step by warp 0 alone (no block barrier), so that the other warps of
// block 0 can update the block's range of the new basis vector meanwhile.  The
// previous rotations applied to the column x = h1 + h2 form the first-order
// recurrence z_0 = x_0, z_{k+1} = -s_k z_k + c_k x_{k+1} with outputs
// y_k = c_k z_k + s_k x_{k+1}: for j <= 32 it is evaluated as an inclusive scan
// of the affine maps z -> a z + b over the lanes (5 shuffle steps instead of
// j dependent steps of one thread on GB300's 2-lane FP64 pipe); longer cycles
// take the serial loop.  gj: g_j staged in shared memory.
__device__ void givens_step_warp0(int j, double hn, double* h1, const double* h2, const double* scs,
                                  const double* ssn, double gj, KPtrs p, KState* s) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;  // warp 0
    const int nv = j + 1;
    for (int k = lane; k < nv; k += 32) h1[k] = h1[k] + h2[k];
    __syncwarp();
    double zj;
    if (j <= 32) {
        const double x0 = h1[0];
        double a = 1.0, b = 0.0, ck = 1.0, sk = 0.0, xk1 = 0.0;
        if (lane < j) {
            ck = scs[lane];
            sk = ssn[lane];
            xk1 = h1[lane + 1];
            a = -sk;
            b = ck * xk1;
        }
        for (int o = 1; o < 32; o <<= 1) {  // (a, b) <- (a, b) o (ap, bp)
            const double ap = __shfl_up_sync(full, a, o), bp = __shfl_up_sync(full, b, o);
            if (lane >= o) {
                b = fma(a, bp, b);
                a *= ap;
            }
        }
        const double znext = fma(a, x0, b);                       // z_{lane+1}
        const double zprev = __shfl_up_sync(full, znext, 1);
        const double zcur = (lane == 0) ? x0 : zprev;             // z_lane
        __syncwarp();
        if (lane < j) h1[lane] = fma(ck, zcur, sk * xk1);         // y_lane
        zj = (j == 0) ? x0 : __shfl_sync(full, znext, j - 1);
    } else {
        if (lane == 0) {
            double* col = h1;
            for (int k = 0; k < j; ++k) {
                const double a = col[k], b = col[k + 1];
                col[k] = scs[k] * a + ssn[k] * b;
                col[k + 1] = -ssn[k] * a + scs[k] * b;
            }
        }
        __syncwarp();
        zj = h1[j];
    }
    __syncwarp();
    if (lane == 0) {
        double* col = h1;
        s->hnext = hn;
        const double r = sqrt(fma(zj, zj, hn * hn));
        const double inv = (r > 0.0) ? 1.0 / r : 0.0;
        const double c = (r > 0.0) ? zj * inv : 1.0;
        const double sn = (r > 0.0) ? hn * inv : 0.0;
        p.cs[j] = c;
        p.sn[j] = sn;
        col[j] = r;
        col[j + 1] = 0.0;
        p.g[j + 1] = -sn * gj;
        p.g[j] = c * gj;
        const double est = fabs(sn * gj);
        s->est = est;
        s->k = j + 1;
        const bool bad = !isfinite(est) || !isfinite(hn);
        if (bad) s->nonfinite = 1;
        if (bad || est <= s->tol * s->bnorm || j + 1 == s->restart || hn == 0.0) s->done = 1;
    }
    __syncwarp();
    double* colg = p.H + (size_t)j * p.ld;
    for (int k = lane; k < j + 2; k += 32) colg[k] = h1[k];
}

__global__ void __launch_bounds__(KT) k_arnoldi(const double* __restrict__ V, int N, int j, double* __restrict__ w,
                                                KPtrs p, KState* s) {
    if (s->done) return;  // set before this launch: the same in every block
    __shared__ double red[8][KD];
    __shared__ double red8[KT / 32][32];
    __shared__ double h1[1025];
    // dynamic: s_pool (h2, the Givens staging and, before they are used, the
    // dots' reduction buffer), then the staging area of the coefficient sums
    extern __shared__ double s_dyn[];
    double* s_pool = s_dyn;
    double* s_stage = s_dyn + kPool;
    double* h2 = s_pool;
    double* scs = s_pool + 1025;
    double* ssn = s_pool + 2049;
    __shared__ double s_hn;
    const int nv = j + 1, nb = gridDim.x;
    const bool staged = nb * (nv + 1) <= kStage;
    const int per = (N + nb - 1) / nb;
    const int i0 = min(N, (int)blockIdx.x * per), i1 = min(N, i0 + per);
    double* part1 = p.part;
    double* part2 = p.part + (size_t)KB_MAX * p.ld;
    // first pass: h1 = V^T w
    range_dots(V, N, nv, w, i0, i1, part1 + (size_t)blockIdx.x * p.ld, red, s_pool, false);
    grid_barrier(s);
    if (staged)
        reduce_coeffs_staged(part1, p.ld, nv, nb, h1, s_stage, red8);
    else
        reduce_coeffs(part1, p.ld, nv, nb, h1, red8);
    // w' = w - V h1 on the block's range, then the second pass h2 = V^T w' with ||w'||^2
    // (fusing this update with the second pass's dots, the basis entries kept in
    // registers, measured slower: 168 registers per thread)
    for (int i = i0 + threadIdx.x; i < i1; i += KT) {
        double acc = w[i];
        for (int k = 0; k < nv; ++k) acc = fma(-h1[k], V[(size_t)k * N + i], acc);
        w[i] = acc;
    }
    __syncthreads();
    range_dots(V, N, nv, w, i0, i1, part2 + (size_t)blockIdx.x * p.ld, red, s_pool, true);
    if (blockIdx.x == 0) givens_stage(j, scs, ssn, p);  // the reduction buffer is free again
    grid_barrier(s);
    if (staged)
        reduce_coeffs_staged(part2, p.ld, nv + 1, nb, h2, s_stage, red8);
    else
        reduce_coeffs(part2, p.ld, nv + 1, nb, h2, red8);
    // ||w' - V h2||^2 = ||w'||^2 - ||h2||^2 for an orthonormal basis; when more
    // than half of ||w'||^2 cancels, the norm is summed again after the update
    if (threadIdx.x < 32) {  // ||h2||^2 by warp 0 (a butterfly: every lane gets the same sum)
        double q = 0.0;
        for (int k = threadIdx.x; k < nv; k += 32) q = fma(h2[k], h2[k], q);
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (threadIdx.x == 0) {
            const double d = h2[nv] - q;
            s_hn = (d > 0.5 * h2[nv]) ? sqrt(d) : -1.0;
        }
    }
    __syncthreads();
    double hn = s_hn;
    if (hn < 0.0) {  // the same decision in every block
        double acc = 0.0;
        for (int i = i0 + threadIdx.x; i < i1; i += KT) {
            double wi = w[i];
            for (int k = 0; k < nv; ++k) wi = fma(-h2[k], V[(size_t)k * N + i], wi);
            w[i] = wi;
            acc = fma(wi, wi, acc);
        }
        acc = block_sum(acc, &red[0][0]);
        if (threadIdx.x == 0) part1[(size_t)blockIdx.x * p.ld] = acc;
        grid_barrier(s);
        if (threadIdx.x < 32) {
            double t = 0.0;
            for (int b = threadIdx.x; b < nb; b += 32) t += __ldcg(part1 + (size_t)b * p.ld);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) s_hn = sqrt(t);
        }
        __syncthreads();
        hn = s_hn;
        if (hn > 0.0 && isfinite(hn)) {
            const double inv = 1.0 / hn;
            for (int i = i0 + threadIdx.x; i < i1; i += KT) w[i] *= inv;
        }
        if (blockIdx.x == 0) givens_step(j, hn, h1, h2, scs, ssn, p, s);
    } else {  // v_{j+1} = (w' - V h2) / h_{j+1,j} in one pass (unused when the cycle stops here)
        const double inv = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 1.0;
        // block 0: warp 0 does the Givens update while the other warps update the range
        const int t0 = (blockIdx.x == 0) ? 32 : 0;
        if (blockIdx.x == 0 && threadIdx.x < 32) givens_step_warp0(j, hn, h1, h2, scs, ssn, scs[1023], p, s);
        for (int i = i0 + (int)threadIdx.x - t0; i < i1; i += KT - t0) {
            if ((int)threadIdx.x < t0) break;
            double wi = w[i];
            for (int k = 0; k < nv; ++k) wi = fma(-h2[k], V[(size_t)k * N + i], wi);
            w[i] = wi * inv;
        }
    }
}

// ---- the same Arnoldi step with the Gram-Schmidt arithmetic in double-float
// on the FP32 pipe (GB300's FP64 pipe has 2 lanes per SM against 128 FP32
// lanes, and each pass is nv multiply-adds per entry), shaped for latency:
// each pass is a handful of dependent memory round trips, so the step is
// built to take as few as possible.
//  * The basis is kept in FP64 (the operator's input and the update of x read
//    it) and as a double-float copy Vd (hi, lo per entry).  At the start, one
//    thread issues bulk asynchronous copies (cp.async.bulk, completion on an
//    mbarrier) of the block's range of Vd_0 .. Vd_j and of w = A v_j into
//    shared memory; every pass then reads shared memory.  (Ranges too long
//    for shared memory read global memory through the same code.)
//  * Dots: warp per basis vector, lanes over the range, a fixed shuffle tree.
//  * Grid barriers: one relaxed-cost arrival (red.release) on a counter that
//    only grows during a solve, and polls (ld.acquire) for the barrier's target
//    count; the target follows from the count seen at the kernel's start.
// Block and grid sums are compensated double-float sums in a fixed order;
// the coefficients stay double-float for the updates and are rounded to FP64
// for the Givens step.  With about 48 significant bits the basis is
// orthonormal to ~1e-14, far below the solver's tolerances; GNK_PREC_FP64
// keeps the FP64 step above.
__device__ __forceinline__ df df_renorm(df a) {
    df r;
    fast_two_sum(a.h, a.l, r.h, r.l);
    return r;
}

__device__ __forceinline__ df df_of(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ float2 f2_of(df v) { return make_float2(v.h, v.l); }
__device__ __forceinline__ double df_dbl(df v) { return (double)v.h + (double)v.l; }
__device__ __forceinline__ df df_minus(df a, df b) { return df_sub(a.h, a.l, b.h, b.l); }
__device__ __forceinline__ df df_plus(df a, df b) { return df_sub(a.h, a.l, -b.h, -b.l); }
__device__ __forceinline__ df df_prod(df a, df b) { return df_renorm(df_mul(a, b)); }

// sqrt(a), a > 0: one Newton step from the rounded FP32 root (the residual
// a.h - y^2 is exact by the FMA), about 46 significant bits
__device__ __forceinline__ df df_sqrt(df a) {
    const float y = __fsqrt_rn(a.h);
    const float e = __fadd_rn(fmaf(-y, y, a.h), a.l);
    df r;
    fast_two_sum(y, __fmul_rn(e, __fdiv_rn(0.5f, y)), r.h, r.l);
    return r;
}

// 1 / a: one Newton step from the rounded FP32 reciprocal (1 - a.h y exact by the FMA)
__device__ __forceinline__ df df_rcp(df a) {
    const float y = __frcp_rn(a.h);
    const float e = __fsub_rn(fmaf(-a.h, y, 1.0f), __fmul_rn(a.l, y));
    df r;
    fast_two_sum(y, __fmul_rn(y, e), r.h, r.l);
    return r;
}

// shared memory of the range (bytes) beyond the pool and the staging area
constexpr int kSliceBytes = 128 * 1024;
constexpr size_t kArnoldiDfDyn = kArnoldiDyn + kSliceBytes;

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on the growing counter: arrive, then wait until the count
// reaches `target` (bounded; a wait that gives up sets bar_err).  The test hook
// block bar_skip passes without arriving.
__device__ __forceinline__ void grid_barrier_count(KState* s, unsigned target) {
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x != s->bar_skip) {
        red_release_add(&s->bar_count, 1u);
        const int limit = s->bar_limit;
        for (int it = 0; (int)(ld_acquire(&s->bar_count) - target) < 0; ++it) {
            if (it >= limit || *(volatile int*)&s->bar_err) {
                atomicExch(&s->bar_err, 1);
                break;
            }
        }
    }
    __syncthreads();
}

// Waits for phase `phase` of the mbarrier with a limit; on a timeout sets
// bar_err and waits once more (also bounded) for the copies in flight.
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned phase, KState* s) {
    const int limit = s->bar_limit;
    if (!mbar_wait(bar, phase, limit)) {
        atomicExch(&s->bar_err, 1);
        mbar_wait(bar, phase, limit);
    }
}

// Threads of the double-float step: one block per multiprocessor, so that the
// block's few hundred entries and short dependent chains have 32 warps to hide
// their latencies.
constexpr int KTD = 1024;

// Block partials of the dots of the range's w (ws, len entries) with the
// rows Vr + k ld, k < nv (and ws . ws when with_norm), to out[0 .. nv(+1)):
// warp w takes k = w, w + 32, ...; lane l the entries l, l + 32, ... in two
// interleaved compensated sums, then a shuffle tree in a fixed order.
__device__ __forceinline__ void slice_dots(const float2* Vr, size_t ld, const float2* ws, int len, int nv,
                                           bool with_norm, float2* out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nt = nv + (with_norm ? 1 : 0);
    for (int k = wid; k < nt; k += KTD / 32) {
        const float2* row = (k < nv) ? Vr + (size_t)k * ld : ws;
        df a0{0.f, 0.f}, a1{0.f, 0.f};
        int e = lane;
        for (; e + 32 < len; e += 64) {
            df_acc(a0, df_mul(df_of(row[e]), df_of(ws[e])));
            df_acc(a1, df_mul(df_of(row[e + 32]), df_of(ws[e + 32])));
        }
        if (e < len) df_acc(a0, df_mul(df_of(row[e]), df_of(ws[e])));
        df_acc(a0, a1);
        for (int o = 16; o > 0; o >>= 1) {
            const df t{__shfl_down_sync(full, a0.h, o), __shfl_down_sync(full, a0.l, o)};
            df_acc(a0, t);
        }
        if (lane == 0) out[k] = f2_of(df_renorm(a0));
    }
}

// hs[k] = sum_b part[b * ld + k] over the nb blocks, k < nv, in double-float:
// staged (the partials loaded at once, up to kStageLoads independent loads per
// thread, into `stage`, at least nb * nv entries) when it fits, else read in
// place; 8 threads per coefficient each add a contiguous eighth of the blocks,
// then the eighths in order.  The result is the same in every block.
constexpr int kStageLoads = 4;

__device__ __forceinline__ void reduce_coeffs_df(const float2* part, int ld, int nv, int nb, float2* hs,
                                                 float2* stage, bool staged, float2 (*red8)[KTD / 8]) {
    if (staged) {
        const int tot = nv * nb;
        for (int e0 = 0; e0 < tot; e0 += kStageLoads * KTD) {
            float2 v[kStageLoads];
#pragma unroll
            for (int u = 0; u < kStageLoads; ++u) {
                const int e = e0 + u * KTD + threadIdx.x;  // e = b * nv + k
                if (e < tot) {
                    const int b = e / nv, k = e - b * nv;
                    v[u] = __ldcg(part + (size_t)b * ld + k);
                }
            }
#pragma unroll
            for (int u = 0; u < kStageLoads; ++u) {
                const int e = e0 + u * KTD + threadIdx.x;
                if (e < tot) stage[e] = v[u];
            }
        }
        __syncthreads();
    }
    const int per = (nb + 7) / 8;
    for (int k0 = 0; k0 < nv; k0 += KTD / 8) {
        const int k = k0 + (threadIdx.x >> 3), slice = threadIdx.x & 7;
        df t{0.f, 0.f};
        if (k < nv) {
            const int b0 = min(nb, slice * per), b1 = min(nb, b0 + per);
            for (int b = b0; b < b1; ++b)
                df_acc(t, df_of(staged ? stage[b * nv + k] : __ldcg(part + (size_t)b * ld + k)));
        }
        red8[slice][threadIdx.x >> 3] = f2_of(t);
        __syncthreads();
        if (threadIdx.x < KTD / 8 && k0 + (int)threadIdx.x < nv) {
            df u = df_of(red8[0][threadIdx.x]);
            for (int sl = 1; sl < 8; ++sl) df_acc(u, df_of(red8[sl][threadIdx.x]));
            hs[k0 + threadIdx.x] = f2_of(df_renorm(u));
        }
        __syncthreads();
    }
}

// sum_k Vr[k ld + e] c_k for k < nv (two interleaved compensated sums)
__device__ __forceinline__ df slice_combo(const float2* Vr, size_t ld, int nv, int e, const float2* c) {
    df s0{0.f, 0.f}, s1{0.f, 0.f};
    int k = 0;
    for (; k + 1 < nv; k += 2) {
        df_acc(s0, df_mul(df_of(Vr[(size_t)k * ld + e]), df_of(c[k])));
        df_acc(s1, df_mul(df_of(Vr[(size_t)(k + 1) * ld + e]), df_of(c[k + 1])));
    }
    if (k < nv) df_acc(s0, df_mul(df_of(Vr[(size_t)k * ld + e]), df_of(c[k])));
    df_acc(s0, s1);
    return s0;
}

// givens_step_warp0 for the double-float step: the column x = hcol (h1 + h2,
// FP64, k <= j) and h_{j+1,j} = hn in double-float.  The previous rotations
// by the same scan; the new rotation (a square root and a reciprocal, each a
// chain of hundreds of cycles on GB300's FP64 pipe) in double-float on the
// FP32 pipe, rounded to FP64 where it is stored.
__device__ void givens_df_warp0(int j, df hn, double* hcol, const double* scs, const double* ssn, double gj,
                                KPtrs p, KState* s) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;  // warp 0
    double zj;
    if (j <= 32) {
        const double x0 = hcol[0];
        double a = 1.0, b = 0.0, ck = 1.0, sk = 0.0, xk1 = 0.0;
        if (lane < j) {
            ck = scs[lane];
            sk = ssn[lane];
            xk1 = hcol[lane + 1];
            a = -sk;
            b = ck * xk1;
        }
        for (int o = 1; o < 32; o <<= 1) {  // (a, b) <- (a, b) o (ap, bp)
            const double ap = __shfl_up_sync(full, a, o), bp = __shfl_up_sync(full, b, o);
            if (lane >= o) {
                b = fma(a, bp, b);
                a *= ap;
            }
        }
        const double znext = fma(a, x0, b);                       // z_{lane+1}
        const double zprev = __shfl_up_sync(full, znext, 1);
        const double zcur = (lane == 0) ? x0 : zprev;             // z_lane
        __syncwarp();
        if (lane < j) hcol[lane] = fma(ck, zcur, sk * xk1);       // y_lane
        zj = (j == 0) ? x0 : __shfl_sync(full, znext, j - 1);
    } else {
        if (lane == 0) {
            for (int k = 0; k < j; ++k) {
                const double a = hcol[k], b = hcol[k + 1];
                hcol[k] = scs[k] * a + ssn[k] * b;
                hcol[k + 1] = -ssn[k] * a + scs[k] * b;
            }
        }
        __syncwarp();
        zj = hcol[j];
    }
    __syncwarp();
    if (lane == 0) {
        const double hnd = df_dbl(hn);
        s->hnext = hnd;
        const df z = df_split(zj);
        const df g = df_split(gj);
        const df r2 = df_plus(df_prod(z, z), df_prod(hn, hn));
        df r{0.f, 0.f}, c{1.f, 0.f}, sn{0.f, 0.f};
        if (r2.h > 0.f) {
            r = df_sqrt(r2);
            const df inv = df_rcp(r);
            c = df_prod(z, inv);
            sn = df_prod(hn, inv);
        }
        const df gn = df_prod(sn, g);
        p.cs[j] = df_dbl(c);
        p.sn[j] = df_dbl(sn);
        hcol[j] = df_dbl(r);
        hcol[j + 1] = 0.0;
        p.g[j + 1] = -df_dbl(gn);
        p.g[j] = df_dbl(df_prod(c, g));
        const double est = fabs(df_dbl(gn));
        s->est = est;
        s->k = j + 1;
        const bool bad = !isfinite(est) || !isfinite(hnd) || !isfinite(zj);
        if (bad) s->nonfinite = 1;
        if (bad || est <= s->tol * s->bnorm || j + 1 == s->restart || hnd == 0.0) s->done = 1;
    }
    __syncwarp();
    double* colg = p.H + (size_t)j * p.ld;
    for (int k = lane; k < j + 2; k += 32) colg[k] = hcol[k];
}

// Entries per block of the double-float step: even, so that every block's
// range starts on a 16-byte boundary of the (even-length) vectors.
__host__ __device__ __forceinline__ int arnoldi_df_per(int N, int nb) {
    const int per = (N + nb - 1) / nb;
    return per + (per & 1);
}

__global__ void __launch_bounds__(KTD) k_arnoldi_df(double* __restrict__ V, float2* __restrict__ Vd, int N,
                                                    int j, float2* __restrict__ wd, KPtrs p, KState* s) {
    if (s->done) return;  // set before this launch: the same in every block
    __shared__ float2 red8[8][KTD / 8];
    __shared__ float2 h1f[1025];
    __shared__ float2 h2f[1025];
    __shared__ double h1[1025];
    __shared__ float2 s_hnf, s_inv;
    __shared__ __align__(8) unsigned long long s_bar;
    // dynamic: pool (h2 and the Givens staging), the staging area of the
    // coefficient sums, then the range of Vd_0 .. Vd_j and w
    extern __shared__ __align__(16) double s_dyn[];
    double* h2 = s_dyn;
    double* scs = s_dyn + 1025;
    double* ssn = s_dyn + 2049;
    float2* s_stage = reinterpret_cast<float2*>(s_dyn + kPool);
    float2* s_slice = reinterpret_cast<float2*>(s_dyn + kPool + kStage);
    const int nv = j + 1, nb = gridDim.x;
    const bool staged = nb * (nv + 1) <= kStage;
    const int per = arnoldi_df_per(N, nb);
    const int i0 = min(N, (int)blockIdx.x * per), i1 = min(N, i0 + per);
    const int len = i1 - i0;
    const bool in_smem = (size_t)(nv + 1) * per * sizeof(float2) <= (size_t)kSliceBytes;
    float2* part1 = reinterpret_cast<float2*>(p.part);
    float2* part2 = reinterpret_cast<float2*>(p.part + (size_t)KB_MAX * p.ld);
    double* w = V + (size_t)(j + 1) * N;  // the product A v_j, overwritten by v_{j+1}
    // the rows of the range: Vr + k ld (k < nv), and w' at ws
    const float2* Vr;
    size_t ld;
    float2* ws;
    unsigned bar_base = 0;
    if (threadIdx.x == 0) {
        const unsigned c = *(volatile unsigned*)&s->bar_count;
        bar_base = c - c % (unsigned)nb;  // no block of this launch has passed a barrier yet
    }
    if (in_smem) {
        Vr = s_slice;
        ld = per;
        ws = s_slice + (size_t)nv * per;
        if (threadIdx.x == 0) {
            mbar_init(&s_bar, 1);
            if (len > 0) {
                const unsigned row = (unsigned)len * sizeof(float2);
                mbar_expect_tx(&s_bar, row * (nv + 1));
                bulk_load(ws, w + i0, row, &s_bar);  // FP64 w, split in place below
                for (int k = 0; k < nv; ++k) bulk_load(s_slice + (size_t)k * per, Vd + (size_t)k * N + i0, row, &s_bar);
            } else {
                mbar_expect_tx(&s_bar, 0);
            }
        }
        __syncthreads();
        mbar_wait_bounded(&s_bar, 0, s);
        const double* wsrc = reinterpret_cast<const double*>(ws);
        for (int e = threadIdx.x; e < len; e += KTD) ws[e] = f2_of(df_split_fast(wsrc[e]));
    } else {
        Vr = Vd + i0;
        ld = N;
        ws = wd + i0;
        for (int e = threadIdx.x; e < len; e += KTD) ws[e] = f2_of(df_split_fast(w[i0 + e]));
    }
    __syncthreads();
    // first pass: h1 = V^T w
    slice_dots(Vr, ld, ws, len, nv, false, part1 + (size_t)blockIdx.x * p.ld);
    grid_barrier_count(s, bar_base + (unsigned)nb);
    reduce_coeffs_df(part1, p.ld, nv, nb, h1f, s_stage, staged, red8);
    // w' = w - V h1 on the range, then the second pass h2 = V^T w' with ||w'||^2
    for (int e = threadIdx.x; e < len; e += KTD) ws[e] = f2_of(df_minus(df_of(ws[e]), slice_combo(Vr, ld, nv, e, h1f)));
    __syncthreads();
    slice_dots(Vr, ld, ws, len, nv, true, part2 + (size_t)blockIdx.x * p.ld);
    if (blockIdx.x == 0) givens_stage(j, scs, ssn, p);
    grid_barrier_count(s, bar_base + 2u * (unsigned)nb);
    reduce_coeffs_df(part2, p.ld, nv + 1, nb, h2f, s_stage, staged, red8);
    // warp 0: ||w' - V h2||^2 = ||w'||^2 - ||h2||^2 (an orthonormal basis) in
    // double-float, its root and reciprocal; when more than half of ||w'||^2
    // cancels, the norm is summed again after the update
    if (threadIdx.x < 32) {
        df q{0.f, 0.f};
        for (int k = threadIdx.x; k < nv; k += 32) {
            const df v = df_of(h2f[k]);
            df_acc(q, df_mul(v, v));
        }
        for (int o = 16; o > 0; o >>= 1) {
            const df t{__shfl_down_sync(0xffffffffu, q.h, o), __shfl_down_sync(0xffffffffu, q.l, o)};
            df_acc(q, t);
        }
        if (threadIdx.x == 0) {
            const df n2 = df_of(h2f[nv]);
            const df d = df_minus(n2, df_renorm(q));
            const df hn = (d.h > 0.5f * n2.h) ? df_sqrt(d) : df{-1.f, 0.f};
            s_hnf = f2_of(hn);
            s_inv = f2_of((hn.h > 0.f && isfinite(hn.h)) ? df_rcp(hn) : df{1.f, 0.f});
        }
    }
    __syncthreads();
    df hn = df_of(s_hnf);
    float2* vnext = Vd + (size_t)(j + 1) * N + i0;
    double* wout = w + i0;
    if (hn.h < 0.f) {  // the same decision in every block
        df acc{0.f, 0.f};
        for (int e = threadIdx.x; e < len; e += KTD) {
            const df wi = df_minus(df_of(ws[e]), slice_combo(Vr, ld, nv, e, h2f));
            ws[e] = f2_of(wi);
            df_acc(acc, df_mul(wi, wi));
        }
        s_stage[threadIdx.x] = f2_of(acc);  // the staging area is free again
        __syncthreads();
        if (threadIdx.x == 0) {
            df t{0.f, 0.f};
            for (int e = 0; e < KTD; ++e) df_acc(t, df_of(s_stage[e]));
            part1[(size_t)blockIdx.x * p.ld] = f2_of(df_renorm(t));
        }
        grid_barrier_count(s, bar_base + 3u * (unsigned)nb);
        if (threadIdx.x == 0) {
            df t{0.f, 0.f};
            for (int b = 0; b < nb; ++b) df_acc(t, df_of(__ldcg(part1 + (size_t)b * p.ld)));
            t = df_renorm(t);
            const df h = (t.h > 0.f) ? df_sqrt(t) : df{0.f, 0.f};
            s_hnf = f2_of(h);
            s_inv = f2_of((h.h > 0.f && isfinite(h.h)) ? df_rcp(h) : df{1.f, 0.f});
        }
        __syncthreads();
        hn = df_of(s_hnf);
        const df inv = df_of(s_inv);
        for (int e = threadIdx.x; e < len; e += KTD) {
            const df v = df_renorm(df_mul(df_of(ws[e]), inv));
            vnext[e] = f2_of(v);
            wout[e] = df_dbl(v);
        }
        if (blockIdx.x == 0) {
            for (int k = threadIdx.x; k <= nv; k += KTD) {
                h1[k] = df_dbl(df_of(h1f[k]));
                h2[k] = df_dbl(df_of(h2f[k]));
            }
            __syncthreads();
            givens_step(j, df_dbl(hn), h1, h2, scs, ssn, p, s);
        }
    } else {  // v_{j+1} = (w' - V h2) / h_{j+1,j} in one pass (unused when the cycle stops here)
        const df inv = df_of(s_inv);
        // block 0: warp 0 does the Givens update while the other warps update the range
        const int t0 = (blockIdx.x == 0) ? 32 : 0;
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            for (int k = threadIdx.x; k < nv; k += 32) h1[k] = df_dbl(df_plus(df_of(h1f[k]), df_of(h2f[k])));
            __syncwarp();
            givens_df_warp0(j, hn, h1, scs, ssn, scs[1023], p, s);
        }
        if ((int)threadIdx.x >= t0) {
            for (int e = (int)threadIdx.x - t0; e < len; e += KTD - t0) {
                const df wi = df_minus(df_of(ws[e]), slice_combo(Vr, ld, nv, e, h2f));
                const df v = df_renorm(df_mul(wi, inv));
                vnext[e] = f2_of(v);
                wout[e] = df_dbl(v);
            }
        }
    }
}

// y = H(0:k, 0:k)^-1 g(0:k) at the end of a cycle (one block), by columns:
// once y_c is known, every row r < c takes its term H(r, c) y_c at once, so
// the dependent chain is one multiply and one multiply-add per column (on
// GB300's 2-lane FP64 pipe a row-by-row loop of one thread costs k^2/2
// dependent steps).  The diagonal's reciprocals are formed first, in
// parallel.  k <= kSmallH: warp 0, H staged in shared memory, two rows per
// lane in registers; longer cycles: the whole block, H read in place.
constexpr int kSmallH = 64;

__global__ void __launch_bounds__(KT) k_solve_y(KPtrs p, const KState* s) {
    __shared__ double sH[kSmallH * kSmallH];  // k > kSmallH: the rows' values and reciprocals instead
    double* sv = sH;
    double* sinv = sH + 1024;
    const int kk = s->k;
    if (kk == 0) return;
    if (kk <= kSmallH) {
        for (int e = threadIdx.x; e < kk * kk; e += KT) sH[e] = p.H[(size_t)(e / kk) * p.ld + (e % kk)];
        __syncthreads();
        if (threadIdx.x >= 32) return;
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x;
        // rows lane and lane + 32: right-hand side and 1 / H(r, r) (0 where H(r, r) = 0)
        double g0 = (lane < kk) ? p.g[lane] : 0.0, g1 = (lane + 32 < kk) ? p.g[lane + 32] : 0.0;
        const double d0 = (lane < kk) ? sH[lane * kk + lane] : 1.0;
        const double d1 = (lane + 32 < kk) ? sH[(lane + 32) * kk + lane + 32] : 1.0;
        const double i0 = (d0 != 0.0) ? 1.0 / d0 : 0.0, i1 = (d1 != 0.0) ? 1.0 / d1 : 0.0;
        for (int c = kk - 1; c >= 0; --c) {  // sH[c * kk + r] = H(r, c)
            const double own = (c < 32) ? g0 * i0 : g1 * i1;
            const double yc = __shfl_sync(full, own, c & 31);
            if (lane == (c & 31)) {
                if (c < 32) g0 = yc; else g1 = yc;
            }
            if (lane < c) g0 = fma(-sH[c * kk + lane], yc, g0);
            if (lane + 32 < c) g1 = fma(-sH[c * kk + lane + 32], yc, g1);
        }
        if (lane < kk) p.y[lane] = g0;
        if (lane + 32 < kk) p.y[lane + 32] = g1;
        return;
    }
    for (int r = threadIdx.x; r < kk; r += KT) {
        sv[r] = p.g[r];
        const double d = p.H[(size_t)r * p.ld + r];
        sinv[r] = (d != 0.0) ? 1.0 / d : 0.0;
    }
    __syncthreads();
    for (int c = kk - 1; c >= 0; --c) {
        const double yc = sv[c] * sinv[c];
        __syncthreads();  // every thread has read sv[c]
        if (threadIdx.x == 0) sv[c] = yc;
        for (int r = threadIdx.x; r < c; r += KT) sv[r] = fma(-p.H[(size_t)c * p.ld + r], yc, sv[r]);
        __syncthreads();
    }
    for (int r = threadIdx.x; r < kk; r += KT) p.y[r] = sv[r];
}

// x += V(:, 0:k) y at the end of a cycle
__global__ void __launch_bounds__(KT) k_update_x(const double* __restrict__ V, int N, KPtrs p,
                                                 double* __restrict__ x, const KState* s) {
    const int kk = s->k;
    if (kk == 0) return;
    __shared__ double ys[1024];
    for (int k = threadIdx.x; k < kk; k += KT) ys[k] = p.y[k];
    __syncthreads();
    for (int i = blockIdx.x * KT + threadIdx.x; i < N; i += gridDim.x * KT) {
        double acc = x[i];
        for (int k = 0; k < kk; ++k) acc = fma(ys[k], V[(size_t)k * N + i], acc);
        x[i] = acc;
    }
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] += d[i];
}

__global__ void k_init_state(KState* s, double tol, int restart, int bar_limit, int bar_skip) {
    s->bnorm = 0.0;
    s->beta = 0.0;
    s->tol = tol;
    s->est = 0.0;
    s->hnext = 0.0;
    s->k = 0;
    s->last_k = 0;
    s->done = 0;
    s->nonfinite = 0;
    s->restart = restart;
    s->counter = 0;
    s->bar_count = 0;
    s->bar_err = 0;
    s->bar_limit = bar_limit;
    s->bar_skip = bar_skip;
}

// Test hook of gnk_debug_barrier_fault, read by every later solve.
std::atomic<int> g_bar_limit{kBarSpin};
std::atomic<int> g_bar_skip{-1};

size_t krylov_basis_bytes(int restart, int N) {
    return (size_t)(restart + 1) * N * (sizeof(double) + sizeof(float2)) + (size_t)N * sizeof(float2);
}

float2* basis_df(const Boundary& b) {
    return reinterpret_cast<float2*>(b.V + (size_t)b.V_cols * b.N);
}

float2* basis_df_scratch(const Boundary& b) {
    return basis_df(b) + (size_t)b.V_cols * b.N;
}

int ensure_krylov(Boundary& b, int restart, cudaStream_t st) {
    if (restart + 1 > 1024) {
        set_error("restart must be below 1024");
        return GNK_EINVAL;
    }
    if (b.V_cols < restart + 1) {
        if (b.V) pool_free(b.V, st);
        b.V = nullptr;
        b.V_cols = 0;
        // V (FP64), its double-float copy Vd and the scratch wd of the
        // double-float Arnoldi step, in one allocation
        if (pool_alloc(reinterpret_cast<void**>(&b.V), krylov_basis_bytes(restart, b.N), st) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate the Krylov basis: %d x %d doubles", restart + 1, b.N);
            return GNK_ENOMEM;
        }
        b.V_cols = restart + 1;
    }
    const size_t need = kry_doubles(restart) * sizeof(double);
    if (b.kry_bytes < need) {
        if (b.kry) pool_free(b.kry, st);
        b.kry = nullptr;
        b.kry_bytes = 0;
        GNK_TRY_CUDA(pool_alloc(reinterpret_cast<void**>(&b.kry), need, st));
        b.kry_bytes = need;
    }
    if (!b.kstate) {
        GNK_TRY_CUDA(pool_alloc(&b.kstate, sizeof(KState), st));
        GNK_TRY_CUDA(cudaMemsetAsync(b.kstate, 0, sizeof(KState), st));
    }
    return GNK_OK;
}

int apply_op(const Boundary& b, int op, const double* x, double* y, int prec, cudaStream_t st,
             const int* done) {
    if (op == OP_ADJ) return op_adjoint(b, x, y, prec, st, done);
    if (op == OP_KT) return op_IminusN_T(b, x, y, prec, st, done);
    return op_IminusN(b, x, y, prec, st, done);
}

int read_state(const Boundary& b, KState* hs, cudaStream_t st) {
    GNK_TRY_CUDA(cudaMemcpyAsync(hs, b.kstate, sizeof(KState), cudaMemcpyDeviceToHost, st));
    int fault = 0;
    const int* fw = fmm_fault_word(b);
    if (fw) GNK_TRY_CUDA(cudaMemcpyAsync(&fault, fw, sizeof(int), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    if (fault) {
        set_error("FMM: a bounded wait of the near field timed out");
        return GNK_ECUDA;
    }
    return GNK_OK;
}

// Blocks of the cooperative Arnoldi launch: one per multiprocessor (all
// resident at once), at most KB_MAX, at most one per KT entries.
static int arnoldi_blocks(int N) {
    static std::mutex mu;
    static std::vector<int> cap;  // per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cap.size() <= dev) cap.resize(dev + 1, 0);
    if (cap[dev] == 0) {
        int occ = 0, occ_df = 0, nsm = 0;
        if (cudaFuncSetAttribute((const void*)k_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kArnoldiDyn) != cudaSuccess ||
            cudaFuncSetAttribute((const void*)k_arnoldi_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kArnoldiDfDyn) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi, KT, kArnoldiDyn) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_df, k_arnoldi_df, KTD, kArnoldiDfDyn) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            occ = occ_df = 1;
            nsm = 1;
        }
        cap[dev] = std::max(1, std::min(std::min(occ, occ_df), 1) * nsm);  // one block per multiprocessor
    }
    return std::max(1, std::min(std::min(cap[dev], KB_MAX), (N + KT - 1) / KT));
}

// Wraps one vector-kernel launch in a profiling event pair (bytes moved as work).
#define KLAUNCH(bytes, launch)                                 \
    do {                                                       \
        const ProfToken t_ = prof_begin(st, PK_KRYLOV);        \
        launch;                                                \
        prof_end(t_, PK_KRYLOV, (double)(bytes), st);          \
    } while (0)

// One restarted GMRES solve of A x = rhs with the operator in precision prec.
// r is a work vector.  Counters are added to *res; *relres receives the final
// true relative residual (in prec).
int gmres(Boundary& b, int adjoint /* OpId */, int prec, const double* rhs, double* x, double* r,
          int restart, int maxit, double tol, gnk_result* res, double* relres, cudaStream_t st,
          double* fc_out, int* fc_valid) {
    if (fc_valid) *fc_valid = 0;
    GNK_TRY(ensure_krylov(b, restart, st));
    const int N = b.N;
    const double vb = 8.0 * N;  // bytes of one vector
    KState* ks = static_cast<KState*>(b.kstate);
    KPtrs p = kry_ptrs(b.kry, restart);
    const int nb = vec_blocks(N);
    const int ng = arnoldi_blocks(N);
    // Gram-Schmidt in double-float for every operator precision but plain FP64
    const bool dfa = prec != GNK_PREC_FP64;
    KState hs;
    k_init_state<<<1, 1, 0, st>>>(ks, tol, restart, g_bar_limit.load(), g_bar_skip.load());
    KLAUNCH(vb, (k_norm<<<nb, KT, 0, st>>>(rhs, N, p, ks, 0)));
    count_launches(2);
    GNK_TRY_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), st));
    GNK_TRY_CUDA(cudaGetLastError());
    // launches of each Arnoldi step of the current cycle, to discount those
    // that the device flag turned into no-ops once the cycle had converged
    std::vector<std::vector<long>> step_ids(restart);
    int status = GNK_ENOTCONV;
    for (int cycle = 0;; ++cycle) {
        if (cycle == 0) {
            GNK_TRY_CUDA(cudaMemcpyAsync(r, rhs, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            GNK_TRY(op_resid(b, adjoint, rhs, x, r, prec, st, fc_out));
            if (prec == GNK_PREC_FP32) res->matvecs_fp32++; else res->matvecs_fp64++;
            if (fc_valid && fc_out) *fc_valid = 1;  // f_C of the current x
        }
        KLAUNCH(vb, (k_norm<<<nb, KT, 0, st>>>(r, N, p, ks, 1)));
        KLAUNCH((dfa ? 3 : 2) * vb, (k_scale_first<<<nb, KT, 0, st>>>(r, b.V, dfa ? basis_df(b) : nullptr, N, ks)));
        count_launches(2);
        GNK_TRY_CUDA(cudaGetLastError());
        // The first cycle is enqueued without waiting for its starting norm: when
        // x0 = 0 already meets the tolerance, k_norm sets the device flag `done`
        // and the cycle's launches do nothing; the next cycle's residual then ends
        // the solve (one product more in that case, one host round trip less in
        // every other).
        const bool wait_state = cycle > 0 || maxit == 0;
        if (!wait_state) {
            res->cycles++;
            goto steps;
        }
        GNK_TRY(read_state(b, &hs, st));
        if (cycle == 1 && hs.last_k == 0 && maxit > 0) res->cycles--;  // the first cycle did no step
        if (hs.bar_err) {
            set_error("GMRES: a grid barrier of the Arnoldi step timed out");
            return GNK_ECUDA;
        }
        if (cycle > 0) {  // the previous cycle's step count is known only now
            res->iterations += hs.last_k;
            if (prec == GNK_PREC_FP32) res->matvecs_fp32 += hs.last_k; else res->matvecs_fp64 += hs.last_k;
            for (int j = hs.last_k; j < restart; ++j)
                for (long id : step_ids[j]) prof_skip(id);
        }
        if (hs.bnorm == 0.0) {
            *relres = 0.0;
            status = GNK_OK;
            break;
        }
        *relres = hs.beta / hs.bnorm;
        if (hs.nonfinite || !std::isfinite(*relres)) {
            status = GNK_ENONFINITE;
            break;
        }
        if (*relres <= tol) {
            status = GNK_OK;
            break;
        }
        if (cycle == maxit) {
            status = GNK_ENOTCONV;
            break;
        }
        res->cycles++;
    steps:
        for (int j = 0; j < restart; ++j) {
            double* vj = b.V + (size_t)j * N;
            double* w = b.V + (size_t)(j + 1) * N;
            const double nv = j + 1;
            prof_collect_begin();
            GNK_TRY(apply_op(b, adjoint, vj, w, prec, st, &ks->done));
            if (dfa) {
                double* Vc = b.V;
                float2* Vdc = basis_df(b);
                float2* wdc = basis_df_scratch(b);
                int Nc = N, jc = j;
                void* args[] = {(void*)&Vc, (void*)&Vdc, (void*)&Nc, (void*)&jc, (void*)&wdc, (void*)&p,
                                (void*)&ks};
                KLAUNCH((3 * nv + 9) * vb, GNK_TRY_CUDA(cudaLaunchCooperativeKernel(
                                               (const void*)k_arnoldi_df, dim3(ng), dim3(KTD), args,
                                               kArnoldiDfDyn, st)));
            } else {
                const double* Vc = b.V;
                int Nc = N, jc = j;
                void* args[] = {(void*)&Vc, (void*)&Nc, (void*)&jc, (void*)&w, (void*)&p, (void*)&ks};
                KLAUNCH((3 * nv + 6) * vb, GNK_TRY_CUDA(cudaLaunchCooperativeKernel(
                                               (const void*)k_arnoldi, dim3(ng), dim3(KT), args, kArnoldiDyn,
                                               st)));
            }
            prof_collect_end(&step_ids[j]);
            GNK_TRY_CUDA(cudaGetLastError());
            count_launches(1);
        }
        KLAUNCH(0.0, (k_solve_y<<<1, KT, 0, st>>>(p, ks)));
        KLAUNCH((restart + 2) * vb, (k_update_x<<<nb, KT, 0, st>>>(b.V, N, p, x, ks)));
        GNK_TRY_CUDA(cudaGetLastError());
        count_launches(2);
        if (fc_valid) *fc_valid = 0;  // x moved
    }
    return status;
}

int norm_host(Boundary& b, const double* v, double* out, cudaStream_t st) {
    KState* ks = static_cast<KState*>(b.kstate);
    KPtrs p = kry_ptrs(b.kry, b.V_cols - 1);
    {
        const ProfToken t_ = prof_begin(st, PK_KRYLOV);
        k_norm<<<vec_blocks(b.N), KT, 0, st>>>(v, b.N, p, ks, 0);
        prof_end(t_, PK_KRYLOV, 8.0 * b.N, st);
    }
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    KState hs;
    GNK_TRY(read_state(b, &hs, st));
    *out = hs.bnorm;
    return GNK_OK;
}

}  // namespace

int debug_barrier_fault(int skip_block, int spin_limit) {
    if (skip_block < -1 || spin_limit < 0) {
        set_error("gnk_debug_barrier_fault: skip_block must be >= -1 and spin_limit >= 0");
        return GNK_EINVAL;
    }
    g_bar_skip.store(skip_block);
    g_bar_limit.store(spin_limit == 0 ? kBarSpin : std::min(spin_limit, kBarSpin));
    return GNK_OK;
}

int outer_precision(int solve_precision) {
    if (solve_precision == GNK_PREC_DF32 || solve_precision == GNK_PREC_MIXED_DF) return GNK_PREC_DF32;
    if (solve_precision == GNK_PREC_FMM || solve_precision == GNK_PREC_MIXED_FMM) return GNK_PREC_FMM;
    return GNK_PREC_FP64;
}

int solve(const Boundary& bc, int adjoint /* OpId */, const double* rhs, double* x, const gnk_options& opt,
          gnk_result* info, cudaStream_t st, double* fc_out, int* fc_valid) {
    Boundary& b = const_cast<Boundary&>(bc);  // workspace only
    gnk_result res;
    std::memset(&res, 0, sizeof(res));
    double relres = 0.0;
    int status;
    const int outer = outer_precision(opt.precision);
    if (fc_valid) *fc_valid = 0;
    if (opt.precision == GNK_PREC_FP64 || opt.precision == GNK_PREC_DF32 || opt.precision == GNK_PREC_FMM) {
        status = gmres(b, adjoint, outer, rhs, x, b.r0, opt.restart, opt.maxit, opt.tol, &res,
                       &relres, st, fc_out, fc_valid);
    } else {
        // FP64 iterative refinement: r = rhs - A x (FP64), A d = r with the
        // FP32 operator to inner_tol, x += d.
        GNK_TRY(ensure_krylov(b, opt.restart, st));
        double* rr = b.r1;
        double* dd = b.r2;
        const int N = b.N;
        GNK_TRY_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), st));
        GNK_TRY_CUDA(cudaMemcpyAsync(rr, rhs, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        double bnorm = 0.0;
        GNK_TRY(norm_host(b, rhs, &bnorm, st));
        status = GNK_ENOTCONV;
        for (int it = 0;; ++it) {
            double rn = 0.0;
            GNK_TRY(norm_host(b, rr, &rn, st));
            relres = (bnorm > 0.0) ? rn / bnorm : 0.0;
            if (!std::isfinite(relres)) {
                status = GNK_ENONFINITE;
                break;
            }
            if (relres <= opt.tol) {
                status = GNK_OK;
                break;
            }
            if (it == opt.max_refine) break;
            double inner_rel = 0.0;
            const int s = gmres(b, adjoint, GNK_PREC_FP32, rr, dd, b.r0, opt.restart, opt.maxit,
                                opt.inner_tol, &res, &inner_rel, st, nullptr, nullptr);
            if (s != GNK_OK && s != GNK_ENOTCONV) {
                // NaN/Inf, a CUDA failure or a timed-out grid barrier in the
                // inner solve: its correction is not applied and its status
                // (and message) is the solve's
                status = s;
                break;
            }
            k_axpy<<<(N + 255) / 256, 256, 0, st>>>(x, dd, N);
            GNK_TRY_CUDA(cudaGetLastError());
            count_launches(1);
            // f_C(x) rides on the residual's Cauchy sum only where this residual is
            // expected to end the refinement; with Im A = 0 the other residuals then
            // need only Im E(q x).  A wrong guess costs one f_C product, never accuracy.
            double* fc_use = fc_out;
            if (fc_out && b.A_real && relres * std::max(inner_rel, 1e-8) > 100.0 * opt.tol)
                fc_use = nullptr;
            GNK_TRY(op_resid(b, adjoint, rhs, x, rr, outer, st, fc_use));
            if (fc_valid) *fc_valid = fc_use != nullptr;
            res.matvecs_fp64++;
            res.refinements++;
        }
    }
    res.status = status;
    res.relres = relres;
    if (info) *info = res;
    return status;
}

}  // namespace gnk
