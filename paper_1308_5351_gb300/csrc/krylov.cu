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
// pass by Pythagoras unless it cancels, then a third); the norms at the start of a cycle
// finish in the last block to arrive (atomic ticket + fence, no spinning).
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

// v0 = r / beta
__global__ void __launch_bounds__(KT) k_scale_first(const double* __restrict__ r, double* __restrict__ v0,
                                                    int N, const KState* s) {
    if (s->done) return;
    const double inv = 1.0 / s->beta;
    for (int i = blockIdx.x * KT + threadIdx.x; i < N; i += gridDim.x * KT) v0[i] = r[i] * inv;
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
    for (int k = threadIdx.x; k < j; k += KT) {
        scs[k] = p.cs[k];
        ssn[k] = p.sn[k];
    }
    if (threadIdx.x == 0) scs[1023] = p.g[j];  // g_j (scs holds at most j <= 1023 rotations before it)
}

__device__ void givens_step(int j, double hn, double* h1, const double* h2, const double* scs, const double* ssn,
                            KPtrs p, KState* s) {
    const int nv = j + 1;
    for (int k = threadIdx.x; k < nv; k += KT) h1[k] = h1[k] + h2[k];
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
    for (int k = threadIdx.x; k < j + 2; k += KT) colg[k] = h1[k];
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

// y = H(0:k, 0:k)^-1 g(0:k) at the end of a cycle (one block; H staged in
// shared memory when k <= kSmallH, else read from global memory)
constexpr int kSmallH = 48;

__global__ void __launch_bounds__(KT) k_solve_y(KPtrs p, const KState* s) {
    __shared__ double sH[kSmallH * kSmallH], sg[kSmallH];
    const int kk = s->k;
    if (kk == 0) return;
    if (kk <= kSmallH) {
        for (int e = threadIdx.x; e < kk * kk; e += KT) sH[e] = p.H[(size_t)(e / kk) * p.ld + (e % kk)];
        for (int e = threadIdx.x; e < kk; e += KT) sg[e] = p.g[e];
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int row = kk - 1; row >= 0; --row) {  // sH[c * kk + r] = H(r, c)
                double v = sg[row];
                for (int c = row + 1; c < kk; ++c) v -= sH[c * kk + row] * sg[c];
                const double d = sH[row * kk + row];
                sg[row] = (d != 0.0) ? v / d : 0.0;  // y overwrites g from the bottom up
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kk; e += KT) p.y[e] = sg[e];
        return;
    }
    if (threadIdx.x != 0) return;
    for (int row = kk - 1; row >= 0; --row) {
        double v = p.g[row];
        for (int c = row + 1; c < kk; ++c) v -= p.H[(size_t)c * p.ld + row] * p.y[c];
        const double d = p.H[(size_t)row * p.ld + row];
        p.y[row] = (d != 0.0) ? v / d : 0.0;
    }
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

int ensure_krylov(Boundary& b, int restart, cudaStream_t st) {
    if (restart + 1 > 1024) {
        set_error("restart must be below 1024");
        return GNK_EINVAL;
    }
    if (b.V_cols < restart + 1) {
        if (b.V) pool_free(b.V, st);
        b.V = nullptr;
        b.V_cols = 0;
        if (pool_alloc(reinterpret_cast<void**>(&b.V), (size_t)(restart + 1) * b.N * sizeof(double), st) !=
            cudaSuccess) {
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
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
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
        int occ = 0, nsm = 0;
        if (cudaFuncSetAttribute((const void*)k_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kArnoldiDyn) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi, KT, kArnoldiDyn) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            occ = 1;
            nsm = 1;
        }
        cap[dev] = std::max(1, std::min(occ, 1) * nsm);  // one block per multiprocessor
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
        KLAUNCH(2 * vb, (k_scale_first<<<nb, KT, 0, st>>>(r, b.V, N, ks)));
        count_launches(2);
        GNK_TRY_CUDA(cudaGetLastError());
        GNK_TRY(read_state(b, &hs, st));
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
        for (int j = 0; j < restart; ++j) {
            double* vj = b.V + (size_t)j * N;
            double* w = b.V + (size_t)(j + 1) * N;
            const double nv = j + 1;
            prof_collect_begin();
            GNK_TRY(apply_op(b, adjoint, vj, w, prec, st, &ks->done));
            {
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
