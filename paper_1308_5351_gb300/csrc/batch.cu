// Batched FBIE: many independent domains of uneven connectivity and n, each
// with several right-hand sides gamma, solved together.
//
// * One persistent launch per operator product: a work list of items
//   (domain, target tile, group of right-hand sides), longest first, that the
//   resident blocks pull with an atomic ticket.  Each item streams all source
//   tiles of its domain through shared memory and finishes with the
//   operator's epilogue (no split-source partials: the list has far more
//   items than the GPU has block slots).
// * The inner products use FP32 pair sums; the refinement residual, the
//   right-hand side and h use double-float pair sums (FP64-class).
// * GMRES runs per system (domain, right-hand side), one thread block per
//   system for the Arnoldi, Givens and update kernels, with a per-system
//   done flag; a converged system's right-hand-side group is skipped by the
//   pair kernel.  The restart cycle's Arnoldi steps are captured once into a
//   CUDA graph and replayed, with one host synchronisation per cycle.
// * Autotuning: the targets per thread and the right-hand-side group size of
//   both pair kernels are chosen at build time by timing each variant on a
//   sample of the batch's work list.
//
// * With GNK_PREC_FMM the systems are solved by the single-domain FBIE path
//   with every Cauchy sum by the FMM (one quadtree, power table and near-field
//   cache per domain, kept with the batch): worker threads, each with a CUDA
//   stream of its own, take the domains in turn (largest first) and solve
//   their right-hand sides one after the other, so that several domains'
//   products run on the GPU at once (a product of a domain of a few thousand
//   nodes fills only part of it).  Domains below kBatchFmmMin nodes use
//   double-float direct sums (GNK_PREC_DF32) instead.
//
// Vector layout: system s = (domain d, rhs r) owns elements
// [vec_off_d + r N_d, vec_off_d + (r+1) N_d) of every batch vector.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {
namespace {

constexpr int BS = kSrcTile32;  // sources per tile (tile of the reference nodes)
constexpr int BT = 256;         // threads per block, batched pair kernels
constexpr int KB = 256;         // threads per block, per-system vector kernels
constexpr float kFarB = 1e18f;

struct BDom {
    int node_off, N, n, m1;
    int tile_off, ntiles;
    long long vec_off;
    int nrhs, sys_off;
};

struct BItem {
    int dom, tile, g, cost;
};

struct BSys {
    long long off;
    int N, dom;
};

enum BEpi : int { BE_K = 0, BE_RESID = 1, BE_RESID_FC = 2, BE_RHS_FB = 3, BE_EONE = 4 };

struct BPairArgs {
    const BDom* dom;
    const BItem* items;
    int nitems;
    unsigned* counter;
    const double2* et;
    const double2* ref64;
    const float4* offdf;
    const float4* et32;
    const float4* ref32;
    const float2* off32;
    const double2* q;
    const float2* q32;
    const double2* A;
    const double* b1;
    const double* d1;
    const double* x;
    const double* rhs;
    const double* Lx;
    double* out;
    double* out2;
    int epi;
    const int* sys_done;
};

__device__ __forceinline__ void bepilogue(const BPairArgs& a, const BDom& D, long long e, int node, double zx,
                                          double zy) {
    const double2 A = a.A[node];
    const double x = a.x[e];
    const double s2n = 2.0 / D.n;
    const double fb = 2.0 * x + a.b1[node] * x + s2n * (A.x * zy + A.y * zx);
    switch (a.epi) {
        case BE_K:
            a.out[e] = fb;
            break;
        case BE_RESID:
            a.out[e] = a.rhs[e] - fb;
            break;
        case BE_RESID_FC:
            a.out[e] = a.rhs[e] - fb;
            a.out2[e] = -s2n * (A.x * zx - A.y * zy) - a.d1[node] * x + a.Lx[e];
            break;
        case BE_RHS_FB:
            a.out[e] = -(-s2n * (A.x * zx - A.y * zy) - a.d1[node] * x + a.Lx[e]);
            a.out2[e] = fb;
            break;
        case BE_EONE:  // x = 1: z = E q
            a.out[e] = -s2n * (A.x * zy + A.y * zx);
            a.out2[e] = -s2n * (A.x * zx - A.y * zy);
            break;
    }
}

// Returns the next item index of the block (same in all threads).
__device__ __forceinline__ int next_item(unsigned* counter, int* s_it) {
    __syncthreads();
    if (threadIdx.x == 0) *s_it = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_it;
}

__device__ __forceinline__ bool group_done(const BPairArgs& a, const BDom& D, int r0, int nr) {
    if (!a.sys_done) return false;
    bool all = true;
    for (int r = 0; r < nr; ++r) all = all && (a.sys_done[D.sys_off + r0 + r] != 0);
    return all;
}

// ---------------------------------------------------------------- FP32 persistent kernel
template <int T, int RG>
__global__ void __launch_bounds__(BT) bpair32_kernel(BPairArgs a) {
    __shared__ float2 s_off[BS];
    __shared__ float2 s_w[RG][BS];
    __shared__ int s_it;
    for (;;) {
        const int it = next_item(a.counter, &s_it);
        if (it >= a.nitems) return;
        const BItem item = a.items[it];
        const BDom D = a.dom[item.dom];
        const int r0 = item.g * RG;
        const int nr = min(RG, D.nrhs - r0);
        if (group_done(a, D, r0, nr)) continue;
        const int tgt0 = item.tile * (BT * T);
        float4 th[T];
        int idx[T];
        float ox[T], oy[T], ax[T][RG], ay[T][RG];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            idx[t] = tgt0 + t * BT + threadIdx.x;
            th[t] = a.et32[D.node_off + min(idx[t], D.N - 1)];
#pragma unroll
            for (int r = 0; r < RG; ++r) ax[t][r] = ay[t][r] = 0.f;
        }
        for (int tile = 0; tile < D.ntiles; ++tile) {
            const int j0 = tile * BS;
            const float4 ref = a.ref32[D.tile_off + tile];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                ox[t] = (th[t].x - ref.x) + (th[t].z - ref.z);
                oy[t] = (th[t].y - ref.y) + (th[t].w - ref.w);
            }
            __syncthreads();
            {
                const int k = threadIdx.x, j = j0 + k;
                if (j < D.N) {
                    s_off[k] = a.off32[D.node_off + j];
                    const float2 sc = a.q32[D.node_off + j];
#pragma unroll
                    for (int r = 0; r < RG; ++r) {
                        const float xv = (r < nr) ? (float)a.x[D.vec_off + (long long)(r0 + r) * D.N + j] : 0.f;
                        s_w[r][k] = make_float2(sc.x * xv, sc.y * xv);
                    }
                } else {
                    s_off[k] = make_float2(kFarB, kFarB);
#pragma unroll
                    for (int r = 0; r < RG; ++r) s_w[r][k] = make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
            const bool diag = (j0 < tgt0 + BT * T) && (tgt0 < j0 + BS);
            if (!diag) {
#pragma unroll 4
                for (int k = 0; k < BS; ++k) {
                    const float2 so = s_off[k];
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const float dx = ox[t] - so.x, dy = oy[t] - so.y;
                        const float inv = recip_f32(fmaf(dx, dx, dy * dy));
                        const float ar = dx * inv, ai = dy * inv;
#pragma unroll
                        for (int r = 0; r < RG; ++r) {
                            const float2 w = s_w[r][k];
                            ax[t][r] = fmaf(w.x, ar, fmaf(w.y, ai, ax[t][r]));
                            ay[t][r] = fmaf(w.y, ar, fmaf(-w.x, ai, ay[t][r]));
                        }
                    }
                }
            } else {
                for (int k = 0; k < BS; ++k) {
                    const float2 so = s_off[k];
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const float dx = ox[t] - so.x, dy = oy[t] - so.y;
                        float inv = recip_f32(fmaf(dx, dx, dy * dy));
                        inv = (j0 + k == idx[t]) ? 0.f : inv;
                        const float ar = dx * inv, ai = dy * inv;
#pragma unroll
                        for (int r = 0; r < RG; ++r) {
                            const float2 w = s_w[r][k];
                            ax[t][r] = fmaf(w.x, ar, fmaf(w.y, ai, ax[t][r]));
                            ay[t][r] = fmaf(w.y, ar, fmaf(-w.x, ai, ay[t][r]));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (idx[t] < D.N) {
#pragma unroll
                for (int r = 0; r < RG; ++r)
                    if (r < nr)
                        bepilogue(a, D, D.vec_off + (long long)(r0 + r) * D.N + idx[t], D.node_off + idx[t],
                                  (double)ax[t][r], (double)ay[t][r]);
            }
        }
    }
}

// ---------------------------------------------------------------- double-float persistent kernel
template <int T, int RG>
__global__ void __launch_bounds__(BT) bpairdf_kernel(BPairArgs a) {
    __shared__ float4 s_off[BS];
    __shared__ float4 s_w[RG][BS];
    __shared__ int s_it;
    for (;;) {
        const int it = next_item(a.counter, &s_it);
        if (it >= a.nitems) return;
        const BItem item = a.items[it];
        const BDom D = a.dom[item.dom];
        const int r0 = item.g * RG;
        const int nr = min(RG, D.nrhs - r0);
        if (group_done(a, D, r0, nr)) continue;
        const int tgt0 = item.tile * (BT * T);
        double2 p[T];
        int idx[T];
        df are[T][RG], aim[T][RG];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            idx[t] = tgt0 + t * BT + threadIdx.x;
            p[t] = a.et[D.node_off + min(idx[t], D.N - 1)];
#pragma unroll
            for (int r = 0; r < RG; ++r) are[t][r] = aim[t][r] = df{0.f, 0.f};
        }
        for (int tile = 0; tile < D.ntiles; ++tile) {
            const int j0 = tile * BS;
            const double2 ref = a.ref64[D.tile_off + tile];
            df ox[T], oy[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                ox[t] = df_split(p[t].x - ref.x);
                oy[t] = df_split(p[t].y - ref.y);
            }
            __syncthreads();
            {
                const int k = threadIdx.x, j = j0 + k;
                if (j < D.N) {
                    s_off[k] = a.offdf[D.node_off + j];
                    const double2 sc = a.q[D.node_off + j];
#pragma unroll
                    for (int r = 0; r < RG; ++r) {
                        const double xv = (r < nr) ? a.x[D.vec_off + (long long)(r0 + r) * D.N + j] : 0.0;
                        const df wx = df_split(sc.x * xv), wy = df_split(sc.y * xv);
                        s_w[r][k] = make_float4(wx.h, wx.l, wy.h, wy.l);
                    }
                } else {
                    s_off[k] = make_float4(kFarB, kFarB, 0.f, 0.f);
#pragma unroll
                    for (int r = 0; r < RG; ++r) s_w[r][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
            const bool diag = (j0 < tgt0 + BT * T) && (tgt0 < j0 + BS);
#pragma unroll 2
            for (int k = 0; k < BS; ++k) {
                const float4 so = s_off[k];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const df dx = df_sub(ox[t].h, ox[t].l, so.x, so.z);
                    const df dy = df_sub(oy[t].h, oy[t].l, so.y, so.w);
                    const float px = __fmul_rn(dx.h, dx.h);
                    float ex = fmaf(dx.h, dx.h, -px);
                    ex = fmaf(dx.h, dx.l + dx.l, ex);
                    const float py = __fmul_rn(dy.h, dy.h);
                    float ey = fmaf(dy.h, dy.h, -py);
                    ey = fmaf(dy.h, dy.l + dy.l, ey);
                    float rh, re;
                    two_sum(px, py, rh, re);
                    const float rl = __fadd_rn(__fadd_rn(ex, ey), re);
                    float y = recip_f32(rh);
                    if (diag && j0 + k == idx[t]) y = 0.f;
                    float e = fmaf(-rh, y, 1.0f);
                    e = fmaf(-rl, y, e);
                    const df inv = df{y, __fmul_rn(y, e)};
                    const df ar = df_mul(dx, inv);
                    const df ai = df_mul(dy, inv);
#pragma unroll
                    for (int r = 0; r < RG; ++r) {
                        const float4 w = s_w[r][k];
                        const df wx{w.x, w.y}, wy{w.z, w.w};
                        df_acc(are[t][r], df_mul(wx, ar));
                        df_acc(are[t][r], df_mul(wy, ai));
                        df_acc(aim[t][r], df_mul(wy, ar));
                        const df qq = df_mul(wx, ai);
                        df_acc(aim[t][r], df{-qq.h, -qq.l});
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (idx[t] < D.N) {
#pragma unroll
                for (int r = 0; r < RG; ++r)
                    if (r < nr)
                        bepilogue(a, D, D.vec_off + (long long)(r0 + r) * D.N + idx[t], D.node_off + idx[t],
                                  (double)are[t][r].h + (double)are[t][r].l,
                                  (double)aim[t][r].h + (double)aim[t][r].l);
            }
        }
    }
}

// ---------------------------------------------------------------- per-system GMRES kernels
struct BKry {
    const BSys* sys;
    int nsys, R;         // systems, restart
    long long L;         // batch vector length
    double* V;           // (R+1) x L
    double* H;           // nsys x (R+1) x R
    double* g;           // nsys x (R+1)
    double* cs;          // nsys x R
    double* sn;          // nsys x R
    double* y;           // nsys x R
    double* h1;          // nsys x (R+1)
    double* h2;          // nsys x (R+1)
    double* beta;        // nsys
    double* bnorm;       // nsys
    int* done;           // nsys
    int* kst;            // nsys
    unsigned* unconv;    // count of unconverged systems at a cycle start
    int* nonfinite;
    double tol;
};

__device__ double bsum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < KB / 32; ++w) t += red[w];
        red[KB / 32] = t;
    }
    __syncthreads();
    return red[KB / 32];
}

__global__ void __launch_bounds__(KB) bk_norm(BKry k, const double* __restrict__ v, double* out) {
    __shared__ double red[KB / 32 + 1];
    const BSys S = k.sys[blockIdx.x];
    double a = 0.0;
    for (int i = threadIdx.x; i < S.N; i += KB) {
        const double t = v[S.off + i];
        a = fma(t, t, a);
    }
    const double s = bsum(a, red);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

// cycle start: beta = ||r||, v0 = r / beta, per-system done flag
__global__ void __launch_bounds__(KB) bk_begin(BKry k, const double* __restrict__ r) {
    __shared__ double red[KB / 32 + 1];
    __shared__ int s_done;
    const int s = blockIdx.x;
    const BSys S = k.sys[s];
    double a = 0.0;
    for (int i = threadIdx.x; i < S.N; i += KB) {
        const double t = r[S.off + i];
        a = fma(t, t, a);
    }
    const double nrm = sqrt(bsum(a, red));
    if (threadIdx.x == 0) {
        k.beta[s] = nrm;
        k.kst[s] = 0;
        double* g = k.g + (size_t)s * (k.R + 1);
        g[0] = nrm;
        for (int j = 1; j <= k.R; ++j) g[j] = 0.0;
        if (!isfinite(nrm)) atomicOr(k.nonfinite, 1);
        const int d = !(nrm > k.tol * k.bnorm[s]) ? 1 : 0;
        k.done[s] = d;
        if (!d) atomicAdd(k.unconv, 1u);
        s_done = d;
    }
    __syncthreads();
    if (s_done) return;
    const double inv = 1.0 / nrm;
    for (int i = threadIdx.x; i < S.N; i += KB) k.V[S.off + i] = r[S.off + i] * inv;
}

// h1 = V(:, 0..j)^T w
__global__ void __launch_bounds__(KB) bk_dots(BKry k, int j) {
    __shared__ double red[KB / 32 + 1];
    const int s = blockIdx.x;
    if (k.done[s]) return;
    const BSys S = k.sys[s];
    const double* w = k.V + (size_t)(j + 1) * k.L + S.off;
    for (int c = 0; c <= j; ++c) {
        const double* v = k.V + (size_t)c * k.L + S.off;
        double a = 0.0;
        for (int i = threadIdx.x; i < S.N; i += KB) a = fma(v[i], w[i], a);
        const double t = bsum(a, red);
        if (threadIdx.x == 0) k.h1[(size_t)s * (k.R + 1) + c] = t;
    }
}

// w -= V h1, then h2 = V^T w
__global__ void __launch_bounds__(KB) bk_update_dots(BKry k, int j) {
    __shared__ double red[KB / 32 + 1];
    __shared__ double hs[1024];
    const int s = blockIdx.x;
    if (k.done[s]) return;
    const BSys S = k.sys[s];
    for (int c = threadIdx.x; c <= j; c += KB) hs[c] = k.h1[(size_t)s * (k.R + 1) + c];
    __syncthreads();
    double* w = k.V + (size_t)(j + 1) * k.L + S.off;
    for (int i = threadIdx.x; i < S.N; i += KB) {
        double acc = w[i];
        for (int c = 0; c <= j; ++c) acc = fma(-hs[c], k.V[(size_t)c * k.L + S.off + i], acc);
        w[i] = acc;
    }
    __syncthreads();
    for (int c = 0; c <= j; ++c) {
        const double* v = k.V + (size_t)c * k.L + S.off;
        double a = 0.0;
        for (int i = threadIdx.x; i < S.N; i += KB) a = fma(v[i], w[i], a);
        const double t = bsum(a, red);
        if (threadIdx.x == 0) k.h2[(size_t)s * (k.R + 1) + c] = t;
    }
}

// w -= V h2, ||w||, Hessenberg column, Givens rotations, convergence test,
// triangular solve at the end of the cycle, v_{j+1} = w / ||w|| otherwise.
__global__ void __launch_bounds__(KB) bk_norm_givens(BKry k, int j) {
    __shared__ double red[KB / 32 + 1];
    __shared__ double hs[1024];
    __shared__ int s_stop;
    __shared__ double s_hn;
    const int s = blockIdx.x;
    if (k.done[s]) return;
    const BSys S = k.sys[s];
    const int ld = k.R + 1;
    for (int c = threadIdx.x; c <= j; c += KB) hs[c] = k.h2[(size_t)s * ld + c];
    __syncthreads();
    double* w = k.V + (size_t)(j + 1) * k.L + S.off;
    double a = 0.0;
    for (int i = threadIdx.x; i < S.N; i += KB) {
        double acc = w[i];
        for (int c = 0; c <= j; ++c) acc = fma(-hs[c], k.V[(size_t)c * k.L + S.off + i], acc);
        w[i] = acc;
        a = fma(acc, acc, a);
    }
    const double hn = sqrt(bsum(a, red));
    if (threadIdx.x == 0) {
        double* H = k.H + (size_t)s * ld * k.R;
        double* col = H + (size_t)j * ld;
        double* g = k.g + (size_t)s * ld;
        double* cs = k.cs + (size_t)s * k.R;
        double* sn = k.sn + (size_t)s * k.R;
        for (int c = 0; c <= j; ++c) col[c] = k.h1[(size_t)s * ld + c] + k.h2[(size_t)s * ld + c];
        col[j + 1] = hn;
        for (int c = 0; c < j; ++c) {
            const double x0 = col[c], x1 = col[c + 1];
            col[c] = cs[c] * x0 + sn[c] * x1;
            col[c + 1] = -sn[c] * x0 + cs[c] * x1;
        }
        const double x0 = col[j], x1 = col[j + 1];
        const double rr = hypot(x0, x1);
        const double c = (rr > 0.0) ? x0 / rr : 1.0;
        const double sg = (rr > 0.0) ? x1 / rr : 0.0;
        cs[j] = c;
        sn[j] = sg;
        col[j] = rr;
        col[j + 1] = 0.0;
        g[j + 1] = -sg * g[j];
        g[j] = c * g[j];
        const double est = fabs(g[j + 1]);
        k.kst[s] = j + 1;
        const bool bad = !isfinite(est) || !isfinite(hn);
        if (bad) atomicOr(k.nonfinite, 1);
        const bool stop = bad || est <= k.tol * k.bnorm[s] || j + 1 == k.R || hn == 0.0;
        if (stop) {
            double* y = k.y + (size_t)s * k.R;
            const int kk = j + 1;
            for (int row = kk - 1; row >= 0; --row) {
                double v = g[row];
                for (int cc = row + 1; cc < kk; ++cc) v -= H[(size_t)cc * ld + row] * y[cc];
                const double d = H[(size_t)row * ld + row];
                y[row] = (d != 0.0) ? v / d : 0.0;
            }
            k.done[s] = 1;
        }
        s_stop = stop;
        s_hn = hn;
    }
    __syncthreads();
    if (s_stop) return;
    const double inv = 1.0 / s_hn;
    for (int i = threadIdx.x; i < S.N; i += KB) w[i] *= inv;
}

__global__ void __launch_bounds__(KB) bk_update_x(BKry k, double* __restrict__ x) {
    __shared__ double ys[1024];
    const int s = blockIdx.x;
    const int kk = k.kst[s];
    if (kk == 0) return;
    const BSys S = k.sys[s];
    for (int c = threadIdx.x; c < kk; c += KB) ys[c] = k.y[(size_t)s * k.R + c];
    __syncthreads();
    for (int i = threadIdx.x; i < S.N; i += KB) {
        double acc = x[S.off + i];
        for (int c = 0; c < kk; ++c) acc = fma(ys[c], k.V[(size_t)c * k.L + S.off + i], acc);
        x[S.off + i] = acc;
    }
}

// Outer check: relres_s = ||r_s|| / ||b_s||; converged systems get r_s = 0 so
// that the inner solve leaves them alone; counts the unconverged ones.
__global__ void __launch_bounds__(KB) bk_outer_check(BKry k, double* __restrict__ r, const double* __restrict__ bn,
                                                     double* __restrict__ relres, double tol, unsigned* unconv,
                                                     int* __restrict__ conv) {
    __shared__ double red[KB / 32 + 1];
    __shared__ int s_conv;
    const int s = blockIdx.x;
    const BSys S = k.sys[s];
    double a = 0.0;
    for (int i = threadIdx.x; i < S.N; i += KB) {
        const double t = r[S.off + i];
        a = fma(t, t, a);
    }
    const double nrm = sqrt(bsum(a, red));
    if (threadIdx.x == 0) {
        const double rel = (bn[s] > 0.0) ? nrm / bn[s] : 0.0;
        relres[s] = rel;
        if (!isfinite(rel)) atomicOr(k.nonfinite, 1);
        s_conv = (rel <= tol) ? 1 : 0;
        conv[s] = s_conv;
        if (!s_conv) atomicAdd(unconv, 1u);
    }
    __syncthreads();
    if (!s_conv) return;
    for (int i = threadIdx.x; i < S.N; i += KB) r[S.off + i] = 0.0;
}

__global__ void bk_axpy(long long L, double* __restrict__ x, const double* __restrict__ d) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < L) x[i] += d[i];
}

__global__ void bk_half_diff(long long L, const double* a, const double* b, double* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < L) out[i] = 0.5 * (a[i] - b[i]);
}

// h_k: mean of h over each component, per system; out[hk_off_s + c]
__global__ void bk_hk(const BSys* sys, const BDom* dom, const int* hk_off, const double* h, double* out) {
    const BSys S = sys[blockIdx.x];
    const BDom D = dom[S.dom];
    for (int c = threadIdx.x; c < D.m1; c += blockDim.x) {
        double t = 0.0;
        for (int p = 0; p < D.n; ++p) t += h[S.off + (long long)c * D.n + p];
        out[hk_off[blockIdx.x] + c] = t / D.n;
    }
}

template <class P>
int dalloc(P** p, size_t count) {
    if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(P) + 16) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch: device allocation of %zu bytes failed", count * sizeof(P));
        return GNK_ENOMEM;
    }
    return GNK_OK;
}

}  // namespace

// ---------------------------------------------------------------- batch handle
struct BatchImpl {
    int ndom = 0, Ntot = 0, ntiles = 0, nsys = 0, nhk = 0, nmax = 0;
    long long L = 0;
    int sms = 0;
    std::vector<BDom> hdom, hdom1;
    BDom* dom = nullptr;    // systems layout (nrhs per domain)
    BDom* dom1 = nullptr;   // one right-hand side per domain (vector = node layout)
    BSys* sys = nullptr;
    int* hk_off = nullptr;
    // geometry
    double2 *et = nullptr, *etp = nullptr, *A = nullptr, *q = nullptr, *ref64 = nullptr, *Eone = nullptr;
    double *b1 = nullptr, *d1 = nullptr, *e = nullptr, *ones = nullptr;
    float4 *et32 = nullptr, *ref32 = nullptr, *offdf = nullptr;
    float2 *off32 = nullptr, *q32 = nullptr, *A32 = nullptr;
    // circulant
    double2* twid = nullptr;
    double* lcol = nullptr;
    int4* cdesc = nullptr;
    long long* cbase = nullptr;
    int ncirc = 0;
    // work lists (per kernel variant: targets per thread T, group size RG)
    int T32 = 2, RG32 = 8, Tdf = 1, RGdf = 4;       // shapes of the current work lists
    int T32t = 2, RG32t = 8, Tdft = 1, RGdft = 4;   // tuned (or default) shapes
    BItem* items32 = nullptr;
    int nitems32 = 0;
    BItem* itemsdf = nullptr;
    int nitemsdf = 0;
    BItem* itemsdf1 = nullptr;
    int nitemsdf1 = 0;
    unsigned* counter = nullptr;
    float tune_ms[8] = {0};
    // vectors (L doubles each)
    double *rhs = nullptr, *x = nullptr, *r = nullptr, *rr = nullptr, *dd = nullptr, *fb = nullptr,
           *fc = nullptr, *Lx = nullptr;
    // Krylov
    int R = 0;
    BKry k;
    double *bnorm_in = nullptr, *bnorm_out = nullptr, *relres = nullptr;
    int* oconv = nullptr;  // per system: converged at the outer (refinement) level
    cudaGraphExec_t graph = nullptr;
    int graph_R = -1;
    double graph_tol = -1.0;
    cudaStream_t graph_stream = nullptr;
    double last_tune_total = 0.0;
    // FMM path: per-domain handles (built on first use), boundedness, the
    // systems' hk offsets, the worker streams
    std::vector<int> hbounded;
    std::vector<int> hhk;
    std::vector<gnk_boundary*> fmm_h;
    std::vector<cudaStream_t> wstreams;
    int device = 0;
};

namespace {

std::vector<BItem> make_items(const std::vector<BDom>& D, int T, int RG) {
    std::vector<BItem> v;
    for (int d = 0; d < (int)D.size(); ++d) {
        const int tiles = (D[d].N + BT * T - 1) / (BT * T);
        const int groups = (D[d].nrhs + RG - 1) / RG;
        for (int t = 0; t < tiles; ++t)
            for (int g = 0; g < groups; ++g) {
                const int nt = std::min(BT * T, D[d].N - t * BT * T);
                const int nr = std::min(RG, D[d].nrhs - g * RG);
                BItem it{d, t, g, 0};
                // cost in units of 4096 pair-evaluations (for the longest-first order)
                it.cost = (int)std::min<long long>((long long)nt * D[d].N * nr / 4096 + 1, 1LL << 30);
                v.push_back(it);
            }
    }
    std::stable_sort(v.begin(), v.end(), [](const BItem& a, const BItem& b) { return a.cost > b.cost; });
    return v;
}

BPairArgs base_args(const BatchImpl& B, const BDom* dom) {
    BPairArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dom = dom;
    a.counter = B.counter;
    a.et = B.et;
    a.ref64 = B.ref64;
    a.offdf = B.offdf;
    a.et32 = B.et32;
    a.ref32 = B.ref32;
    a.off32 = B.off32;
    a.q = B.q;
    a.q32 = B.q32;
    a.A = B.A;
    a.b1 = B.b1;
    a.d1 = B.d1;
    return a;
}

int launch32(const BatchImpl& B, BPairArgs a, int T, int RG, const BItem* items, int nitems, cudaStream_t st) {
    a.items = items;
    a.nitems = nitems;
    GNK_TRY_CUDA(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), st));
    int nb = 1;
    const int slots = B.sms;
    const ProfToken tok = prof_begin(st);
#define L32(TT, GG)                                                                                   \
    if (T == TT && RG == GG) {                                                                        \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bpair32_kernel<TT, GG>, BT, 0);           \
        bpair32_kernel<TT, GG><<<std::max(1, nb) * slots, BT, 0, st>>>(a);                           \
    }
    L32(1, 8) else L32(2, 4) else L32(2, 8) else L32(4, 4) else {
        set_error("batch: no FP32 kernel variant T=%d RG=%d", T, RG);
        return GNK_EINVAL;
    }
#undef L32
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tok, PK_PAIR32, 0.0, st);
    count_launches(2);
    return GNK_OK;
}

int launchdf(const BatchImpl& B, BPairArgs a, int T, int RG, const BItem* items, int nitems, cudaStream_t st) {
    a.items = items;
    a.nitems = nitems;
    GNK_TRY_CUDA(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), st));
    int nb = 1;
    const int slots = B.sms;
    const ProfToken tok = prof_begin(st);
#define LDF(TT, GG)                                                                                   \
    if (T == TT && RG == GG) {                                                                        \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bpairdf_kernel<TT, GG>, BT, 0);           \
        bpairdf_kernel<TT, GG><<<std::max(1, nb) * slots, BT, 0, st>>>(a);                           \
    }
    LDF(1, 1) else LDF(1, 2) else LDF(1, 4) else LDF(2, 2) else {
        set_error("batch: no double-float kernel variant T=%d RG=%d", T, RG);
        return GNK_EINVAL;
    }
#undef LDF
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tok, PK_PAIRDF, 0.0, st);
    count_launches(2);
    return GNK_OK;
}

int upload_items(const std::vector<BItem>& v, BItem** d, int* n, cudaStream_t st) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    GNK_TRY(dalloc(d, std::max<size_t>(1, v.size())));
    if (!v.empty())
        GNK_TRY_CUDA(cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(BItem), cudaMemcpyHostToDevice, st));
    *n = (int)v.size();
    return GNK_OK;
}

// The tile shapes of one call: the tuned shapes, or the override of
// gnk_options.tile_variant (1..4: the FP32 kernel, 5..7: the double-float
// kernel, in the order of gnk_batch_tuning).  The work lists are rebuilt, and
// the captured Arnoldi cycle dropped, only when a shape changes.
int apply_tiles(BatchImpl& B, int variant, cudaStream_t st) {
    static const int v32[][2] = {{1, 8}, {2, 4}, {2, 8}, {4, 4}};
    static const int vdf[][2] = {{1, 2}, {1, 4}, {2, 2}};
    int T32 = B.T32t, RG32 = B.RG32t, Tdf = B.Tdft, RGdf = B.RGdft;
    if (variant >= 1 && variant <= 4) {
        T32 = v32[variant - 1][0];
        RG32 = v32[variant - 1][1];
    } else if (variant >= 5 && variant <= 7) {
        Tdf = vdf[variant - 5][0];
        RGdf = vdf[variant - 5][1];
    }
    if (T32 != B.T32 || RG32 != B.RG32) {
        GNK_TRY(upload_items(make_items(B.hdom, T32, RG32), &B.items32, &B.nitems32, st));
        B.T32 = T32;
        B.RG32 = RG32;
        B.graph_R = -1;
    }
    if (Tdf != B.Tdf || RGdf != B.RGdf) {
        GNK_TRY(upload_items(make_items(B.hdom, Tdf, RGdf), &B.itemsdf, &B.nitemsdf, st));
        B.Tdf = Tdf;
        B.RGdf = RGdf;
        B.graph_R = -1;
    }
    return GNK_OK;
}

// Time `reps` launches of one variant on the sampled item list.
template <class F>
float time_variant(F launch, cudaStream_t st) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int autotune(BatchImpl& B, cudaStream_t st) {
    // sample: every 8th domain (all of them for small batches)
    std::vector<BDom> sample;
    for (int d = 0; d < B.ndom; ++d)
        if (B.ndom < 16 || d % 8 == 0) sample.push_back(B.hdom[d]);
    BDom* dsample = nullptr;
    GNK_TRY(dalloc(&dsample, sample.size()));
    GNK_TRY_CUDA(cudaMemcpyAsync(dsample, sample.data(), sample.size() * sizeof(BDom), cudaMemcpyHostToDevice, st));
    // operands: x = 1 on every system element (weights q), output into fb
    BPairArgs a = base_args(B, dsample);
    a.x = B.fc;
    a.out = B.fb;
    a.epi = BE_K;
    const int v32[][2] = {{1, 8}, {2, 4}, {2, 8}, {4, 4}};
    const int vdf[][2] = {{1, 2}, {1, 4}, {2, 2}};
    float best = 1e30f;
    BItem* it = nullptr;
    int nit = 0;
    int rc = GNK_OK;
    for (int v = 0; v < 4 && rc == GNK_OK; ++v) {
        rc = upload_items(make_items(sample, v32[v][0], v32[v][1]), &it, &nit, st);
        if (rc != GNK_OK) break;
        const float ms = time_variant([&] { launch32(B, a, v32[v][0], v32[v][1], it, nit, st); }, st);
        B.tune_ms[v] = ms;
        if (ms < best) {
            best = ms;
            B.T32 = v32[v][0];
            B.RG32 = v32[v][1];
        }
    }
    best = 1e30f;
    for (int v = 0; v < 3 && rc == GNK_OK; ++v) {
        rc = upload_items(make_items(sample, vdf[v][0], vdf[v][1]), &it, &nit, st);
        if (rc != GNK_OK) break;
        const float ms = time_variant([&] { launchdf(B, a, vdf[v][0], vdf[v][1], it, nit, st); }, st);
        B.tune_ms[4 + v] = ms;
        if (ms < best) {
            best = ms;
            B.Tdf = vdf[v][0];
            B.RGdf = vdf[v][1];
        }
    }
    if (it) cudaFree(it);
    cudaFree(dsample);
    GNK_TRY_CUDA(cudaGetLastError());
    return rc;
}

void release_batch(BatchImpl& B) {
    for (gnk_boundary* h : B.fmm_h)
        if (h) gnk_free_boundary(h);
    B.fmm_h.clear();
    for (cudaStream_t w : B.wstreams)
        if (w) cudaStreamDestroy(w);
    B.wstreams.clear();
    void* p[] = {B.dom, B.dom1, B.sys, B.hk_off, B.et, B.etp, B.A, B.q, B.ref64, B.Eone, B.b1, B.d1, B.e, B.ones,
                 B.et32, B.ref32, B.offdf, B.off32, B.q32, B.A32, B.twid, B.lcol, B.cdesc, B.cbase, B.items32,
                 B.itemsdf, B.itemsdf1, B.counter, B.rhs, B.x, B.r, B.rr, B.dd, B.fb, B.fc, B.Lx, B.k.V, B.k.H,
                 B.k.g, B.k.cs, B.k.sn, B.k.y, B.k.h1, B.k.h2, B.k.beta, B.k.done, B.k.kst,
                 B.k.unconv, B.k.nonfinite, B.bnorm_in, B.bnorm_out, B.relres, B.oconv};
    for (void* q : p)
        if (q) cudaFree(q);
    if (B.graph) cudaGraphExecDestroy(B.graph);
}

int ensure_krylov_batch(BatchImpl& B, int R) {
    if (B.R >= R && B.k.V) return GNK_OK;
    void* p[] = {B.k.V, B.k.H, B.k.g, B.k.cs, B.k.sn, B.k.y, B.k.h1, B.k.h2};
    for (void* q : p)
        if (q) cudaFree(q);
    const size_t ns = B.nsys;
    GNK_TRY(dalloc(&B.k.V, (size_t)(R + 1) * B.L));
    GNK_TRY(dalloc(&B.k.H, ns * (R + 1) * R));
    GNK_TRY(dalloc(&B.k.g, ns * (R + 1)));
    GNK_TRY(dalloc(&B.k.cs, ns * R));
    GNK_TRY(dalloc(&B.k.sn, ns * R));
    GNK_TRY(dalloc(&B.k.y, ns * R));
    GNK_TRY(dalloc(&B.k.h1, ns * (R + 1)));
    GNK_TRY(dalloc(&B.k.h2, ns * (R + 1)));
    B.R = R;
    if (B.graph) {
        cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
        B.graph_R = -1;
    }
    return GNK_OK;
}

// Arnoldi steps of one cycle with the FP32 operator (captured into a graph).
int enqueue_cycle(BatchImpl& B, cudaStream_t st) {
    const int R = B.k.R;
    for (int j = 0; j < R; ++j) {
        BPairArgs a = base_args(B, B.dom);
        a.x = B.k.V + (size_t)j * B.L;
        a.out = B.k.V + (size_t)(j + 1) * B.L;
        a.epi = BE_K;
        a.sys_done = B.k.done;
        GNK_TRY(launch32(B, a, B.T32, B.RG32, B.items32, B.nitems32, st));
        bk_dots<<<B.nsys, KB, 0, st>>>(B.k, j);
        bk_update_dots<<<B.nsys, KB, 0, st>>>(B.k, j);
        bk_norm_givens<<<B.nsys, KB, 0, st>>>(B.k, j);
        GNK_TRY_CUDA(cudaGetLastError());
        count_launches(3);
    }
    return GNK_OK;
}

// Batched GMRES with the FP32 operator: x = K32^-1 rhs per system.
int gmres_batch(BatchImpl& B, const double* rhs, double* x, int R, int maxit, double tol, int* steps,
                int* cycles_out, cudaStream_t st) {
    GNK_TRY(ensure_krylov_batch(B, R));
    B.k.tol = tol;
    B.k.R = R;
    B.k.L = B.L;
    B.k.bnorm = B.bnorm_in;
    const int ns = B.nsys;
    bk_norm<<<ns, KB, 0, st>>>(B.k, rhs, B.bnorm_in);
    GNK_TRY_CUDA(cudaMemsetAsync(x, 0, B.L * sizeof(double), st));
    count_launches(1);
    // graph of one cycle's Arnoldi steps (kernel arguments fixed per handle and R)
    if (!B.graph || B.graph_R != R || B.graph_tol != tol) {
        if (B.graph) cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
        cudaStream_t cs;
        GNK_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        GNK_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        count_suppress(true);
        const int rc = enqueue_cycle(B, cs);
        count_suppress(false);
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        GNK_TRY(rc);
        GNK_TRY_CUDA(e);
        GNK_TRY_CUDA(cudaGraphInstantiate(&B.graph, g, 0));
        cudaGraphDestroy(g);
        B.graph_R = R;
        B.graph_tol = tol;
    }
    *steps = 0;
    int cycles = 0;
    for (int cycle = 0;; ++cycle) {
        if (cycle == 0) {
            GNK_TRY_CUDA(cudaMemcpyAsync(B.r, rhs, B.L * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            BPairArgs a = base_args(B, B.dom);
            a.x = x;
            a.rhs = rhs;
            a.out = B.r;
            a.epi = BE_RESID;
            GNK_TRY(launch32(B, a, B.T32, B.RG32, B.items32, B.nitems32, st));
        }
        GNK_TRY_CUDA(cudaMemsetAsync(B.k.unconv, 0, sizeof(unsigned), st));
        bk_begin<<<ns, KB, 0, st>>>(B.k, B.r);
        count_launches(1);
        unsigned unconv = 0;
        GNK_TRY_CUDA(cudaMemcpyAsync(&unconv, B.k.unconv, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        GNK_TRY_CUDA(cudaStreamSynchronize(st));
        if (unconv == 0 || cycle == maxit) break;
        GNK_TRY_CUDA(cudaGraphLaunch(B.graph, st));
        count_launches((unsigned long long)R * 5);
        bk_update_x<<<ns, KB, 0, st>>>(B.k, x);
        GNK_TRY_CUDA(cudaGetLastError());
        count_launches(1);
        *steps += R;
        ++cycles;
    }
    *cycles_out += cycles;
    return GNK_OK;
}

// ---------------------------------------------------------------- FMM path
constexpr int kBatchFmmMin = 4096;  // nodes: smaller domains use double-float direct sums
constexpr int kBatchWorkers = 8;    // host threads, each with a CUDA stream of its own

}  // namespace

// Solves every system of the batch by gnk_fbie on a per-domain handle (FMM
// products, or double-float direct sums below kBatchFmmMin nodes), the domains
// taken largest first by kBatchWorkers worker threads.  g, x, hv, hkd: device
// batch vectors (gamma in, mu, h and the systems' h_k out).
static int run_batch_fmm(BatchImpl& B, const double* g, double* x, double* hv, double* hkd, const gnk_options& o,
                  gnk_result* res, std::vector<double>* rel, cudaStream_t st) {
    std::vector<int> order(B.ndom);
    for (int d = 0; d < B.ndom; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
        return (long long)B.hdom[u].N * B.hdom[u].nrhs > (long long)B.hdom[v].N * B.hdom[v].nrhs;
    });
    const int nw = std::min(kBatchWorkers, B.ndom);
    while ((int)B.wstreams.size() < nw) {
        cudaStream_t w = nullptr;
        GNK_TRY_CUDA(cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking));
        B.wstreams.push_back(w);
    }
    GNK_TRY_CUDA(cudaStreamSynchronize(st));  // gamma is in place before the workers start
    std::atomic<int> next{0};
    std::mutex mu;
    int first_rc = GNK_OK;
    std::string first_msg;
    std::vector<int> iters(B.nsys, 0), cycles(B.nsys, 0), stat(B.nsys, GNK_OK);
    auto worker = [&](int wi) {
        if (cudaSetDevice(B.device) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            if (first_rc == GNK_OK) {
                first_rc = GNK_ECUDA;
                first_msg = "cudaSetDevice failed in a worker thread";
            }
            return;
        }
        cudaStream_t ws = B.wstreams[wi];
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= B.ndom) break;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (first_rc != GNK_OK) break;
            }
            const int d = order[k];
            const BDom& D = B.hdom[d];
            const int prec = D.N >= kBatchFmmMin ? GNK_PREC_FMM : GNK_PREC_DF32;
            int rc = GNK_OK;
            if (!B.fmm_h[d]) {
                gnk_boundary* h = nullptr;
                rc = gnk_build_boundary_ex(&h, D.m1, D.n, reinterpret_cast<const double*>(B.et + D.node_off),
                                           reinterpret_cast<const double*>(B.etp + D.node_off), nullptr,
                                           reinterpret_cast<const double*>(B.A + D.node_off), nullptr,
                                           B.hbounded[d], prec | GNK_BUILD_DEFER, ws);
                if (rc == GNK_OK) B.fmm_h[d] = h;
            }
            gnk_options od = o;
            od.precision = prec;
            od.timing = 0;
            od.tile_variant = 0;
            for (int r = 0; r < D.nrhs && rc == GNK_OK; ++r) {
                const int sidx = D.sys_off + r;
                const long long off = D.vec_off + (long long)r * D.N;
                gnk_result rr;
                std::memset(&rr, 0, sizeof(rr));
                rc = gnk_fbie(B.fmm_h[d], g + off, x + off, hv + off, hkd + B.hhk[sidx], &od, &rr, ws);
                if (rc == GNK_ENOTCONV || rc == GNK_ENONFINITE) rc = GNK_OK;  // kept per system
                (*rel)[sidx] = rr.relres;
                iters[sidx] = rr.iterations;
                cycles[sidx] = rr.cycles;
                stat[sidx] = rr.status;
            }
            if (rc == GNK_OK && cudaStreamSynchronize(ws) != cudaSuccess) {
                set_error("batch (FMM): %s", cudaGetErrorString(cudaGetLastError()));
                rc = GNK_ECUDA;
            }
            if (rc != GNK_OK) {
                char buf[1024];
                gnk_last_error(buf, sizeof(buf));
                std::lock_guard<std::mutex> lk(mu);
                if (first_rc == GNK_OK) {
                    first_rc = rc;
                    first_msg = buf;
                }
            }
        }
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < nw; ++w) threads.emplace_back(worker, w);
    for (std::thread& t : threads) t.join();
    if (first_rc != GNK_OK) {
        set_error("batch (FMM): %s", first_msg.c_str());
        return first_rc;
    }
    int status = GNK_OK;
    for (int sidx = 0; sidx < B.nsys; ++sidx) {
        res->iterations += iters[sidx];
        res->cycles += cycles[sidx];
        res->matvecs_fp64 += iters[sidx] + 2;
        if (stat[sidx] == GNK_ENONFINITE) status = GNK_ENONFINITE;
        else if (stat[sidx] == GNK_ENOTCONV && status == GNK_OK) status = GNK_ENOTCONV;
    }
    return status;
}

}  // namespace gnk

using namespace gnk;

struct gnk_batch {
    BatchImpl b;
};

extern "C" {

int gnk_build_batch(gnk_batch** out, int ndom, const int* m1, const int* n, const int* nrhs, const int* bounded,
                    const double* et, const double* etp, const double* A, int autotune_flag, void* stream) {
    if (!out || ndom < 1 || !m1 || !n || !nrhs || !bounded || !et || !etp || !A) {
        set_error("gnk_build_batch: bad arguments");
        return GNK_EINVAL;
    }
    *out = nullptr;
    cudaGetLastError();  // a stale, non-sticky error of earlier calls is not ours
    long long Ntot = 0, L = 0;
    int nmax = 0, nsys = 0, nhk = 0, ntiles = 0;
    for (int d = 0; d < ndom; ++d) {
        if (m1[d] < 1 || n[d] < 4 || n[d] > 4096 || (n[d] % 2) || nrhs[d] < 1) {
            set_error("gnk_build_batch: domain %d needs m1 >= 1, even 4 <= n <= 4096, nrhs >= 1", d);
            return GNK_EINVAL;
        }
        const long long N = (long long)m1[d] * n[d];
        Ntot += N;
        L += N * nrhs[d];
        ntiles += (int)((N + BS - 1) / BS);
        nmax = std::max(nmax, n[d]);
        nsys += nrhs[d];
        nhk += nrhs[d] * m1[d];
    }
    if (Ntot > (1LL << 28) || L > (1LL << 34)) {
        set_error("gnk_build_batch: batch too large (nodes %lld, vector length %lld)", Ntot, L);
        return GNK_EINVAL;
    }
    gnk_batch* h = new (std::nothrow) gnk_batch();
    if (!h) return GNK_ENOMEM;
    BatchImpl& B = h->b;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = GNK_OK;
    auto fail = [&](int code) {
        release_batch(B);
        delete h;
        return code;
    };
    B.ndom = ndom;
    B.hbounded.assign(bounded, bounded + ndom);
    B.fmm_h.assign(ndom, nullptr);
    B.Ntot = (int)Ntot;
    B.L = L;
    B.nmax = nmax;
    B.nsys = nsys;
    B.nhk = nhk;
    B.ntiles = ntiles;
    int dev = 0;
    cudaGetDevice(&dev);
    B.device = dev;
    cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, dev);
    // tables
    std::vector<BSys> hsys;
    std::vector<int> hhk;
    std::vector<int4> desc;
    std::vector<long long> base;
    std::vector<double2> twall;
    std::vector<double> colall;
    std::vector<int> nseen, noff;
    int node = 0, tile = 0, sys = 0, hk = 0;
    long long vec = 0;
    for (int d = 0; d < ndom; ++d) {
        BDom D;
        D.node_off = node;
        D.N = m1[d] * n[d];
        D.n = n[d];
        D.m1 = m1[d];
        D.tile_off = tile;
        D.ntiles = (D.N + BS - 1) / BS;
        D.vec_off = vec;
        D.nrhs = nrhs[d];
        D.sys_off = sys;
        B.hdom.push_back(D);
        BDom D1 = D;
        D1.vec_off = node;
        D1.nrhs = 1;
        D1.sys_off = d;
        B.hdom1.push_back(D1);
        // circulant table of this n
        int toff = -1, pow2 = ((n[d] & (n[d] - 1)) == 0) && n[d] <= 4096;
        for (size_t u = 0; u < nseen.size(); ++u)
            if (nseen[u] == n[d]) toff = noff[u];
        if (toff < 0) {
            std::vector<double2> tw;
            std::vector<double> col;
            circulant_tables(n[d], &tw, &col);
            toff = pow2 ? (int)twall.size() : (int)colall.size();
            twall.insert(twall.end(), tw.begin(), tw.end());
            colall.insert(colall.end(), col.begin(), col.end());
            nseen.push_back(n[d]);
            noff.push_back(toff);
        }
        for (int r = 0; r < nrhs[d]; ++r) {
            hsys.push_back(BSys{vec + (long long)r * D.N, D.N, d});
            hhk.push_back(hk);
            hk += m1[d];
            for (int p = 0; p < (m1[d] + 1) / 2; ++p) {
                desc.push_back(make_int4(n[d], m1[d], p, toff | (pow2 << 30)));
                base.push_back(vec + (long long)r * D.N);
            }
        }
        node += D.N;
        tile += D.ntiles;
        sys += nrhs[d];
        vec += (long long)D.N * nrhs[d];
    }
    B.ncirc = (int)desc.size();
    B.hhk = hhk;
    const size_t N = Ntot;
    rc = GNK_OK;
#define TRYB(x)                 \
    do {                        \
        rc = (x);               \
        if (rc != GNK_OK) return fail(rc); \
    } while (0)
    TRYB(dalloc(&B.dom, ndom));
    TRYB(dalloc(&B.dom1, ndom));
    TRYB(dalloc(&B.sys, nsys));
    TRYB(dalloc(&B.hk_off, nsys));
    TRYB(dalloc(&B.et, N));
    TRYB(dalloc(&B.etp, N));
    TRYB(dalloc(&B.A, N));
    TRYB(dalloc(&B.q, N));
    TRYB(dalloc(&B.Eone, N));
    TRYB(dalloc(&B.b1, N));
    TRYB(dalloc(&B.d1, N));
    TRYB(dalloc(&B.e, N));
    TRYB(dalloc(&B.ones, N));
    TRYB(dalloc(&B.et32, N));
    TRYB(dalloc(&B.offdf, N));
    TRYB(dalloc(&B.off32, N));
    TRYB(dalloc(&B.q32, N));
    TRYB(dalloc(&B.A32, N));
    TRYB(dalloc(&B.ref32, (size_t)ntiles));
    TRYB(dalloc(&B.ref64, (size_t)ntiles));
    TRYB(dalloc(&B.twid, std::max<size_t>(1, twall.size())));
    TRYB(dalloc(&B.lcol, std::max<size_t>(1, colall.size())));
    TRYB(dalloc(&B.cdesc, desc.size()));
    TRYB(dalloc(&B.cbase, base.size()));
    TRYB(dalloc(&B.counter, 1));
    const size_t Lz = (size_t)L;
    TRYB(dalloc(&B.rhs, Lz));
    TRYB(dalloc(&B.x, Lz));
    TRYB(dalloc(&B.r, Lz));
    TRYB(dalloc(&B.rr, Lz));
    TRYB(dalloc(&B.dd, Lz));
    TRYB(dalloc(&B.fb, Lz));
    TRYB(dalloc(&B.fc, Lz));
    TRYB(dalloc(&B.Lx, Lz));
    TRYB(dalloc(&B.k.beta, nsys));
    TRYB(dalloc(&B.k.done, nsys));
    TRYB(dalloc(&B.k.kst, nsys));
    TRYB(dalloc(&B.k.unconv, 1));
    TRYB(dalloc(&B.k.nonfinite, 1));
    TRYB(dalloc(&B.bnorm_in, nsys));
    TRYB(dalloc(&B.bnorm_out, nsys));
    TRYB(dalloc(&B.relres, nsys));
    TRYB(dalloc(&B.oconv, nsys));
    B.k.sys = B.sys;
    B.k.nsys = nsys;
    B.k.L = L;
    B.k.bnorm = B.bnorm_in;  // alias, owned through bnorm_in
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess ? GNK_OK : GNK_ECUDA;
    };
    TRYB(up(B.dom, B.hdom.data(), ndom * sizeof(BDom)));
    TRYB(up(B.dom1, B.hdom1.data(), ndom * sizeof(BDom)));
    TRYB(up(B.sys, hsys.data(), nsys * sizeof(BSys)));
    TRYB(up(B.hk_off, hhk.data(), nsys * sizeof(int)));
    if (!twall.empty()) TRYB(up(B.twid, twall.data(), twall.size() * sizeof(double2)));
    if (!colall.empty()) TRYB(up(B.lcol, colall.data(), colall.size() * sizeof(double)));
    TRYB(up(B.cdesc, desc.data(), desc.size() * sizeof(int4)));
    TRYB(up(B.cbase, base.data(), base.size() * sizeof(long long)));
    if (cudaMemcpyAsync(B.et, et, N * sizeof(double2), cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(B.etp, etp, N * sizeof(double2), cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(B.A, A, N * sizeof(double2), cudaMemcpyDefault, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("gnk_build_batch: geometry copy failed");
        return fail(GNK_ECUDA);
    }
    GNK_TRY_CUDA(cudaMemsetAsync(B.k.nonfinite, 0, sizeof(int), st));
    // per-domain node preparation (tiles never cross domains)
    int* flag = nullptr;
    TRYB(dalloc(&flag, 1));
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    for (int d = 0; d < ndom && rc == GNK_OK; ++d) {
        const BDom& D = B.hdom[d];
        Boundary v;
        v.N = D.N;
        v.n = D.n;
        v.m1 = D.m1;
        v.et = B.et + D.node_off;
        v.etp = B.etp + D.node_off;
        v.A = B.A + D.node_off;
        v.q = B.q + D.node_off;
        v.et32 = B.et32 + D.node_off;
        v.off32 = B.off32 + D.node_off;
        v.ref32 = B.ref32 + D.tile_off;
        v.q32 = B.q32 + D.node_off;
        v.A32 = B.A32 + D.node_off;
        v.ref64 = B.ref64 + D.tile_off;
        v.offdf = B.offdf + D.node_off;
        v.e = B.e + D.node_off;
        rc = run_prepare_nodes(v, nullptr, nullptr, flag, st);
    }
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    cudaFree(flag);
    if (rc != GNK_OK) return fail(rc);
    if (hflag & 3) {  // bit 4 (Im A != 0) is information, not an error
        set_error("gnk_build_batch: non-finite geometry or A = 0 at a node");
        return fail(hflag & 1 ? GNK_ENONFINITE : GNK_EINVAL);
    }
    // ones, Eone (double-float), diag(B1), diag(D1)
    {
        std::vector<double> one(N, 1.0);
        TRYB(up(B.ones, one.data(), N * sizeof(double)));
    }
    if (autotune_flag) {
        // the tuning runs use x = 1 on every system element
        std::vector<double> one(std::min<size_t>(Lz, (size_t)1 << 26), 1.0);
        for (size_t o = 0; o < Lz; o += one.size())
            TRYB(up(B.fc + o, one.data(), std::min(one.size(), Lz - o) * sizeof(double)));
        TRYB(autotune(B, st));
    }
    {
        // one right-hand side per domain: the (T = 1, RG = 1) variant
        std::vector<BItem> it1 = make_items(B.hdom1, 1, 1);
        TRYB(upload_items(it1, &B.itemsdf1, &B.nitemsdf1, st));
        BPairArgs a = base_args(B, B.dom1);
        a.x = B.ones;
        a.out = B.b1;
        a.out2 = B.d1;
        a.epi = BE_EONE;
        TRYB(launchdf(B, a, 1, 1, B.itemsdf1, B.nitemsdf1, st));
    }
    B.T32t = B.T32;
    B.RG32t = B.RG32;
    B.Tdft = B.Tdf;
    B.RGdft = B.RGdf;
    TRYB(upload_items(make_items(B.hdom, B.T32, B.RG32), &B.items32, &B.nitems32, st));
    TRYB(upload_items(make_items(B.hdom, B.Tdf, B.RGdf), &B.itemsdf, &B.nitemsdf, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("gnk_build_batch: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GNK_ECUDA);
    }
#undef TRYB
    *out = h;
    return GNK_OK;
}

int gnk_free_batch(gnk_batch* h) {
    if (!h) return GNK_OK;
    release_batch(h->b);
    delete h;
    return GNK_OK;
}

int gnk_batch_sizes(const gnk_batch* h, long long* vec_len, int* systems, int* hk_len) {
    if (!h) {
        set_error("NULL batch");
        return GNK_EINVAL;
    }
    if (vec_len) *vec_len = h->b.L;
    if (systems) *systems = h->b.nsys;
    if (hk_len) *hk_len = h->b.nhk;
    return GNK_OK;
}

int gnk_batch_tuning(const gnk_batch* h, int* fp32_targets, int* fp32_group, int* df_targets, int* df_group,
                     float* variant_ms) {
    if (!h) {
        set_error("NULL batch");
        return GNK_EINVAL;
    }
    const BatchImpl& B = h->b;
    if (fp32_targets) *fp32_targets = B.T32;
    if (fp32_group) *fp32_group = B.RG32;
    if (df_targets) *df_targets = B.Tdf;
    if (df_group) *df_group = B.RGdf;
    if (variant_ms)
        for (int i = 0; i < 7; ++i) variant_ms[i] = B.tune_ms[i];
    return GNK_OK;
}

int gnk_batch_apply_IminusN(const gnk_batch* hc, const double* x, double* y, int precision, void* stream) {
    if (!hc || !x || !y || (precision != GNK_PREC_FP32 && precision != GNK_PREC_DF32)) {
        set_error("gnk_batch_apply_IminusN: NULL argument or precision not FP32/DF32");
        return GNK_EINVAL;
    }
    BatchImpl& B = const_cast<gnk_batch*>(hc)->b;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const size_t Lb = (size_t)B.L * sizeof(double);
    GNK_TRY_CUDA(cudaMemcpyAsync(B.r, x, Lb, cudaMemcpyDefault, st));
    BPairArgs a = base_args(B, B.dom);
    a.x = B.r;
    a.out = B.dd;
    a.epi = BE_K;
    if (precision == GNK_PREC_FP32)
        GNK_TRY(launch32(B, a, B.T32, B.RG32, B.items32, B.nitems32, st));
    else
        GNK_TRY(launchdf(B, a, B.Tdf, B.RGdf, B.itemsdf, B.nitemsdf, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(y, B.dd, Lb, cudaMemcpyDefault, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    return GNK_OK;
}

int gnk_batch_fbie(const gnk_batch* hc, const double* gam, double* mu, double* hv, double* hk,
                   const gnk_options* opt, gnk_result* info, double* relres_per_system, void* stream) {
    if (!hc || !gam || !mu || !hv) {
        set_error("gnk_batch_fbie: NULL argument");
        return GNK_EINVAL;
    }
    BatchImpl& B = const_cast<gnk_batch*>(hc)->b;
    cudaGetLastError();
    gnk_options o;
    gnk_default_options(&o);
    o.precision = GNK_PREC_MIXED_DF;
    if (opt) o = *opt;
    if ((o.precision != GNK_PREC_MIXED_DF && o.precision != GNK_PREC_FMM) || o.restart < 1 || o.restart > 1000 ||
        o.maxit < 1 || !(o.tol > 0) || !(o.inner_tol > 0) || o.max_refine < 0 || o.tile_variant < 0 ||
        o.tile_variant > 7) {
        set_error("gnk_batch_fbie: options need precision GNK_PREC_MIXED_DF or GNK_PREC_FMM, restart 1..1000, "
                  "maxit >= 1, tol > 0, tile_variant 0..7");
        return GNK_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    GNK_TRY(apply_tiles(B, o.tile_variant, st));
    cudaEvent_t t_ev[2] = {nullptr, nullptr};
    if (o.timing) {
        for (auto& e : t_ev) GNK_TRY_CUDA(cudaEventCreate(&e));
        GNK_TRY_CUDA(cudaEventRecord(t_ev[0], st));
    }
    const size_t Lb = (size_t)B.L * sizeof(double);
    // gamma (host or device) is copied into the batch's own vector r
    double* g_dev = B.r;
    GNK_TRY_CUDA(cudaMemcpyAsync(g_dev, gam, Lb, cudaMemcpyDefault, st));
    gnk_result res;
    std::memset(&res, 0, sizeof(res));
    if (o.precision == GNK_PREC_FMM) {
        std::vector<double> rel(B.nsys, 0.0);
        const int s = run_batch_fmm(B, g_dev, B.x, B.dd, B.Lx, o, &res, &rel, st);
        if (s != GNK_OK && s != GNK_ENOTCONV && s != GNK_ENONFINITE) return s;
        GNK_TRY_CUDA(cudaMemcpyAsync(mu, B.x, Lb, cudaMemcpyDefault, st));
        GNK_TRY_CUDA(cudaMemcpyAsync(hv, B.dd, Lb, cudaMemcpyDefault, st));
        if (hk) GNK_TRY_CUDA(cudaMemcpyAsync(hk, B.Lx, (size_t)B.nhk * sizeof(double), cudaMemcpyDefault, st));
        if (o.timing) {
            float ms = 0.f;
            if (cudaEventRecord(t_ev[1], st) == cudaSuccess && cudaEventSynchronize(t_ev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&ms, t_ev[0], t_ev[1]) == cudaSuccess)
                res.solve_ms = ms;
            cudaGetLastError();
            for (auto& e : t_ev) cudaEventDestroy(e);
        }
        GNK_TRY_CUDA(cudaStreamSynchronize(st));
        double mx = 0.0;
        for (double v : rel) mx = std::max(mx, v);
        if (relres_per_system) std::memcpy(relres_per_system, rel.data(), rel.size() * sizeof(double));
        res.status = s;
        res.relres = mx;
        if (info) *info = res;
        if (s == GNK_ENOTCONV) set_error("batch: some systems did not reach tol");
        if (s == GNK_ENONFINITE) set_error("batch: non-finite value in some system");
        return s;
    }
    // right-hand side -y and f_B(gamma) from one double-float product
    GNK_TRY(run_batch_circulant(B.cdesc, B.cbase, B.ncirc, B.nmax, g_dev, B.Lx, B.twid, B.lcol, st));
    {
        BPairArgs a = base_args(B, B.dom);
        a.x = g_dev;
        a.Lx = B.Lx;
        a.out = B.rhs;
        a.out2 = B.fb;
        a.epi = BE_RHS_FB;
        GNK_TRY(launchdf(B, a, B.Tdf, B.RGdf, B.itemsdf, B.nitemsdf, st));
    }
    GNK_TRY_CUDA(cudaMemcpyAsync(B.rr, B.rhs, Lb, cudaMemcpyDeviceToDevice, st));
    const int ns = B.nsys;
    B.k.L = B.L;
    bk_norm<<<ns, KB, 0, st>>>(B.k, B.rhs, B.bnorm_out);
    count_launches(1);
    GNK_TRY_CUDA(cudaMemsetAsync(B.x, 0, Lb, st));
    GNK_TRY_CUDA(cudaMemsetAsync(B.fc, 0, Lb, st));  // f_C(0) = 0 for systems that never move
    bool fc_valid = false;
    int status = GNK_ENOTCONV;
    for (int it = 0;; ++it) {
        GNK_TRY_CUDA(cudaMemsetAsync(B.k.unconv, 0, sizeof(unsigned), st));
        bk_outer_check<<<ns, KB, 0, st>>>(B.k, B.rr, B.bnorm_out, B.relres, o.tol, B.k.unconv, B.oconv);
        count_launches(1);
        unsigned unconv = 0;
        int nonfin = 0;
        cudaMemcpyAsync(&unconv, B.k.unconv, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&nonfin, B.k.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st);
        GNK_TRY_CUDA(cudaStreamSynchronize(st));
        if (nonfin) {
            status = GNK_ENONFINITE;
            break;
        }
        if (unconv == 0) {
            status = GNK_OK;
            break;
        }
        if (it == o.max_refine) break;
        int steps = 0;
        GNK_TRY(gmres_batch(B, B.rr, B.dd, o.restart, o.maxit, o.inner_tol, &steps, &res.cycles, st));
        res.iterations += steps;
        res.matvecs_fp32 += steps;
        bk_axpy<<<(unsigned)((B.L + 255) / 256), 256, 0, st>>>(B.L, B.x, B.dd);
        count_launches(1);
        // outer residual and f_C(x) in double-float
        GNK_TRY(run_batch_circulant(B.cdesc, B.cbase, B.ncirc, B.nmax, B.x, B.Lx, B.twid, B.lcol, st));
        // groups whose systems had all converged are skipped: their x did not
        // move, their residual stays 0 and their f_C(x) stays valid
        BPairArgs a = base_args(B, B.dom);
        a.x = B.x;
        a.rhs = B.rhs;
        a.Lx = B.Lx;
        a.out = B.rr;
        a.out2 = B.fc;
        a.epi = BE_RESID_FC;
        a.sys_done = B.oconv;
        GNK_TRY(launchdf(B, a, B.Tdf, B.RGdf, B.itemsdf, B.nitemsdf, st));
        res.matvecs_fp64++;
        res.refinements++;
        fc_valid = true;
    }
    (void)fc_valid;
    // h = (f_C(mu) - f_B(gamma)) / 2, h_k per system
    bk_half_diff<<<(unsigned)((B.L + 255) / 256), 256, 0, st>>>(B.L, B.fc, B.fb, B.dd);
    count_launches(1);
    GNK_TRY_CUDA(cudaMemcpyAsync(mu, B.x, Lb, cudaMemcpyDefault, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(hv, B.dd, Lb, cudaMemcpyDefault, st));
    if (hk) {
        double* hkd = B.Lx;  // scratch (nhk <= L)
        bk_hk<<<ns, 64, 0, st>>>(B.sys, B.dom, B.hk_off, B.dd, hkd);
        count_launches(1);
        GNK_TRY_CUDA(cudaMemcpyAsync(hk, hkd, (size_t)B.nhk * sizeof(double), cudaMemcpyDefault, st));
    }
    std::vector<double> rel(ns);
    GNK_TRY_CUDA(cudaMemcpyAsync(rel.data(), B.relres, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (double v : rel) mx = std::max(mx, v);
    if (relres_per_system) std::memcpy(relres_per_system, rel.data(), ns * sizeof(double));
    res.status = status;
    res.relres = mx;
    if (o.timing) {
        float ms = 0.f;
        if (cudaEventRecord(t_ev[1], st) == cudaSuccess && cudaEventSynchronize(t_ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, t_ev[0], t_ev[1]) == cudaSuccess)
            res.solve_ms = ms;
        cudaGetLastError();
        for (auto& e : t_ev) cudaEventDestroy(e);
    }
    if (info) *info = res;
    if (status == GNK_ENOTCONV) set_error("batch: some systems did not reach tol");
    return status;
}

}  // extern "C"
