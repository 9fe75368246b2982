// Fast multipole evaluation of the Cauchy sum z_i = sum_{j != i} w_j / (eta_i - eta_j)
// (Sec. 2.5, Eqs. fmm-1, fmm-E: the paper forms E w with the FMM of zfmm2dpart,
// O((m+1)n) operations).  Uniform-depth quadtree over the bounding square of the
// nodes (levels 2..L, empty boxes pruned), expansions of order P scaled by the box
// width r (Greengard & Rokhlin's complex-analytic 2-D FMM):
//   multipole  phi(z) = sum_k a_k r^k / (z - c)^(k+1),  a_k = sum_j w_j ((s_j - c)/r)^k
//   local      phi(z) = sum_l b_l ((z - c)/r)^l
//   M2M  a0_m = sum_{k<=m} C(m,k) ((c1-c0)/r0)^(m-k) 2^-k a1_k
//   M2L  b_l  = (1/r) sum_k (-1)^(k+1) C(k+l,l) delta^-(k+l+1) a_k,  delta = (c1-c0)/r
//   L2L  b1_m = sum_{l>=m} C(l,m) ((c1-c0)/r0)^(l-m) 2^-m b0_l
// The near field (a leaf and its eight neighbours) is summed directly with the
// i = j term excluded.  The truncation error is below 0.43^P of
// sum_j |w_j / (eta_i - eta_j)| (about 2e-12 at P = 32 including round-off;
// checked against direct sums in the tests).
//
// One product is six or seven launches on two streams.  The weights are
// gathered into tree order; the far field runs on a high-priority stream: the
// upward pass (P2M, then the M2M chain carried by the block that completes
// each box's last child, no launch per level), M2L for every box, L2L per leaf
// down its ancestor path.  The near field runs beside it on the caller's
// stream (for the products z = E(q x) streamed from the near-field operator
// cache by bulk asynchronous copies, after x is gathered in the near lists'
// order); L2P adds the two after they join.  M2M and L2L are
// fixed real Pascal matrices between exact Gaussian-integer scalings, M2L a
// fixed real Pascal matrix between two complex scalings per offset: no P x P
// table per relative position.  The far field runs in complex double-float on the FP32
// pipe (GB300's FP64 pipe is 1/64 of it).
//
// The tree is built once per handle (the geometry is fixed for all products),
// on the device when its lookup grids fit (fmm_tree.cu), else on the host:
// Morton keys of 16-bit box coordinates, a sort of (key, node) pairs, leaf
// level L = the deepest level whose non-empty boxes hold at least kFmmLeaf
// nodes on average, interaction and neighbour lists.  Every sum on the device
// runs in a fixed order, so results are reproducible.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "fmm_internal.h"
#include "tma.cuh"
#include "epilogue.cuh"
#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {

namespace {

struct FmmArgs {
    int N, R, P;
    const int* perm;
    const double2* ps;
    const float4* p3;
    const float2* p3b;
    const int* leaf_start;
    const int* leaf_box;
    const double2* center;
    const double* width;
    const int* child_start;
    const int* child_count;
    const int* parent;
    const int* quad;
    const int* il_start;
    const int* il_src;
    const int* il_off;
    const int* nl_start;
    const int* nl_leaf;
    const float2* m2lH;   // C(k+l, l), [k][l] double-float
    const float4* m2lS;   // per offset code: (-1)^(k+1) delta^-(k+1), then delta^-l
    const float2* bUp;    // C(l, m) at [l][m] (0 for l < m): the L2L Pascal sums
    float4* mult;
    float4* loc;
    float4* ws;
    int nbox;
    // weights
    int mode;
    const double2* w0;
    const double2* w1;
    const double* x0;
    const double* x1;
    const double2* s;
    double2* out;  // [R][N] in node order
    const int* done;
    const int2* items;  // near-field work items: (leaf, first target of a chunk of 32)
    int nitems;
    double2* zn;        // [R][N] near-field sums in sorted order
    double2* zf;        // [R][N] near-field sums of w/d^2 in sorted order (EF products)
    double2* outF;      // [R][N] F sums in node order (EF products)
    const int* node_box;  // leaf box of each node in sorted order
    int* ucnt;            // per box: children counted in the upward pass
    float2* xs;           // [R][N] x in sorted order as double-float (cached near field), or null
    const float4* tp;     // [N][P] powers t^k of every node about its leaf centre, or null
    int* fault;           // set by a bounded wait that gave up
};

__global__ void fmm_gather_kernel(FmmArgs a) {
    if (a.done != nullptr && *a.done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int j = a.perm[i];
    for (int r = 0; r < a.R; ++r) {
        double2 w;
        if (a.mode == W_COMPLEX) {
            w = (r == 0) ? a.w0[j] : a.w1[j];
        } else {
            const double2 sc = a.s[j];
            const double x = (r == 0) ? a.x0[j] : a.x1[j];
            w = make_double2(sc.x * x, sc.y * x);
        }
        const df wx = df_split_fast(w.x), wy = df_split_fast(w.y);
        a.ws[(size_t)r * a.N + i] = make_float4(wx.h, wx.l, wy.h, wy.l);
        if (a.xs != nullptr) {  // x alone for the cached near field (W_SCALED)
            const df xv = df_split_fast((r == 0) ? a.x0[j] : a.x1[j]);
            a.xs[(size_t)r * a.N + i] = make_float2(xv.h, xv.l);
        }
    }
}

// ---- complex double-float arithmetic for the far field (FP32 pipe).  The
// expansions and the M2L scalings are stored as float4 (re.h, re.l, im.h,
// im.l); sums keep their rounding errors in the low words (about 2^-46 relative
// per operation), far below the truncation error of the order-32 expansions.
struct cdf {
    df re, im;
};

__device__ __forceinline__ cdf cdf_of(float4 v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ __forceinline__ float4 cdf_pack(cdf c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }
__device__ __forceinline__ cdf cdf_zero() { return cdf{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ cdf cdf_split(double2 v) { return cdf{df_split(v.x), df_split(v.y)}; }
__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

// a + b, renormalised
__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    df r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return cdf{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))),
               df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

// acc += a b
__device__ __forceinline__ void cdf_mac(cdf& acc, cdf a, cdf b) {
    df_acc(acc.re, df_mul(a.re, b.re));
    df_acc(acc.re, df_neg(df_mul(a.im, b.im)));
    df_acc(acc.im, df_mul(a.re, b.im));
    df_acc(acc.im, df_mul(a.im, b.re));
}

__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }

// Translation kernels use kFmmTW warps per target box.
constexpr int kFmmTW = 4;
constexpr int kFmmMaxDepth = 24;  // ancestors of a leaf, the leaf included

// ---- M2M and L2L between exact scalings.  With delta =
// (c1 - c0)/r0 = g/4 for a child in quadrant q, g = (2 qa - 1) + i (2 qb - 1):
//   M2M  a0_m = delta^m sum_{k<=m} C(m,k) [(2 delta)^-k a1_k]
//   L2L  b1_m = (2 delta)^-m sum_{l>=m} C(l,m) [delta^l b0_l]
// and (2 delta)^-1 = conj(g).  The scale factors g^e 4^-e and conj(g)^e are
// Gaussian integers times powers of two, so multiplying by them is exact up
// to one rounding in each part.  The L2L Pascal sum is a product with the
// fixed real triangular matrix C(l,m) (a double-float table of 8 KB that stays
// in L1; C(l,m) < 2^29, exact), lane m accumulating its 32 terms (zero beyond
// the triangle) in two independent compensated sums: one transform has the
// latency of a 32-term dot product instead of 31 dependent passes.  The M2M
// sum takes the passes (binom_lower).
constexpr int kFmmUT = 32 * kFmmTW;  // threads of the upward and downward kernels

// angle of g in units of pi/4 for the quadrant q = 2 qa + qb
__device__ __forceinline__ int gauss_angle(int q) { return (q == 3) ? 1 : (q == 1) ? 3 : (q == 0) ? 5 : 7; }

// x g^e 2^s for g = sqrt(2) e^{i pi ang / 4} (ang odd): g^e = 2^floor(e/2) (c + i d), c, d in {0, +-1}
__device__ __forceinline__ cdf cdf_mul_gpow(cdf x, int ang, int e, int s) {
    const int a8 = (ang * e) & 7;
    const float m = ldexpf(1.f, (e >> 1) + s);
    const float gr = (a8 == 0 || a8 == 1 || a8 == 7) ? m : ((a8 >= 3 && a8 <= 5) ? -m : 0.f);
    const float gi = (a8 >= 1 && a8 <= 3) ? m : ((a8 >= 5) ? -m : 0.f);
    const df p{__fmul_rn(x.re.h, gr), __fmul_rn(x.re.l, gr)}, q{__fmul_rn(-x.im.h, gi), __fmul_rn(-x.im.l, gi)};
    const df u{__fmul_rn(x.im.h, gr), __fmul_rn(x.im.l, gr)}, v{__fmul_rn(x.re.h, gi), __fmul_rn(x.re.l, gi)};
    return cdf{df_add(p, q), df_add(u, v)};
}

__device__ __forceinline__ cdf cdf_shfl_up1(cdf v) {
    return cdf{df{__shfl_up_sync(0xffffffffu, v.re.h, 1), __shfl_up_sync(0xffffffffu, v.re.l, 1)},
               df{__shfl_up_sync(0xffffffffu, v.im.h, 1), __shfl_up_sync(0xffffffffu, v.im.l, 1)}};
}

// lane m: sum_{k<=m} C(m,k) v_k by P - 1 passes (pass i adds the left
// neighbour's pre-pass value on lanes m >= i).  The upward pass keeps this
// form: there the Pascal-table sum below measured slower (more loads while
// the P2M of other leaves competes for the SM).
__device__ __forceinline__ cdf binom_lower(cdf v, int lane) {
#pragma unroll 1
    for (int i = 1; i < kFmmP; ++i) {
        const cdf u = cdf_shfl_up1(v);
        if (lane >= i) v = cdf_add(v, u);
    }
    return v;
}

// lane m: sum_k T[k][m] v_k for a real double-float table T (P x P, [k][m])
// and the complex vector v staged by the warp in sv[0 .. P)
__device__ __forceinline__ cdf pascal_sum(const float2* __restrict__ T, const float4* sv, int lane) {
    df yr{0.f, 0.f}, yi{0.f, 0.f}, zr{0.f, 0.f}, zi{0.f, 0.f};
#pragma unroll 4
    for (int k = 0; k < kFmmP; k += 2) {
        const float2 h0 = __ldg(T + k * kFmmP + lane), h1 = __ldg(T + (k + 1) * kFmmP + lane);
        const float4 x0 = sv[k], x1 = sv[k + 1];
        df_acc(yr, df_mul(df{h0.x, h0.y}, df{x0.x, x0.y}));
        df_acc(yi, df_mul(df{h0.x, h0.y}, df{x0.z, x0.w}));
        df_acc(zr, df_mul(df{h1.x, h1.y}, df{x1.x, x1.y}));
        df_acc(zi, df_mul(df{h1.x, h1.y}, df{x1.z, x1.w}));
    }
    return cdf{df_add(yr, zr), df_add(yi, zi)};
}

// one warp: lane m of a1 (the child's multipole) -> lane m of its contribution
// to the parent's multipole
__device__ __forceinline__ cdf m2m_binom(cdf a1, int q, int lane) {
    const int ang = gauss_angle(q);
    const cdf c = cdf_mul_gpow(a1, 8 - ang, lane, 0);  // (2 delta)^-k a1_k
    return cdf_mul_gpow(binom_lower(c, lane), ang, lane, -2 * lane);  // delta^m S_m
}

__device__ __forceinline__ cdf l2l_pascal(cdf b0, int q, int lane, const float2* bUp, float4* sv) {
    const int ang = gauss_angle(q);
    const cdf e = cdf_mul_gpow(b0, ang, lane, -2 * lane);  // delta^l b0_l
    __syncwarp();
    sv[lane] = cdf_pack(e);
    __syncwarp();
    return cdf_mul_gpow(pascal_sum(bUp, sv, lane), 8 - ang, lane, 0);  // (2 delta)^-m T_m
}

__device__ __forceinline__ cdf reduce_warps(cdf acc, float4 (*s)[32], int wid, int lane) {
    s[wid][lane] = cdf_pack(acc);
    __syncthreads();
    cdf t = cdf_of(s[0][lane]);
    if (wid == 0)
        for (int w = 1; w < kFmmTW; ++w) t = cdf_add(t, cdf_of(s[w][lane]));
    __syncthreads();
    return t;  // valid in warp 0
}

__device__ __forceinline__ cdf cdf_sq(cdf a) { return cdf_mul(a, a); }

// M2L into one box, as a fixed real matrix between two diagonal scalings:
// with x_k = (-1)^(k+1) delta^-(k+1) a_k (delta the source-to-target centre
// offset in box widths),
//   b_l = (1/r) delta^-l sum_k C(k+l, l) x_k.
// The Pascal matrix C(k+l, l) (double-float, 8 KB) is the same for every
// pair and stays in L1; the scalings are 2 x 32 double-float complex values
// per offset code.  The terms are those of the matrix form, so the rounding
// error is of the same size.  Warp w takes the interaction-list entries w,
// w + kFmmTW, ...; the warps' sums are added in warp order; the 1/r factor is
// applied once at the end.  loc then holds the M2L part of the box's local
// expansion.
template <int R>
__device__ __forceinline__ void m2l_box(const FmmArgs& a, int box, int wid, int lane, float4 (*s_acc)[32],
                                        float4 (*s_x)[32]) {
    const int e0 = a.il_start[box], e1 = a.il_start[box + 1];
    const df sc = df_split(1.0 / a.width[box]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cdf acc = cdf_zero();
        for (int e = e0 + wid; e < e1; e += kFmmTW) {
            const float4* S = a.m2lS + (size_t)a.il_off[e] * 2 * kFmmP;
            const cdf x = cdf_mul(cdf_of(__ldcg(a.mult + ((size_t)r * a.nbox + a.il_src[e]) * kFmmP + lane)),
                                  cdf_of(__ldg(S + lane)));
            const cdf post = cdf_of(__ldg(S + kFmmP + lane));
            __syncwarp();
            s_x[wid][lane] = cdf_pack(x);
            __syncwarp();
            df yr{0.f, 0.f}, yi{0.f, 0.f}, zr{0.f, 0.f}, zi{0.f, 0.f};
#pragma unroll 4
            for (int k = 0; k < kFmmP; k += 2) {
                const float2 h0 = __ldg(a.m2lH + k * kFmmP + lane), h1 = __ldg(a.m2lH + (k + 1) * kFmmP + lane);
                const float4 x0 = s_x[wid][k], x1 = s_x[wid][k + 1];
                df_acc(yr, df_mul(df{h0.x, h0.y}, df{x0.x, x0.y}));
                df_acc(yi, df_mul(df{h0.x, h0.y}, df{x0.z, x0.w}));
                df_acc(zr, df_mul(df{h1.x, h1.y}, df{x1.x, x1.y}));
                df_acc(zi, df_mul(df{h1.x, h1.y}, df{x1.z, x1.w}));
            }
            acc = cdf_add(acc, cdf_mul(cdf{df_add(yr, zr), df_add(yi, zi)}, post));
        }
        acc = reduce_warps(acc, s_acc, wid, lane);
        if (wid == 0) a.loc[((size_t)r * a.nbox + box) * kFmmP + lane] = cdf_pack(cdf{df_mul(acc.re, sc), df_mul(acc.im, sc)});
    }
}

// P2M of one leaf (block of kFmmTW warps): for each chunk of 32 nodes, warp
// w forms the powers t_j^k of orders 8w .. 8w + 7 (from t^8 by squaring) in
// shared memory, then sums w_j t_j^k over the chunk's nodes 8w .. 8w + 7 for
// every k (lane = k); the warps' sums are added in warp order.
template <int R>
__device__ __forceinline__ void p2m_leaf(const FmmArgs& a, int leaf, int box, int wid, int lane,
                                         float4 (*s_pow)[33], float4 (*s_w)[32], float4 (*s_acc)[32]) {
    const double2 c = a.center[box];
    const double ir = 1.0 / a.width[box];
    cdf acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = cdf_zero();
    const int j0 = a.leaf_start[leaf], j1 = a.leaf_start[leaf + 1];
    for (int base = j0; base < j1; base += 32) {
        const int j = base + lane;
        if (j < j1) {
            const double2 p = a.ps[j];
            const cdf t = cdf_split(make_double2((p.x - c.x) * ir, (p.y - c.y) * ir));
            const cdf t8 = cdf_sq(cdf_sq(cdf_sq(t)));
            cdf v = cdf{df{1.f, 0.f}, df{0.f, 0.f}};
            if (wid == 1) v = t8;
            if (wid >= 2) v = cdf_sq(t8);
            if (wid == 3) v = cdf_mul(v, t8);
            for (int k = 8 * wid; k < 8 * wid + 8; ++k) {
                s_pow[k][lane] = cdf_pack(v);
                v = cdf_mul(v, t);
            }
            if (wid < R) s_w[wid][lane] = a.ws[(size_t)wid * a.N + j];
        }
        __syncthreads();
        const int q1 = min(8 * wid + 8, j1 - base);
        for (int qn = 8 * wid; qn < q1; ++qn) {
            const cdf pw = cdf_of(s_pow[lane][qn]);
#pragma unroll
            for (int r = 0; r < R; ++r) cdf_mac(acc[r], cdf_of(s_w[r][qn]), pw);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const cdf sm = reduce_warps(acc[r], s_acc, wid, lane);
        if (wid == 0) a.mult[((size_t)r * a.nbox + box) * kFmmP + lane] = cdf_pack(sm);
    }
}

// P2M of one leaf from the cached powers t_j^k (a.tp, [node][k]): warp w
// sums w_j t_j^k over the leaf's nodes j = j0 + w, j0 + w + kFmmTW, ...
// (lane = k), with no block barrier until the warps' sums are added in warp
// order.  The powers (33.5 MB at 65,536 nodes) are read with the default L2
// policy: with the near-field stream marked evict-first they stay in L2
// between products.
template <int R>
__device__ __forceinline__ void p2m_leaf_cached(const FmmArgs& a, int leaf, int box, int wid, int lane,
                                                float4 (*s_acc)[32]) {
    cdf acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = cdf_zero();
    const int j0 = a.leaf_start[leaf], j1 = a.leaf_start[leaf + 1];
    constexpr int U = 8;  // rows loaded before they are used: 8 loads in flight per warp
    for (int j = j0 + wid; j < j1; j += kFmmTW * U) {
        float4 tv[U], wv[R][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int jj = j + u * kFmmTW;
            if (jj < j1) {
                tv[u] = __ldg(a.tp + (size_t)jj * kFmmP + lane);
#pragma unroll
                for (int r = 0; r < R; ++r) wv[r][u] = __ldcg(a.ws + (size_t)r * a.N + jj);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u * kFmmTW < j1) {
                const cdf pw = cdf_of(tv[u]);
#pragma unroll
                for (int r = 0; r < R; ++r) cdf_mac(acc[r], cdf_of(wv[r][u]), pw);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const cdf sm = reduce_warps(acc[r], s_acc, wid, lane);
        if (wid == 0) a.mult[((size_t)r * a.nbox + box) * kFmmP + lane] = cdf_pack(sm);
    }
}

// Upward pass, one block per leaf: P2M (from the cached powers when TP), then
// the multipoles move up the tree without a launch per level: the block that
// completes the last child of a box (an atomic count per box; nothing waits)
// forms that box's M2M from its children (warp w takes child w) and goes on
// to the parent.
template <int R, bool TP>
__global__ void __launch_bounds__(kFmmUT) fmm_up_kernel(FmmArgs a) {
    __shared__ float4 s_pow[TP ? 1 : kFmmP][33];
    __shared__ float4 s_w[R][32];
    __shared__ float4 s_acc[kFmmTW][32];
    __shared__ int s_last;
    if (a.done != nullptr && *a.done) return;
    const int leaf = blockIdx.x, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int box = a.leaf_box[leaf];
    if (TP)
        p2m_leaf_cached<R>(a, leaf, box, wid, lane, s_acc);
    else
        p2m_leaf<R>(a, leaf, box, wid, lane, s_pow, s_w, s_acc);
    for (;;) {
        if (wid == 0) __threadfence();  // the box's multipole (warp 0's stores) before the count
        __syncthreads();
        const int par = a.parent[box];
        if (par < 0) break;  // level 2
        if (threadIdx.x == 0) {
            const int last = atomicAdd(&a.ucnt[par], 1) == a.child_count[par] - 1;
            if (last) {
                a.ucnt[par] = 0;  // every child has counted: ready for the next product
                __threadfence();
            }
            s_last = last;
        }
        __syncthreads();
        if (!s_last) break;
        box = par;
        const int c0 = a.child_start[box], nc = a.child_count[box];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cdf acc = cdf_zero();
            if (wid < nc) {
                const int ch = c0 + wid;
                acc = m2m_binom(cdf_of(__ldcg(a.mult + ((size_t)r * a.nbox + ch) * kFmmP + lane)), a.quad[ch],
                                lane);
            }
            acc = reduce_warps(acc, s_acc, wid, lane);
            if (wid == 0) a.mult[((size_t)r * a.nbox + box) * kFmmP + lane] = cdf_pack(acc);
        }
    }
}

// M2L for every box of levels 2 .. L (block = box)
template <int R>
__global__ void __launch_bounds__(kFmmUT) fmm_m2l_kernel(FmmArgs a) {
    __shared__ float4 s_acc[kFmmTW][32];
    __shared__ float4 s_x[kFmmTW][32];
    if (a.done != nullptr && *a.done) return;
    m2l_box<R>(a, blockIdx.x, threadIdx.x >> 5, threadIdx.x & 31, s_acc, s_x);
}

// L2L, one warp per leaf: the leaf's local expansion is formed from the M2L
// parts of its ancestors, level 2 first, each shifted to the next level by
// the Pascal-matrix L2L (the same operations, in the same order, as a
// level-by-level downward pass; boxes above the leaf are shifted once per
// leaf below them, which costs no waiting), and stored over the leaf's M2L part.
template <int R>
__global__ void __launch_bounds__(32) fmm_l2l_kernel(FmmArgs a) {
    __shared__ int s_path[kFmmMaxDepth];
    __shared__ int s_depth;
    __shared__ float4 s_sv[32];
    if (a.done != nullptr && *a.done) return;
    const int leaf = blockIdx.x, lane = threadIdx.x;
    const int box = a.leaf_box[leaf];
    if (lane == 0) {
        int d = 0;
        for (int bx = box; bx >= 0 && d < kFmmMaxDepth; bx = a.parent[bx]) s_path[d++] = bx;
        s_depth = d;
    }
    __syncwarp();
    const int D = s_depth;  // s_path[D - 1] is on level 2, s_path[0] is the leaf
    if (D < 2) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cdf v = cdf_of(a.loc[((size_t)r * a.nbox + s_path[D - 1]) * kFmmP + lane]);
        for (int d = D - 2; d >= 0; --d) {
            const int bx = s_path[d];
            v = cdf_add(cdf_of(a.loc[((size_t)r * a.nbox + bx) * kFmmP + lane]),
                        l2l_pascal(v, a.quad[bx], lane, a.bUp, s_sv));
        }
        a.loc[((size_t)r * a.nbox + box) * kFmmP + lane] = cdf_pack(v);
    }
}

constexpr int kFmmWarps = kFmmNT / 32;
constexpr int kFmmMaxNbr = 9;  // a leaf and its eight neighbours

// Near field: one block per chunk of up to 32 targets of a leaf (lane = target).
// The sources of the (at most nine) neighbour leaves, taken as one list in
// neighbour order, are split into kFmmWarps equal ranges, one per warp, which
// the warp sums in tiles of 32; the warps' partial sums are added in warp
// order and stored in sorted node order (zn).  The near field runs in
// double-float on the FP32 pipe (GB300's FP64 pipe is 1/64 of it), two
// sources at a time in the two halves of packed float2 instructions (one
// issue for both): d from the exact three-float node coordinates, |d|^2 with
// Dekker products, one Newton step on the reciprocal, compensated
// accumulation into an even-source and an odd-source sum, added at the end.
// EF: also the sums of w_j / (eta_i - eta_j)^2 (to zf), for the gradient.

// d = p - q for two sources (one per half) from exact three-float splits: the
// TwoSums keep every rounding error, so close nodes get d to about 2^-47 |d|.
__device__ __forceinline__ df2 diff3_2(float2 p1, float2 p2, float2 p3, float2 q1, float2 q2, float2 q3) {
    float2 s1, e1, s2, e2, h, l;
    two_diff2(p1, q1, s1, e1);
    two_diff2(p2, q2, s2, e2);
    const float2 s3 = sub2(p3, q3);
    two_sum2(s1, s2, h, l);
    l = add2(l, add2(add2(e1, e2), s3));
    df2 r;
    r.h = add2(h, l);
    r.l = sub2(l, sub2(r.h, h));
    return r;
}

__device__ __forceinline__ df2 df2_neg(df2 a) { return df2{neg2(a.h), neg2(a.l)}; }

// a + b (renormalised), two lanes
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
    float2 s, e;
    two_sum2(a.h, b.h, s, e);
    e = add2(e, add2(a.l, b.l));
    df2 r;
    r.h = add2(s, e);
    r.l = sub2(e, sub2(r.h, s));
    return r;
}

template <int R, bool EF>
__global__ void __launch_bounds__(kFmmNT) fmm_near_kernel(FmmArgs a) {
    constexpr int RS = EF ? 2 * R : R;
    // one tile of 32 sources per warp, component by component, so that a
    // float2 read at pair p gives sources 2p and 2p + 1
    __shared__ float s_c[kFmmWarps][6][32];        // x1, x2, x3, y1, y2, y3
    __shared__ float s_w[kFmmWarps][R][4][32];     // wx.h, wx.l, wy.h, wy.l
    __shared__ int s_j[kFmmWarps][32];             // sorted index of each source (-1: padding)
    __shared__ double2 s_z[kFmmWarps][RS][32];
    __shared__ int s_cum[kFmmMaxNbr + 1];          // prefix sums of the neighbour leaves' sizes
    __shared__ int s_beg[kFmmMaxNbr];              // first source of each neighbour leaf
    if (a.done != nullptr && *a.done) return;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 it = a.items[blockIdx.x];  // (leaf, first target)
    const int leaf = it.x;
    const int t1 = a.leaf_start[leaf + 1];
    const int i = it.y + lane;
    const bool act = i < t1;
    const float4 pa = a.p3[act ? i : it.y];
    const float2 pb = a.p3b[act ? i : it.y];
    const float2 tx1 = f2(pa.x), tx2 = f2(pa.y), tx3 = f2(pa.z), ty1 = f2(pa.w), ty2 = f2(pb.x), ty3 = f2(pb.y);
    df2 are[RS], aim[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) are[r] = aim[r] = df2{f2(0.f), f2(0.f)};
    const int n0 = a.nl_start[leaf], nn = min(a.nl_start[leaf + 1] - n0, kFmmMaxNbr);
    if (threadIdx.x == 0) {
        int c = 0;
        for (int e = 0; e < nn; ++e) {
            const int nl = a.nl_leaf[n0 + e];
            s_beg[e] = a.leaf_start[nl];
            s_cum[e] = c;
            c += a.leaf_start[nl + 1] - a.leaf_start[nl];
        }
        s_cum[nn] = c;
    }
    __syncthreads();
    const int total = s_cum[nn];
    const int q0 = (int)((long long)total * wid / kFmmWarps), q1 = (int)((long long)total * (wid + 1) / kFmmWarps);
    for (int qs = q0; qs < q1; qs += 32) {
        __syncwarp();
        const int cnt = min(32, q1 - qs);
        {
            const int q = qs + min(lane, cnt - 1);  // lanes past the end copy the last source, weight 0
            int e = 0;
            while (e + 1 < nn && s_cum[e + 1] <= q) ++e;
            const int j = s_beg[e] + (q - s_cum[e]);
            const bool pad = lane >= cnt;
            const float4 c4 = a.p3[j];
            const float2 c2 = a.p3b[j];
            s_c[wid][0][lane] = c4.x;
            s_c[wid][1][lane] = c4.y;
            s_c[wid][2][lane] = c4.z;
            s_c[wid][3][lane] = c4.w;
            s_c[wid][4][lane] = c2.x;
            s_c[wid][5][lane] = c2.y;
            s_j[wid][lane] = pad ? -1 : j;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 w4 = pad ? make_float4(0.f, 0.f, 0.f, 0.f) : a.ws[(size_t)r * a.N + j];
                s_w[wid][r][0][lane] = w4.x;
                s_w[wid][r][1][lane] = w4.y;
                s_w[wid][r][2][lane] = w4.z;
                s_w[wid][r][3][lane] = w4.w;
            }
        }
        __syncwarp();
        const int npair = (cnt + 1) >> 1;
        for (int pp = 0; pp < npair; ++pp) {
            const float2 qx1 = reinterpret_cast<const float2*>(s_c[wid][0])[pp];
            const float2 qx2 = reinterpret_cast<const float2*>(s_c[wid][1])[pp];
            const float2 qx3 = reinterpret_cast<const float2*>(s_c[wid][2])[pp];
            const float2 qy1 = reinterpret_cast<const float2*>(s_c[wid][3])[pp];
            const float2 qy2 = reinterpret_cast<const float2*>(s_c[wid][4])[pp];
            const float2 qy3 = reinterpret_cast<const float2*>(s_c[wid][5])[pp];
            const int2 jj = reinterpret_cast<const int2*>(s_j[wid])[pp];
            const df2 dx = diff3_2(tx1, tx2, tx3, qx1, qx2, qx3);
            const df2 dy = diff3_2(ty1, ty2, ty3, qy1, qy2, qy3);
            const float2 px = mul2(dx.h, dx.h);
            float2 ex = fma2(dx.h, dx.h, neg2(px));
            ex = fma2(dx.h, add2(dx.l, dx.l), ex);
            const float2 py = mul2(dy.h, dy.h);
            float2 ey = fma2(dy.h, dy.h, neg2(py));
            ey = fma2(dy.h, add2(dy.l, dy.l), ey);
            float2 rh, re;
            two_sum2(px, py, rh, re);
            const float2 rl = add2(add2(ex, ey), re);
            float2 y = make_float2(recip_f32(rh.x), recip_f32(rh.y));
            // the i = j term is excluded (Eq. fmm-E); padding slots (j < 0) add nothing
            y.x = (jj.x == i || jj.x < 0) ? 0.f : y.x;
            y.y = (jj.y == i || jj.y < 0) ? 0.f : y.y;
            float2 ee = fma2(neg2(rh), y, f2(1.0f));
            ee = fma2(neg2(rl), y, ee);
            const df2 inv{y, mul2(y, ee)};
            const df2 ar = df2_mul(dx, inv), ai = df2_mul(dy, inv);  // 1/d = ar - i ai
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const df2 wx{reinterpret_cast<const float2*>(s_w[wid][r][0])[pp],
                             reinterpret_cast<const float2*>(s_w[wid][r][1])[pp]};
                const df2 wy{reinterpret_cast<const float2*>(s_w[wid][r][2])[pp],
                             reinterpret_cast<const float2*>(s_w[wid][r][3])[pp]};
                df2_acc(are[r], df2_mul(wx, ar));
                df2_acc(are[r], df2_mul(wy, ai));
                df2_acc(aim[r], df2_mul(wy, ar));
                df2_dec(aim[r], df2_mul(wx, ai));
            }
            if (EF) {  // 1/d^2 = (ar - i ai)^2 = gr - i gi
                const df2 a2 = df2_mul(ar, ar), b2 = df2_mul(ai, ai), ab = df2_mul(ar, ai);
                const df2 gr = df2_add(a2, df2_neg(b2));
                const df2 gi{add2(ab.h, ab.h), add2(ab.l, ab.l)};
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const df2 wx{reinterpret_cast<const float2*>(s_w[wid][r][0])[pp],
                                 reinterpret_cast<const float2*>(s_w[wid][r][1])[pp]};
                    const df2 wy{reinterpret_cast<const float2*>(s_w[wid][r][2])[pp],
                                 reinterpret_cast<const float2*>(s_w[wid][r][3])[pp]};
                    df2_acc(are[R + r], df2_mul(wx, gr));
                    df2_acc(are[R + r], df2_mul(wy, gi));
                    df2_acc(aim[R + r], df2_mul(wy, gr));
                    df2_dec(aim[R + r], df2_mul(wx, gi));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RS; ++r) {  // even + odd sums, then to FP64
        const df sr = df_add(df{are[r].h.x, are[r].l.x}, df{are[r].h.y, are[r].l.y});
        const df si = df_add(df{aim[r].h.x, aim[r].l.x}, df{aim[r].h.y, aim[r].l.y});
        s_z[wid][r][lane] = make_double2((double)sr.h + (double)sr.l, (double)si.h + (double)si.l);
    }
    __syncthreads();
    if (wid == 0 && act) {
#pragma unroll
        for (int r = 0; r < RS; ++r) {
            double2 v = s_z[0][r][lane];
            for (int w = 1; w < kFmmWarps; ++w) {
                v.x += s_z[w][r][lane].x;
                v.y += s_z[w][r][lane].y;
            }
            if (r < R)
                a.zn[(size_t)r * a.N + i] = v;
            else
                a.zf[(size_t)(r - R) * a.N + i] = v;
        }
    }
}

// The powers t^k, k < P, of every node about the centre of its leaf in units
// of the leaf width (t = (s - c)/r), double-float complex, [node][k] in sorted
// order: formed once per tree, read by every P2M.
__global__ void fmm_tp_build_kernel(FmmArgs a, float4* __restrict__ tp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int box = a.node_box[i];
    const double2 c = a.center[box];
    const double ir = 1.0 / a.width[box];
    const double2 p = a.ps[i];
    const cdf t = cdf_split(make_double2((p.x - c.x) * ir, (p.y - c.y) * ir));
    cdf v = cdf{df{1.f, 0.f}, df{0.f, 0.f}};
    float4* out = tp + (size_t)i * kFmmP;
    for (int k = 0; k < kFmmP; ++k) {
        out[k] = cdf_pack(v);
        v = cdf_mul(v, t);
    }
}

// ---- Near-field operator cache.  The geometry of a handle is fixed for all
// its products, so the near-field part of z = E(q x), the matrix
//   Q_ij = q_j / (eta_i - eta_j)   (i = j: 0)
// over each work item's targets i (a chunk of tn <= 32 nodes of a leaf) and
// sources j (the nodes of its neighbour leaves, in neighbour order), is
// formed once, in double-float from the exact three-float coordinates like
// the near-field kernel above, and each product then only reads it:
//   z_i = sum_j x_j Q_ij.
// Layout per item, for source pairs p = (2p, 2p + 1) and targets (lanes):
//   nq_re[off + p tn + lane] = (Re Q hi of 2p, of 2p+1, Re Q lo of 2p, of 2p+1)
// and nq_im likewise, so a float4 load gives the packed double-float operand
// of the two sources.  A product that needs only Im z (f_B with real A)
// reads nq_im alone: 8 bytes per pair.

// S (near sources) and tn (targets) of work item `it`; s_beg/s_cum (when
// given) receive the first source and the running count of each neighbour leaf.
__device__ __forceinline__ void nq_item_shape(const FmmArgs& a, int it, int* S, int* tn, int* s_beg, int* s_cum,
                                              int* nn_out) {
    const int2 item = a.items[it];
    const int leaf = item.x;
    *tn = min(32, a.leaf_start[leaf + 1] - item.y);
    const int n0 = a.nl_start[leaf], nn = min(a.nl_start[leaf + 1] - n0, kFmmMaxNbr);
    int c = 0;
    for (int e = 0; e < nn; ++e) {
        const int nl = a.nl_leaf[n0 + e];
        if (s_beg) {
            s_beg[e] = a.leaf_start[nl];
            s_cum[e] = c;
        }
        c += a.leaf_start[nl + 1] - a.leaf_start[nl];
    }
    if (s_cum) s_cum[nn] = c;
    *S = c;
    if (nn_out) *nn_out = nn;
}

__global__ void fmm_nq_count_kernel(FmmArgs a, long long* cnt, long long* scnt) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= a.nitems) return;
    int S, tn;
    nq_item_shape(a, it, &S, &tn, nullptr, nullptr, nullptr);
    cnt[it] = (long long)((S + 1) / 2) * tn;
    scnt[it] = S + (S & 1);  // lists padded to even length (16-byte aligned chunks of x)
}

// off[i] = cnt[0] + ... + cnt[i - 1] for i <= n (one block of 1024 threads,
// each a contiguous range, a block scan of the range sums in between).
__global__ void __launch_bounds__(1024) fmm_nq_scan_kernel(const long long* __restrict__ cnt, int n,
                                                            long long* __restrict__ off) {
    __shared__ long long s[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b0 = min(n, t * per), b1 = min(n, b0 + per);
    long long sum = 0;
    for (int i = b0; i < b1; ++i) sum += cnt[i];
    s[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = (t >= o) ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    long long run = (t == 0) ? 0 : s[t - 1];
    for (int i = b0; i < b1; ++i) {
        off[i] = run;
        run += cnt[i];
    }
    if (t == 1023) off[n] = s[1023];
}

// One block per work item, warp w taking its share of the source pairs.
__global__ void __launch_bounds__(kFmmNT) fmm_nq_build_kernel(FmmArgs a, const double2* __restrict__ q,
                                                              const long long* __restrict__ off,
                                                              const long long* __restrict__ soff,
                                                              float4* __restrict__ nq_re,
                                                              float4* __restrict__ nq_im,
                                                              int4* __restrict__ nq_item,
                                                              int* __restrict__ nq_src) {
    __shared__ float s_c[kFmmWarps][6][32];   // x1, x2, x3, y1, y2, y3 of the tile's sources
    __shared__ float s_q[kFmmWarps][4][32];   // q: re.h, re.l, im.h, im.l
    __shared__ int s_j[kFmmWarps][32];
    __shared__ int s_cum[kFmmMaxNbr + 1];
    __shared__ int s_beg[kFmmMaxNbr];
    __shared__ int s_S, s_tn, s_nn;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x;
    if (threadIdx.x == 0) {
        int S, tn, nn;
        nq_item_shape(a, it, &S, &tn, s_beg, s_cum, &nn);
        s_S = S;
        s_tn = tn;
        s_nn = nn;
    }
    __syncthreads();
    const int S = s_S, tn = s_tn, nn = s_nn;
    const int src0 = (int)soff[it];
    if (threadIdx.x == 0) nq_item[it] = make_int4(S, tn, src0, 0);
    for (int qq = threadIdx.x; qq < S; qq += blockDim.x) {  // the item's source list
        int e = 0;
        while (e + 1 < nn && s_cum[e + 1] <= qq) ++e;
        nq_src[src0 + qq] = s_beg[e] + (qq - s_cum[e]);
    }
    const int i = a.items[it].y + min(lane, tn - 1);
    const float4 pa = a.p3[i];
    const float2 pb = a.p3b[i];
    const float2 tx1 = f2(pa.x), tx2 = f2(pa.y), tx3 = f2(pa.z), ty1 = f2(pa.w), ty2 = f2(pb.x), ty3 = f2(pb.y);
    const int npair = (S + 1) >> 1;
    const int p0 = (int)((long long)npair * wid / kFmmWarps), p1 = (int)((long long)npair * (wid + 1) / kFmmWarps);
    const long long base = off[it];
    for (int ps = p0; ps < p1; ps += 16) {
        __syncwarp();
        const int np = min(16, p1 - ps);
        const int cnt = min(2 * np, S - 2 * ps);  // sources of this tile
        {
            const int qq = 2 * ps + min(lane, cnt - 1);
            int e = 0;
            while (e + 1 < nn && s_cum[e + 1] <= qq) ++e;
            const int j = s_beg[e] + (qq - s_cum[e]);
            const float4 c4 = a.p3[j];
            const float2 c2 = a.p3b[j];
            s_c[wid][0][lane] = c4.x;
            s_c[wid][1][lane] = c4.y;
            s_c[wid][2][lane] = c4.z;
            s_c[wid][3][lane] = c4.w;
            s_c[wid][4][lane] = c2.x;
            s_c[wid][5][lane] = c2.y;
            s_j[wid][lane] = (lane < cnt) ? j : -1;
            const double2 qj = q[a.perm[j]];
            const df qr = df_split(qj.x), qi = df_split(qj.y);
            s_q[wid][0][lane] = qr.h;
            s_q[wid][1][lane] = qr.l;
            s_q[wid][2][lane] = qi.h;
            s_q[wid][3][lane] = qi.l;
        }
        __syncwarp();
        for (int pp = 0; pp < np; ++pp) {
            const float2 qx1 = reinterpret_cast<const float2*>(s_c[wid][0])[pp];
            const float2 qx2 = reinterpret_cast<const float2*>(s_c[wid][1])[pp];
            const float2 qx3 = reinterpret_cast<const float2*>(s_c[wid][2])[pp];
            const float2 qy1 = reinterpret_cast<const float2*>(s_c[wid][3])[pp];
            const float2 qy2 = reinterpret_cast<const float2*>(s_c[wid][4])[pp];
            const float2 qy3 = reinterpret_cast<const float2*>(s_c[wid][5])[pp];
            const int2 jj = reinterpret_cast<const int2*>(s_j[wid])[pp];
            const df2 dx = diff3_2(tx1, tx2, tx3, qx1, qx2, qx3);
            const df2 dy = diff3_2(ty1, ty2, ty3, qy1, qy2, qy3);
            const float2 px = mul2(dx.h, dx.h);
            float2 ex = fma2(dx.h, dx.h, neg2(px));
            ex = fma2(dx.h, add2(dx.l, dx.l), ex);
            const float2 py = mul2(dy.h, dy.h);
            float2 ey = fma2(dy.h, dy.h, neg2(py));
            ey = fma2(dy.h, add2(dy.l, dy.l), ey);
            float2 rh, re;
            two_sum2(px, py, rh, re);
            const float2 rl = add2(add2(ex, ey), re);
            float2 y = make_float2(recip_f32(rh.x), recip_f32(rh.y));
            y.x = (jj.x == i || jj.x < 0) ? 0.f : y.x;  // i = j excluded (Eq. fmm-E); padding
            y.y = (jj.y == i || jj.y < 0) ? 0.f : y.y;
            float2 ee = fma2(neg2(rh), y, f2(1.0f));
            ee = fma2(neg2(rl), y, ee);
            const df2 inv{y, mul2(y, ee)};
            const df2 ar = df2_mul(dx, inv), ai = df2_mul(dy, inv);  // 1/d = ar - i ai
            const df2 qre{reinterpret_cast<const float2*>(s_q[wid][0])[pp], reinterpret_cast<const float2*>(s_q[wid][1])[pp]};
            const df2 qim{reinterpret_cast<const float2*>(s_q[wid][2])[pp], reinterpret_cast<const float2*>(s_q[wid][3])[pp]};
            // q (ar - i ai) = (qre ar + qim ai) + i (qim ar - qre ai)
            df2 Qr = df2_mul(qre, ar), Qi = df2_mul(qim, ar);
            df2_acc(Qr, df2_mul(qim, ai));
            df2_dec(Qi, df2_mul(qre, ai));
            if (lane < tn) {
                const size_t o = (size_t)(base + (long long)(ps + pp) * tn + lane);
                nq_re[o] = make_float4(Qr.h.x, Qr.h.y, Qr.l.x, Qr.l.y);
                nq_im[o] = make_float4(Qi.h.x, Qi.h.y, Qi.l.x, Qi.l.y);
            }
        }
    }
}

// x in the items' source-list order for the cached near field:
// xl[r][q] = xs[r][nq_src[q]] (0 at the lists' padding), so that each chunk of
// a work item's sources is one contiguous, 16-byte aligned run.
__global__ void fmm_nq_xlist_kernel(const int* __restrict__ src, long long qb, int R, int N,
                                    const float2* __restrict__ xs, float2* __restrict__ xl, const int* done) {
    if (done != nullptr && *done) return;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= qb) return;
    const int j = src[q];
    for (int r = 0; r < R; ++r) xl[(size_t)r * qb + q] = (j >= 0) ? xs[(size_t)r * N + j] : make_float2(0.f, 0.f);
}

// The near field of z = E(q x) from the cache, streamed into shared memory by
// the Tensor Memory Accelerator: one block per work item; a producer warp
// issues bulk copies of the item's cache entries (contiguous, pair-major,
// evict-first in L2: the cache is larger than L2 and read once per product) and
// of its sources' x (list order) in chunks of kNbPairs source pairs through a
// ring of kNbStages buffers (full/empty mbarriers); 8 consumer warps, lane =
// target, warp w taking pairs w, w + 8, ... of each chunk.  Even and odd
// sources go to the two halves of packed float2 sums, added at the end, then
// the warps' sums in warp order.  COMP = 1: Im z only (Re z written as 0).
// Every wait is bounded (kNbSpin polls); one that gives up sets a.fault, and
// the producer still waits (bounded) for its copies in flight before leaving.
constexpr int kNbPairs = 32;                 // source pairs per chunk
constexpr int kNbStages = 3;
constexpr int kNbThreads = kFmmNT + 32;      // 8 consumer warps and the producer warp
constexpr int kNbSpin = 1 << 22;

template <int R, int COMP>
struct NbLayout {
    static constexpr int kParts = COMP == 0 ? 2 : 1;
    static constexpr int kQ = kNbPairs * 32;                  // float4 entries of one part (tn <= 32)
    static constexpr int kX = kNbPairs;                       // float4 of x per right-hand side (a pair each)
    static constexpr int kStage = kParts * kQ + R * kX;       // float4 per stage
    static constexpr int kBytes = kNbStages * kStage * 16;    // dynamic shared memory
};

template <int R, int COMP>
__global__ void __launch_bounds__(kNbThreads) fmm_near_bulk_kernel(FmmArgs a, const long long* __restrict__ off,
                                                                   const int4* __restrict__ nq_item,
                                                                   const float4* __restrict__ nq_re,
                                                                   const float4* __restrict__ nq_im,
                                                                   const float2* __restrict__ xl, long long qb) {
    using L = NbLayout<R, COMP>;
    extern __shared__ __align__(16) float4 nb_buf[];
    __shared__ __align__(8) unsigned long long full[kNbStages], empty[kNbStages];
    __shared__ double2 s_z[kFmmWarps][R][32];
    if (a.done != nullptr && *a.done) return;  // set before this launch: the same in every thread
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x;
    const int4 d = __ldg(nq_item + it);  // (S, tn, first source)
    const long long o0 = __ldg(off + it);
    const int S = d.x, tn = d.y, src0 = d.z;
    const int npair = (S + 1) >> 1;
    const int nch = (npair + kNbPairs - 1) / kNbPairs;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kNbStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kFmmWarps);
        }
    }
    __syncthreads();
    if (wid == kFmmWarps) {  // the producer
        if (lane == 0) {
            int c = 0;
            for (; c < nch; ++c) {
                const int st = c % kNbStages;
                if (c >= kNbStages && !mbar_wait(&empty[st], (unsigned)((c / kNbStages - 1) & 1), kNbSpin)) {
                    atomicExch(a.fault, 1);
                    break;
                }
                const int p0 = c * kNbPairs, np = min(kNbPairs, npair - p0);
                const unsigned qbytes = (unsigned)(np * tn) * 16u, xbytes = (unsigned)np * 16u;
                float4* stage = nb_buf + (size_t)st * L::kStage;
                mbar_expect_tx(&full[st], L::kParts * qbytes + R * xbytes);
                bulk_load_stream(stage, nq_im + o0 + (long long)p0 * tn, qbytes, &full[st]);
                if (COMP == 0) bulk_load_stream(stage + L::kQ, nq_re + o0 + (long long)p0 * tn, qbytes, &full[st]);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    bulk_load(stage + L::kParts * L::kQ + r * L::kX, xl + (size_t)r * qb + src0 + 2 * p0, xbytes,
                              &full[st]);
            }
            // the copies still in flight land before the warp leaves
            for (int k = max(0, c - kNbStages); k < c; ++k)
                mbar_wait(&full[k % kNbStages], (unsigned)((k / kNbStages) & 1), kNbSpin);
        }
        return;
    }
    df2 are[R], aim[R];
#pragma unroll
    for (int r = 0; r < R; ++r) are[r] = aim[r] = df2{f2(0.f), f2(0.f)};
    for (int c = 0; c < nch; ++c) {
        const int st = c % kNbStages;
        if (!mbar_wait(&full[st], (unsigned)((c / kNbStages) & 1), kNbSpin)) {
            atomicExch(a.fault, 1);
            break;
        }
        const float4* qi = nb_buf + (size_t)st * L::kStage;
        const float4* qr = qi + L::kQ;
        const float4* xv4 = qi + L::kParts * L::kQ;
        const int np = min(kNbPairs, npair - c * kNbPairs);
        if (lane < tn) {
            for (int pp = wid; pp < np; pp += kFmmWarps) {
                const float4 wi = qi[pp * tn + lane];
                const df2 Qi{make_float2(wi.x, wi.y), make_float2(wi.z, wi.w)};
                df2 Qr{f2(0.f), f2(0.f)};
                if (COMP == 0) {
                    const float4 wr = qr[pp * tn + lane];
                    Qr = df2{make_float2(wr.x, wr.y), make_float2(wr.z, wr.w)};
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 v = xv4[r * L::kX + pp];  // (hi, lo) of sources 2pp and 2pp + 1
                    const df2 xv{make_float2(v.x, v.z), make_float2(v.y, v.w)};
                    if (COMP == 0) df2_acc(are[r], df2_mul(xv, Qr));
                    df2_acc(aim[r], df2_mul(xv, Qi));
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const df sr = df_add(df{are[r].h.x, are[r].l.x}, df{are[r].h.y, are[r].l.y});
        const df si = df_add(df{aim[r].h.x, aim[r].l.x}, df{aim[r].h.y, aim[r].l.y});
        s_z[wid][r][lane] = make_double2((double)sr.h + (double)sr.l, (double)si.h + (double)si.l);
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kFmmNT) : "memory");  // the consumer warps only
    if (wid == 0 && lane < tn) {
        const int i = a.items[it].y + lane;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double2 v = s_z[0][r][lane];
            for (int w = 1; w < kFmmWarps; ++w) {
                v.x += s_z[w][r][lane].x;
                v.y += s_z[w][r][lane].y;
            }
            a.zn[(size_t)r * a.N + i] = v;
        }
    }
}

// L2P by Horner's rule in double-float plus the near-field sum; one thread per
// node in sorted order (the nodes of a leaf are adjacent, so a warp reads the
// same coefficients).  Without the derivative the order-32 polynomial is four
// interleaved Horner chains of 8 coefficients joined by t^8 (a dependent chain
// of 13 steps instead of 31).  EPI: the operator epilogue of the product is applied at
// once (epilogue_apply: e.g. f_B(x) = 2x + diag(B1) x + (2/n) Im(A z)), so the
// sums z never go to memory; otherwise z is written in node order.
// EF: also F = -d/dz of the far field (Horner's rule carries the derivative)
// plus the near-field sums of w/d^2, written to outF.
template <int R, bool EF, bool EPI, int EK = EPI_Z>
__global__ void __launch_bounds__(256) fmm_l2p_kernel(FmmArgs a, ReduceArgs e) {
    if (a.done != nullptr && *a.done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int box = a.node_box[i];
    const double2 c = a.center[box];
    const double ir = recip_f64(a.width[box]);  // (GB300's FP64 division is a long dependent chain)
    const double2 p = a.ps[i];
    const cdf t = cdf{df_split_fast((p.x - c.x) * ir), df_split_fast((p.y - c.y) * ir)};
    const int node = a.perm[i];
    double zx[kMaxRHS] = {0.0, 0.0}, zy[kMaxRHS] = {0.0, 0.0};
    cdf t8{};
    if (!EF) t8 = cdf_sq(cdf_sq(cdf_sq(t)));
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4* b = a.loc + ((size_t)r * a.nbox + box) * kFmmP;
        cdf u, du = cdf_zero();
        if (EF) {  // Horner's rule, carrying the derivative
            u = cdf_of(b[kFmmP - 1]);
            for (int l = kFmmP - 2; l >= 0; --l) {
                du = cdf_add(cdf_mul(du, t), u);
                const cdf m = cdf_mul(u, t);
                const cdf bl = cdf_of(b[l]);
                u = cdf{df_add(m.re, bl.re), df_add(m.im, bl.im)};
            }
        } else {  // four interleaved Horner chains of 8 coefficients, joined by powers of t^8
            cdf h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = cdf_of(b[8 * q + 7]);
#pragma unroll
            for (int m = 6; m >= 0; --m)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const cdf mm = cdf_mul(h[q], t);
                    const cdf bl = cdf_of(b[8 * q + m]);
                    h[q] = cdf{df_add(mm.re, bl.re), df_add(mm.im, bl.im)};
                }
            u = h[3];
#pragma unroll
            for (int q = 2; q >= 0; --q) {
                const cdf mm = cdf_mul(u, t8);
                u = cdf{df_add(mm.re, h[q].re), df_add(mm.im, h[q].im)};
            }
        }
        const double2 zn = a.zn[(size_t)r * a.N + i];
        zx[r] = ((double)u.re.h + (double)u.re.l) + zn.x;
        zy[r] = ((double)u.im.h + (double)u.im.l) + zn.y;
        if (!EPI) a.out[(size_t)r * a.N + node] = make_double2(zx[r], zy[r]);
        if (EF) {
            const double2 zf = a.zf[(size_t)r * a.N + i];
            a.outF[(size_t)r * a.N + node] = make_double2(-ir * ((double)du.re.h + (double)du.re.l) + zf.x,
                                                          -ir * ((double)du.im.h + (double)du.im.l) + zf.y);
        }
    }
    if (EPI) epilogue_apply_as(e, EK, node, make_double2(zx[0], zy[0]), make_double2(zx[1], zy[1]));
}

// ---------------------------------------------------------------- host: tables
using cld = std::complex<long double>;

// a complex value as a double-float pair per part (hi = nearest float, lo = the rest)
float4 cdf_host(const cld& v) {
    const float rh = (float)v.real(), ih = (float)v.imag();
    return make_float4(rh, (float)(v.real() - (long double)rh), ih, (float)(v.imag() - (long double)ih));
}

// The M2L tables: the Pascal matrix C(k+l, l) as double-float pairs (P x P
// float2, in kFmmHSlots float4 slots), then per offset code (dx + 3) 7 + (dy + 3)
// the scalings (-1)^(k+1) delta^-(k+1) and delta^-l, delta = dx + i dy.
// Binomial coefficients by Pascal's triangle and powers by repeated products
// in long double: no library power functions, whose long double forms are
// slow where long double is emulated in software.
constexpr int kFmmHSlots = kFmmP * kFmmP / 2;
constexpr int kFmmSSlots = 49 * 2 * kFmmP;
// then the L2L Pascal table C(l,m) at [l][m] (double-float, zero outside the
// triangle), kFmmHSlots float4 slots

void translation_tables(std::vector<float4>* tab) {
    const int P = kFmmP, PP = 2 * kFmmP + 1;
    std::vector<long double> C((size_t)PP * PP, 0.0L);  // C[n][k], n < 2P + 1
    for (int n = 0; n < PP; ++n) {
        C[(size_t)n * PP] = 1.0L;
        for (int k = 1; k <= n; ++k) C[(size_t)n * PP + k] = C[(size_t)(n - 1) * PP + k - 1] + C[(size_t)(n - 1) * PP + k];
    }
    tab->assign(2 * kFmmHSlots + kFmmSSlots, make_float4(0.f, 0.f, 0.f, 0.f));
    float* BU = reinterpret_cast<float*>(tab->data() + kFmmHSlots + kFmmSSlots);  // [l][m] = C(l, m)
    for (int r = 0; r < P; ++r)
        for (int c = 0; c < P; ++c) {
            const long double up = (r >= c) ? C[(size_t)r * PP + c] : 0.0L;  // C(l = r, m = c)
            BU[2 * (r * P + c)] = (float)up;
            BU[2 * (r * P + c) + 1] = (float)(up - (long double)(float)up);
        }
    float* H = reinterpret_cast<float*>(tab->data());  // [k][l] (hi, lo)
    for (int k = 0; k < P; ++k)
        for (int l = 0; l < P; ++l) {
            const long double v = C[(size_t)(k + l) * PP + l];
            const float hi = (float)v;
            H[2 * (k * P + l)] = hi;
            H[2 * (k * P + l) + 1] = (float)(v - (long double)hi);
        }
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy) {
            if (std::max(std::abs(dx), std::abs(dy)) <= 1) continue;
            const int o = (dx + 3) * 7 + (dy + 3);
            const cld iz = 1.0L / cld((long double)dx, (long double)dy);
            float4* S = tab->data() + kFmmHSlots + (size_t)o * 2 * P;
            cld pw(1.0L, 0.0L);  // delta^-e
            for (int e = 0; e <= P; ++e) {
                if (e < P) S[P + e] = cdf_host(pw);                                       // delta^-l, l = e
                if (e >= 1) S[e - 1] = cdf_host((e % 2 == 1) ? -pw : pw);                // k = e - 1: (-1)^(k+1) = (-1)^e
                pw *= iz;
            }
        }
}

// Pinned host staging for the tree upload (grown on demand, kept for the process).
std::mutex g_stage_mutex;
void* g_stage = nullptr;
size_t g_stage_bytes = 0;

// The M2L tables depend only on P: formed once per process.
const std::vector<float4>& cached_tables() {
    static std::once_flag once;
    static std::vector<float4> tab;
    std::call_once(once, [] { translation_tables(&tab); });
    return tab;
}

// v = s[0] + s[1] + s[2] exactly (each float takes the next 24 bits of the
// double's 53; exact for |v| between 2^-80 and 2^120, which holds for
// boundary nodes in any sane unit)
void split3(double v, float* s) {
    s[0] = (float)v;
    const double r1 = v - (double)s[0];  // exact
    s[1] = (float)r1;
    s[2] = (float)(r1 - (double)s[1]);  // exact: at most 5 bits remain
}

uint32_t spread16(uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

}  // namespace

// The streams and events of FMM handles, kept per device for reuse (at most
// kPoolKeep of each kind), so that a caller that builds and frees a handle
// every step creates none after the first.  A stream returns to the pool only
// after it has been synchronised.
constexpr size_t kPoolKeep = 64;

struct StreamPool {
    std::mutex mu;
    std::vector<std::vector<cudaStream_t>> hi, lo;  // per device: high-priority and normal streams
    std::vector<std::vector<cudaEvent_t>> ev;
};

static StreamPool& stream_pool() {
    static StreamPool* p = new StreamPool();  // never destroyed: the streams outlive static teardown
    return *p;
}

static int fmm_high_priority();

static cudaError_t take_stream(bool high, cudaStream_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    StreamPool& P = stream_pool();
    {
        std::lock_guard<std::mutex> lock(P.mu);
        std::vector<std::vector<cudaStream_t>>& v = high ? P.hi : P.lo;
        if ((int)v.size() > dev && !v[dev].empty()) {
            *out = v[dev].back();
            v[dev].pop_back();
            return cudaSuccess;
        }
    }
    return high ? cudaStreamCreateWithPriority(out, cudaStreamNonBlocking, fmm_high_priority())
                : cudaStreamCreateWithFlags(out, cudaStreamNonBlocking);
}

static cudaError_t take_event(cudaEvent_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    StreamPool& P = stream_pool();
    {
        std::lock_guard<std::mutex> lock(P.mu);
        if ((int)P.ev.size() > dev && !P.ev[dev].empty()) {
            *out = P.ev[dev].back();
            P.ev[dev].pop_back();
            return cudaSuccess;
        }
    }
    return cudaEventCreateWithFlags(out, cudaEventDisableTiming);
}

static void give_stream(bool high, cudaStream_t s, int dev) {
    if (!s) return;
    cudaStreamSynchronize(s);
    StreamPool& P = stream_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    std::vector<std::vector<cudaStream_t>>& v = high ? P.hi : P.lo;
    if ((int)v.size() <= dev) v.resize(dev + 1);
    if (v[dev].size() < kPoolKeep)
        v[dev].push_back(s);
    else
        cudaStreamDestroy(s);
}

static void give_event(cudaEvent_t e, int dev) {
    if (!e) return;
    StreamPool& P = stream_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    if ((int)P.ev.size() <= dev) P.ev.resize(dev + 1);
    if (P.ev[dev].size() < kPoolKeep)
        P.ev[dev].push_back(e);
    else
        cudaEventDestroy(e);
}

void release_fmm(Boundary& b) {
    if (b.fmm) {
        give_stream(true, b.fmm->aux, b.device);
        give_event(b.fmm->ev_fork, b.device);
        give_event(b.fmm->ev_join, b.device);
        give_stream(false, b.fmm->bst, b.device);
        give_event(b.fmm->ev_nq, b.device);

        if (b.fmm->arena || b.fmm->sync || b.fmm->nq_re || b.fmm->tp || b.fmm->fault) {  // once no stream uses them
            cudaDeviceSynchronize();
            cudaGetLastError();
            pool_free(b.fmm->arena, 0);
            pool_free(b.fmm->sync, 0);
            pool_free(b.fmm->nq_cnt, 0);
            pool_free(b.fmm->nq_soff, 0);
            pool_free(b.fmm->nq_off, 0);
            pool_free(b.fmm->nq_item, 0);
            pool_free(b.fmm->nq_src, 0);
            pool_free(b.fmm->nq_re, 0);
            pool_free(b.fmm->nq_im, 0);
            pool_free(b.fmm->xs, 0);
            pool_free(b.fmm->xl, 0);
            pool_free(b.fmm->fault, 0);
            pool_free(b.fmm->tp, 0);
        }
        delete b.fmm;
        b.fmm = nullptr;
    }
}

// Builds the tree of the handle's nodes (once) with workspace for R right-hand sides.
// The host-side tree builder (used when the tree is too deep for the device
// builder's lookup grids): fills t and its device arena.
static int fmm_tree_host(const Boundary& b, FmmTree* t, cudaStream_t st) {
    const int N = b.N;
    std::vector<double2> et(N);
    GNK_TRY_CUDA(cudaMemcpyAsync(et.data(), b.et, (size_t)N * sizeof(double2), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    double xmin = et[0].x, xmax = et[0].x, ymin = et[0].y, ymax = et[0].y;
    for (const double2& p : et) {
        xmin = std::min(xmin, p.x);
        xmax = std::max(xmax, p.x);
        ymin = std::min(ymin, p.y);
        ymax = std::max(ymax, p.y);
    }
    const double W = std::max(std::max(xmax - xmin, ymax - ymin) * (1.0 + 1e-9), 1e-300);
    const double x0 = 0.5 * (xmin + xmax) - 0.5 * W, y0 = 0.5 * (ymin + ymax) - 0.5 * W;
    std::vector<uint32_t> key0(N), key1(N);
    std::vector<int> ord0(N), ord1(N);
    for (int i = 0; i < N; ++i) {
        const double fx = (et[i].x - x0) / W * 65536.0, fy = (et[i].y - y0) / W * 65536.0;
        const uint32_t ix = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(fx)));
        const uint32_t iy = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(fy)));
        key0[i] = (spread16(ix) << 1) | spread16(iy);
        ord0[i] = i;
    }
    // LSD radix sort, four stable passes of 8 bits: (key, node) in increasing order
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 8 * pass;
        int cnt[257] = {0};
        for (int i = 0; i < N; ++i) ++cnt[((key0[i] >> sh) & 0xffu) + 1];
        for (int d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
        for (int i = 0; i < N; ++i) {
            const int dst = cnt[(key0[i] >> sh) & 0xffu]++;
            key1[dst] = key0[i];
            ord1[dst] = ord0[i];
        }
        key0.swap(key1);
        ord0.swap(ord1);
    }
    auto key_at = [&](int i, int l) { return key0[i] >> (2 * (16 - l)); };
    // leaf level: deepest level whose non-empty boxes hold >= kFmmLeaf nodes on
    // average.  Neighbours in key order first differ at level 16 - msb(x)/2.
    std::vector<long long> first_diff(18, 0);
    for (int i = 1; i < N; ++i) {
        const uint32_t x = key0[i] ^ key0[i - 1];
        if (x == 0) continue;
        const int msb = 31 - __builtin_clz(x);
        ++first_diff[16 - msb / 2];  // distinct from this level down
    }
    int L = 2;
    long long distinct = 1;
    for (int l = 1; l <= 16; ++l) {
        distinct += first_diff[l];
        if (l < 3) continue;
        if ((double)N / (double)distinct < kFmmLeaf) break;
        L = l;
    }
    t->L = L;
    // boxes per level (level index l - 2), sorted by key
    const int nlev = L - 1;
    std::vector<std::vector<uint32_t>> keys(nlev);
    std::vector<int> leaf_start;
    for (int i = 0; i < N; ++i) {
        const uint32_t k = key_at(i, L);
        if (i == 0 || k != keys[L - 2].back()) {
            keys[L - 2].push_back(k);
            leaf_start.push_back(i);
        }
    }
    leaf_start.push_back(N);
    for (int l = L - 1; l >= 2; --l)
        for (uint32_t k : keys[l - 1]) {  // children of level l + 1 are keys[l - 1]
            const uint32_t pk = k >> 2;
            if (keys[l - 2].empty() || keys[l - 2].back() != pk) keys[l - 2].push_back(pk);
        }
    t->lvl_off.resize(nlev);
    t->lvl_cnt.resize(nlev);
    int nbox = 0;
    for (int l = 2; l <= L; ++l) {
        t->lvl_off[l - 2] = nbox;
        t->lvl_cnt[l - 2] = (int)keys[l - 2].size();
        nbox += (int)keys[l - 2].size();
    }
    t->nbox = nbox;
    t->nleaf = (int)keys[L - 2].size();
    auto compact = [](uint32_t v) {  // inverse of spread16
        v &= 0x55555555u;
        v = (v | (v >> 1)) & 0x33333333u;
        v = (v | (v >> 2)) & 0x0f0f0f0fu;
        v = (v | (v >> 4)) & 0x00ff00ffu;
        v = (v | (v >> 8)) & 0x0000ffffu;
        return v;
    };
    auto decode = [&](uint32_t key, int* ix, int* iy) {
        *ix = (int)compact(key >> 1);
        *iy = (int)compact(key);
    };
    // box geometry, parents and children: children of a box are contiguous in
    // key order, so one pass over each level links it to the level above
    std::vector<int> bix(nbox), biy(nbox);
    for (int l = 2; l <= L; ++l)
        for (int q = 0; q < t->lvl_cnt[l - 2]; ++q) decode(keys[l - 2][q], &bix[t->lvl_off[l - 2] + q],
                                                           &biy[t->lvl_off[l - 2] + q]);
    std::vector<double2> center(nbox);
    std::vector<double> width(nbox);
    std::vector<int> child_start(nbox, -1), child_count(nbox, 0), parent(nbox, -1), quad(nbox, 0);
    for (int l = 2; l <= L; ++l) {
        const double r = W / (double)(1 << l);
        for (int q = 0; q < t->lvl_cnt[l - 2]; ++q) {
            const int g = t->lvl_off[l - 2] + q;
            center[g] = make_double2(x0 + (bix[g] + 0.5) * r, y0 + (biy[g] + 0.5) * r);
            width[g] = r;
            quad[g] = ((bix[g] & 1) << 1) | (biy[g] & 1);
        }
        if (l == 2) continue;
        int pq = -1;
        uint32_t last = 0;
        for (int q = 0; q < t->lvl_cnt[l - 2]; ++q) {
            const uint32_t pk = keys[l - 2][q] >> 2;
            if (pq < 0 || pk != last) {
                ++pq;
                last = pk;
            }
            const int g = t->lvl_off[l - 2] + q, pg = t->lvl_off[l - 3] + pq;
            parent[g] = pg;
            if (child_start[pg] < 0) child_start[pg] = g;
            ++child_count[pg];
        }
    }
    // neighbour lists (adjacent boxes of the same level, the box itself included)
    // and interaction lists, level by level from the children of the parent's
    // neighbours; level 2 compares all pairs
    std::vector<int> nb_start(nbox + 1, 0), nb;
    std::vector<int> il_start(nbox + 1, 0), il_src, il_off;
    nb.reserve((size_t)nbox * 6);
    il_src.reserve((size_t)nbox * 16);
    il_off.reserve((size_t)nbox * 16);
    auto visit = [&](int g, int c) {
        const int dx = bix[c] - bix[g], dy = biy[c] - biy[g];
        if (std::abs(dx) <= 1 && std::abs(dy) <= 1) {
            nb.push_back(c);
        } else {
            il_src.push_back(c);
            il_off.push_back((dx + 3) * 7 + (dy + 3));
        }
    };
    for (int l = 2; l <= L; ++l)
        for (int q = 0; q < t->lvl_cnt[l - 2]; ++q) {
            const int g = t->lvl_off[l - 2] + q;
            if (l == 2) {
                for (int c = t->lvl_off[0]; c < t->lvl_off[0] + t->lvl_cnt[0]; ++c) visit(g, c);
            } else {
                const int pg = parent[g];
                for (int e = nb_start[pg]; e < nb_start[pg + 1]; ++e) {
                    const int qn = nb[e];
                    for (int c = child_start[qn]; c < child_start[qn] + child_count[qn]; ++c) visit(g, c);
                }
            }
            nb_start[g + 1] = (int)nb.size();
            il_start[g + 1] = (int)il_src.size();
        }
    // neighbour leaves of each leaf (the leaf itself included)
    std::vector<int> nl_start(t->nleaf + 1, 0), nl_leaf, leaf_box(t->nleaf);
    long long near_pairs = 0;
    const int loff = t->lvl_off[L - 2];
    for (int q = 0; q < t->nleaf; ++q) {
        leaf_box[q] = loff + q;
        const long long cnt_t = leaf_start[q + 1] - leaf_start[q];
        for (int e = nb_start[loff + q]; e < nb_start[loff + q + 1]; ++e) {
            const int lq = nb[e] - loff;
            nl_leaf.push_back(lq);
            near_pairs += cnt_t * (leaf_start[lq + 1] - leaf_start[lq]);
        }
        nl_start[q + 1] = (int)nl_leaf.size();
    }
    t->near_pairs = near_pairs;
    // near-field work items: chunks of 32 targets of a leaf, largest leaves first
    std::vector<int2> items;
    for (int q = 0; q < t->nleaf; ++q)
        for (int i = leaf_start[q]; i < leaf_start[q + 1]; i += 32) items.push_back(make_int2(q, i));
    std::stable_sort(items.begin(), items.end(), [&](const int2& u, const int2& v) {
        return (nl_start[u.x + 1] - nl_start[u.x]) > (nl_start[v.x + 1] - nl_start[v.x]);
    });
    t->nitems = (int)items.size();
    t->m2l_pairs = (long long)il_src.size();
    long long m2m_pairs = 0;
    for (int g = 0; g < nbox; ++g) m2m_pairs += child_count[g];
    t->m2m_pairs = m2m_pairs;
    const std::vector<int>& perm = ord0;
    std::vector<double2> ps(N);
    for (int i = 0; i < N; ++i) ps[i] = et[perm[i]];

    // one device allocation for the tree and the expansions
    const size_t P = kFmmP;
    struct Part {
        void** p;
        size_t bytes;
    };
    const size_t nil = std::max<size_t>(il_src.size(), 1), nnl = std::max<size_t>(nl_leaf.size(), 1);
    Part parts[] = {
        {(void**)&t->perm, N * sizeof(int)},
        {(void**)&t->ps, N * sizeof(double2)},
        {(void**)&t->p3, N * sizeof(float4)},
        {(void**)&t->p3b, N * sizeof(float2)},
        {(void**)&t->leaf_start, (t->nleaf + 1) * sizeof(int)},
        {(void**)&t->leaf_box, t->nleaf * sizeof(int)},
        {(void**)&t->center, nbox * sizeof(double2)},
        {(void**)&t->width, nbox * sizeof(double)},
        {(void**)&t->child_start, nbox * sizeof(int)},
        {(void**)&t->child_count, nbox * sizeof(int)},
        {(void**)&t->parent, nbox * sizeof(int)},
        {(void**)&t->quad, nbox * sizeof(int)},
        {(void**)&t->il_start, (nbox + 1) * sizeof(int)},
        {(void**)&t->il_src, nil * sizeof(int)},
        {(void**)&t->il_off, nil * sizeof(int)},
        {(void**)&t->nl_start, (t->nleaf + 1) * sizeof(int)},
        {(void**)&t->nl_leaf, nnl * sizeof(int)},
        {(void**)&t->items, std::max<size_t>(items.size(), 1) * sizeof(int2)},
        {(void**)&t->node_box, N * sizeof(int)},
        {(void**)&t->mult, (size_t)t->R * nbox * P * sizeof(float4)},
        {(void**)&t->loc, (size_t)t->R * nbox * P * sizeof(float4)},
        {(void**)&t->ws, (size_t)t->R * N * sizeof(float4)},
        {(void**)&t->zn, (size_t)t->R * N * sizeof(double2)},
        {(void**)&t->zf, (size_t)t->R * N * sizeof(double2)},
    };
    size_t total = 0;
    for (const Part& p : parts) total += (p.bytes + 255) / 256 * 256;
    if (pool_alloc(&t->arena, total, st) != cudaSuccess) {
        cudaGetLastError();
        t->arena = nullptr;
        set_error("FMM tree: device allocation of %zu bytes failed", total);
        return GNK_ENOMEM;
    }
    char* cur = static_cast<char*>(t->arena);
    for (const Part& p : parts) {
        *p.p = cur;
        cur += (p.bytes + 255) / 256 * 256;
    }
    // everything but the expansions goes up in one copy, staged in a pinned
    // host buffer laid out like the device arena
    const size_t upload = (size_t)((char*)t->mult - (char*)t->arena);
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    if (g_stage_bytes < upload) {
        if (g_stage) cudaFreeHost(g_stage);
        g_stage = nullptr;
        g_stage_bytes = 0;
        if (cudaHostAlloc(&g_stage, upload, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            g_stage = nullptr;
            set_error("FMM tree: pinned staging allocation of %zu bytes failed", upload);
            return GNK_ENOMEM;
        }
        g_stage_bytes = upload;
    }
    char* hb = static_cast<char*>(g_stage);
    auto put = [&](const void* dst, const void* src, size_t bytes) {
        if (bytes) std::memcpy(hb + ((const char*)dst - (const char*)t->arena), src, bytes);
    };
    put(t->perm, perm.data(), N * sizeof(int));
    put(t->ps, ps.data(), N * sizeof(double2));
    float4* p3 = reinterpret_cast<float4*>(hb + ((char*)t->p3 - (char*)t->arena));
    float2* p3b = reinterpret_cast<float2*>(hb + ((char*)t->p3b - (char*)t->arena));
    for (int i = 0; i < N; ++i) {
        float sx[3], sy[3];
        split3(ps[i].x, sx);
        split3(ps[i].y, sy);
        p3[i] = make_float4(sx[0], sx[1], sx[2], sy[0]);
        p3b[i] = make_float2(sy[1], sy[2]);
    }
    put(t->leaf_start, leaf_start.data(), leaf_start.size() * sizeof(int));
    put(t->leaf_box, leaf_box.data(), leaf_box.size() * sizeof(int));
    put(t->center, center.data(), nbox * sizeof(double2));
    put(t->width, width.data(), nbox * sizeof(double));
    put(t->child_start, child_start.data(), nbox * sizeof(int));
    put(t->child_count, child_count.data(), nbox * sizeof(int));
    put(t->parent, parent.data(), nbox * sizeof(int));
    put(t->quad, quad.data(), nbox * sizeof(int));
    put(t->il_start, il_start.data(), il_start.size() * sizeof(int));
    put(t->il_src, il_src.data(), il_src.size() * sizeof(int));
    put(t->il_off, il_off.data(), il_off.size() * sizeof(int));
    put(t->nl_start, nl_start.data(), nl_start.size() * sizeof(int));
    put(t->nl_leaf, nl_leaf.data(), nl_leaf.size() * sizeof(int));
    put(t->items, items.data(), items.size() * sizeof(int2));
    int* nbx = reinterpret_cast<int*>(hb + ((char*)t->node_box - (char*)t->arena));
    for (int q = 0; q < t->nleaf; ++q)
        for (int i = leaf_start[q]; i < leaf_start[q + 1]; ++i) nbx[i] = leaf_box[q];
    // the staging buffer is reused by the next build: finish the copy first
    cudaError_t e = cudaMemcpyAsync(t->arena, hb, upload, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM tree upload failed: %s", cudaGetErrorString(e));
        return GNK_ECUDA;
    }
    return GNK_OK;
}

int fmm_device_tables(const float2** m2lH, const float4** m2lS, const float2** bUp, cudaStream_t st) {
    static std::mutex mu;
    static std::vector<float4*> per_device;  // indexed by device, never freed
    int dev = 0;
    GNK_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_device.size() <= dev) per_device.resize(dev + 1, nullptr);
    if (!per_device[dev]) {
        const std::vector<float4>& c = cached_tables();
        float4* d = nullptr;
        if (cudaMalloc(&d, c.size() * sizeof(float4)) != cudaSuccess) {
            cudaGetLastError();
            set_error("FMM: device allocation of the M2L tables failed");
            return GNK_ENOMEM;
        }
        cudaError_t e = cudaMemcpyAsync(d, c.data(), c.size() * sizeof(float4), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            set_error("FMM: upload of the M2L tables failed");
            return GNK_ECUDA;
        }
        per_device[dev] = d;
    }
    *m2lH = reinterpret_cast<const float2*>(per_device[dev]);
    *m2lS = per_device[dev] + kFmmHSlots;
    *bUp = reinterpret_cast<const float2*>(per_device[dev] + kFmmHSlots + kFmmSSlots);
    return GNK_OK;
}

// The highest stream priority of the device (the far-field chain's stream).
static int fmm_high_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

static void fmm_args(const Boundary& b, FmmArgs& a);

constexpr double kTpMaxBytes = 4.0 * (1 << 30);

// Builds the tree of the handle's nodes (once) with workspace for kMaxRHS
// right-hand sides: on the device when the lookup grids fit, else on the host.
int ensure_fmm(const Boundary& bc, int R, cudaStream_t st) {
    Boundary& b = const_cast<Boundary&>(bc);
    (void)R;
    if (b.fmm) return GNK_OK;
    FmmTree* t = new (std::nothrow) FmmTree();
    if (!t) {
        set_error("host allocation failed");
        return GNK_ENOMEM;
    }
    t->R = kMaxRHS;
    int rc = fmm_tree_device(b, t, st);
    if (rc == kFmmUseHost) rc = fmm_tree_host(b, t, st);
    if (rc == GNK_OK) rc = fmm_device_tables(&t->m2lH, &t->m2lS, &t->bUp, st);
    if (rc == GNK_OK) {  // the upward pass's child counts, all zero
        const size_t nsync = (size_t)t->nbox;
        if (pool_alloc(reinterpret_cast<void**>(&t->sync), nsync * sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(t->sync, 0, nsync * sizeof(int), st) != cudaSuccess ||
            pool_alloc(reinterpret_cast<void**>(&t->fault), sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(t->fault, 0, sizeof(int), st) != cudaSuccess) {
            cudaGetLastError();
            set_error("FMM: allocation of the pass counters failed");
            rc = GNK_ENOMEM;
        }
    }
    // the powers of the P2M: 512 bytes per node, below kTpMaxBytes (else P2M
    // forms them itself)
    if (rc == GNK_OK && (double)b.N * kFmmP * sizeof(float4) <= kTpMaxBytes &&
        pool_alloc(reinterpret_cast<void**>(&t->tp), (size_t)b.N * kFmmP * sizeof(float4), st) == cudaSuccess) {
        FmmArgs a;
        b.fmm = t;
        fmm_args(b, a);
        fmm_tp_build_kernel<<<(b.N + 255) / 256, 256, 0, st>>>(a, t->tp);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("FMM: launch of the power table failed");
            rc = GNK_ECUDA;
        }
    }
    cudaGetLastError();
    if (rc == GNK_OK &&
        (take_stream(true, &t->aux) != cudaSuccess || take_event(&t->ev_fork) != cudaSuccess ||
         take_event(&t->ev_join) != cudaSuccess)) {
        cudaGetLastError();
        set_error("FMM: stream or event creation failed");
        rc = GNK_ECUDA;
    }
    b.fmm = t;  // owned by the handle from here on (freed by release_fmm)
    if (rc != GNK_OK) release_fmm(b);
    return rc;
}

// FP32-pipe instructions of one FMM product, for the roofline.  M2L, per pair
// and lane: 32 (2 Dekker products and 2 compensated sums, 24) for the real
// Pascal matrix, the two complex scalings (38 each) and the sum (22); 840 per
// lane for an L2L transform (32 terms of the Pascal sum at 24 each, two exact
// scalings at 30 and two double-float additions), 742 for an M2M (31 passes
// of a double-float complex addition, 22 each, and the two scalings); P2M: 36 per
// complex double-float power (47 per node: 32 orders, the squarings to t^8 in
// each warp, t^16 and t^24) and 48 R per node and order for the sums; L2P:
// 58 R per node and order (a complex product and sum), twice that with the
// derivative.
// which = 0: M2L; 1: the upward pass (P2M and the M2M climb); 2: L2L; 3: L2P;
// 4: L2P with the derivative.  (The near field: fmm_near_instr.)
double fmm_instr(const Boundary& b, int R, int which) {
    const FmmTree* t = b.fmm;
    if (!t) return 0.0;
    const double P = kFmmP, m2m = 742.0 * P, l2l = 840.0 * P, m2l = (24.0 * P + 98.0) * P;
    switch (which) {
        case 0: return R * m2l * (double)t->m2l_pairs;
        case 1: return R * m2m * (double)t->m2m_pairs + (double)b.N * (t->tp ? 48.0 * R * P : 36.0 * 47.0 + 48.0 * R * P);
        case 2: return R * l2l * (double)t->nleaf * (t->L - 2);
        default: return R * (double)b.N * P * 58.0 * (which == 4 ? 2.0 : 1.0);
    }
}

double fmm_near_instr(const Boundary& b, int R) {
    return b.fmm ? (49.0 + 48.0 * R) * (double)b.fmm->near_pairs : 0.0;
}

// The cached near field per pair and right-hand side: a double-float product
// (4) and a compensated accumulation (8) per part of z; bytes: the cached
// entries read (8 per part and pair).
double fmm_near_cached_instr(const Boundary& b, int R, int comp) {
    return b.fmm ? 12.0 * R * (comp == 1 ? 1.0 : 2.0) * (double)b.fmm->near_pairs : 0.0;
}

double fmm_near_cached_bytes(const Boundary& b, int R, int comp) {
    // 8 bytes per near pair and part of z read from the cache, x in list order
    // (8 bytes per list entry, counted at the lists' bound) and z out (16 bytes
    // per node) per right-hand side
    return b.fmm ? 8.0 * (double)b.fmm->near_pairs * (comp == 1 ? 1.0 : 2.0) +
                       8.0 * R * (double)b.fmm->nq_qb + 16.0 * R * b.N
                 : 0.0;
}

const int* fmm_fault_word(const Boundary& b) {
    return b.fmm ? b.fmm->fault : nullptr;
}

// Forms the near-field operator cache of the products z = E(q x) once per
// handle (count, scan, allocate, build); state -1 when it would exceed
// kNqMaxBytes or when its allocation fails (the products then compute the
// near field directly).
constexpr double kNqMaxBytes = 16.0 * (1 << 30);

static int ensure_near_cache(const Boundary& b, cudaStream_t st) {
    FmmTree* t = b.fmm;
    if (t->nq_state != 0) return GNK_OK;
    t->nq_state = -1;
    if (t->nitems <= 0) return GNK_OK;
    // sizes from bounds the tree already gives, so that nothing waits for the
    // device: sum_items ceil(S/2) tn <= (near pairs + N)/2 entries, and
    // sum_items S <= near pairs sources (each source meets at least one target)
    const size_t ni = (size_t)t->nitems;
    // sum_items S = sum_leaves ceil(n_leaf / 32) S_leaf <= near pairs / 32 + sum_leaves S_leaf, and
    // a leaf is a neighbour of at most kFmmMaxNbr leaves, so sum_leaves S_leaf <= kFmmMaxNbr N;
    // plus one padding entry per item, rounded up to even
    const long long slots = (t->near_pairs + b.N) / 2 + 1;
    long long nsrc = t->near_pairs / 32 + (long long)kFmmMaxNbr * b.N + (long long)ni + 2;
    nsrc += nsrc & 1;
    const size_t bytes = (size_t)slots * sizeof(float4);
    if (nsrc > INT32_MAX || 2.0 * (double)bytes > kNqMaxBytes) return GNK_OK;
    long long *cnt = nullptr, *soff = nullptr;
    if (pool_alloc(reinterpret_cast<void**>(&cnt), 2 * ni * sizeof(long long), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&soff), (ni + 1) * sizeof(long long), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->nq_off), (ni + 1) * sizeof(long long), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->nq_re), bytes, st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->nq_im), bytes, st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->nq_item), ni * sizeof(int4), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->nq_src), (size_t)nsrc * sizeof(int), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->xs), (size_t)kMaxRHS * b.N * sizeof(float2), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&t->xl), (size_t)kMaxRHS * nsrc * sizeof(float2), st) != cudaSuccess) {
        cudaGetLastError();
        pool_free(cnt, st);
        pool_free(soff, st);
        pool_free(t->nq_off, st);
        pool_free(t->nq_re, st);
        pool_free(t->nq_im, st);
        pool_free(t->nq_item, st);
        pool_free(t->nq_src, st);
        pool_free(t->xs, st);
        pool_free(t->xl, st);
        t->xl = nullptr;
        t->nq_off = nullptr;
        t->nq_re = t->nq_im = nullptr;
        t->nq_item = nullptr;
        t->nq_src = nullptr;
        t->xs = nullptr;
        return GNK_OK;
    }
    t->nq_slots = slots;
    t->nq_qb = nsrc;
    t->nq_cnt = cnt;
    t->nq_soff = soff;
    t->nq_state = 2;  // allocated; formed by near_cache_build before the first cached near field
    return GNK_OK;
}

// The launches that form the cache (count, scans, entries), on `st` after the
// product has forked its far field, so that they overlap it.
static int near_cache_build(const Boundary& b, cudaStream_t st) {
    FmmTree* t = b.fmm;
    if (t->nq_state != 2) return GNK_OK;
    FmmArgs a;
    fmm_args(b, a);
    const size_t ni = (size_t)t->nitems;
    long long* cnt = t->nq_cnt;
    long long* scnt = cnt + ni;
    long long* soff = t->nq_soff;
    GNK_TRY_CUDA(cudaMemsetAsync(t->nq_src, 0xff, (size_t)t->nq_qb * sizeof(int), st));  // -1: padding
    fmm_nq_count_kernel<<<(t->nitems + 255) / 256, 256, 0, st>>>(a, cnt, scnt);
    fmm_nq_scan_kernel<<<1, 1024, 0, st>>>(cnt, t->nitems, t->nq_off);
    fmm_nq_scan_kernel<<<1, 1024, 0, st>>>(scnt, t->nitems, soff);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(3);
    const ProfToken tok = prof_begin(st, PK_OTHER);
    fmm_nq_build_kernel<<<t->nitems, kFmmNT, 0, st>>>(a, b.q, t->nq_off, soff, t->nq_re, t->nq_im, t->nq_item,
                                                      t->nq_src);
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tok, PK_OTHER, 0.0, st);
    count_launches(1);
    pool_free(cnt, st);
    pool_free(soff, st);
    t->nq_cnt = nullptr;
    t->nq_soff = nullptr;
    t->nq_state = 1;
    return GNK_OK;
}

// L2P with the product's epilogue, one instantiation per epilogue kind (the
// kind known at compile time: only its case is compiled in).
template <int R, int EK>
static void l2p_epi_launch(const FmmArgs& a, const ReduceArgs& e, int nb, cudaStream_t st) {
    fmm_l2p_kernel<R, false, true, EK><<<nb, 256, 0, st>>>(a, e);
}

template <int R>
static int l2p_epi(const FmmArgs& a, const ReduceArgs& e, int nb, cudaStream_t st) {
    switch (e.job.epi) {
        case EPI_Z: l2p_epi_launch<R, EPI_Z>(a, e, nb, st); break;
        case EPI_IMINUSN: l2p_epi_launch<R, EPI_IMINUSN>(a, e, nb, st); break;
        case EPI_M: l2p_epi_launch<R, EPI_M>(a, e, nb, st); break;
        case EPI_ADJ: l2p_epi_launch<R, EPI_ADJ>(a, e, nb, st); break;
        case EPI_RESID: l2p_epi_launch<R, EPI_RESID>(a, e, nb, st); break;
        case EPI_RESID_ADJ: l2p_epi_launch<R, EPI_RESID_ADJ>(a, e, nb, st); break;
        case EPI_H: l2p_epi_launch<R, EPI_H>(a, e, nb, st); break;
        case EPI_EONE: l2p_epi_launch<R, EPI_EONE>(a, e, nb, st); break;
        case EPI_RHS_FB: l2p_epi_launch<R, EPI_RHS_FB>(a, e, nb, st); break;
        case EPI_RESID_FC: l2p_epi_launch<R, EPI_RESID_FC>(a, e, nb, st); break;
        case EPI_IMINUSN_T: l2p_epi_launch<R, EPI_IMINUSN_T>(a, e, nb, st); break;
        case EPI_RESID_T: l2p_epi_launch<R, EPI_RESID_T>(a, e, nb, st); break;
        case EPI_MT: l2p_epi_launch<R, EPI_MT>(a, e, nb, st); break;
        case EPI_EONE_RHS: l2p_epi_launch<R, EPI_EONE_RHS>(a, e, nb, st); break;
        default:
            set_error("FMM: unknown epilogue kind %d", e.job.epi);
            return GNK_EINVAL;
    }
    return GNK_OK;
}

template <int R, int COMP>
static int launch_near_bulk(const Boundary& b, const FmmArgs& a, cudaStream_t st) {
    using L = NbLayout<R, COMP>;
    static std::mutex mu;
    static std::vector<char> ready;  // per device: the shared-memory attribute is set
    int dev = 0;
    GNK_TRY_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(mu);
        if ((int)ready.size() <= dev) ready.resize(dev + 1, 0);
        if (!ready[dev]) {
            GNK_TRY_CUDA(cudaFuncSetAttribute(fmm_near_bulk_kernel<R, COMP>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes));
            ready[dev] = 1;
        }
    }
    const FmmTree* t = b.fmm;
    fmm_near_bulk_kernel<R, COMP><<<t->nitems, kNbThreads, L::kBytes, st>>>(a, t->nq_off, t->nq_item, t->nq_re,
                                                                            t->nq_im, t->xl, t->nq_qb);
    GNK_TRY_CUDA(cudaGetLastError());
    return GNK_OK;
}

// Starts forming the near-field cache right after the tree, on a stream of its
// own, so that it overlaps whatever the caller enqueues before the first cached
// product (the power table, the right-hand side's circulant, the first
// product's gather and far field); that product waits for it.  For callers
// whose products are z = E(q x) (the FBIE and the equation's solves).
int fmm_start_near_cache(const Boundary& bc, cudaStream_t st) {
    Boundary& b = const_cast<Boundary&>(bc);
    if (b.plain) return GNK_OK;
    GNK_TRY(ensure_fmm(b, kMaxRHS, st));
    FmmTree* t = b.fmm;
    GNK_TRY(ensure_near_cache(b, st));
    if (t->nq_state != 2) return GNK_OK;
    if (!t->bst) {
        if (take_stream(false, &t->bst) != cudaSuccess || take_event(&t->ev_nq) != cudaSuccess) {
            cudaGetLastError();
            return GNK_OK;  // formed by the first cached product instead
        }
    }
    // the cache's buffers were allocated in the order of `st`
    GNK_TRY_CUDA(cudaEventRecord(t->ev_nq, st));
    GNK_TRY_CUDA(cudaStreamWaitEvent(t->bst, t->ev_nq, 0));
    GNK_TRY(near_cache_build(b, t->bst));
    GNK_TRY_CUDA(cudaEventRecord(t->ev_nq, t->bst));
    t->nq_wait = 1;
    return GNK_OK;
}

// One FMM product on the argument block `a` (weights, outputs set by the caller):
// gather, the far-field chain on the high-priority stream, the near field on
// `st`, and L2P after they join.  EF: also the sums of w/d^2 (to a.outF).
static int fmm_product(const Boundary& b, FmmArgs& a, int R, bool EF, const ReduceArgs* epi, cudaStream_t st,
                       int* nlaunch, int cached = -1) {
    const FmmTree* t = b.fmm;
    fmm_gather_kernel<<<(b.N + 255) / 256, 256, 0, st>>>(a);
    GNK_TRY_CUDA(cudaEventRecord(t->ev_fork, st));
    GNK_TRY_CUDA(cudaStreamWaitEvent(t->aux, t->ev_fork, 0));
    cudaStream_t fs = t->aux;
    int launches = 1;
    // the far field on its stream: the upward pass (P2M and the M2M climb in
    // one launch), M2L for every box, L2L per leaf.  (Running the finest
    // level's M2L on a third stream beside the climb measured slower: the two
    // compete for the same SMs.)
    const ProfToken toku = prof_begin(fs, PK_FMMUP);
    if (R == 2 && a.tp)
        fmm_up_kernel<2, true><<<t->nleaf, kFmmUT, 0, fs>>>(a);
    else if (R == 2)
        fmm_up_kernel<2, false><<<t->nleaf, kFmmUT, 0, fs>>>(a);
    else if (a.tp)
        fmm_up_kernel<1, true><<<t->nleaf, kFmmUT, 0, fs>>>(a);
    else
        fmm_up_kernel<1, false><<<t->nleaf, kFmmUT, 0, fs>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(toku, PK_FMMUP, 0.0, fs, fmm_instr(b, R, 1));
    const ProfToken tokm = prof_begin(fs, PK_FMM);
    if (R == 2)
        fmm_m2l_kernel<2><<<t->nbox, kFmmUT, 0, fs>>>(a);
    else
        fmm_m2l_kernel<1><<<t->nbox, kFmmUT, 0, fs>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tokm, PK_FMM, (double)R, fs, fmm_instr(b, R, 0));  // work: Cauchy sums (products)
    launches += 2;
    if (t->L > 2) {
        const ProfToken tokd = prof_begin(fs, PK_FMML2L);
        if (R == 2)
            fmm_l2l_kernel<2><<<t->nleaf, 32, 0, fs>>>(a);
        else
            fmm_l2l_kernel<1><<<t->nleaf, 32, 0, fs>>>(a);
        GNK_TRY_CUDA(cudaGetLastError());
        prof_end(tokd, PK_FMML2L, 0.0, fs, fmm_instr(b, R, 2));
        ++launches;
    }
    GNK_TRY_CUDA(cudaEventRecord(t->ev_join, fs));
    // near field on the caller's stream (from the operator cache when `cached`
    // is 0 (both parts of z) or 1 (Im z only)); the first cached product forms
    // the cache here, beside its far field
    if (cached >= 0) {
        if (t->nq_wait) {  // formed on its own stream since the tree was built
            GNK_TRY_CUDA(cudaStreamWaitEvent(st, t->ev_nq, 0));
            b.fmm->nq_wait = 0;
        } else {
            GNK_TRY(near_cache_build(b, st));
        }
    }
    if (cached >= 0) {  // x in the items' list order
        fmm_nq_xlist_kernel<<<(unsigned)((t->nq_qb + 255) / 256), 256, 0, st>>>(t->nq_src, t->nq_qb, R, b.N, a.xs,
                                                                               t->xl, a.done);
        GNK_TRY_CUDA(cudaGetLastError());
        ++launches;
    }
    const ProfToken tokn = prof_begin(st, PK_FMMNEAR);
    if (cached >= 0) {
        if (R == 2 && cached == 1)
            GNK_TRY((launch_near_bulk<2, 1>(b, a, st)));
        else if (R == 2)
            GNK_TRY((launch_near_bulk<2, 0>(b, a, st)));
        else if (cached == 1)
            GNK_TRY((launch_near_bulk<1, 1>(b, a, st)));
        else
            GNK_TRY((launch_near_bulk<1, 0>(b, a, st)));
    } else if (R == 2 && EF)
        fmm_near_kernel<2, true><<<t->nitems, kFmmNT, 0, st>>>(a);
    else if (R == 2)
        fmm_near_kernel<2, false><<<t->nitems, kFmmNT, 0, st>>>(a);
    else if (EF)
        fmm_near_kernel<1, true><<<t->nitems, kFmmNT, 0, st>>>(a);
    else
        fmm_near_kernel<1, false><<<t->nitems, kFmmNT, 0, st>>>(a);
    ++launches;
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tokn, PK_FMMNEAR, (double)R * t->near_pairs, st,
             cached >= 0 ? fmm_near_cached_instr(b, R, cached) : fmm_near_instr(b, R) * (EF ? 2.0 : 1.0),
             cached >= 0 ? fmm_near_cached_bytes(b, R, cached) : 0.0);
    GNK_TRY_CUDA(cudaStreamWaitEvent(st, t->ev_join, 0));
    const ProfToken tokp = prof_begin(st, PK_FMML2P);
    const int nb = (b.N + 255) / 256;
    const ReduceArgs e = epi ? *epi : ReduceArgs{};
    if (R == 2 && EF)
        fmm_l2p_kernel<2, true, false><<<nb, 256, 0, st>>>(a, e);
    else if (R == 2 && epi)
        GNK_TRY(l2p_epi<2>(a, e, nb, st));
    else if (R == 2)
        fmm_l2p_kernel<2, false, false><<<nb, 256, 0, st>>>(a, e);
    else if (EF)
        fmm_l2p_kernel<1, true, false><<<nb, 256, 0, st>>>(a, e);
    else if (epi)
        GNK_TRY(l2p_epi<1>(a, e, nb, st));
    else
        fmm_l2p_kernel<1, false, false><<<nb, 256, 0, st>>>(a, e);
    ++launches;
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tokp, PK_FMML2P, 0.0, st, fmm_instr(b, R, EF ? 4 : 3));
    *nlaunch = launches;
    return GNK_OK;
}

static void fmm_args(const Boundary& b, FmmArgs& a) {
    const FmmTree* t = b.fmm;
    a.N = b.N;
    a.P = kFmmP;
    a.perm = t->perm;
    a.ps = t->ps;
    a.p3 = t->p3;
    a.p3b = t->p3b;
    a.leaf_start = t->leaf_start;
    a.leaf_box = t->leaf_box;
    a.center = t->center;
    a.width = t->width;
    a.child_start = t->child_start;
    a.child_count = t->child_count;
    a.parent = t->parent;
    a.quad = t->quad;
    a.il_start = t->il_start;
    a.il_src = t->il_src;
    a.il_off = t->il_off;
    a.nl_start = t->nl_start;
    a.nl_leaf = t->nl_leaf;
    a.items = t->items;
    a.nitems = t->nitems;
    a.zn = t->zn;
    a.zf = t->zf;
    a.node_box = t->node_box;
    a.m2lH = t->m2lH;
    a.m2lS = t->m2lS;
    a.bUp = t->bUp;
    a.ucnt = t->sync;
    a.xs = nullptr;
    a.tp = t->tp;
    a.mult = t->mult;
    a.loc = t->loc;
    a.ws = t->ws;
    a.nbox = t->nbox;
    a.outF = nullptr;
    a.done = nullptr;
    a.fault = t->fault;
}

int run_fmm(const Boundary& b, const PairJob& job, cudaStream_t st) {
    GNK_TRY(ensure_fmm(b, job.R, st));
    FmmArgs a;
    fmm_args(b, a);
    a.R = job.R;
    a.mode = job.mode;
    a.w0 = job.w[0];
    a.w1 = job.w[1];
    a.x0 = job.x[0];
    a.x1 = job.x[1];
    a.s = job.s;
    a.out = nullptr;
    a.done = job.done;
    int launches = 0;
    // products with the handle's own weights q x read the near field from
    // the operator cache (formed by the first of them)
    int cached = -1;
    if (job.mode == W_SCALED && job.s == b.q && !b.plain) {
        GNK_TRY(ensure_near_cache(b, st));
        if (b.fmm->nq_state >= 1) {
            cached = pair_component_needed(b, job) == 1 ? 1 : 0;
            a.xs = b.fmm->xs;
        }
    }
    const ReduceArgs e = reduce_args(b, job, 1, 0);  // the epilogue runs inside L2P
    GNK_TRY(fmm_product(b, a, job.R, false, &e, st, &launches, cached));
    count_launches(launches);
    return GNK_OK;
}

// E w and F w (sums of w_j/(eta_i - eta_j) and of w_j/(eta_i - eta_j)^2, i != j)
// for one or two complex weight vectors (w1 may be null), into E and F
// (R x N complex each, node order), by one FMM pass.
int run_fmm_ef(const Boundary& b, const double2* w0, const double2* w1, double2* E, double2* F, cudaStream_t st) {
    const int R = w1 ? 2 : 1;
    GNK_TRY(ensure_fmm(b, R, st));
    FmmArgs a;
    fmm_args(b, a);
    a.R = R;
    a.mode = W_COMPLEX;
    a.w0 = w0;
    a.w1 = w1;
    a.x0 = a.x1 = nullptr;
    a.s = nullptr;
    a.out = E;
    a.outF = F;
    int launches = 0;
    GNK_TRY(fmm_product(b, a, R, true, nullptr, st, &launches));
    count_launches(launches);
    return GNK_OK;
}

}  // namespace gnk
