// All-pairs Cauchy sums z_i = sum_{j != i} w_j / (eta_i - eta_j)  (Sec. 2.5,
// Eqs. fmm-1, fmm-E) and the pointwise operators built on them (Secs. 3.3,
// 3.4, 4.3, 4.4).
//
// Layout of a launch: blocks along x own a tile of targets held in registers
// (T per thread); blocks along y own a contiguous chunk of source tiles, which
// they stream through shared memory.  Each block writes its partial sums to a
// [chunk][rhs][N] buffer; a second kernel adds the chunks in a fixed order
// (deterministic) in FP64 and applies the operator's epilogue.
//
// Per pair the FP64 kernel spends 13 FP64-pipe instructions:
//   2 DADD (d = eta_i - eta_j), DMUL + DFMA (|d|^2), 3 DFMA to refine the
//   hardware reciprocal seed, 2 DMUL (Re, Im of 1/d), 4 DFMA (w / d);
// the FP32 kernel spends 10 FP32-pipe instructions and one MUFU reciprocal;
// the double-float kernel about 97 FP32-pipe instructions and one MUFU.
#include <algorithm>
#include <cmath>

#include "gnk_internal.h"
#include "epilogue.cuh"
#include "pairmath.cuh"

namespace gnk {
namespace {

// Far-away position for padded sources of a ragged last tile: |d|^2 stays
// finite and the zero weight contributes exactly 0.
constexpr double kFar64 = 1e150;
constexpr float kFar32 = 1e18f;

// ------------------------------------------------------------------ FP64
struct Pair64Args {
    const double2* et;
    int N;
    const double2* w0;
    const double2* w1;
    const double* x0;
    const double* x1;
    const double2* s;
    double2* partial;
    int tiles_src;
    int tiles_per_chunk;
    const int* done;
};

template <int R, int MODE>
__global__ void __launch_bounds__(kThreads64) pairsum64_kernel(Pair64Args a) {
    constexpr int S = kSrcTile64, T = kTargets64, NT = kThreads64;
    __shared__ double2 s_pos[S];
    __shared__ double2 s_w[R][S];
    if (a.done != nullptr && *a.done) return;
    const int N = a.N;
    const int tgt0 = blockIdx.x * (NT * T);

    double px[T], py[T], ax[T][R], ay[T][R];
    int idx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        idx[t] = tgt0 + t * NT + threadIdx.x;
        const double2 p = a.et[min(idx[t], N - 1)];
        px[t] = p.x;
        py[t] = p.y;
#pragma unroll
        for (int r = 0; r < R; ++r) ax[t][r] = ay[t][r] = 0.0;
    }

    const int tb = blockIdx.y * a.tiles_per_chunk;
    const int te = min(tb + a.tiles_per_chunk, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        __syncthreads();
        for (int k = threadIdx.x; k < S; k += NT) {
            const int j = j0 + k;
            if (j < N) {
                s_pos[k] = a.et[j];
                if (MODE == W_COMPLEX) {
                    s_w[0][k] = a.w0[j];
                    if (R > 1) s_w[R - 1][k] = a.w1[j];
                } else {
                    const double2 sc = a.s[j];
                    const double x0 = a.x0[j];
                    s_w[0][k] = make_double2(sc.x * x0, sc.y * x0);
                    if (R > 1) {
                        const double x1 = a.x1[j];
                        s_w[R - 1][k] = make_double2(sc.x * x1, sc.y * x1);
                    }
                }
            } else {
                s_pos[k] = make_double2(kFar64, kFar64);
#pragma unroll
                for (int r = 0; r < R; ++r) s_w[r][k] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
        const bool diag = (j0 < tgt0 + NT * T) && (tgt0 < j0 + S);
        if (!diag) {
#pragma unroll 2
            for (int k = 0; k < S; ++k) {
                const double2 sp = s_pos[k];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const double dx = px[t] - sp.x, dy = py[t] - sp.y;
                    const double inv = recip_f64(fma(dx, dx, dy * dy));
                    const double ar = dx * inv, ai = dy * inv;  // 1/d = ar - i ai
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const double2 w = s_w[r][k];
                        ax[t][r] = fma(w.x, ar, ax[t][r]);
                        ax[t][r] = fma(w.y, ai, ax[t][r]);
                        ay[t][r] = fma(w.y, ar, ay[t][r]);
                        ay[t][r] = fma(-w.x, ai, ay[t][r]);
                    }
                }
            }
        } else {
            for (int k = 0; k < S; ++k) {
                const double2 sp = s_pos[k];
                const int j = j0 + k;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const double dx = px[t] - sp.x, dy = py[t] - sp.y;
                    double inv = recip_f64(fma(dx, dx, dy * dy));
                    inv = (j == idx[t]) ? 0.0 : inv;  // the i = j term is excluded (Eq. fmm-E)
                    const double ar = dx * inv, ai = dy * inv;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const double2 w = s_w[r][k];
                        ax[t][r] = fma(w.x, ar, ax[t][r]);
                        ax[t][r] = fma(w.y, ai, ax[t][r]);
                        ay[t][r] = fma(w.y, ar, ay[t][r]);
                        ay[t][r] = fma(-w.x, ai, ay[t][r]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (idx[t] < N) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                a.partial[((size_t)blockIdx.y * R + r) * N + idx[t]] = make_double2(ax[t][r], ay[t][r]);
        }
    }
}

// ------------------------------------------------------------------ FP32
// Source positions are stored relative to one reference node per source tile
// (off32), and each target forms its own offset to that reference from its
// hi/lo split, so that the difference eta_i - eta_j of two nearby nodes keeps
// its leading bits instead of being lost to the magnitude of eta.
struct Pair32Args {
    const float4* et32;
    const float4* ref32;
    const float2* off32;
    int N;
    const double2* w0;
    const double2* w1;
    const double* x0;
    const double* x1;
    const float2* s32;
    float2* partial;
    int tiles_src;
    int tiles_per_chunk;
    const int* done;
};

template <int R, int MODE>
__global__ void __launch_bounds__(kThreads32) pairsum32_kernel(Pair32Args a) {
    constexpr int S = kSrcTile32, T = kTargets32, NT = kThreads32;
    static_assert(S == NT, "one source per thread per tile load");
    __shared__ float4 s_src[S];          // (off.x, off.y, w0.x, w0.y)
    __shared__ float2 s_w1[R > 1 ? S : 1];
    if (a.done != nullptr && *a.done) return;
    const int N = a.N;
    const int tgt0 = blockIdx.x * (NT * T);

    float4 th[T];
    float ox[T], oy[T], ax[T][R], ay[T][R];
    int idx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        idx[t] = tgt0 + t * NT + threadIdx.x;
        th[t] = a.et32[min(idx[t], N - 1)];
#pragma unroll
        for (int r = 0; r < R; ++r) ax[t][r] = ay[t][r] = 0.0f;
    }

    const int tb = blockIdx.y * a.tiles_per_chunk;
    const int te = min(tb + a.tiles_per_chunk, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        const float4 ref = a.ref32[tile];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            ox[t] = (th[t].x - ref.x) + (th[t].z - ref.z);
            oy[t] = (th[t].y - ref.y) + (th[t].w - ref.w);
        }
        __syncthreads();
        {
            const int k = threadIdx.x;
            const int j = j0 + k;
            float4 v;
            float2 w1 = make_float2(0.f, 0.f);
            if (j < N) {
                const float2 off = a.off32[j];
                float2 w0;
                if (MODE == W_COMPLEX) {
                    const double2 w = a.w0[j];
                    w0 = make_float2((float)w.x, (float)w.y);
                    if (R > 1) {
                        const double2 u = a.w1[j];
                        w1 = make_float2((float)u.x, (float)u.y);
                    }
                } else {
                    const float2 sc = a.s32[j];
                    const float x0 = (float)a.x0[j];
                    w0 = make_float2(sc.x * x0, sc.y * x0);
                    if (R > 1) {
                        const float x1 = (float)a.x1[j];
                        w1 = make_float2(sc.x * x1, sc.y * x1);
                    }
                }
                v = make_float4(off.x, off.y, w0.x, w0.y);
            } else {
                v = make_float4(kFar32, kFar32, 0.f, 0.f);
            }
            s_src[k] = v;
            if (R > 1) s_w1[k] = w1;
        }
        __syncthreads();
        const bool diag = (j0 < tgt0 + NT * T) && (tgt0 < j0 + S);
        if (!diag) {
#pragma unroll 4
            for (int k = 0; k < S; ++k) {
                const float4 sv = s_src[k];
                float2 u;
                if (R > 1) u = s_w1[k];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float dx = ox[t] - sv.x, dy = oy[t] - sv.y;
                    const float inv = recip_f32(fmaf(dx, dx, dy * dy));
                    const float ar = dx * inv, ai = dy * inv;
                    ax[t][0] = fmaf(sv.z, ar, ax[t][0]);
                    ax[t][0] = fmaf(sv.w, ai, ax[t][0]);
                    ay[t][0] = fmaf(sv.w, ar, ay[t][0]);
                    ay[t][0] = fmaf(-sv.z, ai, ay[t][0]);
                    if (R > 1) {
                        ax[t][R - 1] = fmaf(u.x, ar, ax[t][R - 1]);
                        ax[t][R - 1] = fmaf(u.y, ai, ax[t][R - 1]);
                        ay[t][R - 1] = fmaf(u.y, ar, ay[t][R - 1]);
                        ay[t][R - 1] = fmaf(-u.x, ai, ay[t][R - 1]);
                    }
                }
            }
        } else {
            for (int k = 0; k < S; ++k) {
                const float4 sv = s_src[k];
                float2 u;
                if (R > 1) u = s_w1[k];
                const int j = j0 + k;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float dx = ox[t] - sv.x, dy = oy[t] - sv.y;
                    float inv = recip_f32(fmaf(dx, dx, dy * dy));
                    inv = (j == idx[t]) ? 0.0f : inv;
                    const float ar = dx * inv, ai = dy * inv;
                    ax[t][0] = fmaf(sv.z, ar, ax[t][0]);
                    ax[t][0] = fmaf(sv.w, ai, ax[t][0]);
                    ay[t][0] = fmaf(sv.w, ar, ay[t][0]);
                    ay[t][0] = fmaf(-sv.z, ai, ay[t][0]);
                    if (R > 1) {
                        ax[t][R - 1] = fmaf(u.x, ar, ax[t][R - 1]);
                        ax[t][R - 1] = fmaf(u.y, ai, ax[t][R - 1]);
                        ay[t][R - 1] = fmaf(u.y, ar, ay[t][R - 1]);
                        ay[t][R - 1] = fmaf(-u.x, ai, ay[t][R - 1]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (idx[t] < N) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                a.partial[((size_t)blockIdx.y * R + r) * N + idx[t]] = make_float2(ax[t][r], ay[t][r]);
        }
    }
}

// Packed FP32 variant: each thread owns 2 x kPairs32 targets, two per float2
// (x and y lanes); sources are stored duplicated so that one packed
// instruction serves both lanes.
constexpr int kPairs32 = kTargets32 / 2;

// z += w / d = w conj(d) / |d|^2 for both lanes, inv = 1/|d|^2 (0 for i = j)
template <int R, int COMP>
__device__ __forceinline__ void accumulate32(const float4 (*s_w)[kSrcTile32], int k, float2 dx, float2 dy,
                                             float2 inv, float2* ax, float2* ay) {
    if (COMP == 0) {
        const float2 ar = mul2(dx, inv), ai = mul2(dy, inv);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 w = s_w[r][k];
            const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
            ax[r] = fma2(wx, ar, fma2(wy, ai, ax[r]));
            ay[r] = fma2(wy, ar, fma2(neg2(wx), ai, ay[r]));
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 w = s_w[r][k];
            const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
            if (COMP == 1)  // Im(w conj d) = wy dx - wx dy
                ay[r] = fma2(fma2(neg2(wx), dy, mul2(wy, dx)), inv, ay[r]);
            else            // Re(w conj d) = wx dx + wy dy
                ax[r] = fma2(fma2(wy, dy, mul2(wx, dx)), inv, ax[r]);
        }
    }
}

// COMP = 1 (2): only Im z (Re z) is formed, 3 instead of 4 + 2 FP32 operations
// per pair and right-hand side; the other part of the partial sum is written as 0.
template <int R, int MODE, int COMP>
__global__ void __launch_bounds__(kThreads32) pairsum32x2_kernel(Pair32Args a) {
    constexpr int S = kSrcTile32, NT = kThreads32, P = kPairs32;
    static_assert(S == NT, "one source per thread per tile load");
    __shared__ float4 s_o[S];          // (ox, ox, oy, oy)
    __shared__ float4 s_w[R][S];       // (wx, wx, wy, wy)
    if (a.done != nullptr && *a.done) return;
    const int N = a.N;
    const int tgt0 = blockIdx.x * (NT * kTargets32);
    float4 th[2 * P];
    int idx[2 * P];
    float2 ax[P][R], ay[P][R];
#pragma unroll
    for (int t = 0; t < 2 * P; ++t) {
        idx[t] = tgt0 + t * NT + threadIdx.x;
        th[t] = a.et32[min(idx[t], N - 1)];
    }
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) ax[u][r] = ay[u][r] = f2(0.f);
    const int tb = blockIdx.y * a.tiles_per_chunk;
    const int te = min(tb + a.tiles_per_chunk, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        const float4 ref = a.ref32[tile];
        float2 ox[P], oy[P];
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const float4 ta = th[2 * u], tb2 = th[2 * u + 1];
            ox[u] = make_float2((ta.x - ref.x) + (ta.z - ref.z), (tb2.x - ref.x) + (tb2.z - ref.z));
            oy[u] = make_float2((ta.y - ref.y) + (ta.w - ref.w), (tb2.y - ref.y) + (tb2.w - ref.w));
        }
        __syncthreads();
        {
            const int k = threadIdx.x;
            const int j = j0 + k;
            if (j < N) {
                const float2 off = a.off32[j];
                s_o[k] = make_float4(off.x, off.x, off.y, off.y);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float2 w;
                    if (MODE == W_COMPLEX) {
                        const double2 wd = (r == 0) ? a.w0[j] : a.w1[j];
                        w = make_float2((float)wd.x, (float)wd.y);
                    } else {
                        const float2 sc = a.s32[j];
                        const float xv = (float)((r == 0) ? a.x0[j] : a.x1[j]);
                        w = make_float2(sc.x * xv, sc.y * xv);
                    }
                    s_w[r][k] = make_float4(w.x, w.x, w.y, w.y);
                }
            } else {
                s_o[k] = make_float4(kFar32, kFar32, kFar32, kFar32);
#pragma unroll
                for (int r = 0; r < R; ++r) s_w[r][k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        const bool diag = (j0 < tgt0 + NT * kTargets32) && (tgt0 < j0 + S);
        if (!diag) {
#pragma unroll 4
            for (int k = 0; k < S; ++k) {
                const float4 so = s_o[k];
                const float2 sx = make_float2(so.x, so.y), sy = make_float2(so.z, so.w);
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const float2 dx = sub2(ox[u], sx), dy = sub2(oy[u], sy);
                    const float2 r2 = fma2(dy, dy, mul2(dx, dx));
                    const float2 inv = make_float2(recip_f32(r2.x), recip_f32(r2.y));
                    accumulate32<R, COMP>(s_w, k, dx, dy, inv, ax[u], ay[u]);
                }
            }
        } else {
            for (int k = 0; k < S; ++k) {
                const float4 so = s_o[k];
                const float2 sx = make_float2(so.x, so.y), sy = make_float2(so.z, so.w);
                const int j = j0 + k;
#pragma unroll
                for (int u = 0; u < P; ++u) {
                    const float2 dx = sub2(ox[u], sx), dy = sub2(oy[u], sy);
                    const float2 r2 = fma2(dy, dy, mul2(dx, dx));
                    float i0 = recip_f32(r2.x), i1 = recip_f32(r2.y);
                    i0 = (j == idx[2 * u]) ? 0.f : i0;
                    i1 = (j == idx[2 * u + 1]) ? 0.f : i1;
                    const float2 inv = make_float2(i0, i1);
                    accumulate32<R, COMP>(s_w, k, dx, dy, inv, ax[u], ay[u]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < P; ++u) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (idx[2 * u] < N)
                a.partial[((size_t)blockIdx.y * R + r) * N + idx[2 * u]] = make_float2(ax[u][r].x, ay[u][r].x);
            if (idx[2 * u + 1] < N)
                a.partial[((size_t)blockIdx.y * R + r) * N + idx[2 * u + 1]] = make_float2(ax[u][r].y, ay[u][r].y);
        }
    }
}

// ------------------------------------------------------------------ double-float (df32)
// (arithmetic helpers in pairmath.cuh)
struct PairDFArgs {
    const double2* et;
    const double2* ref64;
    const float4* offdf;   // per node: (dx.h, dy.h, dx.l, dy.l) of eta_j - ref(tile(j))
    int N;
    const double2* w0;
    const double2* w1;
    const double* x0;
    const double* x1;
    const double2* s;
    float4* partial;       // [chunk][rhs][N]: (re.h, re.l, im.h, im.l)
    int tiles_src;
    int tiles_per_chunk;
    const int* done;
};

template <int R, int MODE>
__global__ void __launch_bounds__(kThreadsDF) pairsumdf_kernel(PairDFArgs a) {
    constexpr int S = kSrcTile32, T = kTargetsDF, NT = kThreadsDF;
    static_assert(S == NT, "one source per thread per tile load");
    __shared__ float4 s_off[S];
    __shared__ float4 s_w[R][S];  // (wx.h, wx.l, wy.h, wy.l)
    if (a.done != nullptr && *a.done) return;
    const int N = a.N;
    const int tgt0 = blockIdx.x * (NT * T);

    double2 p[T];
    df acc_re[T][R], acc_im[T][R];
    int idx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        idx[t] = tgt0 + t * NT + threadIdx.x;
        p[t] = a.et[min(idx[t], N - 1)];
#pragma unroll
        for (int r = 0; r < R; ++r) acc_re[t][r] = acc_im[t][r] = df{0.f, 0.f};
    }

    const int tb = blockIdx.y * a.tiles_per_chunk;
    const int te = min(tb + a.tiles_per_chunk, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        const double2 ref = a.ref64[tile];
        df ox[T], oy[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {  // target offsets, once per tile, in FP64
            ox[t] = df_split(p[t].x - ref.x);
            oy[t] = df_split(p[t].y - ref.y);
        }
        __syncthreads();
        {
            const int k = threadIdx.x;
            const int j = j0 + k;
            if (j < N) {
                s_off[k] = a.offdf[j];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double2 w;
                    if (MODE == W_COMPLEX) {
                        w = (r == 0) ? a.w0[j] : a.w1[j];
                    } else {
                        const double2 sc = a.s[j];
                        const double x = (r == 0) ? a.x0[j] : a.x1[j];
                        w = make_double2(sc.x * x, sc.y * x);
                    }
                    const df wx = df_split(w.x), wy = df_split(w.y);
                    s_w[r][k] = make_float4(wx.h, wx.l, wy.h, wy.l);
                }
            } else {
                s_off[k] = make_float4(kFar32, kFar32, 0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R; ++r) s_w[r][k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        const bool diag = (j0 < tgt0 + NT * T) && (tgt0 < j0 + S);
#pragma unroll 2
        for (int k = 0; k < S; ++k) {
            const float4 so = s_off[k];
            const int j = j0 + k;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const df dx = df_sub(ox[t].h, ox[t].l, so.x, so.z);
                const df dy = df_sub(oy[t].h, oy[t].l, so.y, so.w);
                // |d|^2 = dx.h^2 + dy.h^2 + 2 dx.h dx.l + 2 dy.h dy.l  (lo^2 terms below 2^-48)
                const float px = __fmul_rn(dx.h, dx.h);
                float ex = fmaf(dx.h, dx.h, -px);
                ex = fmaf(dx.h, dx.l + dx.l, ex);
                const float py = __fmul_rn(dy.h, dy.h);
                float ey = fmaf(dy.h, dy.h, -py);
                ey = fmaf(dy.h, dy.l + dy.l, ey);
                float rh, re;
                two_sum(px, py, rh, re);
                const float rl = __fadd_rn(__fadd_rn(ex, ey), re);
                // 1/|d|^2: one Newton step from the 2^-23 seed gives ~2^-46
                float y = recip_f32(rh);
                if (diag && j == idx[t]) y = 0.0f;  // the i = j term is excluded (Eq. fmm-E)
                float e = fmaf(-rh, y, 1.0f);
                e = fmaf(-rl, y, e);
                const df inv = df{y, __fmul_rn(y, e)};
                const df ar = df_mul(dx, inv);  // 1/d = ar - i ai
                const df ai = df_mul(dy, inv);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 w = s_w[r][k];
                    const df wx{w.x, w.y}, wy{w.z, w.w};
                    // z += w (ar - i ai): re += wx ar + wy ai, im += wy ar - wx ai
                    df_acc(acc_re[t][r], df_mul(wx, ar));
                    df_acc(acc_re[t][r], df_mul(wy, ai));
                    df_acc(acc_im[t][r], df_mul(wy, ar));
                    const df q = df_mul(wx, ai);
                    df_acc(acc_im[t][r], df{-q.h, -q.l});
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (idx[t] < N) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                a.partial[((size_t)blockIdx.y * R + r) * N + idx[t]] =
                    make_float4(acc_re[t][r].h, acc_re[t][r].l, acc_im[t][r].h, acc_im[t][r].l);
        }
    }
}

// Packed variant: each thread owns two targets held in the x and y lanes of
// float2 registers; every double-float operation of a pair is one packed
// instruction for both targets.  Source values are stored duplicated (v, v)
// in shared memory so that they broadcast to both lanes.
template <int R, int MODE, int COMP>
__global__ void __launch_bounds__(kThreadsDF) pairsumdf2_kernel(PairDFArgs a) {
    constexpr int S = kSrcTile32, NT = kThreadsDF;
    static_assert(S == NT, "one source per thread per tile load");
    static_assert(kTargetsDF == 2, "two targets per thread, one per lane");
    __shared__ float4 s_off[2][S];       // (xh, xh, yh, yh), (xl, xl, yl, yl)
    __shared__ float4 s_w[R][2][S];      // (wxh, wxh, wxl, wxl), (wyh, wyh, wyl, wyl)
    if (a.done != nullptr && *a.done) return;
    const int N = a.N;
    const int tgt0 = blockIdx.x * (NT * 2);
    const int i0 = tgt0 + threadIdx.x, i1 = tgt0 + NT + threadIdx.x;
    const double2 p0 = a.et[min(i0, N - 1)], p1 = a.et[min(i1, N - 1)];
    df2 are[R], aim[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        are[r] = df2{f2(0.f), f2(0.f)};
        aim[r] = df2{f2(0.f), f2(0.f)};
    }
    const int tb = blockIdx.y * a.tiles_per_chunk;
    const int te = min(tb + a.tiles_per_chunk, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        const double2 ref = a.ref64[tile];
        const df ox0 = df_split(p0.x - ref.x), ox1 = df_split(p1.x - ref.x);
        const df oy0 = df_split(p0.y - ref.y), oy1 = df_split(p1.y - ref.y);
        const float2 oxh = make_float2(ox0.h, ox1.h), oxl = make_float2(ox0.l, ox1.l);
        const float2 oyh = make_float2(oy0.h, oy1.h), oyl = make_float2(oy0.l, oy1.l);
        __syncthreads();
        {
            const int k = threadIdx.x;
            const int j = j0 + k;
            if (j < N) {
                const float4 o = a.offdf[j];
                s_off[0][k] = make_float4(o.x, o.x, o.y, o.y);
                s_off[1][k] = make_float4(o.z, o.z, o.w, o.w);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double2 w;
                    if (MODE == W_COMPLEX) {
                        w = (r == 0) ? a.w0[j] : a.w1[j];
                    } else {
                        const double2 sc = a.s[j];
                        const double x = (r == 0) ? a.x0[j] : a.x1[j];
                        w = make_double2(sc.x * x, sc.y * x);
                    }
                    const df wx = df_split(w.x), wy = df_split(w.y);
                    s_w[r][0][k] = make_float4(wx.h, wx.h, wx.l, wx.l);
                    s_w[r][1][k] = make_float4(wy.h, wy.h, wy.l, wy.l);
                }
            } else {
                s_off[0][k] = make_float4(kFar32, kFar32, kFar32, kFar32);
                s_off[1][k] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    s_w[r][0][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    s_w[r][1][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        __syncthreads();
        const bool diag = (j0 < tgt0 + NT * 2) && (tgt0 < j0 + S);
#pragma unroll 2
        for (int k = 0; k < S; ++k) {
            const float4 oa = s_off[0][k], ob = s_off[1][k];
            const df2 dx = df2_sub(oxh, oxl, make_float2(oa.x, oa.y), make_float2(ob.x, ob.y));
            const df2 dy = df2_sub(oyh, oyl, make_float2(oa.z, oa.w), make_float2(ob.z, ob.w));
            const float2 px = mul2(dx.h, dx.h);
            float2 ex = fma2(dx.h, dx.h, neg2(px));
            ex = fma2(dx.h, add2(dx.l, dx.l), ex);
            const float2 py = mul2(dy.h, dy.h);
            float2 ey = fma2(dy.h, dy.h, neg2(py));
            ey = fma2(dy.h, add2(dy.l, dy.l), ey);
            float2 rh, re;
            two_sum2(px, py, rh, re);
            const float2 rl = add2(add2(ex, ey), re);
            float y0 = recip_f32(rh.x), y1 = recip_f32(rh.y);
            if (diag) {  // the i = j term is excluded (Eq. fmm-E)
                y0 = (j0 + k == i0) ? 0.f : y0;
                y1 = (j0 + k == i1) ? 0.f : y1;
            }
            const float2 y = make_float2(y0, y1);
            float2 e = fma2(neg2(rh), y, f2(1.0f));
            e = fma2(neg2(rl), y, e);
            const df2 inv{y, mul2(y, e)};
            const df2 ar = df2_mul(dx, inv);  // 1/d = ar - i ai
            const df2 ai = df2_mul(dy, inv);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 wa = s_w[r][0][k], wb = s_w[r][1][k];
                const df2 wx{make_float2(wa.x, wa.y), make_float2(wa.z, wa.w)};
                const df2 wy{make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
                if (COMP != 1) {
                    df2_acc(are[r], df2_mul(wx, ar));
                    df2_acc(are[r], df2_mul(wy, ai));
                }
                if (COMP != 2) {
                    df2_acc(aim[r], df2_mul(wy, ar));
                    df2_dec(aim[r], df2_mul(wx, ai));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (i0 < N)
            a.partial[((size_t)blockIdx.y * R + r) * N + i0] =
                make_float4(are[r].h.x, are[r].l.x, aim[r].h.x, aim[r].l.x);
        if (i1 < N)
            a.partial[((size_t)blockIdx.y * R + r) * N + i1] =
                make_float4(are[r].h.y, are[r].l.y, aim[r].h.y, aim[r].l.y);
    }
}

// ------------------------------------------------------------------ reduce + epilogue
__global__ void reduce_epilogue_kernel(ReduceArgs a) {
    const PairJob& j = a.job;
    if (j.done != nullptr && *j.done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int N = a.N;
    double zx[kMaxRHS] = {0.0, 0.0}, zy[kMaxRHS] = {0.0, 0.0};
    for (int r = 0; r < a.R; ++r) {
        double sx = 0.0, sy = 0.0;
        if (a.ptype == 1) {
            for (int ch = 0; ch < a.chunks; ++ch) {
                const float2 p = a.p32[((size_t)ch * a.R + r) * N + i];
                sx += (double)p.x;
                sy += (double)p.y;
            }
        } else if (a.ptype == 2) {
            for (int ch = 0; ch < a.chunks; ++ch) {
                const float4 p = a.pdf[((size_t)ch * a.R + r) * N + i];
                sx += (double)p.x + (double)p.y;
                sy += (double)p.z + (double)p.w;
            }
        } else {
            for (int ch = 0; ch < a.chunks; ++ch) {
                const double2 p = a.p64[((size_t)ch * a.R + r) * N + i];
                sx += p.x;
                sy += p.y;
            }
        }
        zx[r] = sx;
        zy[r] = sy;
    }
    epilogue_apply(a, i, make_double2(zx[0], zy[0]), make_double2(zx[1], zy[1]));
}

cudaError_t launch_reduce(const Boundary& b, const PairJob& job, int chunks, int ptype,
                          cudaStream_t st, const void* partial = nullptr) {
    ReduceArgs ra = reduce_args(b, job, chunks, ptype);
    if (partial) {
        ra.pdf = static_cast<const float4*>(partial);
        ra.p64 = static_cast<const double2*>(partial);
        ra.p32 = static_cast<const float2*>(partial);
    }
    const int threads = 256;
    const ProfToken tok = prof_begin(st, PK_REDUCE);
    reduce_epilogue_kernel<<<(b.N + threads - 1) / threads, threads, 0, st>>>(ra);
    const cudaError_t e = cudaGetLastError();
    // bytes: the partials read plus about four N-vectors of operands and output
    prof_end(tok, PK_REDUCE,
             (double)chunks * job.R * b.N * (ptype == 1 ? 8.0 : 16.0) + 4.0 * 8.0 * b.N, st);
    return e;
}

}  // namespace

// Chunking of the source range: choose the number of source tiles per chunk
// that maximises the fraction of useful block-slots over the launch's waves,
// so the grid covers all SMs even when few target tiles exist.
PairPlan make_plan(int N, int sms, int blocks_per_sm, int targets_per_block, int src_tile) {
    PairPlan p;
    p.tiles_tgt = (N + targets_per_block - 1) / targets_per_block;
    p.tiles_src = (N + src_tile - 1) / src_tile;
    const long slots = std::max(1L, (long)sms * blocks_per_sm);
    double best = -1.0;
    int best_tpc = p.tiles_src;
    const int max_chunks = 64;
    for (int tpc = p.tiles_src; tpc >= 1; --tpc) {
        const int chunks = (p.tiles_src + tpc - 1) / tpc;
        if (chunks > max_chunks) break;
        const long blocks = (long)p.tiles_tgt * chunks;
        const long waves = (blocks + slots - 1) / slots;
        const double eff = (double)p.tiles_tgt * p.tiles_src / ((double)waves * slots * tpc);
        if (eff > best * 1.02) {  // prefer fewer chunks unless clearly better
            best = eff;
            best_tpc = tpc;
        }
    }
    p.tiles_per_chunk = best_tpc;
    p.chunks = (p.tiles_src + best_tpc - 1) / best_tpc;
    return p;
}

int pair_workspace_bytes(const Boundary& b, size_t* bytes) {
    const size_t b64 = (size_t)b.plan64.chunks * kMaxRHS * b.N * sizeof(double2);
    const size_t b32 = (size_t)b.plan32.chunks * kMaxRHS * b.N * sizeof(float2);
    const size_t bdf = (size_t)b.plandf.chunks * kMaxRHS * b.N * sizeof(float4);
    *bytes = std::max(std::max(b64, b32), bdf);
    return GNK_OK;
}

// The plan of one launch: the handle's plan, or, under a source-chunk override
// (gnk_options.tile_chunks), that many chunks (at most one per source tile)
// with a partial-sum workspace large enough for them.
static int launch_plan(const Boundary& b, const PairPlan& base, size_t elem_bytes, PairPlan* p,
                       void** partial, cudaStream_t st) {
    *p = base;
    *partial = b.partial;
    if (b.tile_chunks <= 0) return GNK_OK;
    const int want = std::min(b.tile_chunks, p->tiles_src);
    p->tiles_per_chunk = (p->tiles_src + want - 1) / want;
    p->chunks = (p->tiles_src + p->tiles_per_chunk - 1) / p->tiles_per_chunk;
    const size_t need = (size_t)p->chunks * kMaxRHS * b.N * elem_bytes;
    if (need <= b.partial_bytes) return GNK_OK;
    if (need > b.partial_x_bytes) {
        if (b.partial_x) pool_free(b.partial_x, st);
        b.partial_x = nullptr;
        b.partial_x_bytes = 0;
        if (pool_alloc(&b.partial_x, need, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("pair-sum workspace for %d source chunks: allocation failed", p->chunks);
            return GNK_ENOMEM;
        }
        b.partial_x_bytes = need;
    }
    *partial = b.partial_x;
    return GNK_OK;
}

int run_pairsum64(const Boundary& b, const PairJob& job, cudaStream_t st) {
    PairPlan p;
    void* partial = nullptr;
    GNK_TRY(launch_plan(b, b.plan64, sizeof(double2), &p, &partial, st));
    Pair64Args a;
    a.et = b.et;
    a.N = b.N;
    a.w0 = job.w[0];
    a.w1 = job.w[1];
    a.x0 = job.x[0];
    a.x1 = job.x[1];
    a.s = job.s;
    a.partial = static_cast<double2*>(partial);
    a.tiles_src = p.tiles_src;
    a.tiles_per_chunk = p.tiles_per_chunk;
    a.done = job.done;
    dim3 grid(p.tiles_tgt, p.chunks);
    const ProfToken tok = prof_begin(st);
    if (job.R == 1 && job.mode == W_SCALED)
        pairsum64_kernel<1, W_SCALED><<<grid, kThreads64, 0, st>>>(a);
    else if (job.R == 1)
        pairsum64_kernel<1, W_COMPLEX><<<grid, kThreads64, 0, st>>>(a);
    else if (job.mode == W_SCALED)
        pairsum64_kernel<2, W_SCALED><<<grid, kThreads64, 0, st>>>(a);
    else
        pairsum64_kernel<2, W_COMPLEX><<<grid, kThreads64, 0, st>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    // FP64 pipe per pair: 9 shared (d, |d|^2, reciprocal, 1/d) + 4 per right-hand side
    prof_end(tok, PK_PAIR64, (double)job.R * b.N * (b.N - 1.0), st,
             (9.0 + 4.0 * job.R) * b.N * (b.N - 1.0));
    GNK_TRY_CUDA(launch_reduce(b, job, p.chunks, 0, st, partial));
    count_launches(2);
    return GNK_OK;
}

int run_pairsum32(const Boundary& b, const PairJob& job, cudaStream_t st) {
    PairPlan p;
    void* partial = nullptr;
    GNK_TRY(launch_plan(b, b.plan32, sizeof(float2), &p, &partial, st));
    Pair32Args a;
    a.et32 = b.et32;
    a.ref32 = b.ref32;
    a.off32 = b.off32;
    a.N = b.N;
    a.w0 = job.w[0];
    a.w1 = job.w[1];
    a.x0 = job.x[0];
    a.x1 = job.x[1];
    a.s32 = (job.s == b.q) ? b.q32 : b.A32;
    a.partial = static_cast<float2*>(partial);
    a.tiles_src = p.tiles_src;
    a.tiles_per_chunk = p.tiles_per_chunk;
    a.done = job.done;
    if (job.mode == W_SCALED && job.s != b.q && job.s != b.A) {
        set_error("FP32 pair sum: the scale must be q or A of the handle");
        return GNK_EINVAL;
    }
    dim3 grid(p.tiles_tgt, p.chunks);
    const ProfToken tok = prof_begin(st);
    const int comp = b.f32_scalar ? 0 : job.comp;
    if (!b.f32_scalar) {
        if (job.R == 1 && job.mode == W_SCALED && comp == 1)
            pairsum32x2_kernel<1, W_SCALED, 1><<<grid, kThreads32, 0, st>>>(a);
        else if (job.R == 1 && job.mode == W_SCALED && comp == 2)
            pairsum32x2_kernel<1, W_SCALED, 2><<<grid, kThreads32, 0, st>>>(a);
        else if (job.R == 1 && job.mode == W_SCALED)
            pairsum32x2_kernel<1, W_SCALED, 0><<<grid, kThreads32, 0, st>>>(a);
        else if (job.R == 1)
            pairsum32x2_kernel<1, W_COMPLEX, 0><<<grid, kThreads32, 0, st>>>(a);
        else if (job.mode == W_SCALED)
            pairsum32x2_kernel<2, W_SCALED, 0><<<grid, kThreads32, 0, st>>>(a);
        else
            pairsum32x2_kernel<2, W_COMPLEX, 0><<<grid, kThreads32, 0, st>>>(a);
    } else if (job.R == 1 && job.mode == W_SCALED)
        pairsum32_kernel<1, W_SCALED><<<grid, kThreads32, 0, st>>>(a);
    else if (job.R == 1)
        pairsum32_kernel<1, W_COMPLEX><<<grid, kThreads32, 0, st>>>(a);
    else if (job.mode == W_SCALED)
        pairsum32_kernel<2, W_SCALED><<<grid, kThreads32, 0, st>>>(a);
    else
        pairsum32_kernel<2, W_COMPLEX><<<grid, kThreads32, 0, st>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    // FP32 pipe per pair (plus one MUFU reciprocal): 6 shared + 4 per right-hand
    // side; one part of z only: 4 shared + 3 per right-hand side
    const double per_pair = (comp && job.R == 1) ? 4.0 + 3.0 : 6.0 + 4.0 * job.R;
    prof_end(tok, PK_PAIR32, (double)job.R * b.N * (b.N - 1.0), st, per_pair * b.N * (b.N - 1.0));
    GNK_TRY_CUDA(launch_reduce(b, job, p.chunks, 1, st, partial));
    count_launches(2);
    return GNK_OK;
}

int run_pairsumdf(const Boundary& b, const PairJob& job, cudaStream_t st) {
    PairPlan p;
    void* partial = nullptr;
    GNK_TRY(launch_plan(b, b.plandf, sizeof(float4), &p, &partial, st));
    PairDFArgs a;
    a.et = b.et;
    a.ref64 = b.ref64;
    a.offdf = b.offdf;
    a.N = b.N;
    a.w0 = job.w[0];
    a.w1 = job.w[1];
    a.x0 = job.x[0];
    a.x1 = job.x[1];
    a.s = job.s;
    a.partial = static_cast<float4*>(partial);
    a.tiles_src = p.tiles_src;
    a.tiles_per_chunk = p.tiles_per_chunk;
    a.done = job.done;
    dim3 grid(p.tiles_tgt, p.chunks);
    const ProfToken tok = prof_begin(st);
    const int comp = b.df_scalar ? 0 : job.comp;
    if (!b.df_scalar) {
        if (job.R == 1 && job.mode == W_SCALED && comp == 1)
            pairsumdf2_kernel<1, W_SCALED, 1><<<grid, kThreadsDF, 0, st>>>(a);
        else if (job.R == 1 && job.mode == W_SCALED && comp == 2)
            pairsumdf2_kernel<1, W_SCALED, 2><<<grid, kThreadsDF, 0, st>>>(a);
        else if (job.R == 1 && job.mode == W_SCALED)
            pairsumdf2_kernel<1, W_SCALED, 0><<<grid, kThreadsDF, 0, st>>>(a);
        else if (job.R == 1)
            pairsumdf2_kernel<1, W_COMPLEX, 0><<<grid, kThreadsDF, 0, st>>>(a);
        else if (job.mode == W_SCALED)
            pairsumdf2_kernel<2, W_SCALED, 0><<<grid, kThreadsDF, 0, st>>>(a);
        else
            pairsumdf2_kernel<2, W_COMPLEX, 0><<<grid, kThreadsDF, 0, st>>>(a);
    } else if (job.R == 1 && job.mode == W_SCALED)
        pairsumdf_kernel<1, W_SCALED><<<grid, kThreadsDF, 0, st>>>(a);
    else if (job.R == 1)
        pairsumdf_kernel<1, W_COMPLEX><<<grid, kThreadsDF, 0, st>>>(a);
    else if (job.mode == W_SCALED)
        pairsumdf_kernel<2, W_SCALED><<<grid, kThreadsDF, 0, st>>>(a);
    else
        pairsumdf_kernel<2, W_COMPLEX><<<grid, kThreadsDF, 0, st>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    // FP32 pipe per pair: 49 shared (d, |d|^2, reciprocal, 1/d) + 48 per right-hand
    // side (two products and two compensated sums per part of z)
    const double per_pair = (comp && job.R == 1) ? 49.0 + 24.0 : 49.0 + 48.0 * job.R;
    prof_end(tok, PK_PAIRDF, (double)job.R * b.N * (b.N - 1.0), st, per_pair * b.N * (b.N - 1.0));
    GNK_TRY_CUDA(launch_reduce(b, job, p.chunks, 2, st, partial));
    count_launches(2);
    return GNK_OK;
}

int pair_blocks_per_sm(int precision) {
    int nb = 1;
    cudaError_t e;
    if (precision == GNK_PREC_FP32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pairsum32_kernel<2, W_SCALED>, kThreads32, 0);
    else if (precision == GNK_PREC_DF32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pairsumdf_kernel<2, W_SCALED>, kThreadsDF, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pairsum64_kernel<2, W_SCALED>, kThreads64, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb < 1 ? 1 : nb;
}

// The part of z = E(q x) an epilogue reads: f_B reads Im(A z) and f_C reads
// Re(A z), which with Im A = 0 are A Im z and A Re z.
int pair_component_needed(const Boundary& b, const PairJob& job) {
    if (!b.A_real || job.R != 1 || job.mode != W_SCALED || job.s != b.q) return 0;
    if (job.epi == EPI_IMINUSN || job.epi == EPI_RESID) return 1;
    if (job.epi == EPI_M) return 2;
    return 0;
}

cudaError_t launch_reduce_public(const Boundary& b, const PairJob& job, int chunks, int ptype,
                                 cudaStream_t st) {
    return launch_reduce(b, job, chunks, ptype, st);
}

int run_pairsum(const Boundary& b, const PairJob& job, int precision, cudaStream_t st) {
    if (precision == GNK_PREC_FMM) return run_fmm(b, job, st);
    PairJob j = job;
    j.comp = pair_component_needed(b, job);
    if (precision == GNK_PREC_FP32) return run_pairsum32(b, j, st);
    if (precision == GNK_PREC_DF32) return run_pairsumdf(b, j, st);
    return run_pairsum64(b, j, st);
}

}  // namespace gnk
