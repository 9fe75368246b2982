// Values of an analytic function at points of G from its boundary values:
// the Cauchy integral formula with singularity subtraction (Sec. 5, Eqs.
// cauchy4, cauchy6, listing of FCAU):
//   bounded G:   f(z) = F[f eta'] / F[eta'],
//   unbounded G: f(z) = (f_inf - F[f eta'] / (n i)) / (1 - F[eta'] / (n i)),
// with (F x)(z) = sum_j x_j / (z - eta_j) over all boundary nodes.  The two sums
// share the reciprocal of z - eta_j (one pair kernel with two weight vectors);
// targets are arbitrary points, so no term is excluded.
#include <algorithm>

#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {
namespace {

constexpr int CE_NT64 = 128, CE_T64 = 2, CE_S64 = 128;
constexpr int CE_NTDF = 256;
static_assert(CE_NTDF == kSrcTile32, "one source node per thread in the tile load");

struct CEArgs {
    const double2* et;
    const double2* etp;
    const double2* f;
    const double2* z;
    const double2* ref64;
    const float4* offdf;
    int N, M, tiles_src, tpc;
    void* partial;  // [chunk][2][M]
};

__global__ void __launch_bounds__(CE_NT64) ceval64_kernel(CEArgs a) {
    __shared__ double2 s_pos[CE_S64];
    __shared__ double2 s_w[2][CE_S64];
    const int t0 = blockIdx.x * (CE_NT64 * CE_T64);
    double px[CE_T64], py[CE_T64], ax[CE_T64][2], ay[CE_T64][2];
    int idx[CE_T64];
#pragma unroll
    for (int t = 0; t < CE_T64; ++t) {
        idx[t] = t0 + t * CE_NT64 + threadIdx.x;
        const double2 p = a.z[min(idx[t], a.M - 1)];
        px[t] = p.x;
        py[t] = p.y;
        ax[t][0] = ay[t][0] = ax[t][1] = ay[t][1] = 0.0;
    }
    const int tb = blockIdx.y * a.tpc, te = min(tb + a.tpc, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * CE_S64;
        __syncthreads();
        for (int k = threadIdx.x; k < CE_S64; k += CE_NT64) {
            const int j = j0 + k;
            if (j < a.N) {
                const double2 e = a.etp[j], fv = a.f[j];
                s_pos[k] = a.et[j];
                s_w[0][k] = make_double2(fv.x * e.x - fv.y * e.y, fv.x * e.y + fv.y * e.x);
                s_w[1][k] = e;
            } else {
                s_pos[k] = make_double2(1e150, 1e150);
                s_w[0][k] = s_w[1][k] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
        for (int k = 0; k < CE_S64; ++k) {
            const double2 sp = s_pos[k];
#pragma unroll
            for (int t = 0; t < CE_T64; ++t) {
                const double dx = px[t] - sp.x, dy = py[t] - sp.y;
                const double inv = recip_f64(fma(dx, dx, dy * dy));
                const double ar = dx * inv, ai = dy * inv;  // 1/(z - eta) = ar - i ai
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const double2 w = s_w[r][k];
                    ax[t][r] = fma(w.x, ar, fma(w.y, ai, ax[t][r]));
                    ay[t][r] = fma(w.y, ar, fma(-w.x, ai, ay[t][r]));
                }
            }
        }
    }
    double2* part = static_cast<double2*>(a.partial);
#pragma unroll
    for (int t = 0; t < CE_T64; ++t)
        if (idx[t] < a.M)
#pragma unroll
            for (int r = 0; r < 2; ++r)
                part[((size_t)blockIdx.y * 2 + r) * a.M + idx[t]] = make_double2(ax[t][r], ay[t][r]);
}

// double-float: source offsets from the handle's FP64 tile references
__global__ void __launch_bounds__(CE_NTDF) cevaldf_kernel(CEArgs a) {
    constexpr int S = kSrcTile32;
    __shared__ float4 s_off[S];
    __shared__ float4 s_w[2][2][S];
    const int i = blockIdx.x * CE_NTDF + threadIdx.x;
    const double2 p = a.z[min(i, a.M - 1)];
    df are[2], aim[2];
    are[0] = are[1] = aim[0] = aim[1] = df{0.f, 0.f};
    const int tb = blockIdx.y * a.tpc, te = min(tb + a.tpc, a.tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * S;
        const double2 ref = a.ref64[tile];
        const df ox = df_split(p.x - ref.x), oy = df_split(p.y - ref.y);
        __syncthreads();
        {
            const int k = threadIdx.x, j = j0 + k;
            if (j < a.N) {
                s_off[k] = a.offdf[j];
                const double2 e = a.etp[j], fv = a.f[j];
                const double2 w0 = make_double2(fv.x * e.x - fv.y * e.y, fv.x * e.y + fv.y * e.x);
                const df w0x = df_split(w0.x), w0y = df_split(w0.y), w1x = df_split(e.x), w1y = df_split(e.y);
                s_w[0][0][k] = make_float4(w0x.h, w0x.l, 0.f, 0.f);
                s_w[0][1][k] = make_float4(w0y.h, w0y.l, 0.f, 0.f);
                s_w[1][0][k] = make_float4(w1x.h, w1x.l, 0.f, 0.f);
                s_w[1][1][k] = make_float4(w1y.h, w1y.l, 0.f, 0.f);
            } else {
                s_off[k] = make_float4(1e18f, 1e18f, 0.f, 0.f);
                s_w[0][0][k] = s_w[0][1][k] = s_w[1][0][k] = s_w[1][1][k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        for (int k = 0; k < S; ++k) {
            const float4 so = s_off[k];
            const df dx = df_sub(ox.h, ox.l, so.x, so.z);
            const df dy = df_sub(oy.h, oy.l, so.y, so.w);
            const float px = __fmul_rn(dx.h, dx.h);
            float ex = fmaf(dx.h, dx.h, -px);
            ex = fmaf(dx.h, dx.l + dx.l, ex);
            const float py = __fmul_rn(dy.h, dy.h);
            float ey = fmaf(dy.h, dy.h, -py);
            ey = fmaf(dy.h, dy.l + dy.l, ey);
            float rh, re;
            two_sum(px, py, rh, re);
            const float rl = __fadd_rn(__fadd_rn(ex, ey), re);
            const float y = recip_f32(rh);
            float e = fmaf(-rh, y, 1.0f);
            e = fmaf(-rl, y, e);
            const df inv{y, __fmul_rn(y, e)};
            const df ar = df_mul(dx, inv), ai = df_mul(dy, inv);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float4 a0 = s_w[r][0][k], a1 = s_w[r][1][k];
                const df wx{a0.x, a0.y}, wy{a1.x, a1.y};
                df_acc(are[r], df_mul(wx, ar));
                df_acc(are[r], df_mul(wy, ai));
                df_acc(aim[r], df_mul(wy, ar));
                const df q = df_mul(wx, ai);
                df_acc(aim[r], df{-q.h, -q.l});
            }
        }
    }
    if (i < a.M) {
        float4* part = static_cast<float4*>(a.partial);
        for (int r = 0; r < 2; ++r)
            part[((size_t)blockIdx.y * 2 + r) * a.M + i] = make_float4(are[r].h, are[r].l, aim[r].h, aim[r].l);
    }
}

__global__ void ceval_ratio_kernel(const void* partial, int df32, int M, int chunks, int bounded, int n,
                                   double2 finf, double2* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double s[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < chunks; ++c) {
            const size_t k = ((size_t)c * 2 + r) * M + i;
            if (df32) {
                const float4 v = static_cast<const float4*>(partial)[k];
                s[r][0] += (double)v.x + (double)v.y;
                s[r][1] += (double)v.z + (double)v.w;
            } else {
                const double2 v = static_cast<const double2*>(partial)[k];
                s[r][0] += v.x;
                s[r][1] += v.y;
            }
        }
    double2 num = make_double2(s[0][0], s[0][1]), den = make_double2(s[1][0], s[1][1]);
    if (!bounded) {
        // x / (n i) = -i x / n:  num = f_inf - F[f eta']/(n i),  den = 1 - F[eta']/(n i)
        num = make_double2(finf.x - num.y / n, finf.y + num.x / n);
        den = make_double2(1.0 - den.y / n, den.x / n);
    }
    const double dd = den.x * den.x + den.y * den.y;
    out[i] = make_double2((num.x * den.x + num.y * den.y) / dd, (num.y * den.x - num.x * den.y) / dd);
}

}  // namespace

int cauchy_eval(const Boundary& b, int M, const double2* z, const double2* f, double2 finf, double2* out,
                int precision, cudaStream_t st) {
    const bool dfp = precision == GNK_PREC_DF32;
    const int tpb = dfp ? CE_NTDF : CE_NT64 * CE_T64;
    const int S = dfp ? kSrcTile32 : CE_S64;
    const int tiles_tgt = (M + tpb - 1) / tpb;
    const int tiles_src = (b.N + S - 1) / S;
    int chunks = std::max(1, std::min(tiles_src, (2 * b.sms * 4 + tiles_tgt - 1) / tiles_tgt));
    chunks = std::min(chunks, 32);
    const int tpc = (tiles_src + chunks - 1) / chunks;
    chunks = (tiles_src + tpc - 1) / tpc;
    void* part = nullptr;
    const size_t bytes = (size_t)chunks * 2 * M * (dfp ? sizeof(float4) : sizeof(double2));
    if (pool_alloc(&part, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("gnk_cauchy_eval: workspace allocation of %zu bytes failed", bytes);
        return GNK_ENOMEM;
    }
    CEArgs a;
    a.et = b.et;
    a.etp = b.etp;
    a.f = f;
    a.z = z;
    a.ref64 = b.ref64;
    a.offdf = b.offdf;
    a.N = b.N;
    a.M = M;
    a.tiles_src = tiles_src;
    a.tpc = tpc;
    a.partial = part;
    const ProfToken tok = prof_begin(st);
    if (dfp)
        cevaldf_kernel<<<dim3(tiles_tgt, chunks), CE_NTDF, 0, st>>>(a);
    else
        ceval64_kernel<<<dim3(tiles_tgt, chunks), CE_NT64, 0, st>>>(a);
    prof_end(tok, PK_OTHER, 2.0 * M * b.N, st);
    ceval_ratio_kernel<<<(M + 255) / 256, 256, 0, st>>>(part, dfp ? 1 : 0, M, chunks, b.bounded, b.n, finf, out);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pool_free(part, st);
    if (e != cudaSuccess) {
        set_error("gnk_cauchy_eval: %s", cudaGetErrorString(e));
        return GNK_ECUDA;
    }
    return GNK_OK;
}

}  // namespace gnk
