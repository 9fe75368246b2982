// Gradients of the FBIE outputs (mu, h) with respect to the boundary data
// (eta, eta', A) and gamma, by one transposed solve.
//
// With K = 2I + diag(B1) - B and M = D - diag(D1) + Lhat (Eqs. sys, y), the
// forward computation is K mu = -M gamma, h = (M mu - K gamma)/2 (Eq. bh).
// For a loss L(mu, h) with gradients gm = dL/dmu and gh = dL/dh:
//   lambda = K^-T (gm + M^T gh / 2),
//   dL/dgamma = -K^T gh / 2 - M^T lambda,
// and the geometry enters only through the entries of B and D.  Writing
//   B_ij = -(2/n) Im[A_i q_j/(eta_i - eta_j)],  D_ij = -(2/n) Re[A_i q_j/(eta_i - eta_j)],
// q = eta'/A, the four bilinear forms lambda^T K mu, gh^T K gamma, gh^T M mu,
// lambda^T M gamma combine into (2/n) Re Q with the complex pair form
//   Q = sum_{i != j} [a_i - lambda_i nu_j - gh_i rho_j] A_i q_j / (eta_i - eta_j),
//   nu = -i mu - gamma,  rho = (mu - i gamma)/2,  a = lambda nu + gh rho.
// Q is holomorphic in each A_i, q_j and eta_m, so the gradient of (2/n) Re Q
// with respect to the real and imaginary parts of a complex variable z is
// (2/n) conj(dQ/dz).  The derivatives need six Cauchy sums E w and six
// squared sums (F w)_i = sum_{j != i} w_j/(eta_i - eta_j)^2 of the weights
//   w = q, q nu, q rho, A a, A lambda, A gh,
// which one FP64 kernel forms together (both share 1/(eta_i - eta_j)), or, with
// the FMM precisions, three FMM passes (F from the derivative of the local
// expansions plus the near field's 1/d^2 sums).
#include <algorithm>
#include <cstring>

#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {
namespace {

constexpr int kGR = 6;         // weight vectors
constexpr int kGThreads = 128;
constexpr int kGTile = 64;

// partial[chunk][2 kGR][N]: E w_r in slots 0..5, F w_r in slots 6..11
__global__ void __launch_bounds__(kGThreads) gradsum64_kernel(const double2* __restrict__ et,
                                                              const double2* __restrict__ w, int N,
                                                              int tiles_src, int tpc,
                                                              double2* __restrict__ part) {
    __shared__ double2 s_pos[kGTile];
    __shared__ double2 s_w[kGR][kGTile];
    const int i = blockIdx.x * kGThreads + threadIdx.x;
    const double2 p = et[min(i, N - 1)];
    double ex[kGR], ey[kGR], fx[kGR], fy[kGR];
#pragma unroll
    for (int r = 0; r < kGR; ++r) ex[r] = ey[r] = fx[r] = fy[r] = 0.0;
    const int tb = blockIdx.y * tpc;
    const int te = min(tb + tpc, tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * kGTile;
        __syncthreads();
        for (int k = threadIdx.x; k < kGTile; k += kGThreads) {
            const int j = j0 + k;
            s_pos[k] = (j < N) ? et[j] : make_double2(1e150, 1e150);
#pragma unroll
            for (int r = 0; r < kGR; ++r) s_w[r][k] = (j < N) ? w[(size_t)r * N + j] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int k = 0; k < kGTile; ++k) {
            const double2 sp = s_pos[k];
            const double dx = p.x - sp.x, dy = p.y - sp.y;
            double inv = recip_f64(fma(dx, dx, dy * dy));
            inv = (j0 + k == i) ? 0.0 : inv;
            const double ar = dx * inv, ai = dy * inv;  // 1/d = ar - i ai
            const double gr = fma(ar, ar, -ai * ai);    // 1/d^2 = gr - i gi
            const double gi = 2.0 * ar * ai;
#pragma unroll
            for (int r = 0; r < kGR; ++r) {
                const double2 v = s_w[r][k];
                ex[r] = fma(v.x, ar, fma(v.y, ai, ex[r]));
                ey[r] = fma(v.y, ar, fma(-v.x, ai, ey[r]));
                fx[r] = fma(v.x, gr, fma(v.y, gi, fx[r]));
                fy[r] = fma(v.y, gr, fma(-v.x, gi, fy[r]));
            }
        }
    }
    if (i < N) {
#pragma unroll
        for (int r = 0; r < kGR; ++r) {
            part[((size_t)blockIdx.y * 2 * kGR + r) * N + i] = make_double2(ex[r], ey[r]);
            part[((size_t)blockIdx.y * 2 * kGR + kGR + r) * N + i] = make_double2(fx[r], fy[r]);
        }
    }
}

__global__ void gradsum_reduce_kernel(const double2* __restrict__ part, int N, int chunks,
                                      double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int s = 0; s < 2 * kGR; ++s) {
        double sx = 0.0, sy = 0.0;
        for (int c = 0; c < chunks; ++c) {
            const double2 v = part[((size_t)c * 2 * kGR + s) * N + i];
            sx += v.x;
            sy += v.y;
        }
        out[(size_t)s * N + i] = make_double2(sx, sy);
    }
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cd(double2 a, double2 b) {
    const double s = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / s, (a.y * b.x - a.x * b.y) / s);
}
__device__ __forceinline__ double2 rs(double r, double2 a) { return make_double2(r * a.x, r * a.y); }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// weights w_r (see the file comment) and rhs_T = gm + (M^T gh)/2
__global__ void grad_weights_kernel(int N, const double2* __restrict__ q, const double2* __restrict__ A,
                                    const double* __restrict__ mu, const double* __restrict__ gam,
                                    const double* __restrict__ lam, const double* __restrict__ gh,
                                    double2* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 nu = make_double2(-gam[i], -mu[i]);
    const double2 rho = make_double2(0.5 * mu[i], -0.5 * gam[i]);
    const double2 a = make_double2(lam[i] * nu.x + gh[i] * rho.x, lam[i] * nu.y + gh[i] * rho.y);
    const double2 qi = q[i], Ai = A[i];
    w[0 * (size_t)N + i] = qi;
    w[1 * (size_t)N + i] = cm(qi, nu);
    w[2 * (size_t)N + i] = cm(qi, rho);
    w[3 * (size_t)N + i] = cm(Ai, a);
    w[4 * (size_t)N + i] = rs(lam[i], Ai);
    w[5 * (size_t)N + i] = rs(gh[i], Ai);
}

__global__ void axpby_kernel(int N, const double* __restrict__ x, double a, const double* __restrict__ y,
                             double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = x[i] + a * y[i];
}

// Pointwise assembly of the gradients from the sums S (12 x N complex).
__global__ void grad_assemble_kernel(int N, int n, const double2* __restrict__ q,
                                     const double2* __restrict__ A, const double* __restrict__ b1,
                                     const double* __restrict__ d1, const double* __restrict__ mu,
                                     const double* __restrict__ gam, const double* __restrict__ lam,
                                     const double* __restrict__ gh, const double* __restrict__ Llam,
                                     const double2* __restrict__ S, double2* __restrict__ g_et,
                                     double2* __restrict__ g_etp, double2* __restrict__ g_A,
                                     double* __restrict__ g_gam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double s2n = 2.0 / n;
    const double2 nu = make_double2(-gam[i], -mu[i]);
    const double2 rho = make_double2(0.5 * mu[i], -0.5 * gam[i]);
    const double2 a = make_double2(lam[i] * nu.x + gh[i] * rho.x, lam[i] * nu.y + gh[i] * rho.y);
    const double2 qi = q[i], Ai = A[i];
    const double2 E0 = S[0 * (size_t)N + i], E1 = S[1 * (size_t)N + i], E2 = S[2 * (size_t)N + i];
    const double2 E3 = S[3 * (size_t)N + i], E4 = S[4 * (size_t)N + i], E5 = S[5 * (size_t)N + i];
    const double2 F0 = S[6 * (size_t)N + i], F1 = S[7 * (size_t)N + i], F2 = S[8 * (size_t)N + i];
    const double2 F3 = S[9 * (size_t)N + i], F4 = S[10 * (size_t)N + i], F5 = S[11 * (size_t)N + i];
    // dQ/dA_i (explicit), dQ/dq_i, dQ/deta_i
    const double2 T = sub(sub(cm(a, E0), rs(lam[i], E1)), rs(gh[i], E2));
    const double2 U = rs(-1.0, sub(sub(E3, cm(nu, E4)), cm(rho, E5)));
    const double2 W1 = sub(sub(cm(a, F0), rs(lam[i], F1)), rs(gh[i], F2));
    const double2 W2 = sub(sub(F3, cm(nu, F4)), cm(rho, F5));
    const double2 W = sub(cm(qi, W2), cm(Ai, W1));
    const double2 dA = sub(T, cd(cm(U, qi), Ai));  // through q = eta'/A as well
    const double2 detp = cd(U, Ai);
    g_et[i] = make_double2(s2n * W.x, -s2n * W.y);  // (2/n) conj(.)
    g_etp[i] = make_double2(s2n * detp.x, -s2n * detp.y);
    g_A[i] = make_double2(s2n * dA.x, -s2n * dA.y);
    // dL/dgamma = -(K^T gh)/2 - M^T lambda
    const double ktgh = 2.0 * gh[i] + b1[i] * gh[i] - s2n * (qi.x * E5.y + qi.y * E5.x);
    const double mtl = s2n * (qi.x * E4.x - qi.y * E4.y) - d1[i] * lam[i] - Llam[i];
    g_gam[i] = -0.5 * ktgh - mtl;
}

// dL/dh_i + dL/dh_k / n for the nodes i of component k: h_k is the mean of h
// over its component, so its gradient spreads evenly over the n nodes
__global__ void fold_hk_kernel(int N, int n, const double* __restrict__ gh, const double* __restrict__ ghk,
                               double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = gh[i] + ghk[i / n] / n;
}

}  // namespace

int fbie_backward(const Boundary& bc, const double* mu, const double* gam, const double* gm,
                  const double* gh_nodes, const double* ghk, double2* g_et, double2* g_etp, double2* g_A,
                  double* g_gam, const gnk_options& opt, gnk_result* info, cudaStream_t st) {
    Boundary& b = const_cast<Boundary&>(bc);
    const int N = b.N;
    const int nb = (N + 255) / 256;
    // the loss's gradient with respect to the node values of h, with that of
    // the component means h_k folded in
    const double* gh = gh_nodes;
    double* gh_fold = nullptr;
    if (ghk) {
        if (pool_alloc(reinterpret_cast<void**>(&gh_fold), (size_t)N * sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            set_error("gradient workspace allocation failed");
            return GNK_ENOMEM;
        }
        fold_hk_kernel<<<nb, 256, 0, st>>>(N, b.n, gh_nodes, ghk, gh_fold);
        GNK_TRY_CUDA(cudaGetLastError());
        count_launches(1);
        gh = gh_fold;
    }
    const int rc = fbie_backward_nodes(b, mu, gam, gm, gh, g_et, g_etp, g_A, g_gam, opt, info, st);
    if (gh_fold) pool_free(gh_fold, st);
    return rc;
}

int fbie_backward_nodes(Boundary& b, const double* mu, const double* gam, const double* gm,
                        const double* gh, double2* g_et, double2* g_etp, double2* g_A, double* g_gam,
                        const gnk_options& opt, gnk_result* info, cudaStream_t st) {
    const int N = b.N;
    const int nb = (N + 255) / 256;
    // rhs_T = gm + (M^T gh)/2  (FP64-class products)
    const int outer = outer_precision(opt.precision);
    GNK_TRY(op_MT(b, gh, b.r5, outer, st));
    axpby_kernel<<<nb, 256, 0, st>>>(N, gm, 0.5, b.r5, b.r6);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    // lambda = K^-T rhs_T
    double* lam = b.r4;
    const int s = solve(b, OP_KT, b.r6, lam, opt, info, st);
    if (s != GNK_OK && s != GNK_ENOTCONV) return s;
    // weights and the twelve sums
    double2* w = nullptr;
    double2* S = nullptr;
    double2* part = nullptr;
    const int tiles_src = (N + kGTile - 1) / kGTile;
    const int tiles_tgt = (N + kGThreads - 1) / kGThreads;
    int chunks = std::max(1, std::min(tiles_src, (b.sms * 4 + tiles_tgt - 1) / tiles_tgt));
    chunks = std::min(chunks, 16);
    const int tpc = (tiles_src + chunks - 1) / chunks;
    chunks = (tiles_src + tpc - 1) / tpc;
    int st_alloc = GNK_OK;
    const size_t part_bytes = (outer == GNK_PREC_FMM) ? 0 : (size_t)chunks * 2 * kGR * N * sizeof(double2);
    if (pool_alloc(reinterpret_cast<void**>(&w), (size_t)kGR * N * sizeof(double2), st) != cudaSuccess ||
        pool_alloc(reinterpret_cast<void**>(&S), (size_t)2 * kGR * N * sizeof(double2), st) != cudaSuccess ||
        (part_bytes && pool_alloc(reinterpret_cast<void**>(&part), part_bytes, st) != cudaSuccess)) {
        cudaGetLastError();
        set_error("gradient workspace allocation failed");
        st_alloc = GNK_ENOMEM;
    }
    int rc = st_alloc;
    if (rc == GNK_OK) {
        grad_weights_kernel<<<nb, 256, 0, st>>>(N, b.q, b.A, mu, gam, lam, gh, w);
        count_launches(1);
        if (outer == GNK_PREC_FMM) {
            // the six E and six F sums by three FMM passes of two weights each
            for (int r = 0; r < kGR && rc == GNK_OK; r += 2)
                rc = run_fmm_ef(b, w + (size_t)r * N, w + (size_t)(r + 1) * N, S + (size_t)r * N,
                                S + (size_t)(kGR + r) * N, st);
        } else {
            const ProfToken tok = prof_begin(st);
            gradsum64_kernel<<<dim3(tiles_tgt, chunks), kGThreads, 0, st>>>(b.et, w, N, tiles_src, tpc, part);
            prof_end(tok, PK_OTHER, (double)N * (N - 1.0), st);
            gradsum_reduce_kernel<<<nb, 256, 0, st>>>(part, N, chunks, S);
            count_launches(2);
        }
        cudaError_t e = cudaGetLastError();
        if (rc == GNK_OK && e != cudaSuccess) {
            set_error("gradient kernels: %s", cudaGetErrorString(e));
            rc = GNK_ECUDA;
        }
    }
    if (rc == GNK_OK) rc = run_circulant(b, lam, b.r3, st);
    if (rc == GNK_OK) {
        grad_assemble_kernel<<<nb, 256, 0, st>>>(N, b.n, b.q, b.A, b.b1, b.d1, mu, gam, lam, gh, b.r3, S,
                                                 g_et, g_etp, g_A, g_gam);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("gradient assembly: %s", cudaGetErrorString(e));
            rc = GNK_ECUDA;
        }
    }
    pool_free(w, st);
    pool_free(S, st);
    pool_free(part, st);
    if (rc != GNK_OK) return rc;
    return s;
}

}  // namespace gnk
