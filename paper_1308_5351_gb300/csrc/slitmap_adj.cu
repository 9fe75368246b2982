// Conformal maps onto slit domains by solves of the adjoint equation only
// (Sec. 7, Ex. 3 and Ex. 4: the comparison route of the FBIEad function), for
// theta = pi/2 (circular slit) or 0 (radial slit) per boundary, A of Eq. (A)
// and A~ = eta'/A (Eq. A*), the handle's q.  Writing the map as
// w = (z - alpha) exp(omega), the kernel identities of the generalized Neumann
// kernel formed with A~ (which is -N*, Eq. Nt-N*) give:
//   * the derivative of the boundary correspondence, psi = th' on a circular
//     and -(log rho)' on a radial boundary, solves (I + N* + J) psi = e_0 for
//     bounded G and (I + N* + J) psi = 2 Im[A~/(eta - alpha)] for unbounded G;
//   * its antiderivative S along each boundary (zero at t = 0), by the FFT of
//     the trigonometric interpolant (a direct circulant product when n is not
//     a power of two up to 4096);
//   * the solutions psi_j of (I + N* + J) psi_j = e_j, j = 0..m, and
//     T_j = (1/n) sum_i c_i omega^_i psi_j,i (c = i circular, -1 radial,
//     omega^ = omega without its per-boundary constants), from Cauchy's
//     theorem: rho = log w'(alpha) = Im T_0 (bounded G; 0 for unbounded G),
//     circular k: log R_k = rho - Im T_k, th_k(0) = Re T_k;
//     radial k:   log rho_k(0) = rho + Re T_k, phi_k = Im T_k;
//   * w = R_k exp(i (th_k(0) + S)) or rho_k(0) exp(-S) exp(i phi_k) per node.
// Bounded G needs m + 1 solves (psi_0 is both the derivative and the first
// parameter solution), unbounded G m + 2.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fft.cuh"
#include "gnk_internal.h"

namespace gnk {
namespace {

constexpr int AT = 256;      // threads of the elementwise and per-boundary kernels
constexpr int DOT_T = 512;   // threads of the one-block dot product

// Right-hand sides of Eq. (ie*): e_j for j >= 0; for j < 0 the derivative
// solve of unbounded G, 2 Im[q/(eta - alpha)] with q = eta'/A.
__global__ void adj_rhs_kernel(int N, int n, int j, const double2* __restrict__ q,
                               const double2* __restrict__ et, double2 alpha, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (j >= 0) {
        out[i] = (i / n == j) ? 1.0 : 0.0;
        return;
    }
    const double dx = et[i].x - alpha.x, dy = et[i].y - alpha.y;
    const double2 v = q[i];
    // Im(v / d) = Im(v conj(d)) / |d|^2
    out[i] = 2.0 * (v.y * dx - v.x * dy) / (dx * dx + dy * dy);
}

// A' = e^{i(pi/2 - theta)} eta' (bounded G) or 0 (unbounded G): the derivative
// of the A of the slit map, read by the diagonal of Eq. (sys*).
__global__ void slit_dA_kernel(int N, int n, const double2* __restrict__ etp, const double* __restrict__ theta,
                               int bounded, double2* __restrict__ Ap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (!bounded) {
        Ap[i] = make_double2(0.0, 0.0);
        return;
    }
    double sr, cr;
    sincos(0.5 * M_PI - theta[i / n], &sr, &cr);
    const double2 e = etp[i];
    Ap[i] = make_double2(cr * e.x - sr * e.y, cr * e.y + sr * e.x);
}

// Periodic antiderivative by the FFT, one block per pair of boundaries packed
// as the real and imaginary parts of one signal: the DFT coefficient of
// frequency k (k - n above n/2) is divided by i k, k = 0 and k = n/2 are
// dropped, and S_p = mean t_p + y_p - y_0 (t_p = 2 pi p/n).  The multiplier
// keeps real signals real, so the two boundaries separate after the inverse.
__global__ void antideriv_fft_kernel(const double* __restrict__ x, double* __restrict__ S, int n, int m1,
                                     const double2* __restrict__ tw) {
    extern __shared__ double2 sm[];
    double2* X = sm;
    double2* Y = sm + n;
    const int ca = 2 * blockIdx.x;
    const int cb = ca + 1;
    const bool has_b = cb < m1;
    for (int p = threadIdx.x; p < n; p += blockDim.x)
        X[p] = make_double2(x[(size_t)ca * n + p], has_b ? x[(size_t)cb * n + p] : 0.0);
    __syncthreads();
    double2* F = stockham(X, Y, n, tw, false);
    double2* G = (F == X) ? Y : X;
    const double2 f0 = F[0];  // the two boundaries' sums
    __syncthreads();
    const int half = n >> 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double2 v = F[k];
        if (k == 0 || k == half) {
            F[k] = make_double2(0.0, 0.0);
        } else {
            const double ks = (k < half) ? (double)k : (double)(k - n);
            F[k] = make_double2(v.y / ks, -v.x / ks);  // v / (i ks)
        }
    }
    __syncthreads();
    double2* Z = stockham(F, G, n, tw, true);
    const double2 z0 = Z[0];
    const double inv_n = 1.0 / n;
    const double h = 2.0 * M_PI / n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const double t = h * p;
        S[(size_t)ca * n + p] = f0.x * inv_n * t + (Z[p].x - z0.x) * inv_n;
        if (has_b) S[(size_t)cb * n + p] = f0.y * inv_n * t + (Z[p].y - z0.y) * inv_n;
    }
}

// First column of the same antiderivative as a circulant (any even n):
// K_d = (2/n) sum_{k=1}^{n/2-1} sin(2 pi k d/n)/k, with the argument reduced
// exactly as (k d mod n)/n.
__global__ void antideriv_col_kernel(int n, double* __restrict__ col) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n) return;
    double s = 0.0;
    for (int k = 1; k < n / 2; ++k) {
        const long long r = ((long long)k * d) % n;
        s += sinpi(2.0 * (double)r / n) / k;
    }
    col[d] = 2.0 * s / n;
}

// S_p = sum_q (K_{(p-q) mod n} - K_{(-q) mod n} + t_p/n) x_q: the circulant
// product minus its value at p = 0 plus the mean times t_p.  One block per
// (boundary, tile of AT targets) in a one-dimensional grid of m1 * tiles
// blocks; the boundary's values pass through shared memory in tiles.
__global__ void __launch_bounds__(AT) antideriv_direct_kernel(const double* __restrict__ x, double* __restrict__ S,
                                                              int n, int tiles, const double* __restrict__ col) {
    __shared__ double xs[AT];
    const int comp = blockIdx.x / tiles;
    const int p = (blockIdx.x - comp * tiles) * AT + threadIdx.x;
    const double* xc = x + (size_t)comp * n;
    double acc = 0.0, sum = 0.0;
    for (int q0 = 0; q0 < n; q0 += AT) {
        const int q = q0 + threadIdx.x;
        xs[threadIdx.x] = (q < n) ? xc[q] : 0.0;
        __syncthreads();
        const int cnt = min(AT, n - q0);
        if (p < n) {
            for (int r = 0; r < cnt; ++r) {
                const int qq = q0 + r;
                int d = p - qq;
                d += (d < 0) ? n : 0;
                const int d0 = (qq == 0) ? 0 : n - qq;
                acc = fma(col[d] - col[d0], xs[r], acc);
                sum += xs[r];
            }
        }
        __syncthreads();
    }
    if (p < n) S[(size_t)comp * n + p] = acc + sum * (2.0 * M_PI * p / n) / n;
}

// One block per boundary: log|eta - alpha| and arg(eta - alpha) unwrapped
// along the boundary (a block scan of the wrapped increments in node order),
// then omega^ = -log|eta - alpha| + i (S - arg) on a circular boundary and
// -S - log|eta - alpha| - i arg on a radial one.
__global__ void __launch_bounds__(AT) adj_omega_kernel(const double2* __restrict__ et, int n, double2 alpha,
                                                       const double* __restrict__ theta,
                                                       const double* __restrict__ S, double2* __restrict__ om) {
    __shared__ double s[AT];
    __shared__ double carry, phi0;
    const int k = blockIdx.x;
    const double2* e = et + (size_t)k * n;
    const bool circ = theta[k] != 0.0;
    if (threadIdx.x == 0) {
        carry = 0.0;
        phi0 = atan2(e[0].y - alpha.y, e[0].x - alpha.x);
    }
    __syncthreads();
    for (int base = 0; base < n; base += AT) {
        const int p = base + threadIdx.x;
        double inc = 0.0;
        double2 d = make_double2(1.0, 0.0);
        if (p < n) {
            d = make_double2(e[p].x - alpha.x, e[p].y - alpha.y);
            if (p > 0) {
                inc = atan2(d.y, d.x) - atan2(e[p - 1].y - alpha.y, e[p - 1].x - alpha.x);
                if (inc > M_PI) inc -= 2.0 * M_PI;
                if (inc <= -M_PI) inc += 2.0 * M_PI;
            }
        }
        s[threadIdx.x] = inc;
        __syncthreads();
        for (int off = 1; off < AT; off <<= 1) {  // inclusive scan
            const double v = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0.0;
            __syncthreads();
            s[threadIdx.x] += v;
            __syncthreads();
        }
        if (p < n) {
            const double arg = phi0 + carry + s[threadIdx.x];
            const double lr = 0.5 * log(d.x * d.x + d.y * d.y);
            const size_t i = (size_t)k * n + p;
            const double Si = S[i];
            om[i] = circ ? make_double2(-lr, Si - arg) : make_double2(-Si - lr, -arg);
        }
        __syncthreads();
        if (threadIdx.x == AT - 1) carry += s[AT - 1];
        __syncthreads();
    }
}

// T = (1/n) sum_i c_i omega^_i psi_i (c = i circular, -1 radial) in one block
// with a fixed-order tree sum.
__global__ void __launch_bounds__(DOT_T) adj_dot_kernel(const double2* __restrict__ om,
                                                        const double* __restrict__ theta,
                                                        const double* __restrict__ psi, int N, int n,
                                                        double2* __restrict__ T) {
    __shared__ double rx[DOT_T], ry[DOT_T];
    double sx = 0.0, sy = 0.0;
    for (int i = threadIdx.x; i < N; i += DOT_T) {
        const double2 o = om[i];
        const double p = psi[i];
        if (theta[i / n] != 0.0) {  // i o p
            sx -= o.y * p;
            sy += o.x * p;
        } else {                    // -o p
            sx -= o.x * p;
            sy -= o.y * p;
        }
    }
    rx[threadIdx.x] = sx;
    ry[threadIdx.x] = sy;
    __syncthreads();
    for (int w = DOT_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rx[threadIdx.x] += rx[threadIdx.x + w];
            ry[threadIdx.x] += ry[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *T = make_double2(rx[0] / n, ry[0] / n);
}

// w, omega = omega^ + the boundary's constant, and the parameters (R_k or
// phi_k per boundary, then w'(alpha) for bounded G or 1).
__global__ void adj_assemble_kernel(const double2* __restrict__ om, const double* __restrict__ S,
                                    const double2* __restrict__ T, const double* __restrict__ theta, int N,
                                    int n, int m1, int bounded, double2* __restrict__ w,
                                    double2* __restrict__ omega, double* __restrict__ params) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int k = i / n;
    const double rho = bounded ? T[0].y : 0.0;
    const double2 t = T[k];
    double2 kap, wi;
    double par;
    if (theta[k] != 0.0) {
        const double logR = rho - t.y;  // 0 on the outer boundary of bounded G
        const double R = exp(logR);
        double sn, cs;
        sincos(t.x + S[i], &sn, &cs);
        kap = make_double2(logR, t.x);
        wi = make_double2(R * cs, R * sn);
        par = R;
    } else {
        const double ck = rho + t.x;
        const double mod = exp(ck - S[i]);
        double sn, cs;
        sincos(t.y, &sn, &cs);
        kap = make_double2(ck, t.y);
        wi = make_double2(mod * cs, mod * sn);
        par = t.y;
    }
    w[i] = wi;
    if (omega) omega[i] = make_double2(om[i].x + kap.x, om[i].y + kap.y);
    if (params) {
        if (i == k * n) params[k] = par;
        if (i == 0) params[m1] = bounded ? exp(rho) : 1.0;
    }
}

// Stream-ordered device workspace of one call, returned to the pool on exit.
struct Scratch {
    void* p = nullptr;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        if (p) pool_free(p, st);
    }
};

int launch_check(int launches) {
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(launches);
    return GNK_OK;
}

}  // namespace

int slit_dA(int m1, int n, const double2* etp, const double* theta, int bounded, double2* Ap, cudaStream_t st) {
    const int N = m1 * n;
    slit_dA_kernel<<<(N + AT - 1) / AT, AT, 0, st>>>(N, n, etp, theta, bounded ? 1 : 0, Ap);
    return launch_check(1);
}

int slit_map_adjoint(const Boundary& b, double2 alpha, const double* theta, const gnk_options& opt, double2* w,
                     double2* omega, double* psi_out, double* params, gnk_result* info, cudaStream_t st) {
    const int N = b.N, n = b.n, m1 = b.m1;
    const bool fft = b.fft_pow2 != 0;
    // psi_j, the right-hand side, psi, S (N each), omega^ (2N), T (2 m1), K (n)
    const size_t nd = 4 * (size_t)N + 2 * (size_t)N + 2 * (size_t)m1 + (fft ? 0 : (size_t)n);
    Scratch ws(st);
    if (pool_alloc(&ws.p, nd * sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        set_error("gnk_slit_map_adjoint: device allocation of %zu bytes failed", nd * sizeof(double));
        return GNK_ENOMEM;
    }
    double* psij = static_cast<double*>(ws.p);
    double* rhs = psij + N;
    double* psi = rhs + N;
    double* S = psi + N;
    double2* om = reinterpret_cast<double2*>(S + N);
    double2* T = om + N;
    double* col = reinterpret_cast<double*>(T + m1);

    gnk_result agg;
    std::memset(&agg, 0, sizeof(agg));
    int worst = GNK_OK;
    const int eb = (N + AT - 1) / AT;
    // one GMRES solve of Eq. (sys*); the call's result sums the solves' counts
    // and keeps the largest final residual; a solve that stops at maxit makes
    // the call's status GNK_ENOTCONV, any other failure ends the call
    auto run_solve = [&](const double* r, double* x) -> int {
        gnk_result one;
        std::memset(&one, 0, sizeof(one));
        const int s = solve(b, OP_ADJ, r, x, opt, &one, st);
        agg.iterations += one.iterations;
        agg.cycles += one.cycles;
        agg.refinements += one.refinements;
        agg.matvecs_fp64 += one.matvecs_fp64;
        agg.matvecs_fp32 += one.matvecs_fp32;
        agg.relres = std::max(agg.relres, one.relres);
        if (s == GNK_ENOTCONV) worst = GNK_ENOTCONV;
        if (s != GNK_OK && s != GNK_ENOTCONV && info) {
            agg.status = s;
            *info = agg;
        }
        return s == GNK_ENOTCONV ? GNK_OK : s;
    };

    // derivative of the boundary correspondence
    adj_rhs_kernel<<<eb, AT, 0, st>>>(N, n, b.bounded ? 0 : -1, b.q, b.et, alpha, rhs);
    GNK_TRY(launch_check(1));
    GNK_TRY(run_solve(rhs, psi));
    // its antiderivative along each boundary
    if (fft) {
        const int threads = std::min(512, std::max(32, n / 2));
        const size_t smem = 2 * (size_t)n * sizeof(double2);
        if (smem > 48 * 1024)
            GNK_TRY_CUDA(cudaFuncSetAttribute(antideriv_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        antideriv_fft_kernel<<<(m1 + 1) / 2, threads, smem, st>>>(psi, S, n, m1, b.twiddle);
        GNK_TRY(launch_check(1));
    } else {
        antideriv_col_kernel<<<(n + AT - 1) / AT, AT, 0, st>>>(n, col);
        const int tiles = (n + AT - 1) / AT;
        antideriv_direct_kernel<<<m1 * tiles, AT, 0, st>>>(psi, S, n, tiles, col);
        GNK_TRY(launch_check(2));
    }
    adj_omega_kernel<<<m1, AT, 0, st>>>(b.et, n, alpha, theta, S, om);
    GNK_TRY(launch_check(1));
    // the parameters: one solve and one dot product per boundary
    for (int j = 0; j < m1; ++j) {
        const double* pj = psi;
        if (!(b.bounded && j == 0)) {
            adj_rhs_kernel<<<eb, AT, 0, st>>>(N, n, j, b.q, b.et, alpha, rhs);
            GNK_TRY(launch_check(1));
            GNK_TRY(run_solve(rhs, psij));
            pj = psij;
        }
        adj_dot_kernel<<<1, DOT_T, 0, st>>>(om, theta, pj, N, n, T + j);
        GNK_TRY(launch_check(1));
    }
    adj_assemble_kernel<<<eb, AT, 0, st>>>(om, S, T, theta, N, n, m1, b.bounded, w, omega, params);
    GNK_TRY(launch_check(1));
    if (psi_out) GNK_TRY_CUDA(cudaMemcpyAsync(psi_out, psi, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    agg.status = worst;
    if (info) *info = agg;
    return worst;
}

}  // namespace gnk
