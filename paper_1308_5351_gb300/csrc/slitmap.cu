// Conformal maps onto slit domains by the FBIE route (Sec. 7, Ex. 3 and Ex. 4):
// theta = pi/2 on a boundary that becomes a circular slit, theta = 0 on one that
// becomes a radial slit, gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)] (arg
// continuous along each boundary), and the solution mu and h of Eqs. (ie), (h)
// give the boundary values A f = gamma + h + i mu of an analytic f:
//   bounded G, A = e^{i(pi/2 - theta)} (eta - alpha):
//     w(z) = e^{-h_0} (z - alpha) exp((z - alpha) f(z))  (onto the unit disk);
//   unbounded G, A = e^{i(pi/2 - theta)} (Eq. A), f(inf) = 0:
//     w(z) = (z - alpha) exp(f(z))                        (w = z + O(1) at infinity);
// with f inside G from the Cauchy formula (Eq. cauchy4).
#include <cmath>

#include "gnk_internal.h"

namespace gnk {
namespace {

constexpr int SM_T = 256;

__device__ __forceinline__ double2 cexp2(double2 z) {
    double s, c;
    sincos(z.y, &s, &c);
    const double e = exp(z.x);
    return make_double2(e * c, e * s);
}

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per boundary component: arg(eta - alpha) unwrapped along the
// component by a block scan of the wrapped increments (in node order), then
// A = e^{i(pi/2 - theta)} (eta - alpha) and gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)].
__global__ void __launch_bounds__(SM_T) slit_data_kernel(const double2* __restrict__ et, int n, double2 alpha,
                                                         const double* __restrict__ theta, int bounded,
                                                         double2* A, double* gam) {
    __shared__ double s[SM_T];
    __shared__ double carry, phi0;
    const int k = blockIdx.x;
    const double2* e = et + (size_t)k * n;
    const double th = 0.5 * M_PI - theta[k];
    double sr, cr;
    sincos(th, &sr, &cr);
    if (threadIdx.x == 0) {
        carry = 0.0;
        phi0 = atan2(e[0].y - alpha.y, e[0].x - alpha.x);
    }
    __syncthreads();
    for (int base = 0; base < n; base += SM_T) {
        const int p = base + threadIdx.x;
        double inc = 0.0;
        double2 d = make_double2(0.0, 0.0);
        if (p < n) {
            d = make_double2(e[p].x - alpha.x, e[p].y - alpha.y);
            if (p > 0) {
                const double a1 = atan2(d.y, d.x);
                const double a0 = atan2(e[p - 1].y - alpha.y, e[p - 1].x - alpha.x);
                inc = a1 - a0;
                if (inc > M_PI) inc -= 2.0 * M_PI;
                if (inc <= -M_PI) inc += 2.0 * M_PI;
            }
        }
        s[threadIdx.x] = inc;
        __syncthreads();
        for (int off = 1; off < SM_T; off <<= 1) {  // inclusive scan
            const double v = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0.0;
            __syncthreads();
            s[threadIdx.x] += v;
            __syncthreads();
        }
        if (p < n) {
            const double arg = phi0 + carry + s[threadIdx.x];
            const double lr = 0.5 * log(d.x * d.x + d.y * d.y);
            const size_t i = (size_t)k * n + p;
            A[i] = bounded ? make_double2(cr * d.x - sr * d.y, cr * d.y + sr * d.x) : make_double2(cr, sr);
            gam[i] = -(cr * lr - sr * arg);
        }
        __syncthreads();
        if (threadIdx.x == SM_T - 1) carry += s[SM_T - 1];
        __syncthreads();
    }
}

// f at the nodes: (gamma + h + i mu) / A
__global__ void slit_f_kernel(const double2* __restrict__ A, const double* __restrict__ gam,
                              const double* __restrict__ mu, const double* __restrict__ h, int N, double2* f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 a = A[i];
    const double re = gam[i] + h[i], im = mu[i];
    const double aa = a.x * a.x + a.y * a.y;
    f[i] = make_double2((re * a.x + im * a.y) / aa, (im * a.x - re * a.y) / aa);
}

// w at points z with values f: bounded G, e^{-h_0} (z - alpha) exp((z - alpha) f)
// (h_0 = hk[0]); unbounded G, (z - alpha) exp(f)
__global__ void slit_w_kernel(const double2* __restrict__ z, const double2* __restrict__ f, int M, double2 alpha,
                              const double* __restrict__ hk, int bounded, double2* w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double2 d = make_double2(z[i].x - alpha.x, z[i].y - alpha.y);
    if (bounded) {
        const double c = exp(-hk[0]);
        const double2 v = cmul2(d, cexp2(cmul2(d, f[i])));
        w[i] = make_double2(c * v.x, c * v.y);
    } else {
        w[i] = cmul2(d, cexp2(f[i]));
    }
}

}  // namespace

int slit_data(int m1, int n, const double2* et, double2 alpha, const double* theta, int bounded, double2* A,
              double* gam, cudaStream_t st) {
    slit_data_kernel<<<m1, SM_T, 0, st>>>(et, n, alpha, theta, bounded ? 1 : 0, A, gam);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

int slit_nodes_f(const Boundary& b, const double* gam, const double* mu, const double* h, double2* f,
                 cudaStream_t st) {
    slit_f_kernel<<<(b.N + 255) / 256, 256, 0, st>>>(b.A, gam, mu, h, b.N, f);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

int slit_w(const double2* z, const double2* f, int M, double2 alpha, const double* hk, int bounded, double2* w,
           cudaStream_t st) {
    slit_w_kernel<<<(M + 255) / 256, 256, 0, st>>>(z, f, M, alpha, hk, bounded ? 1 : 0, w);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

}  // namespace gnk
