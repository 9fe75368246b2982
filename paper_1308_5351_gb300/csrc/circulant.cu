// Block-circulant part Lhat x (Sec. 3.3, Eqs. hL-bt, L-bs), per-component
// means (Phat x, Sec. 4.4), and the one-time geometry preparation of a
// boundary handle.
//
// Lhat x: each component's n values are multiplied by the circulant L whose
// first column is b_1 = 0, b_i = (-1)^(i-1) (1/n) cot((i-1) pi / n).  Its
// eigenvalues (the DFT of b) are i 2k/n for 0 <= k < n/2, 0 for k = n/2 and
// i 2(k-n)/n for k > n/2, so L x = IFFT(lambda .* FFT(x)).  Because L is real,
// two components are packed as the real and imaginary parts of one complex
// signal and transformed together.  One thread block per component pair runs
// a radix-2 Stockham FFT in shared memory (no bit reversal), scales by
// lambda, and runs the inverse FFT.  For n not a power of two the product is
// formed directly from the first column b.
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "gnk_internal.h"

namespace gnk {
namespace {

__global__ void circulant_fft_kernel(const double* __restrict__ x, double* __restrict__ y,
                                     int n, int m1, const double2* __restrict__ tw) {
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
    const int half = n >> 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        // lambda_k = i s_k with s_k = 2k/n below n/2, 0 at n/2, 2(k-n)/n above
        const double s = (k < half) ? (2.0 * k) / n : (k == half ? 0.0 : (2.0 * (k - n)) / n);
        const double2 v = F[k];
        F[k] = make_double2(-s * v.y, s * v.x);
    }
    __syncthreads();
    double2* Z = stockham(F, G, n, tw, true);
    const double inv_n = 1.0 / n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const double2 v = Z[p];
        y[(size_t)ca * n + p] = v.x * inv_n;
        if (has_b) y[(size_t)cb * n + p] = v.y * inv_n;
    }
}

// Direct circulant product y_p = sum_q b_{(p - q) mod n} x_q (any even n).
__global__ void circulant_direct_kernel(const double* __restrict__ x, double* __restrict__ y,
                                        int n, const double* __restrict__ bcol) {
    extern __shared__ double xs[];
    const int comp = blockIdx.y;
    for (int q = threadIdx.x; q < n; q += blockDim.x) xs[q] = x[(size_t)comp * n + q];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double acc = 0.0;
    for (int q = 0; q < n; ++q) {
        int d = p - q;
        d += (d < 0) ? n : 0;
        acc = fma(bcol[d], xs[q], acc);
    }
    y[(size_t)comp * n + p] = acc;
}

// Mean of each component (one block per component, fixed-order tree sum).
__global__ void component_means_kernel(const double* __restrict__ x, double* __restrict__ means,
                                       int n) {
    __shared__ double red[256];
    const int comp = blockIdx.x;
    double s = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) s += x[(size_t)comp * n + p];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) means[comp] = red[0] / n;
}

// ---- geometry preparation
struct PrepArgs {
    int N, n, S, has_adj;
    const double2* et;
    const double2* etp;
    const double2* A;
    const double* etpp;  // interleaved complex, may be null
    const double* Ap;    // interleaved complex, may be null
    double2* q;
    float4* et32;
    float2* off32;
    float4* ref32;
    float2* q32;
    float2* A32;
    double2* ref64;
    float4* offdf;
    double* ediag;       // (2/n) Im(eta''/eta' - A'/A), corner limit 0; plain form: 1 + Nd
    int plain;           // plain form: also writes b1 = -1 - Nd and d1 = -M1d
    double* b1;
    double* d1;
    double* ones;        // nullable: filled with 1
    int* flag;           // bit 1: non-finite input, bit 2: A == 0, bit 4: Im A != 0
};

__device__ __forceinline__ float4 split_hilo(double2 z) {
    const float hx = (float)z.x, hy = (float)z.y;
    return make_float4(hx, hy, (float)(z.x - (double)hx), (float)(z.y - (double)hy));
}

__device__ __forceinline__ bool finite2(double2 z) { return isfinite(z.x) && isfinite(z.y); }

__global__ void prepare_geometry_kernel(PrepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const double2 et = a.et[i], etp = a.etp[i], A = a.A[i];
    int bad = 0;
    if (!finite2(et) || !finite2(etp) || !finite2(A)) bad |= 1;
    const double aa = A.x * A.x + A.y * A.y;
    if (aa == 0.0) bad |= 2;
    if (A.y != 0.0) bad |= 4;  // not an error: A is not real-valued
    // q = eta'/A
    const double2 q = make_double2((etp.x * A.x + etp.y * A.y) / aa, (etp.y * A.x - etp.x * A.y) / aa);
    a.q[i] = q;
    a.q32[i] = make_float2((float)q.x, (float)q.y);
    a.A32[i] = make_float2((float)A.x, (float)A.y);
    a.et32[i] = split_hilo(et);
    if (a.ones) a.ones[i] = 1.0;
    const int tile = i / a.S;
    const int j0 = tile * a.S;
    const int cnt = min(a.S, a.N - j0);
    const int r = j0 + cnt / 2;  // reference node of the source tile
    const double2 er = a.et[r];
    a.off32[i] = make_float2((float)(et.x - er.x), (float)(et.y - er.y));
    if (i == r) {
        a.ref32[tile] = split_hilo(er);
        a.ref64[tile] = er;
    }
    // df32 offset to the same reference: hi/lo split of the FP64 difference
    const double ox = et.x - er.x, oy = et.y - er.y;
    const float ohx = (float)ox, ohy = (float)oy;
    a.offdf[i] = make_float4(ohx, ohy, (float)(ox - (double)ohx), (float)(oy - (double)ohy));
    if (a.has_adj) {
        const double2 epp = make_double2(a.etpp[2 * i], a.etpp[2 * i + 1]);
        const double2 Ap = a.Ap ? make_double2(a.Ap[2 * i], a.Ap[2 * i + 1]) : make_double2(0.0, 0.0);
        if (!finite2(epp) || !finite2(Ap)) bad |= 1;
        const double pp = etp.x * etp.x + etp.y * etp.y;
        // Im(eta''/eta') = Im(eta'' conj(eta')) / |eta'|^2 ; Im(A'/A) likewise
        const double im1 = (pp > 0.0) ? (epp.y * etp.x - epp.x * etp.y) / pp : 0.0;
        const double im2 = (Ap.y * A.x - Ap.x * A.y) / aa;
        if (a.plain) {
            // (2 pi/n) N(t,t) and (2 pi/n) M_1(t,t) (Eqs. N-tt, M1-tt)
            const double re1 = (pp > 0.0) ? (epp.x * etp.x + epp.y * etp.y) / pp : 0.0;
            const double re2 = (Ap.x * A.x + Ap.y * A.y) / aa;
            const double Nd = (2.0 / a.n) * (0.5 * im1 - im2);
            const double M1d = (2.0 / a.n) * (0.5 * re1 - re2);
            a.b1[i] = -1.0 - Nd;   // 2x + b1 x - Bx = (I - B - diag(Nd)) x
            a.d1[i] = -M1d;        // Dx - d1 x + L x = (D + diag(M1d) + L) x
            a.ediag[i] = 1.0 + Nd; // e x + B^T x + P x = (I + diag(Nd) + B^T + P) x
        } else {
            a.ediag[i] = (2.0 / a.n) * (im1 - im2);
        }
    }
    if (bad) atomicOr(a.flag, bad);
}

}  // namespace

int run_circulant(const Boundary& b, const double* x, double* y, cudaStream_t st) {
    const ProfToken tok = prof_begin(st, PK_CIRC);
    if (b.fft_pow2) {
        const int pairs = (b.m1 + 1) / 2;
        const int threads = std::min(512, std::max(32, b.n / 2));
        const size_t smem = 2 * (size_t)b.n * sizeof(double2);
        circulant_fft_kernel<<<pairs, threads, smem, st>>>(x, y, b.n, b.m1, b.twiddle);
    } else {
        const int threads = 256;
        dim3 grid((b.n + threads - 1) / threads, b.m1);
        circulant_direct_kernel<<<grid, threads, b.n * sizeof(double), st>>>(x, y, b.n, b.Lcol);
    }
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tok, PK_CIRC, 16.0 * b.N, st);
    count_launches(1);
    return GNK_OK;
}

int run_component_means(const Boundary& b, const double* x, double* means, cudaStream_t st) {
    component_means_kernel<<<b.m1, 256, 0, st>>>(x, means, b.n);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

int run_prepare_nodes(Boundary& b, const double* etpp, const double* Ap, int* d_flag, cudaStream_t st) {
    PrepArgs a;
    a.N = b.N;
    a.n = b.n;
    a.S = kSrcTile32;
    a.has_adj = etpp != nullptr;
    a.et = b.et;
    a.etp = b.etp;
    a.A = b.A;
    a.etpp = etpp;
    a.Ap = Ap;
    a.q = b.q;
    a.et32 = b.et32;
    a.off32 = b.off32;
    a.ref32 = b.ref32;
    a.q32 = b.q32;
    a.A32 = b.A32;
    a.ref64 = b.ref64;
    a.offdf = b.offdf;
    a.ediag = b.e;
    a.plain = b.plain;
    a.b1 = b.b1;
    a.d1 = b.d1;
    a.ones = b.ones;
    a.flag = d_flag;
    prepare_geometry_kernel<<<(b.N + 255) / 256, 256, 0, st>>>(a);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

// Circulant multipliers of one n: twiddles exp(-2 pi i k/n) (k < n/2) when n is
// a power of two up to 4096, else the first column b of L.
void circulant_tables(int n, std::vector<double2>* tw, std::vector<double>* col) {
    if (((n & (n - 1)) == 0) && n <= 4096) {
        tw->resize(n / 2);
        for (int k = 0; k < n / 2; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)n;
            (*tw)[k] = make_double2(std::cos(ang), std::sin(ang));
        }
    } else {
        col->resize(n);
        (*col)[0] = 0.0;
        for (int i = 1; i < n; ++i) (*col)[i] = ((i % 2) ? -1.0 : 1.0) / n / std::tan(M_PI * i / n);
    }
}

namespace {
// Batched circulant: one block per (system, component pair); descriptor
// (vector offset of the system, n, m1, table offset | pow2 << 30).
__global__ void batch_circulant_kernel(const int4* __restrict__ desc, const long long* __restrict__ base,
                                       const double* __restrict__ x, double* __restrict__ y,
                                       const double2* __restrict__ tw, const double* __restrict__ col) {
    extern __shared__ double2 sm[];
    const int4 dd = desc[blockIdx.x];
    const int n = dd.x, m1 = dd.y, pair = dd.z;
    const bool pow2 = (dd.w >> 30) & 1;
    const int toff = dd.w & ((1 << 30) - 1);
    const long long b0 = base[blockIdx.x];
    const int ca = 2 * pair, cb = ca + 1;
    const bool has_b = cb < m1;
    double2* X = sm;
    double2* Y = sm + n;
    for (int p = threadIdx.x; p < n; p += blockDim.x)
        X[p] = make_double2(x[b0 + (long long)ca * n + p], has_b ? x[b0 + (long long)cb * n + p] : 0.0);
    __syncthreads();
    if (pow2) {
        double2* F = stockham(X, Y, n, tw + toff, false);
        double2* G = (F == X) ? Y : X;
        const int half = n >> 1;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double s = (k < half) ? (2.0 * k) / n : (k == half ? 0.0 : (2.0 * (k - n)) / n);
            const double2 v = F[k];
            F[k] = make_double2(-s * v.y, s * v.x);
        }
        __syncthreads();
        double2* Z = stockham(F, G, n, tw + toff, true);
        const double inv_n = 1.0 / n;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            y[b0 + (long long)ca * n + p] = Z[p].x * inv_n;
            if (has_b) y[b0 + (long long)cb * n + p] = Z[p].y * inv_n;
        }
    } else {
        const double* bc = col + toff;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            double ra = 0.0, rb = 0.0;
            for (int q = 0; q < n; ++q) {
                int d = p - q;
                d += (d < 0) ? n : 0;
                ra = fma(bc[d], X[q].x, ra);
                rb = fma(bc[d], X[q].y, rb);
            }
            y[b0 + (long long)ca * n + p] = ra;
            if (has_b) y[b0 + (long long)cb * n + p] = rb;
        }
    }
}
}  // namespace

int run_batch_circulant(const int4* desc, const long long* base, int nblocks, int nmax,
                        const double* x, double* y, const double2* tw, const double* col, cudaStream_t st) {
    if (nblocks == 0) return GNK_OK;
    const size_t smem = 2 * (size_t)nmax * sizeof(double2);
    static bool attr_set = false;
    if (smem > 48 * 1024 && !attr_set) {
        GNK_TRY_CUDA(cudaFuncSetAttribute(batch_circulant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          2 * 4096 * (int)sizeof(double2)));
        attr_set = true;
    }
    const ProfToken tok = prof_begin(st, PK_CIRC);
    batch_circulant_kernel<<<nblocks, 256, smem, st>>>(desc, base, x, y, tw, col);
    GNK_TRY_CUDA(cudaGetLastError());
    prof_end(tok, PK_CIRC, 0.0, st);
    count_launches(1);
    return GNK_OK;
}

int run_prepare_geometry(Boundary& b, const double* etpp, const double* Ap, int* d_flag,
                         cudaStream_t st) {
    GNK_TRY(run_prepare_nodes(b, etpp, Ap, d_flag, st));

    // circulant tables (host, FP64 libm)
    const int n = b.n;
    b.fft_pow2 = ((n & (n - 1)) == 0) && n <= 4096;  // two n-point buffers fit in shared memory
    if (b.fft_pow2) {
        std::vector<double2> tw(n / 2);
        for (int k = 0; k < n / 2; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)n;
            tw[k] = make_double2(std::cos(ang), std::sin(ang));
        }
        GNK_TRY_CUDA(cudaMemcpyAsync(b.twiddle, tw.data(), tw.size() * sizeof(double2),
                                     cudaMemcpyHostToDevice, st));
        if (2 * (size_t)n * sizeof(double2) > 48 * 1024) {
            GNK_TRY_CUDA(cudaFuncSetAttribute(circulant_fft_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(2 * (size_t)n * sizeof(double2))));
        }
    } else {
        std::vector<double> col(n);
        col[0] = 0.0;
        for (int i = 1; i < n; ++i) {
            const double sgn = (i % 2) ? -1.0 : 1.0;  // (-1)^i with 0-based i
            col[i] = sgn / n / std::tan(M_PI * i / n);
        }
        GNK_TRY_CUDA(cudaMemcpyAsync(b.Lcol, col.data(), n * sizeof(double),
                                     cudaMemcpyHostToDevice, st));
        if ((size_t)n * sizeof(double) > 48 * 1024) {
            GNK_TRY_CUDA(cudaFuncSetAttribute(circulant_direct_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(n * sizeof(double))));
        }
    }
    return GNK_OK;
}

}  // namespace gnk
