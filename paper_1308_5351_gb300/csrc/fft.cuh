// Radix-2 Stockham FFT of one block over n = 2^k points in shared memory
// (device code only), used by the circulant part L-hat x and by the periodic
// antiderivative of the slit maps' boundary correspondence.
#pragma once

#include <cuda_runtime.h>

namespace gnk {

static __device__ __forceinline__ double2 fft_cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Autosort (no bit reversal) transform of X with Y as the second buffer;
// returns the buffer that holds the result in natural order.  Twiddles
// tw[k] = exp(-2 pi i k / n), k < n/2; the inverse uses their conjugates and
// does not scale by 1/n.  Every thread of the block takes part; the block is
// synchronised after each stage.
static __device__ double2* stockham(double2* X, double2* Y, int n, const double2* tw, bool inverse) {
    const int half = n >> 1;
    for (int Ns = 1; Ns < n; Ns <<= 1) {
        const int stride = n / (2 * Ns);
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (Ns - 1);
            double2 w = tw[k * stride];
            if (inverse) w.y = -w.y;
            const double2 v0 = X[j];
            const double2 v1 = fft_cmul(X[j + half], w);
            const int d = ((j - k) << 1) + k;
            Y[d] = make_double2(v0.x + v1.x, v0.y + v1.y);
            Y[d + Ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        double2* t = X;
        X = Y;
        Y = t;
    }
    return X;
}

}  // namespace gnk
