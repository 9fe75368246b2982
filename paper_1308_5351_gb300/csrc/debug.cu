// Diagnostics of the library's own arithmetic and failure paths, for tests:
//   gnk_debug_recip_f64     - the FP64 reciprocal of the pair kernels next to
//                             CUDA's correctly rounded 1.0 / x;
//   gnk_debug_split_f64     - the bit-level double-float split of the FMM kernels;
//   gnk_debug_barrier_fault - makes the bounded grid-barrier waits of the
//                             Arnoldi step run out without any fault.
#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {
namespace {

__global__ void recip_check_kernel(const double* __restrict__ x, int n, double* __restrict__ y_lib,
                                   double* __restrict__ y_div) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    y_lib[i] = recip_f64(v);
    y_div[i] = 1.0 / v;  // IEEE division, round to nearest
}

__global__ void split_check_kernel(const double* __restrict__ x, int n, float* __restrict__ hi,
                                   float* __restrict__ lo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df d = df_split_fast(x[i]);
    hi[i] = d.h;
    lo[i] = d.l;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace gnk

using namespace gnk;

extern "C" int gnk_debug_recip_f64(int n, const double* x, double* y_lib, double* y_div, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y_lib || !y_div))) {
        set_error("gnk_debug_recip_f64: n >= 0 and three arrays are required");
        return GNK_EINVAL;
    }
    if (n == 0) return GNK_OK;
    if (!is_device_ptr(x) || !is_device_ptr(y_lib) || !is_device_ptr(y_div)) {
        set_error("gnk_debug_recip_f64: the arrays must be device memory");
        return GNK_EINVAL;
    }
    recip_check_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, n, y_lib, y_div);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

extern "C" int gnk_debug_split_f64(int n, const double* x, float* hi, float* lo, void* stream) {
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) {
        set_error("gnk_debug_split_f64: n >= 0 and three arrays are required");
        return GNK_EINVAL;
    }
    if (n == 0) return GNK_OK;
    if (!is_device_ptr(x) || !is_device_ptr(hi) || !is_device_ptr(lo)) {
        set_error("gnk_debug_split_f64: the arrays must be device memory");
        return GNK_EINVAL;
    }
    split_check_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, n, hi, lo);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

extern "C" int gnk_debug_barrier_fault(int skip_block, int spin_limit) {
    return debug_barrier_fault(skip_block, spin_limit);
}
