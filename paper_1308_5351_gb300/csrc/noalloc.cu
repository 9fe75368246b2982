// gnk_cauchy_sum_noalloc: the FP64 Cauchy sum z = E w for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plugins living inside a host
// application that owns the device memory and forbids allocations of its
// own, and real-time loops where an allocation's implicit device
// synchronisation, or its possible failure, is not acceptable.  They pass in
// device buffers for the inputs and the output and get the same sum as
// gnk_cauchy_sum, with the split-source partial sums kept in a fixed-size
// array that is part of the library's device image.
//
// The array below is reserved on every GPU that loads the library and stays
// there until the process exits.  Its size caps the problem: at most
// kNoAllocMaxNodes nodes.  All calls share it, so two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it; serialise them.  Every call overwrites all the entries it later reads,
// so nothing has to be cleared between calls.
#include <mutex>

#include "gnk_internal.h"
#include "pairmath.cuh"

namespace gnk {
namespace {

constexpr int kNoAllocMaxNodes = 65536;
constexpr int kNoAllocChunks = 4;        // source chunks (blocks along y)
constexpr int kNAThreads = 128;
constexpr int kNATargets = 2;
constexpr int kNATile = 128;
constexpr int kMaxDevices = 64;

// [chunk][node] partial sums: 4 x 65536 x 16 bytes = 4 MiB per device.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocChunks * kNoAllocMaxNodes];

std::mutex g_na_mu;
double2* g_na_ptr[kMaxDevices] = {};

__global__ void __launch_bounds__(kNAThreads) noalloc_pair_kernel(const double2* __restrict__ et,
                                                                  const double2* __restrict__ w,
                                                                  int N, int tiles_src, int tpc,
                                                                  double2* __restrict__ part) {
    __shared__ double2 s_pos[kNATile];
    __shared__ double2 s_w[kNATile];
    const int tgt0 = blockIdx.x * (kNAThreads * kNATargets);
    double px[kNATargets], py[kNATargets], ax[kNATargets], ay[kNATargets];
    int idx[kNATargets];
#pragma unroll
    for (int t = 0; t < kNATargets; ++t) {
        idx[t] = tgt0 + t * kNAThreads + threadIdx.x;
        const double2 p = et[min(idx[t], N - 1)];
        px[t] = p.x;
        py[t] = p.y;
        ax[t] = ay[t] = 0.0;
    }
    const int tb = blockIdx.y * tpc;
    const int te = min(tb + tpc, tiles_src);
    for (int tile = tb; tile < te; ++tile) {
        const int j0 = tile * kNATile;
        __syncthreads();
        {
            const int j = j0 + threadIdx.x;
            s_pos[threadIdx.x] = (j < N) ? et[j] : make_double2(1e150, 1e150);
            s_w[threadIdx.x] = (j < N) ? w[j] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int k = 0; k < kNATile; ++k) {
            const double2 sp = s_pos[k];
            const double2 wk = s_w[k];
            const int j = j0 + k;
#pragma unroll
            for (int t = 0; t < kNATargets; ++t) {
                const double dx = px[t] - sp.x, dy = py[t] - sp.y;
                double inv = recip_f64(fma(dx, dx, dy * dy));
                inv = (j == idx[t]) ? 0.0 : inv;  // no i = j term
                const double ar = dx * inv, ai = dy * inv;
                ax[t] = fma(wk.x, ar, fma(wk.y, ai, ax[t]));
                ay[t] = fma(wk.y, ar, fma(-wk.x, ai, ay[t]));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kNATargets; ++t)
        if (idx[t] < N) part[(size_t)blockIdx.y * N + idx[t]] = make_double2(ax[t], ay[t]);
}

__global__ void noalloc_reduce_kernel(const double2* __restrict__ part, int N, int chunks,
                                      double2* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < chunks; ++c) {
        const double2 p = part[(size_t)c * N + i];
        sx += p.x;
        sy += p.y;
    }
    z[i] = make_double2(sx, sy);
}

// Device memory of the current device (kernels launched here dereference
// it), or managed memory; anything else (host memory, another GPU's memory)
// is refused.
bool on_current_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is not a device address).
int scratch_for_current_device(double2** out) {
    int dev = 0;
    GNK_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gnk_cauchy_sum_noalloc: device ordinal %d not supported", dev);
        return GNK_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("gnk_cauchy_sum_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return GNK_ECUDA;
        }
        g_na_ptr[dev] = static_cast<double2*>(p);
    }
    *out = g_na_ptr[dev];
    return GNK_OK;
}

}  // namespace
}  // namespace gnk

using namespace gnk;

extern "C" int gnk_cauchy_sum_noalloc(int N, const double* et, const double* w, double* z,
                                      void* stream) {
    if (N < 1 || N > kNoAllocMaxNodes) {
        set_error("gnk_cauchy_sum_noalloc: N = %d outside 1..%d (the fixed scratch holds at most %d nodes)",
                  N, kNoAllocMaxNodes, kNoAllocMaxNodes);
        return GNK_EINVAL;
    }
    if (!et || !w || !z) {
        set_error("gnk_cauchy_sum_noalloc: NULL array");
        return GNK_EINVAL;
    }
    int dev = 0;
    GNK_TRY_CUDA(cudaGetDevice(&dev));
    if (!on_current_device(et, dev) || !on_current_device(w, dev) || !on_current_device(z, dev)) {
        set_error("gnk_cauchy_sum_noalloc: et, w and z must be device memory of the current device %d "
                  "(nothing is staged or copied)", dev);
        return GNK_EINVAL;
    }
    double2* part = nullptr;
    GNK_TRY(scratch_for_current_device(&part));
    cudaStream_t st = (cudaStream_t)stream;
    const int tiles_tgt = (N + kNAThreads * kNATargets - 1) / (kNAThreads * kNATargets);
    const int tiles_src = (N + kNATile - 1) / kNATile;
    const int chunks = tiles_src < kNoAllocChunks ? tiles_src : kNoAllocChunks;
    const int tpc = (tiles_src + chunks - 1) / chunks;
    const int used = (tiles_src + tpc - 1) / tpc;  // chunks that receive work
    dim3 grid(tiles_tgt, used);
    noalloc_pair_kernel<<<grid, kNAThreads, 0, st>>>(reinterpret_cast<const double2*>(et),
                                                     reinterpret_cast<const double2*>(w), N,
                                                     tiles_src, tpc, part);
    GNK_TRY_CUDA(cudaGetLastError());
    noalloc_reduce_kernel<<<(N + 255) / 256, 256, 0, st>>>(part, N, used,
                                                           reinterpret_cast<double2*>(z));
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(2);
    return GNK_OK;
}
