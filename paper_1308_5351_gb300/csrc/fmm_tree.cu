// The FMM quadtree built on the device (the geometry of a handle is fixed, so
// this runs once per handle, on the first FMM product):
//   1. bounding square of the nodes;
//   2. 32-bit Morton keys of 16-bit box coordinates;
//   3. stable LSD radix sort of (key, node), three passes of 8 bits (bits 8-31);
//   4. the level at which each node's key first differs from its predecessor's,
//      whose histogram fixes the leaf level L (the deepest level whose non-empty
//      boxes hold >= kFmmLeaf nodes on average);
//   5. per level, box ids by block counts, a scan over blocks and warp ballots;
//   6. box centres, widths, parents and child ranges from the first node of each box;
//   7. dense lookup grids of the boxes of each level, then interaction lists
//      (children of the parent's neighbours that are not adjacent) and the
//      neighbour leaves of each leaf, counted, scanned and filled;
//   8. node order, positions, exact three-float splits and near-field work items.
// Every step is deterministic (counts and scans in a fixed order), so the tree,
// and with it every FMM product, is reproducible.  Three small device-to-host
// reads size the allocations.  Trees deeper than 11 levels (lookup grids of more
// than 4M cells per level) are left to the host builder.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "fmm_internal.h"
#include "gnk_internal.h"

namespace gnk {
namespace {

constexpr int TB = 256;           // threads of the per-node kernels
constexpr int RS_TILE = 2048;     // radix sort: nodes per block (8 warps x 256)
constexpr int LV_BLOCK = 1024;    // level box ids: nodes per block
constexpr int kMaxGridLevel = 11;

__device__ __forceinline__ uint32_t spread16d(uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ uint32_t compact16d(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// ---- 1. bounding square: per-block min/max, the last block combines them
// and forms (x0, y0, W)
__global__ void __launch_bounds__(TB) tb_bbox(const double2* __restrict__ et, int N, double4* part,
                                              unsigned* counter, double* geom) {
    __shared__ double4 red[TB];
    __shared__ bool last;
    double4 m = make_double4(1e300, -1e300, 1e300, -1e300);
    for (int i = blockIdx.x * TB + threadIdx.x; i < N; i += gridDim.x * TB) {
        const double2 p = et[i];
        m.x = fmin(m.x, p.x);
        m.y = fmax(m.y, p.x);
        m.z = fmin(m.z, p.y);
        m.w = fmax(m.w, p.y);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = TB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double4 o = red[threadIdx.x + w];
            double4& r = red[threadIdx.x];
            r.x = fmin(r.x, o.x);
            r.y = fmax(r.y, o.y);
            r.z = fmin(r.z, o.z);
            r.w = fmax(r.w, o.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    // the last block combines the partials in parallel (then the same tree)
    m = make_double4(1e300, -1e300, 1e300, -1e300);
    for (int b = threadIdx.x; b < gridDim.x; b += TB) {
        const double2 lo = __ldcg(reinterpret_cast<const double2*>(part + b));
        const double2 hi = __ldcg(reinterpret_cast<const double2*>(part + b) + 1);
        const double4 o = make_double4(lo.x, lo.y, hi.x, hi.y);
        m.x = fmin(m.x, o.x);
        m.y = fmax(m.y, o.y);
        m.z = fmin(m.z, o.z);
        m.w = fmax(m.w, o.w);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = TB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double4 o = red[threadIdx.x + w];
            double4& q = red[threadIdx.x];
            q.x = fmin(q.x, o.x);
            q.y = fmax(q.y, o.y);
            q.z = fmin(q.z, o.z);
            q.w = fmax(q.w, o.w);
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double4 r = red[0];
    const double W = fmax(fmax(r.y - r.x, r.w - r.z) * (1.0 + 1e-9), 1e-300);
    geom[0] = 0.5 * (r.x + r.y) - 0.5 * W;
    geom[1] = 0.5 * (r.z + r.w) - 0.5 * W;
    geom[2] = W;
    *counter = 0;
}

// ---- 2. Morton keys
__global__ void tb_keys(const double2* __restrict__ et, int N, const double* geom, uint32_t* key, int* idx) {
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i >= N) return;
    const double x0 = geom[0], y0 = geom[1], W = geom[2];
    const double2 p = et[i];
    const double fx = (p.x - x0) / W * 65536.0, fy = (p.y - y0) / W * 65536.0;
    const uint32_t ix = (uint32_t)fmin(65535.0, fmax(0.0, floor(fx)));
    const uint32_t iy = (uint32_t)fmin(65535.0, fmax(0.0, floor(fy)));
    key[i] = (spread16d(ix) << 1) | spread16d(iy);
    idx[i] = i;
}

// ---- 3. radix sort passes
__global__ void __launch_bounds__(TB) tb_hist(const uint32_t* __restrict__ key, int N, int shift,
                                              unsigned* hist, int nb) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE, end = min(base + RS_TILE, N);
    for (int e = base + threadIdx.x; e < end; e += TB) atomicAdd(&h[(key[e] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];  // digit-major
}

// Exclusive scans in place, one block of 1024 threads per array (up to three
// arrays in one launch); each array's total goes to *total when non-null.
// Every thread takes a contiguous range; the ranges' sums are scanned by warp
// shuffles and one pass over the 32 warp totals.
struct ScanArgs {
    unsigned* a[3];
    int len[3];
    unsigned* total[3];
};

__global__ void __launch_bounds__(1024) tb_scan(ScanArgs sa) {
    __shared__ unsigned ws[32];
    unsigned* a = sa.a[blockIdx.x];
    const int len = sa.len[blockIdx.x];
    unsigned* total = sa.total[blockIdx.x];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (len + 1023) / 1024;
    const int b0 = min(len, (int)threadIdx.x * per), b1 = min(b0 + per, len);
    unsigned sum = 0;
    for (int k = b0; k < b1; ++k) sum += a[k];
    unsigned v = sum;  // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(full, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {  // inclusive scan of the warps' totals
        unsigned w = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(full, w, o);
            if (lane >= o) w += t;
        }
        ws[lane] = w;
    }
    __syncthreads();
    unsigned run = (wid > 0 ? ws[wid - 1] : 0u) + v - sum;
    for (int k = b0; k < b1; ++k) {
        const unsigned x = a[k];
        a[k] = run;
        run += x;
    }
    if (total && threadIdx.x == 1023) *total = ws[31];
}

static ScanArgs scan_of(unsigned* a, int len, unsigned* total) {
    ScanArgs sa{};
    sa.a[0] = a;
    sa.len[0] = len;
    sa.total[0] = total;
    return sa;
}

// Stable scatter: warp w of a block owns nodes [base + 256 w, base + 256 (w + 1)),
// counted first, then written in order with ranks from __match_any_sync.
__global__ void __launch_bounds__(TB) tb_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ iin,
                                                 uint32_t* kout, int* iout, int N, int shift,
                                                 const unsigned* __restrict__ hist, int nb) {
    __shared__ unsigned wc[TB / 32][256];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < (TB / 32) * 256; k += TB) (&wc[0][0])[k] = 0u;
    __syncthreads();
    const int wbase = blockIdx.x * RS_TILE + wid * 256;
    for (int r = 0; r < 8; ++r) {
        const int e = wbase + r * 32 + lane;
        if (e < N) atomicAdd(&wc[wid][(kin[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // TB == 256 digits
        unsigned run = hist[(size_t)d * nb + blockIdx.x];
        for (int w = 0; w < TB / 32; ++w) {
            const unsigned c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < 8; ++r) {
        const int e = wbase + r * 32 + lane;
        const bool valid = e < N;
        const uint32_t k = valid ? kin[e] : 0u;
        const unsigned d = valid ? ((k >> shift) & 255u) : 256u + lane;  // invalid lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid) {
            const unsigned pos = wc[wid][d] + __popc(peers & lt);
            kout[pos] = k;
            iout[pos] = iin[e];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[wid][d] += __popc(peers);
        __syncwarp();
    }
}

// ---- 4. first differing level (0 for the first node, 17 for a repeated key)
__global__ void __launch_bounds__(TB) tb_firstdiff(const uint32_t* __restrict__ key, int N, unsigned char* fd,
                                                   unsigned* fdh) {
    __shared__ unsigned h[18];
    if (threadIdx.x < 18) h[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i < N) {
        int f = 0;
        if (i > 0) {
            const uint32_t x = key[i] ^ key[i - 1];
            f = x ? 16 - (31 - __clz(x)) / 2 : 17;
        }
        fd[i] = (unsigned char)f;
        atomicAdd(&h[f], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 18 && h[threadIdx.x]) atomicAdd(&fdh[threadIdx.x], h[threadIdx.x]);
}

// ---- 5. box ids per level: node i starts a box of level l when fd[i] <= l
__global__ void __launch_bounds__(LV_BLOCK) tb_lcount(const unsigned char* __restrict__ fd, int N, int L,
                                                      unsigned* cnt, int nb) {
    const int i = blockIdx.x * LV_BLOCK + threadIdx.x;
    const int f = (i < N) ? fd[i] : 99;
    for (int l = 2; l <= L; ++l) {
        const int c = __syncthreads_count(f <= l);
        if (threadIdx.x == 0) cnt[(size_t)(l - 2) * nb + blockIdx.x] = (unsigned)c;
    }
}

// one block per level: exclusive scan of its row of block counts; row total = boxes of the level
__global__ void __launch_bounds__(1024) tb_lscan(unsigned* cnt, int nb, unsigned* totals) {
    __shared__ unsigned s[1024];
    unsigned* a = cnt + (size_t)blockIdx.x * nb;
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nb);
    unsigned sum = 0;
    for (int k = b0; k < b1; ++k) sum += a[k];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned v = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = s[threadIdx.x] - sum;
    for (int k = b0; k < b1; ++k) {
        const unsigned v = a[k];
        a[k] = run;
        run += v;
    }
    if (threadIdx.x == 1023) totals[blockIdx.x] = s[1023];
}

// box id of every node at every level, and the first node of every box
__global__ void __launch_bounds__(LV_BLOCK) tb_lids(const unsigned char* __restrict__ fd, int N, int L,
                                                    const unsigned* __restrict__ cnt, int nb, int* boxid,
                                                    int* first) {
    __shared__ unsigned wsum[LV_BLOCK / 32];
    const int i = blockIdx.x * LV_BLOCK + threadIdx.x;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = (i < N) ? fd[i] : 99;
    for (int l = 2; l <= L; ++l) {
        const bool start = f <= l;
        const unsigned bal = __ballot_sync(0xffffffffu, start);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        unsigned before = cnt[(size_t)(l - 2) * nb + blockIdx.x];
        for (int w = 0; w < wid; ++w) before += wsum[w];
        before += __popc(bal & ((1u << lane) - 1u));
        if (i < N) {
            const int id = (int)before + (start ? 1 : 0) - 1;  // node 0 starts every level
            boxid[(size_t)(l - 2) * N + i] = id;
            if (start) first[(size_t)(l - 2) * (N + 1) + id] = i;
        }
        __syncthreads();
    }
}

struct TreeDev {
    int N, L, nbox, nleaf;
    const uint32_t* key;     // sorted keys
    const int* boxid;        // [l - 2][N]
    const int* first;        // [l - 2][N + 1]
    const int* lvl_off;      // [L - 1]
    const int* lvl_cnt;
    const double* geom;
    double2* center;
    double* width;
    int* child_start;
    int* child_count;
    int* parent;
    int* quad;
    int* bix;
    int* biy;
    int* leaf_start;
    int* leaf_box;
    int* grid;               // per level l <= L: (2^l)^2 cells, offsets in grid_off
    const long long* grid_off;
    unsigned* il_cnt;        // nbox + 1 (scanned in place)
    unsigned* nl_cnt;        // nleaf + 1
    unsigned* it_cnt;        // nleaf + 1
    int* il_src;
    int* il_off;
    int* nl_leaf;
    int2* items;
    unsigned long long* near_pairs;
};

__device__ __forceinline__ int level_of(const TreeDev& t, int g) {
    int l = 2;
    while (l < t.L && g >= t.lvl_off[l - 1]) ++l;
    return l;
}

// ---- 6. box geometry and links
__global__ void tb_boxes(TreeDev t) {
    const int g = blockIdx.x * TB + threadIdx.x;
    if (g >= t.nbox) return;
    const int l = level_of(t, g);
    const int b = g - t.lvl_off[l - 2];
    const int f = t.first[(size_t)(l - 2) * (t.N + 1) + b];
    const int fn = (b + 1 < t.lvl_cnt[l - 2]) ? t.first[(size_t)(l - 2) * (t.N + 1) + b + 1] : t.N;
    const uint32_t k = t.key[f] >> (2 * (16 - l));
    const int ix = (int)compact16d(k >> 1), iy = (int)compact16d(k);
    const double W = t.geom[2], r = W / (double)(1 << l);
    t.center[g] = make_double2(t.geom[0] + (ix + 0.5) * r, t.geom[1] + (iy + 0.5) * r);
    t.width[g] = r;
    t.quad[g] = ((ix & 1) << 1) | (iy & 1);
    t.bix[g] = ix;
    t.biy[g] = iy;
    t.parent[g] = (l > 2) ? t.lvl_off[l - 3] + t.boxid[(size_t)(l - 3) * t.N + f] : -1;
    if (l < t.L) {
        const int c0 = t.boxid[(size_t)(l - 1) * t.N + f], c1 = t.boxid[(size_t)(l - 1) * t.N + fn - 1];
        t.child_start[g] = t.lvl_off[l - 1] + c0;
        t.child_count[g] = c1 - c0 + 1;
    } else {
        t.child_start[g] = -1;
        t.child_count[g] = 0;
        t.leaf_start[b] = f;
        t.leaf_box[b] = g;
        if (b == t.nleaf - 1) t.leaf_start[t.nleaf] = t.N;
    }
    t.grid[t.grid_off[l - 2] + (long long)ix * (1 << l) + iy] = g;
}

__device__ __forceinline__ int grid_at(const TreeDev& t, int l, int ix, int iy) {
    const int n = 1 << l;
    if (ix < 0 || iy < 0 || ix >= n || iy >= n) return -1;
    return t.grid[t.grid_off[l - 2] + (long long)ix * n + iy];
}

// ---- 7. lists: pass 0 counts, pass 1 fills (after the counts are scanned)
__global__ void tb_lists(TreeDev t, int pass) {
    const int g = blockIdx.x * TB + threadIdx.x;
    if (g >= t.nbox) return;
    const int l = level_of(t, g);
    const int ix = t.bix[g], iy = t.biy[g], pa = ix >> 1, pb = iy >> 1;
    unsigned n = 0, pos = pass ? t.il_cnt[g] : 0u;
    for (int sa = 2 * pa - 2; sa <= 2 * pa + 3; ++sa)
        for (int sb = 2 * pb - 2; sb <= 2 * pb + 3; ++sb) {
            const int dx = sa - ix, dy = sb - iy;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            const int s = grid_at(t, l, sa, sb);
            if (s < 0) continue;
            if (pass) {
                t.il_src[pos] = s;
                t.il_off[pos] = (dx + 3) * 7 + (dy + 3);
                ++pos;
            }
            ++n;
        }
    if (!pass) t.il_cnt[g] = n;
    if (l != t.L) return;
    const int q = g - t.lvl_off[t.L - 2];
    const int cnt_t = t.leaf_start[q + 1] - t.leaf_start[q];
    unsigned m = 0, npos = pass ? t.nl_cnt[q] : 0u;
    unsigned long long pairs = 0;
    for (int sa = ix - 1; sa <= ix + 1; ++sa)
        for (int sb = iy - 1; sb <= iy + 1; ++sb) {
            const int s = grid_at(t, l, sa, sb);
            if (s < 0) continue;
            const int lq = s - t.lvl_off[t.L - 2];
            if (pass) {
                t.nl_leaf[npos++] = lq;
            } else {
                pairs += (unsigned long long)cnt_t * (unsigned long long)(t.leaf_start[lq + 1] - t.leaf_start[lq]);
            }
            ++m;
        }
    if (!pass) {
        t.nl_cnt[q] = m;
        t.it_cnt[q] = (unsigned)((cnt_t + 31) / 32);
        atomicAdd(t.near_pairs, pairs);
    } else {
        unsigned ipos = t.it_cnt[q];
        for (int i = t.leaf_start[q]; i < t.leaf_start[q + 1]; i += 32) t.items[ipos++] = make_int2(q, i);
    }
}

// ---- 8. node arrays in sorted order
__global__ void tb_nodes(const double2* __restrict__ et, int N, const int* __restrict__ sidx,
                         const int* __restrict__ boxid_leaf, int leaf_off, int* perm, double2* ps, float4* p3,
                         float2* p3b, int* node_box) {
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i >= N) return;
    const int j = sidx[i];
    const double2 p = et[j];
    perm[i] = j;
    ps[i] = p;
    float sx[3], sy[3];
    // v = s0 + s1 + s2 exactly: each float takes the next 24 bits of the double
    sx[0] = (float)p.x;
    double r = p.x - (double)sx[0];
    sx[1] = (float)r;
    sx[2] = (float)(r - (double)sx[1]);
    sy[0] = (float)p.y;
    r = p.y - (double)sy[0];
    sy[1] = (float)r;
    sy[2] = (float)(r - (double)sy[1]);
    p3[i] = make_float4(sx[0], sx[1], sx[2], sy[0]);
    p3b[i] = make_float2(sy[1], sy[2]);
    node_box[i] = leaf_off + boxid_leaf[i];
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

int fmm_tree_device(const Boundary& b, FmmTree* t, cudaStream_t st) {
    const int N = b.N;
    const int nbs = (N + RS_TILE - 1) / RS_TILE;      // radix-sort blocks
    const int nbl = (N + LV_BLOCK - 1) / LV_BLOCK;    // level-count blocks
    const int nbb = std::min(1024, (N + TB - 1) / TB);
    const int nlev_max = 15;                          // levels 2..16
    // temporary device memory (freed at the end)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_geom = take(4 * sizeof(double));
    const size_t o_part = take((size_t)nbb * sizeof(double4));
    const size_t o_ctr = take(sizeof(unsigned));
    const size_t o_k0 = take((size_t)N * 4), o_k1 = take((size_t)N * 4);
    const size_t o_i0 = take((size_t)N * 4), o_i1 = take((size_t)N * 4);
    const size_t o_hist = take((size_t)256 * nbs * 4);
    const size_t o_fd = take((size_t)N);
    const size_t o_fdh = take(18 * 4);
    const size_t o_cnt = take((size_t)nlev_max * nbl * 4);
    const size_t o_tot = take((size_t)nlev_max * 4);
    const size_t tmp0 = off;
    char* tmp = nullptr;
    if (pool_alloc(reinterpret_cast<void**>(&tmp), tmp0, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM tree: device allocation of %zu bytes failed", tmp0);
        return GNK_ENOMEM;
    }
    struct Free {  // stream-ordered: no device synchronisation
        char** p;
        cudaStream_t st;
        ~Free() {
            if (*p) pool_free(*p, st);
        }
    } free_tmp{&tmp, st};
    double* geom = (double*)(tmp + o_geom);
    uint32_t* k0 = (uint32_t*)(tmp + o_k0);
    uint32_t* k1 = (uint32_t*)(tmp + o_k1);
    int* i0 = (int*)(tmp + o_i0);
    int* i1 = (int*)(tmp + o_i1);
    unsigned* hist = (unsigned*)(tmp + o_hist);
    unsigned char* fd = (unsigned char*)(tmp + o_fd);
    unsigned* fdh = (unsigned*)(tmp + o_fdh);
    unsigned* cnt = (unsigned*)(tmp + o_cnt);
    unsigned* tot = (unsigned*)(tmp + o_tot);
    GNK_TRY_CUDA(cudaMemsetAsync(tmp + o_ctr, 0, sizeof(unsigned), st));
    GNK_TRY_CUDA(cudaMemsetAsync(fdh, 0, 18 * 4, st));
    tb_bbox<<<nbb, TB, 0, st>>>(b.et, N, (double4*)(tmp + o_part), (unsigned*)(tmp + o_ctr), geom);
    tb_keys<<<(N + TB - 1) / TB, TB, 0, st>>>(b.et, N, geom, k0, i0);
    // LSD passes over bits 8..31 only: the device builder serves trees of at most
    // kMaxGridLevel (11) levels, whose boxes are fixed by the top 22 bits, and the
    // first-difference counts up to level 12 (which decide between this builder
    // and the host's) need the top 24; the order inside a level-12 cell is free
    for (int pass = 1; pass < 4; ++pass) {
        tb_hist<<<nbs, TB, 0, st>>>(k0, N, 8 * pass, hist, nbs);
        tb_scan<<<1, 1024, 0, st>>>(scan_of(hist, 256 * nbs, nullptr));
        tb_scatter<<<nbs, TB, 0, st>>>(k0, i0, k1, i1, N, 8 * pass, hist, nbs);
        std::swap(k0, k1);
        std::swap(i0, i1);
    }
    tb_firstdiff<<<(N + TB - 1) / TB, TB, 0, st>>>(k0, N, fd, fdh);
    GNK_TRY_CUDA(cudaGetLastError());
    unsigned h[18];
    GNK_TRY_CUDA(cudaMemcpyAsync(h, fdh, sizeof(h), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    int L = 2;
    long long distinct = 0;
    for (int l = 0; l <= 16; ++l) {
        distinct += h[l];
        if (l < 3) continue;
        if ((double)N / (double)distinct < kFmmLeaf) break;
        L = l;
    }
    if (L > kMaxGridLevel) return kFmmUseHost;
    t->L = L;
    const int nlev = L - 1;
    // per-level box ids (second temporary block)
    char* tmp2 = nullptr;
    const size_t o2_boxid = 0;
    const size_t o2_first = align256((size_t)nlev * N * 4);
    const size_t tmp2_bytes = o2_first + align256((size_t)nlev * (N + 1) * 4);
    if (pool_alloc(reinterpret_cast<void**>(&tmp2), tmp2_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM tree: device allocation of %zu bytes failed", tmp2_bytes);
        return GNK_ENOMEM;
    }
    Free free_tmp2{&tmp2, st};
    int* boxid = (int*)(tmp2 + o2_boxid);
    int* first = (int*)(tmp2 + o2_first);
    tb_lcount<<<nbl, LV_BLOCK, 0, st>>>(fd, N, L, cnt, nbl);
    tb_lscan<<<nlev, 1024, 0, st>>>(cnt, nbl, tot);
    tb_lids<<<nbl, LV_BLOCK, 0, st>>>(fd, N, L, cnt, nbl, boxid, first);
    GNK_TRY_CUDA(cudaGetLastError());
    std::vector<unsigned> ncnt(nlev);
    GNK_TRY_CUDA(cudaMemcpyAsync(ncnt.data(), tot, nlev * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    t->lvl_off.resize(nlev);
    t->lvl_cnt.resize(nlev);
    int nbox = 0;
    for (int l = 2; l <= L; ++l) {
        t->lvl_off[l - 2] = nbox;
        t->lvl_cnt[l - 2] = (int)ncnt[l - 2];
        nbox += (int)ncnt[l - 2];
    }
    const int nleaf = t->lvl_cnt[L - 2];
    t->nbox = nbox;
    t->nleaf = nleaf;
    std::vector<long long> goff(nlev);
    long long gcells = 0;
    for (int l = 2; l <= L; ++l) {
        goff[l - 2] = gcells;
        gcells += (1LL << (2 * l));
    }
    // upper bounds of the list lengths: 27 interactions per box, 9 neighbours per
    // leaf, one chunk of 32 per leaf plus one per 32 nodes
    const size_t max_il = (size_t)27 * nbox + 1, max_nl = (size_t)9 * nleaf + 1;
    const size_t max_it = (size_t)nleaf + N / 32 + 1;
    // the handle's tree arena (the same layout as the host builder's)
    const size_t P = kFmmP;
    struct Part {
        void** p;
        size_t bytes;
    };
    Part parts[] = {
        {(void**)&t->perm, N * sizeof(int)},
        {(void**)&t->ps, N * sizeof(double2)},
        {(void**)&t->p3, N * sizeof(float4)},
        {(void**)&t->p3b, N * sizeof(float2)},
        {(void**)&t->leaf_start, (nleaf + 1) * sizeof(int)},
        {(void**)&t->leaf_box, nleaf * sizeof(int)},
        {(void**)&t->center, nbox * sizeof(double2)},
        {(void**)&t->width, nbox * sizeof(double)},
        {(void**)&t->child_start, nbox * sizeof(int)},
        {(void**)&t->child_count, nbox * sizeof(int)},
        {(void**)&t->parent, nbox * sizeof(int)},
        {(void**)&t->quad, nbox * sizeof(int)},
        {(void**)&t->il_start, (nbox + 1) * sizeof(int)},
        {(void**)&t->il_src, max_il * sizeof(int)},
        {(void**)&t->il_off, max_il * sizeof(int)},
        {(void**)&t->nl_start, (nleaf + 1) * sizeof(int)},
        {(void**)&t->nl_leaf, max_nl * sizeof(int)},
        {(void**)&t->items, max_it * sizeof(int2)},
        {(void**)&t->node_box, N * sizeof(int)},
        {(void**)&t->mult, (size_t)t->R * nbox * P * sizeof(float4)},
        {(void**)&t->loc, (size_t)t->R * nbox * P * sizeof(float4)},
        {(void**)&t->ws, (size_t)t->R * N * sizeof(float4)},
        {(void**)&t->zn, (size_t)t->R * N * sizeof(double2)},
        {(void**)&t->zf, (size_t)t->R * N * sizeof(double2)},
    };
    size_t total = 0;
    for (const Part& p : parts) total += align256(p.bytes);
    if (pool_alloc(&t->arena, total, st) != cudaSuccess) {
        cudaGetLastError();
        t->arena = nullptr;
        set_error("FMM tree: device allocation of %zu bytes failed", total);
        return GNK_ENOMEM;
    }
    char* cur = static_cast<char*>(t->arena);
    for (const Part& p : parts) {
        *p.p = cur;
        cur += align256(p.bytes);
    }
    // third temporary block: box coordinates, grids, list counts, level tables
    char* tmp3 = nullptr;
    size_t o3 = 0;
    auto take3 = [&](size_t bytes) {
        const size_t o = o3;
        o3 += align256(bytes);
        return o;
    };
    const size_t o3_bix = take3((size_t)nbox * 4), o3_biy = take3((size_t)nbox * 4);
    const size_t o3_grid = take3((size_t)gcells * 4);
    const size_t o3_ilc = take3((size_t)(nbox + 1) * 4);
    const size_t o3_nlc = take3((size_t)(nleaf + 1) * 4), o3_itc = take3((size_t)(nleaf + 1) * 4);
    const size_t o3_lo = take3((size_t)nlev * 4), o3_lc = take3((size_t)nlev * 4);
    const size_t o3_go = take3((size_t)nlev * 8);
    const size_t o3_np = take3(8);
    const size_t o3_tot = take3(3 * 4);
    if (pool_alloc(reinterpret_cast<void**>(&tmp3), o3, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("FMM tree: device allocation of %zu bytes failed", o3);
        return GNK_ENOMEM;
    }
    Free free_tmp3{&tmp3, st};
    GNK_TRY_CUDA(cudaMemsetAsync(tmp3 + o3_grid, 0xff, (size_t)gcells * 4, st));
    GNK_TRY_CUDA(cudaMemsetAsync(tmp3 + o3_np, 0, 8, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(tmp3 + o3_lo, t->lvl_off.data(), nlev * 4, cudaMemcpyHostToDevice, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(tmp3 + o3_lc, t->lvl_cnt.data(), nlev * 4, cudaMemcpyHostToDevice, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(tmp3 + o3_go, goff.data(), nlev * 8, cudaMemcpyHostToDevice, st));
    TreeDev d;
    d.N = N;
    d.L = L;
    d.nbox = nbox;
    d.nleaf = nleaf;
    d.key = k0;
    d.boxid = boxid;
    d.first = first;
    d.lvl_off = (const int*)(tmp3 + o3_lo);
    d.lvl_cnt = (const int*)(tmp3 + o3_lc);
    d.geom = geom;
    d.center = t->center;
    d.width = t->width;
    d.child_start = t->child_start;
    d.child_count = t->child_count;
    d.parent = t->parent;
    d.quad = t->quad;
    d.bix = (int*)(tmp3 + o3_bix);
    d.biy = (int*)(tmp3 + o3_biy);
    d.leaf_start = t->leaf_start;
    d.leaf_box = t->leaf_box;
    d.grid = (int*)(tmp3 + o3_grid);
    d.grid_off = (const long long*)(tmp3 + o3_go);
    d.il_cnt = (unsigned*)(tmp3 + o3_ilc);
    d.nl_cnt = (unsigned*)(tmp3 + o3_nlc);
    d.it_cnt = (unsigned*)(tmp3 + o3_itc);
    d.il_src = t->il_src;
    d.il_off = t->il_off;
    d.nl_leaf = t->nl_leaf;
    d.items = t->items;
    d.near_pairs = (unsigned long long*)(tmp3 + o3_np);
    unsigned* totals = (unsigned*)(tmp3 + o3_tot);
    const int gb = (nbox + TB - 1) / TB;
    tb_boxes<<<gb, TB, 0, st>>>(d);
    tb_lists<<<gb, TB, 0, st>>>(d, 0);
    {
        ScanArgs sa{};
        sa.a[0] = d.il_cnt;
        sa.len[0] = nbox;
        sa.total[0] = totals + 0;
        sa.a[1] = d.nl_cnt;
        sa.len[1] = nleaf;
        sa.total[1] = totals + 1;
        sa.a[2] = d.it_cnt;
        sa.len[2] = nleaf;
        sa.total[2] = totals + 2;
        tb_scan<<<3, 1024, 0, st>>>(sa);
    }
    tb_lists<<<gb, TB, 0, st>>>(d, 1);
    tb_nodes<<<(N + TB - 1) / TB, TB, 0, st>>>(b.et, N, i0, boxid + (size_t)(L - 2) * N, t->lvl_off[L - 2],
                                               t->perm, t->ps, t->p3, t->p3b, t->node_box);
    GNK_TRY_CUDA(cudaGetLastError());
    // CSR starts: the scanned counts with their totals appended
    GNK_TRY_CUDA(cudaMemcpyAsync(t->il_start, d.il_cnt, (size_t)nbox * 4, cudaMemcpyDeviceToDevice, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(t->il_start + nbox, totals + 0, 4, cudaMemcpyDeviceToDevice, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(t->nl_start, d.nl_cnt, (size_t)nleaf * 4, cudaMemcpyDeviceToDevice, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(t->nl_start + nleaf, totals + 1, 4, cudaMemcpyDeviceToDevice, st));
    unsigned tot_h[3];
    unsigned long long np_h = 0;
    GNK_TRY_CUDA(cudaMemcpyAsync(tot_h, totals, sizeof(tot_h), cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaMemcpyAsync(&np_h, d.near_pairs, 8, cudaMemcpyDeviceToHost, st));
    GNK_TRY_CUDA(cudaStreamSynchronize(st));
    t->m2l_pairs = tot_h[0];
    t->nitems = (int)tot_h[2];
    t->near_pairs = (long long)np_h;
    t->m2m_pairs = nbox - t->lvl_cnt[0];
    return GNK_OK;
}

}  // namespace gnk
