// FMM tree shared by the host- and device-side tree builders and the FMM
// product (fmm.cu, fmm_tree.cu).  Internal header.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "gnk_internal.h"

namespace gnk {

constexpr int kFmmP = 32;     // expansion order (one warp lane per coefficient)
#ifndef GNK_FMM_LEAF
#define GNK_FMM_LEAF 64
#endif
constexpr int kFmmLeaf = GNK_FMM_LEAF;  // target mean number of nodes per leaf
constexpr int kFmmNT = 256;   // threads of the near-field kernel: 8 warps

struct FmmTree {
    int L = 0, nbox = 0, nleaf = 0, R = 0;
    std::vector<int> lvl_off;   // first global box index of level l (index l - 2), size L - 1
    std::vector<int> lvl_cnt;
    long long near_pairs = 0, m2l_pairs = 0, m2m_pairs = 0;
    void* arena = nullptr;
    int* perm = nullptr;        // sorted position -> node
    double2* ps = nullptr;      // node positions in sorted order
    float4* p3 = nullptr;       // the same split exactly into three floats: (x1, x2, x3, y1)
    float2* p3b = nullptr;      // (y2, y3)
    int* leaf_start = nullptr;  // nleaf + 1
    int* leaf_box = nullptr;    // global box index of each leaf
    double2* center = nullptr;  // per box
    double* width = nullptr;    // per box
    int* child_start = nullptr; // per box: first child (global), level < L
    int* child_count = nullptr;
    int* parent = nullptr;      // per box, -1 on level 2
    int* quad = nullptr;        // quadrant of a box in its parent: 2 qa + qb
    int* il_start = nullptr;    // interaction lists (nbox + 1), sources, offset codes
    int* il_src = nullptr;
    int* il_off = nullptr;
    int* nl_start = nullptr;    // neighbour leaves of each leaf (nleaf + 1)
    int* nl_leaf = nullptr;
    int2* items = nullptr;      // (leaf, first target) of every chunk of 32 targets
    int nitems = 0;
    const float2* m2lH = nullptr;  // M2L: the Pascal matrix C(k+l, l) [k][l] as double-float,
    const float4* m2lS = nullptr;  // and per offset code the two complex scalings (per-device cache)
    const float2* bUp = nullptr;   // L2L Pascal table C(l,m) [l][m]
    float4* mult = nullptr;     // [R][nbox][P]
    float4* loc = nullptr;      // [R][nbox][P]
    float4* ws = nullptr;       // [R][N] weights in sorted order, double-float complex
    double2* zn = nullptr;      // [R][N] near-field sums in sorted order
    double2* zf = nullptr;      // [R][N] near-field sums of w/d^2 (gradient products)
    int* node_box = nullptr;    // leaf box of each node in sorted order
    int* sync = nullptr;        // [nbox]: children counted by the upward pass (zero between products)
    // near-field operator cache of the products z = E(q x) (fixed geometry):
    // Q_ij = q_j / (eta_i - eta_j) per work item, double-float, for source
    // pairs x targets; state 0 not formed, 2 allocated (formed by the first
    // cached product), 1 formed, -1 not used (too large)
    int nq_state = 0;
    long long* nq_cnt = nullptr;   // build temporaries while state is 2
    long long* nq_soff = nullptr;
    long long nq_slots = 0;     // float4 entries of each of nq_re, nq_im
    long long* nq_off = nullptr;  // per work item: first entry (nitems + 1)
    int4* nq_item = nullptr;    // per work item: (S sources, tn targets, first source in nq_src, -)
    int* nq_src = nullptr;      // the items' sources (sorted node indices), item after item, each
                                // item's list padded to even length with -1 (nq_qb entries)
    long long nq_qb = 0;        // entries of nq_src (a bound on the lists' total, even)
    float4* nq_re = nullptr;
    float4* nq_im = nullptr;
    float2* xs = nullptr;       // [R][N] x in sorted order, double-float (cached products)
    float2* xl = nullptr;       // [R][nq_qb] x in the items' source-list order (0 at padding)
    int* fault = nullptr;       // set by a bounded wait of an FMM kernel that gave up
    float4* tp = nullptr;       // [N][P] powers t^k of each node about its leaf centre (P2M), or null
    cudaStream_t aux = nullptr; // high-priority stream of the far field (the near field runs beside it)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t bst = nullptr; // stream of the near cache's formation when it starts early
    cudaEvent_t ev_nq = nullptr;
    int nq_wait = 0;            // the next cached product waits for ev_nq
};

// Builds the tree on the device (Morton keys, stable radix sort, boxes per level,
// interaction and neighbour lists) into t, with its device arena.  Returns
// GNK_OK, an error code, or kFmmUseHost when the tree is too deep for the
// device lookup grids (then the host builder runs).
constexpr int kFmmUseHost = 1;
int fmm_tree_device(const Boundary& b, FmmTree* t, cudaStream_t st);

// The double-float translation tables on the current device (formed and
// uploaded once per device and process): the M2L Pascal matrix C(k+l, l)
// [P][P] and, per offset code (dx + 3) 7 + (dy + 3), the scalings
// (-1)^(k+1) delta^-(k+1) and delta^-l; the L2L Pascal matrix C(l, m).
int fmm_device_tables(const float2** m2lH, const float4** m2lS, const float2** bUp, cudaStream_t st);

}  // namespace gnk
