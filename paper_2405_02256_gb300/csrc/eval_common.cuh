// Work planning shared by the evaluation kernels (ECT, Radon, hybrid transform and
// its adjoint).
//
// A "pair" is (image b, orthant o) -- for the Radon transform (b, o, part) with part 0
// the sublevel histogram on table o and part 1 the superlevel histogram on table
// o ^ (2^n - 1).  The directions of a pair are the directions of b's direction set
// whose sign vector is o (grouped by dir_prep).  A work item is (pair, tile of
// directions, chunk of the pair's critical table); items are numbered pair by pair,
// tile-major, so that partial results of one direction are laid out in chunk order.
#pragma once

#include "internal.cuh"

namespace topot {

enum EvalMode : int { kModeECT = 0, kModeRadon = 1, kModeHT = 2 };

struct EvalPlan {
    int mode;
    int nsets;                 // 1 (shared directions) or B
    int D;                     // directions per set
    int tile_dirs;             // directions per work item
    int chunk_req;             // requested critical points per item (0 = automatic)
    int target_items;          // automatic chunking aims at about this many items
    int npairs;
    long long max_items;       // capacity of the per-item partial buffers
    const double* dirs;        // [nsets][D][n]
    int* perm;                 // [nsets][D]: direction ids grouped by orthant
    int* rank;                 // [nsets][D]: position of each direction in its group
    int* boff;                 // [nsets][NO + 1]: group offsets
    long long* pair_items;     // [npairs + 1]: exclusive prefix of items
    int* item_pair;            // [max_items]: the pair of every item (written by the planner)
    int* wide_items;           // [max_items]: hybrid FP32C items for the wide-range launch
    int* pair_chunks;          // [npairs]
    int* ctl;                  // [0] item counter, [1] chunk, [2] number of items,
                               // [3] wide-range item counter, [4] wide-range items
    double* thr;               // [T] thresholds (ECT / Radon)
    int T;
    double t_min, t_max;
    // tabulated kernel (hybrid transform with TOPOT_TABLE): K samples of kbar on
    // a + i h; K + 1 padded FP32 pairs (ends (y_0, 0), (y_{K-1}, 0); segment r:
    // (y_r + d_r / 2, d_r)) and the FP64 samples
    const float2* ktab;
    const double* ktab64;
    int ktab_k;
    double ktab_a, ktab_h;
};

__device__ __forceinline__ int orthant_of(const double* xi, int n) {
    int o = 0;
    for (int k = 0; k < n; ++k)
        if (xi[k] < 0.0) o |= 1 << k;   // zero (and -0.0) -> eps_k = +1
    return o;
}

// Pair -> (image, orthant, part).  Hybrid transforms pair an image with a representative
// orthant r < 2^(n-1): the directions of r and of its partner r ^ (2^n - 1) evaluate the
// same Delta table (Delta_{-eps} = -Delta_eps, the sign applied per direction at the
// combine), so they share tiles.
__device__ __forceinline__ void decode_pair(int mode, int NO, int p, int& b, int& o, int& part) {
    part = 0;
    if (mode == kModeHT) {
        b = p / (NO / 2);
        o = p - b * (NO / 2);
        return;
    }
    if (mode == kModeRadon) {
        part = p & 1;
        p >>= 1;
    }
    b = p / NO;
    o = p - b * NO;
}

// Direction group of a direction: its orthant, or for hybrid transforms the
// representative of its orthant's pair.
__device__ __forceinline__ int dir_group(const double* xi, int n, int mode) {
    const int o = orthant_of(xi, n);
    const int NO = 1 << n;
    return (mode == kModeHT && (o & (NO >> 1))) ? (o ^ (NO - 1)) : o;
}

// Segment (table) used by a pair, and the sign applied to its values.
__device__ __forceinline__ int pair_segment(int mode, int NO, int o, int part, int& sign) {
    sign = 1;
    if (mode == kModeECT) return o;
    if (mode == kModeRadon) return part ? (o ^ (NO - 1)) : o;
    // hybrid: representative orthants have bit n-1 clear; the partner's table is -Delta
    if (o & (NO >> 1)) {
        sign = -1;
        return NO + (o ^ (NO - 1));
    }
    return NO + o;
}

// Item -> (pair, tile, chunk): the pair from the planner's map (one load, where a binary
// search over tens of thousands of pairs of a ragged batch took a chain of dependent loads).
__device__ __forceinline__ void decode_item(const EvalPlan& P, long long item, int& pair, int& tile,
                                            int& chunk) {
    const int lo = P.item_pair[item];
    pair = lo;
    const long long local = item - P.pair_items[lo];
    const int nch = P.pair_chunks[lo];
    tile = (int)(local / nch);
    chunk = (int)(local - (long long)tile * nch);
}

// Tabulated kernel in FP64: the piecewise-linear interpolant of the samples (constant
// outside [a, b]) and its slope (zero outside [a, b)), as kernel_table_create states them.
__device__ __forceinline__ double table_kbar64(const EvalPlan& P, double s) {
    const double u = __ddiv_rn(__dsub_rn(s, P.ktab_a), P.ktab_h);
    const int K = P.ktab_k;
    if (u < 0.0) return P.ktab64[0];
    if (!(u < (double)(K - 1))) return P.ktab64[K - 1];
    const double fi = floor(u);
    const int i = (int)fi;
    const double y0 = P.ktab64[i];
    return __dadd_rn(y0, __dmul_rn(__dsub_rn(u, fi), __dsub_rn(P.ktab64[i + 1], y0)));
}

__device__ __forceinline__ double table_kappa64(const EvalPlan& P, double s) {
    const double u = __ddiv_rn(__dsub_rn(s, P.ktab_a), P.ktab_h);
    if (!(u >= 0.0 && u < (double)(P.ktab_k - 1))) return 0.0;
    const int i = (int)floor(u);
    return __ddiv_rn(__dsub_rn(P.ktab64[i + 1], P.ktab64[i]), P.ktab_h);
}

cudaError_t launch_dir_prep(const EvalPlan& P, int n, cudaStream_t st);
cudaError_t launch_plan(const EvalPlan& P, const TablesDev& t, cudaStream_t st);

}  // namespace topot
