// Direction preparation (sign vectors, Section 3) and device-side work planning for
// the evaluation kernels.  Both run on the stream, so that an evaluation needs no
// host synchronisation and can be captured in a CUDA graph.
#include "eval_common.cuh"

namespace topot {

// One block per direction set: stable counting sort of the directions by group (orthant;
// for hybrid transforms the representative of the orthant's pair).
template <int NO>
__global__ void __launch_bounds__(1024) k_dir_prep(EvalPlan P, int n) {
    constexpr int NW = 1024 / 32;
    __shared__ int cnt[NO];
    __shared__ int base[NO];
    __shared__ int wcnt[NW][NO];
    const int set = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double* dirs = P.dirs + (long long)set * P.D * n;
    if (tid < NO) cnt[tid] = 0;
    __syncthreads();
    for (int d = tid; d < P.D; d += 1024) atomicAdd(&cnt[dir_group(dirs + (long long)d * n, n, P.mode)], 1);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        int* bo = P.boff + (long long)set * (NO + 1);
        for (int o = 0; o < NO; ++o) {
            bo[o] = run;
            base[o] = run;
            run += cnt[o];
        }
        bo[NO] = run;
    }
    __syncthreads();
    int* perm = P.perm + (long long)set * P.D;
    for (int d0 = 0; d0 < P.D; d0 += 1024) {
        const int d = d0 + tid;
        const int o = d < P.D ? dir_group(dirs + (long long)d * n, n, P.mode) : -1;
        int myrank = 0;
#pragma unroll
        for (int q = 0; q < NO; ++q) {
            const unsigned bal = __ballot_sync(0xffffffffu, o == q);
            if (o == q) myrank = __popc(bal & lanemask_lt());
            if (lane == 0) wcnt[warp][q] = __popc(bal);
        }
        __syncthreads();
        if (tid < NO) {
            int run = 0;
            for (int w = 0; w < NW; ++w) {
                const int c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            cnt[tid] = run;   // this round's total for orthant tid
        }
        __syncthreads();
        if (o >= 0) {
            const int pos = base[o] + wcnt[warp][o] + myrank;
            perm[pos] = d;
            P.rank[(long long)set * P.D + d] = pos - P.boff[(long long)set * (NO + 1) + o];
        }
        __syncthreads();
        if (tid < NO) base[tid] += cnt[tid];
        __syncthreads();
    }
}

// Hybrid transforms: directions are grouped by the representative of their orthant's
// pair (orthant and partner share a Delta table), and within a group ordered by M = sum_k |xi_k|
// (ties by direction id), so that a tile of 32 DL consecutive directions spans a narrow
// range of |<xi, v>| and its polynomial degree (chosen per tile from the largest M) stays
// low.  One block per direction set sorts the keys
//   orthant (4 bits) | FP32 bits of M (order-preserving for M >= 0) | direction id (28 bits)
// with a bitonic network in shared memory; sets of more than kSortDirsMax directions keep
// the plain orthant grouping.
constexpr int kSortDirsMax = 8192;

__global__ void __launch_bounds__(1024) k_dir_sort(EvalPlan P, int n) {
    extern __shared__ unsigned long long key[];
    __shared__ int cnt[16];
    const int set = blockIdx.x;
    const int tid = threadIdx.x;
    const int NO = 1 << n;
    const double* dirs = P.dirs + (long long)set * P.D * n;
    int L = 1;
    while (L < P.D) L <<= 1;
    if (tid < 16) cnt[tid] = 0;
    __syncthreads();
    for (int d = tid; d < L; d += 1024) {
        unsigned long long k = ~0ull;   // padding sorts last
        if (d < P.D) {
            const double* xi = dirs + (long long)d * n;
            double m = 0.0;
            for (int c = 0; c < n; ++c) m += fabs(xi[c]);
            const int o = dir_group(xi, n, P.mode);
            atomicAdd(&cnt[o], 1);
            k = ((unsigned long long)o << 60) | ((unsigned long long)__float_as_uint((float)m) << 28) |
                (unsigned long long)d;
        }
        key[d] = k;
    }
    __syncthreads();
    for (int size = 2; size <= L; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < L / 2; i += 1024) {
                const int lo = 2 * i - (i & (stride - 1));   // pairs (lo, lo + stride)
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    int* bo = P.boff + (long long)set * (NO + 1);
    if (tid == 0) {
        int run = 0;
        for (int o = 0; o < NO; ++o) {
            bo[o] = run;
            run += cnt[o];
        }
        bo[NO] = run;
    }
    __syncthreads();
    int* perm = P.perm + (long long)set * P.D;
    for (int i = tid; i < P.D; i += 1024) {
        const unsigned long long k = key[i];
        const int d = (int)(k & ((1ull << 28) - 1));
        const int o = (int)(k >> 60);
        perm[i] = d;
        P.rank[(long long)set * P.D + d] = i - bo[o];
    }
}

cudaError_t launch_dir_prep(const EvalPlan& P, int n, cudaStream_t st) {
    if (P.mode == kModeHT && P.D <= kSortDirsMax) {
        static const cudaError_t attr = cudaFuncSetAttribute(k_dir_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                             (int)(sizeof(unsigned long long) * kSortDirsMax));
        if (attr != cudaSuccess) return attr;
        int L = 1;
        while (L < P.D) L <<= 1;
        k_dir_sort<<<P.nsets, 1024, sizeof(unsigned long long) * L, st>>>(P, n);
        return cudaGetLastError();
    }
    if (n == 2) k_dir_prep<4><<<P.nsets, 1024, 0, st>>>(P, n);
    else if (n == 3) k_dir_prep<8><<<P.nsets, 1024, 0, st>>>(P, n);
    else k_dir_prep<16><<<P.nsets, 1024, 0, st>>>(P, n);
    return cudaGetLastError();
}

// Single-block planner: items per pair, chunk size, exclusive prefix, thresholds.
__global__ void __launch_bounds__(1024) k_plan(EvalPlan P, TablesDev t) {
    __shared__ unsigned long long red[32];
    __shared__ long long carry;
    __shared__ int chunk_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NO = 1 << t.n;

    // thresholds t_j = fl(a + fl(fl(j fl(b - a)) / (T - 1)))  (Appendix A.4)
    if (P.thr) {
        const double w = __dsub_rn(P.t_max, P.t_min);
        for (int j = tid; j < P.T; j += 1024)
            P.thr[j] = __dadd_rn(P.t_min, __ddiv_rn(__dmul_rn((double)j, w), (double)(P.T - 1)));
    }

    auto pair_info = [&](int p, long long& tiles, long long& N) {
        int b, o, part, sign;
        decode_pair(P.mode, NO, p, b, o, part);
        const int set = P.nsets == 1 ? 0 : b;
        const int* bo = P.boff + (long long)set * (NO + 1);
        const int nd = bo[o + 1] - bo[o];
        tiles = (nd + P.tile_dirs - 1) / P.tile_dirs;
        const int seg = pair_segment(P.mode, NO, o, part, sign);
        N = t.seg_count[(long long)b * t.S + seg];
    };

    // total work (directions x critical points) for automatic chunking; overflow guard
    unsigned long long work = 0;
    for (int p = tid; p < P.npairs; p += 1024) {
        long long tiles, N;
        pair_info(p, tiles, N);
        work += (unsigned long long)(tiles * P.tile_dirs) * (unsigned long long)N;
    }
    // int32 outputs: |ECT| <= sum_v |Delta^-_o|; |R| <= |ECT(xi)| + |ECT(-xi)| + |chi| <= 3 max_o of it
    // (intermediate int32 sums may wrap: only the final values must fit)
    const long long lim = P.mode == kModeRadon ? (1ll << 31) / 3 : (1ll << 31);
    for (int i = tid; i < t.B * NO; i += 1024)
        if (P.mode != kModeHT && t.absum[i] >= lim) dev_set_error(t.err, kDevErrOverflow);
    work = warp_sum(work);
    if (lane == 0) red[warp] = work;
    __syncthreads();
    if (tid == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < 32; ++w) tot += red[w];
        int chunk = P.chunk_req;
        if (chunk <= 0) {
            const unsigned long long per = tot / ((unsigned long long)P.tile_dirs * P.target_items) + 1;
            long long c = (long long)((per + 255) / 256) * 256;
            c = c < 1024 ? 1024 : c;
            c = c > (1 << 30) ? (1 << 30) : c;
            chunk = (int)c;
        }
        chunk_sh = chunk;
        carry = 0;
        P.ctl[0] = 0;   // item counter
        P.ctl[1] = chunk;
        P.ctl[3] = 0;   // hybrid transforms: wide-range items taken, and set aside
        P.ctl[4] = 0;
    }
    __syncthreads();
    const int chunk = chunk_sh;

    // exclusive prefix of items over pairs, 1024 pairs per round
    for (int p0 = 0; p0 < P.npairs; p0 += 1024) {
        const int p = p0 + tid;
        long long items = 0;
        if (p < P.npairs) {
            long long tiles, N;
            pair_info(p, tiles, N);
            const long long nch = (N + chunk - 1) / chunk;
            items = tiles * nch;
            P.pair_chunks[p] = (int)(nch > 0 ? nch : 1);
            if (nch == 0) items = 0;
        }
        // block inclusive scan of items
        long long v = items;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) red[warp] = (unsigned long long)v;
        __syncthreads();
        if (warp == 0) {
            long long w = (long long)red[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            red[lane] = (unsigned long long)w;   // inclusive over warps
        }
        __syncthreads();
        const long long excl = carry + (warp ? (long long)red[warp - 1] : 0) + v - items;
        if (p < P.npairs) {
            P.pair_items[p] = excl;
            // item -> pair map (items past the buffers' bound are never run)
            for (long long i = excl; i < excl + items && i < P.max_items; ++i) P.item_pair[i] = p;
        }
        __syncthreads();
        if (tid == 0) carry += (long long)red[31];
        __syncthreads();
    }
    if (tid == 0) {
        P.pair_items[P.npairs] = carry;
        // never run more items than the buffers hold (cannot happen with the host's
        // bound; recorded as an error if it ever does)
        if (carry > P.max_items) dev_set_error(t.err, kDevErrOverflow);
        P.ctl[2] = (int)(carry > P.max_items ? P.max_items : carry);
    }
}

cudaError_t launch_plan(const EvalPlan& P, const TablesDev& t, cudaStream_t st) {
    k_plan<<<1, 1024, 0, st>>>(P, t);
    return cudaGetLastError();
}

}  // namespace topot
