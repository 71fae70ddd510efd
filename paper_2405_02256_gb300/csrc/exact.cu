// Exact representations of the ECT and of the Radon transform, and their evaluation
// at arbitrary thresholds (Section 4.3; Appendix A.2 computation, A.3 evaluation).
//
// For one image and one direction xi (eps = eps^xi):
//   kind 0: (T, E) of t -> ECT(xi, t).  T holds the distinct dot products s_v = <xi, x(v)>
//           of the points of the lower table Delta^-_eps, ascending; E the cumulative sums
//           of their values with equal dot products merged.  ECT(xi, t) = E at the largest
//           T <= t (0 if none).
//   kind 1: (T', E') built the same way from the table Delta_eps (the stored partner's
//           table with the sign flipped when eps is outside the stored half).  With the
//           level set split as for the grid Radon transform (sum_v Delta^-_{-eps} = chi),
//             R(xi, t) = sum_{s_v < t} Delta_eps(v) + sum_{s_v = t} Delta^-_eps(v),
//           i.e. E' at the largest T' < t plus the jump of E at t.
//
// Steps, per (image, direction) segment, all on the device:
//   keys   : s_v exactly as the canonical FP64 dot product (one rounding per product and
//            per sum, left to right), -0 turned into +0, mapped to an unsigned 64-bit key
//            whose order is the order of the doubles;
//   sort   : 2048-entry tiles sorted by a bitonic network in shared memory, then merge
//            passes that double the sorted run length: every entry finds its place in
//            the partner run by binary search (entries of the left run go before equal
//            keys of the right run, so the two runs interleave into one sorted run);
//   finish : one block per segment scans the sorted run; a tie group ends where the key
//            changes, and its end writes T and the running sum E;
//   eval   : one binary search per (segment, query).
#include <algorithm>

#include "internal.cuh"

namespace topot {

constexpr int kSortTile = 2048;
constexpr int kSortThreads = 512;
constexpr int kFinishThreads = 1024;

__device__ __forceinline__ unsigned long long order_key(double s) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(s);
    return (u >> 63) ? ~u : (u | (1ull << 63));
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}

template <int NDIM, typename Tval>
__global__ void __launch_bounds__(256) k_exact_keys(ExactArgs a) {
    constexpr int NO = 1 << NDIM;
    const TablesDev& T = a.t;
    for (int seg = blockIdx.y; seg < a.nseg; seg += gridDim.y) {
        const int b = seg / a.D, d = seg - b * a.D;
        const double* xi = a.dirs + ((long long)(a.per_image ? b * a.D : 0) + d) * NDIM;
        double x[NDIM];
        int o = 0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            x[k] = xi[k];
            if (x[k] < 0.0) o |= 1 << k;           // eps_k = -1 only for a negative coordinate
        }
        int tab = o, sg = 1;
        if (a.kind == 1) {
            int r = o;
            if (o >= NO / 2) {
                r = o ^ (NO - 1);
                sg = -1;
            }
            tab = NO + r;
        }
        const ImgDesc& I = T.img[b];
        const long long n = T.seg_count[(long long)b * T.S + tab];
        const long long base = I.seg_base + (long long)tab * I.N;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[seg] = (int)n;
        unsigned long long* K = a.key[0] + (long long)seg * a.cap;
        int* V = a.val[0] + (long long)seg * a.cap;
        const int* ai = T.arena_idx + base;
        const Tval* av = reinterpret_cast<const Tval*>(T.arena_val) + base;
        const int m0 = I.m[0], m1 = I.m[1], m2 = I.m[2], m3 = I.m[3];
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const uint32_t idx = (uint32_t)ai[i];
            int c[4];
            if (NDIM == 4) {   // generic-n tables: plain division
                uint32_t r = idx;
                c[0] = (int)(r % (uint32_t)m0);
                r /= (uint32_t)m0;
                c[1] = (int)(r % (uint32_t)m1);
                r /= (uint32_t)m1;
                c[2] = (int)(r % (uint32_t)m2);
                c[3] = (int)(r / (uint32_t)m2);
            } else {
                const uint32_t q1 = fastdiv(idx, I.div0);
                c[0] = (int)(idx - q1 * (uint32_t)m0);
                if (NDIM == 2) {
                    c[1] = (int)q1;
                } else {
                    const uint32_t q2 = fastdiv(q1, I.div1);
                    c[1] = (int)(q1 - q2 * (uint32_t)m1);
                    c[2] = (int)q2;
                }
            }
            const int mm[4] = {m0, m1, m2, m3};
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NDIM; ++k) {
                const double xk = __ddiv_rn((double)(2 * c[k] - (mm[k] - 1)), (double)(2 * (mm[k] - 1)));
                const double pk = __dmul_rn(x[k], xk);
                s = k == 0 ? pk : __dadd_rn(s, pk);
            }
            s = __dadd_rn(s, 0.0);                  // -0 -> +0: one key per value
            K[i] = order_key(s);
            V[i] = sg * (int)av[i];
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_exact_sort_tiles(ExactArgs a) {
    __shared__ unsigned long long sk[kSortTile];
    __shared__ int sv[kSortTile];
    const int tid = threadIdx.x;
    for (int seg = blockIdx.y; seg < a.nseg; seg += gridDim.y) {
        const int n = a.cnt[seg];
        unsigned long long* K = a.key[0] + (long long)seg * a.cap;
        int* V = a.val[0] + (long long)seg * a.cap;
        for (int start = blockIdx.x * kSortTile; start < n; start += gridDim.x * kSortTile) {
            const int m = min(kSortTile, n - start);
            for (int i = tid; i < kSortTile; i += kSortThreads) {
                sk[i] = i < m ? K[start + i] : ~0ull;
                sv[i] = i < m ? V[start + i] : 0;
            }
            __syncthreads();
            for (int k = 2; k <= kSortTile; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = tid; i < kSortTile; i += kSortThreads) {
                        const int p = i ^ j;
                        if (p > i) {
                            const bool up = (i & k) == 0;
                            const unsigned long long ki = sk[i], kp = sk[p];
                            if ((ki > kp) == up) {
                                sk[i] = kp;
                                sk[p] = ki;
                                const int t = sv[i];
                                sv[i] = sv[p];
                                sv[p] = t;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int i = tid; i < m; i += kSortThreads) {
                K[start + i] = sk[i];
                V[start + i] = sv[i];
            }
            __syncthreads();
        }
    }
}

// number of keys in [lo, hi) that are < key (strict) or <= key
template <bool STRICT>
__device__ __forceinline__ long long count_below(const unsigned long long* K, long long lo, long long hi,
                                                 unsigned long long key) {
    const long long first = lo;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const unsigned long long km = K[mid];
        if (STRICT ? (km < key) : (km <= key)) lo = mid + 1;
        else hi = mid;
    }
    return lo - first;
}

__global__ void __launch_bounds__(256) k_exact_merge(ExactArgs a, int src, long long w) {
    for (int seg = blockIdx.y; seg < a.nseg; seg += gridDim.y) {
        const long long n = a.cnt[seg];
        const unsigned long long* K = a.key[src] + (long long)seg * a.cap;
        const int* V = a.val[src] + (long long)seg * a.cap;
        unsigned long long* K2 = a.key[src ^ 1] + (long long)seg * a.cap;
        int* V2 = a.val[src ^ 1] + (long long)seg * a.cap;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const long long r = i / w, run = r * w;
            const unsigned long long key = K[i];
            long long out;
            if ((r & 1) == 0) {                     // left run; right run may be short or empty
                const long long bs = min(run + w, n), be = min(run + 2 * w, n);
                out = i + count_below<true>(K, bs, be, key);
            } else {                                // right run: after equal keys of the left run
                const long long as = run - w;
                out = as + (i - run) + count_below<false>(K, as, run, key);
            }
            K2[out] = key;
            V2[out] = V[i];
        }
    }
}

__global__ void __launch_bounds__(kFinishThreads) k_exact_finish(ExactArgs a, int src) {
    constexpr int NW = kFinishThreads / 32;
    __shared__ long long w_sum[NW];
    __shared__ int w_cnt[NW];
    __shared__ long long carry_sum;
    __shared__ int carry_cnt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int seg = blockIdx.x; seg < a.nseg; seg += gridDim.x) {
        const int n = a.cnt[seg];
        const unsigned long long* K = a.key[src] + (long long)seg * a.cap;
        const int* V = a.val[src] + (long long)seg * a.cap;
        double* To = a.T + (long long)seg * a.cap;
        int32_t* Eo = a.E + (long long)seg * a.cap;
        if (tid == 0) {
            carry_sum = 0;
            carry_cnt = 0;
        }
        __syncthreads();
        for (int base = 0; base < n; base += kFinishThreads) {
            const int i = base + tid;
            const bool valid = i < n;
            const unsigned long long key = valid ? K[i] : 0ull;
            long long sv = valid ? V[i] : 0;
            int ce = (valid && (i + 1 == n || K[i + 1] != key)) ? 1 : 0;
            const bool end = ce != 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long ys = __shfl_up_sync(0xffffffffu, sv, d);
                const int yc = __shfl_up_sync(0xffffffffu, ce, d);
                if (lane >= d) {
                    sv += ys;
                    ce += yc;
                }
            }
            if (lane == 31) {
                w_sum[warp] = sv;
                w_cnt[warp] = ce;
            }
            __syncthreads();
            if (warp == 0) {
                long long xs = w_sum[lane];
                int xc = w_cnt[lane];
                const long long xs0 = xs;
                const int xc0 = xc;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const long long ys = __shfl_up_sync(0xffffffffu, xs, d);
                    const int yc = __shfl_up_sync(0xffffffffu, xc, d);
                    if (lane >= d) {
                        xs += ys;
                        xc += yc;
                    }
                }
                w_sum[lane] = xs - xs0;              // exclusive over warps
                w_cnt[lane] = xc - xc0;
            }
            __syncthreads();
            const long long run_sum = carry_sum + w_sum[warp] + sv;
            const int run_cnt = carry_cnt + w_cnt[warp] + ce;
            if (end) {
                To[run_cnt - 1] = key_value(key);
                Eo[run_cnt - 1] = (int32_t)run_sum;
            }
            __syncthreads();                         // every thread has read the carries
            if (tid == kFinishThreads - 1) {
                carry_sum = run_sum;
                carry_cnt = run_cnt;
            }
            __syncthreads();
        }
        if (tid == 0) a.len[seg] = carry_cnt;
        __syncthreads();
    }
}

__global__ void k_ect_exact_eval(int nseg, long long cap, const double* T, const int32_t* E, const long long* len,
                                 const double* t, int Q, int32_t* out) {
    const long long total = (long long)nseg * Q;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long seg = k / Q;
        const double tq = t[k - seg * Q];
        const double* Ts = T + seg * cap;
        long long lo = 0, hi = len[seg];
        while (lo < hi) {                           // number of T <= t
            const long long mid = (lo + hi) >> 1;
            if (Ts[mid] <= tq) lo = mid + 1;
            else hi = mid;
        }
        out[k] = lo > 0 ? E[seg * cap + lo - 1] : 0;
    }
}

__device__ __forceinline__ long long count_le(const double* Ts, long long L, double t, bool strict) {
    long long lo = 0, hi = L;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (strict ? (Ts[mid] < t) : (Ts[mid] <= t)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_radon_exact_eval(int nseg, long long cap, const double* Tl, const int32_t* El,
                                   const long long* lenl, long long cap_o, const double* To, const int32_t* Eo,
                                   const long long* leno, const double* t, int Q, int32_t* out) {
    const long long total = (long long)nseg * Q;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long seg = k / Q;
        const double tq = t[k - seg * Q];
        const long long off = seg * cap, off_o = seg * cap_o;
        const long long nb = count_le(To + off_o, leno[seg], tq, true);      // T' < t
        const long long kle = count_le(Tl + off, lenl[seg], tq, false);      // T <= t
        const long long klt = count_le(Tl + off, lenl[seg], tq, true);       // T < t
        const int32_t below = nb > 0 ? Eo[off_o + nb - 1] : 0;
        const int32_t e_le = kle > 0 ? El[off + kle - 1] : 0;
        const int32_t e_lt = klt > 0 ? El[off + klt - 1] : 0;
        out[k] = below + (e_le - e_lt);
    }
}

// ---- host side ------------------------------------------------------------------------------

static unsigned grid_1d(long long work, int threads, int cap_blocks) {
    long long g = (work + threads - 1) / threads;
    return (unsigned)std::max(1ll, std::min(g, (long long)cap_blocks));
}

cudaError_t launch_exact(int n, bool u8, ExactArgs a, long long max_n, int sm_count, cudaStream_t st) {
    const unsigned gy = (unsigned)std::min(a.nseg, 65535);
    const int per_seg_blocks = std::max(1, std::min(4 * sm_count, 65535) / (int)gy);
    dim3 gk(grid_1d(max_n, 256, per_seg_blocks), gy);
    if (n == 2) {
        if (u8) k_exact_keys<2, int16_t><<<gk, 256, 0, st>>>(a);
        else k_exact_keys<2, int32_t><<<gk, 256, 0, st>>>(a);
    } else if (n == 3) {
        if (u8) k_exact_keys<3, int16_t><<<gk, 256, 0, st>>>(a);
        else k_exact_keys<3, int32_t><<<gk, 256, 0, st>>>(a);
    } else {
        if (u8) k_exact_keys<4, int16_t><<<gk, 256, 0, st>>>(a);
        else k_exact_keys<4, int32_t><<<gk, 256, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gs(grid_1d(max_n, kSortTile, per_seg_blocks), gy);
    k_exact_sort_tiles<<<gs, kSortThreads, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int src = 0;
    for (long long w = kSortTile; w < max_n; w *= 2) {
        k_exact_merge<<<gk, 256, 0, st>>>(a, src, w);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        src ^= 1;
    }
    k_exact_finish<<<(unsigned)std::min(a.nseg, 8 * sm_count), kFinishThreads, 0, st>>>(a, src);
    return cudaGetLastError();
}

cudaError_t launch_ect_exact_eval(int nseg, long long cap, const double* T, const int32_t* E, const long long* len,
                                  const double* t, int Q, int32_t* out, int sm_count, cudaStream_t st) {
    k_ect_exact_eval<<<grid_1d((long long)nseg * Q, 256, 16 * sm_count), 256, 0, st>>>(nseg, cap, T, E, len, t, Q,
                                                                                        out);
    return cudaGetLastError();
}

cudaError_t launch_radon_exact_eval(int nseg, long long cap, const double* Tl, const int32_t* El,
                                    const long long* lenl, long long cap_o, const double* To, const int32_t* Eo,
                                    const long long* leno, const double* t, int Q, int32_t* out, int sm_count,
                                    cudaStream_t st) {
    k_radon_exact_eval<<<grid_1d((long long)nseg * Q, 256, 16 * sm_count), 256, 0, st>>>(
        nseg, cap, Tl, El, lenl, cap_o, To, Eo, leno, t, Q, out);
    return cudaGetLastError();
}

}  // namespace topot
