// Generic-n path (n = 4): plain kernels for every step of the method on n-dimensional
// cubical complexes (Section 2.1 states the method for any n; Section 3 uses the 2^n sign
// vectors).  The 2-D and 3-D kernels are specialised (FP32 lattice arithmetic with exact
// filters, packed pairs, staged strips); these favour plainness over speed.
//
// Tables (Section 3, Delta^-; Section 4.2): one thread per vertex.  The 3^n neighbourhood
// is read into registers as phi + C (C = 1 for 8-bit pixels, 2^26 for int32 pixels, so
// that every pixel is > 0) with 0 for "outside the image".  A box of the lower star of v
// spans, per axis k, {i_k} or two neighbouring indices, so its minimum is one of 3^n
// "box minima", obtained by one min-sweep per axis; a box leaving the image has minimum
// 0 and adds nothing.  Delta^-_o(v) = sum over delta of (-1)^|delta| (min - C) over the
// boxes v .. v - delta (.) eps_o.  The tables are compacted in ascending vertex order by
// three passes: per-block counts, an exclusive scan of the counts per (image, table), and
// the write (warp ballots and a block scan within a block).
//
// ECT / Radon (Lemma 3.1; additivity): per (point, direction) the canonical FP64 dot
// product (the oracle's left-to-right rounding) and the exact bin by binary search over
// the FP64 thresholds, added with global integer atomics; k_hist_finish scans.
//
// Hybrid transforms and adjoint (Lemma 3.1): one direction per lane; FP32C forms the
// argument in FP64 and the term in FP32 as the 2-D / 3-D scalar path does beyond its
// FP32 range (kbar(s) - kbar(0) with half-angle sin / cos, Laplace rescaled per round);
// FP64 uses the library FP64 functions.  Partials use the layout of the other kernels,
// so the same combine kernels finish.
#include <algorithm>

#include "eval_common.cuh"

namespace topot {

constexpr int kGenBlock = 256;
constexpr int kGenN = 4;

__host__ __device__ constexpr int pow3(int n) { return n == 0 ? 1 : 3 * pow3(n - 1); }

template <typename Tin>
struct GenPix {
    // offset making every pixel positive; 0 marks a vertex outside the image
    static constexpr int C = sizeof(Tin) == 1 ? 1 : (1 << 26);
};

// int32 pixels: |phi| < 2^25 keeps |Delta^-| <= 2^(n-1) 2^26 = 2^29 and |Delta| <= 2^30 in
// int32 for n = 4 (the 2-D / 3-D kernels allow 2^26)
constexpr long long kGenPixLimit = 1ll << 25;

// Decode a linear vertex index (coordinate 0 fastest).
template <int NDIM>
__device__ __forceinline__ void gen_decode(long long idx, const int* m, int (&i)[NDIM]) {
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        i[k] = (int)(idx % m[k]);
        idx /= m[k];
    }
}

// Delta^-_o(v) for every orthant o of vertex i; *bad set when an int32 pixel is out of range.
template <int NDIM, typename Tin>
__device__ __forceinline__ void gen_lower_star(const Tin* img, const int* m, const int (&i)[NDIM],
                                               long long (&low)[1 << NDIM], bool& bad) {
    constexpr int K = pow3(NDIM);
    constexpr int C = GenPix<Tin>::C;
    int bx[K];   // neighbourhood, then box minima; digit k of the index: axis-k choice
#pragma unroll
    for (int q = 0; q < K; ++q) {
        int rem = q;
        long long lin = 0, stride = 1;
        bool inside = true;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            const int d = rem % 3 - 1;   // -1, 0, +1
            rem /= 3;
            const int c = i[k] + d;
            inside &= c >= 0 && c < m[k];
            lin += (long long)c * stride;
            stride *= m[k];
        }
        int v = 0;
        if (inside) {
            long long p = (long long)img[lin];
            if (sizeof(Tin) == 4 && (p >= kGenPixLimit || p <= -kGenPixLimit)) {
                bad = true;
                p = 0;
            }
            v = (int)p + C;
        }
        bx[q] = v;
    }
    // sweep axis by axis: digit (d = -1, 0, +1) becomes (c = {0}, {-1, 0}, {0, +1})
    int stride = 1;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if ((q / stride) % 3 != 0) continue;   // one line per (other digits)
            const int a = bx[q], b = bx[q + stride], c = bx[q + 2 * stride];
            bx[q] = b;
            bx[q + stride] = min(a, b);
            bx[q + 2 * stride] = min(b, c);
        }
        stride *= 3;
    }
    // signed terms: (-1)^(#axes spanned) (min - C), 0 for a box leaving the image
#pragma unroll
    for (int q = 0; q < K; ++q) {
        int rem = q, span = 0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            span += rem % 3 != 0;
            rem /= 3;
        }
        const int t = bx[q] > 0 ? bx[q] - C : 0;
        bx[q] = (span & 1) ? -t : t;
    }
#pragma unroll
    for (int o = 0; o < (1 << NDIM); ++o) {
        long long s = 0;
#pragma unroll
        for (int dl = 0; dl < (1 << NDIM); ++dl) {
            int q = 0, p3 = 1;
#pragma unroll
            for (int k = 0; k < NDIM; ++k) {
                // delta_k = 0: {i_k}; delta_k = 1: towards -eps_k: eps = +1 -> {i-1, i}, -1 -> {i, i+1}
                const int c = ((dl >> k) & 1) ? (((o >> k) & 1) ? 2 : 1) : 0;
                q += c * p3;
                p3 *= 3;
            }
            s += bx[q];
        }
        low[o] = s;
    }
}

// Block -> image by binary search over the images' first blocks.
__device__ __forceinline__ int gen_image(const TablesDev& T, long long blk) {
    int lo = 0, hi = T.B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.img[mid].tile_begin <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int NDIM>
__device__ __forceinline__ void gen_segments(const long long (&low)[1 << NDIM], long long (&val)[(1 << NDIM) * 3 / 2]) {
    constexpr int NO = 1 << NDIM;
#pragma unroll
    for (int o = 0; o < NO; ++o) val[o] = low[o];
#pragma unroll
    for (int r = 0; r < NO / 2; ++r) val[NO + r] = low[r] - low[r ^ (NO - 1)];
}

// Pass 1: per block and table, the number of non-zero values; chi and sum |Delta^-_o|.
template <int NDIM, typename Tin>
__global__ void __launch_bounds__(kGenBlock) k_gen_count(TablesDev T, const Tin* pixels, long long* cnt) {
    constexpr int NO = 1 << NDIM, S = NO * 3 / 2;
    __shared__ int wc[kGenBlock / 32][S];
    __shared__ long long wl[kGenBlock / 32][NO + 1];
    const long long blk = blockIdx.x;
    const int b = gen_image(T, blk);
    const ImgDesc& I = T.img[b];
    const long long v = (blk - I.tile_begin) * kGenBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long val[S];
#pragma unroll
    for (int s = 0; s < S; ++s) val[s] = 0;
    if (v < I.N) {
        int i[NDIM];
        gen_decode<NDIM>(v, I.m, i);
        long long low[NO];
        bool bad = false;
        gen_lower_star<NDIM, Tin>(pixels + I.offset, I.m, i, low, bad);
        if (bad) dev_set_error(T.err, kDevErrOverflow);
        gen_segments<NDIM>(low, val);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int c = __popc(__ballot_sync(0xffffffffu, val[s] != 0));
        if (lane == 0) wc[warp][s] = c;
    }
    // chi = sum Delta^-_0 and sum |Delta^-_o| (64-bit)
    long long acc[NO + 1];
    acc[0] = val[0];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[1 + o] = val[o] < 0 ? -val[o] : val[o];
#pragma unroll
    for (int q = 0; q <= NO; ++q) {
        long long x = acc[q];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0) wl[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < S) {
        long long c = 0;
        for (int w = 0; w < kGenBlock / 32; ++w) c += wc[w][threadIdx.x];
        cnt[blk * S + threadIdx.x] = c;
    }
    if (threadIdx.x <= NO) {
        long long x = 0;
        for (int w = 0; w < kGenBlock / 32; ++w) x += wl[w][threadIdx.x];
        if (x != 0) {
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(
                threadIdx.x == 0 ? &T.chi[b] : &T.absum[(long long)b * NO + threadIdx.x - 1]);
            atomicAdd(dst, (unsigned long long)x);
        }
    }
}

// Pass 2: per (image, table), exclusive scan of the block counts (in place) and the size.
__global__ void __launch_bounds__(1024) k_gen_scan(TablesDev T, long long* cnt) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int b = blockIdx.x / T.S, s = blockIdx.x - b * T.S;
    const ImgDesc& I = T.img[b];
    const long long nblk = (I.N + kGenBlock - 1) / kGenBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long j0 = 0; j0 < nblk; j0 += 1024) {
        const long long j = j0 + threadIdx.x;
        long long* p = cnt + (I.tile_begin + j) * T.S + s;
        const long long x = j < nblk ? *p : 0;
        long long y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += u;
        }
        if (lane == 31) wsum[warp] = y;
        __syncthreads();
        if (warp == 0) {
            long long w = wsum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const long long excl = carry + (warp ? wsum[warp - 1] : 0) + y - x;
        if (j < nblk) *p = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) T.seg_count[(long long)b * T.S + s] = carry;
}

// Pass 3: write every non-zero value at its place, ascending vertex order.
template <int NDIM, typename Tin, typename Tval>
__global__ void __launch_bounds__(kGenBlock) k_gen_write(TablesDev T, const Tin* pixels, const long long* cnt) {
    constexpr int NO = 1 << NDIM, S = NO * 3 / 2, NW = kGenBlock / 32;
    __shared__ int wc[NW][S];
    const long long blk = blockIdx.x;
    const int b = gen_image(T, blk);
    const ImgDesc& I = T.img[b];
    const long long v = (blk - I.tile_begin) * kGenBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long val[S];
#pragma unroll
    for (int s = 0; s < S; ++s) val[s] = 0;
    if (v < I.N) {
        int i[NDIM];
        gen_decode<NDIM>(v, I.m, i);
        long long low[NO];
        bool bad = false;
        gen_lower_star<NDIM, Tin>(pixels + I.offset, I.m, i, low, bad);
        gen_segments<NDIM>(low, val);
    }
    unsigned bal[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        bal[s] = __ballot_sync(0xffffffffu, val[s] != 0);
        if (lane == 0) wc[warp][s] = __popc(bal[s]);
    }
    __syncthreads();
    Tval* av = reinterpret_cast<Tval*>(T.arena_val);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (val[s] == 0) continue;
        long long pos = cnt[blk * S + s];
        for (int w = 0; w < warp; ++w) pos += wc[w][s];
        pos += __popc(bal[s] & ((1u << lane) - 1u));
        const long long at = I.seg_base + (long long)s * I.N + pos;
        T.arena_idx[at] = (int)v;
        av[at] = (Tval)val[s];
    }
}

template <typename Tin, typename Tval>
static cudaError_t launch_gen_tables(const TablesDev& t, const void* pixels, long long nblk, long long* cnt,
                                     cudaStream_t st) {
    const Tin* px = reinterpret_cast<const Tin*>(pixels);
    k_gen_count<kGenN, Tin><<<(unsigned)nblk, kGenBlock, 0, st>>>(t, px, cnt);
    k_gen_scan<<<(unsigned)(t.B * t.S), 1024, 0, st>>>(t, cnt);
    k_gen_write<kGenN, Tin, Tval><<<(unsigned)nblk, kGenBlock, 0, st>>>(t, px, cnt);
    return cudaGetLastError();
}

int gen_block() { return kGenBlock; }


// ---- small helpers of the evaluation kernels ------------------------------------------------

__device__ __forceinline__ void kahan_add_gen(float& sum, float& c, float term) {
    const float y = __fsub_rn(term, c);
    const float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// s - 2 pi k in [-pi, pi], in FP64, rounded to FP32
__device__ __forceinline__ float gen_reduce_2pi(double s) {
    const double k = rint(s * 0.15915494309189535);
    return (float)fma(-k, 6.283185307179586, s);
}

// ---- evaluation ---------------------------------------------------------------------------

constexpr int kGenSub = 256;   // staged critical points per round

// Stage points [e0, e0 + cnt) of a table: FP64 coordinates x_k(v) (one correctly rounded
// division, as the oracle) and the value.
template <int NDIM, typename Tval>
__device__ __forceinline__ void gen_stage(const TablesDev& t, const ImgDesc& I, long long base, long long e0, int cnt,
                                          double (*X)[NDIM], double* V) {
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);
    for (int i = threadIdx.x; i < cnt; i += kGenBlock) {
        int c[NDIM];
        gen_decode<NDIM>((long long)(uint32_t)t.arena_idx[base + e0 + i], I.m, c);
#pragma unroll
        for (int k = 0; k < NDIM; ++k)
            X[i][k] = __ddiv_rn((double)(2 * c[k] - (I.m[k] - 1)), (double)(2 * (I.m[k] - 1)));
        V[i] = (double)aval[base + e0 + i];
    }
}

// The canonical dot product s = fl(...fl(fl(xi_0 x_0) + fl(xi_1 x_1)) ... + fl(xi_{n-1} x_{n-1})).
template <int NDIM>
__device__ __forceinline__ double gen_dot(const double* xi, const double* x) {
    double s = __dmul_rn(xi[0], x[0]);
#pragma unroll
    for (int k = 1; k < NDIM; ++k) s = __dadd_rn(s, __dmul_rn(xi[k], x[k]));
    return s;
}

// ECT / Radon: every (point, direction) binned exactly, values added to the output rows.
template <int NDIM, typename Tval>
__global__ void __launch_bounds__(kGenBlock) k_hist_gen(EvalPlan P, TablesDev t, int32_t* out_lo, int32_t* out_hi) {
    constexpr int NO = 1 << NDIM, NW = kGenBlock / 32;
    __shared__ double X[kGenSub][NDIM];
    __shared__ double V[kGenSub];
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = P.T;
    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= P.ctl[2]) break;
        int pair, tile, ch, b, o, part, sign;
        decode_item(P, item, pair, tile, ch);
        decode_pair(P.mode, NO, pair, b, o, part);
        const int seg = pair_segment(P.mode, NO, o, part, sign);
        const bool maxbin = part == 1;
        const ImgDesc& I = t.img[b];
        const int set = P.nsets == 1 ? 0 : b;
        const int* bo = P.boff + (long long)set * (NO + 1);
        const int r = tile * 32 + lane;
        const bool valid = r < bo[o + 1] - bo[o];
        const int d = valid ? P.perm[(long long)set * P.D + bo[o] + r] : 0;
        double xi[NDIM];
#pragma unroll
        for (int k = 0; k < NDIM; ++k) xi[k] = P.dirs[((long long)set * P.D + d) * NDIM + k];
        int32_t* row = (maxbin ? out_hi : out_lo) + ((long long)b * P.D + d) * T;
        const long long N = t.seg_count[(long long)b * t.S + seg];
        const long long base = I.seg_base + (long long)seg * I.N;
        const long long e_begin = (long long)ch * P.ctl[1], e_end = min(N, e_begin + P.ctl[1]);
        for (long long e0 = e_begin; e0 < e_end; e0 += kGenSub) {
            const int cnt = (int)min((long long)kGenSub, e_end - e0);
            __syncthreads();
            gen_stage<NDIM, Tval>(t, I, base, e0, cnt, X, V);
            __syncthreads();
            for (int e = warp; valid && e < cnt; e += NW) {
                const double s = gen_dot<NDIM>(xi, X[e]);
                const int v = (int)V[e];
                if (!maxbin) {   // min{j : s <= t_j}, T if none
                    int lo = 0, hi = T;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s <= P.thr[mid]) hi = mid; else lo = mid + 1;
                    }
                    if (lo < T) atomicAdd(&row[lo], v);
                } else {         // max{j : t_j <= s}, -1 if none
                    int lo = -1, hi = T - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (P.thr[mid] <= s) lo = mid; else hi = mid - 1;
                    }
                    if (lo >= 0) atomicAdd(&row[lo], v);
                }
            }
        }
    }
}

// s log2 e in FP64 from the canonical dot product.
__device__ __forceinline__ double gen_lap_exp(double s) { return s * 1.4426950408889634; }

// Forward (ADJ = false) or adjoint of the hybrid transform, one direction per lane.
template <int NDIM, int KERNEL, bool ADJ, typename Tval>
__global__ void __launch_bounds__(kGenBlock) k_ht_gen(EvalPlan P, TablesDev t, int precision, double* part) {
    constexpr int NO = 1 << NDIM, NW = kGenBlock / 32;
    constexpr int NK = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr int NC = ADJ ? NK * NDIM : NK;
    __shared__ double X[kGenSub][NDIM];
    __shared__ double V[kGenSub];
    __shared__ double red[NW][32 * NC];
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool f32 = precision == TOPOT_FP32C;
    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= P.ctl[2]) break;
        int pair, tile, ch, b, o, part_, sign;
        decode_item(P, item, pair, tile, ch);
        decode_pair(P.mode, NO, pair, b, o, part_);
        const int seg = pair_segment(P.mode, NO, o, part_, sign);
        const ImgDesc& I = t.img[b];
        const int set = P.nsets == 1 ? 0 : b;
        const int* bo = P.boff + (long long)set * (NO + 1);
        const int r = tile * 32 + lane;
        const bool valid = r < bo[o + 1] - bo[o];
        const int d = valid ? P.perm[(long long)set * P.D + bo[o] + r] : 0;
        double xi[NDIM];
#pragma unroll
        for (int k = 0; k < NDIM; ++k) xi[k] = P.dirs[((long long)set * P.D + d) * NDIM + k];
        const long long N = t.seg_count[(long long)b * t.S + seg];
        const long long base = I.seg_base + (long long)seg * I.N;
        const long long e_begin = (long long)ch * P.ctl[1], e_end = min(N, e_begin + P.ctl[1]);
        double acc64[NC];                 // FP64 sums (FP64 precision; rescaled Laplace rounds)
        float acc[NC], cmp[NC];           // FP32 compensated sums
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc64[c] = 0.0;
            acc[c] = cmp[c] = 0.0f;
        }
        for (long long e0 = e_begin; e0 < e_end; e0 += kGenSub) {
            const int cnt = (int)min((long long)kGenSub, e_end - e0);
            __syncthreads();
            gen_stage<NDIM, Tval>(t, I, base, e0, cnt, X, V);
            __syncthreads();
            const int per = (cnt + NW - 1) / NW, ws = warp * per, we = min(cnt, ws + per);
            if (!f32) {
                for (int e = ws; e < we; ++e) {
                    const double s = gen_dot<NDIM>(xi, X[e]);
                    double k0 = 0.0, k1 = 0.0;
                    if (KERNEL == TOPOT_LAPLACE) k0 = exp(s);
                    else if (KERNEL == TOPOT_FOURIER) {
                        sincos(s, &k0, &k1);   // (sin, cos): forward (re, im); adjoint (-d im, d re)
                        if (ADJ) { const double c_ = k1; k1 = k0; k0 = c_; }   // (cos, sin)
                    } else if (KERNEL == TOPOT_SINE) k0 = ADJ ? sin(s) : cos(s);
                    else if (KERNEL == TOPOT_BESSEL) k0 = ADJ ? -j1(s) : j0(s);
                    else k0 = ADJ ? table_kappa64(P, s) : table_kbar64(P, s);
                    const double kk[2] = {k0, k1};
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        acc64[c] += V[e] * kk[ADJ ? c / NDIM : c] * (ADJ ? X[e][c % NDIM] : 1.0);
                }
            } else if (KERNEL == TOPOT_LAPLACE) {
                // FP64 exponents, the round scaled by its largest term
                if (ws < we) {
                    double zr = -1e300;
                    for (int e = ws; e < we; ++e) zr = fmax(zr, gen_lap_exp(gen_dot<NDIM>(xi, X[e])));
                    float sr[NC], cr[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) sr[c] = cr[c] = 0.0f;
                    for (int e = ws; e < we; ++e) {
                        const float tk =
                            (float)V[e] * exp2f((float)(gen_lap_exp(gen_dot<NDIM>(xi, X[e])) - zr));
#pragma unroll
                        for (int c = 0; c < NC; ++c) kahan_add_gen(sr[c], cr[c], ADJ ? tk * (float)X[e][c] : tk);
                    }
                    const double sc = exp2(zr);
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc64[c] += ((double)sr[c] - (double)cr[c]) * sc;
                }
            } else {
                for (int e = ws; e < we; ++e) {
                    const double s = gen_dot<NDIM>(xi, X[e]);
                    const float v = (float)V[e];
                    float k0 = 0.0f, k1 = 0.0f;
                    if (KERNEL == TOPOT_FOURIER || KERNEL == TOPOT_SINE) {
                        const float rr = gen_reduce_2pi(s);
                        if (!ADJ) {   // (sin s, cos s - 1) from the half angle
                            float a, c_;
                            sincosf(0.5f * rr, &a, &c_);
                            k0 = KERNEL == TOPOT_FOURIER ? 2.0f * a * c_ : -2.0f * a * a;
                            k1 = -2.0f * a * a;
                        } else {      // (cos s, sin s) for Fourier; sin s for sine
                            float sn, cs;
                            sincosf(rr, &sn, &cs);
                            k0 = KERNEL == TOPOT_FOURIER ? cs : sn;
                            k1 = sn;
                        }
                    } else if (KERNEL == TOPOT_BESSEL) {
                        k0 = ADJ ? -(float)j1(s) : (float)(j0(s) - 1.0);
                    } else {
                        k0 = (float)(ADJ ? table_kappa64(P, s) : table_kbar64(P, s));
                    }
                    const float kk[2] = {k0, k1};
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        kahan_add_gen(acc[c], cmp[c], v * kk[ADJ ? c / NDIM : c] * (ADJ ? (float)X[e][c % NDIM] : 1.0f));
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) red[warp][lane * NC + c] = acc64[c] + ((double)acc[c] - (double)cmp[c]);
        __syncthreads();
        for (int i = tid; i < 32 * NC; i += kGenBlock) {
            double sm = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) sm += red[w][i];
            part[item * (32 * NC) + i] = sm;
        }
    }
}

template <typename Tval>
static cudaError_t launch_hist_gen_t(const EvalPlan& P, const TablesDev& t, int32_t* lo, int32_t* hi, int grid,
                                     cudaStream_t st) {
    k_hist_gen<kGenN, Tval><<<grid, kGenBlock, 0, st>>>(P, t, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_hist_gen(const EvalPlan& P, const TablesDev& t, int32_t* lo, int32_t* hi, int grid,
                            cudaStream_t st) {
    if (t.n != kGenN) return cudaErrorInvalidValue;
    return t.val_bytes == 2 ? launch_hist_gen_t<int16_t>(P, t, lo, hi, grid, st)
                            : launch_hist_gen_t<int32_t>(P, t, lo, hi, grid, st);
}

template <int KERNEL, typename Tval>
static cudaError_t launch_ht_gen_k(const EvalPlan& P, const TablesDev& t, int precision, bool adjoint, int grid,
                                   double* part, cudaStream_t st) {
    if (adjoint) k_ht_gen<kGenN, KERNEL, true, Tval><<<grid, kGenBlock, 0, st>>>(P, t, precision, part);
    else k_ht_gen<kGenN, KERNEL, false, Tval><<<grid, kGenBlock, 0, st>>>(P, t, precision, part);
    return cudaGetLastError();
}

template <typename Tval>
static cudaError_t launch_ht_gen_t(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint,
                                   int grid, double* part, cudaStream_t st) {
    switch (kernel) {
        case TOPOT_LAPLACE: return launch_ht_gen_k<TOPOT_LAPLACE, Tval>(P, t, precision, adjoint, grid, part, st);
        case TOPOT_FOURIER: return launch_ht_gen_k<TOPOT_FOURIER, Tval>(P, t, precision, adjoint, grid, part, st);
        case TOPOT_BESSEL: return launch_ht_gen_k<TOPOT_BESSEL, Tval>(P, t, precision, adjoint, grid, part, st);
        case TOPOT_SINE: return launch_ht_gen_k<TOPOT_SINE, Tval>(P, t, precision, adjoint, grid, part, st);
        case TOPOT_TABLE: return launch_ht_gen_k<TOPOT_TABLE, Tval>(P, t, precision, adjoint, grid, part, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ht_gen(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint, int grid,
                          double* part, cudaStream_t st) {
    if (t.n != kGenN) return cudaErrorInvalidValue;
    return t.val_bytes == 2 ? launch_ht_gen_t<int16_t>(P, t, kernel, precision, adjoint, grid, part, st)
                            : launch_ht_gen_t<int32_t>(P, t, kernel, precision, adjoint, grid, part, st);
}

cudaError_t launch_extract_gen(const TablesDev& t, topot_dtype dtype, const void* pixels, long long nblk,
                               long long* cnt, cudaStream_t st) {
    if (t.n != kGenN) return cudaErrorInvalidValue;
    if (dtype == TOPOT_U8) return launch_gen_tables<uint8_t, int16_t>(t, pixels, nblk, cnt, st);
    return launch_gen_tables<int32_t, int32_t>(t, pixels, nblk, cnt, st);
}

}  // namespace topot
