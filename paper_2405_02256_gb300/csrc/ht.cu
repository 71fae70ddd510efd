// K4 / K5 / K6 / K8: hybrid transforms and their adjoint.
//
// HT(xi) = sum_v Delta_eps(v) kbar(<xi, v>)          (closed form and sign of Lemma 3.1)
// dHT/dxi_k = sum_v Delta_eps(v) kappa(<xi, v>) x_k(v), kappa = kbar'
//
// Work split: persistent grid over the plan's items (pair, tile of 32 * DL
// directions, chunk of the Delta table).  The chunk is staged in shared memory as
// lattice coordinates; every lane owns DL directions and all lanes of a warp read
// the same critical point (shared-memory broadcast), so the kernel evaluations run
// on the FMA and MUFU pipes with no divergence.  Warps take disjoint slices of the
// chunk.
//
// Precision (FP32C): every term is formed in FP32 and added with Kahan compensation
// per lane; at the end of an item the eight warps' (sum - compensation) are added in
// FP64 in warp order and stored as the item's partial; k_ht_combine adds the chunk
// partials of each direction in chunk order in FP64.  The result is deterministic.
// The forward FP32C kernels sum kbar(s) - kbar(0) rather than kbar(s) for the kernels
// with a constant term (Fourier's imaginary part cos s, sine, Bessel): the constant
// drops out of the closed form because sum_v Delta_eps(v) = 0 over a whole table, and
// without it a term stays small where kbar(s) is close to kbar(0) (cos s - 1 = -w q(w),
// J0 - 1 = -y q(y) on the polynomial paths), so small transforms keep their accuracy.
// Laplace: the packed path takes tiles with M = sum_k |xi_k| / 2 <= 1 (|s| <= M), so the
// terms e^s = 2^{s log2 e} lie in [1/e, e] and are summed as they are; wider tiles form
// s log2 e in FP64 and scale every round of staged points by its own largest term, the
// round's sum entering the FP64 partial times that term (no FP32 overflow or underflow).
// Arguments: the packed paths form <xi, v> in FP32 (absolute error <= 3 * 2^-24 M,
// M <= 2); the scalar path does the same up to |s| <= 1.75 (Fourier, sine) or 2
// (Bessel) and beyond forms s in FP64 and reduces it modulo 2 pi in FP64 before the
// FP32 evaluation, so its error does not grow with |s|.
// FP64: the canonical FP64 dot product and library FP64 kernels, plain FP64 sums.
#include <algorithm>

#include "eval_common.cuh"

namespace topot {

constexpr int kHtBlock = 256;
constexpr int kHtWarps = kHtBlock / 32;
constexpr int kHtSub = 1024;        // staged critical points per round

struct alignas(32) Dbl4 {
    double x, y, z, w;
};

__device__ __forceinline__ void kahan_add(float& sum, float& c, float term) {
    const float y = __fsub_rn(term, c);
    const float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// Range limits of the FP32 argument paths, by kernel (largest M = sum_k |xi_k| / 2 of a
// tile, which bounds |<xi, v>|): beyond them the scalar path forms the argument in FP64.
constexpr float kLaplaceM32 = 1.0f;     // Laplace: relative error of e^s <= 3 M log2(e) ln(2) 2^-24
constexpr float kTrigM32 = 1.75f;       // Fourier, sine: polynomial and MUFU range
constexpr float kBesselM32 = 2.0f;      // Bessel: polynomial range

// ---- polynomial kernels -----------------------------------------------------------------------
// Degree-d Chebyshev interpolants on [0, X] written in the power basis (constants derived
// by gen_poly.py from the functions' own series; the listed bounds are the worst absolute
// errors of the FP32 Horner evaluation).  One template serves a float and an f32x2 pair.
__device__ __forceinline__ float fma_v(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_v(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float splat(float c, float) { return c; }
__device__ __forceinline__ float2 splat(float c, float2) { return make_float2(c, c); }

template <int N, typename V>
__device__ __forceinline__ V horner(const float (&c)[N], V x) {
    V p = splat(c[N - 1], x);
#pragma unroll
    for (int k = N - 2; k >= 0; --k) p = fma_v(p, x, splat(c[k], x));
    return p;
}

//   cos(sqrt w): X = 0.5625 (|z| <= 0.75), d = 3, 8e-8;  X = 3.0625 (|z| <= 1.75), d = 5, 7e-8
template <typename V>
__device__ __forceinline__ V cos_short(V w) {
    constexpr float c[4] = {1.000000000e+00f, -4.999988973e-01f, 4.165696725e-02f, -1.361225732e-03f};
    return horner(c, w);
}
template <typename V>
__device__ __forceinline__ V cos_long(V w) {
    constexpr float c[6] = {1.000000000e+00f, -4.999999702e-01f, 4.166659340e-02f, -1.388788689e-03f,
                            2.473820496e-05f, -2.569863113e-07f};
    return horner(c, w);
}
// sin z = z q(z^2): X = 0.5625 (|z| <= 0.75), d = 3, 4e-8;  X = 3.0625 (|z| <= 1.75), d = 5, 7e-8
template <typename V>
__device__ __forceinline__ V sinc_short(V w) {
    constexpr float c[4] = {1.000000000e+00f, -1.666665524e-01f, 8.332253434e-03f, -1.953341998e-04f};
    return horner(c, w);
}
template <typename V>
__device__ __forceinline__ V sinc_long(V w) {
    constexpr float c[6] = {1.000000000e+00f, -1.666666716e-01f, 8.333328180e-03f, -1.984049450e-04f,
                            2.750829026e-06f, -2.361634976e-08f};
    return horner(c, w);
}
// sin z = z q(z^2) for |z| <= 0.5: X = 0.25, d = 2, 1.5e-7 (relative)
template <typename V>
__device__ __forceinline__ V sinc_tiny(V w) {
    constexpr float c[3] = {9.999998808e-01f, -1.666597277e-01f, 8.259218186e-03f};
    return horner(c, w);
}
// cos z - 1 = w r(w), r = -(1 - cos sqrt w) / w (coefficients of gen_poly.py's cosm1q,
// negated): X = 0.5625, d = 2: |w r| error 8e-8, relative 3.5e-7;  X = 3.0625, d = 4:
// 1.1e-7, relative 1e-7
template <typename V>
__device__ __forceinline__ V cosm1_tiny(V w) {   // X = 0.25 (|z| <= 0.5), d = 2: relative 1.2e-7
    constexpr float c[3] = {-5.000000000e-01f, 4.166579992e-02f, -1.379617257e-03f};
    return horner(c, w);
}
template <typename V>
__device__ __forceinline__ V cosm1_short(V w) {
    constexpr float c[3] = {-4.999998510e-01f, 4.166229069e-02f, -1.368109020e-03f};
    return horner(c, w);
}
template <typename V>
__device__ __forceinline__ V cosm1_long(V w) {
    constexpr float c[5] = {-5.000000000e-01f, 4.166664928e-02f, -1.388843870e-03f, 2.476027112e-05f,
                            -2.600190783e-07f};
    return horner(c, w);
}
// J0(z) - 1 = y r(y), y = (z/2)^2, r = -(1 - J0) / y (gen_poly.py's j0m1q, negated):
// X = 0.25 (|z| <= 1), d = 3: |y r| error 1.4e-8, relative 8e-8;  X = 1 (|z| <= 2), d = 4:
// 6e-8, relative 8e-8
template <typename V>
__device__ __forceinline__ V j0m1_tiny(V y) {   // X = 0.0625 (|z| <= 0.5), d = 2: relative 1.1e-7
    constexpr float c[3] = {-1.000000000e+00f, 2.499962002e-01f, -2.761547454e-02f};
    return horner(c, y);
}
template <typename V>
__device__ __forceinline__ V j0m1_short(V y) {
    constexpr float c[4] = {-1.000000000e+00f, 2.499997318e-01f, -2.777241915e-02f, 1.701718429e-03f};
    return horner(c, y);
}
template <typename V>
__device__ __forceinline__ V j0m1_long(V y) {
    constexpr float c[5] = {-1.000000000e+00f, 2.499998212e-01f, -2.777634189e-02f, 1.732071629e-03f,
                            -6.477852730e-05f};
    return horner(c, y);
}
// J1(z) = (z/2) q((z/2)^2): X = 0.25 (|z| <= 1), d = 3, 6e-8;  X = 1 (|z| <= 2), d = 5, 6e-8
template <typename V>
__device__ __forceinline__ V j1q_short(V y) {
    constexpr float c[4] = {1.000000000e+00f, -4.999986589e-01f, 8.330661058e-02f, -6.772808731e-03f};
    return horner(c, y);
}
template <typename V>
__device__ __forceinline__ V j1q_long(V y) {
    constexpr float c[6] = {1.000000000e+00f, -5.000000000e-01f, 8.333322406e-02f, -6.943985354e-03f,
                            3.463324101e-04f, -1.077446268e-05f};
    return horner(c, y);
}

// ---- scalar path: FP32 argument in range, FP64 argument beyond ---------------------------------

// s in FP64 from the staged lattice integers p_k (c_k = 2 i_k - (m_k - 1)) and the
// direction: s = sum_k c_k (xi_k / (2 (m_k - 1))).
template <int NDIM>
__device__ __forceinline__ double arg64(const float4& q, const double (&xi)[3], const double (&inv2m)[3]) {
    double s = (double)q.x * (xi[0] * inv2m[0]);
    s = fma((double)q.y, xi[1] * inv2m[1], s);
    if (NDIM == 3) s = fma((double)q.z, xi[2] * inv2m[2], s);
    return s;
}

// r = s - 2 pi k in [-pi, pi] (FP64; the error of the FP64 constant 2 pi times k stays
// below 1e-10 for |s| <= 1e6), rounded to FP32.
__device__ __forceinline__ float reduce_2pi(double s) {
    const double k = rint(s * 0.15915494309189535);
    return (float)fma(-k, 6.283185307179586, s);
}

// (sin s, cos s - 1).  |z| <= 1.75: polynomials of the FP32 argument z; beyond: the FP64
// argument reduced modulo 2 pi, and with (a, b) = (sin r/2, cos r/2) from the accurate
// sincosf, sin s = 2 a b and cos s - 1 = -2 a^2.
template <int NDIM>
__device__ __forceinline__ void trig_m1(float z, const float4& q, const double (&xi)[3], const double (&inv2m)[3],
                                        float& sn, float& cm1) {
    if (fabsf(z) <= kTrigM32) {
        const float w = z * z;
        sn = z * sinc_long(w);
        cm1 = w * cosm1_long(w);
    } else {
        const float r = reduce_2pi(arg64<NDIM>(q, xi, inv2m));
        float a, b;
        sincosf(0.5f * r, &a, &b);
        sn = 2.0f * a * b;
        cm1 = -2.0f * a * a;
    }
}

// (sin s, cos s) for the adjoint's scalar path, argument as trig_m1.
template <int NDIM>
__device__ __forceinline__ void trig_full(float z, const float4& q, const double (&xi)[3], const double (&inv2m)[3],
                                          float& sn, float& cs) {
    if (fabsf(z) <= kTrigM32) {
        const float w = z * z;
        sn = z * sinc_long(w);
        cs = cos_long(w);
    } else {
        sincosf(reduce_2pi(arg64<NDIM>(q, xi, inv2m)), &sn, &cs);
    }
}

// J0(s) - 1: -y q(y) with y = (z/2)^2 for |z| <= 2; beyond, FP64 j0 of the FP64 argument.
template <int NDIM>
__device__ __forceinline__ float j0m1_scalar(float z, const float4& q, const double (&xi)[3],
                                             const double (&inv2m)[3]) {
    if (fabsf(z) <= kBesselM32) {
        const float y = 0.25f * z * z;
        return y * j0m1_long(y);
    }
    return (float)(j0(arg64<NDIM>(q, xi, inv2m)) - 1.0);
}

// J1(s): (z/2) q((z/2)^2) for |z| <= 2; beyond, FP64 j1 of the FP64 argument.
template <int NDIM>
__device__ __forceinline__ float j1_scalar(float z, const float4& q, const double (&xi)[3],
                                           const double (&inv2m)[3]) {
    if (fabsf(z) <= kBesselM32) {
        const float h = 0.5f * z;
        return h * j1q_long(h * h);
    }
    return (float)j1(arg64<NDIM>(q, xi, inv2m));
}

// Per-lane direction coefficients.
struct HtDir {
    float w[3];      // xi_k / (2 (m_k - 1)) (LAPLACE: times log2 e, so that z = sum_k w_k c_k = s log2 e)
    double xi[3];
    bool valid;
    int d;
};

// Shared prologue of the forward and adjoint kernels: item decode and staging.
struct HtItem {
    int b, o, sign, seg;
    long long base, e_begin, e_end;
    const ImgDesc* I;
    int set, nd;
};

__device__ __forceinline__ HtItem ht_item(const EvalPlan& P, const TablesDev& t, long long item, int NO,
                                          int tile_dirs, int& tile) {
    HtItem it;
    int pair, ch, part;
    decode_item(P, item, pair, tile, ch);
    decode_pair(P.mode, NO, pair, it.b, it.o, part);
    it.seg = pair_segment(P.mode, NO, it.o, part, it.sign);
    it.I = &t.img[it.b];
    it.set = P.nsets == 1 ? 0 : it.b;
    const int* bo = P.boff + (long long)it.set * (NO + 1);
    it.nd = bo[it.o + 1] - bo[it.o];
    const long long N = t.seg_count[(long long)it.b * t.S + it.seg];
    it.base = it.I->seg_base + (long long)it.seg * it.I->N;
    it.e_begin = (long long)ch * P.ctl[1];
    it.e_end = min(N, it.e_begin + P.ctl[1]);
    (void)tile_dirs;
    return it;
}

// Stage critical points [e0, e0 + cnt) as lattice data: A = (p0, p1, p2, value) with the
// lattice integers p_k = c_k = 2 i_k - (m_k - 1) (the same for an orthant and its partner);
// X = (x0, x1, x2) embedding coordinates (adjoint only).
template <int NDIM, int KERNEL, bool WITH_X, typename Tval, bool PACKED = false>
__device__ __forceinline__ void ht_stage(const TablesDev& t, const HtItem& it, long long e0, int cnt,
                                         float4* A, float4* X, int cnt_pad = 0) {
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);
    const ImgDesc& I = *it.I;
    if (PACKED) {   // zero-value points after the last one, up to cnt_pad
        for (int i = cnt + threadIdx.x; i < cnt_pad; i += kHtBlock) {
            A[2 * i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            A[2 * i + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    for (int i = threadIdx.x; i < cnt; i += kHtBlock) {
        const uint32_t idx = (uint32_t)t.arena_idx[it.base + e0 + i];
        const float v = (float)aval[it.base + e0 + i];
        const uint32_t q1 = fastdiv(idx, I.div0);
        int ii[3];
        ii[0] = (int)(idx - q1 * (uint32_t)I.m[0]);
        ii[1] = (int)q1;
        ii[2] = 0;
        if (NDIM == 3) {
            const uint32_t q2 = fastdiv(q1, I.div1);
            ii[1] = (int)(q1 - q2 * (uint32_t)I.m[1]);
            ii[2] = (int)q2;
        }
        float p[3], c[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c[k] = (float)(2 * ii[k] - (I.m[k] - 1));
            p[k] = c[k];
        }
        if (NDIM == 2) p[2] = 0.0f;
        if (PACKED) {
            A[2 * i] = make_float4(p[0], p[0], p[1], p[1]);
            A[2 * i + 1] = make_float4(p[2], p[2], v, v);
        } else {
            A[i] = make_float4(p[0], p[1], p[2], v);
        }
        if (WITH_X) {
            float x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = (k < NDIM) ? c[k] / (float)(2 * (I.m[k] - 1)) : 0.0f;
            X[i] = make_float4(x[0], x[1], x[2], 0.0f);
        }
    }
}

template <int NDIM, int KERNEL>
__device__ __forceinline__ void ht_dir(const EvalPlan& P, const HtItem& it, int r, HtDir& hd) {
    const int NO = 1 << NDIM;
    hd.valid = r < it.nd;
    hd.d = hd.valid ? P.perm[(long long)it.set * P.D + P.boff[(long long)it.set * (NO + 1) + it.o] + r] : 0;
    const double* xp = P.dirs + ((long long)it.set * P.D + hd.d) * NDIM;
    // Laplace works in log2 units (ex2): w_k = xi_k log2 e / (2 (m_k - 1))
    const double f = KERNEL == TOPOT_LAPLACE ? 1.4426950408889634 : 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        hd.xi[k] = k < NDIM ? xp[k] : 0.0;
        hd.w[k] = k < NDIM ? (float)(hd.xi[k] * (f * it.I->inv2m[k])) : 0.0f;
    }
}

// ---- forward, FP32 compensated ------------------------------------------------------------

// Packed FP32 pairs (f32x2: one instruction operates on two directions).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated add of a block sum x into (s, nc) for two sums at once.
__device__ __forceinline__ void kahan2_add(float2& s, float2& nc, float2 x) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 y = add2(x, nc);
    const float2 t = add2(s, y);
    const float2 u = fma2(s, m1, t);
    nc = fma2(u, m1, y);
    s = t;
}

// kbar(s) - kbar(0) for a direction pair.  Fourier: odd pairs take sin and cos from the
// MUFU pipe, even pairs evaluate sin and cos - 1 as polynomials in w = z^2 on the FMA
// pipe; half and half keeps both pipes busy (a MUFU sin/cos costs two XU cycles, the
// polynomial pair about 9 FP32 operations).  The MUFU pairs return cos s itself: their
// constant is removed once per round (the warp's sum of the staged values, see
// ht_packed_range), since MUFU's absolute error would not shrink with cos s - 1 anyway.
template <int KERNEL, int PATH>
__device__ __forceinline__ void kernel_pair(float2 z, float2 (&k)[2], bool mufu_cos) {
    if (KERNEL == TOPOT_LAPLACE) {
        k[0] = make_float2(ex2_approx(z.x), ex2_approx(z.y));
    } else if (KERNEL == TOPOT_FOURIER) {
        if (mufu_cos) {
            k[0] = make_float2(__sinf(z.x), __sinf(z.y));
            k[1] = make_float2(__cosf(z.x), __cosf(z.y));
        } else {
            const float2 w = mul2(z, z);
            k[0] = mul2(z, PATH == 3 ? sinc_tiny(w) : (PATH == 2 ? sinc_short(w) : sinc_long(w)));
            k[1] = mul2(w, PATH == 3 ? cosm1_tiny(w) : (PATH == 2 ? cosm1_short(w) : cosm1_long(w)));
        }
    } else if (KERNEL == TOPOT_SINE) {   // cos s - 1; the sign of kbar = -cos is applied at the combine
        if (mufu_cos) {
            k[0] = make_float2(__cosf(z.x), __cosf(z.y));
        } else {
            const float2 w = mul2(z, z);
            k[0] = mul2(w, PATH == 3 ? cosm1_tiny(w) : (PATH == 2 ? cosm1_short(w) : cosm1_long(w)));
        }
    } else {   // J0 - 1; z is already halved
        const float2 y = mul2(z, z);
        k[0] = mul2(y, PATH == 3 ? j0m1_tiny(y) : (PATH == 2 ? j0m1_short(y) : j0m1_long(y)));
    }
}

// Packed evaluation of staged points [ws, we) for NPR direction pairs.  Terms are
// summed by FMA in blocks of 8 points, and each block sum is added with compensation: a
// block adds at most 8 eps of its terms' magnitudes, the compensated sum 2 eps.  For
// Fourier and sine the pairs on MUFU sin / cos (odd pairs), whose evaluation takes most of
// the error budget, close their block every 4 points.
template <int NDIM, int KERNEL, int NPR, int PATH, int PS>
__device__ __forceinline__ void ht_packed_range(const float4* A, int ws, int we, int g, const float2 (&w)[NPR][3],
                                                float2 (&s2)[NPR][KERNEL == TOPOT_FOURIER ? 2 : 1],
                                                float2 (&n2)[NPR][KERNEL == TOPOT_FOURIER ? 2 : 1]) {
    constexpr int NC = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr bool SPLIT = KERNEL == TOPOT_FOURIER || KERNEL == TOPOT_SINE;
    // [ws, we) is a multiple of 8 PS long (rounds are padded with zero-value points); the
    // lanes of point group g take points ws + g, ws + g + PS, ... (with PS = 2 the two
    // half-warps read neighbouring points: different banks, one shared-memory wavefront).
    // Each block of 8 points is summed in two interleaved chains (even / odd points) to
    // halve the dependency depth, then added with compensation.
    for (int e = ws + g; e < we; e += 8 * PS) {
        float2 ba[NPR][NC], bb[NPR][NC];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 qa = A[2 * (e + u * PS)];
            const float4 qb = A[2 * (e + u * PS) + 1];
            const float2 c0 = make_float2(qa.x, qa.y), c1 = make_float2(qa.z, qa.w);
            const float2 c2 = make_float2(qb.x, qb.y), v2 = make_float2(qb.z, qb.w);
#pragma unroll
            for (int pq = 0; pq < NPR; ++pq) {
                float2 z = mul2(c0, w[pq][0]);
                z = fma2(c1, w[pq][1], z);
                if (NDIM == 3) z = fma2(c2, w[pq][2], z);
                float2 k[2];
                kernel_pair<KERNEL, PATH>(z, k, (pq & 1) == 1);
                const int ub = (SPLIT && (pq & 1)) ? (u & 3) : u;   // position in the pair's block
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (ub == 0) ba[pq][c] = mul2(v2, k[c]);
                    else if (ub == 1) bb[pq][c] = mul2(v2, k[c]);
                    else if (ub & 1) bb[pq][c] = fma2(v2, k[c], bb[pq][c]);
                    else ba[pq][c] = fma2(v2, k[c], ba[pq][c]);
                }
            }
            if (SPLIT && u == 3) {
#pragma unroll
                for (int pq = 1; pq < NPR; pq += 2)
#pragma unroll
                    for (int c = 0; c < NC; ++c) kahan2_add(s2[pq][c], n2[pq][c], add2(ba[pq][c], bb[pq][c]));
            }
        }
#pragma unroll
        for (int pq = 0; pq < NPR; ++pq)
#pragma unroll
            for (int c = 0; c < NC; ++c) kahan2_add(s2[pq][c], n2[pq][c], add2(ba[pq][c], bb[pq][c]));
    }
}

// Sum of the table values of staged points [e0 + i0, e0 + i1) (one warp's slice of a
// round), exact in 64-bit integers; every lane gets it.
template <typename Tval, int PS>
__device__ __forceinline__ long long warp_value_sum(const TablesDev& t, const HtItem& it, long long e0, int i0,
                                                    int i1, int lane) {
    // point group g = lane / (32 / PS) sums points i0 + g, i0 + g + PS, ...
    constexpr int GL = 32 / PS;
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);
    long long v = 0;
    for (int i = i0 + lane / GL + PS * (lane % GL); i < i1; i += 32) v += aval[it.base + e0 + i];
#pragma unroll
    for (int o = GL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Laplace exponent in FP64 for the scalar path: s log2 e from the staged lattice integers
// c_k (s = sum_k c_k xi_k / (2 (m_k - 1))).
template <int NDIM>
__device__ __forceinline__ double lap_arg64(const float4& q, const double (&xi)[3], const double (&inv2m)[3]) {
    constexpr double kLog2e = 1.4426950408889634;
    double s = (double)q.x * (xi[0] * inv2m[0]);
    s = fma((double)q.y, xi[1] * inv2m[1], s);
    if (NDIM == 3) s = fma((double)q.z, xi[2] * inv2m[2], s);
    return s * kLog2e;
}

// Which items a forward or adjoint FP32C launch takes.  With one direction per lane
// (kRoleAll) every item runs on the scalar path.  With two or more, a tile whose
// directions all lie in the FP32 argument range runs on the packed path (kRolePacked)
// and any other tile on the scalar path (kRoleWide): two launches of one item list, each
// skipping the other's tiles, so that the FP64 code of the wide tiles does not weigh on
// the registers of the packed kernel.  Both decide from the same tile maximum of M.
enum HtRole : int { kRoleAll = 0, kRolePacked = 1, kRoleWide = 2 };

// Largest M = sum_k |xi_k| / 2 (a bound on |<xi, v>|) over the tile's directions; every
// lane of the warp gets it.
template <int NDIM, int TDH>
__device__ __forceinline__ float tile_mloc(const EvalPlan& P, const HtItem& it, int tile, int lane) {
    constexpr int NO = 1 << NDIM;
    float m = 0.0f;
#pragma unroll
    for (int j = 0; j < (TDH + 31) / 32; ++j) {
        const int r = tile * TDH + j * 32 + lane;
        if (j * 32 + lane < TDH && r < it.nd) {
            const int d = P.perm[(long long)it.set * P.D + P.boff[(long long)it.set * (NO + 1) + it.o] + r];
            const double* xp = P.dirs + ((long long)it.set * P.D + d) * NDIM;
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < NDIM; ++k) a += fabs(xp[k]);
            m = fmaxf(m, (float)(0.5 * a));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

template <int NDIM, int KERNEL>
__device__ __forceinline__ float packed_limit() {
    return KERNEL == TOPOT_LAPLACE ? kLaplaceM32 : (KERNEL == TOPOT_BESSEL ? kBesselM32 : kTrigM32);
}

template <int NDIM, int KERNEL, int DL, typename Tval, int ROLE, int SPL>
__global__ void __launch_bounds__(kHtBlock) k_ht_f32(EvalPlan P, TablesDev t, double* part) {
    // SPL point groups per warp: lanes l and l + 32 / SPL hold the same DL directions and
    // take alternate points, so a tile is 32 DL / SPL directions (SPL = 2: tiles of 32 or
    // 64 directions with two or four directions per lane, for small direction sets)
    constexpr int NC = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr int GL = 32 / SPL;                // lanes per point group
    constexpr int TDH = GL * DL;
    constexpr int NO = 1 << NDIM;
    constexpr int NPR = DL / 2;                 // direction pairs per lane (packed path)
    constexpr bool SPLIT = KERNEL == TOPOT_FOURIER || KERNEL == TOPOT_SINE;
    constexpr int CCOS = KERNEL == TOPOT_FOURIER ? 1 : 0;   // component holding cos s - 1
    // staging buffer: scalar path (p0, p1, p2, value) per point; packed path
    // (p0, p0, p1, p1), (p2, p2, v, v); reused for the per-item reduction
    __shared__ __align__(16) float4 A[2 * kHtSub];
    static_assert(sizeof(double) * kHtWarps * SPL * TDH * NC <= sizeof(float4) * 2 * kHtSub, "reduction buffer");
    double(*red)[TDH * NC] = reinterpret_cast<double(*)[TDH * NC]>(A);
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = lane / GL, gln = lane % GL;   // point group, lane within the group
    const long long nitems = P.ctl[2];

    while (true) {
        __syncthreads();
        // the wide launch takes the items the packed launch set aside (ctl[4] of them)
        if (tid == 0) {
            if (ROLE == kRoleWide) {
                const int k = atomicAdd(&P.ctl[3], 1);
                sh_item = k < P.ctl[4] ? (long long)P.wide_items[k] : nitems;
            } else {
                sh_item = atomicAdd(&P.ctl[0], 1);
            }
        }
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int tile;
        const HtItem it = ht_item(P, t, item, NO, TDH, tile);
        // tile-uniform choice of the evaluation path (all warps see the same tile)
        const float mloc = tile_mloc<NDIM, TDH>(P, it, tile, lane);
        const bool in_range = mloc <= packed_limit<NDIM, KERNEL>();
        // an item of the other launch: no points and no partial written (a skip that keeps
        // the loop's shape, which the packed path's register allocation prefers)
        const bool mine = !((ROLE == kRolePacked && !in_range) || (ROLE == kRoleWide && in_range));
        if (ROLE == kRolePacked && !mine && tid == 0) P.wide_items[atomicAdd(&P.ctl[4], 1)] = (int)item;
        const long long e_end = mine ? it.e_end : it.e_begin;
        HtDir hd[DL];
#pragma unroll
        for (int j = 0; j < DL; ++j) ht_dir<NDIM, KERNEL>(P, it, tile * TDH + j * GL + gln, hd[j]);
        // 0: scalar path; packed paths by the range of |<xi, v>| <= mloc:
        //   Laplace: 1 (<= 1)
        //   Fourier, sine: 3 (<= 0.5, tiny), 2 (<= 0.75, short), 1 (<= 1.75, long polynomials)
        //   Bessel:  3 (<= 0.5, tiny), 2 (<= 1, short), 1 (<= 2, long)
        // (directions are sorted by M within their orthant, so most tiles are narrow)
        int path = 0;
        if (ROLE == kRolePacked)
            path = (KERNEL == TOPOT_LAPLACE) ? 1
                 : (mloc <= 0.5f ? 3 : (mloc <= (KERNEL == TOPOT_BESSEL ? 1.0f : 0.75f) ? 2 : 1));

        float acc[DL][NC], cmp[DL][NC];
        double off[DL][NC];   // FP64 part of each sum (rescaled Laplace rounds, MUFU constants)
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                acc[j][c] = cmp[j][c] = 0.0f;
                off[j][c] = 0.0;
            }

        if constexpr (ROLE != kRolePacked) {
            // Laplace beyond the packed range: FP64 exponents, each round of staged points
            // scaled by its own largest term (no overflow or underflow, error independent of M)
            const bool rescale = KERNEL == TOPOT_LAPLACE && mloc > kLaplaceM32;
            double inv[3];   // 1 / (2 (m_k - 1))
#pragma unroll
            for (int k = 0; k < 3; ++k)
                inv[k] = k < NDIM ? it.I->inv2m[k] : 0.0;
            for (long long e0 = it.e_begin; e0 < e_end; e0 += kHtSub) {
                const int cnt = (int)min((long long)kHtSub, e_end - e0);
                __syncthreads();
                ht_stage<NDIM, KERNEL, false, Tval>(t, it, e0, cnt, A, nullptr);
                __syncthreads();
                const int per = (cnt + kHtWarps - 1) / kHtWarps;
                const int ws = warp * per, we = min(cnt, ws + per);
                if (KERNEL == TOPOT_LAPLACE && rescale) {
                    if (ws < we) {
#pragma unroll
                        for (int j = 0; j < DL; ++j) {
                            double zr = -1e300;
                            for (int e = ws + grp; e < we; e += SPL) zr = fmax(zr, lap_arg64<NDIM>(A[e], hd[j].xi, inv));
                            float sr = 0.0f, cr = 0.0f;
                            for (int e = ws + grp; e < we; e += SPL) {
                                const float4 q = A[e];
                                kahan_add(sr, cr, q.w * exp2f((float)(lap_arg64<NDIM>(q, hd[j].xi, inv) - zr)));
                            }
                            if (zr > -1e300) off[j][0] += ((double)sr - (double)cr) * exp2(zr);
                        }
                    }
                    continue;
                }
                for (int e = ws + grp; e < we; e += SPL) {
                    const float4 q = A[e];
#pragma unroll
                    for (int j = 0; j < DL; ++j) {
                        float z = q.x * hd[j].w[0];
                        z = fmaf(q.y, hd[j].w[1], z);
                        if (NDIM == 3) z = fmaf(q.z, hd[j].w[2], z);
                        if (KERNEL == TOPOT_LAPLACE) {
                            kahan_add(acc[j][0], cmp[j][0], q.w * exp2f(z));
                        } else if (KERNEL == TOPOT_FOURIER) {
                            float sn, cm;
                            trig_m1<NDIM>(z, q, hd[j].xi, inv, sn, cm);
                            kahan_add(acc[j][0], cmp[j][0], q.w * sn);
                            kahan_add(acc[j][1], cmp[j][1], q.w * cm);
                        } else if (KERNEL == TOPOT_SINE) {
                            float sn, cm;
                            trig_m1<NDIM>(z, q, hd[j].xi, inv, sn, cm);
                            kahan_add(acc[j][0], cmp[j][0], q.w * cm);
                        } else {
                            kahan_add(acc[j][0], cmp[j][0], q.w * j0m1_scalar<NDIM>(z, q, hd[j].xi, inv));
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < DL; ++j)
#pragma unroll
                for (int c = 0; c < NC; ++c) cmp[j][c] = -cmp[j][c];   // report as s + nc
        } else if constexpr (NPR > 0) {
            (void)in_range;
            // packed coefficients: pair p covers directions 2p and 2p + 1 of this lane;
            // Bessel uses z / 2 so that y = (z / 2)^2 is one multiply
            float2 w[NPR][3];   // (w_0, w_1, w_2) of the pair's two directions
            const float wsc = KERNEL == TOPOT_BESSEL ? 0.5f : 1.0f;
#pragma unroll
            for (int pq = 0; pq < NPR; ++pq)
#pragma unroll
                for (int k = 0; k < 3; ++k) w[pq][k] = make_float2(wsc * hd[2 * pq].w[k], wsc * hd[2 * pq + 1].w[k]);
            float2 s2[NPR][NC], n2[NPR][NC];
#pragma unroll
            for (int pq = 0; pq < NPR; ++pq)
#pragma unroll
                for (int c = 0; c < NC; ++c) s2[pq][c] = n2[pq][c] = make_float2(0.0f, 0.0f);
            long long vsum = 0;   // this warp's staged values: the constant of the MUFU pairs' cos

            for (long long e0 = it.e_begin; e0 < e_end; e0 += kHtSub) {
                const int cnt = (int)min((long long)kHtSub, e_end - e0);
                __syncthreads();
                // pad the round to 8 points per warp and point group with zero-value points
                const int cnt_pad = (cnt + kHtWarps * 8 * SPL - 1) / (kHtWarps * 8 * SPL) * (kHtWarps * 8 * SPL);
                ht_stage<NDIM, KERNEL, false, Tval, true>(t, it, e0, cnt, A, nullptr, cnt_pad);
                __syncthreads();
                const int per = cnt_pad / kHtWarps;
                const int ws = warp * per, we = ws + per;
                if (SPLIT && NPR > 1) vsum += warp_value_sum<Tval, SPL>(t, it, e0, ws, min(we, cnt), lane);
                if (KERNEL != TOPOT_LAPLACE && path == 3)
                    ht_packed_range<NDIM, KERNEL, NPR, 3, SPL>(A, ws, we, grp, w, s2, n2);
                else if (KERNEL != TOPOT_LAPLACE && path == 2)
                    ht_packed_range<NDIM, KERNEL, NPR, 2, SPL>(A, ws, we, grp, w, s2, n2);
                else ht_packed_range<NDIM, KERNEL, NPR, 1, SPL>(A, ws, we, grp, w, s2, n2);
            }
#pragma unroll
            for (int pq = 0; pq < NPR; ++pq)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    acc[2 * pq][c] = s2[pq][c].x;
                    cmp[2 * pq][c] = n2[pq][c].x;
                    acc[2 * pq + 1][c] = s2[pq][c].y;
                    cmp[2 * pq + 1][c] = n2[pq][c].y;
                    if (SPLIT && (pq & 1) && c == CCOS) off[2 * pq][c] = off[2 * pq + 1][c] = -(double)vsum;
                }
        }
        // fixed-order FP64 reduction over warps -> item partial (red aliases the stage)
        __syncthreads();
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c)
            {
                double r = (double)acc[j][c] + (double)cmp[j][c];
                if constexpr (ROLE != kRolePacked || SPLIT) r += off[j][c];
                red[warp * SPL + grp][(j * GL + gln) * NC + c] = r;
            }
        __syncthreads();
        for (int i = tid; mine && i < TDH * NC; i += kHtBlock) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kHtWarps * SPL; ++w) s += red[w][i];
            part[item * (TDH * NC) + i] = s;
        }
    }
}

// ---- tabulated kernel -------------------------------------------------------------------------
// kbar is the piecewise-linear interpolant of K samples y_i = kbar(a + i h), constant outside
// [a, b]; kappa is its derivative, the segment slope on [a + i h, a + (i + 1) h) and zero
// outside [a, b).

// FP32: the position p = u + 1/2 is clamped to [0, K] by a saturating FMA on the scaled
// position p / K, and rounded to the nearest integer j by one FMA that adds 1.5 * 2^23
// (j lands in the low mantissa bits: no conversion instruction).  The padded table holds
// K + 1 pairs: entry j = r + 1 (0 <= r <= K - 2) is (y_r + d_r / 2, d_r), d_r = y_{r+1} - y_r,
// and the two ends are (y_0, 0) and (y_{K-1}, 0).  With g = p - j in [-1/2, 1/2]:
// kbar = Y + g D and kappa = D / h, constant ends and zero slope outside [a, b) included.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23; bits 0x4B400000
constexpr int kRoundMagicBits = 0x4B400000;

__device__ __forceinline__ float fma_sat(float a, float b, float c) {
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// ps = p / K in [0, 1]
__device__ __forceinline__ float2 table_entry(const float2* tab, float ps, float Kf, float& g) {
    const float t = fmaf(ps, Kf, kRoundMagic);
    const float j = __fsub_rn(t, kRoundMagic);
    g = fmaf(ps, Kf, -j);
    return tab[__float_as_int(t) - kRoundMagicBits];
}

constexpr int kTabStage = 2048;      // float4 slots of the stage / reduction area (32 KB)
constexpr int kTabMaxK = 16384;      // samples (K + 1 padded FP32 pairs, 128 KB)

// Forward (ADJ = false: one sum per direction) or adjoint (n sums) with the tabulated
// kernel, FP32 compensated.  The scaled position of a term is formed directly,
// p / K = v0 + sum_k c_k w'_k (saturated) with the staged integers c_k = 2 i_k - (m_k - 1),
// w'_k = xi_k / (2 (m_k - 1) h K) and v0 = (1/2 - a / h) / K; the kernel value is then
// one rounding FMA, one shared-memory load and two FMAs.  Blocks of four points are summed
// by FMA and added with compensation; the rounds are padded with zero-value points.
template <int NDIM, int DL, bool ADJ, typename Tval>
__global__ void __launch_bounds__(kHtBlock) k_ht_table_f32(EvalPlan P, TablesDev t, double* part) {
    constexpr int NC = ADJ ? NDIM : 1;
    constexpr int TDH = 32 * DL;
    constexpr int NO = 1 << NDIM;
    constexpr int SUB = ADJ ? kTabStage / 2 : kTabStage;   // staged points per round
    static_assert(sizeof(double) * kHtWarps * TDH * NC <= sizeof(float4) * kTabStage, "reduction buffer");
    extern __shared__ __align__(16) unsigned char smem_tab[];
    float4* A = reinterpret_cast<float4*>(smem_tab);        // (c0, c1, c2, value)
    float4* X = A + SUB;                                     // adjoint: (x0, x1, x2)
    double(*red)[TDH * NC] = reinterpret_cast<double(*)[TDH * NC]>(smem_tab);
    float2* tab = reinterpret_cast<float2*>(smem_tab + sizeof(float4) * kTabStage);
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nitems = P.ctl[2];
    const int K = P.ktab_k;
    for (int i = tid; i <= K; i += kHtBlock) tab[i] = P.ktab[i];
    const float Kf = (float)K;
    const float inv_h = (float)(1.0 / P.ktab_h);
    const float v0 = (float)((0.5 - P.ktab_a / P.ktab_h) / (double)K);
    const double inv_hk = 1.0 / (P.ktab_h * (double)K);

    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int tile;
        const HtItem it = ht_item(P, t, item, NO, TDH, tile);
        float wt[DL][3];
#pragma unroll
        for (int j = 0; j < DL; ++j) {
            HtDir hd;
            ht_dir<NDIM, TOPOT_TABLE>(P, it, tile * TDH + j * 32 + lane, hd);
#pragma unroll
            for (int k = 0; k < 3; ++k) wt[j][k] = k < NDIM ? (float)(hd.xi[k] * (it.I->inv2m[k] * inv_hk)) : 0.0f;
        }
        float acc[DL][NC], cmp[DL][NC];
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[j][c] = cmp[j][c] = 0.0f;

        for (long long e0 = it.e_begin; e0 < it.e_end; e0 += SUB) {
            const int cnt = (int)min((long long)SUB, it.e_end - e0);
            const int cnt_pad = (cnt + kHtWarps * 4 - 1) / (kHtWarps * 4) * (kHtWarps * 4);
            __syncthreads();
            ht_stage<NDIM, TOPOT_TABLE, ADJ, Tval>(t, it, e0, cnt, A, X);
            for (int i = cnt + tid; i < cnt_pad; i += kHtBlock) {
                A[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (ADJ) X[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            __syncthreads();
            const int per = cnt_pad / kHtWarps;
            const int ws = warp * per, we = ws + per;
            for (int e = ws; e < we; e += 4) {
                float blk[DL][NC];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 q = A[e + u];
                    float xs[3] = {0.0f, 0.0f, 0.0f};
                    if (ADJ) {
                        const float4 x = X[e + u];
                        xs[0] = x.x;
                        xs[1] = x.y;
                        xs[2] = x.z;
                    }
                    const float vw = ADJ ? q.w * inv_h : q.w;
#pragma unroll
                    for (int j = 0; j < DL; ++j) {
                        float ps = fmaf(q.x, wt[j][0], v0);
                        if (NDIM == 3) ps = fmaf(q.y, wt[j][1], ps);
                        ps = fma_sat(NDIM == 3 ? q.z : q.y, wt[j][NDIM - 1], ps);
                        float g;
                        const float2 te = table_entry(tab, ps, Kf, g);
                        if (!ADJ) {
                            const float kv = fmaf(g, te.y, te.x);
                            blk[j][0] = u == 0 ? q.w * kv : fmaf(q.w, kv, blk[j][0]);
                        } else {
                            const float tk = vw * te.y;
#pragma unroll
                            for (int c = 0; c < NC; ++c)
                                blk[j][c] = u == 0 ? tk * xs[c] : fmaf(tk, xs[c], blk[j][c]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < DL; ++j)
#pragma unroll
                    for (int c = 0; c < NC; ++c) kahan_add(acc[j][c], cmp[j][c], blk[j][c]);
            }
        }
        __syncthreads();   // red aliases the stage
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                red[warp][(j * 32 + lane) * NC + c] = (double)acc[j][c] - (double)cmp[j][c];
        __syncthreads();
        for (int i = tid; i < TDH * NC; i += kHtBlock) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kHtWarps; ++w) s += red[w][i];
            part[item * (TDH * NC) + i] = s;
        }
    }
}

// ---- forward, plain FP64 ---------------------------------------------------------------------

template <int NDIM, int KERNEL, typename Tval>
__global__ void __launch_bounds__(kHtBlock) k_ht_f64(EvalPlan P, TablesDev t, double* part) {
    constexpr int NC = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr int TDH = 32;
    constexpr int NO = 1 << NDIM;
    __shared__ Dbl4 XA[kHtSub / 2];
    __shared__ double red[kHtWarps][TDH * NC];
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nitems = P.ctl[2];
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);
    constexpr int SUB = kHtSub / 2;

    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int tile;
        const HtItem it = ht_item(P, t, item, NO, TDH, tile);
        HtDir hd;
        ht_dir<NDIM, TOPOT_FOURIER>(P, it, tile * TDH + lane, hd);
        double acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0;
        const ImgDesc& I = *it.I;
        for (long long e0 = it.e_begin; e0 < it.e_end; e0 += SUB) {
            const int cnt = (int)min((long long)SUB, it.e_end - e0);
            __syncthreads();
            for (int i = tid; i < cnt; i += kHtBlock) {
                const uint32_t idx = (uint32_t)t.arena_idx[it.base + e0 + i];
                const double v = (double)aval[it.base + e0 + i];
                const uint32_t q1 = fastdiv(idx, I.div0);
                int ii[3] = {(int)(idx - q1 * (uint32_t)I.m[0]), (int)q1, 0};
                if (NDIM == 3) {
                    const uint32_t q2 = fastdiv(q1, I.div1);
                    ii[1] = (int)(q1 - q2 * (uint32_t)I.m[1]);
                    ii[2] = (int)q2;
                }
                double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < NDIM; ++k)
                    x[k] = __ddiv_rn((double)(2 * ii[k] - (I.m[k] - 1)), (double)(2 * (I.m[k] - 1)));
                XA[i] = Dbl4{x[0], x[1], x[2], v};
            }
            __syncthreads();
            const int per = (cnt + kHtWarps - 1) / kHtWarps;
            const int ws = warp * per, we = min(cnt, ws + per);
            for (int e = ws; e < we; ++e) {
                const Dbl4 q = XA[e];
                double s = __dmul_rn(hd.xi[0], q.x);
                s = __dadd_rn(s, __dmul_rn(hd.xi[1], q.y));
                if (NDIM == 3) s = __dadd_rn(s, __dmul_rn(hd.xi[2], q.z));
                if (KERNEL == TOPOT_LAPLACE) {
                    acc[0] += q.w * exp(s);
                } else if (KERNEL == TOPOT_FOURIER) {
                    double sn, cs;
                    sincos(s, &sn, &cs);
                    acc[0] += q.w * sn;
                    acc[1] += q.w * cs;
                } else if (KERNEL == TOPOT_SINE) {
                    acc[0] += q.w * cos(s);
                } else if (KERNEL == TOPOT_TABLE) {
                    acc[0] += q.w * table_kbar64(P, s);
                } else {
                    acc[0] += q.w * j0(s);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) red[warp][lane * NC + c] = acc[c];
        __syncthreads();
        for (int i = tid; i < TDH * NC; i += kHtBlock) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kHtWarps; ++w) s += red[w][i];
            part[item * (TDH * NC) + i] = s;
        }
    }
}

// ---- adjoint (FP32 compensated and FP64) ----------------------------------------------------
// Partials per direction: LAPLACE / BESSEL: n sums  sum Delta kappa(s) x_k;
// FOURIER: 2n sums  (sum Delta cos(s) x_k, sum Delta sin(s) x_k)  [d Re = +cos, d Im = -sin].

// Packed adjoint over staged points [ws, we) for NPR direction pairs per lane:
//   g_k += v kappa(z) x_k  (Fourier: g_k += v cos z x_k and g_{n+k} += v sin z x_k)
// with x_k rebuilt from the staged integer p_k as x_k = p_k * xa_k + xb_k (shared by the
// pairs: it depends on the point only).  Blocks of four points are summed by FMA, then
// added with compensation (as the forward).
template <int NDIM, int KERNEL, int PATH, int NPR>
__device__ __forceinline__ void ht_adj_packed_range(const float4* A, int ws, int we, const float2 (&w)[NPR][3],
                                                    const float2 (&xa)[3], const float2 (&xb)[3],
                                                    float2 (&s2)[NPR][(KERNEL == TOPOT_FOURIER ? 2 : 1) * NDIM],
                                                    float2 (&n2)[NPR][(KERNEL == TOPOT_FOURIER ? 2 : 1) * NDIM]) {
    constexpr int NC = (KERNEL == TOPOT_FOURIER ? 2 : 1) * NDIM;
    constexpr int BLK = 4;
    for (int e = ws; e < we; e += BLK) {
        float2 blk[NPR][NC];
#pragma unroll
        for (int u = 0; u < BLK; ++u) {
            const float4 qa = A[2 * (e + u)];
            const float4 qb = A[2 * (e + u) + 1];
            const float2 pc[3] = {make_float2(qa.x, qa.y), make_float2(qa.z, qa.w), make_float2(qb.x, qb.y)};
            const float2 v2 = make_float2(qb.z, qb.w);
            float2 x[3];
#pragma unroll
            for (int k = 0; k < NDIM; ++k) x[k] = fma2(pc[k], xa[k], xb[k]);
#pragma unroll
            for (int r = 0; r < NPR; ++r) {
                float2 z = mul2(pc[0], w[r][0]);
                z = fma2(pc[1], w[r][1], z);
                if (NDIM == 3) z = fma2(pc[2], w[r][2], z);
                float2 t[2];
                if (KERNEL == TOPOT_LAPLACE) {
                    t[0] = mul2(v2, make_float2(ex2_approx(z.x), ex2_approx(z.y)));
                } else if (KERNEL == TOPOT_FOURIER) {
                    // odd points on MUFU sin/cos, even points on the polynomials: the
                    // XU pipe takes part of the FMA pipe's load (as the forward's pairs)
                    float2 sn, cs;
                    if (u & 1) {
                        sn = make_float2(__sinf(z.x), __sinf(z.y));
                        cs = make_float2(__cosf(z.x), __cosf(z.y));
                    } else {
                        const float2 ww = mul2(z, z);
                        sn = mul2(z, PATH == 2 ? sinc_short(ww) : sinc_long(ww));
                        cs = PATH == 2 ? cos_short(ww) : cos_long(ww);
                    }
                    t[0] = mul2(v2, cs);
                    t[1] = mul2(v2, sn);
                } else if (KERNEL == TOPOT_SINE) {   // kappa = sin
                    float2 sn;
                    if (u & 1) {
                        sn = make_float2(__sinf(z.x), __sinf(z.y));
                    } else {
                        const float2 ww = mul2(z, z);
                        sn = mul2(z, PATH == 2 ? sinc_short(ww) : sinc_long(ww));
                    }
                    t[0] = mul2(v2, sn);
                } else {   // z is halved: kappa = -J1(2 z) = -z q(z^2)
                    const float2 y = mul2(z, z);
                    const float2 j1 = mul2(z, PATH == 2 ? j1q_short(y) : j1q_long(y));
                    t[0] = mul2(make_float2(-v2.x, -v2.y), j1);
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float2 tc = t[c / NDIM];
                    const float2 xc = x[c % NDIM];
                    blk[r][c] = u == 0 ? mul2(tc, xc) : fma2(tc, xc, blk[r][c]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < NPR; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) kahan2_add(s2[r][c], n2[r][c], blk[r][c]);
    }
}

template <int NDIM, int KERNEL, int DL, typename Tval, int ROLE>
__global__ void __launch_bounds__(kHtBlock) k_ht_adj_f32(EvalPlan P, TablesDev t, double* part) {
    constexpr int NK = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr int NC = NK * NDIM;
    constexpr int TDH = 32 * DL;
    constexpr int NO = 1 << NDIM;
    constexpr int SUB = kHtSub / 2;
    // scalar path: A[0, SUB) = (p0, p1, p2, v), X = A + SUB = (x0, x1, x2); packed path:
    // (p0, p0, p1, p1), (p2, p2, v, v) per point over the whole buffer
    __shared__ __align__(16) float4 A[2 * SUB];
    float4* X = A + SUB;
    __shared__ double red[kHtWarps][TDH * NC];
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nitems = P.ctl[2];

    while (true) {
        __syncthreads();
        // the wide launch takes the items the packed launch set aside (ctl[4] of them)
        if (tid == 0) {
            if (ROLE == kRoleWide) {
                const int k = atomicAdd(&P.ctl[3], 1);
                sh_item = k < P.ctl[4] ? (long long)P.wide_items[k] : nitems;
            } else {
                sh_item = atomicAdd(&P.ctl[0], 1);
            }
        }
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int tile;
        const HtItem it = ht_item(P, t, item, NO, TDH, tile);
        const float mloc = tile_mloc<NDIM, TDH>(P, it, tile, lane);
        const bool in_range = mloc <= packed_limit<NDIM, KERNEL>();
        // an item of the other launch: no points and no partial written (a skip that keeps
        // the loop's shape, which the packed path's register allocation prefers)
        const bool mine = !((ROLE == kRolePacked && !in_range) || (ROLE == kRoleWide && in_range));
        if (ROLE == kRolePacked && !mine && tid == 0) P.wide_items[atomicAdd(&P.ctl[4], 1)] = (int)item;
        const long long e_end = mine ? it.e_end : it.e_begin;
        HtDir hd[DL];
#pragma unroll
        for (int j = 0; j < DL; ++j) ht_dir<NDIM, KERNEL>(P, it, tile * TDH + j * 32 + lane, hd[j]);
        float acc[DL][NC], cmp[DL][NC];
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[j][c] = cmp[j][c] = 0.0f;

        // packed paths: as the forward, DL / 2 direction pairs per lane
        int path = 0;
        if (ROLE == kRolePacked) path = (KERNEL == TOPOT_LAPLACE) ? 1 : (mloc <= (KERNEL == TOPOT_BESSEL ? 1.0f : 0.75f) ? 2 : 1);
        double off[DL][NC];   // FP64 part of each sum (rescaled Laplace rounds)
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) off[j][c] = 0.0;
        if constexpr (ROLE == kRolePacked) {
            constexpr int NPR = DL / 2;
            {
                const float wsc = KERNEL == TOPOT_BESSEL ? 0.5f : 1.0f;
                float2 w[NPR][3], xa[3], xb[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
#pragma unroll
                    for (int r = 0; r < NPR; ++r)
                        w[r][k] = make_float2(wsc * hd[2 * r].w[k], wsc * hd[2 * r + 1].w[k]);
                    const float mk1 = (float)(it.I->m[k] - 1);
                    xa[k] = make_float2(0.5f / mk1, 0.5f / mk1);   // x = c / (2 (m - 1))
                    xb[k] = make_float2(0.0f, 0.0f);
                }

                float2 s2[NPR][NC], n2[NPR][NC];
#pragma unroll
                for (int r = 0; r < NPR; ++r)
#pragma unroll
                    for (int c = 0; c < NC; ++c) s2[r][c] = n2[r][c] = make_float2(0.0f, 0.0f);
                for (long long e0 = it.e_begin; e0 < e_end; e0 += SUB) {
                    const int cnt = (int)min((long long)SUB, e_end - e0);
                    __syncthreads();
                    const int cnt_pad = (cnt + kHtWarps * 8 - 1) / (kHtWarps * 8) * (kHtWarps * 8);
                    ht_stage<NDIM, KERNEL, false, Tval, true>(t, it, e0, cnt, A, nullptr, cnt_pad);
                    __syncthreads();
                    const int per = cnt_pad / kHtWarps;
                    const int ws = warp * per, we = ws + per;
                    if (path == 2) ht_adj_packed_range<NDIM, KERNEL, 2, NPR>(A, ws, we, w, xa, xb, s2, n2);
                    else ht_adj_packed_range<NDIM, KERNEL, 1, NPR>(A, ws, we, w, xa, xb, s2, n2);
                }
#pragma unroll
                for (int r = 0; r < NPR; ++r)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        acc[2 * r][c] = s2[r][c].x;
                        cmp[2 * r][c] = -n2[r][c].x;
                        acc[2 * r + 1][c] = s2[r][c].y;
                        cmp[2 * r + 1][c] = -n2[r][c].y;
                    }
            }
        }
        const bool rescale = KERNEL == TOPOT_LAPLACE && mloc > kLaplaceM32;
        double inv[3];   // 1 / (2 (m_k - 1))
#pragma unroll
        for (int k = 0; k < 3; ++k)
            inv[k] = k < NDIM ? it.I->inv2m[k] : 0.0;
        for (long long e0 = it.e_begin; ROLE != kRolePacked && e0 < e_end; e0 += SUB) {
            const int cnt = (int)min((long long)SUB, e_end - e0);
            __syncthreads();
            ht_stage<NDIM, KERNEL, true, Tval>(t, it, e0, cnt, A, X);
            __syncthreads();
            const int per = (cnt + kHtWarps - 1) / kHtWarps;
            const int ws = warp * per, we = min(cnt, ws + per);
            if (KERNEL == TOPOT_LAPLACE && rescale) {
                // FP64 exponents; each round scaled by its own largest term (as the forward)
                if (ws < we) {
#pragma unroll
                    for (int j = 0; j < DL; ++j) {
                        double zr = -1e300;
                        for (int e = ws; e < we; ++e) zr = fmax(zr, lap_arg64<NDIM>(A[e], hd[j].xi, inv));
                        float sr[NC], cr[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) sr[c] = cr[c] = 0.0f;
                        for (int e = ws; e < we; ++e) {
                            const float4 q = A[e];
                            const float4 x = X[e];
                            const float xs[3] = {x.x, x.y, x.z};
                            const float tk = q.w * exp2f((float)(lap_arg64<NDIM>(q, hd[j].xi, inv) - zr));
#pragma unroll
                            for (int c = 0; c < NC; ++c) kahan_add(sr[c], cr[c], tk * xs[c]);
                        }
                        const double sc = exp2(zr);
#pragma unroll
                        for (int c = 0; c < NC; ++c) off[j][c] += ((double)sr[c] - (double)cr[c]) * sc;
                    }
                }
                continue;
            }
            for (int e = ws; e < we; ++e) {
                const float4 q = A[e];
                const float4 x = X[e];
                const float xs[3] = {x.x, x.y, x.z};
#pragma unroll
                for (int j = 0; j < DL; ++j) {
                    float z = q.x * hd[j].w[0];
                    z = fmaf(q.y, hd[j].w[1], z);
                    if (NDIM == 3) z = fmaf(q.z, hd[j].w[2], z);
                    if (KERNEL == TOPOT_FOURIER) {
                        float sn, cs;
                        trig_full<NDIM>(z, q, hd[j].xi, inv, sn, cs);
                        const float tc = q.w * cs, ts = q.w * sn;
#pragma unroll
                        for (int k = 0; k < NDIM; ++k) {
                            kahan_add(acc[j][k], cmp[j][k], tc * xs[k]);
                            kahan_add(acc[j][NDIM + k], cmp[j][NDIM + k], ts * xs[k]);
                        }
                    } else {
                        float kv;
                        if (KERNEL == TOPOT_LAPLACE) {
                            kv = exp2f(z);
                        } else if (KERNEL == TOPOT_SINE) {   // kappa = sin
                            float cs;
                            trig_full<NDIM>(z, q, hd[j].xi, inv, kv, cs);
                        } else {
                            kv = -j1_scalar<NDIM>(z, q, hd[j].xi, inv);
                        }
                        const float tk = q.w * kv;
#pragma unroll
                        for (int k = 0; k < NDIM; ++k) kahan_add(acc[j][k], cmp[j][k], tk * xs[k]);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < DL; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c)
            {
                double r = (double)acc[j][c] - (double)cmp[j][c];
                if constexpr (ROLE != kRolePacked) r += off[j][c];
                red[warp][(j * 32 + lane) * NC + c] = r;
            }
        __syncthreads();
        for (int i = tid; mine && i < TDH * NC; i += kHtBlock) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kHtWarps; ++w) s += red[w][i];
            part[item * (TDH * NC) + i] = s;
        }
    }
}

template <int NDIM, int KERNEL, typename Tval>
__global__ void __launch_bounds__(kHtBlock) k_ht_adj_f64(EvalPlan P, TablesDev t, double* part) {
    constexpr int NK = KERNEL == TOPOT_FOURIER ? 2 : 1;
    constexpr int NC = NK * NDIM;
    constexpr int TDH = 32;
    constexpr int NO = 1 << NDIM;
    constexpr int SUB = kHtSub / 2;
    __shared__ Dbl4 XA[SUB];
    __shared__ double red[kHtWarps][TDH * NC];
    __shared__ long long sh_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nitems = P.ctl[2];
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);

    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int tile;
        const HtItem it = ht_item(P, t, item, NO, TDH, tile);
        HtDir hd;
        ht_dir<NDIM, TOPOT_FOURIER>(P, it, tile * TDH + lane, hd);
        double acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0;
        const ImgDesc& I = *it.I;
        for (long long e0 = it.e_begin; e0 < it.e_end; e0 += SUB) {
            const int cnt = (int)min((long long)SUB, it.e_end - e0);
            __syncthreads();
            for (int i = tid; i < cnt; i += kHtBlock) {
                const uint32_t idx = (uint32_t)t.arena_idx[it.base + e0 + i];
                const double v = (double)aval[it.base + e0 + i];
                const uint32_t q1 = fastdiv(idx, I.div0);
                int ii[3] = {(int)(idx - q1 * (uint32_t)I.m[0]), (int)q1, 0};
                if (NDIM == 3) {
                    const uint32_t q2 = fastdiv(q1, I.div1);
                    ii[1] = (int)(q1 - q2 * (uint32_t)I.m[1]);
                    ii[2] = (int)q2;
                }
                double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < NDIM; ++k)
                    x[k] = __ddiv_rn((double)(2 * ii[k] - (I.m[k] - 1)), (double)(2 * (I.m[k] - 1)));
                XA[i] = Dbl4{x[0], x[1], x[2], v};
            }
            __syncthreads();
            const int per = (cnt + kHtWarps - 1) / kHtWarps;
            const int ws = warp * per, we = min(cnt, ws + per);
            for (int e = ws; e < we; ++e) {
                const Dbl4 q = XA[e];
                const double xs[3] = {q.x, q.y, q.z};
                double s = __dmul_rn(hd.xi[0], q.x);
                s = __dadd_rn(s, __dmul_rn(hd.xi[1], q.y));
                if (NDIM == 3) s = __dadd_rn(s, __dmul_rn(hd.xi[2], q.z));
                if (KERNEL == TOPOT_FOURIER) {
                    double sn, cs;
                    sincos(s, &sn, &cs);
#pragma unroll
                    for (int k = 0; k < NDIM; ++k) {
                        acc[k] += q.w * cs * xs[k];
                        acc[NDIM + k] += q.w * sn * xs[k];
                    }
                } else {
                    double kv;
                    if (KERNEL == TOPOT_LAPLACE) kv = exp(s);
                    else if (KERNEL == TOPOT_SINE) kv = sin(s);
                    else if (KERNEL == TOPOT_TABLE) kv = table_kappa64(P, s);
                    else kv = -j1(s);
#pragma unroll
                    for (int k = 0; k < NDIM; ++k) acc[k] += q.w * kv * xs[k];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) red[warp][lane * NC + c] = acc[c];
        __syncthreads();
        for (int i = tid; i < TDH * NC; i += kHtBlock) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kHtWarps; ++w) s += red[w][i];
            part[item * (TDH * NC) + i] = s;
        }
    }
}

// ---- combine (K6) ------------------------------------------------------------------------------

// Sum of the chunk partials of direction d of image b, in chunk order.  The hybrid
// transforms group a direction with those of its orthant's partner (same Delta table):
// pair (b, representative orthant).
__device__ __forceinline__ void gather_partials(const EvalPlan& P, int NO, int tdh, int ncomp, int b, int d,
                                                int o, const double* part, double* outc) {
    const int set = P.nsets == 1 ? 0 : b;
    const int r = P.rank[(long long)set * P.D + d];
    const int rep = (o & (NO >> 1)) ? (o ^ (NO - 1)) : o;
    const int pair = b * (NO / 2) + rep;
    const int tile = r / tdh, dd = r - tile * tdh;
    const long long nitems = P.pair_items[pair + 1] - P.pair_items[pair];
    for (int c = 0; c < ncomp; ++c) outc[c] = 0.0;
    if (nitems == 0) return;
    const int nch = P.pair_chunks[pair];
    const long long i0 = P.pair_items[pair] + (long long)tile * nch;
    for (int ch = 0; ch < nch; ++ch) {
        const double* pp = part + (i0 + ch) * (long long)(tdh * ncomp) + (long long)dd * ncomp;
        for (int c = 0; c < ncomp; ++c) outc[c] += pp[c];
    }
}

// vsum (slab handles only, else NULL): the value sums of the tables.  The FP32C kernels
// sum Delta (kbar(s) - kbar(0)) for Fourier's imaginary part, sine and Bessel, which is
// the transform when the table sums to zero (a whole image); a slab's table need not,
// and kbar(0) times its sum is added back here (kbar(0) = 1 for cos and J0).
__global__ void k_ht_combine(EvalPlan P, int n, int B, int kernel, int precision, int tdh,
                             const double* part, const long long* vsum, int S, double* out) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)B * P.D) return;
    const int b = (int)(gid / P.D), d = (int)(gid - (long long)b * P.D);
    const int NO = 1 << n;
    const int set = P.nsets == 1 ? 0 : b;
    const double* xi = P.dirs + ((long long)set * P.D + d) * n;
    const int o = orthant_of(xi, n);
    const int nc = kernel == TOPOT_FOURIER ? 2 : 1;
    double v[2];
    gather_partials(P, NO, tdh, nc, b, d, o, part, v);
    if (vsum && precision == TOPOT_FP32C &&
        (kernel == TOPOT_FOURIER || kernel == TOPOT_SINE || kernel == TOPOT_BESSEL)) {
        const int rep = (o & (NO >> 1)) ? (o ^ (NO - 1)) : o;
        v[nc - 1] += (double)vsum[(long long)b * S + NO + rep];   // cos / J0 component
    }
    const double sign = (o & (NO >> 1)) ? -1.0 : 1.0;
    // sine: the partials hold sum v (cos s - 1), kbar = -cos
    double scale = kernel == TOPOT_SINE ? -sign : sign;
    for (int c = 0; c < nc; ++c) out[gid * nc + c] = v[c] * scale;
}

// gdirs[set][d][k] = sum over images b of the set (all images when shared) of
// sum_c gout[b][d][c] * dOut_c / dxi_k.
__global__ void k_ht_adj_combine(EvalPlan P, int n, int B, int kernel, int precision, int tdh,
                                 const double* part, const double* gout, double* gdirs) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)P.nsets * P.D) return;
    const int set = (int)(gid / P.D), d = (int)(gid - (long long)set * P.D);
    const int NO = 1 << n;
    const double* xi = P.dirs + ((long long)set * P.D + d) * n;
    const int o = orthant_of(xi, n);
    const int nk = kernel == TOPOT_FOURIER ? 2 : 1;
    const int nc = nk * n;
    const double sign = (o & (NO >> 1)) ? -1.0 : 1.0;
    const double scale = sign;
    double g[kMaxDim] = {0.0, 0.0, 0.0, 0.0};
    const int b0 = P.nsets == 1 ? 0 : set, b1 = P.nsets == 1 ? B : set + 1;
    for (int b = b0; b < b1; ++b) {
        double v[2 * kMaxDim];
        gather_partials(P, NO, tdh, nc, b, d, o, part, v);
        const double* go = gout + ((long long)b * P.D + d) * nk;
        for (int k = 0; k < n; ++k) {
            if (kernel == TOPOT_FOURIER)   // Re = sum D sin s: d/dxi = sum D cos s x; Im = sum D cos s: -sum D sin s x
                g[k] += go[0] * v[k] - go[1] * v[n + k];
            else
                g[k] += go[0] * v[k];
        }
    }
    for (int k = 0; k < n; ++k) gdirs[gid * n + k] = g[k] * scale;
}

// ---- launchers ---------------------------------------------------------------------------------

template <int NDIM, int KERNEL, int DL, typename Tval, int SPL>
static void launch_fwd_pair(const EvalPlan& P, const TablesDev& t, int grid, int wide_grid, double* part,
                            cudaStream_t st) {
    k_ht_f32<NDIM, KERNEL, DL, Tval, kRolePacked, SPL><<<grid, kHtBlock, 0, st>>>(P, t, part);
    k_ht_f32<NDIM, KERNEL, DL, Tval, kRoleWide, SPL><<<wide_grid, kHtBlock, 0, st>>>(P, t, part);
}

template <int NDIM, int KERNEL, typename Tval>
static cudaError_t launch_ht_k(const EvalPlan& P, const TablesDev& t, int precision, bool adjoint, int dl,
                               int split, int grid, double* part, cudaStream_t st) {
    if (precision == TOPOT_FP64) {
        if (adjoint) k_ht_adj_f64<NDIM, KERNEL, Tval><<<grid, kHtBlock, 0, st>>>(P, t, part);
        else k_ht_f64<NDIM, KERNEL, Tval><<<grid, kHtBlock, 0, st>>>(P, t, part);
        return cudaGetLastError();
    }
    // two or more directions per lane: the packed launch, then the launch that takes the
    // tiles outside the packed range (it only skips items when there are none)
    const int wide_grid = std::max(1, grid / 4);
    if (adjoint) {
        switch (dl) {
            case 1: k_ht_adj_f32<NDIM, KERNEL, 1, Tval, kRoleAll><<<grid, kHtBlock, 0, st>>>(P, t, part); break;
            case 2:
                k_ht_adj_f32<NDIM, KERNEL, 2, Tval, kRolePacked><<<grid, kHtBlock, 0, st>>>(P, t, part);
                k_ht_adj_f32<NDIM, KERNEL, 2, Tval, kRoleWide><<<wide_grid, kHtBlock, 0, st>>>(P, t, part);
                break;
            case 4:
                if (KERNEL == TOPOT_FOURIER) return cudaErrorInvalidValue;
                k_ht_adj_f32<NDIM, (KERNEL == TOPOT_FOURIER ? TOPOT_LAPLACE : KERNEL), 4, Tval, kRolePacked>
                    <<<grid, kHtBlock, 0, st>>>(P, t, part);
                k_ht_adj_f32<NDIM, (KERNEL == TOPOT_FOURIER ? TOPOT_LAPLACE : KERNEL), 4, Tval, kRoleWide>
                    <<<wide_grid, kHtBlock, 0, st>>>(P, t, part);
                break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        if (split != 1 && (split != 2 || (dl != 2 && dl != 4))) return cudaErrorInvalidValue;
        switch (dl) {
            case 1: k_ht_f32<NDIM, KERNEL, 1, Tval, kRoleAll, 1><<<grid, kHtBlock, 0, st>>>(P, t, part); break;
            case 2:
                if (split == 2) launch_fwd_pair<NDIM, KERNEL, 2, Tval, 2>(P, t, grid, wide_grid, part, st);
                else launch_fwd_pair<NDIM, KERNEL, 2, Tval, 1>(P, t, grid, wide_grid, part, st);
                break;
            case 4:
                if (split == 2) launch_fwd_pair<NDIM, KERNEL, 4, Tval, 2>(P, t, grid, wide_grid, part, st);
                else launch_fwd_pair<NDIM, KERNEL, 4, Tval, 1>(P, t, grid, wide_grid, part, st);
                break;
            case 8:
                if (KERNEL != TOPOT_LAPLACE) return cudaErrorInvalidValue;
                launch_fwd_pair<NDIM, TOPOT_LAPLACE, 8, Tval, 1>(P, t, grid, wide_grid, part, st);
                break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <int NDIM, int DL, bool ADJ, typename Tval>
static cudaError_t launch_ht_table_k(const EvalPlan& P, const TablesDev& t, int grid, double* part,
                                     cudaStream_t st) {
    auto kern = k_ht_table_f32<NDIM, DL, ADJ, Tval>;
    static const cudaError_t attr = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float4) * kTabStage + sizeof(float2) * (kTabMaxK + 1)));
    if (attr != cudaSuccess) return attr;
    if (P.ktab_k < 2 || P.ktab_k > kTabMaxK) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float4) * kTabStage + sizeof(float2) * (size_t)(P.ktab_k + 1);
    kern<<<grid, kHtBlock, smem, st>>>(P, t, part);
    return cudaGetLastError();
}

template <int NDIM, typename Tval>
static cudaError_t launch_ht_table(const EvalPlan& P, const TablesDev& t, int precision, bool adjoint, int dl,
                                   int grid, double* part, cudaStream_t st) {
    if (precision == TOPOT_FP64) {
        if (adjoint) k_ht_adj_f64<NDIM, TOPOT_TABLE, Tval><<<grid, kHtBlock, 0, st>>>(P, t, part);
        else k_ht_f64<NDIM, TOPOT_TABLE, Tval><<<grid, kHtBlock, 0, st>>>(P, t, part);
        return cudaGetLastError();
    }
    switch (dl) {
        case 1: return adjoint ? launch_ht_table_k<NDIM, 1, true, Tval>(P, t, grid, part, st)
                               : launch_ht_table_k<NDIM, 1, false, Tval>(P, t, grid, part, st);
        case 2: return adjoint ? launch_ht_table_k<NDIM, 2, true, Tval>(P, t, grid, part, st)
                               : launch_ht_table_k<NDIM, 2, false, Tval>(P, t, grid, part, st);
        case 4: return adjoint ? launch_ht_table_k<NDIM, 4, true, Tval>(P, t, grid, part, st)
                               : launch_ht_table_k<NDIM, 4, false, Tval>(P, t, grid, part, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NDIM, typename Tval>
static cudaError_t launch_ht_n(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint,
                               int dl, int split, int grid, double* part, cudaStream_t st) {
    switch (kernel) {
        case TOPOT_LAPLACE:
            return launch_ht_k<NDIM, TOPOT_LAPLACE, Tval>(P, t, precision, adjoint, dl, split, grid, part, st);
        case TOPOT_FOURIER:
            return launch_ht_k<NDIM, TOPOT_FOURIER, Tval>(P, t, precision, adjoint, dl, split, grid, part, st);
        case TOPOT_BESSEL:
            return launch_ht_k<NDIM, TOPOT_BESSEL, Tval>(P, t, precision, adjoint, dl, split, grid, part, st);
        case TOPOT_SINE:
            return launch_ht_k<NDIM, TOPOT_SINE, Tval>(P, t, precision, adjoint, dl, split, grid, part, st);
        case TOPOT_TABLE: return launch_ht_table<NDIM, Tval>(P, t, precision, adjoint, dl, grid, part, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ht_gen(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint, int grid,
                          double* part, cudaStream_t st);

cudaError_t launch_ht(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint, int dl,
                      int split, int grid, double* part, cudaStream_t st) {
    if (t.n == 4) return launch_ht_gen(P, t, kernel, precision, adjoint, grid, part, st);   // dl = 1
    if (t.n == 2) {
        if (t.val_bytes == 2)
            return launch_ht_n<2, int16_t>(P, t, kernel, precision, adjoint, dl, split, grid, part, st);
        return launch_ht_n<2, int32_t>(P, t, kernel, precision, adjoint, dl, split, grid, part, st);
    }
    if (t.val_bytes == 2) return launch_ht_n<3, int16_t>(P, t, kernel, precision, adjoint, dl, split, grid, part, st);
    return launch_ht_n<3, int32_t>(P, t, kernel, precision, adjoint, dl, split, grid, part, st);
}

cudaError_t launch_ht_combine(const EvalPlan& P, int n, int B, int kernel, int precision, int tdh,
                              const double* part, const long long* vsum, int S, double* out, cudaStream_t st) {
    const long long rows = (long long)B * P.D;
    k_ht_combine<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(P, n, B, kernel, precision, tdh, part, vsum, S,
                                                                   out);
    return cudaGetLastError();
}

cudaError_t launch_ht_adj_combine(const EvalPlan& P, int n, int B, int kernel, int precision, int tdh,
                                  const double* part, const double* gout, double* gdirs, cudaStream_t st) {
    const long long rows = (long long)P.nsets * P.D;
    k_ht_adj_combine<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(P, n, B, kernel, precision, tdh, part,
                                                                       gout, gdirs);
    return cudaGetLastError();
}

}  // namespace topot
