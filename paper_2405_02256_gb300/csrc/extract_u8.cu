// K1 for 8-bit images and volumes (Section 3, Delta^-; Section 4.2, preprocessing).
//
// The general kernel (extract.cu) handles int32 pixels.  This one is the path of every
// 8-bit batch.  A tile is R full rows of one plane (m_0 <= W_max) or a piece of one row
// of at most W_max columns; one block per tile.  Thread t owns a strip of STRIP
// consecutive vertices of one tile row (8 in 2-D, 4 in 3-D).
//
// Arithmetic.  A pixel value b in [0, 255] is held as the half-precision number 1024 + b
// (bits 0x64:b, one byte permute per two pixels).  Minima keep the common offset, and a
// difference of two such numbers is an integer in [-255, 255].  Grouping
//   Delta^-_o(v) = (phi(v) - e_0) + (f_01 - e_1) + (f_02 - e_2) + (f_12 - c)       (3-D)
//   Delta^-_o(v) = (phi(v) - e_0) + (f_01 - e_1)                                 (2-D)
// (e_k the edge minima, f_kl the square minima, c the cube minimum of the lower star
// fixed by o) keeps every partial sum an integer of magnitude <= 4 * 255 and every Delta
// table value (a difference of two lower-star values) of magnitude <= 2040 < 2048: all
// exact in half precision.  Two vertices share one f16x2 register.
//
// Minima.  With H[x] = min(X[x], X[x+1]) on each staged row X, the vertical edge minima
// V = min(M, U or D) (M the centre row, U / D the rows y -+ 1), Q = min(H_M, H_U or H_D)
// the 2x2 boxes, and in 3-D the same quantities on the planes z -+ 1.  Orthant bit k set
// means eps_k = -1: the lower star leaves v towards +1 on axis k.  A pixel outside the
// image is staged as 0, the smallest value, so every cell that leaves the image
// contributes nothing.
//
// Compaction.  Per segment (2^n lower tables, 2^(n-1) Delta tables) every thread counts
// its non-zero values; a warp scan and a scan of the warp totals give each thread its
// place in a tile-compact shared-memory buffer (one word per entry: tile-local vertex
// index << 16 | half-precision value); the tile aggregates go to the decoupled look-back;
// the block then writes each segment's run.  Warp 0 does the look-back over a window of
// 32 predecessor tiles at a time, for all segments at once, while the other warps fill
// the buffer.
#include <cuda_fp16.h>

#include "internal.cuh"

namespace topot {

namespace {

template <int NDIM> struct U8Cfg;
template <> struct U8Cfg<2> {
    static constexpr int B = 256;       // threads per block
    static constexpr int STRIP = 8;     // vertices per thread
    static constexpr int MINB = 4;      // resident blocks per SM (registers <= 64)
};
template <> struct U8Cfg<3> {
    static constexpr int B = 512;       // 3-D: larger tiles (2048 voxels) halve the per-tile cost
    static constexpr int STRIP = 4;
    static constexpr int MINB = 2;      // registers <= 64
};

constexpr int kPadB = 16;               // staged row interior starts 16 bytes in
constexpr unsigned kFull = 0xffffffffu;
constexpr int kHdrPerWarp = 128;       // shared-memory header bytes per warp

template <int NDIM> struct U8Layout {
    static constexpr int B = U8Cfg<NDIM>::B;
    static constexpr int NW = B / 32;
    static constexpr int STRIP = U8Cfg<NDIM>::STRIP;
    static constexpr int PAIRS = STRIP / 2;
    static constexpr int NO = 1 << NDIM;
    static constexpr int SEG = NO + NO / 2;
    static constexpr int WORDS = SEG / 2;            // two 16-bit counts per word
    static constexpr int CAP = B * STRIP;            // vertices per tile (max); < 2^16
    // header
    static constexpr int OFF_BAR = 0;
    static constexpr int OFF_INT = 8;
    static constexpr int OFF_WSUM = 32;                       // [NW][8] words
    static constexpr int OFF_WEX = OFF_WSUM + NW * 32;        // [NW][8] words
    static constexpr int OFF_TOT = OFF_WEX + NW * 32;         // [8] words
    static constexpr int OFF_PREF = OFF_TOT + 32;             // [SEG] long long
    static constexpr int OFF_OUT = NW * kHdrPerWarp;          // [SEG * CAP] words
    static constexpr int OFF_STAGE = OFF_OUT + 4 * SEG * CAP;
    static_assert(OFF_PREF + 8 * SEG <= NW * kHdrPerWarp, "shared-memory header too small");
    static_assert(CAP <= 65536, "tile-local vertex index must fit 16 bits");
};

__device__ __forceinline__ uint32_t hmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// One staged row around a strip: vertex pairs P[p] = (X[2p], X[2p+1]) and the
// horizontal edge minima HR[p] = (H[2p], H[2p+1]), HL[p] = (H[2p-1], H[2p]).
// sp is STRIP-byte aligned; sp[-1] and sp[STRIP] are the neighbours of the strip, read
// only when hasL / hasR (else outside the image).
template <int PAIRS>
__device__ __forceinline__ void row_pairs(const uint8_t* sp, bool hasL, bool hasR, uint32_t (&P)[PAIRS],
                                          uint32_t (&HR)[PAIRS], uint32_t (&HL)[PAIRS]) {
    constexpr uint32_t K = 0x64646464u;
    uint32_t w[2];
    if constexpr (PAIRS == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(sp);
        w[0] = v.x;
        w[1] = v.y;
    } else {
        w[0] = *reinterpret_cast<const uint32_t*>(sp);
        w[1] = 0;
    }
    const uint32_t l = hasL ? (uint32_t)sp[-1] : 0u;   // 0 = outside the image
    const uint32_t h = hasR ? (uint32_t)sp[2 * PAIRS] : 0u;
#pragma unroll
    for (int p = 0; p < PAIRS; ++p) P[p] = __byte_perm(w[p >> 1], K, (p & 1) ? 0x4342 : 0x4140);
    uint32_t S[PAIRS];                                   // S[p] = (X[2p+1], X[2p+2])
#pragma unroll
    for (int p = 0; p + 1 < PAIRS; ++p) S[p] = __byte_perm(P[p], P[p + 1], 0x5432);
    S[PAIRS - 1] = __byte_perm(P[PAIRS - 1], h, 0x3432);
    const uint32_t L0 = __byte_perm(l, P[0], 0x5450);    // (X[-1], X[0])
#pragma unroll
    for (int p = 0; p < PAIRS; ++p) {
        HR[p] = hmin2(P[p], S[p]);
        HL[p] = hmin2(p == 0 ? L0 : S[p - 1], P[p]);
    }
}

// Segment values of one 2-D strip; sp points at row U (y - 1).  D[o] (o < 4) the lower
// tables, D[4 + r] = D[r] - D[r ^ 3].
__device__ __forceinline__ void strip_values2(const uint8_t* sp, int rs, bool hasL, bool hasR,
                                              uint32_t (&D)[6][4]) {
    uint32_t PM[4], HRM[4], HLM[4];
    row_pairs<4>(sp + rs, hasL, hasR, PM, HRM, HLM);
    uint32_t Al[4], Ar[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        Al[p] = hsub2(PM[p], HLM[p]);
        Ar[p] = hsub2(PM[p], HRM[p]);
    }
#pragma unroll
    for (int yd = 0; yd < 2; ++yd) {                      // 0: row U (eps_1 = +1), 1: row D
        uint32_t PY[4], HRY[4], HLY[4];
        row_pairs<4>(sp + 2 * yd * rs, hasL, hasR, PY, HRY, HLY);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t V = hmin2(PM[p], PY[p]);
            D[2 * yd][p] = hadd2(Al[p], hsub2(hmin2(HLY[p], HLM[p]), V));
            D[2 * yd + 1][p] = hadd2(Ar[p], hsub2(hmin2(HRY[p], HRM[p]), V));
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        D[4][p] = hsub2(D[0][p], D[3][p]);
        D[5][p] = hsub2(D[1][p], D[2][p]);
    }
}

// Segment values of one 3-D strip; sp points at row U of the centre plane, planes are ps
// bytes apart.  D[o] (o < 8) the lower tables, D[8 + r] = D[r] - D[r ^ 7].
__device__ __forceinline__ void strip_values3(const uint8_t* sp, int rs, int ps, bool hasL, bool hasR,
                                              uint32_t (&D)[12][2]) {
    // centre plane: per pair and orthant (x, y) bits the partial sum
    // S1 = (phi - e_0) + (f_01 - e_1), the box minima Q, the edge minima H_M, V
    uint32_t PM[2], HM[2][2], V[2][2], Q[2][2][2], S1[2][2][2];
    {
        uint32_t HRM[2], HLM[2];
        row_pairs<2>(sp + rs, hasL, hasR, PM, HRM, HLM);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            HM[p][0] = HLM[p];
            HM[p][1] = HRM[p];
        }
#pragma unroll
        for (int yd = 0; yd < 2; ++yd) {
            uint32_t PY[2], HRY[2], HLY[2];
            row_pairs<2>(sp + 2 * yd * rs, hasL, hasR, PY, HRY, HLY);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                V[p][yd] = hmin2(PM[p], PY[p]);
                Q[p][0][yd] = hmin2(HLY[p], HLM[p]);
                Q[p][1][yd] = hmin2(HRY[p], HRM[p]);
#pragma unroll
                for (int xd = 0; xd < 2; ++xd)
                    S1[p][xd][yd] = hadd2(hsub2(PM[p], HM[p][xd]), hsub2(Q[p][xd][yd], V[p][yd]));
            }
        }
    }
#pragma unroll
    for (int zd = 0; zd < 2; ++zd) {                      // 0: plane z - 1 (eps_2 = +1), 1: z + 1
        const uint8_t* sz = sp + (2 * zd - 1) * ps;
        uint32_t PMz[2], HRMz[2], HLMz[2];
        row_pairs<2>(sz + rs, hasL, hasR, PMz, HRMz, HLMz);
        uint32_t Vz[2], C[2][2];                          // e_2, and f_02 - e_2 per x side
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            Vz[p] = hmin2(PM[p], PMz[p]);
            C[p][0] = hsub2(hmin2(HM[p][0], HLMz[p]), Vz[p]);
            C[p][1] = hsub2(hmin2(HM[p][1], HRMz[p]), Vz[p]);
        }
#pragma unroll
        for (int yd = 0; yd < 2; ++yd) {
            uint32_t PYz[2], HRYz[2], HLYz[2];
            row_pairs<2>(sz + 2 * yd * rs, hasL, hasR, PYz, HRYz, HLYz);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const uint32_t f12 = hmin2(V[p][yd], hmin2(PMz[p], PYz[p]));
                const uint32_t Qz0 = hmin2(HLYz[p], HLMz[p]);
                const uint32_t Qz1 = hmin2(HRYz[p], HRMz[p]);
                const int o = 2 * yd + 4 * zd;
                D[o][p] = hadd2(hadd2(S1[p][0][yd], C[p][0]), hsub2(f12, hmin2(Q[p][0][yd], Qz0)));
                D[o + 1][p] = hadd2(hadd2(S1[p][1][yd], C[p][1]), hsub2(f12, hmin2(Q[p][1][yd], Qz1)));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int p = 0; p < 2; ++p) D[8 + r][p] = hsub2(D[r][p], D[r ^ 7][p]);
}

// Top-dimensional construction (Section 4.1), corner v with the 2^n pixels X_g = V(v + g),
// g in {0,1}^n, of the u8 corner image V.  The lower-star box of orthant o spanning the
// axes delta takes the minimum t_delta over the pixels with g_k = o_k on those axes, and
//   Delta^-_o(v) = sum_delta (-1)^|delta| t_delta,
// grouped (2-D) as (t_0 - t_x) + (t_xy - t_y) and (3-D) as (t_0 - t_x) + (t_xy - t_y)
// + (t_xz - t_z) + (t_yz - t_xyz): each bracket is a difference of a minimum and a
// minimum over a superset or subset of its pixels, of magnitude <= 255, so every partial
// sum is an exact half-precision integer.

// One staged run of the corner image: P[p] = (X[2p], X[2p+1]), S[p] = (X[2p+1], X[2p+2]);
// sp[2 PAIRS] (the next position) is always staged.
template <int PAIRS>
__device__ __forceinline__ void run_pairs(const uint8_t* sp, uint32_t (&P)[PAIRS], uint32_t (&S)[PAIRS]) {
    constexpr uint32_t K = 0x64646464u;
    uint32_t w[2];
    if constexpr (PAIRS == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(sp);
        w[0] = v.x;
        w[1] = v.y;
    } else {
        w[0] = *reinterpret_cast<const uint32_t*>(sp);
        w[1] = 0;
    }
    const uint32_t h = sp[2 * PAIRS];
#pragma unroll
    for (int p = 0; p < PAIRS; ++p) P[p] = __byte_perm(w[p >> 1], K, (p & 1) ? 0x4342 : 0x4140);
#pragma unroll
    for (int p = 0; p + 1 < PAIRS; ++p) S[p] = __byte_perm(P[p], P[p + 1], 0x5432);
    S[PAIRS - 1] = __byte_perm(P[PAIRS - 1], h, 0x3432);
}

// 2-D: s0 the run of row y, s1 of row y + 1.  D[o] (o < 4) lower tables, D[4 + r] =
// D[r] - D[r ^ 3].
__device__ __forceinline__ void strip_values_top2(const uint8_t* s0, const uint8_t* s1, uint32_t (&D)[6][4]) {
    uint32_t X0[4], X1[4], Y0[4], Y1[4];      // X_{gx gy}: (g_x, g_y) = (0,0), (1,0); (0,1), (1,1)
    run_pairs<4>(s0, X0, X1);
    run_pairs<4>(s1, Y0, Y1);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t cm0 = hmin2(X0[p], Y0[p]), cm1 = hmin2(X1[p], Y1[p]);   // t_x: g_x = 0, 1
        const uint32_t rm0 = hmin2(X0[p], X1[p]), rm1 = hmin2(Y0[p], Y1[p]);   // t_y: g_y = 0, 1
        const uint32_t t0 = hmin2(cm0, cm1);
        const uint32_t a0 = hsub2(t0, cm0), a1 = hsub2(t0, cm1);
        D[0][p] = hadd2(a0, hsub2(X0[p], rm0));
        D[1][p] = hadd2(a1, hsub2(X1[p], rm0));
        D[2][p] = hadd2(a0, hsub2(Y0[p], rm1));
        D[3][p] = hadd2(a1, hsub2(Y1[p], rm1));
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        D[4][p] = hsub2(D[0][p], D[3][p]);
        D[5][p] = hsub2(D[1][p], D[2][p]);
    }
}

// 3-D: sr[2 g_z + g_y] the run of row y + g_y of plane z + g_z.  D[o] (o < 8) lower
// tables, D[8 + r] = D[r] - D[r ^ 7].
__device__ __forceinline__ void strip_values_top3(const uint8_t* const (&sr)[4], uint32_t (&D)[12][2]) {
    uint32_t X[2][2][2][2];                   // [g_z][g_y][g_x][pair]
#pragma unroll
    for (int gz = 0; gz < 2; ++gz)
#pragma unroll
        for (int gy = 0; gy < 2; ++gy) run_pairs<2>(sr[2 * gz + gy], X[gz][gy][0], X[gz][gy][1]);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        uint32_t txy[2][2], txz[2][2], tyz[2][2], tx[2], ty[2], tz[2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                txy[a][c] = hmin2(X[0][a][c][p], X[1][a][c][p]);   // [g_y][g_x]
                txz[a][c] = hmin2(X[a][0][c][p], X[a][1][c][p]);   // [g_z][g_x]
                tyz[a][c] = hmin2(X[a][c][0][p], X[a][c][1][p]);   // [g_z][g_y]
            }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            tx[a] = hmin2(txy[0][a], txy[1][a]);
            ty[a] = hmin2(txy[a][0], txy[a][1]);
            tz[a] = hmin2(txz[a][0], txz[a][1]);
        }
        const uint32_t t0 = hmin2(tx[0], tx[1]);
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            const uint32_t u = hadd2(hsub2(t0, tx[ox]), hsub2(txy[oy][ox], ty[oy]));
            const uint32_t w = hadd2(hsub2(txz[oz][ox], tz[oz]), hsub2(tyz[oz][oy], X[oz][oy][ox][p]));
            D[o][p] = hadd2(u, w);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int p = 0; p < 2; ++p) D[8 + r][p] = hsub2(D[r][p], D[r ^ 7][p]);
}

// Corners of the image (every coordinate 0 or m_k - 1) in the orthant pointing out of
// the image on every axis: every box but the vertex itself has no pixel, and those 255s
// sum to -255 instead of 0.  Adds 255 there and recomputes the Delta tables.
template <int NDIM, int SEG, int PAIRS>
__device__ __forceinline__ void top_corner_fix(uint32_t (&D)[SEG][PAIRS], int xs, int m0, bool ylast, bool zlast) {
    constexpr int NO = 1 << NDIM;
#pragma unroll
    for (int k = 0; k < 2 * PAIRS; ++k) {
        const int x = xs + k;
        if (x == 0 || x == m0 - 1) {
            const int ob = (x == m0 - 1 ? 1 : 0) | (ylast ? 2 : 0) | (zlast ? 4 : 0);
            const uint32_t add = (k & 1) ? 0x5BF80000u : 0x00005BF8u;   // 255.0 in the vertex's half
#pragma unroll
            for (int o = 0; o < NO; ++o)
                if (o == ob) D[o][k >> 1] = hadd2(D[o][k >> 1], add);
        }
    }
#pragma unroll
    for (int r = 0; r < NO / 2; ++r)
#pragma unroll
        for (int p = 0; p < PAIRS; ++p) D[NO + r][p] = hsub2(D[r][p], D[r ^ (NO - 1)][p]);
}

// number of non-zero halves of the pairs
template <int PAIRS>
__device__ __forceinline__ uint32_t count_nonzero(const uint32_t (&d)[PAIRS]) {
    uint32_t c = 0;
#pragma unroll
    for (int p = 0; p < PAIRS; ++p)
        asm("{\n\t.reg .pred a, b;\n\t"
            "setp.ne.f16x2 a|b, %1, %2;\n\t"
            "@a add.u32 %0, %0, 1;\n\t"
            "@b add.u32 %0, %0, 1;\n\t}"
            : "+r"(c) : "r"(d[p]), "r"(0u));
    return c;
}

// appends the non-zero halves of d (tile-local vertex of half 0 is J0 >> 16, of half 1
// J1 >> 16) at shared address a, advancing it
__device__ __forceinline__ void append_pair(uint32_t& a, uint32_t d, uint32_t J0, uint32_t J1) {
    const uint32_t w0 = __byte_perm(d, J0, 0x7610);
    const uint32_t w1 = __byte_perm(d, J1, 0x7632);
    asm volatile("{\n\t.reg .pred a, b;\n\t"
                 "setp.ne.f16x2 a|b, %1, %4;\n\t"
                 "@a st.shared.u32 [%0], %2;\n\t"
                 "@a add.u32 %0, %0, 4;\n\t"
                 "@b st.shared.u32 [%0], %3;\n\t"
                 "@b add.u32 %0, %0, 4;\n\t}"
                 : "+r"(a) : "r"(d), "r"(w0), "r"(w1), "r"(0u) : "memory");
}

template <int WORDS>
__device__ __forceinline__ uint32_t field16(const uint32_t (&w)[WORDS], int s) {
    return (w[s >> 1] >> (16 * (s & 1))) & 0xffffu;
}

__device__ __forceinline__ FastDiv ldg_fastdiv(const FastDiv* f) {
    FastDiv r;
    r.d = 0;
    r.mul = __ldg(&f->mul);
    r.shift = __ldg(&f->shift);
    return r;
}

}  // namespace

// Geometry of one tile (image b, local tile index lt).
struct TileGeo {
    int m0, m1, m2, W, R, spr, RS, segs, tpp, lt, z, nz, y0, x0, rows, cols, packed;
    long long tile_begin;
    const uint8_t* img;
};

template <int NDIM, bool TOP>
__device__ __forceinline__ TileGeo tile_geometry(const ExtractArgs& p, int b, long long ticket) {
    const ImgDesc* Ip = p.t.img + b;
    TileGeo g;
    g.m0 = __ldg(&Ip->m[0]);
    g.m1 = __ldg(&Ip->m[1]);
    g.m2 = __ldg(&Ip->m[2]);
    g.W = __ldg(&Ip->W);
    g.R = __ldg(&Ip->R);
    g.spr = __ldg(&Ip->spr);
    g.RS = __ldg(&Ip->rs);
    g.segs = __ldg(&Ip->segs_per_row);
    g.tpp = __ldg(&Ip->tiles_per_plane);
    g.packed = __ldg(&Ip->packed);
    g.tile_begin = __ldg(&Ip->tile_begin);
    g.lt = (int)(ticket - g.tile_begin);
    if (TOP) {   // a run of positions of the corner image
        const long long Q = (long long)__ldg(&Ip->top_pitch) * g.m1 * g.m2;
        g.z = 0;
        g.nz = 1;
        g.y0 = 0;
        g.x0 = g.lt * g.W;
        g.rows = 1;
        g.cols = (int)min((long long)g.W, Q - g.x0);
        g.img = reinterpret_cast<const uint8_t*>(p.pixels) + __ldg(&Ip->offset);
        return g;
    }
    const int zl = NDIM == 3 ? (int)fastdiv((uint32_t)g.lt, ldg_fastdiv(&Ip->div_tpp)) : 0;   // owned plane
    g.z = NDIM == 3 ? __ldg(&Ip->zlo) + zl : 0;                                            // volume plane
    g.nz = NDIM == 3 ? __ldg(&Ip->nz) : 1;
    const int rem = g.lt - zl * g.tpp;
    const int rb = (int)fastdiv((uint32_t)rem, ldg_fastdiv(&Ip->div_segs));
    const int sg = rem - rb * g.segs;
    g.y0 = rb * g.R;
    g.x0 = sg * g.W;
    g.rows = min(g.R, g.m1 - g.y0);
    g.cols = min(g.W, g.m0 - g.x0);
    // pixels of plane zz at img + zz m_1 m_0: the buffer starts at plane zbase (a slab)
    g.img = reinterpret_cast<const uint8_t*>(p.pixels) + __ldg(&Ip->offset) -
            (NDIM == 3 ? (long long)__ldg(&Ip->zbase) * g.m1 * g.m0 : 0ll);
    return g;
}

// Bulk copies of the tile's staged rows, issued by one thread (the mbarrier counts the
// bytes); rows that need plain loads or zeros are left to the block.
template <int NDIM>
__device__ __forceinline__ void issue_stage_copies(const TileGeo& g, uint8_t* stage, uint64_t* bar) {
    constexpr int kNP = NDIM == 3 ? 3 : 1;
    const int srows = g.rows + 2;
    const int PS = (g.R + 2) * g.RS;
    if (g.packed) {
        if ((reinterpret_cast<uintptr_t>(g.img) & 15) != 0) {   // unaligned pixel buffer: plain loads
            mbar_arrive_expect_tx(bar, 0u);
            return;
        }
        unsigned bytes = 0;
        for (int pl = 0; pl < kNP; ++pl) {
            const int zz = g.z + pl - (NDIM == 3 ? 1 : 0);
            if (zz < 0 || zz >= g.m2) continue;
            bytes += (unsigned)((min(g.y0 + g.rows + 1, g.m1) - max(g.y0 - 1, 0)) * g.m0);
        }
        mbar_arrive_expect_tx(bar, bytes);
        for (int pl = 0; pl < kNP; ++pl) {
            const int zz = g.z + pl - (NDIM == 3 ? 1 : 0);
            if (zz < 0 || zz >= g.m2) continue;
            const int ylo = max(g.y0 - 1, 0), yhi = min(g.y0 + g.rows + 1, g.m1);
            bulk_g2s(stage + kPadB + pl * PS + (ylo - (g.y0 - 1)) * g.m0,
                     g.img + ((long long)zz * g.m1 + ylo) * g.m0, (unsigned)((yhi - ylo) * g.m0), bar);
        }
        return;
    }
    unsigned bytes = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            mbar_arrive_expect_tx(bar, bytes);
            if (bytes == 0) return;
        }
        if ((g.cols & 15) != 0) continue;
        for (int q = 0; q < kNP * srows; ++q) {
            const int pl = NDIM == 3 ? q / srows : 0;
            const int rr = q - pl * srows;
            const int zz = g.z + pl - (NDIM == 3 ? 1 : 0);
            const int yy = g.y0 + rr - 1;
            if (zz < 0 || zz >= g.m2 || yy < 0 || yy >= g.m1) continue;
            const uint8_t* src = g.img + ((long long)zz * g.m1 + yy) * g.m0 + g.x0;
            if ((reinterpret_cast<uintptr_t>(src) & 15) != 0) continue;
            if (pass == 0) bytes += (unsigned)g.cols;
            else bulk_g2s(stage + pl * PS + rr * g.RS + kPadB, src, (unsigned)g.cols, bar);
        }
    }
}

// Top construction: the tile's run and the runs at the offsets of the other pixels of a
// corner (+pitch; in 3-D +plane, +plane+pitch), each W + 16 bytes (the last position reads
// one beyond), clipped at the end of the corner image (the block fills the rest with 255).
template <int NDIM>
__device__ __forceinline__ int top_run_len(const TileGeo& g, int P, int k) {
    const long long plane = (long long)P * g.m1;
    const long long Q = plane * g.m2;
    const long long start = g.x0 + (k & 1) * (long long)P + (k >> 1) * plane;
    return (int)max(0ll, min((long long)g.RS, Q - start));
}

template <int NDIM>
__device__ __forceinline__ void issue_top_copies(const TileGeo& g, int P, uint8_t* stage, uint64_t* bar) {
    constexpr int kNB = NDIM == 3 ? 4 : 2;
    const long long plane = (long long)P * g.m1;
    unsigned bytes = 0;
#pragma unroll
    for (int k = 0; k < kNB; ++k) bytes += (unsigned)top_run_len<NDIM>(g, P, k);
    mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
    for (int k = 0; k < kNB; ++k) {
        const int len = top_run_len<NDIM>(g, P, k);
        if (len > 0)
            bulk_g2s(stage + k * g.RS, g.img + g.x0 + (k & 1) * (long long)P + (k >> 1) * plane, (unsigned)len, bar);
    }
}

template <int NDIM, bool TOP>
__global__ void __launch_bounds__(U8Cfg<NDIM>::B, U8Cfg<NDIM>::MINB) k_extract_u8(ExtractArgs p) {
    using Ly = U8Layout<NDIM>;
    constexpr int kB = Ly::B, kNW = Ly::NW, kSeg = Ly::SEG, kNO = Ly::NO;
    constexpr int kWords = Ly::WORDS, kStrip = Ly::STRIP, kPairs = Ly::PAIRS;
    constexpr int kNP = NDIM == 3 ? 3 : 1;               // staged planes

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Ly::OFF_BAR);
    int* sh_int = reinterpret_cast<int*>(smem_raw + Ly::OFF_INT);
    uint32_t* sh_wsum = reinterpret_cast<uint32_t*>(smem_raw + Ly::OFF_WSUM);
    uint32_t* sh_wex = reinterpret_cast<uint32_t*>(smem_raw + Ly::OFF_WEX);
    uint32_t* sh_tot = reinterpret_cast<uint32_t*>(smem_raw + Ly::OFF_TOT);
    long long* sh_pref = reinterpret_cast<long long*>(smem_raw + Ly::OFF_PREF);
    uint32_t* out = reinterpret_cast<uint32_t*>(smem_raw + Ly::OFF_OUT);
    uint8_t* stage = smem_raw + Ly::OFF_STAGE;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const TablesDev& T = p.t;
    // every volume binary: the binary kernels built all tables (grid-uniform)
    if (p.nonbin && __ldg(&p.nonbin[T.B]) == 0u) return;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        // ticket -> (image, local tile) -> global tile number, which indexes the look-back
        const unsigned ticket = atomicAdd(p.ticket, 1u);
        const int2 bl = __ldg(&p.order[ticket]);
        const int lo = bl.x;
        const long long gt = __ldg(&T.img[lo].tile_begin) + bl.y;
        sh_int[0] = (int)gt;
        sh_int[1] = lo;
        if (p.nonbin && __ldg(&p.nonbin[lo]) == 0u) {
            sh_int[1] = -1;   // a binary volume: the binary kernels build its tables
        } else {
            // the tile's bulk copies go out before the block synchronises
            const TileGeo g0 = tile_geometry<NDIM, TOP>(p, lo, gt);
            if (TOP) issue_top_copies<NDIM>(g0, __ldg(&T.img[lo].top_pitch), stage, bar);
            else issue_stage_copies<NDIM>(g0, stage, bar);
        }
    }
    __syncthreads();

    const long long ticket = (unsigned)sh_int[0];
    const int b = sh_int[1];
    if (b < 0) return;   // block-uniform; no copy was issued
    const ImgDesc* Ip = T.img + b;
    const TileGeo G = tile_geometry<NDIM, TOP>(p, b, ticket);
    const int m0 = G.m0, m1 = G.m1, m2 = G.m2, R = G.R, spr = G.spr, RS = G.RS, tpp = G.tpp;
    const long long tile_begin = G.tile_begin;
    const int lt = G.lt, z = G.z, y0 = G.y0, x0 = G.x0, rows = G.rows, cols = G.cols;
    const int L0 = (z * m1 + y0) * m0 + x0;            // linear index of the tile's first vertex
    const uint8_t* img = G.img;

    // ---- 1. stage rows y0 - 1 .. y0 + rows (planes z - 1 .. z + 1); zeros outside ----------
    // Packed images (full-row tiles, m_0 and the image offset multiples of 16): the rows of
    // a plane are contiguous in the image and in the stage (row stride m_0), so one bulk
    // copy per plane moves them; the strips at the two ends of a row treat their outer
    // neighbour as outside.  Other images: one staged row per image row, with a one-pixel
    // halo and zero tail, interiors by bulk copy where 16-byte aligned.
    const int srows = rows + 2;
    const int PS = (R + 2) * RS;                       // staged plane stride
    const bool packed = __ldg(&Ip->packed) != 0;
    if (TOP) {
        // the clipped ends of the runs: 255 (no pixel)
        const int P = __ldg(&Ip->top_pitch);
#pragma unroll
        for (int k = 0; k < (NDIM == 3 ? 4 : 2); ++k) {
            const int len = top_run_len<NDIM>(G, P, k);
            uint4* dst = reinterpret_cast<uint4*>(stage + k * RS);
            for (int c = (len >> 4) + tid; c < (RS >> 4); c += kB) dst[c] = make_uint4(~0u, ~0u, ~0u, ~0u);
        }
    } else if (packed) {
        // bulk copies need a 16-byte aligned source: the pixel buffer itself may not be
        const bool bulk = (reinterpret_cast<uintptr_t>(img) & 15) == 0;
        if (!bulk) {
            for (int pl = 0; pl < kNP; ++pl) {
                const int zz = z + pl - (NDIM == 3 ? 1 : 0);
                if (zz < 0 || zz >= m2) continue;
                const int ylo = max(y0 - 1, 0), yhi = min(y0 + rows + 1, m1);
                uint8_t* dst = stage + kPadB + pl * PS + (ylo - (y0 - 1)) * m0;
                const uint8_t* src = img + ((long long)zz * m1 + ylo) * m0;
                for (int c = tid; c < (yhi - ylo) * m0; c += kB) dst[c] = src[c];
            }
        }
        // rows and planes outside the image: zeros (16-byte stores; m_0 is a multiple of 16)
        const int n16 = m0 >> 4;
        for (int q = warp; q < kNP * srows; q += kNW) {
            const int pl = NDIM == 3 ? q / srows : 0;
            const int rr = q - pl * srows;
            const int zz = z + pl - (NDIM == 3 ? 1 : 0);
            const int yy = y0 + rr - 1;
            if (zz >= 0 && zz < m2 && yy >= 0 && yy < m1) continue;
            uint4* dst = reinterpret_cast<uint4*>(stage + kPadB + pl * PS + rr * RS);
            for (int c = lane; c < n16; c += 32) dst[c] = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
        const int span = kStrip * spr;                 // bytes read per staged row: [-1, span]
        auto src_row = [&](int q, bool& inside) -> const uint8_t* {
            const int pl = NDIM == 3 ? q / srows : 0;
            const int rr = q - pl * srows;
            const int zz = z + pl - (NDIM == 3 ? 1 : 0);
            const int yy = y0 + rr - 1;
            inside = zz >= 0 && zz < m2 && yy >= 0 && yy < m1;
            return img + ((long long)zz * m1 + yy) * m0 + x0;
        };
        auto dst_row = [&](int q) -> uint8_t* {
            const int pl = NDIM == 3 ? q / srows : 0;
            return stage + pl * PS + (q - pl * srows) * RS + kPadB;
        };
        for (int q = warp; q < kNP * srows; q += kNW) {
            uint8_t* dst = dst_row(q);
            bool inside;
            const uint8_t* src = src_row(q, inside);
            if (!inside) {
                for (int c = lane - 1; c <= span; c += 32) dst[c] = 0;
                continue;
            }
            const bool bulk = ((cols & 15) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
            if (!bulk)
                for (int c = lane; c < cols; c += 32) dst[c] = src[c];
            if (lane == 0) dst[-1] = x0 > 0 ? src[-1] : (uint8_t)0;
            if (lane == 1) dst[cols] = x0 + cols < m0 ? src[cols] : (uint8_t)0;
            for (int c = cols + 1 + lane; c <= span; c += 32) dst[c] = 0;
        }
    }
    mbar_wait_bounded(bar, 0, T.err);
    __syncthreads();

    // ---- 2. segment values of the thread's strip -------------------------------------------
    const int r = (int)fastdiv((uint32_t)tid, ldg_fastdiv(&Ip->div_spr));
    const int g = tid - r * spr;
    uint32_t D[kSeg][kPairs];
    if (r < rows) {
        if constexpr (TOP) {
            // positions past the end of the corner image read 255 everywhere: all zero
            const uint8_t* s0 = stage + kStrip * g;
            if constexpr (NDIM == 2) {
                strip_values_top2(s0, s0 + RS, D);
            } else {
                const uint8_t* const sr[4] = {s0, s0 + RS, s0 + 2 * RS, s0 + 3 * RS};
                strip_values_top3(sr, D);
            }
            // the corners of the image: boxes with no pixel on every axis do not cancel
            const int P = __ldg(&Ip->top_pitch);
            const int q0 = x0 + kStrip * g;
            const int yq = (int)fastdiv((uint32_t)q0, ldg_fastdiv(&Ip->div_pitch));   // z m_1 + y
            const int xs = q0 - yq * P;
            int yy = yq, zz = 0;
            if (NDIM == 3) {
                zz = (int)fastdiv((uint32_t)yq, ldg_fastdiv(&Ip->div1));
                yy = yq - zz * m1;
            }
            if ((yy == 0 || yy == m1 - 1) && (NDIM == 2 || zz == 0 || zz == m2 - 1) &&
                (xs == 0 || (xs <= m0 - 1 && m0 - 1 < xs + kStrip)))
                top_corner_fix<NDIM>(D, xs, m0, yy == m1 - 1, NDIM == 3 && zz == m2 - 1);
        } else {
            const uint8_t* sp = stage + (NDIM == 3 ? PS : 0) + r * RS + kPadB + kStrip * g;
            const bool hasL = !packed || g > 0, hasR = !packed || g < spr - 1;
            if constexpr (NDIM == 2) strip_values2(sp, RS, hasL, hasR, D);
            else strip_values3(sp, RS, PS, hasL, hasR, D);
        }
    } else {
#pragma unroll
        for (int s = 0; s < kSeg; ++s)
#pragma unroll
            for (int q = 0; q < kPairs; ++q) D[s][q] = 0u;
    }

    // ---- 3. counts, warp scan (16-bit fields, two segments per word) -----------------------
    uint32_t cw[kWords];
#pragma unroll
    for (int i = 0; i < kWords; ++i)
        cw[i] = count_nonzero<kPairs>(D[2 * i]) | (count_nonzero<kPairs>(D[2 * i + 1]) << 16);
    uint32_t iw[kWords];
#pragma unroll
    for (int i = 0; i < kWords; ++i) iw[i] = cw[i];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int i = 0; i < kWords; ++i) {
            const uint32_t y = __shfl_up_sync(kFull, iw[i], d);
            if (lane >= d) iw[i] += y;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < kWords; ++i) sh_wsum[warp * 8 + i] = iw[i];
    }
    __syncthreads();

    uint32_t tot[kWords];
    if (warp == 0) {
        // scan of the warp totals; lanes >= kNW carry zeros
        uint32_t v[kWords], x[kWords];
#pragma unroll
        for (int i = 0; i < kWords; ++i) x[i] = v[i] = lane < kNW ? sh_wsum[lane * 8 + i] : 0u;
#pragma unroll
        for (int d = 1; d < kNW; d <<= 1) {
#pragma unroll
            for (int i = 0; i < kWords; ++i) {
                const uint32_t y = __shfl_up_sync(kFull, x[i], d);
                if (lane >= d) x[i] += y;
            }
        }
#pragma unroll
        for (int i = 0; i < kWords; ++i) {
            if (lane < kNW) sh_wex[lane * 8 + i] = x[i] - v[i];
            tot[i] = __shfl_sync(kFull, x[i], kNW - 1);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kWords; ++i) sh_tot[i] = tot[i];
        }
        __syncwarp();
        asm volatile("bar.arrive 1, %0;" ::"r"(kB) : "memory");

        // ---- 4. decoupled look-back (all segments, 32 predecessors per round) -------------
        unsigned long long* st = p.status + ticket * kSeg;
        uint32_t agg = 0;
#pragma unroll
        for (int s = 0; s < kSeg; ++s)
            if (lane == s) agg = field16(tot, s);
        uint32_t pre = 0;                                   // lane s: exclusive prefix of segment s
        if (lt == 0) {
            if (lane < kSeg) st_relaxed_u64(st + lane, kFlagP | agg);
        } else {
            if (lane < kSeg) st_relaxed_u64(st + lane, kFlagA | agg);
            long long q[kSeg];
            uint32_t acc[kSeg];
#pragma unroll
            for (int s = 0; s < kSeg; ++s) {
                q[s] = ticket - 1;
                acc[s] = 0;
            }
            unsigned done = 0;
            const unsigned long long t0 = __shfl_sync(kFull, dev_time_ns(), 0);
            while (true) {
                unsigned long long w[kSeg];
#pragma unroll
                for (int s = 0; s < kSeg; ++s) {
                    const long long qq = q[s] - lane;
                    w[s] = kFlagP;                           // before the image's first tile
                    if (!((done >> s) & 1u) && qq >= tile_begin) w[s] = ld_relaxed_u64(p.status + qq * kSeg + s);
                }
#pragma unroll
                for (int s = 0; s < kSeg; ++s) {
                    if ((done >> s) & 1u) continue;
                    const unsigned flag = (unsigned)(w[s] >> 62);
                    const uint32_t cnt = (uint32_t)(w[s] & kCountMask);   // < 2^31
                    const unsigned mX = __ballot_sync(kFull, flag == 0u);
                    const unsigned mP = __ballot_sync(kFull, flag == 2u);
                    const unsigned stop = mX | mP;
                    if (stop == 0u) {
                        acc[s] += __reduce_add_sync(kFull, cnt);
                        q[s] -= 32;
                    } else {
                        const int L = __ffs(stop) - 1;
                        if ((mP >> L) & 1u) {
                            acc[s] += __reduce_add_sync(kFull, lane <= L ? cnt : 0u);
                            done |= 1u << s;
                        } else {
                            acc[s] += __reduce_add_sync(kFull, lane < L ? cnt : 0u);
                            q[s] -= L;
                        }
                    }
                }
                if (done == (1u << kSeg) - 1u) break;
                const unsigned long long now = __shfl_sync(kFull, dev_time_ns(), 0);
                if (now - t0 > kWaitLimitNs) {
                    if (lane == 0) dev_set_error(T.err, kDevErrTimeout);
#pragma unroll
                    for (int s = 0; s < kSeg; ++s) acc[s] = 0;
                    break;
                }
            }
#pragma unroll
            for (int s = 0; s < kSeg; ++s)
                if (lane == s) pre = acc[s];
            if (lane < kSeg) st_relaxed_u64(st + lane, kFlagP | (unsigned long long)(pre + agg));
        }
        if (lane < kSeg) {
            const long long N = __ldg(&Ip->N);
            sh_pref[lane] = __ldg(&Ip->seg_base) + (long long)lane * N + pre;
            if (lt == tpp * G.nz - 1) T.seg_count[(long long)b * kSeg + lane] = (long long)(pre + agg);
        }
    } else {
        asm volatile("bar.sync 1, %0;" ::"r"(kB) : "memory");
#pragma unroll
        for (int i = 0; i < kWords; ++i) tot[i] = sh_tot[i];
    }

    // ---- 5. append the thread's entries to the tile-compact buffer --------------------------
    {
        uint32_t ex[kWords];
#pragma unroll
        for (int i = 0; i < kWords; ++i) ex[i] = sh_wex[warp * 8 + i] + iw[i] - cw[i];
        const uint32_t jb = (uint32_t)(r * cols + kStrip * g) << 16;
        uint32_t J[kStrip];
#pragma unroll
        for (int k = 0; k < kStrip; ++k) J[k] = jb + ((uint32_t)k << 16);
        // the warp's totals: segments without an entry in this warp skip the appends
        uint32_t wt[kWords];
#pragma unroll
        for (int i = 0; i < kWords; ++i) wt[i] = __shfl_sync(kFull, iw[i], 31);
        const uint32_t out_u32 = smem_u32(out);
        uint32_t base = 0;
#pragma unroll
        for (int s = 0; s < kSeg; ++s) {
            uint32_t a = out_u32 + 4u * (base + field16(ex, s));
            if (field16(wt, s) != 0u) {
#pragma unroll
                for (int q = 0; q < kPairs; ++q) append_pair(a, D[s][q], J[2 * q], J[2 * q + 1]);
            }
            base += field16(tot, s);
        }
    }
    __syncthreads();

    // ---- 6. write the tile's runs; chi and sum |Delta^-_o| from the lower tables -------------
    // Each warp writes one segment: a lower table, or half of a Delta table (about twice as
    // dense), so a thread sets up one run, not every segment's.  A run starts at an
    // arbitrary arena position g0 and is written in groups of four arena slots aligned to
    // four (one 16-byte index store, one 8-byte value store); the partial groups at the two
    // ends store entry by entry.
    static_assert(kNW == kNO + 2 * (kNO / 2), "one warp per lower table, two per Delta table");
    const FastDiv divp = TOP ? ldg_fastdiv(&Ip->div_pitch) : FastDiv{0u, 0u, 0u};
    const int top_p = TOP ? __ldg(&Ip->top_pitch) : 0;
    const int sw = warp < kNO ? warp : kNO + ((warp - kNO) >> 1);   // this warp's segment
    const int part = warp < kNO ? 0 : ((warp - kNO) & 1);
    const int nparts = warp < kNO ? 1 : 2;
    uint32_t base = 0, nseg = 0;
#pragma unroll
    for (int s = 0; s < kSeg; ++s) {
        const uint32_t ns = field16(tot, s);
        if (s < sw) base += ns;
        if (s == sw) nseg = ns;
    }
    {
        const int n = (int)nseg;
        const long long g0 = sh_pref[sw];
        const int ph = (int)(g0 & 3);
        const int ngroups = (ph + n + 3) >> 2;
        const int q1 = (ngroups * (part + 1)) / nparts;
        int* __restrict__ pi = T.arena_idx + (g0 - ph);
        int16_t* __restrict__ pv = reinterpret_cast<int16_t*>(T.arena_val) + (g0 - ph);
        const uint32_t* o = out + base;
        int rabs = 0, rchi = 0;
        for (int q = (ngroups * part) / nparts + lane; q < q1; q += 32) {
            const int e0 = 4 * q - ph;                  // entry of the group's first slot
            int id[4], v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = e0 + k;
                id[k] = 0;
                v[k] = 0;
                if (e >= 0 && e < n) {
                    const uint32_t w = o[e];
                    v[k] = (int)__half2short_rn(__ushort_as_half((unsigned short)(w & 0xffffu)));
                    if constexpr (TOP) {   // position -> vertex index (rows m_0 long)
                        const int qq = x0 + (int)(w >> 16);
                        const int yq = (int)fastdiv((uint32_t)qq, divp);
                        id[k] = yq * m0 + (qq - yq * top_p);
                    } else {
                        id[k] = L0 + (int)(w >> 16);
                    }
                }
                rabs += abs(v[k]);
                rchi += v[k];
            }
            if (e0 >= 0 && e0 + 4 <= n) {
                *reinterpret_cast<int4*>(pi + 4 * q) = make_int4(id[0], id[1], id[2], id[3]);
                *reinterpret_cast<uint2*>(pv + 4 * q) =
                    make_uint2(__byte_perm((uint32_t)v[0], (uint32_t)v[1], 0x5410),
                               __byte_perm((uint32_t)v[2], (uint32_t)v[3], 0x5410));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = e0 + k;
                    if (e >= 0 && e < n) {
                        pi[4 * q + k] = id[k];
                        pv[4 * q + k] = (int16_t)v[k];
                    }
                }
            }
        }
        // the lower tables' sums straight to the image totals (no block barrier at the end)
        if (sw < kNO) {   // warp-uniform
            const int sa = (int)__reduce_add_sync(kFull, (unsigned)rabs);
            const int sc = (int)__reduce_add_sync(kFull, (unsigned)rchi);
            if (lane == 0) {
                if (sa != 0)
                    atomicAdd(reinterpret_cast<unsigned long long*>(&T.absum[(long long)b * kNO + sw]),
                              (unsigned long long)(long long)sa);
                if (sw == 0 && sc != 0)
                    atomicAdd(reinterpret_cast<unsigned long long*>(&T.chi[b]), (unsigned long long)(long long)sc);
            }
        }
    }
}

// ---- host side ----------------------------------------------------------------------------

int extract_u8_threads(int n) { return n == 2 ? U8Cfg<2>::B : U8Cfg<3>::B; }
int extract_u8_strip(int n) { return n == 2 ? U8Cfg<2>::STRIP : U8Cfg<3>::STRIP; }

size_t extract_u8_smem_bytes(int n, int stage_bytes) {
    return (size_t)(n == 2 ? U8Layout<2>::OFF_STAGE : U8Layout<3>::OFF_STAGE) + (size_t)stage_bytes;
}

template <int NDIM, bool TOP>
static cudaError_t launch_u8(const ExtractArgs& a, cudaStream_t st) {
    auto kern = k_extract_u8<NDIM, TOP>;
    static cudaError_t attr = [&] {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    if (attr != cudaSuccess) return attr;
    kern<<<(unsigned)a.num_tiles, U8Cfg<NDIM>::B, extract_u8_smem_bytes(NDIM, a.stage_bytes), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_extract_u8(int n, bool top, const ExtractArgs& a, cudaStream_t st) {
    if (top) return n == 2 ? launch_u8<2, true>(a, st) : launch_u8<3, true>(a, st);
    return n == 2 ? launch_u8<2, false>(a, st) : launch_u8<3, false>(a, st);
}

}  // namespace topot
