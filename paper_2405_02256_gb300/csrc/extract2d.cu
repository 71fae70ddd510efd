// K1, 2-D images of 8-bit pixels (Section 3, Delta^-; Section 4.2, preprocessing).
//
// The general kernel (extract.cu) handles 3-D images and int32 pixels.  This one is the
// path of every 2-D 8-bit batch.  One block of 512 threads per tile; a tile is R full
// rows of an image (m_0 <= 4096) or a piece of one row of at most 4096 columns.  Thread
// t owns a strip of 8 consecutive vertices of one tile row.
//
// Arithmetic.  A pixel value b in [0, 255] is held as the half-precision number 1024 + b
// (bits 0x64:b, one byte permute per two pixels).  Minima keep the common offset, and
// every difference of two such numbers is an integer in [-255, 255]; the lower-star
// value of one orthant is a sum of two such differences and the Delta table value a
// difference of two lower-star values, so every intermediate is an integer of magnitude
// <= 510 < 2048: exact in half precision.  Two vertices share one f16x2 register.
//
// With H[x] = min(X[x], X[x+1]) on each of the rows X = U (y-1), M (y), D (y+1), the
// vertical edge minima V = min(M, U or D) and the 2x2 box minima Q = min(H_U or H_D, H_M),
//   Delta^-_o(v) = (M - H_M[x - 1 or x]) + (Q[x - 1 or x] - V),
// x - 1 for eps_0 = +1 (orthant bit 0 clear), x for eps_0 = -1; U for eps_1 = +1, D for
// eps_1 = -1.  A pixel outside the image is staged as 0, the smallest value, so every
// box that leaves the image contributes nothing.
//
// Compaction.  Per segment (4 lower tables, 2 Delta tables) every thread counts its
// non-zero values, a warp scan and a scan of the 8 warp totals give each thread its
// place in a tile-compact shared-memory buffer (one word per entry: tile-local vertex
// index << 16 | half-precision value), the tile aggregates go to the decoupled
// look-back, and the block then writes each segment's run with consecutive threads on
// consecutive entries.  The look-back is done by warp 0 over a window of 32 predecessor
// tiles at a time, for all six segments at once, while the other warps fill the buffer.
// Two blocks (96 KB of compaction buffer each) share an SM.
#include <cuda_fp16.h>

#include "internal.cuh"

namespace topot {

namespace {

constexpr int kB = 512;                 // threads per block
constexpr int kNW = kB / 32;            // warps
constexpr int kSeg = 6;                 // 4 lower tables + 2 Delta tables
constexpr int kCap = kB * 8;            // vertices per tile (max), entries per segment (max); < 2^16
constexpr int kPadB = 16;               // staged row interior starts 16 bytes in
constexpr unsigned kFull = 0xffffffffu;

// shared-memory header (bytes)
constexpr int kOffBar = 0;              // mbarrier
constexpr int kOffInt = 8;              // ticket, image
constexpr int kOffWsum = 16;            // [kNW][4] packed warp totals
constexpr int kOffWex = kOffWsum + kNW * 16;   // [kNW][4] packed exclusive warp offsets
constexpr int kOffTot = kOffWex + kNW * 16;    // [4] packed tile totals
constexpr int kOffPref = kOffTot + 16;          // [kSeg] long long arena positions
constexpr int kOffRed = kOffPref + 8 * kSeg;    // [8] int: chi, |Delta^-_o| sums
constexpr int kOffOut = 1024;                    // [kSeg * kCap] packed entries
constexpr int kOffStage = kOffOut + 4 * kSeg * kCap;
static_assert(kOffRed + 32 <= kOffOut, "shared-memory header overlaps the compaction buffer");

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

// One staged row: the four vertex pairs P[p] = (X[2p], X[2p+1]) and the horizontal edge
// minima HR[p] = (H[2p], H[2p+1]), HL[p] = (H[2p-1], H[2p]).  sp is 8-byte aligned;
// sp[-1] and sp[8] are the neighbours of the strip.
__device__ __forceinline__ void row_pairs(const uint8_t* sp, uint32_t (&P)[4], uint32_t (&HR)[4],
                                          uint32_t (&HL)[4]) {
    const uint2 w = *reinterpret_cast<const uint2*>(sp);
    const uint32_t l = sp[-1], h = sp[8];
    constexpr uint32_t K = 0x64646464u;
    P[0] = __byte_perm(w.x, K, 0x4140);
    P[1] = __byte_perm(w.x, K, 0x4342);
    P[2] = __byte_perm(w.y, K, 0x4140);
    P[3] = __byte_perm(w.y, K, 0x4342);
    const uint32_t S0 = __byte_perm(P[0], P[1], 0x5432);   // (X[1], X[2])
    const uint32_t S1 = __byte_perm(P[1], P[2], 0x5432);
    const uint32_t S2 = __byte_perm(P[2], P[3], 0x5432);
    const uint32_t S3 = __byte_perm(P[3], h, 0x3432);      // (X[7], X[8])
    const uint32_t L0 = __byte_perm(l, P[0], 0x5450);      // (X[-1], X[0])
    HR[0] = hmin2(P[0], S0);
    HR[1] = hmin2(P[1], S1);
    HR[2] = hmin2(P[2], S2);
    HR[3] = hmin2(P[3], S3);
    HL[0] = hmin2(L0, P[0]);
    HL[1] = hmin2(S0, P[1]);
    HL[2] = hmin2(S1, P[2]);
    HL[3] = hmin2(S2, P[3]);
}

// Segment values of one strip: D[s][p] holds vertices 2p, 2p+1; s < 4 lower tables,
// s = 4 + r the Delta table Delta^-_r - Delta^-_{r^3}.
__device__ __forceinline__ void strip_values(const uint8_t* sp, int rs, uint32_t (&D)[kSeg][4]) {
    uint32_t PM[4], HRM[4], HLM[4];
    row_pairs(sp + rs, PM, HRM, HLM);
    uint32_t Al[4], Ar[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        Al[p] = hsub2(PM[p], HLM[p]);
        Ar[p] = hsub2(PM[p], HRM[p]);
    }
    {
        uint32_t PU[4], HRU[4], HLU[4];
        row_pairs(sp, PU, HRU, HLU);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t V = hmin2(PM[p], PU[p]);
            D[0][p] = hadd2(Al[p], hsub2(hmin2(HLU[p], HLM[p]), V));
            D[1][p] = hadd2(Ar[p], hsub2(hmin2(HRU[p], HRM[p]), V));
        }
    }
    {
        uint32_t PD[4], HRD[4], HLD[4];
        row_pairs(sp + 2 * rs, PD, HRD, HLD);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t V = hmin2(PM[p], PD[p]);
            D[2][p] = hadd2(Al[p], hsub2(hmin2(HLD[p], HLM[p]), V));
            D[3][p] = hadd2(Ar[p], hsub2(hmin2(HRD[p], HRM[p]), V));
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        D[4][p] = hsub2(D[0][p], D[3][p]);
        D[5][p] = hsub2(D[1][p], D[2][p]);
    }
}

// number of non-zero halves of the four pairs
__device__ __forceinline__ uint32_t count_nonzero(const uint32_t (&d)[4]) {
    uint32_t c = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
        asm("{\n\t.reg .pred a, b;\n\t"
            "setp.ne.f16x2 a|b, %1, %2;\n\t"
            "@a add.u32 %0, %0, 1;\n\t"
            "@b add.u32 %0, %0, 1;\n\t}"
            : "+r"(c) : "r"(d[p]), "r"(0u));
    return c;
}

// appends the non-zero halves of d (vertex j of half 0 is J0 >> 16, of half 1 J1 >> 16)
// at shared address *a, advancing it
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

__device__ __forceinline__ uint32_t field16(const uint32_t (&w)[3], int s) {
    return (w[s >> 1] >> (16 * (s & 1))) & 0xffffu;
}

}  // namespace

__global__ void __launch_bounds__(kB, 2) k_extract2d_u8(ExtractArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kOffBar);
    int* sh_int = reinterpret_cast<int*>(smem_raw + kOffInt);
    uint32_t* sh_wsum = reinterpret_cast<uint32_t*>(smem_raw + kOffWsum);
    uint32_t* sh_wex = reinterpret_cast<uint32_t*>(smem_raw + kOffWex);
    uint32_t* sh_tot = reinterpret_cast<uint32_t*>(smem_raw + kOffTot);
    long long* sh_pref = reinterpret_cast<long long*>(smem_raw + kOffPref);
    int* sh_red = reinterpret_cast<int*>(smem_raw + kOffRed);
    uint32_t* out = reinterpret_cast<uint32_t*>(smem_raw + kOffOut);
    uint8_t* stage = smem_raw + kOffStage;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const TablesDev& T = p.t;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        const unsigned ticket = atomicAdd(p.ticket, 1u);
        int lo = 0, hi = T.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&T.img[mid].tile_begin) <= (long long)ticket) lo = mid; else hi = mid - 1;
        }
        sh_int[0] = (int)ticket;
        sh_int[1] = lo;
    }
    if (tid < 8) sh_red[tid] = 0;
    __syncthreads();

    const long long ticket = (unsigned)sh_int[0];
    const int b = sh_int[1];
    const ImgDesc* Ip = T.img + b;
    const int m0 = __ldg(&Ip->m[0]), m1 = __ldg(&Ip->m[1]);
    const int W = __ldg(&Ip->W), R = __ldg(&Ip->R);
    const int spr = __ldg(&Ip->spr), RS = __ldg(&Ip->rs);
    const int segs = __ldg(&Ip->segs_per_row);
    const long long tile_begin = __ldg(&Ip->tile_begin);
    const int lt = (int)(ticket - tile_begin);
    FastDiv dsegs, dspr;
    dsegs.mul = __ldg(&Ip->div_segs.mul);
    dsegs.shift = __ldg(&Ip->div_segs.shift);
    dspr.mul = __ldg(&Ip->div_spr.mul);
    dspr.shift = __ldg(&Ip->div_spr.shift);
    const int rb = (int)fastdiv((uint32_t)lt, dsegs);
    const int sg = lt - rb * segs;
    const int y0 = rb * R, x0 = sg * W;
    const int rows = min(R, m1 - y0);
    const int cols = min(W, m0 - x0);
    const int L0 = y0 * m0 + x0;                       // linear index of the tile's first vertex
    const uint8_t* img = reinterpret_cast<const uint8_t*>(p.pixels) + __ldg(&Ip->offset);

    // ---- 1. stage rows y0 - 1 .. y0 + rows with a one-pixel halo; zeros outside -----------
    const int srows = rows + 2;
    const int span = 8 * spr;                          // bytes read per staged row: [-1, span]
    if (tid == 0) {
        unsigned bytes = 0;
        if ((cols & 15) == 0) {
            for (int rr = 0; rr < srows; ++rr) {
                const int yy = y0 + rr - 1;
                const uint8_t* src = img + (long long)yy * m0 + x0;
                if (yy >= 0 && yy < m1 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) bytes += (unsigned)cols;
            }
        }
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes) {
            for (int rr = 0; rr < srows; ++rr) {
                const int yy = y0 + rr - 1;
                const uint8_t* src = img + (long long)yy * m0 + x0;
                if (yy >= 0 && yy < m1 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0))
                    bulk_g2s(stage + rr * RS + kPadB, src, (unsigned)cols, bar);
            }
        }
    }
    for (int rr = warp; rr < srows; rr += kNW) {
        uint8_t* dst = stage + rr * RS + kPadB;
        const int yy = y0 + rr - 1;
        if (yy < 0 || yy >= m1) {
            for (int c = lane - 1; c <= span; c += 32) dst[c] = 0;
            continue;
        }
        const uint8_t* src = img + (long long)yy * m0 + x0;
        const bool bulk = ((cols & 15) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
        if (!bulk)
            for (int c = lane; c < cols; c += 32) dst[c] = src[c];
        if (lane == 0) dst[-1] = x0 > 0 ? src[-1] : (uint8_t)0;
        if (lane == 1) dst[cols] = x0 + cols < m0 ? src[cols] : (uint8_t)0;
        for (int c = cols + 1 + lane; c <= span; c += 32) dst[c] = 0;
    }
    mbar_wait_bounded(bar, 0, T.err);
    __syncthreads();

    // ---- 2. segment values of the thread's strip -------------------------------------------
    const int r = (int)fastdiv((uint32_t)tid, dspr);
    const int g = tid - r * spr;
    uint32_t D[kSeg][4];
    if (r < rows) {
        strip_values(stage + r * RS + kPadB + 8 * g, RS, D);
    } else {
#pragma unroll
        for (int s = 0; s < kSeg; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) D[s][q] = 0u;
    }

    // ---- 3. counts, warp scan (16-bit fields, two segments per word) -----------------------
    uint32_t cw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) cw[i] = count_nonzero(D[2 * i]) | (count_nonzero(D[2 * i + 1]) << 16);
    uint32_t iw[3] = {cw[0], cw[1], cw[2]};
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const uint32_t y = __shfl_up_sync(kFull, iw[i], d);
            if (lane >= d) iw[i] += y;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < 3; ++i) sh_wsum[warp * 4 + i] = iw[i];
    }
    __syncthreads();

    uint32_t tot[3];
    if (warp == 0) {
        // scan of the warp totals; lanes >= kNW carry zeros
        uint32_t v[3], x[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = v[i] = lane < kNW ? sh_wsum[lane * 4 + i] : 0u;
#pragma unroll
        for (int d = 1; d < kNW; d <<= 1) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const uint32_t y = __shfl_up_sync(kFull, x[i], d);
                if (lane >= d) x[i] += y;
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (lane < kNW) sh_wex[lane * 4 + i] = x[i] - v[i];
            tot[i] = __shfl_sync(kFull, x[i], kNW - 1);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) sh_tot[i] = tot[i];
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
            if (lt == __ldg(&Ip->tiles_per_plane) - 1) T.seg_count[(long long)b * kSeg + lane] = (long long)(pre + agg);
        }
    } else {
        asm volatile("bar.sync 1, %0;" ::"r"(kB) : "memory");
#pragma unroll
        for (int i = 0; i < 3; ++i) tot[i] = sh_tot[i];
    }

    // ---- 5. append the thread's entries to the tile-compact buffer --------------------------
    {
        uint32_t ex[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) ex[i] = sh_wex[warp * 4 + i] + iw[i] - cw[i];
        const uint32_t jb = (uint32_t)(r * cols + 8 * g) << 16;
        uint32_t J[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) J[k] = jb + ((uint32_t)k << 16);
        const uint32_t out_u32 = smem_u32(out);
        uint32_t base = 0;
#pragma unroll
        for (int s = 0; s < kSeg; ++s) {
            uint32_t a = out_u32 + 4u * (base + field16(ex, s));
#pragma unroll
            for (int q = 0; q < 4; ++q) append_pair(a, D[s][q], J[2 * q], J[2 * q + 1]);
            base += field16(tot, s);
        }
    }
    __syncthreads();

    // ---- 6. write the tile's runs; chi and sum |Delta^-_o| from the lower tables -------------
    // Each segment's run starts at an arbitrary arena position g0.  It is written in groups
    // of four arena slots aligned to four (one 16-byte index store, one 8-byte value store);
    // the partial groups at the two ends store entry by entry.  Group numbers continue
    // across segments modulo the block size, so that every thread gets about the same
    // number of groups.
    int chi = 0, ab[4] = {0, 0, 0, 0};
    {
        uint32_t base = 0, cum = 0;
#pragma unroll
        for (int s = 0; s < kSeg; ++s) {
            const int n = (int)field16(tot, s);
            const long long g0 = sh_pref[s];
            const int ph = (int)(g0 & 3);
            const int ngroups = (ph + n + 3) >> 2;
            int* __restrict__ pi = T.arena_idx + (g0 - ph);
            int16_t* __restrict__ pv = reinterpret_cast<int16_t*>(T.arena_val) + (g0 - ph);
            const uint32_t* o = out + base;
            for (int q = (int)(((uint32_t)tid - cum) & (kB - 1)); q < ngroups; q += kB) {
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
                        id[k] = L0 + (int)(w >> 16);
                    }
                    if (s < 4) ab[s & 3] += abs(v[k]);
                    if (s == 0) chi += v[k];
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
            base += (uint32_t)n;
            cum += (uint32_t)ngroups;
        }
    }
    const int red[5] = {chi, ab[0], ab[1], ab[2], ab[3]};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int v = (int)__reduce_add_sync(kFull, (unsigned)red[i]);
        if (lane == 0) atomicAdd(&sh_red[i], v);
    }
    __syncthreads();
    if (tid == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&T.chi[b]), (unsigned long long)(long long)sh_red[0]);
    if (tid >= 1 && tid < 5)
        atomicAdd(reinterpret_cast<unsigned long long*>(&T.absum[(long long)b * 4 + tid - 1]),
                  (unsigned long long)(long long)sh_red[tid]);
}

// ---- host side ----------------------------------------------------------------------------

int extract2d_tile_vertices() { return kCap; }
int extract2d_threads() { return kB; }

size_t extract2d_smem_bytes(int stage_bytes) { return (size_t)kOffStage + (size_t)stage_bytes; }

cudaError_t launch_extract2d_u8(const ExtractArgs& a, cudaStream_t st) {
    static cudaError_t attr = [] {
        cudaError_t e = cudaFuncSetAttribute(k_extract2d_u8, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_extract2d_u8, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    if (attr != cudaSuccess) return attr;
    k_extract2d_u8<<<(unsigned)a.num_tiles, kB, extract2d_smem_bytes(a.stage_bytes), st>>>(a);
    return cudaGetLastError();
}

}  // namespace topot
