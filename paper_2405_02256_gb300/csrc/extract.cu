// K1: critical-table extraction for int32 pixels, and for the top-dimensional
// construction of 8-bit and int32 images through their int32 corner image (Section 3,
// Delta^-; Section 4.1; Section 4.2, preprocessing).  8-bit images in the vertex
// construction use k_extract_u8 (extract_u8.cu).
//
// One block per tile.  A tile is a run of vertices that is contiguous in linear
// vertex order: R full rows of one plane (m_0 <= W) or one W-wide piece of a row.
// The block
//   1. stages the tile's pixels plus a one-vertex halo (three planes in 3-D) in
//      shared memory -- 1-D bulk copies (TMA, cp.async.bulk) for 16-byte aligned row
//      interiors, plain loads for the halo and unaligned rows; pixels outside the
//      image get a sentinel so that a box that leaves the image contributes nothing;
//   2. evaluates, for every vertex and every orthant o, the lower-star value
//      Delta^-_o(v) = sum_{delta in {0,1}^n} (-1)^|delta| min(phi over box(v, v - delta (.) eps_o))
//      from the 3^n neighbourhood (all 2^n orthants share the edge / face minima);
//   3. compacts the non-zero values of the 2^n lower tables and of the 2^(n-1)
//      Delta = Delta^-_r - Delta^-_{-r} tables in vertex order: each thread owns K
//      consecutive vertices and counts its entries per table, warp-shuffle scans and a
//      block scan of the warp totals place them, and a decoupled look-back over the
//      tiles of the same image (tiles are numbered by an atomic ticket, so every
//      predecessor belongs to a block that has already started) gives the tile's start;
//   4. adds chi = sum Delta^-_0 and sum |Delta^-_o| of the tile to per-image totals.
#include <algorithm>

#include "internal.cuh"

namespace topot {

template <typename Tin> struct PixTraits;
template <> struct PixTraits<uint8_t> {
    // u8 values are >= 0: a zero sentinel makes the minimum over any box that leaves
    // the image 0, i.e. that box contributes nothing.
    static constexpr bool kSigned = false;
    __device__ static int sentinel() { return 0; }
    __device__ static int fix(int v) { return v; }
};
template <> struct PixTraits<int32_t> {
    static constexpr bool kSigned = true;
    __device__ static int sentinel() { return INT32_MIN; }
    __device__ static int fix(int v) { return v == INT32_MIN ? 0 : v; }
};

// Lower-star values of one vertex for all 2^NDIM orthants.  `c` points at the vertex
// in the staged buffer; rs = row stride, ps = plane stride (elements).
template <int NDIM, typename Tin>
__device__ __forceinline__ void lower_star(const Tin* c, int rs, int ps, int (&out)[1 << NDIM]) {
    using PT = PixTraits<Tin>;
    auto nb = [&](int dx, int dy, int dz) -> int { return (int)c[dz * ps + dy * rs + dx]; };
    const int a = nb(0, 0, 0);
    if constexpr (NDIM == 2) {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int d0 = (o & 1) ? 1 : -1;
            const int d1 = (o & 2) ? 1 : -1;
            const int e0 = min(a, nb(d0, 0, 0));
            const int e1 = min(a, nb(0, d1, 0));
            const int sq = min(min(e0, e1), nb(d0, d1, 0));
            out[o] = PT::fix(a) - PT::fix(e0) - PT::fix(e1) + PT::fix(sq);
        }
    } else {
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int d0 = (o & 1) ? 1 : -1;
            const int d1 = (o & 2) ? 1 : -1;
            const int d2 = (o & 4) ? 1 : -1;
            const int e0 = min(a, nb(d0, 0, 0));
            const int e1 = min(a, nb(0, d1, 0));
            const int e2 = min(a, nb(0, 0, d2));
            const int f01 = min(min(e0, e1), nb(d0, d1, 0));
            const int f02 = min(min(e0, e2), nb(d0, 0, d2));
            const int f12 = min(min(e1, e2), nb(0, d1, d2));
            const int cu = min(min(f01, f02), min(f12, nb(d0, d1, d2)));
            out[o] = PT::fix(a) - PT::fix(e0) - PT::fix(e1) - PT::fix(e2) + PT::fix(f01) +
                     PT::fix(f02) + PT::fix(f12) - PT::fix(cu);
        }
    }
}

// Lower-star values of one corner vertex for the top-dimensional construction
// (Section 4.1: one top cell per pixel, a lower cell carries the minimum over the pixels
// that contain it).  The extraction runs on the corner image V of shape m + 1 with
// V(v) = pixel(v - 1) and kTopMissing outside the image, so the 2^n pixels around corner
// v are V(v + g), g in {0,1}^n.  The box of the lower star of v for orthant o that spans
// the axes k with delta_k = 1 (towards -eps_k) lies in the pixels with g_k = bit k of o
// on the spanned axes and any g_k on the others; its value is their minimum, and it
// does not exist (adds 0) when none of them is a pixel.
template <int NDIM>
__device__ __forceinline__ void lower_star_top(const int32_t* c, int rs, int ps, int (&out)[1 << NDIM]) {
    constexpr int NO = 1 << NDIM;
    int P[NO];
#pragma unroll
    for (int g = 0; g < NO; ++g) P[g] = c[((g >> 2) & 1) * ps + ((g >> 1) & 1) * rs + (g & 1)];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        int acc = 0;
#pragma unroll
        for (int delta = 0; delta < NO; ++delta) {
            int m = kTopMissing;
#pragma unroll
            for (int g = 0; g < NO; ++g)
                if (((g ^ o) & delta) == 0) m = min(m, P[g]);
            const int term = m == kTopMissing ? 0 : m;
            acc += (__popc(delta) & 1) ? -term : term;
        }
        out[o] = acc;
    }
}

// Corner image V of the top-dimensional construction: V(v) = pixel(v - 1) when every
// v_k >= 1, else kTopMissing; V has m_k + 1 entries per axis.
template <typename Tpix>
__global__ void k_top_prepass(const Tpix* __restrict__ pix, int32_t* __restrict__ V, const TopSrc* __restrict__ src,
                              int B, int n) {
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const TopSrc s = src[b];
        const int M0 = s.m[0] + 1, M1 = s.m[1] + 1, M2 = n == 3 ? s.m[2] + 1 : 1;
        const long long NV = (long long)M0 * M1 * M2;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < NV;
             i += (long long)gridDim.x * blockDim.x) {
            const int x = (int)(i % M0);
            const long long r = i / M0;
            const int y = (int)(r % M1);
            const int z = (int)(r / M1);
            int v = kTopMissing;
            if (x >= 1 && y >= 1 && (n == 2 || z >= 1))
                v = (int)pix[s.pix_offset + ((long long)(n == 3 ? z - 1 : 0) * s.m[1] + (y - 1)) * s.m[0] + (x - 1)];
            V[s.v_offset + i] = v;
        }
    }
}

// u8 corner image of the top-dimensional construction of an 8-bit image: V(v) =
// pixel(v - 1) when every v_k >= 1, else 255; rows padded to `pitch` bytes with 255.
// 255 stands for "no pixel": it is at least every pixel, so a box with some pixels takes
// their minimum, and boxes with none take 255 together and cancel in the alternating
// sum of the lower star -- except at the 2^n corners of the image, which the extraction
// corrects (k_extract_u8).  Blocks over corner-image rows, 16 bytes per thread: from
// 16-byte loads when the pixel row is 16-byte aligned (one byte from the previous chunk),
// else byte by byte.
__global__ void k_top_prepass_u8(const uint8_t* __restrict__ pix, uint8_t* __restrict__ V,
                                 const TopSrc* __restrict__ src, int B, int n) {
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const TopSrc s = src[b];
        const int M1 = s.m[1] + 1, M2 = n == 3 ? s.m[2] + 1 : 1;
        const int chunks = s.pitch >> 4;
        const uint8_t* pb = pix + s.pix_offset;
        uint4* vb = reinterpret_cast<uint4*>(V + s.v_offset);
        for (int row = blockIdx.x; row < M1 * M2; row += gridDim.x) {
            const int z = row / M1, y = row - z * M1;
            const bool inside = y >= 1 && (n == 2 || z >= 1);
            // pixel row (z - 1, y - 1); column x of the corner image is pixel x - 1
            const long long prow = ((long long)(n == 3 ? z - 1 : 0) * s.m[1] + (y - 1)) * s.m[0];
            const uint8_t* pr = pb + (inside ? prow : 0);
            const bool aligned = (reinterpret_cast<uintptr_t>(pr) & 15) == 0;
            for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
                const int x0 = 16 * c;                    // corner columns x0 .. x0 + 15
                uint32_t w[4];
                if (!inside) {
                    w[0] = w[1] = w[2] = w[3] = 0xffffffffu;
                } else if (aligned && x0 + 16 <= s.m[0]) {
                    // pixels x0 - 1 .. x0 + 14: the chunk x0 .. x0 + 15 (inside the row) shifted
                    // up one byte
                    const uint4 q = *reinterpret_cast<const uint4*>(pr + x0);
                    const uint32_t prev = c > 0 ? (uint32_t)pr[x0 - 1] : 255u;
                    w[0] = __byte_perm(prev, q.x, 0x6540);
                    w[1] = __byte_perm(q.x, q.y, 0x6543);
                    w[2] = __byte_perm(q.y, q.z, 0x6543);
                    w[3] = __byte_perm(q.z, q.w, 0x6543);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t v = 0u;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int x = x0 + 4 * j + k;
                            const uint32_t px = (x >= 1 && x <= s.m[0]) ? (uint32_t)pr[x - 1] : 255u;
                            v |= px << (8 * k);
                        }
                        w[j] = v;
                    }
                }
                vb[(long long)row * chunks + c] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

template <int NDIM, typename Tin, typename Tval, int BLOCK, int K, bool TOP>
__global__ void __launch_bounds__(BLOCK, 4) k_extract(ExtractArgs p) {
    using PT = PixTraits<Tin>;
    static_assert(!TOP || sizeof(Tin) == 4, "the corner image of the top construction is int32");
    const Tin kSent = (Tin)(TOP ? kTopMissing : PT::sentinel());   // outside the image
    constexpr int NO = 1 << NDIM;              // orthants
    constexpr int S = NO + NO / 2;             // segments
    constexpr int NW = BLOCK / 32;
    constexpr int PAD = 16 / (int)sizeof(Tin); // interior starts 16 bytes into a row
    constexpr int NP = (NDIM == 3) ? 3 : 1;    // staged planes

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    int* sh_int = reinterpret_cast<int*>(smem_raw + 16);               // [8]
    long long* sh_pref = reinterpret_cast<long long*>(smem_raw + 48);  // [S]
    long long* sh_acc = sh_pref + S;                                   // [1 + NO]
    int* sh_cnt = reinterpret_cast<int*>(sh_acc + 1 + NO);             // [S][NW]
    size_t stage_off = 48 + sizeof(long long) * (S + 1 + NO) + sizeof(int) * S * NW;
    stage_off = (stage_off + 15) & ~size_t(15);
    Tin* stage = reinterpret_cast<Tin*>(smem_raw + stage_off);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const TablesDev& T = p.t;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        // ticket -> (image, local tile) -> global tile number, which indexes the look-back
        const unsigned ticket = atomicAdd(p.ticket, 1u);
        const int2 bl = p.order[ticket];
        sh_int[0] = (int)(T.img[bl.x].tile_begin + bl.y);
        sh_int[1] = bl.x;
    }
    if (tid < 1 + NO) sh_acc[tid] = 0;
    __syncthreads();

    const long long ticket = sh_int[0];
    const int b = sh_int[1];
    // a register copy: the table stores below could alias a reference into global memory
    const ImgDesc I = T.img[b];
    const int m0 = I.m[0], m1 = I.m[1], m2 = I.m[2];
    const long long lt = ticket - I.tile_begin;
    const long long ntiles_img = (long long)I.tiles_per_plane * I.nz;
    const int zl = (int)(lt / I.tiles_per_plane);   // owned plane; volume plane z (slabs: zlo + zl)
    const int z = I.zlo + zl;
    const int rem = (int)(lt - (long long)zl * I.tiles_per_plane);
    const int rb = rem / I.segs_per_row;
    const int sg = rem - rb * I.segs_per_row;
    const int y0 = rb * I.R;
    const int x0 = sg * I.W;
    const int rows = min(I.R, m1 - y0);
    const int cols = min(I.W, m0 - x0);
    const int nverts = rows * cols;
    const long long L0 = ((long long)z * m1 + y0) * m0 + x0;

    // ---- 1. stage pixels + halo -------------------------------------------------------
    // pixels of plane zz at img + zz m_1 m_0: the buffer starts at plane zbase (a slab)
    const Tin* img = reinterpret_cast<const Tin*>(p.pixels) + I.offset - (long long)I.zbase * m1 * m0;
    const int RS = p.row_stride;
    const int PS = p.stage_rows * RS;
    const int srows = rows + 2;
    const bool tma_cols = ((cols * (int)sizeof(Tin)) & 15) == 0;
    unsigned tma_bytes = 0;
    for (int q = tid; q < NP * srows; q += BLOCK) {
        const int pl = q / srows, rr = q - pl * srows;
        const int zz = (NDIM == 3) ? z + pl - 1 : z;
        const int yy = y0 + rr - 1;
        Tin* dst = stage + pl * PS + rr * RS;
        const bool inside = zz >= 0 && zz < m2 && yy >= 0 && yy < m1;
        if (!inside) continue;
        const Tin* src = img + ((long long)zz * m1 + yy) * m0 + x0;
        dst[PAD - 1] = x0 > 0 ? src[-1] : kSent;
        dst[PAD + cols] = (x0 + cols < m0) ? src[cols] : kSent;
    }
    // rows outside the image, and rows whose interior is not 16-byte aligned
    for (int q = 0; q < NP * srows; ++q) {
        const int pl = q / srows, rr = q - pl * srows;
        const int zz = (NDIM == 3) ? z + pl - 1 : z;
        const int yy = y0 + rr - 1;
        Tin* dst = stage + pl * PS + rr * RS;
        const bool inside = zz >= 0 && zz < m2 && yy >= 0 && yy < m1;
        if (!inside) {
            for (int c = tid - 1; c <= cols; c += BLOCK) dst[PAD + c] = kSent;
            continue;
        }
        const Tin* src = img + ((long long)zz * m1 + yy) * m0 + x0;
        const bool aligned = tma_cols && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
        if (aligned) {
            tma_bytes += (unsigned)(cols * sizeof(Tin));
        } else {
            for (int c = tid; c < cols; c += BLOCK) dst[PAD + c] = src[c];
        }
    }
    __syncthreads();   // mbarrier initialised; generic-proxy halo writes done
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, tma_bytes);
        if (tma_bytes) {
            for (int q = 0; q < NP * srows; ++q) {
                const int pl = q / srows, rr = q - pl * srows;
                const int zz = (NDIM == 3) ? z + pl - 1 : z;
                const int yy = y0 + rr - 1;
                if (!(zz >= 0 && zz < m2 && yy >= 0 && yy < m1)) continue;
                const Tin* src = img + ((long long)zz * m1 + yy) * m0 + x0;
                if (tma_cols && ((reinterpret_cast<uintptr_t>(src) & 15) == 0))
                    bulk_g2s(stage + pl * PS + rr * RS + PAD, src, (unsigned)(cols * sizeof(Tin)), bar);
            }
        }
    }
    mbar_wait_bounded(bar, 0, T.err);
    __syncthreads();

    // ---- 2. lower-star values, kept in registers --------------------------------------
    // Blocked layout: thread tid owns the K consecutive vertices j = tid * K + k of the
    // tile, whose linear indices are L0 + j (the tile is a run of full rows, cols == m0, or
    // part of one row).  Their staged positions (r, c) are tracked incrementally.
    int vals[K][NO];
    int chi_acc = 0;          // |Delta^-| <= 2^(n-1) * 255 per vertex for u8, and int32 input
    int abs_acc[NO];          // is limited to |phi| < 2^26 (checked below): K vertices fit int32
#pragma unroll
    for (int o = 0; o < NO; ++o) abs_acc[o] = 0;
    bool bad_pixel = false;
    const Tin* center0 = stage + (NP == 3 ? PS : 0) + RS + PAD;
    const int j0 = tid * K;
    {
        const int W = cols;
        int r = 0, c = j0;
        if (rows > 1 && j0 < nverts) {
            r = (int)fastdiv((uint32_t)j0, I.div0);
            c = j0 - r * W;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (j0 + k < nverts) {
                const Tin* cp = center0 + r * RS + c;
                if constexpr (TOP) lower_star_top<NDIM>(reinterpret_cast<const int32_t*>(cp), RS, PS, vals[k]);
                else lower_star<NDIM, Tin>(cp, RS, PS, vals[k]);
                if constexpr (PT::kSigned) {
                    const int a = (int)cp[0];
                    bad_pixel |= (!TOP || a != kTopMissing) && ((a >= (1 << 26)) || (a <= -(1 << 26)));
                }
                chi_acc += vals[k][0];
#pragma unroll
                for (int o = 0; o < NO; ++o) abs_acc[o] += abs(vals[k][o]);
            } else {
#pragma unroll
                for (int o = 0; o < NO; ++o) vals[k][o] = 0;
            }
            if (++c == W) {
                c = 0;
                ++r;
            }
        }
    }
    if (bad_pixel) dev_set_error(T.err, kDevErrOverflow);

    auto seg_value = [&](int k, int s) -> int {
        return s < NO ? vals[k][s] : vals[k][s - NO] - vals[k][(s - NO) ^ (NO - 1)];
    };

    // ---- 3a. per-thread counts, warp-inclusive scans --------------------------------------
    int incl[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        int c = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) c += seg_value(k, s) != 0;
        incl[s] = c;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl[s], d);
            if (lane >= d) incl[s] += y;
        }
        if (lane == 31) sh_cnt[s * NW + warp] = incl[s];
    }
    // chi and sum |Delta^-| of the tile (64-bit from the warp level up)
    const long long chi_w = warp_sum((long long)chi_acc);
    long long abs_w[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) abs_w[o] = warp_sum((long long)abs_acc[o]);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&sh_acc[0]), (unsigned long long)chi_w);
#pragma unroll
        for (int o = 0; o < NO; ++o)
            atomicAdd(reinterpret_cast<unsigned long long*>(&sh_acc[1 + o]), (unsigned long long)abs_w[o]);
    }
    __syncthreads();

    // ---- 3b. scan of the warp totals per segment + decoupled look-back ---------------------
    if (tid < S) {
        const int s = tid;
        int run = 0;
        int* cs = sh_cnt + s * NW;
        for (int q = 0; q < NW; ++q) {
            const int c = cs[q];
            cs[q] = run;
            run += c;
        }
        const unsigned long long agg = (unsigned long long)run;
        unsigned long long* st = p.status + ticket * S + s;
        long long prefix = 0;
        if (lt == 0) {
            st_relaxed_u64(st, kFlagP | agg);
        } else {
            st_relaxed_u64(st, kFlagA | agg);
            long long q = ticket - 1;
            const unsigned long long t0 = dev_time_ns();
            bool timed_out = false;
            while (true) {
                const unsigned long long w = ld_relaxed_u64(p.status + q * S + s);
                const unsigned long long flag = w & ~kCountMask;
                if (flag == 0) {
                    if (dev_time_ns() - t0 > kWaitLimitNs) { timed_out = true; break; }
                    continue;
                }
                prefix += (long long)(w & kCountMask);
                if (flag == kFlagP) break;
                --q;
            }
            if (timed_out) {
                dev_set_error(T.err, kDevErrTimeout);
                prefix = 0;
            }
            st_relaxed_u64(st, kFlagP | ((unsigned long long)prefix + agg));
        }
        // arena position of this tile's first entry of segment s
        sh_pref[s] = I.seg_base + (long long)s * I.N + prefix;
        if (lt == ntiles_img - 1) T.seg_count[(long long)b * S + s] = prefix + (long long)agg;
    }
    if (tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&T.chi[b]), (unsigned long long)sh_acc[0]);
        for (int o = 0; o < NO; ++o)
            atomicAdd(reinterpret_cast<unsigned long long*>(&T.absum[(long long)b * NO + o]),
                      (unsigned long long)sh_acc[1 + o]);
    }
    __syncthreads();

    // ---- 3c. every thread writes its own run of entries, segment by segment ---------------
    const int vbase = (int)L0 + j0;           // linear index of this thread's first vertex
#pragma unroll
    for (int s = 0; s < S; ++s) {
        int c = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) c += seg_value(k, s) != 0;
        const long long pos0 = sh_pref[s] + sh_cnt[s * NW + warp] + incl[s] - c;
        int* __restrict__ didx = T.arena_idx + pos0;
        Tval* __restrict__ dval = reinterpret_cast<Tval*>(T.arena_val) + pos0;
        int q = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int v = seg_value(k, s);
            if (v != 0) {
                didx[q] = vbase + k;
                dval[q] = (Tval)v;
                ++q;
            }
        }
    }
}

// ---- host-side launch ----------------------------------------------------------------------

template <int NDIM, typename Tin, typename Tval, int BLOCK, int K, bool TOP>
static cudaError_t launch_extract_t(const ExtractArgs& a, size_t smem, cudaStream_t st) {
    auto kern = k_extract<NDIM, Tin, Tval, BLOCK, K, TOP>;
    // attributes once per instantiation, so that launches inside stream capture only launch
    static cudaError_t attr = [&] {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    }();
    if (attr != cudaSuccess) return attr;
    kern<<<(unsigned)a.num_tiles, BLOCK, smem, st>>>(a);
    return cudaGetLastError();
}

// Tile geometry shared with the host code: vertices per tile and block size.
int extract_block(int n) { return n == 2 ? 256 : 256; }
int extract_k(int n) { return n == 2 ? 8 : 4; }

size_t extract_smem_bytes(int n, int elem_bytes, int row_stride, int stage_rows) {
    const int NO = 1 << n, S = NO + NO / 2;
    const int NW = extract_block(n) / 32;
    size_t off = 48 + sizeof(long long) * (S + 1 + NO) + sizeof(int) * S * NW;
    off = (off + 15) & ~size_t(15);
    const int NP = n == 3 ? 3 : 1;
    return off + (size_t)NP * stage_rows * row_stride * elem_bytes;
}

// int32 pixels (vertex construction), or the int32 corner image of the top-dimensional
// construction of 8-bit (int16 tables) or int32 images.  8-bit images in the vertex
// construction go to k_extract_u8 (extract_u8.cu).
cudaError_t launch_extract(int n, topot_dtype dtype, bool top, const ExtractArgs& a, cudaStream_t st) {
    const size_t smem = extract_smem_bytes(n, 4, a.row_stride, a.stage_rows);
    if (!top) {
        if (dtype != TOPOT_I32) return cudaErrorInvalidValue;
        if (n == 2) return launch_extract_t<2, int32_t, int32_t, 256, 8, false>(a, smem, st);
        return launch_extract_t<3, int32_t, int32_t, 256, 4, false>(a, smem, st);
    }
    if (dtype == TOPOT_U8) {
        if (n == 2) return launch_extract_t<2, int32_t, int16_t, 256, 8, true>(a, smem, st);
        return launch_extract_t<3, int32_t, int16_t, 256, 4, true>(a, smem, st);
    }
    if (n == 2) return launch_extract_t<2, int32_t, int32_t, 256, 8, true>(a, smem, st);
    return launch_extract_t<3, int32_t, int32_t, 256, 4, true>(a, smem, st);
}

cudaError_t launch_top_prepass(const void* pixels, topot_dtype dtype, int32_t* V, const TopSrc* src, int B, int n,
                               long long max_nv, int sm_count, cudaStream_t st) {
    const long long per = (max_nv + 255) / 256;
    dim3 grid((unsigned)std::max(1ll, std::min(per, (long long)std::max(1, 8 * sm_count / std::max(1, std::min(B, 65535))))),
              (unsigned)std::min(B, 65535));
    if (dtype == TOPOT_U8)
        k_top_prepass<uint8_t><<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t*>(pixels), V, src, B, n);
    else
        k_top_prepass<int32_t><<<grid, 256, 0, st>>>(reinterpret_cast<const int32_t*>(pixels), V, src, B, n);
    return cudaGetLastError();
}

cudaError_t launch_top_prepass_u8(const uint8_t* pixels, uint8_t* V, const TopSrc* src, int B, int n, int sm_count,
                                  cudaStream_t st) {
    const int gy = std::min(B, 65535);
    const int gx = std::max(1, std::min(65535, 8 * sm_count / gy + 1));
    k_top_prepass_u8<<<dim3(gx, gy), 256, 0, st>>>(pixels, V, src, B, n);
    return cudaGetLastError();
}

}  // namespace topot
