// Internal structures and device helpers of libtopot (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/topot.h"

namespace topot {

constexpr int kMaxDim = 4;   // 2-D and 3-D specialised kernels; 4-D on the generic path

// Device error word bits (OR-ed by kernels, read and cleared by tables_sync).
enum DevErr : unsigned {
    kDevErrOverflow = 1u,   // int32 pixel outside |phi| < 2^26, or |ECT| bound >= 2^31
    kDevErrTimeout = 2u,    // a bounded wait gave up
};

// Time limit (ns of %globaltimer) of every device-side spin (look-back, mbarrier
// waits).  A wait that runs out records kDevErrTimeout and returns instead of hanging.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long dev_time_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Unsigned division by a runtime constant d (1 <= d < 2^31) for dividends n < 2^31:
// q = (n * mul) >> shift with mul = ceil(2^shift / d), shift = 31 + ceil(log2 d).
struct FastDiv {
    uint32_t d;
    uint32_t mul;
    uint32_t shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    f.shift = 31 + l;
    unsigned __int128 num = (unsigned __int128)1 << f.shift;
    f.mul = (uint32_t)((num + d - 1) / d);
    return f;
}

__device__ __forceinline__ uint32_t fastdiv(uint32_t n, const FastDiv& f) {
    return (uint32_t)(((unsigned long long)n * f.mul) >> f.shift);
}

// Per-image description, shared by extraction and evaluation kernels.
struct ImgDesc {
    long long offset;       // element offset of the image in the pixel buffer
    long long N;            // vertices
    long long seg_base;     // arena entry offset of segment 0 (segments are N apart)
    long long tile_begin;   // first extraction tile (global numbering)
    int m[kMaxDim];         // axis lengths, m_0 fastest; 1 beyond n
    int W;                  // extraction tile width (columns)
    int R;                  // extraction tile rows (1 when W < m_0)
    int segs_per_row;       // ceil(m_0 / W)
    int tiles_per_plane;    // ceil(m_1 / R) * segs_per_row
    FastDiv div0;           // division by m_0
    FastDiv div1;           // division by m_1
    // 8-bit extraction kernel only: strips of vertices per tile row, staged row stride
    int spr;                // ceil(W / strip)
    int rs;                 // staged row stride (bytes, multiple of 16)
    int packed;             // 1: full-row tiles, m_0 and offset multiples of 16 (rs = m_0)
    FastDiv div_spr;        // division by spr
    FastDiv div_segs;       // division by segs_per_row
    FastDiv div_tpp;        // division by tiles_per_plane
    // evaluation kernels: 1 / (2 (m_k - 1)) in FP64 (0 for an axis of length 1), so that
    // per-direction weights take a multiply rather than an FP64 division
    double inv2m[kMaxDim];
    // slab of a volume (3-D): the tables hold the vertices of planes [zlo, zlo + nz) of a
    // volume of m_2 planes, whose pixels start at plane zbase (zlo - 1 or zlo) at `offset`.
    // A whole image has zlo = zbase = 0, nz = m_2.
    int zlo;
    int zbase;
    int nz;
    // top-dimensional construction of an 8-bit image: the corner image is a u8 array with
    // rows top_pitch bytes apart (a multiple of 16, >= m_0), planes top_pitch * m_1 apart;
    // extraction tiles are runs of positions of that array.  0 for every other image.
    int top_pitch;
    FastDiv div_pitch;      // division by top_pitch
};

// Device view of a tables handle.
struct TablesDev {
    int n;                      // 2 or 3
    int B;                      // images
    int S;                      // segments per image: 2^n lower + 2^(n-1) delta
    int val_bytes;              // 2 (int16, uint8 input) or 4 (int32 input)
    const ImgDesc* img;         // [B]
    int* arena_idx;             // [sum_b S * N_b]
    void* arena_val;            // same length, int16 or int32
    long long* seg_count;       // [B * S]
    long long* chi;             // [B]
    long long* absum;           // [B * 2^n]  sum_v |Delta^-_o(v)|
    unsigned* err;              // device error word
};

// Arguments of the extraction kernel.
struct ExtractArgs {
    TablesDev t;
    const void* pixels;
    long long num_tiles;
    unsigned* ticket;                 // zeroed before launch
    const int2* order;                // [num_tiles] (image, local tile) taken by ticket t
    unsigned long long* status;       // [num_tiles * S] look-back words (global tile numbers)
    int row_stride;                   // staged row stride (elements, 16-byte multiple)
    int stage_rows;                   // staged rows per plane (max R + 2)
    int stage_bytes;                  // 8-bit kernel: staged bytes per tile (max over images)
    const unsigned* nonbin;           // 3-D 8-bit: [B + 1] from the binary path (null without it)
};

// Binary 8-bit volumes (all voxels 0 or 1): per volume, its packed bits and units.
// The packed bits keep a zero border: (m_2 + 2) planes of (m_1 + 2) rows of (wpr + 2)
// words, voxel word (z, y, xw) at pk_off + ((z + 1)(m_1 + 2) + y + 1)(wpr + 2) + xw + 1, so
// every neighbour word is a fixed offset away and needs no bounds check.
struct BinImg {
    long long pix_off;      // element offset of the voxels in the pixel buffer
    long long pk_off;       // word offset of the packed bits
    long long unit_begin;   // first unit (32 consecutive voxel words) in the global numbering
    long long seg_base;     // arena slot of segment 0 (segments are N apart)
    long long N;            // vertices
    int m0, m1, m2;
    int wpr;                // voxel words per row: ceil(m_0 / 32)
    int nunits;             // ceil(m_2 m_1 wpr / 32)
    FastDiv div_wpr;        // division by wpr
    FastDiv div_m1;         // division by m_1
};

struct BinArgs {
    TablesDev t;
    const BinImg* img;      // [B]
    const void* pixels;
    uint32_t* packed;
    unsigned* nonbin;       // [B + 1] volume b has a voxel above 1; [B]: some volume has (zeroed per build)
    uint32_t* ucount;       // [units][6] per-unit counts, two 16-bit fields per word
    int* uoff;              // [units][12] per-unit offsets within each segment
    int* csum;              // [nchunks][12]
    const int2* blocks;     // [nblocks] (volume, first unit) of each block of the two passes
    int nblocks;
    const int2* chunks;     // [nchunks] (volume, chunk of the volume), volume-major
    int nchunks;
};

// Top-dimensional construction: per image, where its pixels and its corner image live.
constexpr int kTopMissing = 0x7fffffff;   // corner-image value of a pixel outside the image
struct TopSrc {
    long long pix_offset;   // element offset of the pixels in the caller's buffer
    long long v_offset;     // element offset of the corner image in the handle's buffer
    int m[3];               // pixels per axis (m_2 = 1 for n = 2)
    int pitch;              // u8 corner image: row pitch (bytes); 0: int32 corner image, rows m_0 + 1
};

// Arguments of the exact-representation kernels (one segment per image and direction).
struct ExactArgs {
    TablesDev t;
    const double* dirs;
    int D;
    int per_image;
    int kind;
    int nseg;                        // B * D
    long long cap;                   // slots per segment
    unsigned long long* key[2];      // [nseg][cap], ping-pong
    int* val[2];
    int* cnt;                        // [nseg] entries per segment
    int tps;                         // radix tiles per segment (from the largest segment)
    int prod_max;                    // coordinate products staged per direction (0: none)
    unsigned* hist;                  // [nseg][8][256] digit counts (tps > 1), else null
    unsigned long long* status;      // [nseg * tps][256] look-back words (tps > 1), zeroed per call
    int* tile_ctr;                   // [16] tile tickets: the eight passes, then the finish
    double* T;                       // [nseg][cap]
    int32_t* E;
    long long* len;                  // [nseg]
};

// Look-back status words of the extraction kernels: 2-bit flag + 62-bit count.
constexpr unsigned long long kFlagA = 1ull << 62;   // tile aggregate available
constexpr unsigned long long kFlagP = 2ull << 62;   // inclusive prefix available
constexpr unsigned long long kCountMask = (1ull << 62) - 1;

__device__ __forceinline__ void dev_set_error(unsigned* err, unsigned bit) {
    atomicOr(err, bit);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- mbarrier + bulk copy (TMA, non-tensor) helpers --------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Returns true when phase `parity` of the barrier has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait; false (and the error bit set) if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* err,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = dev_time_ns();
    while (dev_time_ns() - t0 < limit_ns) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    dev_set_error(err, kDevErrTimeout);
    return false;
}

// 1-D bulk copy global -> shared (cp.async.bulk), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// ---- warp helpers ---------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace topot
