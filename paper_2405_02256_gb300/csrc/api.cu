// C ABI of libtopot (declared in include/topot.h): validation, handle and workspace
// management, and the launch sequences of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "eval_common.cuh"

namespace topot {
cudaError_t launch_extract(int n, topot_dtype dtype, bool top, const ExtractArgs& a, cudaStream_t st);
cudaError_t launch_segment_sums(const TablesDev& t, long long* vsum, cudaStream_t st);
int gen_block();
cudaError_t launch_extract_gen(const TablesDev& t, topot_dtype dtype, const void* pixels, long long nblk,
                               long long* cnt, cudaStream_t st);
cudaError_t launch_hist_gen(const EvalPlan& P, const TablesDev& t, int32_t* lo, int32_t* hi, int grid,
                            cudaStream_t st);
cudaError_t launch_slab_sum_i32(const int32_t* parts, int P, long long n, int32_t* out, unsigned* err, int sm_count,
                                cudaStream_t st);
cudaError_t launch_slab_sum_f64(const double* parts, int P, long long n, double* out, int sm_count,
                                cudaStream_t st);
cudaError_t launch_top_prepass(const void* pixels, topot_dtype dtype, int32_t* V, const TopSrc* src, int B, int n,
                               long long max_nv, int sm_count, cudaStream_t st);
cudaError_t launch_top_prepass_u8(const uint8_t* pixels, uint8_t* V, const TopSrc* src, int B, int n, int sm_count,
                                  cudaStream_t st);
int extract_block(int n);
int extract_k(int n);
size_t extract_smem_bytes(int n, int elem_bytes, int row_stride, int stage_rows);
cudaError_t launch_extract_u8(int n, bool top, const ExtractArgs& a, cudaStream_t st);
cudaError_t launch_selftest_wait(int which, unsigned long long limit_ns, unsigned long long* flag, unsigned* err,
                                 cudaStream_t st);
int extract_u8_threads(int n);
int bin_unit_warps();
int bin_chunk();
cudaError_t launch_bin_pack(const BinArgs& a, int B, int pack_blocks_per_image, cudaStream_t st);
cudaError_t launch_bin_tables(const BinArgs& a, cudaStream_t st);
int extract_u8_strip(int n);
size_t extract_u8_smem_bytes(int n, int stage_bytes);
size_t hist_smem_bytes(int td, int T);
cudaError_t launch_hist(const EvalPlan& P, const TablesDev& t, int td, int32_t* lo, int32_t* hi, int grid,
                        cudaStream_t st);
cudaError_t launch_hist_finish(int mode, int B, int D, int T, const long long* chi, int32_t* out,
                               const int32_t* hi, cudaStream_t st);
cudaError_t launch_ht(const EvalPlan& P, const TablesDev& t, int kernel, int precision, bool adjoint, int dl,
                      int split, int grid, double* part, cudaStream_t st);
cudaError_t launch_ht_combine(const EvalPlan& P, int n, int B, int kernel, int precision, int tdh,
                              const double* part, const long long* vsum, int S, double* out, cudaStream_t st);
cudaError_t launch_ht_adj_combine(const EvalPlan& P, int n, int B, int kernel, int precision, int tdh,
                                  const double* part, const double* gout, double* gdirs, cudaStream_t st);
}  // namespace topot

using namespace topot;

struct topot_ktable {
    int K = 0;
    double a = 0.0, h = 0.0;
    int device = 0;
    float2* d32 = nullptr;    // K + 1 padded pairs (see kernel_table_create)
    double* d64 = nullptr;    // y_i
};

struct topot_tables {
    int n = 0, B = 0, NO = 0, S = 0;
    topot_dtype dtype = TOPOT_U8;
    int device = 0, sm_count = 0;
    std::vector<ImgDesc> h_img;
    long long total_entries = 0;
    long long num_tiles = 0;
    int row_stride = 0, stage_rows = 0;
    bool u8 = false;          // 8-bit batch: extraction by k_extract_u8 (either construction)
    int stage_bytes = 0;      // its staged bytes per tile (max over images)
    bool top = false;         // top-dimensional construction: corner image, then extraction
                              // (k_extract_u8 on a u8 corner image, k_extract on an int32 one)
    bool gen = false;         // n = 4: the generic-n kernels (generic.cu) for every step
    void* top_buf = nullptr;  // TopSrc[B] followed by the corner images (u8 or int32)
    TopSrc* d_top = nullptr;
    void* d_corner = nullptr;
    long long max_nv = 0;     // largest corner image (elements)
    // device memory
    void* meta = nullptr;             // one block: img, seg_count, chi, absum, err, ticket, status
    ImgDesc* d_img = nullptr;
    long long* seg_count = nullptr;
    long long* chi = nullptr;
    long long* absum = nullptr;
    unsigned* err = nullptr;
    unsigned* ticket = nullptr;
    int2* order = nullptr;            // [num_tiles] extraction order: (image, local tile)
    unsigned long long* status = nullptr;
    long long* vsum = nullptr;        // [B][S] sum of the values of each table (slabs)
    // 3-D 8-bit whole volumes: the binary path (binary3.cu) for volumes of 0 / 1 voxels
    bool bin3 = false;
    void* bbuf = nullptr;
    BinArgs bin{};
    int bin_pack_blocks = 1;
    cudaStream_t side = nullptr;      // the general kernel runs here beside the binary kernels
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool slab = false;                // tables of slabs of volumes (tables_create_slab)
    size_t clear_bytes = 0;           // bytes from `chi` to the end of `vsum` zeroed per build
    int* arena_idx = nullptr;
    void* arena_val = nullptr;
    // host copies (valid after tables_sync)
    bool host_valid = false;
    std::vector<long long> h_seg_count, h_chi, h_absum;
    // evaluation workspaces, grown on demand, one per family of calls (grid transforms,
    // hybrid transforms, exact representations), so that families can run concurrently
    void* ws[3] = {nullptr, nullptr, nullptr};
    size_t ws_bytes[3] = {0, 0, 0};
    topot_tuning tuning{};

    TablesDev dev() const {
        TablesDev t;
        t.n = n;
        t.B = B;
        t.S = S;
        t.val_bytes = dtype == TOPOT_U8 ? 2 : 4;
        t.img = d_img;
        t.arena_idx = arena_idx;
        t.arena_val = arena_val;
        t.seg_count = seg_count;
        t.chi = chi;
        t.absum = absum;
        t.err = err;
        return t;
    }
};

namespace {

thread_local std::string g_last_error;

topot_status fail(topot_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

topot_status cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? TOPOT_ERR_OOM : TOPOT_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define TOPOT_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

enum WsFamily : int { kWsGrid = 0, kWsHybrid = 1, kWsExact = 2, kWsFamilies = 3 };

topot_status ensure_ws(topot_tables* t, int fam, size_t bytes) {
    if (t->ws_bytes[fam] >= bytes) return TOPOT_OK;
    if (t->ws[fam]) {
        cudaError_t e = cudaFree(t->ws[fam]);
        t->ws[fam] = nullptr;
        t->ws_bytes[fam] = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    const size_t sz = align_up(bytes + bytes / 4, 1 << 20);
    cudaError_t e = cudaMalloc(&t->ws[fam], sz);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
    t->ws_bytes[fam] = sz;
    return TOPOT_OK;
}

// Carves a workspace into aligned pieces.
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

bool valid_dirs_args(const topot_tables* t, const void* d_dirs, int D, int per_image_dirs) {
    return t && d_dirs && D >= 1 && (per_image_dirs == 0 || per_image_dirs == 1);
}

// Directions per ECT work item: 8, 16 or 32 per warp, or 64 (two per lane).
int hist_tile(const topot_tables* t, int D, int nsets_dirs_per_orthant, int T) {
    int td = t->tuning.ect_dirs_per_warp;
    if (td != 8 && td != 16 && td != 32 && td != 64) {
        const int per_orthant = nsets_dirs_per_orthant;
        // 64 (two per lane) halves the blocks per SM; measured slower, left to the autotuner
        td = per_orthant >= 24 ? 32 : (per_orthant >= 12 ? 16 : 8);
    }
    (void)D;
    while (td > 8 && hist_smem_bytes(td, T) > 200 * 1024) td >>= 1;
    return td;
}

}  // namespace

extern "C" {

const char* topot_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// tables_create and tables_create_slab: h_zrange (NULL for whole images) gives per image
// the owned planes [z0, z1) of a volume.
static topot_status create_impl(topot_dtype dtype, int n, const int64_t* h_shapes, const int64_t* h_offsets,
                                const int64_t* h_zrange, int B, topot_construction construction,
                                topot_tables** out) {
    if (!out) return fail(TOPOT_ERR_INVALID_ARG, "tables_create: out is NULL");
    *out = nullptr;
    if (h_zrange && (n != 3 || construction != TOPOT_VERTEX))
        return fail(TOPOT_ERR_UNSUPPORTED, "tables_create_slab: slabs of 3-D volumes, vertex construction only");
    if (construction != TOPOT_VERTEX && construction != TOPOT_TOP)
        return fail(TOPOT_ERR_INVALID_ARG, "tables_create: bad construction");
    if (dtype != TOPOT_U8 && dtype != TOPOT_I32) return fail(TOPOT_ERR_INVALID_ARG, "tables_create: bad dtype");
    if (n < 2 || n > 4) return fail(TOPOT_ERR_INVALID_ARG, "tables_create: n must be 2, 3 or 4");
    if (n == 4 && construction == TOPOT_TOP)
        return fail(TOPOT_ERR_UNSUPPORTED, "tables_create: the top-dimensional construction needs n <= 3");
    if (B < 1 || !h_shapes || !h_offsets) return fail(TOPOT_ERR_INVALID_ARG, "tables_create: bad image list");

    topot_tables* t = new (std::nothrow) topot_tables();
    if (!t) return fail(TOPOT_ERR_OOM, "tables_create: host allocation failed");
    t->n = n;
    t->B = B;
    t->dtype = dtype;
    t->NO = 1 << n;
    t->S = t->NO + t->NO / 2;
    cudaError_t e = cudaGetDevice(&t->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "tables_create: device query");
    }
    const bool top = construction == TOPOT_TOP;
    // the top construction extracts from a corner image (m_k + 1 per axis): u8 with padded
    // rows for 8-bit pixels, int32 otherwise
    const int elem = dtype == TOPOT_U8 ? 1 : 4;
    const int pad = 16 / elem;
    const int tile_v = extract_block(n) * extract_k(n);
    const int NP = n == 3 ? 3 : 1;
    const size_t smem_budget = 96 * 1024;
    t->top = top;
    t->gen = n == 4;                      // generic-n kernels for every step
    t->u8 = dtype == TOPOT_U8 && !t->gen;
    std::vector<TopSrc> h_top(top ? B : 0);
    long long v_elems = 0;
    long long tiles = 0, entries = 0;
    int max_w = 1, max_r = 1;
    t->h_img.resize(B);
    for (int b = 0; b < B; ++b) {
        ImgDesc& I = t->h_img[b];
        memset(&I, 0, sizeof(I));
        long long N = 1;
        for (int k = 0; k < kMaxDim; ++k) {
            const long long pm = k < n ? h_shapes[(long long)b * n + k] : 1;
            // vertices per axis: the pixels (vertex construction) or the pixel corners (top)
            const long long m = (top && k < n) ? pm + 1 : pm;
            if (k < n && (pm < (top ? 1 : 2) || m > (1 << 24))) {
                delete t;
                return fail(TOPOT_ERR_INVALID_ARG, top ? "tables_create: every axis needs 1 <= m_k < 2^24 pixels"
                                                       : "tables_create: every axis needs 2 <= m_k <= 2^24");
            }
            I.m[k] = (int)m;
            N *= m;
            if (top && k < 3) h_top[b].m[k] = (int)pm;
        }
        if (N >= (1ll << 31) || h_offsets[b] < 0) {
            delete t;
            return fail(TOPOT_ERR_INVALID_ARG, "tables_create: an image must have < 2^31 vertices and offset >= 0");
        }
        // owned planes: all, or the slab [z0, z1) whose pixels start at plane max(z0 - 1, 0)
        I.zlo = 0;
        I.zbase = 0;
        I.nz = I.m[2];
        if (h_zrange) {
            const int64_t z0 = h_zrange[2 * (long long)b], z1 = h_zrange[2 * (long long)b + 1];
            if (z0 < 0 || z1 <= z0 || z1 > I.m[2]) {
                delete t;
                return fail(TOPOT_ERR_INVALID_ARG, "tables_create_slab: need 0 <= z0 < z1 <= m_2");
            }
            I.zlo = (int)z0;
            I.zbase = z0 > 0 ? (int)z0 - 1 : 0;
            I.nz = (int)(z1 - z0);
            N = (long long)I.m[0] * I.m[1] * I.nz;   // owned vertices: the capacity of a table
        }
        long long top_q = 0;   // u8 corner image: positions (rows padded to top_pitch)
        if (top) {
            // corner images start at 16-byte boundaries
            h_top[b].pix_offset = h_offsets[b];
            h_top[b].v_offset = v_elems;
            I.offset = v_elems;
            if (t->u8) {
                I.top_pitch = (int)align_up((size_t)I.m[0], 16);
                top_q = (long long)I.top_pitch * I.m[1] * I.m[2];
                if (top_q >= (1ll << 31)) {
                    delete t;
                    return fail(TOPOT_ERR_INVALID_ARG, "tables_create: corner image of >= 2^31 bytes");
                }
                h_top[b].pitch = I.top_pitch;
                v_elems += top_q;
            } else {
                v_elems += (N + 3) & ~3ll;
            }
            t->max_nv = std::max(t->max_nv, N);
        } else {
            I.offset = h_offsets[b];
        }
        I.N = N;
        I.seg_base = entries;
        entries += N * t->S;
        I.tile_begin = tiles;
        const int m0 = I.m[0], m1 = I.m[1];
        for (int k = 0; k < kMaxDim; ++k) I.inv2m[k] = I.m[k] > 1 ? 0.5 / (double)(I.m[k] - 1) : 0.0;
        if (t->gen) {   // one block of gen_block() vertices per tile
            tiles += (N + gen_block() - 1) / gen_block();
            continue;
        }
        if (t->u8 && top) {
            // runs of `cap` positions of the corner image (rows and planes at fixed offsets);
            // one staged run per offset of the 2^n pixels around a corner
            const int cap = extract_u8_strip(n) * extract_u8_threads(n);
            I.W = cap;
            I.R = 1;
            I.spr = extract_u8_threads(n);
            I.rs = cap + 16;
            I.nz = 1;
            I.div_pitch = make_fastdiv((uint32_t)I.top_pitch);
            t->stage_bytes = std::max(t->stage_bytes, (n == 3 ? 4 : 2) * I.rs + 32);
            I.segs_per_row = 1;
            I.tiles_per_plane = (int)((top_q + cap - 1) / cap);
        } else if (t->u8) {
            // strips of `strip` vertices, one per thread; R full rows or one piece of a row
            const int strip = extract_u8_strip(n), threads = extract_u8_threads(n);
            I.W = std::min(m0, threads * strip);
            I.spr = (I.W + strip - 1) / strip;
            I.R = I.W == m0 ? std::max(1, std::min(threads / I.spr, m1)) : 1;
            // rows contiguous in the stage when whole rows are 16-byte aligned in the image
            I.packed = I.W == m0 && m0 % 16 == 0 && h_offsets[b] % 16 == 0;
            I.rs = I.packed ? m0 : (int)align_up((size_t)(16 + strip * I.spr + 1), 16);
            t->stage_bytes = std::max(t->stage_bytes, NP * (I.R + 2) * I.rs + 32);
        } else if (m0 <= tile_v) {
            I.W = m0;
            I.R = std::max(1, std::min(tile_v / m0, m1));
            // the staged rows must fit the shared-memory budget
            while (I.R > 1 && (size_t)NP * (I.R + 2) * align_up((size_t)(pad + m0 + 1), pad) * elem > smem_budget)
                --I.R;
        } else {
            I.W = tile_v;
            I.R = 1;
        }
        if (!(t->u8 && top)) {
            I.segs_per_row = (m0 + I.W - 1) / I.W;
            I.tiles_per_plane = ((m1 + I.R - 1) / I.R) * I.segs_per_row;
        }
        tiles += (long long)I.tiles_per_plane * I.nz;
        I.div0 = make_fastdiv((uint32_t)m0);
        I.div1 = make_fastdiv((uint32_t)m1);
        I.div_spr = make_fastdiv((uint32_t)std::max(1, I.spr));
        I.div_segs = make_fastdiv((uint32_t)I.segs_per_row);
        I.div_tpp = make_fastdiv((uint32_t)I.tiles_per_plane);
        max_w = std::max(max_w, I.W);
        max_r = std::max(max_r, I.R);
    }
    t->total_entries = entries;
    t->num_tiles = tiles;
    t->row_stride = (int)align_up((size_t)(pad + max_w + 1), pad);
    t->stage_rows = max_r + 2;

    // device allocations
    size_t off = 0;
    auto place = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t o = off;
        off += bytes;
        return o;
    };
    const size_t o_img = place(sizeof(ImgDesc) * B);
    const size_t o_ord = place(sizeof(int2) * (size_t)tiles);
    const size_t o_cnt = place(sizeof(long long) * B * t->S);
    const size_t o_err = place(sizeof(unsigned));
    const size_t o_chi = place(sizeof(long long) * B);
    const size_t o_abs = place(sizeof(long long) * B * t->NO);
    const size_t o_tic = place(sizeof(unsigned));
    const size_t o_sta = place(sizeof(unsigned long long) * tiles * t->S);
    const size_t o_vsum = place(sizeof(long long) * B * t->S);
    const size_t meta_bytes = off;
    e = cudaMalloc(&t->meta, meta_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&t->arena_idx, sizeof(int) * (size_t)entries);
    if (e == cudaSuccess) e = cudaMalloc(&t->arena_val, (size_t)(dtype == TOPOT_U8 ? 2 : 4) * (size_t)entries);
    if (e != cudaSuccess) {
        free_tables(t);
        return cuda_fail(e, "tables_create: device allocation");
    }
    char* m = reinterpret_cast<char*>(t->meta);
    t->d_img = reinterpret_cast<ImgDesc*>(m + o_img);
    t->seg_count = reinterpret_cast<long long*>(m + o_cnt);
    t->err = reinterpret_cast<unsigned*>(m + o_err);
    t->chi = reinterpret_cast<long long*>(m + o_chi);
    t->absum = reinterpret_cast<long long*>(m + o_abs);
    t->ticket = reinterpret_cast<unsigned*>(m + o_tic);
    t->order = reinterpret_cast<int2*>(m + o_ord);
    t->status = reinterpret_cast<unsigned long long*>(m + o_sta);
    t->vsum = reinterpret_cast<long long*>(m + o_vsum);
    t->slab = h_zrange != nullptr;
    t->clear_bytes = meta_bytes - o_chi;
    if (top) {
        const size_t src_bytes = align_up(sizeof(TopSrc) * B, 256);
        e = cudaMalloc(&t->top_buf, src_bytes + (size_t)elem * (size_t)v_elems);
        if (e != cudaSuccess) {
            free_tables(t);
            return cuda_fail(e, "tables_create: corner image allocation");
        }
        t->d_top = reinterpret_cast<TopSrc*>(t->top_buf);
        t->d_corner = reinterpret_cast<char*>(t->top_buf) + src_bytes;
        e = cudaMemcpy(t->d_top, h_top.data(), sizeof(TopSrc) * B, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_tables(t);
            return cuda_fail(e, "tables_create: corner image descriptors");
        }
    }
    e = cudaMemcpy(t->d_img, t->h_img.data(), sizeof(ImgDesc) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && t->u8 && n == 3 && !top && !h_zrange && B <= 65535) {
        // binary path: packed bits (zero border), per-unit counts and offsets, block and
        // chunk lists
        const long long U = 32, UW = bin_unit_warps(), C = bin_chunk();
        std::vector<BinImg> bi(B);
        std::vector<int2> blk, chk;
        long long pk = 0, ub = 0, most = 1;
        for (int b = 0; b < B; ++b) {
            const ImgDesc& I = t->h_img[b];
            BinImg& Q = bi[b];
            Q.pix_off = h_offsets[b];
            Q.m0 = I.m[0];
            Q.m1 = I.m[1];
            Q.m2 = I.m[2];
            Q.wpr = (I.m[0] + 31) / 32;
            const long long nw = (long long)Q.m2 * Q.m1 * Q.wpr;
            Q.nunits = (int)((nw + U - 1) / U);
            Q.pk_off = pk;
            Q.unit_begin = ub;
            Q.seg_base = I.seg_base;
            Q.N = I.N;
            Q.div_wpr = make_fastdiv((uint32_t)Q.wpr);
            Q.div_m1 = make_fastdiv((uint32_t)Q.m1);
            pk += ((long long)(Q.m2 + 2) * (Q.m1 + 2) * (Q.wpr + 2) + 3) & ~3ll;
            ub += Q.nunits;
            most = std::max(most, nw);
            for (long long lu = 0; lu < Q.nunits; lu += UW) blk.push_back(make_int2(b, (int)lu));
            for (long long j = 0; j * C < Q.nunits; ++j) chk.push_back(make_int2(b, (int)j));
        }
        size_t bo = 0;
        auto bplace = [&](size_t bytes) {
            bo = align_up(bo, 256);
            const size_t o = bo;
            bo += bytes;
            return o;
        };
        const size_t o_bi = bplace(sizeof(BinImg) * B);
        const size_t o_pk = bplace(sizeof(uint32_t) * (size_t)pk);
        const size_t o_nb = bplace(sizeof(unsigned) * (B + 1));
        const size_t o_uc = bplace(sizeof(uint32_t) * 6 * (size_t)ub);
        const size_t o_uo = bplace(sizeof(int) * 12 * (size_t)ub);
        const size_t o_cs = bplace(sizeof(int) * 12 * chk.size());
        const size_t o_bl = bplace(sizeof(int2) * blk.size());
        const size_t o_ch = bplace(sizeof(int2) * chk.size());
        e = cudaMalloc(&t->bbuf, bo);
        if (e == cudaSuccess) {
            char* q = reinterpret_cast<char*>(t->bbuf);
            BinArgs& a = t->bin;
            a.img = reinterpret_cast<BinImg*>(q + o_bi);
            a.packed = reinterpret_cast<uint32_t*>(q + o_pk);
            a.nonbin = reinterpret_cast<unsigned*>(q + o_nb);
            a.ucount = reinterpret_cast<uint32_t*>(q + o_uc);
            a.uoff = reinterpret_cast<int*>(q + o_uo);
            a.csum = reinterpret_cast<int*>(q + o_cs);
            a.blocks = reinterpret_cast<int2*>(q + o_bl);
            a.nblocks = (int)blk.size();
            a.chunks = reinterpret_cast<int2*>(q + o_ch);
            a.nchunks = (int)chk.size();
            e = cudaMemcpy(q + o_bi, bi.data(), sizeof(BinImg) * B, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemset(q + o_pk, 0, sizeof(uint32_t) * (size_t)pk);   // borders stay 0
            if (e == cudaSuccess)
                e = cudaMemcpy(q + o_bl, blk.data(), sizeof(int2) * blk.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(q + o_ch, chk.data(), sizeof(int2) * chk.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming);
            t->bin3 = true;
            t->bin_pack_blocks = (int)std::min<long long>((most + 255) / 256, std::max(1, 4 * t->sm_count / B));
        }
    }
    if (e == cudaSuccess && !t->gen) {
        // Extraction order: round robin over the images by local tile index.  The look-back
        // of a tile waits only on earlier tiles of its own image; interleaving the images
        // keeps few tiles of any one image in flight, so its prefix chain is short.
        std::vector<int2> order;
        order.reserve((size_t)tiles);
        std::vector<long long> ntile(B);
        long long most = 0;
        for (int b = 0; b < B; ++b) {
            const long long nb = (b + 1 < B ? t->h_img[b + 1].tile_begin : tiles) - t->h_img[b].tile_begin;
            ntile[b] = nb;
            most = std::max(most, nb);
        }
        for (long long lt = 0; lt < most; ++lt)
            for (int b = 0; b < B; ++b)
                if (lt < ntile[b]) order.push_back(make_int2(b, (int)lt));
        e = cudaMemcpy(t->order, order.data(), sizeof(int2) * (size_t)tiles, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(t->seg_count, 0, o_chi - o_cnt);   // counts + error word
    if (e != cudaSuccess) {
        free_tables(t);
        return cuda_fail(e, "tables_create: initialise metadata");
    }
    const size_t smem = t->gen ? 0
                               : (t->u8 ? extract_u8_smem_bytes(n, t->stage_bytes)
                                        : extract_smem_bytes(n, elem, t->row_stride, t->stage_rows));
    if (smem > 200 * 1024) {
        free_tables(t);
        return fail(TOPOT_ERR_UNSUPPORTED, "tables_create: rows too wide for the shared-memory stage");
    }
    *out = t;
    return TOPOT_OK;
}

extern "C" {

topot_status tables_create(topot_dtype dtype, int n, const int64_t* h_shapes, const int64_t* h_offsets, int B,
                           topot_construction construction, topot_tables** out) {
    return create_impl(dtype, n, h_shapes, h_offsets, nullptr, B, construction, out);
}

topot_status tables_create_slab(topot_dtype dtype, int n, const int64_t* h_shapes, const int64_t* h_offsets,
                                const int64_t* h_zrange, int B, topot_tables** out) {
    if (!h_zrange) return fail(TOPOT_ERR_INVALID_ARG, "tables_create_slab: h_zrange is NULL");
    return create_impl(dtype, n, h_shapes, h_offsets, h_zrange, B, TOPOT_VERTEX, out);
}

topot_status tables_build(topot_tables* t, const void* d_pixels, void* stream) {
    if (!t || !d_pixels) return fail(TOPOT_ERR_INVALID_ARG, "tables_build: NULL argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    t->host_valid = false;
    TOPOT_CUDA(cudaMemsetAsync(t->chi, 0, t->clear_bytes, st));
    ExtractArgs a;
    a.t = t->dev();
    a.pixels = d_pixels;
    a.num_tiles = t->num_tiles;
    a.ticket = t->ticket;
    a.order = t->order;
    a.status = t->status;
    a.nonbin = nullptr;
    a.row_stride = t->row_stride;
    a.stage_rows = t->stage_rows;
    a.stage_bytes = t->stage_bytes;
    if (t->gen) {
        // per-block counts live in the look-back status words (tiles x S entries)
        TOPOT_CUDA(launch_extract_gen(t->dev(), t->dtype, d_pixels, t->num_tiles,
                                      reinterpret_cast<long long*>(t->status), st));
    } else if (t->top && t->u8) {
        TOPOT_CUDA(launch_top_prepass_u8(reinterpret_cast<const uint8_t*>(d_pixels),
                                         reinterpret_cast<uint8_t*>(t->d_corner), t->d_top, t->B, t->n, t->sm_count,
                                         st));
        a.pixels = t->d_corner;
        TOPOT_CUDA(launch_extract_u8(t->n, true, a, st));
    } else if (t->top) {
        TOPOT_CUDA(launch_top_prepass(d_pixels, t->dtype, reinterpret_cast<int32_t*>(t->d_corner), t->d_top, t->B,
                                      t->n, t->max_nv, t->sm_count, st));
        a.pixels = t->d_corner;
        TOPOT_CUDA(launch_extract(t->n, t->dtype, true, a, st));
    } else if (t->u8) {
        if (t->bin3) {
            // The pack flags the volumes that are not binary.  Then the general kernel (which
            // skips binary volumes) runs on the side stream while the binary kernels run on
            // `st`; the two touch disjoint tables, and `st` waits for both.
            BinArgs b = t->bin;
            b.t = t->dev();
            b.pixels = d_pixels;
            TOPOT_CUDA(cudaMemsetAsync(b.nonbin, 0, sizeof(unsigned) * (t->B + 1), st));
            TOPOT_CUDA(launch_bin_pack(b, t->B, t->bin_pack_blocks, st));
            a.nonbin = b.nonbin;
            TOPOT_CUDA(cudaEventRecord(t->ev_fork, st));
            TOPOT_CUDA(cudaStreamWaitEvent(t->side, t->ev_fork, 0));
            TOPOT_CUDA(launch_extract_u8(t->n, false, a, t->side));
            TOPOT_CUDA(cudaEventRecord(t->ev_join, t->side));
            TOPOT_CUDA(launch_bin_tables(b, st));
            TOPOT_CUDA(cudaStreamWaitEvent(st, t->ev_join, 0));
        } else {
            TOPOT_CUDA(launch_extract_u8(t->n, false, a, st));
        }
    } else {
        TOPOT_CUDA(launch_extract(t->n, t->dtype, false, a, st));
    }
    // a slab's tables need not sum to zero: their value sums let the hybrid transforms
    // put back the constant kbar(0) that the FP32C kernels leave out
    if (t->slab) TOPOT_CUDA(launch_segment_sums(t->dev(), t->vsum, st));
    return TOPOT_OK;
}

topot_status tables_sync(topot_tables* t, void* stream) {
    if (!t) return fail(TOPOT_ERR_INVALID_ARG, "tables_sync: NULL handle");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    TOPOT_CUDA(cudaStreamSynchronize(st));
    t->h_seg_count.resize((size_t)t->B * t->S);
    t->h_chi.resize(t->B);
    t->h_absum.resize((size_t)t->B * t->NO);
    unsigned err = 0;
    TOPOT_CUDA(cudaMemcpy(t->h_seg_count.data(), t->seg_count, sizeof(long long) * t->B * t->S,
                          cudaMemcpyDeviceToHost));
    TOPOT_CUDA(cudaMemcpy(t->h_chi.data(), t->chi, sizeof(long long) * t->B, cudaMemcpyDeviceToHost));
    TOPOT_CUDA(cudaMemcpy(t->h_absum.data(), t->absum, sizeof(long long) * t->B * t->NO, cudaMemcpyDeviceToHost));
    TOPOT_CUDA(cudaMemcpy(&err, t->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) TOPOT_CUDA(cudaMemset(t->err, 0, sizeof(unsigned)));
    t->host_valid = true;
    if (err & kDevErrTimeout) return fail(TOPOT_ERR_TIMEOUT, "device-side wait timed out");
    if (err & kDevErrOverflow)
        return fail(TOPOT_ERR_OVERFLOW, "value out of range (int32 pixel |phi| >= 2^26 or ECT bound >= 2^31)");
    return TOPOT_OK;
}

topot_status build_critical_tables(const void* d_pixels, topot_dtype dtype, int n, const int64_t* h_shapes,
                                   const int64_t* h_offsets, int B, topot_construction construction, void* stream,
                                   topot_tables** out) {
    if (!out) return fail(TOPOT_ERR_INVALID_ARG, "build_critical_tables: out is NULL");
    if (!d_pixels) return fail(TOPOT_ERR_INVALID_ARG, "build_critical_tables: d_pixels is NULL");
    topot_tables* t = nullptr;
    topot_status s = tables_create(dtype, n, h_shapes, h_offsets, B, construction, &t);
    if (s != TOPOT_OK) return s;
    s = tables_build(t, d_pixels, stream);
    if (s == TOPOT_OK) s = tables_sync(t, stream);
    if (s != TOPOT_OK) {
        const std::string msg = g_last_error;
        free_tables(t);
        g_last_error = msg;
        return s;
    }
    *out = t;
    return TOPOT_OK;
}

topot_status tables_info(const topot_tables* t, int image, int orthant, int64_t* n_lower, int64_t* n_delta,
                         int64_t* chi) {
    if (!t) return fail(TOPOT_ERR_INVALID_ARG, "tables_info: NULL handle");
    if (!t->host_valid) return fail(TOPOT_ERR_INVALID_ARG, "tables_info: call tables_sync after tables_build");
    if (image < 0 || image >= t->B || orthant < 0 || orthant >= t->NO)
        return fail(TOPOT_ERR_INVALID_ARG, "tables_info: image or orthant out of range");
    const int rep = (orthant & (t->NO >> 1)) ? (orthant ^ (t->NO - 1)) : orthant;
    const long long* c = t->h_seg_count.data() + (size_t)image * t->S;
    if (n_lower) *n_lower = c[orthant];
    if (n_delta) *n_delta = c[t->NO + rep];
    if (chi) *chi = t->h_chi[image];
    return TOPOT_OK;
}

topot_status tables_copy_to_host(const topot_tables* t, int image, int orthant, int kind, int32_t* h_idx,
                                 int32_t* h_val) {
    if (!t || !h_idx || !h_val) return fail(TOPOT_ERR_INVALID_ARG, "tables_copy_to_host: NULL argument");
    if (!t->host_valid) return fail(TOPOT_ERR_INVALID_ARG, "tables_copy_to_host: call tables_sync first");
    if (image < 0 || image >= t->B || orthant < 0 || orthant >= t->NO || (kind != 0 && kind != 1))
        return fail(TOPOT_ERR_INVALID_ARG, "tables_copy_to_host: bad image, orthant or kind");
    if (kind == 1 && orthant >= t->NO / 2)
        return fail(TOPOT_ERR_INVALID_ARG, "tables_copy_to_host: Delta tables exist for orthants < 2^(n-1)");
    const int seg = kind == 0 ? orthant : t->NO + orthant;
    const ImgDesc& I = t->h_img[image];
    const long long cnt = t->h_seg_count[(size_t)image * t->S + seg];
    const long long base = I.seg_base + (long long)seg * I.N;
    if (cnt == 0) return TOPOT_OK;
    TOPOT_CUDA(cudaMemcpy(h_idx, t->arena_idx + base, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
    if (t->dtype == TOPOT_U8) {
        std::vector<int16_t> tmp((size_t)cnt);
        TOPOT_CUDA(cudaMemcpy(tmp.data(), reinterpret_cast<int16_t*>(t->arena_val) + base, sizeof(int16_t) * cnt,
                              cudaMemcpyDeviceToHost));
        for (long long i = 0; i < cnt; ++i) h_val[i] = tmp[(size_t)i];
    } else {
        TOPOT_CUDA(cudaMemcpy(h_val, reinterpret_cast<int32_t*>(t->arena_val) + base, sizeof(int32_t) * cnt,
                              cudaMemcpyDeviceToHost));
    }
    return TOPOT_OK;
}

topot_status tables_set_tuning(topot_tables* t, const topot_tuning* tuning) {
    if (!t) return fail(TOPOT_ERR_INVALID_ARG, "tables_set_tuning: NULL handle");
    if (!tuning) {
        t->tuning = topot_tuning{};
        return TOPOT_OK;
    }
    const topot_tuning& u = *tuning;
    if ((u.ect_dirs_per_warp && u.ect_dirs_per_warp != 8 && u.ect_dirs_per_warp != 16 &&
         u.ect_dirs_per_warp != 32 && u.ect_dirs_per_warp != 64) ||
        (u.ht_dirs_per_lane && u.ht_dirs_per_lane != 1 && u.ht_dirs_per_lane != 2 && u.ht_dirs_per_lane != 4 &&
         u.ht_dirs_per_lane != 8) ||
        u.ect_chunk < 0 || (u.ect_chunk % 256) != 0 || u.ht_chunk < 0 || (u.ht_chunk % 256) != 0 ||
        u.ect_ctas_per_sm < 0 || u.ect_ctas_per_sm > 32 || u.ht_ctas_per_sm < 0 || u.ht_ctas_per_sm > 32 ||
        (u.ht_warp_split != 0 && u.ht_warp_split != 1 && u.ht_warp_split != 2))
        return fail(TOPOT_ERR_INVALID_ARG, "tables_set_tuning: value out of range");
    t->tuning = u;
    return TOPOT_OK;
}

void free_tables(topot_tables* t) {
    if (!t) return;
    for (int f = 0; f < kWsFamilies; ++f)
        if (t->ws[f]) cudaFree(t->ws[f]);
    if (t->top_buf) cudaFree(t->top_buf);
    if (t->bbuf) cudaFree(t->bbuf);
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    if (t->ev_join) cudaEventDestroy(t->ev_join);
    if (t->side) cudaStreamDestroy(t->side);
    if (t->arena_val) cudaFree(t->arena_val);
    if (t->arena_idx) cudaFree(t->arena_idx);
    if (t->meta) cudaFree(t->meta);
    delete t;
}

// Bound on the work items of a plan: with automatic chunking the planner aims at `target`
// items of balanced size, plus at most one partial chunk per (pair, tile), and every
// direction set has at most D / tile + 2^n tiles over its orthants; with a requested
// chunk, every (tile, chunk) of every image.  `parts`: pairs per (image, orthant).
static long long plan_max_items(const topot_tables* t, int D, int tile, int chunk_req, int parts, int target) {
    const long long tiles = (D + tile - 1) / tile + t->NO;
    if (chunk_req <= 0) return target + (long long)t->B * tiles * parts;
    long long m = 0;
    for (int b = 0; b < t->B; ++b) m += tiles * ((t->h_img[b].N + chunk_req - 1) / chunk_req) * parts;
    return m;
}

// ---- grid transforms ---------------------------------------------------------------------------

static topot_status grid_transform(const char* name, int mode, const topot_tables* tc, const double* d_dirs, int D,
                                   int per_image_dirs, double t_min, double t_max, int T, int32_t* d_out,
                                   void* stream) {
    topot_tables* t = const_cast<topot_tables*>(tc);
    if (!valid_dirs_args(t, d_dirs, D, per_image_dirs) || !d_out)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad handle, directions or output");
    if (T < 2 || !(t_max > t_min) || !std::isfinite(t_min) || !std::isfinite(t_max))
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": need T >= 2 and finite t_min < t_max");
    if (t->host_valid) {
        const long long lim = mode == kModeRadon ? (1ll << 31) / 3 : (1ll << 31);
        for (long long v : t->h_absum)
            if (v >= lim)
                return fail(TOPOT_ERR_OVERFLOW, std::string(name) + ": sum |Delta^-| too large for int32 results");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nsets = per_image_dirs ? t->B : 1;
    const int NO = t->NO;
    const int td = t->gen ? 32 : hist_tile(t, D, D / NO, T);
    if (!t->gen && hist_smem_bytes(td, T) > 200 * 1024)
        return fail(TOPOT_ERR_UNSUPPORTED, std::string(name) + ": too many thresholds for the shared histogram");
    const int npairs = t->B * NO * (mode == kModeRadon ? 2 : 1);
    const size_t out_elems = (size_t)t->B * D * T;
    const long long max_items =
        plan_max_items(t, D, td, t->tuning.ect_chunk, mode == kModeRadon ? 2 : 1, t->sm_count * 16);
    const size_t need = 4096 + sizeof(int) * (size_t)nsets * D * 2 + sizeof(int) * (size_t)nsets * (NO + 1) +
                        sizeof(long long) * (npairs + 1) + sizeof(int) * npairs + sizeof(double) * T +
                        sizeof(int) * (size_t)max_items +
                        (mode == kModeRadon ? sizeof(int32_t) * out_elems : 0) + 9 * 256;
    topot_status s = ensure_ws(t, kWsGrid, need);
    if (s != TOPOT_OK) return s;
    Carver cv{reinterpret_cast<char*>(t->ws[kWsGrid])};
    EvalPlan P{};
    P.mode = mode;
    P.nsets = nsets;
    P.D = D;
    P.tile_dirs = td;
    P.chunk_req = t->tuning.ect_chunk;
    P.target_items = t->sm_count * 16;
    P.npairs = npairs;
    P.max_items = max_items;
    P.dirs = d_dirs;
    P.ctl = cv.take<int>(8);
    P.perm = cv.take<int>((size_t)nsets * D);
    P.rank = cv.take<int>((size_t)nsets * D);
    P.boff = cv.take<int>((size_t)nsets * (NO + 1));
    P.pair_items = cv.take<long long>(npairs + 1);
    P.pair_chunks = cv.take<int>(npairs);
    P.thr = cv.take<double>(T);
    P.item_pair = cv.take<int>((size_t)max_items);
    P.T = T;
    P.t_min = t_min;
    P.t_max = t_max;
    int32_t* hi = mode == kModeRadon ? cv.take<int32_t>(out_elems) : nullptr;

    TOPOT_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int32_t) * out_elems, st));
    if (hi) TOPOT_CUDA(cudaMemsetAsync(hi, 0, sizeof(int32_t) * out_elems, st));
    TOPOT_CUDA(launch_dir_prep(P, t->n, st));
    TOPOT_CUDA(launch_plan(P, t->dev(), st));
    int per_sm = std::max(1, (int)((220 * 1024) / (hist_smem_bytes(td, T) + 1024)));
    per_sm = std::min(per_sm, 8);
    if (t->tuning.ect_ctas_per_sm > 0) per_sm = std::min(per_sm, t->tuning.ect_ctas_per_sm);
    if (t->gen) TOPOT_CUDA(launch_hist_gen(P, t->dev(), d_out, hi, t->sm_count * 8, st));
    else TOPOT_CUDA(launch_hist(P, t->dev(), td, d_out, hi, t->sm_count * per_sm, st));
    TOPOT_CUDA(launch_hist_finish(mode, t->B, D, T, t->chi, d_out, hi, st));
    return TOPOT_OK;
}

topot_status ect(const topot_tables* t, const double* d_dirs, int D, int per_image_dirs, double t_min,
                 double t_max, int T, int32_t* d_out, void* stream) {
    return grid_transform("ect", kModeECT, t, d_dirs, D, per_image_dirs, t_min, t_max, T, d_out, stream);
}

topot_status radon(const topot_tables* t, const double* d_dirs, int D, int per_image_dirs, double t_min,
                   double t_max, int T, int32_t* d_out, void* stream) {
    return grid_transform("radon", kModeRadon, t, d_dirs, D, per_image_dirs, t_min, t_max, T, d_out, stream);
}

// ---- hybrid transforms ----------------------------------------------------------------------

// Tile and chunk choices of one hybrid-transform call, and the scratch they need.  Both
// hybrid_transform (workspace grown with cudaMalloc) and hybrid_transform_noalloc (fixed
// array) size and carve their scratch through these two functions, so that the two give
// the same result for the same call.
struct HtSizing {
    int dl = 1;               // directions per lane
    int split = 1;            // point groups per warp (FP32C forward)
    int tdh = 32;             // directions per tile
    int ncomp = 1;            // FP64 partials per direction and item
    int npairs = 0;
    int target = 0;           // automatic chunking aims at about this many items
    long long max_items = 0;  // capacity of the per-item partials
    size_t part_elems = 0;
    size_t need = 0;          // scratch bytes (plan + partials + alignment slack)
};

static HtSizing ht_sizing(const topot_tables* t, topot_kernel kernel, topot_precision precision, int D,
                          int per_image_dirs, bool adjoint) {
    HtSizing z;
    const int nsets = per_image_dirs ? t->B : 1;
    const int NO = t->NO;
    if (precision == TOPOT_FP32C && !t->gen) {
        z.dl = t->tuning.ht_dirs_per_lane;
        z.split = t->tuning.ht_warp_split;
        const int per_orthant = D / NO;
        if (z.dl == 0) {
            // a tile of 32 dl / split directions: fill it; with fewer than 128 directions per
            // orthant two point groups per warp keep two or four directions per lane
            z.dl = per_orthant >= 64 ? 4 : (per_orthant >= 32 ? 2 : 1);
            if (z.split == 0) z.split = (per_orthant >= 32 && per_orthant < 128) ? 2 : 1;
            if (kernel == TOPOT_LAPLACE && per_orthant >= 256) z.dl = 8;
        }
        if (z.dl == 8 && kernel != TOPOT_LAPLACE) z.dl = 4;
        if (z.split == 0 || z.dl == 1 || z.dl == 8 || adjoint || kernel == TOPOT_TABLE) z.split = 1;
        // adjoint: two direction pairs per lane for the one-component kernels in 2-D, else one
        if (adjoint && kernel != TOPOT_TABLE)
            z.dl = std::min(z.dl, (kernel != TOPOT_FOURIER && t->n == 2) ? 4 : 2);
    }
    z.tdh = 32 * z.dl / z.split;
    const int nk = kernel == TOPOT_FOURIER ? 2 : 1;
    z.ncomp = adjoint ? nk * t->n : nk;
    z.npairs = t->B * NO / 2;   // (image, representative orthant): an orthant shares tiles with its partner
    z.target = t->sm_count * 16;
    z.max_items = plan_max_items(t, D, z.tdh, t->tuning.ht_chunk, 1, z.target);
    z.part_elems = (size_t)z.max_items * z.tdh * z.ncomp;
    z.need = 4096 + sizeof(int) * (size_t)nsets * D * 2 + sizeof(int) * (size_t)nsets * (NO + 1) +
             sizeof(long long) * (z.npairs + 1) + sizeof(int) * z.npairs + sizeof(double) * z.part_elems +
             2 * sizeof(int) * (size_t)z.max_items + 10 * 256;
    return z;
}

// Lays the plan and the partials of a call out in `scratch` (at least z.need bytes).  Every
// field is written by the planning kernels before it is read, so old contents are harmless.
static EvalPlan ht_carve(const topot_tables* t, const HtSizing& z, const double* d_dirs, int D, int per_image_dirs,
                         void* scratch, double** part) {
    const int nsets = per_image_dirs ? t->B : 1;
    Carver cv{reinterpret_cast<char*>(scratch)};
    EvalPlan P{};
    P.mode = kModeHT;
    P.nsets = nsets;
    P.D = D;
    P.tile_dirs = z.tdh;
    P.chunk_req = t->tuning.ht_chunk;
    P.target_items = z.target;
    P.npairs = z.npairs;
    P.max_items = z.max_items;
    P.dirs = d_dirs;
    P.ctl = cv.take<int>(8);
    P.perm = cv.take<int>((size_t)nsets * D);
    P.rank = cv.take<int>((size_t)nsets * D);
    P.boff = cv.take<int>((size_t)nsets * (t->NO + 1));
    P.pair_items = cv.take<long long>(z.npairs + 1);
    P.pair_chunks = cv.take<int>(z.npairs);
    P.thr = nullptr;
    P.T = 0;
    *part = cv.take<double>(z.part_elems);
    P.item_pair = cv.take<int>((size_t)z.max_items);
    P.wide_items = cv.take<int>((size_t)z.max_items);
    return P;
}

static topot_status ht_common(const char* name, const topot_tables* tc, topot_kernel kernel,
                              topot_precision precision, const double* d_dirs, int D, int per_image_dirs,
                              bool adjoint, const double* d_gout, double* d_out, void* stream,
                              const topot_ktable* kt = nullptr) {
    topot_tables* t = const_cast<topot_tables*>(tc);
    if (!valid_dirs_args(t, d_dirs, D, per_image_dirs) || !d_out || (adjoint && !d_gout))
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad handle, directions or output");
    if (kernel == TOPOT_TABLE) {
        if (!kt) return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": TABLE needs hybrid_transform_table");
        if (kt->device != t->device)
            return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": kernel table on another device");
    } else if (kernel != TOPOT_LAPLACE && kernel != TOPOT_FOURIER && kernel != TOPOT_BESSEL && kernel != TOPOT_SINE) {
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad kernel");
    }
    if (precision != TOPOT_FP32C && precision != TOPOT_FP64)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad precision");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const HtSizing z = ht_sizing(t, kernel, precision, D, per_image_dirs, adjoint);
    topot_status s = ensure_ws(t, kWsHybrid, z.need);
    if (s != TOPOT_OK) return s;
    double* part = nullptr;
    EvalPlan P = ht_carve(t, z, d_dirs, D, per_image_dirs, t->ws[kWsHybrid], &part);
    if (kernel == TOPOT_TABLE) {
        P.ktab = kt->d32;
        P.ktab64 = kt->d64;
        P.ktab_k = kt->K;
        P.ktab_a = kt->a;
        P.ktab_h = kt->h;
    }
    const int dl = z.dl, tdh = z.tdh;

    TOPOT_CUDA(launch_dir_prep(P, t->n, st));
    TOPOT_CUDA(launch_plan(P, t->dev(), st));
    const int per_sm = t->tuning.ht_ctas_per_sm > 0 ? t->tuning.ht_ctas_per_sm : 4;
    TOPOT_CUDA(launch_ht(P, t->dev(), kernel, precision, adjoint, dl, z.split, t->sm_count * per_sm, part, st));
    if (adjoint)
        TOPOT_CUDA(launch_ht_adj_combine(P, t->n, t->B, kernel, precision, tdh, part, d_gout, d_out, st));
    else
        TOPOT_CUDA(launch_ht_combine(P, t->n, t->B, kernel, precision, tdh, part, t->slab ? t->vsum : nullptr,
                                     t->S, d_out, st));
    return TOPOT_OK;
}

topot_status hybrid_transform(const topot_tables* t, topot_kernel kernel, topot_precision precision,
                              const double* d_dirs, int D, int per_image_dirs, double* d_out, void* stream) {
    return ht_common("hybrid_transform", t, kernel, precision, d_dirs, D, per_image_dirs, false, nullptr, d_out,
                     stream);
}

topot_status hybrid_transform_grad(const topot_tables* t, topot_kernel kernel, topot_precision precision,
                                   const double* d_dirs, int D, int per_image_dirs, const double* d_gout,
                                   double* d_gdirs, void* stream) {
    return ht_common("hybrid_transform_grad", t, kernel, precision, d_dirs, D, per_image_dirs, true, d_gout,
                     d_gdirs, stream);
}

// ---- tabulated kernels ----------------------------------------------------------------------

topot_status kernel_table_create(const double* h_values, int K, double s_min, double s_max, topot_ktable** out) {
    if (!out) return fail(TOPOT_ERR_INVALID_ARG, "kernel_table_create: out is NULL");
    *out = nullptr;
    if (!h_values || K < 2 || K > 16384)
        return fail(TOPOT_ERR_INVALID_ARG, "kernel_table_create: need 2 <= K <= 16384 samples");
    if (!std::isfinite(s_min) || !std::isfinite(s_max) || !(s_min < s_max))
        return fail(TOPOT_ERR_INVALID_ARG, "kernel_table_create: need finite s_min < s_max");
    for (int i = 0; i < K; ++i) {
        if (!std::isfinite(h_values[i])) return fail(TOPOT_ERR_INVALID_ARG, "kernel_table_create: non-finite sample");
        // the FP32 table holds samples, half-sums and differences: keep them all finite
        if (std::fabs(h_values[i]) > 1e37)
            return fail(TOPOT_ERR_INVALID_ARG, "kernel_table_create: |sample| above 1e37 (FP32 table range)");
    }
    topot_ktable* k = new (std::nothrow) topot_ktable;
    if (!k) return fail(TOPOT_ERR_OOM, "kernel_table_create: host allocation");
    k->K = K;
    k->a = s_min;
    k->h = (s_max - s_min) / (double)(K - 1);
    // FP32 layout of the evaluation kernels: K + 1 pairs, (y_0, 0), then per segment r
    // (y_r + d_r / 2, d_r) with d_r = y_{r+1} - y_r, then (y_{K-1}, 0)
    std::vector<float2> pairs((size_t)K + 1);
    pairs[0] = make_float2((float)h_values[0], 0.0f);
    for (int r = 0; r + 1 < K; ++r) {
        const double d = h_values[r + 1] - h_values[r];
        pairs[r + 1] = make_float2((float)(h_values[r] + 0.5 * d), (float)d);
    }
    pairs[K] = make_float2((float)h_values[K - 1], 0.0f);
    cudaError_t e = cudaGetDevice(&k->device);
    if (e == cudaSuccess) e = cudaMalloc(&k->d32, sizeof(float2) * ((size_t)K + 1));
    if (e == cudaSuccess) e = cudaMalloc(&k->d64, sizeof(double) * (size_t)K);
    if (e == cudaSuccess)
        e = cudaMemcpy(k->d32, pairs.data(), sizeof(float2) * ((size_t)K + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(k->d64, h_values, sizeof(double) * (size_t)K, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        kernel_table_free(k);
        return cuda_fail(e, "kernel_table_create");
    }
    *out = k;
    return TOPOT_OK;
}

void kernel_table_free(topot_ktable* k) {
    if (!k) return;
    if (k->d32) cudaFree(k->d32);
    if (k->d64) cudaFree(k->d64);
    delete k;
}

topot_status hybrid_transform_table(const topot_tables* t, const topot_ktable* k, topot_precision precision,
                                    const double* d_dirs, int D, int per_image_dirs, double* d_out, void* stream) {
    if (!k) return fail(TOPOT_ERR_INVALID_ARG, "hybrid_transform_table: kernel table is NULL");
    return ht_common("hybrid_transform_table", t, TOPOT_TABLE, precision, d_dirs, D, per_image_dirs, false, nullptr,
                     d_out, stream, k);
}

topot_status hybrid_transform_table_grad(const topot_tables* t, const topot_ktable* k, topot_precision precision,
                                         const double* d_dirs, int D, int per_image_dirs, const double* d_gout,
                                         double* d_gdirs, void* stream) {
    if (!k) return fail(TOPOT_ERR_INVALID_ARG, "hybrid_transform_table_grad: kernel table is NULL");
    return ht_common("hybrid_transform_table_grad", t, TOPOT_TABLE, precision, d_dirs, D, per_image_dirs, true,
                     d_gout, d_gdirs, stream, k);
}

}  // extern "C"

// ---- hybrid transform for callers that cannot allocate ---------------------------------------
//
// hybrid_transform() grows a workspace inside the tables handle with cudaMalloc when a
// call needs more than it has.  Code that runs where allocation is not allowed -- inside
// a custom memory pool or allocator callback, under an allocation-free real-time budget,
// or in a host that forbids cudaMalloc after start-up -- cannot use it.  This variant
// takes its scratch (work plan and per-item partial sums) from one fixed array of
// kNoAllocScratchBytes in device global memory that every GPU which loads the library
// holds until the process exits.  Its result is that of hybrid_transform().

#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB per device
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol name is only a
// host-side handle: the address is looked up once per device with that device current.
topot_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "hybrid_transform_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(TOPOT_ERR_UNSUPPORTED, "hybrid_transform_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "hybrid_transform_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return TOPOT_OK;
}

}  // namespace

extern "C" {

topot_status hybrid_transform_noalloc(const topot_tables* tc, topot_kernel kernel, topot_precision precision,
                                      const double* d_dirs, int D, int per_image_dirs, double* d_out,
                                      void* stream) {
    topot_tables* t = const_cast<topot_tables*>(tc);
    const char* name = "hybrid_transform_noalloc";
    if (!valid_dirs_args(t, d_dirs, D, per_image_dirs) || !d_out)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad handle, directions or output");
    if (kernel != TOPOT_LAPLACE && kernel != TOPOT_FOURIER && kernel != TOPOT_BESSEL && kernel != TOPOT_SINE)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad kernel");
    if (precision != TOPOT_FP32C && precision != TOPOT_FP64)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": bad precision");
    int dev = 0;
    TOPOT_CUDA(cudaGetDevice(&dev));
    if (dev != t->device)
        return fail(TOPOT_ERR_INVALID_ARG, std::string(name) + ": the handle's device must be current");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the tile and chunk choices of hybrid_transform (shared helper), hence its result
    const HtSizing z = ht_sizing(t, kernel, precision, D, per_image_dirs, false);
    if (z.need > kNoAllocScratchBytes)
        return fail(TOPOT_ERR_INVALID_ARG,
                    std::string(name) + ": this call needs " + std::to_string(z.need) +
                        " bytes of scratch, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
                        "; use fewer directions or images per call, or hybrid_transform");
    void* scratch = nullptr;
    topot_status s = noalloc_scratch(&scratch);
    if (s != TOPOT_OK) return s;
    double* part = nullptr;
    EvalPlan P = ht_carve(t, z, d_dirs, D, per_image_dirs, scratch, &part);
    const int dl = z.dl, tdh = z.tdh;

    TOPOT_CUDA(launch_dir_prep(P, t->n, st));
    TOPOT_CUDA(launch_plan(P, t->dev(), st));
    const int per_sm = t->tuning.ht_ctas_per_sm > 0 ? t->tuning.ht_ctas_per_sm : 4;
    TOPOT_CUDA(launch_ht(P, t->dev(), kernel, precision, false, dl, z.split, t->sm_count * per_sm, part, st));
    TOPOT_CUDA(launch_ht_combine(P, t->n, t->B, kernel, precision, tdh, part, t->slab ? t->vsum : nullptr, t->S,
                                 d_out, st));
    return TOPOT_OK;
}

}  // extern "C"

// ---- sums over slabs -----------------------------------------------------------------------

static int current_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 1;
    return std::max(sms, 1);
}

extern "C" {

topot_status slab_sum_i32(const int32_t* d_parts, int P, int64_t n, int32_t* d_out, uint32_t* d_overflow,
                          void* stream) {
    if (!d_parts || !d_out || !d_overflow || P < 1 || n < 0)
        return fail(TOPOT_ERR_INVALID_ARG, "slab_sum_i32: bad pointers or sizes");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    TOPOT_CUDA(cudaMemsetAsync(d_overflow, 0, sizeof(uint32_t), st));
    if (n == 0) return TOPOT_OK;
    TOPOT_CUDA(launch_slab_sum_i32(d_parts, P, n, d_out, d_overflow, current_sm_count(), st));
    return TOPOT_OK;
}

topot_status slab_sum_f64(const double* d_parts, int P, int64_t n, double* d_out, void* stream) {
    if (!d_parts || !d_out || P < 1 || n < 0) return fail(TOPOT_ERR_INVALID_ARG, "slab_sum_f64: bad pointers or sizes");
    if (n == 0) return TOPOT_OK;
    TOPOT_CUDA(launch_slab_sum_f64(d_parts, P, n, d_out, current_sm_count(), reinterpret_cast<cudaStream_t>(stream)));
    return TOPOT_OK;
}

}  // extern "C"

// ---- exact representations (Section 4.3; Appendix A.2 / A.3) ----------------------------

namespace topot {
cudaError_t launch_exact(int n, bool u8, ExactArgs a, long long max_n, int sm_count, cudaStream_t st);
int exact_radix_tile();
constexpr int kExactProdLimit = 12288;   // staged coordinate products (96 KB of shared memory)
size_t exact_keys_smem(int prod_max);
cudaError_t launch_ect_exact_eval(int nseg, long long cap, const double* T, const int32_t* E, const long long* len,
                                  const double* t, int Q, int32_t* out, int sm_count, cudaStream_t st);
cudaError_t launch_radon_exact_eval(int nseg, long long cap, const double* Tl, const int32_t* El,
                                    const long long* lenl, long long cap_o, const double* To, const int32_t* Eo,
                                    const long long* leno, const double* t, int Q, int32_t* out, int sm_count,
                                    cudaStream_t st);
}  // namespace topot

extern "C" {

topot_status exact_representation(const topot_tables* tc, int kind, const double* d_dirs, int D, int per_image_dirs,
                                  int64_t cap, double* d_T, int32_t* d_E, int64_t* d_len, void* stream) {
    topot_tables* t = const_cast<topot_tables*>(tc);
    if (!valid_dirs_args(t, d_dirs, D, per_image_dirs) || !d_T || !d_E || !d_len || (kind != 0 && kind != 1))
        return fail(TOPOT_ERR_INVALID_ARG, "exact_representation: bad handle, kind, directions or output");
    if (!t->host_valid) return fail(TOPOT_ERR_INVALID_ARG, "exact_representation: call tables_sync first");
    const long long nseg = (long long)t->B * D;
    if (cap < 1 || nseg > (1ll << 31) - 1 || cap > (1ll << 31) - 1)
        return fail(TOPOT_ERR_INVALID_ARG, "exact_representation: cap or B * D out of range");
    // the largest table the directions can select, and the int32 bound of the sums
    long long max_n = 0;
    for (int b = 0; b < t->B; ++b) {
        const long long* c = t->h_seg_count.data() + (size_t)b * t->S;
        const long long* a = t->h_absum.data() + (size_t)b * t->NO;
        for (int o = 0; o < t->NO; ++o) {
            const int r = (o & (t->NO >> 1)) ? (o ^ (t->NO - 1)) : o;
            max_n = std::max(max_n, kind == 0 ? c[o] : c[t->NO + r]);
            const long long bound = kind == 0 ? a[o] : a[o] + a[o ^ (t->NO - 1)];
            if (bound >= (1ll << 31))
                return fail(TOPOT_ERR_OVERFLOW, "exact_representation: sum |Delta^-| too large for int32 sums");
        }
    }
    if (max_n > cap)
        return fail(TOPOT_ERR_INVALID_ARG, "exact_representation: cap " + std::to_string(cap) +
                                               " < largest table " + std::to_string(max_n));
    const size_t slots = (size_t)nseg * (size_t)cap;
    // radix tiles per segment; with more than one, per-segment digit counts and look-back words
    const long long tile = exact_radix_tile();
    const long long tps = std::max(1ll, (max_n + tile - 1) / tile);
    if (nseg * tps > (1ll << 31) - 1)
        return fail(TOPOT_ERR_INVALID_ARG, "exact_representation: too many radix tiles");
    const size_t hist_n = tps > 1 ? (size_t)nseg * 8 * 256 : 0;
    const size_t status_n = tps > 1 ? (size_t)(nseg * tps) * 256 : 0;
    // per-direction coordinate products staged in shared memory when sum_k m_k fits
    int prod_max = 0;
    for (int b = 0; b < t->B; ++b) {
        int sm = 0;
        for (int k = 0; k < t->n; ++k) sm += t->h_img[b].m[k];
        if (sm <= kExactProdLimit) prod_max = std::max(prod_max, sm);
    }
    const size_t need = 2 * slots * (sizeof(unsigned long long) + sizeof(int)) + sizeof(int) * (size_t)nseg +
                        sizeof(unsigned) * hist_n + sizeof(unsigned long long) * status_n + 9 * 256;
    topot_status s = ensure_ws(t, kWsExact, need);
    if (s != TOPOT_OK) return s;
    Carver cv{reinterpret_cast<char*>(t->ws[kWsExact])};
    ExactArgs a{};
    a.t = t->dev();
    a.dirs = d_dirs;
    a.D = D;
    a.per_image = per_image_dirs;
    a.kind = kind;
    a.nseg = (int)nseg;
    a.cap = cap;
    a.key[0] = cv.take<unsigned long long>(slots);
    a.key[1] = cv.take<unsigned long long>(slots);
    a.val[0] = cv.take<int>(slots);
    a.val[1] = cv.take<int>(slots);
    a.cnt = cv.take<int>((size_t)nseg);
    a.tps = (int)tps;
    a.prod_max = prod_max;
    a.hist = hist_n ? cv.take<unsigned>(hist_n) : nullptr;
    a.status = status_n ? cv.take<unsigned long long>(status_n) : nullptr;
    a.tile_ctr = cv.take<int>(16);
    a.T = d_T;
    a.E = d_E;
    a.len = reinterpret_cast<long long*>(d_len);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    TOPOT_CUDA(cudaMemsetAsync(d_len, 0, sizeof(int64_t) * (size_t)nseg, st));
    TOPOT_CUDA(cudaMemsetAsync(a.tile_ctr, 0, sizeof(int) * 16, st));
    if (hist_n) TOPOT_CUDA(cudaMemsetAsync(a.hist, 0, sizeof(unsigned) * hist_n, st));
    if (status_n) TOPOT_CUDA(cudaMemsetAsync(a.status, 0, sizeof(unsigned long long) * status_n, st));
    TOPOT_CUDA(launch_exact(t->n, t->dtype == TOPOT_U8, a, max_n, t->sm_count, st));
    return TOPOT_OK;
}

topot_status ect_exact_eval(int nrep, int64_t cap, const double* d_T, const int32_t* d_E, const int64_t* d_len,
                            const double* d_t, int Q, int32_t* d_out, void* stream) {
    if (nrep < 1 || cap < 1 || Q < 1 || !d_T || !d_E || !d_len || !d_t || !d_out)
        return fail(TOPOT_ERR_INVALID_ARG, "ect_exact_eval: bad sizes or NULL pointer");
    int dev = 0, sms = 0;
    TOPOT_CUDA(cudaGetDevice(&dev));
    TOPOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TOPOT_CUDA(launch_ect_exact_eval(nrep, cap, d_T, d_E, reinterpret_cast<const long long*>(d_len), d_t, Q, d_out,
                                     sms, reinterpret_cast<cudaStream_t>(stream)));
    return TOPOT_OK;
}

topot_status radon_exact_eval(int nrep, int64_t cap, const double* d_T, const int32_t* d_E, const int64_t* d_len,
                              int64_t cap_ord, const double* d_Tord, const int32_t* d_Eord, const int64_t* d_len_ord,
                              const double* d_t, int Q, int32_t* d_out, void* stream) {
    if (nrep < 1 || cap < 1 || cap_ord < 1 || Q < 1 || !d_T || !d_E || !d_len || !d_Tord || !d_Eord || !d_len_ord || !d_t ||
        !d_out)
        return fail(TOPOT_ERR_INVALID_ARG, "radon_exact_eval: bad sizes or NULL pointer");
    int dev = 0, sms = 0;
    TOPOT_CUDA(cudaGetDevice(&dev));
    TOPOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TOPOT_CUDA(launch_radon_exact_eval(nrep, cap, d_T, d_E, reinterpret_cast<const long long*>(d_len), cap_ord,
                                       d_Tord, d_Eord, reinterpret_cast<const long long*>(d_len_ord), d_t, Q, d_out,
                                       sms, reinterpret_cast<cudaStream_t>(stream)));
    return TOPOT_OK;
}

}  // extern "C"

// ---- self-test of the bounded waits -------------------------------------------------------

extern "C" {

topot_status topot_selftest_wait(int which, int limit_ms, void* stream) {
    if ((which != 0 && which != 1) || limit_ms < 1 || limit_ms > 10000)
        return fail(TOPOT_ERR_INVALID_ARG, "topot_selftest_wait: which must be 0 or 1, limit_ms in [1, 10000]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void* mem = nullptr;
    TOPOT_CUDA(cudaMalloc(&mem, 256));
    unsigned long long* flag = reinterpret_cast<unsigned long long*>(mem);
    unsigned* err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(mem) + 128);
    cudaError_t e = cudaMemsetAsync(mem, 0, 256, st);
    if (e == cudaSuccess) e = launch_selftest_wait(which, (unsigned long long)limit_ms * 1000000ull, flag, err, st);
    unsigned h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(e, "topot_selftest_wait");
    if (h_err & kDevErrTimeout) return fail(TOPOT_ERR_TIMEOUT, "device-side wait timed out (self-test)");
    return TOPOT_OK;
}

}  // extern "C"
