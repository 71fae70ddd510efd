// K1 for binary 8-bit volumes (Section 3, Delta^-; Section 4.2, preprocessing): volumes
// whose voxels are all 0 or 1, vertex construction, whole volumes.
//
// A cell's value is the minimum of its vertices, which for 0/1 voxels is their AND, so
// 32 voxels of a row are handled at once as the bits of a word.  For orthant o let
// d_k = +1 if bit k of o is set (eps_k = -1), else -1; the lower star of v is the box
// v + g d, g in {0,1}^3, and with the box's bits t0 = b(v), x = b(v + d_x e_x), ...,
// xyz = b(v + d):
//   Delta^-_o(v) = t0 (1 - n1 + F - c),   n1 = x + y + z,
//   F = x y xy + x z xz + y z yz (the faces),  c = x y z xy xz yz xyz (the cube),
// a value in {-2, -1, 0, 1} (a face needs two edges, the cube all three faces).  It is
// kept as two bit planes, the 2-bit two's complement (v1, v0):
//   v0 = t0 & ~(s0 ^ F0 ^ c)                        (parity of 1 + n1 + F + c)
//   v1 = t0 & s1 & (s0 ? ~F1 : ~F0)                 (n1 = 2 with no face, n1 = 3 with <= 1)
// where s1 s0 = n1 and F1 F0 = F are bit-sliced sums.  Delta_r = Delta^-_r - Delta^-_{r^7}
// is non-zero where the two codes differ.
//
// Pipeline (one stream): pack the voxels to bits and flag volumes with a voxel above 1;
// count the non-zero values per unit (one warp: 32 consecutive words of a volume, in
// vertex order) and segment; scan the counts per volume (chunk totals, then offsets);
// write the entries at their offsets.  Volumes that are not binary keep the general 8-bit
// kernel, which skips the binary ones.
#include <algorithm>

#include "internal.cuh"

namespace topot {

namespace {

constexpr unsigned kFullB = 0xffffffffu;
constexpr int kSegB = 12;             // 8 lower tables + 4 Delta tables
constexpr int kWordsB = kSegB / 2;    // counts per unit: two 16-bit fields per word
constexpr int kUnitWarps = 8;         // units per block of the count and write passes
constexpr int kBChunk = 1024;         // units per scan chunk (threads of the scan block)

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }

// Padded word index of voxel word (z, y, xw).
__device__ __forceinline__ long long pk_index(const BinImg& I, int z, int y, int xw) {
    return I.pk_off + ((long long)(z + 1) * (I.m1 + 2) + (y + 1)) * (I.wpr + 2) + (xw + 1);
}

// Codes (v1, v0) of the 8 orthants for the 32 voxels of the word at padded index c.
__device__ __forceinline__ void word_codes(const uint32_t* __restrict__ pk, const BinImg& I, long long c,
                                           uint32_t (&v1)[8], uint32_t (&v0)[8]) {
    const long long sy = I.wpr + 2, sz = (long long)(I.m1 + 2) * sy;
    // R[dz][dy][s]: row (z + dz - 1, y + dy - 1), bits of voxel x (s = 0), x + 1 (s = 1), x - 1 (s = 2)
    uint32_t R[3][3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const uint32_t* q = pk + c + (dz - 1) * sz + (dy - 1) * sy;
            const uint32_t w = __ldg(q), wp = __ldg(q - 1), wn = __ldg(q + 1);
            R[dz][dy][0] = w;
            R[dz][dy][1] = __funnelshift_r(w, wn, 1);   // bit i: voxel x_i + 1
            R[dz][dy][2] = __funnelshift_l(wp, w, 1);   // bit i: voxel x_i - 1
        }
    const uint32_t t0 = R[1][1][0];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int sx = (o & 1) ? 1 : 2;          // x shift toward d_x
        const int ry = (o & 2) ? 2 : 0;          // row y + d_y
        const int rz = (o & 4) ? 2 : 0;          // plane z + d_z
        const uint32_t x = R[1][1][sx], y = R[1][ry][0], z = R[rz][1][0];
        const uint32_t xy = R[1][ry][sx], xz = R[rz][1][sx], yz = R[rz][ry][0], xyz = R[rz][ry][sx];
        const uint32_t s0 = x ^ y ^ z, s1 = maj3(x, y, z);
        const uint32_t fxy = x & y & xy, fxz = x & z & xz, fyz = y & z & yz;
        const uint32_t F0 = fxy ^ fxz ^ fyz, F1 = maj3(fxy, fxz, fyz);
        const uint32_t c3 = F0 & F1 & xyz;
        v1[o] = t0 & s1 & ((s0 & ~F1) | (~s0 & ~F0));
        v0[o] = t0 & ~(s0 ^ F0 ^ c3);
    }
}

// Non-zero mask of segment s (0..7 lower tables, 8..11 Delta tables).
__device__ __forceinline__ uint32_t seg_mask(const uint32_t (&v1)[8], const uint32_t (&v0)[8], int s) {
    if (s < 8) return v1[s] | v0[s];
    const int r = s - 8;
    return (v1[r] ^ v1[r ^ 7]) | (v0[r] ^ v0[r ^ 7]);
}

__device__ __forceinline__ int code_at(uint32_t v1, uint32_t v0, int i) {
    return (int)((v0 >> i) & 1u) - 2 * (int)((v1 >> i) & 1u);
}

}  // namespace

// ---- pack: one thread per voxel word ------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin_pack(BinArgs a) {
    const int b = blockIdx.y;
    const BinImg I = a.img[b];
    const int nw = I.m2 * I.m1 * I.wpr;   // < 2^31: fewer words than vertices
    const uint8_t* src0 = reinterpret_cast<const uint8_t*>(a.pixels) + I.pix_off;
    unsigned bad = 0;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const int row = (int)fastdiv((uint32_t)w, I.div_wpr);
        const int xw = w - row * I.wpr;
        const int z = (int)fastdiv((uint32_t)row, I.div_m1);
        const int y = row - z * I.m1;
        const int x0 = 32 * xw;
        const uint8_t* src = src0 + (long long)row * I.m0 + x0;
        uint32_t bits = 0;
        if (x0 + 32 <= I.m0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const uint4 q0 = *reinterpret_cast<const uint4*>(src);
            const uint4 q1 = *reinterpret_cast<const uint4*>(src + 16);
            const uint32_t q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                bad |= q[k] & 0xFEFEFEFEu;
                // bytes b0..b3 in {0, 1}: byte 3 of q * 0x01020408 is b0 | b1 << 1 | b2 << 2 | b3 << 3
                // (no byte of the product exceeds 15, so no carry reaches byte 3)
                bits |= ((q[k] * 0x01020408u) >> 24) << (4 * k);
            }
        } else {
            const int nx = min(32, I.m0 - x0);
            for (int k = 0; k < nx; ++k) {
                const uint32_t v = src[k];
                bad |= v & 0xFEu;
                bits |= (v & 1u) << k;
            }
        }
        a.packed[pk_index(I, z, y, xw)] = bits;
    }
    if (__any_sync(kFullB, bad != 0u) && (threadIdx.x & 31) == 0) {
        atomicOr(&a.nonbin[b], 1u);
        atomicOr(&a.nonbin[a.t.B], 1u);
    }
}

// ---- count (WRITE = false) and write (WRITE = true) passes: one unit per warp -------------
template <bool WRITE>
__global__ void __launch_bounds__(32 * kUnitWarps) k_bin_extract(BinArgs a) {
    __shared__ long long bsum[9];
    const int2 bl = __ldg(&a.blocks[blockIdx.x]);   // (volume, first unit of the block)
    const int b = bl.x;
    if (__ldg(&a.nonbin[b]) != 0u) return;   // block-uniform: the general kernel takes this volume
    const BinImg I = a.img[b];
    const int lane = threadIdx.x & 31;
    const int lu = bl.y + (int)(threadIdx.x >> 5);
    const bool unit_ok = lu < I.nunits;      // warp-uniform: a volume's last block may overhang
    const long long u = I.unit_begin + lu;
    if (!WRITE) {
        if (threadIdx.x < 9) bsum[threadIdx.x] = 0;
        __syncthreads();
    }
    const int nw = I.m2 * I.m1 * I.wpr;
    const int w = unit_ok ? 32 * lu + lane : nw;
    uint32_t v1[8], v0[8];
    int z = 0, y = 0, xw = 0;
    if (w < nw) {
        const int row = (int)fastdiv((uint32_t)w, I.div_wpr);
        xw = w - row * I.wpr;
        z = (int)fastdiv((uint32_t)row, I.div_m1);
        y = row - z * I.m1;
        word_codes(a.packed, I, pk_index(I, z, y, xw), v1, v0);
    } else {
#pragma unroll
        for (int o = 0; o < 8; ++o) v1[o] = v0[o] = 0u;
    }
    // per lane counts, two segments per word
    uint32_t cw[kWordsB];
#pragma unroll
    for (int i = 0; i < kWordsB; ++i)
        cw[i] = (uint32_t)__popc(seg_mask(v1, v0, 2 * i)) | ((uint32_t)__popc(seg_mask(v1, v0, 2 * i + 1)) << 16);
    if constexpr (!WRITE) {
        uint32_t mine = 0;
#pragma unroll
        for (int i = 0; i < kWordsB; ++i) {
            const uint32_t t = __reduce_add_sync(kFullB, cw[i]);
            if (lane == i) mine = t;
        }
        if (unit_ok && lane < kWordsB) a.ucount[u * kWordsB + lane] = mine;
        // chi = sum Delta^-_0 and sum |Delta^-_o| (|v| = v0 + 2 v1 ~v0 per voxel)
        int sums[9];
#pragma unroll
        for (int o = 0; o < 8; ++o) sums[o] = __popc(v0[o]) + 2 * __popc(v1[o] & ~v0[o]);
        sums[8] = __popc(v0[0]) - 2 * __popc(v1[0]);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int t = (int)__reduce_add_sync(kFullB, (unsigned)sums[i]);
            if (lane == 0 && t != 0)
                atomicAdd(reinterpret_cast<unsigned long long*>(&bsum[i]), (unsigned long long)(long long)t);
        }
        __syncthreads();
        if (threadIdx.x < 9 && bsum[threadIdx.x] != 0) {
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(
                threadIdx.x == 8 ? &a.t.chi[b] : &a.t.absum[(long long)b * 8 + threadIdx.x]);
            atomicAdd(dst, (unsigned long long)bsum[threadIdx.x]);
        }
    } else {
        if (!unit_ok) return;
        uint32_t ex[kWordsB];
#pragma unroll
        for (int i = 0; i < kWordsB; ++i) {
            uint32_t x = cw[i];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(kFullB, x, d);
                if (lane >= d) x += t;
            }
            ex[i] = x - cw[i];
        }
        const int uo = lane < kSegB ? __ldg(&a.uoff[u * kSegB + lane]) : 0;
        const int base_idx = (int)(((long long)z * I.m1 + y) * I.m0 + 32 * xw);
        int* const aidx = a.t.arena_idx;
        int16_t* const aval = reinterpret_cast<int16_t*>(a.t.arena_val);
#pragma unroll
        for (int s = 0; s < kSegB; ++s) {
            uint32_t m = seg_mask(v1, v0, s);
            const int us = __shfl_sync(kFullB, uo, s);
            if (!__any_sync(kFullB, m != 0u)) continue;
            const long long rel = (long long)us + ((ex[s >> 1] >> (16 * (s & 1))) & 0xffffu);
            if (us < 0 || rel + __popc(m) > I.N) {   // both passes count alike, so never
                dev_set_error(a.t.err, kDevErrOverflow);
                m = 0u;
            }
            long long pos = I.seg_base + (long long)s * I.N + rel;
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1u;
                const int v = s < 8 ? code_at(v1[s], v0[s], i)
                                    : code_at(v1[s - 8], v0[s - 8], i) - code_at(v1[(s - 8) ^ 7], v0[(s - 8) ^ 7], i);
                aidx[pos] = base_idx + i;
                aval[pos] = (int16_t)v;
                ++pos;
            }
        }
    }
}

// ---- scan of the unit counts per volume ---------------------------------------------------

// Per chunk: the totals of each segment.
__global__ void __launch_bounds__(kBChunk) k_bin_chunk_sum(BinArgs a) {
    const int2 cb = __ldg(&a.chunks[blockIdx.x]);
    if (__ldg(&a.nonbin[cb.x]) != 0u) return;   // block-uniform
    const BinImg& I = a.img[cb.x];
    __shared__ uint32_t tot[kSegB];
    if (threadIdx.x < kSegB) tot[threadIdx.x] = 0;
    __syncthreads();
    const int lu = cb.y * kBChunk + threadIdx.x;
    uint32_t c[kSegB];
#pragma unroll
    for (int i = 0; i < kWordsB; ++i) {
        const uint32_t x = lu < I.nunits ? __ldg(&a.ucount[(I.unit_begin + lu) * kWordsB + i]) : 0u;
        c[2 * i] = x & 0xffffu;
        c[2 * i + 1] = x >> 16;
    }
#pragma unroll
    for (int s = 0; s < kSegB; ++s) {
        const uint32_t t = __reduce_add_sync(kFullB, c[s]);
        if ((threadIdx.x & 31) == 0 && t != 0u) atomicAdd(&tot[s], t);
    }
    __syncthreads();
    if (threadIdx.x < kSegB) a.csum[(long long)blockIdx.x * kSegB + threadIdx.x] = (int)tot[threadIdx.x];
}

// Per chunk: unit offsets = (earlier chunks of the volume) + (earlier units of the chunk);
// the last chunk of a volume writes the table sizes.
__global__ void __launch_bounds__(kBChunk) k_bin_scan(BinArgs a) {
    constexpr int NWS = kBChunk / 32;
    const int2 cb = __ldg(&a.chunks[blockIdx.x]);
    if (__ldg(&a.nonbin[cb.x]) != 0u) return;   // block-uniform
    const BinImg& I = a.img[cb.x];
    __shared__ uint32_t pre[kSegB];
    __shared__ uint32_t wtot[NWS][kSegB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kSegB) pre[tid] = 0;
    __syncthreads();
    for (int q = tid; q < cb.y * kSegB; q += kBChunk)
        atomicAdd(&pre[q % kSegB],
                  (uint32_t)__ldg(&a.csum[((long long)blockIdx.x - cb.y + q / kSegB) * kSegB + q % kSegB]));
    const int lu = cb.y * kBChunk + tid;
    uint32_t c[kSegB], inc[kSegB];
#pragma unroll
    for (int i = 0; i < kWordsB; ++i) {
        const uint32_t x = lu < I.nunits ? __ldg(&a.ucount[(I.unit_begin + lu) * kWordsB + i]) : 0u;
        c[2 * i] = x & 0xffffu;
        c[2 * i + 1] = x >> 16;
    }
#pragma unroll
    for (int s = 0; s < kSegB; ++s) {
        uint32_t x = c[s];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(kFullB, x, d);
            if (lane >= d) x += t;
        }
        inc[s] = x;
    }
    if (lane == 31) {
#pragma unroll
        for (int s = 0; s < kSegB; ++s) wtot[warp][s] = inc[s];
    }
    __syncthreads();
    if (warp == 0) {   // exclusive scan of the warp totals, in place
#pragma unroll
        for (int s = 0; s < kSegB; ++s) {
            const uint32_t v = wtot[lane][s];
            uint32_t x = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(kFullB, x, d);
                if (lane >= d) x += t;
            }
            wtot[lane][s] = x - v;
        }
    }
    __syncthreads();
    uint32_t o[kSegB];
#pragma unroll
    for (int s = 0; s < kSegB; ++s) o[s] = pre[s] + wtot[warp][s] + inc[s] - c[s];
    if (lu < I.nunits) {
#pragma unroll
        for (int s = 0; s < kSegB; ++s) a.uoff[(I.unit_begin + lu) * kSegB + s] = (int)o[s];
    }
    if (tid == kBChunk - 1 && (cb.y + 1) * kBChunk >= I.nunits) {
#pragma unroll
        for (int s = 0; s < kSegB; ++s) a.t.seg_count[(long long)cb.x * kSegB + s] = (long long)(o[s] + c[s]);
    }
}

// ---- host side ----------------------------------------------------------------------------

int bin_unit_warps() { return kUnitWarps; }
int bin_chunk() { return kBChunk; }

cudaError_t launch_bin_pack(const BinArgs& a, int B, int pack_blocks_per_image, cudaStream_t st) {
    k_bin_pack<<<dim3((unsigned)pack_blocks_per_image, (unsigned)B), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bin_tables(const BinArgs& a, cudaStream_t st) {
    cudaError_t e;
    k_bin_extract<false><<<(unsigned)a.nblocks, 32 * kUnitWarps, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bin_chunk_sum<<<(unsigned)a.nchunks, kBChunk, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bin_scan<<<(unsigned)a.nchunks, kBChunk, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_bin_extract<true><<<(unsigned)a.nblocks, 32 * kUnitWarps, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace topot
