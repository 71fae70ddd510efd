// Slabs of a volume (the paper's parallelisation over vertex subsets, Section 5.3).
//
// A slab handle holds the tables of the vertices of planes [z0, z1) of a volume.  Every
// transform is a sum over vertices (Lemma 3.1: ECT and Radon are sums of Delta^- over
// sublevel / superlevel sets, the hybrid transform a sum of Delta kbar), so the
// transforms of the slabs of a partition add up to the transform of the volume.  This
// file holds the two device pieces that the split needs beyond the extraction:
//   k_segment_sums  the sum of the values of every table of a slab handle (a slab's
//                   Delta tables need not sum to zero, and the FP32C hybrid kernels leave
//                   the constant kbar(0) out);
//   k_slab_sum_*    the sum of P slabs' results, in slab order: exact for the int32
//                   grids (int64 accumulation, range checked), Neumaier-compensated FP64
//                   for the hybrid transforms, so the result does not depend on which
//                   device or rank computed which slab.
#include <algorithm>

#include "internal.cuh"

namespace topot {

// One block per (image, table): sum of the table's values.
template <typename Tval>
__global__ void __launch_bounds__(256) k_segment_sums(TablesDev t, long long* vsum) {
    __shared__ long long red[8];
    const int b = blockIdx.x / t.S, seg = blockIdx.x - b * t.S;
    const ImgDesc& I = t.img[b];
    const long long n = t.seg_count[(long long)b * t.S + seg];
    const Tval* v = reinterpret_cast<const Tval*>(t.arena_val) + I.seg_base + (long long)seg * I.N;
    long long acc = 0;
    for (long long i = threadIdx.x; i < n; i += 256) acc += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < 8; ++w) s += red[w];
        vsum[blockIdx.x] = s;
    }
}

cudaError_t launch_segment_sums(const TablesDev& t, long long* vsum, cudaStream_t st) {
    const unsigned grid = (unsigned)(t.B * t.S);
    if (t.val_bytes == 2) k_segment_sums<int16_t><<<grid, 256, 0, st>>>(t, vsum);
    else k_segment_sums<int32_t><<<grid, 256, 0, st>>>(t, vsum);
    return cudaGetLastError();
}

// out[i] = sum_p parts[p][i] (p = 0 .. P-1 in order), int64 accumulation; an element out
// of the int32 range sets *err.
__global__ void k_slab_sum_i32(const int32_t* parts, int P, long long n, int32_t* out, unsigned* err) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long s = 0;
        for (int p = 0; p < P; ++p) s += parts[(long long)p * n + i];
        if (s > 2147483647ll || s < -2147483648ll) {
            atomicOr(err, 1u);
            s = 0;
        }
        out[i] = (int32_t)s;
    }
}

// out[i] = sum_p parts[p][i] in slab order with Neumaier's compensation (the running sum
// and the lost low parts; Neumaier 1974, improved Kahan-Babuska summation).
__global__ void k_slab_sum_f64(const double* parts, int P, long long n, double* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = 0.0, c = 0.0;
        for (int p = 0; p < P; ++p) {
            const double x = parts[(long long)p * n + i];
            const double t = s + x;
            c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
            s = t;
        }
        out[i] = s + c;
    }
}

cudaError_t launch_slab_sum_i32(const int32_t* parts, int P, long long n, int32_t* out, unsigned* err, int sm_count,
                                cudaStream_t st) {
    const long long blocks = std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
    k_slab_sum_i32<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(parts, P, n, out, err);
    return cudaGetLastError();
}

cudaError_t launch_slab_sum_f64(const double* parts, int P, long long n, double* out, int sm_count,
                                cudaStream_t st) {
    const long long blocks = std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
    k_slab_sum_f64<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, st>>>(parts, P, n, out);
    return cudaGetLastError();
}

}  // namespace topot
