// K2 / K3: ECT and Radon transform on a grid of directions x thresholds.
//
// ECT(xi, t_j) = sum_{v : s_v <= t_j} Delta^-_{eps(xi)}(v)       (Lemma 3.1; Appendix A.4)
// R(xi, t_j)   = sum_{s_v <= t_j} Delta^-_o + sum_{s_v >= t_j} Delta^-_{o^(2^n-1)} - chi
//                                                      (additivity of the Euler integral)
// with s_v = <xi, x(v)>.  Each critical point is binned once per direction:
//   sublevel bin   j(v) = min{j : s_v <= t_j}   (T when none)
//   superlevel bin j(v) = max{j : t_j <= s_v}   (-1 when none)
// and its value is added to a shared-memory histogram; an exact integer prefix
// (suffix) sum over the bins gives the transform.
//
// Exactness of the bin: the FP32 estimate u = (s - a) / h of the bin coordinate,
// computed from the lattice form s = sum_k xi_k c_k / (2 (m_k - 1)), c_k = 2 i_k - (m_k - 1),
// is within delta of the exact value of the FP64 s_v; when u is farther than delta
// from every integer, ceil(u) (floor(u)) is the bin the FP64 comparison gives.
// Otherwise the lane recomputes s_v and compares with t_j exactly as the FP64
// expressions do (__ddiv_rn / __dmul_rn / __dadd_rn, no contraction).
//
// Work split: one persistent grid walks the work items of the plan (pair, tile of
// TD directions, chunk of the table).  A warp evaluates one critical point for TD
// directions at once (lane = direction; with TD < 32, 32/TD groups of lanes take
// critical points far apart in the chunk so that equal bins rarely collide).  The
// chunk is staged in shared memory as decoded lattice coordinates.  Histograms are
// merged into the output with integer atomics: the result is exact and does not
// depend on the order.
#include <type_traits>

#include "eval_common.cuh"

namespace topot {

constexpr int kHistBlock = 512;
constexpr int kHistSub = 1024;   // staged critical points per round

struct DirCoef {
    float a0, a1, a2, beta, delta;
};

__device__ __forceinline__ DirCoef make_coef(const double* xi, int n, const int* m, double t_min,
                                             double t_max, int T) {
    const double h = (t_max - t_min) / (double)(T - 1);
    double A[3] = {0.0, 0.0, 0.0};
    double Mu = 0.0;
    for (int k = 0; k < n; ++k) {
        A[k] = xi[k] / (2.0 * (double)(m[k] - 1) * h);
        Mu += fabs(A[k]) * (double)(m[k] - 1);
    }
    const double beta = -t_min / h;
    Mu += fabs(beta);
    DirCoef c;
    c.a0 = (float)A[0];
    c.a1 = (float)A[1];
    c.a2 = (float)A[2];
    c.beta = (float)beta;
    // rounding of the coefficients and of the n FMAs: <= 4 * 2^-24 * Mu; FP64 errors of
    // s, t_j and the coefficients: far below 1e-12 (Mu + T + 1)
    const double d = ldexp(Mu, -22) + 1e-12 * (Mu + (double)T + 1.0);
    c.delta = (Mu < 4194304.0) ? (float)(d * (1.0 + 1e-6)) : __int_as_float(0x7f800000);
    return c;
}

// Exact bin of one critical point (rare path).
template <int NDIM, bool MAXBIN>
__device__ __noinline__ int exact_bin(float c0, float c1, float c2, const double* xi, const int* m,
                                      const double* thr, int T, float u) {
    const float cc[3] = {c0, c1, c2};
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        const double xk = __ddiv_rn((double)cc[k], (double)(2 * (m[k] - 1)));
        const double pk = __dmul_rn(xi[k], xk);
        s = (k == 0) ? pk : __dadd_rn(s, pk);
    }
    float uc = fminf(fmaxf(u, -2.0f), (float)T + 1.0f);
    if (uc != uc) uc = 0.0f;
    int j = (int)rintf(uc);
    if (!MAXBIN) {   // min{j : s <= t_j}, T if none
        j = min(max(j, 0), T);
        while (j > 0 && s <= thr[j - 1]) --j;
        while (j < T && s > thr[j]) ++j;
        return j;
    } else {         // max{j : t_j <= s}, -1 if none; stored shifted by one
        j = min(max(j, -1), T - 1);
        while (j >= 0 && thr[j] > s) --j;
        while (j + 1 < T && thr[j + 1] <= s) ++j;
        return j + 1;
    }
}

template <int NDIM, int TD, int DPL, typename Tval>
__global__ void __launch_bounds__(kHistBlock, DPL == 1 ? 2 : 1) k_hist(EvalPlan P, TablesDev t, int32_t* out_lo,
                                                                     int32_t* out_hi) {
    // TD directions share a warp (lane = direction for TD = 32; 32/TD point groups
    // otherwise); with DPL = 2 every lane bins two directions (64 per warp), which halves
    // the per-update instruction overhead at the cost of a twice larger histogram.
    constexpr int NW = kHistBlock / 32;
    constexpr int G = 32 / TD;
    constexpr int NO = 1 << NDIM;
    constexpr int TDT = TD * DPL;                           // directions per work item
    static_assert(DPL == 1 || TD == 32, "two directions per lane only with 32 per warp");
    extern __shared__ float4 stage[];                       // [kHistSub]
    int* hist = reinterpret_cast<int*>(stage + kHistSub);   // [T + 1][TDT]
    __shared__ long long sh_item;
    __shared__ int sh_dir[TDT];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = P.T;
    const int HS = T + 1;
    const int dl = lane % TD, g = lane / TD;
    const long long nitems = P.ctl[2];
    const int chunk = P.ctl[1];
    const Tval* aval = reinterpret_cast<const Tval*>(t.arena_val);

    while (true) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(&P.ctl[0], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item >= nitems) break;
        int pair, tile, ch;
        decode_item(P, item, pair, tile, ch);
        int b, o, part, sign;
        decode_pair(P.mode, NO, pair, b, o, part);
        const int seg = pair_segment(P.mode, NO, o, part, sign);
        const bool maxbin = part == 1;
        const ImgDesc& I = t.img[b];
        const int set = P.nsets == 1 ? 0 : b;
        const int* bo = P.boff + (long long)set * (NO + 1);
        const int nd = bo[o + 1] - bo[o];
        double xi[DPL][3];
        DirCoef cf[DPL];
        int* row[DPL];
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            const int r = tile * TDT + j * TD + dl;
            const bool dvalid = r < nd;
            const int d = dvalid ? P.perm[(long long)set * P.D + bo[o] + r] : 0;
            if (g == 0 && warp == 0) sh_dir[j * TD + dl] = dvalid ? d : -1;
            const double* xp = P.dirs + ((long long)set * P.D + d) * NDIM;
#pragma unroll
            for (int k = 0; k < 3; ++k) xi[j][k] = k < NDIM ? xp[k] : 0.0;
            cf[j] = make_coef(xi[j], NDIM, I.m, P.t_min, P.t_max, T);
            // bin-major histogram [T + 1][TDT]: the 32 lanes of a warp update 32 different
            // columns, so a lane's bank is fixed by its direction and the shared atomics of
            // one instruction do not conflict (TD = 32); lanes of directions past the tile
            // end bin into columns nobody reads
            row[j] = hist + (j * TD + dl);
        }

        // u = (s - t_min) / h of every point lies in beta +- sum_k |A_k| (m_k - 1); when that
        // range is inside [-0.25, T - 0.75] for every direction of the block, the clamp of u
        // before the rounding can be left out (block-uniform choice)
        int inside = 1;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            const float S = fabsf(cf[j].a0) * (float)(I.m[0] - 1) + fabsf(cf[j].a1) * (float)(I.m[1] - 1) +
                            fabsf(cf[j].a2) * (float)(I.m[2] - 1);
            inside &= (cf[j].beta - S >= -0.25f) && (cf[j].beta + S <= (float)T - 0.75f);
        }
        const bool clamp = !__syncthreads_and(inside);

        for (int i = tid; i < TDT * HS; i += kHistBlock) hist[i] = 0;

        const long long N = t.seg_count[(long long)b * t.S + seg];
        const long long base = I.seg_base + (long long)seg * I.N;
        const long long e_begin = (long long)ch * chunk;
        const long long e_end = min(N, e_begin + chunk);

        // Staging is software-pipelined: the raw entries of the next round are loaded
        // into registers while the current round is binned.
        constexpr int PF = kHistSub / kHistBlock;     // entries per thread per round
        uint32_t pidx[PF];
        int pval[PF];
        auto prefetch = [&](long long e0) {
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const long long e = e0 + tid + k * kHistBlock;
                pidx[k] = e < e_end ? (uint32_t)t.arena_idx[base + e] : 0u;
                pval[k] = e < e_end ? (int)aval[base + e] : 0;
            }
        };
        prefetch(e_begin);
        for (long long e0 = e_begin; e0 < e_end; e0 += kHistSub) {
            const int cnt = (int)min((long long)kHistSub, e_end - e0);
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int i = tid + k * kHistBlock;
                const uint32_t idx = pidx[k];
                const uint32_t q1 = fastdiv(idx, I.div0);
                const int i0 = (int)(idx - q1 * (uint32_t)I.m[0]);
                int i1 = (int)q1, i2 = 0;
                if (NDIM == 3) {
                    const uint32_t q2 = fastdiv(q1, I.div1);
                    i1 = (int)(q1 - q2 * (uint32_t)I.m[1]);
                    i2 = (int)q2;
                }
                // entries past the chunk end carry value 0 and add nothing
                stage[i] = make_float4((float)(2 * i0 - (I.m[0] - 1)), (float)(2 * i1 - (I.m[1] - 1)),
                                       (float)(2 * i2 - (I.m[2] - 1)), __int_as_float(pval[k]));
            }
            __syncthreads();
            if (e0 + kHistSub < e_end) prefetch(e0 + kHistSub);
            {
                // rounds are padded with zero-value entries to a multiple of 4 per warp group
                const int cnt4 = (cnt + 3) & ~3;
                const int per = (((cnt4 + NW - 1) / NW) + 3) & ~3;
                const int ws = warp * per;
                const int we = min(cnt4, ws + per);
                const int len = max(0, we - ws);
                const int gl = (((len + G - 1) / G) + 3) & ~3;
                const int gs = ws + g * gl;
                const int ge = min(we, gs + gl);
                const float umax = (float)T - 0.5f;
                // Bin from u without float->int conversions: adding 1.5 * 2^23 rounds u to
                // an integer r (ties to even) held in the low mantissa bits.  u is clamped to
                // [-0.5, T - 0.5] first (unless no point can leave that range), so the
                // sublevel bin ceil(u) and the superlevel index floor(u) + 1 both land in
                // [0, T].  Points within delta of a bin edge are binned exactly on a slow
                // path, checked once per 4 points.  The clamp and the bin side are
                // compile-time choices of the loop, taken per work item (block-uniform).
                auto bin_round = [&](auto cl, auto mb) {
                    constexpr bool CL = decltype(cl)::value;
                    constexpr bool MB = decltype(mb)::value;
                    for (int e = gs; e < ge; e += 4) {
                        bool amb[4][DPL];
                        bool any = false;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float4 q = stage[e + k];
#pragma unroll
                            for (int j = 0; j < DPL; ++j) {
                                float u;
                                if (NDIM == 3)
                                    u = fmaf(q.x, cf[j].a0, fmaf(q.y, cf[j].a1, fmaf(q.z, cf[j].a2, cf[j].beta)));
                                else
                                    u = fmaf(q.x, cf[j].a0, fmaf(q.y, cf[j].a1, cf[j].beta));
                                const float uc = CL ? fminf(fmaxf(u, -0.5f), umax) : u;
                                const float f = uc + 12582912.0f;
                                const float rf = f - 12582912.0f;
                                const int r = __float_as_int(f) - 0x4B400000;
                                const int bin = MB ? (uc < rf ? r : r + 1) : (uc > rf ? r + 1 : r);
                                amb[k][j] = !(fabsf(u - rf) >= cf[j].delta);
                                any |= amb[k][j];
                                if (!amb[k][j]) atomicAdd(&row[j][bin * TDT], __float_as_int(q.w));
                            }
                        }
                        // rare: exact FP64 binning.  A per-lane branch: lane groups of one warp
                        // may run different trip counts, so no warp-wide vote may be used here.
                        if (any) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
#pragma unroll
                                for (int j = 0; j < DPL; ++j) {
                                    if (amb[k][j]) {
                                        const float4 q = stage[e + k];
                                        float u;
                                        if (NDIM == 3)
                                            u = fmaf(q.x, cf[j].a0,
                                                     fmaf(q.y, cf[j].a1, fmaf(q.z, cf[j].a2, cf[j].beta)));
                                        else
                                            u = fmaf(q.x, cf[j].a0, fmaf(q.y, cf[j].a1, cf[j].beta));
                                        const int bin = exact_bin<NDIM, MB>(q.x, q.y, q.z, xi[j], I.m, P.thr, T, u);
                                        atomicAdd(&row[j][bin * TDT], __float_as_int(q.w));
                                    }
                                }
                            }
                        }
                    }
                };
                using T1 = std::true_type;
                using F0 = std::false_type;
                if (clamp) {
                    if (maxbin) bin_round(T1{}, T1{}); else bin_round(T1{}, F0{});
                } else {
                    if (maxbin) bin_round(F0{}, T1{}); else bin_round(F0{}, F0{});
                }
            }
        }
        __syncthreads();
        int32_t* out = maxbin ? out_hi : out_lo;
        const int off = maxbin ? 1 : 0;
        for (int i = tid; i < TDT * T; i += kHistBlock) {
            const int j = i / TDT;
            const int q = i - j * TDT;
            const int v = hist[(j + off) * TDT + q];
            const int dd = sh_dir[q];
            if (v != 0 && dd >= 0) atomicAdd(&out[((long long)b * P.D + dd) * T + j], v);
        }
    }
}

// Prefix sums over thresholds: ECT, or Radon = prefix(lo) + suffix(hi) - chi.
__global__ void k_hist_finish(int mode, int B, int D, int T, const long long* chi, int32_t* out,
                              const int32_t* hi) {
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= (long long)B * D) return;
    int32_t* o = out + row * T;
    int carry = 0;
    for (int j0 = 0; j0 < T; j0 += 32) {
        const int j = j0 + lane;
        int v = j < T ? o[j] : 0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, s);
            if (lane >= s) v += u;
        }
        v += carry;
        if (j < T) o[j] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    if (mode != kModeRadon) return;
    const int b = (int)(row / D);
    const int32_t c = (int32_t)chi[b];
    const int32_t* h = hi + row * T;
    carry = 0;
    for (int j0 = T - 1; j0 >= 0; j0 -= 32) {   // suffix sums, walking down
        const int j = j0 - lane;
        int v = j >= 0 ? h[j] : 0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, s);
            if (lane >= s) v += u;
        }
        v += carry;
        if (j >= 0) o[j] += v - c;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// Kernel attributes are set once per instantiation (largest dynamic shared memory, max
// shared carveout), so that later launches -- also inside stream capture -- only launch.
static cudaError_t set_smem_attrs(const void* k) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int NDIM, typename Tval>
static cudaError_t launch_hist_n(const EvalPlan& P, const TablesDev& t, int td, int32_t* lo, int32_t* hi,
                                 int grid, cudaStream_t st) {
    const size_t smem = sizeof(float4) * kHistSub + sizeof(int) * (size_t)td * (P.T + 1);
#define TOPOT_HIST_CASE(TDV)                                                                   \
    case TDV: {                                                                                \
        auto k = k_hist<NDIM, (TDV > 32 ? 32 : TDV), (TDV > 32 ? 2 : 1), Tval>;                \
        static cudaError_t attr = set_smem_attrs(reinterpret_cast<const void*>(k));            \
        if (attr != cudaSuccess) return attr;                                                  \
        k<<<grid, kHistBlock, smem, st>>>(P, t, lo, hi);                                       \
        break;                                                                                 \
    }
    switch (td) {
        TOPOT_HIST_CASE(8)
        TOPOT_HIST_CASE(16)
        TOPOT_HIST_CASE(32)
        TOPOT_HIST_CASE(64)
        default: return cudaErrorInvalidValue;
    }
#undef TOPOT_HIST_CASE
    return cudaGetLastError();
}

size_t hist_smem_bytes(int td, int T) { return sizeof(float4) * kHistSub + sizeof(int) * (size_t)td * (T + 1); }

cudaError_t launch_hist(const EvalPlan& P, const TablesDev& t, int td, int32_t* lo, int32_t* hi, int grid,
                        cudaStream_t st) {
    if (t.n == 2) {
        if (t.val_bytes == 2) return launch_hist_n<2, int16_t>(P, t, td, lo, hi, grid, st);
        return launch_hist_n<2, int32_t>(P, t, td, lo, hi, grid, st);
    }
    if (t.val_bytes == 2) return launch_hist_n<3, int16_t>(P, t, td, lo, hi, grid, st);
    return launch_hist_n<3, int32_t>(P, t, td, lo, hi, grid, st);
}

cudaError_t launch_hist_finish(int mode, int B, int D, int T, const long long* chi, int32_t* out,
                               const int32_t* hi, cudaStream_t st) {
    const long long rows = (long long)B * D;
    const int wpb = 8;
    const long long blocks = (rows + wpb - 1) / wpb;
    k_hist_finish<<<(unsigned)blocks, wpb * 32, 0, st>>>(mode, B, D, T, chi, out, hi);
    return cudaGetLastError();
}

}  // namespace topot
