// Exact representations of the ECT and of the Radon transform, and their evaluation
// at arbitrary thresholds (Section 4.3; Appendix A.2 computation, A.3 evaluation).
//
// For one image and one direction xi (eps = eps^xi):
//   kind 0: (T, E) of t -> ECT(xi, t).  T holds the distinct dot products s_v = <xi, x(v)>
//           of the points of the lower table Delta^-_eps, ascending; E the cumulative sums
//           of their values with equal dot products merged.  ECT(xi, t) = E at the largest
//           T <= t (0 if none).
//   kind 1: (T', E') built the same way from the table Delta_eps (the stored partner's
//           table with the sign flipped when eps is outside the stored half).  With the
//           level set split as for the grid Radon transform (sum_v Delta^-_{-eps} = chi),
//             R(xi, t) = sum_{s_v < t} Delta_eps(v) + sum_{s_v = t} Delta^-_eps(v),
//           i.e. E' at the largest T' < t plus the jump of E at t.
//
// Steps, per (image, direction) segment, all on the device:
//   keys   : s_v exactly as the canonical FP64 dot product (one rounding per product and
//            per sum, left to right), mapped (-0 with +0) to an unsigned 64-bit key
//            whose order is the order of the doubles.  The products xi_k x_k(c) of one
//            direction take m_0 + ... + m_{n-1} values; a block stages them in shared
//            memory once per direction, so that an entry costs n - 1 FP64 additions and no
//            division.  The same pass counts the eight 8-bit digits of every key per
//            segment (segments longer than one radix tile);
//   sort   : least-significant-digit radix sort, eight stable passes of 8-bit digits.  A
//            pass takes one 4096-entry tile per block (tickets in launch order), ranks the
//            tile's keys by digit (warp peers from ballots, per-warp counters, one scan
//            over warps), publishes the tile's digit counts and finds the counts of the
//            segment's earlier tiles by decoupled look-back, reorders the tile by digit in
//            shared memory and writes it out in runs of equal digit;
//   finish : one block per segment scans the sorted run; a tie group ends where the key
//            changes, and its end writes T and the running sum E;
//   eval   : one binary search per (segment, query).
#include <algorithm>

#include "internal.cuh"

namespace topot {

constexpr int kRadixBins = 256;
constexpr int kRadixPasses = 8;
constexpr int kRadixThreads = 512;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kKeysThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Radix look-back words: pass + 1 in bits 63..60 (words of an earlier pass read as not
// yet published), flag in bits 59..58 (1: tile count, 2: inclusive prefix), count below.
constexpr unsigned long long kRadixA = 1ull << 58;
constexpr unsigned long long kRadixP = 2ull << 58;
constexpr unsigned long long kRadixCount = (1ull << 58) - 1;

// -0 and +0 map to one key (that of +0)
__device__ __forceinline__ unsigned long long order_key(double s) {
    unsigned long long u = (unsigned long long)__double_as_longlong(s);
    if (u == (1ull << 63)) u = 0ull;
    return (u >> 63) ? ~u : (u | (1ull << 63));
}

__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}

// Lanes of the warp with the same 8-bit digit (lanes with ok false form a group of their
// own): nine ballots, one per digit bit and one for ok.  (match.any runs on the
// address-divergence unit at a fraction of this rate.)
template <bool ALL_OK>
__device__ __forceinline__ unsigned digit_peers(unsigned dg, bool ok) {
    unsigned peers = kFull;
    if (!ALL_OK) {
        const unsigned okm = __ballot_sync(kFull, ok);
        peers = ok ? okm : ~okm;
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bb = __ballot_sync(kFull, (dg >> b) & 1u);
        peers &= bb ^ (((dg >> b) & 1u) - 1u);   // bb where the bit is set, ~bb where clear
    }
    return peers;
}

// x_k(c) = (2c - (m - 1)) / (2(m - 1)): the vertex coordinate in [-1/2, 1/2] (one rounding)
__device__ __forceinline__ double vertex_coord(int c, int m) {
    return __ddiv_rn((double)(2 * c - (m - 1)), (double)(2 * (m - 1)));
}

template <int NDIM, typename Tval>
__global__ void __launch_bounds__(kKeysThreads) k_exact_keys(ExactArgs a) {
    constexpr int NO = 1 << NDIM;
    extern __shared__ __align__(16) unsigned char keys_smem[];
    unsigned* hist = reinterpret_cast<unsigned*>(keys_smem);                       // [8][256]
    double* prod = reinterpret_cast<double*>(keys_smem + sizeof(unsigned) * kRadixPasses * kRadixBins);
    const TablesDev& T = a.t;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool count_digits = a.hist != nullptr;
    for (int seg = blockIdx.y; seg < a.nseg; seg += gridDim.y) {
        const int b = seg / a.D, d = seg - b * a.D;
        const double* xi = a.dirs + ((long long)(a.per_image ? b * a.D : 0) + d) * NDIM;
        double x[NDIM];
        int o = 0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            x[k] = xi[k];
            if (x[k] < 0.0) o |= 1 << k;           // eps_k = -1 only for a negative coordinate
        }
        int tab = o, sg = 1;
        if (a.kind == 1) {
            int r = o;
            if (o >= NO / 2) {
                r = o ^ (NO - 1);
                sg = -1;
            }
            tab = NO + r;
        }
        const ImgDesc& I = T.img[b];
        const long long n = T.seg_count[(long long)b * T.S + tab];
        const long long base = I.seg_base + (long long)tab * I.N;
        if (blockIdx.x == 0 && tid == 0) a.cnt[seg] = (int)n;
        const int mm[4] = {I.m[0], I.m[1], I.m[2], I.m[3]};
        const FastDiv div0 = I.div0, div1 = I.div1;       // registers: the stores below may alias
        int off[NDIM + 1];
        off[0] = 0;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) off[k + 1] = off[k] + mm[k];
        const bool staged = off[NDIM] <= a.prod_max;
        if (staged) {
#pragma unroll
            for (int k = 0; k < NDIM; ++k)
                for (int j = tid; j < mm[k]; j += kKeysThreads) prod[off[k] + j] = __dmul_rn(x[k], vertex_coord(j, mm[k]));
        }
        if (count_digits)
            for (int j = tid; j < kRadixPasses * kRadixBins; j += kKeysThreads) hist[j] = 0u;
        __syncthreads();
        unsigned long long* K = a.key[0] + (long long)seg * a.cap;
        int* V = a.val[0] + (long long)seg * a.cap;
        const int* ai = T.arena_idx + base;
        const Tval* av = reinterpret_cast<const Tval*>(T.arena_val) + base;
        // warp-uniform trip count: every lane of a warp takes part in the digit counts
        for (long long i = (long long)blockIdx.x * kKeysThreads + tid; i - lane < n;
             i += (long long)gridDim.x * kKeysThreads) {
            const bool ok = i < n;
            unsigned long long key = 0ull;
            if (ok) {
                const uint32_t idx = (uint32_t)ai[i];
                int c[4];
                if (NDIM == 4) {   // generic-n tables: plain division
                    uint32_t r = idx;
                    c[0] = (int)(r % (uint32_t)mm[0]);
                    r /= (uint32_t)mm[0];
                    c[1] = (int)(r % (uint32_t)mm[1]);
                    r /= (uint32_t)mm[1];
                    c[2] = (int)(r % (uint32_t)mm[2]);
                    c[3] = (int)(r / (uint32_t)mm[2]);
                } else {
                    const uint32_t q1 = fastdiv(idx, div0);
                    c[0] = (int)(idx - q1 * (uint32_t)mm[0]);
                    if (NDIM == 2) {
                        c[1] = (int)q1;
                    } else {
                        const uint32_t q2 = fastdiv(q1, div1);
                        c[1] = (int)(q1 - q2 * (uint32_t)mm[1]);
                        c[2] = (int)q2;
                    }
                }
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < NDIM; ++k) {
                    const double pk = staged ? prod[off[k] + c[k]] : __dmul_rn(x[k], vertex_coord(c[k], mm[k]));
                    s = k == 0 ? pk : __dadd_rn(s, pk);
                }
                key = order_key(s);
                K[i] = key;
                V[i] = sg * (int)av[i];
            }
            if (count_digits) {
                // a digit the whole warp shares (the high digits of neighbouring vertices)
                // takes one atomic; otherwise every lane adds its own
                const unsigned okm = __ballot_sync(kFull, ok);
#pragma unroll
                for (int p = 0; p < kRadixPasses; ++p) {
                    const unsigned dg = (unsigned)(key >> (8 * p)) & 255u;
                    const unsigned d0 = __shfl_sync(kFull, dg, 0);
                    if (__all_sync(kFull, !ok || dg == d0)) {
                        if (lane == 0 && ok) atomicAdd(hist + p * kRadixBins + d0, (unsigned)__popc(okm));
                    } else if (ok) {
                        atomicAdd(hist + p * kRadixBins + dg, 1u);
                    }
                }
            }
        }
        __syncthreads();
        if (count_digits) {
            unsigned* gh = a.hist + (long long)seg * kRadixPasses * kRadixBins;
            for (int j = tid; j < kRadixPasses * kRadixBins; j += kKeysThreads)
                if (hist[j]) atomicAdd(gh + j, hist[j]);
            __syncthreads();
        }
    }
}

// Exclusive scan of one 64-bit value per thread of a kRadixThreads block.
__device__ __forceinline__ long long radix_block_scan(long long v, long long* tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long x = v;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, dd);
        if (lane >= dd) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kRadixWarps ? tmp[lane] : 0;
        const long long w0 = w;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const long long y = __shfl_up_sync(kFull, w, dd);
            if (lane >= dd) w += y;
        }
        if (lane < kRadixWarps) tmp[lane] = w - w0;
    }
    __syncthreads();
    return tmp[warp] + x - v;
}

struct RadixSmem {
    unsigned long long k[kRadixTile];     // the tile reordered by digit
    int v[kRadixTile];
    int whist[kRadixWarps][kRadixBins];   // per-warp digit counts, then exclusive over warps
    long long gbase[kRadixBins];          // output position of local position 0 of each digit
    int lstart[kRadixBins];               // first local position of each digit
    long long scan[kRadixWarps];
    int tile;
};

// One stable counting pass on bits [8 pass, 8 pass + 8) of the keys: buffer (pass & 1)
// to buffer (pass & 1) ^ 1.
__global__ void __launch_bounds__(kRadixThreads) k_exact_radix_pass(ExactArgs a, int pass) {
    extern __shared__ __align__(16) unsigned char radix_smem[];
    RadixSmem& S = *reinterpret_cast<RadixSmem*>(radix_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) S.tile = atomicAdd(a.tile_ctr + pass, 1);
    __syncthreads();
    // tickets run over the segments first: a tile's predecessor in its segment took its
    // ticket nseg tickets earlier, so look-back rarely walks more than a tile or two
    const int lt = S.tile / a.nseg, seg = S.tile - lt * a.nseg;
    const long long tile = (long long)seg * a.tps + lt;    // look-back word index
    const int n = a.cnt[seg];
    const int start = lt * kRadixTile;
    if (start >= n) return;                    // past the end of the segment (block-uniform)
    for (int j = tid; j < kRadixWarps * kRadixBins; j += kRadixThreads) (&S.whist[0][0])[j] = 0;
    __syncthreads();
    const int m = min(kRadixTile, n - start);
    const int src = pass & 1, shift = 8 * pass;
    const long long sbase = (long long)seg * a.cap;
    const unsigned long long* K = a.key[src] + sbase + start;
    const int* V = a.val[src] + sbase + start;

    // load warp-striped (a warp's items in tile order), rank within the warp
    unsigned long long key[kRadixItems];
    int val[kRadixItems], rank[kRadixItems];
    int* wh = S.whist[warp];
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int idx = warp * 32 * kRadixItems + i * 32 + lane;
        key[i] = idx < m ? K[idx] : 0ull;
        val[i] = idx < m ? V[idx] : 0;
    }
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int idx = warp * 32 * kRadixItems + i * 32 + lane;
        const bool ok = idx < m;
        const unsigned dg = (unsigned)(key[i] >> shift) & 255u;
        const unsigned peers = m == kRadixTile ? digit_peers<true>(dg, true) : digit_peers<false>(dg, ok);
        const int lower = __popc(peers & below);
        int old = 0;
        if (ok && lower == 0) {
            old = wh[dg];
            wh[dg] = old + __popc(peers);
        }
        old = __shfl_sync(kFull, old, __ffs(peers) - 1);
        rank[i] = old + lower;
        __syncwarp();
    }
    __syncthreads();

    // per digit: exclusive offsets over warps, the tile's count, the segment's count
    long long packed = 0;
    int tcount = 0;
    if (tid < kRadixBins) {
        int run = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            const int c = S.whist[w][tid];
            S.whist[w][tid] = run;
            run += c;
        }
        tcount = run;
        // the digit's count in the whole segment (the tile itself when it is the only one)
        const long long segc =
            a.tps > 1 ? (long long)a.hist[((long long)seg * kRadixPasses + pass) * kRadixBins + tid] : (long long)run;
        packed = (segc << 32) | (long long)run;   // tile counts <= 4096: no carry into the high half
    }
    const long long excl = radix_block_scan(packed, S.scan);
    if (tid < kRadixBins) {
        const int lstart = (int)(excl & 0xffffffffll);
        long long prefix = 0;                     // this digit in the segment's earlier tiles
        if (a.tps > 1) {
            unsigned long long* st = a.status + tile * kRadixBins + tid;
            const unsigned long long tag = (unsigned long long)(pass + 1) << 60;
            if (lt == 0) {
                st_relaxed_u64(st, tag | kRadixP | (unsigned long long)tcount);
            } else {
                st_relaxed_u64(st, tag | kRadixA | (unsigned long long)tcount);
                const long long first = tile - lt;
                long long j = tile - 1;
                const unsigned long long t0 = dev_time_ns();
                while (j >= first) {
                    const unsigned long long w = ld_relaxed_u64(a.status + j * kRadixBins + tid);
                    const unsigned long long flag = w & (3ull << 58);
                    if ((w >> 60) == (unsigned long long)(pass + 1) && flag != 0ull) {
                        prefix += (long long)(w & kRadixCount);
                        if (flag == kRadixP) break;
                        --j;
                    } else if (dev_time_ns() - t0 > kWaitLimitNs) {
                        dev_set_error(a.t.err, kDevErrTimeout);
                        break;
                    }
                }
                st_relaxed_u64(st, tag | kRadixP | (unsigned long long)(prefix + tcount));
            }
        }
        S.lstart[tid] = lstart;
        S.gbase[tid] = (excl >> 32) + prefix - lstart;
    }
    __syncthreads();

    // reorder the tile by digit, then write runs of equal digit
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int idx = warp * 32 * kRadixItems + i * 32 + lane;
        if (idx < m) {
            const int dg = (int)(key[i] >> shift) & 255;
            const int pos = S.lstart[dg] + wh[dg] + rank[i];
            S.k[pos] = key[i];
            S.v[pos] = val[i];
        }
    }
    __syncthreads();
    unsigned long long* K2 = a.key[src ^ 1] + sbase;
    int* V2 = a.val[src ^ 1] + sbase;
    for (int idx = tid; idx < m; idx += kRadixThreads) {
        const unsigned long long kk = S.k[idx];
        const long long out = S.gbase[(int)(kk >> shift) & 255] + idx;
        K2[out] = kk;
        V2[out] = S.v[idx];
    }
}

// Pair scan (exclusive) of (count, sum) over a kRadixThreads block.
__device__ __forceinline__ void radix_block_scan2(long long& c, long long& s, long long* tc, long long* ts) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long c0 = c, s0 = s;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const long long yc = __shfl_up_sync(kFull, c, dd);
        const long long ys = __shfl_up_sync(kFull, s, dd);
        if (lane >= dd) {
            c += yc;
            s += ys;
        }
    }
    if (lane == 31) {
        tc[warp] = c;
        ts[warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
        long long wc = lane < kRadixWarps ? tc[lane] : 0, ws = lane < kRadixWarps ? ts[lane] : 0;
        const long long wc0 = wc, ws0 = ws;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const long long yc = __shfl_up_sync(kFull, wc, dd);
            const long long ys = __shfl_up_sync(kFull, ws, dd);
            if (lane >= dd) {
                wc += yc;
                ws += ys;
            }
        }
        if (lane < kRadixWarps) {
            tc[lane] = wc - wc0;
            ts[lane] = ws - ws0;
        }
        if (lane == kRadixWarps - 1) {       // block totals
            tc[kRadixWarps] = wc;
            ts[kRadixWarps] = ws;
        }
    }
    __syncthreads();
    c = tc[warp] + c - c0;
    s = ts[warp] + s - s0;
}

// Decoupled look-back over one quantity of the tiles of a segment (tile words spaced by
// kRadixBins, quantity q at offset q): publishes the tile's aggregate, returns the sum
// over the earlier tiles and publishes the inclusive value.  Values are two's complement
// in 58 bits.
__device__ long long finish_lookback(const ExactArgs& a, long long tile, int lt, int q, long long agg) {
    const unsigned long long tag = 9ull << 60;
    unsigned long long* st = a.status + tile * kRadixBins + q;
    const unsigned long long enc = (unsigned long long)agg & kRadixCount;
    if (lt == 0) {
        st_relaxed_u64(st, tag | kRadixP | enc);
        return 0;
    }
    st_relaxed_u64(st, tag | kRadixA | enc);
    long long prefix = 0, j = tile - 1;
    const long long first = tile - lt;
    const unsigned long long t0 = dev_time_ns();
    while (j >= first) {
        const unsigned long long w = ld_relaxed_u64(a.status + j * kRadixBins + q);
        const unsigned long long flag = w & (3ull << 58);
        if ((w >> 60) == 9ull && flag != 0ull) {
            prefix += ((long long)(w << 6)) >> 6;
            if (flag == kRadixP) break;
            --j;
        } else if (dev_time_ns() - t0 > kWaitLimitNs) {
            dev_set_error(a.t.err, kDevErrTimeout);
            break;
        }
    }
    st_relaxed_u64(st, tag | kRadixP | ((unsigned long long)(prefix + agg) & kRadixCount));
    return prefix;
}

struct FinishSmem {
    unsigned long long k[kRadixTile + 1];    // the tile's keys and the next key; then T
    int v[kRadixTile];                        // values; then E
    long long tc[kRadixWarps + 1], ts[kRadixWarps + 1];
    long long pre[2];
    int tile;
};

// Tie groups of the sorted segments: a group ends where the key changes; its end writes
// T (the value) and E (the running sum of the values).  Tiles of 4096 sorted entries;
// the number of groups and the value sum of the segment's earlier tiles by look-back.
__global__ void __launch_bounds__(kRadixThreads) k_exact_finish(ExactArgs a) {
    extern __shared__ __align__(16) unsigned char finish_smem[];
    FinishSmem& S = *reinterpret_cast<FinishSmem*>(finish_smem);
    const int tid = threadIdx.x;
    if (tid == 0) S.tile = atomicAdd(a.tile_ctr + kRadixPasses, 1);
    __syncthreads();
    const int lt = S.tile / a.nseg, seg = S.tile - lt * a.nseg;
    const long long tile = (long long)seg * a.tps + lt;
    const int n = a.cnt[seg];
    const int start = lt * kRadixTile;
    if (start >= n) {
        if (lt == 0 && tid == 0) a.len[seg] = 0;
        return;
    }
    const int m = min(kRadixTile, n - start);
    const bool last = start + m == n;
    const long long sbase = (long long)seg * a.cap;
    const unsigned long long* K = a.key[0] + sbase + start;
    const int* V = a.val[0] + sbase + start;
    for (int i = tid; i < m; i += kRadixThreads) {
        S.k[i] = K[i];
        S.v[i] = V[i];
    }
    if (tid == 0) S.k[m] = last ? ~K[m - 1] : K[m];   // after the segment: any other key
    __syncthreads();
    // warp-striped items (a warp's items in tile order): group ends by ballot, value sums
    // by warp scans
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned below = (1u << lane) - 1u;
    unsigned long long key[kRadixItems];
    int pos[kRadixItems];
    long long run[kRadixItems];
    unsigned ends = 0u;
    long long wc = 0, ws = 0;                 // groups and sum of the warp's earlier items
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int idx = warp * 32 * kRadixItems + i * 32 + lane;
        const bool ok = idx < m;
        key[i] = ok ? S.k[idx] : 0ull;
        int x = ok ? S.v[idx] : 0;
        const bool e = ok && S.k[idx + 1] != key[i];
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const int y = __shfl_up_sync(kFull, x, dd);
            if (lane >= dd) x += y;
        }
        const unsigned bal = __ballot_sync(kFull, e);
        if (e) ends |= 1u << i;
        pos[i] = (int)wc + __popc(bal & below);
        run[i] = ws + x;
        wc += __popc(bal);
        ws += __shfl_sync(kFull, x, 31);
    }
    // one value per warp into the block scan (other lanes contribute zero)
    long long c = lane == 31 ? wc : 0, sum = lane == 31 ? ws : 0;
    radix_block_scan2(c, sum, S.tc, S.ts);
    const long long wpre_c = __shfl_sync(kFull, c, 31), wpre_s = __shfl_sync(kFull, sum, 31);
    if (a.tps > 1) {
        if (tid == 0) S.pre[0] = finish_lookback(a, tile, lt, 0, S.tc[kRadixWarps]);
        if (tid == 32) S.pre[1] = finish_lookback(a, tile, lt, 1, S.ts[kRadixWarps]);
    } else if (tid == 0) {
        S.pre[0] = 0;
        S.pre[1] = 0;
    }
    __syncthreads();                          // the keys are in registers: S.k, S.v take T, E
    const long long gc = S.pre[0];
    const int tile_groups = (int)S.tc[kRadixWarps];
    const long long base_s = S.pre[1] + wpre_s;
    double* Ts = reinterpret_cast<double*>(S.k);
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        if ((ends >> i) & 1u) {
            const int p = (int)wpre_c + pos[i];
            Ts[p] = key_value(key[i]);
            S.v[p] = (int)(base_s + run[i]);
        }
    }
    __syncthreads();
    double* To = a.T + sbase + gc;
    int32_t* Eo = a.E + sbase + gc;
    for (int i = tid; i < tile_groups; i += kRadixThreads) {
        To[i] = Ts[i];
        Eo[i] = S.v[i];
    }
    if (last && tid == 0) a.len[seg] = gc + tile_groups;
}

__global__ void k_ect_exact_eval(int nseg, long long cap, const double* T, const int32_t* E, const long long* len,
                                 const double* t, int Q, int32_t* out) {
    const long long total = (long long)nseg * Q;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long seg = k / Q;
        const double tq = t[k - seg * Q];
        const double* Ts = T + seg * cap;
        long long lo = 0, hi = len[seg];
        while (lo < hi) {                           // number of T <= t
            const long long mid = (lo + hi) >> 1;
            if (Ts[mid] <= tq) lo = mid + 1;
            else hi = mid;
        }
        out[k] = lo > 0 ? E[seg * cap + lo - 1] : 0;
    }
}

__device__ __forceinline__ long long count_le(const double* Ts, long long L, double t, bool strict) {
    long long lo = 0, hi = L;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (strict ? (Ts[mid] < t) : (Ts[mid] <= t)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_radon_exact_eval(int nseg, long long cap, const double* Tl, const int32_t* El,
                                   const long long* lenl, long long cap_o, const double* To, const int32_t* Eo,
                                   const long long* leno, const double* t, int Q, int32_t* out) {
    const long long total = (long long)nseg * Q;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long seg = k / Q;
        const double tq = t[k - seg * Q];
        const long long off = seg * cap, off_o = seg * cap_o;
        const long long nb = count_le(To + off_o, leno[seg], tq, true);      // T' < t
        const long long kle = count_le(Tl + off, lenl[seg], tq, false);      // T <= t
        const long long klt = count_le(Tl + off, lenl[seg], tq, true);       // T < t
        const int32_t below = nb > 0 ? Eo[off_o + nb - 1] : 0;
        const int32_t e_le = kle > 0 ? El[off + kle - 1] : 0;
        const int32_t e_lt = klt > 0 ? El[off + klt - 1] : 0;
        out[k] = below + (e_le - e_lt);
    }
}

// ---- host side ------------------------------------------------------------------------------

static unsigned grid_1d(long long work, int threads, int cap_blocks) {
    long long g = (work + threads - 1) / threads;
    return (unsigned)std::max(1ll, std::min(g, (long long)cap_blocks));
}

int exact_radix_tile() { return kRadixTile; }

size_t exact_keys_smem(int prod_max) {
    return sizeof(unsigned) * kRadixPasses * kRadixBins + sizeof(double) * (size_t)prod_max;
}

template <int NDIM, typename Tval>
static cudaError_t launch_keys(const ExactArgs& a, dim3 grid, cudaStream_t st) {
    const size_t smem = exact_keys_smem(a.prod_max);
    cudaError_t e = cudaFuncSetAttribute(k_exact_keys<NDIM, Tval>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_exact_keys<NDIM, Tval><<<grid, kKeysThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_exact(int n, bool u8, ExactArgs a, long long max_n, int sm_count, cudaStream_t st) {
    const unsigned gy = (unsigned)std::min(a.nseg, 65535);
    const int per_seg_blocks = std::max(1, std::min(4 * sm_count, 65535) / (int)gy);
    dim3 gk(grid_1d(max_n, kKeysThreads, per_seg_blocks), gy);
    cudaError_t e;
    if (n == 2) e = u8 ? launch_keys<2, int16_t>(a, gk, st) : launch_keys<2, int32_t>(a, gk, st);
    else if (n == 3) e = u8 ? launch_keys<3, int16_t>(a, gk, st) : launch_keys<3, int32_t>(a, gk, st);
    else e = u8 ? launch_keys<4, int16_t>(a, gk, st) : launch_keys<4, int32_t>(a, gk, st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(RadixSmem);
    e = cudaFuncSetAttribute(k_exact_radix_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned tiles = (unsigned)((long long)a.nseg * a.tps);
    for (int pass = 0; pass < kRadixPasses; ++pass) {
        k_exact_radix_pass<<<tiles, kRadixThreads, smem, st>>>(a, pass);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const size_t fsmem = sizeof(FinishSmem);
    e = cudaFuncSetAttribute(k_exact_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
    if (e != cudaSuccess) return e;
    k_exact_finish<<<tiles, kRadixThreads, fsmem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ect_exact_eval(int nseg, long long cap, const double* T, const int32_t* E, const long long* len,
                                  const double* t, int Q, int32_t* out, int sm_count, cudaStream_t st) {
    k_ect_exact_eval<<<grid_1d((long long)nseg * Q, 256, 16 * sm_count), 256, 0, st>>>(nseg, cap, T, E, len, t, Q,
                                                                                        out);
    return cudaGetLastError();
}

cudaError_t launch_radon_exact_eval(int nseg, long long cap, const double* Tl, const int32_t* El,
                                    const long long* lenl, long long cap_o, const double* To, const int32_t* Eo,
                                    const long long* leno, const double* t, int Q, int32_t* out, int sm_count,
                                    cudaStream_t st) {
    k_radon_exact_eval<<<grid_1d((long long)nseg * Q, 256, 16 * sm_count), 256, 0, st>>>(
        nseg, cap, Tl, El, lenl, cap_o, To, Eo, leno, t, Q, out);
    return cudaGetLastError();
}

}  // namespace topot
