/*
 * topot.h -- C ABI of libtopot.so: topological integral transforms of images and
 * volumes on one GPU (critical-point tables, Euler characteristic transform, Radon
 * transform, hybrid transforms and their gradient).
 *
 * Method: Lebovici, Oudot, Passe, "Efficient computation of topological integral
 * transforms" (SEA 2024, arXiv 2405.02256).  Each entry point names the passage that
 * defines the operation it performs.
 *
 * Conventions shared by every call
 * --------------------------------
 * - An image with n in {2, 3, 4} axes has lengths m_0 .. m_{n-1}, m_0 being the FASTEST
 *   memory axis; every m_k >= 2.  Vertex v = (i_0, .., i_{n-1}) has linear index
 *   i_0 + m_0 (i_1 + m_1 (i_2 + m_2 i_3)).  The method holds in any dimension (Section
 *   2.1); n = 2 and 3 run on specialised kernels, n = 4 on plain generic-n kernels (same
 *   calls, same results, slower).
 * - Complex: "dual"/vertex construction (Section 5): pixels are vertices, a cube
 *   exists iff all its vertices are pixels, and carries the minimum of their values.
 *   The top-dimensional construction (TOPOT_TOP) is described at topot_construction;
 *   with it, m_k below means the number of pixel corners, m_k + 1.
 * - Embedding (Section 4.1): x_k(i) = (2 i - (m_k - 1)) / (2 (m_k - 1)), in [-0.5, 0.5].
 * - Orthant o in [0, 2^n): bit k set <=> eps_k = -1.  The sign vector of a direction
 *   xi is eps_k = +1 if xi_k >= 0 (zero included), else -1 (Section 3, Lemma 3.2).
 * - Dot products <xi, x(v)> and thresholds t_j = a + j (b - a) / (T - 1) (Appendix A.4)
 *   are decided exactly as the FP64 expressions
 *       s   = fl(fl(fl(xi_0 x_0) + fl(xi_1 x_1)) + fl(xi_2 x_2))
 *       t_j = fl(a + fl(fl(j fl(b - a)) / (T - 1)))
 *   would decide them (the sum continuing left to right for n = 4); integer results
 *   (tables, ECT, Radon) are therefore exact.
 * - Pointers named d_* are DEVICE pointers, h_* HOST pointers; the caller owns them.
 *   `stream` is a cudaStream_t (NULL = legacy default stream).  Unless stated
 *   otherwise calls only enqueue work on `stream` and return; outputs are valid once
 *   the stream has reached that point.  A handle owns one workspace per family of
 *   calls: (ect, radon), (hybrid transforms and gradients, tabulated or not),
 *   (exact_representation).  Calls of one family on one handle must be ordered on one
 *   stream; calls of different families may run concurrently once the tables are built,
 *   and tables_build must be ordered with all of them.
 * - No exception crosses the ABI.  Every call returns a topot_status; on error the
 *   outputs are unspecified and topot_last_error() gives a message (thread-local).
 * - Directions must be finite.
 */
#ifndef TOPOT_H
#define TOPOT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TOPOT_API __attribute__((visibility("default")))
#else
#define TOPOT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TOPOT_OK = 0,
    TOPOT_ERR_INVALID_ARG = 1,   /* bad shape, pointer, size or enum value          */
    TOPOT_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement     */
    TOPOT_ERR_OOM = 3,           /* device allocation failed                        */
    TOPOT_ERR_CUDA = 4,          /* a CUDA runtime call failed                      */
    TOPOT_ERR_OVERFLOW = 5,      /* a result would not fit its integer type          */
    TOPOT_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up              */
} topot_status;

typedef enum { TOPOT_U8 = 0, TOPOT_I32 = 1 } topot_dtype;

/* TOPOT_VERTEX: dual construction (Section 5): pixels are vertices, a cube carries the
 * minimum of its vertices.  TOPOT_TOP: top-dimensional construction (Section 4.1): one
 * top cube per pixel, every lower cell carries the minimum over the pixels containing
 * it; the vertices are the pixel corners, so the tables, the embedding and every
 * transform live on a grid of m_k + 1 vertices per axis (m_k >= 1 pixels). */
typedef enum { TOPOT_VERTEX = 0, TOPOT_TOP = 1 } topot_construction;

/* Kernel primitives kbar of the hybrid transform (Section 2.2; Lemma 3.1):
 *   LAPLACE  kbar(s) = e^s             (Appendix A.2 uses kbar = exp)
 *   FOURIER  kbar(s) = sin s + i cos s (kappa(t) = e^{-i t}); output (re, im)
 *   BESSEL   kbar(s) = J_0(s)          (kappa = -J_1)
 *   SINE     kbar(s) = -cos s          (kappa = sin, the kernel of the experiments of
 *                                       Section 5); real output
 *   TABLE    kbar given by samples (kernel_table_create); only through
 *            hybrid_transform_table / hybrid_transform_table_grad               */
typedef enum { TOPOT_LAPLACE = 0, TOPOT_FOURIER = 1, TOPOT_BESSEL = 2, TOPOT_SINE = 3, TOPOT_TABLE = 4 } topot_kernel;

/* FP32C: FP32 terms, Kahan-compensated per thread, FP64 cross-block combine
 *        (Laplace terms beyond |s| <= 1 are scaled per round of points, so no FP32
 *        term overflows or underflows).  FP64: plain FP64 terms and sums. */
typedef enum { TOPOT_FP32C = 0, TOPOT_FP64 = 1 } topot_precision;

typedef struct topot_tables topot_tables;   /* opaque; owns the device tables */

/* Tile shapes of the evaluation kernels, per operation; 0 = library default.  Set by
 * the autotuner of the Python binding, or by hand. */
typedef struct {
    int ect_dirs_per_warp;    /* ECT / Radon: 8, 16, 32 per warp, or 64 (two per lane)    */
    int ect_chunk;            /* ECT / Radon: critical points per work item (x256)        */
    int ect_ctas_per_sm;      /* ECT / Radon: resident blocks per SM of the persistent grid */
    int ht_dirs_per_lane;     /* hybrid FP32C: 1, 2, 4 (8: Laplace) directions per lane    */
    int ht_chunk;             /* hybrid: critical points per work item (x256)             */
    int ht_ctas_per_sm;       /* hybrid: resident blocks per SM of the persistent grid     */
    int ht_warp_split;        /* hybrid FP32C forward: 1 or 2 point groups per warp; with 2
                                 (and 2 or 4 directions per lane) a tile has 16 x directions
                                 per lane, for small direction sets                        */
} topot_tuning;

/* ---------------------------------------------------------------------------
 * Critical tables (Section 3: Delta^-; Section 4.2: preprocessing)
 * ---------------------------------------------------------------------------
 * For each image b and orthant o, the table of classical critical values
 *   Delta^-_o(v) = chi(phi restricted to LwSt(eps_o, v))
 *               = sum over delta in {0,1}^n, box v..v - delta (.) eps existing,
 *                 of (-1)^|delta| min(phi over the box)
 * keeps every vertex with Delta^-_o(v) != 0, in ascending vertex index; and for
 * each representative orthant r < 2^(n-1) the table of
 *   Delta_r(v) = Delta^-_r(v) - Delta^-_{r ^ (2^n - 1)}(v)    (= -Delta^ord_r)
 * (Delta_{-eps} = -Delta_eps).  chi(phi) = sum_v Delta^-_o(v) for any o.
 *
 * d_pixels : image data (uint8 or int32, see dtype); image b starts at element
 *            h_offsets[b] and has h_shapes[b*n + k] = m_k.  Images must not alias
 *            outputs.  int32 values must satisfy |phi| < 2^26 (n = 4: 2^25).
 * B        : number of images, >= 1.  n: 2, 3 or 4 (4: vertex construction only,
 *            TOPOT_TOP gives UNSUPPORTED).
 * out      : receives a new handle; release it with free_tables().
 * Synchronous: allocates, launches the extraction on `stream`, waits for it and
 * reads the table sizes back.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA,
 * OVERFLOW (int32 input out of range), TIMEOUT.
 */
TOPOT_API topot_status build_critical_tables(const void* d_pixels, topot_dtype dtype, int n,
                                   const int64_t* h_shapes, const int64_t* h_offsets,
                                   int B, topot_construction construction,
                                   void* stream, topot_tables** out);

/* Allocate a handle for images of the given shapes without launching anything.
 * Same arguments as build_critical_tables minus the pixels and stream. */
TOPOT_API topot_status tables_create(topot_dtype dtype, int n, const int64_t* h_shapes,
                           const int64_t* h_offsets, int B,
                           topot_construction construction, topot_tables** out);

/* Slabs of volumes (the paper parallelises the preprocessing over vertex subsets and the
 * evaluation over directions, Section 5.3).  As tables_create for 3-D images (n = 3,
 * vertex construction, else UNSUPPORTED), where image b is the part of a volume of shape
 * h_shapes[b] (m_0, m_1, m_2: the WHOLE volume) made of the planes
 * z in [z0, z1) = [h_zrange[2b], h_zrange[2b+1]) (0 <= z0 < z1 <= m_2, else INVALID_ARG).
 * Its pixel buffer (at h_offsets[b]) holds planes max(z0 - 1, 0) .. min(z1 + 1, m_2) - 1:
 * the slab and the neighbouring plane on each side that exists (staged for the stencil,
 * owned by the neighbouring slab).  The handle's tables hold the owned vertices only,
 * with their linear index in the whole volume and the volume's embedding; chi and
 * sum |Delta^-| (tables_info) are the slab's parts.  Every transform of a slab handle is
 * the slab's part of the volume's transform: ECT and Radon of the slabs of a partition of
 * [0, m_2) sum exactly to the volume's, hybrid transforms and gradients to within their
 * accuracy (slab_sum_i32 / slab_sum_f64 add the parts in slab order).  Exact
 * representations of a slab handle represent the slab's part. */
TOPOT_API topot_status tables_create_slab(topot_dtype dtype, int n, const int64_t* h_shapes,
                                          const int64_t* h_offsets, const int64_t* h_zrange, int B,
                                          topot_tables** out);

/* Sums of slab parts, in slab order (Section 5.3; the exchange step of a volume split
 * across devices).  d_parts is [P][n] (P >= 1 parts of n elements each, for example the
 * ECT, Radon or hybrid outputs of P slabs gathered from P devices), d_out [n].
 *   slab_sum_i32: exact integer sums; *d_overflow (device, caller-owned) is set to 0 and
 *     then to 1 if some sum leaves the int32 range (that element is written as 0).
 *   slab_sum_f64: compensated (Neumaier) FP64 sums in slab order, deterministic.
 * Asynchronous on `stream`; INVALID_ARG on NULL pointers or bad sizes. */
TOPOT_API topot_status slab_sum_i32(const int32_t* d_parts, int P, int64_t n, int32_t* d_out,
                                    uint32_t* d_overflow, void* stream);
TOPOT_API topot_status slab_sum_f64(const double* d_parts, int P, int64_t n, double* d_out, void* stream);

/* Enqueue the extraction of all tables of `t` from d_pixels on `stream`
 * (asynchronous, no allocation, no host synchronisation: may be captured in a
 * CUDA graph once the handle exists).  Table sizes stay on the device; the
 * evaluation calls read them there.  tables_sync() makes them visible on the host.
 * Whole 3-D volumes of 8-bit voxels that are all 0 or 1 (decided on the device at each
 * build) take a bit-sliced path (Section 3's lower-star values as AND/XOR bit planes);
 * for such handles the general kernel runs on a stream of the handle, forked from and
 * joined back to `stream` by events, so the call stays ordered on `stream`.  Tables are
 * identical whichever path builds them. */
TOPOT_API topot_status tables_build(topot_tables* t, const void* d_pixels, void* stream);

/* Wait for `stream`, read table sizes, chi and the device error word of `t`.
 * Returns the first device-side error recorded since the last sync (OVERFLOW,
 * TIMEOUT) and clears it. */
TOPOT_API topot_status tables_sync(topot_tables* t, void* stream);

/* Sizes of one table set after a sync: n_lower = |{v: Delta^-_o(v) != 0}|,
 * n_delta = |{v: Delta_r(v) != 0}| with r the representative of o (the partner's
 * table is the negation), chi = chi(phi) of image `image`. */
TOPOT_API topot_status tables_info(const topot_tables* t, int image, int orthant,
                         int64_t* n_lower, int64_t* n_delta, int64_t* chi);

/* Copy one table to host memory (synchronous).  kind 0: Delta^-_orthant;
 * kind 1: Delta_orthant (orthant must be a representative, < 2^(n-1)).
 * h_idx / h_val need room for the size tables_info() reports. */
TOPOT_API topot_status tables_copy_to_host(const topot_tables* t, int image, int orthant, int kind,
                                 int32_t* h_idx, int32_t* h_val);

/* Override the evaluation tile shapes of a handle (NULL restores defaults). */
TOPOT_API topot_status tables_set_tuning(topot_tables* t, const topot_tuning* tuning);

TOPOT_API void free_tables(topot_tables* t);

/* ---------------------------------------------------------------------------
 * Transforms on a grid of directions x thresholds
 * ---------------------------------------------------------------------------
 * d_dirs : FP64 directions, [D][n] shared by every image (per_image_dirs = 0) or
 *          [B][D][n] (per_image_dirs = 1).
 * Thresholds t_j = a + j (b - a) / (T - 1), j < T, T >= 2, a = t_min, b = t_max.
 * d_out  : int32 [B][D][T].
 *
 * ect (Lemma 3.1; Section 4.3; Appendix A.4 vectorisation):
 *   ECT(xi, t_j) = sum over v with <xi, v> <= t_j of Delta^-_{eps(xi)}(v).
 * radon (Section 2.2; additivity of the Euler integral, Appendix B):
 *   R(xi, t_j) = chi({xi = t_j}) = ECT(xi, t_j) + ECT(-xi, -t_j) - chi(phi)
 *             = sum_{s_v <= t_j} Delta^-_{o}(v) + sum_{s_v >= t_j} Delta^-_{o^(2^n-1)}(v) - chi
 *   exact for every xi, generic or not.
 * Errors: INVALID_ARG; OVERFLOW when the sum of |Delta^-| of an image reaches 2^31
 * (checked on the host when the sizes are known, else recorded on the device and
 * reported by tables_sync). */
TOPOT_API topot_status ect(const topot_tables* t, const double* d_dirs, int D, int per_image_dirs,
                 double t_min, double t_max, int T, int32_t* d_out, void* stream);
TOPOT_API topot_status radon(const topot_tables* t, const double* d_dirs, int D, int per_image_dirs,
                   double t_min, double t_max, int T, int32_t* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Exact representations and evaluation at arbitrary thresholds
 * (Section 4.3; Appendix A.2 computation, A.3 evaluation)
 * ---------------------------------------------------------------------------
 * One representation per image b and direction d (segment b * D + d), eps = eps^xi_d:
 *   kind 0: (T, E) of t -> ECT(xi, t).  T = the distinct dot products <xi, x(v)> (the
 *           canonical FP64 dot product) of the points of the lower table Delta^-_eps,
 *           ascending; E = the cumulative sums of their values, equal dot products
 *           merged.  ECT(xi, t) = E at the largest T <= t, 0 if none.
 *   kind 1: (T', E') the same from the table Delta_eps (= -Delta^ord of the paper, so
 *           E' is the negative of the printed E').  R(xi, t) = E' at the largest T' < t
 *           for every t that is not a critical value.
 * d_T [B][D][cap] FP64, d_E [B][D][cap] int32: entries 0 .. d_len[b][D]-1 of each
 * segment are written, the rest left as they are; d_len [B][D] int64.  cap must be at
 * least the largest table the kind can select (tables_info: n_lower for kind 0,
 * n_delta for kind 1), else INVALID_ARG.  The handle must have been synchronised
 * (tables_sync).  Allocates in the handle's workspace (24 B per slot); asynchronous.
 * Errors: INVALID_ARG; OVERFLOW when a sum of |values| of a selectable table reaches
 * 2^31; OOM when the workspace cannot grow. */
TOPOT_API topot_status exact_representation(const topot_tables* t, int kind, const double* d_dirs, int D,
                                            int per_image_dirs, int64_t cap, double* d_T, int32_t* d_E,
                                            int64_t* d_len, void* stream);

/* ECT(xi, t_q) from kind-0 representations: d_out[r][q] = E at the largest T <= t_q of
 * representation r (0 if none), r < nrep = B * D, q < Q; d_t [Q] FP64 (not NaN).
 * Arrays as written by exact_representation with the same cap.  INVALID_ARG on bad
 * sizes or NULL pointers. */
TOPOT_API topot_status ect_exact_eval(int nrep, int64_t cap, const double* d_T, const int32_t* d_E,
                                      const int64_t* d_len, const double* d_t, int Q, int32_t* d_out,
                                      void* stream);

/* R(xi, t_q) at every t_q from a kind-0 (cap, d_T, d_E, d_len) and a kind-1 (cap_ord,
 * d_Tord, d_Eord, d_len_ord) representation of the same images and directions:
 *   R(xi, t) = sum_{s_v < t} Delta_eps(v) + sum_{s_v = t} Delta^-_eps(v)
 *            = E' at the largest T' < t  +  the jump of E at t (0 if t is not in T),
 * the level set {xi = t} split as {xi <= t} + {xi >= t} - everything (additivity of the
 * Euler integral).  d_out [nrep][Q] int32. */
TOPOT_API topot_status radon_exact_eval(int nrep, int64_t cap, const double* d_T, const int32_t* d_E,
                                        const int64_t* d_len, int64_t cap_ord, const double* d_Tord,
                                        const int32_t* d_Eord, const int64_t* d_len_ord, const double* d_t, int Q,
                                        int32_t* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Hybrid transforms (Section 2.2; closed form and sign of Lemma 3.1)
 * ---------------------------------------------------------------------------
 *   HT(xi) = - sum_v Delta^ord_eps(v) kbar(<xi, v>) = sum_v Delta_eps(v) kbar(<xi, v>)
 * (= -int kappa(t) R(xi, t) dt).  d_out: FP64 [B][D] (LAPLACE, BESSEL, SINE) or
 * [B][D][2] (FOURIER: re, im).  Deterministic for a given tuning and direction set.
 * Accuracy, with M = sum_k |xi_k| / 2 >= |<xi, v>|:
 *   FP32C: |HT - exact| <= 1e-6 sum_v |Delta kbar(<xi, v>)| (complex modulus for FOURIER)
 *     for every finite xi with M <= 1e6; LAPLACE overflows (inf or NaN) once some
 *     <xi, v> exceeds ~709, as in FP64.
 *     The terms are kbar(s) - kbar(0) (the constant cancels: sum_v Delta_eps(v) = 0),
 *     so transforms much smaller than that bound (small |xi|) keep their relative
 *     accuracy; tiles with M above 1 (LAPLACE), 1.75 (FOURIER, SINE) or 2 (BESSEL)
 *     form <xi, v> in FP64 and reduce it modulo 2 pi before the FP32 evaluation.
 *     Beyond M ~ 1e6 the FP64 rounding of <xi, v> (2^-53 |<xi, v>|) dominates.
 *   FP64: plain FP64 terms and sums (error of the order of 1e-15 sum_v |Delta kbar|);
 *     LAPLACE overflows (inf or NaN) once some <xi, v> exceeds ~709. */
TOPOT_API topot_status hybrid_transform(const topot_tables* t, topot_kernel kernel,
                              topot_precision precision, const double* d_dirs, int D,
                              int per_image_dirs, double* d_out, void* stream);

/* Adjoint: d_gdirs = sum over images and outputs of d_gout * d HT / d xi, with
 *   d HT(xi) / d xi_k = sum_v Delta_eps(v) kappa(<xi, v>) x_k(v),  kappa = kbar'
 * (Lemma 3.1 differentiated inside an orthant, where the tables are constant by
 * Lemma 3.2).  d_gout is shaped like d_out of hybrid_transform; d_gdirs like d_dirs
 * (FP64).  For FOURIER, gout = (g_re, g_im) and the result is
 * g_re d Re/d xi + g_im d Im/d xi.  With per_image_dirs = 0 the gradients of all
 * images are summed per direction.  Accuracy (FP32C): 2e-6 of sum_v |Delta kappa x_k|
 * per component over the ranges of hybrid_transform (same paths, same LAPLACE limit). */
TOPOT_API topot_status hybrid_transform_grad(const topot_tables* t, topot_kernel kernel,
                                   topot_precision precision, const double* d_dirs, int D,
                                   int per_image_dirs, const double* d_gout,
                                   double* d_gdirs, void* stream);

/* hybrid_transform() for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment variant.  hybrid_transform() may call cudaMalloc to
 * grow the handle's workspace; code running where allocation is forbidden (inside an
 * allocator or memory-pool callback, under a no-allocation real-time budget, in a host
 * that disallows cudaMalloc after start-up) can call this entry point instead.
 * Arguments and result are those of hybrid_transform(); the handle's device must be
 * current.  Its scratch (work plan and partial sums) lives in one fixed 16 MiB device
 * array that every GPU loading the library holds until the process exits.  The first
 * call on a device looks the array's address up (cudaGetSymbolAddress); with CUDA's lazy
 * module loading (the default) that first call also loads the library's device code on
 * that device, which is when the 16 MiB are reserved.  So make the first call during
 * start-up, outside any context that forbids allocation, and before any stream capture;
 * later calls reserve nothing and call no cudaMalloc / cudaFree.  The address is kept per
 * device for the life of the process: after cudaDeviceReset the device code is reloaded
 * elsewhere, so do not call this entry point on a device that has been reset.  A call
 * whose scratch would exceed 16 MiB returns TOPOT_ERR_INVALID_ARG with the size in the
 * message.  All calls on a device share the array: calls that may overlap on the GPU
 * (different streams, no ordering) race and must be serialised by the caller. */
TOPOT_API topot_status hybrid_transform_noalloc(const topot_tables* t, topot_kernel kernel,
                                               topot_precision precision, const double* d_dirs,
                                               int D, int per_image_dirs, double* d_out,
                                               void* stream);

/* ---------------------------------------------------------------------------
 * Tabulated kernels (Section 2.2 admits any locally integrable kappa; Lemma 3.1 needs
 * only its primitive kbar)
 * ---------------------------------------------------------------------------
 * h_values[i] = kbar(s_min + i h), i < K, h = (s_max - s_min) / (K - 1) (FP64, host,
 * copied; the caller keeps ownership).  kbar is the piecewise-linear interpolant of the
 * samples, constant outside [s_min, s_max]:
 *   u = (s - s_min) / h, i = floor(u), f = u - i:  kbar(s) = y_i + f (y_{i+1} - y_i)
 *   for 0 <= u < K - 1;  y_0 for u < 0;  y_{K-1} for u >= K - 1,
 * and kappa = kbar' the step function (y_{i+1} - y_i) / h on [s_min + i h,
 * s_min + (i + 1) h), zero outside [s_min, s_max).  2 <= K <= 16384, finite samples of
 * magnitude <= 1e37 (the FP32 table range), s_min < s_max (finite), else INVALID_ARG.  The handle owns device copies on the
 * current device (for FP32C, K + 1 FP32 pairs: (y_0, 0), (y_r + d_r / 2, d_r) per
 * segment r with d_r = y_{r+1} - y_r, (y_{K-1}, 0); for FP64 the samples); free it with
 * kernel_table_free after the last call that uses it has completed. */
typedef struct topot_ktable topot_ktable;
TOPOT_API topot_status kernel_table_create(const double* h_values, int K, double s_min, double s_max,
                                           topot_ktable** out);
TOPOT_API void kernel_table_free(topot_ktable* k);

/* hybrid_transform / hybrid_transform_grad with the tabulated kernel k (real output,
 * d_out [B][D]; the gradient as hybrid_transform_grad).  FP32C accuracy:
 * |HT - exact| <= 1e-6 sum_v |Delta kbar| when |kappa| (s_max - s_min) is of the order of
 * |kbar| (the FP32 position u carries an absolute error of a few units of 2^-24 K).
 * Gradient: at a dot product within rounding of a knot either neighbouring slope may be
 * taken. */
TOPOT_API topot_status hybrid_transform_table(const topot_tables* t, const topot_ktable* k,
                                              topot_precision precision, const double* d_dirs, int D,
                                              int per_image_dirs, double* d_out, void* stream);
TOPOT_API topot_status hybrid_transform_table_grad(const topot_tables* t, const topot_ktable* k,
                                                   topot_precision precision, const double* d_dirs, int D,
                                                   int per_image_dirs, const double* d_gout, double* d_gdirs,
                                                   void* stream);

/* Self-test of the bounded device-side waits.  Every spin of the library (extraction
 * look-back, wait for staged pixels) gives up after a time limit, records the timeout
 * and returns, so that a lost predecessor or copy becomes TOPOT_ERR_TIMEOUT rather than a
 * hung GPU.  This call makes one such wait run out on purpose, limited to limit_ms
 * (1 .. 10000): which = 0 spins on a device flag that nothing sets, which = 1 waits on an
 * mbarrier phase that never completes (no copy is issued).  Synchronous on `stream`.
 * Returns TOPOT_ERR_TIMEOUT when the wait ran out as designed; INVALID_ARG, CUDA. */
TOPOT_API topot_status topot_selftest_wait(int which, int limit_ms, void* stream);

/* Message of the last failed call on this thread ("" if none). */
TOPOT_API const char* topot_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TOPOT_H */
