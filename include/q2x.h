/*
 * q2x.h -- C ABI of the Q2X (quadrature-to-expansion) library for GB300.
 *
 * Q2X computes, for every simplex element (line segment, flat triangle,
 * tetrahedron) carrying a density, the multipole coefficients of its Laplace
 * layer potential about an expansion centre r*, up to degree p, and sums them
 * into one coefficient vector per octree leaf box (Sec. 2, Eq. (st4)):
 *
 *   K_n^m = J/(4pi) (-1)^n p_n^{-m}   segment,     single layer   Eq. (bas10)
 *   L_n^m = J/(4pi) (-1)^n i_n^{-m}   triangle,    single layer
 *   M_n^m = J/(4pi) (-1)^n l_n^{-m}   triangle,    double layer
 *   N_n^m = J/(4pi) (-1)^n a_n^{-m}   tetrahedron, single (volume) layer
 *
 * with R_n^m normalised as in Eq. (bas1), J the Jacobian of Eq. (map4) and
 * p_n^m, i_n^m, a_n^m the integrals of Eq. (bas9) of R_n^m(y - r*) over the
 * unit simplices.  They are computed by the paper's O(1)-per-moment recursions
 * (Lemmas 1-5, Eqs. (rec10)-(rec15)) in CUDA kernels for sm_103a.
 *
 * CONVENTIONS (all entry points)
 *  - Degree: p is the MAXIMUM degree kept, n = 0..p, so (p+1)^2 real numbers
 *    per expansion.  (The paper's truncation number counts degrees 0..p-1.)
 *  - Packing: real index k = n*n + n + m, -n <= m <= n.  Entry k holds
 *    Re F_n^m for m >= 0 and Im F_n^{|m|} for m < 0 (negative orders follow
 *    from F_n^{-m} = (-1)^m conj(F_n^m), Eq. (bas2.1); Im F_n^0 = 0).
 *  - Norm: Q2X_NORM_COEFF gives the coefficients above (expansion of the
 *    potential in S_n^m, Eq. (bas3)); Q2X_NORM_MOMENT gives the raw moments
 *    int density * R_n^m(y - r*) (double layer: int density * n.grad R_n^m).
 *  - Memory: every array pointer is DEVICE memory owned by the caller.  The
 *    plan owns its workspace.  SoA layouts:
 *      vxyz   double[3 * n_vert]    x block, then y block, then z block
 *      idx    int32 [k * n_elem]    vertex j of element e at idx[j*n_elem + e]
 *                                   (k = 2 segment, 3 triangle, 4 tetrahedron;
 *                                    vertex order x1, x2, x3[, x4] of Eq. (map2))
 *      leaf_off int64[n_leaves + 1] CSR: elements of leaf L are
 *                                   [leaf_off[L], leaf_off[L+1]); elements must
 *                                   be sorted by leaf; leaf_off[0] = 0,
 *                                   leaf_off[n_leaves] = n_elem
 *      leaf_c double[3 * n_leaves]  expansion centres r* (SoA)
 *      leaf_rho double[n_leaves]    length scale of each leaf (e.g. its
 *                                   half-diagonal or the largest distance from
 *                                   r* to a vertex); only the power of two
 *                                   above it is used, to keep the FP32 path in
 *                                   range.  NULL: computed from the geometry
 *      leaf_p int32[n_leaves]       per-leaf degree 0..p_max, NULL = p_max;
 *                                   entries above a leaf's degree are zero
 *      coef   double[n_leaves * (p_max+1)^2]   output, real packing
 *    leaf_off == NULL selects per-element expansions: n_leaves must equal
 *    n_elem and leaf_c holds one centre per element.
 *  - accumulate: 0 overwrites coef, 1 adds into it (several element kinds
 *    into the same leaves).
 *  - Streams: calls are asynchronous on the plan's stream.  Host-side argument
 *    checks return a status synchronously.  Device-side checks (vertex index
 *    out of range, non-finite input, bad leaf degree, bad leaf offsets) set a
 *    device error word; q2x_sync() reports it as
 *    Q2X_ERR_DEVICE_INPUT and clears it.  Invalid elements contribute zero.
 *  - No CPU fallback: without a usable CUDA device every call fails with
 *    Q2X_ERR_CUDA.  No exception crosses the ABI.
 *  - Thread safety: a plan may be used by one host thread at a time; distinct
 *    plans are independent.
 */
#ifndef Q2X_H
#define Q2X_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    Q2X_OK = 0,
    Q2X_ERR_ARG = 1,          /* bad argument (NULL pointer, negative size, ...) */
    Q2X_ERR_RANGE = 2,        /* p outside 0..Q2X_P_MAX or above the plan's p_max */
    Q2X_ERR_CUDA = 3,         /* a CUDA runtime call failed (message in q2x_last_error) */
    Q2X_ERR_OOM = 4,          /* workspace allocation failed */
    Q2X_ERR_DEVICE_INPUT = 5, /* the device error word was set by a previous call */
    Q2X_ERR_TIMEOUT = 6,      /* reserved: a bounded device wait gave up */
    Q2X_ERR_UNSUPPORTED = 7   /* combination not implemented */
} q2x_status;

typedef enum { Q2X_NORM_COEFF = 0, Q2X_NORM_MOMENT = 1 } q2x_norm;
typedef enum { Q2X_FP64 = 0, Q2X_FP32_MIXED = 1 } q2x_precision;
typedef enum { Q2X_DENSITY_CONST = 0, Q2X_DENSITY_LINEAR = 1 } q2x_density;

#define Q2X_P_MAX 20

/* Bits of the device error word (q2x_device_errors). */
#define Q2X_DEVERR_INDEX 1u      /* a vertex index outside [0, n_vert) */
#define Q2X_DEVERR_NONFINITE 2u  /* a non-finite coordinate, centre or density */
#define Q2X_DEVERR_LEAF_P 4u     /* leaf_p outside [0, p_max] */
#define Q2X_DEVERR_LEAF_OFF 8u   /* leaf_off not monotone or not spanning [0, n_elem] */

typedef struct q2x_plan_s* q2x_plan_t;

/* Create a plan for degrees up to p_max (0..Q2X_P_MAX) in the given norm and
 * precision, bound to a CUDA stream (cudaStream_t; NULL = legacy default
 * stream) on the current device.  Q2X_FP64 runs the whole recursion in FP64.
 * Q2X_FP32_MIXED runs it in FP32 in a per-leaf scaled local frame; the
 * translation to the leaf centre keeps FP64 accuracy (exact double -> float
 * splitting), per-leaf sums are FP32 with compensated combination of partial
 * sums, and the result is rescaled exactly into FP64.
 * Ownership: *out must be released with q2x_plan_destroy. */
q2x_status q2x_plan(q2x_plan_t* out, int p_max, q2x_norm norm, q2x_precision precision,
                    void* cuda_stream);
q2x_status q2x_plan_destroy(q2x_plan_t plan);
q2x_status q2x_plan_set_stream(q2x_plan_t plan, void* cuda_stream);

/* Last error message of this plan (static storage owned by the plan), or of
 * the last failed q2x_plan() call when plan == NULL. */
const char* q2x_last_error(q2x_plan_t plan);

/* Synchronise the plan's stream; return Q2X_ERR_DEVICE_INPUT (and clear the
 * word) if any device-side check failed since the last report. */
q2x_status q2x_sync(q2x_plan_t plan);
/* Synchronise and return the raw device error bits (Q2X_DEVERR_*), clearing them. */
q2x_status q2x_device_errors(q2x_plan_t plan, uint32_t* bits);

/* Pre-size the workspace for up to n_elem elements and n_leaves leaves so that
 * later calls of that size allocate nothing (needed before graph capture). */
q2x_status q2x_reserve(q2x_plan_t plan, int64_t n_elem, int64_t n_leaves);
/* Bytes of device workspace the plan currently holds. */
int64_t q2x_workspace_bytes(q2x_plan_t plan);

/* Profiling hooks.  q2x_plan_set_kernel_timing(plan, 1) makes the plan
 * bracket every element-kernel launch with a pair of its own CUDA events on its
 * stream; q2x_plan_kernel_timing() synchronises the stream, returns the summed
 * duration (ms) and number of the element-kernel launches timed since the
 * previous query, and resets both.  q2x_launch_count: number of CUDA kernels
 * this plan has launched since it was created (all of them: checks, element
 * kernels, fix-ups, reductions). */
q2x_status q2x_plan_set_kernel_timing(q2x_plan_t plan, int enable);
q2x_status q2x_plan_kernel_timing(q2x_plan_t plan, double* total_ms, int64_t* n_launches);
int64_t q2x_launch_count(q2x_plan_t plan);

/* Segments: K coefficients (Lemma 1, Eqs. (rec10)-(rec11)), constant line
 * density sigma[n_elem]; Jacobian |x2 - x1|. */
q2x_status q2x_segments(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                        const int32_t* idx, const double* sigma, int64_t n_leaves,
                        const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                        const int32_t* leaf_p, double* coef, int accumulate);

/* Triangles, single and/or double layer in ONE pass (Lemmas 2-3,
 * Eqs. (rec12)-(rec15)).  density Q2X_DENSITY_CONST: sigma[n_elem];
 * Q2X_DENSITY_LINEAR: sigma[n_vert] (value at each vertex, interpolated
 * linearly over the triangle).  coef_single (L) and/or coef_double (M) may be
 * NULL to skip that layer (not both).  The double-layer normal is
 * n = (x2 - x1) x (x3 - x1) / J (right-hand rule on the vertex order). */
q2x_status q2x_triangles(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                         const int32_t* idx, q2x_density density, const double* sigma,
                         int64_t n_leaves, const int64_t* leaf_off, const double* leaf_c,
                         const double* leaf_rho, const int32_t* leaf_p, double* coef_single,
                         double* coef_double, int accumulate);
q2x_status q2x_triangles_single(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                const double* vxyz, const int32_t* idx, q2x_density density,
                                const double* sigma, int64_t n_leaves, const int64_t* leaf_off,
                                const double* leaf_c, const double* leaf_rho,
                                const int32_t* leaf_p, double* coef, int accumulate);
q2x_status q2x_triangles_double(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                const double* vxyz, const int32_t* idx, q2x_density density,
                                const double* sigma, int64_t n_leaves, const int64_t* leaf_off,
                                const double* leaf_c, const double* leaf_rho,
                                const int32_t* leaf_p, double* coef, int accumulate);

/* Tetrahedra: N coefficients (Lemmas 4-5, Eqs. (rec14.1)-(rec14.2)),
 * constant volume density sigma[n_elem]; Jacobian |(Ru x Rv).Rw|. */
q2x_status q2x_tetra(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                     const int32_t* idx, const double* sigma, int64_t n_leaves,
                     const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                     const int32_t* leaf_p, double* coef, int accumulate);

/* Triangles without any device allocation.  There is no counterpart in the
 * paper: this is a deployment variant of q2x_triangles for callers that cannot
 * call cudaMalloc -- solvers that have handed all device memory to their own
 * pool, code paths that must never synchronise the device (cudaMalloc and
 * cudaFree may synchronise), and callers that must not meet an out-of-memory
 * failure at call time.  It takes no plan: the degree bound, norm, precision
 * and stream come as arguments; the remaining arguments and layouts are those
 * of q2x_triangles (leaf mode only: leaf_off is required, and leaf_rho is
 * required in Q2X_FP32_MIXED).
 * Scratch: the partial sums of leaves that straddle warp ranges live in one
 * file-scope device array of Q2X_NOALLOC_SCRATCH_BYTES (16 MiB), which every
 * GPU that loads the library holds until the process exits.  Each warp range
 * covers Q2X_NOALLOC_RANGE elements and needs 4 (p_max+1)^2 8 bytes (FP64
 * partial sums in both precisions), so the call accepts
 *   n_elem <= Q2X_NOALLOC_RANGE * floor(Q2X_NOALLOC_SCRATCH_BYTES / (32 (p_max+1)^2))
 * (e.g. 794,112 triangles at p_max = 12) and returns Q2X_ERR_RANGE above
 * that, having launched nothing.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it: make that
 * first call before any stream capture.  cuda_stream must belong to the
 * current device (Q2X_ERR_ARG otherwise).  Every call shares the array; calls
 * that overlap on the GPU race on it and on the device error word.  Device-side
 * input checks are not reported by this entry point: an invalid element
 * contributes zero, and a leaf_off that is not non-decreasing from 0 to n_elem
 * gives undefined coefficients (every memory access stays in bounds).
 * Asynchronous on cuda_stream; no allocation, no synchronisation. */
#define Q2X_NOALLOC_SCRATCH_BYTES (16u << 20)
#define Q2X_NOALLOC_RANGE 256
q2x_status q2x_triangles_noalloc(int p_max, q2x_norm norm, q2x_precision precision,
                                 void* cuda_stream, int64_t n_elem, int64_t n_vert,
                                 const double* vxyz, const int32_t* idx, q2x_density density,
                                 const double* sigma, int64_t n_leaves, const int64_t* leaf_off,
                                 const double* leaf_c, const double* leaf_rho,
                                 const int32_t* leaf_p, double* coef_single, double* coef_double,
                                 int accumulate);

/* Adjoint of q2x_triangles_single with constant density (the derivative of
 * loss = sum_{leaves, c} grad_coef[L][c] * coef[L][c] with respect to the
 * vertex coordinates and the densities).  Derived from Eq. (bas10) and the
 * derivative rules of Eq. (bas5)-(bas8): d coef / d x_k is a Jacobian term
 * plus J * int lambda_k grad R_n^{-m}, and each component of the latter is a
 * double-layer moment (Eq. (rec15)) with a coordinate axis as the normal and
 * the barycentric weight lambda_k of vertex k as a linear density.
 *   grad_coef  double[n_leaves * (p_max+1)^2]  (device, read)
 *   grad_vxyz  double[3 * n_vert] SoA (device): d loss / d vxyz is ADDED
 *              (FP64 atomic accumulation over the elements sharing a vertex;
 *              the summation order is not fixed)
 *   grad_sigma double[n_elem] (device) or NULL: d loss / d sigma, overwritten
 * Other arguments as in q2x_triangles_single.  In Q2X_FP32_MIXED the
 * per-element sums run in FP32 (weights rho^{n+1} G, which flush to zero
 * below the FP32 range), the accumulation into grad_vxyz in FP64. */
q2x_status q2x_triangles_single_vjp(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                    const double* vxyz, const int32_t* idx, const double* sigma,
                                    int64_t n_leaves, const int64_t* leaf_off,
                                    const double* leaf_c, const double* leaf_rho,
                                    const int32_t* leaf_p, const double* grad_coef,
                                    double* grad_vxyz, double* grad_sigma);

/* ---- Ragged mixed batch in one CUDA-graph replay -----------------------
 * Several element kinds (segments, triangles, tetrahedra) share one leaf set;
 * every leaf has its own degree p_leaf <= p_max and its own element counts.
 * q2x_batch_build (a set-up call: it copies leaf_p and the leaf offsets to the
 * host, allocates the batch's device memory and synchronises) cuts the work
 * into tiles of at most tile_elems elements of one kind inside one leaf,
 * orders them (by degree bin, kind and cost, most expensive first) and captures
 * [counter reset, one persistent kernel per (kind, degree bin) group of tiles,
 * per-leaf combine] in a CUDA graph.  q2x_batch_run replays that graph on the plan's stream: coef
 * (n_leaves x (p_max+1)^2) receives, per leaf, the sum of the single-layer
 * coefficients of all its elements of all kinds (zero above p_leaf), added in
 * a fixed order.  The descriptor's device arrays must stay valid and
 * unchanged in shape while the batch exists; their values may change between
 * runs.  tile_elems <= 0 picks the default (256).  Triangles may carry
 * constant or linear density; double layers are not part of a batch.
 * leaf_rho is required in Q2X_FP32_MIXED. */
typedef struct {
    int64_t n_elem;           /* 0: kind absent */
    int64_t n_vert;
    const double* vxyz;       /* SoA 3 x n_vert */
    const int32_t* idx;       /* SoA k x n_elem */
    const double* sigma;      /* n_elem, or n_vert for linear-density triangles */
    const int64_t* leaf_off;  /* CSR over the batch's leaves, n_leaves + 1 entries */
    q2x_density density;      /* triangles only */
} q2x_batch_elements;

typedef struct {
    int64_t n_leaves;
    const double* leaf_c;     /* SoA 3 x n_leaves */
    const double* leaf_rho;   /* n_leaves */
    const int32_t* leaf_p;    /* n_leaves, degrees 0..p_max; NULL = p_max */
    q2x_batch_elements segments, triangles, tetra;
    double* coef;             /* n_leaves x (p_max+1)^2 */
    int accumulate;
} q2x_batch_desc;

typedef struct q2x_batch_s* q2x_batch_t;

q2x_status q2x_batch_build(q2x_plan_t plan, const q2x_batch_desc* desc, int tile_elems, q2x_batch_t* out);
q2x_status q2x_batch_run(q2x_batch_t batch);
q2x_status q2x_batch_destroy(q2x_batch_t batch);
/* Number of tiles and of partial rows of a built batch. */
q2x_status q2x_batch_info(q2x_batch_t batch, int64_t* n_tiles, int64_t* n_slots, int* tile_elems);

/* Autotuner: build the batch with each candidate tile size, time reps graph
 * replays of each (CUDA events on the plan's stream, after one warm-up), and
 * return the fastest candidate in *best and the mean time of every candidate
 * in ms[n_candidates].  The caller persists the choice (the Python binding
 * keeps a JSON table keyed by device and workload shape). */
q2x_status q2x_batch_tune(q2x_plan_t plan, const q2x_batch_desc* desc, const int* candidates,
                          int n_candidates, int reps, int* best, float* ms);

/* Translation of expansions to new centres: the multipole-to-multipole step
 * that consumes the leaf coefficients (the paper stops at Eq. (st4); the
 * formula follows from the derivative rules of Eq. (bas5), whose Taylor
 * series gives R_n^m(x + t) = sum_{k<=n} sum_{|l|<=k} R_k^l(t) R_{n-k}^{m-l}(x)):
 *   COEFF : F_n^m(dst) = sum_{k,l} (-1)^k R_k^l(t) F_{n-k}^{m+l}(src)
 *   MOMENT: M_n^m(dst) = sum_{k,l} R_k^l(t) M_{n-k}^{m-l}(src)
 * with t = src centre - dst centre; exact for every degree n <= p (no
 * truncation), single and double layer alike.  The plan's norm selects the
 * formula.
 *   p          degree, 0..the plan's p_max; every row has (p+1)^2 entries
 *   src_coef   double[n_src * (p+1)^2], packed like coef above (device)
 *   src_c      double[3 * n_src] SoA source centres (device)
 *   dst_off    int64[n_dst + 1] CSR: destination d receives the sources
 *              dst_off[d] .. dst_off[d+1]-1 (device); a bad range sets the
 *              device error word (bit 8) and that destination gets zeros
 *   dst_c      double[3 * n_dst] SoA destination centres (device)
 *   dst_coef   double[n_dst * (p+1)^2] (device): overwritten, or added to
 *              with accumulate = 1
 * Sums run in source order (deterministic).  FP64 arithmetic in both
 * precisions of the plan.  One upward pass of an octree is one call per
 * level (children -> parents). */
q2x_status q2x_translate(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef,
                         const double* src_c, int64_t n_dst, const int64_t* dst_off,
                         const double* dst_c, double* dst_coef, int accumulate);

/* The solid harmonics R_n^m(t), n <= p, of n_t translation vectors t
 * (double[3 * n_t] SoA, device) into rt (double[n_t * (p+1)^2], device),
 * packed like the coefficients: Re R_n^m at n^2+n+m for m >= 0 and
 * Im R_n^|m| at n^2+n-|m| (R_n^{-m} = (-1)^m conj R_n^m).  Built by the
 * point recursion of Eq. (rec2), as q2x_translate does per source; a tree
 * whose shifts are fixed computes them once (an octree level has eight).
 * FP64; p <= the plan's p_max. */
q2x_status q2x_translation_rows(q2x_plan_t plan, int p, int64_t n_t, const double* t, double* rt);

/* q2x_translate with R(t) read from precomputed rows instead of built per
 * source: source s uses row t_idx[s] (int32, device) of rt (n_t rows from
 * q2x_translation_rows), which must hold R(c_src - c_dst) for the source's
 * destination; the centres are then not needed.  An index outside
 * [0, n_t) sets bit 1 of the device error word and that source adds zero.
 * Other arguments and the results as q2x_translate (up to the rounding of
 * R_n^{-m} taken from R_n^m). */
q2x_status q2x_translate_rt(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef, int64_t n_t,
                            const double* rt, const int32_t* t_idx, int64_t n_dst, const int64_t* dst_off,
                            double* dst_coef, int accumulate);

/* Far-field evaluation (the M2P step fed by the leaf or box coefficients):
 * out[t] (+)= sum over the expansions e listed for target t of
 *   phi_e(x_t) = sum_{n<=p} sum_{|m|<=n} F_n^m S_n^m(x_t - c_e)      (Eq. (bas3))
 * with F the COEFF coefficients, or (1/4pi)(-1)^n M_n^{-m} for MOMENT
 * coefficients (the plan's norm).  The value is real (Eq. (bas2.1)); the
 * series converges for |x_t - c_e| larger than the expansion's radius, and
 * an expansion evaluated exactly at its centre contributes 0.
 *   coef     double[n_exp * (p+1)^2] packed (device); exp_c double[3 * n_exp] SoA
 *   tgt      double[3 * n_tgt] SoA target points (device)
 *   tgt_off  int64[n_tgt + 1] CSR into exp_idx (device); exp_idx int64 list of
 *            expansion indices (device; may be NULL when every list is
 *            empty); an index out of range sets the device error word (bit 1)
 *            and is skipped, a bad range (or a non-empty list with exp_idx
 *            NULL) sets bit 8 and the target gets 0
 *   out      double[n_tgt] (device), overwritten or added to (accumulate = 1)
 * FP64 arithmetic in both precisions of the plan; S_n^m by the
 * associated-Legendre recurrences in Cartesian form (Eqs. (bas1)-(bas2)). */
q2x_status q2x_evaluate(q2x_plan_t plan, int p, int64_t n_exp, const double* coef, const double* exp_c,
                        int64_t n_tgt, const double* tgt, const int64_t* tgt_off, const int64_t* exp_idx,
                        double* out, int accumulate);

/* Curl of the far field of vector expansions (Biot-Savart, Eq. (st3)):
 * expansion e has three component rows F^(k) (k = x, y, z), e.g. segment
 * coefficients computed with the components of a vector line density as
 * sigma; A_k(x) = sum_{n,m} F^(k)_n^m S_n^m(x - c_e) and
 *   out3[d][t] (+)= (curl A)_d at target t, summed over the listed expansions,
 * i.e. H(x) = (1/4pi) int I x (x - y)/|x - y|^3 dl for line currents I.
 *   coef3   double[3 * n_exp * (p+1)^2]: component-major [3][n_exp][np] (device)
 *   out3    double[3 * n_tgt] SoA (device)
 * Other arguments as q2x_evaluate.  The gradients of S_n^m are carried
 * through the same recurrences in forward mode (no derivative tables).  COEFF
 * norm only (Q2X_ERR_UNSUPPORTED otherwise).  FP64. */
q2x_status q2x_evaluate_curl(q2x_plan_t plan, int p, int64_t n_exp, const double* coef3, const double* exp_c,
                             int64_t n_tgt, const double* tgt, const int64_t* tgt_off, const int64_t* exp_idx,
                             double* out3, int accumulate);

/* Near field: exact potentials of constant-density elements at targets,
 *   out[t] (+)= sum over the elements e listed for target t of
 *               sigma[e] / (4 pi) * int_e 1/|r_t - y| dmu(y)          (layer 0)
 *               sigma[e] / (4 pi) * int_e n.(r_t - y)/|r_t - y|^3 dS   (layer 1,
 *               triangles: the double-layer kernel, a signed solid angle)
 * by the closed forms of Sec. 4.1 (Eqs. (num1)-(num3) for segments, the
 * edge-sum form of Eq. (num5) for flat triangles, the divergence-theorem face sum of
 * Eqs. (num7)-(num8) for tetrahedra).  kind 0 segment, 1 triangle, 2
 * tetrahedron; vxyz, idx, sigma (per element) as q2x_segments/-triangles/
 * -tetra; tgt double[3 * n_tgt] SoA; tgt_off int64[n_tgt + 1] CSR into the
 * element list elem_idx (int64; may be NULL when every list is empty); out
 * double[n_tgt], overwritten or added to (accumulate = 1); all device
 * arrays.  Targets on an element are handled where the integral exists
 * (vertices and edges of a triangle, and any point of a tetrahedron, give
 * finite values; a target inside a segment gives inf).  A target within
 * rounding of a triangle's plane is taken in it, where the double layer
 * has its direct value 0.  An element or vertex index out of range sets
 * the device error word (bit 1) and the element is skipped; a bad range
 * (or a non-empty list with elem_idx NULL) sets bit 8 and the target gets
 * 0.  Errors: Q2X_ERR_UNSUPPORTED for layer 1 with kind != 1, Q2X_ERR_ARG
 * for bad kinds, sizes or NULL arrays.  Launches one frame kernel (kinds 1,
 * 2; the face frames live in the plan's workspace) and one target kernel on
 * the plan's stream.  FP64. */
q2x_status q2x_nearfield(q2x_plan_t plan, int kind, int layer, int64_t n_elem, int64_t n_vert,
                         const double* vxyz, const int32_t* idx, const double* sigma, int64_t n_tgt,
                         const double* tgt, const int64_t* tgt_off, const int64_t* elem_idx, double* out,
                         int accumulate);

/* Receiver-side (Galerkin) integration over triangles: for every triangle e
 * of leaf L,
 *   out[e] = sum_c w[L][c] P_c(e),
 * P(e) the packed coefficients of triangle e alone with constant density
 * sigma[e] (layer 0: single layer, Eq. (bas4); layer 1: double layer, with
 * n.grad) in the plan's norm, about leaf L's centre, up to the plan's p_max.
 * With the MOMENT norm and the weights of a local expansion
 * phi(y) = sum_{n,m} L_n^m R_n^m(y - c) (w = L_n^0 at (n, 0), 2 Re L_n^m at
 * (n, m > 0), -2 Im L_n^m at (n, -m)), out[e] is the integral of
 * sigma[e] phi (layer 0) or sigma[e] n.grad phi (layer 1) over the triangle,
 * i.e. the receiving side of a Galerkin boundary-element FMM.  Computed by
 * the same recursions as the Q2X element kernels (Lemmas 2-3), contracted per
 * element instead of summed per leaf.
 *   vxyz, idx, sigma, leaf_off, leaf_c, leaf_rho: as q2x_triangles_single
 *   (sigma required: the per-element weights)
 *   w    double[n_leaves * (p_max+1)^2] (device)
 *   out  double[n_elem] (device), overwritten
 * FP64 arithmetic in both precisions of the plan; deterministic. */
q2x_status q2x_galerkin_triangles(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                                  const int32_t* idx, const double* sigma, int64_t n_leaves,
                                  const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                                  int layer, const double* w, double* out);

/* Segmented sum of per-element coefficient rows into leaves (Eq. (st4)):
 * coef[L] (+)= sum_{e in leaf L} elem[e], elem double[n_elem * (p+1)^2],
 * coef double[n_leaves * (p+1)^2], leaf_off as above (required).  FP64,
 * deterministic (fixed summation order).  p <= the plan's p_max. */
q2x_status q2x_leaf_reduce(q2x_plan_t plan, int64_t n_elem, int p, const double* elem,
                           int64_t n_leaves, const int64_t* leaf_off, double* coef,
                           int accumulate);

/* Vector line density (Eq. (st3)): the coefficients of the three components
 * of a current constant per segment, current double[3 * n_elem] (component
 * j at current + j * n_elem), into coef3 double[3 * n_leaves * (p_max+1)^2]
 * (component j's block at coef3 + j * n_leaves * (p_max+1)^2), otherwise the
 * arguments of q2x_segments (leaf_off required).  The moments are geometric
 * and each component multiplies them, so the recursion runs once per
 * element, with unit density: each round's moments are staged once and summed
 * per leaf three times, weighted by the components (one pass of the element
 * kernel; no temporary beyond the plan workspace).  Same results as three
 * q2x_segments calls with the components as densities, up to rounding;
 * deterministic.  A non-finite component sets Q2X_DEVERR_NONFINITE and its
 * segment contributes zero. */
q2x_status q2x_segments_vector(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                               const int32_t* idx, const double* current, int64_t n_leaves,
                               const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                               const int32_t* leaf_p, double* coef3, int accumulate);

/* Weighted segmented sums of per-element rows, n_w components at once
 * (1 <= n_w <= 4):
 *   coef[j][L] (+)= sum_{e in leaf L} w[j][e] * elem[e],   j < n_w,
 * component j's weights at w + j * w_stride (n_elem doubles each) and its
 * output block (n_leaves * (p+1)^2 doubles) at coef + j * coef_stride.  With
 * the unit-density moments of each element as elem, these are the
 * coefficients of a vector density (Eq. (st3): the moments are geometric and
 * each component multiplies them), so the three components of a line
 * current share one recursion pass.  FP64, deterministic (each sum in
 * element order, one FMA per element); leaf_off as above (required; a bad
 * range sets bit 8 of the device error word and is clamped). */
q2x_status q2x_leaf_reduce_weighted(q2x_plan_t plan, int64_t n_elem, int p, const double* elem, int n_w,
                                    const double* w, int64_t w_stride, int64_t n_leaves,
                                    const int64_t* leaf_off, double* coef, int64_t coef_stride,
                                    int accumulate);

/* ---- Measurement aid (no counterpart in the paper) ----------------------
 * ALU peak probe: the element kernels are bound by the FP64 or FP32 FMA
 * pipes, so their roofline divides by the FMA rate this device actually
 * sustains.  One launch, asynchronous on cuda_stream (cudaStream_t, NULL =
 * legacy default stream) of the current device, of 4 CTAs x 256 threads per
 * SM, each thread running 8 independent chains x <- a x + b for iters steps
 * (rounded up to a multiple of 16):
 *   Q2X_PEAK_DFMA   FP64 fma            2 flops per FMA
 *   Q2X_PEAK_FFMA   FP32 fma            2 flops per FMA
 *   Q2X_PEAK_FFMA2  packed fma.rn.f32x2 4 flops per instruction
 * *flops (host) receives the floating-point operations the launch performs;
 * the caller times the launch with CUDA events on the same stream.
 * sink: device double[1], written only if a chain sum takes a value it never
 * takes (it keeps the chains live; nothing is stored in practice).
 * Q2X_ERR_ARG for a bad kind, iters outside 1..2^40 or a NULL pointer. */
typedef enum { Q2X_PEAK_DFMA = 0, Q2X_PEAK_FFMA = 1, Q2X_PEAK_FFMA2 = 2 } q2x_peak_kind;
q2x_status q2x_alu_peak_probe(int kind, int64_t iters, double* sink, void* cuda_stream, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* Q2X_H */
