/*
 * fmm.h -- C ABI of a single-GPU fast multipole method for the 3-D Laplace
 * (1/r) kernel on NVIDIA GB300 (sm_103a).
 *
 * The method is the FMM of Yokota & Barba, "A Tuned and Scalable Fast
 * Multipole Method as a Preeminent Algorithm for Exascale Systems"
 * (arXiv:1106.2176): a Morton-indexed octree (Sec. 2.2, Sec. 5), multipole and
 * local expansions of p terms (Sec. 2.1), the operators P2M,
 * M2M, M2L, L2L, L2P and the direct near-field P2P (Sec. 2.1, Fig.
 * flow_chart; Sec. 3.1 names P2P and M2L as the dominant kernels).
 *
 * Given N particles x_i with charges q_i the library computes
 *     phi_i  = sum_{j != i, r_ij > 0} q_j / |x_i - x_j|
 *     grad_i = d phi_i / d x_i = - sum_{j != i, r_ij > 0} q_j (x_i - x_j) / |x_i - x_j|^3
 * to the accuracy set by p and theta (no 1/(4 pi) factor, no softening;
 * coincident pairs contribute nothing).
 *
 * Conventions shared by every entry point:
 *   - Return value: FMM_OK (0) on success, a negative FMM_E* code on error.
 *     No C++ exception crosses this boundary. fmm_last_error() gives a
 *     message for the calling thread.
 *   - Pointers to particle data are device pointers unless FMM_HOST_MEM is
 *     OR-ed into the dtype argument of fmm_build; then x, q and the outputs
 *     of fmm_evaluate are host pointers and the library copies them.
 *   - The caller owns x, q, phi and grad. The handle owns every workspace;
 *     fmm_destroy frees them. fmm_build copies what it needs, so x and q may
 *     be reused once the handle's stream has passed the build.
 *   - All device work is asynchronous on the handle's stream (the legacy
 *     default stream unless fmm_set_stream was called). fmm_build makes a
 *     few host synchronisations to size the tree and the lists; fmm_evaluate
 *     with device pointers makes none.
 *   - A handle is not thread safe; use one handle per thread.
 */
#ifndef FMM_H
#define FMM_H

#include <stdint.h>

#if defined(__GNUC__)
#define FMM_API __attribute__((visibility("default")))
#else
#define FMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx *fmm_handle;
typedef struct fmm_batch_s *fmm_batch;

/* status codes */
enum {
    FMM_OK = 0,
    FMM_EINVAL = -1,     /* bad argument (null pointer, size or range) */
    FMM_ENOMEM = -2,     /* device or host allocation failed */
    FMM_ESTATE = -3,     /* call out of order, e.g. evaluate before build */
    FMM_ECUDA = -4,      /* a CUDA runtime call or kernel launch failed */
    FMM_ENONFINITE = -5, /* a position is NaN or infinite */
    FMM_ENODEV = -6      /* no usable sm_103 device */
};

/* element types of x, q, phi, grad; FMM_HOST_MEM may be OR-ed in */
enum { FMM_F32 = 0, FMM_F64 = 1, FMM_HOST_MEM = 0x100 };

/* arithmetic of the evaluation */
enum {
    FMM_FP64 = 0,  /* every stage in FP64 (the on-device reference path) */
    FMM_MIXED = 1  /* FP32 P2P and expansions, M2L on the tensor cores in
                      split TF32 with FP32 accumulation (p <= 11; FP32
                      rotation M2L above), FP64 tree, FP64 offsets and final
                      sums */
};

/* M2L engine of the same-level pairs (fmm_set_m2l_engine) */
enum { FMM_M2L_AUTO = 0, FMM_M2L_TENSOR = 1, FMM_M2L_CUDACORE = 2, FMM_M2L_ROTATION = 3 };

/* arithmetic pipes fmm_measure_peak can time */
enum {
    FMM_PEAK_FP32_FMA = 0,   /* scalar FP32 FMA on the CUDA cores */
    FMM_PEAK_FP32X2_FMA = 1, /* packed FP32 pair FMA (fma.rn.f32x2), 4 flop per instruction */
    FMM_PEAK_TF32_MMA = 2    /* tcgen05.mma kind::tf32, FP32 accumulator in tensor memory */
};

typedef struct {
    int64_t n;              /* particles of the last build */
    int64_t ncells;         /* cells of the tree */
    int64_t nleaves;
    int32_t depth;          /* deepest level */
    int32_t precision;      /* FMM_FP64 or FMM_MIXED */
    int64_t n_p2p_pairs;    /* leaf pairs in the P2P lists, (A, A) included */
    int64_t n_m2l_pairs;    /* accepted cell pairs, same-level and other */
    int64_t n_m2l_irregular;/* accepted pairs whose cells sit on different levels */
    int64_t n_interactions; /* sum over P2P pairs of n_A * n_B, minus n */
    int64_t n_stencil;      /* same-level M2L translation vectors (all octants) */
    int32_t m2l_engine;     /* engine used by the last evaluate */
    int32_t async_error;    /* nonzero if a device-side wait of the last evaluate timed out */
    /* milliseconds of the last build / evaluate, measured with CUDA events */
    double ms_build, ms_evaluate;
    double ms_p2m, ms_m2m, ms_m2l, ms_l2l, ms_l2p, ms_p2p, ms_combine;
    int64_t kernel_launches; /* kernels this handle launched since creation */
    int32_t uniform_path;    /* 1 if the last build took the full-octree fast path */
    int32_t lattice_levels;  /* bit l: level l's M2L sources come by TMA tile loads (fmm_set_m2l_lattice) */
} fmm_stats;

/* Sizes of the arrays fmm_export_tree writes. */
typedef struct {
    int64_t n, ncells, n_p2p, n_m2l;
    int32_t depth, p;
} fmm_tree_sizes;

/*
 * Create a handle for up to N particles with expansions of p terms (degrees
 * 0..p-1, Sec. 2.1), multipole acceptance parameter theta and leaf size
 * ncrit. Limits: N >= 1, 1 <= p <= 20, 0 < theta < 1, ncrit >= 1. The cell
 * accepted for M2L against cell B when r_A + r_B < theta |c_A - c_B|, r the
 * half diagonal of the box. Precomputes the level-independent translation
 * operators. Returns FMM_EINVAL, FMM_ENODEV, FMM_ENOMEM or FMM_ECUDA on error;
 * *out is set to NULL then.
 */
FMM_API int fmm_create(int64_t N, int p, double theta, int ncrit, fmm_handle *out);

/* Select FMM_FP64 (default) or FMM_MIXED. Takes effect at the next build. */
FMM_API int fmm_set_precision(fmm_handle h, int mode);

/* Select the M2L engine; takes effect at the next build. FMM_M2L_AUTO: the
 * tensor cores for FMM_MIXED with p <= 11, otherwise rotation for p <= 16
 * (FP64 included), otherwise the CUDA-core dense contraction. FMM_M2L_TENSOR: split-TF32 tcgen05 contraction (FMM_MIXED,
 * p <= 11). FMM_M2L_CUDACORE: dense O(p^4) contraction on the CUDA cores.
 * FMM_M2L_ROTATION: rotate each translation onto the z axis, translate along
 * z and rotate back, O(p^3) per pair (either precision, p <= 16). The
 * different-level pairs of adaptive trees always take the per-pair kernel.
 * Returns FMM_EINVAL for an unknown engine or one that does not support p. */
FMM_API int fmm_set_m2l_engine(fmm_handle h, int engine);

/* Scheduling of fmm_evaluate. on = 1 (default): the far field (P2M .. L2P)
 * and the near field (P2P) run concurrently on two library streams, joined
 * back to the caller's stream before the combine. on = 0: both run in turn on
 * the caller's stream, so the phase times in fmm_stats are those of each
 * phase alone. Results are bitwise the same either way. The paper runs the two
 * in turn on one device; this is an addition. Returns FMM_EINVAL for a NULL
 * handle or on not 0/1. */
FMM_API int fmm_set_overlap(fmm_handle h, int on);

/* Uniform-tree fast path (Sec. 5: for uniform distributions the cells of a
 * level and the interaction lists follow from the Morton index alone).
 * on = 1 (default): when the cell build yields a full octree (every leaf on
 * the deepest level L and every level full), fmm_build skips the dual
 * traversal: the P2P rows of the leaves come from the near-field lattice
 * stencil of level L (the offsets the MAC rejects, cut at the lattice
 * boundary, ancestors checked as the traversal does), there are no pairs
 * across levels, and the implicit same-level M2L pairs are counted in closed
 * form. The lists, and so the results, are identical to the traversal's.
 * on = 0: always traverse. Takes effect at the next build; fmm_stats
 * .uniform_path says which path the last build took. Returns FMM_EINVAL for a
 * NULL handle or on not 0/1. */
FMM_API int fmm_set_uniform_path(fmm_handle h, int on);

/*
 * Same-level M2L tiles (the tensor-core and dense engines): tiles hold the
 * cells of one level and one octant, except on levels with at most max_cells
 * cells, which are pooled over the 8 octants into tiles that walk the union
 * of the 8 stencils (fuller tiles, longer walks; Sec. 5's grouping of work
 * into large, contiguous pieces). max_cells = -1: the default, 4 tiles' worth
 * (512 cells for the tensor-core engine); 0: no pooling. Takes effect at the
 * next build. Returns FMM_EINVAL for a NULL handle or max_cells < -1.
 */
FMM_API int fmm_set_m2l_pool(fmm_handle h, int max_cells);

/*
 * Sources of the tensor-core M2L on complete levels (Sec. 2.2: every box of a
 * level present, boxes indexed by lattice position). on = 1 (default): on a
 * complete level with at least 8^4 cells (above the pooling threshold, at
 * most level 9) each evaluation first copies the level's M~ into lattice
 * order (octant bits, then z, y, x of the halved position), and the kernel
 * brings a tile's sources for one translation as TMA tile loads of a shifted
 * block, positions outside the level as zeros; no per-row lookups or row
 * gathers. on = 0: per-row lookups and gathers on every level. The results
 * are bitwise the same. Takes effect at the next build; fmm_stats
 * .lattice_levels says which levels the last build set up (bit l: level l).
 * Returns FMM_EINVAL for a NULL handle or on not 0/1.
 */
FMM_API int fmm_set_m2l_lattice(fmm_handle h, int on);

/* Use the given cudaStream_t (NULL = legacy default stream) for all work. */
FMM_API int fmm_set_stream(fmm_handle h, void *stream);

/*
 * Build the octree and the interaction lists (Sec. 2.1 hierarchical
 * subdivision into near and far; Sec. 2.2 Morton-indexed boxes; Sec. 5
 * sorted indices with start/offset ranges).
 *   x: n*3 positions, row-major (x0 y0 z0 x1 ...); q: n charges;
 *   dtype: FMM_F32 or FMM_F64, optionally | FMM_HOST_MEM;
 *   1 <= n <= N of fmm_create.
 * Errors: FMM_EINVAL (null pointer, n out of range, bad dtype),
 * FMM_ENONFINITE (a coordinate is NaN or infinite), FMM_ENOMEM, FMM_ECUDA.
 */
FMM_API int fmm_build(fmm_handle h, const void *x, const void *q, int64_t n, int dtype);

/*
 * Evaluate the potential and its gradient at every particle of the last
 * build, in the caller's particle order (Sec. 2.1, Fig. flow_chart: P2M,
 * M2M, M2L, L2L, L2P and P2P).
 *   phi: n values; grad: n*3 values row-major, or NULL to skip the gradient
 *   (it is computed anyway). Element type and memory kind are the build's.
 * Errors: FMM_ESTATE (no successful build), FMM_EINVAL, FMM_ECUDA.
 */
FMM_API int fmm_evaluate(fmm_handle h, void *phi, void *grad);

/* Weighted energy and its adjoint (differentiation of the evaluation).
 *
 * The paper evaluates potentials and forces (Sec. 2); these calls add the
 * derivatives of the weighted energy E = 1/2 sum_i w_i q_i phi_i. The Laplace
 * kernel is symmetric, so with psi the potential of the charges w_j q_j at the
 * same positions:
 *   dE/dq_k = 1/2 (w_k phi_k + psi_k),
 *   dE/dx_k = 1/2 q_k (w_k grad phi_k + grad psi_k),
 *   dE/dw_k = 1/2 q_k phi_k.
 * psi comes from one more evaluation on the same tree: fmm_update_charges(h,
 * q, w) then fmm_evaluate. */

/* Replace the charges of the built tree by q (times w if w is not NULL), in
 * the caller's order, same dtype and memory kind as at build; the positions and
 * the tree stay. The next fmm_evaluate uses them. Returns FMM_ESTATE before a
 * build, FMM_EINVAL for NULL h or q. */
FMM_API int fmm_update_charges(fmm_handle h, const void *q, const void *w);

/* *out = 1/2 sum_i w_i q_i phi_i over the built n particles, summed in FP64 in
 * a fixed order. w, q, phi: device arrays of the build's dtype, caller's order.
 * Returns FMM_ESTATE before a build, FMM_EINVAL on NULL arguments or a
 * host-memory build. Synchronises the stream. */
FMM_API int fmm_energy(fmm_handle h, const void *w, const void *q, const void *phi, double *out);

/* Adjoint of fmm_energy scaled by gE: dq = gE dE/dq, dx = gE dE/dx (n x 3),
 * dw = gE dE/dw, from phi, grad (the evaluation with charges q) and psi, gpsi
 * (the evaluation with charges w q). Device arrays of the build's dtype,
 * caller's order; any of dq, dx, dw may be NULL (dx needs grad and gpsi).
 * Returns FMM_ESTATE before a build, FMM_EINVAL on NULL inputs or a
 * host-memory build. */
FMM_API int fmm_energy_adjoint(fmm_handle h, double gE, const void *w, const void *q, const void *phi,
                               const void *grad, const void *psi, const void *gpsi, void *dq, void *dx, void *dw);

/* Counters and phase timings of the last build and evaluate; synchronises
 * the handle's stream. */
FMM_API int fmm_get_stats(fmm_handle h, fmm_stats *out);

/* The same counters, with each phase time (ms_*) the mean over the last k
 * builds and the last k evaluations of the handle (1 <= k <= 32, and at most
 * the number of builds and of evaluations done; FMM_EINVAL otherwise). The
 * handle records the CUDA events of its 32 most recent builds and evaluations
 * on the streams that launch each phase, so a timed loop of builds and
 * evaluations needs no host synchronisation to be broken down by phase
 * afterwards. Synchronises the handle's streams. */
FMM_API int fmm_get_stats_mean(fmm_handle h, int k, fmm_stats *out);

/* Sizes of the arrays written by fmm_export_tree (after a build). */
FMM_API int fmm_get_tree_sizes(fmm_handle h, fmm_tree_sizes *out);

/*
 * Copy the tree and the lists of the last build to HOST buffers (any may be
 * NULL). Sizes from fmm_get_tree_sizes. Used to check the GPU tree bit for
 * bit against an independent implementation.
 *   keys[n]       sorted 63-bit Morton keys
 *   perm[n]       perm[k] = input index of the k-th sorted particle
 *   level[ncells], anchor[ncells] (Morton key of the cell's lowest corner),
 *   begin[ncells], end[ncells] (sorted particle range), child[ncells]
 *   (first child or -1), nchild[ncells], parent[ncells] (-1 for the root);
 *   cells in breadth-first order, key order within a level
 *   p2p_ptr[ncells+1], p2p_idx[n_p2p]: CSR by target cell, sources ascending
 *   m2l_ptr[ncells+1], m2l_idx[n_m2l]: CSR by target cell, sources ascending
 *   box[4]: origin x, y, z of the root cube and its half width R0
 * Synchronises the handle's stream.
 */
FMM_API int fmm_export_tree(fmm_handle h, uint64_t *keys, int32_t *perm, int32_t *level, uint64_t *anchor,
                    int32_t *begin, int32_t *end, int32_t *child, int32_t *nchild, int32_t *parent,
                    int64_t *p2p_ptr, int32_t *p2p_idx, int64_t *m2l_ptr, int32_t *m2l_idx,
                    double *box);

/*
 * Copy the multipole and local expansions of the last evaluate to HOST
 * buffers M and L (ncells * p * p doubles each, either may be NULL). Entry
 * [c][k] is the k-th real coefficient of cell c in the packed real layout:
 * for degree n at offset n*n, Re(n,0), then Re(n,m), Im(n,m) for m = 1..n.
 * Coefficients are scaled by the cell width w: M_n^m / w^n and L_n^m w^(n+1).
 * Synchronises the handle's stream.
 */
FMM_API int fmm_export_expansions(fmm_handle h, double *M, double *L);

/*
 * FP64 direct sum on the device (the quantity the FMM approximates), for the
 * targets tidx[0..nt) (device int64 indices) or all n particles when tidx is
 * NULL. x, q: device FP64 (n*3, n); phi[nt], grad[nt*3]: device FP64. Sums
 * run over j in index order. Runs on the handle's stream; the handle only
 * supplies the stream and the launch counter.
 */
FMM_API int fmm_direct(fmm_handle h, const double *x, const double *q, int64_t n, const int64_t *tidx,
               int64_t nt, double *phi, double *grad);

/* Rotation-based M2L of one expansion on the host, FP64, no GPU needed: the
 * packed multipole M (p^2 reals: for each degree n, Re M_n^0, then Re and Im
 * of M_n^m, m = 1..n) about c_M is translated into the local expansion L
 * (same layout, overwritten) about c_L, u = c_L - c_M (|u| > 0), by rotating
 * u onto the z axis, translating along z (only equal orders couple, O(p^3))
 * and rotating back; the result equals the dense M2L
 * L_n^m = (-1)^n sum_{j,k} M_j^k I_{j+n}^{k+m}(u) to 1e-13 relative up to
 * p = 20 (the rotation maps are the closed-form Wigner small-d matrices,
 * evaluated in FP64). It uses the rotation maps of the FMM_M2L_ROTATION
 * engine. Returns FMM_EINVAL
 * for p outside [1, 20], a NULL pointer or u = 0. */
FMM_API int fmm_m2l_rotation_host(int p, const double *u, const double *M, double *L);

FMM_API int fmm_destroy(fmm_handle h);

/*
 * Batched evaluation of many independent systems (the paper's GPU task queue,
 * Sec. 5: work handed to the GPU in large contiguous pieces). Each system has
 * its own handle, built with fmm_build (mixed precision, FP32 device inputs,
 * all with the same p in [2, 10] on one device). fmm_batch_create fixes the
 * systems and their outputs: phi[i] (n_i floats) and grad[i] (n_i x 3 floats),
 * device memory, caller's order. The handles must outlive the batch and must
 * not be rebuilt while it exists. Returns FMM_EINVAL (mismatched handles, p,
 * precision or NULL arguments), FMM_ESTATE (a handle not built), FMM_ECUDA.
 *
 * fmm_batch_evaluate evaluates every system with a fixed number of launches
 * (about eight, whatever the number of systems), asynchronously on `stream`
 * (NULL: legacy default), which may be captured into a CUDA graph. Work items
 * (system, phase, cell or tile) come from device queues: the upward and
 * downward passes are persistent kernels whose items wait, bounded by about a
 * second, for the level they depend on; the M2L and P2P kernels draw (system,
 * tile) and (system, leaf) items. Each system's phi and grad are bitwise those
 * of fmm_evaluate on its handle.
 *
 * fmm_batch_status synchronises the device and reports in *async_error the
 * device-side waits of the last evaluation that gave up (bit 0: a dependency
 * wait of the upward or downward pass, bit 1: tensor-core M2L, bit 2: P2P;
 * the outputs of that evaluation are then void) and, if kernel_launches is
 * not NULL, the kernels one evaluation launches.
 *
 * For failure-detection tests: fmm_batch_items reads work item `item` of pass
 * 0 (upward) or 1 (downward) (its system, kind 0 P2M / 1 M2M / 2 L2L / 3 L2P,
 * cell and level); fmm_batch_withhold removes it from the queue, so that the
 * items that depend on it time out and report bit 0.
 */
FMM_API int fmm_batch_create(const fmm_handle *handles, int nsys, void *const *phi, void *const *grad, fmm_batch *out);
FMM_API int fmm_batch_evaluate(fmm_batch b, void *stream);
FMM_API int fmm_batch_status(fmm_batch b, int *async_error, int64_t *kernel_launches);
FMM_API int fmm_batch_items(fmm_batch b, int pass, int64_t item, int *system, int *kind, int *cell, int *level);
FMM_API int fmm_batch_withhold(fmm_batch b, int pass, int64_t item);
FMM_API int fmm_batch_destroy(fmm_batch b);

/*
 * Allocation-free Morton keys and stable sort (the paper has no counterpart:
 * this is an interface for callers that cannot allocate device memory, such
 * as a loop with a fixed device-memory budget, where a cudaMalloc may block
 * on the device or fail part-way through a run, or an application whose
 * device memory is owned by another framework's allocator, which a library
 * allocating behind its back would starve).
 *   x: n*3 positions on the device, dtype FMM_F32 or FMM_F64 (no host memory);
 *   keys[n], perm[n]: device outputs, the same sorted 63-bit Morton keys and
 *   permutation (perm[k] = input index of the k-th sorted particle) that
 *   fmm_build computes and fmm_export_tree returns;
 *   stream: cudaStream_t (NULL = legacy default stream).
 * No allocation: temporaries live in one fixed array that the library
 * reserves on every GPU that loads it (about 12.3 MB, held until the process
 * exits); n above 1048576 is rejected with FMM_EINVAL. The first call on a
 * device looks up the array's device address with that device current; make
 * that first call before any stream capture. All calls share the array: calls
 * that overlap on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller. Positions must be finite. Runs
 * asynchronously on the stream; no handle is needed. Errors: FMM_EINVAL,
 * FMM_ENODEV, FMM_ECUDA (message in fmm_last_error(NULL)).
 */
FMM_API int fmm_morton_sort_noalloc(const void *x, int64_t n, int dtype, uint64_t *keys, int32_t *perm, void *stream);

/*
 * Measured peak rate of one arithmetic pipe of the current device, in TFLOP/s
 * (2 flop per multiply-add). The paper has no counterpart: these are the
 * denominators of the roofline fractions the benchmark reports for P2P (FP32
 * FMA) and for the tensor-core M2L (TF32 MMA).
 *   kind FMM_PEAK_FP32_FMA / FMM_PEAK_FP32X2_FMA: every thread of a full-
 *     occupancy grid runs 8 independent FMA chains (param ignored);
 *   kind FMM_PEAK_TF32_MMA: one CTA per SM, one thread issuing M = 128,
 *     N = param (128 or 256), K = 8 MMAs from two fixed 128B-swizzled
 *     shared-memory operands into one tensor-memory accumulator.
 * One untimed launch, then the best of reps (1..100) launches timed with CUDA
 * events. Runs on the legacy default stream; allocates and frees a few bytes
 * of device memory; synchronises the device. Errors: FMM_EINVAL (kind, param,
 * reps or NULL tflops), FMM_ENODEV, FMM_ECUDA.
 */
FMM_API int fmm_measure_peak(int kind, int param, int reps, double *tflops);

/* Message of the last error on the calling thread ("" if none). */
FMM_API const char *fmm_last_error(fmm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H */
