/*
 * libgpp: General Plasmon Pole (GPP) self-energy summation on one NVIDIA GB300 (sm_103a).
 *
 * The operation (paper §II-A, the loop nest over band, igp, ig and iw; §III v2, the
 * three-way branch; §III v3, predicates on squared moduli). For every band b, local column
 * p, G-vector ig and frequency iw:
 *
 *   g      = indinv[inv_igp_index[p]]  (global column; if inv_igp_index[p] is outside
 *                                       [0, ncouls] or g is outside [0, ncouls), column p
 *                                       contributes nothing -- indinv[ncouls] = ncouls is
 *                                       the sentinel)
 *   M      = conj(aqsmtemp[b][g]) * aqsntemp[b][ig] * vcoul[g]
 *   x      = wx_array[b][iw],  w = wtilde_array[p][ig],  I = I_eps_array[p][ig]
 *   wdiff  = x - w,  wdiffr = |wdiff|^2,  delw = w / wdiff,  delwr = |delw|^2
 *   branch 1, wdiffr > 0.25 and delwr < 2.5e5:  sch = delw I,  ssx = w^2 I / (x^2 - w^2)
 *   branch 2, else if delwr > 1e-12:           sch = 0,       ssx = -I delw / (4 delw + 2)
 *   branch 3, else:                             sch = 0,       ssx = 0
 *   achtemp[iw] = sum M sch,   asxtemp[iw] = sum occ(b) M ssx
 *
 * with occ(b) = 1 (GPP_OCC_ALL) or [b < nvband] (GPP_OCC_OCCUPIED). The paper names the
 * three thresholds without printing them or the sch/ssx formulas; the values above are the
 * generalised plasmon-pole terms of BerkeleyGW, which the paper's kernel is taken from.
 *
 * Conventions for every entry point:
 *  - Arrays are C row-major with the last index contiguous; complex arrays are interleaved
 *    (re, im) pairs, the layout of torch complex128 / complex64. Shapes:
 *      aqsmtemp, aqsntemp [number_bands][ncouls]; I_eps_array, wtilde_array
 *      [ngpown][ncouls]; vcoul [ncouls]; inv_igp_index [ngpown]; indinv [ncouls + 1];
 *      wx_array [number_bands][nw]; achtemp, asxtemp [nw].
 *  - Data pointers are DEVICE pointers owned by the caller; inputs are only read, outputs
 *    are fully overwritten. Complex arrays must be 16-byte aligned (c128) or 8-byte aligned
 *    (c64). The caller provides the workspace; the library allocates no device memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *    default stream) unless stated otherwise.
 *  - Results are bit-for-bit deterministic for fixed inputs, options and device.
 *  - Return GPP_OK (0) or a negative gpp_status; gpp_last_error() then describes it.
 */
#ifndef GPP_H
#define GPP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GPP_API __attribute__((visibility("default")))
#else
#define GPP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gpp_status {
    GPP_OK = 0,
    GPP_ERR_NULL_PTR = -1,    /* a required pointer is NULL */
    GPP_ERR_BAD_SIZE = -2,    /* a size is negative, nw outside [1, GPP_MAX_NW], or a size exceeds 32-bit indexing */
    GPP_ERR_BAD_INDEX = -3,   /* debug_checks found an index outside its range */
    GPP_ERR_WORKSPACE = -4,   /* workspace NULL, misaligned or smaller than required */
    GPP_ERR_CUDA = -5,        /* a CUDA call or kernel launch failed */
    GPP_ERR_UNSUPPORTED = -6, /* option combination not supported */
    GPP_ERR_TIMEOUT = -7,     /* a bounded device-side wait gave up */
    GPP_ERR_BAD_OPTION = -8   /* an option field has an unknown value */
} gpp_status;

typedef enum gpp_precision {
    GPP_FP64 = 0,      /* every step in FP64 */
    GPP_FP32_BULK = 1  /* FP32 complex arithmetic (complex64 aqsntemp copy), FP64 branch
                          decisions near the threshold, FP64 near the wdiff pole, compensated
                          FP32 accumulation folded into FP64 reductions */
} gpp_precision;

typedef enum gpp_occ_mode {
    GPP_OCC_ALL = 0,      /* occ(b) = 1: every band enters asxtemp (the paper's loop nest) */
    GPP_OCC_OCCUPIED = 1  /* occ(b) = [b < nvband] */
} gpp_occ_mode;

/* Options of the Sigma code around the kernel (BerkeleyGW; not part of the paper's loop
 * nest), bits of gpp_options.physics: */
typedef enum gpp_physics {
    GPP_PHYS_CH_HALF = 1,   /* achtemp[iw] = (1/2) sum M sch: the factor 1/2 of the Coulomb hole */
    GPP_PHYS_SX_CUTOFF = 2  /* a term with x < 0 and |ssx| > sexcut |I| takes ssx = 0 (the
                               screened-exchange cutoff; sexcut from gpp_options.sexcut) */
} gpp_physics;

#define GPP_MAX_NW 8

typedef struct gpp_c128 {
    double re, im;
} gpp_c128;

typedef struct gpp_c64 {
    float re, im;
} gpp_c64;

/* One GPP instance. Names follow the paper's kernel. */
typedef struct gpp_problem {
    int64_t number_bands; /* B >= 0 */
    int64_t nvband;       /* V >= 0, used by GPP_OCC_OCCUPIED */
    int64_t ncouls;       /* G >= 0 */
    int64_t ngpown;       /* P >= 0 */
    int64_t nw;           /* W, 1 <= W <= GPP_MAX_NW */
    const gpp_c128 *aqsmtemp;     /* [B][G] */
    const gpp_c128 *aqsntemp;     /* [B][G] */
    const gpp_c128 *I_eps_array;  /* [P][G] */
    const gpp_c128 *wtilde_array; /* [P][G] */
    const double *vcoul;          /* [G] */
    const int32_t *inv_igp_index; /* [P] */
    const int32_t *indinv;        /* [G + 1] */
    const double *wx_array;       /* [B][W] */
    /* complex64 copy of aqsntemp, read by GPP_FP32_BULK for its per-band loads (ignored
     * otherwise). NULL lets the library make it: the call then converts aqsntemp into its
     * workspace first (an HBM-bound copy, counted in gpp_sigma_workspace_size: B * G * 8
     * bytes more). The (igp, ig) arrays are read once per pair in FP64 and rounded in
     * registers, and the gathered weights are rounded by the gather kernel, so no other
     * copies are needed. */
    const gpp_c64 *aqsntemp_c64; /* [B][G] */
    gpp_c128 *achtemp; /* [W] output */
    gpp_c128 *asxtemp; /* [W] output */
} gpp_problem;

typedef struct gpp_options {
    int32_t precision;     /* gpp_precision */
    int32_t occ_mode;      /* gpp_occ_mode */
    int32_t block_threads; /* threads per CTA of the main kernel: 0 = default (128), else a multiple of 32 in [64, 256] */
    int32_t blocks_per_sm; /* resident CTAs per SM for the persistent grid: 0 = as many as fit */
    int32_t debug_checks;  /* 1: validate indices on the device and synchronise (GPP_ERR_BAD_INDEX) */
    int32_t ig_per_thread; /* G-vectors each thread takes per tile: 0 = default (4 in GPP_FP64,
                              2 in GPP_FP32_BULK), max 8; a tile is
                              one igp column x block_threads * ig_per_thread G-vectors x all bands */
    int32_t physics;       /* bit set of gpp_physics: 0 = the paper's sum */
    int32_t reserved;      /* must be 0 */
    /* NULL, or an array of 4 cudaEvent_t (passed as void*) that the call records on its
     * stream: [0] before the column gather, [1] before the main sum, [2] after it, [3] after
     * the final reduction. For timing the main kernel; the events belong to the caller. */
    void *const *stage_events;
    double sexcut;         /* with GPP_PHYS_SX_CUTOFF: the cutoff factor (> 0, finite; BerkeleyGW
                              uses 4); ignored otherwise. The kernels test |w|^2 / |x^2 - w^2| >
                              sexcut (branch 1) and |w| / (2 |x + w|) > sexcut (branch 2), which
                              equal |ssx| / |I| there, so a term within rounding of the cutoff can
                              be decided either way */
} gpp_options;

/* Fills *opt with the defaults (GPP_FP64, GPP_OCC_ALL, default tiles, no debug checks, no
 * physics options). */
GPP_API void gpp_options_default(gpp_options *opt);

/*
 * Workspace bytes that gpp_sigma needs for this problem and these options on the current
 * device (it depends on the SM count). 0 with gpp_last_error() set if the arguments are
 * invalid. Pure host computation; no device memory is touched.
 */
GPP_API size_t gpp_sigma_workspace_size(const gpp_problem *prob, const gpp_options *opt);

/*
 * The forward sum (achtemp, asxtemp) of one instance. `workspace` is a device buffer of at
 * least gpp_sigma_workspace_size() bytes, 256-byte aligned, owned by the caller and not
 * used concurrently by another call. The call enqueues three kernels on `stream` (column
 * gather, main sum over tiles taken from a counter by a persistent grid with one partial
 * per tile, fixed-order reduction of the partials) and returns without synchronising,
 * except with debug_checks = 1, where it synchronises `stream` to report bad indices.
 * A problem with number_bands, ngpown or ncouls equal to 0 is an empty sum: the outputs
 * are set to zero on `stream`, no input is read and the workspace may be NULL.
 * Errors: NULL_PTR, BAD_SIZE, BAD_OPTION, WORKSPACE, CUDA, BAD_INDEX (debug_checks only).
 */
GPP_API int gpp_sigma(const gpp_problem *prob, const gpp_options *opt, void *workspace,
              size_t workspace_bytes, void *stream);

/*
 * Device bytes that gpp_sigma_host needs: room for device copies of every input array
 * plus gpp_sigma's own workspace.
 */
GPP_API size_t gpp_sigma_host_workspace_size(const gpp_problem *prob, const gpp_options *opt);

/*
 * gpp_sigma on HOST arrays: every pointer in `prob` (inputs and outputs) is a host pointer
 * (page-locked memory gives the fastest copies and lets them overlap the sum). The inputs
 * are copied into `workspace` (a device buffer of gpp_sigma_host_workspace_size() bytes),
 * except aqsmtemp when it is page-locked and mapped into the device's address space (as
 * cudaHostAlloc memory is): the column gather then reads its number_bands x ngpown
 * elements at the gathered columns in place instead of waiting for a copy of the whole
 * array,
 * the sum runs, the outputs are copied back, and the call returns after `stream` has
 * finished (it synchronises). The copies of aqsntemp, I_eps_array and wtilde_array go in
 * up to 8 chunks of G-vectors (of doubling size, so that the sum starts after a small
 * first chunk) on a copy stream while the sum runs the chunks already copied, alternating between `stream` and a second stream (the library creates both
 * streams on a device's first call and keeps them); the result equals gpp_sigma's bit for
 * bit.
 */
GPP_API int gpp_sigma_host(const gpp_problem *prob, const gpp_options *opt, void *workspace,
                   size_t workspace_bytes, void *stream);

/*
 * gpp_sigma without a caller-supplied workspace, for callers that cannot allocate device
 * memory for it: a Fortran or C host code that links this library through its C interface
 * and keeps no device allocator of its own, or a process whose device memory is owned and
 * accounted by another runtime. (No counterpart in the paper: it is an interface option.)
 * The scratch lives in a fixed array of GPP_NOALLOC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library holds until the process exits. The call allocates
 * nothing and frees nothing. Problems whose gpp_sigma_workspace_size() exceeds the array
 * are rejected with GPP_ERR_WORKSPACE, unless `ig_per_thread` is 0 and tiles of 8
 * G-vectors per thread (half the per-tile partials) fit, which the call then uses (the
 * benchmark shape B=512, P=1638, G=32768, nw=3 needs about 24 MB in FP64 and 30 MB in
 * FP32-bulk with the default tiles). Every call looks up the array's device address in
 * the current device's context (cudaGetSymbolAddress), so a call on another device, in
 * another context or after a device reset uses that context's copy; the first call on a
 * device can load the library's device code, so make it before any stream capture. All
 * calls share the one array, so calls that overlap on the GPU (other streams, other
 * threads) race: serialise them. Everything that must start at zero is cleared by every
 * call. Results equal gpp_sigma's with the tile shape used, bit for bit. Asynchronous on
 * `stream`. Errors as gpp_sigma (NULL_PTR, BAD_SIZE, BAD_OPTION, ... with the same codes),
 * plus WORKSPACE for a problem beyond the array and CUDA if the lookup fails.
 */
#define GPP_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
GPP_API int gpp_sigma_noalloc(const gpp_problem *prob, const gpp_options *opt, void *stream);

/* Gradients written by gpp_sigma_backward (device pointers; NULL skips that gradient). */
typedef struct gpp_grads {
    gpp_c128 *wtilde_array; /* [P][G] */
    gpp_c128 *I_eps_array;  /* [P][G] */
    gpp_c128 *aqsmtemp;     /* [B][G]; entries of global columns no igp reaches are 0 */
    gpp_c128 *aqsntemp;     /* [B][G] */
} gpp_grads;

/* Workspace bytes gpp_sigma_backward needs (0 with gpp_last_error() set on bad input). */
GPP_API size_t gpp_sigma_backward_workspace_size(const gpp_problem *prob, const gpp_options *opt);

/*
 * Adjoint of gpp_sigma in FP64 (a derivative of the sum that the paper does not treat).
 * Given the cotangents of the outputs in PyTorch's convention for complex tensors,
 * grad_achtemp[iw] = dL/dRe achtemp[iw] + i dL/dIm achtemp[iw] (likewise grad_asxtemp;
 * device arrays of nw), writes dL/dRe z + i dL/dIm z for z = wtilde_array, I_eps_array,
 * aqsmtemp, aqsntemp into `grads` (overwritten, not accumulated). Inside a branch every
 * term is holomorphic in wtilde, I_eps and aqsntemp and anti-holomorphic in aqsmtemp;
 * the branch predicates contribute no derivative. Terms are recomputed from the inputs,
 * not stored. prob->achtemp / asxtemp are not used. opt->precision must be GPP_FP64.
 * Asynchronous on `stream`; deterministic. Errors as gpp_sigma, plus UNSUPPORTED.
 */
GPP_API int gpp_sigma_backward(const gpp_problem *prob, const gpp_options *opt,
                               const gpp_c128 *grad_achtemp, const gpp_c128 *grad_asxtemp,
                               const gpp_grads *grads, void *workspace, size_t workspace_bytes,
                               void *stream);

/*
 * Batched sums: n independent instances (uneven sizes allowed, the same nw) in one
 * persistent kernel (an extension of the paper's single-instance kernel). Tiles (one igp
 * column x block_threads * ig_per_thread G-vectors x all bands) of all instances are taken
 * from an atomic counter by a grid of blocks_per_sm CTAs per SM, largest band count first;
 * each tile writes its own partial and a per-instance kernel sums them in a fixed order,
 * so results are deterministic and equal to gpp_sigma's up to summation order.
 * `probs` is a host array of n problems with device pointers (each with its own outputs).
 * The caller provides one device workspace of gpp_batched_workspace_size() bytes.
 */
typedef struct gpp_batched_plan gpp_batched_plan; /* opaque host object */

GPP_API size_t gpp_batched_workspace_size(const gpp_problem *probs, int n, const gpp_options *opt);

/*
 * Prepares a batch: validates every instance, writes the instance descriptors into the
 * workspace (the call synchronises `stream` once for that), and, with use_graph = 1,
 * captures gather + persistent kernel + reduction into a CUDA graph (on a private stream;
 * runs launch it on the caller's stream). The
 * problems' device arrays and the workspace must stay valid until the plan is destroyed.
 */
GPP_API int gpp_batched_plan_create(gpp_batched_plan **plan, const gpp_problem *probs, int n,
                                    const gpp_options *opt, void *workspace,
                                    size_t workspace_bytes, int use_graph, void *stream);
/* Runs a prepared batch on `stream` (a graph launch if the plan holds a graph). */
GPP_API int gpp_batched_plan_run(gpp_batched_plan *plan, void *stream);
/* Frees the host-side plan and its graph. */
GPP_API int gpp_batched_plan_destroy(gpp_batched_plan *plan);
/* One-shot: create (no graph), run, destroy. */
GPP_API int gpp_sigma_batched(const gpp_problem *probs, int n, const gpp_options *opt,
                              void *workspace, size_t workspace_bytes, void *stream);

/*
 * dst[i] = src[i] rounded to complex64 (round to nearest, both parts), i < n: the complex64
 * copy of aqsntemp that GPP_FP32_BULK reads, made once by a caller that keeps it across
 * calls. Device arrays; asynchronous on `stream`. Errors: NULL_PTR, BAD_SIZE (n < 0), CUDA.
 */
GPP_API int gpp_convert_c64(const gpp_c128 *src, gpp_c64 *dst, int64_t n, void *stream);

/* Thread-local description of the last error on this host thread ("" if none). */
GPP_API const char *gpp_last_error(void);

/* Library version string. */
GPP_API const char *gpp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPP_H */
