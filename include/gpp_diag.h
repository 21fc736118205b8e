/*
 * libgpp machine characterisation and numerics diagnostics.
 *
 * The paper reports its kernel against measured machine peaks (§I, the Empirical Roofline
 * Toolkit; §III v8, the FMA-ratio-adjusted FP64 peak). Copy-bandwidth and bf16
 * GEMM rates do not cover the FP64 and FP32 pipes that bound the GPP sum, so the library
 * carries its own throughput kernels. Conventions as in gpp.h (device pointers, async on
 * `stream`, negative gpp_status on error, gpp_last_error()).
 */
#ifndef GPP_DIAG_H
#define GPP_DIAG_H

#include <stddef.h>
#include <stdint.h>

#include "gpp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gpp_peak_kind {
    GPP_PEAK_DFMA = 0,    /* FP64 fused multiply-add chains (2 FLOP each) */
    GPP_PEAK_FFMA = 1,    /* FP32 fused multiply-add chains (2 FLOP each) */
    GPP_PEAK_DADD = 2,    /* FP64 add chains (1 FLOP each) */
    GPP_PEAK_DMUL = 3,    /* FP64 multiply chains (1 FLOP each) */
    GPP_PEAK_DRCP = 4,    /* the sum's FP64 reciprocal: approximation + 3 FMA (1 op each) */
    GPP_PEAK_DRCP_RN = 5, /* CUDA's correctly rounded FP64 reciprocal __drcp_rn (1 op each) */
    GPP_PEAK_DRCP_APPROX = 6, /* the hardware FP64 reciprocal approximation alone (1 op each) */
    GPP_PEAK_FSEL = 7,    /* FP32 select on a data-dependent predicate (1 op each) */
    GPP_PEAK_FSETP = 8,   /* FP32 compare feeding an integer select (1 op each) */
    GPP_PEAK_ISEL = 9,    /* 32-bit integer select (1 op each) */
    GPP_PEAK_F2F = 10     /* FP64 -> FP32 -> FP64 round trip (1 op each) */
} gpp_peak_kind;

/* Independent dependency chains per thread in every throughput kernel. */
#define GPP_PEAK_CHAINS 8

/*
 * Launches one throughput kernel: `blocks` CTAs of `threads` threads, each thread running
 * GPP_PEAK_CHAINS independent chains of `iters` operations of `kind`. The operation count
 * of one launch is blocks * threads * GPP_PEAK_CHAINS * iters; time it with events on
 * `stream`. `sink` is a device double that receives a value only under a condition that
 * never holds (it keeps the work alive); it may not be NULL.
 */
GPP_API int gpp_peak_launch(int kind, int64_t iters, int blocks, int threads, double *sink,
                    void *stream);

/*
 * out[i] = the FP64 reciprocal the GPP kernels use, applied to in[i] (i < n), for tests
 * that compare it with 1.0 / in[i]. Device arrays of n doubles.
 */
GPP_API int gpp_diag_rcp(const double *in, double *out, int64_t n, void *stream);

/*
 * Host-side fault injection for tests of the error paths. After this call, the n-th CUDA
 * runtime call whose status a libgpp entry point checks on this host thread (1 = the next
 * one) reports failure as if it had failed: the call itself has been made, and the entry
 * point takes its error path (GPP_ERR_CUDA, with "[injected by
 * gpp_diag_inject_cuda_failure]" in gpp_last_error()). Nothing fails on the device. n <= 0
 * disarms; a countdown not reached stays armed.
 */
GPP_API void gpp_diag_inject_cuda_failure(int n);

#ifdef __cplusplus
}
#endif

#endif /* GPP_DIAG_H */
