/*
 * sv_diag.h -- diagnostics of libsvgb.so (not part of the simulation API).
 */
#ifndef SVGB_SV_DIAG_H
#define SVGB_SV_DIAG_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * One product on the tensor-core path used by sv_apply_circuit with
 * precision = 1: d[m][n] = sum_k a[m][k] * b[n][k] for m < 128, n, k < 32,
 * with a (float32, row-major 128 x 32) split into TF32 hi/lo parts on the
 * device, b (double, row-major 32 x 32) split on the host, and the three
 * products a_hi*b_hi + a_hi*b_lo + a_lo*b_hi accumulated in float32 by
 * tcgen05.mma (kind::tf32, A in tensor memory, B in shared memory).  All
 * pointers are host memory owned by the caller; d receives 128 x 32 floats.
 * Runs on the current device; synchronous.  Returns SV_OK, SV_ERR_TIMEOUT if
 * the bounded wait for MMA completion gave up, or SV_ERR_CUDA.
 */
int sv_tc_selftest(const float *a, const double *b, float *d);

/*
 * The same product for a stage of r register qubits (r = 4 or 5): K = 2^(r+1)
 * columns, d[m][n] = sum_k a[m][k] * b[n][k] for m < 128, n, k < K, with a
 * (float32, row-major 128 x K), b (double, row-major K x K) and d (128 x K
 * floats) host memory owned by the caller.  r = 4 is sv_tc_selftest; r = 5 is
 * the 64 x 64 real product of a 5-qubit stage (a 32 x 32 complex block), issued
 * as 16 MMAs of N = 128 and N = 64.  Returns as sv_tc_selftest, and SV_ERR_ARG
 * for another r.
 */
int sv_tc_selftest_r(int r, const float *a, const double *b, float *d);

/*
 * Exercises the device-side timeout path without faulting or hanging the GPU:
 * one CTA waits on an mbarrier that nothing arrives on, with the same
 * %globaltimer bound the tensor-core kernels use (limit_ms in [1, 10000]).
 * Returns SV_ERR_TIMEOUT (the expected outcome), SV_ERR_ARG or SV_ERR_CUDA.
 * Synchronous, current device.
 */
int sv_diag_bounded_wait(int limit_ms);

#ifdef __cplusplus
}
#endif

#endif /* SVGB_SV_DIAG_H */
