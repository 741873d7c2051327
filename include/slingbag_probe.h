/*
 * slingbag_probe.h -- throughput probes of the units that bound the hot
 * kernels of libslingbag (the paper has no counterpart: these measure the
 * roofline denominators on the GPU at hand).
 *
 * Each probe launches its kernel on the current device, times it with CUDA
 * events on a private stream, synchronises, and writes an operation rate:
 *   sbp_probe_fp32_fma:     thread-level FP32 fused multiply-adds per second
 *                           (independent chains, no memory traffic);
 *   sbp_probe_fp32x2_fma:   the same FMAs issued as packed pairs (one
 *                           instruction performs the FMAs of both halves of
 *                           a float2; sm_100 and later);
 *   sbp_probe_issue:        warp instructions issued per second by a loop of
 *                           independent integer adds (ALU pipe);
 *   sbp_probe_smem_atomic:  shared-memory atomic adds per second, by kind:
 *                           0 = 32-bit integer, 1 = 64-bit integer,
 *                           2 = 32-bit float; every lane of a warp targets its
 *                           own bank, so bank conflicts do not limit the rate.
 * Returns SBP_OK, SBP_ERR_ARG for a null pointer or unknown kind, or
 * SBP_ERR_CUDA when a launch or event fails (see sbp_last_error).
 */
#ifndef SLINGBAG_PROBE_H
#define SLINGBAG_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

int sbp_probe_fp32_fma(double* fma_per_s);
int sbp_probe_fp32x2_fma(double* fma_per_s);
int sbp_probe_issue(double* warp_inst_per_s);
int sbp_probe_smem_atomic(int kind, double* atomics_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SLINGBAG_PROBE_H */
