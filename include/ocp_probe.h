/*
 * ocp_probe.h -- measurement utility of the GB300 linearisation library.
 *
 * The paper has no counterpart: this entry point measures the sustained FP64
 * fused-multiply-add rate of a device, the denominator of the roofline of
 * the library's FP64-bound kernels (on GB300 the FP64 pipe, not HBM, bounds
 * the linearisation, the block-CSR product and the adjoint).
 */
#ifndef OCP_PROBE_H
#define OCP_PROBE_H

#include "ocp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs two FP64 FMA throughput kernels on `device` (16 independent FMA
 * chains per thread, 8 CTAs of 256 threads per SM), `reps` times each: chains
 * through the multiplicand with constant operands (v = v*a + b) and
 * accumulation chains with loop-invariant register multiplicands
 * (v = x*y + v), which GB300 issues about 18 % faster.  Returns the best rate
 * of either in *dfma_per_s (FMA thread-operations per second; 2 flops each).
 * Allocates and frees a small device buffer; synchronises the device.
 * Returns OCP_ERR_INVALID_ARG for a NULL output or reps < 1. */
ocp_status ocp_probe_fp64(int device, int reps, double* dfma_per_s);

#ifdef __cplusplus
}
#endif
#endif /* OCP_PROBE_H */
