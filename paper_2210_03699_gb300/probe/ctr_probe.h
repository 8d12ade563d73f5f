/*
 * ctr_probe.h -- arithmetic-throughput probes used as roofline denominators.
 *
 * The pair sum of the CTR-IBIM operator (Eqs. 2.14-2.15) is bound by the
 * FP32 pipe and the special-function unit, whose peaks the driver-measured
 * copy bandwidth and bf16 GEMM rate do not give.  These probes run dependent
 * chains of one instruction kind on every SM and report the rate.  They are
 * measurement tooling of the benchmark, built as libctr_probe.so apart from the
 * solver library.
 */
#ifndef CTR_PROBE_H
#define CTR_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CTR_PROBE_FFMA = 0,     /* fma.rn.f32, 8 independent chains per thread */
    CTR_PROBE_FFMA2 = 1,    /* fma.rn.f32x2 (two FP32 lanes per instruction) */
    CTR_PROBE_EX2 = 2,      /* ex2.approx.ftz.f32 (SFU) */
    CTR_PROBE_RSQRT = 3,    /* rsqrt.approx.ftz.f32 (SFU) */
    CTR_PROBE_DFMA = 4      /* fma.rn.f64 */
};

/*
 * Runs probe `kind` on the current device for `iters` iterations per chain
 * and writes the achieved rate in operations per second to *ops_per_s
 * (one FP32 lane operation = 1; an f32x2 FMA counts 2; FMA counts 1, not 2
 * flops) and the kernel time in *seconds.  Returns 0, -1 for a bad argument,
 * -4 on a CUDA error, -5 when its 2 KB output buffer cannot be allocated.
 */
int ctr_probe_rate(int kind, int64_t iters, double* ops_per_s, double* seconds);

#ifdef __cplusplus
}
#endif

#endif /* CTR_PROBE_H */
