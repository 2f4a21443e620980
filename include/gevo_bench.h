/*
 * gevo_bench.h -- measurement helpers (no counterpart in the paper): kernels
 * that saturate the FP32 FMA pipe and the MUFU ex2 unit, so that the peak the
 * blend kernels' ALU roofline is derived from (SMs x 128 lanes x 2 FLOP x
 * clock) and the exponential rate can be measured on the device instead of
 * assumed.  The caller times them with events on `stream`.
 */
#ifndef GEVO_BENCH_H
#define GEVO_BENCH_H

#include "gevo.h"

#ifdef __cplusplus
extern "C" {
#endif

/* blocks x 256 threads, each running 8 independent FMA chains for `iters`
 * steps: 16 * iters FLOP per thread.  sink: DEVICE float[blocks * 256]
 * (written, keeps the chains live). */
gevo_status gevo_bench_fma(int32_t blocks, int32_t iters, float* sink, void* stream);

/* The same shape with 8 independent ex2.approx chains: 8 * iters
 * exponentials per thread. */
gevo_status gevo_bench_ex2(int32_t blocks, int32_t iters, float* sink, void* stream);

/* The FMA shape with the paired instruction (fma.rn.f32x2): 8 independent
 * packed chains, 16 FMAs = 32 FLOP per thread and step.  Tells whether the
 * paired form raises the FP32 rate or only halves the instructions issued. */
gevo_status gevo_bench_fma2(int32_t blocks, int32_t iters, float* sink, void* stream);

/* 8 independent chains x <- rcp.approx(x) + 0.5: 8 * iters reciprocals per
 * thread (the MUFU operation of the reverse walk's transmittance recovery). */
gevo_status gevo_bench_rcp(int32_t blocks, int32_t iters, float* sink, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GEVO_BENCH_H */
