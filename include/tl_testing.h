/*
 * tl_testing.h -- test hooks of libtl (not part of the stable API).
 *
 * tl_testing_ff applies one float-float primitive of the TL_F64_FF kernels (pairs of binary32 values
 * carried as hi + lo, converted to and from binary64 with integer operations) elementwise, so the
 * primitives can be checked against exact rational arithmetic:
 *   op 0: y[i] = merge(normalize(split(a[i])))       (conversion round trip)
 *   op 1: y[i] = merge(split(a[i]) - split(b[i]))     (pair subtraction)
 *   op 2: y[i] = merge(dot3(split(a), split(b), split(c), split(d), split(e), split(f)))[i]
 *         = a b + c d + e f                           (the contraction kernel's dot product)
 * All pointers are DEVICE arrays of n doubles (b..f may be NULL when the op does not read them); the
 * work is enqueued on `stream`.  Returns a tl_status code (0 = OK).
 *
 * tl_testing_f32_staged_stall runs the staged binary32 forward kernel over the full 512-point tiles of
 * n points with every stage announcing 16 bytes more than its copies deliver, so that no stage
 * completes: each block's bounded wait runs out (after about 0.5 s), the block counts it in the
 * counter tl_wait_timeouts reads, waits (bounded again) for the copies it issued, and leaves without
 * writing outputs.  Tables as for tl_dtg_forward with TL_F32 (inputs 16-byte aligned, else
 * TL_ERR_ALIGNMENT).  Exercises the failure path of the waits without a device fault.
 */
#ifndef TL_TESTING_H
#define TL_TESTING_H
#include "tl.h"
#ifdef __cplusplus
extern "C" {
#endif

TL_API tl_status tl_testing_ff(int op, const double *a, const double *b, const double *c, const double *d,
                               const double *e, const double *f, double *y, int64_t n, tl_stream stream);
/*
 * tl_testing_f64_int applies one binary64 operation elementwise, as the kernels' integer-pipe form or
 * the hardware instruction, so the integer forms can be checked bit for bit:
 *   op 0: y[i] = a[i] * b[i]           (integer-pipe product, mul_int)
 *   op 1: y[i] = 1 / a[i]              (the kernels' reciprocal, rcp_f64: binary32 seed and one
 *                                       third-order step; within one ulp of the IEEE quotient)
 *   op 3: y[i] = fma(a[i], b[i], c[i]) (hardware fused multiply-add, reference)
 * (op 2 is reserved).  DEVICE arrays of n doubles; b not read by op 1, c only for op 3.  Enqueued on
 * `stream`.
 */
TL_API tl_status tl_testing_f64_int(int op, const double *a, const double *b, const double *c, double *y, int64_t n,
                                    tl_stream stream);
TL_API tl_status tl_testing_f32_staged_stall(const tl_dtg_in *in, const tl_dtg_out *out, int64_t n,
                                             tl_stream stream);
/*
 * tl_testing_batched_staged_stall launches a plan whose staging depth is 2 or 3 (tl_batch_plan_set_staging)
 * once, with every stage announcing 16 bytes more than its copies deliver, so that no stage completes:
 * each block's bounded wait runs out, the block counts it in the counter tl_wait_timeouts reads, waits
 * (bounded again) for the stages it issued, and leaves without writing outputs.  TL_ERR_INVALID_ARG for a
 * plan that does not stage.  Exercises the failure path of the staged batched kernel's waits.
 */
TL_API tl_status tl_testing_batched_staged_stall(const tl_batch_plan *plan, tl_stream stream);
/*
 * tl_testing_pipe_rate launches `blocks` blocks of `threads` threads (a multiple of 32, at most 1024),
 * each thread running 8 independent chains of `iters` rounds of one operation:
 *   op 0: DFMA   op 1: DADD   op 2: DMUL   op 3: binary64 -> binary32 -> binary64 conversion pair
 *         (two F2F and one binary32 multiply per round)   op 4: an addition written as an FMA by 1.0
 *   (an immediate operand); ops 0-4 read their other operands from the parameter bank.
 *   op 5: DFMA   op 6: DADD   op 7: DMUL, with register operands   op 8: an addition written as an FMA
 *   whose factor 1.0 comes from constant memory (register addend)
 * so that, timed by the caller, blocks x threads x 8 x iters / time is the issue rate of that
 * operation (op 3: of conversion pairs).  `sink` is a DEVICE array of blocks x threads doubles that
 * is never written for these operands (it only keeps the chains alive).  Enqueued on `stream`.
 */
TL_API tl_status tl_testing_pipe_rate(int op, int64_t iters, int32_t blocks, int32_t threads, double *sink,
                                      tl_stream stream);
/*
 * tl_testing_jit_min_blocks: the blocks per SM of 256 threads that a compiled program's kernel is built
 * for (its launch bound): 3 unless that spills more than 128 bytes per thread, then 2.  Decided from the
 * ptxas report in the compile log when it has one, and checked again against the loaded kernel's local
 * memory at its first launch on a device.  Host only.
 */
TL_API tl_status tl_testing_jit_min_blocks(const tl_jit_kernel *k, int32_t *blocks);
/*
 * tl_testing_memory_info: the device's peak memory clock (kHz) and global memory bus width (bits), from
 * which the nominal HBM bandwidth is clock x 2 x width / 8.  TL_ERR_INVALID_ARG for NULL outputs
 * (checked before any CUDA call), TL_ERR_CUDA when the device cannot be queried.
 */
TL_API tl_status tl_testing_memory_info(int32_t device, int32_t *clock_khz, int32_t *bus_bits);

#ifdef __cplusplus
}
#endif
#endif
