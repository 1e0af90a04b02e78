/*
 * fst_testing.h -- host-emulation entry points of libfst_gb300.so, for CPU tests.
 *
 * A plan made by fst_emu_plan_op runs every kernel body of the library on the host
 * (one thread block at a time, the threads of a block looped between barriers),
 * with all buffers in host memory.  Every other entry point of fst.h accepts such
 * a plan; its signal pointers are then HOST pointers and `stream` is ignored.
 * This checks the library's index arithmetic and plan logic without a GPU; it is
 * slow and not meant for production use.
 */
#ifndef FST_GB300_TESTING_H
#define FST_GB300_TESTING_H

#include "fst.h"

#ifdef __cplusplus
extern "C" {
#endif

/* as fst_plan_op, executed by the host emulator.  Same argument rules and errors. */
fst_status fst_emu_plan_op(fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op, double alpha);

/* as fst_plan_many, executed by the host emulator. */
fst_status fst_emu_plan_many(fst_plan_t *out, int64_t count, const int64_t *N, const double *W,
                             const int64_t *K, const double *eps);

/* 1 if the plan runs on the host emulator, 0 otherwise (including NULL). */
int fst_plan_is_emulated(fst_plan_t plan);

/*
 * Test hook for the failure path of the bounded device waits (no GPU fault involved):
 * the next `launches` launches of the tensor-core correction first wait on a barrier
 * that nothing completes, give up after limit_s seconds (0 < limit_s <= 2) before
 * issuing any copy or product, and take the kernel's normal give-up path (tensor
 * memory freed, NaN partial sums, error word raised).  Calls made while a stall is
 * pending launch directly (no CUDA graph is recorded or replayed).
 * Errors: FST_EINVAL (launches < 0 or limit_s out of range).
 */
fst_status fst_test_tc_stall(int launches, double limit_s);

#ifdef __cplusplus
}
#endif

#endif /* FST_GB300_TESTING_H */
