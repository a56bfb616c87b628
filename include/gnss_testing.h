/* gnss_testing.h -- entry points of libgnss.so for tests and measurement,
 * kept apart from the acquisition API in gnss.h.  None of them has a
 * counterpart in the paper; they fault nothing on the device. */
#ifndef GNSS_TESTING_H
#define GNSS_TESTING_H

#include "gnss.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Testing hook: make the k-th next device allocation of the dispatcher fail
 * (k = 0: the next one; negative: never), as if the device were out of
 * memory; the requests of that batch end with GNSS_ENOMEM and the server
 * carries on.  Nothing is faulted on the device. */
GNSS_API gnss_status gnss_server_inject_alloc_failure(gnss_server* srv, int k);

/* FP32 FMA throughput probe (a measurement aid with no counterpart in the
 * paper; it states the ALU roof the acquisition kernels are held against):
 * 'iters' rounds of 128 dependent-chain FMAs per thread, 4 CTAs of 512
 * threads per SM.  Writes TFLOP/s (2 flops per FMA) and the kernel time in
 * ms (ms may be NULL).  Synchronous. */
GNSS_API gnss_status gnss_probe_ffma(int iters, double* tflops, double* ms, void* stream);

/* Testing hook: every wait of the staged correlate variant (variant code
 * 16 | GNSS_TUNE_STAGED) on the current device polls its bulk copy at most
 * 'iters' times before it gives up (default 4194304; 0 makes every wait give
 * up at once).  A CTA whose wait gave up issues no further copy, reads the
 * rest of its spectra from global memory, flags its call's records with
 * GNSS_DET_STAGE_TIMEOUT and waits for the copy still in flight with the
 * full bound before it leaves, so the records stay complete.  Affects every
 * later launch on the device until it is set back.  Synchronous on 'stream'.
 * Errors: GNSS_ECUDA. */
GNSS_API gnss_status gnss_testing_set_stage_wait_limit(uint32_t iters, void* stream);

/* Testing hook: every wait of the correlate's occupancy form at N = 4096,
 * 8192 and 16384 (variant code 16 | GNSS_TUNE_TMEM | GNSS_TUNE_OCC, one
 * shared-memory exchange buffer per CTA) for the release of that buffer by the CTA's other
 * warps polls at most 'iters' times before it gives up (default 4194304; 0
 * makes every wait give up at once).  A wait that gave up flags its call's
 * records with GNSS_DET_WAIT_TIMEOUT and the CTA goes on: its warps may then
 * overwrite buffer slots another warp has yet to read (shared memory only,
 * within the CTA's buffer), so the flagged call's records and surfaces are
 * not valid; nothing is faulted and nothing waits unboundedly.  Affects
 * every later launch on the device until it is set back.  Synchronous on
 * 'stream'.  Errors: GNSS_ECUDA. */
GNSS_API gnss_status gnss_testing_set_buf_wait_limit(uint32_t iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GNSS_TESTING_H */
