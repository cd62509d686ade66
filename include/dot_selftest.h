/* dot_selftest.h -- self-test of the library's failure handling (no counterpart in
 * the paper).
 *
 * Every mbarrier wait in the tensor-core kernels gives up after about one second
 * (global timer), records the failure in a device flag that the host reads with
 * the stopping measures (dot_solve then returns DOT_ECUDA), waits for its own
 * copies and MMAs in flight and frees its TMEM, so that the context stays usable.
 * This entry point exercises that path without faulting the GPU: it runs one
 * 128-row tcgen05 DCT pass (K = 32, one CTA) on zero data, on a private stream of
 * the current device, in which -- when inject != 0 -- the stage barrier expects 16
 * bytes more than its TMA load delivers, i.e. a phase that nothing completes.
 *
 *   inject   : 0 = a normal pass, 1 = the barrier that never completes
 *   seconds  : out, host wall time from launch to the end of the stream
 *   flag     : out, the pass's error flag (1 = a wait gave up)
 *
 * Returns 0 when the pass ran and the flag was read, -1 when the pass could not be
 * launched on the tensor cores, -3 when a CUDA call failed.  Allocates and frees
 * about 50 KB of device memory. */
#ifndef DOT_SELFTEST_H
#define DOT_SELFTEST_H

#ifdef __cplusplus
extern "C" {
#endif

int dot_selftest_pipeline_timeout(int inject, double *seconds, int *flag);

#ifdef __cplusplus
}
#endif

#endif /* DOT_SELFTEST_H */
