/*
 * Measurement probes for the roofline of the stereo ray tracer (sm_103a).
 *
 * The traversal kernel is bound by FP32 issue; two further ceilings enter its
 * roofline and are not published for this part, so they are measured:
 *   - the MUFU (special-function) pipe, which serves one reciprocal per
 *     triangle test, one square root per sphere test and one reciprocal
 *     square root per normalised ray (the primitive tests of Sec. 2 as built
 *     here);
 *   - the L2 read bandwidth, against which the bytes the rays fetch (64 B per
 *     node visit, 48 B per primitive test) are a diagnostic: the BVH of the
 *     benchmark scene fits in L2, so its node fetches never reach HBM.
 *
 * Conventions as in rt_stereo.h: 0 = RT_OK, negative codes on error, work
 * enqueued on `cuda_stream` (NULL = legacy default stream), asynchronous;
 * the caller times the launch with events on that stream. Buffers are
 * caller-owned device memory.
 */
#ifndef RT_PROBES_H
#define RT_PROBES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Read `n_vec` 16-byte vectors of `buf` `reps` times with loads that bypass
 * L1 (cache-global), every CTA starting at a different offset each pass so
 * no SM re-reads its own lines back to back. The first pass pulls the buffer
 * into L2; with a buffer well below L2's capacity the remaining passes are L2
 * hits. Bytes read = 16 * n_vec * reps. One 16-byte word per thread of the
 * grid is written to `sink` (n_sink >= grid threads, else RT_ERR_INVALID_ARG)
 * so no load is dead. `buf` must be 16-byte aligned. Grid: 4 CTAs of 512
 * threads per SM. */
int rt_probe_l2_read(const void* buf, uint64_t n_vec, uint32_t reps, void* sink,
                     uint64_t n_sink, void* cuda_stream);

/* Grid threads needed by rt_probe_l2_read's `sink` on the current device. */
uint64_t rt_probe_l2_threads(void);

/* Issue `iters` x 8 independent MUFU reciprocal-square-root operations per
 * thread over a grid of 8 CTAs of 256 threads per SM; operations issued =
 * rt_probe_mufu_threads() * iters * 8. Each thread stores one float to `sink`
 * (n_sink >= rt_probe_mufu_threads(), else RT_ERR_INVALID_ARG). */
int rt_probe_mufu(uint32_t iters, float* sink, uint64_t n_sink, void* cuda_stream);

/* Grid threads of rt_probe_mufu on the current device. */
uint64_t rt_probe_mufu_threads(void);

#ifdef __cplusplus
}
#endif

#endif /* RT_PROBES_H */
