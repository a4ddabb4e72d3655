/*
 * dpcs_probe.h -- roof probes of the DPCS measurement library
 * (libdpcs_probe.so, built beside libdpcs.so and loaded only by the
 * benchmark and its tests).  Measurement helpers with no counterpart in the
 * paper: the render and replay kernels load a scene and textures that stay
 * resident in L2, and the replay scatters gradients with float4 atomics;
 * these calls measure both rates on a device so that the kernels' rooflines
 * can be stated against them.  Each call selects `device`, allocates its own
 * device buffer for the call's duration, runs on the legacy default stream,
 * times the best of three launches after one warm-up with CUDA events, and
 * returns after synchronising.  Return value: 0 on success, -1 for a bad
 * argument, -2 when the buffer cannot be allocated, -3 when a CUDA call
 * fails (the same codes as dpcs.h's DPCS_OK / DPCS_ERR_INVALID_ARG /
 * DPCS_ERR_OOM / DPCS_ERR_CUDA).
 *
 * dpcs_probe_l2_load: reads a zeroed `bytes` buffer `passes` times with
 * 16-byte loads that cache in L2 only; *gbs = bytes * passes / time in GB/s.
 * bytes must be a positive multiple of 16 up to 64 MiB (so it stays in L2)
 * and passes in [1, 4096].
 *
 * dpcs_probe_atomic4: about n_atomics float4 atomic adds (rounded up to a
 * whole number per thread) at pseudo-random texels of a `texels`-entry float4
 * buffer, so the lanes of a warp hit unrelated addresses; *gatomics = adds
 * per second / 1e9.  texels in [1, 2^24], n_atomics in [1, 2^34].
 */
#ifndef DPCS_PROBE_H
#define DPCS_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int32_t dpcs_probe_l2_load(int32_t device, size_t bytes, int32_t passes, double *gbs);
int32_t dpcs_probe_atomic4(int32_t device, int32_t texels, int64_t n_atomics, double *gatomics);

#ifdef __cplusplus
}
#endif

#endif /* DPCS_PROBE_H */
