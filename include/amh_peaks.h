/*
 * amh_peaks.h -- microbenchmarks of the units that bound the sweeps
 * (libamh_peaks.so, separate from the sampler's libamh.so).
 *
 * The global sweep's pair term is FP32-pipe work (FFMA/FADD) plus one MUFU
 * square root and one table gather from L1/L2, so its roofline is stated
 * against the FP32 FMA issue rate, the MUFU rate and the L2 read bandwidth
 * measured on the device that runs the benchmark.  The paper has no
 * counterpart; it times its own GPU against a CPU.
 */
#ifndef AMH_PEAKS_H
#define AMH_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * amh_measure_peaks -- on the current CUDA device, synchronously:
 *   fp32_fma_per_s       FFMA instructions per second, whole GPU (8
 *                        independent chains per thread, 2048 threads per SM)
 *   mufu_sqrt_per_s      sqrt.approx.f32 per second, whole GPU
 *   l2_read_bytes_per_s  bytes per second read from a buffer of half the L2
 *                        size, resident in L2 (16-byte loads that bypass L1)
 * All three outputs are host pointers owned by the caller.  Allocates and
 * frees about L2/2 bytes of device memory.  Returns 0, or the CUDA error
 * code of the first failing call (outputs then undefined).
 */
int amh_measure_peaks(double* fp32_fma_per_s, double* mufu_sqrt_per_s,
                      double* l2_read_bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* AMH_PEAKS_H */
