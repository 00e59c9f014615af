/*
 * ed_probes.h -- measured on-chip ceilings of the current CUDA device
 * (libed_probes.so).  Measurement support for the roofline of the H v kernel
 * of libhubbard_ed.so: when its DRAM traffic is already at the algorithmic
 * bytes, the rates below (how fast L2 and shared memory deliver data to the
 * SMs, and the FMA rates) are the ones that bound it.  No passage of the paper
 * corresponds; the paper runs on CPUs.
 */
#ifndef HUBBARD_ED_PROBES_H
#define HUBBARD_ED_PROBES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double l2_read_gbs;       /* 16-byte ld.global.cg reads of a 32 MB buffer held in L2,
                               100 passes, 8 CTAs of 256 threads per SM              */
  double hbm_read_gbs;      /* one streaming read of a 4 GB buffer (read bytes only)  */
  double smem_read_gbs;     /* conflict-free 16-byte shared-memory reads, all SMs     */
  double fp32_fma_tflops;   /* scalar FFMA, 2 flops per FMA                            */
  double fp32x2_fma_tflops; /* packed fma.rn.f32x2, 4 flops per instruction            */
  double fp64_fma_tflops;   /* DFMA, 2 flops per FMA                                   */
  int sms;                  /* multiprocessors of the device                           */
} ed_ceilings;

/* Run every probe once (after a warm-up launch each) on the current device
 * and fill *out.  Allocates 4 GB + 32 MB of device memory for the duration of
 * the call and takes about a second.  Returns 0, or the cudaError_t code of
 * the first failing CUDA call (out partially filled).                       */
int ed_probe_ceilings(ed_ceilings* out);

/* Launch, once each, four one-warp kernels (k_probe_lds<0..3>) that load
 * 16-byte words from shared memory in fixed patterns: one address for all
 * lanes; 32 consecutive words; every quarter warp 2-way in four bank groups
 * with the two quarters of each half warp in disjoint groups; every quarter
 * warp 8-way.  The call only launches them; the wavefronts each pattern
 * costs are read with a profiler.  Allocates 128 bytes of device memory for
 * the duration of the call.  Returns 0, or the cudaError_t code of the first
 * failing CUDA call.                                                          */
int ed_probe_shared_loads(void);

#ifdef __cplusplus
}
#endif

#endif /* HUBBARD_ED_PROBES_H */
