/*
 * perm_probe.h -- issue-rate probes used by the benchmark to measure the roofline
 * denominators of this GPU (the FP64 pipe, the FP64 tensor cores and the integer
 * pipes).  They are measurement tools, not part of the paper's method.
 */
#ifndef PERM_PROBE_H_
#define PERM_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PERM_PROBE_DFMA = 0,  /* FP64 fused multiply-add instructions per second */
  PERM_PROBE_DMMA = 1,  /* FP64 tensor-core (mma.sync m8n8k4) flops per second */
  PERM_PROBE_IMAD = 2,  /* 32-bit integer multiply-add instructions per second */
  PERM_PROBE_IADD = 3,  /* 32-bit integer add instructions per second */
  PERM_PROBE_FFMA = 4   /* FP32 fused multiply-add instructions per second */
} perm_probe_kind;

/* Run a dependent-chain throughput kernel of the given kind on `device` for about
 * 50 ms (best of three launches on `stream`, timed with CUDA events) and write the
 * measured rate to *rate (unit per kind above).  Returns 0 (PERM_OK) or the
 * perm_status of the failure (PERM_EINVAL for an unknown kind or null rate,
 * PERM_ECUDA for a CUDA error). */
int perm_probe_rate(int device, int kind, void* stream, double* rate);

#ifdef __cplusplus
}
#endif

#endif /* PERM_PROBE_H_ */
