// KPM runners for complex FP32 vectors and FP32 matrix values (the step
// kernels of every FP32 shape are instantiated here).
#include "kpm_runner.cuh"

GPUTB_DEFINE_KPM_ENTRY(float)
