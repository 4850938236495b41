// KPM runners for complex FP64 vectors and FP64 matrix values (the step
// kernels of every FP64 shape are instantiated here).
#include "kpm_runner.cuh"

GPUTB_DEFINE_KPM_ENTRY(double)
