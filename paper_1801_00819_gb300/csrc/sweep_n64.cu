// Sweep, gradient and coefficient-table kernels instantiated for nx = 64.
#include "lsm_sweep.cuh"
LSM_DEFINE_N(64)
