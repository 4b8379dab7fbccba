// Sweep, gradient and coefficient-table kernels instantiated for nx = 96.
#include "lsm_sweep.cuh"
LSM_DEFINE_N(96)
