// Sweep, gradient and coefficient-table kernels instantiated for nx = 1024.
#include "lsm_sweep.cuh"
LSM_DEFINE_N(1024)
