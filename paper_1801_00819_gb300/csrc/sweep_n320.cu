// Sweep, gradient and coefficient-table kernels instantiated for nx = 320.
#include "lsm_sweep.cuh"
LSM_DEFINE_N(320)
