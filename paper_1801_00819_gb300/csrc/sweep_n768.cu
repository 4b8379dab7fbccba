// Sweep, gradient and coefficient-table kernels instantiated for nx = 768.
#include "lsm_sweep.cuh"
LSM_DEFINE_N(768)
