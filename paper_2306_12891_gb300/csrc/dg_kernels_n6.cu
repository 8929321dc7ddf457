// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 6.
#define DG_N 6
#include "dg_kernels.cuh"
