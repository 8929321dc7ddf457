// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 1.
#define DG_N 1
#include "dg_kernels.cuh"
