// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 3.
#define DG_N 3
#include "dg_kernels.cuh"
