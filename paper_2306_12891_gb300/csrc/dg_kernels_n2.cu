// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 2.
#define DG_N 2
#include "dg_kernels.cuh"
