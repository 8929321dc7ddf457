// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 7.
#define DG_N 7
#include "dg_kernels.cuh"
