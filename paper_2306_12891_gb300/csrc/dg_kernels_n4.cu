// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 4.
#define DG_N 4
#include "dg_kernels.cuh"
