// Kernels of the split-form DGSEM right-hand side for polynomial degree N = 5.
#define DG_N 5
#include "dg_kernels.cuh"
