// Kernels of the split-form DGSEM right-hand side and its adjoint for polynomial degree N = 4.
#define DG_N 4
#include "dg_kernels.cuh"
#include "dg_adjoint.cuh"
#include "dg_table.cuh"
