// dg_table.cuh -- the kernel table of one polynomial degree (forward and adjoint launchers),
// included last by dg_kernels_nN.cu.
#pragma once

#define DG_CAT2(a, b) a##b
#define DG_CAT(a, b) DG_CAT2(a, b)
const DgKernelTable DG_CAT(dg_kernels_n, DG_N) = {
    N,                 upload,          launch_metrics,    launch_face_normals, launch_face,
    launch_lift,       launch_volume,   launch_indicator,  launch_spread,       launch_invariants,
    launch_max_dt,     launch_shadow,   launch_adj_face,   launch_adj_visc,     launch_adj_volume,
    launch_ke_grad};
