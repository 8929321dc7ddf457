// dg_fp32.cuh -- the FP32-bulk volume and lifting kernels without the blend, for ONE polynomial
// degree: the node-per-thread volume kernel, its TMA-fed and warp-specialised persistent forms, the
// pair-symmetric line kernel (N = 7) and the TMA-fed lifting kernel. Part of dg_kernels.cuh, which
// includes it after its shared definitions (degree constants, tables, flux helpers, k_lift's per-node
// functions); the code lives in the same unnamed namespace.
#pragma once

namespace {

// ---------------------------------------------------------------------------------------------
// FP32-bulk volume kernel without the blend: one thread per node. FP32 flux arithmetic is cheap on
// this GPU, so the pair symmetry that halves the FP64 work is given up here: each thread forms
// all 3(n-1) two-point fluxes of its node's lines and keeps its sums in registers, which removes
// the partner accumulators and two block barriers of the line-per-thread layout, and the metric
// terms are staged in shared memory with the primitives (one coalesced load per element).
// ---------------------------------------------------------------------------------------------
constexpr int NODE_EPB = nnn >= 256 ? 1 : 256 / nnn;
constexpr int NODE_THREADS = round32(NODE_EPB * nnn);
constexpr int NODE_SLOTS = 7 + 9 + 12;  // staged primitives, metric terms, contravariant viscous flux


// scaled two-point flux of the staged nodes a and b through the metric sums Sj (see line_fluxdiff);
// P holds the staged quantities [7][nnn] (node index, no padding)
template <int VF>
__device__ __forceinline__ void pair_flux_f(const float *__restrict__ P, int a, int b, float Sjx, float Sjy,
                                            float Sjz, float gam, float pref, float F[5]) {
  const float ri = P[a], ui = P[nnn + a], vi = P[2 * nnn + a], wi = P[3 * nnn + a];
  const float rm = P[b], um = P[nnn + b], vm = P[2 * nnn + b], wm = P[3 * nnn + b];
  if (VF == VF_PIR || VF == VF_KG) {
    const float Su = ui + um, Sv = vi + vm, Sw = wi + wm;
    const float Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;
    F[0] = (ri + rm) * Vp;
    const float Sp = P[4 * nnn + a] + P[4 * nnn + b];
    F[1] = F[0] * Su + Sp * Sjx;
    F[2] = F[0] * Sv + Sp * Sjy;
    F[3] = F[0] * Sw + Sp * Sjz;
    if (VF == VF_PIR) F[4] = F[0] * (P[5 * nnn + a] + P[5 * nnn + b]);
    else F[4] = F[0] * (P[5 * nnn + a] + P[5 * nnn + b]) + (P[6 * nnn + a] + P[6 * nnn + b]) * Vp;
  } else {
    const float av[3] = {0.5f * Sjx, 0.5f * Sjy, 0.5f * Sjz};
    if (VF == VF_EC) {
      ec_flux<float>(ri, ui, vi, wi, P[6 * nnn + a], rm, um, vm, wm, P[6 * nnn + b], av, gam, pref, F);
    } else {
      const float Vi = ui * av[0] + vi * av[1] + wi * av[2], Vm = um * av[0] + vm * av[1] + wm * av[2];
      const float pm2 = 0.125f * (P[4 * nnn + a] + P[4 * nnn + b]);
      F[0] = 0.5f * (ri * Vi + rm * Vm);
      F[1] = 0.5f * (ri * ui * Vi + rm * um * Vm) + pm2 * av[0];
      F[2] = 0.5f * (ri * vi * Vi + rm * vm * Vm) + pm2 * av[1];
      F[3] = 0.5f * (ri * wi * Vi + rm * wm * Vm) + pm2 * av[2];
      F[4] = 0.5f * (P[5 * nnn + a] * Vi + P[5 * nnn + b] * Vm);
    }
  }
}

// staged quantities of one node (rho, u, v, w, 4p', X, Y; see k_volume) from its FP32 shadow state;
// Pn points at the node's entry of P [7][nnn]
template <int VF>
__device__ __forceinline__ void f32_stage(const DgDevice &d, const float Uv[5], float *Pn) {
  const float gm1 = d.gm1_f, pref = d.p_ref_f;
  const float r = Uv[0], ir = 1.0f / r;
  const float u = Uv[1] * ir, v = Uv[2] * ir, w = Uv[3] * ir;
  const float pm = gm1 * (Uv[4] - 0.5f * (Uv[1] * u + Uv[2] * v + Uv[3] * w));
  const float p = pm + pref;
  const float Et = Uv[4] + (float)d.eref;
  if (!(r > 0.0f) || !(p > 0.0f) || !isfinite(Uv[4])) flag_set(d.flag, 1);
  Pn[0] = r; Pn[nnn] = u; Pn[2 * nnn] = v; Pn[3 * nnn] = w; Pn[4 * nnn] = 4.0f * pm;
  if (VF == VF_PIR) Pn[5 * nnn] = (Et + p) * ir;
  else if (VF == VF_KG) { Pn[5 * nnn] = Et * ir; Pn[6 * nnn] = 2.0f * p; }
  else if (VF == VF_EC) Pn[6 * nnn] = p;
  else Pn[5 * nnn] = Et + p;
}

// D_im with a zero diagonal, rows padded to n + 1 floats, in shared memory: the node-per-thread
// kernels index it by the thread's own node, which would serialise a constant-memory load
constexpr int DZ_STRIDE = n + 1;
__device__ __forceinline__ void fill_dz(float *Dz, int tid, int nthreads) {
  for (int t = tid; t < nn; t += nthreads) Dz[(t / n) * DZ_STRIDE + t % n] = 0.5f * f_D2[t];  // exact
}

// the node's flux differencing, surface terms and (Navier-Stokes) viscous divergence with the
// neighbour's or the wall's viscous trace, summed into s. P [7][nnn], J [9][nnn] (slot 3d + c),
// F [12][nnn] (contravariant viscous flux of this element) staged; Fs = this element's face slots
// [6][5][nn] (shared or global memory); Dz from fill_dz.
// The line sums skip the zero diagonal (partner m = mm or mm + 1) and take D itself; the split-form
// scalings D/4 (mass), D/8 (momentum, energy) or 2D (EC, central) are powers of two, applied once at
// the end, so the flux-differencing sums are those of the scaled tables bit for bit.
template <int VF>
__device__ __forceinline__ void f32_node_terms(const DgDevice &d, const float *__restrict__ P,
                                               const float *__restrict__ J, const float *__restrict__ F,
                                               const float *__restrict__ Fs, const float *__restrict__ Dz,
                                               int e, int node, float s[5]) {
  const float gam = d.gamma_f, pref = d.p_ref_f;
  const bool ns = d.equations == 1;
  const int ijk[3] = {node % n, (node / n) % n, node / nn};
  float a[5];  // flux differencing with D
#pragma unroll
  for (int v = 0; v < 5; ++v) a[v] = s[v] = 0.0f;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    const int id = ijk[dd];
    const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
    const int base = node - id * st;
    const float *Dr = Dz + id * DZ_STRIDE;
    const float *Fvd = F + (dd * 4) * nnn;
    const float jx = J[(3 * dd) * nnn + node], jy = J[(3 * dd + 1) * nnn + node], jz = J[(3 * dd + 2) * nnn + node];
    float vq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int mm = 0; mm < N; ++mm) {
      const int m = mm + (mm >= id ? 1 : 0);
      const int am = base + m * st;
      const float c = Dr[m];
      float Fp[5];
      pair_flux_f<VF>(P, node, am, jx + J[(3 * dd) * nnn + am], jy + J[(3 * dd + 1) * nnn + am],
                      jz + J[(3 * dd + 2) * nnn + am], gam, pref, Fp);
#pragma unroll
      for (int v = 0; v < 5; ++v) a[v] += c * Fp[v];
      if (ns) {  // viscous divergence along the line
#pragma unroll
        for (int q = 0; q < 4; ++q) vq[q] += c * Fvd[q * nnn + am];
      }
    }
    const bool face = id == 0 || id == N;
    const int f = 2 * dd + (id == N ? 1 : 0);
    const int pp = dd == 0 ? ijk[1] : ijk[0], qq = dd == 2 ? ijk[1] : ijk[2];
    const float iw = id == 0 ? f_invw[0] : f_invw[N];  // two uniform constant loads
    if (face) {  // surface term: (1/w_b) times the outward face flux
      const float *fs = Fs + f * 5 * nn + pp + n * qq;
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] += iw * fs[v * nn];
    }
    if (ns) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s[1 + q] -= vq[q];
      // the neighbour's outward normal viscous flux -(1/(2 w_b)) phi_nb at the element faces
      if (face) {
        const int *ef = d.ef + ((size_t)e * 6 + f) * 4;
        const int nb = ef[0], fnb = ef[1], o = ef[2];
        if (nb < 0) {  // wall-model flux: (1/w_b) (F*_wall - (+-) Fv_own / 2), see k_volume
          const float *fw = d.Fwall_f + (size_t)ef[3] * 4 * nn + pp + n * qq;
          const float hs = (id == N) ? 0.5f : -0.5f;
#pragma unroll
          for (int q = 0; q < 4; ++q) s[1 + q] -= iw * (fw[q * nn] - hs * F[(dd * 4 + q) * nnn + node]);
        } else {
          int p2, q2;
          orient_map(o, pp, qq, p2, q2);
          const int nbnode = face_node(fnb, p2, q2);
          const float sg = (fnb & 1) ? 0.5f : -0.5f;
          const float *Fvn = d.Fv_f + ((size_t)nb * 12 + (fnb >> 1) * 4) * nnn + nbnode;
#pragma unroll
          for (int q = 0; q < 4; ++q) s[1 + q] += iw * sg * Fvn[q * nnn];
        }
      }
    }
  }
  if (VF == VF_PIR || VF == VF_KG) {
    s[0] += 0.25f * a[0];
#pragma unroll
    for (int v = 1; v < 5; ++v) s[v] += 0.125f * a[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += 2.0f * a[v];
  }
}

// -1/J and the output / LSERK(5,4) stage in FP64 for one node; Ue, ge point at this element's state
// and register slices [5][nnn] to read (shared or global memory), out and g are global
__device__ __forceinline__ void f32_finish_reg(const DgDevice &d, const double Uv[5], const double gv0[5],
                                               float cf, double *out, double *__restrict__ g, int e, int node,
                                               const float s[5], int mode, int first, double dt, double A,
                                               double B) {
  // Uv, gv0: this node's U and g; cf: its float(1/J) (mode 0) or float(dt (-1/J)) (mode 1, formed in
  // FP64 and rounded once per step size by dg_api's k_stage_factor).
  // The right-hand side -s/J, or the stage increment dt (-1/J) s, is one FP32 product of the FP32 sum
  // s with the factor -1/J or dt (-1/J) (GB300 issues FP64 at 1/64 of the FP32 rate, and this
  // epilogue bounds the kernel); the LSERK register and the state accumulate in FP64. Explicit
  // roundings (no compiler contraction) keep every kernel variant's bits.
  (void)dt;
  const size_t gi = (size_t)e * 5 * nnn + node;
  if (mode == 0) {
    const float c = -cf;  // float(-1/J) = -float(1/J): rounding to nearest is symmetric
#pragma unroll
    for (int v = 0; v < 5; ++v) out[gi + v * nnn] = f2d_int(__fmul_rn(s[v], c));
    return;
  }
  const float c = cf;
  const double eref = d.eref;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double du = f2d_int(__fmul_rn(s[v], c));
    const double gv = first ? du : __fma_rn(A, gv0[v], du);
    g[gi + v * nnn] = gv;
    const double un = __fma_rn(B, gv, Uv[v]);
    out[gi + v * nnn] = un;
    d.Uf[gi + v * nnn] = d2f_int(v == 4 ? __dsub_rn(un, eref) : un);
  }
}

// the same with this element's U, g and 1/J read from global memory or a shared-memory copy
__device__ __forceinline__ void f32_finish(const DgDevice &d, const double *Ue, const double *ge,
                                           const float *ce, double *out, double *__restrict__ g, int e,
                                           int node, const float s[5], int mode, int first, double dt,
                                           double A, double B) {
  double Uv[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gv0[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (mode == 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Uv[v] = Ue[node + v * nnn];
      if (!first) gv0[v] = ge[node + v * nnn];
    }
  }
  f32_finish_reg(d, Uv, gv0, ce[node], out, g, e, node, s, mode, first, dt, A, B);
}

template <int VF>
__global__ void __launch_bounds__(NODE_THREADS, 2) k_volume_f32(const DgDevice d, const double *U, double *out,
                                                                 double *__restrict__ g, int mode, int first,
                                                                 double dt, double A, double B) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float *P = reinterpret_cast<float *>(sm_raw);  // [EPB][7][nnn] staged primitives
  float *JS = P + NODE_EPB * 7 * nnn;            // [EPB][9][nnn] metric terms Ja^d_c, slot 3d + c
  float *FS = JS + NODE_EPB * 9 * nnn;           // [EPB][12][nnn] contravariant viscous flux (NS)
  __shared__ float s_Dz[n * DZ_STRIDE];
  fill_dz(s_Dz, threadIdx.x, blockDim.x);
  const int e0 = blockIdx.x * NODE_EPB;
  for (int t = threadIdx.x; t < NODE_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    float Uv[5];
    load_state<float>(d, U, e, node, Uv);
    f32_stage<VF>(d, Uv, P + le * 7 * nnn + node);
    const float *Jn = d.Jaf + (size_t)e * 9 * nnn + node;
    float *Je = JS + le * 9 * nnn + node;
#pragma unroll
    for (int k = 0; k < 9; ++k) Je[k * nnn] = Jn[k * nnn];
    if (d.equations == 1) {
      const float *Fn = d.Fv_f + (size_t)e * 12 * nnn + node;
      float *Fe = FS + le * 12 * nnn + node;
#pragma unroll
      for (int k = 0; k < 12; ++k) Fe[k * nnn] = Fn[k * nnn];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NODE_EPB * nnn; t += blockDim.x) {
    const int le = t / nnn, node = t % nnn, e = e0 + le;
    if (e >= d.nE) continue;
    float s[5];
    f32_node_terms<VF>(d, P + le * 7 * nnn, JS + le * 9 * nnn, FS + le * 12 * nnn,
                       d.Fsurf_f + (size_t)e * 6 * 5 * nn, s_Dz, e, node, s);
    const size_t ge0 = (size_t)e * 5 * nnn;
    f32_finish(d, U + ge0, g + ge0, (mode ? d.facf : d.invJf) + (size_t)e * nnn, out, g, e, node, s, mode, first,
               dt, A, B);
  }
}

// ---------------------------------------------------------------------------------------------
// The same FP32-bulk volume operator as a persistent kernel fed by TMA bulk copies: one CTA per SM
// (or two) walks its elements; each element's contiguous slices -- FP32 state, metric terms,
// viscous flux, face slots and the FP64 state and LSERK register -- are copied into shared memory
// with cp.async.bulk one element ahead (double buffer, one mbarrier per buffer), so the next
// element's loads overlap this element's arithmetic. Needs element slices that are multiples of
// 16 bytes (N = 3, 5, 7) and 16-byte aligned U, g and output.
// ---------------------------------------------------------------------------------------------
constexpr bool TMA_OK = (N == 3 || N == 5 || N == 7);
constexpr int TMA_THREADS = round32(nnn);
constexpr unsigned TB_UF = 5u * nnn * 4u, TB_JA = 9u * nnn * 4u, TB_FV = 12u * nnn * 4u, TB_FS = 30u * nn * 4u;
// TB_IJ: the node factor of the epilogue, float(1/J) or float(dt (-1/J)) (f32_finish_reg)
constexpr unsigned TB_U = 5u * nnn * 8u, TB_G = 5u * nnn * 8u, TB_IJ = nnn * 4u;
constexpr unsigned TB_BUF = TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G + TB_IJ;
constexpr unsigned TB_P = 7u * nnn * 4u;
constexpr unsigned TB_SMEM = 2u * TB_BUF + TB_P + 16u;
static_assert(!TMA_OK || (TB_UF % 16 == 0 && TB_JA % 16 == 0 && TB_FV % 16 == 0 && TB_FS % 16 == 0 &&
                          TB_U % 16 == 0 && TB_IJ % 16 == 0 && TB_P % 16 == 0), "TMA slices must be multiples of 16 bytes");
static_assert(!TMA_OK || TB_SMEM <= 232448, "TMA kernel exceeds the shared memory of one CTA");

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// wait for the phase with the given parity, giving up after ~2^31 clock cycles (about a second)
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int VF>
__global__ void __launch_bounds__(TMA_THREADS, 1) k_volume_f32_tma(const DgDevice d, const double *U, double *out,
                                                                    double *g, int mode, int first, double dt,
                                                                    double A, double B) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *P = reinterpret_cast<float *>(sm_tma + 2 * TB_BUF);
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm_tma + 2 * TB_BUF + TB_P);
  __shared__ int s_ok;
  __shared__ float s_Dz[n * DZ_STRIDE];
  const bool ns = d.equations == 1;
  const bool needU = mode == 1, needG = mode == 1 && !first;
  const unsigned bytes =
      TB_UF + TB_JA + TB_FS + TB_IJ + (ns ? TB_FV : 0u) + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fill_dz(s_Dz, tid, blockDim.x);
  __syncthreads();
  // copies of element group k into buffer k & 1 (thread 0)
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * TB_BUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, bytes);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV), d.Fsurf_f + e * 30 * nn, TB_FS, mb);
    if (needU) bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS), U + e * 5 * nnn, TB_U, mb);
    if (needG) bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U), g + e * 5 * nnn, TB_G, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G), (mode ? d.facf : d.invJf) + e * nnn,
             TB_IJ, mb);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  for (int k = 0;; ++k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) break;
    const unsigned mb = smem_addr(&bar[k & 1]), parity = (unsigned)((k >> 1) & 1);
    if (tid == 0) s_ok = mbar_wait(mb, parity) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {  // a copy never completed: report, wait (bounded) for the other buffer's copy, stop
      if (tid == 0) {
        flag_set(d.flag, 4);
        if (e + gridDim.x < d.nE) mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
      return;
    }
    mbar_wait(mb, parity);  // completed: returns at once and orders this thread's reads after the copy
    const unsigned char *b = sm_tma + (k & 1) * TB_BUF;
    const float *Uf = reinterpret_cast<const float *>(b);
    const float *Jb = reinterpret_cast<const float *>(b + TB_UF);
    const float *Fb = reinterpret_cast<const float *>(b + TB_UF + TB_JA);
    const float *Sb = reinterpret_cast<const float *>(b + TB_UF + TB_JA + TB_FV);
    const double *Ub = reinterpret_cast<const double *>(b + TB_UF + TB_JA + TB_FV + TB_FS);
    const double *Gb = reinterpret_cast<const double *>(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U);
    const float *Ib = reinterpret_cast<const float *>(b + TB_UF + TB_JA + TB_FV + TB_FS + TB_U + TB_G);
    if (tid < nnn) {
      const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
      f32_stage<VF>(d, Uv, P + tid);
    }
    __syncthreads();
    if (tid < nnn) {
      float s[5];
      f32_node_terms<VF>(d, P, Jb, Fb, Sb, s_Dz, (int)e, tid, s);
      f32_finish(d, Ub, Gb, Ib, out, g, (int)e, tid, s, mode, first, dt, A, B);
    }
    __syncthreads();  // buffer k & 1 and P are free again
    if (tid == 0) issue(k + 2);
  }
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised form of the TMA kernel: 16 compute warps stage the primitives and form the
// per-node sums of element k while 4 epilogue warps apply -1/J and the FP64 LSERK update to element
// k-1, so the FP64 epilogue overlaps the FP32 flux arithmetic instead of following it. The sums
// pass through shared memory (two buffers); hand-offs use mbarriers: full[b] (the compute threads
// arrive when sums are written) and empty[b] (the epilogue threads arrive when they are consumed).
// Every wait is bounded; the compute warps leave their loop together after a block-level barrier
// among themselves.
// ---------------------------------------------------------------------------------------------
constexpr int WS_COMPUTE = TMA_THREADS;
constexpr int WS_EPI = 128;
constexpr int WS_THREADS = WS_COMPUTE + WS_EPI;
constexpr unsigned WS_CBUF = TB_UF + TB_JA + TB_FV + TB_FS;  // per-element TMA slices (no U, g)
constexpr unsigned WS_S = 5u * nnn * 4u;                      // per-node sums of one element
constexpr unsigned WS_UG = TB_U + TB_G + TB_IJ;              // FP64 state, register and 1/J of one element
constexpr unsigned WS_SMEM = 2u * WS_CBUF + TB_P + 2u * WS_S + WS_UG + 64u;
static_assert(!TMA_OK || WS_SMEM <= 232448, "warp-specialised kernel exceeds the shared memory of one CTA");

__device__ __forceinline__ void mbar_init_n(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int VF>
__global__ void __launch_bounds__(WS_THREADS, 1) k_volume_f32_ws(const DgDevice d, const double *U, double *out,
                                                                  double *g, int mode, int first, double dt,
                                                                  double A, double B) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *P = reinterpret_cast<float *>(sm_tma + 2 * WS_CBUF);
  float *S = reinterpret_cast<float *>(sm_tma + 2 * WS_CBUF + TB_P);  // [2][5][nnn]
  unsigned char *UG = sm_tma + 2 * WS_CBUF + TB_P + 2 * WS_S;  // U [5][nnn], g [5][nnn], 1/J [nnn] (FP64)
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(UG + WS_UG);
  // bar[0..1]: TMA arrival per buffer; bar[2..3]: sums full; bar[4..5]: sums empty; bar[6]: U, g arrival
  __shared__ int s_abort, s_abort_e;
  __shared__ float s_Dz[n * DZ_STRIDE];
  const bool ns = d.equations == 1;
  const unsigned bytes = TB_UF + TB_JA + TB_FS + (ns ? TB_FV : 0u);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    mbar_init_n(smem_addr(&bar[2]), WS_COMPUTE);
    mbar_init_n(smem_addr(&bar[3]), WS_COMPUTE);
    mbar_init_n(smem_addr(&bar[4]), WS_EPI);
    mbar_init_n(smem_addr(&bar[5]), WS_EPI);
    mbar_init(smem_addr(&bar[6]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_abort_e = 0;
  }
  fill_dz(s_Dz, tid, blockDim.x);
  __syncthreads();
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * WS_CBUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, bytes);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + TB_FV), d.Fsurf_f + e * 30 * nn, TB_FS, mb);
  };
  if (tid < WS_COMPUTE) {
    if (tid == 0) {
      issue(0);
      issue(1);
    }
    int k = 0;
    for (;; ++k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) break;
      const int b = k & 1;
      const unsigned parity = (unsigned)((k >> 1) & 1);
      if (!mbar_wait(smem_addr(&bar[b]), parity)) s_abort = 1;
      const unsigned char *buf = sm_tma + b * WS_CBUF;
      const float *Uf = reinterpret_cast<const float *>(buf);
      if (tid < nnn && !s_abort) {
        const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
        f32_stage<VF>(d, Uv, P + tid);
      }
      named_sync(1, WS_COMPUTE);
      if (s_abort) break;
      float sv[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (tid < nnn)
        f32_node_terms<VF>(d, P, reinterpret_cast<const float *>(buf + TB_UF),
                           reinterpret_cast<const float *>(buf + TB_UF + TB_JA),
                           reinterpret_cast<const float *>(buf + TB_UF + TB_JA + TB_FV), s_Dz, (int)e, tid, sv);
      // the sums buffer b is free once the epilogue has consumed element k - 2
      if (k >= 2 && !mbar_wait(smem_addr(&bar[4 + b]), (unsigned)(((k >> 1) - 1) & 1))) s_abort = 1;
      if (tid < nnn) {
        float *Sb = S + b * 5 * nnn + tid;
#pragma unroll
        for (int v = 0; v < 5; ++v) Sb[v * nnn] = sv[v];
      }
      mbar_arrive(smem_addr(&bar[2 + b]));
      named_sync(1, WS_COMPUTE);  // buffer b and P are free again
      if (s_abort) break;
      if (tid == 0) issue(k + 2);
    }
    if (s_abort && tid == 0) {  // report; wait (bounded) for the next element's copy still in flight
      flag_set(d.flag, 4);
      if ((long long)blockIdx.x + (long long)(k + 1) * gridDim.x < d.nE)
        mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
    }
  } else {
    // epilogue warps: the FP64 state, register and 1/J of each element arrive by TMA one element
    // ahead (issued by the group's first thread once the whole group has finished with the buffer)
    const int et = tid - WS_COMPUTE;
    const bool needU = mode == 1, needG = mode == 1 && !first;
    const unsigned ug_bytes = TB_IJ + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
    auto issue_ug = [&](int k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) return;
      const unsigned mb = smem_addr(&bar[6]);
      mbar_expect_tx(mb, ug_bytes);
      if (needU) bulk_g2s(smem_addr(UG), U + e * 5 * nnn, TB_U, mb);
      if (needG) bulk_g2s(smem_addr(UG + TB_U), g + e * 5 * nnn, TB_G, mb);
      bulk_g2s(smem_addr(UG + TB_U + TB_G), (mode ? d.facf : d.invJf) + e * nnn, TB_IJ, mb);
    };
    if (et == 0) issue_ug(0);
    int k = 0;
    for (;; ++k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) break;
      const int b = k & 1;
      if (!mbar_wait(smem_addr(&bar[2 + b]), (unsigned)((k >> 1) & 1))) s_abort_e = 1;
      if (!mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1))) s_abort_e = 1;
      if (!s_abort_e) {
        const float *Sb = S + b * 5 * nnn;
        const double *Ue = reinterpret_cast<const double *>(UG), *ge = reinterpret_cast<const double *>(UG + TB_U);
        const float *iJe = reinterpret_cast<const float *>(UG + TB_U + TB_G);
        // all of the thread's nodes at once (unrolled): their conversion and FP64 chains overlap
#pragma unroll
        for (int r = 0; r < (nnn + WS_EPI - 1) / WS_EPI; ++r) {
          const int node = et + r * WS_EPI;
          if (node < nnn) {
            const float sv[5] = {Sb[node], Sb[nnn + node], Sb[2 * nnn + node], Sb[3 * nnn + node],
                                 Sb[4 * nnn + node]};
            f32_finish(d, Ue, ge, iJe, out, g, (int)e, node, sv, mode, first, dt, A, B);
          }
        }
      }
      mbar_arrive(smem_addr(&bar[4 + b]));
      named_sync(2, WS_EPI);  // the group is done with the U, g buffer
      if (s_abort_e) break;
      if (et == 0) issue_ug(k + 1);
    }
    if (s_abort_e && et == 0) {  // report; wait (bounded) for this element's copy, the one in flight
      flag_set(d.flag, 4);
      mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP32-bulk volume operator with pair symmetry (N = 7). 192 line threads (one per x, y or z line of
// the element) form each two-point flux once, for both of its nodes, and keep the sums of their
// line's eight nodes in registers. The per-direction sums go to shared memory, where 8 epilogue
// warps add the three directions and apply -1/J and the FP64 LSERK update to element k-1 while the
// line threads work on element k. The FP32 state, metric terms and viscous flux arrive by TMA bulk
// copies one element ahead (as in k_volume_f32_ws); the face slots and the neighbours' viscous
// traces at a line's two end nodes come from global memory at the start of its line phase. Staged
// primitives and the sums use an XOR-swizzled node order (ln_sw), so that x, y and z lines and
// node-consecutive warps all access them without shared-memory bank conflicts.
// The sums are kept unscaled: the split-form factors (1/4 mass, 1/8 momentum and energy for KG and
// Pirozzoli; 2 for EC and central) are powers of two, applied once by the epilogue, and the surface
// and viscous terms enter divided by them (exact).
// ---------------------------------------------------------------------------------------------
constexpr bool LN_OK = (N == 7);
// four warp groups: two of epilogue warps (threads 0-255), two of line warps (256-511: 192 line
// threads, 64 that only help staging); setmaxnreg moves registers from the epilogue groups to the
// line groups, whose eight nodes' values and sums need ~168 per thread
constexpr int LN_EPI = 256;
constexpr int LN_GROUP = 256;       // threads of the line warp groups
constexpr int LN_COMPUTE = 3 * nn;  // line threads
constexpr int LN_THREADS = LN_EPI + LN_GROUP;
constexpr int LN_REG_LAUNCH = 65536 / LN_THREADS, LN_REG_LINE = 168, LN_REG_EPI = 88;
static_assert(LN_EPI * LN_REG_EPI + LN_GROUP * LN_REG_LINE <= LN_THREADS * LN_REG_LAUNCH,
              "the register split must fit the registers the block is launched with");
constexpr unsigned LN_CBUF = TB_UF + TB_JA + TB_FV;  // per-element TMA slices of the line phase
constexpr unsigned LN_ACC = 15u * nnn * 4u;          // [3 d][5][nnn] per-direction sums
constexpr unsigned LN_SMEM = 2u * LN_CBUF + TB_P + 2u * LN_ACC + WS_UG + 64u;
static_assert(!LN_OK || LN_SMEM <= 232448 - 256, "line kernel exceeds the shared memory of one CTA");
static_assert(!LN_OK || (LN_CBUF % 16 == 0 && LN_ACC % 16 == 0), "shared-memory regions must stay 16-byte aligned");
static_assert(!LN_OK || (nnn % LN_EPI == 0 && nnn % LN_GROUP == 0 && LN_COMPUTE <= LN_GROUP),
              "the epilogue and staging threads take whole nodes");

// bijective swizzle of node (i, j, k) = i + 8 j + 64 k for N = 7 (identity otherwise): the five
// low bits (the bank) are (i ^ j, (j ^ k) mod 4), which differ across the 32 lanes of an x, y or z
// line warp and of a warp of consecutive nodes
__device__ __forceinline__ int ln_sw(int node) {
  if (N != 7) return node;
  const int i = node & 7, j = (node >> 3) & 7, k = node >> 6;
  return ((i ^ j) & 7) | (((j ^ k) & 3) << 3) | ((j >> 2) << 5) | (k << 6);
}

// two-point flux of staged values held in registers (slots as in f32_stage); Sj = Ja_i + Ja_m
template <int VF>
__device__ __forceinline__ void pair_flux_reg(float ri, float ui, float vi, float wi, float p4i, float xi, float yi,
                                              float rm, float um, float vm, float wm, float p4m, float xm, float ym,
                                              float Sjx, float Sjy, float Sjz, float gam, float pref, float F[5]) {
  if (VF == VF_PIR || VF == VF_KG) {
    const float Su = ui + um, Sv = vi + vm, Sw = wi + wm;
    const float Vp = Su * Sjx + Sv * Sjy + Sw * Sjz;
    F[0] = (ri + rm) * Vp;
    const float Sp = p4i + p4m;
    F[1] = F[0] * Su + Sp * Sjx;
    F[2] = F[0] * Sv + Sp * Sjy;
    F[3] = F[0] * Sw + Sp * Sjz;
    if (VF == VF_PIR) F[4] = F[0] * (xi + xm);
    else F[4] = F[0] * (xi + xm) + (yi + ym) * Vp;
  } else {
    const float av[3] = {0.5f * Sjx, 0.5f * Sjy, 0.5f * Sjz};
    if (VF == VF_EC) {
      ec_flux<float>(ri, ui, vi, wi, yi, rm, um, vm, wm, ym, av, gam, pref, F);
    } else {
      const float Vi = ui * av[0] + vi * av[1] + wi * av[2], Vm = um * av[0] + vm * av[1] + wm * av[2];
      const float pm2 = 0.125f * (p4i + p4m);
      F[0] = 0.5f * (ri * Vi + rm * Vm);
      F[1] = 0.5f * (ri * ui * Vi + rm * um * Vm) + pm2 * av[0];
      F[2] = 0.5f * (ri * vi * Vi + rm * vm * Vm) + pm2 * av[1];
      F[3] = 0.5f * (ri * wi * Vi + rm * wm * Vm) + pm2 * av[2];
      F[4] = 0.5f * (xi * Vi + xm * Vm);
    }
  }
}

// the line's values and sums (registers); pairs (I, M), I < M, visited by template recursion so
// that every array index is a compile-time constant
struct LineRegs {
  float r[n], u[n], v[n], w[n], p4[n], x[n], y[n], jx[n], jy[n], jz[n];
  float acc[n][5];
};
template <int VF, int I, int M>
__device__ __forceinline__ void line_pairs(LineRegs &R, float gam, float pref) {
  if constexpr (I < n - 1) {
    float F[5];
    pair_flux_reg<VF>(R.r[I], R.u[I], R.v[I], R.w[I], R.p4[I], R.x[I], R.y[I], R.r[M], R.u[M], R.v[M], R.w[M],
                      R.p4[M], R.x[M], R.y[M], R.jx[I] + R.jx[M], R.jy[I] + R.jy[M], R.jz[I] + R.jz[M], gam, pref, F);
    const float ci = f_D[I * n + M], cm = f_D[M * n + I];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R.acc[I][v] += ci * F[v];
      R.acc[M][v] += cm * F[v];
    }
    if constexpr (M + 1 < n) line_pairs<VF, I, M + 1>(R, gam, pref);
    else line_pairs<VF, I + 1, I + 2>(R, gam, pref);
  }
}

__device__ __forceinline__ void regs_inc_line() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(LN_REG_LINE));
}
__device__ __forceinline__ void regs_dec_epi() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(LN_REG_EPI));
}

template <int VF>
__global__ void __launch_bounds__(LN_THREADS, 1) k_volume_f32_line(const DgDevice d, const double *U, double *out,
                                                                    double *g, int mode, int first, double dt,
                                                                    double A, double B) {
  if constexpr (LN_OK) {
    extern __shared__ __align__(128) unsigned char sm_tma[];
    float *P = reinterpret_cast<float *>(sm_tma + 2 * LN_CBUF);            // [7][nnn], swizzled
    float *ACC = reinterpret_cast<float *>(sm_tma + 2 * LN_CBUF + TB_P);  // [2][3][5][nnn], swizzled
    unsigned char *UG = sm_tma + 2 * LN_CBUF + TB_P + 2 * LN_ACC;          // U, g, 1/J (FP64)
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(UG + WS_UG);
    // bar[0..1]: TMA arrival per buffer; bar[2..3]: sums full; bar[4..5]: sums empty; bar[6]: U, g, 1/J
    __shared__ int s_abort, s_abort_e;
    constexpr bool SPLIT = (VF == VF_PIR || VF == VF_KG);
    // 1 / (split-form factor) per variable: the sums are unscaled (see above)
    constexpr float ISC0 = SPLIT ? 4.0f : 0.5f, ISC1 = SPLIT ? 8.0f : 0.5f;
    const bool ns = d.equations == 1;
    const unsigned bytes = TB_UF + TB_JA + (ns ? TB_FV : 0u);
    const int tid = threadIdx.x;
    if (tid == 0) {
      mbar_init(smem_addr(&bar[0]));
      mbar_init(smem_addr(&bar[1]));
      mbar_init_n(smem_addr(&bar[2]), LN_GROUP);
      mbar_init_n(smem_addr(&bar[3]), LN_GROUP);
      mbar_init_n(smem_addr(&bar[4]), LN_EPI);
      mbar_init_n(smem_addr(&bar[5]), LN_EPI);
      mbar_init(smem_addr(&bar[6]));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_abort = 0;
      s_abort_e = 0;
    }
    __syncthreads();
    auto issue = [&](int k) {
      const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
      if (e >= d.nE) return;
      unsigned char *b = sm_tma + (k & 1) * LN_CBUF;
      const unsigned mb = smem_addr(&bar[k & 1]);
      mbar_expect_tx(mb, bytes);
      bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
      bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
      if (ns) bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.Fv_f + e * 12 * nnn, TB_FV, mb);
    };
    if (tid >= LN_EPI) {
      regs_inc_line();
      const int ct = tid - LN_EPI;  // thread of the line warp groups
      const bool line = ct < LN_COMPUTE;
      if (ct == 0) {
        issue(0);
        issue(1);
      }
      // this thread's line: direction dd (warp-uniform), position (la, lb) on the faces 2dd, 2dd+1
      const int dd = line ? ct / nn : 0, L = ct % nn, la = L % n, lb = L / n;
      const int st = dd == 0 ? 1 : dd == 1 ? n : nn;
      const int base = dd == 0 ? n * la + nn * lb : dd == 1 ? la + nn * lb : la + n * lb;
      const float gam = d.gamma_f, pref = d.p_ref_f;
      const float iw0 = f_invw[0], iwN = f_invw[N];
      // face records of the line's two faces, loaded one element ahead (a warp issues in order: an
      // address computed from a just-loaded record would stall it for a full memory latency)
      int4 rec_next[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
      if (ns && line && blockIdx.x < d.nE) {
        rec_next[0] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)blockIdx.x * 6 + 2 * dd) * 4);
        rec_next[1] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)blockIdx.x * 6 + 2 * dd + 1) * 4);
      }
      int k = 0;
      for (;; ++k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) break;
        const int b = k & 1;
        const int4 rec[2] = {rec_next[0], rec_next[1]};
        if (ns && line && e + gridDim.x < d.nE) {
          rec_next[0] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)(e + gridDim.x) * 6 + 2 * dd) * 4);
          rec_next[1] = *reinterpret_cast<const int4 *>(d.ef + ((size_t)(e + gridDim.x) * 6 + 2 * dd + 1) * 4);
        }
        if (!mbar_wait(smem_addr(&bar[b]), (unsigned)((k >> 1) & 1))) s_abort = 1;
        const unsigned char *buf = sm_tma + b * LN_CBUF;
        const float *Uf = reinterpret_cast<const float *>(buf);
        const float *Jb = reinterpret_cast<const float *>(buf + TB_UF);
        const float *Fb = reinterpret_cast<const float *>(buf + TB_UF + TB_JA);
        if (!s_abort)
          for (int t = ct; t < nnn; t += LN_GROUP) {
            const float Uv[5] = {Uf[t], Uf[nnn + t], Uf[2 * nnn + t], Uf[3 * nnn + t], Uf[4 * nnn + t]};
            f32_stage<VF>(d, Uv, P + ln_sw(t));
          }
        named_sync(1, LN_GROUP);
        if (s_abort) break;
        if (line) {
        // end-node data from global memory, loaded before the pair sums so that its latency overlaps them
        float fs[2][5], fnb[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        int wall[2] = {0, 0};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int f = 2 * dd + side;
          const float *Fs = d.Fsurf_f + ((size_t)e * 6 + f) * 5 * nn + L;
#pragma unroll
          for (int v = 0; v < 5; ++v) fs[side][v] = Fs[v * nn];
          if (ns) {
            const int4 r4 = rec[side];
            if (r4.x >= 0) {
              int p2, q2;
              orient_map(r4.z, la, lb, p2, q2);
              const float *Fvn = d.Fv_f + ((size_t)r4.x * 12 + (r4.y >> 1) * 4) * nnn + face_node(r4.y, p2, q2);
#pragma unroll
              for (int q = 0; q < 4; ++q) fnb[side][q] = Fvn[q * nnn];
            } else {  // wall: the wall-model flux, combined with the own trace below
              const float *fw = d.Fwall_f + (size_t)r4.w * 4 * nn + L;
#pragma unroll
              for (int q = 0; q < 4; ++q) fnb[side][q] = fw[q * nn];
              wall[side] = 1;
            }
          }
        }
        // the line's staged values and metric terms Ja^dd
        LineRegs R;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const int nd = base + i * st, sw = ln_sw(nd);
          R.r[i] = P[sw]; R.u[i] = P[nnn + sw]; R.v[i] = P[2 * nnn + sw]; R.w[i] = P[3 * nnn + sw];
          R.p4[i] = P[4 * nnn + sw];
          R.x[i] = (VF == VF_EC) ? 0.0f : P[5 * nnn + sw];
          R.y[i] = (VF == VF_KG || VF == VF_EC) ? P[6 * nnn + sw] : 0.0f;
          R.jx[i] = Jb[(3 * dd) * nnn + nd];
          R.jy[i] = Jb[(3 * dd + 1) * nnn + nd];
          R.jz[i] = Jb[(3 * dd + 2) * nnn + nd];
#pragma unroll
          for (int v = 0; v < 5; ++v) R.acc[i][v] = 0.0f;
        }
        // each pair (i, m), i < m, once: node i takes D_im F, node m takes D_mi F (F is symmetric)
        line_pairs<VF, 0, 1>(R, gam, pref);
        float (&acc)[n][5] = R.acc;
        // surface terms: (1/w_b) times the outward face flux at the end nodes
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float isc = v == 0 ? ISC0 : ISC1;
          acc[0][v] += (isc * iw0) * fs[0][v];
          acc[N][v] += (isc * iwN) * fs[1][v];
        }
        if (ns) {
          // viscous divergence along the line, then the neighbour's normal viscous flux or the wall
          // term at the end nodes (see k_volume)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float fv[n];
#pragma unroll
            for (int m = 0; m < n; ++m) fv[m] = Fb[(dd * 4 + q) * nnn + base + m * st];
#pragma unroll
            for (int i = 0; i < n; ++i) {
              float t = 0.0f;
#pragma unroll
              for (int m = 0; m < n; ++m)
                if (m != i) t += f_D[i * n + m] * fv[m];
              acc[i][1 + q] -= ISC1 * t;
            }
            const float sg0 = (rec[0].y & 1) ? 0.5f : -0.5f, sg1 = (rec[1].y & 1) ? 0.5f : -0.5f;
            acc[0][1 + q] += wall[0] ? -(ISC1 * iw0) * (fnb[0][q] + 0.5f * fv[0]) : (ISC1 * iw0 * sg0) * fnb[0][q];
            acc[N][1 + q] += wall[1] ? -(ISC1 * iwN) * (fnb[1][q] - 0.5f * fv[N]) : (ISC1 * iwN * sg1) * fnb[1][q];
          }
        }
        // the sums buffer b is free once the epilogue has consumed element k - 2
        if (k >= 2 && !mbar_wait(smem_addr(&bar[4 + b]), (unsigned)(((k >> 1) - 1) & 1))) s_abort = 1;
        float *Ab = ACC + (b * 3 + dd) * 5 * nnn;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const int sw = ln_sw(base + i * st);
#pragma unroll
          for (int v = 0; v < 5; ++v) Ab[v * nnn + sw] = acc[i][v];
        }
        }  // line
        mbar_arrive(smem_addr(&bar[2 + b]));
        named_sync(1, LN_GROUP);  // buffer b and P are free again
        if (s_abort) break;
        if (ct == 0) issue(k + 2);
      }
      if (s_abort && ct == 0) {  // report; wait (bounded) for the next element's copy still in flight
        flag_set(d.flag, 4);
        if ((long long)blockIdx.x + (long long)(k + 1) * gridDim.x < d.nE)
          mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
    } else {
      // epilogue warps: sum the three directions, scale, -1/J and the FP64 LSERK stage; the FP64
      // state, register and 1/J arrive by TMA one element ahead (issued once the group is done)
      regs_dec_epi();
      const int et = tid;
      const bool needU = mode == 1, needG = mode == 1 && !first;
      const unsigned ug_bytes = TB_IJ + (needU ? TB_U : 0u) + (needG ? TB_G : 0u);
      auto issue_ug = [&](int k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) return;
        const unsigned mb = smem_addr(&bar[6]);
        mbar_expect_tx(mb, ug_bytes);
        if (needU) bulk_g2s(smem_addr(UG), U + e * 5 * nnn, TB_U, mb);
        if (needG) bulk_g2s(smem_addr(UG + TB_U), g + e * 5 * nnn, TB_G, mb);
        bulk_g2s(smem_addr(UG + TB_U + TB_G), (mode ? d.facf : d.invJf) + e * nnn, TB_IJ, mb);
      };
      if (et == 0) issue_ug(0);
      constexpr float SC0 = SPLIT ? 0.25f : 2.0f, SC1 = SPLIT ? 0.125f : 2.0f;
      int k = 0;
      for (;; ++k) {
        const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
        if (e >= d.nE) break;
        const int b = k & 1;
        if (!mbar_wait(smem_addr(&bar[2 + b]), (unsigned)((k >> 1) & 1))) s_abort_e = 1;
        if (!mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1))) s_abort_e = 1;
        // the thread's nodes' sums, U, g and 1/J into registers first; then the sums buffer and the
        // U, g, 1/J buffer are released (the next element's copy overlaps this element's FP64 stage)
        constexpr int R = nnn / LN_EPI;
        float sv[R][5];
        double Uv[R][5], gv0[R][5];
        float iJ[R];
        if (!s_abort_e) {
          const float *A0 = ACC + (b * 3) * 5 * nnn, *A1 = A0 + 5 * nnn, *A2 = A1 + 5 * nnn;
          const double *Ue = reinterpret_cast<const double *>(UG), *ge = reinterpret_cast<const double *>(UG + TB_U);
          const float *iJe = reinterpret_cast<const float *>(UG + TB_U + TB_G);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int node = et + r * LN_EPI, sw = ln_sw(node);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              sv[r][v] = (v == 0 ? SC0 : SC1) * ((A0[v * nnn + sw] + A1[v * nnn + sw]) + A2[v * nnn + sw]);
              Uv[r][v] = needU ? Ue[node + v * nnn] : 0.0;
              gv0[r][v] = needG ? ge[node + v * nnn] : 0.0;
            }
            iJ[r] = iJe[node];
          }
        }
        mbar_arrive(smem_addr(&bar[4 + b]));
        named_sync(2, LN_EPI);  // the group is done with the U, g, 1/J buffer
        if (s_abort_e) break;
        if (et == 0) issue_ug(k + 1);
#pragma unroll
        for (int r = 0; r < R; ++r)
          f32_finish_reg(d, Uv[r], gv0[r], iJ[r], out, g, (int)e, et + r * LN_EPI, sv[r], mode, first, dt, A, B);
      }
      if (s_abort_e && et == 0) {  // report; wait (bounded) for this element's copy, the one in flight
        flag_set(d.flag, 4);
        mbar_wait(smem_addr(&bar[6]), (unsigned)(k & 1));
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP32-bulk BR1 lifting as a persistent kernel fed by TMA (N = 3, 5, 7): one thread per node, two
// CTAs per SM; each element's FP32 state, metric terms, 1/J and BR1 face jumps arrive by
// cp.async.bulk one element ahead into a double buffer, so the loads of the next element overlap
// this element's arithmetic. The per-node arithmetic is lift_prim / lift_node, as in k_lift.
// ---------------------------------------------------------------------------------------------
constexpr int LT_THREADS = TMA_THREADS;
constexpr unsigned LT_IJ = nnn * 4u, LT_WS = 24u * nn * 4u;
constexpr unsigned LT_BUF = TB_UF + TB_JA + LT_IJ + LT_WS;
constexpr unsigned LT_SMEM = 2u * LT_BUF + 4u * nnn * 4u + 16u;
static_assert(!TMA_OK || (LT_IJ % 16 == 0 && LT_WS % 16 == 0 && LT_BUF % 16 == 0),
              "TMA slices must be multiples of 16 bytes");

__global__ void __launch_bounds__(LT_THREADS, 2) k_lift_f32_tma(const DgDevice d) {
  extern __shared__ __align__(128) unsigned char sm_tma[];
  float *W = reinterpret_cast<float *>(sm_tma + 2 * LT_BUF);  // [4][nnn]
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm_tma + 2 * LT_BUF + 4 * nnn * 4);
  __shared__ float sD[n][n + 1];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  for (int t = tid; t < nn; t += blockDim.x) sD[t / n][t % n] = f_D[t];
  if (tid == 0) {
    mbar_init(smem_addr(&bar[0]));
    mbar_init(smem_addr(&bar[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) return;
    unsigned char *b = sm_tma + (k & 1) * LT_BUF;
    const unsigned mb = smem_addr(&bar[k & 1]);
    mbar_expect_tx(mb, LT_BUF);
    bulk_g2s(smem_addr(b), d.Uf + e * 5 * nnn, TB_UF, mb);
    bulk_g2s(smem_addr(b + TB_UF), d.Jaf + e * 9 * nnn, TB_JA, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA), d.invJf + e * nnn, LT_IJ, mb);
    bulk_g2s(smem_addr(b + TB_UF + TB_JA + LT_IJ), d.Wsurf_f + e * 24 * nn, LT_WS, mb);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  const float gm1 = d.gm1_f, iR = d.iR_f, pref = d.p_ref_f, mu = d.mu_f, kappa = d.kappa_f;
  for (int k = 0;; ++k) {
    const long long e = (long long)blockIdx.x + (long long)k * gridDim.x;
    if (e >= d.nE) break;
    const unsigned mb = smem_addr(&bar[k & 1]), parity = (unsigned)((k >> 1) & 1);
    if (tid == 0) s_ok = mbar_wait(mb, parity) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {  // a copy never completed: report, wait (bounded) for the other buffer's copy, stop
      if (tid == 0) {
        flag_set(d.flag, 4);
        if (e + gridDim.x < d.nE) mbar_wait(smem_addr(&bar[(k + 1) & 1]), (unsigned)(((k + 1) >> 1) & 1));
      }
      return;
    }
    mbar_wait(mb, parity);  // completed: returns at once and orders this thread's reads after the copy
    const unsigned char *b = sm_tma + (k & 1) * LT_BUF;
    const float *Uf = reinterpret_cast<const float *>(b);
    const float *Jb = reinterpret_cast<const float *>(b + TB_UF);
    const float *Ib = reinterpret_cast<const float *>(b + TB_UF + TB_JA);
    const float *Sb = reinterpret_cast<const float *>(b + TB_UF + TB_JA + LT_IJ);
    if (tid < nnn) {
      const float Uv[5] = {Uf[tid], Uf[nnn + tid], Uf[2 * nnn + tid], Uf[3 * nnn + tid], Uf[4 * nnn + tid]};
      float Wn[4];
      lift_prim<float>(Uv, gm1, iR, pref, Wn);
#pragma unroll
      for (int q = 0; q < 4; ++q) W[q * nnn + tid] = Wn[q];
    }
    __syncthreads();
    if (tid < nnn) lift_node<float>(d, tid, W, sD, Jb, Sb, Ib[tid], mu, kappa, d.Fv_f + (size_t)e * 12 * nnn);
    __syncthreads();  // buffer k & 1 and W are free again
    if (tid == 0) issue(k + 2);
  }
}

}  // namespace
