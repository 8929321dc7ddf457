// dg_api.cu -- the C ABI of libdg (declared in include/dg.h): context set-up, mesh validation,
// device buffers, the per-stage launch sequence and the LSERK(5,4) driver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_convert.cuh"
#include "dg_internal.h"

namespace {

const DgKernelTable *kernels_for(int N) {
  switch (N) {
    case 1: return &dg_kernels_n1;
    case 2: return &dg_kernels_n2;
    case 3: return &dg_kernels_n3;
    case 4: return &dg_kernels_n4;
    case 5: return &dg_kernels_n5;
    case 6: return &dg_kernels_n6;
    case 7: return &dg_kernels_n7;
    default: return nullptr;
  }
}

// constant-memory tables are per device and per degree; upload once
std::mutex g_upload_mutex;
std::vector<unsigned> g_uploaded;  // bitmask of degrees per device

enum KernelClass {
  KC_FACE = 0, KC_LIFT, KC_VOLUME, KC_INDICATOR, KC_SPREAD, KC_OTHER, KC_ADJ_FACE, KC_ADJ_VISC, KC_ADJ_VOLUME,
  KC_COUNT
};
const char *kKernelNames[KC_COUNT] = {"face",  "lift",     "volume",   "indicator", "spread",
                                      "other", "adj_face", "adj_visc", "adj_volume"};

// LSERK(5,4) of Carpenter and Kennedy, 2N-storage form (published coefficients)
const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};
// (the stage times t + c_s dt are not needed: no boundary condition or source depends on t)

}  // namespace

struct dg_ctx {
  int N = 0, device = 0;
  dg_params params{};
  DgDevice d{};
  const DgKernelTable *K = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  double *g = nullptr;         // LSERK register
  double *Ustage = nullptr;    // device copy for the host-buffer entry point (lazy)
  double *small = nullptr;     // 16 doubles of device scratch for reductions' results
  int *flag_host = nullptr;
  std::string err;
  long long launches = 0;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<int> ev_class;
  size_t ev_used = 0;
  double t_ms[KC_COUNT] = {0};
  long long t_count[KC_COUNT] = {0};
  size_t n_state = 0;          // doubles in U
  size_t n_tau = 0;            // doubles in a viscous stress record [nE][6][n^3] (Navier-Stokes adjoint)
  // adjoint: library-owned state buffers (stage states, gbar, checkpoints), allocated on first use
  std::vector<double *> adj_pool;
  // adjoint, Navier-Stokes: the lifting's viscous stress record of each state the reverse sweep
  // differentiates at (one step's stages, or a segment's)
  std::vector<double *> tau_pool;
  size_t adj_limit = 0;        // bytes the adjoint's buffers may use (0: free memory less 10%)
  // recorded forward run (dg_lserk_steps_record): every stage state (with its stress record), or
  // checkpoints
  std::vector<double *> tape_pool, tape_tau;
  long long tape_id = 0, tape_serial = 0;
  int tape_steps = 0, tape_interval = 0;
  bool tape_all = false;
  double tape_dt = 0.0;
  double fac_dt = std::nan("");  // step size of the FP32-bulk stage factor d.facf (NaN: not formed yet)
  // CUDA graph of one LSERK step, replayed by the multi-step calls on a library stream that is
  // ordered after (and before) the caller's stream with events
  int use_graphs = 1;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  // host-buffer entry point: the state's copies are split over library streams (one copy each), so
  // that several copy engines move it at once
  static constexpr int kCopyStreams = 4;
  cudaStream_t cstream[kCopyStreams] = {};
  cudaEvent_t cev[kCopyStreams + 1] = {};
  cudaGraphExec_t step_graph = nullptr;
  const double *graph_U = nullptr;
  double graph_dt = 0.0;
  long long graph_launches = 0;
};

namespace {

dg_status fail(dg_ctx *c, dg_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

dg_status cuda_fail(dg_ctx *c, cudaError_t e, const char *where) {
  return fail(c, DG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
dg_status dev_alloc(dg_ctx *c, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return DG_OK;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DG_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return DG_OK;
}

// Run one launch (a callable) with launch counting, optional event timing and error check.
template <class F>
dg_status launch(dg_ctx *c, int kc, F &&f) {
  if (c->timing) {
    if (c->ev_used == c->ev_pool.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      c->ev_pool.push_back({a, b});
      c->ev_class.push_back(kc);
    }
    c->ev_class[c->ev_used] = kc;
    cudaEventRecord(c->ev_pool[c->ev_used].first, c->stream);
  }
  f();
  cudaError_t e = cudaGetLastError();
  if (c->timing) {
    cudaEventRecord(c->ev_pool[c->ev_used].second, c->stream);
    ++c->ev_used;
  }
  ++c->launches;
  if (e != cudaSuccess) return cuda_fail(c, e, kKernelNames[kc]);
  return DG_OK;
}

#define DG_TRY(x)                  \
  do {                             \
    dg_status _s = (x);            \
    if (_s != DG_OK) return _s;    \
  } while (0)

// alpha for this stage (shock capturing with the indicator)
dg_status stage_alpha(dg_ctx *c, const double *U) {
  if (!c->d.shock_capturing || c->d.alpha_fixed >= 0.0) return DG_OK;
  DG_TRY(launch(c, KC_INDICATOR, [&] { c->K->indicator(c->d, U, c->stream); }));
  DG_TRY(launch(c, KC_SPREAD, [&] { c->K->spread(c->d, c->d.alpha, c->stream); }));
  return DG_OK;
}

// one right-hand-side evaluation; mode 0 writes Ut, mode 1 performs LSERK stage `stage`; tau
// (Navier-Stokes, optional): the lifting also writes its viscous stress record of U there
dg_status stage(dg_ctx *c, const double *U, double *out, int mode, int st, double dt, double *tau = nullptr) {
  DG_TRY(stage_alpha(c, U));
  DG_TRY(launch(c, KC_FACE, [&] { c->K->face(c->d, U, c->stream); }));
  if (c->d.equations == DG_NAVIER_STOKES)
    DG_TRY(launch(c, KC_LIFT, [&] { c->K->lift(c->d, U, tau, c->stream); }));
  const double A = mode ? kA[st] : 0.0, B = mode ? kB[st] : 0.0;
  DG_TRY(launch(c, KC_VOLUME, [&] { c->K->volume(c->d, U, out, c->g, mode, st == 0, dt, A, B, c->stream); }));
  return DG_OK;
}

__global__ void k_fill(double *p, int count, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

__global__ void k_scale(double *__restrict__ y, const double *__restrict__ x, double a, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// ---- discrete adjoint ----

dg_status adjoint_supported(dg_ctx *c, const char *who) {
  const DgDevice &d = c->d;
  if (d.precision != DG_FP64 || d.shock_capturing || d.n_walls ||
      (d.vflux != DG_VFLUX_KG && d.vflux != DG_VFLUX_PIROZZOLI))
    return fail(c, DG_ERR_UNSUPPORTED, std::string(who) +
                ": the adjoint needs DG_FP64, no shock capturing, no wall faces and the KG or Pirozzoli volume flux");
  return DG_OK;
}

// at least `count` library-owned state buffers in the adjoint pool
dg_status adj_pool(dg_ctx *c, size_t count) {
  while (c->adj_pool.size() < count) {
    double *p = nullptr;
    DG_TRY(dev_alloc(c, &p, c->n_state));
    c->adj_pool.push_back(p);
  }
  return DG_OK;
}

// at least `count` viscous stress records in the adjoint's pool (Navier-Stokes; none for Euler)
dg_status tau_fill(dg_ctx *c, size_t count) {
  if (!c->n_tau) return DG_OK;
  while (c->tau_pool.size() < count) {
    double *p = nullptr;
    DG_TRY(dev_alloc(c, &p, c->n_tau));
    c->tau_pool.push_back(p);
  }
  return DG_OK;
}

// the viscous stress record of U alone (the face and lifting kernels of a stage, no volume work)
dg_status record_tau(dg_ctx *c, const double *U, double *tau) {
  if (c->d.equations != DG_NAVIER_STOKES) return DG_OK;
  DG_TRY(launch(c, KC_FACE, [&] { c->K->face(c->d, U, c->stream); }));
  DG_TRY(launch(c, KC_LIFT, [&] { c->K->lift(c->d, U, tau, c->stream); }));
  return DG_OK;
}

// stress record i of the pool (null for Euler)
double *tau_at(dg_ctx *c, size_t i) { return c->n_tau ? c->tau_pool[i] : nullptr; }

// one vector-Jacobian product of L at U with cotangent lam (see DgKernelTable::adj_volume for modes);
// tau: the lifting's stress record of U (Navier-Stokes). The forward work buffers serve as scratch:
// Fsurf = face slots, Fv = cotW, Wsurf = sigma
dg_status vjp(dg_ctx *c, const double *U, const double *lam, double *out, int mode, double dt, double A, double B,
              int update_g, const double *tau) {
  DgDevice &d = c->d;
  DG_TRY(launch(c, KC_ADJ_FACE, [&] { c->K->adj_face(d, U, lam, d.Fsurf, c->stream); }));
  if (d.equations == DG_NAVIER_STOKES)
    DG_TRY(launch(c, KC_ADJ_VISC, [&] { c->K->adj_visc(d, U, lam, tau, d.Fv, d.Wsurf, c->stream); }));
  DG_TRY(launch(c, KC_ADJ_VOLUME, [&] {
    c->K->adj_volume(d, U, lam, d.Fsurf, d.Fv, d.Wsurf, out, const_cast<double *>(lam), mode, dt, A, B, update_g,
                     c->stream);
  }));
  return DG_OK;
}

dg_status copy_state(dg_ctx *c, double *dst, const double *src) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * c->n_state, cudaMemcpyDeviceToDevice, c->stream);
  return e ? cuda_fail(c, e, "state copy") : DG_OK;
}

// reverse of one LSERK step whose five stage input states are S[0..4], with their stress records
// T[0..4] (gbar in pool[4]):
// gbar = B_5 Ubar; for s = 5..1: Ubar += dt (dL/dU)(S[s-1])^T gbar; gbar = A_s gbar + B_(s-1) Ubar
dg_status reverse_stages(dg_ctx *c, double *const S[5], double *const T[5], double *Ubar, double dt) {
  double *gbar = c->adj_pool[4];
  DG_TRY(launch(c, KC_OTHER, [&] { k_scale<<<8 * 152, 256, 0, c->stream>>>(gbar, Ubar, kB[4], c->n_state); }));
  for (int st = 4; st >= 0; --st)
    DG_TRY(vjp(c, S[st], gbar, Ubar, 1, dt, kA[st], st > 0 ? kB[st - 1] : 0.0, st > 0, T[st]));
  return DG_OK;
}

dg_status steps_impl(dg_ctx *c, double *U, double dt, int n_steps);

// device bytes of `states` state buffers and `taus` stress records
size_t adj_bytes(const dg_ctx *c, size_t states, size_t taus) {
  return sizeof(double) * (states * c->n_state + taus * c->n_tau);
}

// bytes the adjoint's and the tape's buffers hold now
size_t adj_held(const dg_ctx *c) {
  return adj_bytes(c, c->adj_pool.size() + c->tape_pool.size(), c->tau_pool.size() + c->tape_tau.size());
}

// whether buffers of `need` bytes fit in the adjoint's memory budget, counting `have` already held
bool budget_allows(dg_ctx *c, size_t need, size_t have) {
  if (c->adj_limit) return need <= c->adj_limit;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t extra = need > have ? need - have : 0;
  return extra + total_b / 10 < free_b;
}

// at least `count` library-owned buffers of `doubles` doubles (default: a state) in `pool`
dg_status pool_fill(dg_ctx *c, std::vector<double *> &pool, size_t count, size_t doubles = 0) {
  while (pool.size() < count) {
    double *p = nullptr;
    DG_TRY(dev_alloc(c, &p, doubles ? doubles : c->n_state));
    pool.push_back(p);
  }
  return DG_OK;
}

// reverse of one LSERK step from U, recomputing its four inner stage states into pool[0..3] and the
// five stress records into the stress pool [0..4]
dg_status step_vjp(dg_ctx *c, const double *U, double *Ubar, double dt) {
  DG_TRY(adj_pool(c, 5));
  DG_TRY(tau_fill(c, 5));
  double *S[5] = {const_cast<double *>(U), c->adj_pool[0], c->adj_pool[1], c->adj_pool[2], c->adj_pool[3]};
  double *T[5] = {tau_at(c, 0), tau_at(c, 1), tau_at(c, 2), tau_at(c, 3), tau_at(c, 4)};
  for (int st = 0; st < 4; ++st) DG_TRY(stage(c, S[st], S[st + 1], 1, st, dt, T[st]));
  DG_TRY(record_tau(c, S[4], T[4]));
  return reverse_stages(c, S, T, Ubar, dt);
}

// Reverse sweep over n_steps from checkpoints cp[j] = state at step j * interval: each segment is
// recomputed once from its checkpoint and reversed step by step. When the budget allows, the
// recomputation keeps all five stage states of the segment and their stress records (5 interval
// buffers of each); otherwise the step start states only (interval - 1 buffers) and each step's
// stages are recomputed before reversal. Segment buffers live in the adjoint pool from index `first`
// on, segment stress records in the stress pool from index 0 on.
dg_status reverse_from_checkpoints(dg_ctx *c, const std::vector<double *> &cp, int interval, int n_steps,
                                   double *Ubar, double dt, size_t first) {
  const int ncp = (int)cp.size();
  const bool store = budget_allows(c, adj_bytes(c, first + 5 * (size_t)interval, 5 * (size_t)interval),
                                   adj_held(c));
  DG_TRY(adj_pool(c, first + (store ? 5 * (size_t)interval : (size_t)interval - 1)));
  if (store) DG_TRY(tau_fill(c, 5 * (size_t)interval));
  double **seg = c->adj_pool.data() + first;
  for (int j = ncp - 1; j >= 0; --j) {
    const int len = std::min(interval, n_steps - j * interval);
    if (store) {
      // S(i, s): input state of stage s of step i of the segment; S(0, 0) is the checkpoint
      auto S = [&](int i, int st) { return (i == 0 && st == 0) ? cp[j] : seg[5 * i + st]; };
      auto T = [&](int i, int st) { return tau_at(c, 5 * (size_t)i + st); };
      for (int i = 0; i < len; ++i)
        for (int st = 0; st < 5; ++st) {
          if (i == len - 1 && st == 4) {  // the segment's end state is not needed, its input's record is
            DG_TRY(record_tau(c, S(i, st), T(i, st)));
            break;
          }
          double *out = st < 4 ? S(i, st + 1) : S(i + 1, 0);
          DG_TRY(stage(c, S(i, st), out, 1, st, dt, T(i, st)));
        }
      for (int i = len - 1; i >= 0; --i) {
        double *st5[5] = {S(i, 0), S(i, 1), S(i, 2), S(i, 3), S(i, 4)};
        double *tau5[5] = {T(i, 0), T(i, 1), T(i, 2), T(i, 3), T(i, 4)};
        DG_TRY(reverse_stages(c, st5, tau5, Ubar, dt));
      }
    } else {
      auto state = [&](int i) { return i == 0 ? cp[j] : seg[i - 1]; };
      for (int i = 1; i < len; ++i) {
        DG_TRY(copy_state(c, state(i), state(i - 1)));
        DG_TRY(steps_impl(c, state(i), dt, 1));
      }
      for (int i = len - 1; i >= 0; --i) DG_TRY(step_vjp(c, state(i), Ubar, dt));
    }
  }
  return DG_OK;
}
}  // namespace

extern "C" {

const char *dg_status_string(int s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_MESH: return "inconsistent mesh";
    case DG_ERR_JACOBIAN: return "non-positive Jacobian";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_NONPHYSICAL: return "non-physical state";
    case DG_ERR_UNSUPPORTED: return "unsupported";
    case DG_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

const char *dg_last_error(const dg_ctx *c) { return c ? c->err.c_str() : "null context"; }

dg_status dg_basis(int N, double *xi, double *w, double *D) {
  if (N < 1 || N > DG_NMAX || !xi || !w || !D) return DG_ERR_ARG;
  DgTables t;
  if (dg_build_tables(N, &t) != 0) return DG_ERR_ARG;
  const int n = N + 1;
  for (int i = 0; i < n; ++i) { xi[i] = t.xi[i]; w[i] = t.w[i]; }
  for (int i = 0; i < n * n; ++i) D[i] = t.D[i];
  return DG_OK;
}

void dg_free(dg_ctx *c) {
  if (!c) return;
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  if (c->gev_in) cudaEventDestroy(c->gev_in);
  if (c->gev_out) cudaEventDestroy(c->gev_out);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  for (cudaStream_t st : c->cstream)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : c->cev)
    if (ev) cudaEventDestroy(ev);
  for (void *p : c->allocs) cudaFree(p);
  for (auto &pr : c->ev_pool) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (c->flag_host) cudaFreeHost(c->flag_host);
  delete c;
}

dg_status dg_init(const dg_mesh *mesh, int N, int nodes, const dg_params *prm, void *cuda_stream, dg_ctx **out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  if (!mesh || !prm || !mesh->xyz || !mesh->face) return DG_ERR_ARG;
  if (N < 1 || N > DG_NMAX || nodes != DG_NODES_LGL || mesh->n_geo != N) return DG_ERR_ARG;
  if (mesh->n_elems <= 0 || mesh->n_faces <= 0) return DG_ERR_ARG;
  if (prm->equations < 0 || prm->equations > 1 || prm->volume_flux < 0 || prm->volume_flux > 3 ||
      prm->surface_flux < 0 || prm->surface_flux > 2 || prm->precision < 0 || prm->precision > 1)
    return DG_ERR_ARG;
  if (!(prm->gamma > 1.0) || !(prm->R > 0.0) || !(prm->mu >= 0.0) || !(prm->Pr > 0.0)) return DG_ERR_ARG;
  if (!std::isfinite(prm->p_ref) || prm->p_ref < 0.0) return DG_ERR_ARG;
  const int nE = mesh->n_elems, nF = mesh->n_faces, n = N + 1, nn = n * n, nnn = nn * n;

  // element-face connectivity: every (element, local face) slot used exactly once; a wall face
  // (elemR = -1) fills one slot: (-1, boundary kind, 0, face id)
  std::vector<int> ef((size_t)nE * 24, -1);
  std::vector<char> used((size_t)nE * 6, 0);
  int n_walls = 0;
  for (int f = 0; f < nF; ++f) {
    const int *F = mesh->face + 5 * f;
    const int eL = F[0], fL = F[1], eR = F[2], fR = F[3], o = F[4];
    if (eR == -1) {
      if (eL < 0 || eL >= nE || fL < 0 || fL > 5 || fR != DG_BC_WALL_MODEL || used[(size_t)eL * 6 + fL])
        return DG_ERR_MESH;
      if (prm->wm_index < 1 || prm->wm_index > N) return DG_ERR_ARG;
      used[(size_t)eL * 6 + fL] = 1;
      int *sL = &ef[((size_t)eL * 6 + fL) * 4];
      sL[0] = -1; sL[1] = fR; sL[2] = 0; sL[3] = f;
      ++n_walls;
      continue;
    }
    if (eL < 0 || eL >= nE || eR < 0 || eR >= nE || fL < 0 || fL > 5 || fR < 0 || fR > 5 || o < 0 || o > 7)
      return DG_ERR_MESH;
    int *sL = &ef[((size_t)eL * 6 + fL) * 4], *sR = &ef[((size_t)eR * 6 + fR) * 4];
    if (used[(size_t)eL * 6 + fL] || used[(size_t)eR * 6 + fR] || (eL == eR && fL == fR)) return DG_ERR_MESH;
    used[(size_t)eL * 6 + fL] = used[(size_t)eR * 6 + fR] = 1;
    // inverse orientation: a transposed map swaps the roles of the two flip bits
    const int inv = (o & 4) ? (4 | ((o & 1) << 1) | ((o & 2) >> 1)) : o;
    sL[0] = eR; sL[1] = fR; sL[2] = o; sL[3] = f;
    sR[0] = eL; sR[1] = fL; sR[2] = inv; sR[3] = f;
  }
  for (char u : used)
    if (!u) return DG_ERR_MESH;
  if (n_walls && !(prm->wm_uinf >= 0.0 && prm->wm_mainf >= 0.0)) return DG_ERR_ARG;

  dg_ctx *c = new dg_ctx();
  c->N = N;
  c->params = *prm;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { dg_status s = cuda_fail(c, e, "cudaGetDevice"); *out = nullptr; delete c; return s; }
  c->K = kernels_for(N);
  {
    std::lock_guard<std::mutex> lk(g_upload_mutex);
    if ((int)g_uploaded.size() <= c->device) g_uploaded.resize(c->device + 1, 0u);
    if (!(g_uploaded[c->device] & (1u << N))) {
      DgTables t;
      dg_build_tables(N, &t);
      e = c->K->upload(t);
      if (e != cudaSuccess) { cuda_fail(c, e, "constant tables"); dg_free(c); return DG_ERR_CUDA; }
      g_uploaded[c->device] |= (1u << N);
    }
  }
  DgDevice &d = c->d;
  d.N = N; d.nE = nE; d.nF = nF;
  d.equations = prm->equations; d.vflux = prm->volume_flux; d.sflux = prm->surface_flux;
  d.precision = prm->precision; d.shock_capturing = prm->shock_capturing ? 1 : 0;
  d.gamma = prm->gamma; d.R = prm->R; d.mu = prm->mu;
  d.kappa = prm->mu * prm->gamma * prm->R / ((prm->gamma - 1.0) * prm->Pr);
  d.alpha_min = prm->alpha_min; d.alpha_max = prm->alpha_max; d.sharpness = prm->sharpness;
  d.ind_T = 0.5 * std::pow(10.0, -1.8 * std::pow((double)(N + 1), 0.25));
  d.ind_k = -prm->sharpness / d.ind_T;
  d.alpha_fixed = prm->alpha_fixed;
  d.p_ref = prm->precision == DG_FP32_BULK ? prm->p_ref : 0.0;
  d.gm1 = d.gamma - 1.0;
  d.igm1 = 1.0 / d.gm1;
  d.igm1_f = (float)d.igm1;
  d.iR = 1.0 / d.R;
  d.href = d.p_ref * d.gamma / (d.gamma - 1.0);
  d.eref = d.p_ref / (d.gamma - 1.0);
  d.gamma_f = (float)d.gamma;
  d.gm1_f = (float)d.gamma - 1.0f;
  d.iR_f = 1.0f / (float)d.R;
  d.p_ref_f = (float)d.p_ref;
  d.href_f = (float)d.href;
  d.mu_f = (float)d.mu;
  d.kappa_f = (float)d.kappa;
  d.use_tma = 3;  // N = 7: pair-symmetric line kernel; other N: warp-specialised node kernel
  d.n_walls = n_walls;
  d.wm_index = prm->wm_index;
  d.wm_vd = prm->wm_van_driest ? 1 : 0;
  d.wm_uinf = prm->wm_uinf;
  {
    const double m = 0.5 * (prm->gamma - 1.0) * prm->wm_mainf * prm->wm_mainf * std::cbrt(prm->Pr);
    d.wm_b = std::sqrt(m) / std::sqrt(1.0 + m);  // van Driest transform (Sec. 3, Eq. (5))
  }
  c->n_state = (size_t)nE * 5 * nnn;
  c->n_tau = prm->equations == DG_NAVIER_STOKES ? (size_t)nE * 6 * nnn : 0;
  const bool fp32 = prm->precision == DG_FP32_BULK;

  double *xyz = nullptr;
  int *face = nullptr;
  dg_status s = DG_OK;
#define DG_ALLOC(p, cnt) \
  do {                        \
    if (s == DG_OK) s = dev_alloc(c, &(p), (size_t)(cnt)); \
  } while (0)
  DG_ALLOC(xyz, (size_t)nE * 3 * nnn);
  DG_ALLOC(face, (size_t)nF * 5);
  DG_ALLOC(d.ef, (size_t)nE * 24);
  DG_ALLOC(d.Ja, (size_t)nE * 9 * nnn);
  DG_ALLOC(d.J, (size_t)nE * nnn);
  DG_ALLOC(d.invJ, (size_t)nE * nnn);
  DG_ALLOC(d.nrm, (size_t)nF * 4 * nn);
  if (fp32) {  // FP32-bulk: FP32 copies of the geometry and FP32 work buffers
    DG_ALLOC(d.Jaf, (size_t)nE * 9 * nnn);
    DG_ALLOC(d.nrm_f, (size_t)nF * 4 * nn);
    DG_ALLOC(d.invJf, (size_t)nE * nnn);
    DG_ALLOC(d.facf, (size_t)nE * nnn);
    DG_ALLOC(d.Uf, (size_t)nE * 5 * nnn);
    DG_ALLOC(d.Fsurf_f, (size_t)nE * 6 * 5 * nn);
    if (prm->equations == DG_NAVIER_STOKES) {
      DG_ALLOC(d.Wsurf_f, (size_t)nE * 6 * 4 * nn);
      DG_ALLOC(d.Fv_f, (size_t)nE * 12 * nnn);
    }
  } else {
    DG_ALLOC(d.Fsurf, (size_t)nE * 6 * 5 * nn);
    if (prm->equations == DG_NAVIER_STOKES) {
      DG_ALLOC(d.Wsurf, (size_t)nE * 6 * 4 * nn);
      DG_ALLOC(d.Fv, (size_t)nE * 12 * nnn);
    }
  }
  if (n_walls && prm->equations == DG_NAVIER_STOKES) {  // wall model: exchange distances and wall fluxes
    DG_ALLOC(d.hwm, (size_t)nF * nn);
    if (fp32) {
      DG_ALLOC(d.Fwall_f, (size_t)nF * 4 * nn);
    } else {
      DG_ALLOC(d.Fwall, (size_t)nF * 4 * nn);
    }
  }
  DG_ALLOC(d.alpha_raw, (size_t)nE);
  DG_ALLOC(d.alpha, (size_t)nE);
  DG_ALLOC(d.red, (size_t)DG_RED_DOUBLES);
  DG_ALLOC(d.flag, (size_t)1);
  DG_ALLOC(c->g, c->n_state);
  DG_ALLOC(c->small, (size_t)16);
#undef DG_ALLOC
  if (s != DG_OK) { dg_free(c); return s; }
  d.xyz = xyz;
  d.face = face;
  if ((e = cudaMallocHost(&c->flag_host, sizeof(int))) != cudaSuccess) {
    cuda_fail(c, e, "cudaMallocHost");
    dg_free(c);
    return DG_ERR_OOM;
  }
  cudaStream_t st = c->stream;
  e = cudaMemcpyAsync(xyz, mesh->xyz, sizeof(double) * (size_t)nE * 3 * nnn, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(face, mesh->face, sizeof(int) * (size_t)nF * 5, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(d.ef, ef.data(), sizeof(int) * (size_t)nE * 24, cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemsetAsync(d.flag, 0, sizeof(int), st);
  if (!e) e = cudaMemsetAsync(d.alpha, 0, sizeof(double) * nE, st);
  if (!e) e = cudaMemsetAsync(d.alpha_raw, 0, sizeof(double) * nE, st);
  if (e) { cuda_fail(c, e, "init copies"); dg_free(c); return DG_ERR_CUDA; }
  if ((s = launch(c, KC_OTHER, [&] { c->K->metrics(c->d, st); })) != DG_OK) { dg_free(c); return s; }
  if ((s = launch(c, KC_OTHER, [&] { c->K->face_normals(c->d, st); })) != DG_OK) { dg_free(c); return s; }
  if (d.shock_capturing && d.alpha_fixed >= 0.0) {
    if ((s = launch(c, KC_OTHER, [&] { k_fill<<<(nE + 255) / 256, 256, 0, st>>>(d.alpha, nE, d.alpha_fixed); })) !=
        DG_OK) { dg_free(c); return s; }
  }
  e = cudaMemcpyAsync(c->flag_host, d.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) { cuda_fail(c, e, "init"); dg_free(c); return DG_ERR_CUDA; }
  if (*c->flag_host & 2) { dg_free(c); return DG_ERR_JACOBIAN; }
  d.xyz = nullptr;  // coordinates are not needed after the metrics
  *out = c;
  return DG_OK;
}

}  // extern "C"

namespace {
// FP32-bulk: refresh the FP32 shadow of a caller state (the volume kernel keeps it current afterwards)
dg_status refresh_shadow(dg_ctx *c, const double *U) {
  if (c->d.precision != DG_FP32_BULK) return DG_OK;
  return launch(c, KC_OTHER, [&] { c->K->shadow(c->d, U, c->stream); });
}

// FP32-bulk: the epilogue's stage factor float(dt (-1/J)) per node, formed in FP64 and rounded once,
// whenever the step size changes (outside any graph capture: steps_impl calls this first)
__global__ void k_stage_factor(float *__restrict__ fac, const double *__restrict__ invJ, double dt, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    fac[i] = d2f_int(__dmul_rn(dt, -invJ[i]));
}

dg_status ensure_stage_factor(dg_ctx *c, double dt) {
  if (c->d.precision != DG_FP32_BULK || c->fac_dt == dt) return DG_OK;
  const size_t n = (size_t)c->d.N + 1, count = (size_t)c->d.nE * n * n * n;
  DG_TRY(launch(c, KC_OTHER, [&] { k_stage_factor<<<8 * 152, 256, 0, c->stream>>>(c->d.facf, c->d.invJ, dt, count); }));
  c->fac_dt = dt;
  return DG_OK;
}
dg_status plain_steps(dg_ctx *c, double *U, double dt, int n_steps) {
  for (int k = 0; k < n_steps; ++k)
    for (int st = 0; st < 5; ++st) DG_TRY(stage(c, U, U, 1, st, dt));
  return DG_OK;
}

// capture one LSERK step on U with step dt into c->step_graph (launches go to the library stream)
dg_status capture_step(dg_ctx *c, double *U, double dt) {
  if (c->step_graph) { cudaGraphExecDestroy(c->step_graph); c->step_graph = nullptr; }
  cudaStream_t user = c->stream;
  c->stream = c->gstream;
  const long long l0 = c->launches;
  cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
  dg_status st = e ? DG_ERR_CUDA : DG_OK;
  if (st == DG_OK) st = plain_steps(c, U, dt, 1);
  cudaGraph_t g = nullptr;
  if (!e) {
    const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
    if (!e && e2) e = e2;
  }
  c->graph_launches = c->launches - l0;
  c->launches = l0;  // captured, not run
  c->stream = user;
  if (!e && st == DG_OK) e = cudaGraphInstantiate(&c->step_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e) {
    cudaGetLastError();
    c->step_graph = nullptr;
    return cuda_fail(c, e, "step graph");
  }
  if (st != DG_OK) return st;
  c->graph_U = U;
  c->graph_dt = dt;
  return DG_OK;
}

// n_steps LSERK steps. With graphs on (and kernel timing off) the step's launch sequence is
// captured once per (U, dt) and replayed: one graph launch per step instead of 10-20 kernel
// launches, which is what bounds small meshes.
dg_status steps_impl(dg_ctx *c, double *U, double dt, int n_steps) {
  DG_TRY(refresh_shadow(c, U));
  DG_TRY(ensure_stage_factor(c, dt));
  if (n_steps <= 0) return DG_OK;
  if (!c->use_graphs || c->timing || n_steps < 2) return plain_steps(c, U, dt, n_steps);
  cudaError_t e = cudaSuccess;
  if (!c->gstream) {
    e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming);
    if (e) return cuda_fail(c, e, "graph stream");
  }
  if (!(c->step_graph && c->graph_U == U && c->graph_dt == dt)) {
    DG_TRY(plain_steps(c, U, dt, 1));  // first step directly (also sets kernel attributes outside capture)
    --n_steps;
    if (capture_step(c, U, dt) != DG_OK) {  // no graph on this stream: launch the kernels directly
      c->use_graphs = 0;
      c->err.clear();
      return plain_steps(c, U, dt, n_steps);
    }
  }
  e = cudaEventRecord(c->gev_in, c->stream);
  if (!e) e = cudaStreamWaitEvent(c->gstream, c->gev_in, 0);
  for (int k = 0; k < n_steps && !e; ++k) e = cudaGraphLaunch(c->step_graph, c->gstream);
  if (!e) e = cudaEventRecord(c->gev_out, c->gstream);
  if (!e) e = cudaStreamWaitEvent(c->stream, c->gev_out, 0);
  if (e) return cuda_fail(c, e, "step graph launch");
  c->launches += c->graph_launches * n_steps;
  return DG_OK;
}
// state copy by the SMs through the host-device link, 16 bytes per thread and step; for page-locked host
// memory, which the device addresses directly
__global__ void k_copy16(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// one copy of `bytes` split into dg_ctx::kCopyStreams pieces on the library copy streams, ordered
// after the work already on the context stream and before the work enqueued on it afterwards
dg_status copy_split(dg_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  constexpr int K = dg_ctx::kCopyStreams;
  cudaError_t e = cudaSuccess;
  if (!c->cstream[0]) {
    for (int k = 0; k < K && !e; ++k) e = cudaStreamCreateWithFlags(&c->cstream[k], cudaStreamNonBlocking);
    for (int k = 0; k <= K && !e; ++k) e = cudaEventCreateWithFlags(&c->cev[k], cudaEventDisableTiming);
    if (e) return cuda_fail(c, e, "copy streams");
  }
  const size_t chunk = ((bytes + K - 1) / K + 255) / 256 * 256;
  e = cudaEventRecord(c->cev[K], c->stream);
  for (int k = 0; k < K && !e; ++k) {
    const size_t off = (size_t)k * chunk;
    if (off >= bytes) break;
    const size_t len = std::min(chunk, bytes - off);
    e = cudaStreamWaitEvent(c->cstream[k], c->cev[K], 0);
    if (!e) e = cudaMemcpyAsync(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, len, kind,
                                c->cstream[k]);
    if (!e) e = cudaEventRecord(c->cev[k], c->cstream[k]);
    if (!e) e = cudaStreamWaitEvent(c->stream, c->cev[k], 0);
  }
  if (e) return cuda_fail(c, e, kind == cudaMemcpyHostToDevice ? "H2D" : "D2H");
  return DG_OK;
}

// a host <-> device copy of the state: page-locked host memory that the device can address is copied by
// k_copy16 on the context stream (the SMs keep many 16-byte loads in flight over the host-device link);
// other host memory, or an unaligned buffer, by copy engines (copy_split)
// the device's address of page-locked host memory `host` when it is 16-byte aligned and `bytes` is a
// multiple of 16, else null (other host memory, or a failed query, whose error is not left behind)
void *host_device_pointer(const void *host, size_t bytes) {
  cudaPointerAttributes a{};
  const cudaError_t qe = cudaPointerGetAttributes(&a, host);
  if (qe != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer && bytes % 16 == 0 &&
      (reinterpret_cast<uintptr_t>(a.devicePointer) & 15u) == 0)
    return a.devicePointer;
  return nullptr;
}

dg_status copy_state_host(dg_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  void *hdev = host_device_pointer(kind == cudaMemcpyHostToDevice ? src : dst, bytes);
  if (hdev && (reinterpret_cast<uintptr_t>(kind == cudaMemcpyHostToDevice ? dst : src) & 15u)) hdev = nullptr;
  if (!hdev) return copy_split(c, dst, src, bytes, kind);
  const uint4 *from = static_cast<const uint4 *>(kind == cudaMemcpyHostToDevice ? hdev : src);
  uint4 *to = static_cast<uint4 *>(kind == cudaMemcpyHostToDevice ? dst : hdev);
  return launch(c, KC_OTHER, [&] { k_copy16<<<8 * 152, 256, 0, c->stream>>>(from, to, bytes / 16); });
}

}  // namespace

extern "C" {

dg_status dg_rhs(dg_ctx *c, const double *U, double *Ut, double t) {
  (void)t;
  if (!c || !U || !Ut || U == Ut) return fail(c, DG_ERR_ARG, "dg_rhs: null or aliased arrays");
  DG_TRY(refresh_shadow(c, U));
  return stage(c, U, Ut, 0, 0, 0.0);
}

dg_status dg_lserk_step(dg_ctx *c, double *U, double dt, double t) {
  (void)t;
  if (!c || !U || !std::isfinite(dt)) return fail(c, DG_ERR_ARG, "dg_lserk_step: bad argument");
  return steps_impl(c, U, dt, 1);
}

dg_status dg_lserk_steps(dg_ctx *c, double *U, double dt, double t, int n_steps) {
  (void)t;
  if (!c || !U || n_steps < 0 || !std::isfinite(dt)) return fail(c, DG_ERR_ARG, "dg_lserk_steps: bad argument");
  return steps_impl(c, U, dt, n_steps);
}

dg_status dg_lserk_step_host(dg_ctx *c, double *U_host, double dt, double t) {
  if (!c || !U_host) return fail(c, DG_ERR_ARG, "dg_lserk_step_host: null array");
  if (!std::isfinite(dt)) return fail(c, DG_ERR_ARG, "dg_lserk_step_host: bad argument");
  if (!c->Ustage) DG_TRY(dev_alloc(c, &c->Ustage, c->n_state));
  const size_t bytes = sizeof(double) * c->n_state;
  DG_TRY(copy_state_host(c, c->Ustage, U_host, bytes, cudaMemcpyHostToDevice));
  if (double *hdev = static_cast<double *>(host_device_pointer(U_host, bytes))) {
    // page-locked host state: the last stage's volume kernel writes the new state straight into it
    // over the host link, spread over the kernel's run, instead of a copy after it (same kernels,
    // same bits)
    DG_TRY(refresh_shadow(c, c->Ustage));
    DG_TRY(ensure_stage_factor(c, dt));
    for (int st = 0; st < 5; ++st) DG_TRY(stage(c, c->Ustage, st < 4 ? c->Ustage : hdev, 1, st, dt));
  } else {
    DG_TRY(dg_lserk_step(c, c->Ustage, dt, t));
    DG_TRY(copy_state_host(c, U_host, c->Ustage, bytes, cudaMemcpyDeviceToHost));
  }
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "D2H");
  return DG_OK;
}

dg_status dg_rhs_vjp(dg_ctx *c, const double *U, const double *lambda, double *Ubar, double t) {
  (void)t;
  if (!c || !U || !lambda || !Ubar || Ubar == U || Ubar == lambda)
    return fail(c, DG_ERR_ARG, "dg_rhs_vjp: null or aliased arrays");
  DG_TRY(adjoint_supported(c, "dg_rhs_vjp"));
  DG_TRY(tau_fill(c, 1));
  DG_TRY(record_tau(c, U, tau_at(c, 0)));
  return vjp(c, U, lambda, Ubar, 0, 0.0, 0.0, 0.0, 0, tau_at(c, 0));
}

dg_status dg_lserk_step_vjp(dg_ctx *c, const double *U, double *Ubar, double dt, double t) {
  (void)t;
  if (!c || !U || !Ubar || U == Ubar || !std::isfinite(dt)) return fail(c, DG_ERR_ARG, "dg_lserk_step_vjp: bad argument");
  DG_TRY(adjoint_supported(c, "dg_lserk_step_vjp"));
  return step_vjp(c, U, Ubar, dt);
}

dg_status dg_lserk_steps_vjp(dg_ctx *c, const double *U0, double *Ubar, double dt, double t, int n_steps,
                             int interval) {
  (void)t;
  if (!c || !U0 || !Ubar || U0 == Ubar || n_steps < 0 || interval < 1 || !std::isfinite(dt))
    return fail(c, DG_ERR_ARG, "dg_lserk_steps_vjp: bad argument");
  DG_TRY(adjoint_supported(c, "dg_lserk_steps_vjp"));
  if (n_steps == 0) return DG_OK;
  if (interval > n_steps) interval = n_steps;
  const int ncp = (n_steps + interval - 1) / interval;
  DG_TRY(adj_pool(c, 5 + (size_t)ncp));
  double **cp = c->adj_pool.data() + 5;
  // forward sweep: checkpoints every `interval` steps
  DG_TRY(copy_state(c, cp[0], U0));
  for (int j = 1; j < ncp; ++j) {
    DG_TRY(copy_state(c, cp[j], cp[j - 1]));
    DG_TRY(steps_impl(c, cp[j], dt, interval));
  }
  std::vector<double *> cps(cp, cp + ncp);  // (the pool may grow below)
  return reverse_from_checkpoints(c, cps, interval, n_steps, Ubar, dt, 5 + ncp);
}

dg_status dg_lserk_steps_record(dg_ctx *c, double *U, double dt, double t, int n_steps, int interval,
                                long long *tape) {
  (void)t;
  if (!c || !U || !tape || n_steps < 1 || interval < 1 || !std::isfinite(dt))
    return fail(c, DG_ERR_ARG, "dg_lserk_steps_record: bad argument");
  DG_TRY(adjoint_supported(c, "dg_lserk_steps_record"));
  c->tape_id = 0;  // any earlier tape is invalid from here on
  if (interval > n_steps) interval = n_steps;
  const size_t full = 5 * (size_t)n_steps, ncp = (size_t)((n_steps + interval - 1) / interval);
  // every stage state and its stress record when the budget holds them (and the reverse sweep's 5
  // scratch buffers), else checkpoints every `interval` steps
  const bool store_all = budget_allows(c, adj_bytes(c, full + 5, full), adj_held(c));
  DG_TRY(pool_fill(c, c->tape_pool, store_all ? full : ncp));
  if (store_all && c->n_tau) DG_TRY(pool_fill(c, c->tape_tau, full, c->n_tau));
  double **T = c->tape_pool.data();
  if (store_all) {
    DG_TRY(copy_state(c, T[0], U));
    for (int k = 0; k < n_steps; ++k)
      for (int st = 0; st < 5; ++st) {
        double *out = st < 4 ? T[5 * k + st + 1] : (k + 1 < n_steps ? T[5 * (k + 1)] : U);
        DG_TRY(stage(c, T[5 * k + st], out, 1, st, dt, c->n_tau ? c->tape_tau[5 * k + st] : nullptr));
      }
  } else {
    for (int j = 0; j < (int)ncp; ++j) {
      DG_TRY(copy_state(c, T[j], U));
      DG_TRY(steps_impl(c, U, dt, std::min(interval, n_steps - j * interval)));
    }
  }
  c->tape_steps = n_steps;
  c->tape_interval = interval;
  c->tape_all = store_all;
  c->tape_dt = dt;
  c->tape_id = ++c->tape_serial;
  *tape = c->tape_id;
  return DG_OK;
}

dg_status dg_lserk_steps_vjp_recorded(dg_ctx *c, long long tape, double *Ubar) {
  if (!c || !Ubar) return fail(c, DG_ERR_ARG, "dg_lserk_steps_vjp_recorded: bad argument");
  if (tape <= 0 || tape != c->tape_id)
    return fail(c, DG_ERR_ARG, "dg_lserk_steps_vjp_recorded: no such tape (recorded over or never recorded)");
  DG_TRY(adjoint_supported(c, "dg_lserk_steps_vjp_recorded"));
  const int n_steps = c->tape_steps;
  const double dt = c->tape_dt;
  if (c->tape_all) {
    DG_TRY(adj_pool(c, 5));  // gbar
    double **T = c->tape_pool.data();
    for (int k = n_steps - 1; k >= 0; --k) {
      double *S[5] = {T[5 * k], T[5 * k + 1], T[5 * k + 2], T[5 * k + 3], T[5 * k + 4]};
      double *tau5[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
      if (c->n_tau)
        for (int st = 0; st < 5; ++st) tau5[st] = c->tape_tau[5 * k + st];
      DG_TRY(reverse_stages(c, S, tau5, Ubar, dt));
    }
    return DG_OK;
  }
  const int ncp = (n_steps + c->tape_interval - 1) / c->tape_interval;
  std::vector<double *> cps(c->tape_pool.begin(), c->tape_pool.begin() + ncp);
  return reverse_from_checkpoints(c, cps, c->tape_interval, n_steps, Ubar, dt, 5);
}

dg_status dg_tape_current(const dg_ctx *c, long long *tape) {
  if (!c || !tape) return DG_ERR_ARG;
  *tape = c->tape_id;
  return DG_OK;
}

dg_status dg_adjoint_memory_limit(dg_ctx *c, double bytes) {
  if (!c || !(bytes >= 0.0)) return fail(c, DG_ERR_ARG, "dg_adjoint_memory_limit: bad argument");
  c->adj_limit = (size_t)bytes;
  return DG_OK;
}

dg_status dg_kinetic_energy_grad(dg_ctx *c, const double *U, double *grad) {
  if (!c || !U || !grad || U == grad) return fail(c, DG_ERR_ARG, "dg_kinetic_energy_grad: bad argument");
  return launch(c, KC_OTHER, [&] { c->K->ke_grad(c->d, U, grad, c->stream); });
}

dg_status dg_indicator(dg_ctx *c, const double *U, double *alpha) {
  if (!c || !U || !alpha) return fail(c, DG_ERR_ARG, "dg_indicator: null array");
  DG_TRY(launch(c, KC_INDICATOR, [&] { c->K->indicator(c->d, U, c->stream); }));
  DG_TRY(launch(c, KC_SPREAD, [&] { c->K->spread(c->d, alpha, c->stream); }));
  return DG_OK;
}

dg_status dg_invariants(dg_ctx *c, const double *U, const double *Ut, double out[8]) {
  if (!c || !U || !Ut || !out) return fail(c, DG_ERR_ARG, "dg_invariants: null array");
  DG_TRY(launch(c, KC_OTHER, [&] { c->K->invariants(c->d, U, Ut, c->small, c->stream); }));
  cudaError_t e = cudaMemcpyAsync(out, c->small, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "dg_invariants");
  return DG_OK;
}

dg_status dg_max_dt(dg_ctx *c, const double *U, double cfl, double *dt) {
  if (!c || !U || !dt || !(cfl > 0.0)) return fail(c, DG_ERR_ARG, "dg_max_dt: bad argument");
  DG_TRY(launch(c, KC_OTHER, [&] { c->K->max_dt(c->d, U, c->small + 8, c->stream); }));
  double v = 0.0;
  cudaError_t e = cudaMemcpyAsync(&v, c->small + 8, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "dg_max_dt");
  *dt = cfl * v;
  return DG_OK;
}

dg_status dg_check(dg_ctx *c) {
  if (!c) return DG_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(c->flag_host, c->d.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "dg_check");
  const int f = *c->flag_host;
  e = cudaMemsetAsync(c->d.flag, 0, sizeof(int), c->stream);
  if (e) return cuda_fail(c, e, "dg_check");
  if (f & 4) return fail(c, DG_ERR_CUDA, "a device-side wait for a bulk copy timed out");
  if (f & 1) return fail(c, DG_ERR_NONPHYSICAL, "a kernel met rho <= 0, p <= 0 or a non-finite state");
  return DG_OK;
}

dg_status dg_get_metrics(dg_ctx *c, double *Ja, double *J) {
  if (!c || !Ja || !J) return fail(c, DG_ERR_ARG, "dg_get_metrics: null array");
  const int n = c->N + 1;
  const size_t nnn = (size_t)n * n * n;
  cudaError_t e = cudaMemcpyAsync(Ja, c->d.Ja, sizeof(double) * c->d.nE * 9 * nnn, cudaMemcpyDeviceToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(J, c->d.J, sizeof(double) * c->d.nE * nnn, cudaMemcpyDeviceToDevice, c->stream);
  if (e) return cuda_fail(c, e, "dg_get_metrics");
  return DG_OK;
}

dg_status dg_use_tma(dg_ctx *c, int enable) {
  if (!c) return DG_ERR_ARG;
  if (enable < 0 || enable > 3) return fail(c, DG_ERR_ARG, "dg_use_tma: mode 0, 1, 2 or 3");
  c->d.use_tma = enable;
  if (c->step_graph) { cudaGraphExecDestroy(c->step_graph); c->step_graph = nullptr; }  // kernels change
  return DG_OK;
}

dg_status dg_use_graphs(dg_ctx *c, int enable) {
  if (!c) return DG_ERR_ARG;
  c->use_graphs = enable != 0;
  return DG_OK;
}

dg_status dg_timing_enable(dg_ctx *c, int enable) {
  if (!c) return DG_ERR_ARG;
  c->timing = enable != 0;
  return DG_OK;
}

int dg_timing_get(dg_ctx *c, const char **names, double *ms, long long *launches, int cap) {
  if (!c) return -1;
  if (c->ev_used) {
    cudaStreamSynchronize(c->stream);
    for (size_t i = 0; i < c->ev_used; ++i) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, c->ev_pool[i].first, c->ev_pool[i].second);
      c->t_ms[c->ev_class[i]] += t;
      c->t_count[c->ev_class[i]] += 1;
    }
    c->ev_used = 0;
  }
  int k = 0;
  for (; k < KC_COUNT && k < cap; ++k) {
    if (names) names[k] = kKernelNames[k];
    if (ms) ms[k] = c->t_ms[k];
    if (launches) launches[k] = c->t_count[k];
  }
  for (int j = 0; j < KC_COUNT; ++j) { c->t_ms[j] = 0.0; c->t_count[j] = 0; }
  return k;
}

long long dg_launch_count(const dg_ctx *c) { return c ? c->launches : -1; }

}  // extern "C"
