// C-ABI of the GB300 SSCN solver (declared in include/dgpe.h): parameter checks, the
// workspace layout, the step sequence K1..K7 (replayed from a CUDA graph) and the
// synchronising calls.  All arithmetic of the step runs in the kernels of
// dgpe_device.cuh; this file only orders them on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "dgpe.h"
#include "dgpe_internal.h"

using namespace dgpe;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool is_2a3b5c7d(int n) {
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  while (n % 7 == 0) n /= 7;
  return n == 1;
}

bool finite(double v) { return isfinite(v) != 0; }

// Radix plan.  style 0: as many radix-8 stages as possible, then one radix-4 or radix-2
// stage for the rest of the power of two, then the radix-3, 5 and 7 stages.  style 1:
// radix-4 stages (and one radix-2), then the odd radices.  style 2: radix-3 stages first,
// then as style 0.
FftPlan make_plan(int n, int style = 0) {
  FftPlan p{};
  p.n = n;
  int m = n, k = 0;
  if (style == 2)
    while (m % 3 == 0) {
      p.radix[k++] = 3;
      m /= 3;
    }
  if (style != 1)
    while (m % 8 == 0) {
      p.radix[k++] = 8;
      m /= 8;
    }
  while (m % 4 == 0) {
    p.radix[k++] = 4;
    m /= 4;
  }
  if (m % 2 == 0) {
    p.radix[k++] = 2;
    m /= 2;
  }
  while (m % 3 == 0) {
    p.radix[k++] = 3;
    m /= 3;
  }
  while (m % 5 == 0) {
    p.radix[k++] = 5;
    m /= 5;
  }
  while (m % 7 == 0) {
    p.radix[k++] = 7;
    m /= 7;
  }
  p.nstages = k;
  int off = 0, ns = 1;
  for (int s = 0; s < k; ++s) {
    p.twoff[s] = off;
    off += ns * (p.radix[s] - 1);
    ns *= p.radix[s];
  }
  return p;
}

// Interior points per lane of the chunked Thomas solve: the smallest power of two >= 2
// with 32 lanes covering the m = n - 2 unknowns (a power of two keeps the slot arithmetic
// to shifts; an even chunk gives an odd slot stride, so the lanes hit distinct banks).
int cn_chunk(int n) {
  const int m = n - 2;
  int c = 2;
  while (c * kWarp < m) c *= 2;
  return c;
}

int log2_int(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int check_shape(const dgpe_params *p) {
  const int dims[3] = {p->nx, p->ny, p->nz};
  for (int d = 0; d < 3; ++d) {
    const int n = dims[d];
    if (n < 4 || n > 512 || n % 2 != 0 || !is_2a3b5c7d(n)) return DGPE_EINVAL;
    if (cn_chunk(n) > kCnMaxChunk) return DGPE_EUNSUPPORTED;
  }
  if (p->precision != DGPE_FP64 && p->precision != DGPE_MIXED && p->precision != DGPE_DF64) return DGPE_EINVAL;
  return DGPE_OK;
}

int check_physics(const dgpe_params *p) {
  if (!(p->hx > 0 && p->hy > 0 && p->hz > 0) || !finite(p->hx) || !finite(p->hy) || !finite(p->hz))
    return DGPE_EINVAL;
  if (p->mode != DGPE_REAL_TIME && p->mode != DGPE_IMAG_TIME) return DGPE_EINVAL;
  if (!finite(p->dt) || p->dt == 0.0) return DGPE_EINVAL;
  if (p->mode == DGPE_IMAG_TIME && !(p->dt > 0)) return DGPE_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!finite(p->nu[d])) return DGPE_EINVAL;
  if (!finite(p->g) || !finite(p->gdd) || !finite(p->cutoff)) return DGPE_EINVAL;
  if (p->integration != DGPE_RECTANGLE && p->integration != DGPE_SIMPSON) return DGPE_EINVAL;
  if (p->kinetic != DGPE_KINETIC_LAPLACIAN3 && p->kinetic != DGPE_KINETIC_GRADIENT5) return DGPE_EINVAL;
  return DGPE_OK;
}

struct Layout {
  size_t state, partials, tw[3], cn[3], cn_adj[3], cnz, cn8[3], cn8_adj[2], dtv[3], psi, spec, utab, ybuf, total;
};

// FP32 contexts whose compile-time K5 (nz = 128, 256, 384, 512) solves along z at a chunk
// other than the sweeps' power of two (nz = 384: 12 points per lane) get their own tables.
bool needs_cnz(const dgpe_params *p) {
  const int nz = p->nz;
  return p->precision == DGPE_MIXED && (nz == 128 || nz == 256 || nz == 384 || nz == 512) &&
         k5_chunk(nz) != cn_chunk(nz);
}

Layout layout_of(const dgpe_params *p, const KernelSet *ks, int max_blocks) {
  const size_t e = (size_t)(p->precision == DGPE_MIXED ? 8 : 16);
  const int n[3] = {p->nx, p->ny, p->nz};
  Layout L{};
  size_t off = 0;
  L.state = off;
  off += align_up(sizeof(DevState));
  L.partials = off;
  off += align_up((size_t)max_blocks * 8 * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    L.tw[d] = off;
    off += align_up((size_t)n[d] * e);
  }
  for (int d = 0; d < 3; ++d) {
    L.cn[d] = off;
    // lane-interleaved tables, scan factors, then the twist pivot of the two-thread sweeps
    off += align_up((size_t)(4 * cn_chunk(n[d]) + 11) * kWarp * e);
    L.cn_adj[d] = off;   // the same for dt -> -dt (adjoint)
    off += align_up((size_t)(4 * cn_chunk(n[d]) + 11) * kWarp * e);
  }
  L.cnz = 0;   // K5's z tables at their own chunk (FP32 where the compile-time K5 needs them)
  if (needs_cnz(p)) {
    L.cnz = off;
    off += align_up((size_t)(4 * k5_chunk(p->nz) + 11) * kWarp * e);
  }
  // tables in the 8-lane layout: the x and y sweeps' (FP32 short lines), K5's z solve (FP32,
  // the compile-time K5 of nz = 64, 96, 128)
  for (int d = 0; d < 3; ++d) {
    L.cn8[d] = 0;
    if (p->precision == DGPE_MIXED && (d < 2 ? short_cn_chunk(n[d]) != 0 : k5_short_z(n[d]))) {
      L.cn8[d] = off;
      off += align_up((size_t)(4 * 8 * short_cn_chunk(n[d]) + 49) * e);
    }
  }
  for (int d = 0; d < 2; ++d) {   // the same for dt -> -dt (the adjoint x and y sweeps)
    L.cn8_adj[d] = 0;
    if (L.cn8[d]) {
      L.cn8_adj[d] = off;
      off += align_up((size_t)(4 * 8 * short_cn_chunk(n[d]) + 49) * e);
    }
  }
  for (int d = 0; d < 3; ++d) {
    L.dtv[d] = off;
    off += align_up((size_t)n[d] * (e / 2));
  }
  L.psi = off;
  off += align_up((size_t)p->nx * p->ny * p->nz * e);
  L.spec = off;
  off += align_up((size_t)(p->nz / 2 + 1) * p->nx * p->ny * e);
  L.utab = off;   // FP64 and double-float (8-byte entries); the FP32 kernels evaluate it in place
  if (p->precision != DGPE_MIXED) off += align_up((size_t)(p->nz / 2 + 1) * p->nx * p->ny * 8);
  L.ybuf = off;   // the forward-elimination values of the FP64 per-line sweeps
  if (p->precision == DGPE_FP64) off += align_up((size_t)p->nx * p->ny * p->nz * e);
  L.total = off;
  (void)ks;
  return L;
}

const KernelSet *kernel_set(int precision) {
  return precision == DGPE_FP64 ? kernels_f64() : precision == DGPE_DF64 ? kernels_df64() : kernels_f32();
}

// d = f + l: f its FP32 rounding, l = fl32(d - f) (the double-float pair of d)
void split_df(double d, float *f, float *l) {
  *f = (float)d;
  *l = (float)(d - (double)*f);
}

KArgs base_args(const dgpe_params *p) {
  KArgs a{};
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.nzh = p->nz / 2 + 1;
  for (int d = 0; d < 3; ++d) {
    const int n = d == 0 ? p->nx : d == 1 ? p->ny : p->nz;
    a.plan[d] = make_plan(n, 0);
    a.cn[d].m = n - 2;
    a.cn[d].chunk = cn_chunk(n);
    a.cn[d].lchunk = log2_int(a.cn[d].chunk);
  }
  return a;
}

void set_physics(KArgs &a, const dgpe_params *p) {
  a.hx = p->hx;
  a.hy = p->hy;
  a.hz = p->hz;
  a.dt = p->dt;
  a.cutoff = p->cutoff;
  a.has_cutoff = p->cutoff > 0.0;
  a.cutoff_f = (float)p->cutoff;
  a.kf[0] = (float)(2.0 * M_PI / (p->nx * p->hx));
  a.kf[1] = (float)(2.0 * M_PI / (p->ny * p->hy));
  a.kf[2] = (float)(2.0 * M_PI / (p->nz * p->hz));
  a.simpson = p->integration == DGPE_SIMPSON;
  a.kinetic5 = p->kinetic == DGPE_KINETIC_GRADIENT5;
  a.g = p->g;
  a.gdd = p->gdd;
  a.vx = 0.5 * p->nu[0] * p->nu[0];
  a.vy = 0.5 * p->nu[1] * p->nu[1];
  a.vz = 0.5 * p->nu[2] * p->nu[2];
  a.inv_ntot = 1.0 / ((double)p->nx * p->ny * p->nz);
  split_df(a.inv_ntot, &a.inv_ntot_f, &a.inv_ntot_l);
  a.imag = p->mode == DGPE_IMAG_TIME;
  const double h[3] = {p->hx, p->hy, p->hz};
  for (int d = 0; d < 3; ++d) {
    a.cn_r[d] = p->dt / (4.0 * h[d] * h[d]);
    split_df(a.cn_r[d], &a.cn_rf[d], &a.cn_rl[d]);
  }
  a.dt_nuz = p->dt * p->nu[2];
  a.dtg = p->dt * p->g;
  a.dtgdd_n = p->dt * p->gdd * a.inv_ntot;
  split_df(a.dtg, &a.dtg_f, &a.dtg_l);
  split_df(a.dtgdd_n, &a.dtgdd_n_f, &a.dtgdd_n_l);
}

thread_local char g_last_cuda_error[128] = "";

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return DGPE_OK;
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return DGPE_ENOMEM;
  return DGPE_ECUDA;
}

const char *kKernelNames[kNumKernels] = {"k1_density_r2c_z",  "k2_fft_y",            "k3_fft_x_dipolar_ifft_x",
                                         "k4_ifft_y",         "k5_c2r_z_phase_cn_z", "k6_cn_y",
                                         "k7_cn_x_reduce",    "materialize",         "observables",
                                         "adj_phase_r2c_z",   "adj_combine"};

}  // namespace

struct dgpe_ctx {
  dgpe_params p;
  const KernelSet *ks;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  void *ws;
  bool owns_ws;
  Layout L;
  KArgs args;
  cudaGraphExec_t graph;
  bool graph_valid;
  bool timing;
  std::vector<cudaEvent_t> ev_free;
  struct Pending {
    int kernel;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double total_ms[kNumKernels];
  long long launches[kNumKernels];
  int latched;
  int plan_style[3];
  unsigned generation;   // bumped whenever the captured step would change (batches rebuild)
  // real time, FP32-mixed: every step restores the norm the real-time run began with (off
  // during dgpe_grad_z2, whose adjoint differentiates the plain step)
  bool restore_norm;
  // dgpe_step_host: a second psi buffer (successive states alternate between the two, each
  // with its own captured step), the output staging of double-float, one copy stream each
  // way, and their events
  void *psi_main, *psi_alt, *stage_out;
  cudaGraphExec_t graph_alt;
  bool graph_alt_valid;
  cudaStream_t cs_in, cs_out;
  cudaEvent_t ev_in_ready, ev_out_ready, ev_stage_free, ev_main_done[2], ev_d2h_done[2];
  bool host_io;
};

struct dgpe_batch {
  std::vector<dgpe_ctx *> ctxs;
  std::vector<unsigned> gens;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> events;
  std::map<int, cudaGraphExec_t> graphs;   // steps per branch -> instantiated graph
  // same-shaped FP32 contexts stepped together (each kernel one launch for the group): the
  // members, their arguments on the host and in device memory (args_dev: one array for all
  // groups, allocated at dgpe_batch_create)
  struct Group {
    std::vector<int> members;
    size_t offset;   // first entry of the group in args_dev
  };
  std::vector<Group> groups;
  std::vector<int> singles;   // contexts stepped on their own
  std::vector<KArgs> args_host;
  KArgs *args_dev = nullptr;
};

namespace {

void *at(dgpe_ctx *c, size_t off) { return static_cast<char *>(c->ws) + off; }

double kernel_bytes(const dgpe_ctx *c, int k) {
  const double e = c->ks->elem_bytes;
  const double ntot = (double)c->p.nx * c->p.ny * c->p.nz;
  const double nspec = (double)(c->p.nz / 2 + 1) * c->p.nx * c->p.ny;
  switch (k) {
    case kK1DensityR2Cz: return e * (ntot + nspec);
    case kK2FftY:
    case kK4IfftY: return 2 * e * nspec;
    // FP64 reads the dipolar kernel table (one real value per spectral point) as well
    case kK3FftXDipolar: return 2 * e * nspec + (c->p.precision != DGPE_MIXED ? e / 2 * nspec : 0.0);
    case kK5C2RzPhaseCnz: return e * (nspec + 2 * ntot);
    case kK6CnY:
    case kK7CnXReduce:
    case kKMaterialize: return 2 * e * ntot;
    case kKObs: return e * (nspec + 5 * ntot);
    case kKAdjPhase: return e * (2 * nspec + 4 * ntot);
    case kKAdjCombine: return e * (nspec + 3 * ntot);
    default: return 0;
  }
}

cudaEvent_t get_event(dgpe_ctx *c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch one kernel of the step on stream st, timed with events when timing is on.
template <typename F>
int launch(dgpe_ctx *c, cudaStream_t st, int kernel, F &&f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->timing) {
    a = get_event(c);
    b = get_event(c);
    if (!a || !b) return DGPE_ECUDA;
    if (cudaEventRecord(a, st) != cudaSuccess) return DGPE_ECUDA;
  }
  const int rc = map_cuda(f());
  if (rc != DGPE_OK) return rc;
  if (c->timing) {
    if (cudaEventRecord(b, st) != cudaSuccess) return DGPE_ECUDA;
    c->pending.push_back({kernel, a, b});
  }
  return DGPE_OK;
}

int enqueue_potential_transforms(dgpe_ctx *c, cudaStream_t st) {
  const KArgs &a = c->args;
  const KernelSet *ks = c->ks;
  int rc;
  if ((rc = launch(c, st, kK1DensityR2Cz, [&] { return ks->k1(a, st); }))) return rc;
  if ((rc = launch(c, st, kK2FftY, [&] { return ks->k2(a, st); }))) return rc;
  if ((rc = launch(c, st, kK3FftXDipolar, [&] { return ks->k3(a, st); }))) return rc;
  if ((rc = launch(c, st, kK4IfftY, [&] { return ks->k4(a, st); }))) return rc;
  return DGPE_OK;
}

int enqueue_step(dgpe_ctx *c, cudaStream_t st) {
  const KArgs &a = c->args;
  const KernelSet *ks = c->ks;
  int rc;
  if ((rc = enqueue_potential_transforms(c, st))) return rc;
  if ((rc = launch(c, st, kK5C2RzPhaseCnz, [&] { return ks->k5(a, kZStep, st); }))) return rc;
  if ((rc = launch(c, st, kK6CnY, [&] { return ks->k6(a, st); }))) return rc;
  const int renorm = a.imag ? kRenormUnit : (c->restore_norm ? kRenormRestore : kRenormNone);
  if ((rc = launch(c, st, kK7CnXReduce, [&] { return ks->k7(a, 1, renorm, st); }))) return rc;
  return DGPE_OK;
}

// The captured step of the psi buffer the context currently holds (the workspace's, or the
// second buffer of dgpe_step_host).
bool on_alt_psi(const dgpe_ctx *c) { return c->psi_alt && c->args.psi == c->psi_alt; }

// Work that changes psi first waits for the output copy of the last dgpe_step_host call,
// which reads the state buffer itself.
int wait_host_output(dgpe_ctx *c, cudaStream_t st) {
  if (!c->host_io) return DGPE_OK;
  return map_cuda(cudaStreamWaitEvent(st, c->ev_d2h_done[on_alt_psi(c) ? 1 : 0], 0));
}

int build_graph(dgpe_ctx *c) {
  const bool alt = on_alt_psi(c);
  cudaGraphExec_t &graph = alt ? c->graph_alt : c->graph;
  bool &valid = alt ? c->graph_alt_valid : c->graph_valid;
  if (valid) return DGPE_OK;
  if (graph) {
    cudaGraphExecDestroy(graph);
    graph = nullptr;
  }
  const bool timing = c->timing;
  c->timing = false;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c->timing = timing;
    return map_cuda(e);
  }
  const int rc = enqueue_step(c, c->cap_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &g);
  c->timing = timing;
  if (rc != DGPE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return map_cuda(e);
  e = cudaGraphInstantiate(&graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    graph = nullptr;
    return map_cuda(e);
  }
  valid = true;
  return DGPE_OK;
}

// Per-axis tables of the physics: dt v_d x^2 (always), the Crank-Nicolson factor tables
// (only when dt, h or the mode changed, or on the first call) and the dipolar kernel on the
// half spectrum (only when h or the cutoff changed, or on the first call).
int setup_tables(dgpe_ctx *c, bool cn_changed, bool ut_changed) {
  const dgpe_params *p = &c->p;
  const double h[3] = {p->hx, p->hy, p->hz};
  const int n[3] = {p->nx, p->ny, p->nz};
  const double v[3] = {c->args.vx, c->args.vy, c->args.vz};
  CnJobs jobs{};
  jobs.imag = p->mode == DGPE_IMAG_TIME;
  for (int d = 0; d < 3; ++d) {
    int rc = map_cuda(c->ks->axis_potential(at(c, c->L.dtv[d]), n[d], h[d], v[d], p->dt, c->stream));
    if (rc) return rc;
    if (!cn_changed) continue;
    jobs.job[jobs.n++] = {at(c, c->L.cn[d]), c->args.cn[d].m, c->args.cn[d].chunk, c->args.cn_r[d], kWarp};
    if (p->mode == DGPE_REAL_TIME)   // the adjoint sweep is the sweep with dt -> -dt
      jobs.job[jobs.n++] = {at(c, c->L.cn_adj[d]), c->args.cn[d].m, c->args.cn[d].chunk, -c->args.cn_r[d], kWarp};
    if (c->L.cn8[d]) jobs.job[jobs.n++] = {at(c, c->L.cn8[d]), c->args.cn[d].m, n[d] / 8, c->args.cn_r[d], 8};
    if (d < 2 && c->L.cn8_adj[d] && p->mode == DGPE_REAL_TIME)
      jobs.job[jobs.n++] = {at(c, c->L.cn8_adj[d]), c->args.cn[d].m, n[d] / 8, -c->args.cn_r[d], 8};
  }
  if (cn_changed && c->L.cnz)
    jobs.job[jobs.n++] = {at(c, c->L.cnz), c->args.cn[2].m, k5_chunk(p->nz), c->args.cn_r[2], kWarp};
  if (jobs.n) {
    const int rc = map_cuda(c->ks->cn_tables(jobs, c->stream));
    if (rc) return rc;
  }
  if (ut_changed) return map_cuda(c->ks->dipolar_table(c->args, c->stream));
  return DGPE_OK;
}

// Read the device flags after a synchronisation; latch a device error.
int check_device_flags(dgpe_ctx *c) {
  unsigned int flags = 0;
  cudaError_t e = cudaMemcpy(&flags, &static_cast<DevState *>(at(c, c->L.state))->flags, sizeof(flags),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return map_cuda(e);
  if (flags & kFlagNonFinite) c->latched = DGPE_ENONFINITE;
  return c->latched;
}

}  // namespace

namespace {

// The sweeps of the adjoint step run on the cotangent with the conjugate (dt -> -dt) tables.
KArgs adjoint_sweep_args(dgpe_ctx *c, void *gbar) {
  KArgs a = c->args;
  a.psi = gbar;
  for (int d = 0; d < 3; ++d) {
    a.cn[d].tab = at(c, c->L.cn_adj[d]);
    // the adjoint x and y sweeps of short lines on their own 8-lane tables; K5's z solve does
    // not run in the adjoint step
    a.cn8_tab[d] = d < 2 && c->L.cn8_adj[d] ? at(c, c->L.cn8_adj[d]) : nullptr;
    a.cn_r[d] = -a.cn_r[d];
    a.cn_rf[d] = -a.cn_rf[d];
    a.cn_rl[d] = -a.cn_rl[d];
  }
  return a;
}

// Adjoint of one real-time step (GPU order P, Z, Y, X): X^H, Y^H, Z^H on gbar, then the
// adjoint of the potential step, which needs Phi of |psi_k|^2 and then Phi of s.
int enqueue_adjoint_step(dgpe_ctx *c, const void *psi_k, void *gbar, double *nu_slot) {
  cudaStream_t st = c->stream;
  const KernelSet *ks = c->ks;
  const KArgs sw = adjoint_sweep_args(c, gbar);
  int rc;
  if ((rc = launch(c, st, kK7CnXReduce, [&] { return ks->k7(sw, 0, 0, st); }))) return rc;
  if ((rc = launch(c, st, kK6CnY, [&] { return ks->k6(sw, st); }))) return rc;
  if ((rc = launch(c, st, kK5C2RzPhaseCnz, [&] { return ks->k5(sw, kZCnOnly, st); }))) return rc;
  KArgs fa = c->args;
  fa.psi = const_cast<void *>(psi_k);
  fa.gbar = gbar;
  fa.unit_scale = 1;
  fa.grad_nu_slot = nu_slot;
  if ((rc = launch(c, st, kK1DensityR2Cz, [&] { return ks->k1(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK2FftY, [&] { return ks->k2(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK3FftXDipolar, [&] { return ks->k3(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK4IfftY, [&] { return ks->k4(fa, st); }))) return rc;
  if ((rc = launch(c, st, kKAdjPhase, [&] { return ks->adj_phase(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK2FftY, [&] { return ks->k2(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK3FftXDipolar, [&] { return ks->k3(fa, st); }))) return rc;
  if ((rc = launch(c, st, kK4IfftY, [&] { return ks->k4(fa, st); }))) return rc;
  return launch(c, st, kKAdjCombine, [&] { return ks->adj_combine(fa, st); });
}

// nu_z during a trajectory: only the z table of dt v_z z^2 is rebuilt (the captured step
// graph stays valid).
int set_nu_z(dgpe_ctx *c, double v) {
  if (v == c->p.nu[2]) return DGPE_OK;
  c->p.nu[2] = v;
  c->args.vz = 0.5 * v * v;
  c->args.dt_nuz = c->p.dt * v;
  return map_cuda(c->ks->axis_potential(at(c, c->L.dtv[2]), c->p.nz, c->p.hz, c->args.vz, c->p.dt, c->stream));
}

int grad_steps_per_checkpoint(int nsteps) {
  int k = 1;
  while ((long)k * k < nsteps) ++k;
  return k;
}

struct GradLayout {
  size_t state, ckpt, seg, gbar, dnu, total;
  int k, nck;
};

GradLayout grad_layout(const dgpe_ctx *c, int nseg, int steps_per_seg) {
  GradLayout g{};
  const int n = nseg * steps_per_seg;
  g.k = grad_steps_per_checkpoint(n);
  g.nck = (n + g.k - 1) / g.k;
  g.state = align_up((size_t)c->p.nx * c->p.ny * c->p.nz * c->ks->elem_bytes);
  g.ckpt = 0;
  g.seg = g.ckpt + (size_t)g.nck * g.state;
  g.gbar = g.seg + (size_t)g.k * g.state;
  g.dnu = g.gbar + g.state;
  g.total = g.dnu + align_up((size_t)nseg * sizeof(double));
  return g;
}

}  // namespace

namespace {

// Drain the timing events of the launches enqueued with timing on: per-kernel milliseconds.
int drain_kernel_times(dgpe_ctx *c, double *ms) {
  int rc = map_cuda(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < kNumKernels; ++q) ms[q] = 0;
  for (const auto &pd : c->pending) {
    float t = 0.f;
    if (rc == DGPE_OK && cudaEventElapsedTime(&t, pd.a, pd.b) == cudaSuccess) ms[pd.kernel] += t;
    c->ev_free.push_back(pd.a);
    c->ev_free.push_back(pd.b);
  }
  c->pending.clear();
  return rc;
}

int apply_tuning(dgpe_ctx *c, const dgpe_tuning &t) {
  const int n[3] = {c->p.nx, c->p.ny, c->p.nz};
  int rc = DGPE_OK;
  for (int d = 0; d < 3; ++d) {
    const bool changed = c->plan_style[d] != t.plan_style[d];
    c->plan_style[d] = t.plan_style[d];
    c->args.plan[d] = make_plan(n[d], t.plan_style[d]);
    // the twiddle tables are laid out per stage of the plan
    if (changed && !rc) rc = map_cuda(c->ks->twiddles(const_cast<void *>(c->args.tw[d]), c->args.plan[d], c->stream));
  }
  c->args.ylines = t.ylines;
  c->args.fft_threads = t.fft_threads;
  c->args.cn_per_sm = t.cn_per_sm;
  c->graph_valid = c->graph_alt_valid = false;
  ++c->generation;
  return rc;
}

bool tuning_valid(const dgpe_ctx *c, const dgpe_tuning &t) {
  for (int d = 0; d < 3; ++d)
    if (t.plan_style[d] < 0 || t.plan_style[d] > 2) return false;
  if (t.fft_threads != 128 && t.fft_threads != 256) return false;
  if (t.ylines < 2 || t.ylines > 32 || (t.ylines & (t.ylines - 1))) return false;
  if (c->ks->y_smem(c->p.ny, t.ylines) + 8192 > 227 * 1024) return false;
  if (t.cn_per_sm < 1 || t.cn_per_sm > 2) return false;
  return true;
}

dgpe_tuning current_tuning(const dgpe_ctx *c) {
  dgpe_tuning t{};
  for (int d = 0; d < 3; ++d) t.plan_style[d] = c->plan_style[d];
  t.ylines = c->args.ylines;
  t.fft_threads = c->args.fft_threads;
  t.cn_per_sm = c->args.cn_per_sm;
  return t;
}

}  // namespace

extern "C" {

const char *dgpe_strerror(int code) {
  switch (code) {
    case DGPE_OK: return "ok";
    case DGPE_EINVAL: return "invalid argument or parameter";
    case DGPE_ENOMEM: return "out of device memory or workspace too small";
    case DGPE_ECUDA: return "CUDA runtime error";
    case DGPE_ENONFINITE: return "non-finite value in a device reduction";
    case DGPE_ETIMEOUT: return "device-side wait timed out";
    case DGPE_EUNSUPPORTED: return "unsupported by this build";
    default: return "unknown error code";
  }
}

const char *dgpe_last_cuda_error(void) { return g_last_cuda_error; }

int dgpe_workspace_bytes(const dgpe_params *p, size_t *bytes) {
  if (!p || !bytes) return DGPE_EINVAL;
  int rc = check_shape(p);
  if (rc) return rc;
  // the block count of the reducing kernels depends only on shape and precision
  const KernelSet *ks = kernel_set(p->precision);
  *bytes = layout_of(p, ks, ks->max_blocks(base_args(p))).total;
  return DGPE_OK;
}

int dgpe_create(const dgpe_params *p, void *cuda_stream, dgpe_ctx **out) {
  if (!p || !out) return DGPE_EINVAL;
  *out = nullptr;
  int rc = check_shape(p);
  if (rc) return rc;
  if ((rc = check_physics(p))) return rc;
  size_t need = 0;
  dgpe_workspace_bytes(p, &need);
  if (p->workspace) {
    if (p->workspace_bytes < need) return DGPE_ENOMEM;
    if (reinterpret_cast<uintptr_t>(p->workspace) % kAlign) return DGPE_EINVAL;
  }
  dgpe_ctx *c = new (std::nothrow) dgpe_ctx();
  if (!c) return DGPE_ENOMEM;
  c->p = *p;
  c->restore_norm = p->precision == DGPE_MIXED;
  c->ks = kernel_set(p->precision);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->args = base_args(p);
  set_physics(c->args, p);
  c->L = layout_of(p, c->ks, c->ks->max_blocks(c->args));
  c->args.ylines = c->ks->default_ylines(p->ny);
  c->args.fft_threads = 256;
  c->args.cn_per_sm = 2;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      c->args.nsm = nsm;
  }
  rc = map_cuda(c->ks->init());
  if (!rc) rc = map_cuda(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!rc) {
    if (p->workspace) {
      c->ws = p->workspace;
      c->owns_ws = false;
    } else {
      rc = map_cuda(cudaMalloc(&c->ws, c->L.total));
      c->owns_ws = rc == DGPE_OK;
    }
  }
  if (rc) {
    dgpe_destroy(c);
    return rc;
  }
  KArgs &a = c->args;
  a.state = static_cast<DevState *>(at(c, c->L.state));
  a.partials = static_cast<double *>(at(c, c->L.partials));
  a.psi = at(c, c->L.psi);
  c->psi_main = a.psi;
  a.spec = at(c, c->L.spec);
  for (int d = 0; d < 3; ++d) {
    a.tw[d] = at(c, c->L.tw[d]);
    a.cn[d].tab = at(c, c->L.cn[d]);
    a.dtv[d] = at(c, c->L.dtv[d]);
  }
  a.utab = at(c, c->L.utab);
  a.ybuf = at(c, c->L.ybuf);
  a.cnz_tab = c->L.cnz ? at(c, c->L.cnz) : nullptr;
  for (int d = 0; d < 3; ++d) a.cn8_tab[d] = c->L.cn8[d] ? at(c, c->L.cn8[d]) : nullptr;
  const int n[3] = {p->nx, p->ny, p->nz};
  rc = map_cuda(cudaMemsetAsync(a.psi, 0, (size_t)p->nx * p->ny * p->nz * c->ks->elem_bytes, c->stream));
  if (!rc) rc = map_cuda(c->ks->reset_state(a.state, c->stream));
  for (int d = 0; d < 3 && !rc; ++d) rc = map_cuda(c->ks->twiddles(const_cast<void *>(a.tw[d]), a.plan[d], c->stream));
  (void)n;
  if (!rc) rc = setup_tables(c, true, true);
  if (rc) {
    dgpe_destroy(c);
    return rc;
  }
  *out = c;
  return DGPE_OK;
}

int dgpe_set_params(dgpe_ctx *c, const dgpe_params *p) {
  if (!c || !p) return DGPE_EINVAL;
  if (p->nx != c->p.nx || p->ny != c->p.ny || p->nz != c->p.nz || p->precision != c->p.precision)
    return DGPE_EINVAL;
  int rc = check_physics(p);
  if (rc) return rc;
  const bool cn_changed = p->dt != c->p.dt || p->hx != c->p.hx || p->hy != c->p.hy || p->hz != c->p.hz ||
                          p->mode != c->p.mode;
  const bool ut_changed = p->hx != c->p.hx || p->hy != c->p.hy || p->hz != c->p.hz || p->cutoff != c->p.cutoff;
  const bool step_args_changed = cn_changed || p->g != c->p.g || p->gdd != c->p.gdd || p->cutoff != c->p.cutoff ||
                                 p->integration != c->p.integration;
  void *ws = c->p.workspace;
  const size_t wsb = c->p.workspace_bytes;
  c->p = *p;
  c->p.workspace = ws;
  c->p.workspace_bytes = wsb;
  set_physics(c->args, p);
  // the step kernels read the trap only through the per-axis tables rebuilt below, so a
  // change of nu alone keeps the captured graph valid
  if (step_args_changed) {
    c->graph_valid = c->graph_alt_valid = false;
    ++c->generation;
  }
  return setup_tables(c, cn_changed, ut_changed);
}

int dgpe_set_psi(dgpe_ctx *c, const void *psi, int where) {
  if (!c || !psi || (where != DGPE_HOST && where != DGPE_DEVICE)) return DGPE_EINVAL;
  if (const int w = wait_host_output(c, c->stream)) return w;
  const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz;
  const size_t bytes = n * c->ks->elem_bytes;
  int rc;
  if (c->p.precision == DGPE_DF64) {
    // complex128 in, double-float pairs (same 16 bytes per value) in the workspace: copy,
    // then split in place
    rc = map_cuda(cudaMemcpyAsync(c->args.psi, psi, bytes,
                                  where == DGPE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    if (!rc) rc = map_cuda(c->ks->from_c128(c->args.psi, c->args.psi, n, c->stream));
  } else {
    rc = map_cuda(cudaMemcpyAsync(c->args.psi, psi, bytes,
                                  where == DGPE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
  }
  if (!rc) rc = map_cuda(c->ks->reset_state(c->args.state, c->stream));
  if (!rc && where == DGPE_HOST) rc = map_cuda(cudaStreamSynchronize(c->stream));
  if (!rc) c->latched = DGPE_OK;
  return rc;
}

int dgpe_get_psi(dgpe_ctx *c, void *out, int where) {
  if (!c || !out || (where != DGPE_HOST && where != DGPE_DEVICE)) return DGPE_EINVAL;
  if (const int w = wait_host_output(c, c->stream)) return w;
  const size_t bytes = (size_t)c->p.nx * c->p.ny * c->p.nz * c->ks->elem_bytes;
  int rc = launch(c, c->stream, kKMaterialize, [&] { return c->ks->materialize(c->args, c->stream); });
  if (rc) return rc;
  if (c->p.precision == DGPE_DF64) {
    // double-float pairs -> complex128, through a stream-ordered temporary for a host buffer
    const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz;
    if (where == DGPE_DEVICE) {
      rc = map_cuda(c->ks->to_c128(c->args.psi, out, n, c->stream));
    } else {
      void *tmp = nullptr;
      rc = map_cuda(cudaMallocAsync(&tmp, bytes, c->stream));
      if (!rc) rc = map_cuda(c->ks->to_c128(c->args.psi, tmp, n, c->stream));
      if (!rc) rc = map_cuda(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->stream));
      if (tmp) cudaFreeAsync(tmp, c->stream);
    }
  } else {
    rc = map_cuda(cudaMemcpyAsync(out, c->args.psi, bytes,
                                  where == DGPE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
  }
  if (rc) return rc;
  if (where == DGPE_HOST) {
    rc = map_cuda(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    return check_device_flags(c);
  }
  return DGPE_OK;
}

int dgpe_step(dgpe_ctx *c, int nsteps) {
  if (!c || nsteps < 0) return DGPE_EINVAL;
  if (nsteps == 0) return DGPE_OK;
  if (const int w = wait_host_output(c, c->stream)) return w;
  if (c->timing) {
    for (int s = 0; s < nsteps; ++s) {
      const int rc = enqueue_step(c, c->stream);
      if (rc) return rc;
    }
    return DGPE_OK;
  }
  int rc = build_graph(c);
  if (rc) return rc;
  cudaGraphExec_t graph = on_alt_psi(c) ? c->graph_alt : c->graph;
  for (int s = 0; s < nsteps; ++s) {
    rc = map_cuda(cudaGraphLaunch(graph, c->stream));
    if (rc) return rc;
  }
  return DGPE_OK;
}

int dgpe_substep(dgpe_ctx *c, int which) {
  if (!c) return DGPE_EINVAL;
  if (const int w = wait_host_output(c, c->stream)) return w;
  const KArgs &a = c->args;
  const KernelSet *ks = c->ks;
  cudaStream_t st = c->stream;
  switch (which) {
    case DGPE_SUB_POTENTIAL: {
      // absorb the pending renormalisation first: the phase step then runs with s = 1
      int rc = launch(c, st, kKMaterialize, [&] { return ks->materialize(a, st); });
      if (!rc) rc = enqueue_potential_transforms(c, st);
      if (!rc) rc = launch(c, st, kK5C2RzPhaseCnz, [&] { return ks->k5(a, kZPhaseOnly, st); });
      return rc;
    }
    case DGPE_SUB_CN_X: return launch(c, st, kK7CnXReduce, [&] { return ks->k7(a, 0, 0, st); });
    case DGPE_SUB_CN_Y: return launch(c, st, kK6CnY, [&] { return ks->k6(a, st); });
    case DGPE_SUB_CN_Z: return launch(c, st, kK5C2RzPhaseCnz, [&] { return ks->k5(a, kZCnOnly, st); });
    default: return DGPE_EINVAL;
  }
}

int dgpe_observables(dgpe_ctx *c, dgpe_obs *o) {
  if (!c || !o) return DGPE_EINVAL;
  int rc = enqueue_potential_transforms(c, c->stream);
  if (!rc) rc = launch(c, c->stream, kKObs, [&] { return c->ks->k5(c->args, kZObs, c->stream); });
  if (rc) return rc;
  double v[10];
  rc = map_cuda(cudaMemcpyAsync(v, c->args.state->obs, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = map_cuda(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  o->norm = v[0];
  o->mu = v[1];
  o->energy = v[2];
  o->rms[0] = v[3];
  o->rms[1] = v[4];
  o->rms[2] = v[5];
  o->e_kin = v[6];
  o->e_trap = v[7];
  o->e_contact = v[8];
  o->e_dipolar = v[9];
  return check_device_flags(c);
}

int dgpe_get_phi(dgpe_ctx *c, void *out, int where) {
  if (!c || !out || (where != DGPE_HOST && where != DGPE_DEVICE)) return DGPE_EINVAL;
  const size_t bytes = (size_t)c->p.nx * c->p.ny * c->p.nz * (c->ks->elem_bytes / 2);
  void *dst = out;
  int rc = DGPE_OK;
  if (where == DGPE_HOST) {
    rc = map_cuda(cudaMallocAsync(&dst, bytes, c->stream));
    if (rc) return rc;
  }
  KArgs a = c->args;
  a.out = dst;
  rc = enqueue_potential_transforms(c, c->stream);
  if (!rc) rc = map_cuda(c->ks->k5(a, kZPhi, c->stream));
  if (where == DGPE_HOST) {
    if (!rc) rc = map_cuda(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    cudaFreeAsync(dst, c->stream);
    if (!rc) rc = map_cuda(cudaStreamSynchronize(c->stream));
    if (!rc) rc = check_device_flags(c);
  }
  return rc;
}

int dgpe_adjoint_step(dgpe_ctx *c, const void *psi_k, void *gbar) {
  if (!c || !psi_k || !gbar) return DGPE_EINVAL;
  if (c->p.mode != DGPE_REAL_TIME || c->p.precision == DGPE_DF64) return DGPE_EUNSUPPORTED;
  return enqueue_adjoint_step(c, psi_k, gbar, nullptr);
}

int dgpe_adjoint_grads(dgpe_ctx *c, double *out, int reset) {
  if (!c || !out) return DGPE_EINVAL;
  double *dev = c->args.state->grads;
  int rc = map_cuda(cudaMemcpyAsync(out, dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (!rc && reset) rc = map_cuda(cudaMemsetAsync(dev, 0, 4 * sizeof(double), c->stream));
  if (!rc) rc = map_cuda(cudaStreamSynchronize(c->stream));
  return rc;
}

int dgpe_grad_z2_workspace_bytes(const dgpe_ctx *c, int nseg, int steps_per_seg, size_t *bytes) {
  if (!c || !bytes || nseg < 1 || steps_per_seg < 1) return DGPE_EINVAL;
  *bytes = grad_layout(c, nseg, steps_per_seg).total;
  return DGPE_OK;
}

int dgpe_grad_z2(dgpe_ctx *c, int nseg, int steps_per_seg, const double *nu_z, void *work, size_t work_bytes,
                 double *loss, double *dnu, double *dg, double *dgdd) {
  if (!c || !nu_z || !work || !loss || !dnu || !dg || !dgdd || nseg < 1 || steps_per_seg < 1) return DGPE_EINVAL;
  if (c->p.mode != DGPE_REAL_TIME || c->p.precision == DGPE_DF64) return DGPE_EUNSUPPORTED;
  for (int s = 0; s < nseg; ++s)
    if (!isfinite(nu_z[s])) return DGPE_EINVAL;
  const GradLayout g = grad_layout(c, nseg, steps_per_seg);
  if (work_bytes < g.total) return DGPE_ENOMEM;
  if (reinterpret_cast<uintptr_t>(work) % kAlign) return DGPE_EINVAL;
  if (const int w = wait_host_output(c, c->stream)) return w;
  char *w = static_cast<char *>(work);
  const int n = nseg * steps_per_seg;
  const size_t sb = (size_t)c->p.nx * c->p.ny * c->p.nz * c->ks->elem_bytes;
  cudaStream_t st = c->stream;
  void *psi = c->args.psi;
  void *gbar = w + g.gbar;
  double *dnu_dev = reinterpret_cast<double *>(w + g.dnu);
  const double nu_z0 = c->p.nu[2];
  int rc = DGPE_OK;
  auto chk = [&](int r) {
    if (rc == DGPE_OK) rc = r;
    return rc == DGPE_OK;
  };
  // the adjoint differentiates the plain step: no norm restoration (FP32-mixed) while the
  // trajectory runs, so that every checkpoint and recomputed state is the state itself
  const bool restore = c->restore_norm;
  auto set_restore = [&](bool on) {
    if (c->restore_norm == on) return;
    c->restore_norm = on;
    c->graph_valid = c->graph_alt_valid = false;
    ++c->generation;
  };
  set_restore(false);
  // absorb a pending renormalisation so that every checkpoint is the state itself
  chk(launch(c, st, kKMaterialize, [&] { return c->ks->materialize(c->args, st); }));
  chk(map_cuda(cudaMemsetAsync(c->args.state->grads, 0, 4 * sizeof(double), st)));
  chk(map_cuda(cudaMemsetAsync(dnu_dev, 0, (size_t)nseg * sizeof(double), st)));
  // forward trajectory with a checkpoint of psi every k steps
  for (int t = 0; t < n && rc == DGPE_OK; ++t) {
    if (t % g.k == 0) chk(map_cuda(cudaMemcpyAsync(w + g.ckpt + (size_t)(t / g.k) * g.state, psi, sb,
                                                   cudaMemcpyDeviceToDevice, st)));
    chk(set_nu_z(c, nu_z[t / steps_per_seg]));
    chk(dgpe_step(c, 1));
  }
  // L = h^3 sum z^2 |psi_N|^2 is the last x-sweep's z^2 moment; its cotangent seeds gbar
  double sum_z2 = 0;
  chk(map_cuda(cudaMemcpyAsync(&sum_z2, &c->args.state->sums[3], sizeof(double), cudaMemcpyDeviceToHost, st)));
  KArgs la = c->args;
  la.gbar = gbar;
  chk(map_cuda(c->ks->loss_z2(la, st)));
  chk(map_cuda(cudaStreamSynchronize(st)));
  *loss = c->p.hx * c->p.hy * c->p.hz * sum_z2;
  // backward, segment by segment: recompute the states of a segment from its checkpoint,
  // then run the adjoint steps through it in reverse
  for (int ck = g.nck - 1; ck >= 0 && rc == DGPE_OK; --ck) {
    const int t0 = ck * g.k, t1 = (t0 + g.k < n) ? t0 + g.k : n;
    chk(map_cuda(cudaMemcpyAsync(psi, w + g.ckpt + (size_t)ck * g.state, sb, cudaMemcpyDeviceToDevice, st)));
    for (int t = t0; t < t1 && rc == DGPE_OK; ++t) {
      chk(map_cuda(cudaMemcpyAsync(w + g.seg + (size_t)(t - t0) * g.state, psi, sb, cudaMemcpyDeviceToDevice, st)));
      if (t + 1 < t1) {   // the state after the segment's last step is not needed
        chk(set_nu_z(c, nu_z[t / steps_per_seg]));
        chk(dgpe_step(c, 1));
      }
    }
    for (int t = t1 - 1; t >= t0 && rc == DGPE_OK; --t) {
      chk(set_nu_z(c, nu_z[t / steps_per_seg]));
      chk(enqueue_adjoint_step(c, w + g.seg + (size_t)(t - t0) * g.state, gbar, dnu_dev + t / steps_per_seg));
    }
  }
  // leave the context at the initial state and the initial nu_z
  chk(map_cuda(cudaMemcpyAsync(psi, w + g.ckpt, sb, cudaMemcpyDeviceToDevice, st)));
  chk(set_nu_z(c, nu_z0));
  double gr[4] = {0, 0, 0, 0};
  chk(map_cuda(cudaMemcpyAsync(gr, c->args.state->grads, sizeof(gr), cudaMemcpyDeviceToHost, st)));
  chk(map_cuda(cudaMemcpyAsync(dnu, dnu_dev, (size_t)nseg * sizeof(double), cudaMemcpyDeviceToHost, st)));
  chk(map_cuda(cudaStreamSynchronize(st)));
  set_restore(restore);
  if (rc) return rc;
  *dg = gr[0];
  *dgdd = gr[1];
  return check_device_flags(c);
}

int dgpe_set_tuning(dgpe_ctx *c, const dgpe_tuning *t) {
  if (!c || !t || !tuning_valid(c, *t)) return DGPE_EINVAL;
  return apply_tuning(c, *t);
}

int dgpe_step_launches(const dgpe_ctx *c, int *n) {
  if (!c || !n) return DGPE_EINVAL;
  *n = 6 + c->ks->k5_launches;   // K1 K2 K3 K4, K5 (1 or 2), K6 K7
  return DGPE_OK;
}

int dgpe_get_tuning(const dgpe_ctx *c, dgpe_tuning *out) {
  if (!c || !out) return DGPE_EINVAL;
  *out = current_tuning(c);
  return DGPE_OK;
}

int dgpe_autotune(dgpe_ctx *c, dgpe_tuning *out) {
  if (!c || !out) return DGPE_EINVAL;
  if (const int w = wait_host_output(c, c->stream)) return w;
  const size_t sb = (size_t)c->p.nx * c->p.ny * c->p.nz * c->ks->elem_bytes;
  void *saved = nullptr;
  DevState st_saved;
  int rc = map_cuda(cudaMallocAsync(&saved, sb, c->stream));
  if (!rc) rc = map_cuda(cudaMemcpyAsync(saved, c->args.psi, sb, cudaMemcpyDeviceToDevice, c->stream));
  if (!rc) rc = map_cuda(cudaMemcpyAsync(&st_saved, c->args.state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  if (!rc) rc = map_cuda(cudaStreamSynchronize(c->stream));
  if (rc) {
    if (saved) cudaFreeAsync(saved, c->stream);
    return rc;
  }
  const dgpe_tuning base = current_tuning(c);
  const int ylines_opts[5] = {2, 4, 8, 16, 32};
  const int threads_opts[2] = {256, 128};
  const int steps = 3;
  // per option, the summed time of the kernels it affects
  double t_style[3][3] = {{1e30, 1e30, 1e30}, {1e30, 1e30, 1e30}, {1e30, 1e30, 1e30}};
  double t_y[5][2], t_x[2] = {1e30, 1e30}, t_cn[2] = {1e30, 1e30};
  for (auto &r : t_y) r[0] = r[1] = 1e30;
  double default_ms = 0;
  const bool timing = c->timing;
  c->timing = true;
  for (int round = 0; round < 10 && rc == DGPE_OK; ++round) {
    dgpe_tuning t = base;
    const int yi = round % 5, ti = (round / 5) % 2, si = round % 3, ci = round % 2;
    if (round > 0) {
      t.ylines = ylines_opts[yi];
      t.fft_threads = threads_opts[ti];
      for (int d = 0; d < 3; ++d) t.plan_style[d] = si;
      t.cn_per_sm = 1 + ci;
    }
    if (!tuning_valid(c, t)) continue;
    rc = apply_tuning(c, t);
    if (!rc) rc = enqueue_step(c, c->stream);   // warm-up step of this configuration
    double ms[kNumKernels];
    if (!rc) rc = drain_kernel_times(c, ms);
    for (int s = 0; s < steps && rc == DGPE_OK; ++s) rc = enqueue_step(c, c->stream);
    if (!rc) rc = drain_kernel_times(c, ms);
    if (rc) break;
    double total = 0;
    for (int q = 0; q < kNumKernels; ++q) total += ms[q];
    if (round == 0) default_ms = total / steps;
    const double tz = ms[kK1DensityR2Cz] + ms[kK5C2RzPhaseCnz], ty = ms[kK2FftY] + ms[kK4IfftY],
                 tx = ms[kK3FftXDipolar], tcn = ms[kK6CnY] + ms[kK7CnXReduce];
    const int sidx[3] = {t.plan_style[0], t.plan_style[1], t.plan_style[2]};
    t_style[0][sidx[0]] = fmin(t_style[0][sidx[0]], tx);
    t_style[1][sidx[1]] = fmin(t_style[1][sidx[1]], ty);
    t_style[2][sidx[2]] = fmin(t_style[2][sidx[2]], tz);
    int yk = 0;
    while (ylines_opts[yk] != t.ylines) ++yk;
    const int tk = t.fft_threads == 256 ? 0 : 1;
    t_y[yk][tk] = fmin(t_y[yk][tk], ty);
    t_x[tk] = fmin(t_x[tk], tx);
    t_cn[t.cn_per_sm - 1] = fmin(t_cn[t.cn_per_sm - 1], tcn);
  }
  dgpe_tuning best = base;
  if (rc == DGPE_OK) {
    // another radix order only when it is faster by more than the timing noise (3 %): the
    // default order is the one with compile-time kernels (faster in grouped launches, where
    // a single context's few-microsecond kernels do not show it)
    for (int d = 0; d < 3; ++d) {
      int b = base.plan_style[d];
      for (int k = 0; k < 3; ++k)
        if (t_style[d][k] < 0.97 * t_style[d][b]) b = k;
      best.plan_style[d] = b;
    }
    // y-pass shape and transform threads: the (ylines, threads) pair with the least y + x time
    double bestv = 1e30;
    for (int yk = 0; yk < 5; ++yk)
      for (int tk = 0; tk < 2; ++tk) {
        const double v = t_y[yk][tk] + t_x[tk];
        if (v < bestv) {
          bestv = v;
          best.ylines = ylines_opts[yk];
          best.fft_threads = threads_opts[tk];
        }
      }
    best.cn_per_sm = t_cn[1] < t_cn[0] ? 2 : 1;
    if (!tuning_valid(c, best)) best = base;
    rc = apply_tuning(c, best);
    for (int s = 0; s < 1 + steps && rc == DGPE_OK; ++s) {
      rc = enqueue_step(c, c->stream);
      if (s == 0 && !rc) {
        double ms0[kNumKernels];
        rc = drain_kernel_times(c, ms0);
      }
    }
    double ms[kNumKernels];
    if (!rc) rc = drain_kernel_times(c, ms);
    double total = 0;
    for (int q = 0; q < kNumKernels; ++q) total += ms[q];
    best.step_ms_default = default_ms;
    best.step_ms_tuned = total / steps;
  }
  c->timing = timing;
  // restore the state the tuning steps advanced
  int rc2 = map_cuda(cudaMemcpyAsync(c->args.psi, saved, sb, cudaMemcpyDeviceToDevice, c->stream));
  if (!rc2) rc2 = map_cuda(cudaMemcpyAsync(c->args.state, &st_saved, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  cudaFreeAsync(saved, c->stream);
  if (!rc2) rc2 = map_cuda(cudaStreamSynchronize(c->stream));
  if (rc == DGPE_OK) rc = rc2;
  if (rc == DGPE_OK) *out = best;
  return rc;
}

int dgpe_batch_create(dgpe_ctx *const *ctxs, int n, void *cuda_stream, dgpe_batch **out) {
  if (!ctxs || n < 1 || !out) return DGPE_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return DGPE_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return DGPE_EINVAL;
  }
  dgpe_batch *b = new (std::nothrow) dgpe_batch();
  if (!b) return DGPE_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + n);
  b->gens.assign(n, ~0u);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = map_cuda(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  b->branches.assign(n, nullptr);
  b->events.assign(n + 1, nullptr);
  for (int i = 0; i < n && !rc; ++i) rc = map_cuda(cudaStreamCreateWithFlags(&b->branches[i], cudaStreamNonBlocking));
  for (int i = 0; i <= n && !rc; ++i) rc = map_cuda(cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming));
  // the argument array of the grouped launches (at most every context in one group)
  if (!rc) rc = map_cuda(cudaMalloc(reinterpret_cast<void **>(&b->args_dev), (size_t)n * sizeof(KArgs)));
  if (rc) {
    dgpe_batch_destroy(b);
    return rc;
  }
  *out = b;
  return DGPE_OK;
}

// Contexts whose step kernels can run as one grouped launch: FP32, and the same shape,
// mode, norm handling and launch shape (radix orders, y lines per CTA, transform threads,
// sweep CTAs per SM).
static bool same_group(const dgpe_ctx *x, const dgpe_ctx *y) {
  const KArgs &a = x->args, &b = y->args;
  if (x->ks != y->ks || !x->ks->step_group) return false;
  if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.imag != b.imag || x->restore_norm != y->restore_norm)
    return false;
  if (a.ylines != b.ylines || a.fft_threads != b.fft_threads || a.cn_per_sm != b.cn_per_sm) return false;
  for (int d = 0; d < 3; ++d)
    if (x->plan_style[d] != y->plan_style[d]) return false;
  return true;
}

// Sort the contexts into groups (two or more members) and singles, and copy every group's
// arguments to the device array, stream-ordered on the batch stream (before any later
// launch of the batch's graphs).
static int batch_group(dgpe_batch *b) {
  const int n = (int)b->ctxs.size();
  b->groups.clear();
  b->singles.clear();
  b->args_host.clear();
  std::vector<char> used(n, 0);
  for (int i = 0; i < n; ++i) {
    if (used[i]) continue;
    dgpe_batch::Group g;
    g.members.push_back(i);
    for (int j = i + 1; j < n; ++j)
      if (!used[j] && same_group(b->ctxs[i], b->ctxs[j])) {
        g.members.push_back(j);
        used[j] = 1;
      }
    if (g.members.size() < 2) {
      b->singles.push_back(i);
      continue;
    }
    g.offset = b->args_host.size();
    for (int m : g.members) b->args_host.push_back(b->ctxs[m]->args);
    b->groups.push_back(g);
  }
  // branch priorities: the less work a branch (group or single) has, the higher its stream
  // priority, so that the short, latency-bound chains of small grids get SMs as soon as the
  // large grids' blocks free them instead of waiting behind whole launches (the graph keeps
  // each kernel's priority from the stream it was captured on)
  {
    std::vector<std::pair<double, int>> work;   // (points x members, branch leader)
    for (const dgpe_batch::Group &g : b->groups) {
      const KArgs &a = b->ctxs[g.members[0]]->args;
      work.push_back({(double)a.nx * a.ny * a.nz * g.members.size(), g.members[0]});
    }
    for (int i : b->singles) {
      const KArgs &a = b->ctxs[i]->args;
      work.push_back({(double)a.nx * a.ny * a.nz, i});
    }
    std::sort(work.begin(), work.end(), [](const std::pair<double, int> &x, const std::pair<double, int> &y) {
      return x.first > y.first;
    });
    int least = 0, greatest = 0;
    int rc0 = map_cuda(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (size_t k = 0; k < work.size() && !rc0; ++k) {
      const int prio = least - (int)std::min<size_t>(k, (size_t)(least - greatest));
      cudaStream_t &st = b->branches[work[k].second];
      if (st) cudaStreamDestroy(st);
      st = nullptr;
      rc0 = map_cuda(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio));
    }
    if (rc0) return rc0;
  }
  if (b->args_host.empty()) return DGPE_OK;
  int rc = DGPE_OK;
  for (const dgpe_batch::Group &g : b->groups)
    if (!rc) rc = map_cuda(b->ctxs[g.members[0]]->ks->init_group());
  if (!rc) rc = map_cuda(cudaMemcpyAsync(b->args_dev, b->args_host.data(), b->args_host.size() * sizeof(KArgs),
                                         cudaMemcpyHostToDevice, b->stream));
  // the host copy is read by the transfer: keep it unchanged until it has run
  if (!rc) rc = map_cuda(cudaStreamSynchronize(b->stream));
  return rc;
}

// Kernel nodes of one batch graph at most; a longer run launches several graphs.
constexpr long long kBatchMaxNodes = 1LL << 18;
constexpr size_t kBatchMaxGraphs = 4;   // cached step counts per batch

static void batch_drop_graphs(dgpe_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// The graph of `steps` steps of every context: a fork from the capture stream to one
// branch per context, each branch that context's step kernels `steps` times in a row, then
// one join.  The branches are independent chains, so a small grid's steps never wait for a
// large grid's; the GPU interleaves the chains' kernels.
static int batch_graph(dgpe_batch *b, int steps, cudaGraphExec_t *out) {
  bool stale = false;
  for (size_t i = 0; i < b->ctxs.size(); ++i) stale = stale || b->gens[i] != b->ctxs[i]->generation;
  if (stale || b->graphs.size() >= kBatchMaxGraphs) batch_drop_graphs(b);
  const auto it = b->graphs.find(steps);
  if (it != b->graphs.end()) {
    *out = it->second;
    return DGPE_OK;
  }
  if (b->graphs.empty()) {   // (re)building: the contexts' arguments may have changed
    const int grc = batch_group(b);
    if (grc) return grc;
  }
  const int n = (int)b->ctxs.size();
  std::vector<char> timing(n);
  for (int i = 0; i < n; ++i) {
    timing[i] = b->ctxs[i]->timing;
    b->ctxs[i]->timing = false;
  }
  int rc = map_cuda(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  if (!rc) rc = map_cuda(cudaEventRecord(b->events[n], b->cap));
  // a branch per group (its first member's stream and event) and per single context
  auto branch = [&](int i, auto &&enqueue) {
    if (!rc) rc = map_cuda(cudaStreamWaitEvent(b->branches[i], b->events[n], 0));
    for (int s = 0; s < steps && !rc; ++s) rc = enqueue(b->branches[i]);
    if (!rc) rc = map_cuda(cudaEventRecord(b->events[i], b->branches[i]));
    if (!rc) rc = map_cuda(cudaStreamWaitEvent(b->cap, b->events[i], 0));
  };
  for (const dgpe_batch::Group &g : b->groups) {
    const dgpe_ctx *c0 = b->ctxs[g.members[0]];
    const KArgs &a0 = c0->args;
    const int renorm = a0.imag ? kRenormUnit : (c0->restore_norm ? kRenormRestore : kRenormNone);
    branch(g.members[0], [&](cudaStream_t st) {
      return map_cuda(c0->ks->step_group(a0, b->args_dev + g.offset, (int)g.members.size(), renorm, st));
    });
  }
  for (int i : b->singles) branch(i, [&](cudaStream_t st) { return enqueue_step(b->ctxs[i], st); });
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  for (int i = 0; i < n; ++i) b->ctxs[i]->timing = timing[i];
  if (!rc) rc = map_cuda(e);
  cudaGraphExec_t exec = nullptr;
  if (!rc) rc = map_cuda(cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority));
  if (g) cudaGraphDestroy(g);
  if (rc) return rc;
  b->graphs[steps] = exec;
  for (int i = 0; i < n; ++i) b->gens[i] = b->ctxs[i]->generation;
  *out = exec;
  return DGPE_OK;
}

int dgpe_batch_step(dgpe_batch *b, int nsteps) {
  if (!b || nsteps < 0) return DGPE_EINVAL;
  if (nsteps == 0) return DGPE_OK;
  long long per_step = 0;   // kernel nodes of one step of every context
  for (dgpe_ctx *c : b->ctxs) per_step += 6 + c->ks->k5_launches;
  const int per_graph = (int)std::max<long long>(1, std::min<long long>(nsteps, kBatchMaxNodes / per_step));
  int rc = DGPE_OK;
  for (size_t i = 0; i < b->ctxs.size() && !rc; ++i) rc = wait_host_output(b->ctxs[i], b->stream);
  for (int done = 0; done < nsteps && !rc;) {
    const int k = std::min(per_graph, nsteps - done);
    cudaGraphExec_t exec = nullptr;
    rc = batch_graph(b, k, &exec);
    if (!rc) rc = map_cuda(cudaGraphLaunch(exec, b->stream));
    done += k;
  }
  return rc;
}

int dgpe_batch_sync(dgpe_batch *b) {
  if (!b) return DGPE_EINVAL;
  int rc = map_cuda(cudaStreamSynchronize(b->stream));
  for (size_t i = 0; i < b->ctxs.size() && !rc; ++i) rc = check_device_flags(b->ctxs[i]);
  return rc;
}

void dgpe_batch_destroy(dgpe_batch *b) {
  if (!b) return;
  if (b->stream || b->cap) cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  if (b->args_dev) cudaFree(b->args_dev);
  for (cudaEvent_t e : b->events)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : b->branches)
    if (st) cudaStreamDestroy(st);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

int dgpe_sync(dgpe_ctx *c) {
  if (!c) return DGPE_EINVAL;
  int rc = map_cuda(cudaStreamSynchronize(c->stream));
  if (!rc && c->host_io) rc = map_cuda(cudaStreamSynchronize(c->cs_in));
  if (!rc && c->host_io) rc = map_cuda(cudaStreamSynchronize(c->cs_out));
  if (rc) return rc;
  return check_device_flags(c);
}

namespace {
// The second psi buffer, staging, streams and events of dgpe_step_host, created at its
// first call.
int host_io_setup(dgpe_ctx *c) {
  if (c->host_io) return DGPE_OK;
  const size_t bytes = (size_t)c->p.nx * c->p.ny * c->p.nz * c->ks->elem_bytes;
  // a failed earlier attempt keeps what it created (dgpe_destroy frees it); create the rest
  int rc = DGPE_OK;
  if (!c->psi_alt) rc = map_cuda(cudaMalloc(&c->psi_alt, bytes));
  if (!rc && c->p.precision == DGPE_DF64 && !c->stage_out) rc = map_cuda(cudaMalloc(&c->stage_out, bytes));
  if (!rc && !c->cs_in) rc = map_cuda(cudaStreamCreateWithFlags(&c->cs_in, cudaStreamNonBlocking));
  if (!rc && !c->cs_out) rc = map_cuda(cudaStreamCreateWithFlags(&c->cs_out, cudaStreamNonBlocking));
  cudaEvent_t *ev[7] = {&c->ev_in_ready,    &c->ev_out_ready,   &c->ev_stage_free, &c->ev_main_done[0],
                        &c->ev_main_done[1], &c->ev_d2h_done[0], &c->ev_d2h_done[1]};
  for (int q = 0; q < 7 && !rc; ++q)
    if (!*ev[q]) rc = map_cuda(cudaEventCreateWithFlags(ev[q], cudaEventDisableTiming));
  if (rc) return rc;
  c->host_io = true;
  return DGPE_OK;
}
}  // namespace

// Successive calls alternate between the workspace's psi buffer and a second one: the input
// of a call is copied into the buffer that does not hold the current state while the steps
// of the previous call still run, and its result is copied out of it while the next call's
// steps run, with no device-side copy.  A buffer is written again once the main stream has
// left it (ev_main_done, recorded where the state moves to the other buffer) and its
// previous output copy has finished (ev_d2h_done).  Double-float converts its input in place
// and its output through a staging buffer (the state itself stays in pairs).
int dgpe_step_host(dgpe_ctx *c, const void *in, void *out, int nsteps) {
  if (!c || !in || !out || nsteps < 0) return DGPE_EINVAL;
  int rc = host_io_setup(c);
  if (rc) return rc;
  const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz;
  const size_t bytes = n * c->ks->elem_bytes;
  const int cur = on_alt_psi(c) ? 1 : 0, tgt = 1 - cur;
  void *const buf[2] = {c->psi_main, c->psi_alt};
  // host -> the free buffer on the input copy stream
  rc = map_cuda(cudaStreamWaitEvent(c->cs_in, c->ev_main_done[tgt], 0));
  if (!rc) rc = map_cuda(cudaStreamWaitEvent(c->cs_in, c->ev_d2h_done[tgt], 0));
  if (!rc) rc = map_cuda(cudaMemcpyAsync(buf[tgt], in, bytes, cudaMemcpyHostToDevice, c->cs_in));
  if (!rc) rc = map_cuda(cudaEventRecord(c->ev_in_ready, c->cs_in));
  // the state moves to that buffer: from here on the main stream leaves the other one alone
  if (!rc) rc = map_cuda(cudaStreamWaitEvent(c->stream, c->ev_in_ready, 0));
  if (!rc) rc = map_cuda(cudaEventRecord(c->ev_main_done[cur], c->stream));
  if (rc) return rc;
  c->args.psi = buf[tgt];
  ++c->generation;   // batches holding this context capture its new buffer
  if (c->p.precision == DGPE_DF64) rc = map_cuda(c->ks->from_c128(buf[tgt], buf[tgt], n, c->stream));
  if (!rc) rc = map_cuda(c->ks->reset_state(c->args.state, c->stream));
  if (rc) return rc;
  c->latched = DGPE_OK;
  rc = dgpe_step(c, nsteps);
  if (rc) return rc;
  // the pending scale (imaginary time; real time where the mixed path restores the norm:
  // FP64 and double-float real-time steps leave s = 1)
  if (c->p.mode == DGPE_IMAG_TIME || c->restore_norm)
    rc = launch(c, c->stream, kKMaterialize, [&] { return c->ks->materialize(c->args, c->stream); });
  const void *src = buf[tgt];
  if (!rc && c->p.precision == DGPE_DF64) {
    // pairs -> complex128 into the staging, once the previous output copy has left it
    rc = map_cuda(cudaStreamWaitEvent(c->stream, c->ev_stage_free, 0));
    if (!rc) rc = map_cuda(c->ks->to_c128(buf[tgt], c->stage_out, n, c->stream));
    src = c->stage_out;
  }
  if (!rc) rc = map_cuda(cudaEventRecord(c->ev_out_ready, c->stream));
  // the result -> host on the output copy stream
  if (!rc) rc = map_cuda(cudaStreamWaitEvent(c->cs_out, c->ev_out_ready, 0));
  if (!rc) rc = map_cuda(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, c->cs_out));
  if (!rc) rc = map_cuda(cudaEventRecord(c->ev_d2h_done[tgt], c->cs_out));
  if (!rc && c->p.precision == DGPE_DF64) rc = map_cuda(cudaEventRecord(c->ev_stage_free, c->cs_out));
  return rc;
}

int dgpe_set_timing(dgpe_ctx *c, int enable) {
  if (!c) return DGPE_EINVAL;
  c->timing = enable != 0;
  return DGPE_OK;
}

int dgpe_kernel_times(dgpe_ctx *c, dgpe_kernel_time *out, int max, int *n) {
  if (!c || (!out && max > 0) || !n) return DGPE_EINVAL;
  int rc = map_cuda(cudaStreamSynchronize(c->stream));
  if (rc) return rc;
  for (const auto &pd : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pd.a, pd.b) == cudaSuccess) {
      c->total_ms[pd.kernel] += ms;
      c->launches[pd.kernel] += 1;
    }
    c->ev_free.push_back(pd.a);
    c->ev_free.push_back(pd.b);
  }
  c->pending.clear();
  int k = 0;
  for (int q = 0; q < kNumKernels; ++q) {
    if (c->launches[q] == 0) continue;
    if (k < max) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kKernelNames[q], sizeof(out[k].name) - 1);
      out[k].total_ms = c->total_ms[q];
      out[k].launches = c->launches[q];
      out[k].bytes_per_launch = kernel_bytes(c, q);
    }
    ++k;
    c->total_ms[q] = 0;
    c->launches[q] = 0;
  }
  *n = k;
  return DGPE_OK;
}

void dgpe_destroy(dgpe_ctx *c) {
  if (!c) return;
  if (c->ws) cudaStreamSynchronize(c->stream);
  if (c->cs_in) cudaStreamSynchronize(c->cs_in);
  if (c->cs_out) cudaStreamSynchronize(c->cs_out);
  for (cudaEvent_t e : {c->ev_in_ready, c->ev_out_ready, c->ev_stage_free, c->ev_main_done[0], c->ev_main_done[1],
                        c->ev_d2h_done[0], c->ev_d2h_done[1]})
    if (e) cudaEventDestroy(e);
  if (c->cs_in) cudaStreamDestroy(c->cs_in);
  if (c->cs_out) cudaStreamDestroy(c->cs_out);
  if (c->psi_alt) cudaFree(c->psi_alt);
  if (c->stage_out) cudaFree(c->stage_out);
  if (c->graph_alt) cudaGraphExecDestroy(c->graph_alt);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (const auto &pd : c->pending) {
    cudaEventDestroy(pd.a);
    cudaEventDestroy(pd.b);
  }
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
