// Internal interface between the C-ABI host code (dgpe_api.cu) and the kernel translation
// units (kernels_f64.cu, kernels_f32.cu).  Plain structs only; no CUDA device code here.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace dgpe {

constexpr int kMaxStages = 12;
constexpr int kWarp = 32;
constexpr int kCnMaxChunk = 16;   // interior points per lane of the chunked Thomas solve

// Mixed-radix plan of one transform length: n = radix[0] * radix[1] * ...
// Twiddles are stored per stage: stage s (radix P, ns = product of the earlier radices)
// keeps e^{-2 pi i r k / (ns P)} for k < ns, r = 1..P-1 at twoff[s] + k (P - 1) + r - 1;
// the stages together hold n - 1 entries.
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int twoff[kMaxStages];
};

// Crank-Nicolson factor tables of one direction (interior size m = n - 2, chunk length c):
// four arrays [alpha | beta | H | G] of 32*c coefficients each (complex in real time,
// real in imaginary time, in the kernel precision), lane-interleaved: the entry of interior
// point t*c + e sits at e*32 + t, so the 32 lanes of a warp read one contiguous segment;
// then 10 x 32 scan factors of the lane carries (5 forward steps, 5 backward), then
// 1/gamma, the pivot of the twist point m/2 of the FP64 two-thread sweeps.
// Factor tables to build in one launch (one block each): the three axes, forward and (real
// time) the dt -> -dt tables of the adjoint sweeps.
struct CnJob {
  void *tab;
  int m, chunk;
  double r;    // dt / (4 h^2), negated for the adjoint tables
  int lanes;   // lanes per line of the layout: 32, or 8 (the short-line sweeps)
};
constexpr int kMaxCnJobs = 12;

// FP32 sweeps of short lines: n = 8 CH points (CH = 4, 6, 8, 12 or 16) are solved on 8 lanes
// per line, CH points each; 0 where the line takes the 32-lane solver.
__host__ __device__ constexpr int short_cn_chunk(int n) {
  return (n == 32 || n == 48 || n == 64 || n == 96 || n == 128) ? n / 8 : 0;
}
// FP32 compile-time K5 lengths whose z solve runs on 8 lanes per line (8-lane z tables)
__host__ __device__ constexpr bool k5_short_z(int n) { return n == 64 || n == 96 || n == 128; }

// Interior points per lane of K5's z solve at a compile-time length n: the least chunk with
// 32 chunks covering the n - 2 unknowns (12 for n = 384; the sweeps' power of two for 128,
// 256, 512), so that the line pads to 32 whole chunks with at most a few padded unknowns.
__host__ __device__ constexpr int k5_chunk(int n) { return (n - 2 + 31) / 32; }
struct CnJobs {
  CnJob job[kMaxCnJobs];
  int n;
  int imag;   // the same for every job of a call
};

struct CnTab {
  const void *tab;
  int m;
  int chunk;    // interior points per lane, a power of two
  int lchunk;   // log2(chunk)
};

// Device-resident solver state (lives in the workspace).
struct DevState {
  double s;          // pending renormalisation factor: the state is s * psi_buf
  float sf, s2f;     // s and s^2 rounded to FP32 (read by the FP32 kernels)
  float sl, s2l;     // the FP32 remainders: (sf, sl) and (s2f, s2l) are double-float pairs
  double norm;       // hx hy hz sum |psi_buf|^2 after the last full step
  double norm_in;    // the true norm (s^2 norm) of the state the next step starts from; 0: unknown
  double norm_ref;   // the norm real-time steps restore (FP32-mixed); 0: not yet taken
  double sums[8];    // last reduction (step: n, 0 (x^2 n is not summed), y^2 n, z^2 n; obs: 8 terms)
  double obs[12];    // observables of the last dgpe_observables call
  double grads[4];      // adjoint accumulators: dL/dg, dL/dgdd, dL/dnu_z
  unsigned int flags;   // bit 0: non-finite norm
  unsigned int ticket;  // last-block-done counter of the fused reductions
  unsigned long long steps;
};
constexpr unsigned kFlagNonFinite = 1u;

// Everything a kernel needs, passed by value.
struct KArgs {
  int nx, ny, nz, nzh;         // nzh = nz/2 + 1 (half-spectrum length along z)
  double hx, hy, hz;
  double dt, g, gdd;
  double cutoff;               // spherical cutoff radius of the dipolar kernel (<= 0: none)
  int has_cutoff;              // cutoff > 0
  float cutoff_f;
  int simpson;                 // 1: composite Simpson weights in the norm and observables
  int kinetic5;                // 1: kinetic energy from the 5-point gradient
  double vx, vy, vz;           // 0.5 * nu_d^2
  double inv_ntot;             // 1 / (nx ny nz)
  float inv_ntot_f, inv_ntot_l;   // FP32 rounding and remainder (the double-float pair)
  int imag;                    // 1 = imaginary time
  double cn_r[3];              // dt / (4 h_d^2), the Crank-Nicolson coefficient magnitude
  float cn_rf[3], cn_rl[3];
  double dtg, dtgdd_n;         // dt g and dt gdd / (nx ny nz) (Phi's 1/N folded in)
  float dtg_f, dtgdd_n_f, dtg_l, dtgdd_n_l;
  const void *dtv[3];          // dt v_d x_i^2 per axis (kernel precision)
  void *psi;                   // [nx][ny][nz] complex
  void *spec;                  // [nzh][nx][ny] complex, the z-half-spectrum-major layout
  const void *utab;            // Ut(k) (times the cutoff factor) on [nzh][nx][ny], FP64 only
  void *ybuf;                  // [point][line] forward-elimination scratch of the FP64
                               // one-thread-per-line sweeps (nx ny nz complex values)
  float kf[3];                 // 2 pi / (n_d h_d): wavenumber per frequency index (FP32 K3)
  DevState *state;
  double *partials;            // per-block reduction partials
  const void *tw[3];           // per-stage twiddle tables of plan[d] (layout in FftPlan), d = x, y, z
  FftPlan plan[3];
  CnTab cn[3];
  const void *cnz_tab;         // K5's z tables at k5_chunk(nz) points per lane, where that is not
                               // cn[2].chunk (FP32, compile-time nz); else null
  const void *cn8_tab[3];      // tables in the 8-lane layout: the x and y sweeps' (FP32 lines of
                               // short_cn_chunk(n) != 0) and K5's z solve (FP32, k5_short_z(nz)); else null
  void *out;                   // optional output (Phi for get_phi)
  // adjoint step
  void *gbar;                  // cotangent field (same layout as psi)
  double dt_nuz;               // dt * nu_z (the nu_z derivative of theta is dt nu_z z^2)
  double *grad_nu_slot;        // optional extra accumulator of dL/dnu_z (schedule segment)
  int unit_scale;              // K1: ignore the pending renormalisation (s = 1)
  // launch shapes (defaults set at create; dgpe_autotune may change them)
  int ylines;                  // K2/K4 lines per CTA (power of two, <= 32)
  int fft_threads;             // K2/K3/K4 threads per CTA (128 or 256)
  int cn_per_sm;               // K6/K7 persistent CTAs per SM (1 or 2; capped by shared memory)
  int nsm;                     // SMs of the device: the FP32 tile kernels prefetch into L2 the tile of
                               // the CTA one resident wave ahead (residency x nsm; 0: no prefetch)
};

// Modes of the z-line kernel (C2R along z + potential step + CN along z).
// What the x sweep's last block does with the norm it sums (see finish_sweep_sums).
enum RenormMode : int { kRenormNone = 0, kRenormUnit = 1, kRenormRestore = 2 };

enum ZMode : int {
  kZStep = 0,        // phase, then CN-z
  kZPhaseOnly = 1,   // phase only
  kZCnOnly = 2,      // CN-z only (no transform)
  kZPhi = 3,         // write Phi to args.out
  kZObs = 4,         // observables reduction
};

// Kernel identifiers (timing records, launch table).
enum KernelId : int {
  kK1DensityR2Cz = 0,
  kK2FftY,
  kK3FftXDipolar,
  kK4IfftY,
  kK5C2RzPhaseCnz,
  kK6CnY,
  kK7CnXReduce,
  kKMaterialize,
  kKObs,
  kKAdjPhase,
  kKAdjCombine,
  kNumKernels
};

// Host-side launchers of one precision (implemented in kernels_f64.cu / kernels_f32.cu).
struct KernelSet {
  int elem_bytes;  // sizeof complex element
  cudaError_t (*init)();
  cudaError_t (*twiddles)(void *tw, const FftPlan &pl, cudaStream_t st);
  cudaError_t (*cn_tables)(const CnJobs &jobs, cudaStream_t st);
  cudaError_t (*axis_potential)(void *out, int n, double h, double v, double dt, cudaStream_t st);
  cudaError_t (*dipolar_table)(const KArgs &a, cudaStream_t st);   // fills utab
  // double-float only: complex128 -> the kernels' pairs (in place allowed), and back with the
  // pending renormalisation applied
  cudaError_t (*from_c128)(const void *src, void *psi, size_t n, cudaStream_t st);
  cudaError_t (*to_c128)(const void *psi, void *dst, size_t n, cudaStream_t st);
  cudaError_t (*reset_state)(DevState *st_ptr, cudaStream_t st);
  cudaError_t (*k1)(const KArgs &a, cudaStream_t st);
  cudaError_t (*k2)(const KArgs &a, cudaStream_t st);   // forward FFT along y
  cudaError_t (*k3)(const KArgs &a, cudaStream_t st);   // FFT-x, x Ut, IFFT-x
  cudaError_t (*k4)(const KArgs &a, cudaStream_t st);   // inverse FFT along y
  cudaError_t (*k5)(const KArgs &a, int zmode, cudaStream_t st);
  cudaError_t (*k6)(const KArgs &a, cudaStream_t st);   // CN-y
  cudaError_t (*k7)(const KArgs &a, int reduce, int renorm, cudaStream_t st);  // CN-x
  cudaError_t (*materialize)(const KArgs &a, cudaStream_t st);
  cudaError_t (*adj_phase)(const KArgs &a, cudaStream_t st);     // u = e^{i theta} gbar, s, R2C(s)
  cudaError_t (*adj_combine)(const KArgs &a, cudaStream_t st);   // gbar = u + 2 dt (g s + gdd Phi[s]) psi
  cudaError_t (*loss_z2)(const KArgs &a, cudaStream_t st);       // gbar = 2 h^3 z^2 psi
  int (*max_blocks)(const KArgs &a);   // upper bound on blocks of any reducing kernel
  int k5_launches;                     // kernels behind one k5 step call (1 fused, or 2)
  int (*default_ylines)(int ny);
  size_t (*y_smem)(int ny, int ylines);
  // one step of a group of same-shaped condensates, each kernel launched once for all of
  // them (ga: their arguments in device memory; a: one member's); null where the precision
  // has no grouped kernels (FP64, double-float)
  cudaError_t (*init_group)();
  cudaError_t (*step_group)(const KArgs &a, const KArgs *ga, int n, int renorm, cudaStream_t st);
};

cudaError_t group_init_f32();
cudaError_t group_step_f32(const KArgs &a, const KArgs *ga, int n, int renorm, cudaStream_t st);

const KernelSet *kernels_f64();
const KernelSet *kernels_f32();
const KernelSet *kernels_df64();

}  // namespace dgpe
