// dgpe_moments_noalloc: the norm and rms sizes of a caller's psi, computed without any
// device allocation.  The scratch memory of its reduction (per-block partial sums and the
// last-block counter) is a file-scope __device__ array of fixed size, so the call needs
// neither a context nor a workspace.  The paper has no counterpart of this entry point.
//
// Scratch: kNoAllocMaxBlocks x 4 doubles of partial sums + one counter, 256 KiB in all (the
// grid is capped at kNoAllocMaxBlocks blocks whatever the size).
// Every GPU that loads libdgpe.so holds one copy of it until the process exits, and every
// call on that GPU shares it: calls whose work overlaps on the GPU (different streams
// without ordering between them) race on it and give wrong results.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "dgpe.h"
#include "dgpe_device.cuh"

using namespace dgpe;

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 8192;
constexpr int kNoAllocMaxN = 512;   // points per axis (the library's grid limit)

struct NoAllocScratch {
  unsigned int ticket;            // last-block counter: must be 0 when a reduction starts
  unsigned int pad[63];
  double partials[kNoAllocMaxBlocks * 4];
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of this GPU's copy of the scratch array, looked up once per device with
// that device current (in host code the symbol itself is only a host-side stand-in).
int scratch_address(NoAllocScratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DGPE_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DGPE_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<NoAllocScratch *>(g_scratch_addr[dev]);
  return DGPE_OK;
}

// Sums n, x^2 n, y^2 n, z^2 n (FP64, weighted by the quadrature rule) with one warp per
// z-line at a time (grid-stride over the nx*ny lines): the line's (i, j) costs one division
// per line, the z weights come from a shared table.  The last block turns the sums into
// norm = hx hy hz sum w n and rms_d = sqrt(sum w d^2 n / sum w n).
template <typename R>
__global__ void __launch_bounds__(kNoAllocThreads)
    k_moments_noalloc(const cplx<R> *__restrict__ psi, int nx, int ny, int nz, double hx, double hy, double hz,
                      int simpson, NoAllocScratch *scr, double *out) {
  __shared__ double wz[kNoAllocMaxN], wz2[kNoAllocMaxN];   // w_k and w_k z_k^2
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const double z = coordinate(k, nz, hz), w = quad_weight(k, nz, simpson);
    wz[k] = w;
    wz2[k] = w * z * z;
  }
  __syncthreads();
  const int lane = threadIdx.x & (kWarp - 1);
  const long long nlines = (long long)nx * ny;
  const long long nwarps = (long long)gridDim.x * (blockDim.x / kWarp);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long l = (long long)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp; l < nlines; l += nwarps) {
    const int i = (int)(l / ny), j = (int)(l - (long long)i * ny);
    const cplx<R> *line = psi + l * nz;
    double s0 = 0.0, sz = 0.0;
    for (int k = lane; k < nz; k += kWarp) {
      const cplx<R> w = line[k];
      const double d = (double)w.re * w.re + (double)w.im * w.im;
      s0 = fma(wz[k], d, s0);
      sz = fma(wz2[k], d, sz);
    }
    const double x = coordinate(i, nx, hx), y = coordinate(j, ny, hy);
    const double t = quad_weight(i, nx, simpson) * quad_weight(j, ny, simpson) * s0;
    v[0] += t;
    v[1] += x * x * t;
    v[2] += y * y * t;
    v[3] += quad_weight(i, nx, simpson) * quad_weight(j, ny, simpson) * sz;
  }
  if (reduce_across_blocks<4>(v, scr->partials, &scr->ticket) && threadIdx.x == 0) {
    out[0] = hx * hy * hz * v[0];
    out[1] = sqrt(v[1] / v[0]);
    out[2] = sqrt(v[2] / v[0]);
    out[3] = sqrt(v[3] / v[0]);
  }
}

}  // namespace

extern "C" int dgpe_moments_noalloc(const void *psi, const dgpe_params *p, double *out, void *cuda_stream) {
  if (!psi || !p || !out) return DGPE_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return DGPE_EINVAL;
  if (!(p->hx > 0 && p->hy > 0 && p->hz > 0) || !isfinite(p->hx) || !isfinite(p->hy) || !isfinite(p->hz))
    return DGPE_EINVAL;
  if (p->precision != DGPE_FP64 && p->precision != DGPE_MIXED && p->precision != DGPE_DF64) return DGPE_EINVAL;
  if (p->integration != DGPE_RECTANGLE && p->integration != DGPE_SIMPSON) return DGPE_EINVAL;
  if (p->nx > kNoAllocMaxN || p->ny > kNoAllocMaxN || p->nz > kNoAllocMaxN) return DGPE_EUNSUPPORTED;
  NoAllocScratch *scr = nullptr;
  int rc = scratch_address(&scr);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the counter must start at zero (a reduction that was cut short may have left it set)
  if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return DGPE_ECUDA;
  const long long nlines = (long long)p->nx * p->ny;
  const long long warps_per_block = kNoAllocThreads / kWarp;
  const unsigned blocks = (unsigned)std::min<long long>((nlines + warps_per_block - 1) / warps_per_block,
                                                        kNoAllocMaxBlocks);
  const int simpson = p->integration == DGPE_SIMPSON;
  if (p->precision != DGPE_MIXED)   // complex128 (FP64, and the double-float mode's caller format)
    k_moments_noalloc<double><<<blocks, kNoAllocThreads, 0, st>>>(static_cast<const cplx<double> *>(psi), p->nx,
                                                                  p->ny, p->nz, p->hx, p->hy, p->hz, simpson,
                                                                  scr, out);
  else
    k_moments_noalloc<float><<<blocks, kNoAllocThreads, 0, st>>>(static_cast<const cplx<float> *>(psi), p->nx,
                                                                 p->ny, p->nz, p->hx, p->hy, p->hz, simpson,
                                                                 scr, out);
  return cudaGetLastError() == cudaSuccess ? DGPE_OK : DGPE_ECUDA;
}
