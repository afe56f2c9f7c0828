// Far-field pattern without any device allocation (igabem_farfield_noalloc).
//
// igabem_farfield stages its inputs and its per-Gauss-point scratch in memory that the library
// allocates on demand.  Some callers cannot let a library allocate: a host program whose own caching
// allocator has reserved the device memory (a raw cudaMalloc then fails or fragments its pool), or
// a serving loop that must not stall on the implicit device synchronisation of cudaMalloc/cudaFree.
// This file gives them the same computation with a fixed scratch area: a file-scope device array
// that the CUDA module holds from its load until the process exits, on every device that loads the
// library.  The caller passes device-resident inputs and outputs; nothing here calls cudaMalloc,
// cudaFree or any allocating routine.
#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"
#include "k_common.cuh"

// Scratch of the allocation-free far field: 2^21 complex doubles (32 MiB), one weighted density value
// per (element, Gauss point, right-hand side).  Host code must not use this name as an address; it
// asks the runtime for the device address (see noalloc_scratch below).
static constexpr size_t kNoallocScratchComplex = size_t(1) << 21;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchComplex];

namespace igabem {

namespace {

// density at the Gauss points weighted by w_q h^2 (same sum as the allocating path), written to rho
__global__ void k_density_noalloc(const int *__restrict__ x2g, const double *__restrict__ phi1,
                                  const double *__restrict__ gw, const double2 *__restrict__ x, long E,
                                  int n1, int nb, int p, int ng, int R, double h, double2 *__restrict__ rho) {
  const int p1 = p + 1, nq = ng * ng;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < E * nq * R; o += (long)gridDim.x * blockDim.x) {
    long e = o / (nq * R);
    int q = int((o / R) % nq), r = int(o % R), q1 = q / ng, q2 = q % ng;
    int j = int(e / ((long)n1 * n1)), ix = int((e / n1) % n1), iy = int(e % n1);
    double2 acc = cmk(0, 0);
    for (int ka = 0; ka < p1; ++ka)
      for (int kb = 0; kb < p1; ++kb) {
        long X = ((long)j * nb + ix + ka) * nb + iy + kb;
        double w = phi1[(ix * ng + q1) * p1 + ka] * phi1[(iy * ng + q2) * p1 + kb];
        acc = cadd(acc, cscale(x[(long)x2g[X] * R + r], w));
      }
    rho[o] = cscale(acc, gw[q1] * gw[q2] * h * h);
  }
}

// u_inf[k][r] = sum over Gauss points of rho exp(-i kappa x^_k . x) times -a/(4 pi) (sound-soft) or
// -i kappa (x^_k . n~)/(4 pi) (sound-hard); one block per (direction, right-hand side)
__global__ void k_farfield_noalloc(const double *__restrict__ gpx, const double *__restrict__ gpn,
                                   const double *__restrict__ gpa, long gst, const double2 *__restrict__ rho,
                                   int R, double kappa, bool hard, const double *__restrict__ xhat,
                                   double2 *__restrict__ uinf) {
  __shared__ double2 red[256];
  const int k = blockIdx.x, r = blockIdx.y;
  const double *xh = xhat + 3 * k;
  double2 acc = cmk(0, 0);
  for (long i = threadIdx.x; i < gst; i += blockDim.x) {
    double s, c;
    sincos(-kappa * (xh[0] * gpx[i] + xh[1] * gpx[gst + i] + xh[2] * gpx[2 * gst + i]), &s, &c);
    double2 v = cmul(rho[i * R + r], cmk(c, s));
    if (hard) {
      double xn = xh[0] * gpn[i] + xh[1] * gpn[gst + i] + xh[2] * gpn[2 * gst + i];
      v = cmul(v, cmk(0.0, -kappa * xn));
    } else {
      v = cscale(v, -gpa[i]);
    }
    acc = cadd(acc, v);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) uinf[(long)k * gridDim.y + r] = cscale(red[0], 0.25 / IGA_PI);
}

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_noalloc_mu;
double2 *g_noalloc_ptr[128] = {};

int noalloc_scratch(int device, double2 **out) {
  if (device < 0 || device >= 128) {
    set_error("device ordinal out of range for the allocation-free far field");
    return IGABEM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("cudaGetSymbolAddress of the far-field scratch failed: ") + cudaGetErrorString(e));
      return IGABEM_ECUDA;
    }
    g_noalloc_ptr[device] = static_cast<double2 *>(ptr);
  }
  *out = g_noalloc_ptr[device];
  return IGABEM_OK;
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace igabem

extern "C" int igabem_farfield_noalloc(igabem_problem *P, int n_rhs, const void *density, int n_dir,
                                       const double *xhat, void *uinf) {
  using namespace igabem;
  set_error("");
  if (!P || !density || !xhat || !uinf || n_rhs <= 0 || n_dir <= 0) {
    set_error("invalid arguments to igabem_farfield_noalloc");
    return IGABEM_EINVAL;
  }
  const HostSetup &S = P->S;
  const long gst = (long)S.E * S.ng * S.ng;
  if ((size_t)gst * (size_t)n_rhs > kNoallocScratchComplex) {
    set_error("igabem_farfield_noalloc: n_elements * gauss_regular^2 * n_rhs = " +
              std::to_string(gst * (long)n_rhs) + " exceeds the fixed scratch of " +
              std::to_string(kNoallocScratchComplex) + " values (32 MiB); use igabem_farfield");
    return IGABEM_EINVAL;
  }
  const int dev = P->geom->ctx->device;
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return IGABEM_ECUDA;
  }
  if (!on_device(density) || !on_device(xhat) || !on_device(uinf)) {
    set_error("igabem_farfield_noalloc: density, xhat and uinf must be device memory of the context's device");
    return IGABEM_EINVAL;
  }
  double2 *rho = nullptr;
  int rc = noalloc_scratch(dev, &rho);
  if (rc != IGABEM_OK) return rc;
  cudaStream_t st = P->geom->ctx->stream;
  const DeviceProblem &d = P->d;
  long tot = gst * n_rhs;
  int grid = (int)std::max<long>(1, std::min<long>((tot + 255) / 256, 152L * 32));
  // every scratch entry that k_farfield_noalloc reads is written first by k_density_noalloc, so the
  // contents left by an earlier call never need clearing
  k_density_noalloc<<<grid, 256, 0, st>>>(d.x2g, d.phi1, d.gw, static_cast<const double2 *>(density), S.E,
                                          S.n1, S.nb, S.p, S.ng, n_rhs, S.h, rho);
  dim3 g2(n_dir, n_rhs);
  k_farfield_noalloc<<<g2, 256, 0, st>>>(d.gpx, d.gpn, d.gpa, gst, rho, n_rhs, P->opt.kappa, S.hard, xhat,
                                         static_cast<double2 *>(uinf));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("igabem_farfield_noalloc: ") + cudaGetErrorString(e));
    return IGABEM_ECUDA;
  }
  return IGABEM_OK;
}
