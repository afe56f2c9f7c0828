// Far-field pattern without any device allocation (igabem_farfield_noalloc).
//
// igabem_farfield stages its inputs and its per-Gauss-point scratch in memory that the library
// allocates on demand.  Some callers cannot let a library allocate: a host program whose own caching
// allocator has reserved the device memory (a raw cudaMalloc then fails or fragments its pool), or
// a serving loop that must not stall on the implicit device synchronisation of cudaMalloc/cudaFree.
// This file gives them the same computation -- the same kernels as igabem_farfield, through
// launch_farfield -- with a fixed scratch area: a file-scope device array that the CUDA module holds
// from its load until the process exits, on every device that loads the library.  The caller passes
// device-resident inputs and outputs; nothing here calls cudaMalloc, cudaFree or any allocating
// routine.
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.h"

// Scratch of the allocation-free far field: 2^21 complex doubles (32 MiB), one weighted density value
// per (element, Gauss point, right-hand side).  Host code must not use this name as an address; it
// asks the runtime for the device address (see noalloc_scratch below).
static constexpr size_t kNoallocScratchComplex = size_t(1) << 21;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchComplex];

namespace igabem {

namespace {

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_noalloc_mu;
double2 *g_noalloc_ptr[128] = {};

double2 *noalloc_scratch(int device) {
  if (device < 0 || device >= 128) fail(IGABEM_EINVAL, "device ordinal out of range for the allocation-free far field");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(IGABEM_ECUDA, std::string("cudaGetSymbolAddress of the far-field scratch failed: ") + cudaGetErrorString(e));
    }
    g_noalloc_ptr[device] = static_cast<double2 *>(ptr);
  }
  return g_noalloc_ptr[device];
}

// true for memory the kernels on `device` can read and write in place: device memory of that device
// (not of another GPU), or managed memory
bool on_device(const void *p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

}  // namespace igabem

extern "C" int igabem_farfield_noalloc(igabem_problem *P, int n_rhs, const void *density, int n_dir,
                                       const double *xhat, void *uinf) {
  using namespace igabem;
  return run_guarded([&] {
    if (!P || !density || !xhat || !uinf || n_rhs <= 0 || n_dir <= 0)
      fail(IGABEM_EINVAL, "invalid arguments to igabem_farfield_noalloc");
    // the far-field kernel runs one thread block per (direction, right-hand side), the right-hand sides
    // along the grid's y dimension
    if (n_rhs > 65535) fail(IGABEM_EINVAL, "igabem_farfield_noalloc: at most 65535 right-hand sides per call");
    const HostSetup &S = P->S;
    const long gst = (long)S.E * S.ng * S.ng;
    if ((size_t)gst * (size_t)n_rhs > kNoallocScratchComplex)
      fail(IGABEM_EINVAL, "igabem_farfield_noalloc: n_elements * gauss_regular^2 * n_rhs = " +
                              std::to_string(gst * (long)n_rhs) + " exceeds the fixed scratch of " +
                              std::to_string(kNoallocScratchComplex) + " values (32 MiB); use igabem_farfield");
    const int dev = P->geom->ctx->device;
    IGA_CUDA(cudaSetDevice(dev));
    if (!on_device(density, dev) || !on_device(xhat, dev) || !on_device(uinf, dev))
      fail(IGABEM_EINVAL, "igabem_farfield_noalloc: density, xhat and uinf must be device memory of the context's "
                          "device (host memory and other GPUs' memory are refused)");
    double2 *rho = noalloc_scratch(dev);
    cudaStream_t st = P->stream;
    // every scratch entry that the far-field kernel reads is written first by the density kernel, so
    // the contents left by an earlier call never need clearing
    launch_farfield(P->d, S, P->opt, n_rhs, static_cast<const double *>(density), n_dir, xhat,
                    static_cast<double *>(uinf), reinterpret_cast<double *>(rho), st);
    IGA_CUDA(cudaStreamSynchronize(st));
    P->prof.flush();
  });
}
