// dds_stress_noalloc: a stress evaluation that allocates no device memory.
//
// Its work buffers (the intermediate spectra between the five passes) live in one
// file-scope device array of DDS_NOALLOC_SCRATCH_BYTES instead of buffers the
// context allocated.  Host code cannot use the array's name as a device address,
// so the address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.  The look-up happens in
// dds_build_kernels (noalloc_prepare), a set-up step: under lazy module loading it is
// the look-up that places this file's module, and with it the array, on the device,
// so no call of dds_stress_noalloc is the one that allocates it.
#include <algorithm>
#include <mutex>

#include "dds_internal.h"

namespace dds {
namespace {

constexpr size_t SCRATCH_ELEMS = (size_t)DDS_NOALLOC_SCRATCH_BYTES / sizeof(float2);

// Shared by every call on a device; each GPU that loads the library holds it until exit.
static __device__ __align__(256) float2 g_scratch[SCRATCH_ELEMS];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
float2 *g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_scratch on device `dev`, which must be current; looked up on
// the first request for that device.
cudaError_t scratch_address(int dev, float2 **out) {
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_addr[dev] = static_cast<float2 *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t round256(size_t elems) {   // float2 elements, rounded up to 256 bytes
  return (elems + 31) / 32 * 32;
}

}  // namespace

// Called by dds_build_kernels with the context's device current.
cudaError_t noalloc_prepare(int dev) {
  if (dev < 0 || dev >= MAX_DEVICES) return cudaSuccess;   // dds_stress_noalloc refuses such devices
  float2 *p = nullptr;
  return scratch_address(dev, &p);
}

}  // namespace dds

using namespace dds;

extern "C" int dds_stress_noalloc(dds_ctx *ctx, const void *rho, int rho_dtype, float *sigma,
                                  void *cuda_stream) {
  if (!ctx) return DDS_ERR_INVALID_ARG;
  if (!ctx->built) return fail(ctx, DDS_ERR_NOT_READY, "stress_noalloc: call dds_build_kernels first");
  if (!rho || !sigma) return fail(ctx, DDS_ERR_INVALID_ARG, "stress_noalloc: NULL pointer");
  if (rho_dtype != DDS_F32 && rho_dtype != DDS_BF16)
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_noalloc: unknown density type %d", rho_dtype);
  if (((uintptr_t)rho & 15) || ((uintptr_t)sigma & 15))
    return fail(ctx, DDS_ERR_INVALID_ARG, "stress_noalloc: rho and sigma must be 16-byte aligned");
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return fail(ctx, DDS_ERR_UNSUPPORTED, "stress_noalloc: device %d beyond %d", ctx->device, MAX_DEVICES);

  // Work space of the five passes for this shape (complex FP32 elements).
  const Shape &sh = ctx->shape;
  const size_t fe = (size_t)(sh.fe > 0 ? sh.fe : 1);
  const size_t M = sh.M, ny = sh.ny, nz = sh.nz, py = sh.py;
  const size_t a = round256(std::max(fe * nz * ny * M, 6 * nz * py * M));
  const size_t b = round256(std::max(fe * nz * py * M, 6 * nz * ny * M));
  const size_t na = round256(std::max(fe * ny * nz, 6 * py * nz));
  const size_t nb = round256(std::max(fe * py * nz, 6 * ny * nz));
  const size_t need = a + b + na + nb;
  if (need > SCRATCH_ELEMS)
    return fail(ctx, DDS_ERR_UNSUPPORTED,
                "stress_noalloc: this grid needs %.1f MB of work space; the fixed area holds %.1f MB",
                need * sizeof(float2) / 1048576.0, (double)DDS_NOALLOC_SCRATCH_BYTES / 1048576.0);

  DeviceGuard guard(ctx->device);
  if (!guard.ok) return fail(ctx, DDS_ERR_CUDA, "stress_noalloc: cannot make device %d current", ctx->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ctx->fe == 0) {
    const cudaError_t err = cudaMemsetAsync(sigma, 0, sizeof(float) * 6 * (size_t)ctx->nx * ctx->ny * ctx->nz, s);
    return err == cudaSuccess ? DDS_OK : fail(ctx, DDS_ERR_CUDA, "stress_noalloc: %s", cudaGetErrorString(err));
  }
  float2 *base = nullptr;
  const cudaError_t err = scratch_address(ctx->device, &base);
  if (err != cudaSuccess)
    return fail(ctx, DDS_ERR_CUDA, "stress_noalloc: cannot locate the work area: %s", cudaGetErrorString(err));
  // Nothing in the area needs to start at zero: every element a pass reads was
  // written by an earlier pass of the same call.
  return enqueue_stress_buffers(ctx, rho, rho_dtype, sigma, base, base + a, base + a + b, base + a + b + na, s);
}
