// Allocation-free variant of the batched Hermitian eigen-solver step.
//
// Some callers cannot call cudaMalloc while they run: code inside a host
// framework that owns all device memory and forbids libraries from
// allocating, real-time loops that cannot afford the allocator's latency or
// the device-wide synchronisation cudaFree implies, and programs that reserve
// all memory they will ever use before they start.  For them,
// spod_eigh_batched_noalloc takes its scratch from a fixed array in this
// file instead of from the allocator.  The array (kNoAllocScratchBytes) is
// part of the library image, so every GPU that loads the library holds it
// until the process exits.
#include <mutex>

#include "spod_internal.cuh"

namespace spod {
namespace {

// Scratch of the eigen-solver: [256 B status word][per-frequency working
// copies A and V, 2 * nb * nb complex FP64 each, used when nb exceeds the
// shared-memory limit of the solver].
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr size_t kFlagsBytes = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the array.
// In host code the array's name is only a host-side stand-in, never a device
// address, so kernels must be given this pointer instead.
cudaError_t scratch_for_device(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace spod

using namespace spod;

extern "C" spod_status spod_eigh_batched_noalloc(const double* d_gram, int nf, int nb, double* d_lambda,
                                                 double* d_psi, void* stream) {
  if (!d_gram || !d_lambda || !d_psi) {
    set_error("spod_eigh_batched_noalloc: NULL pointer");
    return SPOD_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_gram) % 16 || reinterpret_cast<uintptr_t>(d_psi) % 16 ||
      reinterpret_cast<uintptr_t>(d_lambda) % 8) {
    set_error("spod_eigh_batched_noalloc: d_gram and d_psi must be 16-byte aligned, d_lambda 8-byte aligned");
    return SPOD_EINVAL;
  }
  if (nf < 1 || nb < 1 || nb > kMaxNb) {
    set_error("spod_eigh_batched_noalloc: need nf >= 1 and 1 <= nb <= 1024");
    return SPOD_EINVAL;
  }
  const size_t work = nb > kEigSmemMaxNb ? (size_t)nf * 4 * (size_t)nb * nb * sizeof(double) : 0;
  if (kFlagsBytes + work > kNoAllocScratchBytes) {
    set_error("spod_eigh_batched_noalloc: nf * 32 * nb^2 bytes of scratch needed (" +
              std::to_string(kFlagsBytes + work) + ") exceeds the fixed 32 MiB array");
    return SPOD_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_for_device(dev, &base);
  if (e != cudaSuccess) {
    set_error(std::string("spod_eigh_batched_noalloc: scratch set-up: ") + cudaGetErrorString(e));
    return SPOD_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* flags = static_cast<unsigned*>(base);
  double* gws = nb > kEigSmemMaxNb ? reinterpret_cast<double*>(static_cast<char*>(base) + kFlagsBytes) : nullptr;
  // the status word keeps the previous call's value: clear it
  e = cudaMemsetAsync(flags, 0, kFlagsBytes, s);
  if (e == cudaSuccess) e = launch_eig_buffers(d_gram, nf, nb, d_lambda, d_psi, gws, flags, s);
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("spod_eigh_batched_noalloc: ") + cudaGetErrorString(e));
    return SPOD_ECUDA;
  }
  if (h & FLAG_NOTCONV) {
    set_error("spod_eigh_batched_noalloc: eigen-solver reached its sweep cap");
    return SPOD_ENOTCONVERGED;
  }
  return SPOD_OK;
}
