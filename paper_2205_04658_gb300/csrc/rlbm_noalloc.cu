// Energy spectrum of caller-provided device velocity fields with no memory allocation:
// the FFT work buffers live in a fixed-size array in the library's own device memory.
//
// Who needs it: callers that cannot call cudaMalloc.  Some own every byte of device
// memory through their own allocator or a fixed budget (a framework's memory pool that
// must not be bypassed, an embedded service with a hard cap); others run in loops where
// cudaMalloc's implicit device-wide synchronisation would stall unrelated streams.  The
// regular rlbm_spectrum works on a context, whose workspace the caller allocates.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/rlbm.h"
#include "rlbm_launch.h"

namespace rlbm {
void set_thread_error(const std::string &msg);  // message of rlbm_last_error(NULL)
}

namespace {

constexpr int kMaxCells = 131072;  // nx * ny <= 2^17 (for example 512 x 256)
constexpr int kMaxDim = 16384;     // nx, ny <= 2^14
constexpr int kMaxBins = 8200;     // every shell round(|k|) of every accepted lattice (|k| <= 8193)
constexpr size_t kZBytes = sizeof(double2) * kMaxCells;
constexpr size_t kTwBytes = sizeof(double2) * kMaxDim;
constexpr size_t kScratchBytes = 2 * kZBytes + 2 * kTwBytes + sizeof(double) * kMaxBins;

// The scratch: two complex work arrays, the twiddles of both directions and the bins,
// kScratchBytes = 4 784 192 bytes (about 4.8 MB, 4.56 MiB).  Every GPU that loads the
// library holds it until the process exits.  In host code the name is only a stand-in; its
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static_assert(kScratchBytes == 4784192, "the size the header states");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_ptr[kMaxDevices];  // device address of the scratch per device, once looked up

// The scratch's device address on device `dev` (current), looked up on the first call that
// succeeds: a failed lookup is not kept, so a later call tries again.
cudaError_t scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();  // clear the error this lookup left, so that it is not reported again later
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}


// exp(-2 pi i t / n) for t < n
__global__ void twiddle_kernel(double2 *tw, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s, c;
  sincospi(2.0 * t / n, &s, &c);
  tw[t] = make_double2(c, -s);
}

}  // namespace

extern "C" RLBM_API rlbm_status rlbm_spectrum_noalloc(const double *d_ux, const double *d_uy, int32_t nx, int32_t ny,
                                                      int32_t nbins, double *d_E, void *cuda_stream) {
  if (!d_ux || !d_uy || !d_E) { rlbm::set_thread_error("d_ux, d_uy and d_E must be device pointers"); return RLBM_E_INVAL; }
  if (nx < 8 || ny < 8 || nx > kMaxDim || ny > kMaxDim || (long long)nx * ny > kMaxCells) {
    rlbm::set_thread_error("rlbm_spectrum_noalloc handles 8 <= nx, ny <= " + std::to_string(kMaxDim) +
                           " and nx * ny <= " + std::to_string(kMaxCells) + " cells; got " + std::to_string(nx) +
                           " x " + std::to_string(ny));
    return RLBM_E_INVAL;
  }
  if (nbins < 1 || nbins > kMaxBins) {
    rlbm::set_thread_error("nbins must lie in [1, " + std::to_string(kMaxBins) + "]");
    return RLBM_E_INVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    rlbm::set_thread_error(std::string("no usable current device: ") + cudaGetErrorString(e));
    return RLBM_E_CUDA;
  }
  // set-up, once per device, with that device current (retried on the next call if it fails)
  void *scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess) {
    rlbm::set_thread_error(std::string("cudaGetSymbolAddress of the scratch failed: ") + cudaGetErrorString(e));
    return RLBM_E_CUDA;
  }
  unsigned char *base = static_cast<unsigned char *>(scratch);
  double2 *z0 = reinterpret_cast<double2 *>(base);
  double2 *z1 = reinterpret_cast<double2 *>(base + kZBytes);
  double2 *twx = reinterpret_cast<double2 *>(base + 2 * kZBytes);
  double2 *twy = reinterpret_cast<double2 *>(base + 2 * kZBytes + kTwBytes);
  double *bins = reinterpret_cast<double *>(base + 2 * kZBytes + 2 * kTwBytes);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  twiddle_kernel<<<(nx + 255) / 256, 256, 0, st>>>(twx, nx);
  twiddle_kernel<<<(ny + 255) / 256, 256, 0, st>>>(twy, ny);
  if ((e = cudaGetLastError()) != cudaSuccess) { rlbm::set_thread_error(std::string("twiddle kernel: ") + cudaGetErrorString(e)); return RLBM_E_CUDA; }
  // launch_spectrum zeroes the bins before it accumulates into them
  e = rlbm::launch_spectrum(d_ux, d_uy, nx, ny, twx, twy, z0, z1, bins, nbins, st);
  if (e != cudaSuccess) { rlbm::set_thread_error(std::string("spectrum kernels: ") + cudaGetErrorString(e)); return RLBM_E_CUDA; }
  e = cudaMemcpyAsync(d_E, bins, sizeof(double) * nbins, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) { rlbm::set_thread_error(std::string("copy of the bins: ") + cudaGetErrorString(e)); return RLBM_E_CUDA; }
  return RLBM_OK;
}
