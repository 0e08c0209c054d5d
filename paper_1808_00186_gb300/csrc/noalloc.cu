// Allocation-free form of the weight gradient of the learned preconditioner's 3x3x3 convolution
// (declared in include/petgem.h as petgem_nn_conv3d_wgrad_noalloc).
//
// petgem_nn_conv3d_wgrad takes its split-K partial sums and its error flag from cudaMallocAsync
// on every call.  Some callers cannot allocate device memory inside such a call: a host framework
// whose own caching allocator already holds the free device memory (a driver allocation then
// fails, or fragments the pool it manages), or a training step that runs with allocation
// forbidden because an allocation can wait on the allocator's lock and a release can synchronise
// the device.  This entry point serves them: its scratch is one fixed array in the library's own
// device memory (a module global, reserved when the library's device code is loaded), sized for
// grids of up to PETGEM_NOALLOC_MAX_VOXELS voxels; it calls no cudaMalloc, cudaMallocAsync,
// cudaFree or other allocating routine.
//
// The scratch is shared by every call on a device, so calls that overlap in time (on two streams,
// or from two host threads) race on it and corrupt each other's partial sums.
#include <mutex>

#include "learned.cuh"

namespace {

// wgrad_splits(V) = ceil(V / 4096) for V up to the limit: 32 split-K slices of the largest
// partial-sum block (27 taps x 32 x 32 channels, FP32), then the error flag on its own 256 B.
constexpr int kMaxSplits = PETGEM_NOALLOC_MAX_VOXELS / 4096;
constexpr size_t kPartBytes = (size_t)kMaxSplits * 27 * 32 * 32 * sizeof(float);
constexpr size_t kScratchBytes = kPartBytes + 256;
static_assert(kPartBytes % 256 == 0, "the error flag must start on a 256-byte boundary");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices];  // the scratch's device address, per device ordinal

}  // namespace

// 3,538,944 B of partial sums + 256 B for the error flag, per device.
static __device__ __align__(256) unsigned char g_wgrad_scratch[kScratchBytes];

namespace {

// Address of the scratch on the current device, looked up once per device with that device
// current (the first call on a device does this set-up).
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PETGEM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PETGEM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_wgrad_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PETGEM_ERR_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return PETGEM_OK;
}

}  // namespace

extern "C" int petgem_nn_conv3d_wgrad_noalloc(void* stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin,
                                              int32_t cout, const void* x, const void* dy, float* dw) {
  if (gx < 1 || gy < 1 || gz < 1 || !x || !dy || !dw) return PETGEM_ERR_INVALID_ARG;
  if ((cin != 16 && cin != 32) || (cout != 16 && cout != 32)) return PETGEM_ERR_UNSUPPORTED;
  // Each dimension is checked before the product is formed: three dimensions up to the limit
  // multiply to at most 2^51, so the 64-bit product below cannot wrap.
  const int64_t lim = PETGEM_NOALLOC_MAX_VOXELS;
  if (gx > lim || gy > lim || gz > lim) return PETGEM_ERR_UNSUPPORTED;
  const int64_t V = (int64_t)gx * gy * gz;
  if (V > lim) return PETGEM_ERR_UNSUPPORTED;  // beyond the fixed scratch
  const int splits = petgem::nn::wgrad_splits(V);
  if (splits > kMaxSplits) return PETGEM_ERR_UNSUPPORTED;
  unsigned char* base = nullptr;
  const int st = scratch_address(&base);
  if (st != PETGEM_OK) return st;
  float* part = reinterpret_cast<float*>(base);  // every slice is written before it is read
  int* err = reinterpret_cast<int*>(base + kPartBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return PETGEM_ERR_CUDA;  // starts at zero
  petgem::Status r = petgem::nn::conv3d_wgrad(s, gx, gy, gz, cin, cout, static_cast<const __nv_bfloat16*>(x),
                                              static_cast<const __nv_bfloat16*>(dy), part, splits, dw, false, err);
  if (r.ok()) r = petgem::nn::check_err(s, err, "petgem_nn_conv3d_wgrad_noalloc");
  return r.code;
}
