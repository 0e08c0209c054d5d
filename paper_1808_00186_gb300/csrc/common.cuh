// Shared device-side definitions of the petgem CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "petgem.h"

namespace petgem {

// ------------------------------------------------------------------ complex helpers
// Storage types: complex128 = double2, complex64 = float2 (interleaved re, im).
struct c128 { double x, y; };
struct c64 { float x, y; };

template <typename T> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };

__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ------------------------------------------------------------------ device error flags
// One 32-bit word per context; kernels OR bits in, the host reads it at sync points.
enum DeviceFlag : uint32_t {
  kFlagBadNode = 1u << 0,       // a tet references a node id outside [0, n_nodes)
  kFlagRepeatedNode = 1u << 1,  // a tet repeats a node
  kFlagNonManifold = 1u << 2,   // a face is shared by more than two tets
  kFlagDegenerate = 1u << 3,    // a tet has (near) zero volume
  kFlagSegmentTooLong = 1u << 4,
  kFlagNaN = 1u << 5,
};

// ------------------------------------------------------------------ launch helpers
inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Host-side status carrier used inside the library.
struct Status {
  int code = PETGEM_OK;
  std::string msg;
  bool ok() const { return code == PETGEM_OK; }
};

#define PG_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return petgem::Status{PETGEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    }                                                                                     \
  } while (0)

// Programmatic dependent launch.  A kernel started with pdl_launch may be scheduled while the
// kernel before it in the stream is still finishing (its launch is processed early); it must call
// pdl_wait() before it reads anything that kernel wrote, and may call pdl_trigger() to let the
// kernel after it be scheduled once every one of its own blocks has started.  Both are no-ops for
// a kernel started with a plain launch.
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool cooperative,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  int na = 1;
  if (cooperative) {
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    na = 2;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

#define PG_TRY(expr)                   \
  do {                                 \
    petgem::Status s_ = (expr);        \
    if (!s_.ok()) return s_;           \
  } while (0)

// Exclusive prefix sum of n int32 counts into out[0..n] (out[n] = total), int64 results,
// on `stream`.  Scratch comes from the stream-ordered allocator.
Status exclusive_scan(const int32_t* in, int64_t* out, int64_t n, cudaStream_t stream);

}  // namespace petgem
