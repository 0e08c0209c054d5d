// Kernels of the learned preconditioner's network: 3x3x3 convolutions as implicit GEMMs on the
// tcgen05 tensor cores (forward, and the input gradient through flipped weights), the weight
// gradient as a split-K tcgen05 GEMM, and the grid element-wise operations.
//
// Grid tensors: BF16 [V][C], voxel v = x + gx (y + gy z), channels innermost (C = 16 or 32).
// Convolution weights: W[t][co][ci], tap t = (dx+1) + 3 (dy+1) + 9 (dz+1), zero "same" padding:
//   y[v][co] = b[co] + sum_t sum_ci W[t][co][ci] x[v + (dx, dy, dz)][ci].
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace petgem {
namespace nn {

constexpr int kConvRows = 128;  // output voxels per CTA (the MMA's M)

// Dynamic shared memory of k_conv3d<CIN, COUT>: two A buffers and all 27 taps of the weights.
__host__ __device__ constexpr int conv_smem(int cin, int cout) { return 2 * kConvRows * cin * 2 + 27 * cout * cin * 2; }

// One CTA: 128 consecutive output voxels x COUT channels.  For every tap, the 128 neighbour rows
// (CIN channels each) are gathered into a double-buffered shared tile laid out as K-major core
// matrices, and one thread issues CIN/16 MMAs (K = 16 each) accumulating in TMEM; the buffer is
// refilled only after the tcgen05.commit of the MMAs that read it has arrived on its mbarrier.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv3d(const __nv_bfloat16* __restrict__ X,
                                                const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                                                int gx, int gy, int gz, int relu, __nv_bfloat16* __restrict__ Ybf,
                                                float* __restrict__ Yf, int* __restrict__ err,
                                                const int* __restrict__ stop) {
  static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 32, "channel counts");
  if (stop && *stop) return;  // block-uniform: before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                               // 2 x 128 x CIN bf16
  unsigned char* sW = smem + 2 * kConvRows * CIN * 2;     // 27 x COUT x CIN bf16
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ unsigned tbase;
  __shared__ int s_ok;  // block-uniform outcome of the last mbarrier wait (thread 0 waits)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int V = gx * gy * gz;
  // weights -> core-matrix layout (8 input channels = one 16-byte core row)
  for (int idx = tid; idx < 27 * COUT * (CIN / 8); idx += 128) {
    const int c8 = idx % (CIN / 8), row = idx / (CIN / 8);  // row = t * COUT + co
    const int t = row / COUT, co = row - t * COUT;
    const uint4 w = *reinterpret_cast<const uint4*>(W + (size_t)row * CIN + 8 * c8);
    *reinterpret_cast<uint4*>(sW + t * COUT * CIN * 2 + tc::core_offset(co, 8 * c8, CIN)) = w;
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0]);
    tc::mbar_init(&bar[1]);
    tc::mbar_init_fence();
    s_ok = 1;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = tbase;
  const int v = blockIdx.x * kConvRows + tid;
  const int x = v % gx, y = (v / gx) % gy, z = v / (gx * gy);
  const uint32_t idesc = tc::idesc_bf16(kConvRows, COUT);
  const unsigned sbo = (CIN / 8) * 128;
  // A timed-out wait stops the tap loop for the whole block: no further buffer rewrite or MMA
  // issue, no TMEM load; the MMAs already issued are drained with one more bounded wait before
  // TMEM is freed, and the error flag is set.
  int issued = 0;  // taps whose MMAs were issued
  for (int t = 0; t < 27; ++t) {
    const int buf = t & 1;
    if (t >= 2) {
      if (tid == 0 && !tc::mbar_wait(&bar[buf], ((t - 2) >> 1) & 1)) s_ok = 0;
      __syncthreads();
      if (!s_ok) break;
    }
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int nx = x + dx, ny = y + dy, nz = z + dz;
    const bool in = v < V && nx >= 0 && nx < gx && ny >= 0 && ny < gy && nz >= 0 && nz < gz;
    const __nv_bfloat16* src = X + (size_t)(nx + gx * (ny + gy * nz)) * CIN;
    unsigned char* dstA = sA + buf * kConvRows * CIN * 2;
#pragma unroll
    for (int c8 = 0; c8 < CIN / 8; ++c8) {
      const uint4 a = in ? *reinterpret_cast<const uint4*>(src + 8 * c8) : make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(dstA + tc::core_offset(tid, 8 * c8, CIN)) = a;
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int ks = 0; ks < CIN / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(dstA) + ks * 256, 128, sbo);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sW + t * COUT * CIN * 2) + ks * 256, 128, sbo);
        tc::mma_bf16(tmem, ad, bd, idesc, t > 0 || ks > 0);
      }
      tc::commit(&bar[buf]);
    }
    issued = t + 1;
  }
  // the commit of the last issued tap covers every MMA issued before it (after all 27 taps: the
  // 14th commit on buffer 0, parity 1)
  if (tid == 0 && issued > 0) {
    const int last = issued - 1;
    if (!tc::mbar_wait(&bar[last & 1], (last >> 1) & 1)) s_ok = 0;
  }
  __syncthreads();
  tc::fence_after();
  const bool ok = s_ok != 0 && issued == 27;
  if (ok) {
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + c0, acc);
      if (v < V) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float r = acc[i] + bias[c0 + i];
          if (relu) r = fmaxf(r, 0.f);
          acc[i] = r;
        }
        if (Yf) {
#pragma unroll
          for (int i = 0; i < 16; ++i) Yf[(size_t)v * COUT + c0 + i] = acc[i];
        } else {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16(acc[i]);
          *reinterpret_cast<uint4*>(Ybf + (size_t)v * COUT + c0) = *reinterpret_cast<uint4*>(o);
          *reinterpret_cast<uint4*>(Ybf + (size_t)v * COUT + c0 + 8) = *reinterpret_cast<uint4*>(o + 8);
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// Weight gradient as a GEMM over voxels: D[(t, ci)][co] = sum_v X[v + off_t][ci] dY[v][co].
// CTA (m, s): rows (t, ci) in [128 m, 128 m + 128) of 27 CIN, voxel chunks s, s + splits, ...
// of 64 voxels (K = 64: four MMAs).  Each chunk's im2col-transposed tile and dY tile are built in
// shared memory; the FP32 partial sums go to part[s][row][co] for a fixed-order reduction.
constexpr int kWgChunk = 64;
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ X,
                                                      const __nv_bfloat16* __restrict__ dY, int gx, int gy, int gz,
                                                      float* __restrict__ part, int* __restrict__ err) {
  __shared__ __align__(1024) unsigned char sA[kConvRows * kWgChunk * 2];
  __shared__ __align__(1024) unsigned char sB[COUT * kWgChunk * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tbase;
  __shared__ int s_ok;  // block-uniform outcome of the last mbarrier wait (thread 0 waits)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int V = gx * gy * gz;
  const int rows = 27 * CIN;
  const int row0 = blockIdx.x * kConvRows;
  const int splits = gridDim.y, split = blockIdx.y;
  const int nchunks = (V + kWgChunk - 1) / kWgChunk;
  if (tid == 0) {
    tc::mbar_init(&bar);
    tc::mbar_init_fence();
    s_ok = 1;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = tbase;
  const uint32_t idesc = tc::idesc_bf16(kConvRows, COUT);
  const unsigned sbo = (kWgChunk / 8) * 128;
  // thread -> (voxel column k, half of the 8-channel chunks)
  const int k = tid & (kWgChunk - 1), half = tid >> 6;
  // the taps whose rows meet this tile
  const int t_lo = row0 / CIN, t_hi = min(26, (row0 + kConvRows - 1) / CIN);
  int issued = 0;
  for (int ch = split; ch < nchunks; ch += splits) {
    const int v = ch * kWgChunk + k;
    const bool vin = v < V;
    const int x = v % gx, y = (v / gx) % gy, z = v / (gx * gy);
    // A: rows (t, ci) of this tile, column k = X[v + off_t][ci]
    for (int t = t_lo; t <= t_hi; ++t) {
      const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
      const int nx = x + dx, ny = y + dy, nz = z + dz;
      const bool in = vin && nx >= 0 && nx < gx && ny >= 0 && ny < gy && nz >= 0 && nz < gz;
      const __nv_bfloat16* src = X + (size_t)(nx + gx * (ny + gy * nz)) * CIN;
      for (int c8 = half; c8 < CIN / 8; c8 += 2) {
        const int r = t * CIN + 8 * c8 - row0;  // tile row of channel 8 c8
        if (r < 0 || r >= kConvRows) continue;
        __align__(16) __nv_bfloat16 e[8];
        *reinterpret_cast<uint4*>(e) = in ? *reinterpret_cast<const uint4*>(src + 8 * c8) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          *reinterpret_cast<__nv_bfloat16*>(sA + tc::core_offset(r + i, k, kWgChunk)) = e[i];
      }
    }
    // rows past 27 CIN are zero
    if (row0 + kConvRows > rows)
      for (int r = max(0, rows - row0) + half; r < kConvRows; r += 2)
        *reinterpret_cast<__nv_bfloat16*>(sA + tc::core_offset(r, k, kWgChunk)) = __float2bfloat16(0.f);
    // B: rows co, column k = dY[v][co]
    for (int c8 = half; c8 < COUT / 8; c8 += 2) {
      __align__(16) __nv_bfloat16 e[8];
      *reinterpret_cast<uint4*>(e) = vin ? *reinterpret_cast<const uint4*>(dY + (size_t)v * COUT + 8 * c8)
                                         : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::core_offset(8 * c8 + i, k, kWgChunk)) = e[i];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int ks = 0; ks < kWgChunk / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(sA) + ks * 256, 128, sbo);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + ks * 256, 128, sbo);
        tc::mma_bf16(tmem, ad, bd, idesc, issued > 0 || ks > 0);
      }
      tc::commit(&bar);
    }
    // the tiles are rewritten next chunk: wait for these MMAs.  On a timeout the whole block
    // stops issuing (the decision is block-uniform), skips the TMEM loads and sets the error flag;
    // a timed-out commit gets one more bounded wait before TMEM is freed.
    if (tid == 0 && !tc::mbar_wait(&bar, issued & 1)) {
      s_ok = 0;
      tc::mbar_wait(&bar, issued & 1);
    }
    ++issued;
    __syncthreads();
    tc::fence_after();
    if (!s_ok) break;
  }
  const bool ok = s_ok != 0;
  if (ok) {
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      float acc[16];
      if (issued > 0) {
        tc::tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + c0, acc);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      }
      const int r = row0 + warp * 32 + (tid & 31);
      if (r < rows) {
#pragma unroll
        for (int i = 0; i < 16; ++i) part[((size_t)split * rows + r) * COUT + c0 + i] = acc[i];
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// dW[t][co][ci] (+)= sum_s part[s][t CIN + ci][co], fixed order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int splits, int cin, int cout, float* __restrict__ dW,
                               int accumulate) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over 27 cout cin, layout of dW
  if (idx >= 27 * cout * cin) return;
  const int ci = idx % cin, co = (idx / cin) % cout, t = idx / (cin * cout);
  const int rows = 27 * cin, r = t * cin + ci;
  float s = 0.f;
  for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * rows + r) * cout + co];
  dW[idx] = accumulate ? dW[idx] + s : s;
}

}  // namespace nn
}  // namespace petgem
