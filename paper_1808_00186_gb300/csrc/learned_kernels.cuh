// Kernels of the learned preconditioner's network: the 3x3x3 convolution on the tcgen05 tensor
// cores (forward, and the input gradient through flipped weights; one halo brick per CTA, the
// taps as descriptor offsets into it), the packing of its weights into the kernel's shared-memory
// image, and the weight gradient as a split-K tcgen05 GEMM.  Pooling, upsampling and the
// auxiliary maps are in learned.cu.
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

constexpr int kConvRows = 128;  // output voxels per tensor-core tile (the MMA's M)

// Convolution tile: 8 (x) by 16 (y) voxels of one z-plane, 128 rows of the MMA, row m at
// (x0 + m % 8, y0 + m / 8).  A CTA computes NZ such tiles stacked in z from one halo brick, the
// input voxels x0-1 .. x0+8, y0-1 .. y0+16, z0-1 .. z0+NZ (zero outside the grid), held in shared
// memory as CIN/8 "planes" of 8 channels, 16 bytes per voxel, voxel (x', y', z') of the brick at
// ((z' kHaloY + y') kHaloX + x') * 16 in its plane.  In that layout the A operand of every tap is
// already a K-major core-matrix tile: core matrix i (line y0 + i, rows x0 .. x0+7) is 8 voxels 16
// bytes apart, line i + 1 is kHaloX voxels further on (the stride byte offset), the next 8 input
// channels one plane further on (the leading byte offset), and tap (dx, dy, dz) only moves the
// start address.  So all 27 taps read the one brick: no per-tap gather.
constexpr int kBrickX = 8, kBrickY = 16;
constexpr int kHaloX = kBrickX + 2, kHaloY = kBrickY + 2;
static_assert(kBrickX * kBrickY == kConvRows, "tile rows");

// Bytes of one plane of the halo brick of nz output planes (128-byte aligned).
__host__ __device__ constexpr int brick_plane(int nz) { return (kHaloX * kHaloY * (nz + 2) * 16 + 127) / 128 * 128; }
// Dynamic shared memory of k_conv3d<CIN, COUT, NZ>: the brick, all 27 taps of the weights, the
// bias, and the slack that aligns the brick to 128 bytes.
__host__ __device__ constexpr int conv_smem(int cin, int cout, int nz) {
  return (cin / 8) * brick_plane(nz) + 27 * cout * cin * 2 + cout * 4 + 128;
}
// Planes per CTA from which the MMAs are shared between output planes: the A operand of tap dz
// for output plane zl is brick plane zl + dz, so one MMA per brick plane and (dy, dx) with the
// three z-taps' weights stacked (N = 3 COUT) adds that plane's contribution to three output
// planes' accumulators at once: (NZ + 2) 9 MMAs instead of 27 NZ (54 against 108 at NZ = 4), at
// the same issue cost (an M = 128 MMA costs the issuing thread the same for any N up to 64 and
// little more up to 128).  The accumulators of planes -2, -1, NZ and NZ + 1 are scratch.
__host__ __device__ constexpr bool conv_shares(int nz) { return nz >= 2; }
// TMEM columns: NZ accumulators of COUT FP32 columns, NZ + 4 when the MMAs are shared (a power
// of two, at least 32).
__host__ __device__ constexpr unsigned conv_tmem_cols(int cout, int nz) {
  return (conv_shares(nz) ? nz + 4 : nz) * cout <= 32    ? 32u
         : (conv_shares(nz) ? nz + 4 : nz) * cout <= 64  ? 64u
         : (conv_shares(nz) ? nz + 4 : nz) * cout <= 128 ? 128u
                                                         : 256u;
}
// Dynamic shared memory a launch requests: at least conv_smem, and enough that the CTAs one SM
// holds (233,472 bytes of shared memory, 1 KB reserved per CTA) never ask for more than the 512
// TMEM columns, so no allocation waits for another CTA.
__host__ __device__ constexpr int conv_smem_launch(int cin, int cout, int nz) {
  return conv_smem(cin, cout, nz) > 233472 / (int)(512 / conv_tmem_cols(cout, nz) + 1) - 1024 + 16
             ? conv_smem(cin, cout, nz)
             : 233472 / (int)(512 / conv_tmem_cols(cout, nz) + 1) - 1024 + 16;
}

// Convolution weights as the kernel's shared-memory image, grouped by (dy, dx): group
// g = 3 (dy+1) + (dx+1) is one K-major core-matrix tile of 3 COUT rows (CIN columns), the
// weights of dz = +1, 0, -1 stacked in that order, so that a group is the B operand of a shared
// MMA and one dz block of it (COUT rows, COUT CIN elements further per block) the B operand of a
// single tap.  Element (t, co, ci) of W[t][co][ci], t = (dx+1) + 3 (dy+1) + 9 (dz+1), sits at
// g 3 COUT CIN + core_offset((1 - dz) COUT + co, ci, CIN) / 2.  One bulk copy loads all 27 taps.
__host__ __device__ inline int64_t conv_weight_index(int t, int co, int ci, int cin, int cout) {
  const int g = t % 9, j = 2 - t / 9;
  return (int64_t)g * 3 * cout * cin + tc::core_offset(j * cout + co, ci, cin) / 2;
}

// X: BF16 [gz][gy][gx][CIN]; Wc: the weights in the order above.  Grid: one CTA per (x-tile,
// y-tile, z-group of NZ planes), x fastest.  Thread 0 starts the bulk copy of the weights; all
// threads copy the brick (16-byte cp.async, zeros outside the grid) and the bias; thread 0 then
// issues the MMAs (K = 16 each) into the TMEM accumulators and one commit: (NZ + 2) 9 CIN/16
// shared ones of N = 3 COUT when NZ >= 2 (conv_shares; the accumulators zeroed first), else
// 27 CIN/16 of N = COUT; the four warps read their 32 TMEM lanes each and store bias + (ReLU) to
// the voxels inside the grid.
template <int CIN, int COUT, int NZ>
__global__ void __launch_bounds__(128) k_conv3d(const __nv_bfloat16* __restrict__ X,
                                                const __nv_bfloat16* __restrict__ Wc, const float* __restrict__ bias,
                                                int gx, int gy, int gz, int relu, __nv_bfloat16* __restrict__ Ybf,
                                                float* __restrict__ Yf, int* __restrict__ err,
                                                const int* __restrict__ stop) {
  static_assert(CIN % 16 == 0 && CIN <= 32 && COUT % 16 == 0 && COUT <= 32 && NZ >= 1 && NZ <= 4, "tile shape");
  constexpr int NC = CIN / 8;
  constexpr int kPlane = brick_plane(NZ);
  constexpr int kVox = kHaloX * kHaloY * (NZ + 2);
  constexpr unsigned kWBytes = 27 * COUT * CIN * 2;
  constexpr unsigned kCols = conv_tmem_cols(COUT, NZ);
  constexpr bool kShare = conv_shares(NZ);
  const int stopped = stop ? *stop : 0;  // consumed after the barrier set-up, which hides its latency
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sX = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);  // NC planes
  unsigned char* sW = sX + NC * kPlane;                                                // 27 x COUT x CIN
  float* sB = reinterpret_cast<float*>(sW + kWBytes);                                  // COUT
  __shared__ __align__(8) uint64_t bar[2];  // 0: the weights have landed; 1: the MMAs are done
  __shared__ unsigned tbase;
  __shared__ int s_ok;  // block-uniform outcome of the bounded waits (thread 0 waits)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tiles_x = (gx + kBrickX - 1) / kBrickX, tiles_y = (gy + kBrickY - 1) / kBrickY;
  const int x0 = (int)(blockIdx.x % tiles_x) * kBrickX;
  const int y0 = (int)((blockIdx.x / tiles_x) % tiles_y) * kBrickY;
  const int z0 = (int)(blockIdx.x / (tiles_x * tiles_y)) * NZ;
  if (tid == 0) {
    tc::mbar_init(&bar[0]);
    tc::mbar_init(&bar[1]);
    tc::mbar_init_fence();
    s_ok = 1;
  }
  __syncthreads();
  if (stopped) return;  // block-uniform: no copy, MMA or TMEM allocation yet
  if (tid == 0) {
    tc::mbar_expect_tx(&bar[0], kWBytes);
    tc::bulk_load(sW, Wc, kWBytes, &bar[0]);
  }
  if (tid < COUT) tc::cp_async4(sB + tid, bias + tid);
  // brick: consecutive threads on consecutive 16-byte pieces of the input (8 channels of a voxel)
  for (int idx = tid; idx < kVox * NC; idx += 128) {
    const int c = idx % NC, b = idx / NC;
    const int xh = b % kHaloX, yh = (b / kHaloX) % kHaloY, zh = b / (kHaloX * kHaloY);
    const int x = x0 - 1 + xh, y = y0 - 1 + yh, z = z0 - 1 + zh;
    unsigned char* dst = sX + c * kPlane + b * 16;
    if (x >= 0 && x < gx && y >= 0 && y < gy && z >= 0 && z < gz)
      tc::cp_async16(dst, X + ((size_t)x + (size_t)gx * ((size_t)y + (size_t)gy * (size_t)z)) * CIN + 8 * c);
    else
      *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
  }
  tc::cp_async_commit();
  if (warp == 0) tc::tmem_alloc(&tbase, kCols);
  if (kShare) {  // every shared MMA accumulates: the accumulators start at zero
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
#pragma unroll
    for (unsigned c = 0; c < (NZ + 4) * COUT; c += 16) tc::tmem_zero16(tbase + ((unsigned)(warp * 32) << 16) + c);
    tc::tmem_wait_st();
  }
  tc::cp_async_wait_all();
  tc::fence_proxy_async();  // the brick (generic proxy) becomes visible to the tensor core
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const unsigned tmem = tbase;
  // A timed-out wait issues nothing more: the weights' copy is let land (a second bounded wait)
  // before the CTA leaves, issued MMAs are drained before TMEM is freed, and the flag is set.
  if (tid == 0) {
    if (!tc::mbar_wait(&bar[0], 0)) {
      s_ok = 0;
      tc::mbar_wait(&bar[0], 0);
    } else {
      const uint64_t ad0 = tc::smem_desc(tc::smem_u32(sX), kPlane, kHaloX * 16);
      const uint64_t bd0 = tc::smem_desc(tc::smem_u32(sW), 128, (CIN / 8) * 128);
      // descriptor start addresses are in 16-byte units: a tap, K-step or plane adds its offset / 16
      if (kShare) {
        // brick plane p, tap (dy, dx): D columns [p COUT, (p + 3) COUT) are the accumulators of
        // output planes p - 2, p - 1, p (dz = +1, 0, -1), accumulator a of plane a - 2
        const uint32_t idesc = tc::idesc_bf16(kConvRows, 3 * COUT);
#pragma unroll
        for (int p = 0; p < NZ + 2; ++p) {
#pragma unroll
          for (int g = 0; g < 9; ++g) {
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ++ks) {
              const int aoff = ((p * kHaloY + g / 3) * kHaloX + g % 3) * 16 + 2 * ks * kPlane;
              const uint64_t bd = bd0 + (uint64_t)((g * 3 * COUT * CIN * 2 + ks * 256) >> 4);
              tc::mma_bf16(tmem + p * COUT, ad0 + (uint64_t)(aoff >> 4), bd, idesc, true);
            }
          }
        }
      } else {
        const uint32_t idesc = tc::idesc_bf16(kConvRows, COUT);
#pragma unroll
        for (int t = 0; t < 27; ++t) {
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ++ks) {
            const int woff = (t % 9) * 3 * COUT * CIN * 2 + (2 - t / 9) * COUT * CIN * 2 + ks * 256;
            const uint64_t bd = bd0 + (uint64_t)(woff >> 4);
#pragma unroll
            for (int zl = 0; zl < NZ; ++zl) {
              const int aoff = (((zl + t / 9) * kHaloY + (t / 3) % 3) * kHaloX + t % 3) * 16 + 2 * ks * kPlane;
              tc::mma_bf16(tmem + zl * COUT, ad0 + (uint64_t)(aoff >> 4), bd, idesc, t > 0 || ks > 0);
            }
          }
        }
      }
      tc::commit(&bar[1]);
      if (!tc::mbar_wait(&bar[1], 0)) {
        s_ok = 0;
        tc::mbar_wait(&bar[1], 0);
      }
    }
  }
  __syncthreads();
  tc::fence_after();
  if (s_ok) {
    const int x = x0 + (tid & 7), y = y0 + (tid >> 3);  // row m = tid (warp w: TMEM lanes 32w ..)
#pragma unroll
    for (int zl = 0; zl < NZ; ++zl) {
      const int z = z0 + zl;
      const bool in = x < gx && y < gy && z < gz;
      const size_t v = (size_t)x + (size_t)gx * ((size_t)y + (size_t)gy * (size_t)z);
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((zl + (kShare ? 2 : 0)) * COUT + c0), acc);
        if (in) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float r = acc[i] + sB[c0 + i];
            if (relu) r = fmaxf(r, 0.f);
            acc[i] = r;
          }
          if (Yf) {
#pragma unroll
            for (int i = 0; i < 16; i += 4)
              *reinterpret_cast<float4*>(Yf + v * COUT + c0 + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
          } else {
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = __float2bfloat16(acc[i]);
            *reinterpret_cast<uint4*>(Ybf + v * COUT + c0) = *reinterpret_cast<uint4*>(o);
            *reinterpret_cast<uint4*>(Ybf + v * COUT + c0 + 8) = *reinterpret_cast<uint4*>(o + 8);
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// Weights -> the convolution's shared-memory image (conv_weight_index), BF16.  flip: the layer
// cout' x cin' = cin x cout with W'[t][o][i] = W[26 - t][i][o], the convolution that takes the
// output gradient of the layer W (cin -> cout) to its input gradient.  Wf: FP32 [27][cout][cin].
__global__ void k_pack_conv_weights(const float* __restrict__ Wf, int cin, int cout, int flip,
                                    __nv_bfloat16* __restrict__ Wc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 27 * cin * cout) return;
  const int ci2 = flip ? cout : cin, co2 = flip ? cin : cout;  // the packed layer's shape
  const int i = idx % ci2, o = (idx / ci2) % co2, t = idx / (ci2 * co2);
  const float w = flip ? Wf[((26 - t) * cout + i) * cin + o] : Wf[(t * cout + o) * cin + i];
  Wc[conv_weight_index(t, o, i, ci2, co2)] = __float2bfloat16(w);
}

// The same from BF16 [27][cout][cin] weights, not flipped.
__global__ void k_pack_conv_weights_bf16(const __nv_bfloat16* __restrict__ W, int cin, int cout,
                                         __nv_bfloat16* __restrict__ Wc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 27 * cin * cout) return;
  const int i = idx % cin, o = (idx / cin) % cout, t = idx / (cin * cout);
  Wc[conv_weight_index(t, o, i, cin, cout)] = W[idx];
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
