// Restarted GMRES(m) for the assembled complex-symmetric system (the paper solves it with
// PETSc's GMRES, Section 5.1), right-preconditioned by Jacobi.
//
// Right Jacobi preconditioning is a column scaling: with D = diag(A) and Ahat = A D^{-1}
// (stored once), the solver iterates on Ahat u = b and returns x = D^{-1} u.
//
// Precision:
//   c128: Krylov vectors and Ahat in complex128, all arithmetic FP64.
//   mixed: Krylov vectors and Ahat in complex64; every cycle restarts from the residual
//     b - Ahat u computed in FP64 with u in complex128 (iterative refinement: each GMRES cycle
//     solves for a correction, added to u in FP64).  Dot products take FP32 products over 8
//     rows per thread and sum everything across threads in FP64.
//
// Arnoldi with classical Gram-Schmidt and a conditional second pass: after w <- w - V (V^H w),
// the pass is repeated when ||w|| fell below eta * ||w_before|| (eta = 1/sqrt(2)).
// Each Krylov vector V_k is stored unnormalised with its scale 1/||V_k|| on the device, so no
// separate normalisation pass is needed.  The Hessenberg column, its Givens rotations and the
// stopping test run in the last block of each reduction kernel: a cycle of m iterations needs
// no host synchronisation, and kernels after the stop return at once.
#include <math.h>

#include <algorithm>

#include "krylov.cuh"
#include "learned.cuh"

namespace petgem {

namespace {

// ------------------------------------------------------------------ kernels
// Output scaling of the Arnoldi SpMV.  complex64: FP32 only (no FP64 instruction in the kernel:
// on this GPU a single FP64 multiply per row costs as much as the row's memory traffic).
template <typename T> __device__ inline T scale_out(typename Acc<T>::type acc, const GState* st, int j);
template <> __device__ inline float2 scale_out<float2>(float2 acc, const GState* st, int j) {
  const float s = st->inv_beta32[j];
  return make_float2(acc.x * s, acc.y * s);
}
template <> __device__ inline double2 scale_out<double2>(double2 acc, const GState* st, int j) {
  const double s = st->inv_beta[j];
  return make_double2(acc.x * s, acc.y * s);
}

// y = (Ahat x) * scale, G lanes per row.  x = V_j, y = V_{j+1}, scale = 1/||V_j||.
template <typename T, int G>
__global__ void __launch_bounds__(256) k_spmv_arnoldi(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const T* __restrict__ val, const T* __restrict__ x,
                                                      T* __restrict__ y, int64_t n, const GState* __restrict__ st,
                                                      int j) {
  if (st->done) return;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t row = gid / G;
  int lane = (int)(gid % G);
  typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
  if (row < n) {
    const int64_t p1 = rp[row + 1];
    int64_t p = rp[row] + lane;
    for (; p + G < p1; p += 2 * G) {  // two entries per lane in flight
      const int32_t c0 = __ldg(&col[p]), c1 = __ldg(&col[p + G]);
      const T a0 = __ldg(&val[p]), a1 = __ldg(&val[p + G]);
      fma_c(acc, a0, __ldg(&x[c0]));
      fma_c(acc2, a1, __ldg(&x[c1]));
    }
    if (p < p1) fma_c(acc, __ldg(&val[p]), __ldg(&x[__ldg(&col[p])]));
  }
  acc.x += acc2.x;
  acc.y += acc2.y;
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) y[row] = scale_out<T>(acc, st, j);
}

// r = b - Ahat u in FP64 (complex128 matrix and vectors).
template <int G>
__global__ void __launch_bounds__(256) k_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                  const double2* __restrict__ val, const double2* __restrict__ u,
                                                  const double2* __restrict__ b, double2* __restrict__ r, int64_t n) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t row = gid / G;
  int lane = (int)(gid % G);
  double2 acc = make_double2(0.0, 0.0);
  if (row < n) {
    int64_t p1 = rp[row + 1];
    for (int64_t p = rp[row] + lane; p < p1; p += G) fma_c(acc, val[p], u[col[p]]);
  }
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) r[row] = csub(b[row], acc);
}

// Cycle start: V_0 = r (rounded to T), ||r||^2 in FP64, ||V_0||^2, then (last block) the
// Arnoldi state: g = (||V_0||, 0, ...), 1/||V_0||, stop threshold.
template <typename T>
__global__ void __launch_bounds__(kT) k_cycle_init(const double2* __restrict__ r, T* __restrict__ V0, int64_t n,
                                                   GState* __restrict__ st, double2* __restrict__ partials,
                                                   double tol_abs, double inner_rel) {
  __shared__ double2 red[kT / 32];
  __shared__ double2 fin[2];
  double rr = 0.0, vv = 0.0;
  int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    if (i < n) {
      double2 v = r[i];
      T t = from_d2<T>(v);
      V0[i] = t;
      rr += nrm2(v);
      vv += nrm2(to_d2(t));
    }
  }
  double2 a = warp_sum(make_double2(rr, vv));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < kT / 32; ++w) s = cadd(s, red[w]);
    partials[(int64_t)blockIdx.x * kPStride] = s;
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, 1, fin);
  if (threadIdx.x == 0) {
    double r2 = fin[0].x, v2 = fin[0].y;
    st->rnorm2 = r2;
    double b0 = sqrt(v2);
    st->beta0 = b0;
    st->g[0] = make_double2(b0, 0.0);
    for (int i = 1; i <= kMaxM; ++i) st->g[i] = make_double2(0.0, 0.0);
    st->inv_beta[0] = b0 > 0.0 ? 1.0 / b0 : 0.0;
    st->inv_beta32[0] = (float)st->inv_beta[0];
    st->k = 0;
    st->refine = 0;
    st->n_refine = 0;
    for (int i = 0; i < kMaxM; ++i) st->refined[i] = 0;
    st->stop_abs = fmax(tol_abs, inner_rel * sqrt(r2));
    // Converged before the first step (FP64 residual already small), nothing to do, or not finite.
    if (!isfinite(r2) || !isfinite(b0))
      st->done = 2;
    else
      st->done = (b0 > 0.0 && sqrt(r2) > tol_abs) ? 0 : 1;
    st->counter = 0;
  }
}

// ------------------------------------------------------------------ TMA-staged Gram-Schmidt
// One persistent kernel, three modes, for classical Gram-Schmidt with one re-orthogonalisation
// (CGS2) of w = V_{j+1} against V_0..V_j:
//   mode 0: h1 = V^H w, ||w||^2
//   mode 1: w <- w - V c1 (c1 = h1 scaled), then h2 = V^H w on the updated w
//   mode 2: w <- w - V c2, ||w||^2; the last block finishes the Hessenberg column
// so V is read three times per Arnoldi step.  Each block walks row tiles; for a tile, one thread
// issues a 1-D bulk copy (cp.async.bulk, completion on an mbarrier) of every vector's 2 KB slice
// into shared memory, double-buffered so the next tile streams in while this one is used.  Rows
// per tile: 128 (complex64) or 64 (complex128).  ld is a multiple of 256 elements, so every slice
// is whole and 16-byte aligned; rows >= n are zero padding.  Two blocks per SM hide each other's
// waits; each block double-buffers its own tiles.
constexpr int kMaxSlice = 2048;   // largest per-vector slice of a row tile (bytes)
constexpr int kSlicePad = 16;     // pad between slices: shifts shared-memory banks, keeps 16-byte alignment
constexpr int kMaxStages = 4;
constexpr int kCgsThreads = 256;
constexpr int kCgsBlocksPerSM = 2;
// Dynamic shared memory per block: two blocks per SM must fit in the SM's 228 KB together with
// their ~5 KB of static shared memory and the 1 KB each block reserves.
constexpr int kCgsDynSmem = 105 * 1024;
constexpr int kCgsRedBytes = (kCgsThreads / 32) * 64 * 16;  // end-of-kernel reduction, aliased on the stages
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s: no copy takes that long

// Slice size and stage count for nv staged vectors: 1 KB slices, double-buffered (the fastest
// measured shape on this GPU; deeper staging with smaller slices lost more to per-tile overhead).
struct CgsShape {
  int slice, stages;
};
inline CgsShape cgs_shape(int nv) {
  const int st = kCgsDynSmem / (nv * (1024 + kSlicePad));
  return CgsShape{1024, st >= 2 ? 2 : 1};
}

// ------------------------------------------------------------------ projections (dot pass)
// h = V^H w and ||w||^2 for w = V_{j+1}: each thread keeps kR rows of w in registers and streams
// the basis two vectors at a time (2 kR independent loads in flight), high occupancy.  complex64:
// FP32 products over the thread's rows and an FP32 tree over the warp (256 rows); the warp totals
// are turned into FP64 only at the end, and everything across warps and blocks is FP64.
template <typename T>
__global__ void __launch_bounds__(kT) k_mdot(const T* __restrict__ V, int64_t ld, int64_t n, int j,
                                             GState* __restrict__ st, double2* __restrict__ partials) {
  if (st->done) return;
  using A = typename Acc<T>::type;
  __shared__ A red[kMaxM + 2][kT / 32];
  __shared__ double2 fin[kMaxM + 2];
  const int nk = j + 1, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* w = V + (int64_t)(j + 1) * ld;
  const int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
  T wr[kR];
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    const int64_t i = base + (int64_t)q * kT;
    wr[q] = i < n ? w[i] : zero<T>();
  }
  auto warp_tree = [&](A a) {
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    return a;
  };
  {
    A a = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) a.x += nrm2(wr[q]);
    a = warp_tree(a);
    if (lane == 0) red[nk][wid] = a;
  }
  int k = 0;
  for (; k + 1 < nk; k += 2) {
    const T* v0 = V + (int64_t)k * ld;
    const T* v1 = v0 + ld;
    T a0[kR], a1[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      const int64_t i = base + (int64_t)q * kT;
      a0[q] = i < n ? v0[i] : zero<T>();
      a1[q] = i < n ? v1[i] : zero<T>();
    }
    A s0 = zero<T>(), s1 = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      fma_conj(s0, a0[q], wr[q]);
      fma_conj(s1, a1[q], wr[q]);
    }
    s0 = warp_tree(s0);
    s1 = warp_tree(s1);
    if (lane == 0) {
      red[k][wid] = s0;
      red[k + 1][wid] = s1;
    }
  }
  for (; k < nk; ++k) {
    const T* v0 = V + (int64_t)k * ld;
    A s0 = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      const int64_t i = base + (int64_t)q * kT;
      if (i < n) fma_conj(s0, v0[i], wr[q]);
    }
    s0 = warp_tree(s0);
    if (lane == 0) red[k][wid] = s0;
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk <= nk; kk += kT) {
    double2 sum = make_double2(0.0, 0.0);
    for (int ww = 0; ww < kT / 32; ++ww) sum = cadd(sum, to_d2(red[kk][ww]));
    partials[(int64_t)blockIdx.x * kPStride + kk] = sum;
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, nk + 1, fin);
  for (int kk = threadIdx.x; kk < nk; kk += kT) {
    const double ib = st->inv_beta[kk];
    const double2 h = cscale(fin[kk], ib);  // v_k^H w with v_k = V_k / ||V_k||
    st->h[kk] = h;
    st->c[kk] = cscale(h, ib);              // w -= V_k * (h_k / ||V_k||)
  }
  if (threadIdx.x == 0) {
    st->nrm_w = fin[nk].x;
    st->counter = 0;
  }
}

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false if the phase did not complete within kWaitLimitNs.
__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}
__device__ inline void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kCgsThreads, kCgsBlocksPerSM) k_cgs(T* __restrict__ V, int64_t ld, int64_t n, int j,
                                                        GState* __restrict__ st, double2* __restrict__ partials,
                                                        int n_tiles, int slice, int n_stages, int pass,
                                                        int need_refine, double eta2) {
  if (st->done || (need_refine && !st->refine)) return;
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ uint64_t bar[kMaxStages];
  __shared__ T cs[kMaxM + 1];
  __shared__ double2 fin[kMaxM + 2];
  __shared__ __align__(16) unsigned char wraw[kMaxSlice];  // updated w of the tile (never a copy target)
  __shared__ bool aborted;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int nwarps = kCgsThreads / 32;
  T* wbuf = (T*)wraw;
  const int TR = slice / (int)sizeof(T);  // rows per tile: 32..256, a power of two
  const int stride = slice + kSlicePad;
  const int nv = j + 2;                   // staged slices: V_0..V_j and w = V_{j+1}
  const size_t stage_bytes = (size_t)nv * stride;
  const int my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int i = 0; i < n_stages; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    aborted = false;
  }
  if (MODE != 0)
    for (int k = tid; k <= j; k += kCgsThreads) cs[k] = from_d2<T>(st->c[k]);
  __syncthreads();
  auto issue = [&](int it) {
    const int sidx = it % n_stages;
    const int64_t r0 = (int64_t)(blockIdx.x + (int64_t)it * gridDim.x) * TR;
    unsigned char* base = stage_mem + sidx * stage_bytes;
    mbar_expect_tx(&bar[sidx], (unsigned)(nv * slice));
    for (int k = 0; k < nv; ++k) bulk_g2s(base + (size_t)k * stride, V + (int64_t)k * ld + r0, slice, &bar[sidx]);
  };
  if (tid == 0)
    for (int it = 0; it < n_stages && it < my_tiles; ++it) issue(it);
  // Update mode: one thread per row (threads beyond TR rows idle: fewer instructions measured faster
  // than sharing a row between threads).
  const int split = 1;
  const int urow = tid, usub = 0;
  typename Acc<T>::type a_hi = zero<T>();
  typename Acc<T>::type f0 = zero<T>(), f1 = zero<T>();  // FP32 (complex64) running sums of the slots
  double2 acc0 = make_double2(0.0, 0.0), acc1 = make_double2(0.0, 0.0);
  double nrm = 0.0;
  const int k0 = lane, k1 = lane + 32;
  const bool has0 = k0 <= j + 1, has1 = k1 <= j + 1;
  for (int it = 0; it < my_tiles; ++it) {
    const int sidx = it % n_stages;
    const unsigned parity = (unsigned)((it / n_stages) & 1);
    if (!mbar_wait(&bar[sidx], parity)) aborted = true;
    __syncthreads();
    if (aborted) break;
    // Staged slices are only ever written by the bulk copies; the updated w goes to wbuf.
    const unsigned char* base = stage_mem + sidx * stage_bytes;
    const T* ws = (const T*)(base + (size_t)(j + 1) * stride);
    const int64_t r0 = (int64_t)(blockIdx.x + (int64_t)it * gridDim.x) * TR;
    if (MODE != 0) {  // w -= sum_k V_k c_k, rows over threads (split threads per row for short tiles)
      if (urow < TR) {
        T w = usub == 0 ? ws[urow] : zero<T>(), w2 = zero<T>();
        int k = usub;
        for (; k + split <= j; k += 2 * split) {  // two independent chains
          sub_mul(w, ((const T*)(base + (size_t)k * stride))[urow], cs[k]);
          sub_mul(w2, ((const T*)(base + (size_t)(k + split) * stride))[urow], cs[k + split]);
        }
        if (k <= j) sub_mul(w, ((const T*)(base + (size_t)k * stride))[urow], cs[k]);
        w.x += w2.x;
        w.y += w2.y;
        for (int o = 1; o < split; o <<= 1) {  // the split threads are adjacent lanes
          w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
          w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
        }
        const int64_t r = r0 + urow;
        if (usub == 0) {
          if (r < n) {
            V[(int64_t)(j + 1) * ld + r] = w;
            if (MODE == 2) a_hi.x += nrm2(w);
          }
          if (MODE == 1) wbuf[urow] = w;
        }
      }
      __syncthreads();
    }
    if (MODE != 2) {  // lane owns slots k0 and k1 (slot j + 1 is ||w||^2); rows staggered by lane
      const T* wsrc = MODE == 0 ? ws : wbuf;
      const T* v0 = (const T*)(base + (size_t)k0 * stride);
      const T* v1 = (const T*)(base + (size_t)k1 * stride);
      const int mask = TR - 1;
      typename Acc<T>::type t0 = zero<T>(), t1 = zero<T>();  // second row of each pair
      for (int r = wid; r < TR; r += 2 * nwarps) {
        const int ra = (r + lane) & mask, rb = (r + nwarps + lane) & mask;
        const T wa = wsrc[ra], wb = wsrc[rb];
        if (has0) {
          fma_conj(f0, v0[ra], wa);
          fma_conj(t0, v0[rb], wb);
        }
        if (has1) {
          fma_conj(f1, v1[ra], wa);
          fma_conj(t1, v1[rb], wb);
        }
      }
      f0.x += t0.x;
      f0.y += t0.y;
      f1.x += t1.x;
      f1.y += t1.y;
      if ((it & 3) == 3) {  // FP32 sums over at most 4 tiles (<= 128 rows per lane), then FP64
        acc0 = cadd(acc0, to_d2(f0));
        acc1 = cadd(acc1, to_d2(f1));
        f0 = zero<T>();
        f1 = zero<T>();
      }
    } else if ((it & 7) == 7) {  // flush the FP32 norm every 8 tiles (<= 8 rows per thread)
      nrm += (double)a_hi.x;
      a_hi = zero<T>();
    }
    __syncthreads();  // every thread is done with this stage
    if (tid == 0 && it + n_stages < my_tiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(it + n_stages);
    }
  }
  if (aborted) {
    // Give the copies still in flight a bounded chance to land before the block's shared memory
    // is released, report, and leave the rest of the cycle to skip.
    if (tid == 0) {
      for (int sidx = 0; sidx < n_stages; ++sidx) mbar_wait(&bar[sidx], 0), mbar_wait(&bar[sidx], 1);
      st->timeout = 1;
      atomicExch(&st->done, 2);
    }
    return;
  }
  nrm += (double)a_hi.x;
  acc0 = cadd(acc0, to_d2(f0));
  acc1 = cadd(acc1, to_d2(f1));
  // Every issued copy has been waited for, so the stage memory is free for the block reduction.
  double2(*red)[64] = reinterpret_cast<double2(*)[64]>(stage_mem);
  if (MODE != 2) {
    red[wid][k0] = acc0;
    red[wid][k1] = acc1;
  } else {
    double t = warp_sum(nrm);
    if (lane == 0) red[wid][0] = make_double2(t, 0.0);
  }
  __syncthreads();
  const int nslots = MODE == 2 ? 1 : j + 2;
  for (int k = tid; k < nslots; k += kCgsThreads) {
    double2 sum = make_double2(0.0, 0.0);
    for (int w2 = 0; w2 < nwarps; ++w2) sum = cadd(sum, red[w2][k]);
    partials[(int64_t)blockIdx.x * kPStride + k] = sum;
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, nslots, fin);
  if (MODE == 0) {
    for (int k = tid; k <= j; k += kCgsThreads) {
      const double ib = st->inv_beta[k];
      const double2 h = cscale(fin[k], ib);
      if (pass == 0)
        st->h[k] = h;
      else
        st->h2[k] = h;
      st->c[k] = cscale(h, ib);
    }
    if (tid == 0) {
      if (pass == 0) st->nrm_w = fin[j + 1].x;
      st->counter = 0;
    }
  } else if (MODE == 1) {
    for (int k = tid; k <= j; k += kCgsThreads) {
      const double ib = st->inv_beta[k];
      const double2 h = cscale(fin[k], ib);
      st->h2[k] = h;
      st->c[k] = cscale(h, ib);
    }
    if (tid == 0) st->counter = 0;
  } else {
    // pass 0 with eta2 > 0: keep this single pass only if ||w|| kept more than eta of its norm.
    if (pass == 0 && eta2 > 0.0 && fin[0].x < eta2 * st->nrm_w) {
      if (tid == 0) {
        st->refine = 1;
        st->counter = 0;
      }
      return;
    }
    __shared__ double2 hsum[kMaxM + 1];
    for (int k = tid; k <= j; k += kCgsThreads) hsum[k] = pass == 1 ? cadd(st->h[k], st->h2[k]) : st->h[k];
    __syncthreads();
    if (tid == 0) {
      finish_column(st, j, hsum, fin[0].x);
      if (pass == 1) {
        st->refined[j] = 1;
        st->n_refine += 1;
      }
      st->refine = 0;
      st->counter = 0;
    }
  }
}

// y = H(0:k, 0:k)^{-1} g(0:k), scaled by 1/||V_i|| for the unnormalised basis.  One warp:
// column-oriented back substitution (lane l keeps the running right-hand side of rows l, l+32).
__global__ void k_backsolve(GState* st) { backsolve_warp(st, threadIdx.x); }

// u += sum_k V_k y_k.  complex128: in FP64.  complex64: the correction sum_k V_k y_k is formed in
// FP32 (it is the inner solve's correction, accurate to complex64 anyway) and added to u in FP64.
template <typename T>
__global__ void __launch_bounds__(kT) k_xupdate(const T* __restrict__ V, int64_t ld, int64_t n,
                                                double2* __restrict__ u, const GState* __restrict__ st) {
  __shared__ T ys[kMaxM];
  const int kk = st->done == 2 ? 0 : st->k;  // a failed cycle leaves u untouched
  for (int k = threadIdx.x; k < kk; k += kT) ys[k] = from_d2<T>(st->y[k]);
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x;
  if (i >= n || kk == 0) return;
  typename Acc<T>::type acc = zero<T>();
  for (int k = 0; k < kk; ++k) fma_c(acc, V[(int64_t)k * ld + i], ys[k]);
  u[i] = cadd(u[i], to_d2(acc));
}

__global__ void k_scale_in(const double2* __restrict__ x, const double2* __restrict__ d, double2* __restrict__ u,
                           int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] = cmul(d[i], x[i]);
}
__global__ void k_scale_out(const double2* __restrict__ u, const double2* __restrict__ d, double2* __restrict__ x,
                            int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = cdiv(u[i], d[i]);
}

// Ahat = A D^{-1} (column scaling) in complex128 and its complex64 rounding.
__global__ void k_scale_matrix(const double2* __restrict__ val, const int32_t* __restrict__ col,
                               const double2* __restrict__ d, int64_t nnz, double2* __restrict__ a128,
                               float2* __restrict__ a64) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  double2 a = cdiv(val[p], d[col[p]]);
  a128[p] = a;
  a64[p] = make_float2((float)a.x, (float)a.y);
}

// Plain y = A x (complex128) for the public SpMV entry point.
template <int G>
__global__ void __launch_bounds__(256) k_spmv_plain(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                    const double2* __restrict__ val, const double2* __restrict__ x,
                                                    double2* __restrict__ y, int64_t n) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t row = gid / G;
  int lane = (int)(gid % G);
  double2 acc = make_double2(0.0, 0.0);
  if (row < n) {
    int64_t p1 = rp[row + 1];
    for (int64_t p = rp[row] + lane; p < p1; p += G) fma_c(acc, val[p], x[col[p]]);
  }
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) y[row] = acc;
}

// ||b||^2 in FP64 (last-block reduction into st->rnorm2).
__global__ void __launch_bounds__(kT) k_norm2(const double2* __restrict__ b, int64_t n, GState* __restrict__ st,
                                              double2* __restrict__ partials) {
  __shared__ double red[kT / 32];
  __shared__ double2 fin[1];
  double s = 0.0;
  int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    if (i < n) s += nrm2(b[i]);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    partials[(int64_t)blockIdx.x * kPStride] = make_double2(t, 0.0);
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, 1, fin);
  if (threadIdx.x == 0) {
    st->rnorm2 = fin[0].x;
    st->counter = 0;
  }
}


// ------------------------------------------------------------------ host side

Status read_state(petgem_ctx* c, HostState* hs) {
  Solver* S = c->solver;
  PG_CUDA(cudaMemcpyAsync(hs, S->state.ptr, sizeof(HostState), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return Status{};
}

// Scaled matrices (once per assembly) and device facts; then, for the single-source driver, its
// workspaces.  The multi-source driver (block.cu) sizes its own.
Status prepare(petgem_ctx* c, int m, int prec, bool single) {
  if (!c->solver) c->solver = new Solver();
  Solver* S = c->solver;
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  if (S->version != c->assembly_version) {
    PG_TRY(S->ahat128.reserve(c->nnz * sizeof(double2)));
    PG_TRY(S->ahat64.reserve(c->nnz * sizeof(float2)));
    k_scale_matrix<<<blocks_for(c->nnz, 256), 256, 0, s>>>(c->val.as<double2>(), c->col.as<int32_t>(),
                                                          c->diag.as<double2>(), c->nnz, S->ahat128.as<double2>(),
                                                          S->ahat64.as<float2>());
    c->launches++;
    PG_CUDA(cudaGetLastError());
    S->version = c->assembly_version;
  }
  if (S->sms == 0) {
    PG_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, c->device));
    for (auto f : {(const void*)k_cgs<float2, 0>, (const void*)k_cgs<float2, 1>, (const void*)k_cgs<float2, 2>,
                   (const void*)k_cgs<double2, 0>, (const void*)k_cgs<double2, 1>, (const void*)k_cgs<double2, 2>})
      PG_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kCgsDynSmem));
  }
  S->n = n;
  S->ld = (n + 255) / 256 * 256;  // whole slices for the staged Gram-Schmidt kernel
  S->m = m;
  S->n_blocks = (n + kRows - 1) / kRows;
  if (!single) return Status{};
  const size_t vbytes_all = (size_t)(m + 1) * S->ld * (prec == PETGEM_PREC_MIXED ? sizeof(float2) : sizeof(double2));
  // The staged Gram-Schmidt kernel reads whole slices, so the rows n..ld-1 of every basis vector
  // must be zero.  Kernels never write them, but complex64 and complex128 vectors place their
  // padding at different byte offsets: clear the buffer when it grows or the layout changes.
  const bool fresh = S->V.bytes < vbytes_all || S->prec != prec || S->ld_used != S->ld;
  PG_TRY(S->V.reserve(vbytes_all));
  if (fresh) PG_CUDA(cudaMemsetAsync(S->V.ptr, 0, S->V.bytes, s));
  S->prec = prec;
  S->ld_used = S->ld;
  // Partials: one row per block of the widest reduction grid (vector kernels: n_blocks; the
  // persistent Gram-Schmidt kernel: two blocks per SM).
  PG_TRY(S->partials.reserve((size_t)std::max<int64_t>(std::max<int64_t>(S->n_blocks, kCgsBlocksPerSM * S->sms), 1) *
                             kPStride * sizeof(double2)));
  PG_TRY(S->u.reserve(n * sizeof(double2)));
  PG_TRY(S->r.reserve(n * sizeof(double2)));
  PG_TRY(S->state.reserve(sizeof(GState)));
  PG_CUDA(cudaMemsetAsync(S->state.ptr, 0, sizeof(GState), s));
  return Status{};
}

template <typename T>
Status run_cycle(petgem_ctx* c, const T* ahat, int m, int orth, double tol_abs, double inner_rel, bool learned,
                 HostState* hs) {
  Solver* S = c->solver;
  cudaStream_t s = c->stream;
  const int64_t n = S->n, ld = S->ld;
  T* V = S->V.as<T>();
  GState* st = S->state.as<GState>();
  double2* part = S->partials.as<double2>();
  const unsigned nb = (unsigned)S->n_blocks;
  const double vbytes = (double)sizeof(T) * n;
  const bool c128 = sizeof(T) == 16;
  const size_t pending0 = c->pending.size();
  {
    KernelTimer kt(c, c128 ? "cycle_init_c128" : "cycle_init_c64", 16.0 * n + vbytes);
    k_cycle_init<T><<<nb, kT, 0, s>>>(S->r.as<double2>(), V, n, st, part, tol_abs, inner_rel);
    c->launches++;
  }
  const double spmv_bytes = (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 2.0 * vbytes;
  const unsigned spmv_blocks = blocks_for(n * kGroup, 256);
  // Flexible GMRES with the learned preconditioner: z_j = N-corrected v_j, stored in Z, and the
  // solution update uses Z instead of V.
  T* Z = learned ? S->Z.as<T>() : nullptr;
  for (int j = 0; j < m; ++j) {
    T* vj = V + (int64_t)j * ld;
    T* vn = vj + ld;
    const T* xin = vj;
    if (learned) {  // odd steps: the network's direction; even steps: Jacobi (z = v)
      T* zj = Z + (int64_t)j * ld;
      if (j & 1) {
        KernelTimer kt(c, "learned_apply", 0.0, j, 0);
        PG_TRY(c->net->apply<T>(s, vj, c->slots.as<int32_t>(), n, zj));
        c->launches += 20;
      } else {
        PG_CUDA(cudaMemcpyAsync(zj, vj, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      }
      xin = zj;
    }
    {
      KernelTimer kt(c, c128 ? "spmv_c128" : "spmv_c64", spmv_bytes, j, 0);
      k_spmv_arnoldi<T, kGroup><<<spmv_blocks, 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), ahat, xin,
                                                            vn, n, st, j);
    }
    const int nv = j + 2;
    const CgsShape shp = cgs_shape(nv);
    const size_t dyn = std::max<size_t>((size_t)shp.stages * nv * (shp.slice + kSlicePad), kCgsRedBytes);
    const int tiles = (int)(ld * sizeof(T) / shp.slice);
    const unsigned grid = (unsigned)std::min(tiles, kCgsBlocksPerSM * S->sms);
    const int64_t wb = (int64_t)vbytes;
    auto cgs = [&](int mode, int pass, int need_refine, double eta2, const char* name, double bytes, int tag) {
      KernelTimer kt(c, name, bytes, j, tag);
      if (mode == 0)
        k_cgs<T, 0><<<grid, kCgsThreads, dyn, s>>>(V, ld, n, j, st, part, tiles, shp.slice, shp.stages, pass, need_refine, eta2);
      else if (mode == 1)
        k_cgs<T, 1><<<grid, kCgsThreads, dyn, s>>>(V, ld, n, j, st, part, tiles, shp.slice, shp.stages, pass, need_refine, eta2);
      else
        k_cgs<T, 2><<<grid, kCgsThreads, dyn, s>>>(V, ld, n, j, st, part, tiles, shp.slice, shp.stages, pass, need_refine, eta2);
      c->launches++;
    };
    const double dot_b = (double)(j + 2) * wb, upd_b = (double)(j + 3) * wb;
    auto mdot = [&]() {
      KernelTimer kt(c, c128 ? "mdot_c128" : "mdot_c64", dot_b, j, 0);
      k_mdot<T><<<nb, kT, 0, s>>>(V, ld, n, j, st, part);
      c->launches++;
    };
    if (orth == 0) {  // CGS2: dots, update + dots, update + norm
      mdot();
      cgs(1, 0, 0, 0.0, c128 ? "cgs_upd_dot_c128" : "cgs_upd_dot_c64", upd_b, 0);
      cgs(2, 1, 0, 0.0, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0);
    } else if (orth == 1) {  // CGS: dots, update + norm
      mdot();
      cgs(2, 0, 0, 0.0, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0);
    } else {  // CGS, second pass when the norm fell below 1/sqrt(2) of its value
      mdot();
      cgs(2, 0, 0, 0.5, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0);
      cgs(0, 1, 1, 0.0, c128 ? "cgs_dot2_c128" : "cgs_dot2_c64", dot_b, 1);
      cgs(2, 1, 1, 0.0, c128 ? "cgs_upd2_c128" : "cgs_upd2_c64", upd_b, 1);
    }
    c->launches += 1;
  }
  PG_CUDA(cudaGetLastError());
  k_backsolve<<<1, 32, 0, s>>>(st);
  {
    KernelTimer kt(c, c128 ? "xupdate_c128" : "xupdate_c64", 32.0 * n + (double)m * vbytes);
    k_xupdate<T><<<blocks_for(n, kT), kT, 0, s>>>(learned ? Z : V, ld, n, S->u.as<double2>(), st);
  }
  c->launches += 2;
  PG_CUDA(cudaGetLastError());
  PG_TRY(read_state(c, hs));
  if (c->profiling) drop_idle_timings(c, pending0, hs->done == 2 ? 0 : hs->k, hs->refined);
  return Status{};
}

}  // namespace

void destroy_solver(petgem_ctx* c) {
  if (!c->solver) return;
  Solver* S = c->solver;
  S->ahat128.release();
  S->ahat64.release();
  S->dinv.release();
  S->V.release();
  S->u.release();
  S->r.release();
  S->partials.release();
  S->state.release();
  delete S;
  c->solver = nullptr;
}

Status run_spmv(petgem_ctx* c, const double2* x, double2* y) {
  k_spmv_plain<kGroup><<<blocks_for(c->n_edges * kGroup, 256), 256, 0, c->stream>>>(
      c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->val.as<double2>(), x, y, c->n_edges);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status run_solve(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info) {
  const int m = o.restart;
  if (m < 1 || m > kMaxRestart) return Status{PETGEM_ERR_UNSUPPORTED, "restart must be in [1, 62]"};
  const bool block = o.batch != 1 && c->n_src > 1 && o.precond != PETGEM_PRECOND_LEARNED;
  PG_TRY(prepare(c, m, o.precision, !block));
  if (block) return run_solve_block(c, o, x, info);
  Solver* S = c->solver;
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  GState* st = S->state.as<GState>();
  double2* part = S->partials.as<double2>();
  const unsigned nb = (unsigned)S->n_blocks;
  const unsigned rb = blocks_for(n * kGroup, 256);
  Status worst;
  for (int32_t src = 0; src < c->n_src; ++src) {
    petgem_solve_info& inf = info[src];
    inf = petgem_solve_info{};
    const double2* b = c->b.as<double2>() + (int64_t)src * n;
    double2* xs = x + (int64_t)src * n;
    HostState hs;
    k_norm2<<<nb, kT, 0, s>>>(b, n, st, part);
    c->launches++;
    PG_TRY(read_state(c, &hs));
    const double bnorm = sqrt(hs.rnorm2);
    if (bnorm == 0.0) {
      PG_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double2), s));
      inf.status = PETGEM_OK;
      continue;
    }
    k_scale_in<<<blocks_for(n, 256), 256, 0, s>>>(xs, c->diag.as<double2>(), S->u.as<double2>(), n);
    c->launches++;
    int64_t iters = 0, cycles = 0, reorth = 0;
    int status = PETGEM_OK;
    double relres = 0.0, prev_relres = 0.0;
    // Learned preconditioner: the first cycle runs with Jacobi and measures its residual reduction
    // per cycle; learned cycles follow while each reduces the FP64 residual more than that.
    bool want_learned = o.precond == PETGEM_PRECOND_LEARNED;
    bool learned = false;
    double jacobi_rate = -1.0;
    int fell_back = 0;
    if (want_learned) {
      PG_TRY(S->Z.reserve((size_t)m * S->ld * (o.precision == PETGEM_PREC_MIXED ? sizeof(float2) : sizeof(double2))));
      PG_TRY(S->usave.reserve(n * sizeof(double2)));
      PG_TRY(c->net->features(s, c->sigma.as<double>(), c->sigma_p, c->omega, c->lattice_h));
    }
    bool prev_learned = false;
    auto residual = [&]() -> Status {
      KernelTimer kt(c, "residual_c128", (double)c->nnz * 20 + 8.0 * (n + 1) + 48.0 * n);
      k_residual<kGroup><<<rb, 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), S->ahat128.as<double2>(),
                                            S->u.as<double2>(), b, S->r.as<double2>(), n);
      c->launches++;
      PG_CUDA(cudaGetLastError());
      return Status{};
    };
    while (true) {
      PG_TRY(residual());
      if (want_learned && cycles > 0) {
        k_norm2<<<nb, kT, 0, s>>>(S->r.as<double2>(), n, st, part);
        c->launches++;
        PG_TRY(read_state(c, &hs));
        const double rate = sqrt(hs.rnorm2) / bnorm / prev_relres;
        if (prev_learned && !(rate < jacobi_rate)) {
          // the learned cycle just run did no better than a Jacobi cycle: undo it, stay with Jacobi
          PG_CUDA(cudaMemcpyAsync(S->u.ptr, S->usave.ptr, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
          PG_TRY(residual());
          want_learned = false;
          fell_back = 1;
        } else if (!prev_learned && jacobi_rate < 0.0) {
          jacobi_rate = rate;
        }
      }
      learned = want_learned && jacobi_rate >= 0.0;
      if (learned) PG_CUDA(cudaMemcpyAsync(S->usave.ptr, S->u.ptr, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
      const int mj = (int)std::min<int64_t>(m, std::max<int64_t>(o.max_iters - iters, 0));
      const double tol_abs = o.tol * bnorm;
      // Learned cycles always re-orthogonalise: the network's directions can be nearly dependent.
      const int orth = learned ? PETGEM_ORTH_CGS2 : o.orth;
      // A cycle whose starting residual already meets tol runs no iteration (k = 0).
      if (o.precision == PETGEM_PREC_MIXED)
        PG_TRY(run_cycle<float2>(c, S->ahat64.as<float2>(), mj, orth, tol_abs, o.inner_tol, learned, &hs));
      else
        PG_TRY(run_cycle<double2>(c, S->ahat128.as<double2>(), mj, orth, tol_abs, 0.0, learned, &hs));
      relres = sqrt(hs.rnorm2) / bnorm;  // FP64 residual of u before this cycle's update
      if (!isfinite(relres)) {
        status = PETGEM_ERR_BREAKDOWN;
        break;
      }
      if (relres <= o.tol) break;
      if (mj == 0) {
        status = PETGEM_ERR_NOT_CONVERGED;
        break;
      }
      iters += hs.k;
      cycles += 1;
      reorth += hs.n_refine;
      prev_learned = learned;
      prev_relres = relres;
      if (hs.done == 2) {  // u was left as it was before this cycle
        status = hs.timeout ? PETGEM_ERR_TIMEOUT : PETGEM_ERR_BREAKDOWN;
        break;
      }
    }
    k_scale_out<<<blocks_for(n, 256), 256, 0, s>>>(S->u.as<double2>(), c->diag.as<double2>(), xs, n);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    inf.iters = iters;
    inf.restarts = cycles;
    inf.refinements = cycles;
    inf.true_rel_residual = relres;
    inf.status = status;
    inf.reorth = (int32_t)std::min<int64_t>(reorth, INT32_MAX);
    inf.fell_back = fell_back;
    if (o.precond == PETGEM_PRECOND_LEARNED) PG_TRY(nn::check_err(s, c->net->err.as<int>(), "petgem_solve (learned)"));
    if (status != PETGEM_OK && worst.ok()) worst = Status{status, "source " + std::to_string(src) + " did not converge"};
  }
  PG_CUDA(cudaStreamSynchronize(s));
  return worst;
}

}  // namespace petgem
