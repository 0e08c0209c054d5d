// Classical Gram-Schmidt kernels over the Krylov basis: the projections h = V^H w (with ||w||^2)
// and the update w <- w - V c (with ||w||^2 and the new Hessenberg column), for one source
// (P = 1) or P interleaved sources (element (row i, source s) at i * P + s).
//
// Both are HBM-bound streams over j + 2 vectors, written with plain coalesced loads: on this GPU
// enough independent loads per thread keep the copy rate at the HBM limit, where a single
// bulk-copy (TMA) issuer per block did not (about three copies per microsecond per block).
//
// Projections (k_pdot): a persistent cooperative grid of two 512-thread blocks per SM; block b
// owns an even share of the rows.  For a tile of 512 x R elements every thread keeps its R
// elements of w in registers and streams the basis two vectors at a time (2R loads in flight),
// forming FP32 products over its R elements and a tree over the lanes of one source; per tile the
// block sums the warps in FP32 (one slot per warp for P = 1, shared-memory atomics over the
// sources otherwise) and then adds into FP64 registers.  After a grid
// barrier block b finishes slots b, b + G, ... in FP64 over the blocks, so the cross-block
// reduction is spread over every SM (FP64 runs at 1/58 of the FP32 rate on this part: one block
// reducing every slot would be a serial tail).
// Update (k_pupd): a persistent grid, one element per thread at a time, w -= sum_k c_k V_k with
// eight basis loads in flight; ||w||^2 in FP32 over at most 32 elements, then FP64; the last block
// to finish reduces ||w||^2 (parallel loads) and closes the Hessenberg column(s), one warp per
// source (finish_column_warp).
//
// The grid barrier is a 64-bit arrival counter that only grows; its wait is bounded
// (kGsWaitNs), after which the launch abandons the cycle with a timeout status.
#pragma once
#include "krylov.cuh"

namespace petgem {
namespace {

constexpr int kDotThreads = 512;
constexpr int kDotBlocksPerSM = 2;
constexpr int kUpdThreads = 512;
constexpr int kUpdBlocksPerSM = 2;
constexpr unsigned long long kGsWaitNs = 2000000000ull;  // 2 s

template <typename T> struct DotRows;  // elements per thread per tile
template <> struct DotRows<float2> { static constexpr int value = 8; };
template <> struct DotRows<double2> { static constexpr int value = 4; };

__device__ inline unsigned long long gs_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sums over the lanes that hold the same source (lane mod P).
template <int P>
__device__ inline float2 lane_tree(float2 a) {
#pragma unroll
  for (int o = 16; o >= P; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  return a;
}
template <int P>
__device__ inline double2 lane_tree(double2 a) {
#pragma unroll
  for (int o = 16; o >= P; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  return a;
}
template <int P>
__device__ inline float lane_tree(float a) {
#pragma unroll
  for (int o = 16; o >= P; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}
template <int P>
__device__ inline double lane_tree(double a) {
#pragma unroll
  for (int o = 16; o >= P; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

__device__ inline void red_add(float2* r, float2 a) {
  atomicAdd(&r->x, a.x);
  atomicAdd(&r->y, a.y);
}
__device__ inline void red_add(double2* r, double2 a) {
  atomicAdd(&r->x, a.x);
  atomicAdd(&r->y, a.y);
}

// A bounded wait gave up: abandon the cycle of every source of the launch.
template <int P>
__device__ inline void gs_fail(GState* sts, int* stop) {
  for (int s = 0; s < P; ++s) {
    sts[s].timeout = 1;
    atomicExch(&sts[s].done, 2);
  }
  if (P > 1) atomicExch(stop, 1);
}

// ------------------------------------------------------------------ projections
// h_s = V^H w_s (slots 0..j, scaled by 1 / ||V_k|| into h and c = h / ||V_k||) and ||w_s||^2
// (slot j + 1, kept as nrm_w on pass 0); pass 1 writes h2 instead of h.  Launched cooperatively
// (every block resident).  stop: the early-exit flag (the source's done, or the group's all_done);
// gbar: the grid barrier's arrival counter (0 when the state is cleared).
template <typename T, int P>
__global__ void __launch_bounds__(kDotThreads, kDotBlocksPerSM)
    k_pdot(const T* __restrict__ V, int64_t ldv, int64_t n, int j, GState* __restrict__ sts, int* stop,
           unsigned long long* gbar, double2* __restrict__ partials, int pass, int need_refine) {
  pdl_trigger();
  pdl_wait();
  if (*(volatile int*)stop) return;
  if (P == 1 && need_refine && !sts[0].refine) return;
  using A = typename Acc<T>::type;
  constexpr int R = DotRows<T>::value, TILE = kDotThreads * R;
  constexpr int NOWN = (kPStride * P + kDotThreads - 1) / kDotThreads;  // (k, s) slots per thread
  constexpr int NW = kDotThreads / 32;
  // per-tile sums: P > 1 by shared atomics on red[k * P + s]; P = 1 by one slot per warp
  // (redw[k][warp]: sixteen warps adding into one address would serialise)
  __shared__ A red[P == 1 ? 1 : kPStride * P];
  __shared__ A redw[P == 1 ? kPStride : 1][P == 1 ? NW : 1];
  __shared__ int bar_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nk = j + 1, nslot = (nk + 1) * P;  // slot (k, s) at k * P + s; k = nk is ||w||^2
  if (P > 1)
    for (int i = tid; i < nslot; i += kDotThreads) red[i] = zero<T>();
  auto put = [&](int k, A a) {  // after lane_tree: lanes < P hold the warp's sums
    if (P == 1) {
      if (lane == 0) redw[k][warp] = a;
    } else if (lane < P) {
      red_add(&red[k * P + lane], a);
    }
  };
  double2 acc[NOWN];
#pragma unroll
  for (int m = 0; m < NOWN; ++m) acc[m] = make_double2(0.0, 0.0);
  const int64_t e0 = n * blockIdx.x / gridDim.x * P, e1 = n * (blockIdx.x + 1) / gridDim.x * P;
  const T* W = V + (int64_t)(j + 1) * ldv;
  __syncthreads();
  for (int64_t base = e0; base < e1; base += TILE) {
    T wr[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int64_t e = base + tid + (int64_t)kDotThreads * q;
      wr[q] = e < e1 ? W[e] : zero<T>();
    }
    {
      A a = zero<T>();
#pragma unroll
      for (int q = 0; q < R; ++q) a.x += nrm2(wr[q]);
      put(nk, lane_tree<P>(a));
    }
    int k = 0;
    for (; k + 1 < nk; k += 2) {
      const T* v0 = V + (int64_t)k * ldv;
      const T* v1 = v0 + ldv;
      T a0[R], a1[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int64_t e = base + tid + (int64_t)kDotThreads * q;
        a0[q] = e < e1 ? v0[e] : zero<T>();
        a1[q] = e < e1 ? v1[e] : zero<T>();
      }
      A s0 = zero<T>(), s1 = zero<T>();
#pragma unroll
      for (int q = 0; q < R; ++q) {
        fma_conj(s0, a0[q], wr[q]);
        fma_conj(s1, a1[q], wr[q]);
      }
      put(k, lane_tree<P>(s0));
      put(k + 1, lane_tree<P>(s1));
    }
    if (k < nk) {
      const T* v0 = V + (int64_t)k * ldv;
      A s0 = zero<T>();
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int64_t e = base + tid + (int64_t)kDotThreads * q;
        if (e < e1) fma_conj(s0, v0[e], wr[q]);
      }
      put(k, lane_tree<P>(s0));
    }
    __syncthreads();
    if (P == 1) {
      if (tid < nslot) {
        A a = zero<T>();
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          a.x += redw[tid][w].x;
          a.y += redw[tid][w].y;
        }
        acc[0] = cadd(acc[0], to_d2(a));
      }
    } else {
#pragma unroll
      for (int m = 0; m < NOWN; ++m) {
        const int i = tid + kDotThreads * m;
        if (i < nslot) {
          acc[m] = cadd(acc[m], to_d2(red[i]));
          red[i] = zero<T>();
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < NOWN; ++m) {
    const int i = tid + kDotThreads * m;
    if (i < nslot) partials[(int64_t)blockIdx.x * kPStride * P + i] = acc[m];
  }
  // grid barrier: every block arrives once per launch, so the counter is a multiple of the grid
  // size when the launch starts and this launch's arrivals are the next gridDim.x tickets.
  // Arrival is a release add and the wait acquire loads; the block barriers on either side carry
  // the ordering to the block's other threads.
  __syncthreads();
  if (tid == 0) {
    const unsigned long long G = gridDim.x;
    unsigned long long ticket;
    asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(ticket) : "l"(gbar) : "memory");
    const unsigned long long target = (ticket / G + 1) * G;
    bool okb = true;
    const unsigned long long w0 = gs_time();
    while (true) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(gbar) : "memory");
      if (v >= target) break;
      if (gs_time() - w0 > kGsWaitNs) {
        okb = false;
        break;
      }
    }
    if (!okb) gs_fail<P>(sts, stop);
    bar_ok = okb;
  }
  __syncthreads();
  if (!bar_ok) return;
  // One warp per slot i, warps spread over the grid: lane l sums blocks l, l + 32, ... with its
  // loads in flight together (eight at a time), then an FP64 tree; fixed order.
  const int G = gridDim.x, nwarps = G * NW;
  for (int i = (warp % NW) * G + blockIdx.x; i < nslot; i += nwarps) {
    double2 sum = make_double2(0.0, 0.0);
    for (int b0 = 0; b0 < G; b0 += 256) {
      double2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int b = b0 + lane + 32 * m;
        v[m] = b < G ? __ldcg(&partials[(int64_t)b * kPStride * P + i]) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) sum = cadd(sum, v[m]);
    }
    sum = warp_sum(sum);
    if (lane != 0) continue;
    const int k = i / P, s = i - k * P;
    GState* st = &sts[s];
    if (k < nk) {
      const double ib = st->inv_beta[k];
      const double2 h = cscale(sum, ib);  // v_k^H w with v_k = V_k / ||V_k||
      if (pass == 0)
        st->h[k] = h;
      else
        st->h2[k] = h;
      st->c[k] = cscale(h, ib);  // w -= V_k (h_k / ||V_k||)
    } else if (pass == 0) {
      st->nrm_w = sum.x;
    }
  }
}

// ------------------------------------------------------------------ update
// w_s <- w_s - sum_k V_k c_k,s for the n rows.  finish != 0: also ||w_s||^2, and the last block to
// finish closes the Hessenberg column(s) (P = 1: pass 0 with eta2 > 0 instead flags a second pass
// when ||w||^2 fell below eta2 ||w_before||^2; pass 1 adds h2 to h).  counter: the solver's
// last-block counter (left at 0).  A persistent grid of kUpdBlocksPerSM blocks per SM walks the
// elements; eight basis loads per thread are in flight at a time.
template <typename T, int P>
__global__ void __launch_bounds__(kUpdThreads, kUpdBlocksPerSM)
    k_pupd(T* __restrict__ V, int64_t ldv, int64_t n, int j, GState* __restrict__ sts, int* stop, unsigned* counter,
           double2* __restrict__ partials, int pass, int need_refine, double eta2, int finish) {
  pdl_trigger();
  pdl_wait();
  if (*(volatile int*)stop) return;
  if (P == 1 && need_refine && !sts[0].refine) return;
  constexpr int NW = kUpdThreads / 32;
  __shared__ T cs[(kMaxM + 1) * P];
  __shared__ double red[NW][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < (j + 1) * P; i += kUpdThreads) {
    const int k = i / P, s = i - k * P;
    cs[i] = from_d2<T>(sts[s].c[k]);
  }
  __syncthreads();
  T* W = V + (int64_t)(j + 1) * ldv;
  const int s = tid % P;  // the grid stride is a multiple of P
  const int64_t total = n * P;
  double nrm = 0.0;
  typename Acc<T>::type part = zero<T>();
  int cnt = 0;
  for (int64_t e = blockIdx.x * (int64_t)kUpdThreads + tid; e < total; e += (int64_t)gridDim.x * kUpdThreads) {
    T w = W[e], w2 = zero<T>();
    int k = 0;
    for (; k + 8 <= j + 1; k += 8) {  // eight independent loads in flight
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V[(int64_t)(k + u) * ldv + e];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        sub_mul(w, v[u], cs[(k + u) * P + s]);
        sub_mul(w2, v[u + 1], cs[(k + u + 1) * P + s]);
      }
    }
    for (; k + 1 <= j; k += 2) {
      const T v0 = V[(int64_t)k * ldv + e], v1 = V[(int64_t)(k + 1) * ldv + e];
      sub_mul(w, v0, cs[k * P + s]);
      sub_mul(w2, v1, cs[(k + 1) * P + s]);
    }
    if (k <= j) sub_mul(w, V[(int64_t)k * ldv + e], cs[k * P + s]);
    w.x += w2.x;
    w.y += w2.y;
    W[e] = w;
    part.x += nrm2(w);
    if (++cnt == 32) {  // FP32 over at most 32 elements, then FP64
      nrm += (double)part.x;
      part = zero<T>();
      cnt = 0;
    }
  }
  if (!finish) return;
  // the thread's total and the warp tree in the accumulator's precision, FP64 across warps
  using AS = decltype(part.x);
  const AS tot = lane_tree<P>((AS)(nrm + (double)part.x));
  if (lane < P) red[warp][lane] = (double)tot;
  __syncthreads();
  if (tid < P) {
    double a = 0.0;
    for (int w = 0; w < NW; ++w) a += red[w][tid];
    partials[(int64_t)blockIdx.x * P + tid] = make_double2(a, 0.0);
  }
  if (!last_block(counter)) return;
  __shared__ double beta2[P];
  // ||w_s||^2 over the blocks: warp q sums source q (lanes take blocks lane, lane + 32, ...,
  // eight loads in flight at a time), fixed order.
  for (int q = warp; q < P; q += NW) {
    double a = 0.0;
    for (int b0 = 0; b0 < (int)gridDim.x; b0 += 256) {
      double v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int b = b0 + lane + 32 * m;
        v[m] = b < (int)gridDim.x ? __ldcg(&partials[(int64_t)b * P + q]).x : 0.0;
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) a += v[m];
    }
    a = warp_sum(a);
    if (lane == 0) beta2[q] = a;
  }
  __syncthreads();
  if (P == 1) {
    GState* st = &sts[0];
    if (pass == 0 && eta2 > 0.0 && beta2[0] < eta2 * st->nrm_w) {
      if (tid == 0) {
        st->refine = 1;
        *counter = 0;
      }
      return;
    }
    __shared__ double2 hsum[kMaxM + 1];
    for (int k = tid; k <= j; k += kUpdThreads) hsum[k] = pass == 1 ? cadd(st->h[k], st->h2[k]) : st->h[k];
    __syncthreads();
    if (warp == 0) finish_column_warp(st, j, hsum, beta2[0]);
    if (tid == 0) {
      if (pass == 1) {
        st->refined[j] = 1;
        st->n_refine += 1;
      }
      st->refine = 0;
      *counter = 0;
    }
  } else {
    for (int q = warp; q < P; q += NW)  // one warp per live source
      if (sts[q].done == 0) finish_column_warp(&sts[q], j, sts[q].h, beta2[q]);
    __syncthreads();
    if (tid == 0) {
      int alive = 0;
      for (int q = 0; q < P; ++q) alive += sts[q].done == 0;
      *stop = alive == 0;
      *counter = 0;
    }
  }
}

// ------------------------------------------------------------------ host side
// Check, once per process, that the projection kernel's grid (kDotBlocksPerSM per SM) can be
// resident at once, as its grid barrier needs.
template <typename T, int P>
Status gs_setup() {
  static bool done = false;
  if (done) return Status{};
  int nb = 0;
  PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pdot<T, P>, kDotThreads, 0));
  if (nb < kDotBlocksPerSM) return Status{PETGEM_ERR_UNSUPPORTED, "projection kernel: too few resident blocks per SM"};
  done = true;
  return Status{};
}

template <typename T, int P>
Status launch_pdot(cudaStream_t s, int sms, const T* V, int64_t ldv, int64_t n, int j, GState* sts, int* stop,
                   unsigned long long* gbar, double2* part, int pass, int need_refine) {
  PG_CUDA(pdl_launch(k_pdot<T, P>, dim3(kDotBlocksPerSM * sms), dim3(kDotThreads), 0, s, true, V, ldv, n, j, sts,
                     stop, gbar, part, pass, need_refine));
  return Status{};
}

inline int pupd_grid(int64_t n, int P, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n * P + kUpdThreads - 1) / kUpdThreads, kUpdBlocksPerSM * sms));
}

template <typename T, int P>
Status launch_pupd(cudaStream_t s, int sms, T* V, int64_t ldv, int64_t n, int j, GState* sts, int* stop,
                   unsigned* counter, double2* part, int pass, int need_refine, double eta2, int finish) {
  PG_CUDA(pdl_launch(k_pupd<T, P>, dim3(pupd_grid(n, P, sms)), dim3(kUpdThreads), 0, s, false, V, ldv, n, j, sts,
                     stop, counter, part, pass, need_refine, eta2, finish));
  return Status{};
}

}  // namespace
}  // namespace petgem
