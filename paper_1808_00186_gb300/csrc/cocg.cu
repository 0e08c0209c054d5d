// Conjugate orthogonal conjugate gradient (COCG) for the complex-symmetric system of eq. 9: a
// short-recurrence alternative to GMRES (the paper's mesh-adaptation study, Section 5.3, solves the
// same system with a method of this family, symmetric QMR).  COCG is CG with the bilinear form
// u^T v instead of the Hermitian product; A^T = A makes the residuals orthogonal in that form, so
// no basis is stored and an iteration moves about half the bytes of a GMRES(50) step.
//
// Jacobi enters as a symmetric scaling, Atil = S A S with S = D^{-1/2} (principal complex square
// root of the diagonal), which keeps the operator complex symmetric (a one-sided scaling A D^{-1}
// would not be, and COCG diverges on it).  An inner solve iterates on Atil y = S r and returns
// x += S y.
//
// The iterations run in one persistent cooperative kernel (k_cg_inner): per iteration the SpMV
// q = Atil p with the bilinear p^T q fused into it, the residual update (r -= alpha q, r^T r and
// ||r||^2) and the pass y += alpha p, p = r + beta p, separated by barriers over the grid instead
// of kernel boundaries.  The scalars never leave the device; the host looks at the state once per
// chunk of iterations.  Mixed precision: Atil and the vectors in complex64 (FP32
// products within a thread and its warp, FP64 beyond); each inner solve runs until its residual fell
// by inner_tol and restarts from the FP64 true residual b - A x (iterative refinement).  c128:
// everything in FP64, one inner solve to the final tolerance.
#include <math.h>

#include <algorithm>
#include <vector>

#include "krylov.cuh"
#include "bands.cuh"

namespace petgem {
namespace {

struct CState {
  int done;  // 0 running, 1 inner threshold reached, 2 breakdown of the bilinear form
  int k;     // iterations of this inner solve
  unsigned counter;
  int pad;
  unsigned long long gbar;  // arrivals at the persistent kernel's barriers (only grows)
  unsigned long long grel;  // the last release of a reducing barrier (the arrival count it closed)
  double2 sc;               // the scalar a reducing barrier published (alpha or beta)
  int sc_dn;                // and its stopping decision
  int pad2;
  double2 sc2;              // SQMR: c^2 alpha, the weight of p in the smoothing direction d
  double sc3;               // SQMR: c^2 theta_prev^2, the weight of the previous d
  double tau, theta;        // SQMR: quasi-residual norm and theta of the last step
  double2 rho;  // r^T r
  double2 alpha, beta;
  float2 alpha32, beta32;
  double nr0, nr, stop2;  // ||r||^2 at the start and now; stop when nr <= stop2
  double rn2;             // FP64 ||v||^2 of the last k_cg_norm
};

constexpr int kCgG = 4;  // lanes per row of the CSR products (rows hold at most ~19 entries)
constexpr int kCgU = 5;  // entries per lane in one batch
constexpr unsigned long long kCgWaitNs = 2000000000ull;  // bound of a barrier wait (2 s)
template <typename T> struct CgOcc { static constexpr int value = 4; };
template <> struct CgOcc<double2> { static constexpr int value = 3; };

__device__ inline void bil_fma(float2& acc, float2 a, float2 b) { fma_c(acc, a, b); }  // acc += a b
__device__ inline void bil_fma(double2& acc, double2 a, double2 b) { fma_c(acc, a, b); }

// Warp-parallel FP64 sum of partials[b * kPStride + slot] over b < nb (eight loads in flight per
// lane at a time, then a tree): every lane returns the total.
__device__ inline double2 warp_sum_partials(const double2* partials, int nb, int slot) {
  const int lane = threadIdx.x & 31;
  double2 a = make_double2(0.0, 0.0);
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int b = b0 + lane + 32 * m;
      v[m] = b < nb ? __ldcg(&partials[(int64_t)b * kPStride + slot]) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) a = cadd(a, v[m]);
  }
  return warp_sum(a);
}

// Warp tree in the accumulator's own precision (FP32 for complex64 data: an FP64 add costs ~60
// cycles per warp instruction on this GPU).
__device__ inline float2 warp_tree(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ inline double2 warp_tree(double2 v) { return warp_sum(v); }

// Block sums of two complex accumulators into partials[b][0..1]: the warp tree in the
// accumulator's precision, FP64 across the warps.
template <int NT, typename A>
__device__ inline void block_partials2(A a0, A a1, double2* partials) {
  __shared__ double2 red[NT / 32][2];
  a0 = warp_tree(a0);
  a1 = warp_tree(a1);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = to_d2(a0);
    red[threadIdx.x >> 5][1] = to_d2(a1);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) s = cadd(s, red[w][threadIdx.x]);
    partials[(int64_t)blockIdx.x * kPStride + threadIdx.x] = s;
  }
}

// Scaled operator Atil = S A S, S = diag(sq): row by row (one thread per row).
__global__ void k_cg_scale(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, const double2* __restrict__ sq, int64_t n,
                           double2* __restrict__ a128, float2* __restrict__ a64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 si = sq[i];
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    const double2 v = cmul(cmul(si, val[p]), sq[col[p]]);
    a128[p] = v;
    a64[p] = make_float2((float)v.x, (float)v.y);
  }
}

// sq = D^{-1/2}: principal complex square root of the diagonal, inverted.
__global__ void k_cg_sqrt_diag(const double2* __restrict__ d, int64_t n, double2* __restrict__ sq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 z = d[i];
  const double m = sqrt(cabs2(z));
  // sqrt(z) = (sqrt((m + x) / 2), sign(y) sqrt((m - x) / 2)), the root with non-negative real part
  const double re = sqrt(fmax(0.5 * (m + z.x), 0.0));
  double im = sqrt(fmax(0.5 * (m - z.x), 0.0));
  if (z.y < 0.0) im = -im;
  sq[i] = cdiv(make_double2(1.0, 0.0), make_double2(re, im));
}

// r64 = b - A x (FP64, the assembled matrix), G lanes per row.
template <int G>
__global__ void __launch_bounds__(256) k_cg_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                     const double2* __restrict__ val, const double2* __restrict__ x,
                                                     const double2* __restrict__ b, double2* __restrict__ r,
                                                     int64_t n) {
  // loads of a lane's first five entries first, then their gathers, then the FMAs (two chains)
  constexpr int U = 5;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / G;
  const int lane = (int)(gid % G);
  double2 acc = make_double2(0.0, 0.0), acc2 = acc;
  if (row < n) {
    const int64_t p0 = rp[row] + lane, p1 = rp[row + 1];
    int32_t c[U];
    double2 a[U], xv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t q = p0 + (int64_t)k * G;
      c[k] = q < p1 ? __ldg(&col[q]) : 0;
      a[k] = q < p1 ? __ldg(&val[q]) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) xv[k] = p0 + (int64_t)k * G < p1 ? x[c[k]] : make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < U; ++k) fma_c((k & 1) ? acc2 : acc, a[k], xv[k]);
    for (int64_t p = p0 + (int64_t)U * G; p < p1; p += G) fma_c(acc, val[p], x[col[p]]);
  }
  acc.x += acc2.x;
  acc.y += acc2.y;
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) r[row] = csub(b[row], acc);
}

// ||v||^2 in FP64 into st->rn2.
__global__ void __launch_bounds__(kT) k_cg_norm(const double2* __restrict__ v, int64_t n, CState* __restrict__ st,
                                                double2* __restrict__ partials) {
  double s = 0.0;
  const int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    const int64_t i = base + (int64_t)q * kT;
    if (i < n) s += nrm2(v[i]);
  }
  block_partials2<kT>(make_double2(s, 0.0), make_double2(0.0, 0.0), partials);
  if (!last_block(&st->counter)) return;
  if (threadIdx.x < 32) {
    const double2 t = warp_sum_partials(partials, gridDim.x, 0);
    if (threadIdx.x == 0) {
      st->rn2 = t.x;
      st->counter = 0;
    }
  }
}

// Inner-solve start: r = p = scale S r64 (rounded to T), y = 0, rho = r^T r, ||r||^2, threshold.
// scale = 1 / ||r64|| keeps the complex64 vectors of O(1) size: after a few refinements the
// residual's entries are ~1e-20 and their squares would underflow in FP32.
// SQMR (dvec != null): also d = 0, tau = ||r||, theta = 0.  perm != null: the iteration vectors
// are in the SELL layout's renumbering (entry i is edge perm[i]).
template <typename T>
__global__ void __launch_bounds__(kT) k_cg_start(const double2* __restrict__ r64, const double2* __restrict__ sq,
                                                 const int32_t* __restrict__ perm, T* __restrict__ r,
                                                 T* __restrict__ p, T* __restrict__ y, T* __restrict__ dvec, int64_t n,
                                                 CState* __restrict__ st, double2* __restrict__ partials, double inner,
                                                 double scale) {
  using A = typename Acc<T>::type;
  A rho = zero<T>(), nr = zero<T>();
  const int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    const int64_t i = base + (int64_t)q * kT;
    if (i < n) {
      const int64_t o = perm ? perm[i] : i;  // renumbered vectors (SELL layout) gather the original entry
      const T t = from_d2<T>(cscale(cmul(sq[o], r64[o]), scale));
      r[i] = t;
      p[i] = t;
      y[i] = zero<T>();
      if (dvec) dvec[i] = zero<T>();
      bil_fma(rho, t, t);
      nr.x += nrm2(t);
    }
  }
  block_partials2<kT>(rho, nr, partials);
  if (!last_block(&st->counter)) return;
  if (threadIdx.x < 32) {
    const double2 a = warp_sum_partials(partials, gridDim.x, 0);
    const double2 b = warp_sum_partials(partials, gridDim.x, 1);
    if (threadIdx.x == 0) {
      st->rho = a;
      st->nr0 = b.x;
      st->nr = b.x;
      st->stop2 = inner * inner * b.x;
      st->k = 0;
      st->done = (b.x > 0.0 && isfinite(b.x)) ? 0 : (b.x == 0.0 ? 1 : 2);
      st->gbar = 0;
      st->grel = 0;
      st->tau = sqrt(b.x);
      st->theta = 0.0;
      st->counter = 0;
    }
  }
}

template <typename T, int G>
__device__ inline void cg_fetch(const int32_t* __restrict__ col, const T* __restrict__ val, int64_t p0, int64_t p1,
                                int32_t* c, T* a) {
#pragma unroll
  for (int u = 0; u < kCgU; ++u) {
    const int64_t q = p0 + (int64_t)u * G;
    c[u] = q < p1 ? __ldg(&col[q]) : 0;
    a[u] = q < p1 ? __ldg(&val[q]) : zero<T>();
  }
}

// One system of a persistent COCG launch: its CSR operator (row pointers, columns, values of
// Atil), its four vectors, its state and block partials, and the range of blocks that serve it.
template <typename T>
struct CgSys {
  const int64_t* rp;
  const int32_t* col;
  const T* val;
  T *p, *q, *r, *y;
  T* d;           // SQMR: the smoothing direction (unused by COCG)
  const int64_t* sp;    // SELL-32 layout of the operator (rows and vectors renumbered; null: CSR)
  const int32_t* scol;
  const T* sval;
  int64_t ns;           // slices
  int64_t n;
  CState* st;
  double2* part;  // [nb][kCgSlots]: slot 0 r^T r, 1 ||r||^2, 2 p^T q
  int64_t kmax;   // the inner solve stops when its iteration count reaches kmax
  int b0, nb;
};
constexpr int kCgSlots = 4;

__device__ inline unsigned long long cg_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over the nb blocks of one system.  gbar counts arrivals and only grows; every block
// arrives once per barrier, so each barrier's arrivals are the next nb tickets.  Thread 0 arrives
// with a release add and waits with acquire loads; the block barriers on either side carry the
// ordering to the other threads, so every block's writes before the barrier are visible to every
// block's reads after it.  The wait is bounded (kCgWaitNs): false in every thread of the block when
// it gave up.
__device__ inline bool cg_barrier(unsigned long long* gbar, unsigned nb, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(t) : "l"(gbar) : "memory");
    const unsigned long long target = (t / nb + 1) * nb;
    int ok = 1;
    const unsigned long long w0 = cg_now();
    while (true) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(gbar) : "memory");
      if (v >= target) break;
      if (cg_now() - w0 > kCgWaitNs) {
        ok = 0;
        break;
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Fixed-order FP64 sums of part[b * kCgSlots + s0] and part[b * kCgSlots + s1] over b < nb by the
// whole block: each thread a few partials (all loads in flight at once), a warp tree, then one over
// the warps; out[0], out[1] (shared) receive the totals.
template <int NT>
__device__ inline void cg_sum_blocks2(const double2* part, int nb, int s0, int s1, double2* out) {
  __shared__ double2 red[NT / 32][2];
  double2 a = make_double2(0.0, 0.0), b = a;
  for (int k = threadIdx.x; k < nb; k += NT) {
    a = cadd(a, __ldcg(&part[(int64_t)k * kCgSlots + s0]));
    b = cadd(b, __ldcg(&part[(int64_t)k * kCgSlots + s1]));
  }
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = a;
    red[warp][1] = b;
  }
  __syncthreads();
  if (warp == 0) {
    double2 u = lane < NT / 32 ? red[lane][0] : make_double2(0.0, 0.0);
    double2 v = lane < NT / 32 ? red[lane][1] : make_double2(0.0, 0.0);
#pragma unroll
    for (int o = NT / 64; o > 0; o >>= 1) {
      u.x += __shfl_xor_sync(0xffffffffu, u.x, o);
      u.y += __shfl_xor_sync(0xffffffffu, u.y, o);
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) {
      out[0] = u;
      out[1] = v;
    }
  }
}

// Reducing barrier over the nb blocks of one system: the last block to arrive (it sees every
// other block's partials) sums the block partials once, with all its threads, forms the step's
// scalar and decision in the state, and releases the others, which read the published scalar
// (sc, sc_dn).  One block reads the partials instead of every block (which would make every block
// fetch the same lines from L2 and spend the SM's scarce FP64 issue slots on the same sums).
//   stage 0 (after the SpMV): alpha = rho / p^T q, or a breakdown of the bilinear form.
//   stage 1 (after the update): r^T r and ||r||^2; the stopping test, beta = rho' / rho, k, nr.
// The wait is bounded (kCgWaitNs); the result is false in every thread when it gave up.  On
// return *s_sc and *s_dn hold the scalar and decision in every block.
template <int NT, int STAGE, bool QMR>
__device__ inline bool cg_reduce_barrier(CState* st, const double2* part, unsigned nb, int* s_ok, int* s_last,
                                         double2* s_sc, int* s_dn, double2* s_sc2, double* s_sc3) {
  __syncthreads();
  unsigned long long target = 0;  // this barrier's closing arrival count (thread 0)
  if (threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(t) : "l"(&st->gbar) : "memory");
    target = (t / nb + 1) * nb;
    *s_last = t + 1 == target;
    int ok = 1;
    if (t + 1 != target) {
      const unsigned long long w0 = cg_now();
      while (true) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&st->grel) : "memory");
        if (v >= target) break;
        if (cg_now() - w0 > kCgWaitNs) {
          ok = 0;
          break;
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  if (!*s_ok) return false;
  if (*s_last) {
    __shared__ double2 tot[2];
    cg_sum_blocks2<NT>(part, nb, STAGE == 0 ? 2 : 0, STAGE == 0 ? 3 : 1, tot);
    __syncthreads();
    if (threadIdx.x == 0) {
      int d = 0;
      double2 sc = make_double2(0.0, 0.0);
      if (STAGE == 0) {
        const double2 pq = tot[0];
        if (!(cabs2(pq) > 0.0) || !isfinite(pq.x) || !isfinite(pq.y)) {
          d = 2;
        } else {
          sc = cdiv(st->rho, pq);
          st->alpha = sc;
        }
      } else {
        const double nrm = tot[1].x;
        st->k += 1;
        st->nr = nrm;
        // SQMR: quasi-minimal-residual smoothing of the step (theta, c, tau) and the weights of
        // d = c^2 theta_prev^2 d + c^2 alpha p; the stopping test is on the quasi-residual tau
        double test = nrm;
        if (QMR) {  // no smoothing step when the norm is not finite
          st->sc2 = make_double2(0.0, 0.0);
          st->sc3 = 0.0;
        }
        if (QMR && isfinite(nrm)) {
          const double th = sqrt(nrm) / st->tau;
          const double c2 = 1.0 / (1.0 + th * th);
          const double tau = st->tau * th * sqrt(c2);
          st->sc2 = cscale(st->alpha, c2);
          st->sc3 = c2 * st->theta * st->theta;
          st->theta = th;
          st->tau = tau;
          test = tau * tau;
        }
        if (!isfinite(nrm))
          d = 2;
        else if (test <= st->stop2)
          d = 1;
        else if (!(cabs2(st->rho) > 0.0))
          d = 2;
        if (!d) {
          sc = cdiv(tot[0], st->rho);
          st->beta = sc;
          st->rho = tot[0];
        }
      }
      if (d) st->done = d;
      st->sc = sc;
      st->sc_dn = d;
      *s_sc = sc;
      *s_dn = d;
      if (QMR && STAGE == 1) {
        *s_sc2 = st->sc2;
        *s_sc3 = st->sc3;
      }
      asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(&st->grel), "l"(target) : "memory");
    }
  } else if (threadIdx.x == 0) {
    *s_sc = __ldcg(&st->sc);
    *s_dn = __ldcg(&st->sc_dn);
    if (QMR && STAGE == 1) {
      *s_sc2 = __ldcg(&st->sc2);
      *s_sc3 = __ldcg(&st->sc3);
    }
  }
  __syncthreads();
  return true;
}

// Block sums of two accumulators into out[0], out[1] (warp tree in the accumulator's precision,
// FP64 across warps).
template <int NT, typename A>
__device__ inline void cg_block_sums(A a0, A a1, double2* out) {
  __shared__ double2 red[NT / 32][2];
  a0 = warp_tree(a0);
  a1 = warp_tree(a1);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = to_d2(a0);
    red[threadIdx.x >> 5][1] = to_d2(a1);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) s = cadd(s, red[w][threadIdx.x]);
    out[threadIdx.x] = s;
  }
}

// q = Atil p over the rows row0, row0 + groups, ... (G lanes per row), software-pipelined: the
// gathers of row i overlap the column/value loads of row i + 1 and the row pointers of row i + 2.
// Returns this thread's share of the bilinear p^T q.  p is written by other blocks of the same
// launch between calls, so its gathers are plain (coherent after the barrier) loads, not
// read-only-cache loads; the matrix is read-only.
template <typename T, int G>
__device__ inline typename Acc<T>::type cg_spmv_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                     const T* __restrict__ val, const T* p, T* q, int64_t n,
                                                     int64_t row, int64_t groups) {
  constexpr int U = kCgU;
  using A = typename Acc<T>::type;
  const int lane = threadIdx.x % G;
  int64_t p0 = 0, p1 = 0;
  if (row < n) {
    p0 = __ldg(&rp[row]) + lane;
    p1 = __ldg(&rp[row + 1]);
  }
  int32_t c[U];
  T a[U];
  cg_fetch<T, G>(col, val, p0, p1, c, a);
  int64_t nrow = row + groups, np0 = 0, np1 = 0;
  if (nrow < n) {
    np0 = __ldg(&rp[nrow]) + lane;
    np1 = __ldg(&rp[nrow + 1]);
  }
  A dot = zero<T>();
  while (__any_sync(0xffffffffu, row < n)) {
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = p0 + (int64_t)u * G < p1 ? p[c[u]] : zero<T>();
    const T prow = (row < n && lane == 0) ? p[row] : zero<T>();
    int32_t c2[U];
    T a2[U];
    cg_fetch<T, G>(col, val, np0, np1, c2, a2);
    const int64_t nnrow = nrow + groups;
    int64_t nnp0 = 0, nnp1 = 0;
    if (nnrow < n) {
      nnp0 = __ldg(&rp[nnrow]) + lane;
      nnp1 = __ldg(&rp[nnrow + 1]);
    }
    A acc = zero<T>(), acc2 = zero<T>();
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      fma_c(acc, a[u], xv[u]);
      if (u + 1 < U) fma_c(acc2, a[u + 1], xv[u + 1]);
    }
    for (int64_t qq = p0 + (int64_t)U * G; qq < p1; qq += G) fma_c(acc, __ldg(&val[qq]), p[__ldg(&col[qq])]);
    acc.x += acc2.x;
    acc.y += acc2.y;
    for (int o = G / 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (row < n && lane == 0) {
      const T qv = from_d2<T>(to_d2(acc));
      q[row] = qv;
      bil_fma(dot, prow, qv);
    }
    row = nrow;
    p0 = np0;
    p1 = np1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = c2[u];
      a[u] = a2[u];
    }
    nrow = nnrow;
    np0 = nnp0;
    np1 = nnp1;
  }
  return dot;
}

// q = Atil p over the SELL-32 slices w0, w0 + nwarps, ... of the renumbered operator (one warp per
// slice, lane = row), five entries of a slice at a time with the next five's columns and values in
// flight during this chunk's gathers; returns this thread's share of the bilinear p^T q.  As in
// cg_spmv_rows, p's gathers are plain loads (other blocks wrote p since the last barrier).
// (Contiguous slice ranges of equal stored entries per warp measured far slower than this
// interleaving: one block took 2.6x the others.)
template <typename T>
__device__ inline typename Acc<T>::type cg_sell_rows(const int64_t* __restrict__ sp, const int32_t* __restrict__ scol,
                                                     const T* __restrict__ sval, const T* p, T* q, int64_t n,
                                                     int64_t ns, int64_t w0, int64_t nwarps) {
  constexpr int U = 5;
  using A = typename Acc<T>::type;
  const int lane = threadIdx.x & 31;
  A dot = zero<T>();
  int64_t s = w0, b = 0, w = 0, t = 0;
  if (s < ns) {
    b = __ldg(&sp[s]);
    w = (__ldg(&sp[s + 1]) - b) >> 5;
  }
  int32_t c[U];
  T a[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const bool ok = u < w;
    c[u] = ok ? __ldg(&scol[b + u * 32 + lane]) : 0;
    a[u] = ok ? __ldg(&sval[b + u * 32 + lane]) : zero<T>();
  }
  A acc = zero<T>(), acc2 = zero<T>();
  while (s < ns) {
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = t + u < w ? p[c[u]] : zero<T>();
    int64_t s2 = s, b2 = b, w2 = w, t2 = t + U;
    if (t2 >= w) {  // the next chunk is the next slice's first
      s2 = s + nwarps;
      t2 = 0;
      w2 = 0;
      if (s2 < ns) {
        b2 = __ldg(&sp[s2]);
        w2 = (__ldg(&sp[s2 + 1]) - b2) >> 5;
      }
    }
    int32_t c2[U];
    T a2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = t2 + u < w2;
      c2[u] = ok ? __ldg(&scol[b2 + (t2 + u) * 32 + lane]) : 0;
      a2[u] = ok ? __ldg(&sval[b2 + (t2 + u) * 32 + lane]) : zero<T>();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) fma_c((u & 1) ? acc2 : acc, a[u], xv[u]);
    if (t2 == 0) {  // this slice is complete
      const int64_t r = s * 32 + lane;
      if (r < n) {
        acc.x += acc2.x;
        acc.y += acc2.y;
        const T qv = from_d2<T>(to_d2(acc));
        q[r] = qv;
        bil_fma(dot, p[r], qv);
      }
      acc = zero<T>();
      acc2 = zero<T>();
    }
    s = s2;
    b = b2;
    w = w2;
    t = t2;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = c2[u];
      a[u] = a2[u];
    }
  }
  return dot;
}

// The iterations of an inner COCG solve, persistent: one launch runs up to max_steps iterations
// of every system in sys[0, nsys), each on its own blocks [b0, b0 + nb), and stops a system when
// its residual met the inner threshold or its bilinear form broke down.  Per iteration and system
// three phases, each closed by a barrier over the system's blocks:
//   SpMV    q = Atil p and the block sums of p^T q;  (reducing barrier: alpha)
//   update  r -= alpha q, block sums of r^T r and ||r||^2;  (reducing barrier: beta, the stopping
//           test)
//   then    y += alpha p and the direction p = r + beta p (one pass over p).
// The scalars are formed once per barrier, by the block that arrives last, and the state always
// holds the current rho, k and ||r||^2.  The grid must be resident at once (cooperative launch).
// A barrier that gives up sets done = 3.
template <typename T, int G, bool QMR, bool SELL = false>
__global__ void __launch_bounds__(256, CgOcc<T>::value)
    k_cg_inner(const CgSys<T>* __restrict__ sys, int nsys, int max_steps) {
  __shared__ int s_sys, s_ok, s_dn, s_last;
  __shared__ double2 s_sc, s_sc2;
  __shared__ double s_sc3;
  pdl_wait();
  const int tid = threadIdx.x;
  if (tid == 0) {
    int k = 0;
    while (k + 1 < nsys && (int)blockIdx.x >= sys[k + 1].b0) ++k;
    s_sys = k;
  }
  __syncthreads();
  const CgSys<T>* S = &sys[s_sys];
  const int lb = (int)blockIdx.x - S->b0, nb = S->nb;
  if (lb < 0 || lb >= nb) return;  // blocks past the last system's range (none when the host sizes the grid)
  CState* st = S->st;
  // read before the first barrier: the barriers' last blocks rewrite the state after it
  if (st->done) return;
  const int64_t steps = std::min<int64_t>(max_steps, S->kmax - st->k);
  const int64_t n = S->n;
  const int64_t* rp = S->rp;
  const int32_t* col = S->col;
  const T* val = S->val;
  T *p = S->p, *q = S->q, *r = S->r, *y = S->y;
  T* dq = S->d;
  double2* part = S->part;
  using A = typename Acc<T>::type;
  const int64_t groups = (int64_t)nb * (256 / G);
  const int64_t row0 = (int64_t)lb * (256 / G) + tid / G;
  const int64_t stride = (int64_t)nb * 256, first = (int64_t)lb * 256 + tid;
  bool fail = false;
  for (int64_t step = 0; step < steps; ++step) {
    A dot;
    if constexpr (SELL)
      dot = cg_sell_rows<T>(S->sp, S->scol, S->sval, p, q, n, S->ns, (int64_t)lb * 8 + (tid >> 5), (int64_t)nb * 8);
    else
      dot = cg_spmv_rows<T, G>(rp, col, val, p, q, n, row0, groups);
    cg_block_sums<256>(dot, zero<T>(), part + (int64_t)lb * kCgSlots + 2);
    if (!cg_reduce_barrier<256, 0, QMR>(st, part, nb, &s_ok, &s_last, &s_sc, &s_dn, &s_sc2, &s_sc3)) {
      fail = true;
      break;
    }
    if (s_dn) break;
    const T al = from_d2<T>(s_sc);
    A rh = zero<T>(), nr = zero<T>();
    double2 rh64 = make_double2(0.0, 0.0), nr64 = rh64;
    int cnt = 0;
    // r -= alpha q (y += alpha p waits for the direction pass, which reads p anyway); four
    // elements per thread in flight, then the ragged tail one by one
    int64_t i = first;
    for (; i + 3 * stride < n; i += 4 * stride) {
      T qv[4], rv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qv[v] = __ldcg(&q[i + v * stride]);
        rv[v] = r[i + v * stride];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sub_mul(rv[v], qv[v], al);
        r[i + v * stride] = rv[v];
        bil_fma(rh, rv[v], rv[v]);
        nr.x += nrm2(rv[v]);
      }
      cnt += 4;
      if (cnt >= 32) {  // the accumulator's precision over at most 32 elements, then FP64
        rh64 = cadd(rh64, to_d2(rh));
        nr64 = cadd(nr64, to_d2(nr));
        rh = zero<T>();
        nr = zero<T>();
        cnt = 0;
      }
    }
    for (; i < n; i += stride) {
      T rv = r[i];
      sub_mul(rv, __ldcg(&q[i]), al);
      r[i] = rv;
      bil_fma(rh, rv, rv);
      nr.x += nrm2(rv);
    }
    rh.x += (decltype(rh.x))rh64.x;
    rh.y += (decltype(rh.x))rh64.y;
    nr.x += (decltype(nr.x))nr64.x;
    cg_block_sums<256>(rh, nr, part + (int64_t)lb * kCgSlots);
    if (!cg_reduce_barrier<256, 1, QMR>(st, part, nb, &s_ok, &s_last, &s_sc, &s_dn, &s_sc2, &s_sc3)) {
      fail = true;
      break;
    }
    if (QMR) {
      // SQMR: d = c^2 theta_prev^2 d + c^2 alpha p, y += d (the smoothed iterate), p = r + beta p
      const T wp = from_d2<T>(s_sc2);
      const decltype(wp.x) wd = (decltype(wp.x))s_sc3;
      if (s_dn) {  // stopped: the iterate still takes this step's smoothing
        for (int64_t j = first; j < n; j += stride) {
          T dv = dq[j];
          dv.x *= wd;
          dv.y *= wd;
          fma_c(dv, wp, p[j]);
          dq[j] = dv;
          T yv = y[j];
          yv.x += dv.x;
          yv.y += dv.y;
          y[j] = yv;
        }
        break;
      }
      const T be = from_d2<T>(s_sc);
      int64_t j = first;
      for (; j + stride < n; j += 2 * stride) {
        T a[2], b[2], c[2], e[2];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          a[v] = r[j + v * stride];
          b[v] = p[j + v * stride];
          c[v] = y[j + v * stride];
          e[v] = dq[j + v * stride];
        }
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          e[v].x *= wd;
          e[v].y *= wd;
          fma_c(e[v], wp, b[v]);
          dq[j + v * stride] = e[v];
          c[v].x += e[v].x;
          c[v].y += e[v].y;
          y[j + v * stride] = c[v];
          fma_c(a[v], be, b[v]);
          p[j + v * stride] = a[v];
        }
      }
      for (; j < n; j += stride) {
        const T pv = p[j];
        T dv = dq[j];
        dv.x *= wd;
        dv.y *= wd;
        fma_c(dv, wp, pv);
        dq[j] = dv;
        T yv = y[j], rv = r[j];
        yv.x += dv.x;
        yv.y += dv.y;
        y[j] = yv;
        fma_c(rv, be, pv);
        p[j] = rv;
      }
    } else {
      if (s_dn) {  // stopped: the iterate still takes this step's alpha p
        for (int64_t j = first; j < n; j += stride) {
          T yv = y[j];
          fma_c(yv, al, p[j]);
          y[j] = yv;
        }
        break;
      }
      // y += alpha p and p = r + beta p
      const T be = from_d2<T>(s_sc);
      int64_t j = first;
      for (; j + 3 * stride < n; j += 4 * stride) {
        T a[4], b[4], c[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          a[v] = r[j + v * stride];
          b[v] = p[j + v * stride];
          c[v] = y[j + v * stride];
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          fma_c(c[v], al, b[v]);
          y[j + v * stride] = c[v];
          fma_c(a[v], be, b[v]);
          p[j + v * stride] = a[v];
        }
      }
      for (; j < n; j += stride) {
        const T pv = p[j];
        T yv = y[j], rv = r[j];
        fma_c(yv, al, pv);
        y[j] = yv;
        fma_c(rv, be, pv);
        p[j] = rv;
      }
    }
    if (!cg_barrier(&st->gbar, nb, &s_ok)) {
      fail = true;
      break;
    }
  }
  if (fail && tid == 0) atomicExch(&st->done, 3);
}

constexpr int kCgChunk = 1024;  // iterations per persistent launch (the host checks the state between)
constexpr int64_t kCgInnerMax = 4096;  // iterations of one complex64 inner solve at most

// Whether the persistent kernel's grid (CgOcc blocks per SM) can be resident at once.
template <typename T, int G, bool QMR = false, bool SELL = false>
Status cg_setup() {
  static bool done = false;
  if (done) return Status{};
  int nb = 0;
  PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_inner<T, G, QMR, SELL>, 256, 0));
  if (nb < CgOcc<T>::value) return Status{PETGEM_ERR_UNSUPPORTED, "COCG kernel: too few resident blocks per SM"};
  done = true;
  return Status{};
}

template <typename T> __device__ inline T cg_alpha(const CState* st);
template <> __device__ inline float2 cg_alpha<float2>(const CState* st) { return st->alpha32; }
template <> __device__ inline double2 cg_alpha<double2>(const CState* st) { return st->alpha; }
template <typename T> __device__ inline T cg_beta(const CState* st);
template <> __device__ inline float2 cg_beta<float2>(const CState* st) { return st->beta32; }
template <> __device__ inline double2 cg_beta<double2>(const CState* st) { return st->beta; }

// x += unscale S y (FP64).
template <typename T>
__global__ void k_cg_finish(const T* __restrict__ y, const double2* __restrict__ sq, const int32_t* __restrict__ perm,
                            double2* __restrict__ x, int64_t n, double unscale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = perm ? perm[i] : i;
  x[o] = cadd(x[o], cscale(cmul(sq[o], to_d2(y[i])), unscale));
}

struct BatchBuffers;

struct CgBuffers {
  DevBuf sq, a128, a64, r64, r, p, q, y, d, state, partials, sys;
  DevBuf s64, s128;  // the operator's values in the SELL-32 layout (when the mesh has one)
  BatchBuffers* batch = nullptr;  // workspace of petgem_solve_batch (when this context leads one)
  // multi-source solve: interleaved right-hand sides, iterate and residual (c128), vectors (T),
  // per-source states, group flags and per-source scales / inner targets
  DevBuf Bt, X, R, rb, pb, qb, yb, bstates, bgrp, bscal;
  int64_t version = -1;
};

CgBuffers* cg_bufs(petgem_ctx* c) {
  if (!c->cocg) c->cocg = new CgBuffers();
  return static_cast<CgBuffers*>(c->cocg);
}

Status read_cstate(petgem_ctx* c, CgBuffers* B, CState* h) {
  PG_CUDA(cudaMemcpyAsync(h, B->state.ptr, sizeof(CState), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return Status{};
}

template <typename T, bool QMR>
Status cocg_source(petgem_ctx* c, const petgem_solve_opts& o, CgBuffers* B, const double2* b, double2* x,
                   petgem_solve_info& inf, int sms) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  CState* st = B->state.as<CState>();
  double2* part = B->partials.as<double2>();
  const bool c128 = sizeof(T) == 16;
  const T* at = c128 ? (const T*)B->a128.ptr : (const T*)B->a64.ptr;
  T *r = B->r.as<T>(), *p = B->p.as<T>(), *q = B->q.as<T>(), *y = B->y.as<T>();
  T* dq = QMR ? B->d.as<T>() : nullptr;
  const unsigned nb = blocks_for(n, kRows);
  // the persistent kernel's grid: CgOcc blocks per SM (all resident), fewer for a small system
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(blocks_for(n * kCgG, 256), (int64_t)CgOcc<T>::value * sms));
  const bool sell = c->sell_ok;
  if (sell)
    PG_TRY((cg_setup<T, kCgG, QMR, true>()));
  else
    PG_TRY((cg_setup<T, kCgG, QMR, false>()));
  const int32_t* perm = sell ? c->sell_perm.as<int32_t>() : nullptr;
  const double vb = (double)sizeof(T) * n;
  // per iteration: SpMV nnz (values + columns) + row pointers + p gathered once, p of the row and
  // q written; update q, r read and r written; direction r, p, y read and p, y written (SQMR: and
  // d read and written)
  const double iter_bytes =
      (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 3.0 * vb + 3.0 * vb + (QMR ? 7.0 : 5.0) * vb;
  const T* sv = sell ? (c128 ? (const T*)B->s128.ptr : (const T*)B->s64.ptr) : nullptr;
  CgSys<T> hsys{(const int64_t*)c->row_ptr.as<int64_t>(),
                (const int32_t*)c->col.as<int32_t>(),
                at,
                p,
                q,
                r,
                y,
                dq,
                sell ? (const int64_t*)c->sell_sp.as<int64_t>() : nullptr,
                sell ? (const int32_t*)c->sell_col.as<int32_t>() : nullptr,
                sv,
                sell ? c->sell_ns : 0,
                n,
                st,
                part,
                0,
                0,
                grid};
  PG_TRY(B->sys.reserve(sizeof(CgSys<T>)));
  const CgSys<T>* dsys = B->sys.as<CgSys<T>>();
  CState hs;
  auto norm = [&](const double2* v, double* out) -> Status {
    k_cg_norm<<<nb, kT, 0, s>>>(v, n, st, part);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    PG_TRY(read_cstate(c, B, &hs));
    *out = hs.rn2;
    return Status{};
  };
  double bn2 = 0.0;
  PG_TRY(norm(b, &bn2));
  const double bnorm = sqrt(bn2);
  if (bnorm == 0.0) {
    PG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
    inf.status = PETGEM_OK;
    return Status{};
  }
  int64_t iters = 0, solves = 0;
  double relres = 0.0;
  int status = PETGEM_OK, stalls = 0;
  double prev = INFINITY;
  while (true) {
    {
      KernelTimer kt(c, "cg_residual_c128", (double)c->nnz * 20 + 8.0 * (n + 1) + 48.0 * n);
      k_cg_residual<kCgG><<<blocks_for(n * kCgG, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                                    c->val.as<double2>(), x, b, B->r64.as<double2>(),
                                                                    n);
      c->launches++;
    }
    double rn2 = 0.0;
    PG_TRY(norm(B->r64.as<double2>(), &rn2));
    relres = sqrt(rn2) / bnorm;
    if (!isfinite(relres)) {
      status = PETGEM_ERR_BREAKDOWN;
      break;
    }
    if (relres <= o.tol) break;
    if (iters >= o.max_iters) {
      status = PETGEM_ERR_NOT_CONVERGED;
      break;
    }
    // restarts that no longer halve the FP64 residual: stagnation at the rounding floor
    stalls = relres > 0.5 * prev ? stalls + 1 : 0;
    if (stalls >= 3) {
      status = PETGEM_ERR_NOT_CONVERGED;
      break;
    }
    prev = relres;
    // Inner target: reduce the scaled residual by inner_tol (mixed) but not much below what the
    // final tolerance still needs (0.3 tol ||b|| / ||r||, a margin for the scaling by S); c128
    // aims at that need directly.
    const double rnorm = sqrt(rn2);
    const double need = 0.3 * o.tol * bnorm / rnorm;
    const double inner = c128 ? need : std::min(std::max(o.inner_tol, need), 0.5);
    k_cg_start<T><<<nb, kT, 0, s>>>(B->r64.as<double2>(), B->sq.as<double2>(), perm, r, p, y, dq, n, st, part, inner,
                                    1.0 / rnorm);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    hs.k = 0;
    // this inner solve's iteration budget: what is left, and in complex64 at most kCgInnerMax (the
    // recursively updated residual drifts from the true one in FP32 over long solves; a fresh FP64
    // residual bounds the drift)
    hsys.kmax = std::min<int64_t>(o.max_iters - iters, c128 ? INT64_MAX : kCgInnerMax);
    PG_CUDA(cudaMemcpyAsync(B->sys.ptr, &hsys, sizeof(hsys), cudaMemcpyHostToDevice, s));
    // the iterations of this inner solve: persistent launches of up to kCgChunk iterations each
    while (true) {
      const int steps = (int)std::min<int64_t>(kCgChunk, hsys.kmax - hs.k);
      if (steps <= 0) break;
      {
        KernelTimer kt(c, QMR ? (c128 ? "qmr_inner_c128" : "qmr_inner_c64") : (c128 ? "cg_inner_c128" : "cg_inner_c64"),
                       0.0);
        if (sell)
          PG_CUDA(pdl_launch(k_cg_inner<T, kCgG, QMR, true>, dim3(grid), dim3(256), 0, s, true, dsys, 1, steps));
        else
          PG_CUDA(pdl_launch(k_cg_inner<T, kCgG, QMR, false>, dim3(grid), dim3(256), 0, s, true, dsys, 1, steps));
      }
      c->launches++;
      const int k0 = hs.k;
      PG_TRY(read_cstate(c, B, &hs));
      set_last_timing_bytes(c, (hs.k - k0) * iter_bytes);
      if (hs.done) break;
    }
    k_cg_finish<T><<<blocks_for(n, 256), 256, 0, s>>>(y, B->sq.as<double2>(), perm, x, n, rnorm);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    iters += hs.k;
    solves += 1;
    if (hs.done == 3) {  // a barrier of the persistent kernel gave up
      status = PETGEM_ERR_TIMEOUT;
      break;
    }
    if (hs.done == 2 && hs.k == 0) {  // the bilinear form broke down at once: no progress possible
      status = PETGEM_ERR_BREAKDOWN;
      break;
    }
  }
  inf.iters = iters;
  inf.restarts = solves;
  inf.refinements = solves;
  inf.true_rel_residual = relres;
  inf.status = status;
  return Status{};
}

// ------------------------------------------------------------------ multi-source COCG
// P sources of one frequency iterate in lockstep (element (row i, source s) at i * P + s), each
// with its own scalars, normalisation and stopping test; the matrix is read once per step for all
// of them (the SpMM).  A source that met its inner target, or is already converged, stops updating
// while the others go on.
struct BGrp {
  unsigned counter;
  int all_done;
};

template <int P>
__global__ void k_bcg_in(const double2* __restrict__ b, const double2* __restrict__ x, int64_t n, int S_g,
                         double2* __restrict__ Bt, double2* __restrict__ X) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t i = e / P;
  const int s = (int)(e - i * P);
  Bt[e] = s < S_g ? b[(int64_t)s * n + i] : make_double2(0.0, 0.0);
  X[e] = s < S_g ? x[(int64_t)s * n + i] : make_double2(0.0, 0.0);
}

template <int P>
__global__ void k_bcg_out(const double2* __restrict__ X, int64_t n, int S_g, double2* __restrict__ x) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t i = e / P;
  const int s = (int)(e - i * P);
  if (s < S_g) x[(int64_t)s * n + i] = X[e];
}

// R = Bt - A X in FP64, P lanes per row (lane = source).
template <int P>
__global__ void __launch_bounds__(256) k_bcg_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const double2* __restrict__ val, const double2* __restrict__ X,
                                                      const double2* __restrict__ Bt, double2* __restrict__ R,
                                                      int64_t n) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / P;
  const int s = (int)(gid % P);
  if (row >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t p = rp[row]; p < rp[row + 1]; ++p) fma_c(acc, __ldg(&val[p]), X[(int64_t)__ldg(&col[p]) * P + s]);
  R[row * P + s] = csub(Bt[row * P + s], acc);
}

// Per-source sums of partials[b * P + s] (double2) over b < nb, one warp per source; every lane of
// warp w returns the total of source w.
template <int P>
__device__ inline double2 source_total(const double2* partials, int nb, int s) {
  const int lane = threadIdx.x & 31;
  double2 a = make_double2(0.0, 0.0);
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int b = b0 + lane + 32 * m;
      v[m] = b < nb ? __ldcg(&partials[((int64_t)b * 2) * P + s]) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) a = cadd(a, v[m]);
  }
  return warp_sum(a);
}
template <int P>
__device__ inline double2 source_total2(const double2* partials, int nb, int s) {
  const int lane = threadIdx.x & 31;
  double2 a = make_double2(0.0, 0.0);
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int b = b0 + lane + 32 * m;
      v[m] = b < nb ? __ldcg(&partials[((int64_t)b * 2 + 1) * P + s]) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) a = cadd(a, v[m]);
  }
  return warp_sum(a);
}

// Block sums of two per-source accumulators into partials[(b * 2 + slot) * P + s]: the thread's
// source is tid mod P (grid strides are multiples of P); tree over the lanes of one source in the
// accumulator's precision, FP64 across warps.
template <int NT, int P, typename A>
__device__ inline void source_partials2(A a0, A a1, double2* partials) {
  __shared__ double2 red[NT / 32][2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= P; o >>= 1) {
    a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
    a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
    a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
    a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
  }
  if (lane < P) {
    red[warp][0][lane] = to_d2(a0);
    red[warp][1][lane] = to_d2(a1);
  }
  __syncthreads();
  if (threadIdx.x < 2 * P) {
    const int slot = threadIdx.x / P, s = threadIdx.x % P;
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) t = cadd(t, red[w][slot][s]);
    partials[((int64_t)blockIdx.x * 2 + slot) * P + s] = t;
  }
}

constexpr int kBcgThreads = 512;  // persistent vector kernels: two blocks per SM

// Per-source ||v_s||^2 (FP64 data) into sts[s].rn2.
template <int P>
__global__ void __launch_bounds__(kBcgThreads) k_bcg_norms(const double2* __restrict__ V, int64_t n,
                                                           CState* __restrict__ sts, BGrp* __restrict__ g,
                                                           double2* __restrict__ partials) {
  double a = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)kBcgThreads + threadIdx.x; e < n * P; e += (int64_t)gridDim.x * kBcgThreads)
    a += nrm2(V[e]);
  source_partials2<kBcgThreads, P>(make_double2(a, 0.0), make_double2(0.0, 0.0), partials);
  if (!last_block(&g->counter)) return;
  const int warp = threadIdx.x >> 5;
  for (int s = warp; s < P; s += kBcgThreads / 32) {
    const double2 t = source_total<P>(partials, gridDim.x, s);
    if ((threadIdx.x & 31) == 0) sts[s].rn2 = t.x;
  }
  __syncthreads();
  if (threadIdx.x == 0) g->counter = 0;
}

// Inner-solve start per source: r = p = scale_s S R (rounded to T), y = 0; rho_s, ||r_s||^2, the
// threshold inner_s^2 ||r_s||^2; scale_s = 0 marks a source that takes no part (done at once).
template <typename T, int P>
__global__ void __launch_bounds__(kBcgThreads) k_bcg_start(const double2* __restrict__ R,
                                                           const double2* __restrict__ sq,
                                                           const double* __restrict__ scal, T* __restrict__ r,
                                                           T* __restrict__ p, T* __restrict__ y, int64_t n,
                                                           CState* __restrict__ sts, BGrp* __restrict__ g,
                                                           double2* __restrict__ partials) {
  using A = typename Acc<T>::type;
  const int s = threadIdx.x % P;
  const double sc = scal[s];
  A rho = zero<T>(), nr = zero<T>();
  for (int64_t e = blockIdx.x * (int64_t)kBcgThreads + threadIdx.x; e < n * P;
       e += (int64_t)gridDim.x * kBcgThreads) {
    const T t = from_d2<T>(cscale(cmul(sq[e / P], R[e]), sc));
    r[e] = t;
    p[e] = t;
    y[e] = zero<T>();
    bil_fma(rho, t, t);
    nr.x += nrm2(t);
  }
  source_partials2<kBcgThreads, P>(rho, nr, partials);
  if (!last_block(&g->counter)) return;
  const int warp = threadIdx.x >> 5;
  for (int q = warp; q < P; q += kBcgThreads / 32) {
    const double2 a = source_total<P>(partials, gridDim.x, q);
    const double2 b = source_total2<P>(partials, gridDim.x, q);
    if ((threadIdx.x & 31) == 0) {
      CState* st = &sts[q];
      const double inner = scal[P + q];
      st->rho = a;
      st->nr0 = b.x;
      st->nr = b.x;
      st->stop2 = inner * inner * b.x;
      st->k = 0;
      st->done = (scal[q] != 0.0 && b.x > 0.0 && isfinite(b.x)) ? 0 : ((scal[q] == 0.0 || b.x == 0.0) ? 1 : 2);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int alive = 0;
    for (int q = 0; q < P; ++q) alive += sts[q].done == 0;
    g->all_done = alive == 0;
    g->counter = 0;
  }
}


// Q = Atil Pm for all P sources: the row's entries read by its lane group four at a time (the
// wavefront form of the block GMRES SpMM).
template <typename T, int P>
__global__ void __launch_bounds__(256) k_bcg_spmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                  const T* __restrict__ val, const T* __restrict__ Pm,
                                                  T* __restrict__ Q, int64_t n, const BGrp* __restrict__ g) {
  pdl_trigger();
  pdl_wait();
  if (g->all_done) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / P;
  const int s = (int)(gid % P);
  if (row >= n) return;
  typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
  const int64_t p1 = rp[row + 1];
  int64_t pp = rp[row];
  for (; pp + 4 <= p1; pp += 4) {
    int64_t cc[4];
    T aa[4], xx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cc[u] = __ldg(&col[pp + u]);
      aa[u] = __ldg(&val[pp + u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xx[u] = Pm[cc[u] * P + s];
    fma_c(acc, aa[0], xx[0]);
    fma_c(acc2, aa[1], xx[1]);
    fma_c(acc, aa[2], xx[2]);
    fma_c(acc2, aa[3], xx[3]);
  }
  for (; pp < p1; ++pp) fma_c(acc, __ldg(&val[pp]), Pm[(int64_t)__ldg(&col[pp]) * P + s]);
  acc.x += acc2.x;
  acc.y += acc2.y;
  Q[row * P + s] = from_d2<T>(to_d2(acc));
}

// Per-source p_s^T q_s; the last block forms alpha_s for every live source.
template <typename T, int P>
__global__ void __launch_bounds__(kBcgThreads) k_bcg_pq(const T* __restrict__ Pm, const T* __restrict__ Q, int64_t n,
                                                        CState* __restrict__ sts, BGrp* __restrict__ g,
                                                        double2* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (g->all_done) return;
  using A = typename Acc<T>::type;
  A d = zero<T>();
  for (int64_t e = blockIdx.x * (int64_t)kBcgThreads + threadIdx.x; e < n * P; e += (int64_t)gridDim.x * kBcgThreads)
    bil_fma(d, Pm[e], Q[e]);
  source_partials2<kBcgThreads, P>(d, zero<T>(), partials);
  if (!last_block(&g->counter)) return;
  const int warp = threadIdx.x >> 5;
  for (int q = warp; q < P; q += kBcgThreads / 32) {
    const double2 pq = source_total<P>(partials, gridDim.x, q);
    if ((threadIdx.x & 31) == 0) {
      CState* st = &sts[q];
      if (st->done == 0) {
        if (!(cabs2(pq) > 0.0) || !isfinite(pq.x) || !isfinite(pq.y)) {
          st->done = 2;
        } else {
          const double2 al = cdiv(st->rho, pq);
          st->alpha = al;
          st->alpha32 = make_float2((float)al.x, (float)al.y);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) g->counter = 0;
}

// y_s += alpha_s p_s, r_s -= alpha_s q_s for live sources; rho'_s, ||r_s||^2; the last block forms
// beta_s and the stopping tests.
template <typename T, int P>
__global__ void __launch_bounds__(kBcgThreads) k_bcg_update(const T* __restrict__ Pm, const T* __restrict__ Q,
                                                            T* __restrict__ r, T* __restrict__ y, int64_t n,
                                                            CState* __restrict__ sts, BGrp* __restrict__ g,
                                                            double2* __restrict__ partials) {
  pdl_trigger();
  pdl_wait();
  if (g->all_done) return;
  using A = typename Acc<T>::type;
  const int s = threadIdx.x % P;
  const bool live = sts[s].done == 0;
  const T al = cg_alpha<T>(&sts[s]);
  A rho = zero<T>(), nr = zero<T>();
  if (live)
    for (int64_t e = blockIdx.x * (int64_t)kBcgThreads + threadIdx.x; e < n * P;
         e += (int64_t)gridDim.x * kBcgThreads) {
      const T pv = Pm[e], qv = Q[e];
      T yv = y[e], rv = r[e];
      fma_c(yv, al, pv);
      sub_mul(rv, qv, al);
      y[e] = yv;
      r[e] = rv;
      bil_fma(rho, rv, rv);
      nr.x += nrm2(rv);
    }
  source_partials2<kBcgThreads, P>(rho, nr, partials);
  if (!last_block(&g->counter)) return;
  const int warp = threadIdx.x >> 5;
  for (int q = warp; q < P; q += kBcgThreads / 32) {
    const double2 rh = source_total<P>(partials, gridDim.x, q);
    const double2 nn = source_total2<P>(partials, gridDim.x, q);
    if ((threadIdx.x & 31) == 0) {
      CState* st = &sts[q];
      if (st->done == 0) {
        st->k += 1;
        st->nr = nn.x;
        if (!isfinite(nn.x)) {
          st->done = 2;
        } else if (nn.x <= st->stop2) {
          st->done = 1;
        } else if (!(cabs2(st->rho) > 0.0)) {
          st->done = 2;
        } else {
          const double2 be = cdiv(rh, st->rho);
          st->beta = be;
          st->beta32 = make_float2((float)be.x, (float)be.y);
          st->rho = rh;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int alive = 0;
    for (int q = 0; q < P; ++q) alive += sts[q].done == 0;
    g->all_done = alive == 0;
    g->counter = 0;
  }
}

// p_s = r_s + beta_s p_s for live sources.
template <typename T, int P>
__global__ void __launch_bounds__(kBcgThreads) k_bcg_dir(const T* __restrict__ r, T* __restrict__ Pm, int64_t n,
                                                         const CState* __restrict__ sts,
                                                         const BGrp* __restrict__ g) {
  pdl_trigger();
  pdl_wait();
  if (g->all_done) return;
  const int s = threadIdx.x % P;
  if (sts[s].done != 0) return;
  const T be = cg_beta<T>(&sts[s]);
  for (int64_t e = blockIdx.x * (int64_t)kBcgThreads + threadIdx.x; e < n * P;
       e += (int64_t)gridDim.x * kBcgThreads) {
    T pv = r[e];
    fma_c(pv, be, Pm[e]);
    Pm[e] = pv;
  }
}

// X_s += ||r_s|| S y_s for the sources that took part (scale != 0).
template <typename T, int P>
__global__ void k_bcg_finish(const T* __restrict__ y, const double2* __restrict__ sq, const double* __restrict__ scal,
                             double2* __restrict__ X, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int s = (int)(e % P);
  const double sc = scal[s];
  if (sc == 0.0) return;
  X[e] = cadd(X[e], cscale(cmul(sq[e / P], to_d2(y[e])), 1.0 / sc));
}

template <typename T, int P>
Status cocg_group(petgem_ctx* c, const petgem_solve_opts& o, CgBuffers* B, const double2* b, double2* x, int S_g,
                  petgem_solve_info* info, int sms) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges, nP = n * P;
  const bool c128 = sizeof(T) == 16;
  PG_TRY(B->Bt.reserve(nP * sizeof(double2)));
  PG_TRY(B->X.reserve(nP * sizeof(double2)));
  PG_TRY(B->R.reserve(nP * sizeof(double2)));
  for (DevBuf* d : {&B->rb, &B->pb, &B->qb, &B->yb}) PG_TRY(d->reserve(nP * sizeof(T)));
  PG_TRY(B->bstates.reserve(P * sizeof(CState)));
  PG_TRY(B->bgrp.reserve(sizeof(BGrp)));
  PG_TRY(B->bscal.reserve(2 * P * sizeof(double)));
  const unsigned vgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_for(nP, kBcgThreads), 2LL * sms));
  PG_TRY(B->partials.reserve((size_t)vgrid * 2 * P * sizeof(double2) +
                             (size_t)std::max<int64_t>(blocks_for(n, kRows), 8LL * sms) * kPStride * sizeof(double2)));
  CState* sts = B->bstates.as<CState>();
  BGrp* grp = B->bgrp.as<BGrp>();
  double2* part = B->partials.as<double2>();
  double* scal = B->bscal.as<double>();
  const T* at = c128 ? (const T*)B->a128.ptr : (const T*)B->a64.ptr;
  T *r = B->rb.as<T>(), *pm = B->pb.as<T>(), *q = B->qb.as<T>(), *y = B->yb.as<T>();
  double2 *Bt = B->Bt.as<double2>(), *X = B->X.as<double2>(), *R = B->R.as<double2>();
  PG_CUDA(cudaMemsetAsync(sts, 0, P * sizeof(CState), s));
  PG_CUDA(cudaMemsetAsync(grp, 0, sizeof(BGrp), s));
  k_bcg_in<P><<<blocks_for(nP, 256), 256, 0, s>>>(b, x, n, S_g, Bt, X);
  c->launches++;
  std::vector<CState> hs(P);
  auto norms = [&](const double2* V) -> Status {
    k_bcg_norms<P><<<vgrid, kBcgThreads, 0, s>>>(V, n, sts, grp, part);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    PG_CUDA(cudaMemcpyAsync(hs.data(), sts, P * sizeof(CState), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    return Status{};
  };
  PG_TRY(norms(Bt));
  std::vector<double> bn(P), relres(P, 0.0), prev(P, INFINITY), hscal(2 * P, 0.0);
  std::vector<int64_t> iters(P, 0), solves(P, 0);
  std::vector<int> status(P, PETGEM_OK), finished(P, 0), stalls(P, 0);
  for (int i = 0; i < P; ++i) {
    bn[i] = sqrt(hs[i].rn2);
    if (i >= S_g || bn[i] == 0.0) finished[i] = 1;
  }
  const int chunk = std::max(1, o.restart);
  const double vb = (double)nP * sizeof(T);
  const double spmm_bytes = (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 2.0 * vb;
  int64_t max_done = 0;
  const unsigned spmm_grid = blocks_for(nP, 256);
  // SpMM form for this mesh and group size (autotuned on the direction and product buffers before
  // the first inner solve writes them; the group state is zero, so every launch runs in full)
  int spmm_form = -1;
  if (o.spmv_lanes == 0) {
    PG_TRY((tune_spmm<T, P>(c, s, at, pm, q,
                            [&]() -> Status {
                              PG_CUDA(pdl_launch(k_bcg_spmm<T, P>, dim3(spmm_grid), dim3(256), 0, s, false,
                                                 (const int64_t*)c->row_ptr.as<int64_t>(),
                                                 (const int32_t*)c->col.as<int32_t>(), at, (const T*)pm, q, n,
                                                 (const BGrp*)grp));
                              return Status{};
                            },
                            &spmm_form)));
  } else if (o.spmv_lanes != 1) {
    spmm_form = o.spmv_lanes == 16 ? 0 : o.spmv_lanes == 32 ? 1 : o.spmv_lanes == 64 ? 2 : -2;
    if (spmm_form < 0) return Status{PETGEM_ERR_UNSUPPORTED, "block SpMM: spmv_lanes must be 0, 1, 16, 32 or 64"};
    PG_TRY(band_layout(c, spmm_form));
    if ((size_t)c->bands[spmm_form].max_u * P * sizeof(T) > kBandSmemMax)
      return Status{PETGEM_ERR_UNSUPPORTED, "block SpMM: the bands of this height are too wide"};
  }
  while (true) {
    {
      KernelTimer kt(c, "bcg_residual_c128", (double)c->nnz * 20 + 48.0 * nP);
      k_bcg_residual<P><<<blocks_for(nP, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                           c->val.as<double2>(), X, Bt, R, n);
      c->launches++;
    }
    PG_TRY(norms(R));
    bool all = true;
    for (int i = 0; i < P; ++i) {
      if (finished[i]) {
        hscal[i] = 0.0;
        continue;
      }
      const double rn = sqrt(hs[i].rn2);
      relres[i] = rn / bn[i];
      if (!isfinite(relres[i])) {
        status[i] = PETGEM_ERR_BREAKDOWN;
        finished[i] = 1;
      } else if (relres[i] <= o.tol) {
        finished[i] = 1;
      } else if (iters[i] >= o.max_iters) {
        status[i] = PETGEM_ERR_NOT_CONVERGED;
        finished[i] = 1;
      } else {
        stalls[i] = relres[i] > 0.5 * prev[i] ? stalls[i] + 1 : 0;
        if (stalls[i] >= 3) {
          status[i] = PETGEM_ERR_NOT_CONVERGED;
          finished[i] = 1;
        }
      }
      prev[i] = relres[i];
      if (finished[i]) {
        hscal[i] = 0.0;
        continue;
      }
      all = false;
      const double need = 0.3 * o.tol * bn[i] / rn;
      hscal[i] = 1.0 / rn;
      hscal[P + i] = c128 ? need : std::min(std::max(o.inner_tol, need), 0.5);
    }
    if (all) break;
    PG_CUDA(cudaMemcpyAsync(scal, hscal.data(), 2 * P * sizeof(double), cudaMemcpyHostToDevice, s));
    k_bcg_start<T, P><<<vgrid, kBcgThreads, 0, s>>>(R, B->sq.as<double2>(), scal, r, pm, y, n, sts, grp, part);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    int64_t done_iters = 0;
    BGrp hg{};
    while (true) {
      // complex64 inner solves stop after at most kCgInnerMax iterations, as the single-source
      // solver's do (a complex64 COCG left running drifts); the FP64 refinement restarts them
      int64_t steps = std::min<int64_t>(chunk, o.max_iters - max_done - done_iters);
      if (!c128) steps = std::min<int64_t>(steps, kCgInnerMax - done_iters);
      if (steps <= 0) break;
      for (int64_t k = 0; k < steps; ++k) {
        {
          KernelTimer kt(c, c128 ? "bcg_spmm_c128" : "bcg_spmm_c64", spmm_bytes);
          if (spmm_form >= 0)
            PG_TRY((launch_spmm_band<T, P>(c, s, spmm_form, at, (const T*)pm, q, &grp->all_done, SpmmStorePlain{})));
          else
            PG_CUDA(pdl_launch(k_bcg_spmm<T, P>, dim3(spmm_grid), dim3(256), 0, s, false,
                               (const int64_t*)c->row_ptr.as<int64_t>(), (const int32_t*)c->col.as<int32_t>(), at,
                               (const T*)pm, q, n, (const BGrp*)grp));
        }
        {
          KernelTimer kt(c, c128 ? "bcg_pq_c128" : "bcg_pq_c64", 2.0 * vb);
          PG_CUDA(pdl_launch(k_bcg_pq<T, P>, dim3(vgrid), dim3(kBcgThreads), 0, s, false, (const T*)pm, (const T*)q, n,
                             sts, grp, part));
        }
        {
          KernelTimer kt(c, c128 ? "bcg_update_c128" : "bcg_update_c64", 6.0 * vb);
          PG_CUDA(pdl_launch(k_bcg_update<T, P>, dim3(vgrid), dim3(kBcgThreads), 0, s, false, (const T*)pm,
                             (const T*)q, r, y, n, sts, grp, part));
        }
        {
          KernelTimer kt(c, c128 ? "bcg_dir_c128" : "bcg_dir_c64", 3.0 * vb);
          PG_CUDA(pdl_launch(k_bcg_dir<T, P>, dim3(vgrid), dim3(kBcgThreads), 0, s, false, (const T*)r, pm, n,
                             (const CState*)sts, (const BGrp*)grp));
        }
        c->launches += 4;
      }
      done_iters += steps;
      PG_CUDA(cudaMemcpyAsync(&hg, grp, sizeof(BGrp), cudaMemcpyDeviceToHost, s));
      PG_CUDA(cudaStreamSynchronize(s));
      if (hg.all_done) break;
    }
    PG_CUDA(cudaMemcpyAsync(hs.data(), sts, P * sizeof(CState), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    k_bcg_finish<T, P><<<blocks_for(nP, 256), 256, 0, s>>>(y, B->sq.as<double2>(), scal, X, n);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    for (int i = 0; i < P; ++i) {
      if (finished[i]) continue;
      iters[i] += hs[i].k;
      solves[i] += 1;
      max_done = std::max(max_done, iters[i]);
      if (hs[i].done == 2 && hs[i].k == 0) {  // the bilinear form broke down at once
        status[i] = PETGEM_ERR_BREAKDOWN;
        finished[i] = 1;
      }
    }
  }
  k_bcg_out<P><<<blocks_for(nP, 256), 256, 0, s>>>(X, n, S_g, x);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  for (int i = 0; i < S_g; ++i) {
    info[i] = petgem_solve_info{};
    info[i].iters = iters[i];
    info[i].restarts = solves[i];
    info[i].refinements = solves[i];
    info[i].true_rel_residual = relres[i];
    info[i].status = status[i];
    info[i].spmv_lanes = spmm_form >= 0 ? kBandHeights[spmm_form] : 1;
  }
  return Status{};
}

template <typename T>
Status cocg_group_p(petgem_ctx* c, const petgem_solve_opts& o, CgBuffers* B, const double2* b, double2* x, int S_g,
                    petgem_solve_info* info, int sms) {
  if (S_g <= 2) return cocg_group<T, 2>(c, o, B, b, x, S_g, info, sms);
  if (S_g <= 4) return cocg_group<T, 4>(c, o, B, b, x, S_g, info, sms);
  if (S_g <= 8) return cocg_group<T, 8>(c, o, B, b, x, S_g, info, sms);
  if (S_g <= 16) return cocg_group<T, 16>(c, o, B, b, x, S_g, info, sms);
  return cocg_group<T, 32>(c, o, B, b, x, S_g, info, sms);
}

// The scaled operator Atil = S A S (complex128 and complex64) and S = D^{-1/2} of the context's
// current assembly, built once per assembly on the context's stream.
Status cg_prepare(petgem_ctx* c) {
  CgBuffers* B = cg_bufs(c);
  if (B->version == c->assembly_version) return Status{};
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  PG_TRY(B->sq.reserve(n * sizeof(double2)));
  PG_TRY(B->a128.reserve(c->nnz * sizeof(double2)));
  PG_TRY(B->a64.reserve(c->nnz * sizeof(float2)));
  k_cg_sqrt_diag<<<blocks_for(n, 256), 256, 0, s>>>(c->diag.as<double2>(), n, B->sq.as<double2>());
  k_cg_scale<<<blocks_for(n, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->val.as<double2>(),
                                                B->sq.as<double2>(), n, B->a128.as<double2>(), B->a64.as<float2>());
  c->launches += 2;
  PG_CUDA(cudaGetLastError());
  // the same operator in the SELL-32 layout
  PG_TRY(sell_prepare(c));
  if (c->sell_ok) {
    PG_TRY(B->s64.reserve(c->sell_nnz * sizeof(float2)));
    PG_TRY(B->s128.reserve(c->sell_nnz * sizeof(double2)));
    PG_TRY(sell_values<float2>(c, B->a64.as<float2>(), B->s64.as<float2>()));
    PG_TRY(sell_values<double2>(c, B->a128.as<double2>(), B->s128.as<double2>()));
  }
  B->version = c->assembly_version;
  return Status{};
}

// ------------------------------------------------------------------ batch of meshes
// The systems of several contexts (meshes of different sizes, each with its sources) solved
// together.  Their inner iterations share one persistent launch (k_cg_inner over a table of
// systems, each on its own blocks); their FP64 refinement steps run as five launches per round
// for all systems at once (finish, residual, norm, decide, start: each kernel's blocks are divided
// among the systems), which a CUDA graph replays when asked.

// Refinement-side view of one system.
struct CgCtl {
  double bnorm, relres, prev, scale, inner;  // scale = 1 / ||r|| of the current inner solve
  int64_t iters, solves;
  int stalls, status, active, ran;
};
template <typename T>
struct CgRef {
  const int64_t* rp;
  const int32_t* col;
  const double2* val;  // the assembled FP64 matrix (true residual)
  const double2* sq;   // S = D^{-1/2}
  const double2* b;
  double2* x;
  double2* r64;
  T *r, *p, *y;
  const int32_t* perm;  // the inner solve's vectors in the SELL renumbering (null: original order)
  CState* st;
  double2* part;
  CgCtl* ctl;
  int64_t n;
  int v0, vnb;  // blocks of the vector kernels (256 elements each)
  int r0, rnb;  // blocks of the residual kernel (256 / kCgG rows each)
};
constexpr int kBatchMax = 64;        // systems per batch
constexpr int kBatchTuneSteps = 2;   // iterations per timed launch of the autotuner

// The system whose block range [v0, v0 + vnb) (resid: [r0, r0 + rnb)) holds this block.
template <typename T, bool RESID>
__device__ inline int batch_sys(const CgRef<T>* R, int ns) {
  __shared__ int s_k;
  if (threadIdx.x == 0) {
    int k = 0;
    while (k + 1 < ns && (int)blockIdx.x >= (RESID ? R[k + 1].r0 : R[k + 1].v0)) ++k;
    s_k = k;
  }
  __syncthreads();
  return s_k;
}

// "Last block of this system" handshake over nb blocks with the system's own counter.
__device__ inline bool last_of(unsigned* counter, unsigned nb) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == nb - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// x += ||r|| S y for the systems whose inner solve ran in the last round.
template <typename T>
__global__ void __launch_bounds__(256) k_cgb_finish(const CgRef<T>* __restrict__ R, int ns) {
  const int k = batch_sys<T, false>(R, ns);
  const CgRef<T>& S = R[k];
  if (!S.ctl->ran) return;
  const double unscale = 1.0 / S.ctl->scale;
  for (int64_t i = (int64_t)(blockIdx.x - S.v0) * 256 + threadIdx.x; i < S.n; i += (int64_t)S.vnb * 256) {
    const int64_t o = S.perm ? S.perm[i] : i;
    S.x[o] = cadd(S.x[o], cscale(cmul(S.sq[o], to_d2(S.y[i])), unscale));
  }
}

// r64 = b - A x (FP64) for the active systems, kCgG lanes per row.
template <typename T>
__global__ void __launch_bounds__(256) k_cgb_residual(const CgRef<T>* __restrict__ R, int ns) {
  const int k = batch_sys<T, true>(R, ns);
  const CgRef<T>& S = R[k];
  if (!S.ctl->active) return;
  const int lane = threadIdx.x % kCgG;
  for (int64_t row = (int64_t)(blockIdx.x - S.r0) * (256 / kCgG) + threadIdx.x / kCgG;
       __any_sync(0xffffffffu, row < S.n); row += (int64_t)S.rnb * (256 / kCgG)) {
    double2 acc = make_double2(0.0, 0.0);
    if (row < S.n)
      for (int64_t q = S.rp[row] + lane; q < S.rp[row + 1]; q += kCgG) fma_c(acc, S.val[q], S.x[S.col[q]]);
    for (int o = kCgG / 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (row < S.n && lane == 0) S.r64[row] = csub(S.b[row], acc);
  }
}

// ||v||^2 (v = r64, or b when of_b) into st->rn2 for the active systems (every system when of_b).
template <typename T>
__global__ void __launch_bounds__(256) k_cgb_norm(const CgRef<T>* __restrict__ R, int ns, int of_b) {
  const int k = batch_sys<T, false>(R, ns);
  const CgRef<T>& S = R[k];
  if (!of_b && !S.ctl->active) return;
  const double2* v = of_b ? S.b : S.r64;
  const int lb = blockIdx.x - S.v0;
  double a = 0.0;
  for (int64_t i = (int64_t)lb * 256 + threadIdx.x; i < S.n; i += (int64_t)S.vnb * 256) a += nrm2(v[i]);
  cg_block_sums<256>(make_double2(a, 0.0), make_double2(0.0, 0.0), S.part + (int64_t)lb * kCgSlots);
  if (!last_of(&S.st->counter, S.vnb)) return;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < S.vnb; b += 32) t += __ldcg(&S.part[(int64_t)b * kCgSlots]).x;
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      S.st->rn2 = t;
      S.st->counter = 0;
      if (of_b) {  // the batch's start: ||b||, and which systems have anything to solve
        CgCtl* c = S.ctl;
        c->bnorm = sqrt(t);
        c->relres = 0.0;
        c->prev = INFINITY;
        c->iters = c->solves = 0;
        c->stalls = 0;
        c->status = PETGEM_OK;
        c->active = c->bnorm > 0.0;
        c->ran = 0;
      }
    }
  }
}

// One thread per system: book the inner solve that just ran, then the stopping decision on the
// FP64 residual and the next inner solve's target and scale (the host-side rules of the
// single-system solver, on the device so that the round needs no host round trip).
__global__ void k_cgb_decide(CgCtl* __restrict__ ctl, const CState* __restrict__ st, int ns, double tol,
                             double inner_tol, int64_t max_iters, int c128) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  CgCtl& c = ctl[k];
  if (c.ran) {
    c.iters += st[k].k;
    c.solves += 1;
    if (st[k].done == 3) {
      c.status = PETGEM_ERR_TIMEOUT;
      c.active = 0;
    } else if (st[k].done == 2 && st[k].k == 0) {
      c.status = PETGEM_ERR_BREAKDOWN;
      c.active = 0;
    }
    c.ran = 0;
  }
  if (!c.active) return;
  const double rnorm = sqrt(st[k].rn2);
  c.relres = rnorm / c.bnorm;
  if (!isfinite(c.relres)) {
    c.status = PETGEM_ERR_BREAKDOWN;
    c.active = 0;
  } else if (c.relres <= tol) {
    c.active = 0;
  } else if (c.iters >= max_iters) {
    c.status = PETGEM_ERR_NOT_CONVERGED;
    c.active = 0;
  } else {
    c.stalls = c.relres > 0.5 * c.prev ? c.stalls + 1 : 0;  // no longer halving: rounding floor
    if (c.stalls >= 3) {
      c.status = PETGEM_ERR_NOT_CONVERGED;
      c.active = 0;
    }
  }
  c.prev = c.relres;
  if (!c.active) return;
  const double need = 0.3 * tol * c.bnorm / rnorm;
  c.inner = c128 ? need : fmin(fmax(inner_tol, need), 0.5);
  c.scale = 1.0 / rnorm;
}

// Inner-solve start of every active system (as k_cg_start); an inactive system is marked done so
// that the persistent kernel's blocks skip it.
template <typename T>
__global__ void __launch_bounds__(256) k_cgb_start(const CgRef<T>* __restrict__ R, int ns) {
  const int k = batch_sys<T, false>(R, ns);
  const CgRef<T>& S = R[k];
  const int lb = blockIdx.x - S.v0;
  if (!S.ctl->active) {
    if (lb == 0 && threadIdx.x == 0) S.st->done = 1;
    return;
  }
  using A = typename Acc<T>::type;
  const double scale = S.ctl->scale;
  A rho = zero<T>(), nr = zero<T>();
  for (int64_t i = (int64_t)lb * 256 + threadIdx.x; i < S.n; i += (int64_t)S.vnb * 256) {
    const int64_t o = S.perm ? S.perm[i] : i;
    const T t = from_d2<T>(cscale(cmul(S.sq[o], S.r64[o]), scale));
    S.r[i] = t;
    S.p[i] = t;
    S.y[i] = zero<T>();
    bil_fma(rho, t, t);
    nr.x += nrm2(t);
  }
  cg_block_sums<256>(rho, nr, S.part + (int64_t)lb * kCgSlots);
  if (!last_of(&S.st->counter, S.vnb)) return;
  __shared__ double2 tot[2];
  cg_sum_blocks2<256>(S.part, S.vnb, 0, 1, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    CState* st = S.st;
    const double2 a = tot[0], b = tot[1];
    const double inner = S.ctl->inner;
    st->rho = a;
    st->nr0 = b.x;
    st->nr = b.x;
    st->stop2 = inner * inner * b.x;
    st->k = 0;
    st->done = (b.x > 0.0 && isfinite(b.x)) ? 0 : (b.x == 0.0 ? 1 : 2);
    st->gbar = 0;
    st->grel = 0;
    st->counter = 0;
    S.ctl->ran = 1;
  }
}

// Blocks of the persistent kernel for the active systems: in proportion to each system's matrix
// entries times its expected iterations (the last inner solve's, or E^(1/3) before any ran), at
// least one and at most what its rows fill.
inline void batch_partition(const std::vector<int>& act, const std::vector<double>& work,
                            const std::vector<int64_t>& cap, int total, std::vector<int>& nb) {
  double sum = 0.0;
  for (int k : act) sum += work[k];
  int used = 0;
  for (int k : act) {
    nb[k] = (int)std::max<int64_t>(1, std::min<int64_t>(cap[k], (int64_t)(total * work[k] / sum)));
    used += nb[k];
  }
  // hand out what rounding left, to the systems with the most work per block
  while (used < total) {
    int best = -1;
    double bw = 0.0;
    for (int k : act)
      if (nb[k] < cap[k] && work[k] / nb[k] > bw) {
        bw = work[k] / nb[k];
        best = k;
      }
    if (best < 0) break;
    nb[best] += 1;
    used += 1;
  }
  while (used > total) {  // more systems than blocks' worth of minimums cannot happen (kBatchMax)
    int best = -1;
    double bw = INFINITY;
    for (int k : act)
      if (nb[k] > 1 && work[k] / nb[k] < bw) {
        bw = work[k] / nb[k];
        best = k;
      }
    if (best < 0) break;
    nb[best] -= 1;
    used -= 1;
  }
}

struct BatchBuffers {
  DevBuf vec, st, part, ctl, sys, ref;
  cudaStream_t cap = nullptr;
};

template <int G, typename T>
Status batch_inner_launch(cudaStream_t s, const CgSys<T>* dsys, int na, int grid, int steps) {
  PG_TRY((cg_setup<T, G>()));
  PG_CUDA(pdl_launch(k_cg_inner<T, G, false>, dim3(grid), dim3(256), 0, s, true, dsys, na, steps));
  return Status{};
}

template <typename T>
Status batch_inner(int G, cudaStream_t s, const CgSys<T>* dsys, int na, int grid, int steps) {
  if (G == 1) {  // the SELL-32 products
    PG_TRY((cg_setup<T, kCgG, false, true>()));
    PG_CUDA(pdl_launch(k_cg_inner<T, kCgG, false, true>, dim3(grid), dim3(256), 0, s, true, dsys, na, steps));
    return Status{};
  }
  if (G == 2) return batch_inner_launch<2, T>(s, dsys, na, grid, steps);
  if (G == 8) return batch_inner_launch<8, T>(s, dsys, na, grid, steps);
  return batch_inner_launch<4, T>(s, dsys, na, grid, steps);
}

template <typename T>
Status solve_batch(petgem_ctx* const* ctxs, int n_ctx, const petgem_solve_opts& o, double2* const* x,
                   petgem_solve_info* info) {
  petgem_ctx* c0 = ctxs[0];
  cudaStream_t s = c0->stream;
  const bool c128 = sizeof(T) == 16;
  int sms = 0;
  PG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
  CgBuffers* B0 = cg_bufs(c0);
  if (!B0->batch) B0->batch = new BatchBuffers();
  BatchBuffers* W = B0->batch;
  // the systems
  struct Sys {
    petgem_ctx* c;
    int src;
    int64_t n, nnz;
  };
  std::vector<Sys> sys;
  for (int k = 0; k < n_ctx; ++k)
    for (int j = 0; j < ctxs[k]->n_src; ++j) sys.push_back(Sys{ctxs[k], j, ctxs[k]->n_edges, ctxs[k]->nnz});
  const int ns = (int)sys.size();
  if (ns == 0) return Status{};
  if (ns > kBatchMax) return Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve_batch: more than 64 systems"};
  // workspace: per system r, p, q, y (T) and r64 (FP64), each on a 256-byte boundary
  const int pgrid = CgOcc<T>::value * sms;
  std::vector<size_t> off(ns);
  size_t bytes = 0;
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  for (int k = 0; k < ns; ++k) {
    off[k] = bytes;
    bytes += 4 * al(sys[k].n * sizeof(T)) + al(sys[k].n * sizeof(double2));
  }
  std::vector<int> vnb(ns), rnb(ns);
  size_t part_rows = 0;
  for (int k = 0; k < ns; ++k) {
    vnb[k] = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_for(sys[k].n, 256), 2LL * sms));
    rnb[k] = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_for(sys[k].n * kCgG, 256), 4LL * sms));
    part_rows += std::max(vnb[k], pgrid);
  }
  PG_TRY(W->vec.reserve(bytes));
  PG_TRY(W->st.reserve(ns * sizeof(CState)));
  PG_TRY(W->part.reserve(part_rows * kCgSlots * sizeof(double2)));
  PG_TRY(W->ctl.reserve(ns * sizeof(CgCtl)));
  PG_TRY(W->sys.reserve(ns * sizeof(CgSys<T>)));
  PG_TRY(W->ref.reserve(ns * sizeof(CgRef<T>)));
  CState* dst = W->st.as<CState>();
  CgCtl* dctl = W->ctl.as<CgCtl>();
  PG_CUDA(cudaMemsetAsync(dst, 0, ns * sizeof(CState), s));
  // tables
  std::vector<CgRef<T>> ref(ns);
  std::vector<CgSys<T>> tab(ns);
  int v0 = 0, r0 = 0;
  size_t prow = 0;
  unsigned char* base = W->vec.as<unsigned char>();
  for (int k = 0; k < ns; ++k) {
    petgem_ctx* c = sys[k].c;
    CgBuffers* Bc = cg_bufs(c);
    const int64_t n = sys[k].n;
    unsigned char* v = base + off[k];
    T* r = (T*)v;
    T* p = (T*)(v + al(n * sizeof(T)));
    T* q = (T*)(v + 2 * al(n * sizeof(T)));
    T* y = (T*)(v + 3 * al(n * sizeof(T)));
    double2* r64 = (double2*)(v + 4 * al(n * sizeof(T)));
    double2* part = W->part.as<double2>() + prow * kCgSlots;
    prow += std::max(vnb[k], pgrid);
    ref[k] = CgRef<T>{c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->val.as<double2>(), Bc->sq.as<double2>(),
                      c->b.as<double2>() + (int64_t)sys[k].src * n, nullptr,
                      r64, r, p, y, nullptr, dst + k, part, dctl + k, n, v0, vnb[k], r0, rnb[k]};
    v0 += vnb[k];
    r0 += rnb[k];
    const T* at = c128 ? (const T*)Bc->a128.ptr : (const T*)Bc->a64.ptr;
    const bool sl = c->sell_ok;
    tab[k] = CgSys<T>{c->row_ptr.as<int64_t>(),
                      c->col.as<int32_t>(),
                      at,
                      p,
                      q,
                      r,
                      y,
                      nullptr,
                      sl ? c->sell_sp.as<int64_t>() : nullptr,
                      sl ? c->sell_col.as<int32_t>() : nullptr,
                      sl ? (c128 ? (const T*)Bc->s128.ptr : (const T*)Bc->s64.ptr) : nullptr,
                      sl ? c->sell_ns : 0,
                      n,
                      dst + k,
                      part,
                      0,
                      0,
                      0};
  }
  bool all_sell = true;  // every mesh has the SELL-32 layout: the layout is one of the candidates
  for (int k = 0; k < ns; ++k) all_sell = all_sell && sys[k].c->sell_ok;
  // the inner solves' vector order: the SELL renumbering (layout 1) or the original (CSR)
  auto set_layout = [&](bool sell) -> Status {
    for (int k = 0; k < ns; ++k) {
      petgem_ctx* ck = sys[k].c;
      ref[k].perm = sell ? ck->sell_perm.as<int32_t>() : nullptr;
    }
    PG_CUDA(cudaMemcpyAsync(W->ref.ptr, ref.data(), ns * sizeof(CgRef<T>), cudaMemcpyHostToDevice, s));
    return Status{};
  };
  // solution pointers: context k's sources in order
  {
    int k = 0;
    for (int ci = 0; ci < n_ctx; ++ci)
      for (int j = 0; j < ctxs[ci]->n_src; ++j, ++k) ref[k].x = x[ci] + (int64_t)j * ctxs[ci]->n_edges;
  }
  PG_CUDA(cudaMemcpyAsync(W->ref.ptr, ref.data(), ns * sizeof(CgRef<T>), cudaMemcpyHostToDevice, s));
  const CgRef<T>* dref = W->ref.as<CgRef<T>>();
  const int vgrid = v0, rgrid = r0;
  // ||b|| of every system and the control block
  k_cgb_norm<T><<<vgrid, 256, 0, s>>>(dref, ns, 1);
  c0->launches++;
  PG_CUDA(cudaGetLastError());
  std::vector<CgCtl> hctl(ns);
  PG_CUDA(cudaMemcpyAsync(hctl.data(), dctl, ns * sizeof(CgCtl), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < ns; ++k)
    if (!hctl[k].active) PG_CUDA(cudaMemsetAsync(ref[k].x, 0, sys[k].n * sizeof(double2), s));
  // the refinement round: direct launches, or their graph
  auto round = [&](cudaStream_t rs) -> Status {
    k_cgb_finish<T><<<vgrid, 256, 0, rs>>>(dref, ns);
    k_cgb_residual<T><<<rgrid, 256, 0, rs>>>(dref, ns);
    k_cgb_norm<T><<<vgrid, 256, 0, rs>>>(dref, ns, 0);
    k_cgb_decide<<<1, kBatchMax, 0, rs>>>(dctl, dst, ns, o.tol, o.inner_tol, o.max_iters, c128 ? 1 : 0);
    k_cgb_start<T><<<vgrid, 256, 0, rs>>>(dref, ns);
    PG_CUDA(cudaGetLastError());
    return Status{};
  };
  cudaGraphExec_t gexec = nullptr;
  if (o.use_graphs) {
    if (!W->cap) PG_CUDA(cudaStreamCreateWithFlags(&W->cap, cudaStreamNonBlocking));
    PG_CUDA(cudaStreamBeginCapture(W->cap, cudaStreamCaptureModeThreadLocal));
    const Status r = round(W->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(W->cap, &g);
    if (!r.ok()) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return Status{PETGEM_ERR_CUDA, std::string("batch round capture: ") + cudaGetErrorString(e)};
    const cudaError_t ei = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return Status{PETGEM_ERR_CUDA, std::string("batch round graph: ") + cudaGetErrorString(ei)};
  }
  struct GraphGuard {
    cudaGraphExec_t g;
    ~GraphGuard() {
      if (g) cudaGraphExecDestroy(g);
    }
  } guard{gexec};
  // rounds
  // layout: 1 = SELL-32 (one lane per row), 2 / 4 / 8 = CSR with that many lanes per row
  int G = o.spmv_lanes ? o.spmv_lanes : kCgG;
  if (G == 1 && !all_sell) G = kCgG;
  bool tuned = o.spmv_lanes != 0;
  if (G == 1) PG_TRY(set_layout(true));
  std::vector<double> work(ns);
  std::vector<int64_t> cap(ns), lastk(ns, 0);
  std::vector<CState> hst(ns);
  std::vector<int> nb(ns, 0);
  Status st_all;
  while (true) {
    if (gexec)
      PG_CUDA(cudaGraphLaunch(gexec, s));
    else
      PG_TRY(round(s));
    c0->launches += 5;
    PG_CUDA(cudaMemcpyAsync(hctl.data(), dctl, ns * sizeof(CgCtl), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    std::vector<int> act;
    for (int k = 0; k < ns; ++k)
      if (hctl[k].active) act.push_back(k);
    if (act.empty()) break;
    // scheduler: the blocks of the persistent grid divided among the active systems
    auto plan = [&]() -> Status {
      for (int k : act) {
        const double expect = lastk[k] > 0 ? (double)lastk[k] : std::cbrt((double)sys[k].n);
        work[k] = (double)sys[k].nnz * expect;
        // the same cap for every lane count: the partition, and so the barrier counters' block
        // counts, must not change between the launches of one inner solve
        cap[k] = std::max<int64_t>(1, blocks_for(sys[k].n * 8, 256));
      }
      batch_partition(act, work, cap, pgrid, nb);
      std::vector<CgSys<T>> at;
      int b = 0;
      for (int k : act) {
        CgSys<T> e = tab[k];
        e.b0 = b;
        e.nb = nb[k];
        e.kmax = std::min<int64_t>(o.max_iters - hctl[k].iters, c128 ? INT64_MAX : kCgInnerMax);
        b += nb[k];
        at.push_back(e);
      }
      PG_CUDA(cudaMemcpyAsync(W->sys.ptr, at.data(), at.size() * sizeof(CgSys<T>), cudaMemcpyHostToDevice, s));
      return Status{};
    };
    auto grid_of = [&]() {
      int g = 0;
      for (int k : act) g += nb[k];
      return g;
    };
    const CgSys<T>* dsys = W->sys.as<CgSys<T>>();
    auto all_done = [&]() -> Status {
      PG_CUDA(cudaMemcpyAsync(hst.data(), dst, ns * sizeof(CState), cudaMemcpyDeviceToHost, s));
      PG_CUDA(cudaStreamSynchronize(s));
      return Status{};
    };
    auto running = [&]() {
      for (int k : act)
        if (hst[k].done == 0 && hst[k].k < std::min<int64_t>(o.max_iters - hctl[k].iters, c128 ? INT64_MAX : kCgInnerMax))
          return true;
      return false;
    };
    PG_TRY(plan());
    if (!tuned) {
      // autotuner: a few iterations with each layout of the product (CSR with 2, 4 or 8 lanes per
      // row, and SELL-32 when every mesh has it), two passes over the candidates with the faster of
      // each pair kept, timed with events on the stream; each probe restarts the inner solve, and
      // the solve proper restarts once more with the winner
      PG_TRY((cg_setup<T, 2>()));
      PG_TRY((cg_setup<T, 4>()));
      PG_TRY((cg_setup<T, 8>()));
      PG_TRY((cg_setup<T, kCgG, false, true>()));
      struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
          for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
        }
      } ev;
      PG_CUDA(cudaEventCreate(&ev.e[0]));
      PG_CUDA(cudaEventCreate(&ev.e[1]));
      float best[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
      const int cand[4] = {2, 4, 8, 1};
      const int nc = all_sell ? 4 : 3;
      bool sell_now = false;
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < nc; ++i) {
          // every candidate starts the inner solve afresh in its own vector order
          if ((cand[i] == 1) != sell_now) {
            sell_now = cand[i] == 1;
            PG_TRY(set_layout(sell_now));
          }
          k_cgb_start<T><<<vgrid, 256, 0, s>>>(dref, ns);
          c0->launches++;
          PG_CUDA(cudaEventRecord(ev.e[0], s));
          PG_TRY(batch_inner<T>(cand[i], s, dsys, (int)act.size(), grid_of(), kBatchTuneSteps));
          PG_CUDA(cudaEventRecord(ev.e[1], s));
          c0->launches++;
          PG_CUDA(cudaEventSynchronize(ev.e[1]));
          float ms = 0.f;
          PG_CUDA(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
          best[i] = std::min(best[i], ms);
        }
      G = cand[std::min_element(best, best + nc) - best];
      if ((G == 1) != sell_now) PG_TRY(set_layout(G == 1));
      k_cgb_start<T><<<vgrid, 256, 0, s>>>(dref, ns);  // the solve proper, from the start
      c0->launches++;
      PG_CUDA(cudaGetLastError());
      tuned = true;
    }
    PG_TRY(all_done());
    while (running()) {
      PG_TRY(batch_inner<T>(G, s, dsys, (int)act.size(), grid_of(), kCgChunk));
      c0->launches++;
      PG_TRY(all_done());
    }
    for (int k : act) lastk[k] = std::max<int64_t>(1, hst[k].k);
  }
  int k = 0;
  for (int ci = 0; ci < n_ctx; ++ci)
    for (int j = 0; j < ctxs[ci]->n_src; ++j, ++k) {
      petgem_solve_info& inf = info[k];
      inf = petgem_solve_info{};
      inf.iters = hctl[k].iters;
      inf.restarts = hctl[k].solves;
      inf.refinements = hctl[k].solves;
      inf.true_rel_residual = hctl[k].relres;
      inf.status = hctl[k].status;
      inf.spmv_lanes = G;
      if (inf.status != PETGEM_OK && st_all.ok())
        st_all = Status{inf.status, "context " + std::to_string(ci) + " source " + std::to_string(j) +
                                        " did not converge (COCG batch)"};
    }
  return st_all;
}

}  // namespace

Status run_solve_cocg(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info) {
  CgBuffers* B = cg_bufs(c);
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  int sms = 0;
  PG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  const bool c128 = o.precision != PETGEM_PREC_MIXED;
  PG_TRY(cg_prepare(c));
  const size_t tb = c128 ? sizeof(double2) : sizeof(float2);
  PG_TRY(B->r64.reserve(n * sizeof(double2)));
  const bool qmr = o.method == PETGEM_METHOD_SQMR;
  for (DevBuf* d : {&B->r, &B->p, &B->q, &B->y}) PG_TRY(d->reserve(n * tb));
  if (qmr) PG_TRY(B->d.reserve(n * tb));
  PG_TRY(B->state.reserve(sizeof(CState)));
  PG_TRY(B->partials.reserve((size_t)std::max<int64_t>(blocks_for(n, kRows), 8LL * sms) * kPStride * sizeof(double2)));
  PG_CUDA(cudaMemsetAsync(B->state.ptr, 0, sizeof(CState), s));
  Status worst;
  if (!qmr && o.batch != 1 && c->n_src > 1) {  // sources of one frequency together, up to 32 per group
    const int group = o.batch <= 0 ? 32 : std::min(o.batch, 32);
    for (int s0 = 0; s0 < c->n_src; s0 += group) {
      const int S_g = std::min(group, c->n_src - s0);
      const double2* b = c->b.as<double2>() + (int64_t)s0 * n;
      if (c128)
        PG_TRY(cocg_group_p<double2>(c, o, B, b, x + (int64_t)s0 * n, S_g, info + s0, sms));
      else
        PG_TRY(cocg_group_p<float2>(c, o, B, b, x + (int64_t)s0 * n, S_g, info + s0, sms));
    }
    PG_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < c->n_src; ++i)
      if (info[i].status != PETGEM_OK && worst.ok())
        worst = Status{info[i].status, "source " + std::to_string(i) + " did not converge (COCG)"};
    return worst;
  }
  for (int32_t src = 0; src < c->n_src; ++src) {
    petgem_solve_info& inf = info[src];
    inf = petgem_solve_info{};
    const double2* b = c->b.as<double2>() + (int64_t)src * n;
    double2* xs = x + (int64_t)src * n;
    Status r;
    if (c128)
      r = qmr ? cocg_source<double2, true>(c, o, B, b, xs, inf, sms) : cocg_source<double2, false>(c, o, B, b, xs, inf, sms);
    else
      r = qmr ? cocg_source<float2, true>(c, o, B, b, xs, inf, sms) : cocg_source<float2, false>(c, o, B, b, xs, inf, sms);
    PG_TRY(r);
    if (inf.status != PETGEM_OK && worst.ok())
      worst = Status{inf.status, "source " + std::to_string(src) + (qmr ? " did not converge (SQMR)"
                                                                         : " did not converge (COCG)")};
  }
  PG_CUDA(cudaStreamSynchronize(s));
  return worst;
}

Status run_solve_batch(petgem_ctx* const* ctxs, int n_ctx, const petgem_solve_opts& o, double2* const* x,
                       petgem_solve_info* info) {
  petgem_ctx* c0 = ctxs[0];
  for (int k = 0; k < n_ctx; ++k) PG_TRY(cg_prepare(ctxs[k]));
  // order: every context's queued work before the batch (on ctxs[0]'s stream), the batch before
  // anything queued on them afterwards
  std::vector<cudaEvent_t> ev;
  auto join = [&](cudaStream_t from, cudaStream_t to) -> Status {
    if (from == to) return Status{};
    cudaEvent_t e;
    PG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
    PG_CUDA(cudaEventRecord(e, from));
    PG_CUDA(cudaStreamWaitEvent(to, e, 0));
    return Status{};
  };
  Status r;
  for (int k = 1; k < n_ctx && r.ok(); ++k) r = join(ctxs[k]->stream, c0->stream);
  if (r.ok())
    r = o.precision == PETGEM_PREC_MIXED ? solve_batch<float2>(ctxs, n_ctx, o, x, info)
                                         : solve_batch<double2>(ctxs, n_ctx, o, x, info);
  for (int k = 1; k < n_ctx; ++k) {
    const Status j = join(c0->stream, ctxs[k]->stream);
    if (r.ok() && !j.ok()) r = j;
  }
  cudaStreamSynchronize(c0->stream);
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  return r;
}

void destroy_cocg(petgem_ctx* c) {
  if (!c->cocg) return;
  CgBuffers* B = static_cast<CgBuffers*>(c->cocg);
  if (B->batch) {
    for (DevBuf* d : {&B->batch->vec, &B->batch->st, &B->batch->part, &B->batch->ctl, &B->batch->sys, &B->batch->ref})
      d->release();
    if (B->batch->cap) cudaStreamDestroy(B->batch->cap);
    delete B->batch;
  }
  for (DevBuf* d : {&B->sq, &B->a128, &B->a64, &B->r64, &B->r, &B->p, &B->q, &B->y, &B->d, &B->state, &B->partials, &B->sys, &B->s64, &B->s128, &B->Bt,
                    &B->X, &B->R, &B->rb, &B->pb, &B->qb, &B->yb, &B->bstates, &B->bgrp, &B->bscal})
    d->release();
  delete B;
  c->cocg = nullptr;
}

}  // namespace petgem
