// Multicolour symmetric SOR (SSOR) preconditioner and the SQMR solver it preconditions: the
// configuration of the paper's Section 5.3 runs (SQMR with an SOR preconditioner).  FP64 residuals
// around inner solves in complex64 or complex128.
//
// Colouring.  A Gauss-Seidel sweep is sequential row by row; on the GPU the rows are coloured so
// that rows of one colour share no matrix entry and the sweep takes one colour per launch, all its
// rows at once.  The colouring is Jones-Plassmann's: row i has the priority key
// (splitmix64(i), i) (SplitMix64's output function, Steele, Lea and Flood 2014); in round k every
// uncoloured row whose key exceeds those of all its uncoloured neighbours takes the smallest colour
// none of its coloured neighbours holds.  The result is the greedy colouring in decreasing key
// order, deterministic and independent of the launch shape.  Neighbours are the off-diagonal
// entries of the CSR pattern; a Kuhn mesh's edge matrix takes 12 or 13 colours in 35 to 40 rounds.
//
// SSOR.  With A = D + L + U split in the colour order (L: entries whose column has a lower colour
// than the row, U: a higher one), M = (D + w L) D^{-1} (D + w U), complex symmetric because
// U = L^T.  SQMR takes the symmetric split M1 = (D + w L) D^{-1/2}, M2 = M1^T:
//   M1^{-1} v = D^{1/2} F v and M2^{-1} t = B D^{1/2} t, F = (D + w L)^{-1} (forward sweep),
//   B = (D + w U)^{-1} (backward sweep).
// Neither D^{1/2} is formed: SQMR needs ||M1^{-1} r||, whose squares are |d_i| |(F r)_i|^2, and
// M2^{-1} M1^{-1} r = B (D F r), whose backward sweep reads y = F r directly:
//   forward, colours ascending:  y_i = (r_i - w sum_{col(j) < col(i)} a_ij y_j) / d_i
//   backward, colours descending: u_i = y_i - (w / d_i) sum_{col(j) > col(i)} a_ij u_j.
//
// Layout.  The solver works in the colour order: rows (and columns) renumbered so that each
// colour's rows are consecutive (ascending original ids inside a colour), every row holding its
// off-diagonal entries split as [lower-colour entries | higher-colour entries] with renumbered
// columns, the diagonal apart.  A sweep over one colour then streams a contiguous block of rows
// and only the half of each row it needs (no per-entry colour test), and the product reads both
// halves plus the diagonal: one matrix pass per sweep pair beyond the product.  Values are gathered
// into the layout once per assembly (complex128 and complex64); the vectors are permuted at the
// start of an inner solve and scattered back at its end.
//
// SQMR (Freund and Nachtigal 1994), in the order of the method: t = A q; sigma = q^T t;
// alpha = rho / sigma; r -= alpha t; y = F r; theta' = ||D^{1/2} y|| / tau; c^2 = 1 / (1 + theta'^2);
// tau = tau theta' c; d = c^2 theta^2 d + c^2 alpha q; x += d; u = B D y; rho' = r^T u;
// beta = rho' / rho; q = u + beta q.  The kernels fuse neighbouring steps: the residual update into
// the forward sweep, the d and x updates and rho' into the backward sweep, and the direction update
// into the next product (q_new = u + beta q_old formed on the fly, double-buffered).  Every
// reduction writes one partial per block; a one-block kernel sums them in a fixed order and forms
// the scalars on the device.  No kernel waits on another: the iterations are plain launches, and
// the host reads the state every kSsChunk iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"

namespace petgem {
namespace {

constexpr int kSsLanes = 4;     // lanes per row (rows hold at most ~19 entries)
constexpr int kSsThreads = 256;
constexpr int kSsMaxColours = 64;
constexpr int kSsChunk = 16;    // iterations enqueued between host reads of the state

struct SsState {
  double2 rho, sigma, alpha, beta, dc2, sum;
  double tau, tau_stop, theta, dc1;
  long long k, kmax;
  int done;    // 0 running; 1 stop test met or budget used; 2 breakdown of the bilinear form
  int finish;  // the stop test was met in this iteration: done follows once x is updated
};

struct SsBuffers {
  // colour-order layout of the pattern (mesh version `layout`): row offsets, lower/upper split,
  // renumbered columns, CSR entry each slot takes its value from, old -> new row ids
  DevBuf prp, psp, pcol, psrc, inv;
  int64_t layout = -1, noff = 0;
  // values in that layout (assembly version `version`): off-diagonal entries, diagonal, 1 / d
  // (complex128 and complex64) and |d|
  DevBuf pv128, pv64, dg128, dg64, id128, id64, absd;
  int64_t version = -1;
  DevBuf r64, r, t, y, u, qa, qb, dv, e, state, part;  // inner vectors sized for complex128
};

__device__ __forceinline__ unsigned long long ss_key(unsigned long long s) {
  unsigned long long z = s + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One Jones-Plassmann round.  rnd[i]: the round row i was coloured in (-1: not yet).  A neighbour
// coloured in this same round counts as uncoloured (it was when the round began); its colour is
// never read in this round.
__global__ void k_jp_round(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n, int32_t round,
                           int32_t* __restrict__ rnd, int32_t* __restrict__ colour,
                           unsigned long long* __restrict__ coloured, int32_t* __restrict__ overflow) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool chosen = false;
  if (i < n && rnd[i] < 0) {
    const unsigned long long ki = ss_key((unsigned long long)i);
    unsigned long long used = 0;
    bool waits = false;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t j = col[p];
      if (j == i) continue;
      const int32_t rj = rnd[j];
      if (rj < 0 || rj == round) {
        const unsigned long long kj = ss_key((unsigned long long)j);
        if (kj > ki || (kj == ki && j > i)) {
          waits = true;
          break;
        }
      } else {
        used |= 1ull << colour[j];
      }
    }
    if (!waits) {
      if (used == ~0ull) {
        *overflow = 1;
      } else {
        colour[i] = __ffsll((long long)~used) - 1;
        rnd[i] = round;
        chosen = true;
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, chosen);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(coloured, (unsigned long long)__popc(m));
}

__global__ void k_ss_flag(const int32_t* __restrict__ colour, int64_t n, int32_t c, int32_t* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = colour[i] == c;
}

__global__ void k_ss_place(const int32_t* __restrict__ flag, const int64_t* __restrict__ rank, int64_t n, int64_t base,
                           int32_t* __restrict__ rows) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && flag[i]) rows[base + rank[i]] = (int32_t)i;
}

// Layout construction.  inv[perm[r]] = r.
__global__ void k_ss_inv(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) inv[perm[r]] = (int32_t)r;
}

// Off-diagonal entries of new row r (the pattern holds every row's diagonal).
__global__ void k_ss_offlen(const int64_t* __restrict__ rp, const int32_t* __restrict__ perm, int64_t n,
                            int32_t* __restrict__ len) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int32_t i = perm[r];
  len[r] = (int32_t)(rp[i + 1] - rp[i]) - 1;
}

// New row r: its lower-colour entries, then its higher-colour ones, each in CSR order, with
// renumbered columns and the CSR entry they come from; psp[r] = the first higher-colour slot.
__global__ void k_ss_split(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ colour, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ inv, const int64_t* __restrict__ prp, int64_t n,
                           int32_t* __restrict__ pcol, int32_t* __restrict__ psrc, int64_t* __restrict__ psp,
                           int32_t* __restrict__ bad) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int32_t i = perm[r];
  const int32_t ci = colour[i];
  int64_t q = prp[r];
  const int64_t end = prp[r + 1];
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) psp[r] = q;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t j = col[p];
      if (j == i) continue;
      const int32_t cj = colour[j];
      if (cj == ci) *bad = 1;  // not a colouring of this pattern
      if ((pass == 0) != (cj < ci)) continue;
      if (q >= end) {
        *bad = 1;
        return;
      }
      pcol[q] = inv[j];
      psrc[q] = (int32_t)p;
      ++q;
    }
  }
  if (q != end) *bad = 1;
}

// Values into the layout: off-diagonal entries (complex128 and complex64) ...
__global__ void k_ss_values(const int32_t* __restrict__ psrc, int64_t m, const double2* __restrict__ val,
                            double2* __restrict__ v128, float2* __restrict__ v64) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= m) return;
  const double2 a = val[psrc[q]];
  v128[q] = a;
  v64[q] = make_float2((float)a.x, (float)a.y);
}

// ... and d_r, 1 / d_r (both precisions) and |d_r| in the new order.
__global__ void k_ss_diag(const double2* __restrict__ d, const int32_t* __restrict__ perm, int64_t n,
                          double2* __restrict__ dg128, float2* __restrict__ dg64, double2* __restrict__ id128,
                          float2* __restrict__ id64, double* __restrict__ absd) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double2 di = d[perm[r]];
  const double2 ii = cdiv(make_double2(1.0, 0.0), di);
  dg128[r] = di;
  dg64[r] = make_float2((float)di.x, (float)di.y);
  id128[r] = ii;
  id64[r] = make_float2((float)ii.x, (float)ii.y);
  absd[r] = sqrt(cabs2(di));
}

__device__ __forceinline__ double2 ss_lanes_sum(double2 a) {
  for (int o = 1; o < kSsLanes; o <<= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  return a;
}

// Block sum of v (fixed order), written by thread 0 to *out.
__device__ __forceinline__ void ss_block_partial(double2 v, double2* out) {
  __shared__ double2 sh[kSsThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = sh[0];
    for (int w = 1; w < kSsThreads / 32; ++w) s = cadd(s, sh[w]);
    *out = s;
  }
}

// r = b - A x with partial sums of |r_i|^2 (mode 0), or partial sums of |v_i|^2 (mode 1: v = b).
__global__ void __launch_bounds__(kSsThreads) k_ss_residual(const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const double2* __restrict__ val,
                                                            const double2* __restrict__ x,
                                                            const double2* __restrict__ b, int64_t n, int mode,
                                                            double2* __restrict__ r, double2* __restrict__ part) {
  const int64_t i = (blockIdx.x * (int64_t)kSsThreads + threadIdx.x) / kSsLanes;
  const int lane = threadIdx.x & (kSsLanes - 1);
  double2 acc = make_double2(0.0, 0.0);
  if (mode == 0 && i < n)
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += kSsLanes) acc = cadd(acc, cmul(val[p], x[col[p]]));
  acc = ss_lanes_sum(acc);
  double s = 0.0;
  if (i < n && lane == 0) {
    const double2 ri = mode == 0 ? csub(b[i], acc) : b[i];
    if (mode == 0) r[i] = ri;
    s = cabs2(ri);
  }
  ss_block_partial(make_double2(s, 0.0), part + blockIdx.x);
}

// Precision of the inner solve: complex128 (T = double2) or complex64 (T = float2) vectors and
// matrix; every sum across rows is taken in FP64 (the block partials).
__device__ __forceinline__ void ss_fma(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ void ss_fma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ __forceinline__ double2 ss_d2(double2 a) { return a; }
__device__ __forceinline__ double2 ss_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T> __device__ __forceinline__ T ss_t(double2 a);
template <> __device__ __forceinline__ double2 ss_t<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 ss_t<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <typename T> __device__ __forceinline__ T ss_zero() { T z; z.x = 0; z.y = 0; return z; }
template <typename T> __device__ __forceinline__ T ss_lanes_sum_t(T a) {
  for (int o = 1; o < kSsLanes; o <<= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  return a;
}

// acc += sum over the slots [beg, end) of lane `lane` (every kSsLanes-th slot) of pv[k] x[pcol[k]]:
// kSsU slots per lane at a time, their columns and values loaded together, then the gathers, then
// the products, so that each lane keeps kSsU loads in flight (a row's half holds at most ~18).
constexpr int kSsU = 5;
template <typename T>
__device__ __forceinline__ void ss_row_sum(const int32_t* __restrict__ pcol, const T* __restrict__ pv,
                                           const T* __restrict__ x, int64_t beg, int64_t end, int lane, T& acc) {
  for (int64_t b = beg + lane; b < end; b += kSsLanes * kSsU) {
    int32_t j[kSsU];
    T a[kSsU], xv[kSsU];
#pragma unroll
    for (int u = 0; u < kSsU; ++u) {
      const int64_t k = b + (int64_t)u * kSsLanes;
      j[u] = k < end ? pcol[k] : -1;
      a[u] = k < end ? pv[k] : ss_zero<T>();
    }
#pragma unroll
    for (int u = 0; u < kSsU; ++u) xv[u] = j[u] >= 0 ? x[j[u]] : ss_zero<T>();
#pragma unroll
    for (int u = 0; u < kSsU; ++u) ss_fma(acc, a[u], xv[u]);
  }
}

// The same for the product with q_new = u + beta q_old formed on the fly (first: q_new = u).
template <typename T>
__device__ __forceinline__ void ss_row_sum2(const int32_t* __restrict__ pcol, const T* __restrict__ pv,
                                            const T* __restrict__ u, const T* __restrict__ qold, T beta, bool first,
                                            int64_t beg, int64_t end, int lane, T& acc) {
  for (int64_t b = beg + lane; b < end; b += kSsLanes * kSsU) {
    int32_t j[kSsU];
    T a[kSsU], uv[kSsU], qv[kSsU];
#pragma unroll
    for (int k = 0; k < kSsU; ++k) {
      const int64_t s = b + (int64_t)k * kSsLanes;
      j[k] = s < end ? pcol[s] : -1;
      a[k] = s < end ? pv[s] : ss_zero<T>();
    }
#pragma unroll
    for (int k = 0; k < kSsU; ++k) {
      uv[k] = j[k] >= 0 ? u[j[k]] : ss_zero<T>();
      qv[k] = (j[k] >= 0 && !first) ? qold[j[k]] : ss_zero<T>();
    }
#pragma unroll
    for (int k = 0; k < kSsU; ++k) {
      ss_fma(uv[k], beta, qv[k]);
      ss_fma(acc, a[k], uv[k]);
    }
  }
}

// Inner right-hand side r = T(r64 * scale) in the new order and correction e = 0.
template <typename T>
__global__ void k_ss_start(const double2* __restrict__ r64, const int32_t* __restrict__ perm, double scale, int64_t n,
                           T* __restrict__ r, T* __restrict__ e) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = ss_t<T>(cscale(r64[perm[i]], scale));
  e[i] = ss_zero<T>();
}

// x += e * scale (FP64), back in the original order.
template <typename T>
__global__ void k_ss_finish(const T* __restrict__ e, const int32_t* __restrict__ perm, double scale, int64_t n,
                            double2* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t o = perm[i];
  x[o] = cadd(x[o], cscale(ss_d2(e[i]), scale));
}

// Forward sweep over the rows [r0, r0 + cnt) of one colour: with iter, first r_i -= alpha t_i;
// then y_i = (r_i - w sum_lower a_ij y_j) / d_i; partial sums of |d_i| |y_i|^2.
template <typename T>
__global__ void __launch_bounds__(kSsThreads) k_ss_forward(const int64_t* __restrict__ prp,
                                                           const int64_t* __restrict__ psp,
                                                           const int32_t* __restrict__ pcol,
                                                           const T* __restrict__ pv, int64_t r0, int64_t cnt,
                                                           double omega, const T* __restrict__ inv_d,
                                                           const double* __restrict__ absd,
                                                           const T* __restrict__ t, T* __restrict__ r,
                                                           T* __restrict__ y, const SsState* __restrict__ st,
                                                           double2* __restrict__ part, int iter) {
  if (st->done) return;
  const int64_t g = (blockIdx.x * (int64_t)kSsThreads + threadIdx.x) / kSsLanes;
  const int lane = threadIdx.x & (kSsLanes - 1);
  const int64_t i = r0 + g;
  T acc = ss_zero<T>();
  if (g < cnt) ss_row_sum(pcol, pv, y, prp[i], psp[i], lane, acc);
  acc = ss_lanes_sum_t(acc);
  double s = 0.0;
  if (g < cnt && lane == 0) {
    T ri = r[i];
    if (iter) {
      const T al = ss_t<T>(st->alpha);
      T mt = ss_zero<T>();
      ss_fma(mt, al, t[i]);
      ri.x -= mt.x;
      ri.y -= mt.y;
      r[i] = ri;
    }
    T v = ri;
    v.x -= (decltype(v.x))omega * acc.x;
    v.y -= (decltype(v.y))omega * acc.y;
    T yi = ss_zero<T>();
    ss_fma(yi, v, inv_d[i]);
    y[i] = yi;
    s = absd[i] * cabs2(ss_d2(yi));
  }
  ss_block_partial(make_double2(s, 0.0), part + blockIdx.x);
}

// Backward sweep over the rows [r0, r0 + cnt) of one colour: u_i = y_i - (w / d_i) sum_upper a_ij u_j;
// with iter, d_i = dc1 d_i + dc2 q_i and e_i += d_i, else d_i = 0; partial sums of r_i u_i.
template <typename T>
__global__ void __launch_bounds__(kSsThreads) k_ss_backward(const int64_t* __restrict__ prp,
                                                            const int64_t* __restrict__ psp,
                                                            const int32_t* __restrict__ pcol,
                                                            const T* __restrict__ pv, int64_t r0, int64_t cnt,
                                                            double omega, const T* __restrict__ inv_d,
                                                            const T* __restrict__ y, T* __restrict__ u,
                                                            const T* __restrict__ r, const T* __restrict__ q,
                                                            T* __restrict__ dv, T* __restrict__ e,
                                                            const SsState* __restrict__ st,
                                                            double2* __restrict__ part, int iter) {
  if (st->done) return;
  const int64_t g = (blockIdx.x * (int64_t)kSsThreads + threadIdx.x) / kSsLanes;
  const int lane = threadIdx.x & (kSsLanes - 1);
  const int64_t i = r0 + g;
  T acc = ss_zero<T>();
  if (g < cnt) ss_row_sum(pcol, pv, u, psp[i], prp[i + 1], lane, acc);
  acc = ss_lanes_sum_t(acc);
  double2 s = make_double2(0.0, 0.0);
  if (g < cnt && lane == 0) {
    T w = ss_zero<T>();
    ss_fma(w, inv_d[i], acc);
    T ui = y[i];
    ui.x -= (decltype(ui.x))omega * w.x;
    ui.y -= (decltype(ui.y))omega * w.y;
    u[i] = ui;
    if (iter) {
      const T c2 = ss_t<T>(st->dc2);
      T di = dv[i];
      const auto c1 = (decltype(di.x))st->dc1;
      di.x *= c1;
      di.y *= c1;
      ss_fma(di, c2, q[i]);
      dv[i] = di;
      T ei = e[i];
      ei.x += di.x;
      ei.y += di.y;
      e[i] = ei;
    } else {
      dv[i] = ss_zero<T>();
    }
    s = cmul(ss_d2(r[i]), ss_d2(ui));
  }
  ss_block_partial(s, part + blockIdx.x);
}

// t = A q_new with q_new = u + beta q_old formed on the fly (first: q_new = u): both halves of
// each row plus the diagonal; writes q_new and partial sums of q_new^T t.
template <typename T>
__global__ void __launch_bounds__(kSsThreads) k_ss_spmv(const int64_t* __restrict__ prp,
                                                        const int32_t* __restrict__ pcol,
                                                        const T* __restrict__ pv, const T* __restrict__ dg,
                                                        int64_t n, const T* __restrict__ u,
                                                        const T* __restrict__ qold, T* __restrict__ qnew,
                                                        T* __restrict__ t, const SsState* __restrict__ st,
                                                        double2* __restrict__ part, int first) {
  if (st->done) return;
  const int64_t i = (blockIdx.x * (int64_t)kSsThreads + threadIdx.x) / kSsLanes;
  const int lane = threadIdx.x & (kSsLanes - 1);
  const T beta = ss_t<T>(st->beta);
  T acc = ss_zero<T>();
  if (i < n) ss_row_sum2(pcol, pv, u, qold, beta, first != 0, prp[i], prp[i + 1], lane, acc);
  acc = ss_lanes_sum_t(acc);
  double2 s = make_double2(0.0, 0.0);
  if (i < n && lane == 0) {
    T qi = u[i];
    if (!first) ss_fma(qi, beta, qold[i]);
    ss_fma(acc, dg[i], qi);
    qnew[i] = qi;
    t[i] = acc;
    s = cmul(ss_d2(qi), ss_d2(acc));
  }
  ss_block_partial(s, part + blockIdx.x);
}

// Sum of np partials (fixed order) and the scalar step of a stage:
//   0  after the first forward sweep: tau = tau0 = sqrt(sum); stop at tau <= arg tau0
//   1  after the first backward sweep: rho = sum
//   2  after the product: sigma = sum, alpha = rho / sigma (breakdown: sigma or rho zero)
//   3  after the forward sweep: theta, c^2, tau, the coefficients of d; stop test
//   4  after the backward sweep: rho' = sum, beta = rho' / rho
//   5  plain sum (norms of the outer loop)
template <int STAGE>
__global__ void __launch_bounds__(kSsThreads) k_ss_scalar(SsState* __restrict__ st, const double2* __restrict__ part,
                                                          int64_t np, double arg, long long kmax) {
  if (STAGE >= 2 && STAGE <= 4 && st->done) return;
  double2 v = make_double2(0.0, 0.0);
  for (int64_t k = threadIdx.x; k < np; k += kSsThreads) v = cadd(v, part[k]);
  __shared__ double2 tot;
  {
    __shared__ double2 sh[kSsThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 s = sh[0];
      for (int w = 1; w < kSsThreads / 32; ++w) s = cadd(s, sh[w]);
      tot = s;
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double2 sum = tot;
  if (STAGE == 0) {
    st->tau = sqrt(sum.x);
    st->tau_stop = arg * st->tau;
    st->theta = 0.0;
    st->k = 0;
    st->kmax = kmax;
    st->finish = 0;
    st->beta = make_double2(0.0, 0.0);
    st->done = !isfinite(st->tau) ? 2 : (st->tau == 0.0 || kmax <= 0 ? 1 : 0);
  } else if (STAGE == 1) {
    st->rho = sum;
  } else if (STAGE == 2) {
    st->sigma = sum;
    if (cabs2(sum) == 0.0 || cabs2(st->rho) == 0.0 || !isfinite(sum.x) || !isfinite(sum.y)) {
      st->done = 2;
      return;
    }
    st->alpha = cdiv(st->rho, sum);
  } else if (STAGE == 3) {
    const double th = sqrt(sum.x) / st->tau;
    const double c2 = 1.0 / (1.0 + th * th);
    st->dc1 = c2 * st->theta * st->theta;
    st->dc2 = cscale(st->alpha, c2);
    st->tau = st->tau * th * sqrt(c2);
    st->theta = th;
    st->k += 1;
    if (!(st->tau > st->tau_stop) || st->k >= st->kmax) st->finish = 1;  // NaN tau stops too
  } else if (STAGE == 4) {
    st->beta = cdiv(sum, st->rho);
    st->rho = sum;
    if (st->finish) st->done = 1;
  } else {
    st->sum = sum;
  }
}

SsBuffers* ss_bufs(petgem_ctx* c) {
  if (!c->ssor) c->ssor = new SsBuffers();
  return static_cast<SsBuffers*>(c->ssor);
}

}  // namespace

Status ssor_colouring(petgem_ctx* c) {
  if (c->ss_version == c->mesh_version) return Status{};
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  if (n >= (1ll << 31)) return Status{PETGEM_ERR_UNSUPPORTED, "SSOR colouring: more than 2^31 rows"};
  PG_TRY(c->ss_colour.reserve(n * sizeof(int32_t)));
  PG_TRY(c->ss_rows.reserve(n * sizeof(int32_t)));
  DevBuf work;
  PG_TRY(work.reserve((size_t)n * 4 + 64 + (size_t)(n + 1) * 8 + 64));
  int32_t* rnd = work.as<int32_t>();  // later reused as the flags of one colour
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(work.ptr) + ((n * 4 + 15) / 16) * 16);
  int32_t* overflow = reinterpret_cast<int32_t*>(ctr + 1);
  int64_t* rank = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(ctr) + 64);
  int32_t* colour = c->ss_colour.as<int32_t>();
  auto body = [&]() -> Status {
    PG_CUDA(cudaMemsetAsync(rnd, 0xff, n * sizeof(int32_t), s));
    PG_CUDA(cudaMemsetAsync(colour, 0xff, n * sizeof(int32_t), s));
    PG_CUDA(cudaMemsetAsync(ctr, 0, 16, s));
    int32_t round = 0;
    while (true) {
      if (round > n) return Status{PETGEM_ERR_CUDA, "SSOR colouring made no progress"};
      k_jp_round<<<blocks_for(n, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), n, round, rnd,
                                                    colour, ctr, overflow);
      c->launches++;
      PG_CUDA(cudaGetLastError());
      ++round;
      unsigned long long h[2] = {0, 0};
      PG_CUDA(cudaMemcpyAsync(h, ctr, 16, cudaMemcpyDeviceToHost, s));
      PG_CUDA(cudaStreamSynchronize(s));
      if ((int32_t)h[1] != 0)
        return Status{PETGEM_ERR_UNSUPPORTED, "SSOR colouring: a row needs more than 64 colours"};
      if ((int64_t)h[0] >= n) break;
    }
    // rows grouped by colour, ascending row ids inside a colour
    c->ss_off.assign(1, 0);
    for (int32_t k = 0; c->ss_off.back() < n; ++k) {
      if (k >= kSsMaxColours) return Status{PETGEM_ERR_CUDA, "SSOR colouring: colours do not cover the rows"};
      k_ss_flag<<<blocks_for(n, 256), 256, 0, s>>>(colour, n, k, rnd);
      c->launches++;
      PG_CUDA(cudaGetLastError());
      PG_TRY(exclusive_scan(rnd, rank, n, s));
      k_ss_place<<<blocks_for(n, 256), 256, 0, s>>>(rnd, rank, n, c->ss_off.back(), c->ss_rows.as<int32_t>());
      c->launches++;
      PG_CUDA(cudaGetLastError());
      int64_t cnt = 0;
      PG_CUDA(cudaMemcpyAsync(&cnt, rank + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      PG_CUDA(cudaStreamSynchronize(s));
      c->ss_off.push_back(c->ss_off.back() + cnt);
    }
    c->ss_rounds = round;
    return Status{};
  };
  const Status st = body();
  cudaStreamSynchronize(s);  // the work buffer is released on return
  work.release();
  if (!st.ok()) {
    c->ss_off.clear();
    return st;
  }
  c->ss_version = c->mesh_version;
  return Status{};
}

namespace {

constexpr int64_t kSsInnerMax = 4096;  // iterations of one complex64 inner solve at most

__global__ void k_ss_scatter(const double2* __restrict__ v, const int32_t* __restrict__ perm, int64_t n,
                             double2* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[perm[i]] = v[i];
}

struct SsLaunch {
  petgem_ctx* c;
  SsBuffers* B;
  int64_t n, nb, np_sweep;
  double omega;
  std::vector<int64_t> pbase;  // first partial of each colour's sweep launch
};

// The colour-order layout of the pattern (once per mesh).
Status ss_layout(petgem_ctx* c, SsBuffers* B) {
  if (B->layout == c->mesh_version) return Status{};
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  const int64_t m = c->nnz - n;  // off-diagonal entries
  if (c->nnz >= (1ll << 31)) return Status{PETGEM_ERR_UNSUPPORTED, "SSOR layout: more than 2^31 entries"};
  const int32_t* perm = c->ss_rows.as<int32_t>();
  PG_TRY(B->inv.reserve(n * sizeof(int32_t)));
  PG_TRY(B->prp.reserve((n + 1) * sizeof(int64_t)));
  PG_TRY(B->psp.reserve(n * sizeof(int64_t)));
  PG_TRY(B->pcol.reserve(std::max<int64_t>(m, 1) * sizeof(int32_t)));
  PG_TRY(B->psrc.reserve(std::max<int64_t>(m, 1) * sizeof(int32_t)));
  DevBuf work;
  PG_TRY(work.reserve((size_t)n * sizeof(int32_t) + 16));
  int32_t* len = work.as<int32_t>();
  int32_t* bad = len + n;
  auto body = [&]() -> Status {
    PG_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    k_ss_inv<<<blocks_for(n, 256), 256, 0, s>>>(perm, n, B->inv.as<int32_t>());
    k_ss_offlen<<<blocks_for(n, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), perm, n, len);
    c->launches += 2;
    PG_CUDA(cudaGetLastError());
    PG_TRY(exclusive_scan(len, B->prp.as<int64_t>(), n, s));
    int64_t total = 0;
    PG_CUDA(cudaMemcpyAsync(&total, B->prp.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (total != m) return Status{PETGEM_ERR_CUDA, "SSOR layout: a pattern row lacks its diagonal"};
    k_ss_split<<<blocks_for(n, 128), 128, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                  c->ss_colour.as<int32_t>(), perm, B->inv.as<int32_t>(),
                                                  B->prp.as<int64_t>(), n, B->pcol.as<int32_t>(),
                                                  B->psrc.as<int32_t>(), B->psp.as<int64_t>(), bad);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    int32_t hbad = 0;
    PG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (hbad) return Status{PETGEM_ERR_CUDA, "SSOR layout: the colouring does not match the pattern"};
    return Status{};
  };
  const Status st = body();
  cudaStreamSynchronize(s);  // the work buffer is released on return
  work.release();
  if (!st.ok()) return st;
  B->noff = m;
  B->layout = c->mesh_version;
  B->version = -1;  // values follow the new layout
  return Status{};
}

Status ss_setup(petgem_ctx* c, double omega, SsLaunch& L) {
  PG_TRY(ssor_colouring(c));
  SsBuffers* B = ss_bufs(c);
  PG_TRY(ss_layout(c, B));
  const int64_t n = c->n_edges;
  for (DevBuf* d : {&B->r64, &B->r, &B->t, &B->y, &B->u, &B->qa, &B->qb, &B->dv, &B->e, &B->dg128, &B->id128})
    PG_TRY(d->reserve(n * sizeof(double2)));
  PG_TRY(B->dg64.reserve(n * sizeof(float2)));
  PG_TRY(B->id64.reserve(n * sizeof(float2)));
  PG_TRY(B->absd.reserve(n * sizeof(double)));
  PG_TRY(B->pv128.reserve(std::max<int64_t>(B->noff, 1) * sizeof(double2)));
  PG_TRY(B->pv64.reserve(std::max<int64_t>(B->noff, 1) * sizeof(float2)));
  PG_TRY(B->state.reserve(sizeof(SsState)));
  const int ncol = (int)c->ss_off.size() - 1;
  L.c = c;
  L.B = B;
  L.n = n;
  L.nb = blocks_for(n * kSsLanes, kSsThreads);
  L.omega = omega;
  L.pbase.assign(ncol + 1, 0);
  for (int k = 0; k < ncol; ++k)
    L.pbase[k + 1] = L.pbase[k] + blocks_for((c->ss_off[k + 1] - c->ss_off[k]) * kSsLanes, kSsThreads);
  L.np_sweep = L.pbase[ncol];
  PG_TRY(B->part.reserve((size_t)std::max<int64_t>(L.np_sweep, L.nb) * sizeof(double2)));
  PG_CUDA(cudaMemsetAsync(B->state.ptr, 0, sizeof(SsState), c->stream));
  if (B->version != c->assembly_version) {
    if (B->noff > 0)
      k_ss_values<<<blocks_for(B->noff, 256), 256, 0, c->stream>>>(B->psrc.as<int32_t>(), B->noff,
                                                                   c->val.as<double2>(), B->pv128.as<double2>(),
                                                                   B->pv64.as<float2>());
    k_ss_diag<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->diag.as<double2>(), c->ss_rows.as<int32_t>(), n,
                                                         B->dg128.as<double2>(), B->dg64.as<float2>(),
                                                         B->id128.as<double2>(), B->id64.as<float2>(),
                                                         B->absd.as<double>());
    c->launches += 2;
    PG_CUDA(cudaGetLastError());
    B->version = c->assembly_version;
  }
  return Status{};
}

template <typename T> struct SsVals;
template <> struct SsVals<double2> {
  static const double2* pv(const SsBuffers* B) { return B->pv128.as<double2>(); }
  static const double2* dg(const SsBuffers* B) { return B->dg128.as<double2>(); }
  static const double2* id(const SsBuffers* B) { return B->id128.as<double2>(); }
};
template <> struct SsVals<float2> {
  static const float2* pv(const SsBuffers* B) { return B->pv64.as<float2>(); }
  static const float2* dg(const SsBuffers* B) { return B->dg64.as<float2>(); }
  static const float2* id(const SsBuffers* B) { return B->id64.as<float2>(); }
};

// One sweep over all colours (ascending for the forward one).
template <typename T>
Status ss_forward(const SsLaunch& L, const T* t, T* r, T* y, int iter) {
  petgem_ctx* c = L.c;
  const int ncol = (int)c->ss_off.size() - 1;
  const double vb = sizeof(T);
  // the lower halves (values and columns, y gathered once), row offsets and splits; r read (and
  // written), t, 1 / d, |d| read, y written
  const double bytes = 0.5 * (double)L.B->noff * (vb + 4) + 16.0 * L.n + L.n * (vb * (iter ? 6 : 4) + 8);
  KernelTimer kt(c, sizeof(T) == 16 ? "ssor_forward_c128" : "ssor_forward_c64", bytes);
  for (int k = 0; k < ncol; ++k) {
    const int64_t cnt = c->ss_off[k + 1] - c->ss_off[k];
    if (cnt == 0) continue;
    k_ss_forward<T><<<blocks_for(cnt * kSsLanes, kSsThreads), kSsThreads, 0, c->stream>>>(
        L.B->prp.as<int64_t>(), L.B->psp.as<int64_t>(), L.B->pcol.as<int32_t>(), SsVals<T>::pv(L.B), c->ss_off[k], cnt,
        L.omega, SsVals<T>::id(L.B), L.B->absd.as<double>(), t, r, y, L.B->state.as<SsState>(),
        L.B->part.as<double2>() + L.pbase[k], iter);
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status ss_backward(const SsLaunch& L, const T* y, T* u, const T* r, const T* q, T* e, int iter) {
  petgem_ctx* c = L.c;
  const int ncol = (int)c->ss_off.size() - 1;
  const double vb = sizeof(T);
  // the upper halves as the forward sweep's lower ones; y, r, 1 / d read, u written, and with
  // iter d, q, e read and d, e written
  const double bytes = 0.5 * (double)L.B->noff * (vb + 4) + 16.0 * L.n + L.n * vb * (iter ? 9 : 5);
  KernelTimer kt(c, sizeof(T) == 16 ? "ssor_backward_c128" : "ssor_backward_c64", bytes);
  for (int k = ncol - 1; k >= 0; --k) {
    const int64_t cnt = c->ss_off[k + 1] - c->ss_off[k];
    if (cnt == 0) continue;
    k_ss_backward<T><<<blocks_for(cnt * kSsLanes, kSsThreads), kSsThreads, 0, c->stream>>>(
        L.B->prp.as<int64_t>(), L.B->psp.as<int64_t>(), L.B->pcol.as<int32_t>(), SsVals<T>::pv(L.B), c->ss_off[k], cnt,
        L.omega, SsVals<T>::id(L.B), y, u, r, q, L.B->dv.as<T>(), e, L.B->state.as<SsState>(),
        L.B->part.as<double2>() + L.pbase[k], iter);
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  return Status{};
}

template <int STAGE>
Status ss_scalar(const SsLaunch& L, int64_t np, double arg = 0.0, long long kmax = 0) {
  k_ss_scalar<STAGE><<<1, kSsThreads, 0, L.c->stream>>>(L.B->state.as<SsState>(), L.B->part.as<double2>(), np, arg,
                                                        kmax);
  L.c->launches++;
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status ss_read(const SsLaunch& L, SsState* h) {
  PG_CUDA(cudaMemcpyAsync(h, L.B->state.ptr, sizeof(SsState), cudaMemcpyDeviceToHost, L.c->stream));
  PG_CUDA(cudaStreamSynchronize(L.c->stream));
  return Status{};
}

// ||v||^2 (mode 1) or ||b - A x||^2 with the residual into r64 (mode 0), all in FP64.
Status ss_norm2(const SsLaunch& L, const double2* x, const double2* v, int mode, double* out) {
  petgem_ctx* c = L.c;
  {
    KernelTimer kt(c, mode == 0 ? "ssor_residual_c128" : "ssor_norm",
                   mode == 0 ? (double)c->nnz * 20 + 8.0 * (L.n + 1) + 48.0 * L.n : 16.0 * L.n);
    k_ss_residual<<<L.nb, kSsThreads, 0, c->stream>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                      c->val.as<double2>(), x, v, L.n, mode, L.B->r64.as<double2>(),
                                                      L.B->part.as<double2>());
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  PG_TRY(ss_scalar<5>(L, L.nb));
  SsState h;
  PG_TRY(ss_read(L, &h));
  *out = h.sum.x;
  return Status{};
}

// One source: FP64 residuals r = b - A x; each inner solve runs SQMR in T on A e = r / ||r||
// (e0 = 0) until tau fell by its target, then x += ||r|| e in FP64.
template <typename T>
Status ssor_sqmr_source(const SsLaunch& L, const petgem_solve_opts& o, const double2* b, double2* x,
                        petgem_solve_info& inf) {
  petgem_ctx* c = L.c;
  SsBuffers* B = L.B;
  const int64_t n = L.n;
  const bool c128 = sizeof(T) == 16;
  T *r = B->r.as<T>(), *t = B->t.as<T>(), *y = B->y.as<T>(), *u = B->u.as<T>(), *e = B->e.as<T>();
  T* qbuf[2] = {B->qa.as<T>(), B->qb.as<T>()};
  double bn2 = 0.0;
  PG_TRY(ss_norm2(L, x, b, 1, &bn2));
  const double bnorm = sqrt(bn2);
  if (bnorm == 0.0) {
    PG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), c->stream));
    inf.status = PETGEM_OK;
    return Status{};
  }
  const double vb = sizeof(T);
  // off-diagonal values and columns, row offsets, the diagonal; u and q_old gathered once and
  // read by row, q_new and t written
  const double spmv_bytes = (double)B->noff * (vb + 4) + 8.0 * (n + 1) + vb * n * 7;
  int64_t iters = 0, solves = 0;
  double relres = 0.0, prev = INFINITY;
  int status = PETGEM_OK, stalls = 0;
  SsState hs;
  while (true) {
    double rn2 = 0.0;
    PG_TRY(ss_norm2(L, x, b, 0, &rn2));
    relres = sqrt(rn2) / bnorm;
    if (!std::isfinite(relres)) {
      status = PETGEM_ERR_BREAKDOWN;
      break;
    }
    if (relres <= o.tol) break;
    if (iters >= o.max_iters) {
      status = PETGEM_ERR_NOT_CONVERGED;
      break;
    }
    stalls = relres > 0.5 * prev ? stalls + 1 : 0;  // restarts at the rounding floor
    if (stalls >= 3) {
      status = PETGEM_ERR_NOT_CONVERGED;
      break;
    }
    prev = relres;
    // inner target on tau, relative to its start: what the final tolerance still needs (with a
    // margin for the difference between tau and the true residual); complex64 inner solves stop
    // at inner_tol at most and run kSsInnerMax iterations at most (their recursively updated
    // residual drifts from the true one in FP32; a fresh FP64 residual bounds the drift)
    const double rnorm = sqrt(rn2);
    const double need = 0.3 * o.tol * bnorm / rnorm;
    const double inner = c128 ? need : std::min(std::max(o.inner_tol, need), 0.5);
    const int64_t kmax = std::min<int64_t>(o.max_iters - iters, c128 ? INT64_MAX : kSsInnerMax);
    k_ss_start<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(B->r64.as<double2>(), c->ss_rows.as<int32_t>(),
                                                             1.0 / rnorm, n, r, e);
    c->launches++;
    PG_CUDA(cudaMemsetAsync(B->state.ptr, 0, sizeof(SsState), c->stream));  // running again
    PG_TRY(ss_forward<T>(L, nullptr, r, y, 0));
    PG_TRY(ss_scalar<0>(L, L.np_sweep, inner, (long long)kmax));
    PG_TRY(ss_backward<T>(L, y, u, r, nullptr, e, 0));
    PG_TRY(ss_scalar<1>(L, L.np_sweep));
    int cur = 0;
    for (int64_t it = 0;; ++it) {
      {
        KernelTimer kt(c, c128 ? "ssor_spmv_c128" : "ssor_spmv_c64", spmv_bytes);
        k_ss_spmv<T><<<L.nb, kSsThreads, 0, c->stream>>>(B->prp.as<int64_t>(), B->pcol.as<int32_t>(),
                                                         SsVals<T>::pv(B), SsVals<T>::dg(B), n, u, qbuf[cur],
                                                         qbuf[cur ^ 1], t, B->state.as<SsState>(),
                                                         B->part.as<double2>(), it == 0);
        c->launches++;
      }
      PG_CUDA(cudaGetLastError());
      cur ^= 1;  // q_new
      PG_TRY(ss_scalar<2>(L, L.nb));
      PG_TRY(ss_forward<T>(L, t, r, y, 1));
      PG_TRY(ss_scalar<3>(L, L.np_sweep));
      PG_TRY(ss_backward<T>(L, y, u, r, qbuf[cur], e, 1));
      PG_TRY(ss_scalar<4>(L, L.np_sweep));
      if ((it + 1) % kSsChunk == 0) {
        PG_TRY(ss_read(L, &hs));
        if (hs.done) break;
      }
    }
    k_ss_finish<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(e, c->ss_rows.as<int32_t>(), rnorm, n, x);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    iters += hs.k;
    solves += 1;
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

}  // namespace

Status run_solve_ssor(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info) {
  SsLaunch L;
  PG_TRY(ss_setup(c, o.omega, L));
  Status worst;
  for (int32_t src = 0; src < c->n_src; ++src) {
    petgem_solve_info& inf = info[src];
    inf = petgem_solve_info{};
    const double2* b = c->b.as<double2>() + (int64_t)src * L.n;
    double2* xs = x + (int64_t)src * L.n;
    if (o.precision == PETGEM_PREC_MIXED)
      PG_TRY(ssor_sqmr_source<float2>(L, o, b, xs, inf));
    else
      PG_TRY(ssor_sqmr_source<double2>(L, o, b, xs, inf));
    if (inf.status != PETGEM_OK && worst.ok())
      worst = Status{inf.status, "source " + std::to_string(src) + " did not converge (SQMR, SSOR)"};
  }
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return worst;
}

Status run_ssor_apply(petgem_ctx* c, double omega, const double2* r_in, double2* z) {
  SsLaunch L;
  PG_TRY(ss_setup(c, omega, L));
  double2 *r = L.B->r.as<double2>(), *u = L.B->u.as<double2>();
  const int32_t* perm = c->ss_rows.as<int32_t>();
  k_ss_start<double2><<<blocks_for(L.n, 256), 256, 0, c->stream>>>(r_in, perm, 1.0, L.n, r, L.B->e.as<double2>());
  c->launches++;
  PG_CUDA(cudaGetLastError());
  PG_TRY(ss_forward<double2>(L, nullptr, r, L.B->y.as<double2>(), 0));
  PG_TRY(ss_backward<double2>(L, L.B->y.as<double2>(), u, r, nullptr, nullptr, 0));
  k_ss_scatter<<<blocks_for(L.n, 256), 256, 0, c->stream>>>(u, perm, L.n, z);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return Status{};
}

void destroy_ssor(petgem_ctx* c) {
  if (!c->ssor) return;
  SsBuffers* B = static_cast<SsBuffers*>(c->ssor);
  for (DevBuf* d : {&B->prp, &B->psp, &B->pcol, &B->psrc, &B->inv, &B->pv128, &B->pv64, &B->dg128, &B->dg64, &B->id128,
                    &B->id64, &B->absd, &B->r64, &B->r, &B->t, &B->y, &B->u, &B->qa, &B->qb, &B->dv, &B->e, &B->state,
                    &B->part})
    d->release();
  delete B;
  c->ssor = nullptr;
}

}  // namespace petgem
