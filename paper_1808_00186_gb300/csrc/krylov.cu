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

#include "ctx.cuh"

namespace petgem {

constexpr int kMaxM = 64;  // largest restart length

struct GState {
  int m, k, done, refine;
  unsigned counter;
  int pad0;
  double stop_abs;
  double nrm_w;    // ||w||^2 before orthogonalisation (pass 0)
  double rnorm2;   // ||r||^2 of the FP64 residual at the start of the cycle
  double beta0;
  double2 H[(kMaxM + 1) * kMaxM];  // column j at H[j * (kMaxM + 1) + i], rotated in place
  double2 g[kMaxM + 1];
  double cs_c[kMaxM];
  double2 cs_s[kMaxM];
  double2 h[kMaxM + 1];   // projections of the current column, pass 0
  double2 h2[kMaxM + 1];  // projections, pass 1
  double2 c[kMaxM + 1];   // update coefficients inv_beta[k] * h[k] of the running pass
  double inv_beta[kMaxM + 1];
  double2 y[kMaxM];       // cycle solution, already scaled by inv_beta
};

struct Solver {
  int64_t n = 0, ld = 0;
  int m = 0;
  int prec = -1;
  int64_t version = -1;  // assembly version the scaled matrices belong to
  DevBuf ahat128, ahat64, dinv;  // scaled matrix (c128, c64)
  DevBuf V, u, r, partials, state;
  int64_t n_blocks = 0;
};

namespace {

constexpr int kT = 256;   // threads per block of the vector kernels
constexpr int kR = 8;     // rows per thread of the vector kernels
constexpr int kRows = kT * kR;
constexpr int kPStride = kMaxM + 2;

// ------------------------------------------------------------------ precision traits
__device__ inline double2 to_d2(double2 a) { return a; }
__device__ inline double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename T> __device__ inline T from_d2(double2 a);
template <> __device__ inline double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ inline float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <typename T> __device__ inline T zero();
template <> __device__ inline double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ inline float2 zero<float2>() { return make_float2(0.f, 0.f); }

// Accumulator of a thread's products: FP64 for complex128 data, FP32 for complex64 data
// (only over the thread's kR rows; everything across threads is summed in FP64).
template <typename T> struct Acc;
template <> struct Acc<double2> { using type = double2; };
template <> struct Acc<float2> { using type = float2; };

__device__ inline void fma_conj(double2& acc, double2 a, double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
__device__ inline void fma_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__device__ inline void fma_c(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ inline void fma_c(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ inline void sub_mul(double2& w, double2 v, double2 c) {  // w -= v c
  w.x = fma(-v.x, c.x, fma(v.y, c.y, w.x));
  w.y = fma(-v.x, c.y, fma(-v.y, c.x, w.y));
}
__device__ inline void sub_mul(float2& w, float2 v, float2 c) {
  w.x = fmaf(-v.x, c.x, fmaf(v.y, c.y, w.x));
  w.y = fmaf(-v.x, c.y, fmaf(-v.y, c.x, w.y));
}
__device__ inline double nrm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline float nrm2(float2 a) { return a.x * a.x + a.y * a.y; }

__device__ inline double2 warp_sum(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-level "last block done" handshake: returns true in exactly one block, after every block
// has published its partials.
__device__ inline bool last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum partials[b * kPStride + k] over blocks b for k in [0, nk) in a fixed order; result in out[k].
__device__ void reduce_partials(const double2* partials, int nblocks, int nk, double2* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = w; k < nk; k += kT / 32) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = lane; b < nblocks; b += 32) {
      double2 p = __ldcg(&partials[(int64_t)b * kPStride + k]);
      s.x += p.x;
      s.y += p.y;
    }
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  __syncthreads();
}

// New Hessenberg column j from the projections h (summed over passes) and beta = ||V_{j+1}||:
// earlier rotations, a new complex Givens rotation, the residual estimate and the stopping test.
__device__ void finish_column(GState* st, int j, const double2* h, double beta2) {
  double beta = sqrt(beta2);
  double2* Hc = &st->H[j * (kMaxM + 1)];
  for (int i = 0; i <= j; ++i) Hc[i] = h[i];
  Hc[j + 1] = make_double2(beta, 0.0);
  st->inv_beta[j + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int i = 0; i < j; ++i) {
    double2 a = Hc[i], b = Hc[i + 1];
    double c = st->cs_c[i];
    double2 s = st->cs_s[i];
    Hc[i] = cadd(cscale(a, c), cmul(s, b));
    Hc[i + 1] = csub(cscale(b, c), cconjmul(s, a));  // -conj(s) a + c b
  }
  double2 a = Hc[j];
  double aa = sqrt(cabs2(a));
  double rho = sqrt(aa * aa + beta * beta);
  double c;
  double2 s;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    c = aa / rho;
    s = cscale(a, beta / (aa * rho));
  }
  st->cs_c[j] = c;
  st->cs_s[j] = s;
  Hc[j] = cadd(cscale(a, c), cscale(s, beta));
  Hc[j + 1] = make_double2(0.0, 0.0);
  double2 gj = st->g[j];
  st->g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
  st->g[j] = cscale(gj, c);
  st->k = j + 1;
  double res = sqrt(cabs2(st->g[j + 1]));
  if (!isfinite(res) || !isfinite(beta) || !(rho > 0.0))
    st->done = 2;
  else if (res <= st->stop_abs || beta == 0.0)
    st->done = 1;
}

// ------------------------------------------------------------------ kernels
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
  typename Acc<T>::type acc = zero<T>();
  if (row < n) {
    int64_t p1 = rp[row + 1];
    for (int64_t p = rp[row] + lane; p < p1; p += G) fma_c(acc, val[p], x[col[p]]);
  }
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) {
    double s = st->inv_beta[j];
    y[row] = from_d2<T>(make_double2((double)acc.x * s, (double)acc.y * s));
  }
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
    st->k = 0;
    st->refine = 0;
    st->stop_abs = fmax(tol_abs, inner_rel * sqrt(r2));
    // Converged before the first step (FP64 residual already small), nothing to do, or not finite.
    if (!isfinite(r2) || !isfinite(b0))
      st->done = 2;
    else
      st->done = (b0 > 0.0 && sqrt(r2) > tol_abs) ? 0 : 1;
    st->counter = 0;
  }
}

// Projections of w = V_{j+1} on V_0..V_j (scaled to the normalised basis) and ||w||^2.
template <typename T>
__global__ void __launch_bounds__(kT) k_mdot(const T* __restrict__ V, int64_t ld, int64_t n, int j,
                                             GState* __restrict__ st, double2* __restrict__ partials, int pass) {
  if (st->done || (pass == 1 && !st->refine)) return;
  __shared__ double2 red[kMaxM + 2][kT / 32];
  __shared__ double2 fin[kMaxM + 2];
  const int nk = j + 1, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* w = V + (int64_t)(j + 1) * ld;
  int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
  T wr[kR];
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    wr[q] = i < n ? w[i] : zero<T>();
  }
  {
    typename Acc<T>::type a = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) a.x += nrm2(wr[q]);
    double2 s = warp_sum(make_double2((double)a.x, 0.0));
    if (lane == 0) red[nk][wid] = s;
  }
  int k = 0;
  for (; k + 1 < nk; k += 2) {  // two vectors per step: 16 independent loads in flight
    const T* v0 = V + (int64_t)k * ld;
    const T* v1 = v0 + ld;
    T a0[kR], a1[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      int64_t i = base + (int64_t)q * kT;
      a0[q] = i < n ? v0[i] : zero<T>();
      a1[q] = i < n ? v1[i] : zero<T>();
    }
    typename Acc<T>::type s0 = zero<T>(), s1 = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      fma_conj(s0, a0[q], wr[q]);
      fma_conj(s1, a1[q], wr[q]);
    }
    double2 d0 = warp_sum(to_d2(s0)), d1 = warp_sum(to_d2(s1));
    if (lane == 0) {
      red[k][wid] = d0;
      red[k + 1][wid] = d1;
    }
  }
  for (; k < nk; ++k) {
    const T* v0 = V + (int64_t)k * ld;
    typename Acc<T>::type s0 = zero<T>();
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      int64_t i = base + (int64_t)q * kT;
      if (i < n) fma_conj(s0, v0[i], wr[q]);
    }
    double2 d0 = warp_sum(to_d2(s0));
    if (lane == 0) red[k][wid] = d0;
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk <= nk; kk += kT) {
    double2 s = make_double2(0.0, 0.0);
    for (int ww = 0; ww < kT / 32; ++ww) s = cadd(s, red[kk][ww]);
    partials[(int64_t)blockIdx.x * kPStride + kk] = s;
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, nk + 1, fin);
  for (int kk = threadIdx.x; kk < nk; kk += kT) {
    double ib = st->inv_beta[kk];
    double2 h = cscale(fin[kk], ib);  // v_k^H w with v_k = V_k / ||V_k||
    if (pass == 0)
      st->h[kk] = h;
    else
      st->h2[kk] = h;
    st->c[kk] = cscale(h, ib);        // w -= V_k * (h_k / ||V_k||)
  }
  if (threadIdx.x == 0) {
    if (pass == 0) st->nrm_w = fin[nk].x;
    st->counter = 0;
  }
}

// w = V_{j+1} <- w - sum_k V_k c_k, ||w||^2; the last block decides on a second pass or
// finishes the Hessenberg column.
template <typename T>
__global__ void __launch_bounds__(kT) k_mupdate(T* __restrict__ V, int64_t ld, int64_t n, int j,
                                                GState* __restrict__ st, double2* __restrict__ partials, int pass) {
  if (st->done || (pass == 1 && !st->refine)) return;
  __shared__ T cs[kMaxM + 1];
  __shared__ double red[kT / 32];
  __shared__ double2 fin[1];
  __shared__ double2 hsum[kMaxM + 1];
  const int nk = j + 1;
  for (int k = threadIdx.x; k < nk; k += kT) cs[k] = from_d2<T>(st->c[k]);
  __syncthreads();
  T* w = V + (int64_t)(j + 1) * ld;
  int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
  T wr[kR];
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    wr[q] = i < n ? w[i] : zero<T>();
  }
  int k = 0;
  for (; k + 1 < nk; k += 2) {
    const T* v0 = V + (int64_t)k * ld;
    const T* v1 = v0 + ld;
    T a0[kR], a1[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      int64_t i = base + (int64_t)q * kT;
      a0[q] = i < n ? v0[i] : zero<T>();
      a1[q] = i < n ? v1[i] : zero<T>();
    }
    const T c0 = cs[k], c1 = cs[k + 1];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      sub_mul(wr[q], a0[q], c0);
      sub_mul(wr[q], a1[q], c1);
    }
  }
  for (; k < nk; ++k) {
    const T* v0 = V + (int64_t)k * ld;
    const T c0 = cs[k];
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      int64_t i = base + (int64_t)q * kT;
      if (i < n) sub_mul(wr[q], v0[i], c0);
    }
  }
  double nn = 0.0;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    if (i < n) {
      w[i] = wr[q];
      nn += (double)nrm2(wr[q]);
    }
  }
  nn = warp_sum(nn);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int ww = 0; ww < kT / 32; ++ww) s += red[ww];
    partials[(int64_t)blockIdx.x * kPStride] = make_double2(s, 0.0);
  }
  if (!last_block(&st->counter)) return;
  reduce_partials(partials, gridDim.x, 1, fin);
  const double n2 = fin[0].x;
  if (pass == 0 && n2 < 0.5 * st->nrm_w) {  // lost more than 1 - 1/sqrt(2) of the norm: one more pass
    if (threadIdx.x == 0) {
      st->refine = 1;
      st->counter = 0;
    }
    return;
  }
  for (int kk = threadIdx.x; kk < nk; kk += kT) hsum[kk] = pass == 0 ? st->h[kk] : cadd(st->h[kk], st->h2[kk]);
  __syncthreads();
  if (threadIdx.x == 0) {
    finish_column(st, j, hsum, n2);
    st->refine = 0;
    st->counter = 0;
  }
}

// y = H(0:k, 0:k)^{-1} g(0:k), scaled by 1/||V_i|| for the unnormalised basis.
__global__ void k_backsolve(GState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int kk = st->k;
  for (int i = kk - 1; i >= 0; --i) {
    double2 acc = st->g[i];
    for (int l = i + 1; l < kk; ++l) acc = csub(acc, cmul(st->H[l * (kMaxM + 1) + i], st->y[l]));
    st->y[i] = cdiv(acc, st->H[i * (kMaxM + 1) + i]);
  }
  for (int i = 0; i < kk; ++i) st->y[i] = cscale(st->y[i], st->inv_beta[i]);
}

// u += sum_k V_k y_k in FP64.
template <typename T>
__global__ void __launch_bounds__(kT) k_xupdate(const T* __restrict__ V, int64_t ld, int64_t n,
                                                double2* __restrict__ u, const GState* __restrict__ st) {
  __shared__ double2 ys[kMaxM];
  const int kk = st->done == 2 ? 0 : st->k;  // a failed cycle leaves u untouched
  for (int k = threadIdx.x; k < kk; k += kT) ys[k] = st->y[k];
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x;
  if (i >= n || kk == 0) return;
  double2 acc = u[i];
  for (int k = 0; k < kk; ++k) fma_c(acc, to_d2(V[(int64_t)k * ld + i]), ys[k]);
  u[i] = acc;
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

constexpr int kGroup = 8;  // lanes per row in the CSR kernels (rows hold at most ~19 entries)

// ------------------------------------------------------------------ host side
struct HostState {
  int m, k, done, refine;
  unsigned counter;
  int pad0;
  double stop_abs, nrm_w, rnorm2, beta0;
};

Status read_state(petgem_ctx* c, HostState* hs) {
  Solver* S = c->solver;
  PG_CUDA(cudaMemcpyAsync(hs, S->state.ptr, sizeof(HostState), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  return Status{};
}

Status prepare(petgem_ctx* c, int m) {
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
  S->n = n;
  S->ld = (n + 63) / 64 * 64;
  S->m = m;
  S->n_blocks = (n + kRows - 1) / kRows;
  PG_TRY(S->V.reserve((size_t)(m + 1) * S->ld * sizeof(double2)));
  PG_TRY(S->u.reserve(n * sizeof(double2)));
  PG_TRY(S->r.reserve(n * sizeof(double2)));
  PG_TRY(S->partials.reserve((size_t)std::max<int64_t>(S->n_blocks, 1) * kPStride * sizeof(double2)));
  PG_TRY(S->state.reserve(sizeof(GState)));
  PG_CUDA(cudaMemsetAsync(S->state.ptr, 0, sizeof(GState), s));
  return Status{};
}

template <typename T>
Status run_cycle(petgem_ctx* c, const T* ahat, int m, double tol_abs, double inner_rel, HostState* hs) {
  Solver* S = c->solver;
  cudaStream_t s = c->stream;
  const int64_t n = S->n, ld = S->ld;
  T* V = S->V.as<T>();
  GState* st = S->state.as<GState>();
  double2* part = S->partials.as<double2>();
  const unsigned nb = (unsigned)S->n_blocks;
  const double vbytes = (double)sizeof(T) * n;
  k_cycle_init<T><<<nb, kT, 0, s>>>(S->r.as<double2>(), V, n, st, part, tol_abs, inner_rel);
  c->launches++;
  const char* spmv_name = sizeof(T) == 16 ? "spmv_c128" : "spmv_c64";
  const char* dot_name = sizeof(T) == 16 ? "mdot_c128" : "mdot_c64";
  const char* upd_name = sizeof(T) == 16 ? "mupdate_c128" : "mupdate_c64";
  const double spmv_bytes = (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 2.0 * vbytes;
  const unsigned spmv_blocks = blocks_for(n * kGroup, 256);
  for (int j = 0; j < m; ++j) {
    T* vj = V + (int64_t)j * ld;
    T* vn = vj + ld;
    {
      KernelTimer kt(c, spmv_name, spmv_bytes);
      k_spmv_arnoldi<T, kGroup><<<spmv_blocks, 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), ahat, vj,
                                                            vn, n, st, j);
    }
    {
      KernelTimer kt(c, dot_name, (j + 2) * vbytes);
      k_mdot<T><<<nb, kT, 0, s>>>(V, ld, n, j, st, part, 0);
    }
    {
      KernelTimer kt(c, upd_name, (j + 3) * vbytes);
      k_mupdate<T><<<nb, kT, 0, s>>>(V, ld, n, j, st, part, 0);
    }
    k_mdot<T><<<nb, kT, 0, s>>>(V, ld, n, j, st, part, 1);
    k_mupdate<T><<<nb, kT, 0, s>>>(V, ld, n, j, st, part, 1);
    c->launches += 5;
  }
  PG_CUDA(cudaGetLastError());
  k_backsolve<<<1, 32, 0, s>>>(st);
  k_xupdate<T><<<blocks_for(n, kT), kT, 0, s>>>(V, ld, n, S->u.as<double2>(), st);
  c->launches += 2;
  PG_CUDA(cudaGetLastError());
  return read_state(c, hs);
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
  if (m < 1 || m > kMaxM) return Status{PETGEM_ERR_UNSUPPORTED, "restart must be in [1, 64]"};
  PG_TRY(prepare(c, m));
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
    int64_t iters = 0, cycles = 0;
    int status = PETGEM_OK;
    double relres = 0.0;
    while (true) {
      {
        KernelTimer kt(c, "residual_c128", (double)c->nnz * 20 + 8.0 * (n + 1) + 48.0 * n);
        k_residual<kGroup><<<rb, 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                              S->ahat128.as<double2>(), S->u.as<double2>(), b, S->r.as<double2>(), n);
        c->launches++;
      }
      PG_CUDA(cudaGetLastError());
      const int mj = (int)std::min<int64_t>(m, std::max<int64_t>(o.max_iters - iters, 0));
      const double tol_abs = o.tol * bnorm;
      // A cycle whose starting residual already meets tol runs no iteration (k = 0).
      if (o.precision == PETGEM_PREC_MIXED)
        PG_TRY(run_cycle<float2>(c, S->ahat64.as<float2>(), mj, tol_abs, o.inner_tol, &hs));
      else
        PG_TRY(run_cycle<double2>(c, S->ahat128.as<double2>(), mj, tol_abs, 0.0, &hs));
      relres = sqrt(hs.rnorm2) / bnorm;  // FP64 residual of the current u
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
      if (hs.done == 2) {  // u was left as it was before this cycle
        status = PETGEM_ERR_BREAKDOWN;
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
    if (status != PETGEM_OK && worst.ok()) worst = Status{status, "source " + std::to_string(src) + " did not converge"};
  }
  PG_CUDA(cudaStreamSynchronize(s));
  return worst;
}

}  // namespace petgem
