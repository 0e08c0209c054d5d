// Krylov-solver definitions shared by the single-source (krylov.cu) and the multi-source
// (block.cu) GMRES drivers: device state of one Arnoldi cycle, precision traits, reductions and
// the Hessenberg / Givens update.
#pragma once
#include <math.h>

#include "ctx.cuh"

namespace petgem {

constexpr int kMaxM = 64;        // capacity of the Hessenberg arrays
constexpr int kMaxRestart = 62;  // Gram-Schmidt slots j + 2 <= 64

struct GState {
  int m, k, done, refine;
  unsigned counter;
  int n_refine;    // steps of this cycle that took a second Gram-Schmidt pass
  int timeout;     // a bounded wait in a kernel gave up
  int pad1;
  double stop_abs;
  double nrm_w;    // ||w||^2 before orthogonalisation (pass 0)
  double rnorm2;   // ||r||^2 of the FP64 residual at the start of the cycle
  double beta0;
  uint8_t refined[kMaxM];
  double2 H[(kMaxM + 1) * kMaxM];  // column j at H[j * (kMaxM + 1) + i], rotated in place
  double2 g[kMaxM + 1];
  double cs_c[kMaxM];
  double2 cs_s[kMaxM];
  double2 h[kMaxM + 1];   // projections of the current column, pass 0
  double2 h2[kMaxM + 1];  // projections, pass 1
  double2 c[kMaxM + 1];   // update coefficients inv_beta[k] * h[k] of the running pass
  double inv_beta[kMaxM + 1];
  float inv_beta32[kMaxM + 1];  // the same scales in FP32, for the complex64 kernels
  double2 y[kMaxM];       // cycle solution, already scaled by inv_beta
  unsigned long long gbar;  // arrivals at the projection kernel's grid barrier (only grows)
};

struct Solver {
  int64_t n = 0, ld = 0;
  int m = 0;
  int prec = -1;
  int64_t version = -1;  // assembly version the scaled matrices belong to
  DevBuf ahat128, ahat64, dinv;  // scaled matrix (c128, c64)
  DevBuf V, u, r, partials, state, Z, usave;
  // multi-source solve (block.cu): interleaved basis / iterate / residual / right-hand sides,
  // one Arnoldi state per source, a group flag and the per-source stopping thresholds
  DevBuf Vb, Ub, Rb, Bb, bstates, bgroup, btol;
  int bprec = -1;
  int64_t bld_used = 0;
  int64_t n_blocks = 0;
  int64_t ld_used = 0;
  int sms = 0;
  // one Arnoldi cycle captured as a CUDA graph (use_graphs): the launches after the cycle's
  // initialisation, for the buffers, sizes and options the key hashes
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_key = 0;
  int64_t graph_launches = 0;
  cudaStream_t cap_stream = nullptr;  // private stream the capture runs on
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

__device__ inline double shfl_d(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ inline double2 shfl_d2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// New Hessenberg column j from the projections h[0..j] (summed over passes; global or shared
// memory) and beta = ||V_{j+1}||: the earlier rotations in order, a new complex Givens rotation,
// the residual estimate and the stopping test.  Called by all 32 lanes of one warp: lane l loads
// rotation l and l + 32 and entries l and l + 32 of the column at once, so the sequential chain of
// rotations runs on registers and shuffles instead of a chain of memory round trips.
__device__ __forceinline__ void finish_column_warp(GState* st, int j, const double2* h, double beta2) {
  const int l = threadIdx.x & 31;
  const double beta = sqrt(beta2);
  const double2 z = make_double2(0.0, 0.0);
  const double c_lo = l < j ? st->cs_c[l] : 0.0, c_hi = l + 32 < j ? st->cs_c[l + 32] : 0.0;
  const double2 s_lo = l < j ? st->cs_s[l] : z, s_hi = l + 32 < j ? st->cs_s[l + 32] : z;
  const double2 h_lo = l <= j ? h[l] : z, h_hi = l + 32 <= j ? h[l + 32] : z;
  double2 out_lo = h_lo, out_hi = h_hi;  // rotated entries of the column
  double2 carry = shfl_d2(h_lo, 0);      // entry i after rotations 0..i-1
  for (int i = 0; i < j; ++i) {
    const bool hi = i >= 32, hi1 = i + 1 >= 32;
    const double c = shfl_d(hi ? c_hi : c_lo, i & 31);
    const double2 s = shfl_d2(hi ? s_hi : s_lo, i & 31);
    const double2 b = shfl_d2(hi1 ? h_hi : h_lo, (i + 1) & 31);
    const double2 top = cadd(cscale(carry, c), cmul(s, b));
    carry = csub(cscale(b, c), cconjmul(s, carry));  // -conj(s) a + c b
    if (l == (i & 31)) {
      if (hi)
        out_hi = top;
      else
        out_lo = top;
    }
  }
  // new rotation on (carry, beta)
  const double aa = sqrt(cabs2(carry));
  const double rho = sqrt(aa * aa + beta * beta);
  double c;
  double2 s;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    c = aa / rho;
    s = cscale(carry, beta / (aa * rho));
  }
  const double2 hj = cadd(cscale(carry, c), cscale(s, beta));
  if (l == (j & 31)) {
    if (j >= 32)
      out_hi = hj;
    else
      out_lo = hj;
  }
  double2* Hc = &st->H[j * (kMaxM + 1)];
  if (l <= j) Hc[l] = out_lo;
  if (l + 32 <= j) Hc[l + 32] = out_hi;
  if (l == 0) {
    Hc[j + 1] = z;
    st->inv_beta[j + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
    st->inv_beta32[j + 1] = (float)st->inv_beta[j + 1];
    st->cs_c[j] = c;
    st->cs_s[j] = s;
    const double2 gj = st->g[j];
    const double2 g1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
    st->g[j + 1] = g1;
    st->g[j] = cscale(gj, c);
    st->k = j + 1;
    const double res = sqrt(cabs2(g1));
    if (!isfinite(res) || !isfinite(beta) || !(rho > 0.0))
      st->done = 2;
    else if (res <= st->stop_abs || beta == 0.0)
      st->done = 1;
  }
  __syncwarp();
}

// y = H(0:k, 0:k)^{-1} g(0:k), scaled by 1/||V_i|| for the unnormalised basis.  One warp:
// column-oriented back substitution (lane l keeps the running right-hand side of rows l, l+32).
__device__ inline void backsolve_warp(GState* st, int lane) {
  const int kk = st->k;
  double2 rhs0 = lane < kk ? st->g[lane] : make_double2(0.0, 0.0);
  double2 rhs1 = lane + 32 < kk ? st->g[lane + 32] : make_double2(0.0, 0.0);
  for (int i = kk - 1; i >= 0; --i) {
    double2 ri = i < 32 ? rhs0 : rhs1;
    double2 yi = make_double2(__shfl_sync(0xffffffffu, ri.x, i & 31), __shfl_sync(0xffffffffu, ri.y, i & 31));
    yi = cdiv(yi, st->H[i * (kMaxM + 1) + i]);
    if (lane == 0) st->y[i] = cscale(yi, st->inv_beta[i]);
    const double2* Hc = &st->H[i * (kMaxM + 1)];
    if (lane < i) rhs0 = csub(rhs0, cmul(Hc[lane], yi));
    if (lane + 32 < i) rhs1 = csub(rhs1, cmul(Hc[lane + 32], yi));
  }
}

struct HostState {  // leading fields of GState
  int m, k, done, refine;
  unsigned counter;
  int n_refine, timeout, pad1;
  double stop_abs, nrm_w, rnorm2, beta0;
  uint8_t refined[kMaxM];
};

constexpr int kGroup = 4;  // lanes per row in the CSR kernels (rows hold at most ~19 entries)

}  // namespace
}  // namespace petgem
