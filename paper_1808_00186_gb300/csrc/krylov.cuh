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
  DevBuf sell128, sell64;        // the scaled matrix in the SELL-32 layout (sell.cu)
  DevBuf V, u, r, partials, state, Z, usave;
  // multi-source solve (block.cu): interleaved basis / iterate / residual / right-hand sides,
  // one Arnoldi state per source, a group flag and the per-source stopping thresholds
  DevBuf Vb, Ub, Rb, Bb, bstates, bgroup, btol;
  DevBuf Zb, Usb, bnorm2;  // learned block FGMRES: Z basis, saved solution, per-source norms
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
// the residual estimate and the stopping test.  Called by all 32 lanes of one warp.
//
// Rotation i maps the pair (carry_i, h_{i+1}) to (top_i, carry_{i+1}) with
//   top_i = c_i carry_i + s_i h_{i+1},   carry_{i+1} = c_i h_{i+1} - conj(s_i) carry_i,
// starting from carry_0 = h_0.  The carries follow a first-order linear recurrence, i.e. the
// composition of the affine maps A_i(x) = -conj(s_i) x + c_i h_{i+1}; composition is associative,
// so lane l composes its two maps (i = 2l, 2l + 1) and a warp scan over the lanes forms every
// prefix in log2(32) steps instead of a chain of j dependent steps (each ~60-cycle FP64
// operations on this part).  The tops then follow elementwise.
__device__ __forceinline__ void finish_column_warp(GState* st, int j, const double2* h, double beta2) {
  const int l = threadIdx.x & 31;
  const double beta = sqrt(beta2);
  const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
  const int e0 = 2 * l, e1 = 2 * l + 1;
  const double c0 = e0 < j ? st->cs_c[e0] : 1.0, c1 = e1 < j ? st->cs_c[e1] : 1.0;
  const double2 s0 = e0 < j ? st->cs_s[e0] : z, s1 = e1 < j ? st->cs_s[e1] : z;
  const double2 h0 = e0 <= j ? h[e0] : z, h1 = e1 <= j ? h[e1] : z, h2 = e1 + 1 <= j ? h[e1 + 1] : z;
  // A_e(x) = a_e x + b_e (identity past the last rotation)
  const double2 a0 = e0 < j ? make_double2(-s0.x, s0.y) : one, b0 = e0 < j ? cscale(h1, c0) : z;
  const double2 a1 = e1 < j ? make_double2(-s1.x, s1.y) : one, b1 = e1 < j ? cscale(h2, c1) : z;
  // this lane's pair A_1 o A_0, then the inclusive scan over lanes (earlier maps apply first)
  double2 A = cmul(a1, a0), B = cadd(cmul(a1, b0), b1);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double2 Ap = make_double2(__shfl_up_sync(0xffffffffu, A.x, d), __shfl_up_sync(0xffffffffu, A.y, d));
    const double2 Bp = make_double2(__shfl_up_sync(0xffffffffu, B.x, d), __shfl_up_sync(0xffffffffu, B.y, d));
    if (l >= d) {
      B = cadd(cmul(A, Bp), B);
      A = cmul(A, Ap);
    }
  }
  // exclusive prefix (the maps of the lanes before) applied to carry_0 = h_0
  double2 Ae = make_double2(__shfl_up_sync(0xffffffffu, A.x, 1), __shfl_up_sync(0xffffffffu, A.y, 1));
  double2 Be = make_double2(__shfl_up_sync(0xffffffffu, B.x, 1), __shfl_up_sync(0xffffffffu, B.y, 1));
  if (l == 0) {
    Ae = one;
    Be = z;
  }
  const double2 hz = shfl_d2(h0, 0);
  const double2 k0 = cadd(cmul(Ae, hz), Be);  // carry_{2l}
  const double2 k1 = cadd(cmul(a0, k0), b0);  // carry_{2l+1}
  double2 out_lo = e0 < j ? cadd(cscale(k0, c0), cmul(s0, h1)) : h0;  // rotated entries 2l, 2l+1
  double2 out_hi = e1 < j ? cadd(cscale(k1, c1), cmul(s1, h2)) : h1;
  const double2 kj = (j & 1) ? k1 : k0;
  const double2 carry = shfl_d2(kj, (j >> 1) & 31);  // carry_j: entry j after rotations 0..j-1
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
  if (e0 == j) out_lo = hj;
  if (e1 == j) out_hi = hj;
  double2* Hc = &st->H[j * (kMaxM + 1)];
  if (e0 <= j) Hc[e0] = out_lo;
  if (e1 <= j) Hc[e1] = out_hi;
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
  const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
  double2 rhs0 = lane < kk ? st->g[lane] : z;
  double2 rhs1 = lane + 32 < kk ? st->g[lane + 32] : z;
  // the diagonal's reciprocals, every lane two at once (a complex division is a long FP64 chain)
  const double2 inv0 = lane < kk ? cdiv(one, st->H[lane * (kMaxM + 1) + lane]) : z;
  const double2 inv1 = lane + 32 < kk ? cdiv(one, st->H[(lane + 32) * (kMaxM + 1) + lane + 32]) : z;
  // column i's entries above the diagonal, loaded one column ahead of their use
  auto col = [&](int i, int r) { return (i >= 0 && r < i) ? st->H[i * (kMaxM + 1) + r] : z; };
  double2 c0 = col(kk - 1, lane), c1 = col(kk - 1, lane + 32);
  for (int i = kk - 1; i >= 0; --i) {
    const double2 n0 = col(i - 1, lane), n1 = col(i - 1, lane + 32);
    const double2 ri = i < 32 ? rhs0 : rhs1;
    const double2 inv = i < 32 ? inv0 : inv1;
    const double2 yi = cmul(shfl_d2(ri, i & 31), shfl_d2(inv, i & 31));
    if (lane == 0) st->y[i] = cscale(yi, st->inv_beta[i]);
    if (lane < i) rhs0 = csub(rhs0, cmul(c0, yi));
    if (lane + 32 < i) rhs1 = csub(rhs1, cmul(c1, yi));
    c0 = n0;
    c1 = n1;
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
