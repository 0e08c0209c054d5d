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
//     solves for a correction, added to u in FP64).  Dot products take FP32 products over a
//     thread's 8 elements and its warp (256 elements) and sum everything beyond in FP64.
//
// Arnoldi with classical Gram-Schmidt (gs.cuh): one projection pass and one update pass (CGS, the
// default), two of each (CGS2), or a second pair only when ||w|| fell below eta * ||w_before||
// (eta = 1/sqrt(10), kReorthEta2).  Each Krylov vector V_k is stored unnormalised with its scale 1/||V_k|| on
// the device, so no separate normalisation pass is needed.  The Hessenberg column, its Givens
// rotations and the stopping test run in the last block of the update kernel: a cycle of m
// iterations needs no host synchronisation, and kernels after the stop return at once.
#include <math.h>

#include <algorithm>

#include "krylov.cuh"
#include "learned.cuh"
#include "gs.cuh"

namespace petgem {

namespace {

// Conditional second Gram-Schmidt pass: taken when the first pass left less than 1/sqrt(10) of
// the vector's norm (||w'||^2 < 0.1 ||w||^2).  One classical pass loses orthogonality in
// proportion to the cancellation ||w|| / ||w'|| times the unit rounding, so below that factor
// (sqrt(10)) a single complex64 pass stays near 2e-7, far inside what an inner cycle that FP64
// refinement restarts needs; the classical 1/sqrt(2) test fired on nearly every step of the
// learned cycles (whose new directions lose 30-70% of their norm) for no change in iterations.
constexpr double kReorthEta2 = 0.1;

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
// Latency, not bandwidth, bounds a plain row-per-group CSR product here (a row costs three
// dependent round trips: row pointers, then columns and values, then the gathers of x), so the
// kernel is software-pipelined: a persistent grid of lane groups walks rows g, g + groups, ...,
// and while it gathers x for row i it already loads the columns and values of row i + 1 and the
// row pointers of row i + 2.  A lane takes up to U of its row's entries in one batch (rows of
// these meshes hold at most 19 entries: G = 4, U = 5); longer rows finish in a loop.
constexpr int kSpmvU = 5;
template <typename T> struct SpmvOcc { static constexpr int value = 4; };  // resident 256-thread blocks per SM
template <> struct SpmvOcc<double2> { static constexpr int value = 3; };

template <typename T, int G>
__device__ inline void spmv_fetch(const int32_t* __restrict__ col, const T* __restrict__ val, int64_t p0, int64_t p1,
                                  int32_t* c, T* a) {
#pragma unroll
  for (int u = 0; u < kSpmvU; ++u) {
    const int64_t q = p0 + (int64_t)u * G;
    c[u] = q < p1 ? __ldg(&col[q]) : 0;
    a[u] = q < p1 ? __ldg(&val[q]) : zero<T>();
  }
}

template <typename T, int G>
__global__ void __launch_bounds__(256, SpmvOcc<T>::value)
    k_spmv_arnoldi(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const T* __restrict__ val,
                   const T* __restrict__ x, T* __restrict__ y, int64_t n, const GState* __restrict__ st, int j) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  constexpr int U = kSpmvU;
  const int64_t groups = (int64_t)gridDim.x * (256 / G);
  const int lane = threadIdx.x % G;
  int64_t row = blockIdx.x * (int64_t)(256 / G) + threadIdx.x / G;
  // pipeline state: row (pointers, columns, values), row + groups (pointers)
  int64_t p0 = 0, p1 = 0;
  if (row < n) {
    p0 = rp[row] + lane;
    p1 = rp[row + 1];
  }
  int32_t c[U];
  T a[U];
  spmv_fetch<T, G>(col, val, p0, p1, c, a);
  int64_t nrow = row + groups, np0 = 0, np1 = 0;
  if (nrow < n) {
    np0 = rp[nrow] + lane;
    np1 = rp[nrow + 1];
  }
  while (__any_sync(0xffffffffu, row < n)) {
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = p0 + (int64_t)u * G < p1 ? __ldg(&x[c[u]]) : zero<T>();
    int32_t c2[U];
    T a2[U];
    spmv_fetch<T, G>(col, val, np0, np1, c2, a2);
    const int64_t nnrow = nrow + groups;
    int64_t nnp0 = 0, nnp1 = 0;
    if (nnrow < n) {
      nnp0 = rp[nnrow] + lane;
      nnp1 = rp[nnrow + 1];
    }
    typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
#pragma unroll
    for (int u = 0; u < U; u += 2) {
      fma_c(acc, a[u], xv[u]);
      if (u + 1 < U) fma_c(acc2, a[u + 1], xv[u + 1]);
    }
    for (int64_t q = p0 + (int64_t)U * G; q < p1; q += G) fma_c(acc, __ldg(&val[q]), __ldg(&x[__ldg(&col[q])]));
    acc.x += acc2.x;
    acc.y += acc2.y;
    for (int o = G / 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (row < n && lane == 0) y[row] = scale_out<T>(acc, st, j);
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
}

// r = b - Ahat u in FP64 (complex128 matrix and vectors).
template <int G>
__global__ void __launch_bounds__(256) k_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                  const double2* __restrict__ val, const double2* __restrict__ u,
                                                  const double2* __restrict__ b, double2* __restrict__ r, int64_t n) {
  // A lane's first five entries: all column and value loads, then all gathers, then the FMAs on two
  // accumulators (one memory round trip per stage instead of two per entry, and two FP64 chains).
  constexpr int U = 5;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t row = gid / G;
  int lane = (int)(gid % G);
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
    for (int k = 0; k < U; ++k) xv[k] = p0 + (int64_t)k * G < p1 ? u[c[k]] : make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < U; ++k) fma_c((k & 1) ? acc2 : acc, a[k], xv[k]);
    for (int64_t p = p0 + (int64_t)U * G; p < p1; p += G) fma_c(acc, val[p], u[col[p]]);
  }
  acc.x += acc2.x;
  acc.y += acc2.y;
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (row < n && lane == 0) r[row] = csub(b[row], acc);
}

// Cycle start: V_0 = r (rounded to T), ||r||^2 in FP64, ||V_0||^2, then (last block) the
// Arnoldi state: g = (||V_0||, 0, ...), 1/||V_0||, stop threshold.
// y = (Ahat x) * scale over the SELL-32 layout (rows and vectors renumbered, sell.cu): one warp per
// slice, lane = row, slices interleaved over the grid; five entries of a slice at a time with the
// next five's columns and values in flight during this chunk's gathers.  Grouping the rows by edge
// kind makes a slice's 32 rows consecutive lattice edges of one kind, so the column, value and
// gather loads of each entry are coalesced, which lifts the product from the L1 limit of the CSR
// form to close to the HBM rate.
template <typename T>
__global__ void __launch_bounds__(256, SpmvOcc<T>::value)
    k_spmv_sell(const int64_t* __restrict__ sp, const int32_t* __restrict__ scol, const T* __restrict__ sval,
                const T* __restrict__ x, T* __restrict__ y, int64_t n, int64_t ns, const GState* __restrict__ st, int j) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  constexpr int U = 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, b = 0, w = 0, t = 0;
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
  typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
  while (s < ns) {
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = t + u < w ? __ldg(&x[c[u]]) : zero<T>();
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
        y[r] = scale_out<T>(acc, st, j);
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
}

template <typename T>
__global__ void __launch_bounds__(kT) k_cycle_init(const double2* __restrict__ r, const int32_t* __restrict__ perm,
                                                   T* __restrict__ V0, int64_t n, GState* __restrict__ st,
                                                   double2* __restrict__ partials, double tol_abs, double inner_rel) {
  __shared__ double2 red[kT / 32];
  __shared__ double2 fin[2];
  double rr = 0.0, vv = 0.0;
  int64_t base = blockIdx.x * (int64_t)kRows + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    int64_t i = base + (int64_t)q * kT;
    if (i < n) {
      double2 v = r[perm ? perm[i] : i];  // the basis is in the SELL renumbering when perm is set
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

// y = H(0:k, 0:k)^{-1} g(0:k), scaled by 1/||V_i|| for the unnormalised basis.  One warp:
// column-oriented back substitution (lane l keeps the running right-hand side of rows l, l+32).
__global__ void __launch_bounds__(32) k_backsolve(GState* st) { backsolve_warp(st, threadIdx.x); }

// u += sum_k V_k y_k.  complex128: in FP64.  complex64: the correction sum_k V_k y_k is formed in
// FP32 (it is the inner solve's correction, accurate to complex64 anyway) and added to u in FP64.
template <typename T>
__global__ void __launch_bounds__(kT) k_xupdate(const T* __restrict__ V, const int32_t* __restrict__ perm, int64_t ld,
                                                int64_t n, double2* __restrict__ u, const GState* __restrict__ st) {
  __shared__ T ys[kMaxM];
  const int kk = st->done == 2 ? 0 : st->k;  // a failed cycle leaves u untouched
  for (int k = threadIdx.x; k < kk; k += kT) ys[k] = from_d2<T>(st->y[k]);
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x;
  if (i >= n || kk == 0) return;
  typename Acc<T>::type acc = zero<T>();
  for (int k = 0; k < kk; ++k) fma_c(acc, V[(int64_t)k * ld + i], ys[k]);
  const int64_t o = perm ? perm[i] : i;
  u[o] = cadd(u[o], to_d2(acc));
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
    // the same matrix in the SELL-32 layout (single-source Jacobi cycles use it)
    PG_TRY(sell_prepare(c));
    if (c->sell_ok) {
      PG_TRY(S->sell64.reserve(c->sell_nnz * sizeof(float2)));
      PG_TRY(S->sell128.reserve(c->sell_nnz * sizeof(double2)));
      PG_TRY(sell_values<float2>(c, S->ahat64.as<float2>(), S->sell64.as<float2>()));
      PG_TRY(sell_values<double2>(c, S->ahat128.as<double2>(), S->sell128.as<double2>()));
    }
    S->version = c->assembly_version;
  }
  if (S->sms == 0) PG_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, c->device));
  PG_TRY((gs_setup<float2, 1>()));
  PG_TRY((gs_setup<double2, 1>()));
  S->n = n;
  S->ld = (n + 255) / 256 * 256;
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
  // Partials: one row of kPStride per block of the widest reduction grid (vector kernels:
  // n_blocks; the projection kernel: kDotBlocksPerSM per SM), and one value per update block.
  PG_TRY(S->partials.reserve(((size_t)std::max<int64_t>(S->n_blocks, (int64_t)kDotBlocksPerSM * S->sms) * kPStride +
                              (size_t)kUpdBlocksPerSM * S->sms) *
                             sizeof(double2)));
  PG_TRY(S->u.reserve(n * sizeof(double2)));
  PG_TRY(S->r.reserve(n * sizeof(double2)));
  PG_TRY(S->state.reserve(sizeof(GState)));
  PG_CUDA(cudaMemsetAsync(S->state.ptr, 0, sizeof(GState), s));
  return Status{};
}

// FNV-1a over the values that fix a captured cycle's launches.
inline uint64_t cycle_key(std::initializer_list<uint64_t> v) {
  uint64_t h = 1469598103934665603ull;
  for (uint64_t x : v)
    for (int b = 0; b < 8; ++b) h = (h ^ ((x >> (8 * b)) & 0xffu)) * 1099511628211ull;
  return h;
}

template <typename T>
Status run_cycle(petgem_ctx* c, const T* ahat, int m, int orth, double tol_abs, double inner_rel, bool learned,
                 bool graph, HostState* hs) {
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
  // SELL-32 products (renumbered basis) when the mesh has the layout; learned cycles then run the
  // network's maps in the same row order (Net::renumber)
  const bool sell = c->sell_ok;
  const int32_t* perm = sell ? c->sell_perm.as<int32_t>() : nullptr;
  {
    KernelTimer kt(c, c128 ? "cycle_init_c128" : "cycle_init_c64", 16.0 * n + vbytes);
    k_cycle_init<T><<<nb, kT, 0, s>>>(S->r.as<double2>(), perm, V, n, st, part, tol_abs, inner_rel);
    c->launches++;
  }
  const double spmv_bytes = sell ? (double)c->sell_nnz * (sizeof(T) + 4) + 8.0 * (c->sell_ns + 1) + 2.0 * vbytes
                                 : (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 2.0 * vbytes;
  const unsigned spmv_blocks =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_for(n * kGroup, 256), (int64_t)SpmvOcc<T>::value * S->sms));
  const unsigned sell_blocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(blocks_for(c->sell_ns * 32, 256), (int64_t)SpmvOcc<T>::value * S->sms));
  // Flexible GMRES with the learned preconditioner: z_j = N-corrected v_j, stored in Z, and the
  // solution update uses Z instead of V.
  T* Z = learned ? S->Z.as<T>() : nullptr;
  // the launches of one cycle after its initialisation: the m Arnoldi steps (each returns at once
  // after the cycle stopped), the back substitution and the solution update
  auto cycle_body = [&]() -> Status {
    for (int j = 0; j < m; ++j) {
      T* vj = V + (int64_t)j * ld;
      T* vn = vj + ld;
      const T* xin = vj;
      if (learned) {  // every step: z = D (D^{-1} v + G phi + Pi w), the network's auxiliary-space direction
        T* zj = Z + (int64_t)j * ld;
        KernelTimer kt(c, "learned_apply", 0.0, j, 0);
        PG_TRY(c->net->apply<T>(s, vj, c->slots.as<int32_t>(), n, zj, false, &st->done, 1, 0, sell));
        c->launches += 28;
        xin = zj;
      }
      {
        KernelTimer kt(c, c128 ? "spmv_c128" : "spmv_c64", spmv_bytes, j, 0);
        if (sell)
          PG_CUDA(pdl_launch(k_spmv_sell<T>, dim3(sell_blocks), dim3(256), 0, s, false,
                             (const int64_t*)c->sell_sp.as<int64_t>(), (const int32_t*)c->sell_col.as<int32_t>(),
                             (const T*)(c128 ? S->sell128.ptr : S->sell64.ptr), xin, vn, n, c->sell_ns,
                             (const GState*)st, j));
        else
          PG_CUDA(pdl_launch(k_spmv_arnoldi<T, kGroup>, dim3(spmv_blocks), dim3(256), 0, s, false,
                             (const int64_t*)c->row_ptr.as<int64_t>(), (const int32_t*)c->col.as<int32_t>(), ahat, xin,
                             vn, n, (const GState*)st, j));
      }
      const double dot_b = (double)(j + 2) * vbytes, upd_b = (double)(j + 3) * vbytes;
      auto sdot = [&](int pass, int need_refine, const char* name, double bytes, int tag) -> Status {
        KernelTimer kt(c, name, bytes, j, tag);
        c->launches++;
        return launch_pdot<T, 1>(s, S->sms, V, ld, n, j, st, &st->done, &st->gbar, part, pass, need_refine);
      };
      auto supd = [&](int pass, int need_refine, double eta2, int finish, const char* name, double bytes,
                      int tag) -> Status {
        KernelTimer kt(c, name, bytes, j, tag);
        c->launches++;
        return launch_pupd<T, 1>(s, S->sms, V, ld, n, j, st, &st->done, &st->counter, part, pass, need_refine, eta2,
                                 finish);
      };
      if (orth == 0) {  // CGS2: dots, update, dots of the updated w, update + norm
        PG_TRY(sdot(0, 0, c128 ? "mdot_c128" : "mdot_c64", dot_b, 0));
        PG_TRY(supd(0, 0, 0.0, 0, c128 ? "cgs_upd1_c128" : "cgs_upd1_c64", upd_b, 0));
        PG_TRY(sdot(1, 0, c128 ? "cgs_dot2_c128" : "cgs_dot2_c64", dot_b, 0));
        PG_TRY(supd(1, 0, 0.0, 1, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0));
      } else if (orth == 1) {  // CGS: dots, update + norm
        PG_TRY(sdot(0, 0, c128 ? "mdot_c128" : "mdot_c64", dot_b, 0));
        PG_TRY(supd(0, 0, 0.0, 1, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0));
      } else {  // CGS, second pass when the norm fell below 1/sqrt(10) of its value
        PG_TRY(sdot(0, 0, c128 ? "mdot_c128" : "mdot_c64", dot_b, 0));
        PG_TRY(supd(0, 0, kReorthEta2, 1, c128 ? "cgs_upd_c128" : "cgs_upd_c64", upd_b, 0));
        PG_TRY(sdot(1, 1, c128 ? "cgs_dot2_c128" : "cgs_dot2_c64", dot_b, 1));
        PG_TRY(supd(1, 1, 0.0, 1, c128 ? "cgs_upd2_c128" : "cgs_upd2_c64", upd_b, 1));
      }
      c->launches += 1;
    }
    PG_CUDA(cudaGetLastError());
    k_backsolve<<<1, 32, 0, s>>>(st);
    {
      KernelTimer kt(c, c128 ? "xupdate_c128" : "xupdate_c64", 32.0 * n + (double)m * vbytes);
      k_xupdate<T><<<blocks_for(n, kT), kT, 0, s>>>(learned ? Z : V, perm, ld, n, S->u.as<double2>(), st);
    }
    c->launches += 2;
    PG_CUDA(cudaGetLastError());
    return Status{};
  };
  if (!graph || c->profiling) {
    PG_TRY(cycle_body());
  } else {
    // CUDA graph: captured once for these buffers, sizes and options, replayed every cycle (the
    // kernels read the cycle's scalars from the device state, so one capture serves every cycle)
    const uint64_t key = cycle_key({(uint64_t)(uintptr_t)ahat, (uint64_t)(uintptr_t)V, (uint64_t)(uintptr_t)st,
                                    (uint64_t)(uintptr_t)part, (uint64_t)(uintptr_t)c->row_ptr.ptr,
                                    (uint64_t)(uintptr_t)c->col.ptr, (uint64_t)(uintptr_t)S->u.ptr, (uint64_t)n,
                                    (uint64_t)ld, (uint64_t)m, (uint64_t)orth, (uint64_t)sizeof(T),
                                    (uint64_t)spmv_blocks, (uint64_t)S->sms, (uint64_t)sell,
                                    (uint64_t)(uintptr_t)(sell ? (c128 ? S->sell128.ptr : S->sell64.ptr) : nullptr),
                                    (uint64_t)(uintptr_t)c->sell_perm.ptr, (uint64_t)(uintptr_t)c->sell_sp.ptr,
                                    (uint64_t)(uintptr_t)c->sell_col.ptr, (uint64_t)c->sell_ns,
                                    (uint64_t)(uintptr_t)c->val.ptr, (uint64_t)(uintptr_t)S->r.ptr,
                                    (uint64_t)learned, (uint64_t)(uintptr_t)Z, (uint64_t)(uintptr_t)c->net,
                                    (uint64_t)(c->net ? c->net->alloc_gen : 0),
                                    (uint64_t)(uintptr_t)c->slots.ptr, (uint64_t)(uintptr_t)c->diag.ptr,
                                    (uint64_t)(uintptr_t)c->sell_inv.ptr});
    if (!S->graph || S->graph_key != key) {
      if (S->graph) cudaGraphExecDestroy(S->graph);
      S->graph = nullptr;
      // captured on a private stream (the context's may be the legacy default stream, which
      // cannot be captured); the graph is then launched on the context's stream
      if (!S->cap_stream) PG_CUDA(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
      const int64_t l0 = c->launches;
      s = S->cap_stream;
      PG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const Status r = cycle_body();
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(s, &g);
      s = c->stream;
      if (!r.ok()) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return Status{PETGEM_ERR_CUDA, std::string("cycle capture: ") + cudaGetErrorString(e)};
      cudaGraphExec_t ex = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return Status{PETGEM_ERR_CUDA, std::string("cycle graph: ") + cudaGetErrorString(ei)};
      S->graph = ex;
      S->graph_key = key;
      S->graph_launches = c->launches - l0;
      c->launches = l0;
    }
    PG_CUDA(cudaGraphLaunch(S->graph, s));
    c->launches += S->graph_launches;
  }
  PG_TRY(read_state(c, hs));
  if (c->profiling) drop_idle_timings(c, pending0, hs->done == 2 ? 0 : hs->k, hs->refined);
  return Status{};
}

}  // namespace

void destroy_solver(petgem_ctx* c) {
  if (!c->solver) return;
  Solver* S = c->solver;
  for (DevBuf* d : {&S->ahat128, &S->ahat64, &S->sell128, &S->sell64, &S->dinv, &S->V, &S->u, &S->r, &S->partials, &S->state, &S->Z, &S->usave, &S->Zb, &S->Usb, &S->bnorm2,
                    &S->Vb, &S->Ub, &S->Rb, &S->Bb, &S->bstates, &S->bgroup, &S->btol})
    d->release();
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
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
  if (o.method == PETGEM_METHOD_COCG || o.method == PETGEM_METHOD_SQMR) return run_solve_cocg(c, o, x, info);
  const bool block = o.batch != 1 && c->n_src > 1;
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
    // Learned preconditioner: learned cycles from the start while each removes at least 10 % of
    // the FP64 residual; one that does not is undone and the solve goes on with Jacobi alone.
    bool want_learned = o.precond == PETGEM_PRECOND_LEARNED;
    bool learned = false;
    constexpr double kLearnedRate = 0.9;
    int fell_back = 0;
    if (want_learned) {
      PG_TRY(S->Z.reserve((size_t)m * S->ld * (o.precision == PETGEM_PREC_MIXED ? sizeof(float2) : sizeof(double2))));
      PG_TRY(S->usave.reserve(n * sizeof(double2)));
      PG_TRY(c->net->features(s, c->sigma.as<double>(), c->sigma_p, c->omega, c->lattice_h));
      if (c->sell_ok) PG_TRY(c->net->renumber(c));
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
        if (prev_learned && !(rate < kLearnedRate)) {
          // the learned cycle just run removed too little of the residual: undo it, stay with Jacobi
          PG_CUDA(cudaMemcpyAsync(S->u.ptr, S->usave.ptr, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
          PG_TRY(residual());
          want_learned = false;
          fell_back = 1;
        }
      }
      learned = want_learned;
      if (learned) PG_CUDA(cudaMemcpyAsync(S->usave.ptr, S->u.ptr, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
      const int mj = (int)std::min<int64_t>(m, std::max<int64_t>(o.max_iters - iters, 0));
      const double tol_abs = o.tol * bnorm;
      // Learned cycles take a second Gram-Schmidt pass whenever the first one lost more than a
      // factor 1/sqrt(10) of the norm (the network's directions can be nearly dependent).
      const int orth = learned && o.orth == PETGEM_ORTH_CGS ? PETGEM_ORTH_CGS_IFNEEDED : o.orth;
      // A cycle whose starting residual already meets tol runs no iteration (k = 0).
      if (o.precision == PETGEM_PREC_MIXED)
        PG_TRY(run_cycle<float2>(c, S->ahat64.as<float2>(), mj, orth, tol_abs, o.inner_tol, learned, o.use_graphs != 0, &hs));
      else
        PG_TRY(run_cycle<double2>(c, S->ahat128.as<double2>(), mj, orth, tol_abs, 0.0, learned, o.use_graphs != 0, &hs));
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
      if (hs.k == 0 && hs.done != 2) {
        // The cycle stopped before its first step although the FP64 residual is above tol (its
        // working-precision start vector had norm zero, e.g. every entry of r underflowed in
        // complex64): a repeat would do the same, so stop instead of cycling without progress.
        status = PETGEM_ERR_BREAKDOWN;
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
