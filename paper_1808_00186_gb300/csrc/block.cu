// Multi-source GMRES: all sources of one frequency share the matrix, so up to 32 of them are
// iterated in lockstep and every Arnoldi step does one sparse matrix times block-of-vectors product
// (SpMM) instead of one SpMV per source.  Each source keeps its own Krylov space, Hessenberg
// matrix, Givens rotations and stopping test (the result is that of independent solves, as the
// paper's per-source runs in Section 5.2), with classical Gram-Schmidt.
//
// Layout: a "block vector" holds element (row i, source s) at i * P + s, P = the group size padded
// to a power of two (2..32); padding sources have a zero right-hand side and stop at once.
//
// With the learned preconditioner the group runs flexible GMRES: each step applies the network to
// every live source's column of V_j (read and written in place in the interleaved layout) into
// the block vector Z_j, the SpMM takes Z_j, and the solution update uses Z.  As in the
// single-source solve, a source whose learned cycle removes less than 10 % of its FP64 residual
// has that cycle undone and goes on with Jacobi alone (its Z columns are copies of V's).
#include <math.h>

#include <algorithm>
#include <vector>

#include "krylov.cuh"
#include "gs.cuh"
#include "bands.cuh"
#include "learned.cuh"

namespace petgem {
namespace {

constexpr int kBMaxP = 32;

struct BGroup {
  unsigned counter;
  int all_done;
  unsigned long long gbar;  // arrivals at the projection kernel's grid barrier (only grows)
};

// -------------------------------------------------------------------- per-source columns
// dst[i P + s] = src[i P + s] for the n rows (one source's column of a block vector).
template <typename T, int P>
__global__ void k_bcol_copy(const T* __restrict__ src, T* __restrict__ dst, int64_t n, int s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i * P + s] = src[i * P + s];
}

// out[s] += sum_i |v[i P + s]|^2 for every source (one pass over the block vector; FP64 partial
// sums per block, added atomically: the result decides only whether a cycle gained 10 %).
template <int P>
__global__ void __launch_bounds__(256) k_bcol_norm2(const double2* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double red[256];
  const int tid = threadIdx.x;
  double a = 0.0;
  for (int64_t e = blockIdx.x * 256 + tid; e < n * P; e += (int64_t)gridDim.x * 256) a += v[e].x * v[e].x + v[e].y * v[e].y;
  red[tid] = a;  // the grid stride is a multiple of P, so thread tid always sees source tid % P
  __syncthreads();
  if (tid < P) {
    double t = 0.0;
    for (int k = tid; k < 256; k += P) t += red[k];
    atomicAdd(&out[tid], t);
  }
}

// -------------------------------------------------------------------- layout changes
template <int P>
__global__ void k_btrans_in(const double2* __restrict__ b, const double2* __restrict__ x0,
                            const double2* __restrict__ d, int64_t n, int S_g, double2* __restrict__ Bt,
                            double2* __restrict__ U) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t i = e / P;
  const int s = (int)(e - i * P);
  if (s < S_g) {
    Bt[e] = b[(int64_t)s * n + i];
    U[e] = cmul(d[i], x0[(int64_t)s * n + i]);  // u = D x (right Jacobi)
  } else {
    Bt[e] = make_double2(0.0, 0.0);
    U[e] = make_double2(0.0, 0.0);
  }
}

template <int P>
__global__ void k_btrans_out(const double2* __restrict__ U, const double2* __restrict__ d, int64_t n, int S_g,
                             double2* __restrict__ x) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t i = e / P;
  const int s = (int)(e - i * P);
  if (s < S_g) x[(int64_t)s * n + i] = cdiv(U[e], d[i]);
}

// Scaled store of one SpMM output: complex64 in FP32 (no FP64 instruction), complex128 in FP64.
__device__ inline void store_scaled(float2* y, float2 acc, const GState& g, int j) {
  const float f = g.inv_beta32[j];
  *y = make_float2(acc.x * f, acc.y * f);
}
__device__ inline void store_scaled(double2* y, double2 acc, const GState& g, int j) {
  const double f = g.inv_beta[j];
  *y = make_double2(acc.x * f, acc.y * f);
}

// Epilogue of the staged SpMM for block GMRES: V_{j+1} = (Ahat V_j) / ||V_j|| per source, zero for a
// source whose cycle stopped (as k_bspmm).
struct SpmmStoreGmres {
  const GState* sts;
  int j;
  template <typename T>
  __device__ void operator()(T* Y, int64_t row, int s, int P, typename Acc<T>::type acc) const {
    const GState& g = sts[s];
    if (g.done)
      Y[row * P + s] = zero<T>();
    else
      store_scaled(&Y[row * P + s], acc, g, j);
  }
};

// Per-source sums of partials[b * P + s] over b < nb with the whole block (P divides 256); the
// results land in out[0..P) (shared memory), visible after the call.
template <int P>
__device__ void source_sums(const double2* partials, int nb, double2* red /*[256]*/, double2* out) {
  const int tid = threadIdx.x, s = tid % P;
  double2 a = make_double2(0.0, 0.0);
  for (int b = tid / P; b < nb; b += 256 / P) a = cadd(a, __ldcg(&partials[(int64_t)b * P + s]));
  red[tid] = a;
  __syncthreads();
  if (tid < P) {
    double2 t = make_double2(0.0, 0.0);
    for (int m = tid; m < 256; m += P) t = cadd(t, red[m]);
    out[tid] = t;
  }
  __syncthreads();
}

// -------------------------------------------------------------------- sparse products
// R = B - Ahat U in FP64; P lanes per row, lane = source: the row's entries are read once for
// all sources (broadcast within the lane group), the block vector's rows are contiguous.
template <int P>
__global__ void __launch_bounds__(256) k_bresidual(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                   const double2* __restrict__ val, const double2* __restrict__ U,
                                                   const double2* __restrict__ B, double2* __restrict__ R, int64_t n) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / P;
  const int s = (int)(gid % P);
  if (row >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t p = rp[row]; p < rp[row + 1]; ++p) fma_c(acc, __ldg(&val[p]), U[(int64_t)__ldg(&col[p]) * P + s]);
  R[row * P + s] = csub(B[row * P + s], acc);
}


// Y = (Ahat X) diag(1 / ||X_s||), zero for stopped sources.  P lanes per row, lane = source: the
// row's entries are read by the whole lane group (one broadcast transaction) four at a time, all
// index and value loads of a batch ahead of its gathers of X.  Blocks are short (256 / P rows
// each) and start in row order, so the rows in flight at any time form one narrow band and the
// rows of X they gather stay in L2.  Every nonzero moves P values of X through L1 (256 B for 32
// complex64 sources): the product is bound by the L1 data path, not by HBM (persistent sweeps,
// SM-contiguous bands and whole-row gather batches all measured slower than this form).
template <typename T, int P>
__global__ void __launch_bounds__(256) k_bspmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                               const T* __restrict__ val, const T* __restrict__ X, T* __restrict__ Y,
                                               int64_t n, const GState* __restrict__ sts,
                                               const BGroup* __restrict__ grp, int j) {
  pdl_trigger();
  pdl_wait();
  if (grp->all_done) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / P;
  const int s = (int)(gid % P);
  if (row >= n) return;
  typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
  const int64_t p1 = rp[row + 1];
  int64_t p = rp[row];
  for (; p + 4 <= p1; p += 4) {
    int64_t cc[4];
    T aa[4], xx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cc[u] = __ldg(&col[p + u]);
      aa[u] = __ldg(&val[p + u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xx[u] = X[cc[u] * P + s];
    fma_c(acc, aa[0], xx[0]);
    fma_c(acc2, aa[1], xx[1]);
    fma_c(acc, aa[2], xx[2]);
    fma_c(acc2, aa[3], xx[3]);
  }
  for (; p < p1; ++p) fma_c(acc, __ldg(&val[p]), X[(int64_t)__ldg(&col[p]) * P + s]);
  acc.x += acc2.x;
  acc.y += acc2.y;
  const GState& g = sts[s];
  if (g.done)
    Y[row * P + s] = zero<T>();
  else
    store_scaled(&Y[row * P + s], acc, g, j);
}

// -------------------------------------------------------------------- cycle start
// V_0 = R rounded to T; per source ||R_s||^2 (FP64) and ||V_0,s||^2; the last block starts every
// source's Arnoldi state (a source whose residual already meets its threshold is stopped).
template <typename T, int P>
__global__ void __launch_bounds__(256) k_bcycle_init(const double2* __restrict__ R, T* __restrict__ V0, int64_t n,
                                                     GState* __restrict__ sts, BGroup* __restrict__ grp,
                                                     double2* __restrict__ partials, const double* __restrict__ tol_abs,
                                                     double inner_rel) {
  __shared__ double2 red[256];
  __shared__ double2 fin[kBMaxP];
  const int tid = threadIdx.x;
  double rr = 0.0, vv = 0.0;  // thread tid only meets source tid % P: the stride is a multiple of P
  for (int64_t e = blockIdx.x * (int64_t)256 + tid; e < n * P; e += (int64_t)gridDim.x * 256) {
    const double2 v = R[e];
    const T t = from_d2<T>(v);
    V0[e] = t;
    rr += nrm2(v);
    vv += nrm2(to_d2(t));
  }
  red[tid] = make_double2(rr, vv);
  __syncthreads();
  if (tid < P) {
    double2 sum = make_double2(0.0, 0.0);
    for (int m = tid; m < 256; m += P) sum = cadd(sum, red[m]);
    partials[(int64_t)blockIdx.x * P + tid] = sum;
  }
  if (!last_block(&grp->counter)) return;
  source_sums<P>(partials, gridDim.x, red, fin);
  if (tid < P) {
    GState* st = &sts[tid];
    const double r2 = fin[tid].x, b0 = sqrt(fin[tid].y);
    st->rnorm2 = r2;
    st->beta0 = b0;
    st->g[0] = make_double2(b0, 0.0);
    for (int i = 1; i <= kMaxM; ++i) st->g[i] = make_double2(0.0, 0.0);
    st->inv_beta[0] = b0 > 0.0 ? 1.0 / b0 : 0.0;
    st->inv_beta32[0] = (float)st->inv_beta[0];
    st->k = 0;
    st->refine = 0;
    st->n_refine = 0;
    st->stop_abs = fmax(tol_abs[tid], inner_rel * sqrt(r2));
    if (!isfinite(r2) || !isfinite(b0))
      st->done = 2;
    else
      st->done = (b0 > 0.0 && sqrt(r2) > tol_abs[tid]) ? 0 : 1;
  }
  __syncthreads();
  if (tid == 0) {
    int alive = 0;
    for (int s = 0; s < P; ++s) alive += sts[s].done == 0;
    grp->all_done = alive == 0;
    grp->counter = 0;
  }
}

// One warp per source: y = H^{-1} g for that source's cycle.
// One block of 32 threads per source (each source's back substitution is one warp's work).
__global__ void __launch_bounds__(32) k_bbacksolve(GState* sts) { backsolve_warp(&sts[blockIdx.x], threadIdx.x); }

// U += sum_k V_k y_k per source (complex64 basis: correction in FP32, added in FP64).
template <typename T, int P>
__global__ void __launch_bounds__(256) k_bxupdate(const T* __restrict__ V, int64_t ldb, int64_t n,
                                                  double2* __restrict__ U, const GState* __restrict__ sts, int kmax) {
  __shared__ T ys[kMaxM * P];
  for (int idx = threadIdx.x; idx < kmax * P; idx += blockDim.x) {
    const int k = idx / P, s = idx - k * P;
    const GState& g = sts[s];
    const int kk = g.done == 2 ? 0 : g.k;
    ys[idx] = k < kk ? from_d2<T>(g.y[k]) : zero<T>();
  }
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int s = (int)(e % P);
  typename Acc<T>::type acc = zero<T>();
  for (int k = 0; k < kmax; ++k) fma_c(acc, V[(int64_t)k * ldb + e], ys[k * P + s]);
  U[e] = cadd(U[e], to_d2(acc));
}

// ||b_s||^2 of the group's right-hand sides (one block per source).
__global__ void k_bnorms(const double2* __restrict__ b, int64_t n, int S_g, double* __restrict__ out) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  double a = 0.0;
  if (s < S_g)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += nrm2(b[(int64_t)s * n + i]);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[s] = red[0];
}

// -------------------------------------------------------------------- host driver
template <typename T, int P>
Status run_group(petgem_ctx* c, const petgem_solve_opts& o, const double2* b, double2* x, int S_g,
                 petgem_solve_info* info) {
  Solver* S = c->solver;
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges;
  const int m = o.restart;
  const int64_t ldb = (n + 255) / 256 * 256 * P;
  const int prec = sizeof(T) == 8 ? PETGEM_PREC_MIXED : PETGEM_PREC_C128;
  const size_t vbytes_all = (size_t)(m + 1) * ldb * sizeof(T);
  const bool fresh = S->Vb.bytes < vbytes_all || S->bprec != prec || S->bld_used != ldb;
  PG_TRY(S->Vb.reserve(vbytes_all));
  if (fresh) PG_CUDA(cudaMemsetAsync(S->Vb.ptr, 0, S->Vb.bytes, s));
  S->bprec = prec;
  S->bld_used = ldb;
  const bool learned_req = o.precond == PETGEM_PRECOND_LEARNED;
  if (learned_req) {
    PG_TRY(S->Zb.reserve((size_t)m * ldb * sizeof(T)));
    PG_CUDA(cudaMemsetAsync(S->Zb.ptr, 0, (size_t)m * ldb * sizeof(T), s));  // finite in every column
    PG_TRY(S->Usb.reserve(n * P * sizeof(double2)));
    PG_TRY(S->bnorm2.reserve(P * sizeof(double)));
  }
  PG_TRY(S->Ub.reserve(n * P * sizeof(double2)));
  PG_TRY(S->Rb.reserve(n * P * sizeof(double2)));
  PG_TRY(S->Bb.reserve(n * P * sizeof(double2)));
  PG_TRY(S->bstates.reserve(P * sizeof(GState)));
  PG_TRY(S->bgroup.reserve(sizeof(BGroup)));
  PG_TRY(S->btol.reserve(2 * P * sizeof(double)));
  PG_TRY((gs_setup<T, P>()));
  const unsigned grid_init = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_for(n * P, 256), 8 * S->sms));
  const size_t part_rows = std::max<size_t>({(size_t)kDotBlocksPerSM * S->sms * kPStride * P, (size_t)grid_init * P,
                                             (size_t)pupd_grid(n, P, S->sms) * P});
  PG_TRY(S->partials.reserve(part_rows * sizeof(double2)));
  PG_CUDA(cudaMemsetAsync(S->bstates.ptr, 0, P * sizeof(GState), s));
  PG_CUDA(cudaMemsetAsync(S->bgroup.ptr, 0, sizeof(BGroup), s));
  GState* sts = S->bstates.as<GState>();
  BGroup* grp = S->bgroup.as<BGroup>();
  double2* part = S->partials.as<double2>();
  T* V = S->Vb.as<T>();
  const double2* ahat128 = S->ahat128.as<double2>();
  const T* ahat = sizeof(T) == 8 ? (const T*)S->ahat64.ptr : (const T*)S->ahat128.ptr;

  // ||b_s|| and thresholds
  double* dnorm = S->btol.as<double>() + P;
  k_bnorms<<<P, 256, 0, s>>>(b, n, S_g, dnorm);
  std::vector<double> bn2(P), tol_abs(P);
  PG_CUDA(cudaMemcpyAsync(bn2.data(), dnorm, P * sizeof(double), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < P; ++i) tol_abs[i] = o.tol * sqrt(bn2[i]);
  PG_CUDA(cudaMemcpyAsync(S->btol.ptr, tol_abs.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
  k_btrans_in<P><<<blocks_for(n * P, 256), 256, 0, s>>>(b, x, c->diag.as<double2>(), n, S_g, S->Bb.as<double2>(),
                                                        S->Ub.as<double2>());
  c->launches += 2;
  PG_CUDA(cudaGetLastError());

  std::vector<int64_t> iters(P, 0), cycles(P, 0);
  std::vector<double> relres(P, 0.0);
  std::vector<int> status(P, PETGEM_OK), finished(P, 0);
  for (int i = 0; i < P; ++i)
    if (i >= S_g || bn2[i] == 0.0) finished[i] = 1;
  std::vector<HostState> hs(P);
  const unsigned spmm_grid = blocks_for(n * P, 256);
  // SpMM form for this mesh and group size: the autotuner times the row-per-lane kernel and the
  // staged band kernels on the basis buffers (before the first cycle writes them) and caches the
  // choice; the states are zero here, so every launch runs in full.
  int spmm_form = -1;
  if (o.spmv_lanes == 0) {
    PG_TRY((tune_spmm<T, P>(c, s, ahat, V, V + ldb,
                            [&]() -> Status {
                              PG_CUDA(pdl_launch(k_bspmm<T, P>, dim3(spmm_grid), dim3(256), 0, s, false,
                                                 (const int64_t*)c->row_ptr.as<int64_t>(),
                                                 (const int32_t*)c->col.as<int32_t>(), ahat, (const T*)V, V + ldb, n,
                                                 (const GState*)sts, (const BGroup*)grp, 0));
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
  const double spmm_bytes = (double)c->nnz * (sizeof(T) + 4) + 8.0 * (n + 1) + 2.0 * n * P * sizeof(T);
  int64_t max_done = 0;
  // learned preconditioner, per source: on from the start; the previous cycle's state
  constexpr double kLearnedRate = 0.9;
  std::vector<int> learned_on(P, 0), prev_learned(P, 0), fell_back(P, 0);
  std::vector<double> prev_rel(P, 0.0);
  for (int i = 0; i < S_g; ++i) learned_on[i] = learned_req && !finished[i];
  T* Zb = learned_req ? S->Zb.as<T>() : nullptr;
  const unsigned ncol = blocks_for(n, 256);
  auto residual = [&]() -> Status {
    KernelTimer kt(c, "bresidual_c128", (double)c->nnz * 20 + 48.0 * n * P);
    k_bresidual<P><<<blocks_for(n * P, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), ahat128,
                                                          S->Ub.as<double2>(), S->Bb.as<double2>(),
                                                          S->Rb.as<double2>(), n);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    return Status{};
  };
  while (true) {
    PG_TRY(residual());
    if (learned_req) {
      bool judge = false, any_on = false;
      for (int i = 0; i < S_g; ++i) judge |= !finished[i] && prev_learned[i];
      if (judge) {  // did each source's learned cycle remove at least 10 % of its FP64 residual?
        std::vector<double> rn2(P, 0.0);
        PG_CUDA(cudaMemsetAsync(S->bnorm2.ptr, 0, P * sizeof(double), s));
        k_bcol_norm2<P><<<std::min<unsigned>(blocks_for(n * P, 256), 8 * S->sms), 256, 0, s>>>(
            S->Rb.as<double2>(), n, S->bnorm2.as<double>());
        PG_CUDA(cudaMemcpyAsync(rn2.data(), S->bnorm2.ptr, P * sizeof(double), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
        bool undone = false;
        for (int i = 0; i < S_g; ++i) {
          if (finished[i] || !prev_learned[i]) continue;
          const double rate = sqrt(rn2[i] / bn2[i]) / prev_rel[i];
          if (!(rate < kLearnedRate)) {  // undo that source's learned cycle; Jacobi from here on
            k_bcol_copy<double2, P><<<ncol, 256, 0, s>>>(S->Usb.as<double2>(), S->Ub.as<double2>(), n, i);
            learned_on[i] = 0;
            fell_back[i] = 1;
            undone = true;
          }
        }
        c->launches += 2;
        if (undone) PG_TRY(residual());
      }
      for (int i = 0; i < S_g; ++i) any_on |= !finished[i] && learned_on[i];
      if (any_on)
        PG_CUDA(cudaMemcpyAsync(S->Usb.ptr, S->Ub.ptr, n * P * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }
    k_bcycle_init<T, P><<<grid_init, 256, 0, s>>>(S->Rb.as<double2>(), V, n, sts, grp, part, S->btol.as<double>(),
                                                  prec == PETGEM_PREC_MIXED ? o.inner_tol : 0.0);
    c->launches += 1;
    const int mj = (int)std::min<int64_t>(m, std::max<int64_t>(o.max_iters - max_done, 0));
    for (int j = 0; j < mj; ++j) {
      T* vj = V + (int64_t)j * ldb;
      const T* xin = vj;
      if (learned_req) {  // z_j of every live source: the network (learned) or v_j itself (Jacobi)
        T* zj = Zb + (int64_t)j * ldb;
        for (int i = 0; i < S_g; ++i) {
          if (finished[i]) continue;
          if (learned_on[i]) {
            KernelTimer kt(c, "learned_apply", 0.0, j, i);
            PG_TRY(c->net->apply<T>(s, vj, c->slots.as<int32_t>(), n, zj, false, &sts[i].done, P, i));
            c->launches += 28;
          } else {
            k_bcol_copy<T, P><<<ncol, 256, 0, s>>>(vj, zj, n, i);
            c->launches++;
          }
        }
        xin = zj;
      }
      {
        KernelTimer kt(c, sizeof(T) == 8 ? "bspmm_c64" : "bspmm_c128", spmm_bytes);
        if (spmm_form >= 0)
          PG_TRY((launch_spmm_band<T, P>(c, s, spmm_form, ahat, xin, vj + ldb, &grp->all_done,
                                         SpmmStoreGmres{sts, j})));
        else
          PG_CUDA(pdl_launch(k_bspmm<T, P>, dim3(spmm_grid), dim3(256), 0, s, false,
                             (const int64_t*)c->row_ptr.as<int64_t>(), (const int32_t*)c->col.as<int32_t>(), ahat,
                             xin, vj + ldb, n, (const GState*)sts, (const BGroup*)grp, j));
      }
      {
        KernelTimer kt(c, sizeof(T) == 8 ? "bmdot_c64" : "bmdot_c128", (double)(j + 2) * n * P * sizeof(T));
        PG_TRY((launch_pdot<T, P>(s, S->sms, V, ldb, n, j, sts, &grp->all_done, &grp->gbar, part, 0, 0)));
      }
      {
        KernelTimer kt(c, sizeof(T) == 8 ? "bmupdate_c64" : "bmupdate_c128", (double)(j + 3) * n * P * sizeof(T));
        PG_TRY((launch_pupd<T, P>(s, S->sms, V, ldb, n, j, sts, &grp->all_done, &grp->counter, part, 0, 0, 0.0,
                                  1)));
      }
      c->launches += 3;
    }
    PG_CUDA(cudaGetLastError());
    k_bbacksolve<<<P, 32, 0, s>>>(sts);
    k_bxupdate<T, P><<<blocks_for(n * P, 256), 256, 0, s>>>(learned_req ? Zb : V, ldb, n, S->Ub.as<double2>(), sts,
                                                            std::max(mj, 1));
    c->launches += 2;
    PG_CUDA(cudaGetLastError());
    PG_CUDA(cudaMemcpy2DAsync(hs.data(), sizeof(HostState), sts, sizeof(GState), sizeof(HostState), P,
                              cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int i = 0; i < S_g; ++i) {
      if (finished[i]) continue;
      relres[i] = sqrt(hs[i].rnorm2) / sqrt(bn2[i]);
      if (!isfinite(relres[i])) {
        status[i] = PETGEM_ERR_BREAKDOWN;
        finished[i] = 1;
        continue;
      }
      if (relres[i] <= o.tol) {
        finished[i] = 1;
        continue;
      }
      if (mj == 0) {
        status[i] = PETGEM_ERR_NOT_CONVERGED;
        finished[i] = 1;
        continue;
      }
      iters[i] += hs[i].k;
      cycles[i] += 1;
      max_done = std::max(max_done, iters[i]);
      prev_learned[i] = learned_on[i];
      prev_rel[i] = relres[i];
      if (hs[i].done == 2) {
        status[i] = hs[i].timeout ? PETGEM_ERR_TIMEOUT : PETGEM_ERR_BREAKDOWN;
        finished[i] = 1;
        continue;
      }
      all = false;
    }
    if (all) break;
  }
  k_btrans_out<P><<<blocks_for(n * P, 256), 256, 0, s>>>(S->Ub.as<double2>(), c->diag.as<double2>(), n, S_g, x);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  for (int i = 0; i < S_g; ++i) {
    info[i] = petgem_solve_info{};
    info[i].iters = iters[i];
    info[i].restarts = cycles[i];
    info[i].refinements = cycles[i];
    info[i].true_rel_residual = bn2[i] == 0.0 ? 0.0 : relres[i];
    info[i].status = status[i];
    info[i].spmv_lanes = spmm_form >= 0 ? kBandHeights[spmm_form] : 1;
    info[i].fell_back = fell_back[i];
  }
  if (learned_req) PG_TRY(nn::check_err(s, c->net->err.as<int>(), "petgem_solve (learned, block)"));
  return Status{};
}

template <typename T>
Status run_group_p(petgem_ctx* c, const petgem_solve_opts& o, const double2* b, double2* x, int S_g,
                   petgem_solve_info* info) {
  if (S_g <= 2) return run_group<T, 2>(c, o, b, x, S_g, info);
  if (S_g <= 4) return run_group<T, 4>(c, o, b, x, S_g, info);
  if (S_g <= 8) return run_group<T, 8>(c, o, b, x, S_g, info);
  if (S_g <= 16) return run_group<T, 16>(c, o, b, x, S_g, info);
  return run_group<T, 32>(c, o, b, x, S_g, info);
}

}  // namespace

Status run_solve_block(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info) {
  const int64_t n = c->n_edges;
  if (o.precond == PETGEM_PRECOND_LEARNED)
    PG_TRY(c->net->features(c->stream, c->sigma.as<double>(), c->sigma_p, c->omega, c->lattice_h));
  const int group = o.batch <= 0 ? kBMaxP : std::min(o.batch, kBMaxP);
  for (int s0 = 0; s0 < c->n_src; s0 += group) {
    const int S_g = std::min(group, c->n_src - s0);
    const double2* b = c->b.as<double2>() + (int64_t)s0 * n;
    double2* xs = x + (int64_t)s0 * n;
    if (o.precision == PETGEM_PREC_MIXED)
      PG_TRY(run_group_p<float2>(c, o, b, xs, S_g, info + s0));
    else
      PG_TRY(run_group_p<double2>(c, o, b, xs, S_g, info + s0));
  }
  PG_CUDA(cudaStreamSynchronize(c->stream));
  Status worst;
  for (int i = 0; i < c->n_src; ++i)
    if (info[i].status != PETGEM_OK && worst.ok())
      worst = Status{info[i].status, "source " + std::to_string(i) + " did not converge"};
  return worst;
}

}  // namespace petgem
