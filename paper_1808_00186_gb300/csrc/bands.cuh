// Block SpMM Y = A X with the rows of X staged in shared memory band by band (multi-source
// solvers: X is n x P, row-major, the P sources of a row contiguous).
//
// Each nonzero of A needs a whole row of X (P values).  Consecutive rows of a band share most of
// their columns (the edges of neighbouring tets), so a CTA first copies every distinct X row its
// band of R rows needs into shared memory with coalesced 16-byte loads, once, and then forms the
// band's outputs from shared memory: a warp lane per source, the matrix value broadcast to the
// lanes of the row.  The band layout (bands.cu) gives every band its sorted distinct columns and
// every nonzero its index in that list (16 bits).
#pragma once
#include <math.h>

#include "common.cuh"
#include "krylov.cuh"

namespace petgem {

// Output of the staged product for row `row`, source `s`: the functor decides what is stored.
struct SpmmStorePlain {
  template <typename T>
  __device__ void operator()(T* Y, int64_t row, int s, int P, typename Acc<T>::type acc) const {
    Y[row * P + s] = from_d2<T>(to_d2(acc));
  }
};

template <typename T, int P, int R, typename Store>
__global__ void __launch_bounds__(256) k_spmm_band(const int64_t* __restrict__ band_off,
                                                   const int32_t* __restrict__ ucol,
                                                   const int64_t* __restrict__ rp, const uint16_t* __restrict__ lcol,
                                                   const T* __restrict__ val, const T* __restrict__ X,
                                                   T* __restrict__ Y, int64_t n, const int* __restrict__ all_done,
                                                   Store store) {
  static_assert(P >= 1 && P <= 32 && (32 % P) == 0, "sources per row");
  pdl_trigger();
  pdl_wait();
  if (all_done && *all_done) return;  // block-uniform
  extern __shared__ __align__(16) unsigned char smem_band[];
  T* Xs = reinterpret_cast<T*>(smem_band);  // [U][P]
  const int64_t band = blockIdx.x;
  const int64_t u0 = band_off[band];
  const int U = (int)(band_off[band + 1] - u0);
  // stage the band's distinct X rows: 16-byte pieces, consecutive threads on consecutive pieces
  constexpr int kRowBytes = P * (int)sizeof(T);
  if (kRowBytes % 16 == 0) {
    constexpr int kPieces = kRowBytes / 16;
    for (int k = threadIdx.x; k < U * kPieces; k += blockDim.x) {
      const int u = k / kPieces, q = k - u * kPieces;
      // plain loads: X was written by the kernel before this one (programmatic dependent launch)
      const uint4* src = reinterpret_cast<const uint4*>(X + (int64_t)__ldg(&ucol[u0 + u]) * P) + q;
      reinterpret_cast<uint4*>(Xs + u * P)[q] = *src;
    }
  } else {
    for (int k = threadIdx.x; k < U * P; k += blockDim.x) {
      const int u = k / P, s = k - u * P;
      Xs[k] = X[(int64_t)__ldg(&ucol[u0 + u]) * P + s];
    }
  }
  __syncthreads();
  // rows: a lane per source; 256 / P rows of the band in flight per pass
  constexpr int kRowsPerPass = 256 / P;
  const int s = threadIdx.x % P;
  for (int r = threadIdx.x / P; r < R; r += kRowsPerPass) {
    const int64_t row = band * R + r;
    if (row >= n) break;
    typename Acc<T>::type acc = zero<T>(), acc2 = zero<T>();
    const int64_t p1 = rp[row + 1];
    int64_t p = rp[row];
    for (; p + 4 <= p1; p += 4) {
      int l[4];
      T a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        l[u] = __ldg(&lcol[p + u]);
        a[u] = __ldg(&val[p + u]);
      }
      fma_c(acc, a[0], Xs[l[0] * P + s]);
      fma_c(acc2, a[1], Xs[l[1] * P + s]);
      fma_c(acc, a[2], Xs[l[2] * P + s]);
      fma_c(acc2, a[3], Xs[l[3] * P + s]);
    }
    for (; p < p1; ++p) fma_c(acc, __ldg(&val[p]), Xs[__ldg(&lcol[p]) * P + s]);  // as the row kernels
    acc.x += acc2.x;
    acc.y += acc2.y;
    store(Y, row, s, P, acc);
  }
}

// Band heights the layout is built for, and their index in petgem_ctx::bands.
constexpr int kBandHeights[3] = {16, 32, 64};
constexpr size_t kBandSmemMax = 200 * 1024;  // shared memory a band may use (its distinct X rows)

}  // namespace petgem

#include "ctx.cuh"

namespace petgem {

template <typename T, int P, int R, typename Store>
Status launch_spmm_band_r(petgem_ctx* c, cudaStream_t s, const BandLayout& B, const T* val, const T* X, T* Y,
                          const int* all_done, Store store) {
  static bool attr = false;  // once per instantiation
  if (!attr) {
    PG_CUDA(cudaFuncSetAttribute(k_spmm_band<T, P, R, Store>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBandSmemMax));
    attr = true;
  }
  const size_t smem = (size_t)B.max_u * P * sizeof(T);
  PG_CUDA(pdl_launch(k_spmm_band<T, P, R, Store>, dim3((unsigned)B.nb), dim3(256), smem, s, false,
                     (const int64_t*)B.off.as<int64_t>(), (const int32_t*)B.ucol.as<int32_t>(),
                     (const int64_t*)c->row_ptr.as<int64_t>(), (const uint16_t*)B.lcol.as<uint16_t>(), val, X, Y,
                     c->n_edges, all_done, store));
  return Status{};
}

// Y = A X with the staged kernel of band height kBandHeights[which] (its layout must exist).
template <typename T, int P, typename Store>
Status launch_spmm_band(petgem_ctx* c, cudaStream_t s, int which, const T* val, const T* X, T* Y, const int* all_done,
                        Store store) {
  const BandLayout& B = c->bands[which];
  if ((size_t)B.max_u * P * sizeof(T) > kBandSmemMax) return Status{PETGEM_ERR_UNSUPPORTED, "band too wide"};
  switch (which) {
    case 0: return launch_spmm_band_r<T, P, 16, Store>(c, s, B, val, X, Y, all_done, store);
    case 1: return launch_spmm_band_r<T, P, 32, Store>(c, s, B, val, X, Y, all_done, store);
    default: return launch_spmm_band_r<T, P, 64, Store>(c, s, B, val, X, Y, all_done, store);
  }
}

// Autotuner of the block SpMM: on the solver's own operands (val, X; Y is overwritten) it times
// the solver's row kernel (rows(), a launch of it) and the staged kernel for every band height
// (the band layouts are built on first use), one warm-up and ten timed launches each with CUDA
// events on the stream, and keeps the fastest for this problem shape: rows, nonzeros, source
// count and value type.  A new mesh of the same shape (a re-meshed model) keeps the choice, and
// a band form then gets its layout for the new mesh where it is launched.
// *choice: -1 for the row kernel, else the band height's index.
template <typename T, int P, typename Rows>
Status tune_spmm(petgem_ctx* c, cudaStream_t s, const T* val, const T* X, T* Y, Rows rows, int* choice) {
  const uint64_t key = ((uint64_t)c->n_edges << 24) ^ ((uint64_t)c->nnz << 8) ^ ((uint64_t)P << 4) ^ (uint64_t)sizeof(T);
  auto it = c->spmm_choice.find(key);
  if (it != c->spmm_choice.end()) {
    *choice = it->second;
    return Status{};
  }
  cudaEvent_t e0, e1;
  PG_CUDA(cudaEventCreate(&e0));
  PG_CUDA(cudaEventCreate(&e1));
  float best = INFINITY;
  int pick = -1;
  auto time_it = [&](auto&& launch, float* ms) -> Status {
    PG_TRY(launch());
    PG_CUDA(cudaEventRecord(e0, s));
    for (int k = 0; k < 10; ++k) PG_TRY(launch());
    PG_CUDA(cudaEventRecord(e1, s));
    PG_CUDA(cudaEventSynchronize(e1));
    PG_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return Status{};
  };
  Status st;
  float t = 0.f;
  st = time_it(rows, &t);
  if (st.ok()) best = t;
  for (int w = 0; w < 3 && st.ok(); ++w) {
    st = band_layout(c, w);
    if (!st.ok()) break;
    if ((size_t)c->bands[w].max_u * P * sizeof(T) > kBandSmemMax) continue;
    st = time_it([&]() { return launch_spmm_band<T, P>(c, s, w, val, X, Y, nullptr, SpmmStorePlain{}); }, &t);
    if (st.ok() && t < best) {
      best = t;
      pick = w;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PG_TRY(st);
  c->spmm_choice[key] = pick;
  *choice = pick;
  return Status{};
}

}  // namespace petgem
