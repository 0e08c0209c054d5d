// Sliced-ELL (SELL-32) layout of the system matrix, rows in lattice-class order, for the
// bandwidth-bound sparse products of the Krylov solvers.
//
// CSR with four lanes per row leaves every nonzero's gather of x (8 bytes through L1) to an
// uncoalesced access, and the product is bound by the L1 data path (~75 % of the HBM rate).
// Here 32 consecutive rows form a slice, stored column-major: entry t of the slice's 32 rows is one
// 128-byte column index and one 256-byte value load.  The rows are renumbered so that a slice's
// 32 rows are 32 edges of the same kind at consecutive lattice nodes: edges are grouped by their
// node-id difference hi - lo (on a Kuhn lattice the 7 edge directions of a node), keeping their
// order (lo, hi) inside a group, so that consecutive rows have consecutive lower nodes.  With
// every row's entries sorted by the renumbered column, entry t of a slice then points at 32
// consecutive entries of x, and its gather is coalesced too.  A mesh with more than kSellMaxKinds
// distinct differences keeps the original order (the slices still stream their entries).
//
// The solvers that use it work on the renumbered vectors: x_new[r] = x[perm[r]].  The pattern is
// built once per mesh; values are gathered from any CSR value array of that pattern.
#include <algorithm>
#include <vector>

#include "ctx.cuh"

namespace petgem {
namespace {

constexpr int kSellMaxKinds = 64;   // distinct hi - lo differences that still get grouped
constexpr int kSellMaxRow = 64;     // longest row the layout takes

// Each edge's difference hi - lo into an open-addressing table of kSellMaxKinds keys (empty = -1).
__global__ void k_sell_kinds(const int32_t* __restrict__ edges, int64_t n, int32_t* __restrict__ table,
                             int32_t* __restrict__ overflow) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t d = edges[2 * e + 1] - edges[2 * e];
  int h = (int)(((uint32_t)d * 2654435761u) >> 26) & (kSellMaxKinds - 1);
  for (int probe = 0; probe < kSellMaxKinds; ++probe) {
    const int32_t k = table[h];
    if (k == d) return;
    if (k == -1) {
      const int32_t old = atomicCAS(&table[h], -1, d);
      if (old == -1 || old == d) return;
    }
    h = (h + 1) & (kSellMaxKinds - 1);
  }
  *overflow = 1;
}

// flag[e] = 1 when edge e has difference d (one kind at a time).
__global__ void k_sell_flag(const int32_t* __restrict__ edges, int64_t n, int32_t d, int32_t* __restrict__ flag) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  flag[e] = (edges[2 * e + 1] - edges[2 * e]) == d;
}

// Edges of one kind to their new positions base + (rank among the kind's edges).
__global__ void k_sell_place(const int32_t* __restrict__ flag, const int64_t* __restrict__ rank, int64_t n, int64_t base,
                             int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n || !flag[e]) return;
  const int64_t r = base + rank[e];
  perm[r] = (int32_t)e;
  inv[e] = (int32_t)r;
}

__global__ void k_sell_identity(int64_t n, int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  perm[e] = (int32_t)e;
  inv[e] = (int32_t)e;
}

// Slice widths (the longest renumbered row of each 32), times 32: one warp per slice.
__global__ void k_sell_width(const int64_t* __restrict__ rp, const int32_t* __restrict__ perm, int64_t n, int64_t ns,
                             int32_t* __restrict__ w32, int32_t* __restrict__ too_long) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= ns) return;
  const int64_t r = gw * 32 + lane;
  int len = 0;
  if (r < n) {
    const int64_t o = perm[r];
    len = (int)(rp[o + 1] - rp[o]);
  }
  for (int d = 16; d > 0; d >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, d));
  if (lane == 0) {
    w32[gw] = len * 32;
    if (len > kSellMaxRow) *too_long = 1;
  }
}

// Renumbered row r: its entries sorted by renumbered column into the slice's columns; src holds
// the CSR entry each slot takes its value from (-1: padding, column = the row itself).
__global__ void k_sell_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                            const int64_t* __restrict__ sp, int64_t n, int64_t ns, int32_t* __restrict__ scol,
                            int32_t* __restrict__ src) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= ns * 32) return;
  const int64_t s = r >> 5;
  const int lane = (int)(r & 31);
  const int64_t base = sp[s];
  const int w = (int)((sp[s + 1] - base) >> 5);
  int32_t c[kSellMaxRow];
  int32_t q[kSellMaxRow];
  int len = 0;
  if (r < n) {
    const int64_t o = perm[r];
    for (int64_t p = rp[o]; p < rp[o + 1] && len < kSellMaxRow; ++p, ++len) {
      // insertion by renumbered column
      const int32_t cc = inv[col[p]];
      int k = len;
      while (k > 0 && c[k - 1] > cc) {
        c[k] = c[k - 1];
        q[k] = q[k - 1];
        --k;
      }
      c[k] = cc;
      q[k] = (int32_t)p;
    }
  }
  const int32_t self = (int32_t)(r < n ? r : n - 1);
  for (int t = 0; t < w; ++t) {
    scol[base + (int64_t)t * 32 + lane] = t < len ? c[t] : self;
    src[base + (int64_t)t * 32 + lane] = t < len ? q[t] : -1;
  }
}

template <typename T>
__global__ void k_sell_values(const int32_t* __restrict__ src, int64_t m, const T* __restrict__ val, T* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int32_t q = src[i];
  T z;
  z.x = 0;
  z.y = 0;
  out[i] = q >= 0 ? val[q] : z;
}

}  // namespace

Status sell_prepare(petgem_ctx* c) {
  if (c->sell_version == c->mesh_version) return Status{};
  cudaStream_t s = c->stream;
  const int64_t n = c->n_edges, ns = (n + 31) / 32;
  c->sell_ok = false;
  if (n >= (1ll << 31) || c->nnz >= (1ll << 31)) {
    c->sell_version = c->mesh_version;
    return Status{};
  }
  PG_TRY(c->sell_perm.reserve(n * sizeof(int32_t)));
  PG_TRY(c->sell_inv.reserve(n * sizeof(int32_t)));
  int32_t* perm = c->sell_perm.as<int32_t>();
  int32_t* inv = c->sell_inv.as<int32_t>();
  const int32_t* edges = c->edges.as<int32_t>();
  // kinds of edges (node-id differences)
  DevBuf work;
  PG_TRY(work.reserve((kSellMaxKinds + 2) * sizeof(int32_t) + (size_t)n * sizeof(int32_t) + (size_t)(n + 1) * 8 + 64));
  int32_t* table = work.as<int32_t>();
  int32_t* flags = table + kSellMaxKinds;  // [0] overflow, [1] row too long
  int32_t* flag = table + kSellMaxKinds + 2;
  int64_t* rank = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(flag) + ((n * 4 + 15) / 16) * 16);
  Status st;
  auto body = [&]() -> Status {
    PG_CUDA(cudaMemsetAsync(table, 0xff, kSellMaxKinds * sizeof(int32_t), s));
    PG_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s));
    k_sell_kinds<<<blocks_for(n, 256), 256, 0, s>>>(edges, n, table, flags);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    int32_t htab[kSellMaxKinds + 2];
    PG_CUDA(cudaMemcpyAsync(htab, table, sizeof(htab), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> kinds;
    for (int i = 0; i < kSellMaxKinds; ++i)
      if (htab[i] != -1) kinds.push_back(htab[i]);
    std::sort(kinds.begin(), kinds.end());
    if (htab[kSellMaxKinds] || kinds.empty()) {
      k_sell_identity<<<blocks_for(n, 256), 256, 0, s>>>(n, perm, inv);
      c->launches++;
      PG_CUDA(cudaGetLastError());
    } else {
      int64_t base = 0;
      for (int32_t d : kinds) {
        k_sell_flag<<<blocks_for(n, 256), 256, 0, s>>>(edges, n, d, flag);
        c->launches++;
        PG_CUDA(cudaGetLastError());
        PG_TRY(exclusive_scan(flag, rank, n, s));
        k_sell_place<<<blocks_for(n, 256), 256, 0, s>>>(flag, rank, n, base, perm, inv);
        c->launches++;
        PG_CUDA(cudaGetLastError());
        int64_t cnt = 0;
        PG_CUDA(cudaMemcpyAsync(&cnt, rank + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
        base += cnt;
      }
      if (base != n) return Status{PETGEM_ERR_CUDA, "sell_prepare: edge kinds do not cover the edges"};
    }
    // slice widths and offsets
    int32_t* w32 = flag;  // reuse: ns <= n entries
    k_sell_width<<<blocks_for(ns * 32, 256), 256, 0, s>>>(c->row_ptr.as<int64_t>(), perm, n, ns, w32, flags + 1);
    c->launches++;
    PG_CUDA(cudaGetLastError());
    PG_TRY(c->sell_sp.reserve((ns + 1) * sizeof(int64_t)));
    PG_TRY(exclusive_scan(w32, c->sell_sp.as<int64_t>(), ns, s));
    int64_t total = 0;
    int32_t too_long = 0;
    PG_CUDA(cudaMemcpyAsync(&total, c->sell_sp.as<int64_t>() + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaMemcpyAsync(&too_long, flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (too_long) return Status{};  // rows too long for the layout: the solvers keep CSR
    PG_TRY(c->sell_col.reserve(total * sizeof(int32_t)));
    PG_TRY(c->sell_src.reserve(total * sizeof(int32_t)));
    k_sell_fill<<<blocks_for(ns * 32, 128), 128, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), perm, inv,
                                                         c->sell_sp.as<int64_t>(), n, ns, c->sell_col.as<int32_t>(),
                                                         c->sell_src.as<int32_t>());
    c->launches++;
    PG_CUDA(cudaGetLastError());
    c->sell_ns = ns;
    c->sell_nnz = total;
    c->sell_ok = true;
    return Status{};
  };
  st = body();
  cudaStreamSynchronize(s);  // the work buffer is released on return
  work.release();
  if (!st.ok()) return st;
  c->sell_version = c->mesh_version;
  return Status{};
}

template <typename T>
Status sell_values(petgem_ctx* c, const T* csr_val, T* out) {
  k_sell_values<T><<<blocks_for(c->sell_nnz, 256), 256, 0, c->stream>>>(c->sell_src.as<int32_t>(), c->sell_nnz, csr_val,
                                                                       out);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  return Status{};
}
template Status sell_values<float2>(petgem_ctx*, const float2*, float2*);
template Status sell_values<double2>(petgem_ctx*, const double2*, double2*);

}  // namespace petgem
