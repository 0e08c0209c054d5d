// Mesh topology on the GPU: global edge numbering and orientation (Appendix B eq. B.16),
// boundary edges (Section 2 Dirichlet condition) and the CSR pattern with its deterministic
// gather map.
//
// Every "sort" here is a counting sort on the first key (a node id or an edge id, with
// atomics only deciding slot positions) followed by an in-segment sort on the remaining key
// and the payload.  The output is therefore fully determined by the input: the same
// lexicographic order a global sort would give, with no dependence on atomic ordering.
#include "ctx.cuh"

namespace petgem {
namespace {

// Local edge i joins local nodes (kA[i], kB[i]) and its basis is W_{kA kB} (Appendix B,
// eqs. B.1-B.6; N5 runs from node 4 to node 2).
__constant__ int kA[6] = {0, 0, 0, 1, 3, 2};
__constant__ int kB[6] = {1, 2, 3, 2, 1, 3};

constexpr int kThreads = 256;
constexpr int kLocalSort = 48;  // segments up to this length are sorted in registers/local memory

// ---------------------------------------------------------------- edges
__global__ void k_edge_count(const int32_t* __restrict__ tets, int64_t n_tets, int64_t n_nodes,
                             int32_t* __restrict__ cnt, int8_t* __restrict__ signs,
                             uint32_t* __restrict__ flags) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 6 * n_tets) return;
  int64_t t = idx / 6;
  int e = (int)(idx - 6 * t);
  int32_t n1 = tets[4 * t + kA[e]], n2 = tets[4 * t + kB[e]];
  if (n1 < 0 || n2 < 0 || n1 >= n_nodes || n2 >= n_nodes) {
    atomicOr(flags, kFlagBadNode);
    signs[idx] = 0;
    return;
  }
  if (n1 == n2) {
    atomicOr(flags, kFlagRepeatedNode);
    signs[idx] = 0;
    return;
  }
  signs[idx] = n2 > n1 ? (int8_t)1 : (int8_t)-1;  // eq. B.16: sign of node_i2 - node_i1
  atomicAdd(&cnt[min(n1, n2)], 1);
}

__global__ void k_edge_scatter(const int32_t* __restrict__ tets, int64_t n_tets, int64_t n_nodes,
                               const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                               uint64_t* __restrict__ keys) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 6 * n_tets) return;
  int64_t t = idx / 6;
  int e = (int)(idx - 6 * t);
  int32_t n1 = tets[4 * t + kA[e]], n2 = tets[4 * t + kB[e]];
  if (n1 < 0 || n2 < 0 || n1 >= n_nodes || n2 >= n_nodes || n1 == n2) return;
  int32_t lo = min(n1, n2), hi = max(n1, n2);
  int64_t pos = off[lo] + atomicAdd(&cursor[lo], 1);
  keys[pos] = ((uint64_t)(uint32_t)hi << 32) | (uint64_t)(uint32_t)idx;
}

// Sort keys[begin, end) ascending (insertion sort; segments are short: a node is the low end of
// a handful of edges, each shared by a handful of tets).  `aux` (optional) moves with the keys.
__device__ void sort_segment(uint64_t* keys, uint8_t* aux, int64_t begin, int64_t end) {
  int64_t len = end - begin;
  if (len <= 1) return;
  if (len <= kLocalSort) {
    uint64_t k[kLocalSort];
    uint8_t a[kLocalSort];
    for (int i = 0; i < len; ++i) {
      k[i] = keys[begin + i];
      a[i] = aux ? aux[begin + i] : 0;
    }
    for (int i = 1; i < len; ++i) {
      uint64_t kv = k[i];
      uint8_t av = a[i];
      int j = i - 1;
      while (j >= 0 && k[j] > kv) {
        k[j + 1] = k[j];
        a[j + 1] = a[j];
        --j;
      }
      k[j + 1] = kv;
      a[j + 1] = av;
    }
    for (int i = 0; i < len; ++i) {
      keys[begin + i] = k[i];
      if (aux) aux[begin + i] = a[i];
    }
    return;
  }
  for (int64_t i = begin + 1; i < end; ++i) {
    uint64_t kv = keys[i];
    uint8_t av = aux ? aux[i] : 0;
    int64_t j = i - 1;
    while (j >= begin && keys[j] > kv) {
      keys[j + 1] = keys[j];
      if (aux) aux[j + 1] = aux[j];
      --j;
    }
    keys[j + 1] = kv;
    if (aux) aux[j + 1] = av;
  }
}

// Sort each node's segment by (high id, slot) and count its distinct high ids.
__global__ void k_edge_segments(const int64_t* __restrict__ off, uint64_t* __restrict__ keys, int64_t n,
                                int32_t* __restrict__ ucnt) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  int64_t b = off[v], e = off[v + 1];
  sort_segment(keys, nullptr, b, e);
  int32_t u = 0;
  uint32_t prev = 0xffffffffu;
  for (int64_t p = b; p < e; ++p) {
    uint32_t hi = (uint32_t)(keys[p] >> 32);
    if (hi != prev) ++u;
    prev = hi;
  }
  ucnt[v] = u;
}

// Edge id = rank of (low, high): the node's base plus the rank of high within its segment.
__global__ void k_edge_assign(const int64_t* __restrict__ off, const uint64_t* __restrict__ keys, int64_t n,
                              const int64_t* __restrict__ ebase, int32_t* __restrict__ tet_edges,
                              int32_t* __restrict__ edges, int32_t* __restrict__ occ,
                              int64_t* __restrict__ eptr) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  int64_t b = off[v], e = off[v + 1];
  int64_t id = ebase[v] - 1;
  uint32_t prev = 0xffffffffu;
  for (int64_t p = b; p < e; ++p) {
    uint32_t hi = (uint32_t)(keys[p] >> 32);
    uint32_t slot = (uint32_t)(keys[p] & 0xffffffffu);
    if (hi != prev) {
      ++id;
      edges[2 * id] = (int32_t)v;
      edges[2 * id + 1] = (int32_t)hi;
      eptr[id] = p;
    }
    prev = hi;
    tet_edges[slot] = (int32_t)id;
    occ[p] = (int32_t)slot;
  }
}

// ---------------------------------------------------------------- boundary faces
__device__ inline void face_nodes(const int32_t* tets, int64_t t, int o, int32_t& a, int32_t& b, int32_t& c) {
  int32_t v[3];
  int m = 0;
  for (int j = 0; j < 4; ++j)
    if (j != o) v[m++] = tets[4 * t + j];
  a = min(v[0], min(v[1], v[2]));
  c = max(v[0], max(v[1], v[2]));
  b = v[0] + v[1] + v[2] - a - c;
}

__global__ void k_face_count(const int32_t* __restrict__ tets, int64_t n_tets, int32_t* __restrict__ cnt) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 4 * n_tets) return;
  int32_t a, b, c;
  face_nodes(tets, idx >> 2, (int)(idx & 3), a, b, c);
  atomicAdd(&cnt[a], 1);
}

__global__ void k_face_scatter(const int32_t* __restrict__ tets, int64_t n_tets, const int64_t* __restrict__ off,
                               int32_t* __restrict__ cursor, uint64_t* __restrict__ fkey,
                               uint32_t* __restrict__ fpay) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 4 * n_tets) return;
  int32_t a, b, c;
  face_nodes(tets, idx >> 2, (int)(idx & 3), a, b, c);
  int64_t pos = off[a] + atomicAdd(&cursor[a], 1);
  fkey[pos] = ((uint64_t)(uint32_t)b << 32) | (uint32_t)c;
  fpay[pos] = (uint32_t)idx;
}

// Faces of one node's segment: a run of length 1 is a boundary face and flags its three edges;
// a run longer than 2 is a non-manifold face.  Payload order inside a run does not matter.
__global__ void k_face_mark(const int64_t* __restrict__ off, const uint64_t* __restrict__ fkey,
                            const uint32_t* __restrict__ fpay, int64_t n,
                            const int32_t* __restrict__ tet_edges, uint8_t* __restrict__ boundary,
                            uint32_t* __restrict__ flags) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  int64_t b = off[v], e = off[v + 1];
  for (int64_t p = b; p < e; ++p) {
    // Faces with the same low node are few: count the copies of this face in the segment.
    uint64_t k = fkey[p];
    int64_t run = 0;
    for (int64_t r = b; r < e; ++r) run += (fkey[r] == k);
    if (run > 2) atomicOr(flags, kFlagNonManifold);
    if (run == 1) {
      uint32_t pay = fpay[p];
      int64_t t = pay >> 2;
      int o = (int)(pay & 3);
      for (int i = 0; i < 6; ++i)
        if (kA[i] != o && kB[i] != o) boundary[tet_edges[6 * t + i]] = 1;
    }
  }
}

// ---------------------------------------------------------------- CSR pattern
// Row r of an interior edge couples to the interior edges of every tet holding r.  One pair
// (r, c) per (tet, i, j) with r = te[t][i], c = te[t][j] both interior.
__global__ void k_pair_count(const int32_t* __restrict__ te, const uint8_t* __restrict__ boundary,
                             int64_t n_tets, int32_t* __restrict__ cnt) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 6 * n_tets) return;
  int64_t t = idx / 6;
  int32_t r = te[idx];
  if (boundary[r]) return;
  int k = 0;
  for (int j = 0; j < 6; ++j) k += boundary[te[6 * t + j]] ? 0 : 1;
  atomicAdd(&cnt[r], k);
}

__global__ void k_pair_scatter(const int32_t* __restrict__ te, const uint8_t* __restrict__ boundary,
                               int64_t n_tets, const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                               uint64_t* __restrict__ pkey, uint8_t* __restrict__ pij) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 6 * n_tets) return;
  int64_t t = idx / 6;
  int i = (int)(idx - 6 * t);
  int32_t r = te[idx];
  if (boundary[r]) return;
  int k = 0;
  for (int j = 0; j < 6; ++j) k += boundary[te[6 * t + j]] ? 0 : 1;
  int64_t pos = off[r] + atomicAdd(&cursor[r], k);
  for (int j = 0; j < 6; ++j) {
    int32_t c = te[6 * t + j];
    if (boundary[c]) continue;
    pkey[pos] = ((uint64_t)(uint32_t)c << 32) | (uint64_t)(uint32_t)t;
    pij[pos] = (uint8_t)(6 * i + j);
    ++pos;
  }
}

__global__ void k_pair_segments(const int64_t* __restrict__ off, uint64_t* __restrict__ pkey,
                                uint8_t* __restrict__ pij, const uint8_t* __restrict__ boundary, int64_t n,
                                int32_t* __restrict__ ucnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  if (boundary[r]) {
    ucnt[r] = 1;
    return;
  }
  int64_t b = off[r], e = off[r + 1];
  sort_segment(pkey, pij, b, e);
  int32_t u = 0;
  uint32_t prev = 0xffffffffu;
  for (int64_t p = b; p < e; ++p) {
    uint32_t c = (uint32_t)(pkey[p] >> 32);
    if (c != prev) ++u;
    prev = c;
  }
  ucnt[r] = u;
}

__global__ void k_pattern_write(const int64_t* __restrict__ off, const uint64_t* __restrict__ pkey,
                                const uint8_t* __restrict__ boundary, int64_t n,
                                const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                int64_t* __restrict__ gptr) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int64_t q = row_ptr[r];
  if (boundary[r]) {  // identity row: its gather range is empty
    col[q] = (int32_t)r;
    gptr[q] = off[r];
    return;
  }
  uint32_t prev = 0xffffffffu;
  for (int64_t p = off[r]; p < off[r + 1]; ++p) {
    uint32_t c = (uint32_t)(pkey[p] >> 32);
    if (c != prev) {
      col[q] = (int32_t)c;
      gptr[q] = p;
      ++q;
    }
    prev = c;
  }
}

// Stream-ordered temporaries released (in stream order) when the owner goes out of scope,
// also on early error returns.
struct Temps {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Temps(cudaStream_t st) : s(st) {}
  ~Temps() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  Status alloc(T** p, size_t count) {
    PG_CUDA(cudaMallocAsync((void**)p, count * sizeof(T) + 16, s));
    ptrs.push_back(*p);
    return Status{};
  }
};

}  // namespace

// ---------------------------------------------------------------- scan
namespace {
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

template <typename In>
__global__ void k_scan_tiles(const In* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ tile_sums) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
    run += v[i];
  }
  // inclusive scan of per-thread totals within the block
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = run;
  for (int d = 1; d < 32; d <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  int64_t wofs = 0;
  for (int k = 0; k < w; ++k) wofs += warp_tot[k];
  int64_t excl = wofs + x - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = excl;
    excl += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tile_ofs) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_ofs[i / kScanTile];
}

template <typename In>
Status scan_impl(const In* in, int64_t* out, int64_t n, cudaStream_t s) {
  // out[0..n-1] exclusive; out[n] = total.
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) {
    PG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return Status{};
  }
  if (tiles == 1) {  // one tile: its total lands directly in out[n]
    k_scan_tiles<In><<<1, kScanThreads, 0, s>>>(in, out, n, out + n);
    PG_CUDA(cudaGetLastError());
    return Status{};
  }
  int64_t* sums = nullptr;
  int64_t* sums_scan = nullptr;
  Temps tmp(s);
  PG_TRY(tmp.alloc(&sums, tiles));
  PG_TRY(tmp.alloc(&sums_scan, tiles + 1));
  k_scan_tiles<In><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
  PG_CUDA(cudaGetLastError());
  PG_TRY(scan_impl<int64_t>(sums, sums_scan, tiles, s));
  k_scan_add<<<blocks_for(n, 256), 256, 0, s>>>(out, n, sums_scan);
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaMemcpyAsync(out + n, sums_scan + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  return Status{};
}
}  // namespace

Status exclusive_scan(const int32_t* in, int64_t* out, int64_t n, cudaStream_t stream) {
  return scan_impl<int32_t>(in, out, n, stream);
}

// ---------------------------------------------------------------- driver
Status build_topology(petgem_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t Nn = c->n_nodes, T = c->n_tets;
  const int32_t* tets = c->tets.as<int32_t>();
  uint32_t* flags = c->flags.as<uint32_t>();
  PG_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
  Temps tmp(s);

  // -- edges: counting sort on the low node id, then (high id, slot) inside each node's segment
  int32_t* cnt = nullptr;
  int64_t* off = nullptr;
  uint64_t* keys = nullptr;
  PG_TRY(tmp.alloc(&cnt, Nn));
  PG_TRY(tmp.alloc(&off, Nn + 1));
  PG_TRY(tmp.alloc(&keys, 6 * T));
  PG_TRY(c->signs.reserve(6 * T));
  PG_CUDA(cudaMemsetAsync(cnt, 0, Nn * sizeof(int32_t), s));
  k_edge_count<<<blocks_for(6 * T, kThreads), kThreads, 0, s>>>(tets, T, Nn, cnt, c->signs.as<int8_t>(), flags);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  PG_TRY(check_flags(c, "petgem_mesh_edges"));
  PG_TRY(exclusive_scan(cnt, off, Nn, s));
  c->launches += 3;
  PG_CUDA(cudaMemsetAsync(cnt, 0, Nn * sizeof(int32_t), s));
  k_edge_scatter<<<blocks_for(6 * T, kThreads), kThreads, 0, s>>>(tets, T, Nn, off, cnt, keys);
  k_edge_segments<<<blocks_for(Nn, 128), 128, 0, s>>>(off, keys, Nn, cnt);
  c->launches += 2;
  PG_CUDA(cudaGetLastError());
  int64_t* ebase = nullptr;
  PG_TRY(tmp.alloc(&ebase, Nn + 1));
  PG_TRY(exclusive_scan(cnt, ebase, Nn, s));
  c->launches += 3;
  int64_t E = 0;
  PG_CUDA(cudaMemcpyAsync(&E, ebase + Nn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  c->n_edges = E;
  PG_TRY(c->edges.reserve(2 * E * sizeof(int32_t)));
  PG_TRY(c->tet_edges.reserve(6 * T * sizeof(int32_t)));
  PG_TRY(c->occ.reserve(6 * T * sizeof(int32_t)));
  PG_TRY(c->eptr.reserve((E + 1) * sizeof(int64_t)));
  k_edge_assign<<<blocks_for(Nn, 128), 128, 0, s>>>(off, keys, Nn, ebase, c->tet_edges.as<int32_t>(),
                                                    c->edges.as<int32_t>(), c->occ.as<int32_t>(),
                                                    c->eptr.as<int64_t>());
  c->launches++;
  PG_CUDA(cudaGetLastError());
  int64_t six_t = 6 * T;
  PG_CUDA(cudaMemcpyAsync(c->eptr.as<int64_t>() + E, &six_t, sizeof(int64_t), cudaMemcpyHostToDevice, s));

  // -- boundary: faces keyed by their sorted node triple; a face seen once is on the boundary
  uint64_t* fkey = nullptr;
  uint32_t* fpay = nullptr;
  PG_TRY(tmp.alloc(&fkey, 4 * T));
  PG_TRY(tmp.alloc(&fpay, 4 * T));
  PG_CUDA(cudaMemsetAsync(cnt, 0, Nn * sizeof(int32_t), s));
  k_face_count<<<blocks_for(4 * T, kThreads), kThreads, 0, s>>>(tets, T, cnt);
  PG_TRY(exclusive_scan(cnt, off, Nn, s));
  PG_CUDA(cudaMemsetAsync(cnt, 0, Nn * sizeof(int32_t), s));
  k_face_scatter<<<blocks_for(4 * T, kThreads), kThreads, 0, s>>>(tets, T, off, cnt, fkey, fpay);
  PG_TRY(c->boundary.reserve(E));
  PG_CUDA(cudaMemsetAsync(c->boundary.ptr, 0, E, s));
  k_face_mark<<<blocks_for(Nn, 128), 128, 0, s>>>(off, fkey, fpay, Nn, c->tet_edges.as<int32_t>(),
                                                  c->boundary.as<uint8_t>(), flags);
  c->launches += 6;
  PG_CUDA(cudaGetLastError());
  PG_TRY(check_flags(c, "petgem_mesh_edges"));

  // -- CSR pattern over interior rows + identity boundary rows, with the gather map
  int32_t* rcnt = nullptr;
  int64_t* poff = nullptr;
  PG_TRY(tmp.alloc(&rcnt, E));
  PG_TRY(tmp.alloc(&poff, E + 1));
  PG_CUDA(cudaMemsetAsync(rcnt, 0, E * sizeof(int32_t), s));
  const int32_t* te = c->tet_edges.as<int32_t>();
  const uint8_t* bd = c->boundary.as<uint8_t>();
  k_pair_count<<<blocks_for(6 * T, kThreads), kThreads, 0, s>>>(te, bd, T, rcnt);
  c->launches++;
  PG_TRY(exclusive_scan(rcnt, poff, E, s));
  c->launches += 3;
  int64_t P = 0;
  PG_CUDA(cudaMemcpyAsync(&P, poff + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  c->n_pairs = P;
  PG_TRY(c->pkey.reserve((P + 1) * sizeof(uint64_t)));
  PG_TRY(c->pij.reserve(P + 16));
  PG_CUDA(cudaMemsetAsync(rcnt, 0, E * sizeof(int32_t), s));
  k_pair_scatter<<<blocks_for(6 * T, kThreads), kThreads, 0, s>>>(te, bd, T, poff, rcnt, c->pkey.as<uint64_t>(),
                                                                 c->pij.as<uint8_t>());
  k_pair_segments<<<blocks_for(E, 128), 128, 0, s>>>(poff, c->pkey.as<uint64_t>(), c->pij.as<uint8_t>(), bd, E,
                                                     rcnt);
  c->launches += 2;
  PG_CUDA(cudaGetLastError());
  PG_TRY(c->row_ptr.reserve((E + 1) * sizeof(int64_t)));
  PG_TRY(exclusive_scan(rcnt, c->row_ptr.as<int64_t>(), E, s));
  c->launches += 3;
  int64_t nnz = 0;
  PG_CUDA(cudaMemcpyAsync(&nnz, c->row_ptr.as<int64_t>() + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  c->nnz = nnz;
  PG_TRY(c->col.reserve(nnz * sizeof(int32_t)));
  PG_TRY(c->gptr.reserve((nnz + 1) * sizeof(int64_t)));
  k_pattern_write<<<blocks_for(E, 128), 128, 0, s>>>(poff, c->pkey.as<uint64_t>(), bd, E, c->row_ptr.as<int64_t>(),
                                                     c->col.as<int32_t>(), c->gptr.as<int64_t>());
  c->launches++;
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaMemcpyAsync(c->gptr.as<int64_t>() + nnz, &c->n_pairs, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PG_CUDA(cudaStreamSynchronize(s));
  return Status{};
}

}  // namespace petgem
