// Band layout of the CSR pattern for the staged block SpMM (bands.cuh): built once per mesh and
// band height on the host from the pattern (deterministic: columns sorted within a band).
#include <algorithm>
#include <vector>

#include "bands.cuh"
#include "ctx.cuh"

namespace petgem {

Status band_layout(petgem_ctx* c, int which) {
  BandLayout& B = c->bands[which];
  if (B.version == c->mesh_version) return Status{};
  const int R = kBandHeights[which];
  const int64_t n = c->n_edges, nnz = c->nnz;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> col(nnz);
  PG_CUDA(cudaMemcpyAsync(rp.data(), c->row_ptr.ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaMemcpyAsync(col.data(), c->col.ptr, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t nb = (n + R - 1) / R;
  std::vector<int64_t> off(nb + 1, 0);
  std::vector<int32_t> ucol;
  ucol.reserve((size_t)nnz / 3 + 16);
  std::vector<uint16_t> lcol(nnz);
  std::vector<int32_t> tmp;
  int max_u = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t p0 = rp[b * R], p1 = rp[std::min<int64_t>(n, (b + 1) * R)];
    tmp.assign(col.begin() + p0, col.begin() + p1);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    if (tmp.size() > 65535) return Status{PETGEM_ERR_UNSUPPORTED, "band layout: a band has over 65535 columns"};
    for (int64_t p = p0; p < p1; ++p)
      lcol[p] = (uint16_t)(std::lower_bound(tmp.begin(), tmp.end(), col[p]) - tmp.begin());
    ucol.insert(ucol.end(), tmp.begin(), tmp.end());
    off[b + 1] = (int64_t)ucol.size();
    max_u = std::max(max_u, (int)tmp.size());
  }
  PG_TRY(B.off.reserve((nb + 1) * sizeof(int64_t)));
  PG_TRY(B.ucol.reserve(std::max<size_t>(ucol.size(), 1) * sizeof(int32_t)));
  PG_TRY(B.lcol.reserve(std::max<int64_t>(nnz, 1) * sizeof(uint16_t)));
  PG_CUDA(cudaMemcpyAsync(B.off.ptr, off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  PG_CUDA(cudaMemcpyAsync(B.ucol.ptr, ucol.data(), ucol.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  PG_CUDA(cudaMemcpyAsync(B.lcol.ptr, lcol.data(), nnz * sizeof(uint16_t), cudaMemcpyHostToDevice, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
  B.nb = nb;
  B.max_u = max_u;
  B.version = c->mesh_version;
  return Status{};
}

}  // namespace petgem
