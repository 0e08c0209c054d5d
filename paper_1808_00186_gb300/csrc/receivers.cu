// Field at receivers (Section 3 eq. 7): locate the tet holding each receiver, then
// E_s(x) = sum_i S_i N_i(x) e_g(i) with the Nedelec basis of Appendix B, plus E_p(x; sigma_p).
#include <math.h>

#include "ctx.cuh"
#include "physics.cuh"

namespace petgem {
namespace {

using namespace phys;

constexpr int kRxChunk = 512;  // receivers staged in shared memory per pass

// One thread per tet: test every receiver against the tet's bounding box, then against its
// barycentric coordinates; the lowest tet id with all coordinates >= -1e-12 wins (atomicMin).
__global__ void k_locate(const double* __restrict__ nodes, const int32_t* __restrict__ tets, int64_t n_tets,
                         const double* __restrict__ rx, int n_rcv, int32_t* __restrict__ found) {
  __shared__ double srx[kRxChunk][3];
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  TetGeom G;
  bool ok = false;
  double lo[3], hi[3];
  if (t < n_tets) {
    ok = tet_geometry(nodes, tets, t, G);
    for (int d = 0; d < 3; ++d) {
      lo[d] = fmin(fmin(G.p[0][d], G.p[1][d]), fmin(G.p[2][d], G.p[3][d]));
      hi[d] = fmax(fmax(G.p[0][d], G.p[1][d]), fmax(G.p[2][d], G.p[3][d]));
      double pad = 1e-9 * (hi[d] - lo[d]);
      lo[d] -= pad;
      hi[d] += pad;
    }
  }
  for (int r0 = 0; r0 < n_rcv; r0 += kRxChunk) {
    int nr = min(kRxChunk, n_rcv - r0);
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nr; i += blockDim.x) srx[i / 3][i % 3] = rx[3 * (int64_t)r0 + i];
    __syncthreads();
    if (!ok) continue;
    for (int r = 0; r < nr; ++r) {
      const double x = srx[r][0], y = srx[r][1], z = srx[r][2];
      if (x < lo[0] || x > hi[0] || y < lo[1] || y > hi[1] || z < lo[2] || z > hi[2]) continue;
      double d[3] = {x - G.p[0][0], y - G.p[0][1], z - G.p[0][2]};
      double l1 = dot(G.g[1], d), l2 = dot(G.g[2], d), l3 = dot(G.g[3], d);
      double l0 = 1.0 - l1 - l2 - l3;
      if (l0 >= -1e-12 && l1 >= -1e-12 && l2 >= -1e-12 && l3 >= -1e-12) atomicMin(&found[r0 + r], (int32_t)t);
    }
  }
}

// One thread per (source, receiver): out[s][r] = (E_p, E_s, E_p + E_s), NaN when not located.
__global__ void k_rcv_eval(const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                           const int32_t* __restrict__ tet_edges, const int8_t* __restrict__ signs,
                           const double* __restrict__ rx, int n_rcv, const int32_t* __restrict__ found,
                           const double2* __restrict__ xs, int64_t n_edges, int n_src, const double* __restrict__ src5,
                           double sigma_p, double kappa, const double2* __restrict__ ep_pre,
                           double2* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_src * n_rcv) return;
  int s = (int)(idx / n_rcv), r = (int)(idx - (int64_t)s * n_rcv);
  double2* o = out + idx * 9;
  int32_t t = found[r];
  TetGeom G;
  if (t == 0x7fffffff || !tet_geometry(nodes, tets, t, G)) {
    for (int k = 0; k < 9; ++k) o[k] = make_double2(nan(""), nan(""));
    return;
  }
  const double x[3] = {rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]};
  double d0[3] = {x[0] - G.p[0][0], x[1] - G.p[0][1], x[2] - G.p[0][2]};
  double lam[4];
  lam[1] = dot(G.g[1], d0);
  lam[2] = dot(G.g[2], d0);
  lam[3] = dot(G.g[3], d0);
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
  double2 Es[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  const double2* xv = xs + (int64_t)s * n_edges;
  for (int k = 0; k < 6; ++k) {
    const int a = kA[k], b = kB[k];
    double2 e = xv[tet_edges[6 * (int64_t)t + k]];
    double sg = (double)signs[6 * (int64_t)t + k];
    for (int dd = 0; dd < 3; ++dd) {
      double nk = sg * G.len[k] * (lam[a] * G.g[b][dd] - lam[b] * G.g[a][dd]);
      Es[dd].x += nk * e.x;
      Es[dd].y += nk * e.y;
    }
  }
  const double* sp = src5 + 5 * s;
  double dv[3] = {x[0] - sp[0], x[1] - sp[1], x[2] - sp[2]};
  double2 Ep[3];
  if (ep_pre) {  // layered background: E_p computed beforehand at the receivers
    for (int dd = 0; dd < 3; ++dd) Ep[dd] = ep_pre[idx * 3 + dd];
  } else {
    dipole_field(dv, (int)sp[4], sp[3], sigma_p, kappa, Ep);
  }
  for (int dd = 0; dd < 3; ++dd) {
    o[dd] = Ep[dd];
    o[3 + dd] = Es[dd];
    o[6 + dd] = cadd(Ep[dd], Es[dd]);
  }
}

}  // namespace

Status run_receivers(petgem_ctx* c, int32_t n_rcv, const double* rx, const double2* x, double2* out, bool* outside) {
  cudaStream_t s = c->stream;
  int32_t* found = nullptr;
  double* src5 = nullptr;
  PG_CUDA(cudaMallocAsync((void**)&found, n_rcv * sizeof(int32_t), s));
  PG_CUDA(cudaMallocAsync((void**)&src5, 5 * sizeof(double) * c->n_src, s));
  std::vector<double> h5(5 * c->n_src);
  for (int i = 0; i < c->n_src; ++i) {  // (x, y, z, moment, axis)
    h5[5 * i] = c->src[i].x;
    h5[5 * i + 1] = c->src[i].y;
    h5[5 * i + 2] = c->src[i].z;
    h5[5 * i + 3] = c->src[i].moment;
    h5[5 * i + 4] = (double)c->src[i].axis;
  }
  PG_CUDA(cudaMemcpyAsync(src5, h5.data(), h5.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  PG_CUDA(cudaMemsetAsync(found, 0x7f, n_rcv * sizeof(int32_t), s));  // 0x7f7f7f7f > any tet id
  {
    KernelTimer kt(c, "rcv_locate", (double)c->n_tets * 64);
    k_locate<<<blocks_for(c->n_tets, 128), 128, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(), c->n_tets, rx,
                                                        n_rcv, found);
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  // Receivers never located keep 0x7f7f7f7f; map them to the "not found" marker.
  std::vector<int32_t> hf(n_rcv);
  PG_CUDA(cudaMemcpyAsync(hf.data(), found, n_rcv * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  *outside = false;
  for (auto& f : hf)
    if (f >= c->n_tets) {
      f = 0x7fffffff;
      *outside = true;
    }
  PG_CUDA(cudaMemcpyAsync(found, hf.data(), n_rcv * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const double kappa = sqrt(c->omega * phys::kMu0 * c->sigma_p * 0.5);
  double2* ep = nullptr;
  if (c->bg_layers > 0) {  // layered background: E_p of every source at every receiver
    PG_CUDA(cudaMallocAsync((void**)&ep, (size_t)c->n_src * n_rcv * 3 * sizeof(double2), s));
    for (int i = 0; i < c->n_src; ++i) PG_TRY(layered_primary(c, c->src[i], n_rcv, rx, ep + (int64_t)i * n_rcv * 3));
  }
  k_rcv_eval<<<blocks_for((int64_t)c->n_src * n_rcv, 128), 128, 0, s>>>(
      c->nodes.as<double>(), c->tets.as<int32_t>(), c->tet_edges.as<int32_t>(), c->signs.as<int8_t>(), rx, n_rcv,
      found, x, c->n_edges, c->n_src, src5, c->sigma_p, kappa, ep, out);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  PG_CUDA(cudaFreeAsync(found, s));
  PG_CUDA(cudaFreeAsync(src5, s));
  if (ep) PG_CUDA(cudaFreeAsync(ep, s));
  PG_CUDA(cudaStreamSynchronize(s));
  return Status{};
}

}  // namespace petgem
