// Element matrices, primary-field right-hand sides and the deterministic global assembly.
//
// Section 3 eq. 9 with the mass term scaled by mu0 as in eqs. 3 and 6:
//   (K^e + i w mu0 sigma_e M^e) E_s^e = -i w mu0 (sigma_e - sigma_p) R^e,
// K^e and M^e from Appendix B eqs. B.14-B.15 (signed by eq. B.16), R^e_k = int S_k N_k . E_p,
// E_p the whole-space dipole field of Appendix A.  All in FP64.
#include <math.h>

#include "ctx.cuh"
#include "physics.cuh"

namespace petgem {
namespace {

using namespace phys;

// Packed upper-triangle index of (i, j), i <= j, row-major: 0..20.
__constant__ int kSym[36] = {0, 1, 2,  3,  4,  5,  1, 6,  7,  8,  9,  10, 2,  7,  11, 12, 13, 14,
                             3, 8, 12, 15, 16, 17, 4, 9, 13, 16, 18, 19, 5, 10, 14, 17, 19, 20};

// One thread per tet: the 21 distinct entries of the symmetric signed K^e and M^e (eqs. B.14-B.15).
// curl N_i = 2 l_i grad l_a x grad l_b is constant, so K_ij = V (curl N_i S_i) . (curl N_j S_j);
// M_ij = S_i S_j l_i l_j int (l_a gl_b - l_b gl_a) . (l_c gl_d - l_d gl_c) with
// int l_p l_q = V (1 + delta_pq) / 20.
__global__ void k_element(const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                          const int8_t* __restrict__ signs, int64_t n_tets, double* __restrict__ K21,
                          double* __restrict__ M21, double* __restrict__ vol, uint32_t* __restrict__ flags) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  TetGeom G;
  if (!tet_geometry(nodes, tets, t, G)) {
    atomicOr(flags, kFlagDegenerate);
    for (int k = 0; k < 21; ++k) {
      K21[k * n_tets + t] = 0.0;
      M21[k * n_tets + t] = 0.0;
    }
    vol[t] = 0.0;
    return;
  }
  double S[6], cu[6][3];
  for (int i = 0; i < 6; ++i) {
    S[i] = (double)signs[6 * t + i];
    cross(G.g[kA[i]], G.g[kB[i]], cu[i]);
    double f = 2.0 * G.len[i] * S[i];
    for (int d = 0; d < 3; ++d) cu[i][d] *= f;
  }
  double gg[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = a; b < 4; ++b) gg[a][b] = gg[b][a] = dot(G.g[a], G.g[b]);
  const double v20 = G.vol / 20.0;
  int k = 0;
  for (int i = 0; i < 6; ++i) {
    const int a = kA[i], b = kB[i];
    for (int j = i; j < 6; ++j, ++k) {
      const int c = kA[j], d = kB[j];
      double Iac = v20 * (a == c ? 2.0 : 1.0), Iad = v20 * (a == d ? 2.0 : 1.0);
      double Ibc = v20 * (b == c ? 2.0 : 1.0), Ibd = v20 * (b == d ? 2.0 : 1.0);
      double m = Iac * gg[b][d] - Iad * gg[b][c] - Ibc * gg[a][d] + Ibd * gg[a][c];
      K21[k * n_tets + t] = G.vol * dot(cu[i], cu[j]);
      M21[k * n_tets + t] = S[i] * S[j] * G.len[i] * G.len[j] * m;
    }
  }
  vol[t] = G.vol;
}

struct DipoleDev {
  double x, y, z, moment;
  int axis;
};

// One thread per (tet, source of this chunk): R^e_k = sum_q (V/4) S_k N_k(x_q) . E_p(x_q) on the
// symmetric 4-point rule (barycentric alpha, beta, beta, beta and permutations), then scaled by
// -i w mu0 (sigma_e - sigma_p).  Tets with sigma_e == sigma_p write zeros.  be layout:
// [slot = 6 t + k][chunk source].
__global__ void k_rhs(const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                      const int8_t* __restrict__ signs, const double* __restrict__ sigma, int64_t n_tets,
                      double sigma_p, double omega, const DipoleDev* __restrict__ src, int n_chunk,
                      double2* __restrict__ be) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_tets * n_chunk) return;
  int64_t t = idx / n_chunk;
  int sc = (int)(idx - t * n_chunk);
  double dsig = sigma[t] - sigma_p;
  if (dsig == 0.0) {
    for (int k = 0; k < 6; ++k) be[(6 * t + k) * n_chunk + sc] = make_double2(0.0, 0.0);
    return;
  }
  TetGeom G;
  if (!tet_geometry(nodes, tets, t, G)) {
    for (int k = 0; k < 6; ++k) be[(6 * t + k) * n_chunk + sc] = make_double2(0.0, 0.0);
    return;
  }
  const double alpha = 0.58541019662496845446, beta = 0.13819660112501051518;  // (5 +- ...) / 20
  const double kappa = sqrt(omega * kMu0 * sigma_p * 0.5);
  const DipoleDev D = src[sc];
  double2 R[6];
  for (int k = 0; k < 6; ++k) R[k] = make_double2(0.0, 0.0);
  for (int q = 0; q < 4; ++q) {
    double lam[4] = {beta, beta, beta, beta};
    lam[q] = alpha;
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = lam[0] * G.p[0][d] + lam[1] * G.p[1][d] + lam[2] * G.p[2][d] + lam[3] * G.p[3][d];
    double dv[3] = {x[0] - D.x, x[1] - D.y, x[2] - D.z};
    double2 E[3];
    dipole_field(dv, D.axis, D.moment, sigma_p, kappa, E);
    for (int k = 0; k < 6; ++k) {
      const int a = kA[k], b = kB[k];
      double N[3];
      for (int d = 0; d < 3; ++d) N[d] = G.len[k] * (lam[a] * G.g[b][d] - lam[b] * G.g[a][d]);
      double2 ne = make_double2(N[0] * E[0].x + N[1] * E[1].x + N[2] * E[2].x,
                                N[0] * E[0].y + N[1] * E[1].y + N[2] * E[2].y);
      R[k] = cadd(R[k], ne);
    }
  }
  // -i w mu0 dsig * (V/4) * S_k * R_k
  const double f = omega * kMu0 * dsig * G.vol * 0.25;
  for (int k = 0; k < 6; ++k) {
    double s = (double)signs[6 * t + k] * f;
    be[(6 * t + k) * n_chunk + sc] = make_double2(s * R[k].y, -s * R[k].x);
  }
}

// ---- layered background (Section 2): sigma_p varies by layer, E_p from the layered kernel
struct BgLayers {
  int nl;
  double zif[7];
  double sig[8];
};
// Layer holding height z (a point on an interface belongs to the layer above it).
__device__ inline int bg_layer(double z, const BgLayers& B) {
  int j = 0;
  while (j < B.nl - 1 && z < B.zif[j]) ++j;
  return j;
}
// Tets whose conductivity differs from their layer's (layer of the centroid): dsig[t], and with
// pts given, a slot each (tet_slot[t], -1 for the others) holding the four quadrature points of
// the 4-point rule (pts[4 slot + q][3]); *count receives the number of such tets.
__global__ void k_rhs_layered_points(const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                                     const double* __restrict__ sigma, int64_t n_tets, BgLayers B,
                                     int32_t* __restrict__ count, int32_t* __restrict__ tet_slot,
                                     double* __restrict__ dsig, double* __restrict__ pts) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  double p[4][3], zc = 0.0;
  for (int j = 0; j < 4; ++j) {
    const int64_t v = tets[4 * t + j];
    for (int d = 0; d < 3; ++d) p[j][d] = nodes[3 * v + d];
    zc += 0.25 * p[j][2];
  }
  const double ds = sigma[t] - B.sig[bg_layer(zc, B)];
  if (!pts) {
    dsig[t] = ds;
    if (ds != 0.0) atomicAdd(count, 1);
    return;
  }
  if (ds == 0.0) {
    tet_slot[t] = -1;
    return;
  }
  const int32_t slot = atomicAdd(count, 1);
  tet_slot[t] = slot;
  const double alpha = 0.58541019662496845446, beta = 0.13819660112501051518;
  for (int q = 0; q < 4; ++q) {
    double lam[4] = {beta, beta, beta, beta};
    lam[q] = alpha;
    for (int d = 0; d < 3; ++d)
      pts[(4 * (int64_t)slot + q) * 3 + d] = lam[0] * p[0][d] + lam[1] * p[1][d] + lam[2] * p[2][d] + lam[3] * p[3][d];
  }
}
// k_rhs with the primary field read from Ep[source][4 slot + q][3] (computed at the same points).
__global__ void k_rhs_layered(const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                              const int8_t* __restrict__ signs, const double* __restrict__ dsig,
                              const int32_t* __restrict__ tet_slot, int64_t n_tets, double omega,
                              const double2* __restrict__ Ep, int64_t n_pts, int s0, int n_chunk,
                              double2* __restrict__ be) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_tets * n_chunk) return;
  int64_t t = idx / n_chunk;
  int sc = (int)(idx - t * n_chunk);
  const int32_t slot = tet_slot[t];
  TetGeom G;
  if (slot < 0 || !tet_geometry(nodes, tets, t, G)) {
    for (int k = 0; k < 6; ++k) be[(6 * t + k) * n_chunk + sc] = make_double2(0.0, 0.0);
    return;
  }
  const double alpha = 0.58541019662496845446, beta = 0.13819660112501051518;
  const double2* ep = Ep + ((int64_t)(s0 + sc) * n_pts + 4 * (int64_t)slot) * 3;
  double2 R[6];
  for (int k = 0; k < 6; ++k) R[k] = make_double2(0.0, 0.0);
  for (int q = 0; q < 4; ++q) {
    double lam[4] = {beta, beta, beta, beta};
    lam[q] = alpha;
    const double2* E = ep + 3 * q;
    for (int k = 0; k < 6; ++k) {
      const int a = kA[k], b = kB[k];
      double N[3];
      for (int d = 0; d < 3; ++d) N[d] = G.len[k] * (lam[a] * G.g[b][d] - lam[b] * G.g[a][d]);
      R[k] = cadd(R[k], make_double2(N[0] * E[0].x + N[1] * E[1].x + N[2] * E[2].x,
                                     N[0] * E[0].y + N[1] * E[1].y + N[2] * E[2].y));
    }
  }
  const double f = omega * kMu0 * dsig[t] * G.vol * 0.25;
  for (int k = 0; k < 6; ++k) {
    double sg = (double)signs[6 * t + k] * f;
    be[(6 * t + k) * n_chunk + sc] = make_double2(sg * R[k].y, -sg * R[k].x);
  }
}

// b[s][e] = sum over the occurrences of edge e (sorted by slot = 6 t + k) of be; 0 on the boundary.
__global__ void k_rhs_gather(const int64_t* __restrict__ eptr, const int32_t* __restrict__ occ,
                             const uint8_t* __restrict__ boundary, int64_t n_edges, const double2* __restrict__ be,
                             int n_chunk, int s0, double2* __restrict__ b) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_edges * n_chunk) return;
  int sc = (int)(idx / n_edges);
  int64_t e = idx - (int64_t)sc * n_edges;
  double2 acc = make_double2(0.0, 0.0);
  if (!boundary[e]) {
    for (int64_t p = eptr[e]; p < eptr[e + 1]; ++p) acc = cadd(acc, be[(int64_t)occ[p] * n_chunk + sc]);
  }
  b[(int64_t)(s0 + sc) * n_edges + e] = acc;
}

// One thread per row: the global K[q] and M_sigma[q] = sums of the gathered element entries K^e
// and sigma_t M^e in (tet, i, j) order (an empty gather range is a Dirichlet identity entry:
// K = 1, M_sigma = 0), kept for later frequencies, and A[q] = K + i w mu0 M_sigma (eq. 9).  Also
// the diagonal.
__global__ void k_matrix_gather(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const int64_t* __restrict__ gptr, const uint64_t* __restrict__ pkey,
                                const uint8_t* __restrict__ pij, const double* __restrict__ K21,
                                const double* __restrict__ M21, const double* __restrict__ sigma,
                                int64_t n_tets, int64_t n_edges, double wmu0, double* __restrict__ kval,
                                double* __restrict__ mval, double2* __restrict__ val, double2* __restrict__ diag) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n_edges) return;
  double2 dg = make_double2(0.0, 0.0);
  for (int64_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
    int64_t g0 = gptr[q], g1 = gptr[q + 1];
    double ks = 0.0, ms = 0.0;
    if (g0 == g1) {
      ks = 1.0;
    } else {
      for (int64_t p = g0; p < g1; ++p) {
        int64_t t = (int64_t)(uint32_t)(pkey[p] & 0xffffffffu);
        int k = kSym[pij[p]];
        ks += K21[k * n_tets + t];
        ms += sigma[t] * M21[k * n_tets + t];
      }
    }
    kval[q] = ks;
    mval[q] = ms;
    const double2 a = make_double2(ks, wmu0 * ms);
    val[q] = a;
    if (col[q] == r) dg = a;
  }
  diag[r] = dg;
}

// Another frequency on the same mesh and conductivities: A[q] = K[q] + i w mu0 M_sigma[q] from
// the kept real matrices (eq. 9 is linear in w), one thread per row; also the diagonal.
__global__ void k_matrix_frequency(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const double* __restrict__ kval, const double* __restrict__ mval,
                                   int64_t n_edges, double wmu0, double2* __restrict__ val,
                                   double2* __restrict__ diag) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n_edges) return;
  double2 dg = make_double2(0.0, 0.0);
  for (int64_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
    const double2 a = make_double2(kval[q], wmu0 * mval[q]);
    val[q] = a;
    if (col[q] == r) dg = a;
  }
  diag[r] = dg;
}

}  // namespace

Status build_assembly(petgem_ctx* c, const double* sigma_dev) {
  cudaStream_t s = c->stream;
  const int64_t T = c->n_tets, E = c->n_edges, S = c->n_src;
  uint32_t* flags = c->flags.as<uint32_t>();
  PG_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
  PG_TRY(c->sigma.reserve(T * sizeof(double)));
  PG_CUDA(cudaMemcpyAsync(c->sigma.ptr, sigma_dev, T * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PG_TRY(c->K21.reserve(21 * T * sizeof(double)));
  PG_TRY(c->M21.reserve(21 * T * sizeof(double)));
  PG_TRY(c->vol.reserve(T * sizeof(double)));
  {
    KernelTimer kt(c, "element", (double)T * (4 * 4 + 12 * 8 + 6 + 43 * 8));
    k_element<<<blocks_for(T, 128), 128, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(), c->signs.as<int8_t>(),
                                                  T, c->K21.as<double>(), c->M21.as<double>(), c->vol.as<double>(),
                                                  flags);
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  PG_TRY(check_flags(c, "petgem_assemble"));

  PG_TRY(c->val.reserve(c->nnz * sizeof(double2)));
  PG_TRY(c->diag.reserve(E * sizeof(double2)));
  PG_TRY(c->kval.reserve(c->nnz * sizeof(double)));
  PG_TRY(c->mval.reserve(c->nnz * sizeof(double)));
  {
    KernelTimer kt(c, "matrix_gather", (double)c->nnz * (8 + 16 + 16 + 8) + (double)c->n_pairs * (9 + 24));
    k_matrix_gather<<<blocks_for(E, 128), 128, 0, s>>>(
        c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->gptr.as<int64_t>(), c->pkey.as<uint64_t>(),
        c->pij.as<uint8_t>(), c->K21.as<double>(), c->M21.as<double>(), c->sigma.as<double>(), T, E, c->omega * kMu0,
        c->kval.as<double>(), c->mval.as<double>(), c->val.as<double2>(), c->diag.as<double2>());
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  PG_TRY(build_rhs(c));
  c->assembled = true;
  c->assembly_version++;
  return Status{};
}

Status build_frequency(petgem_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t E = c->n_edges;
  uint32_t* flags = c->flags.as<uint32_t>();
  PG_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
  {
    KernelTimer kt(c, "matrix_frequency", (double)c->nnz * (8 + 8 + 4 + 16) + 8.0 * (E + 1) + 16.0 * E);
    k_matrix_frequency<<<blocks_for(E, 128), 128, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                           c->kval.as<double>(), c->mval.as<double>(), E,
                                                           c->omega * kMu0, c->val.as<double2>(), c->diag.as<double2>());
    c->launches++;
  }
  PG_CUDA(cudaGetLastError());
  PG_TRY(build_rhs(c));
  c->assembled = true;
  c->assembly_version++;
  return Status{};
}

// Right-hand sides of the context's sources at its frequency (eq. 6, App. A).
Status build_rhs(petgem_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t T = c->n_tets, E = c->n_edges, S = c->n_src;

  // Right-hand sides, in chunks of sources so the per-slot buffer stays near 1 GB.
  PG_TRY(c->b.reserve(S * E * sizeof(double2)));
  int64_t per_src = 6 * T * (int64_t)sizeof(double2);
  int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(1ll << 30) / std::max<int64_t>(per_src, 1)));
  double2* be = nullptr;
  PG_CUDA(cudaMallocAsync((void**)&be, per_src * chunk, s));
  DipoleDev* dsrc = nullptr;
  PG_CUDA(cudaMallocAsync((void**)&dsrc, sizeof(DipoleDev) * S, s));
  std::vector<DipoleDev> hsrc(S);
  for (int64_t i = 0; i < S; ++i)
    hsrc[i] = DipoleDev{c->src[i].x, c->src[i].y, c->src[i].z, c->src[i].moment, c->src[i].axis};
  PG_CUDA(cudaMemcpyAsync(dsrc, hsrc.data(), sizeof(DipoleDev) * S, cudaMemcpyHostToDevice, s));
  // layered background: the quadrature points of the tets whose conductivity differs from their
  // layer's, and the layered primary field of every source there
  int32_t *lcount = nullptr, *tet_slot = nullptr;
  double *dsig = nullptr, *lpts = nullptr;
  double2* Ep = nullptr;
  int64_t n_pts = 0;
  if (c->bg_layers > 0) {
    BgLayers B{};
    B.nl = c->bg_layers;
    for (int j = 0; j < 7; ++j) B.zif[j] = c->bg_z[j];
    for (int j = 0; j < 8; ++j) B.sig[j] = c->bg_sig[j];
    PG_CUDA(cudaMallocAsync((void**)&lcount, sizeof(int32_t), s));
    PG_CUDA(cudaMallocAsync((void**)&tet_slot, T * sizeof(int32_t), s));
    PG_CUDA(cudaMallocAsync((void**)&dsig, T * sizeof(double), s));
    PG_CUDA(cudaMemsetAsync(lcount, 0, sizeof(int32_t), s));
    k_rhs_layered_points<<<blocks_for(T, 256), 256, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(),
                                                            c->sigma.as<double>(), T, B, lcount, tet_slot, dsig, nullptr);
    int32_t hcount = 0;
    PG_CUDA(cudaMemcpyAsync(&hcount, lcount, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    n_pts = 4 * (int64_t)hcount;
    PG_CUDA(cudaMallocAsync((void**)&lpts, std::max<int64_t>(n_pts, 1) * 3 * sizeof(double), s));
    PG_CUDA(cudaMallocAsync((void**)&Ep, std::max<int64_t>(n_pts * S, 1) * 3 * sizeof(double2), s));
    PG_CUDA(cudaMemsetAsync(lcount, 0, sizeof(int32_t), s));
    k_rhs_layered_points<<<blocks_for(T, 256), 256, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(),
                                                            c->sigma.as<double>(), T, B, lcount, tet_slot, dsig, lpts);
    c->launches += 2;
    PG_CUDA(cudaGetLastError());
    for (int64_t i = 0; i < S; ++i) PG_TRY(layered_primary(c, c->src[i], n_pts, lpts, Ep + i * n_pts * 3));
  }
  for (int s0 = 0; s0 < S; s0 += chunk) {
    int n_chunk = (int)std::min<int64_t>(chunk, S - s0);
    {
      KernelTimer kt(c, "rhs", (double)T * n_chunk * 6 * 16);
      if (c->bg_layers > 0)
        k_rhs_layered<<<blocks_for(T * n_chunk, 128), 128, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(),
                                                                    c->signs.as<int8_t>(), dsig, tet_slot, T,
                                                                    c->omega, Ep, n_pts, s0, n_chunk, be);
      else
        k_rhs<<<blocks_for(T * n_chunk, 128), 128, 0, s>>>(c->nodes.as<double>(), c->tets.as<int32_t>(),
                                                            c->signs.as<int8_t>(), c->sigma.as<double>(), T,
                                                            c->sigma_p, c->omega, dsrc + s0, n_chunk, be);
      c->launches++;
    }
    PG_CUDA(cudaGetLastError());
    k_rhs_gather<<<blocks_for(E * n_chunk, 256), 256, 0, s>>>(c->eptr.as<int64_t>(), c->occ.as<int32_t>(),
                                                              c->boundary.as<uint8_t>(), E, be, n_chunk, s0,
                                                              c->b.as<double2>());
    c->launches++;
    PG_CUDA(cudaGetLastError());
  }
  PG_CUDA(cudaFreeAsync(be, s));
  PG_CUDA(cudaFreeAsync(dsrc, s));
  if (c->bg_layers > 0) {
    PG_CUDA(cudaFreeAsync(lcount, s));
    PG_CUDA(cudaFreeAsync(tet_slot, s));
    PG_CUDA(cudaFreeAsync(dsig, s));
    PG_CUDA(cudaFreeAsync(lpts, s));
    PG_CUDA(cudaFreeAsync(Ep, s));
  }
  PG_TRY(check_flags(c, "petgem_assemble"));
  return Status{};
}

}  // namespace petgem
