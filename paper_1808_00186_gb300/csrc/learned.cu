// Learned preconditioner: a small 3-D convolutional U-Net on the node lattice of a Kuhn-split
// mesh, acting through the two auxiliary spaces of lowest-order edge elements (the
// Hiptmair-Xu decomposition): nodal gradients G phi, which the curl-curl term annihilates, and
// nodal vector fields Pi w.  For a residual r the preconditioner returns
//     z = D^{-1} r + G phi + Pi w,   (phi, w) = network(G^T r, Pi^T r, model features),
// the additive auxiliary-space preconditioner with the two nodal solves (G^T A G and Pi^T A Pi,
// nodal problems on the lattice) replaced by the network.  The edge degrees of freedom are
// tangential components, so (G phi)_e = (phi_hi - phi_lo) / |t_e| and
// (Pi w)_e = (w_lo + w_hi) . t_e / (2 |t_e|); phi, w vanish on the outer boundary (Dirichlet).
// Trained on the GPU with the library's own tensor-core kernels on solver residuals, loss = the
// residual angle of one step along z.  Inside flexible GMRES every step uses z (in the solver's
// Jacobi-scaled variables, D z).  Not part of the paper: the paper solves with GMRES / SQMR /
// MUMPS (Sections 5.1-5.3); the plain solver stays the fallback.
//
// Network (levels G0 = lattice nodes, G1 .. G(L-1) = successive 2x average poolings until the
// coarsest level has at most 3 nodes per axis, L >= 3; BF16 activations, FP32 accumulation and
// master weights).  Seven weight sets serve any depth:
//   e0 = relu(c1 16->16 on G0)                  e1 = relu(c2 16->32 on pool e0)
//   e_l = relu(c3 32->32 on pool e_(l-1))       for 2 <= l <= L-2 (c3 shared by these levels)
//   e_(L-1) = relu(c4 32->32 on pool e_(L-2))   (the coarsest level)
//   d_l = relu(c5 32->32 on up(d_(l+1)) + e_l)  for L-2 >= l >= 2 (d_(L-1) = e_(L-1); c5 shared)
//   d1 = relu(c6 32->16 on up(d2) + e1)         y = c7 16->16 on up(d1) + e0
//   (channels 8..15 of y unused; with L = 3 the c3 / c5 levels are absent)
// Input channels (sg = |diag(G^T A G)|^{-1/2}, sp = |diag(Pi^T A Pi)|^{-1/2} per node and axis,
// zero on boundary nodes; fg = sg G^T r, fp = sp Pi^T r; s = RMS of (fg, fp) over the interior
// nodes' four complex values): Re fg / s, Im fg / s, Re fp / s (x, y, z), Im fp / s (x, y, z),
// log10(sigma / sigma_p), log10(w mu0 sigma h^2) of the cell at the node, six zeros.
// Output: phi = s sg (y0 + i y1), w = s sp (y2..4 + i y5..7).
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "learned_kernels.cuh"
#include "learned.cuh"

namespace petgem {
namespace nn {
namespace {

constexpr int kIn = 16;

__device__ inline void grid_coords(int64_t v, int gx, int gy, int& x, int& y, int& z) {
  x = (int)(v % gx);
  y = (int)((v / gx) % gy);
  z = (int)(v / ((int64_t)gx * gy));
}

// Average of the existing children 2c + {0,1}^3 of every coarse voxel; one thread per coarse
// voxel and 8 channels (16-byte loads and stores).
__global__ void k_pool(const __nv_bfloat16* __restrict__ in, int gx, int gy, int gz, int C,
                       __nv_bfloat16* __restrict__ out, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int cx = (gx + 1) / 2, cy = (gy + 1) / 2, cz = (gz + 1) / 2;
  const int C8 = C / 8;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)cx * cy * cz * C8) return;
  const int c8 = (int)(idx % C8);
  int x, y, z;
  grid_coords(idx / C8, cx, cy, x, y, z);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int n = 0;
  for (int o = 0; o < 8; ++o) {
    const int fx = 2 * x + (o & 1), fy = 2 * y + ((o >> 1) & 1), fz = 2 * z + (o >> 2);
    if (fx < gx && fy < gy && fz < gz) {
      const uint4 u = *reinterpret_cast<const uint4*>(in + ((int64_t)fx + gx * ((int64_t)fy + (int64_t)gy * fz)) * C + 8 * c8);
      const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(b[k]);
      ++n;
    }
  }
  __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) o8[k] = __float2bfloat16(s[k] / n);
  *reinterpret_cast<uint4*>(out + (idx / C8) * C + 8 * c8) = *reinterpret_cast<const uint4*>(o8);
}
// din[f] += dout[parent(f)] / (children of the parent)
__global__ void k_pool_bwd_add(const __nv_bfloat16* __restrict__ dout, int gx, int gy, int gz, int C,
                               __nv_bfloat16* __restrict__ din) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)gx * gy * gz * C) return;
  const int c = (int)(idx % C);
  int x, y, z;
  grid_coords(idx / C, gx, gy, x, y, z);
  const int cx = (gx + 1) / 2, cy = (gy + 1) / 2;
  const int px = x / 2, py = y / 2, pz = z / 2;
  const int nx = (2 * px + 1 < gx) ? 2 : 1, ny = (2 * py + 1 < gy) ? 2 : 1, nz = (2 * pz + 1 < gz) ? 2 : 1;
  const float g = __bfloat162float(dout[((int64_t)px + cx * ((int64_t)py + (int64_t)cy * pz)) * C + c]) / (nx * ny * nz);
  din[idx] = __float2bfloat16(__bfloat162float(din[idx]) + g);
}
// out[f] = coarse[parent(f)] + skip[f]; one thread per fine voxel and 8 channels.
__global__ void k_up_add(const __nv_bfloat16* __restrict__ coarse, const __nv_bfloat16* __restrict__ skip, int gx,
                         int gy, int gz, int C, __nv_bfloat16* __restrict__ out, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int C8 = C / 8;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)gx * gy * gz * C8) return;
  const int c8 = (int)(idx % C8);
  const int64_t v = idx / C8;
  int x, y, z;
  grid_coords(v, gx, gy, x, y, z);
  const int cx = (gx + 1) / 2, cy = (gy + 1) / 2;
  const uint4 a = *reinterpret_cast<const uint4*>(
      coarse + ((int64_t)(x / 2) + cx * ((int64_t)(y / 2) + (int64_t)cy * (z / 2))) * C + 8 * c8);
  const uint4 b = *reinterpret_cast<const uint4*>(skip + v * C + 8 * c8);
  const __nv_bfloat16* pa = reinterpret_cast<const __nv_bfloat16*>(&a);
  const __nv_bfloat16* pb = reinterpret_cast<const __nv_bfloat16*>(&b);
  __align__(16) __nv_bfloat16 o8[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) o8[k] = __float2bfloat16(__bfloat162float(pa[k]) + __bfloat162float(pb[k]));
  *reinterpret_cast<uint4*>(out + v * C + 8 * c8) = *reinterpret_cast<const uint4*>(o8);
}
// dcoarse[c] = sum of dfine over c's children
__global__ void k_up_bwd(const __nv_bfloat16* __restrict__ dfine, int gx, int gy, int gz, int C,
                         __nv_bfloat16* __restrict__ dcoarse) {
  const int cx = (gx + 1) / 2, cy = (gy + 1) / 2, cz = (gz + 1) / 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)cx * cy * cz * C) return;
  const int c = (int)(idx % C);
  int x, y, z;
  grid_coords(idx / C, cx, cy, x, y, z);
  float s = 0.f;
  for (int o = 0; o < 8; ++o) {
    const int fx = 2 * x + (o & 1), fy = 2 * y + ((o >> 1) & 1), fz = 2 * z + (o >> 2);
    if (fx < gx && fy < gy && fz < gz) s += __bfloat162float(dfine[((int64_t)fx + gx * ((int64_t)fy + (int64_t)gy * fz)) * C + c]);
  }
  dcoarse[idx] = __float2bfloat16(s);
}
// dy *= (y > 0)
__global__ void k_relu_bwd(__nv_bfloat16* __restrict__ dy, const __nv_bfloat16* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16(0.f);
}
// db[co] (+)= sum_v dy[v][co]: one block per channel, fixed order.
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, int64_t V, int C, float* __restrict__ db, int acc) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int64_t v = threadIdx.x; v < V; v += 256) s += __bfloat162float(dy[v * C + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = acc ? db[c] + red[0] : red[0];
}

// ------------------------------------------------------------ edges <-> grid
// slot of every edge: low node * 7 + class; -1 when the edge is not a lattice step.
__global__ void k_edge_slots(const int32_t* __restrict__ edges, int64_t E, int gx, int gy, int gz,
                             int32_t* __restrict__ slot, int* __restrict__ bad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int64_t lo = edges[2 * e], hi = edges[2 * e + 1];
  int x0, y0, z0, x1, y1, z1;
  grid_coords(lo, gx, gy, x0, y0, z0);
  grid_coords(hi, gx, gy, x1, y1, z1);
  const int dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
  int cls = -1;
  if (dx == 1 && dy == 0 && dz == 0) cls = 0;
  else if (dx == 0 && dy == 1 && dz == 0) cls = 1;
  else if (dx == 0 && dy == 0 && dz == 1) cls = 2;
  else if (dx == 1 && dy == 1 && dz == 0) cls = 3;
  else if (dx == 1 && dy == 0 && dz == 1) cls = 4;
  else if (dx == 0 && dy == 1 && dz == 1) cls = 5;
  else if (dx == 1 && dy == 1 && dz == 1) cls = 6;
  if (cls < 0 || hi >= (int64_t)gx * gy * gz) {
    atomicOr(bad, 1);
    slot[e] = -1;
  } else {
    slot[e] = (int32_t)(lo * 7 + cls);
  }
}
// Model features at every node: log10(sigma / sigma_p) and log10(w mu0 sigma h^2) of the cell
// whose lowest corner is the node (the last node layer repeats its neighbour's cell).
__global__ void k_node_features(const double* __restrict__ sigma, int nx, int ny, int nz, double sigma_p,
                                double wmu0h2, float* __restrict__ feat) {
  const int gx = nx + 1, gy = ny + 1, gz = nz + 1;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= (int64_t)gx * gy * gz) return;
  int x, y, z;
  grid_coords(v, gx, gy, x, y, z);
  const int cxi = min(x, nx - 1), cyi = min(y, ny - 1), czi = min(z, nz - 1);
  const int64_t cell = cxi + (int64_t)nx * (cyi + (int64_t)ny * czi);
  double s = 0.0;  // the cell's six tets share one sigma in the synthetic models; average them
  for (int p = 0; p < 6; ++p) s += sigma[6 * cell + p];
  s /= 6.0;
  feat[2 * v] = (float)log10(s / sigma_p);
  feat[2 * v + 1] = (float)log10(wmu0h2 * s);
}
// Lattice step from the low to the high node of each edge class.
__constant__ int kStep[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

// Edge of every slot, and the slot's unit tangent t / |t| with 1 / |t| (the edge's true geometry,
// so jittered lattices are handled exactly).
__global__ void k_slot_geometry(const int32_t* __restrict__ edges, const int32_t* __restrict__ slot, int64_t E,
                                const double* __restrict__ nodes, int32_t* __restrict__ slot_edge,
                                float4* __restrict__ tang) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t sl = slot[e];
  if (sl < 0) return;
  const int64_t lo = edges[2 * e], hi = edges[2 * e + 1];
  const double tx = nodes[3 * hi] - nodes[3 * lo], ty = nodes[3 * hi + 1] - nodes[3 * lo + 1],
               tz = nodes[3 * hi + 2] - nodes[3 * lo + 2];
  const double l = sqrt(tx * tx + ty * ty + tz * tz);
  slot_edge[sl] = (int32_t)e;
  tang[sl] = make_float4((float)(tx / l), (float)(ty / l), (float)(tz / l), (float)(1.0 / l));
}

__device__ inline bool interior(int x, int y, int z, int gx, int gy, int gz) {
  return x >= 1 && y >= 1 && z >= 1 && x <= gx - 2 && y <= gy - 2 && z <= gz - 2;
}

// The 14 edge slots at node v with their coefficients in G (g) and Pi (p = t / (2 |t|)): slot 2c
// is the edge leaving v in lattice direction c (v its low node, g = -1/|t|), slot 2c + 1 the edge
// arriving from v - step_c.  A slot without an edge has e = -1 and zero coefficients (its tangent
// entry is zero), so every array index is a compile-time constant once the loops are unrolled
// and the slots stay in registers; the 14 edge ids and tangents are independent loads.
struct Incident {
  int32_t e[14];
  float g[14];
  float3 p[14];
};
__device__ inline void incident_edges(int64_t v, int x, int y, int z, int gx, int gy, const int32_t* slot_edge,
                                      const float4* tang, Incident& I) {
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const int64_t so = v * 7 + c;
    const float4 t = tang[so];
    I.e[2 * c] = slot_edge[so];
    I.g[2 * c] = -t.w;
    I.p[2 * c] = make_float3(0.5f * t.x, 0.5f * t.y, 0.5f * t.z);
    const int ux = x - kStep[c][0], uy = y - kStep[c][1], uz = z - kStep[c][2];
    int32_t ei = -1;
    float4 ti = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ux >= 0 && uy >= 0 && uz >= 0) {
      const int64_t si = ((int64_t)ux + (int64_t)gx * ((int64_t)uy + (int64_t)gy * uz)) * 7 + c;
      ei = slot_edge[si];
      ti = tang[si];
    }
    I.e[2 * c + 1] = ei;
    I.g[2 * c + 1] = ti.w;
    I.p[2 * c + 1] = make_float3(0.5f * ti.x, 0.5f * ti.y, 0.5f * ti.z);
  }
}

// Per-node scales (sg, sp_x, sp_y, sp_z) = |diag|^{-1/2} of G^T A G and Pi^T A Pi, from the
// assembled A (complex128 CSR, ascending columns): diag_v = sum over incident edge pairs (e, f) of
// coef_e coef_f A_ef (entries outside the pattern are zero).  Zero on boundary nodes.
__global__ void k_hx_diag(const int32_t* __restrict__ slot_edge, const float4* __restrict__ tang,
                          const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double2* __restrict__ val, int gx, int gy, int gz, float4* __restrict__ aux) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= (int64_t)gx * gy * gz) return;
  int x, y, z;
  grid_coords(v, gx, gy, x, y, z);
  if (!interior(x, y, z, gx, gy, gz)) {
    aux[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  Incident I;
  incident_edges(v, x, y, z, gx, gy, slot_edge, tang, I);
  double2 dg = make_double2(0.0, 0.0), dp[3] = {dg, dg, dg};
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    if (I.e[i] < 0) continue;
    const int64_t r0 = rp[I.e[i]], r1 = rp[I.e[i] + 1];
#pragma unroll
    for (int j = 0; j < 14; ++j) {
      if (I.e[j] < 0) continue;
      int64_t lo = r0, hi = r1;  // binary search for column e_j in row e_i
      const int32_t want = I.e[j];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < want) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= r1 || col[lo] != want) continue;
      const double2 a = val[lo];
      dg = cadd(dg, cscale(a, (double)I.g[i] * I.g[j]));
      dp[0] = cadd(dp[0], cscale(a, (double)I.p[i].x * I.p[j].x));
      dp[1] = cadd(dp[1], cscale(a, (double)I.p[i].y * I.p[j].y));
      dp[2] = cadd(dp[2], cscale(a, (double)I.p[i].z * I.p[j].z));
    }
  }
  auto inv_sqrt_abs = [](double2 d) -> float {
    const double m = sqrt(d.x * d.x + d.y * d.y);
    return m > 0.0 ? (float)(1.0 / sqrt(m)) : 0.f;
  };
  aux[v] = make_float4(inv_sqrt_abs(dg), inv_sqrt_abs(dp[0]), inv_sqrt_abs(dp[1]), inv_sqrt_abs(dp[2]));
}

// Node fields of an edge vector r: [sg Re G^T r, sg Im G^T r, sp Re Pi^T r (x, y, z), sp Im Pi^T r
// (x, y, z)] per node, and per-block sums of their squares (FP64) for the scale s.  The sums run
// in the vector's own precision (FP32 for complex64: FP64 arithmetic per node would cost more
// than the node's memory traffic on this GPU).
template <typename T>
__global__ void __launch_bounds__(256) k_hx_in(const T* __restrict__ r, const int32_t* __restrict__ slot_edge,
                                               const float4* __restrict__ tang, const float4* __restrict__ aux,
                                               int gx, int gy, int gz, float* __restrict__ out,
                                               double* __restrict__ part, const int* __restrict__ stop,
                                               int64_t stride, int64_t off) {
  if (stop && *stop) return;
  using R = typename real_of<T>::type;
  __shared__ double red[8];
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float ss = 0.f;
  if (v < (int64_t)gx * gy * gz) {
    const float4 a = aux[v];
    float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (a.x > 0.f) {
      int x, y, z;
      grid_coords(v, gx, gy, x, y, z);
      Incident I;
      incident_edges(v, x, y, z, gx, gy, slot_edge, tang, I);
      T rv[14];
#pragma unroll
      for (int k = 0; k < 14; ++k) rv[k] = I.e[k] >= 0 ? r[(int64_t)I.e[k] * stride + off] : T{0, 0};
      R gr = 0, gi = 0, pr[3] = {0, 0, 0}, pi[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < 14; ++k) {
        const T re = rv[k];
        const R xr = (R)re.x, xi = (R)re.y;
        gr += (R)I.g[k] * xr;
        gi += (R)I.g[k] * xi;
        pr[0] += (R)I.p[k].x * xr;
        pi[0] += (R)I.p[k].x * xi;
        pr[1] += (R)I.p[k].y * xr;
        pi[1] += (R)I.p[k].y * xi;
        pr[2] += (R)I.p[k].z * xr;
        pi[2] += (R)I.p[k].z * xi;
      }
      o[0] = (float)(a.x * gr);
      o[1] = (float)(a.x * gi);
      o[2] = (float)(a.y * pr[0]);
      o[3] = (float)(a.z * pr[1]);
      o[4] = (float)(a.w * pr[2]);
      o[5] = (float)(a.y * pi[0]);
      o[6] = (float)(a.z * pi[1]);
      o[7] = (float)(a.w * pi[2]);
#pragma unroll
      for (int k = 0; k < 8; ++k) ss += o[k] * o[k];
    }
    reinterpret_cast<float4*>(out)[2 * v] = make_float4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<float4*>(out)[2 * v + 1] = make_float4(o[4], o[5], o[6], o[7]);
  }
  double sd = ss;
  for (int off = 16; off > 0; off >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
// s = sqrt(sum / (4 n_interior)) (1 when the sum is zero) -> scal[0] = 1 / s, scal[1] = s.
__global__ void k_hx_scale(const double* __restrict__ part, int nb, int64_t n_interior, float* __restrict__ scal, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) a += part[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double sc = n_interior > 0 ? sqrt(red[0] / (4.0 * (double)n_interior)) : 0.0;
    if (!(sc > 0.0) || !isfinite(sc)) sc = 1.0;
    scal[0] = (float)(1.0 / sc);
    scal[1] = (float)sc;
  }
}
__global__ void k_hx_pack(const float* __restrict__ nodes8, const float* __restrict__ feat, int64_t V,
                          const float* __restrict__ scal, __nv_bfloat16* __restrict__ x, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float is = scal[0];
  const float4 a = reinterpret_cast<const float4*>(nodes8)[2 * v], b = reinterpret_cast<const float4*>(nodes8)[2 * v + 1];
  const float2 f = reinterpret_cast<const float2*>(feat)[v];
  __align__(16) __nv_bfloat16 o[16];
  const float in[10] = {a.x * is, a.y * is, a.z * is, a.w * is, b.x * is, b.y * is, b.z * is, b.w * is, f.x, f.y};
#pragma unroll
  for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(c < 10 ? in[c] : 0.f);
  reinterpret_cast<uint4*>(x)[2 * v] = reinterpret_cast<const uint4*>(o)[0];
  reinterpret_cast<uint4*>(x)[2 * v + 1] = reinterpret_cast<const uint4*>(o)[1];
}
// z_e = D^{-1} r_e + (G phi + Pi w)_e (XS) or r_e + D_e (G phi + Pi w)_e, from the network output y
// [V][16] (FP32): phi = s sg (y0 + i y1), w_k = s sp_k (y_{2+k} + i y_{5+k}) at the edge's nodes.
// Arithmetic, and the diagonal D, in the vector's precision (FP32 for complex64).
template <typename T, bool XS>
__global__ void k_hx_out(const T* __restrict__ r, const int32_t* __restrict__ slot, int64_t E,
                         const float* __restrict__ y, const float4* __restrict__ aux, const float4* __restrict__ tang,
                         const float* __restrict__ scal, const T* __restrict__ diag, int gx, int gy,
                         T* __restrict__ z, const int* __restrict__ stop, int64_t stride, int64_t off,
                         const int32_t* __restrict__ zrow) {
  if (stop && *stop) return;
  using R = typename real_of<T>::type;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t sl = slot[e];
  const int64_t er = zrow ? (int64_t)zrow[e] : e;  // zrow: r and z in the SELL-32 row order
  const T re = r[er * stride + off];
  R cr = 0, ci = 0;
  if (sl >= 0) {
    const int64_t lo = sl / 7;
    const int c = sl - (int)(lo * 7);
    const int64_t hi = lo + kStep[c][0] + (int64_t)gx * (kStep[c][1] + (int64_t)gy * kStep[c][2]);
    const float4 t = tang[sl];
    const R s = scal[1];
    const float4 al = aux[lo], ah = aux[hi];
    const float4* yl = reinterpret_cast<const float4*>(y + lo * 16);
    const float4* yh = reinterpret_cast<const float4*>(y + hi * 16);
    const float4 l0 = yl[0], l1 = yl[1], h0 = yh[0], h1 = yh[1];
    // G phi: (phi_hi - phi_lo) / |t|
    cr = (R)t.w * s * ((R)ah.x * h0.x - (R)al.x * l0.x);
    ci = (R)t.w * s * ((R)ah.x * h0.y - (R)al.x * l0.y);
    // Pi w: (w_lo + w_hi) . t / (2 |t|); channels: Re x,y,z = 2,3,4; Im x,y,z = 5,6,7
    const R hs = (R)0.5 * s;
    cr += hs * ((R)t.x * ((R)al.y * l0.z + (R)ah.y * h0.z) + (R)t.y * ((R)al.z * l0.w + (R)ah.z * h0.w) +
                (R)t.z * ((R)al.w * l1.x + (R)ah.w * h1.x));
    ci += hs * ((R)t.x * ((R)al.y * l1.y + (R)ah.y * h1.y) + (R)t.y * ((R)al.z * l1.z + (R)ah.z * h1.z) +
                (R)t.z * ((R)al.w * l1.w + (R)ah.w * h1.w));
  }
  const T dd = diag[e];
  const R dr = dd.x, di = dd.y;
  const R rr = (R)re.x, ri = (R)re.y;
  T o;
  if (XS) {  // r / d + corr
    const R den = dr * dr + di * di;
    o.x = (rr * dr + ri * di) / den + cr;
    o.y = (ri * dr - rr * di) / den + ci;
  } else {  // r + d corr
    o.x = rr + (dr * cr - di * ci);
    o.y = ri + (dr * ci + di * cr);
  }
  z[er * stride + off] = o;
}
// Slot si -> the SELL-32 row of its edge, inv[slot_edge[si]] (-1 for a slot without an edge).
__global__ void k_renumber_slots(const int32_t* __restrict__ slot_edge, int64_t n_slots, const int32_t* __restrict__ inv,
                                 int32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n_slots) out[i] = slot_edge[i] >= 0 ? inv[slot_edge[i]] : -1;
}
// The diagonal of A in single precision, for the complex64 application.
__global__ void k_diag_f32(const double2* __restrict__ d, int64_t n, float2* __restrict__ o) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) o[i] = make_float2((float)d[i].x, (float)d[i].y);
}
// Gradient of the loss with respect to the network output: with gzp = Ahat^H gw and
// g = conj(D) gzp = A^H gw (the gradient at z in the unscaled variables),
// dy[v] = s [sg Re G^T g, sg Im G^T g, sp Re Pi^T g (x, y, z), sp Im Pi^T g (x, y, z), 0 ...].
__global__ void k_hx_dy(const double2* __restrict__ gzp, const double2* __restrict__ diag,
                        const int32_t* __restrict__ slot_edge, const float4* __restrict__ tang,
                        const float4* __restrict__ aux, const float* __restrict__ scal, int gx, int gy, int gz,
                        __nv_bfloat16* __restrict__ dy) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= (int64_t)gx * gy * gz) return;
  const float4 a = aux[v];
  float o[16];
  for (int k = 0; k < 16; ++k) o[k] = 0.f;
  if (a.x > 0.f) {
    int x, y, z;
    grid_coords(v, gx, gy, x, y, z);
    Incident I;
    incident_edges(v, x, y, z, gx, gy, slot_edge, tang, I);
    double gr = 0.0, gi = 0.0, pr[3] = {0.0, 0.0, 0.0}, pi[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      if (I.e[k] < 0) continue;
      const double2 g = cconjmul(diag[I.e[k]], gzp[I.e[k]]);
      gr += I.g[k] * g.x;
      gi += I.g[k] * g.y;
      pr[0] += I.p[k].x * g.x;
      pi[0] += I.p[k].x * g.y;
      pr[1] += I.p[k].y * g.x;
      pi[1] += I.p[k].y * g.y;
      pr[2] += I.p[k].z * g.x;
      pi[2] += I.p[k].z * g.y;
    }
    const double s = scal[1];
    o[0] = (float)(s * a.x * gr);
    o[1] = (float)(s * a.x * gi);
    o[2] = (float)(s * a.y * pr[0]);
    o[3] = (float)(s * a.z * pr[1]);
    o[4] = (float)(s * a.w * pr[2]);
    o[5] = (float)(s * a.y * pi[0]);
    o[6] = (float)(s * a.z * pi[1]);
    o[7] = (float)(s * a.w * pi[2]);
  }
  for (int k = 0; k < 16; ++k) dy[v * 16 + k] = __float2bfloat16(o[k]);
}
// Adam (Kingma & Ba 2015) on FP32 master weights.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, float gscale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] * gscale;
  g[i] = gi;  // keep the mean gradient readable
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// r = b - A x (one thread per row, FP64) and du = D (x* - x).
__global__ void k_res_err(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double2* __restrict__ val, const double2* __restrict__ b, const double2* __restrict__ d,
                          const double2* __restrict__ x, const double2* __restrict__ xs, int64_t n,
                          double2* __restrict__ r, double2* __restrict__ du) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = b[i];
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = csub(acc, cmul(val[p], x[col[p]]));
  r[i] = acc;
  du[i] = cmul(d[i], csub(xs[i], x[i]));
}

// w = Ahat z = A D^{-1} z (complex128, one thread per row).
__global__ void k_ahat_apply(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double2* __restrict__ val, const double2* __restrict__ d,
                             const double2* __restrict__ z, int64_t n, double2* __restrict__ w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    const int32_t j = col[p];
    acc = cadd(acc, cmul(val[p], cdiv(z[j], d[j])));
  }
  w[i] = acc;
}
// g = Ahat^H y = conj(D)^{-1} conj(A) y (A complex symmetric).
__global__ void k_ahat_adjoint(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double2* __restrict__ val, const double2* __restrict__ d,
                               const double2* __restrict__ y, int64_t n, double2* __restrict__ g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = cadd(acc, cconjmul(val[p], y[col[p]]));
  g[i] = cdiv(acc, make_double2(d[i].x, -d[i].y));
}
// dv = (<r, w>, |w|^2, |r|^2) in FP64 (one block), and loss += 1 - |<r,w>|^2 / (|w|^2 |r|^2).
__global__ void k_angle_dots(const double2* __restrict__ r, const double2* __restrict__ w, int64_t n,
                             double* __restrict__ dv, double* __restrict__ loss) {
  __shared__ double red[4][1024];
  double ax = 0.0, ay = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 ri = r[i], wi = w[i];
    ax += ri.x * wi.x + ri.y * wi.y;
    ay += ri.x * wi.y - ri.y * wi.x;
    b += wi.x * wi.x + wi.y * wi.y;
    c += ri.x * ri.x + ri.y * ri.y;
  }
  red[0][threadIdx.x] = ax;
  red[1][threadIdx.x] = ay;
  red[2][threadIdx.x] = b;
  red[3][threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) dv[q] = red[q][0];
    const double bc = red[2][0] * red[3][0];
    *loss += bc > 0.0 ? 1.0 - (red[0][0] * red[0][0] + red[1][0] * red[1][0]) / bc : 1.0;
  }
}
// dL/dw (real and imaginary parts as one complex number): -2 (a r / (c b) - |a|^2 w / (c b^2)).
__global__ void k_angle_gw(const double2* __restrict__ r, const double2* __restrict__ w, int64_t n,
                           const double* __restrict__ dv, double2* __restrict__ gw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 a = make_double2(dv[0], dv[1]);
  const double b = dv[2], c = dv[3];
  if (!(b > 0.0 && c > 0.0)) {
    gw[i] = make_double2(0.0, 0.0);
    return;
  }
  const double a2 = a.x * a.x + a.y * a.y;
  const double2 t1 = cscale(cmul(a, r[i]), 1.0 / (c * b));
  const double2 t2 = cscale(w[i], a2 / (c * b * b));
  gw[i] = cscale(csub(t1, t2), -2.0);
}

unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------ host side
Status conv3d_attributes() {
  static bool done = false;
  if (done) return Status{};
#define PG_ATTR(CI, CO, NZ) \
  PG_CUDA(cudaFuncSetAttribute(k_conv3d<CI, CO, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                               conv_smem_launch(CI, CO, NZ)));
#define PG_ATTR_NZ(CI, CO) PG_ATTR(CI, CO, 1) PG_ATTR(CI, CO, 2) PG_ATTR(CI, CO, 4)
  PG_ATTR_NZ(16, 16)
  PG_ATTR_NZ(16, 32)
  PG_ATTR_NZ(32, 16)
  PG_ATTR_NZ(32, 32)
#undef PG_ATTR_NZ
#undef PG_ATTR
  done = true;
  return Status{};
}

Status conv3d(cudaStream_t s, int gx, int gy, int gz, int cin, int cout, const __nv_bfloat16* x,
              const __nv_bfloat16* w, const float* bias, bool relu, __nv_bfloat16* ybf, float* yf, int* err,
              const int* stop) {
  if ((cin != 16 && cin != 32) || (cout != 16 && cout != 32))
    return Status{PETGEM_ERR_UNSUPPORTED, "conv3d: channel counts must be 16 or 32"};
  if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)ybf | (uintptr_t)yf) & 15)
    return Status{PETGEM_ERR_INVALID_ARG, "conv3d: x, w and y must be 16-byte aligned"};
  PG_TRY(conv3d_attributes());
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    PG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  // planes per CTA: the most (fewer brick and weight loads per voxel) that still leave two CTAs per SM
  const int64_t txy = (int64_t)((gx + kBrickX - 1) / kBrickX) * ((gy + kBrickY - 1) / kBrickY);
  const int nz = txy * ((gz + 3) / 4) >= 2 * sms ? 4 : txy * ((gz + 1) / 2) >= 2 * sms ? 2 : 1;
  const unsigned grid = (unsigned)(txy * ((gz + nz - 1) / nz));
#define PG_CONV(CI, CO, NZ)                                                                                      \
  if (cin == CI && cout == CO && nz == NZ) {                                                                     \
    k_conv3d<CI, CO, NZ><<<grid, 128, conv_smem_launch(CI, CO, NZ), s>>>(x, w, bias, gx, gy, gz, relu ? 1 : 0, ybf, yf, err, \
                                                                   stop);                                       \
    PG_CUDA(cudaGetLastError());                                                                                 \
    return Status{};                                                                                             \
  }
#define PG_CONV_NZ(CI, CO) PG_CONV(CI, CO, 1) PG_CONV(CI, CO, 2) PG_CONV(CI, CO, 4)
  PG_CONV_NZ(16, 16)
  PG_CONV_NZ(16, 32)
  PG_CONV_NZ(32, 16)
  PG_CONV_NZ(32, 32)
#undef PG_CONV_NZ
#undef PG_CONV
  return Status{PETGEM_ERR_UNSUPPORTED, "conv3d: channel counts must be 16 or 32"};
}

Status pack_conv_weights(cudaStream_t s, const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wc) {
  k_pack_conv_weights_bf16<<<nb(27 * cin * cout), 256, 0, s>>>(w, cin, cout, wc);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status conv3d_wgrad(cudaStream_t s, int gx, int gy, int gz, int cin, int cout, const __nv_bfloat16* x,
                    const __nv_bfloat16* dy, float* part, int splits, float* dw, bool accumulate, int* err) {
  const dim3 grid((27 * cin + kConvRows - 1) / kConvRows, splits);
#define PG_WG(CI, CO)                                                                                  \
  if (cin == CI && cout == CO) {                                                                       \
    k_conv3d_wgrad<CI, CO><<<grid, 128, 0, s>>>(x, dy, gx, gy, gz, part, err);                         \
    PG_CUDA(cudaGetLastError());                                                                       \
    k_wgrad_reduce<<<nb(27 * cin * cout), 256, 0, s>>>(part, splits, cin, cout, dw, accumulate ? 1 : 0); \
    PG_CUDA(cudaGetLastError());                                                                       \
    return Status{};                                                                                   \
  }
  PG_WG(16, 16)
  PG_WG(16, 32)
  PG_WG(32, 16)
  PG_WG(32, 32)
#undef PG_WG
  return Status{PETGEM_ERR_UNSUPPORTED, "conv3d_wgrad: channel counts must be 16 or 32"};
}

int wgrad_splits(int64_t V) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, (V + 4095) / 4096)); }

Status Net::init(petgem_ctx* c, int nx_, int ny_, int nz_) {
  ctx = c;
  nx = nx_;
  ny = ny_;
  nz = nz_;
  g[0][0] = nx + 1;
  g[0][1] = ny + 1;
  g[0][2] = nz + 1;
  nlev = net_levels(g[0][0], g[0][1], g[0][2]);
  if (nlev > kMaxLevels) return Status{PETGEM_ERR_UNSUPPORTED, "learned network: grid too large"};
  for (int l = 1; l < nlev; ++l)
    for (int a = 0; a < 3; ++a) g[l][a] = (g[l - 1][a] + 1) / 2;
  for (int l = 0; l < nlev; ++l) V[l] = (int64_t)g[l][0] * g[l][1] * g[l][2];
  const int spec[7][3] = {{16, 16, 1}, {16, 32, 1}, {32, 32, 1}, {32, 32, 1},
                          {32, 32, 1}, {32, 16, 1}, {16, 16, 0}};  // cin, cout, relu
  n_params = 0;
  for (int i = 0; i < 7; ++i) {
    L[i].cin = spec[i][0];
    L[i].cout = spec[i][1];
    L[i].relu = spec[i][2];
    L[i].w_off = n_params;
    n_params += 27 * L[i].cin * L[i].cout;
    L[i].b_off = n_params;
    n_params += L[i].cout;
  }
  PG_TRY(params.reserve(n_params * sizeof(float)));
  PG_TRY(grads.reserve(n_params * sizeof(float)));
  PG_TRY(adam_m.reserve(n_params * sizeof(float)));
  PG_TRY(adam_v.reserve(n_params * sizeof(float)));
  PG_TRY(wb.reserve(n_params * sizeof(__nv_bfloat16)));
  PG_TRY(wd.reserve(n_params * sizeof(__nv_bfloat16)));
  cudaStream_t s = c->stream;
  PG_CUDA(cudaMemsetAsync(params.ptr, 0, n_params * sizeof(float), s));
  PG_CUDA(cudaMemsetAsync(adam_m.ptr, 0, n_params * sizeof(float), s));
  PG_CUDA(cudaMemsetAsync(adam_v.ptr, 0, n_params * sizeof(float), s));
  adam_t = 0;
  // activations and their gradients (BF16) by level
  auto act = [&](DevBuf& b, int lvl, int ch) { return b.reserve((size_t)V[lvl] * ch * sizeof(__nv_bfloat16) + 64); };
  for (int l = 0; l < nlev; ++l) {
    PG_TRY(act(q[l], l, ch_q(l)));
    PG_TRY(act(e[l], l, ch_e(l)));
    PG_TRY(act(dd[l], l, l == 0 ? 16 : (l == nlev - 1 ? ch_e(l) : ch_d(l))));
    if (l < nlev - 1) {
      PG_TRY(act(sk[l], l, ch_e(l)));
      PG_TRY(act(ds[l], l, ch_e(l)));
      if (l > 0) PG_TRY(act(d[l], l, ch_d(l)));
    }
    if (l > 0) PG_TRY(act(dq[l], l, ch_q(l)));
  }
  PG_TRY(y.reserve((size_t)V[0] * 16 * sizeof(float)));
  PG_TRY(feat.reserve((size_t)V[0] * 2 * sizeof(float)));
  PG_TRY(scal.reserve(16 * sizeof(float)));
  PG_TRY(loss_acc.reserve(sizeof(double)));
  PG_TRY(err.reserve(sizeof(int)));
  PG_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
  PG_TRY(zbias.reserve(32 * sizeof(float)));
  PG_CUDA(cudaMemsetAsync(zbias.ptr, 0, 32 * sizeof(float), s));
  const int splits = wgrad_splits(V[0]);
  PG_TRY(wpart.reserve((size_t)splits * 27 * 32 * 32 * sizeof(float)));
  PG_CUDA(cudaMemsetAsync(feat.ptr, 0, (size_t)V[0] * 2 * sizeof(float), s));
  geom_version = -1;
  aux_version = -1;
  ++alloc_gen;
  PG_TRY(conv3d_attributes());
  ready = true;
  return Status{};
}

// Forward and input-gradient weights of every layer as the convolution kernel's shared-memory
// image (BF16).
Status Net::pack_weights(cudaStream_t s) {
  for (int i = 0; i < 7; ++i) {
    const float* w = params.as<float>() + L[i].w_off;
    const unsigned g = nb(27 * L[i].cin * L[i].cout);
    k_pack_conv_weights<<<g, 256, 0, s>>>(w, L[i].cin, L[i].cout, 0, wb.as<__nv_bfloat16>() + L[i].w_off);
    k_pack_conv_weights<<<g, 256, 0, s>>>(w, L[i].cin, L[i].cout, 1, wd.as<__nv_bfloat16>() + L[i].w_off);
  }
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status Net::conv(cudaStream_t s, int i, int lvl, const __nv_bfloat16* in, __nv_bfloat16* out, float* outf,
                 const int* stop) {
  const int* gg = g[lvl];
  // timed (when profiling) with its floating-point operations in place of bytes
  const double flops = 2.0 * 27.0 * L[i].cin * L[i].cout * (double)gg[0] * gg[1] * gg[2];
  KernelTimer kt(ctx, "conv3d_fwd", flops);
  return conv3d(s, gg[0], gg[1], gg[2], L[i].cin, L[i].cout, in, wb.as<__nv_bfloat16>() + L[i].w_off,
                params.as<float>() + L[i].b_off, L[i].relu != 0, out, outf, err.as<int>(), stop);
}

// Input grid q[0] (BF16 [V0][16]) -> y (FP32 [V0][16]): encoder down to the coarsest level, then
// decoder levels that add the upsampled coarse output to the encoder's.
Status Net::forward(cudaStream_t s, const int* stop) {
  using B = __nv_bfloat16;
  for (int l = 0; l < nlev; ++l) {
    if (l > 0)
      k_pool<<<nb(V[l] * ch_e(l - 1) / 8), 256, 0, s>>>(e[l - 1].as<B>(), g[l - 1][0], g[l - 1][1], g[l - 1][2],
                                                        ch_e(l - 1), q[l].as<B>(), stop);
    PG_TRY(conv(s, enc(l), l, q[l].as<B>(), e[l].as<B>(), nullptr, stop));
  }
  for (int l = nlev - 2; l >= 0; --l) {
    const B* coarse = (l + 1 == nlev - 1) ? e[l + 1].as<B>() : d[l + 1].as<B>();
    k_up_add<<<nb(V[l] * ch_e(l) / 8), 256, 0, s>>>(coarse, e[l].as<B>(), g[l][0], g[l][1], g[l][2], ch_e(l),
                                                    sk[l].as<B>(), stop);
    if (l == 0)
      PG_TRY(conv(s, dec(0), 0, sk[0].as<B>(), nullptr, y.as<float>(), stop));
    else
      PG_TRY(conv(s, dec(l), l, sk[l].as<B>(), d[l].as<B>(), nullptr, stop));
  }
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status Net::dgrad(cudaStream_t s, int i, int lvl, const __nv_bfloat16* dout, __nv_bfloat16* din) {
  const int* gg = g[lvl];  // the input gradient has no bias term: zbias is all zeros
  return conv3d(s, gg[0], gg[1], gg[2], L[i].cout, L[i].cin, dout, wd.as<__nv_bfloat16>() + L[i].w_off,
                zbias.as<float>(), false, din, nullptr, err.as<int>());
}

Status Net::wgrad(cudaStream_t s, int i, int lvl, const __nv_bfloat16* in, const __nv_bfloat16* dout, bool acc) {
  const int* gg = g[lvl];
  const int64_t Vl = (int64_t)gg[0] * gg[1] * gg[2];
  PG_TRY(conv3d_wgrad(s, gg[0], gg[1], gg[2], L[i].cin, L[i].cout, in, dout, wpart.as<float>(), wgrad_splits(Vl),
                      grads.as<float>() + L[i].w_off, acc, err.as<int>()));
  k_bias_grad<<<L[i].cout, 256, 0, s>>>(dout, Vl, L[i].cout, grads.as<float>() + L[i].b_off, acc ? 1 : 0);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

// dd[0] (BF16 [V0][16], the gradient at y) -> parameter gradients (accumulated when acc; a
// layer that acts on several levels collects every level's gradient).
Status Net::backward(cudaStream_t s, bool acc) {
  using B = __nv_bfloat16;
  bool touched[7] = {false, false, false, false, false, false, false};
  auto W = [&](int i, int lvl, const B* in, const B* dout) -> Status {
    const bool a = acc || touched[i];
    touched[i] = true;
    return wgrad(s, i, lvl, in, dout, a);
  };
  // decoder, finest level first: ds[l] is the gradient at sk[l], and (skip path) at e[l]
  for (int l = 0; l <= nlev - 2; ++l) {
    const int ci = ch_e(l);
    if (l > 0) k_relu_bwd<<<nb(V[l] * ch_d(l)), 256, 0, s>>>(dd[l].as<B>(), d[l].as<B>(), V[l] * ch_d(l));
    PG_TRY(W(dec(l), l, sk[l].as<B>(), dd[l].as<B>()));
    PG_TRY(dgrad(s, dec(l), l, dd[l].as<B>(), ds[l].as<B>()));
    k_up_bwd<<<nb(V[l + 1] * ci), 256, 0, s>>>(ds[l].as<B>(), g[l][0], g[l][1], g[l][2], ci, dd[l + 1].as<B>());
  }
  // encoder, coarsest level first: the gradient at e[l] is dd[nlev-1] (bottom) or ds[l]
  for (int l = nlev - 1; l >= 0; --l) {
    B* de = l == nlev - 1 ? dd[l].as<B>() : ds[l].as<B>();
    k_relu_bwd<<<nb(V[l] * ch_e(l)), 256, 0, s>>>(de, e[l].as<B>(), V[l] * ch_e(l));
    PG_TRY(W(enc(l), l, q[l].as<B>(), de));
    if (l > 0) {
      PG_TRY(dgrad(s, enc(l), l, de, dq[l].as<B>()));
      B* de_below = l - 1 == nlev - 1 ? dd[l - 1].as<B>() : ds[l - 1].as<B>();
      k_pool_bwd_add<<<nb(V[l - 1] * ch_q(l)), 256, 0, s>>>(dq[l].as<B>(), g[l - 1][0], g[l - 1][1], g[l - 1][2],
                                                             ch_q(l), de_below);
    }
  }
  PG_CUDA(cudaGetLastError());
  return Status{};
}

// Slot map and tangents of the current mesh, and the auxiliary scales of the current assembly.
Status Net::prepare_aux(petgem_ctx* c) {
  cudaStream_t s = c->stream;
  const int gx = g[0][0], gy = g[0][1], gz = g[0][2];
  // captured graphs hold these buffers' addresses: the generation moves only when one of them
  // moved (a new mesh or assembly of the same sizes keeps the graphs)
  const void* before[6] = {slot_edge.ptr, tang.ptr, aux.ptr, nodes8.ptr, npart.ptr, diag32.ptr};
  if (geom_version != c->mesh_version) {
    PG_TRY(slot_edge.reserve((size_t)V[0] * 7 * sizeof(int32_t)));
    PG_TRY(tang.reserve((size_t)V[0] * 7 * sizeof(float4)));
    PG_CUDA(cudaMemsetAsync(slot_edge.ptr, 0xff, (size_t)V[0] * 7 * sizeof(int32_t), s));  // -1: no edge
    PG_CUDA(cudaMemsetAsync(tang.ptr, 0, (size_t)V[0] * 7 * sizeof(float4), s));
    k_slot_geometry<<<nb(c->n_edges), 256, 0, s>>>(c->edges.as<int32_t>(), c->slots.as<int32_t>(), c->n_edges,
                                                    c->nodes.as<double>(), slot_edge.as<int32_t>(), tang.as<float4>());
    PG_CUDA(cudaGetLastError());
    geom_version = c->mesh_version;
    aux_version = -1;
  }
  if (aux_version != c->assembly_version) {
    PG_TRY(aux.reserve((size_t)V[0] * sizeof(float4)));
    PG_TRY(nodes8.reserve((size_t)V[0] * 8 * sizeof(float)));
    PG_TRY(npart.reserve((size_t)nb(V[0]) * sizeof(double)));
    k_hx_diag<<<nb(V[0]), 256, 0, s>>>(slot_edge.as<int32_t>(), tang.as<float4>(), c->row_ptr.as<int64_t>(),
                                       c->col.as<int32_t>(), c->val.as<double2>(), gx, gy, gz, aux.as<float4>());
    PG_TRY(diag32.reserve((size_t)c->n_edges * sizeof(float2)));
    k_diag_f32<<<nb(c->n_edges), 256, 0, s>>>(c->diag.as<double2>(), c->n_edges, diag32.as<float2>());
    PG_CUDA(cudaGetLastError());
    aux_version = c->assembly_version;
  }
  const void* after[6] = {slot_edge.ptr, tang.ptr, aux.ptr, nodes8.ptr, npart.ptr, diag32.ptr};
  for (int k = 0; k < 6; ++k)
    if (before[k] != after[k]) {
      ++alloc_gen;
      break;
    }
  return Status{};
}

// Network input x0 from an edge vector r (a residual): the gathered, scaled node fields, the scale
// s in scal[0..1] (1 / s, s), the two features.
template <typename T>
Status Net::load_input(cudaStream_t s, const T* r, int64_t E, const int* stop, int64_t stride, int64_t off,
                       bool renum) {
  (void)E;
  const int gx = g[0][0], gy = g[0][1], gz = g[0][2];
  const unsigned blocks = nb(V[0]);
  // algorithmic bytes: every edge value read twice (once from each end node), each node's 14
  // slots (edge id and tangent) read once, 32 B of node output written
  {
    KernelTimer kt(ctx, sizeof(T) == 8 ? "hx_in_c64" : "hx_in_c128",
                   2.0 * sizeof(T) * (double)ctx->n_edges + (double)V[0] * (14.0 * 20.0 + 32.0 + 16.0));
    k_hx_in<T><<<blocks, 256, 0, s>>>(r, (renum ? slot_edge_r : slot_edge).as<int32_t>(), tang.as<float4>(),
                                      aux.as<float4>(), gx, gy, gz,
                                      nodes8.as<float>(), npart.as<double>(), stop, stride, off);
  }
  const int64_t n_in = (int64_t)std::max(gx - 2, 0) * std::max(gy - 2, 0) * std::max(gz - 2, 0);
  k_hx_scale<<<1, 256, 0, s>>>(npart.as<double>(), (int)blocks, n_in, scal.as<float>(), stop);
  k_hx_pack<<<nb(V[0]), 256, 0, s>>>(nodes8.as<float>(), feat.as<float>(), V[0], scal.as<float>(),
                                     q[0].as<__nv_bfloat16>(), stop);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

template <typename T>
Status Net::apply(cudaStream_t s, const T* r, const int32_t* slot, int64_t E, T* z, bool xspace,
                  const int* stop, int64_t stride, int64_t off, bool renum) {
  // renum: the node-wise map gathers r through its slots' SELL-32 rows; the edge-wise map runs in
  // edge order, where an edge's node data are adjacent (measured faster than over the rows), and
  // reads r and writes z at the edge's row
  const int32_t* zrow = renum ? ctx->sell_inv.as<int32_t>() : nullptr;
  PG_TRY(load_input(s, r, E, stop, stride, off, renum));
  PG_TRY(forward(s, stop));
  const T* d = sizeof(T) == 8 ? reinterpret_cast<const T*>(diag32.as<float2>())
                              : reinterpret_cast<const T*>(ctx->diag.as<double2>());
  // algorithmic bytes per edge: r, z, diag, slot, tangent, and 2 x (32 B of y + 16 B of scales)
  KernelTimer kt(ctx, sizeof(T) == 8 ? "hx_out_c64" : "hx_out_c128",
                 (double)E * (3.0 * sizeof(T) + 4.0 + 16.0 + 96.0));
  if (xspace)
    k_hx_out<T, true><<<nb(E), 256, 0, s>>>(r, slot, E, y.as<float>(), aux.as<float4>(), tang.as<float4>(),
                                            scal.as<float>(), d, g[0][0], g[0][1], z, stop, stride, off, zrow);
  else
    k_hx_out<T, false><<<nb(E), 256, 0, s>>>(r, slot, E, y.as<float>(), aux.as<float4>(), tang.as<float4>(),
                                             scal.as<float>(), d, g[0][0], g[0][1], z, stop, stride, off, zrow);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

template Status Net::apply<float2>(cudaStream_t, const float2*, const int32_t*, int64_t, float2*, bool,
                                  const int*, int64_t, int64_t, bool);
template Status Net::apply<double2>(cudaStream_t, const double2*, const int32_t*, int64_t, double2*, bool,
                                   const int*, int64_t, int64_t, bool);

Status Net::renumber(petgem_ctx* c) {
  if (!c->sell_ok) return Status{PETGEM_ERR_UNSUPPORTED, "learned network: the mesh has no SELL-32 layout"};
  if (renum_mesh == c->mesh_version) return Status{};
  const int64_t ns = V[0] * 7;
  const void* before = slot_edge_r.ptr;
  PG_TRY(slot_edge_r.reserve((size_t)ns * sizeof(int32_t)));
  if (slot_edge_r.ptr != before) ++alloc_gen;
  k_renumber_slots<<<nb(ns), 256, 0, c->stream>>>(slot_edge.as<int32_t>(), ns, c->sell_inv.as<int32_t>(),
                                                  slot_edge_r.as<int32_t>());
  PG_CUDA(cudaGetLastError());
  renum_mesh = c->mesh_version;
  return Status{};
}

// One training sample, r = the residual of a solver iterate (complex128 edge vector).  Loss: the
// residual angle L = 1 - |<r, A z>|^2 / (|r|^2 |A z|^2) of the preconditioned direction
// z = D^{-1} r + G phi + Pi w (scale-free, as flexible GMRES is), back-propagated through A^H and
// the auxiliary maps to the network output.  A z = Ahat (D z) with Ahat = A D^{-1}.
Status Net::sample_grad(cudaStream_t s, petgem_ctx* c, const double2* r, const int32_t* slot, int64_t E, bool acc) {
  PG_TRY(load_input(s, r, E));
  PG_TRY(forward(s));
  double2* zu = dutmp.as<double2>();
  double2* w = wtmp.as<double2>();
  double2* gw = gtmp.as<double2>();
  k_hx_out<double2, false><<<nb(E), 256, 0, s>>>(r, slot, E, y.as<float>(), aux.as<float4>(), tang.as<float4>(),
                                                 scal.as<float>(), c->diag.as<double2>(), g[0][0], g[0][1], zu,
                                                 nullptr, 1, 0, nullptr);
  k_ahat_apply<<<nb(E), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->val.as<double2>(),
                                     c->diag.as<double2>(), zu, E, w);
  k_angle_dots<<<1, 1024, 0, s>>>(r, w, E, dvec.as<double>(), loss_acc.as<double>());
  k_angle_gw<<<nb(E), 256, 0, s>>>(r, w, E, dvec.as<double>(), gw);
  k_ahat_adjoint<<<nb(E), 256, 0, s>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(), c->val.as<double2>(),
                                       c->diag.as<double2>(), gw, E, zu);
  k_hx_dy<<<nb(V[0]), 256, 0, s>>>(zu, c->diag.as<double2>(), slot_edge.as<int32_t>(), tang.as<float4>(),
                                   aux.as<float4>(), scal.as<float>(), g[0][0], g[0][1], g[0][2],
                                   dd[0].as<__nv_bfloat16>());
  PG_CUDA(cudaGetLastError());
  PG_TRY(backward(s, acc));
  return Status{};
}

Status Net::adam_step(cudaStream_t s, float lr, float gscale) {
  ++adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)adam_t), c2 = 1.f - powf(b2, (float)adam_t);
  k_adam<<<nb(n_params), 256, 0, s>>>(params.as<float>(), grads.as<float>(), adam_m.as<float>(), adam_v.as<float>(),
                                      n_params, lr, b1, b2, 1e-8f, c1, c2, gscale);
  PG_CUDA(cudaGetLastError());
  return pack_weights(s);
}

Status Net::features(cudaStream_t s, const double* sigma, double sigma_p, double omega, double h) {
  PG_TRY(prepare_aux(ctx));
  const double mu0 = 4.0e-7 * 3.141592653589793238462643383279502884;
  k_node_features<<<nb(V[0]), 256, 0, s>>>(sigma, nx, ny, nz, sigma_p, omega * mu0 * h * h, feat.as<float>());
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status edge_slots(cudaStream_t s, const int32_t* edges, int64_t E, int gx, int gy, int gz, int32_t* slot, int* bad) {
  k_edge_slots<<<nb(E), 256, 0, s>>>(edges, E, gx, gy, gz, slot, bad);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status residual_and_error(petgem_ctx* c, const double2* x, const double2* xstar, double2* r, double2* du) {
  k_res_err<<<nb(c->n_edges), 256, 0, c->stream>>>(c->row_ptr.as<int64_t>(), c->col.as<int32_t>(),
                                                   c->val.as<double2>(), c->b.as<double2>(), c->diag.as<double2>(), x,
                                                   xstar, c->n_edges, r, du);
  PG_CUDA(cudaGetLastError());
  return Status{};
}

Status check_err(cudaStream_t s, const int* err, const char* where) {
  int h = 0;
  PG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PG_CUDA(cudaStreamSynchronize(s));
  if (h) return Status{PETGEM_ERR_TIMEOUT, std::string(where) + ": a tensor-core wait timed out"};
  return Status{};
}

}  // namespace nn
}  // namespace petgem
