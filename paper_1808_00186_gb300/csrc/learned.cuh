// Host-side interface of the learned preconditioner's network (learned.cu).
#pragma once
#include <cuda_bf16.h>

#include "ctx.cuh"

namespace petgem {
namespace nn {

struct Layer {
  int cin, cout, relu, level;
  int64_t w_off, b_off;  // offsets into the parameter vector: W[27][cout][cin] then b[cout]
};

struct Net {
  petgem_ctx* ctx = nullptr;
  bool ready = false;
  int nx = 0, ny = 0, nz = 0;
  int g[4][3];      // grid dimensions of levels 0..3
  int64_t V[4];     // voxels per level
  Layer L[7];
  int64_t n_params = 0;
  int64_t adam_t = 0;
  DevBuf params, grads, adam_m, adam_v, wb, wd, zbias;
  DevBuf x0, a1, p1, a2, p2, a3, p3, a4, s5, a5, s6, a6, s7, y;
  DevBuf dy, ds7, da6, ds6, da5, ds5, da4, dp3, dp2, dp1;
  DevBuf g32, feat, scal, loss_acc, err, wpart, rtmp, dutmp, wtmp, gtmp, dvec;
  // auxiliary spaces on the lattice: edge of every slot (node * 7 + class, -1 if none), the
  // slot's unit tangent and inverse length, per-node scales (sg, sp_x, sp_y, sp_z), the gathered
  // node fields [V0][8] and per-block partial sums
  DevBuf slot_edge, tang, aux, nodes8, npart;
  int64_t aux_version = -1;    // assembly the scales belong to
  int64_t geom_version = -1;   // mesh the slot map and tangents belong to

  Status init(petgem_ctx* c, int nx, int ny, int nz);
  Status pack_weights(cudaStream_t s);
  Status conv(cudaStream_t s, int i, const __nv_bfloat16* in, __nv_bfloat16* out, float* outf);
  Status dgrad(cudaStream_t s, int i, const __nv_bfloat16* dout, __nv_bfloat16* din);
  Status wgrad(cudaStream_t s, int i, const __nv_bfloat16* in, const __nv_bfloat16* dout, bool acc);
  Status forward(cudaStream_t s);
  Status backward(cudaStream_t s, bool acc);
  Status prepare_aux(petgem_ctx* c);
  template <typename T> Status load_input(cudaStream_t s, const T* r, int64_t E);
  // z = D (D^{-1} r + G phi + Pi w) (the solver's Jacobi-scaled variables) or, with xspace,
  // z = D^{-1} r + G phi + Pi w, for the residual r of E entries.
  template <typename T> Status apply(cudaStream_t s, const T* r, const int32_t* slot, int64_t E, T* z,
                                     bool xspace = false);
  Status sample_grad(cudaStream_t s, petgem_ctx* c, const double2* r, const int32_t* slot, int64_t E, bool acc);
  Status adam_step(cudaStream_t s, float lr, float gscale);
  Status features(cudaStream_t s, const double* sigma, double sigma_p, double omega, double h);
};

Status conv3d(cudaStream_t s, int gx, int gy, int gz, int cin, int cout, const __nv_bfloat16* x,
              const __nv_bfloat16* w, const float* bias, bool relu, __nv_bfloat16* ybf, float* yf, int* err);
Status conv3d_wgrad(cudaStream_t s, int gx, int gy, int gz, int cin, int cout, const __nv_bfloat16* x,
                    const __nv_bfloat16* dy, float* part, int splits, float* dw, bool accumulate, int* err);
int wgrad_splits(int64_t V);
// The convolution kernels index voxels (and voxels x 32 channels) in 32 bits: a grid fits when
// gx gy gz 32 < 2^31.  Each factor is bounded before the next product, so nothing wraps.
inline bool grid_fits(int64_t gx, int64_t gy, int64_t gz) {
  const int64_t lim = (int64_t(1) << 31) / 32;
  if (gx < 1 || gy < 1 || gz < 1 || gx > lim || gy > lim || gz > lim) return false;
  const int64_t xy = gx * gy;
  return xy < lim && xy * gz < lim;
}
Status edge_slots(cudaStream_t s, const int32_t* edges, int64_t E, int gx, int gy, int gz, int32_t* slot, int* bad);
Status check_err(cudaStream_t s, const int* err, const char* where);
// r = b - A x and du = D (x* - x) for the context's assembled system (source 0), complex128.
Status residual_and_error(petgem_ctx* c, const double2* x, const double2* xstar, double2* r, double2* du);

}  // namespace nn
}  // namespace petgem
