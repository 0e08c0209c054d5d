// Host-side interface of the learned preconditioner's network (learned.cu).
#pragma once
#include <cuda_bf16.h>

#include "ctx.cuh"

namespace petgem {
namespace nn {

struct Layer {
  int cin, cout, relu;
  int64_t w_off, b_off;  // offsets into the parameter vector: W[27][cout][cin] then b[cout]
};

constexpr int kMaxLevels = 12;

// Levels of a grid: poolings until the coarsest grid has at most 3 nodes per axis (at least 3).
inline int net_levels(int gx, int gy, int gz) {
  int L = 1;
  while (gx > 3 || gy > 3 || gz > 3) {
    gx = (gx + 1) / 2;
    gy = (gy + 1) / 2;
    gz = (gz + 1) / 2;
    ++L;
  }
  return L < 3 ? 3 : L;
}

struct Net {
  petgem_ctx* ctx = nullptr;
  bool ready = false;
  int nx = 0, ny = 0, nz = 0;
  int nlev = 0;                // levels (net_levels of the node grid)
  int g[kMaxLevels][3];        // grid dimensions per level
  int64_t V[kMaxLevels];       // voxels per level
  Layer L[7];
  int64_t n_params = 0;
  int64_t adam_t = 0;
  DevBuf params, grads, adam_m, adam_v, wb, wd, zbias;
  // per level l: q = encoder input (q[0] = the network input), e = encoder output, sk = decoder
  // input (upsampled coarse + e), d = decoder output (d[0] is y, FP32; d[nlev-1] is e[nlev-1]);
  // dd = gradient at d (dd[0] = dy), ds = gradient at sk, dq = gradient at q
  DevBuf q[kMaxLevels], e[kMaxLevels], sk[kMaxLevels], d[kMaxLevels];
  DevBuf dd[kMaxLevels], ds[kMaxLevels], dq[kMaxLevels];
  DevBuf y;
  DevBuf feat, scal, loss_acc, err, wpart, rtmp, dutmp, wtmp, gtmp, dvec;
  // auxiliary spaces on the lattice: edge of every slot (node * 7 + class, -1 if none), the
  // slot's unit tangent and inverse length, per-node scales (sg, sp_x, sp_y, sp_z), the gathered
  // node fields [V0][8] and per-block partial sums
  DevBuf slot_edge, tang, aux, nodes8, npart, diag32;  // diag32: diag(A) as complex64
  DevBuf slot_edge_r;                                  // slot -> SELL-32 row of its edge (renumbered application)
  int64_t renum_mesh = -1;
  int64_t aux_version = -1;    // assembly the scales belong to
  int64_t geom_version = -1;   // mesh the slot map and tangents belong to
  int64_t alloc_gen = 0;       // bumped whenever a buffer may have moved (captured graphs key on it)
  Status init(petgem_ctx* c, int nx, int ny, int nz);
  Status pack_weights(cudaStream_t s);
  // layer i on level lvl
  Status conv(cudaStream_t s, int i, int lvl, const __nv_bfloat16* in, __nv_bfloat16* out, float* outf,
              const int* stop = nullptr);
  Status dgrad(cudaStream_t s, int i, int lvl, const __nv_bfloat16* dout, __nv_bfloat16* din);
  Status wgrad(cudaStream_t s, int i, int lvl, const __nv_bfloat16* in, const __nv_bfloat16* dout, bool acc);
  int enc(int l) const { return l == 0 ? 0 : l == 1 ? 1 : l == nlev - 1 ? 3 : 2; }  // c1, c2, c4, c3
  int dec(int l) const { return l == 0 ? 6 : l == 1 ? 5 : 4; }                        // c7, c6, c5
  static int ch_e(int l) { return l == 0 ? 16 : 32; }
  static int ch_q(int l) { return l <= 1 ? 16 : 32; }
  static int ch_d(int l) { return l == 1 ? 16 : 32; }
  // stop: optional device flag; when nonzero every kernel of the pass returns at once (a FGMRES
  // cycle that already stopped)
  Status forward(cudaStream_t s, const int* stop = nullptr);
  Status backward(cudaStream_t s, bool acc);
  Status prepare_aux(petgem_ctx* c);
  template <typename T> Status load_input(cudaStream_t s, const T* r, int64_t E, const int* stop = nullptr,
                                          int64_t stride = 1, int64_t off = 0, bool renum = false);
  // z = D (D^{-1} r + G phi + Pi w) (the solver's Jacobi-scaled variables) or, with xspace,
  // z = D^{-1} r + G phi + Pi w, for the residual r of E entries.  Entry e of r and z sits at
  // e stride + off (one source of an interleaved block vector: stride = the group size).
  // renum: r and z are in the SELL-32 row order of the context (renumber() first): the node-wise
  // map gathers r through the rows of its slots' edges, the edge-wise map runs in edge order.
  template <typename T> Status apply(cudaStream_t s, const T* r, const int32_t* slot, int64_t E, T* z,
                                     bool xspace = false, const int* stop = nullptr, int64_t stride = 1,
                                     int64_t off = 0, bool renum = false);
  // The slot map of the renumbered application (after prepare_aux, before any stream capture).
  Status renumber(petgem_ctx* c);
  Status sample_grad(cudaStream_t s, petgem_ctx* c, const double2* r, const int32_t* slot, int64_t E, bool acc);
  Status adam_step(cudaStream_t s, float lr, float gscale);
  Status features(cudaStream_t s, const double* sigma, double sigma_p, double omega, double h);
};

// The tensor-core convolution (k_conv3d): any grid size; w packed by k_pack_conv_weights (the
// kernel's shared-memory image); x, w and y 16-byte aligned.
Status conv3d(cudaStream_t s, int gx, int gy, int gz, int cin, int cout, const __nv_bfloat16* x,
              const __nv_bfloat16* w, const float* bias, bool relu, __nv_bfloat16* ybf, float* yf, int* err,
              const int* stop = nullptr);
// BF16 weights [27][cout][cin] -> the convolution kernel's shared-memory image (wc, 27 cin cout).
Status pack_conv_weights(cudaStream_t s, const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wc);
// Dynamic shared-memory limits of the tensor-core convolutions (once per process; before any
// stream capture).
Status conv3d_attributes();
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
