// Element geometry and the primary field, shared by the assembly and receiver kernels.
#pragma once
#include <math.h>

#include "common.cuh"

namespace petgem {
namespace phys {

static __constant__ int kA[6] = {0, 0, 0, 1, 3, 2};  // Appendix B eqs. B.1-B.6
static __constant__ int kB[6] = {1, 2, 3, 2, 1, 3};

static constexpr double kPi = 3.141592653589793238462643383279502884;
static constexpr double kMu0 = 4.0e-7 * kPi;

struct TetGeom {
  double p[4][3];
  double g[4][3];  // grad lambda_i
  double det;      // 6 x signed volume
  double vol;
  double len[6];
};

__device__ inline void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ inline double dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Barycentric gradients by the cofactor formula: with e_k = p_k - p_0 and det = e1 . (e2 x e3),
// grad l1 = (e2 x e3)/det, grad l2 = (e3 x e1)/det, grad l3 = (e1 x e2)/det, grad l0 = -sum.
__device__ inline bool tet_geometry(const double* __restrict__ nodes, const int32_t* __restrict__ tets, int64_t t,
                                    TetGeom& G) {
  for (int j = 0; j < 4; ++j) {
    int64_t v = tets[4 * t + j];
    G.p[j][0] = nodes[3 * v];
    G.p[j][1] = nodes[3 * v + 1];
    G.p[j][2] = nodes[3 * v + 2];
  }
  double e[3][3];
  for (int k = 1; k < 4; ++k)
    for (int d = 0; d < 3; ++d) e[k - 1][d] = G.p[k][d] - G.p[0][d];
  double c23[3], c31[3], c12[3];
  cross(e[1], e[2], c23);
  cross(e[2], e[0], c31);
  cross(e[0], e[1], c12);
  G.det = dot(e[0], c23);
  G.vol = fabs(G.det) / 6.0;
  double lmax2 = 0.0;
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      double q = G.p[kB[i]][d] - G.p[kA[i]][d];
      s += q * q;
    }
    G.len[i] = sqrt(s);
    lmax2 = fmax(lmax2, s);
  }
  if (!(fabs(G.det) > 1e-13 * lmax2 * sqrt(lmax2))) return false;
  double inv = 1.0 / G.det;
  for (int d = 0; d < 3; ++d) {
    G.g[1][d] = c23[d] * inv;
    G.g[2][d] = c31[d] * inv;
    G.g[3][d] = c12[d] * inv;
    G.g[0][d] = -(G.g[1][d] + G.g[2][d] + G.g[3][d]);
  }
  return true;
}

// Whole-space dipole field (Appendix A, eqs. A.1-A.3) at distance vector d from the source,
// background sigma, kappa = sqrt(w mu0 sigma / 2).  With the decaying root k = (1 - i) kappa
// (eq. 6's operator carries +i w mu0 sigma, so k^2 = -i w mu0 sigma):
//   e^{-ikr} = e^{-kappa r} (cos kappa r - i sin kappa r),  ikr = (1 + i) kappa r,
//   k^2 r^2 = -2 i kappa^2 r^2,
// and component j = p / (4 pi sigma r^3) e^{-ikr} [ (d_a d_j / r^2) A + delta_aj B ] with
//   A = -k^2 r^2 + 3ikr + 3 = (3 + 3 kappa r) + i (2 kappa^2 r^2 + 3 kappa r),
//   B =  k^2 r^2 - ikr - 1  = -(1 + kappa r) - i (2 kappa^2 r^2 + kappa r).
__device__ inline void dipole_field(const double d[3], int axis, double moment, double sigma, double kappa,
                                    double2 E[3]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double r = sqrt(r2);
  double kr = kappa * r;
  double s, c;
  sincos(kr, &s, &c);
  double amp = moment * exp(-kr) / (4.0 * kPi * sigma * r * r2);
  double2 pre = make_double2(amp * c, -amp * s);
  double2 A = make_double2(3.0 + 3.0 * kr, 2.0 * kr * kr + 3.0 * kr);
  double2 B = make_double2(-(1.0 + kr), -(2.0 * kr * kr + kr));
  double inv_r2 = 1.0 / r2;
  for (int j = 0; j < 3; ++j) {
    double f = d[axis] * d[j] * inv_r2;
    double2 br = make_double2(f * A.x + (j == axis ? B.x : 0.0), f * A.y + (j == axis ? B.y : 0.0));
    E[j] = cmul(pre, br);
  }
}


}  // namespace phys
}  // namespace petgem
