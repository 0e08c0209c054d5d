// Primary field of a horizontal electric dipole in a horizontally layered Earth (Section 2: for a
// layered background the primary field is computed semi-analytically by Hankel transforms).
//
// The field is the source layer's whole-space field (App. A, closed form) plus Hankel integrals
// of the difference between the layered and the whole-space mode spectra.  For a horizontal
// wavenumber lambda the dipole's field splits into a TE and a TM problem in z (u_j^2 = lambda^2 +
// i w mu0 sigma_j, Re u_j > 0; f'' = u^2 f in every layer; f and f'/eps continuous at interfaces,
// eps = 1 for TE and sigma for TM; at the source TE has [f'] = 1, TM [f] = -1).  Here each is
// solved by admittance recursion: from the top half-space down and from the bottom half-space up
// to the source layer, the admittance Y = f' / (eps f) of the solution that decays away from the
// source, carried through every layer by its reflection coefficient; the amplitudes at the source
// follow from the jump conditions, and the field at z from products of bounded ratios of the
// layer solutions.  With (rho, theta) the horizontal offset of the point,
//   E_x = p/(4 pi) int lambda [(E_TM + E_TE) J0 - (E_TM - E_TE) J2 cos 2theta]
//   E_y = -p/(4 pi) int lambda (E_TM - E_TE) J2 sin 2theta,  E_z = i p/(2 pi) int lambda E_z,TM J1 cos theta,
// E_TE = i w mu0 f_TE, E_TM = -f_TM' / sigma, E_z,TM = i lambda f_TM / sigma.  A y-directed dipole
// is the x-directed one rotated by 90 degrees.
//
// Quadrature (the paper names Hankel filters and gives none; the integrals are evaluated by this
// rule): lambda_max = 36 / D, D the length over which the difference spectrum decays (the shortest
// path source - interface - point when the point lies in the source layer, else |z - z_s|, at
// least 1e-3 m); panels [0, k_min / 16], then panels doubling in width up to w = min(pi / rho,
// lambda_max / 16), then of width w (at most 16384 panels); 8-point Gauss-Legendre per panel.
#include <math.h>

#include <cmath>

#include "ctx.cuh"
#include "physics.cuh"

namespace petgem {
namespace {

constexpr int kMaxLayers = 8;
constexpr int kGL = 8;
constexpr double kDecay = 36.0;
constexpr int64_t kMaxPanels = 16384;

struct Layered {
  int nl;                       // layers; nl - 1 interfaces
  double zif[kMaxLayers - 1];   // interfaces, strictly decreasing (z up)
  double sig[kMaxLayers];       // conductivity of each layer, top first
  double omega, kmin;           // angular frequency, smallest |k_j| = sqrt(w mu0 sigma_j)
  double glx[kGL], glw[kGL];    // Gauss-Legendre nodes and weights on [-1, 1]
};

__device__ inline double2 cexp_(double2 z) {
  double s, c;
  sincos(z.y, &s, &c);
  const double e = exp(z.x);
  return make_double2(e * c, e * s);
}
// principal square root of a + ib with a >= 0 or b != 0 (here a = lambda^2, b = w mu0 sigma > 0)
__device__ inline double2 csqrt_(double2 z) {
  const double r = hypot(z.x, z.y);
  const double re = sqrt(0.5 * (r + z.x));
  return make_double2(re, re > 0.0 ? 0.5 * z.y / re : sqrt(0.5 * (r - z.x)));
}
__device__ inline double2 cone_plus(double2 a) { return make_double2(1.0 + a.x, a.y); }
__device__ inline double2 cone_minus(double2 a) { return make_double2(1.0 - a.x, -a.y); }

// Layer holding height z; a point on an interface belongs to the layer above it.
__host__ __device__ inline int layer_of(double z, const Layered& M) {
  int j = 0;
  while (j < M.nl - 1 && z < M.zif[j]) ++j;
  return j;
}

// f and f' at height z (layer jz) of the mode solution for the source at zs (layer s).
__device__ void mode_solution(const Layered& M, int s, int jz, double lam, double z, double zs, bool tm, double2& f,
                              double2& df) {
  double2 u[kMaxLayers];
  double eps[kMaxLayers];
  for (int j = 0; j < M.nl; ++j) {
    u[j] = csqrt_(make_double2(lam * lam, M.omega * phys::kMu0 * M.sig[j]));
    eps[j] = tm ? M.sig[j] : 1.0;
  }
  // from the top: reflection coefficient r_j (relative to the top of layer j) of the solution
  // decaying upward; the top half-space has r = 0
  double2 r[kMaxLayers], q[kMaxLayers];
  r[0] = make_double2(0.0, 0.0);
  if (s > 0) {
    double2 Y = cscale(u[0], -1.0 / eps[0]);
    for (int j = 1; j <= s; ++j) {
      const double2 y = cscale(cdiv(Y, u[j]), eps[j]);
      r[j] = cdiv(cone_plus(y), cone_minus(y));
      if (j < s) {
        const double2 E2 = cexp_(cscale(u[j], -2.0 * (M.zif[j - 1] - M.zif[j])));
        const double2 rE = cmul(r[j], E2);
        const double2 yb = cdiv(make_double2(rE.x - 1.0, rE.y), cone_plus(rE));
        Y = cscale(cmul(u[j], yb), 1.0 / eps[j]);
      }
    }
  }
  // from the bottom: q_j (relative to the bottom of layer j) of the solution decaying downward
  const int L = M.nl - 1;
  q[L] = make_double2(0.0, 0.0);
  if (s < L) {
    double2 Y = cscale(u[L], 1.0 / eps[L]);
    for (int j = L - 1; j >= s; --j) {
      const double2 y = cscale(cdiv(Y, u[j]), eps[j]);
      q[j] = cdiv(cone_minus(y), cone_plus(y));
      if (j > s) {
        const double2 E2 = cexp_(cscale(u[j], -2.0 * (M.zif[j - 1] - M.zif[j])));
        const double2 qE = cmul(q[j], E2);
        const double2 yt = cdiv(cone_minus(qE), cone_plus(qE));
        Y = cscale(cmul(u[j], yt), 1.0 / eps[j]);
      }
    }
  }
  // normalised admittances y = f' / (u_s f) at the source from above and from below
  const double2 us = u[s];
  const double t_up = s > 0 ? M.zif[s - 1] - zs : 0.0;
  const double t_dn = s < L ? zs - M.zif[s] : 0.0;
  const double2 rE = cmul(r[s], cexp_(cscale(us, -2.0 * t_up)));
  const double2 qE = cmul(q[s], cexp_(cscale(us, -2.0 * t_dn)));
  const double2 y_up = cdiv(make_double2(rE.x - 1.0, rE.y), cone_plus(rE));
  const double2 y_dn = cdiv(cone_minus(qE), cone_plus(qE));
  const double2 dy = csub(y_up, y_dn);
  // amplitudes of the solution normalised to 1 at zs, above (A) and below (B)
  double2 A, B;
  if (!tm) {
    A = cdiv(make_double2(1.0, 0.0), cmul(us, dy));
    B = A;
  } else {
    A = cdiv(y_dn, dy);
    B = cdiv(y_up, dy);
  }
  double2 cur = make_double2(1.0, 0.0);
  if (z >= zs) {  // walk up from zs to z
    double za = zs;
    for (int j = s;; --j) {
      const bool last = j == jz;
      const double zb = last ? z : M.zif[j - 1];
      const double2 uj = u[j];
      double2 g = cexp_(cscale(uj, -(zb - za)));
      double2 eb = make_double2(0.0, 0.0);
      if (j > 0) {  // (1 + r e^{2u(zb - top)}) / (1 + r e^{2u(za - top)})
        const double top = M.zif[j - 1];
        eb = cmul(r[j], cexp_(cscale(uj, 2.0 * (zb - top))));
        const double2 ea = cmul(r[j], cexp_(cscale(uj, 2.0 * (za - top))));
        g = cmul(g, cdiv(cone_plus(eb), cone_plus(ea)));
      }
      cur = cmul(cur, g);
      if (last) {
        f = cmul(A, cur);
        df = cmul(f, cmul(uj, cdiv(make_double2(eb.x - 1.0, eb.y), cone_plus(eb))));
        return;
      }
      za = zb;
    }
  } else {  // walk down from zs to z
    double za = zs;
    for (int j = s;; ++j) {
      const bool last = j == jz;
      const double zb = last ? z : M.zif[j];
      const double2 uj = u[j];
      double2 g = cexp_(cscale(uj, zb - za));
      double2 eb = make_double2(0.0, 0.0);
      if (j < L) {  // (1 + q e^{-2u(zb - bot)}) / (1 + q e^{-2u(za - bot)})
        const double bot = M.zif[j];
        eb = cmul(q[j], cexp_(cscale(uj, -2.0 * (zb - bot))));
        const double2 ea = cmul(q[j], cexp_(cscale(uj, -2.0 * (za - bot))));
        g = cmul(g, cdiv(cone_plus(eb), cone_plus(ea)));
      }
      cur = cmul(cur, g);
      if (last) {
        f = cmul(B, cur);
        df = cmul(f, cmul(uj, cdiv(cone_minus(eb), cone_plus(eb))));
        return;
      }
      za = zb;
    }
  }
}

__device__ inline double bessel_j2(double x, double j0x, double j1x) {
  if (x < 1e-3) return 0.125 * x * x * (1.0 - x * x / 12.0);  // series: J2 = x^2/8 - x^4/96 + ...
  return 2.0 * j1x / x - j0x;
}

// One block per point.  out[i][c] (complex128) for the dipole (xs, ys, zs, axis, moment).
__global__ void __launch_bounds__(256) k_layered_primary(Layered M, double xs, double ys, double zs, int axis,
                                                         double mom, const double* __restrict__ pts, int64_t n,
                                                         double2* __restrict__ out) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  double dx = pts[3 * i] - xs, dy = pts[3 * i + 1] - ys;
  const double z = pts[3 * i + 2];
  if (axis == 1) {  // rotate the offset by -90 degrees: the x-dipole's frame
    const double t = dx;
    dx = dy;
    dy = -t;
  }
  const double rho = hypot(dx, dy);
  const double th = rho > 0.0 ? atan2(dy, dx) : 0.0;
  const int s = layer_of(zs, M), jz = layer_of(z, M);
  // decay length of the difference spectrum
  double D;
  if (jz != s) {
    D = fabs(z - zs);
  } else {
    D = INFINITY;
    if (s > 0) D = fmin(D, (M.zif[s - 1] - zs) + (M.zif[s - 1] - z));
    if (s < M.nl - 1) D = fmin(D, (zs - M.zif[s]) + (z - M.zif[s]));
  }
  D = fmax(D, 1e-3);
  // panel rule: [0, a], doubling panels while the current edge is <= w, then width w; lmax last
  const double lmax = kDecay / D;
  double w = lmax / 16.0;
  if (rho > 0.0) w = fmin(w, phys::kPi / rho);
  const double a = fmin(M.kmin / 16.0, lmax);
  int m = 0;  // doubling panels
  double E = a;
  while (E < lmax && E <= w && 1 + m < kMaxPanels) {
    E = fmin(2.0 * E, lmax);
    ++m;
  }
  int64_t P = 1 + m;
  if (E < lmax) P += (int64_t)ceil((lmax - E) / w);
  P = P < kMaxPanels ? P : kMaxPanels;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // (E_TM + E_TE) J0, (E_TM - E_TE) J2, Ez J1 (re, im)
  const double2 te_ws_pre = make_double2(0.0, -M.omega * phys::kMu0);  // -i w mu0
  for (int64_t k = threadIdx.x; k < P * kGL; k += blockDim.x) {
    const int64_t p = k / kGL;
    const int g = (int)(k - p * kGL);
    double lo, hi;
    if (p == 0) {
      lo = 0.0;
      hi = a;
    } else if (p <= m) {
      lo = a * ldexp(1.0, (int)p - 1);
      hi = fmin(2.0 * lo, lmax);
    } else {
      lo = E + (double)(p - m - 1) * w;
      hi = fmin(lo + w, lmax);
    }
    if (!(hi > lo)) continue;
    const double lam = lo + 0.5 * (hi - lo) * (M.glx[g] + 1.0);
    const double wt = 0.5 * (hi - lo) * M.glw[g];
    double2 fte, dfte, ftm, dftm;
    mode_solution(M, s, jz, lam, z, zs, false, fte, dfte);
    mode_solution(M, s, jz, lam, z, zs, true, ftm, dftm);
    const double sj = M.sig[jz], ss = M.sig[s];
    double2 te = cmul(make_double2(0.0, M.omega * phys::kMu0), fte);
    double2 tmv = cscale(dftm, -1.0 / sj);
    double2 tz = cscale(cmul(make_double2(0.0, lam), ftm), 1.0 / sj);
    // minus the whole-space spectra of the source layer
    const double2 us = csqrt_(make_double2(lam * lam, M.omega * phys::kMu0 * ss));
    const double2 ex = cexp_(cscale(us, -fabs(z - zs)));
    const double sgn = z >= zs ? 1.0 : -1.0;
    te = csub(te, cdiv(cmul(te_ws_pre, ex), cscale(us, 2.0)));
    tmv = csub(tmv, cscale(cmul(us, ex), -0.5 / ss));
    tz = csub(tz, cscale(cmul(make_double2(0.0, lam), ex), -0.5 * sgn / ss));
    const double x = lam * rho;
    const double j0x = j0(x), j1x = j1(x), j2x = bessel_j2(x, j0x, j1x);
    const double c = wt * lam;
    acc[0] += c * (tmv.x + te.x) * j0x;
    acc[1] += c * (tmv.y + te.y) * j0x;
    acc[2] += c * (tmv.x - te.x) * j2x;
    acc[3] += c * (tmv.y - te.y) * j2x;
    acc[4] += c * tz.x * j1x;
    acc[5] += c * tz.y * j1x;
  }
  __shared__ double red[8][6];
  for (int q = 0; q < 6; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 6; ++q) red[threadIdx.x >> 5][q] = acc[q];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp)
    for (int q = 0; q < 6; ++q) t[q] += red[wp][q];
  double s2, c2, s1, c1;
  sincos(2.0 * th, &s2, &c2);
  sincos(th, &s1, &c1);
  const double k4 = mom / (4.0 * phys::kPi), k2 = mom / (2.0 * phys::kPi);
  double2 e[3];
  e[0] = make_double2(k4 * (t[0] - t[2] * c2), k4 * (t[1] - t[3] * c2));
  e[1] = make_double2(-k4 * t[2] * s2, -k4 * t[3] * s2);
  e[2] = make_double2(-k2 * t[5] * c1, k2 * t[4] * c1);  // i * (re + i im)
  if (axis == 1) {  // rotate the field back by +90 degrees
    const double2 ex0 = e[0];
    e[0] = make_double2(-e[1].x, -e[1].y);
    e[1] = ex0;
  }
  // plus the source layer's whole-space field (App. A)
  const double d[3] = {pts[3 * i] - xs, pts[3 * i + 1] - ys, z - zs};
  double2 Ew[3];
  phys::dipole_field(d, axis, mom, M.sig[s], sqrt(0.5 * M.omega * phys::kMu0 * M.sig[s]), Ew);
  for (int c = 0; c < 3; ++c) out[3 * i + c] = cadd(e[c], Ew[c]);
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the three-term recurrence of
// the Legendre polynomials.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Model of n layers (validated), Gauss-Legendre nodes included.
int make_model(int32_t n_layers, const double* z_interfaces, const double* sigma_layers, double freq_hz, Layered& M) {
  if (n_layers < 1 || !sigma_layers || !(freq_hz > 0.0) || (n_layers > 1 && !z_interfaces)) return PETGEM_ERR_INVALID_ARG;
  if (n_layers > kMaxLayers) return PETGEM_ERR_UNSUPPORTED;
  M = Layered{};
  M.nl = n_layers;
  double smin = INFINITY;
  for (int j = 0; j < n_layers; ++j) {
    if (!(sigma_layers[j] > 0.0) || !std::isfinite(sigma_layers[j])) return PETGEM_ERR_INVALID_ARG;
    M.sig[j] = sigma_layers[j];
    smin = std::fmin(smin, sigma_layers[j]);
  }
  for (int j = 0; j + 1 < n_layers; ++j) {
    if (!std::isfinite(z_interfaces[j]) || (j > 0 && !(z_interfaces[j] < z_interfaces[j - 1])))
      return PETGEM_ERR_INVALID_ARG;
    M.zif[j] = z_interfaces[j];
  }
  M.omega = 2.0 * phys::kPi * freq_hz;
  M.kmin = std::sqrt(M.omega * phys::kMu0 * smin);
  gauss_legendre(kGL, M.glx, M.glw);
  return PETGEM_OK;
}

}  // namespace

Status layered_primary(petgem_ctx* c, const petgem_dipole& src, int64_t n, const double* pts, double2* out) {
  Layered M;
  const int st = make_model(c->bg_layers, c->bg_z, c->bg_sig, c->freq, M);
  if (st != PETGEM_OK) return Status{st, "layered background"};
  if (src.axis != 0 && src.axis != 1) return Status{PETGEM_ERR_UNSUPPORTED, "layered background: horizontal dipoles only"};
  if (n == 0) return Status{};
  KernelTimer kt(c, "layered_primary", (double)n);
  k_layered_primary<<<(unsigned)n, 256, 0, c->stream>>>(M, src.x, src.y, src.z, src.axis, src.moment, pts, n, out);
  c->launches++;
  PG_CUDA(cudaGetLastError());
  return Status{};
}

}  // namespace petgem

extern "C" int petgem_primary_layered(void* stream, int32_t n_layers, const double* z_interfaces,
                                      const double* sigma_layers, double freq_hz, const petgem_dipole* src,
                                      int32_t n_pts, const double* pts, void* out) {
  using namespace petgem;
  if (!src || n_pts < 0) return PETGEM_ERR_INVALID_ARG;
  if (n_pts > 0 && (!pts || !out)) return PETGEM_ERR_INVALID_ARG;
  Layered M;
  const int st = make_model(n_layers, z_interfaces, sigma_layers, freq_hz, M);
  if (st != PETGEM_OK) return st;
  if (src->axis != 0 && src->axis != 1) return PETGEM_ERR_UNSUPPORTED;
  if (n_pts == 0) return PETGEM_OK;
  k_layered_primary<<<(unsigned)n_pts, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      M, src->x, src->y, src->z, src->axis, src->moment, pts, n_pts, static_cast<double2*>(out));
  return cudaGetLastError() == cudaSuccess ? PETGEM_OK : PETGEM_ERR_CUDA;
}
