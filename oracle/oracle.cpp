// CPU oracle for the secondary-field CSEM forward problem on Nedelec edge elements.
//
// TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Plain, slow, FP64 (std::complex<double>)
// restatement of what the paper computes, used only by tests/, by the smoke check and by
// the benchmark's CPU-baseline leg.  It shares no code, header or table with the CUDA
// library, and the CUDA library never calls it.
//
// What it follows (Castillo-Reyes, de la Puente, Cela, "PETGEM", Comput. Geosci. 2018):
//   * curl-curl secondary-field equation, Section 2 eq. 6, Dirichlet E_s = 0 on the boundary;
//   * element system K^e + i w mu0 sigma_e M^e, right-hand side -i w mu0 dsigma_e R^e, Section 3 eq. 9;
//   * whole-space dipole primary field, Appendix A eqs. A.1-A.3;
//   * lowest-order Nedelec basis, local edge table, K^e, M^e and edge signs, Appendix B eqs. B.1-B.16;
//   * interpolation E(x) = sum_i N_i(x) E_i, Section 3 eq. 7;
//   * GMRES as the Krylov solver (Section 5.1), Jacobi-preconditioned.
// Readings where the paper is silent or garbled are written next to the code that takes them.
// Parity status: every function here is pinned by tests that do not call it back (closed
// forms, exact rational integrals, brute force, finite-difference PDE residuals, dense LU).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846;
const double kMu0 = 4.0e-7 * kPi;  // free-space permeability; the paper does not print a value

// Status codes (mirrors nothing: the oracle's own).
enum { ORC_OK = 0, ORC_BAD_INPUT = 1, ORC_DEGENERATE = 2, ORC_NOT_CONVERGED = 3, ORC_OUTSIDE = 4,
       ORC_SINGULAR = 5 };

// Appendix B, eqs. B.1-B.6: local edge i joins local nodes (a, b) and its basis is W_ab:
// N1 = W12, N2 = W13, N3 = W14, N4 = W23, N5 = W42, N6 = W34 (1-based in the paper).
const int kEdgeA[6] = {0, 0, 0, 1, 3, 2};
const int kEdgeB[6] = {1, 2, 3, 2, 1, 3};

// ------------------------------------------------------------------------------------------
// Element geometry: barycentric coordinates lambda_i(x) = c0_i + g_i . x with lambda_i(x_j) =
// delta_ij.  Appendix B eq. B.7 writes grad lambda_i = (b_i, c_i, d_i) / (6V); here the
// coefficients come from solving [1 x_j y_j z_j] C = I by Gaussian elimination with partial
// pivoting, which gives the same gradients for either vertex orientation.
struct Geom {
  double c0[4];
  double g[4][3];
  double vol;  // |det| / 6
  double len[6];
};

int solve4_inverse(const double m_in[4][4], double inv[4][4], double* det) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = c < 4 ? m_in[r][c] : (c - 4 == r ? 1.0 : 0.0);
  double d = 1.0;
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return ORC_DEGENERATE;
    if (piv != col) {
      for (int c = 0; c < 8; ++c) std::swap(a[piv][c], a[col][c]);
      d = -d;
    }
    d *= a[col][col];
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      double f = a[r][col] / a[col][col];
      for (int c = col; c < 8; ++c) a[r][c] -= f * a[col][c];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) inv[r][c] = a[r][c + 4] / a[r][r];
  *det = d;
  return ORC_OK;
}

int geometry(const double p[4][3], Geom* G) {
  double m[4][4], inv[4][4], det;
  for (int j = 0; j < 4; ++j) {
    m[j][0] = 1.0;
    m[j][1] = p[j][0];
    m[j][2] = p[j][1];
    m[j][3] = p[j][2];
  }
  // Row j of m evaluates (c0, g) at vertex j, so column i of m^{-1} holds lambda_i's coefficients.
  if (solve4_inverse(m, inv, &det) != ORC_OK) return ORC_DEGENERATE;
  G->vol = std::fabs(det) / 6.0;
  if (!(G->vol > 0.0)) return ORC_DEGENERATE;
  for (int i = 0; i < 4; ++i) {
    G->c0[i] = inv[0][i];
    for (int k = 0; k < 3; ++k) G->g[i][k] = inv[k + 1][i];
  }
  for (int e = 0; e < 6; ++e) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
      double d = p[kEdgeB[e]][k] - p[kEdgeA[e]][k];
      s += d * d;
    }
    G->len[e] = std::sqrt(s);
  }
  return ORC_OK;
}

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Appendix B eqs. B.14-B.15 with signs S_i (eq. B.16).
// Curl of W_ab = lambda_a grad lambda_b - lambda_b grad lambda_a is the constant
// 2 grad lambda_a x grad lambda_b, so K_ij = V * (2 l_i S_i ga x gb) . (2 l_j S_j gc x gd).
// M_ij integrates the products of the four terms with int lambda_p lambda_q dV = V (1 + d_pq) / 20.
void element_km(const Geom& G, const int8_t* S, double K[36], double M[36]) {
  double curl[6][3];
  for (int e = 0; e < 6; ++e) {
    cross3(G.g[kEdgeA[e]], G.g[kEdgeB[e]], curl[e]);
    for (int k = 0; k < 3; ++k) curl[e][k] *= 2.0 * G.len[e] * S[e];
  }
  auto I = [&](int p, int q) { return G.vol * (p == q ? 2.0 : 1.0) / 20.0; };
  auto gg = [&](int p, int q) { return dot3(G.g[p], G.g[q]); };
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      K[i * 6 + j] = G.vol * dot3(curl[i], curl[j]);
      int a = kEdgeA[i], b = kEdgeB[i], c = kEdgeA[j], d = kEdgeB[j];
      double w = I(a, c) * gg(b, d) - I(a, d) * gg(b, c) - I(b, c) * gg(a, d) + I(b, d) * gg(a, c);
      M[i * 6 + j] = S[i] * S[j] * G.len[i] * G.len[j] * w;
    }
  }
}

// Appendix A eqs. A.1-A.3: whole-space electric dipole of moment I dS along `axis`, in a
// medium of conductivity sigma (the background sigma_p).  Reading of the garbled x-dipole
// bracket, taken from the y- and z-dipole lines: component j is
//   p / (4 pi sigma r^3) e^{-ikr} [ (d_a d_j / r^2)(-k^2 r^2 + 3ikr + 3) + delta_aj (k^2 r^2 - ikr - 1) ]
// with d = x - x_s.  The curl-curl operator of eq. 6 carries +i w mu0 sigma, so k^2 = -i w mu0 sigma
// and the root with Im k < 0 makes e^{-ikr} decay.
void primary_field(const double* x, const double* src, double sigma, double omega, cd E[3]) {
  double d[3] = {x[0] - src[0], x[1] - src[1], x[2] - src[2]};
  int axis = (int)src[3];
  double moment = src[4];
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double r = std::sqrt(r2);
  cd k = std::sqrt(cd(0.0, -omega * kMu0 * sigma));
  if (k.imag() > 0.0) k = -k;
  const cd I1(0.0, 1.0);
  cd ikr = I1 * k * r;
  cd k2r2 = k * k * r2;
  cd pre = moment / (4.0 * kPi * sigma * r * r2) * std::exp(-ikr);
  cd A = -k2r2 + 3.0 * ikr + 3.0;
  cd B = k2r2 - ikr - 1.0;
  for (int j = 0; j < 3; ++j) E[j] = pre * ((d[axis] * d[j] / r2) * A + (j == axis ? B : cd(0.0)));
}

// Section 3 eq. 9 says the right-hand side is integrated numerically but names no rule.
// Reading: the symmetric 4-point degree-2 rule on the tetrahedron, barycentric points
// (alpha, beta, beta, beta) and permutations, alpha = (5 + 3 sqrt 5) / 20, beta = (5 - sqrt 5) / 20,
// each with weight V / 4.
void quad_points(double bary[4][4]) {
  double alpha = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, beta = (5.0 - std::sqrt(5.0)) / 20.0;
  for (int q = 0; q < 4; ++q)
    for (int i = 0; i < 4; ++i) bary[q][i] = (i == q) ? alpha : beta;
}

// Nedelec basis at barycentric point lam (eqs. B.1-B.6): N_e = l_e (lam_a grad lam_b - lam_b grad lam_a).
void basis_at(const Geom& G, const double lam[4], double N[6][3]) {
  for (int e = 0; e < 6; ++e) {
    int a = kEdgeA[e], b = kEdgeB[e];
    for (int k = 0; k < 3; ++k) N[e][k] = G.len[e] * (lam[a] * G.g[b][k] - lam[b] * G.g[a][k]);
  }
}

void tet_points(const double* nodes, const int32_t* tet, double p[4][3]) {
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 3; ++k) p[j][k] = nodes[3 * (int64_t)tet[j] + k];
}

// ------------------------------------------------------------------------------------------
struct System {
  int64_t n_nodes = 0, n_tets = 0, n_edges = 0, n_src = 0;
  std::vector<double> nodes;
  std::vector<int32_t> tets;
  std::vector<int32_t> edges;      // [E][2] (low id, high id)
  std::vector<int32_t> tet_edges;  // [T][6]
  std::vector<int8_t> signs;       // [T][6]
  std::vector<uint8_t> boundary;   // [E]
  std::vector<int64_t> row_ptr;    // [E + 1]
  std::vector<int32_t> col;
  std::vector<cd> val;
  std::vector<cd> diag;            // Jacobi diagonal D = diag(A)
  std::vector<cd> b;               // [S][E]
  std::vector<double> src;         // [S][5]
  double sigma_p = 1.0, omega = 0.0;
};

// Appendix B eq. B.16 and the text around it: a global edge points from its lower to its higher
// node id; S_i = sign(node_i2 - node_i1) for local edge i running node_i1 -> node_i2 as in W_ab.
// The paper imports the edge numbering from files and does not fix an order.  Reading: global
// edge id = rank of (low, high) in lexicographic order.
int number_edges(System& s) {
  struct Occ { int32_t lo, hi; int64_t slot; };
  std::vector<Occ> occ((size_t)s.n_tets * 6);
  s.signs.assign((size_t)s.n_tets * 6, 0);
  for (int64_t t = 0; t < s.n_tets; ++t) {
    for (int e = 0; e < 6; ++e) {
      int32_t n1 = s.tets[4 * t + kEdgeA[e]], n2 = s.tets[4 * t + kEdgeB[e]];
      if (n1 == n2) return ORC_BAD_INPUT;
      occ[6 * t + e] = {std::min(n1, n2), std::max(n1, n2), 6 * t + e};
      s.signs[6 * t + e] = n2 > n1 ? 1 : -1;
    }
  }
  std::sort(occ.begin(), occ.end(), [](const Occ& a, const Occ& b) {
    if (a.lo != b.lo) return a.lo < b.lo;
    if (a.hi != b.hi) return a.hi < b.hi;
    return a.slot < b.slot;
  });
  s.tet_edges.assign((size_t)s.n_tets * 6, -1);
  s.edges.clear();
  for (size_t i = 0; i < occ.size(); ++i) {
    if (i == 0 || occ[i].lo != occ[i - 1].lo || occ[i].hi != occ[i - 1].hi) {
      s.edges.push_back(occ[i].lo);
      s.edges.push_back(occ[i].hi);
    }
    s.tet_edges[occ[i].slot] = (int32_t)(s.edges.size() / 2 - 1);
  }
  s.n_edges = (int64_t)s.edges.size() / 2;
  return ORC_OK;
}

// Section 2: E_s = 0 on the outer boundary.  Reading: the boundary is the union of the faces
// that belong to exactly one tet, and its edges are the Dirichlet edges (Table 1's DOF column
// is the edge count minus these).
int find_boundary(System& s) {
  struct Face { int32_t v[3]; int64_t tet; int opp; };
  std::vector<Face> faces((size_t)s.n_tets * 4);
  for (int64_t t = 0; t < s.n_tets; ++t) {
    for (int o = 0; o < 4; ++o) {
      Face f;
      int m = 0;
      for (int j = 0; j < 4; ++j)
        if (j != o) f.v[m++] = s.tets[4 * t + j];
      std::sort(f.v, f.v + 3);
      f.tet = t;
      f.opp = o;
      faces[4 * t + o] = f;
    }
  }
  std::sort(faces.begin(), faces.end(), [](const Face& a, const Face& b) {
    for (int k = 0; k < 3; ++k)
      if (a.v[k] != b.v[k]) return a.v[k] < b.v[k];
    return a.tet < b.tet;
  });
  s.boundary.assign((size_t)s.n_edges, 0);
  size_t i = 0;
  while (i < faces.size()) {
    size_t j = i + 1;
    while (j < faces.size() && std::equal(faces[j].v, faces[j].v + 3, faces[i].v)) ++j;
    if (j - i > 2) return ORC_BAD_INPUT;  // a face shared by three or more tets
    if (j - i == 1) {
      const Face& f = faces[i];
      for (int e = 0; e < 6; ++e)
        if (kEdgeA[e] != f.opp && kEdgeB[e] != f.opp) s.boundary[s.tet_edges[6 * f.tet + e]] = 1;
    }
    i = j;
  }
  return ORC_OK;
}

// Section 3 eq. 9 summed over elements (Section 4: every element adds its contributions to the
// global system), then the Dirichlet rows of Section 2.  mu0 multiplies the mass term as in
// eqs. 3 and 6 (eq. 9 drops it).  Optional g holds prescribed boundary values [S][E] (NULL =
// homogeneous, the paper's condition); interior rows then move A_IB g to the right-hand side.
int assemble(System& s, const double* sigma, double freq, const cd* g) {
  const cd I1(0.0, 1.0);
  s.omega = 2.0 * kPi * freq;
  const int64_t E = s.n_edges, T = s.n_tets, S = s.n_src;
  // Element matrices and right-hand sides, one tet at a time.
  std::vector<cd> Ae((size_t)T * 36);
  std::vector<cd> be((size_t)T * 6 * S, cd(0.0));
  double qb[4][4];
  quad_points(qb);
  for (int64_t t = 0; t < T; ++t) {
    double p[4][3];
    tet_points(s.nodes.data(), &s.tets[4 * t], p);
    Geom G;
    if (geometry(p, &G) != ORC_OK) return ORC_DEGENERATE;
    double K[36], M[36];
    const int8_t* Sg = &s.signs[6 * t];
    element_km(G, Sg, K, M);
    for (int k = 0; k < 36; ++k) Ae[36 * t + k] = K[k] + I1 * s.omega * kMu0 * sigma[t] * M[k];
    double dsig = sigma[t] - s.sigma_p;
    if (dsig == 0.0) continue;
    for (int64_t sc = 0; sc < S; ++sc) {
      cd R[6] = {};
      for (int q = 0; q < 4; ++q) {
        double xq[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < 4; ++j)
          for (int k = 0; k < 3; ++k) xq[k] += qb[q][j] * p[j][k];
        cd Ep[3];
        primary_field(xq, &s.src[5 * sc], s.sigma_p, s.omega, Ep);
        double N[6][3];
        basis_at(G, qb[q], N);
        for (int e = 0; e < 6; ++e)
          R[e] += (G.vol / 4.0) * (double)Sg[e] * (N[e][0] * Ep[0] + N[e][1] * Ep[1] + N[e][2] * Ep[2]);
      }
      for (int e = 0; e < 6; ++e) be[(6 * t + e) * S + sc] = -I1 * s.omega * kMu0 * dsig * R[e];
    }
  }
  // Global rows: gather, for every edge, the contributions of the tets that hold it.
  std::vector<std::vector<std::pair<int64_t, int>>> holders((size_t)E);  // (tet, local edge)
  for (int64_t t = 0; t < T; ++t)
    for (int e = 0; e < 6; ++e) holders[s.tet_edges[6 * t + e]].push_back({t, e});
  s.b.assign((size_t)S * E, cd(0.0));
  s.row_ptr.assign((size_t)E + 1, 0);
  s.col.clear();
  s.val.clear();
  s.diag.assign((size_t)E, cd(0.0));
  for (int64_t r = 0; r < E; ++r) {
    if (s.boundary[r]) {  // identity row, right-hand side = prescribed value
      s.col.push_back((int32_t)r);
      s.val.push_back(1.0);
      s.diag[r] = 1.0;
      for (int64_t sc = 0; sc < S; ++sc) s.b[sc * E + r] = g ? g[sc * E + r] : cd(0.0);
      s.row_ptr[r + 1] = (int64_t)s.col.size();
      continue;
    }
    std::vector<std::pair<int32_t, cd>> row;
    for (auto& h : holders[r]) {
      for (int j = 0; j < 6; ++j) row.push_back({s.tet_edges[6 * h.first + j], Ae[36 * h.first + 6 * h.second + j]});
      for (int64_t sc = 0; sc < S; ++sc) s.b[sc * E + r] += be[(6 * h.first + h.second) * S + sc];
    }
    std::stable_sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    size_t i = 0;
    while (i < row.size()) {
      int32_t c = row[i].first;
      cd v = 0.0;
      size_t j = i;
      for (; j < row.size() && row[j].first == c; ++j) v += row[j].second;
      if (s.boundary[c]) {
        if (g)
          for (int64_t sc = 0; sc < S; ++sc) s.b[sc * E + r] -= v * g[sc * E + c];
      } else {
        s.col.push_back(c);
        s.val.push_back(v);
        if (c == r) s.diag[r] = v;
      }
      i = j;
    }
    s.row_ptr[r + 1] = (int64_t)s.col.size();
  }
  return ORC_OK;
}

void spmv(const System& s, const cd* x, cd* y) {
  for (int64_t r = 0; r < s.n_edges; ++r) {
    cd acc = 0.0;
    for (int64_t p = s.row_ptr[r]; p < s.row_ptr[r + 1]; ++p) acc += s.val[p] * x[s.col[p]];
    y[r] = acc;
  }
}

double norm2(const cd* v, int64_t n) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc += std::norm(v[i]);
  return std::sqrt(acc);
}

// Restarted GMRES(m) with right Jacobi preconditioning (solve A D^{-1} u = b, x = D^{-1} u),
// modified Gram-Schmidt Arnoldi with Hermitian inner products, complex Givens rotations, and a
// restart from the true residual b - A x.  Stops when ||b - A x|| / ||b|| <= tol, checked on the
// true residual at the end of each cycle.  The paper uses PETSc's GMRES (Section 5.1) and gives no
// details; these are the textbook choices (Saad, Iterative Methods for Sparse Linear Systems, 6.5).
int gmres(const System& s, const cd* b, cd* x, int m, double tol, int64_t maxit, int64_t* iters,
          int64_t* restarts, double* relres) {
  const int64_t n = s.n_edges;
  *iters = 0;
  *restarts = 0;
  double bnorm = norm2(b, n);
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    return ORC_OK;
  }
  std::vector<cd> V((size_t)(m + 1) * n), w(n), z(n), r(n);
  std::vector<cd> H((size_t)(m + 1) * m), gv(m + 1), cs_s(m);
  std::vector<double> cs_c(m);
  while (true) {
    spmv(s, x, r.data());
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = norm2(r.data(), n);
    *relres = beta / bnorm;
    if (*relres <= tol) return ORC_OK;
    if (*iters >= maxit) return ORC_NOT_CONVERGED;
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    std::fill(gv.begin(), gv.end(), cd(0.0));
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m && *iters < maxit; ++j) {
      const cd* vj = &V[(size_t)j * n];
      for (int64_t i = 0; i < n; ++i) z[i] = vj[i] / s.diag[i];
      spmv(s, z.data(), w.data());
      ++*iters;
      for (int i = 0; i <= j; ++i) {
        const cd* vi = &V[(size_t)i * n];
        cd h = 0.0;
        for (int64_t l = 0; l < n; ++l) h += std::conj(vi[l]) * w[l];
        H[(size_t)i * m + j] = h;
        for (int64_t l = 0; l < n; ++l) w[l] -= h * vi[l];
      }
      double hn = norm2(w.data(), n);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (int64_t l = 0; l < n; ++l) V[(size_t)(j + 1) * n + l] = w[l] / hn;
      for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
        cd a = H[(size_t)i * m + j], c2 = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs_c[i] * a + cs_s[i] * c2;
        H[(size_t)(i + 1) * m + j] = -std::conj(cs_s[i]) * a + cs_c[i] * c2;
      }
      cd a = H[(size_t)j * m + j];
      double bb = hn, rho = std::sqrt(std::norm(a) + bb * bb);
      if (std::abs(a) == 0.0) {
        cs_c[j] = 0.0;
        cs_s[j] = 1.0;
      } else {
        cs_c[j] = std::abs(a) / rho;
        cs_s[j] = (a / std::abs(a)) * bb / rho;
      }
      H[(size_t)j * m + j] = cs_c[j] * a + cs_s[j] * bb;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -std::conj(cs_s[j]) * gv[j];
      gv[j] = cs_c[j] * gv[j];
      k = j + 1;
      if (std::abs(gv[j + 1]) / bnorm <= tol || hn == 0.0) break;
    }
    std::vector<cd> y(k);
    for (int i = k - 1; i >= 0; --i) {
      cd acc = gv[i];
      for (int l = i + 1; l < k; ++l) acc -= H[(size_t)i * m + l] * y[l];
      y[i] = acc / H[(size_t)i * m + i];
    }
    for (int64_t l = 0; l < n; ++l) {
      cd acc = 0.0;
      for (int i = 0; i < k; ++i) acc += V[(size_t)i * n + l] * y[i];
      x[l] += acc / s.diag[l];
    }
    ++*restarts;
  }
}

}  // namespace

// ============================================================================ C interface
extern "C" {

// Element matrices of one tet (Appendix B eqs. B.14-B.15): p = 4 vertices x 3 coordinates,
// S = 6 edge signs; K, M out as 6x6 row-major; vol out.
int orc_element(const double* p12, const int8_t* S, double* K, double* M, double* vol) {
  double p[4][3];
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 3; ++k) p[j][k] = p12[3 * j + k];
  Geom G;
  if (geometry(p, &G) != ORC_OK) return ORC_DEGENERATE;
  element_km(G, S, K, M);
  *vol = G.vol;
  return ORC_OK;
}

// Barycentric gradients (row i = grad lambda_i) and edge lengths of one tet.
int orc_geometry(const double* p12, double* c0, double* grads, double* len, double* vol) {
  double p[4][3];
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 3; ++k) p[j][k] = p12[3 * j + k];
  Geom G;
  if (geometry(p, &G) != ORC_OK) return ORC_DEGENERATE;
  for (int i = 0; i < 4; ++i) {
    c0[i] = G.c0[i];
    for (int k = 0; k < 3; ++k) grads[3 * i + k] = G.g[i][k];
  }
  for (int e = 0; e < 6; ++e) len[e] = G.len[e];
  *vol = G.vol;
  return ORC_OK;
}

// Primary field (Appendix A) at n points; src = (x, y, z, axis, moment); out complex [n][3].
int orc_primary_field(int64_t n, const double* pts, const double* src, double sigma_p, double freq,
                      double* out) {
  cd* E = reinterpret_cast<cd*>(out);
  for (int64_t i = 0; i < n; ++i) primary_field(&pts[3 * i], src, sigma_p, 2.0 * kPi * freq, &E[3 * i]);
  return ORC_OK;
}

// The 4-point quadrature rule (barycentric [4][4]) so tests can state what the oracle integrates with.
int orc_quadrature(double* bary16) {
  double qb[4][4];
  quad_points(qb);
  std::memcpy(bary16, qb, sizeof(qb));
  return ORC_OK;
}

// Whole forward setup: edges, boundary, element matrices, right-hand sides, CSR with Dirichlet rows.
// src = [S][5]; g = optional prescribed boundary values, complex [S][E] (NULL = E_s = 0).
void* orc_build(int64_t n_nodes, const double* nodes, int64_t n_tets, const int32_t* tets,
                const double* sigma, double sigma_p, double freq, int64_t n_src, const double* src,
                const double* g, int* status) {
  System* s = new System();
  s->n_nodes = n_nodes;
  s->n_tets = n_tets;
  s->n_src = n_src;
  s->sigma_p = sigma_p;
  s->nodes.assign(nodes, nodes + 3 * n_nodes);
  s->tets.assign(tets, tets + 4 * n_tets);
  s->src.assign(src, src + 5 * n_src);
  for (int64_t i = 0; i < 4 * n_tets; ++i)
    if (tets[i] < 0 || tets[i] >= n_nodes) {
      *status = ORC_BAD_INPUT;
      delete s;
      return nullptr;
    }
  int st = number_edges(*s);
  if (st == ORC_OK) st = find_boundary(*s);
  if (st == ORC_OK) st = assemble(*s, sigma, freq, reinterpret_cast<const cd*>(g));
  *status = st;
  if (st != ORC_OK) {
    delete s;
    return nullptr;
  }
  return s;
}

// Topology only (edges + boundary), for meshes too large to assemble on the CPU in a test.
void* orc_topology(int64_t n_nodes, int64_t n_tets, const int32_t* tets, int* status) {
  System* s = new System();
  s->n_nodes = n_nodes;
  s->n_tets = n_tets;
  s->tets.assign(tets, tets + 4 * n_tets);
  int st = number_edges(*s);
  if (st == ORC_OK) st = find_boundary(*s);
  *status = st;
  if (st != ORC_OK) {
    delete s;
    return nullptr;
  }
  return s;
}

void orc_free(void* h) { delete static_cast<System*>(h); }

int orc_sizes(void* h, int64_t* out3) {
  System* s = static_cast<System*>(h);
  out3[0] = s->n_edges;
  out3[1] = s->row_ptr.empty() ? 0 : s->row_ptr.back();
  out3[2] = s->n_src;
  return ORC_OK;
}

int orc_get_topology(void* h, int32_t* edges, int32_t* tet_edges, int8_t* signs, uint8_t* boundary) {
  System* s = static_cast<System*>(h);
  if (edges) std::memcpy(edges, s->edges.data(), s->edges.size() * sizeof(int32_t));
  if (tet_edges) std::memcpy(tet_edges, s->tet_edges.data(), s->tet_edges.size() * sizeof(int32_t));
  if (signs) std::memcpy(signs, s->signs.data(), s->signs.size());
  if (boundary) std::memcpy(boundary, s->boundary.data(), s->boundary.size());
  return ORC_OK;
}

int orc_get_system(void* h, int64_t* row_ptr, int32_t* col, double* val, double* b) {
  System* s = static_cast<System*>(h);
  if (row_ptr) std::memcpy(row_ptr, s->row_ptr.data(), s->row_ptr.size() * sizeof(int64_t));
  if (col) std::memcpy(col, s->col.data(), s->col.size() * sizeof(int32_t));
  if (val) std::memcpy(val, s->val.data(), s->val.size() * sizeof(cd));
  if (b) std::memcpy(b, s->b.data(), s->b.size() * sizeof(cd));
  return ORC_OK;
}

// Solve every source's system; x complex [S][E] is the initial guess in and the solution out.
// info = [S][3] doubles: iterations, restarts, true relative residual.
int orc_solve(void* h, int restart, double tol, int64_t maxit, double* x, double* info) {
  System* s = static_cast<System*>(h);
  cd* X = reinterpret_cast<cd*>(x);
  int worst = ORC_OK;
  for (int64_t sc = 0; sc < s->n_src; ++sc) {
    int64_t it, rs;
    double rr;
    int st = gmres(*s, &s->b[sc * s->n_edges], &X[sc * s->n_edges], restart, tol, maxit, &it, &rs, &rr);
    info[3 * sc + 0] = (double)it;
    info[3 * sc + 1] = (double)rs;
    info[3 * sc + 2] = rr;
    if (st != ORC_OK) worst = st;
  }
  return worst;
}

// y = A x for one complex vector (test helper).
int orc_spmv(void* h, const double* x, double* y) {
  System* s = static_cast<System*>(h);
  spmv(*s, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y));
  return ORC_OK;
}

// Section 3 eq. 7 at receivers.  Point location reading: the receiver belongs to the lowest-id tet
// whose barycentric coordinates are all >= -1e-12.  out complex [S][R][3 kinds][3], kinds =
// primary (sigma_p), secondary (sum_i S_i N_i x_g(i)), total = primary + secondary.
int orc_receivers(void* h, const double* x, int64_t n_rcv, const double* rx, double* out) {
  System* s = static_cast<System*>(h);
  const cd* X = reinterpret_cast<const cd*>(x);
  cd* O = reinterpret_cast<cd*>(out);
  int st_all = ORC_OK;
  for (int64_t r = 0; r < n_rcv; ++r) {
    const double* q = &rx[3 * r];
    int64_t found = -1;
    Geom G;
    double lam[4];
    for (int64_t t = 0; t < s->n_tets && found < 0; ++t) {
      double p[4][3];
      tet_points(s->nodes.data(), &s->tets[4 * t], p);
      bool maybe = true;  // cheap bounding-box rejection before the barycentric test
      for (int k = 0; k < 3 && maybe; ++k) {
        double lo = std::min(std::min(p[0][k], p[1][k]), std::min(p[2][k], p[3][k]));
        double hi = std::max(std::max(p[0][k], p[1][k]), std::max(p[2][k], p[3][k]));
        double pad = 1e-9 * (hi - lo);
        if (q[k] < lo - pad || q[k] > hi + pad) maybe = false;
      }
      if (!maybe) continue;
      if (geometry(p, &G) != ORC_OK) return ORC_DEGENERATE;
      bool in = true;
      for (int i = 0; i < 4; ++i) {
        lam[i] = G.c0[i] + dot3(G.g[i], q);
        if (lam[i] < -1e-12) in = false;
      }
      if (in) found = t;
    }
    for (int64_t sc = 0; sc < s->n_src; ++sc) {
      cd* o = &O[(sc * n_rcv + r) * 9];
      if (found < 0) {
        for (int k = 0; k < 9; ++k) o[k] = cd(NAN, NAN);
        st_all = ORC_OUTSIDE;
        continue;
      }
      cd Ep[3];
      primary_field(q, &s->src[5 * sc], s->sigma_p, s->omega, Ep);
      double N[6][3];
      basis_at(G, lam, N);
      cd Es[3] = {};
      for (int e = 0; e < 6; ++e) {
        cd xe = X[sc * s->n_edges + s->tet_edges[6 * found + e]] * (double)s->signs[6 * found + e];
        for (int k = 0; k < 3; ++k) Es[k] += N[e][k] * xe;
      }
      for (int k = 0; k < 3; ++k) {
        o[k] = Ep[k];
        o[3 + k] = Es[k];
        o[6 + k] = Ep[k] + Es[k];
      }
    }
  }
  return st_all;
}

// Dense complex LU with partial pivoting (test pin for tiny meshes): A [n][n] row-major, b [n].
int orc_dense_solve(int64_t n, const double* A_in, const double* b_in, double* x_out) {
  std::vector<cd> A(reinterpret_cast<const cd*>(A_in), reinterpret_cast<const cd*>(A_in) + n * n);
  std::vector<cd> b(reinterpret_cast<const cd*>(b_in), reinterpret_cast<const cd*>(b_in) + n);
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::abs(A[r * n + c]) > std::abs(A[piv * n + c])) piv = r;
    if (std::abs(A[piv * n + c]) == 0.0) return ORC_SINGULAR;
    if (piv != c) {
      for (int64_t k = 0; k < n; ++k) std::swap(A[piv * n + k], A[c * n + k]);
      std::swap(b[piv], b[c]);
    }
    for (int64_t r = c + 1; r < n; ++r) {
      cd f = A[r * n + c] / A[c * n + c];
      if (f == cd(0.0)) continue;
      for (int64_t k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  cd* x = reinterpret_cast<cd*>(x_out);
  for (int64_t r = n - 1; r >= 0; --r) {
    cd acc = b[r];
    for (int64_t k = r + 1; k < n; ++k) acc -= A[r * n + k] * x[k];
    x[r] = acc / A[r * n + r];
  }
  return ORC_OK;
}

}  // extern "C"
