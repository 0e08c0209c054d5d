// Context object behind the opaque petgem_ctx handle, and the device buffer helper.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace petgem {

// Device buffer owned by the context (cudaMalloc / cudaFree; grows, never shrinks).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  Status reserve(size_t n) {
    if (n <= bytes && ptr) return Status{};
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    if (n == 0) return Status{};
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return Status{PETGEM_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(n) + " bytes failed"};
    }
    bytes = n;
    return Status{};
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Per-kernel timing while profiling is on: CUDA events around each launch on the ctx stream.
struct KernelStat {
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

struct PendingTiming {
  std::string name;
  cudaEvent_t start, stop;
  double bytes;
  int iter;   // Arnoldi step of the launch (-1: not part of a cycle)
  int pass;   // 0: runs whenever the cycle is alive, 1: only when that step re-orthogonalised
};

// Band layout of the CSR pattern for the staged block SpMM (bands.cu): bands of R consecutive
// rows, each band's sorted distinct columns (ucol, band b at off[b] .. off[b + 1]) and, per
// nonzero, its index in its band's list (lcol).
struct BandLayout {
  int64_t version = -1;  // mesh version the layout belongs to
  int64_t nb = 0;        // bands
  int max_u = 0;         // most distinct columns of one band
  DevBuf off, ucol, lcol;
};

struct Solver;  // Krylov workspaces (krylov.cu)
namespace nn {
struct Net;  // learned preconditioner (learned.cu)
}

}  // namespace petgem

struct petgem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  int64_t launches = 0;

  // ---- mesh
  int64_t n_nodes = 0, n_tets = 0, n_edges = 0, n_pairs = 0, nnz = 0;
  petgem::DevBuf nodes, tets;              // copies of the caller's arrays
  petgem::DevBuf edges, tet_edges, signs, boundary;
  petgem::DevBuf occ, eptr;                // edge occurrences sorted by (edge, slot); offsets
  petgem::DevBuf row_ptr, col, gptr, pkey, pij;  // CSR pattern and its gather map
  petgem::DevBuf flags;                    // uint32 device error word
  int64_t mesh_version = 0;                // bumped by every petgem_mesh_edges

  // ---- SELL-32 layout of the pattern, rows in edge-kind order (sell.cu)
  int64_t sell_version = -1;               // mesh version the layout belongs to
  bool sell_ok = false;                    // false: the solvers use CSR
  int64_t sell_ns = 0, sell_nnz = 0;       // slices, stored entries (with padding)
  petgem::DevBuf sell_perm, sell_inv;      // renumbered row r holds edge perm[r]; inv = perm^-1
  petgem::DevBuf sell_sp, sell_col, sell_src;  // slice offsets, columns, CSR entry per slot (-1 pad)

  // ---- multicolour SSOR (ssor.cu): colour of each row, rows grouped by colour, group offsets
  int64_t ss_version = -1;                 // mesh version the colouring belongs to
  int32_t ss_rounds = 0;                   // Jones-Plassmann rounds it took
  petgem::DevBuf ss_colour, ss_rows;
  std::vector<int64_t> ss_off;             // rows of colour k: ss_rows[ss_off[k] .. ss_off[k + 1])
  void* ssor = nullptr;                    // SSOR-SQMR workspaces

  // ---- assembly
  bool assembled = false;
  int64_t assembly_version = 0;
  double freq = 0.0, omega = 0.0, sigma_p = 1.0;
  // layered background (petgem_assemble_layered): bg_layers > 0 layers top first, their
  // interfaces (decreasing z) and conductivities; 0 = the homogeneous background sigma_p
  int32_t bg_layers = 0;
  double bg_z[7] = {0, 0, 0, 0, 0, 0, 0};
  double bg_sig[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t n_src = 0;
  std::vector<petgem_dipole> src;
  petgem::DevBuf sigma, K21, M21, vol;
  petgem::DevBuf val, diag, b;             // A (complex128), diag(A), b [n_src][E]
  petgem::DevBuf kval, mval;               // real K and M_sigma on the pattern (A = K + i w mu0 M_sigma)

  // ---- solver state (krylov.cu)
  petgem::Solver* solver = nullptr;

  // ---- staged block SpMM (bands.cu): layouts for band heights 16, 32, 64 and the autotuner's
  // choice per (mesh, rows, nonzeros, sources, value size): -1 the row-per-lane kernel, else the
  // index of the band height
  petgem::BandLayout bands[3];
  std::map<uint64_t, int> spmm_choice;

  // ---- learned preconditioner (learned.cu): network, edge -> grid slots of the current mesh
  petgem::nn::Net* net = nullptr;
  void* cocg = nullptr;  // COCG solver workspaces (cocg.cu)
  petgem::DevBuf slots;
  bool slots_ready = false;
  double lattice_h = 0.0;

  // ---- profiling
  bool profiling = false;
  std::vector<cudaEvent_t> event_pool;
  std::vector<petgem::PendingTiming> pending;
  std::map<std::string, petgem::KernelStat> stats;
};

namespace petgem {

// Timing scope: while profiling, records an event pair around the launches inside it.
struct KernelTimer {
  petgem_ctx* c;
  std::string name;
  double bytes;
  int iter, pass;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KernelTimer(petgem_ctx* ctx, const char* nm, double b, int it = -1, int ps = 0);
  ~KernelTimer();
};

// Drop the timings, recorded since pending index `from`, of cycle launches that returned at
// once: steps >= k, and second-pass launches of steps that did not re-orthogonalise.
void drop_idle_timings(petgem_ctx* c, size_t from, int k, const uint8_t* refined);

// Set the byte count of the most recent timing (for a launch whose work is known only after it).
void set_last_timing_bytes(petgem_ctx* c, double bytes);

Status resolve_timings(petgem_ctx* c);
Status check_flags(petgem_ctx* c, const char* where);

// Stages implemented in the .cu files.
Status build_topology(petgem_ctx* c);
Status build_assembly(petgem_ctx* c, const double* sigma_dev);
Status sell_prepare(petgem_ctx* c);
template <typename T> Status sell_values(petgem_ctx* c, const T* csr_val, T* out);
Status build_frequency(petgem_ctx* c);
Status build_rhs(petgem_ctx* c);
Status run_receivers(petgem_ctx* c, int32_t n_rcv, const double* rx, const double2* x, double2* out,
                     bool* outside);
Status run_solve(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info);
Status run_solve_block(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info);
Status run_solve_cocg(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info);
Status run_solve_batch(petgem_ctx* const* ctxs, int n_ctx, const petgem_solve_opts& o, double2* const* x,
                       petgem_solve_info* info);
Status run_spmv(petgem_ctx* c, const double2* x, double2* y);
// Band layout for band height kBandHeights[which] of the current mesh (bands.cu).
Status band_layout(petgem_ctx* c, int which);
// Primary field of dipole src in the context's layered background at n device points (layered.cu).
Status layered_primary(petgem_ctx* c, const petgem_dipole& src, int64_t n, const double* pts, double2* out);
Status ssor_colouring(petgem_ctx* c);
Status run_solve_ssor(petgem_ctx* c, const petgem_solve_opts& o, double2* x, petgem_solve_info* info);
Status run_ssor_apply(petgem_ctx* c, double omega, const double2* r, double2* z);
void destroy_ssor(petgem_ctx* c);
void destroy_solver(petgem_ctx* c);
void destroy_cocg(petgem_ctx* c);

}  // namespace petgem
