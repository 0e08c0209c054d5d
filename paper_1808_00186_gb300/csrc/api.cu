// C ABI of the petgem library (declared in include/petgem.h).  Argument checking, context
// lifetime, error reporting and the per-kernel timers; the stages themselves live in
// topology.cu, assembly.cu, krylov.cu and receivers.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ctx.cuh"
#include "learned.cuh"

namespace petgem {

KernelTimer::KernelTimer(petgem_ctx* ctx, const char* nm, double b, int it, int ps)
    : c(ctx), name(nm), bytes(b), iter(it), pass(ps) {
  if (!c->profiling) return;
  for (cudaEvent_t* e : {&e0, &e1}) {
    if (!c->event_pool.empty()) {
      *e = c->event_pool.back();
      c->event_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      *e = nullptr;
    }
  }
  if (e0 && e1) cudaEventRecord(e0, c->stream);
}

KernelTimer::~KernelTimer() {
  if (!c->profiling || !e0 || !e1) return;
  cudaEventRecord(e1, c->stream);
  c->pending.push_back(PendingTiming{name, e0, e1, bytes, iter, pass});
}

void set_last_timing_bytes(petgem_ctx* c, double bytes) {
  if (c->profiling && !c->pending.empty()) c->pending.back().bytes = bytes;
}

void drop_idle_timings(petgem_ctx* c, size_t from, int k, const uint8_t* refined) {
  std::vector<PendingTiming> keep(c->pending.begin(), c->pending.begin() + std::min(from, c->pending.size()));
  for (size_t i = from; i < c->pending.size(); ++i) {
    const PendingTiming& p = c->pending[i];
    bool idle = p.iter >= 0 && (p.iter >= k || (p.pass == 1 && !refined[p.iter]));
    if (idle) {
      c->event_pool.push_back(p.start);
      c->event_pool.push_back(p.stop);
    } else {
      keep.push_back(p);
    }
  }
  c->pending.swap(keep);
}

Status resolve_timings(petgem_ctx* c) {
  for (auto& p : c->pending) {
    PG_CUDA(cudaEventSynchronize(p.stop));
    float ms = 0.f;
    PG_CUDA(cudaEventElapsedTime(&ms, p.start, p.stop));
    KernelStat& k = c->stats[p.name];
    k.launches++;
    k.ms += ms;
    k.bytes += p.bytes;
    c->event_pool.push_back(p.start);
    c->event_pool.push_back(p.stop);
  }
  c->pending.clear();
  return Status{};
}

Status check_flags(petgem_ctx* c, const char* where) {
  uint32_t f = 0;
  PG_CUDA(cudaMemcpyAsync(&f, c->flags.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  PG_CUDA(cudaStreamSynchronize(c->stream));
  if (f & (kFlagBadNode | kFlagRepeatedNode | kFlagNonManifold))
    return Status{PETGEM_ERR_BAD_MESH,
                  std::string(where) + ": " +
                      ((f & kFlagBadNode)        ? "node id out of range"
                       : (f & kFlagRepeatedNode) ? "a tet repeats a node"
                                                 : "a face is shared by more than two tets")};
  if (f & kFlagDegenerate) return Status{PETGEM_ERR_DEGENERATE_TET, std::string(where) + ": a tet has zero volume"};
  return Status{};
}

}  // namespace petgem

using petgem::Status;

namespace {

int finish(petgem_ctx* c, const Status& s) {
  if (c) c->last_error = s.ok() ? std::string() : s.msg;
  return s.code;
}

Status set_device(petgem_ctx* c) {
  PG_CUDA(cudaSetDevice(c->device));
  return Status{};
}

#define PG_CUDA_S(st, call)                                                            \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) st = Status{PETGEM_ERR_CUDA, cudaGetErrorString(e_)};       \
  } while (0)

}  // namespace

extern "C" {

int petgem_create(petgem_ctx** out, int device, void* cuda_stream) {
  if (!out) return PETGEM_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PETGEM_ERR_CUDA;
  }
  petgem_ctx* c = new (std::nothrow) petgem_ctx();
  if (!c) return PETGEM_ERR_OUT_OF_MEMORY;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  Status s = set_device(c);
  if (s.ok()) s = c->flags.reserve(sizeof(uint32_t));
  if (!s.ok()) {
    delete c;
    return s.code;
  }
  *out = c;
  return PETGEM_OK;
}

int petgem_destroy(petgem_ctx* c) {
  if (!c) return PETGEM_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  petgem::destroy_solver(c);
  petgem::destroy_cocg(c);
  petgem::destroy_ssor(c);
  delete c->net;
  c->net = nullptr;
  c->slots.release();
  for (petgem::DevBuf* b : {&c->nodes, &c->tets, &c->edges, &c->tet_edges, &c->signs, &c->boundary, &c->occ, &c->eptr,
                            &c->row_ptr, &c->col, &c->gptr, &c->pkey, &c->pij, &c->flags, &c->sigma, &c->K21, &c->M21,
                            &c->vol, &c->val, &c->diag, &c->b, &c->kval, &c->mval, &c->sell_perm, &c->sell_inv,
                            &c->sell_sp, &c->sell_col, &c->sell_src})
    b->release();
  for (auto& p : c->pending) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  delete c;
  return PETGEM_OK;
}

const char* petgem_status_string(int s) {
  switch (s) {
    case PETGEM_OK: return "ok";
    case PETGEM_ERR_INVALID_ARG: return "invalid argument";
    case PETGEM_ERR_BAD_MESH: return "bad mesh";
    case PETGEM_ERR_DEGENERATE_TET: return "degenerate tetrahedron";
    case PETGEM_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PETGEM_ERR_CUDA: return "CUDA error";
    case PETGEM_ERR_NOT_CONVERGED: return "not converged";
    case PETGEM_ERR_BREAKDOWN: return "Krylov breakdown";
    case PETGEM_ERR_RECEIVER_OUTSIDE: return "receiver outside the mesh";
    case PETGEM_ERR_UNSUPPORTED: return "unsupported size or option";
    case PETGEM_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* petgem_last_error(const petgem_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

int petgem_mesh_edges(petgem_ctx* c, int64_t n_nodes, const double* nodes, int64_t n_tets, const int32_t* tets,
                      int64_t* n_edges_out) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!nodes || !tets || n_nodes < 4 || n_tets < 1)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_mesh_edges: need nodes, tets, n_nodes >= 4, n_tets >= 1"});
  if (n_nodes >= (1ll << 31) || 6 * n_tets >= (1ll << 31))
    return finish(c, Status{PETGEM_ERR_UNSUPPORTED, "petgem_mesh_edges: n_nodes < 2^31 and 6 n_tets < 2^31 required"});
  Status s = set_device(c);
  if (!s.ok()) return finish(c, s);
  c->assembled = false;
  c->slots_ready = false;  // the learned preconditioner's edge map belongs to the previous mesh
  c->n_nodes = n_nodes;
  c->n_tets = n_tets;
  s = c->nodes.reserve(3 * n_nodes * sizeof(double));
  if (s.ok()) s = c->tets.reserve(4 * n_tets * sizeof(int32_t));
  if (s.ok() && cudaMemcpyAsync(c->nodes.ptr, nodes, 3 * n_nodes * sizeof(double), cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess)
    s = Status{PETGEM_ERR_CUDA, "copy of nodes failed"};
  if (s.ok() && cudaMemcpyAsync(c->tets.ptr, tets, 4 * n_tets * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess)
    s = Status{PETGEM_ERR_CUDA, "copy of tets failed"};
  if (s.ok()) s = petgem::build_topology(c);
  c->mesh_version++;
  if (!s.ok()) {
    c->n_edges = 0;
    cudaGetLastError();
    return finish(c, s);
  }
  if (n_edges_out) *n_edges_out = c->n_edges;
  return finish(c, s);
}

int petgem_get_topology(petgem_ctx* c, int32_t* edges, int32_t* tet_edges, int8_t* signs, uint8_t* boundary) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_get_topology: no mesh"});
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  if (edges && e == cudaSuccess) e = cudaMemcpyAsync(edges, c->edges.ptr, 2 * c->n_edges * 4, cudaMemcpyDeviceToDevice, s);
  if (tet_edges && e == cudaSuccess)
    e = cudaMemcpyAsync(tet_edges, c->tet_edges.ptr, 6 * c->n_tets * 4, cudaMemcpyDeviceToDevice, s);
  if (signs && e == cudaSuccess) e = cudaMemcpyAsync(signs, c->signs.ptr, 6 * c->n_tets, cudaMemcpyDeviceToDevice, s);
  if (boundary && e == cudaSuccess)
    e = cudaMemcpyAsync(boundary, c->boundary.ptr, c->n_edges, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return finish(c, Status{PETGEM_ERR_CUDA, cudaGetErrorString(e)});
  return finish(c, Status{});
}

int petgem_assemble(petgem_ctx* c, double freq_hz, const double* sigma, double sigma_p, int32_t n_src,
                    const petgem_dipole* src) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble: call petgem_mesh_edges first"});
  if (!sigma || !(freq_hz > 0.0) || !(sigma_p > 0.0) || n_src < 1 || !src)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble: need sigma, freq > 0, sigma_p > 0, n_src >= 1"});
  for (int32_t i = 0; i < n_src; ++i)
    if (src[i].axis < 0 || src[i].axis > 2 || !std::isfinite(src[i].x) || !std::isfinite(src[i].y) ||
        !std::isfinite(src[i].z) || !std::isfinite(src[i].moment))
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble: bad dipole " + std::to_string(i)});
  Status s = set_device(c);
  if (!s.ok()) return finish(c, s);
  c->freq = freq_hz;
  c->omega = 2.0 * 3.141592653589793238462643383279502884 * freq_hz;
  c->sigma_p = sigma_p;
  c->bg_layers = 0;
  c->n_src = n_src;
  c->src.assign(src, src + n_src);
  c->assembled = false;
  s = petgem::build_assembly(c, sigma);
  if (!s.ok()) cudaGetLastError();
  return finish(c, s);
}

int petgem_assemble_layered(petgem_ctx* c, double freq_hz, const double* sigma, int32_t n_layers,
                            const double* z_interfaces, const double* sigma_layers, int32_t n_src,
                            const petgem_dipole* src) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_layered: call petgem_mesh_edges first"});
  if (!sigma || !(freq_hz > 0.0) || n_src < 1 || !src || n_layers < 1 || !sigma_layers || (n_layers > 1 && !z_interfaces))
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_layered: bad arguments"});
  if (n_layers > 8) return finish(c, Status{PETGEM_ERR_UNSUPPORTED, "petgem_assemble_layered: at most 8 layers"});
  for (int32_t j = 0; j < n_layers; ++j)
    if (!(sigma_layers[j] > 0.0) || !std::isfinite(sigma_layers[j]))
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_layered: layer conductivities must be > 0"});
  for (int32_t j = 0; j + 1 < n_layers; ++j)
    if (!std::isfinite(z_interfaces[j]) || (j > 0 && !(z_interfaces[j] < z_interfaces[j - 1])))
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_layered: interfaces must decrease"});
  for (int32_t i = 0; i < n_src; ++i) {
    if (!std::isfinite(src[i].x) || !std::isfinite(src[i].y) || !std::isfinite(src[i].z) ||
        !std::isfinite(src[i].moment) || src[i].axis < 0 || src[i].axis > 2)
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_layered: bad dipole " + std::to_string(i)});
    if (src[i].axis == 2)
      return finish(c, Status{PETGEM_ERR_UNSUPPORTED, "petgem_assemble_layered: horizontal dipoles only"});
  }
  Status s = set_device(c);
  if (!s.ok()) return finish(c, s);
  c->freq = freq_hz;
  c->omega = 2.0 * 3.141592653589793238462643383279502884 * freq_hz;
  c->bg_layers = n_layers;
  for (int32_t j = 0; j < 7; ++j) c->bg_z[j] = j + 1 < n_layers ? z_interfaces[j] : 0.0;
  for (int32_t j = 0; j < 8; ++j) c->bg_sig[j] = j < n_layers ? sigma_layers[j] : 0.0;
  {  // sigma_p of the context: the conductivity of the first source's layer
    int32_t j = 0;
    while (j + 1 < n_layers && src[0].z < z_interfaces[j]) ++j;
    c->sigma_p = sigma_layers[j];
  }
  c->n_src = n_src;
  c->src.assign(src, src + n_src);
  c->assembled = false;
  s = petgem::build_assembly(c, sigma);
  if (!s.ok()) cudaGetLastError();
  return finish(c, s);
}

int petgem_assemble_frequency(petgem_ctx* c, double freq_hz, int32_t n_src, const petgem_dipole* src) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_frequency: call petgem_assemble first"});
  if (!(freq_hz > 0.0) || n_src < 1 || !src)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_frequency: need freq > 0 and n_src >= 1"});
  for (int32_t i = 0; i < n_src; ++i)
    if (src[i].axis < 0 || src[i].axis > 2 || !std::isfinite(src[i].x) || !std::isfinite(src[i].y) ||
        !std::isfinite(src[i].z) || !std::isfinite(src[i].moment))
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_assemble_frequency: bad dipole " + std::to_string(i)});
  Status s = set_device(c);
  if (!s.ok()) return finish(c, s);
  c->freq = freq_hz;
  c->omega = 2.0 * 3.141592653589793238462643383279502884 * freq_hz;
  c->n_src = n_src;
  c->src.assign(src, src + n_src);
  c->assembled = false;
  s = petgem::build_frequency(c);
  if (!s.ok()) cudaGetLastError();
  return finish(c, s);
}

int petgem_get_system(petgem_ctx* c, int64_t* nnz_out, int64_t* row_ptr, int32_t* col, void* val, void* b,
                      void* diag) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_get_system: no mesh"});
  if ((val || b || diag) && !c->assembled)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_get_system: not assembled"});
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  if (row_ptr) e = cudaMemcpyAsync(row_ptr, c->row_ptr.ptr, (c->n_edges + 1) * 8, cudaMemcpyDeviceToDevice, s);
  if (col && e == cudaSuccess) e = cudaMemcpyAsync(col, c->col.ptr, c->nnz * 4, cudaMemcpyDeviceToDevice, s);
  if (val && e == cudaSuccess) e = cudaMemcpyAsync(val, c->val.ptr, c->nnz * 16, cudaMemcpyDeviceToDevice, s);
  if (b && e == cudaSuccess) e = cudaMemcpyAsync(b, c->b.ptr, (int64_t)c->n_src * c->n_edges * 16, cudaMemcpyDeviceToDevice, s);
  if (diag && e == cudaSuccess) e = cudaMemcpyAsync(diag, c->diag.ptr, c->n_edges * 16, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return finish(c, Status{PETGEM_ERR_CUDA, cudaGetErrorString(e)});
  if (nnz_out) *nnz_out = c->nnz;
  return finish(c, Status{});
}

int petgem_get_elements(petgem_ctx* c, double* K21, double* M21, double* vol) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_get_elements: not assembled"});
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  if (K21) e = cudaMemcpyAsync(K21, c->K21.ptr, 21 * c->n_tets * 8, cudaMemcpyDeviceToDevice, s);
  if (M21 && e == cudaSuccess) e = cudaMemcpyAsync(M21, c->M21.ptr, 21 * c->n_tets * 8, cudaMemcpyDeviceToDevice, s);
  if (vol && e == cudaSuccess) e = cudaMemcpyAsync(vol, c->vol.ptr, c->n_tets * 8, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return finish(c, Status{PETGEM_ERR_CUDA, cudaGetErrorString(e)});
  return finish(c, Status{});
}

int petgem_solve(petgem_ctx* c, const petgem_solve_opts* opts, void* x, petgem_solve_info* info) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: call petgem_assemble first"});
  if (!x || !info) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: need x and info"});
  petgem_solve_opts o{};
  o.restart = 50;
  o.precision = PETGEM_PREC_C128;
  o.precond = PETGEM_PRECOND_JACOBI;
  o.batch = 1;
  o.tol = 1e-8;
  o.inner_tol = 1e-4;
  o.max_iters = 200000;
  o.orth = PETGEM_ORTH_CGS;
  o.use_graphs = 0;
  o.method = PETGEM_METHOD_GMRES;
  if (opts) o = *opts;
  if (o.method != PETGEM_METHOD_GMRES && o.method != PETGEM_METHOD_COCG && o.method != PETGEM_METHOD_SQMR)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: unknown method"});
  if (o.precond == PETGEM_PRECOND_SSOR) {
    if (o.method != PETGEM_METHOD_SQMR)
      return finish(c, Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve: SSOR preconditions SQMR only"});
    if (o.omega == 0.0) o.omega = 1.0;
    if (!(o.omega > 0.0 && o.omega < 2.0))
      return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: SSOR needs 0 < omega < 2"});
  } else if (o.method != PETGEM_METHOD_GMRES && o.precond != PETGEM_PRECOND_JACOBI) {
    return finish(c, Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve: COCG takes the Jacobi preconditioner only"});
  }
  if (!(o.tol > 0.0) || o.max_iters < 0 || (o.precision != PETGEM_PREC_C128 && o.precision != PETGEM_PREC_MIXED) ||
      (o.precond != PETGEM_PRECOND_JACOBI && o.precond != PETGEM_PRECOND_LEARNED &&
       o.precond != PETGEM_PRECOND_SSOR) ||
      !(o.inner_tol >= 0.0 && o.inner_tol < 1.0) || o.orth < 0 ||
      o.orth > PETGEM_ORTH_CGS_IFNEEDED)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: bad options"});
  if (o.precond == PETGEM_PRECOND_LEARNED && (!c->net || !c->slots_ready))
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve: learned preconditioner needs petgem_learned_create"});
  Status s = set_device(c);
  if (s.ok())
    s = o.precond == PETGEM_PRECOND_SSOR ? petgem::run_solve_ssor(c, o, static_cast<double2*>(x), info)
                                         : petgem::run_solve(c, o, static_cast<double2*>(x), info);
  if (s.code == PETGEM_ERR_CUDA || s.code == PETGEM_ERR_OUT_OF_MEMORY) cudaGetLastError();
  return finish(c, s);
}

int petgem_solve_batch(petgem_ctx* const* ctxs, int32_t n_ctx, const petgem_solve_opts* opts, void* const* x,
                       petgem_solve_info* info) {
  if (n_ctx == 0) return PETGEM_OK;
  if (!ctxs || n_ctx < 0 || !ctxs[0]) return PETGEM_ERR_INVALID_ARG;
  petgem_ctx* c0 = ctxs[0];
  if (!opts || !x || !info) return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: need opts, x and info"});
  for (int k = 0; k < n_ctx; ++k) {
    if (!ctxs[k] || !x[k]) return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: null context or x"});
    if (!ctxs[k]->assembled)
      return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: a context is not assembled"});
    if (ctxs[k]->device != c0->device)
      return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: contexts on different devices"});
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: a context twice"});
  }
  const petgem_solve_opts& o = *opts;
  if (o.method != PETGEM_METHOD_COCG)
    return finish(c0, Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve_batch: the batch solver is COCG"});
  if (o.precond != PETGEM_PRECOND_JACOBI)
    return finish(c0, Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve_batch: Jacobi preconditioner only"});
  if (o.spmv_lanes != 0 && o.spmv_lanes != 1 && o.spmv_lanes != 2 && o.spmv_lanes != 4 && o.spmv_lanes != 8)
    return finish(c0, Status{PETGEM_ERR_UNSUPPORTED, "petgem_solve_batch: spmv_lanes must be 0, 1, 2, 4 or 8"});
  if (!(o.tol > 0.0) || o.max_iters < 0 || (o.precision != PETGEM_PREC_C128 && o.precision != PETGEM_PREC_MIXED) ||
      !(o.inner_tol >= 0.0 && o.inner_tol < 1.0))
    return finish(c0, Status{PETGEM_ERR_INVALID_ARG, "petgem_solve_batch: bad options"});
  Status s = set_device(c0);
  if (s.ok())
    s = petgem::run_solve_batch(ctxs, n_ctx, o, reinterpret_cast<double2* const*>(x), info);
  if (s.code == PETGEM_ERR_CUDA || s.code == PETGEM_ERR_OUT_OF_MEMORY) cudaGetLastError();
  return finish(c0, s);
}

int petgem_spmv(petgem_ctx* c, const void* x, void* y) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled || !x || !y) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_spmv: not assembled or null"});
  Status s = set_device(c);
  if (s.ok()) s = petgem::run_spmv(c, static_cast<const double2*>(x), static_cast<double2*>(y));
  return finish(c, s);
}

int petgem_colouring(petgem_ctx* c, int32_t* colour, int32_t* n_colours, int32_t* n_rounds) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_colouring: call petgem_mesh_edges first"});
  Status s = set_device(c);
  if (s.ok()) s = petgem::ssor_colouring(c);
  if (s.ok() && colour) {
    cudaError_t e = cudaMemcpyAsync(colour, c->ss_colour.ptr, c->n_edges * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = Status{PETGEM_ERR_CUDA, cudaGetErrorString(e)};
  }
  if (s.ok() && n_colours) *n_colours = (int32_t)c->ss_off.size() - 1;
  if (s.ok() && n_rounds) *n_rounds = c->ss_rounds;
  return finish(c, s);
}

int petgem_ssor_apply(petgem_ctx* c, double omega, const void* r, void* z) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled || !r || !z) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_ssor_apply: not assembled or null"});
  if (omega == 0.0) omega = 1.0;
  if (!(omega > 0.0 && omega < 2.0)) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_ssor_apply: 0 < omega < 2"});
  if (r == z) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_ssor_apply: r and z must not alias"});
  Status s = set_device(c);
  if (s.ok()) s = petgem::run_ssor_apply(c, omega, static_cast<const double2*>(r), static_cast<double2*>(z));
  return finish(c, s);
}

int petgem_receivers(petgem_ctx* c, int32_t n_rcv, const double* rx, const void* x, void* out) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->assembled) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_receivers: call petgem_assemble first"});
  if (n_rcv < 1 || !rx || !x || !out) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_receivers: bad arguments"});
  Status s = set_device(c);
  bool outside = false;
  if (s.ok()) s = petgem::run_receivers(c, n_rcv, rx, static_cast<const double2*>(x), static_cast<double2*>(out), &outside);
  if (s.ok() && outside) s = Status{PETGEM_ERR_RECEIVER_OUTSIDE, "petgem_receivers: a receiver lies in no tet"};
  return finish(c, s);
}

int petgem_learned_create(petgem_ctx* c, int32_t nx, int32_t ny, int32_t nz) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (c->n_edges == 0 || nx < 1 || ny < 1 || nz < 1 ||
      (int64_t)(nx + 1) * (ny + 1) * (nz + 1) != c->n_nodes || (int64_t)6 * nx * ny * nz != c->n_tets)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_learned_create: mesh must be an (nx+1)(ny+1)(nz+1)-node lattice"});
  Status s = set_device(c);
  if (!s.ok()) return finish(c, s);
  if (!c->net) c->net = new petgem::nn::Net();
  if (!c->net->ready || c->net->nx != nx || c->net->ny != ny || c->net->nz != nz) {
    // new grid size: reallocate the activations, keep the parameters
    std::vector<float> keep;
    if (c->net->ready) {
      keep.resize(c->net->n_params);
      cudaMemcpy(keep.data(), c->net->params.ptr, keep.size() * sizeof(float), cudaMemcpyDeviceToHost);
    }
    s = c->net->init(c, nx, ny, nz);
    if (s.ok() && !keep.empty())
      if (cudaMemcpyAsync(c->net->params.ptr, keep.data(), keep.size() * sizeof(float), cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
        s = Status{PETGEM_ERR_CUDA, "petgem_learned_create: parameter copy failed"};
    if (s.ok()) s = c->net->pack_weights(c->stream);
    if (s.ok() && keep.empty()) cudaStreamSynchronize(c->stream);
  }
  if (s.ok()) s = c->slots.reserve(c->n_edges * sizeof(int32_t));
  if (s.ok()) {
    PG_CUDA_S(s, cudaMemsetAsync(c->net->err.ptr, 0, sizeof(int), c->stream));
    if (s.ok())
      s = petgem::nn::edge_slots(c->stream, c->edges.as<int32_t>(), c->n_edges, nx + 1, ny + 1, nz + 1,
                                 c->slots.as<int32_t>(), c->net->err.as<int>());
    int bad = 0;
    if (s.ok() && (cudaMemcpyAsync(&bad, c->net->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                   cudaStreamSynchronize(c->stream) != cudaSuccess))
      s = Status{PETGEM_ERR_CUDA, "petgem_learned_create: CUDA error"};
    if (s.ok() && bad) s = Status{PETGEM_ERR_UNSUPPORTED, "petgem_learned_create: an edge is not a lattice step"};
    cudaMemsetAsync(c->net->err.ptr, 0, sizeof(int), c->stream);
  }
  if (s.ok()) {  // lattice spacing from the first cell's corner nodes
    double p0[3], px[3], py[3], pz[3];
    const double* nd = c->nodes.as<double>();
    cudaMemcpy(p0, nd, 24, cudaMemcpyDeviceToHost);
    cudaMemcpy(px, nd + 3 * 1, 24, cudaMemcpyDeviceToHost);
    cudaMemcpy(py, nd + 3 * (int64_t)(nx + 1), 24, cudaMemcpyDeviceToHost);
    cudaMemcpy(pz, nd + 3 * (int64_t)(nx + 1) * (ny + 1), 24, cudaMemcpyDeviceToHost);
    const double hx = fabs(px[0] - p0[0]), hy = fabs(py[1] - p0[1]), hz = fabs(pz[2] - p0[2]);
    c->lattice_h = cbrt(hx * hy * hz);
  }
  c->slots_ready = s.ok();
  return finish(c, s);
}

int petgem_learned_params(petgem_ctx* c, const float* set, float* get, float* grad, int64_t* n_params) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->net || !c->net->ready) return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_learned_params: no network"});
  petgem::nn::Net* N = c->net;
  Status s = set_device(c);
  if (n_params) *n_params = N->n_params;
  if (s.ok() && set) {
    if (cudaMemcpy(N->params.ptr, set, N->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      s = Status{PETGEM_ERR_CUDA, "petgem_learned_params: copy failed"};
    if (s.ok()) s = N->pack_weights(c->stream);
    N->adam_t = 0;
    cudaMemsetAsync(N->adam_m.ptr, 0, N->n_params * sizeof(float), c->stream);
    cudaMemsetAsync(N->adam_v.ptr, 0, N->n_params * sizeof(float), c->stream);
  }
  if (s.ok() && get) {
    if (cudaMemcpyAsync(get, N->params.ptr, N->n_params * sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      s = Status{PETGEM_ERR_CUDA, "petgem_learned_params: copy failed"};
  }
  if (s.ok() && grad) {
    if (cudaMemcpyAsync(grad, N->grads.ptr, N->n_params * sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      s = Status{PETGEM_ERR_CUDA, "petgem_learned_params: copy failed"};
  }
  return finish(c, s);
}

int petgem_learned_train_step(petgem_ctx* c, int32_t n_samples, const void* x_iters, float lr, double* loss) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->net || !c->slots_ready || !c->assembled || n_samples < 1 || !x_iters || !(lr > 0.f))
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_learned_train_step: bad arguments or state"});
  petgem::nn::Net* N = c->net;
  cudaStream_t st = c->stream;
  const int64_t E = c->n_edges;
  Status s = set_device(c);
  for (petgem::DevBuf* b : {&N->rtmp, &N->dutmp, &N->wtmp, &N->gtmp})
    if (s.ok()) s = b->reserve(E * sizeof(double2));
  if (s.ok()) s = N->dvec.reserve(8 * sizeof(double));
  if (s.ok()) s = N->features(st, c->sigma.as<double>(), c->sigma_p, c->omega, c->lattice_h);
  if (s.ok() && cudaMemsetAsync(N->loss_acc.ptr, 0, sizeof(double), st) != cudaSuccess)
    s = Status{PETGEM_ERR_CUDA, "memset"};
  for (int32_t i = 0; i < n_samples && s.ok(); ++i) {
    const double2* xi = static_cast<const double2*>(x_iters) + (int64_t)i * E;
    s = petgem::nn::residual_and_error(c, xi, xi, N->rtmp.as<double2>(), N->dutmp.as<double2>());
    if (s.ok()) s = N->sample_grad(st, c, N->rtmp.as<double2>(), c->slots.as<int32_t>(), E, i > 0);
    c->launches += 70;
  }
  if (s.ok()) s = N->adam_step(st, lr, 1.f / (float)n_samples);
  if (s.ok()) s = petgem::nn::check_err(st, N->err.as<int>(), "petgem_learned_train_step");
  double l = 0.0;
  if (s.ok() && (cudaMemcpyAsync(&l, N->loss_acc.ptr, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaStreamSynchronize(st) != cudaSuccess))
    s = Status{PETGEM_ERR_CUDA, "petgem_learned_train_step: CUDA error"};
  if (loss) *loss = l / n_samples;
  return finish(c, s);
}

int petgem_learned_apply(petgem_ctx* c, const void* r, void* z) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  if (!c->net || !c->slots_ready || !c->assembled || !r || !z)
    return finish(c, Status{PETGEM_ERR_INVALID_ARG, "petgem_learned_apply: bad arguments or state"});
  petgem::nn::Net* N = c->net;
  Status s = set_device(c);
  if (s.ok()) s = N->features(c->stream, c->sigma.as<double>(), c->sigma_p, c->omega, c->lattice_h);
  if (s.ok())
    s = N->apply<double2>(c->stream, static_cast<const double2*>(r), c->slots.as<int32_t>(), c->n_edges,
                          static_cast<double2*>(z), true);
  c->launches += 20;
  if (s.ok()) s = petgem::nn::check_err(c->stream, N->err.as<int>(), "petgem_learned_apply");
  return finish(c, s);
}

int petgem_nn_conv3d(void* stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin, int32_t cout, const void* x,
                     const void* w, const float* bias, int32_t relu, void* y, int32_t y_fp32) {
  if (gx < 1 || gy < 1 || gz < 1 || !x || !w || !bias || !y) return PETGEM_ERR_INVALID_ARG;
  if (!petgem::nn::grid_fits(gx, gy, gz)) return PETGEM_ERR_UNSUPPORTED;
  if ((cin != 16 && cin != 32) || (cout != 16 && cout != 32)) return PETGEM_ERR_UNSUPPORTED;
  if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)y) & 15) return PETGEM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  __nv_bfloat16* wc = nullptr;  // the weights as the kernel's shared-memory image
  const int nw = 27 * cin * cout;
  if (cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) return PETGEM_ERR_OUT_OF_MEMORY;
  if (cudaMallocAsync((void**)&wc, nw * sizeof(__nv_bfloat16), s) != cudaSuccess) {
    cudaFreeAsync(err, s);
    return PETGEM_ERR_OUT_OF_MEMORY;
  }
  cudaMemsetAsync(err, 0, sizeof(int), s);
  Status st = petgem::nn::pack_conv_weights(s, static_cast<const __nv_bfloat16*>(w), cin, cout, wc);
  if (st.ok())
    st = petgem::nn::conv3d(s, gx, gy, gz, cin, cout, static_cast<const __nv_bfloat16*>(x), wc, bias,
                            relu != 0, y_fp32 ? nullptr : static_cast<__nv_bfloat16*>(y),
                            y_fp32 ? static_cast<float*>(y) : nullptr, err);
  if (st.ok()) st = petgem::nn::check_err(s, err, "petgem_nn_conv3d");
  cudaFreeAsync(wc, s);
  cudaFreeAsync(err, s);
  return st.code;
}

int petgem_nn_conv3d_wgrad(void* stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin, int32_t cout, const void* x,
                           const void* dy, float* dw) {
  if (gx < 1 || gy < 1 || gz < 1 || !x || !dy || !dw) return PETGEM_ERR_INVALID_ARG;
  if (!petgem::nn::grid_fits(gx, gy, gz)) return PETGEM_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t V = (int64_t)gx * gy * gz;
  const int splits = petgem::nn::wgrad_splits(V);
  int* err = nullptr;
  float* part = nullptr;
  if (cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) return PETGEM_ERR_OUT_OF_MEMORY;
  if (cudaMallocAsync((void**)&part, (size_t)splits * 27 * 32 * 32 * sizeof(float), s) != cudaSuccess) {
    cudaFreeAsync(err, s);
    return PETGEM_ERR_OUT_OF_MEMORY;
  }
  cudaMemsetAsync(err, 0, sizeof(int), s);
  Status st = petgem::nn::conv3d_wgrad(s, gx, gy, gz, cin, cout, static_cast<const __nv_bfloat16*>(x),
                                       static_cast<const __nv_bfloat16*>(dy), part, splits, dw, false, err);
  if (st.ok()) st = petgem::nn::check_err(s, err, "petgem_nn_conv3d_wgrad");
  cudaFreeAsync(part, s);
  cudaFreeAsync(err, s);
  return st.code;
}

int petgem_profile(petgem_ctx* c, int enable) {
  if (!c) return PETGEM_ERR_INVALID_ARG;
  Status s = petgem::resolve_timings(c);
  c->stats.clear();
  c->profiling = enable != 0;
  return finish(c, s);
}

int petgem_kernel_stats(petgem_ctx* c, const char* name, int64_t* launches, double* total_ms, double* bytes) {
  if (!c || !name) return PETGEM_ERR_INVALID_ARG;
  Status s = petgem::resolve_timings(c);
  if (!s.ok()) return finish(c, s);
  auto it = c->stats.find(name);
  petgem::KernelStat k = it == c->stats.end() ? petgem::KernelStat{} : it->second;
  if (launches) *launches = k.launches;
  if (total_ms) *total_ms = k.ms;
  if (bytes) *bytes = k.bytes;
  return finish(c, Status{});
}

int64_t petgem_launch_count(const petgem_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
