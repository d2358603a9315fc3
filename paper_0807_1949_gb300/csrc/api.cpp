// C ABI entry points (include/vtm.h): argument checks, error codes and thread-local messages.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace vtm {
void build_partition(const vtm_csr* A, const vtm_partition_spec* spec, vtm_partition* p);
vtm_solver* create_solver(const vtm_partition* p, const vtm_setup_opts* o, void* cuda_stream);
void solver_set_rhs(vtm_solver* s, const double* b, int64_t ldb);
void reset_waves(vtm_solver* s);
void solver_iterate(vtm_solver* s, int k);
int solver_solve(vtm_solver* s, const double* b, double* x, int64_t ld, double rtol, int maxit, vtm_stats* st);
void solver_get_state(vtm_solver* s, double* waves);
void solver_set_state(vtm_solver* s, const double* waves);
void solver_get_copies(vtm_solver* s, double* out);
void solver_get_info(const vtm_solver* s, vtm_solver_info* info);
void solver_get_history(const vtm_solver* s, int32_t* count, int32_t* sweeps, double* rel, double* inner);
void solver_input_impedances(vtm_solver* s, double* r);
void line_features(const vtm_partition* p, float* out);
void line_pairs(const vtm_partition* p, std::vector<int64_t>& pairs, std::vector<double>& wts);
void element_pieces(const vtm_partition_spec* sp, int32_t* out);
void solver_get_impedances(const vtm_solver* s, double* z);
void solver_get_piece_precision(const vtm_solver* s, int32_t* bits);
vtm_mlp* mlp_create(uint64_t seed);
void mlp_set_params(vtm_mlp* m, const float* host);
void mlp_get_params(const vtm_mlp* m, float* host);
void mlp_get_grads(const vtm_mlp* m, float* host);
void mlp_forward(const vtm_mlp* m, const float* X, float* y, int64_t n, cudaStream_t st);
float mlp_loss_grad(vtm_mlp* m, const float* X, const float* t, int64_t n, cudaStream_t st);
void mlp_adam(vtm_mlp* m, float lr, float b1, float b2, float eps, cudaStream_t st);
void mlp_destroy(vtm_mlp* m);
void solver_destroy(vtm_solver* s);

static thread_local std::string g_last_error;

void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace vtm

using vtm::Error;

template <class F>
static int guarded(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    vtm::g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    vtm::g_last_error = "host allocation failed";
    return VTM_ERR_OOM;
  } catch (const std::exception& e) {
    vtm::g_last_error = e.what();
    return VTM_ERR_INVALID;
  } catch (...) {
    vtm::g_last_error = "unknown error";
    return VTM_ERR_INVALID;
  }
}

extern "C" {

int vtm_partition_evs(const vtm_csr* A, const vtm_partition_spec* spec, vtm_partition** out) {
  return guarded([&] {
    if (!out) vtm::fail(VTM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    vtm_partition* p = new vtm_partition();
    try {
      vtm::build_partition(A, spec, p);
    } catch (...) {
      delete p;
      throw;
    }
    *out = p;
    return VTM_OK;
  });
}

int vtm_rcb(const double* coords, int64_t n, int32_t dim, int32_t nparts, int32_t* out) {
  return guarded([&] {
    if (!coords || !out || n < 1 || dim < 1 || dim > 3 || nparts < 1 || nparts > n)
      vtm::fail(VTM_ERR_INVALID, "vtm_rcb: bad arguments");
    vtm_partition_spec sp{};
    sp.nelem = n;
    sp.elem_coords = coords;
    sp.coord_dim = dim;
    sp.npieces = nparts;
    vtm::element_pieces(&sp, out);
    return VTM_OK;
  });
}

int vtm_partition_get_info(const vtm_partition* p, vtm_partition_info* info) {
  return guarded([&] {
    if (!p || !info) vtm::fail(VTM_ERR_INVALID, "null argument");
    info->n = p->n;
    info->npieces = p->npieces;
    info->ncopies = p->piece_ptr.empty() ? 0 : p->piece_ptr.back();
    info->nlines = (int64_t)p->line_a.size();
    info->nboundary = p->nboundary;
    int64_t mx = 0;
    for (int32_t j = 0; j < p->npieces; ++j) mx = std::max(mx, p->piece_ptr[j + 1] - p->piece_ptr[j]);
    info->max_piece = mx;
    return VTM_OK;
  });
}

int vtm_partition_get_piece(const vtm_partition* p, int32_t j, int64_t* n_j, int64_t* nnz_j, int64_t* vertices,
                            double* shares, int64_t* rowptr, int32_t* col, double* val) {
  return guarded([&] {
    if (!p || j < 0 || j >= p->npieces) vtm::fail(VTM_ERR_INVALID, "bad partition or piece index");
    const int64_t c0 = p->piece_ptr[j], c1 = p->piece_ptr[j + 1];
    const int64_t k0 = p->l_rowptr[c0], k1 = p->l_rowptr[c1];
    if (n_j) *n_j = c1 - c0;
    if (nnz_j) *nnz_j = k1 - k0;
    if (vertices) std::memcpy(vertices, p->copy_vertex.data() + c0, (c1 - c0) * sizeof(int64_t));
    if (shares) std::memcpy(shares, p->copy_share.data() + c0, (c1 - c0) * sizeof(double));
    if (rowptr)
      for (int64_t c = c0; c <= c1; ++c) rowptr[c - c0] = p->l_rowptr[c] - k0;
    if (col) std::memcpy(col, p->l_col.data() + k0, (k1 - k0) * sizeof(int32_t));
    if (val) std::memcpy(val, p->l_val.data() + k0, (k1 - k0) * sizeof(double));
    return VTM_OK;
  });
}

int vtm_partition_get_lines(const vtm_partition* p, int64_t* quads) {
  return guarded([&] {
    if (!p || !quads) vtm::fail(VTM_ERR_INVALID, "null argument");
    auto piece_of = [&](int64_t c) {
      return (int64_t)(std::upper_bound(p->piece_ptr.begin(), p->piece_ptr.end(), c) - p->piece_ptr.begin() - 1);
    };
    for (size_t t = 0; t < p->line_a.size(); ++t) {
      const int64_t a = p->line_a[t], b = p->line_b[t];
      const int64_t ja = piece_of(a), jb = piece_of(b);
      quads[4 * t + 0] = ja;
      quads[4 * t + 1] = a - p->piece_ptr[ja];
      quads[4 * t + 2] = jb;
      quads[4 * t + 3] = b - p->piece_ptr[jb];
    }
    return VTM_OK;
  });
}

int vtm_partition_line_pairs(const vtm_partition* p, int64_t* count, int64_t* pairs, double* weights) {
  return guarded([&] {
    if (!p || !count) vtm::fail(VTM_ERR_INVALID, "null argument");
    std::vector<int64_t> pr;
    std::vector<double> w;
    vtm::line_pairs(p, pr, w);
    *count = (int64_t)w.size();
    if (pairs) std::copy(pr.begin(), pr.end(), pairs);
    if (weights) std::copy(w.begin(), w.end(), weights);
    return VTM_OK;
  });
}

void vtm_partition_destroy(vtm_partition* p) { delete p; }

int vtm_setup(const vtm_partition* p, const vtm_setup_opts* opts, void* cuda_stream, vtm_solver** out) {
  return guarded([&] {
    if (!out) vtm::fail(VTM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    // load the allocation-free residual's scratch now, while the caller can still allocate
    vtm::noalloc_prepare_current_device();
    *out = vtm::create_solver(p, opts, cuda_stream);
    return VTM_OK;
  });
}

int vtm_solver_get_info(const vtm_solver* s, vtm_solver_info* info) {
  return guarded([&] {
    if (!s || !info) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::solver_get_info(s, info);
    return VTM_OK;
  });
}

int vtm_solver_get_history(const vtm_solver* s, int32_t* count, int32_t* sweeps, double* rel, double* inner) {
  return guarded([&] {
    if (!s || !count) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::solver_get_history(s, count, sweeps, rel, inner);
    return VTM_OK;
  });
}

void vtm_solver_destroy(vtm_solver* s) {
  if (s) vtm::solver_destroy(s);
}

int vtm_set_rhs(vtm_solver* s, const double* b, int64_t ldb) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_set_rhs(s, b, ldb);
    return VTM_OK;
  });
}

int vtm_reset(vtm_solver* s) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::reset_waves(s);
    return VTM_OK;
  });
}

int vtm_iterate(vtm_solver* s, int32_t sweeps) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_iterate(s, sweeps);
    return VTM_OK;
  });
}

int vtm_solve(vtm_solver* s, const double* b, double* x, int64_t ld, double rtol, int32_t maxit, vtm_stats* st) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    return vtm::solver_solve(s, b, x, ld, rtol, maxit, st);
  });
}

int vtm_input_impedances(vtm_solver* s, double* r_in) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_input_impedances(s, r_in);
    return VTM_OK;
  });
}

int vtm_solver_get_impedances(const vtm_solver* s, double* z_lines) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_get_impedances(s, z_lines);
    return VTM_OK;
  });
}

int vtm_solver_get_piece_precision(const vtm_solver* s, int32_t* bits) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_get_piece_precision(s, bits);
    return VTM_OK;
  });
}

int vtm_get_state(vtm_solver* s, double* waves) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_get_state(s, waves);
    return VTM_OK;
  });
}

int vtm_set_state(vtm_solver* s, const double* waves) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_set_state(s, waves);
    return VTM_OK;
  });
}

int vtm_get_copies(vtm_solver* s, double* copies) {
  return guarded([&] {
    if (!s) vtm::fail(VTM_ERR_INVALID, "null solver");
    vtm::solver_get_copies(s, copies);
    return VTM_OK;
  });
}

int vtm_line_features(const vtm_partition* p, float* feats) {
  return guarded([&] {
    if (!p || !feats) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::line_features(p, feats);
    return VTM_OK;
  });
}

int vtm_mlp_create(uint64_t seed, vtm_mlp** out) {
  return guarded([&] {
    if (!out) vtm::fail(VTM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    *out = vtm::mlp_create(seed);
    return VTM_OK;
  });
}

void vtm_mlp_destroy(vtm_mlp* m) {
  if (m) vtm::mlp_destroy(m);
}

int vtm_mlp_get_params(const vtm_mlp* m, float* params) {
  return guarded([&] {
    if (!m || !params) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::mlp_get_params(m, params);
    return VTM_OK;
  });
}

int vtm_mlp_set_params(vtm_mlp* m, const float* params) {
  return guarded([&] {
    if (!m || !params) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::mlp_set_params(m, params);
    return VTM_OK;
  });
}

int vtm_mlp_get_grads(const vtm_mlp* m, float* grads) {
  return guarded([&] {
    if (!m || !grads) vtm::fail(VTM_ERR_INVALID, "null argument");
    vtm::mlp_get_grads(m, grads);
    return VTM_OK;
  });
}

int vtm_mlp_forward(const vtm_mlp* m, const float* X, float* y, int64_t n, void* cuda_stream) {
  return guarded([&] {
    if (!m || (n > 0 && (!X || !y)) || n < 0) vtm::fail(VTM_ERR_INVALID, "bad argument");
    vtm::mlp_forward(m, X, y, n, static_cast<cudaStream_t>(cuda_stream));
    return VTM_OK;
  });
}

int vtm_mlp_loss_grad(vtm_mlp* m, const float* X, const float* target, int64_t n, float* loss, void* cuda_stream) {
  return guarded([&] {
    if (!m || !X || !target || n <= 0) vtm::fail(VTM_ERR_INVALID, "bad argument");
    const float l = vtm::mlp_loss_grad(m, X, target, n, static_cast<cudaStream_t>(cuda_stream));
    if (loss) *loss = l;
    return VTM_OK;
  });
}

int vtm_mlp_adam_step(vtm_mlp* m, float lr, float beta1, float beta2, float eps, void* cuda_stream) {
  return guarded([&] {
    if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
      vtm::fail(VTM_ERR_INVALID, "bad Adam hyper-parameters");
    vtm::mlp_adam(m, lr, beta1, beta2, eps, static_cast<cudaStream_t>(cuda_stream));
    return VTM_OK;
  });
}

const char* vtm_last_error(void) { return vtm::g_last_error.c_str(); }

int vtm_version(void) { return VTM_VERSION_MAJOR * 100 + VTM_VERSION_MINOR; }

}  // extern "C"
