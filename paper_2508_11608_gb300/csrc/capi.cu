// C ABI of the library (include/cutmg.h): argument checking, error
// translation, dispatch to the (dim, degree)-specialised engines.
#include <cuda_runtime.h>
#include <omp.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "../../include/cutmg.h"
#include "batch_api.hpp"
#include "engine_api.hpp"
#include "problem.hpp"
#include "setup.hpp"

using namespace cutmg;


struct cf_batch {
  std::vector<std::unique_ptr<BatchGroupBase>> groups;
  std::vector<std::vector<int>> members;  // input index of each group member
  int count = 0;
};

namespace {

thread_local std::string g_err;

cf_status fail(cf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

template <typename F>
cf_status guarded(F&& f) {
  try {
    f();
    return CF_OK;
  } catch (const std::invalid_argument& e) {
    return fail(CF_EINVAL, e.what());
  } catch (const OomError& e) {
    return fail(CF_ENOMEM, e.what());
  } catch (const std::bad_alloc&) {
    return fail(CF_ENOMEM, "host allocation failed");
  } catch (const CudaError& e) {
    return fail(CF_ECUDA, e.what());
  } catch (const TimeoutError& e) {
    return fail(CF_ETIMEOUT, e.what());
  } catch (const std::exception& e) {
    return fail(CF_EINVAL, e.what());
  }
}

bool bad_level(const cf_problem* pb, int level) {
  return !pb || level < 0 || level >= (int)pb->H.levels.size();
}

bool no_device(const cf_problem* pb) { return !pb || !pb->eng; }

bool bad_prec(int p) { return p != CF_FP64 && p != CF_MIXED; }

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

cf_status cutmg_set_error(cf_status s, const char* msg) { return fail(s, msg); }

#define CUTMG_CHECK(expr)                                                                   \
  do {                                                                                     \
    cudaError_t e__ = (expr);                                                              \
    if (e__ != cudaSuccess) throw CudaError(std::string(#expr) + ": " + cudaGetErrorString(e__)); \
  } while (0)

extern "C" {

cf_status cutmg_noalloc_engine(cf_problem* pb, EngineBase** eng, int* device) {
  if (no_device(pb)) return fail(CF_EINVAL, "null or host-only problem");
  *eng = pb->eng.get();
  *device = pb->device;
  return CF_OK;
}

const char* cf_last_error(void) { return g_err.c_str(); }

// cf_mesh / cf_levelset / cf_params -> SetupParams, with the argument checks
// of cf_setup
static cf_status translate(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                           SetupParams& prm, int& precision, int& threads) {
  if (!mesh || !ls) return fail(CF_EINVAL, "null argument");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(CF_EINVAL, "dim must be 2 or 3");
  if (degree < 1 || degree > 4) return fail(CF_EINVAL, "degree must be 1, 2, 3 or 4");
  if (mesh->dim == 3 && degree > 2) return fail(CF_EUNSUPPORTED, "dim 3 supports degree 1 and 2");
  if (mesh->n_cells < 1 || mesh->n_levels < 1) return fail(CF_EINVAL, "n_cells and n_levels must be positive");
  if (ls->kind < CF_LS_SPHERE || ls->kind > CF_LS_CALLBACK) return fail(CF_EINVAL, "unknown level-set kind");
  if (ls->kind == CF_LS_CALLBACK && (!ls->phi || !ls->grad))
    return fail(CF_EINVAL, "a callback level set needs phi and grad");
  if (ls->kind == CF_LS_SPHERE && !(ls->radius > 0.0)) return fail(CF_EINVAL, "radius must be positive");
  if ((ls->kind == CF_LS_ELLIPSOID || ls->kind == CF_LS_TORUS) && mesh->dim != 3)
    return fail(CF_EINVAL, "ellipsoid and torus level sets are three-dimensional");
  if (ls->kind == CF_LS_FLOWER && mesh->dim != 2) return fail(CF_EINVAL, "the flower level set is two-dimensional");
  if (ls->kind == CF_LS_ELLIPSOID && !(ls->axes[0] > 0 && ls->axes[1] > 0 && ls->axes[2] > 0))
    return fail(CF_EINVAL, "ellipsoid semi-axes must be positive");
  if (ls->kind == CF_LS_TORUS && !(ls->major > ls->radius && ls->radius > 0))
    return fail(CF_EINVAL, "torus radii must satisfy major > minor > 0");
  if (ls->kind == CF_LS_FLOWER && !(ls->radius > ls->amplitude && ls->amplitude >= 0 && ls->lobes >= 1))
    return fail(CF_EINVAL, "flower needs radius > amplitude >= 0 and lobes >= 1");
  prm = SetupParams();
  prm.dim = mesh->dim;
  prm.degree = degree;
  prm.n_cells = mesh->n_cells;
  prm.n_levels = mesh->n_levels;
  prm.lo = mesh->lo;
  prm.hi = mesh->hi;
  prm.gamma_D = 20.0 * degree * degree;
  prm.n_c = 2;
  prm.quad_q = degree + 2;
  precision = CF_FP64;
  if (params) {
    if (params->gamma_D > 0) prm.gamma_D = params->gamma_D;
    for (int k = 0; k < 4; ++k)
      if (params->gamma_ghost[k] > 0) prm.gamma_ghost[k] = params->gamma_ghost[k];
    if (params->n_c > 0) prm.n_c = params->n_c;
    if (params->quad_q > 0) prm.quad_q = params->quad_q;
    if (bad_prec(params->precision)) return fail(CF_EINVAL, "bad precision");
    precision = params->precision;
    if (params->smoother != CF_SMOOTHER_MVS && params->smoother != CF_SMOOTHER_CHEBYSHEV)
      return fail(CF_EINVAL, "bad smoother");
    prm.smoother = params->smoother;
    if (params->smoother_degree < 0 || params->smoother_degree > 32) return fail(CF_EINVAL, "bad smoother degree");
    if (params->smoother_degree > 0) prm.cheb_degree = params->smoother_degree;
    if (params->setup_threads < 0) return fail(CF_EINVAL, "bad setup thread count");
  }
  threads = params ? params->setup_threads : 0;
  prm.ls.kind = ls->kind;
  prm.ls.d = mesh->dim;
  for (int k = 0; k < 3; ++k) {
    prm.ls.c[k] = ls->center[k];
    prm.ls.nrm[k] = ls->normal[k];
  }
  prm.ls.r = ls->radius;
  prm.ls.off = ls->offset;
  for (int k = 0; k < 3; ++k) prm.ls.ax[k] = ls->axes[k];
  if (ls->kind == CF_LS_ELLIPSOID || ls->kind == CF_LS_TORUS)
    for (int k = 0; k < 9; ++k) prm.ls.R[k] = ls->rot[k];
  prm.ls.major = ls->major;
  prm.ls.lobes = ls->lobes;
  prm.ls.amp = ls->amplitude;
  prm.ls.phase = ls->phase;
  if (ls->kind == CF_LS_CALLBACK) {
    prm.ls.uphi = ls->phi;
    prm.ls.ugrad = ls->grad;
    prm.ls.user = ls->user;
    static std::atomic<uint64_t> epochs{0};
    prm.ls.epoch = ++epochs;
  }
  return CF_OK;
}

// the calling thread's OpenMP team size for the setup, restored on exit
struct ThreadCount {
  int saved;
  explicit ThreadCount(int n) : saved(omp_get_max_threads()) {
    if (n > 0) omp_set_num_threads(n);
  }
  ~ThreadCount() { omp_set_num_threads(saved); }
};

static cf_status setup_impl(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                            cf_problem** out, bool device, cudaStream_t stream, bool device_inverse) {
  if (!out) return fail(CF_EINVAL, "null argument");
  *out = nullptr;
  SetupParams prm;
  int precision = CF_FP64, threads = 0;
  cf_status tr = translate(mesh, ls, degree, params, prm, precision, threads);
  if (tr != CF_OK) return tr;
  prm.device_inverse = device_inverse;
  std::unique_ptr<cf_problem> pb;
  cf_status st = guarded([&] {
    ThreadCount tc(threads);
    pb.reset(new cf_problem());
    build_hierarchy(prm, pb->H);
    if (device) {
      if (cudaGetDevice(&pb->device) != cudaSuccess) throw CudaError("no CUDA device");
      pb->eng = mesh->dim == 2 ? make_engine_d2(degree, pb->H, stream) : make_engine_d3(degree, pb->H, stream);
    }
    pb->precision = precision;
  });
  if (st != CF_OK) return st;
  *out = pb.release();
  return CF_OK;
}

cf_status cf_setup(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params, void* stream,
                   cf_problem** out) {
  return setup_impl(mesh, ls, degree, params, out, true, S(stream), true);
}

cf_status cutmg_build_host(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                           cf_problem** out) {
  // the served form attaches a device right after: its inverses are formed there
  return setup_impl(mesh, ls, degree, params, out, false, nullptr, true);
}

cf_status cutmg_attach_device(cf_problem* pb, cudaStream_t stream) {
  if (!pb) return fail(CF_EINVAL, "null problem");
  if (pb->eng) return CF_OK;
  return guarded([&] {
    if (cudaGetDevice(&pb->device) != cudaSuccess) throw CudaError("no CUDA device");
    pb->eng = pb->H.prm.dim == 2 ? make_engine_d2(pb->H.prm.degree, pb->H, stream)
                                 : make_engine_d3(pb->H.prm.degree, pb->H, stream);
  });
}

// the device bytes of a hierarchy built with or without prm.dry (sizes only)
size_t cutmg_estimate_hierarchy_bytes(const Hierarchy& H) {
  // mirrors the allocations of Engine (both precisions) and its CG vectors
  const int d = H.prm.dim, p = H.prm.degree;
  size_t nb = 1;
  for (int k = 0; k < d; ++k) nb *= (size_t)(p + 1);
  const size_t nt = d == 2 ? (size_t)(p + 1) : (size_t)(p + 1) * (p + 1);
  size_t tot = 0;
  for (size_t l = 0; l < H.levels.size(); ++l) {
    const auto& L = H.levels[l];
    const size_t nbox = L.nact.size(), ncell = L.cflag.size();
    tot += ncell * 5 + nbox + L.dofs.size() * 8 + (L.bulk_pos.size() + L.bnd_node.size()) * 4;
    tot += (L.cart_vert.size() + L.cut_vert.size() * 3 + L.member_node.size() + L.fent.size() + L.fofs.size() +
            L.ghost_faces.size() + L.cfaces.size() + L.face_id.size() + L.cut_fo.size() + L.cut_cell.size() +
            L.cut_item_off.size()) * 4 + L.cut_vert.size() * 8 + L.members.size() * 2 + L.cut_items.size();
    tot += (L.pro_col.size() + L.res_col.size()) * 4;
    const size_t ncoarse = l == 0 ? L.dofs.size() * L.dofs.size() : 0;
    // cut-patch storage: explicit inverses (warp kernel) or records and the
    // boundary-face moment slots (pipelined kernel)
    const bool pipe = !L.cut_roff.empty();
    const size_t ncp = L.cut_vert.size();
    const size_t cutstore = pipe ? (size_t)L.n_rec + (size_t)(L.cut_gboff.empty() ? 0 : L.cut_gboff.back()) * p * nt
                                 : (size_t)L.n_inv;
    size_t typed = (size_t)L.n_cut * nb * nb + nb * nb + cutstore + L.pro_w.size() + L.res_w.size() +
                   ncoarse + 3 * nbox + L.members.size() + L.ghost_faces.size() * p * nt;
    if (pipe) {
      size_t words = 0;
      for (size_t j = 0; j < ncp; ++j) words += (size_t)(L.cut_item_off[j + 1] - L.cut_item_off[j] + 3) / 4;
      tot += 4 * L.members.size() + 4 * words + 8 * ncp + 4 * L.cut_pk.size() + 8 * L.cut_gmask.size() +
             8 * L.cut_roff.size() + 4 * L.cut_gboff.size() + 4 * L.bf_face.size() + 4 * L.bf_dst.size() +
             4 * L.cut_geoff.size() + 2 * L.cut_gent.size();
    }
    if (l > 0) {  // interior-patch dense map: transposed copy and the tensor-core operand (FP32 only)
      size_t nc = 1, ni = 1;
      for (int k = 0; k < d; ++k) {
        nc *= (size_t)(2 * p + 1);
        ni *= (size_t)(2 * p - 1);
      }
      const size_t np_tc = ni <= 16 ? 16 : (ni + 15) / 16 * 16;
      tot += 4 * (2 * nc * ((ni + 7) / 8 * 8) + np_tc * ((nc + 7) / 8 * 8));
    }
    if (l > 0) {
      const size_t nf = L.n, nc = H.levels[l - 1].n;
      typed += d == 3 ? nc * nf * nf + nc * nc * nf + nf * nc * nc + nf * nf * nc : 2 * nc * nf;
    }
    tot += typed * 12;  // FP64 + FP32 copies
  }
  tot += 9 * H.levels.back().nact.size() * 8 + H.levels.back().dofs.size() * 8 + 64 * 1024;
  return tot;
}

size_t cutmg_estimate_device_bytes(const cf_problem* pb) { return cutmg_estimate_hierarchy_bytes(pb->H); }

cf_status cf_setup_host(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                        cf_problem** out) {
  return setup_impl(mesh, ls, degree, params, out, false, nullptr, false);
}

void cf_destroy(cf_problem* pb) { delete pb; }

cf_status cf_footprint(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                       size_t* bytes) {
  if (!bytes) return fail(CF_EINVAL, "null argument");
  SetupParams prm;
  int precision = CF_FP64, threads = 0;
  cf_status tr = translate(mesh, ls, degree, params, prm, precision, threads);
  if (tr != CF_OK) return tr;
  prm.dry = true;
  return guarded([&] {
    ThreadCount tc(threads);
    Hierarchy H;
    build_hierarchy(prm, H);
    *bytes = cutmg_estimate_hierarchy_bytes(H);
  });
}

cf_status cf_problem_footprint(const cf_problem* pb, size_t* bytes) {
  if (!pb || !bytes) return fail(CF_EINVAL, "null argument");
  *bytes = cutmg_estimate_device_bytes(pb);
  return CF_OK;
}

int cf_n_levels(const cf_problem* pb) { return pb ? (int)pb->H.levels.size() : 0; }

int64_t cf_n_dofs(const cf_problem* pb) { return pb ? (int64_t)pb->H.levels.back().dofs.size() : 0; }

int64_t cf_level_n_dofs(const cf_problem* pb, int level) {
  return bad_level(pb, level) ? 0 : (int64_t)pb->H.levels[level].dofs.size();
}

cf_status cf_dof_lattice(const cf_problem* pb, int level, int64_t* h_idx) {
  if (bad_level(pb, level) || !h_idx) return fail(CF_EINVAL, "bad level or null output");
  const auto& d = pb->H.levels[level].dofs;
  std::memcpy(h_idx, d.data(), d.size() * sizeof(int64_t));
  return CF_OK;
}

cf_status cf_dof_coords(const cf_problem* pb, int level, double* h_xyz) {
  if (bad_level(pb, level) || !h_xyz) return fail(CF_EINVAL, "bad level or null output");
  const HostLevel& L = pb->H.levels[level];
  Poly1D b(L.p);
  for (size_t i = 0; i < L.dofs.size(); ++i) {
    int64_t t = L.dofs[i];
    for (int k = 0; k < L.d; ++k) {
      int ik = (int)(t % L.n);
      t /= L.n;
      int c = std::min(ik / L.p, L.N - 1);
      h_xyz[i * L.d + k] = L.lo + L.h * (c + b.nodes[ik - L.p * c]);
    }
  }
  return CF_OK;
}

cf_status cf_stats(const cf_problem* pb, int level, int64_t* h_out6) {
  if (bad_level(pb, level) || !h_out6) return fail(CF_EINVAL, "bad level or null output");
  const HostLevel& L = pb->H.levels[level];
  h_out6[0] = L.n_active;
  h_out6[1] = L.n_cut;
  h_out6[2] = L.n_ghost;
  h_out6[3] = (int64_t)(L.cart_vert.size() + L.cut_vert.size());
  h_out6[4] = (int64_t)L.cut_vert.size();
  h_out6[5] = (int64_t)L.inv.size();
  return CF_OK;
}

cf_status cf_work_model(const cf_problem* pb, int level, int kind, int colour, double* h_out3) {
  if (bad_level(pb, level) || !h_out3 || kind < 0 || kind > 2) return fail(CF_EINVAL, "bad argument");
  const HostLevel& L = pb->H.levels[level];
  if (colour < 0 || colour >= (1 << L.d)) return fail(CF_EINVAL, "bad colour");
  const auto& w = kind == 0 ? L.work_cart : (kind == 1 ? L.work_cut : L.work_face);
  for (int i = 0; i < 3; ++i) h_out3[i] = (colour < (int)w.size()) ? w[colour][i] : 0.0;
  return CF_OK;
}

cf_status cf_host_rhs_user(const cf_problem* pb, double (*f)(const double*, void*),
                           double (*g)(const double*, void*), void* user, double* h_b) {
  if (!pb || !h_b) return fail(CF_EINVAL, "null argument");
  return guarded([&] {
    std::vector<double> b;
    build_rhs_user(pb->H, f, g, user, b);
    std::copy(b.begin(), b.end(), h_b);
  });
}

cf_status cf_rhs_user(cf_problem* pb, double (*f)(const double*, void*), double (*g)(const double*, void*),
                      void* user, double* d_b, void* stream) {
  if (no_device(pb) || !d_b) return fail(CF_EINVAL, "null argument");
  return guarded([&] {
    std::vector<double> b;
    build_rhs_user(pb->H, f, g, user, b);
    cudaStream_t st = S(stream);
    CUTMG_CHECK(cudaMemcpyAsync(d_b, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, st));
    CUTMG_CHECK(cudaStreamSynchronize(st));
  });
}

cf_status cf_set_precision(cf_problem* pb, int precision) {
  if (!pb || bad_prec(precision)) return fail(CF_EINVAL, "bad precision");
  pb->precision = precision;
  return CF_OK;
}

cf_status cf_set_kernel_variant(cf_problem* pb, int family, int variant) {
  if (no_device(pb)) return fail(CF_EINVAL, "null or host-only problem");
  return guarded([&] { pb->eng->set_variant(family, variant); });
}

cf_status cf_set_wait_limit(cf_problem* pb, int64_t polls) {
  if (no_device(pb)) return fail(CF_EINVAL, "null or host-only problem");
  if (polls < 0 || polls > (int64_t)1 << 30) return fail(CF_EINVAL, "wait limit must be in [0, 2^30]");
  return guarded([&] { pb->eng->set_wait_limit((int)polls); });
}

cf_status cf_rhs(cf_problem* pb, double* d_b, void* stream) {
  if (no_device(pb) || !d_b) return fail(CF_EINVAL, "null argument");
  return guarded([&] { pb->eng->rhs(d_b, S(stream)); });
}

cf_status cf_apply(cf_problem* pb, const double* d_x, double* d_y, void* stream) {
  if (no_device(pb) || !d_x || !d_y) return fail(CF_EINVAL, "null argument");
  return guarded([&] { pb->eng->apply_fine(d_x, d_y, S(stream)); });
}

cf_status cf_vcycle(cf_problem* pb, const double* d_r, double* d_z, void* stream) {
  if (no_device(pb) || !d_r || !d_z) return fail(CF_EINVAL, "null argument");
  return guarded([&] { pb->eng->vcycle(pb->precision, d_r, d_z, S(stream)); });
}

cf_status cf_solve(cf_problem* pb, const double* d_b, double* d_x, double rtol, int maxit,
                   cf_info* info, void* stream) {
  if (no_device(pb) || !d_b || !d_x) return fail(CF_EINVAL, "null argument");
  if (!(rtol > 0.0) || maxit < 1) return fail(CF_EINVAL, "rtol must be positive and maxit >= 1");
  int it = 0;
  double rel = 0, trel = 0;
  float ms = 0;
  cf_status st = guarded([&] {
    it = pb->eng->solve(pb->precision, d_b, d_x, rtol, maxit, &rel, &trel, &ms, S(stream));
  });
  if (st != CF_OK) return st;
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->true_rel_residual = trel;
    info->solve_ms = ms;
  }
  if (rel > rtol) return fail(CF_ENOCONV, "CG reached maxit before the tolerance");
  return CF_OK;
}

cf_status cf_solve_vcycle(cf_problem* pb, const double* d_b, double* d_x, double rtol, int maxit,
                          cf_info* info, void* stream) {
  if (no_device(pb) || !d_b || !d_x) return fail(CF_EINVAL, "null argument");
  if (!(rtol > 0.0) || maxit < 1) return fail(CF_EINVAL, "rtol must be positive and maxit >= 1");
  int it = 0;
  double rel = 0, trel = 0;
  float ms = 0;
  cf_status st = guarded([&] {
    it = pb->eng->solve_vcycle(pb->precision, d_b, d_x, rtol, maxit, &rel, &trel, &ms, S(stream));
  });
  if (st != CF_OK) return st;
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->true_rel_residual = trel;
    info->solve_ms = ms;
  }
  if (rel > rtol) return fail(CF_ENOCONV, "the V-cycle iteration reached maxit before the tolerance");
  return CF_OK;
}

cf_status cf_solve_gmres(cf_problem* pb, const double* d_b, double* d_x, double rtol, int restart, int maxit,
                         cf_info* info, void* stream) {
  if (no_device(pb) || !d_b || !d_x) return fail(CF_EINVAL, "null argument");
  if (!(rtol > 0.0) || maxit < 1 || restart < 1) return fail(CF_EINVAL, "rtol > 0, maxit >= 1, restart >= 1");
  int it = 0;
  double rel = 0, trel = 0;
  float ms = 0;
  cf_status st = guarded([&] {
    it = pb->eng->solve_gmres(pb->precision, d_b, d_x, rtol, restart, maxit, &rel, &trel, &ms, S(stream));
  });
  if (st != CF_OK) return st;
  if (info) {
    info->iterations = it;
    info->rel_residual = rel;
    info->true_rel_residual = trel;
    info->solve_ms = ms;
  }
  if (rel > rtol) return fail(CF_ENOCONV, "GMRES reached maxit before the tolerance");
  return CF_OK;
}

cf_status cf_level_apply(cf_problem* pb, int level, int precision, const double* d_x, double* d_y,
                         void* stream) {
  if (bad_level(pb, level) || no_device(pb) || bad_prec(precision) || !d_x || !d_y) return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->level_apply(level, precision, d_x, d_y, S(stream)); });
}

cf_status cf_level_colour_step(cf_problem* pb, int level, int precision, int cut, int colour,
                               double* d_x, const double* d_b, void* stream) {
  if (bad_level(pb, level) || no_device(pb) || bad_prec(precision) || !d_x || !d_b) return fail(CF_EINVAL, "bad argument");
  if (colour < 0 || colour >= (1 << pb->H.prm.dim)) return fail(CF_EINVAL, "bad colour");
  return guarded([&] { pb->eng->level_colour(level, precision, cut, colour, d_x, d_b, S(stream)); });
}

cf_status cf_level_smooth(cf_problem* pb, int level, int precision, int post, double* d_x,
                          const double* d_b, void* stream) {
  if (bad_level(pb, level) || no_device(pb) || bad_prec(precision) || !d_x || !d_b) return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->level_smooth(level, precision, post, d_x, d_b, S(stream)); });
}

cf_status cf_level_restrict(cf_problem* pb, int level, int precision, const double* d_r_fine,
                            double* d_b_coarse, void* stream) {
  if (bad_level(pb, level) || no_device(pb) || level < 1 || bad_prec(precision) || !d_r_fine || !d_b_coarse)
    return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->level_restrict(level, precision, d_r_fine, d_b_coarse, S(stream)); });
}

cf_status cf_level_prolongate(cf_problem* pb, int level, int precision, const double* d_x_coarse,
                              double* d_x_fine, void* stream) {
  if (bad_level(pb, level) || no_device(pb) || level < 1 || bad_prec(precision) || !d_x_coarse || !d_x_fine)
    return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->level_prolongate(level, precision, d_x_coarse, d_x_fine, S(stream)); });
}

cf_status cf_coarse_solve(cf_problem* pb, int precision, const double* d_b0, double* d_x0, void* stream) {
  if (no_device(pb) || bad_prec(precision) || !d_b0 || !d_x0) return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->coarse_solve(precision, d_b0, d_x0, S(stream)); });
}


int64_t cf_launch_count(const cf_problem* pb) { return no_device(pb) ? 0 : pb->eng->launches(); }

cf_status cf_profile_start(cf_problem* pb, int kernel) { return cf_profile_start_level(pb, kernel, -1); }

cf_status cf_profile_start_level(cf_problem* pb, int kernel, int level) {
  if (no_device(pb) || kernel < 1 || kernel > 5 || level < -1 || level >= (int)pb->H.levels.size())
    return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->profile_start(kernel, level); });
}

cf_status cf_profile_read(cf_problem* pb, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (no_device(pb) || !ms || !launches || !flops || !bytes) return fail(CF_EINVAL, "bad argument");
  return guarded([&] { pb->eng->profile_read(ms, launches, flops, bytes); });
}

cf_status cf_batch_create(cf_problem* const* problems, int count, cf_batch** out) {
  if (!problems || count < 1 || !out) return fail(CF_EINVAL, "empty batch");
  *out = nullptr;
  int dev = -1;
  for (int i = 0; i < count; ++i) {
    if (no_device(problems[i])) return fail(CF_EINVAL, "null or host-only problem in batch");
    if (i == 0) dev = problems[i]->device;
    if (problems[i]->device != dev) return fail(CF_EINVAL, "problems on different devices");
  }
  std::unique_ptr<cf_batch> bt(new cf_batch());
  bt->count = count;
  cf_status st = guarded([&] {
    int grouped = 0;
    for (int dim = 2; dim <= 3; ++dim)
      for (int deg = 1; deg <= 4; ++deg) {
        std::vector<EngineBase*> inst;
        std::vector<int> idx;
        int n_c = -1;
        for (int i = 0; i < count; ++i) {
          const auto& prm = problems[i]->H.prm;
          if (prm.dim != dim || prm.degree != deg) continue;
          if (n_c >= 0 && prm.n_c != n_c) throw std::invalid_argument("n_c differs within a batch group");
          if (prm.smoother != 0) throw std::invalid_argument("the batched form runs the vertex-patch smoother only");
          n_c = prm.n_c;
          inst.push_back(problems[i]->eng.get());
          idx.push_back(i);
        }
        if (inst.empty()) continue;
        bt->groups.push_back(dim == 2 ? make_batch_group_d2(deg, inst, n_c) : make_batch_group_d3(deg, inst, n_c));
        bt->members.push_back(idx);
        grouped += (int)idx.size();
      }
    if (grouped != count) throw std::invalid_argument("a problem of the batch fits no (dim, degree) group");
    cudaStream_t s;
    CUTMG_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto& g : bt->groups) g->autotune(s);
    CUTMG_CHECK(cudaStreamSynchronize(s));
    cudaStreamDestroy(s);
  });
  if (st != CF_OK) return st;
  *out = bt.release();
  return CF_OK;
}

cf_status cf_batch_solve(cf_batch* bt, int precision, const double* const* d_b, double* const* d_x, double rtol,
                         int maxit, cf_info* infos, void* stream) {
  if (!bt || !d_b || !d_x || bad_prec(precision)) return fail(CF_EINVAL, "bad argument");
  if (!(rtol > 0.0) || maxit < 1) return fail(CF_EINVAL, "rtol must be positive and maxit >= 1");
  bool noconv = false;
  cf_status st = guarded([&] {
    cudaStream_t s = S(stream);
    cudaEvent_t e0, e1;
    CUTMG_CHECK(cudaEventCreate(&e0));
    CUTMG_CHECK(cudaEventCreate(&e1));
    CUTMG_CHECK(cudaEventRecord(e0, s));
    const size_t G = bt->groups.size();
    std::vector<std::vector<double>> bn(G), rr(G);
    for (size_t g = 0; g < G; ++g) {
      std::vector<const double*> b;
      for (int i : bt->members[g]) b.push_back(d_b[i]);
      bt->groups[g]->start(precision, b.data(), s);
      bn[g].assign(bt->members[g].size(), 0.0);
      rr[g].assign(bt->members[g].size(), 0.0);
      bt->groups[g]->bnorms(bn[g].data());
    }
    int it = 0;
    while (it < maxit) {
      bool any = false;
      for (size_t g = 0; g < G; ++g)
        if (bt->groups[g]->active() > 0) {
          bt->groups[g]->half_a(s);
          any = true;
        }
      if (!any) break;
      ++it;
      bool left = false;
      for (size_t g = 0; g < G; ++g) {
        if (bt->groups[g]->active() == 0) continue;
        bt->groups[g]->read_rr(rr[g].data(), s);
        std::vector<int> done;
        for (size_t i = 0; i < rr[g].size(); ++i)
          if (!(std::sqrt(rr[g][i]) > rtol * bn[g][i])) done.push_back((int)i);
        bt->groups[g]->deactivate(done);
        if (bt->groups[g]->active() > 0) left = true;
      }
      if (!left) break;
      for (size_t g = 0; g < G; ++g)
        if (bt->groups[g]->active() > 0) bt->groups[g]->half_b(precision, s);
    }
    CUTMG_CHECK(cudaEventRecord(e1, s));
    CUTMG_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUTMG_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t g = 0; g < G; ++g) {
      const size_t n = bt->members[g].size();
      std::vector<double*> x;
      for (int i : bt->members[g]) x.push_back(d_x[i]);
      std::vector<BatchInfo> inf(n);
      bt->groups[g]->finish(x.data(), inf.data(), s);
      for (size_t k = 0; k < n; ++k) {
        const int i = bt->members[g][k];
        if (inf[k].rel > rtol) noconv = true;
        if (infos) {
          infos[i].iterations = inf[k].iterations;
          infos[i].rel_residual = inf[k].rel;
          infos[i].true_rel_residual = inf[k].true_rel;
          infos[i].solve_ms = ms;
        }
      }
    }
  });
  if (st != CF_OK) return st;
  if (noconv) return fail(CF_ENOCONV, "a problem of the batch reached maxit before the tolerance");
  return CF_OK;
}

int64_t cf_batch_launch_count(const cf_batch* bt) {
  if (!bt) return 0;
  int64_t n = 0;
  for (auto& g : bt->groups) n += g->launches();
  return n;
}

void cf_batch_destroy(cf_batch* bt) { delete bt; }

cf_status cf_host_rhs(const cf_problem* pb, double* h_b) {
  if (!pb || !h_b) return fail(CF_EINVAL, "null argument");
  std::memcpy(h_b, pb->H.rhs.data(), pb->H.rhs.size() * sizeof(double));
  return CF_OK;
}

cf_status cf_host_cell_matrix(const cf_problem* pb, int level, int64_t cell, double* h_out) {
  if (bad_level(pb, level) || !h_out) return fail(CF_EINVAL, "bad level or null output");
  const HostLevel& L = pb->H.levels[level];
  if (cell < 0 || cell >= (int64_t)L.cflag.size() || !(L.cflag[cell] & kFlagActive))
    return fail(CF_EINVAL, "cell out of range or inactive");
  const size_t nb2 = L.Kref.size();
  const double* src = (L.cflag[cell] & kFlagCut) ? &L.cutmat[(size_t)L.cut_id[cell] * nb2] : L.Kref.data();
  std::memcpy(h_out, src, nb2 * sizeof(double));
  return CF_OK;
}

cf_status cf_host_patch_counts(const cf_problem* pb, int level, int64_t* n_interior, int64_t* n_cut) {
  if (bad_level(pb, level) || !n_interior || !n_cut) return fail(CF_EINVAL, "bad argument");
  *n_interior = (int64_t)pb->H.levels[level].cart_vert.size();
  *n_cut = (int64_t)pb->H.levels[level].cut_vert.size();
  return CF_OK;
}

cf_status cf_host_diagonal(const cf_problem* pb, int level, double* h_d) {
  if (bad_level(pb, level) || !h_d || level < 1) return fail(CF_EINVAL, "bad level or null output");
  const auto& D = pb->H.levels[level].diag;
  std::copy(D.begin(), D.end(), h_d);
  return CF_OK;
}

cf_status cf_host_coarse_inverse(const cf_problem* pb, double* h_inv) {
  if (!pb || !h_inv) return fail(CF_EINVAL, "null handle or output");
  const auto& A = pb->H.levels[0].coarse_inv;
  std::copy(A.begin(), A.end(), h_inv);
  return CF_OK;
}

cf_status cf_host_interior_update(const cf_problem* pb, int level, double* h_W) {
  if (bad_level(pb, level) || !h_W || level < 1) return fail(CF_EINVAL, "bad level or null output");
  const auto& W = pb->H.levels[level].Wcart;
  std::copy(W.begin(), W.end(), h_W);
  return CF_OK;
}

cf_status cf_host_interior_patch(const cf_problem* pb, int level, int64_t j, int64_t* vertex) {
  if (bad_level(pb, level) || !vertex) return fail(CF_EINVAL, "bad argument");
  const HostLevel& L = pb->H.levels[level];
  if (j < 0 || j >= (int64_t)L.cart_vert.size()) return fail(CF_EINVAL, "patch index out of range");
  *vertex = L.cart_vert[j];
  return CF_OK;
}

cf_status cf_host_cut_patch(const cf_problem* pb, int level, int64_t j, int64_t* vertex, int* m,
                            int64_t* h_nodes, double* h_inv) {
  if (bad_level(pb, level) || !vertex || !m || !h_nodes) return fail(CF_EINVAL, "bad argument");
  const HostLevel& L = pb->H.levels[level];
  if (j < 0 || j >= (int64_t)L.cut_vert.size()) return fail(CF_EINVAL, "patch index out of range");
  const int np = L.N + 1, C = 2 * L.p + 1;
  *vertex = L.cut_vert[j];
  *m = L.cut_n[j];
  int v[3] = {0, 0, 0};
  int64_t t = L.cut_vert[j];
  for (int k = 0; k < L.d; ++k) {
    v[k] = (int)(t % np);
    t /= np;
  }
  for (int e = 0; e < L.cut_n[j]; ++e) {
    int o = L.members[L.cut_moff[j] + e];
    int64_t node = 0, st = 1;
    for (int k = 0; k < L.d; ++k) {
      node += (int64_t)(L.p * (v[k] - 1) + o % C) * st;
      o /= C;
      st *= L.n;
    }
    h_nodes[e] = node;
  }
  if (h_inv) {
    if (!L.inv_on_device) {
      std::memcpy(h_inv, &L.inv[L.cut_ioff[j]], sizeof(double) * L.cut_n[j] * L.cut_n[j]);
    } else {
      // formed on the device: read back from the FP64 record
      if (!pb->eng) return fail(CF_EINVAL, "cut-patch inverses of this handle live on a device that was not attached");
      cf_status st = guarded([&] { pb->eng->cut_inverse(level, j, h_inv); });
      if (st != CF_OK) return st;
    }
  }
  return CF_OK;
}

}  // extern "C"
