// Served form: a stream of solve requests with arrival times, solved with
// continuous batching on one GPU.
//
//  * A pool of host workers builds the requests' hierarchies (classification,
//    cut quadrature, cell and patch matrices), each once its request has
//    arrived, in arrival order and at most kLookahead requests ahead of
//    admission; the workers share the host cores (one setup alone scales
//    sublinearly with threads, so concurrent setups raise the rate).  A
//    setup takes the cores no other running setup holds, at least its share
//    of them, so a request that arrives alone is built on every core.
//  * Admission (FIFO): a prepared request enters as soon as its device
//    footprint (estimated before its setup by cf_footprint) fits the HBM budget next to
//    the resident problems and an active slot is free; its hierarchy is
//    uploaded and its CG is started (x = 0, r = b, z = B r, p = z).
//  * Every tick runs one CG iteration for all active problems together: each
//    step of the V-cycle and of CG is one launch over all of them (the batched
//    kernels), so requests that arrive while others run share the device.
//  * A problem whose residual reaches its tolerance (or maxit) retires at once:
//    its true residual is computed, its solution copied to the host if asked,
//    its device memory freed for the next admissions.
// A problem performs the same floating-point operations whether it runs
// alone or in the mix (the batched kernels reuse the single-problem device
// code and reduction partitions).
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cutmg.h"
#include "batch_api.hpp"
#include "problem.hpp"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kLookahead = 8;
constexpr int kMaxSetupWorkers = 4;  // host setups built concurrently
constexpr int kThreadsPerSetup = 4;

struct Request {
  int64_t id = 0;
  cf_mesh mesh{};
  cf_levelset ls{};
  int degree = 2;
  cf_params params{};
  double rtol = 1e-8;
  int maxit = 500;
  double arrival = 0.0;  // seconds after cf_server_run starts
  // state
  int state = 0;  // 0 waiting, 1 prepared, 2 active, 3 done, -1 failed
  cf_problem* pb = nullptr;
  double* d_b = nullptr;
  double* d_x = nullptr;
  size_t bytes = 0;
  double bn = 0.0;
  int iterations = 0;
  double rel = 0.0, true_rel = 0.0;
  double t_admit = 0.0, t_done = 0.0;
  int64_t ndof = 0;
  std::vector<double> x;
  std::string error;
};

}  // namespace

struct cf_server {
  size_t budget = 0;
  int max_active = 64;
  int precision = CF_FP64;
  int keep = 0;
  std::vector<Request> reqs;
  size_t peak_bytes = 0;
  int peak_active = 0;
  int64_t ticks = 0;
  double run_s = 0.0;
};

namespace cutmg {
std::unique_ptr<BatchGroupBase> make_batch_group_d2(int degree, const std::vector<EngineBase*>& inst, int n_c);
std::unique_ptr<BatchGroupBase> make_batch_group_d3(int degree, const std::vector<EngineBase*>& inst, int n_c);
}  // namespace cutmg

extern "C" {

cf_status cf_server_create(size_t hbm_budget_bytes, int max_active, int precision, int keep_solutions,
                           cf_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_active < 1 || (precision != CF_FP64 && precision != CF_MIXED))
    return cutmg_set_error(CF_EINVAL, "bad server parameters");
  cf_server* s = new cf_server();
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->precision = precision;
  s->keep = keep_solutions;
  *out = s;
  return CF_OK;
}

void cf_server_destroy(cf_server* s) {
  if (!s) return;
  for (auto& r : s->reqs) {
    if (r.d_b) cudaFree(r.d_b);
    if (r.d_x) cudaFree(r.d_x);
    cf_destroy(r.pb);
  }
  delete s;
}

cf_status cf_server_submit(cf_server* s, const cf_mesh* mesh, const cf_levelset* ls, int degree,
                           const cf_params* params, double rtol, int maxit, double arrival_s, int64_t* id) {
  if (!s || !mesh || !ls || !(rtol > 0.0) || maxit < 1 || !(arrival_s >= 0.0))
    return cutmg_set_error(CF_EINVAL, "bad request");
  Request r;
  r.id = (int64_t)s->reqs.size();
  r.mesh = *mesh;
  r.ls = *ls;
  r.degree = degree;
  if (params) r.params = *params;
  r.rtol = rtol;
  r.maxit = maxit;
  r.arrival = arrival_s;
  if (!s->reqs.empty() && arrival_s < s->reqs.back().arrival)
    return cutmg_set_error(CF_EINVAL, "requests must be submitted in arrival order");
  s->reqs.push_back(std::move(r));
  if (id) *id = s->reqs.back().id;
  return CF_OK;
}

cf_status cf_server_run(cf_server* s, void* stream) {
  if (!s) return cutmg_set_error(CF_EINVAL, "null server");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)s->reqs.size();
  if (n == 0) return CF_OK;
  std::mutex mu;
  std::condition_variable cv;
  int admitted = 0;  // requests taken off the prepared queue (admitted or failed)
  bool stop = false;
  const auto t0 = Clock::now();
  auto now = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };

  // host workers: each claims the next request in arrival order, at most
  // kLookahead ahead of admission, and builds its hierarchy after arrival
  const int hw = std::max(1, (int)std::thread::hardware_concurrency());
  const int nworkers = std::max(1, std::min(kMaxSetupWorkers, hw / kThreadsPerSetup));
  const int threads_each = std::max(1, hw / nworkers);
  int claimed = 0;
  int threads_busy = 0;  // OpenMP threads of the setups in progress
  auto work = [&] {
    omp_set_num_threads(threads_each);
    for (;;) {
      int i;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || claimed >= n || claimed - admitted < kLookahead; });
        if (stop || claimed >= n) return;
        i = claimed++;
      }
      Request& r = s->reqs[i];
      const double wait = r.arrival - now();
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
      cf_params prm = r.params;
      int mine = 0;
      if (prm.setup_threads == 0) {  // the caller left the thread count open
        std::lock_guard<std::mutex> lk(mu);
        mine = std::max(threads_each, hw - threads_busy);
        threads_busy += mine;
        prm.setup_threads = mine;
      }
      // admission estimate before the setup (cf_footprint: sizes only, no
      // quadrature, matrices or inverses); a request that can never fit is
      // refused without building it
      size_t est = 0;
      cf_problem* pb = nullptr;
      cf_status rc = cf_footprint(&r.mesh, &r.ls, r.degree, &prm, &est);
      std::string why;
      if (rc == CF_OK && est > s->budget) {
        rc = CF_ENOMEM;
        why = "device footprint exceeds the server's HBM budget";
      } else if (rc == CF_OK) {
        rc = cutmg_build_host(&r.mesh, &r.ls, r.degree, &prm, &pb);
      }
      if (rc != CF_OK && why.empty()) why = cf_last_error();
      std::lock_guard<std::mutex> lk(mu);
      threads_busy -= mine;
      if (rc != CF_OK) {
        r.state = -1;
        r.error = why;
      } else {
        r.pb = pb;
        r.bytes = est;
        r.state = 1;
      }
      cv.notify_all();
    }
  };
  std::vector<std::thread> workers;
  for (int w = 0; w < nworkers; ++w) workers.emplace_back(work);

  cf_status result = CF_OK;
  std::vector<int> active;
  std::vector<std::unique_ptr<cutmg::BatchGroupBase>> groups;
  std::vector<std::vector<int>> gmem;
  bool regroup = true;
  size_t used = 0;
  int next = 0, done = 0, tile_w = 0, tile_b = 0;
  try {
    while (done < n) {
      // admissions (FIFO)
      while (next < n) {
        Request& r = s->reqs[next];
        {
          std::unique_lock<std::mutex> lk(mu);
          if (r.state == 0) {
            if (!active.empty()) break;
            cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
          }
        }
        if (r.state == -1) {
          ++next;
          ++done;
          std::lock_guard<std::mutex> lk(mu);
          ++admitted;
          cv.notify_all();
          continue;
        }
        if ((int)active.size() >= s->max_active) break;
        if (used + r.bytes > s->budget) {
          if (active.empty()) {  // never fits: fail this request
            r.state = -1;
            r.error = "device footprint exceeds the server's HBM budget";
            cf_destroy(r.pb);
            r.pb = nullptr;
            ++next;
            ++done;
            std::lock_guard<std::mutex> lk(mu);
            ++admitted;
            cv.notify_all();
            continue;
          }
          break;
        }
        cf_status rc = cutmg_attach_device(r.pb, st);
        if (rc != CF_OK) throw cutmg::CudaError(cf_last_error());
        r.ndof = cf_n_dofs(r.pb);
        if (cudaMalloc(&r.d_b, sizeof(double) * std::max<int64_t>(1, r.ndof)) != cudaSuccess ||
            cudaMalloc(&r.d_x, sizeof(double) * std::max<int64_t>(1, r.ndof)) != cudaSuccess)
          throw cutmg::OomError("request vectors");
        used += r.pb->eng->device_bytes() + 2 * sizeof(double) * r.ndof;
        s->peak_bytes = std::max(s->peak_bytes, used);
        r.pb->eng->rhs(r.d_b, st);
        r.bn = r.pb->eng->cg_begin(s->precision, r.d_b, st);
        r.t_admit = now();
        r.state = 2;
        if (!(r.bn > 0.0)) {  // zero right-hand side: x = 0
          r.true_rel = 0.0;
          r.pb->eng->cg_end(r.d_x, st);
          r.state = 3;
          r.t_done = now();
          ++done;
        } else {
          active.push_back(next);
          regroup = true;
        }
        ++next;
        std::lock_guard<std::mutex> lk(mu);
        ++admitted;
        cv.notify_all();
      }
      if (active.empty()) continue;
      s->peak_active = std::max<int>(s->peak_active, (int)active.size());
      if (regroup) {
        groups.clear();
        gmem.clear();
        for (int dim = 2; dim <= 3; ++dim)
          for (int deg = 1; deg <= 4; ++deg) {
            std::vector<cutmg::EngineBase*> inst;
            std::vector<int> mem;
            int n_c = -1;
            for (int i : active) {
              const auto& prm = s->reqs[i].pb->H.prm;
              if (prm.dim != dim || prm.degree != deg) continue;
              if (n_c >= 0 && prm.n_c != n_c) throw std::invalid_argument("n_c differs within a group");
              n_c = prm.n_c;
              inst.push_back(s->reqs[i].pb->eng.get());
              mem.push_back(i);
            }
            if (inst.empty()) continue;
            groups.push_back(dim == 2 ? cutmg::make_batch_group_d2(deg, inst, n_c)
                                      : cutmg::make_batch_group_d3(deg, inst, n_c));
            if (tile_w == 0) {
              groups.back()->autotune(st);
              groups.back()->get_tile(&tile_w, &tile_b);
            } else {
              groups.back()->set_tile(tile_w, tile_b);
            }
            gmem.push_back(mem);
          }
        regroup = false;
      }
      // one CG iteration for every active problem
      ++s->ticks;
      for (auto& g : groups)
        if (g->active() > 0) g->half_a(st);
      std::vector<int> retire;
      for (size_t g = 0; g < groups.size(); ++g) {
        if (groups[g]->active() == 0) continue;
        std::vector<double> rr(gmem[g].size());
        groups[g]->read_rr(rr.data(), st);
        std::vector<int> fin;
        for (size_t k = 0; k < gmem[g].size(); ++k) {
          Request& r = s->reqs[gmem[g][k]];
          if (r.state != 2) continue;
          r.iterations += 1;
          r.rel = std::sqrt(rr[k]) / r.bn;
          if (!(r.rel > r.rtol) || r.iterations >= r.maxit) {
            fin.push_back((int)k);
            retire.push_back(gmem[g][k]);
          }
        }
        groups[g]->deactivate(fin);
      }
      for (auto& g : groups)
        if (g->active() > 0) g->half_b(s->precision, st);
      for (int i : retire) {
        Request& r = s->reqs[i];
        r.true_rel = r.pb->eng->cg_end(r.d_x, st) / r.bn;
        if (s->keep) {
          r.x.resize(r.ndof);
          cudaMemcpyAsync(r.x.data(), r.d_x, sizeof(double) * r.ndof, cudaMemcpyDeviceToHost, st);
          cudaStreamSynchronize(st);
        }
        r.t_done = now();
        r.state = 3;
        used -= r.pb->eng->device_bytes() + 2 * sizeof(double) * r.ndof;
        cudaFree(r.d_b);
        cudaFree(r.d_x);
        r.d_b = r.d_x = nullptr;
        cf_destroy(r.pb);
        r.pb = nullptr;
        active.erase(std::find(active.begin(), active.end(), i));
        ++done;
        regroup = true;
      }
      if (!retire.empty()) groups.clear();
    }
  } catch (const std::exception& e) {
    result = cutmg_set_error(CF_ECUDA, e.what());
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
    cv.notify_all();
  }
  for (auto& w : workers) w.join();
  s->run_s = now();
  return result;
}

cf_status cf_server_result(const cf_server* s, int64_t id, cf_info* info, double* times3, int64_t* ndof,
                           double* h_x) {
  if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return cutmg_set_error(CF_EINVAL, "bad request id");
  const Request& r = s->reqs[id];
  if (r.state == -1) return cutmg_set_error(CF_EINVAL, ("request failed: " + r.error).c_str());
  if (r.state != 3) return cutmg_set_error(CF_EINVAL, "request not finished");
  if (info) {
    info->iterations = r.iterations;
    info->rel_residual = r.rel;
    info->true_rel_residual = r.true_rel;
    info->solve_ms = 1e3 * (r.t_done - r.t_admit);
  }
  if (times3) {
    times3[0] = r.arrival;
    times3[1] = r.t_admit;
    times3[2] = r.t_done;
  }
  if (ndof) *ndof = r.ndof;
  if (h_x) {
    if (!s->keep) return cutmg_set_error(CF_EINVAL, "solutions were not kept");
    std::copy(r.x.begin(), r.x.end(), h_x);
  }
  return CF_OK;
}

cf_status cf_server_stats(const cf_server* s, double* out4) {
  if (!s || !out4) return cutmg_set_error(CF_EINVAL, "bad argument");
  out4[0] = (double)s->peak_bytes;
  out4[1] = (double)s->peak_active;
  out4[2] = (double)s->ticks;
  out4[3] = s->run_s;
  return CF_OK;
}

}  // extern "C"
