// C ABI of the batched ensemble (declared in include/spfc.h).
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/spfc.h"
#include "spfc_internal.h"

#include "spfc_batch.cuh"

namespace spfc {
#define SPFC_BATCH_DECL(P)                                                                                      \
  BatchClassBase* make_batch_class_##P##_small(int, const std::vector<Params>&, cudaStream_t, int*, std::string*); \
  BatchClassBase* make_batch_class_##P##_128(int, const std::vector<Params>&, cudaStream_t, int*, std::string*);   \
  BatchClassBase* make_batch_class_##P##_256(int, const std::vector<Params>&, cudaStream_t, int*, std::string*);   \
  BatchClassBase* make_batch_class_##P##_512(int, const std::vector<Params>&, cudaStream_t, int*, std::string*);
SPFC_BATCH_DECL(f32)
SPFC_BATCH_DECL(f64)
#undef SPFC_BATCH_DECL

// A class of grid size N with a batch schedule (-1: the default of the size
// and precision).
static BatchClassBase* make_class(int N, int precision, int sched, const std::vector<Params>& ps, cudaStream_t st,
                                  int* status, std::string* err) {
  const bool f64 = precision == SPFC_FP64;
  if (sched < 0) {
    if (N >= 128) sched = f64 ? 5 : (N >= 256 ? 4 : 0);
    else sched = 0;
  }
  if (!batch_schedule_valid(N, sched)) {
    *status = SPFC_EINVAL;
    *err = "batch schedule " + std::to_string(sched) + " is not compiled for N = " + std::to_string(N);
    return nullptr;
  }
  switch (N) {
    case 16: case 32: case 64:
      return f64 ? make_batch_class_f64_small(N, ps, st, status, err) : make_batch_class_f32_small(N, ps, st, status, err);
    case 128: return f64 ? make_batch_class_f64_128(sched, ps, st, status, err) : make_batch_class_f32_128(sched, ps, st, status, err);
    case 256: return f64 ? make_batch_class_f64_256(sched, ps, st, status, err) : make_batch_class_f32_256(sched, ps, st, status, err);
    case 512: return f64 ? make_batch_class_f64_512(sched, ps, st, status, err) : make_batch_class_f32_512(sched, ps, st, status, err);
    default:
      *status = SPFC_EINVAL;
      *err = "batch grid sizes must be one of 16, 32, 64, 128, 256, 512";
      return nullptr;
  }
}
}  // namespace spfc

using spfc::BatchClassBase;
using spfc::Params;
using spfc::SavScal;

struct spfc_batch_s {
  std::vector<std::unique_ptr<BatchClassBase>> classes;
  std::vector<std::pair<int, int>> where;  // run -> (class, index within class)
  std::vector<int> n;
  cudaStream_t st = nullptr, cap = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> evs;
  cudaGraphExec_t g1 = nullptr, g8 = nullptr;
  bool w_ready = false;
  int64_t points = 0;
  std::string err;

  ~spfc_batch_s() {
    if (g1) cudaGraphExecDestroy(g1);
    if (g8) cudaGraphExecDestroy(g8);
    for (auto e : evs) cudaEventDestroy(e);
    for (auto s : side) cudaStreamDestroy(s);
    if (cap) cudaStreamDestroy(cap);
  }

  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }

  // nsteps steps of every class: each class a chain of its own steps, the
  // classes as parallel branches of the graph joined once at its end (their
  // runs share nothing, so a class never waits for another between steps)
  int capture(int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(SPFC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    int rc = 0;
    const size_t nc = classes.size();
    cudaEventRecord(evs[0], cap);
    for (size_t c = 0; c < nc; ++c) cudaStreamWaitEvent(side[c], evs[0], 0);
    for (int s = 0; s < nsteps && !rc; ++s)
      for (size_t c = 0; c < nc && !rc; ++c) {
        rc = classes[c]->launch_step(side[c]);
        if (rc) err = classes[c]->err;
      }
    for (size_t c = 0; c < nc; ++c) {  // joined also after a failed launch, so that the capture ends
      cudaEventRecord(evs[1 + c], side[c]);
      cudaStreamWaitEvent(cap, evs[1 + c], 0);
    }
    e = cudaStreamEndCapture(cap, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(SPFC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SPFC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return 0;
  }
};

static thread_local std::string g_batch_create_err;

extern "C" {

int spfc_batch_create(int nruns, const int* n, const double* L, const double* eps, const double* beta, double dt,
                      int precision, void* cuda_stream, spfc_batch_t* out) {
  return spfc_batch_create_scheduled(nruns, n, L, eps, beta, dt, precision, cuda_stream, nullptr, out);
}

int spfc_batch_schedule_valid(int n, int schedule) { return spfc::batch_schedule_valid(n, schedule) ? 1 : 0; }

int spfc_batch_schedule(spfc_batch_t b, int n) {
  if (!b) return -1;
  for (auto& c : b->classes)
    if (c->N == n) return c->schedule;
  return -1;
}

int spfc_batch_create_scheduled(int nruns, const int* n, const double* L, const double* eps, const double* beta,
                                double dt, int precision, void* cuda_stream, const int* schedules,
                                spfc_batch_t* out) {
  if (!out) { g_batch_create_err = "out is NULL"; return SPFC_EINVAL; }
  *out = nullptr;
  if (nruns <= 0 || !n || !L || !eps || !beta) { g_batch_create_err = "invalid run list"; return SPFC_EINVAL; }
  if (!(dt > 0.0) || !std::isfinite(dt)) { g_batch_create_err = "dt must be positive"; return SPFC_EINVAL; }
  if (precision != SPFC_FP64 && precision != SPFC_FP32_BULK) { g_batch_create_err = "unknown precision"; return SPFC_EINVAL; }
  std::map<int, std::vector<int>> by_n;
  std::map<int, int> sched_of;
  for (int r = 0; r < nruns; ++r) {
    const int sr = schedules ? schedules[r] : -1;
    auto it = sched_of.find(n[r]);
    if (it == sched_of.end()) sched_of[n[r]] = sr;
    else if (it->second != sr) {
      g_batch_create_err = "runs of one grid size must share one schedule";
      return SPFC_EINVAL;
    }
  }
  for (int r = 0; r < nruns; ++r) {
    if (!(L[r] > 0.0) || !(1.0 - eps[r] > 0.0) || !(beta[r] > 0.0)) {
      g_batch_create_err = "run " + std::to_string(r) + ": need L > 0, 1 - eps > 0, beta > 0";
      return SPFC_EINVAL;
    }
    by_n[n[r]].push_back(r);
  }
  auto b = std::make_unique<spfc_batch_s>();
  b->st = (cudaStream_t)cuda_stream;
  b->where.assign(nruns, {-1, -1});
  b->n.assign(n, n + nruns);
  for (auto& kv : by_n) {
    std::vector<Params> ps;
    for (int r : kv.second) {
      Params P{};
      P.d = 2;
      P.N = kv.first;
      P.NH = kv.first / 2 + 1;
      P.kf[0] = P.kf[1] = 2.0 * M_PI / L[r];
      P.kf[2] = 0.0;
      const double h = L[r] / kv.first;
      P.hd = h * h;
      P.vol = L[r] * L[r];
      P.P = (double)kv.first * kv.first;
      P.a = 1.0 - eps[r];
      P.beta = beta[r];
      P.C = 1.0 + 1.0 / beta[r];
      P.dt = dt;
      spfc::fill_float_params(&P);
      ps.push_back(P);
      b->points += (int64_t)kv.first * kv.first;
    }
    int status = 0;
    std::string err;
    BatchClassBase* c = spfc::make_class(kv.first, precision, sched_of[kv.first], ps, b->st, &status, &err);
    if (!c) { g_batch_create_err = err; return status ? status : SPFC_ECUDA; }
    c->runs = kv.second;
    for (size_t i = 0; i < kv.second.size(); ++i) b->where[kv.second[i]] = {(int)b->classes.size(), (int)i};
    b->classes.emplace_back(c);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (size_t c = 0; c < b->classes.size() && e == cudaSuccess; ++c) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->side.push_back(s);
  }
  const size_t nev = 1 + b->classes.size();  // the graph's fork and one join per class
  for (size_t i = 0; i < nev && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->evs.push_back(ev);
  }
  if (e != cudaSuccess) { g_batch_create_err = cudaGetErrorString(e); return SPFC_ECUDA; }
  *out = b.release();
  return SPFC_OK;
}

int spfc_batch_init(spfc_batch_t b, int run, const double* phi0, int mode) {
  if (!b || !phi0) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  if (mode < 0 || mode > 2) return b->fail(SPFC_EINVAL, "unknown start mode");
  auto w = b->where[run];
  int rc = b->classes[w.first]->load_run(w.second, phi0, mode);
  if (rc) return b->fail(rc, b->classes[w.first]->err);
  b->w_ready = false;
  return SPFC_OK;
}

int spfc_batch_set_state(spfc_batch_t b, int run, const double* phi, const double* phi_prev, double r,
                         double r_prev) {
  if (!b || !phi || !phi_prev) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  if (!std::isfinite(r) || !std::isfinite(r_prev)) return b->fail(SPFC_EINVAL, "r and r_prev must be finite");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return b->fail(SPFC_ECUDA, cudaGetErrorString(e));
  auto w = b->where[run];
  int rc = b->classes[w.first]->set_run_state(w.second, phi, phi_prev, r, r_prev);
  if (rc) return b->fail(rc, b->classes[w.first]->err);
  b->w_ready = false;
  return SPFC_OK;
}

int spfc_batch_set_gamma3(spfc_batch_t b, int run, double gamma3) {
  if (!b) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  if (!(gamma3 >= 0.0) || !std::isfinite(gamma3)) return b->fail(SPFC_EINVAL, "gamma3 must be finite and >= 0");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return b->fail(SPFC_ECUDA, cudaGetErrorString(e));
  auto w = b->where[run];
  int rc = b->classes[w.first]->set_gamma3(w.second, gamma3);
  if (rc) return b->fail(rc, b->classes[w.first]->err);
  // the class may switch to the phi^4 passes: new graphs, and W prepared again
  if (b->g1) { cudaGraphExecDestroy(b->g1); b->g1 = nullptr; }
  if (b->g8) { cudaGraphExecDestroy(b->g8); b->g8 = nullptr; }
  b->w_ready = false;
  return SPFC_OK;
}

int spfc_batch_step(spfc_batch_t b, int64_t nsteps) {
  if (!b) return SPFC_EINVAL;
  if (nsteps < 0) return b->fail(SPFC_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return SPFC_OK;
  if (!b->w_ready) {
    for (auto& c : b->classes) {
      int rc = c->prepare(b->st);
      if (rc) return b->fail(rc, c->err);
    }
    b->w_ready = true;
  }
  if (!b->g1) { int rc = b->capture(1, &b->g1); if (rc) return rc; }
  if (!b->g8) { int rc = b->capture(8, &b->g8); if (rc) return rc; }
  for (int64_t i = 0; i < nsteps / 8; ++i) {
    cudaError_t e = cudaGraphLaunch(b->g8, b->st);
    if (e != cudaSuccess) return b->fail(SPFC_ECUDA, cudaGetErrorString(e));
  }
  for (int64_t i = 0; i < nsteps % 8; ++i) {
    cudaError_t e = cudaGraphLaunch(b->g1, b->st);
    if (e != cudaSuccess) return b->fail(SPFC_ECUDA, cudaGetErrorString(e));
  }
  return SPFC_OK;
}

int spfc_batch_sync(spfc_batch_t b) {
  if (!b) return SPFC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return b->fail(SPFC_ECUDA, cudaGetErrorString(e));
  return SPFC_OK;
}

int spfc_batch_get_field(spfc_batch_t b, int run, double* out, int which) {
  if (!b || !out) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  int rc = spfc_batch_sync(b);
  if (rc) return rc;
  auto w = b->where[run];
  rc = b->classes[w.first]->run_field(w.second, out, which);
  if (rc) return b->fail(rc, b->classes[w.first]->err);
  return SPFC_OK;
}

int spfc_batch_scalars(spfc_batch_t b, int run, double* out, int nout) {
  if (!b || !out) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  int rc = spfc_batch_sync(b);
  if (rc) return rc;
  auto w = b->where[run];
  SavScal h;
  rc = b->classes[w.first]->run_scalars(w.second, &h);
  const double v[8] = {h.r1, h.r0, h.xi, h.gamma, h.E1, (double)h.nsteps, h.zm[h.p], (double)h.status};
  for (int i = 0; i < nout && i < 8; ++i) out[i] = v[i];
  if (rc) return b->fail(rc, "device status latched for this run");
  return SPFC_OK;
}

int spfc_batch_energy(spfc_batch_t b, int run, double* E3) {
  if (!b || !E3) return SPFC_EINVAL;
  if (run < 0 || run >= (int)b->where.size()) return b->fail(SPFC_EINVAL, "run index out of range");
  int rc = spfc_batch_sync(b);
  if (rc) return rc;
  auto w = b->where[run];
  rc = b->classes[w.first]->run_energy(w.second, E3);
  if (rc) return b->fail(rc, b->classes[w.first]->err);
  return SPFC_OK;
}

int64_t spfc_batch_points(spfc_batch_t b) { return b ? b->points : 0; }

void spfc_batch_destroy(spfc_batch_t b) { delete b; }

const char* spfc_batch_last_error(spfc_batch_t b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

}  // extern "C"
