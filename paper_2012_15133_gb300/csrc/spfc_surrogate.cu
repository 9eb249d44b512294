// Jump-with-fallback loop of the learned surrogate (declared in
// include/spfc.h). One network call predicts phi^{n+K} for every run of a
// round; each prediction is judged by the modified-energy test (eq.
// discrete energy of the live two-level state against that of the
// copy-restarted prediction) and, every
// check_every rounds, against K plain SAV steps taken from the same state
// by a twin solver; a rejected jump falls back to the plain steps. The loop
// composes the library's own entry points (solver handles, the network, the
// allocation-free energy) and adds three small kernels: the float64 <->
// float32 conversions of the fields and the rel-L2 of a checked jump.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "../../include/spfc.h"
#include "spfc_common.cuh"
#include "spfc_internal.h"

namespace {

thread_local std::string g_sur_err;

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// One block: sum a^4 over n values in a fixed order (the phi^4 term of E_1).
__global__ void __launch_bounds__(1024) k_sum_pow4(const double* __restrict__ a, size_t n, double* __restrict__ out) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = a[i] * a[i];
    s += v * v;
  }
  s = spfc::block_sum(s, scratch);
  if (threadIdx.x == 0) out[0] = s;
}

// One block: sum (a - b)^2 and sum b^2 over n values in a fixed order.
__global__ void __launch_bounds__(1024) k_rel_parts(const double* __restrict__ a, const double* __restrict__ b,
                                                    size_t n, double* __restrict__ out) {
  __shared__ double scratch[32];
  double s1 = 0.0, s2 = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = a[i] - b[i];
    s1 += d * d;
    s2 += b[i] * b[i];
  }
  s1 = spfc::block_sum(s1, scratch);
  __syncthreads();
  s2 = spfc::block_sum(s2, scratch);
  if (threadIdx.x == 0) {
    out[0] = s1;
    out[1] = s2;
  }
}

int failx(int code, const std::string& msg) {
  g_sur_err = msg;
  return code;
}

// device buffers of one call, freed on every return path
struct Bufs {
  std::vector<void*> p;
  ~Bufs() {
    for (void* q : p) cudaFree(q);
  }
  template <typename T> bool get(T** out, size_t count) {
    if (cudaMalloc((void**)out, count * sizeof(T)) != cudaSuccess) return false;
    p.push_back(*out);
    return true;
  }
};

}  // namespace

extern "C" {

int spfc_surrogate_advance(spfc_fno_t net, spfc_t* runs, spfc_t* twins, int nruns, int K, int jumps, int check_every,
                           double tol, int64_t* counts, int8_t* decisions, double* check_err) {
  g_sur_err.clear();
  if (!net || !runs || nruns < 1 || K < 1 || jumps < 0 || check_every < 0 || !(tol >= 0.0))
    return failx(SPFC_EINVAL, "bad argument (net, runs, nruns >= 1, K >= 1, jumps >= 0, check_every >= 0, tol >= 0)");
  int n = 0, bmax = 0;
  cudaStream_t st = nullptr;
  spfc::fno_shape(net, &n, &bmax, &st);
  if (nruns > bmax) return failx(SPFC_EINVAL, "more runs than the network's largest batch");
  if (n > 256) return failx(SPFC_EINVAL, "the energy test takes grids of at most 256 x 256");
  if (check_every > 0 && !twins) return failx(SPFC_EINVAL, "periodic checks need one twin handle per run");
  for (int i = 0; i < nruns; ++i) {
    const spfc_t h = runs[i];
    if (!h || !h->s->inited) return failx(SPFC_ESTATE, "every run must be an initialised handle");
    const spfc::Params& P = h->s->P;
    if (P.d != 2 || P.N != n || P.Lbox[0] != P.Lbox[1])
      return failx(SPFC_EINVAL, "runs must be square 2D grids of the network's size");
    if (P.pfc) return failx(SPFC_EINVAL, "the surrogate serves SPFC runs (not the PFC model)");
    for (int k = 0; k < i; ++k)
      if (runs[k] == h) return failx(SPFC_EINVAL, "a run appears twice");
    if (check_every > 0) {
      const spfc_t t = twins[i];
      if (!t) return failx(SPFC_EINVAL, "each run needs a twin handle of its own");
      for (int k = 0; k < nruns; ++k)
        if (runs[k] == t) return failx(SPFC_EINVAL, "a twin must not be one of the runs");
      for (int k = 0; k < i; ++k)
        if (twins[k] == t) return failx(SPFC_EINVAL, "a twin appears twice");
      const spfc::Params& Q = t->s->P;
      if (Q.d != 2 || Q.N != n || Q.Lbox[0] != P.Lbox[0] || Q.Lbox[1] != P.Lbox[1] || Q.eps != P.eps ||
          Q.beta != P.beta || Q.dt != P.dt || Q.stab != P.stab || Q.g3 != P.g3 ||
          t->s->precision != h->s->precision)
        return failx(SPFC_EINVAL, "a twin must have its run's grid, parameters and precision");
    }
  }
  const size_t P = (size_t)n * n, RP = (size_t)nruns * P;
  Bufs b;
  double *cur = nullptr, *prev = nullptr, *pred = nullptr, *plain = nullptr, *plain_prev = nullptr, *parts = nullptr;
  float *cur32 = nullptr, *prev32 = nullptr, *pred32 = nullptr;
  if (!b.get(&cur, RP) || !b.get(&prev, RP) || !b.get(&pred, RP) || !b.get(&plain, P) || !b.get(&plain_prev, P) ||
      !b.get(&parts, 2) || !b.get(&cur32, RP) || !b.get(&prev32, RP) || !b.get(&pred32, RP))
    return failx(SPFC_ENOMEM, "device allocation failed");
  std::vector<double> eps(nruns), beta(nruns);
  for (int i = 0; i < nruns; ++i) {
    eps[i] = runs[i]->s->P.eps;
    beta[i] = runs[i]->s->P.beta;
  }
  int64_t cnt[5] = {0, 0, 0, 0, 0};  // jumps, accepted, rejected by energy, rejected by check, checks
  const int cvt_blocks = (int)std::min<size_t>((RP + 255) / 256, 2048);
  auto run_err = [](spfc_t h, int rc, const char* what) {
    return failx(rc, std::string(what) + ": " + spfc_last_error(h));
  };
  for (int j = 0; j < jumps; ++j) {
    for (int i = 0; i < nruns; ++i) {
      int rc = spfc_get_field(runs[i], cur + i * P, 1, 0);
      if (!rc) rc = spfc_get_field(runs[i], prev + i * P, 1, 1);
      if (rc) return run_err(runs[i], rc, "reading a run");
    }
    k_d2f<<<cvt_blocks, 256, 0, st>>>(cur, cur32, RP);
    k_d2f<<<cvt_blocks, 256, 0, st>>>(prev, prev32, RP);
    int rc = spfc_fno_predict(net, nruns, cur32, prev32, eps.data(), beta.data(), pred32);
    if (rc) return failx(rc, std::string("network: ") + spfc_fno_last_error(net));
    k_f2d<<<cvt_blocks, 256, 0, st>>>(pred32, pred, RP);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return failx(SPFC_ECUDA, std::string("prediction: ") + cudaGetErrorString(e));
    const bool check = check_every > 0 && j % check_every == 0;
    for (int i = 0; i < nruns; ++i) {
      const spfc_t h = runs[i];
      const double L2[2] = {h->s->P.Lbox[0], h->s->P.Lbox[1]};
      const spfc::Params& Pr = h->s->P;
      double e_new[3], e_live = 0.0, s4 = 0.0;
      ++cnt[0];
      if (check_err) check_err[(size_t)j * nruns + i] = std::numeric_limits<double>::quiet_NaN();
      // before: the modified energy of the live state (phi^n, phi^{n-1}, r^n, r^{n-1})
      rc = spfc_energy(h, nullptr, &e_live, nullptr);
      if (rc) return run_err(h, rc, "energy test");
      // after the copy restart (phi^{n+K-1} = phi^{n+K}, r = sqrt(E_1)) the
      // modified energy is E_N(prediction) + C_beta |Omega|, E_N with the
      // run's phi^4 term
      rc = spfc_field_energy_noalloc(n, L2, eps[i], beta[i], pred + i * P, e_new, st);
      if (rc) return failx(rc, std::string("energy test: ") + spfc_noalloc_last_error());
      if (Pr.g3 != 0.0) {
        k_sum_pow4<<<1, 1024, 0, st>>>(pred + i * P, P, parts);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s4, parts, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return failx(SPFC_ECUDA, std::string("energy test: ") + cudaGetErrorString(e));
      }
      const double e_after = e_new[0] + 0.25 * Pr.g3 * Pr.hd * s4 + Pr.C * Pr.vol;
      if (e_after > e_live) {
        ++cnt[2];
        if (decisions) decisions[(size_t)j * nruns + i] = 1;
        if ((rc = spfc_step(h, K))) return run_err(h, rc, "fallback steps");
        continue;
      }
      if (check) {
        const spfc_t t = twins[i];
        double sc[2], ts[2], pp[2];
        rc = spfc_sav_scalars(h, sc, 2);
        if (rc) return run_err(h, rc, "reading r");
        rc = spfc_set_state(t, cur + i * P, prev + i * P, sc[0], sc[1], 1);
        if (!rc) rc = spfc_step(t, K);
        if (!rc) rc = spfc_get_field(t, plain, 1, 0);
        if (rc) return run_err(t, rc, "check steps");
        k_rel_parts<<<1, 1024, 0, st>>>(pred + i * P, plain, P, parts);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(pp, parts, sizeof(pp), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return failx(SPFC_ECUDA, std::string("check: ") + cudaGetErrorString(e));
        const double err = std::sqrt(pp[0]) / std::sqrt(pp[1]);
        ++cnt[4];
        if (check_err) check_err[(size_t)j * nruns + i] = err;
        if (err > tol) {
          // keep the plain result
          ++cnt[3];
          if (decisions) decisions[(size_t)j * nruns + i] = 2;
          rc = spfc_sav_scalars(t, ts, 2);
          if (!rc) rc = spfc_get_field(t, plain_prev, 1, 1);
          if (rc) return run_err(t, rc, "reading the check");
          if ((rc = spfc_set_state(h, plain, plain_prev, ts[0], ts[1], 1))) return run_err(h, rc, "fallback state");
          continue;
        }
      }
      ++cnt[1];
      if (decisions) decisions[(size_t)j * nruns + i] = 0;
      if ((rc = spfc_init(h, pred + i * P, 1, SPFC_START_COPY))) return run_err(h, rc, "restart from the jump");
    }
  }
  if (counts)
    for (int k = 0; k < 5; ++k) counts[k] = cnt[k];
  return SPFC_OK;
}

const char* spfc_surrogate_last_error(void) { return g_sur_err.c_str(); }

}  // extern "C"
