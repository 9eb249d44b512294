// C ABI of the SPFC solver (declared in include/spfc.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/spfc.h"
#include "spfc_internal.h"

using spfc::SolverBase;

static thread_local std::string g_create_err;

// phi[j] = mean + amp (2 u_j - 1), u_j = (x_j >> 11) 2^-53 with x_j output j of
// SplitMix64 (Steele, Lea & Flood 2014) seeded with `seed`, used as a
// counter-based generator: x_j is the finaliser applied to
// seed + (j + 1) * 0x9E3779B97F4A7C15 (mod 2^64). The arithmetic is rounded
// explicitly (no contraction), so the field is the same on every platform.
__global__ void k_noise_field(double* __restrict__ phi, size_t count, unsigned long long seed, double mean,
                              double amp) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < count; j += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = __dmul_rn((double)(z >> 11), 0x1.0p-53);
    const double c = __dadd_rn(__dmul_rn(2.0, u), -1.0);
    phi[j] = __dadd_rn(mean, __dmul_rn(amp, c));
  }
}

static int fail(spfc_t h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_err = msg;
  return code;
}

// Default launch schedule per grid: the autotuner's choice on GB300 (the
// smallest sum of flushed and L2-resident step time; autotune_cache.json).
// float32 bulk: the persistent step (6) at 512, its 4-values-per-lane form
// (7) at 256 and 128, the persistent step (1) below; float64: the persistent
// step (6) at 512, 5 at 128 and 256, 0 below.
static int default_schedule(int d, int n, int precision) {
  if (d != 2) return 0;
  if (precision == SPFC_FP64) return n == 512 ? 6 : ((n == 128 || n == 256) ? 5 : 0);
  if (n == 512) return 6;
  return (n == 128 || n == 256) ? 7 : 1;
}

static int wrap(spfc_t h, int rc) {
  if (rc) h->err = h->s->err;
  return rc;
}

extern "C" {

int spfc_create(int d, const int* n, const double* L, double eps, double beta, double dt, int precision,
                void* cuda_stream, spfc_t* out) {
  return spfc_create_scheduled(d, n, L, eps, beta, dt, precision, cuda_stream, -1, out);
}

int spfc_num_schedules(int d, int n) { return spfc::num_schedules(d, n); }

int spfc_schedule(spfc_t h) { return h ? h->s->schedule : -1; }

int spfc_create_scheduled(int d, const int* n, const double* L, double eps, double beta, double dt, int precision,
                          void* cuda_stream, int schedule, spfc_t* out) {
  if (!out) return fail(nullptr, SPFC_EINVAL, "out is NULL");
  *out = nullptr;
  if (d != 2 && d != 3) return fail(nullptr, SPFC_EINVAL, "d must be 2 or 3");
  if (!n || !L) return fail(nullptr, SPFC_EINVAL, "n and L must not be NULL");
  for (int i = 0; i < d; ++i) {
    if (n[i] != n[0]) return fail(nullptr, SPFC_EINVAL, "the GPU solver needs the same N on every axis");
    if (!(L[i] > 0.0) || !std::isfinite(L[i])) return fail(nullptr, SPFC_EINVAL, "L must be positive");
  }
  if (!(1.0 - eps > 0.0) || !std::isfinite(eps)) return fail(nullptr, SPFC_EINVAL, "a = 1 - eps must be positive");
  if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, SPFC_EINVAL, "beta must be positive");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, SPFC_EINVAL, "dt must be positive");
  if (precision != SPFC_FP64 && precision != SPFC_FP32_BULK) return fail(nullptr, SPFC_EINVAL, "unknown precision");
  spfc::Params P{};
  P.d = d;
  P.N = n[0];
  P.NH = n[0] / 2 + 1;
  double hd = 1.0, vol = 1.0;
  for (int i = 0; i < 3; ++i) P.kf[i] = P.Lbox[i] = 0.0;
  for (int i = 0; i < d; ++i) {
    P.Lbox[i] = L[i];
    P.kf[i] = 2.0 * M_PI / L[i];
    hd *= L[i] / n[i];
    vol *= L[i];
  }
  P.hd = hd;
  P.vol = vol;
  P.P = std::pow((double)n[0], d);
  P.a = 1.0 - eps;
  P.eps = eps;
  P.beta = beta;
  P.C = 1.0 + 1.0 / beta;
  P.dt = dt;
  spfc::fill_float_params(&P);
  int status = 0;
  std::string err;
  if (schedule < 0) schedule = default_schedule(d, n[0], precision);
  SolverBase* s = (precision == SPFC_FP64)
                      ? spfc::make_solver_f64(P, (cudaStream_t)cuda_stream, schedule, &status, &err)
                      : spfc::make_solver_f32(P, (cudaStream_t)cuda_stream, schedule, &status, &err);
  if (!s) return fail(nullptr, status ? status : SPFC_ECUDA, err);
  s->precision = precision;
  spfc_t h = new spfc_s;
  h->s = s;
  *out = h;
  return SPFC_OK;
}

int spfc_init(spfc_t h, const double* phi0, int on_device, int mode) {
  if (!h || !phi0) return fail(h, SPFC_EINVAL, "NULL argument");
  if (mode < 0 || mode > 2) return fail(h, SPFC_EINVAL, "unknown start mode");
  return wrap(h, h->s->init(phi0, on_device != 0, mode));
}

int spfc_init_random(spfc_t h, double mean, double amp, uint64_t seed, int mode) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (mode < 0 || mode > 2) return fail(h, SPFC_EINVAL, "unknown start mode");
  if (!std::isfinite(mean) || !std::isfinite(amp)) return fail(h, SPFC_EINVAL, "mean and amp must be finite");
  const spfc::Params& P = h->s->P;
  const size_t count = (size_t)std::llround(P.P);
  double* phi = nullptr;
  cudaError_t e = cudaMalloc(&phi, count * sizeof(double));
  if (e != cudaSuccess) return fail(h, SPFC_ENOMEM, std::string("allocation: ") + cudaGetErrorString(e));
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
  k_noise_field<<<blocks, 256>>>(phi, count, (unsigned long long)seed, mean, amp);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  int rc = (e == cudaSuccess) ? wrap(h, h->s->init(phi, true, mode))
                              : fail(h, SPFC_ECUDA, std::string("noise field: ") + cudaGetErrorString(e));
  cudaFree(phi);  // synchronises with the device: the start-up has consumed the field
  return rc;
}

int spfc_set_state(spfc_t h, const double* phi, const double* phi_prev, double r, double r_prev, int on_device) {
  if (!h || !phi || !phi_prev) return fail(h, SPFC_EINVAL, "NULL argument");
  if (!(r > 0.0) || !(r_prev > 0.0)) return fail(h, SPFC_EINVAL, "r must be positive");
  return wrap(h, h->s->set_state(phi, phi_prev, r, r_prev, on_device != 0));
}

int spfc_step(spfc_t h, int64_t nsteps) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(h, SPFC_EINVAL, "nsteps must be >= 0");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "spfc_step before spfc_init");
  return wrap(h, h->s->step(nsteps));
}

int spfc_energy(spfc_t h, double* E_orig, double* E_mod, double* E_breve) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  return wrap(h, h->s->energy(E_orig, E_mod, E_breve));
}

int spfc_mass(spfc_t h, double* mass, double* mean) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  return wrap(h, h->s->mass(mass, mean));
}

int spfc_sav_scalars(spfc_t h, double* out, int nout) {
  if (!h || !out) return fail(h, SPFC_EINVAL, "NULL argument");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  spfc::SavScal sc;
  int rc = h->s->scalars(&sc);
  if (rc) return wrap(h, rc);
  const double v[10] = {sc.r1, sc.r0, sc.xi, sc.gamma, sc.E1, (double)sc.nsteps, sc.eta, sc.theta, sc.denom, sc.LHS};
  for (int i = 0; i < nout && i < 10; ++i) out[i] = v[i];
  return SPFC_OK;
}

int spfc_get_field(spfc_t h, double* out, int on_device, int which) {
  if (!h || !out) return fail(h, SPFC_EINVAL, "NULL argument");
  if (which != 0 && which != 1) return fail(h, SPFC_EINVAL, "which must be 0 or 1");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  return wrap(h, h->s->get_field(out, on_device != 0, which));
}

int spfc_set_stabilization(spfc_t h, double A) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!(A >= 0.0) || !std::isfinite(A)) return fail(h, SPFC_EINVAL, "the stabiliser A must be finite and >= 0");
  if (!h->s->inited) {  // before spfc_init: the start-up step uses it too
    h->s->P.stab = A;
    spfc::fill_float_params(&h->s->P);
    return SPFC_OK;
  }
  return wrap(h, h->s->set_stab(A));
}

int spfc_set_gamma3(spfc_t h, double gamma3) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!(gamma3 >= 0.0) || !std::isfinite(gamma3)) return fail(h, SPFC_EINVAL, "gamma3 must be finite and >= 0");
  return wrap(h, h->s->set_gamma3(gamma3));
}

int spfc_dt_change(spfc_t h, double dt_new) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!(dt_new > 0.0) || !std::isfinite(dt_new)) return fail(h, SPFC_EINVAL, "dt must be positive");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  return wrap(h, h->s->dt_change(dt_new));
}

// Checkpoint file: magic, then int32 {d, N, precision, blob bytes}, then
// float64 {kf0, kf1, kf2, dt, a, beta, A, gamma3, model (1 = PFC)}, then the raw state blob
// (scalar record and both spectral levels), so that a resumed run is
// bit-identical.
static const char kMagic[8] = {'S', 'P', 'F', 'C', 'C', 'K', 'P', '5'};

int spfc_save(spfc_t h, const char* path) {
  if (!h || !path) return fail(h, SPFC_EINVAL, "NULL argument");
  if (!h->s->inited) return fail(h, SPFC_ESTATE, "not initialised");
  const spfc::Params& P = h->s->P;
  std::string blob;
  int rc = h->s->dump(&blob);
  if (rc) return wrap(h, rc);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(h, SPFC_EINVAL, std::string("cannot open ") + path);
  const int32_t hdr[4] = {P.d, P.N, h->s->precision, (int32_t)blob.size()};
  const double sv[9] = {P.kf[0], P.kf[1], P.kf[2], P.dt, P.a, P.beta, P.stab, P.g3, (double)P.pfc};
  bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 &&
            std::fwrite(sv, sizeof(sv), 1, fp) == 1 && std::fwrite(blob.data(), 1, blob.size(), fp) == blob.size();
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(h, SPFC_EINVAL, std::string("write failed: ") + path);
  return SPFC_OK;
}

int spfc_load(spfc_t h, const char* path) {
  if (!h || !path) return fail(h, SPFC_EINVAL, "NULL argument");
  const spfc::Params& P = h->s->P;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(h, SPFC_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[4];
  double sv[9];
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, fp) == 1 && std::fread(sv, sizeof(sv), 1, fp) == 1;
  if (!ok || hdr[0] != P.d || hdr[1] != P.N || hdr[2] != h->s->precision || hdr[3] <= 0) {
    std::fclose(fp);
    return fail(h, SPFC_EINVAL, "checkpoint does not match this handle (grid or precision)");
  }
  const double want[9] = {P.kf[0], P.kf[1], P.kf[2], P.dt, P.a, P.beta, P.stab, P.g3, (double)P.pfc};
  for (int i = 0; i < 9; ++i)
    if (std::fabs(sv[i] - want[i]) > 1e-12 * std::fabs(want[i])) {
      std::fclose(fp);
      return fail(h, SPFC_EINVAL,
                  "checkpoint parameters (L, dt, eps, beta, stabiliser, gamma3 or model) differ from this handle's");
    }
  std::string blob((size_t)hdr[3], '\0');
  ok = std::fread(&blob[0], 1, blob.size(), fp) == blob.size();
  std::fclose(fp);
  if (!ok) return fail(h, SPFC_EINVAL, "truncated checkpoint");
  return wrap(h, h->s->restore(blob));
}

int spfc_set_pfc(spfc_t h, double gamma3) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!(gamma3 >= 0.0) || !std::isfinite(gamma3)) return fail(h, SPFC_EINVAL, "gamma3 must be finite and >= 0");
  return wrap(h, h->s->set_pfc(gamma3));
}

int spfc_set_scalar_ring(spfc_t h, double* host_ring, int64_t capacity) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  if (!host_ring) return wrap(h, h->s->set_ring(nullptr, 0));
  if (capacity < 1) return fail(h, SPFC_EINVAL, "capacity must be >= 1 when a ring is given");
  void* dev = nullptr;
  cudaError_t e = cudaHostGetDevicePointer(&dev, host_ring, 0);
  if (e != cudaSuccess || !dev) {
    cudaGetLastError();  // clear the sticky-free error of the failed lookup
    return fail(h, SPFC_EINVAL, "the ring must be page-locked host memory mapped into the device address space");
  }
  return wrap(h, h->s->set_ring(static_cast<double*>(dev), (long long)capacity));
}

int spfc_sync(spfc_t h) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  return wrap(h, h->s->sync());
}

int spfc_set_timing(spfc_t h, int on) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  return wrap(h, h->s->set_timing(on != 0));
}

int spfc_kernel_times(spfc_t h, int max, const char** names, int64_t* launches, double* ms) {
  if (!h) return fail(h, SPFC_EINVAL, "NULL handle");
  static const char* kNames[] = {"col_inv",  "row",    "col_fwd", "col_fused", "y_fwd",
                                 "z_fwd",    "scalar", "z_inv",   "y_inv",     "col_inv+col_fwd", "step"};
  spfc::KernelTimes kt;
  int rc = h->s->kernel_times(&kt);
  if (rc) return wrap(h, rc);
  const int n = (int)kt.ms.size();
  for (int i = 0; i < n && i < max; ++i) {
    if (names) {
      names[i] = "kernel";
      for (const char* k : kNames)
        if (kt.names[i] == k) names[i] = k;
    }
    if (launches) launches[i] = kt.launches[i];
    if (ms) ms[i] = kt.ms[i];
  }
  return n;
}

int64_t spfc_device_bytes(spfc_t h) { return h ? h->s->device_bytes() : 0; }

void spfc_destroy(spfc_t h) {
  if (!h) return;
  delete h->s;
  delete h;
}

const char* spfc_last_error(spfc_t h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

}  // extern "C"
