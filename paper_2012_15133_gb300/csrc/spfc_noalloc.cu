// Allocation-free variant of the energy diagnostics for a caller-supplied 2D
// field (declared in include/spfc.h as spfc_field_energy_noalloc).
//
// Some callers cannot allocate device memory: code that runs under a fixed
// memory budget owned by another allocator (a framework's caching pool, an
// embedded or real-time host loop), or code that must not synchronise the
// device, which cudaMalloc / cudaFree may do. For them this entry point keeps
// all of its scratch (spectra, work arrays, partial sums, the scalar record
// and the twiddle table) in one file-scope __device__ array of fixed size; the
// caller passes only the input field and receives the results.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/spfc.h"
#include "spfc_internal.h"
#include "spfc_solver2d.cuh"

namespace spfc {
namespace {

// Largest grid: 256 x 256 in float64. Three complex half spectra
// (N x (N/2+1) x 16 bytes each) plus partial sums, the scalar record and the
// twiddle table.
constexpr int NOALLOC_MAX_N = 256;
constexpr size_t kSpec = (size_t)NOALLOC_MAX_N * (NOALLOC_MAX_N / 2 + 1) * sizeof(double2);
constexpr size_t kPart = 64 * 1024;
constexpr size_t kTw = TW_LEN * sizeof(double2);
constexpr size_t kScal = 1024;
constexpr size_t kBytes = 3 * kSpec + kPart + kTw + kScal;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kBytes];

struct DevSlot {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_scratch on this device
};
// A marker written into the array after the twiddle table: a new context on
// the device (after cudaDeviceReset) reloads the module with the array
// zeroed, possibly at another address, so each call checks both.
constexpr unsigned long long kMagic = 0x5350464354574431ull;
constexpr size_t kMagicOff = kBytes - sizeof(unsigned long long);
constexpr int kMaxDev = 64;
DevSlot g_dev[kMaxDev];
std::mutex g_mu;
thread_local std::string g_err;

// Every call, with the device current: look up the device address of the
// scratch array (a host-side name of a __device__ array is only a stand-in,
// never a device address); once per device context, write the twiddle table
// and the marker into it.
int setup_device(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDev) { g_err = "device index out of range"; return SPFC_EINVAL; }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess) { g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return SPFC_ECUDA; }
  if (g_dev[dev].ready) {
    unsigned long long m = 0;
    e = cudaMemcpy(&m, (unsigned char*)ptr + kMagicOff, sizeof(m), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { g_err = std::string("scratch check: ") + cudaGetErrorString(e); return SPFC_ECUDA; }
    if (ptr != (void*)g_dev[dev].base || m != kMagic) g_dev[dev].ready = false;  // a new context
  }
  if (!g_dev[dev].ready) {
    std::vector<double2> tw;
    host_twiddles<double>(tw);
    e = cudaMemcpy((unsigned char*)ptr + 3 * kSpec + kPart, tw.data(), kTw, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { g_err = std::string("twiddle upload: ") + cudaGetErrorString(e); return SPFC_ECUDA; }
    e = cudaMemcpy((unsigned char*)ptr + kMagicOff, &kMagic, sizeof(kMagic), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { g_err = std::string("scratch marker: ") + cudaGetErrorString(e); return SPFC_ECUDA; }
    g_dev[dev].base = (unsigned char*)ptr;
    g_dev[dev].ready = true;
  }
  *base = g_dev[dev].base;
  return SPFC_OK;
}

template <int N>
int run(const Params& P, const double* phi, double* out, cudaStream_t st, unsigned char* base) {
  using C = double2;
  using SH = Shape2D<N>;
  constexpr int E = SH::E, CT = SH::CT, RPC = SH::RPC, T = SH::T;
  constexpr int NH = N / 2 + 1;
  constexpr int GCOL = (NH + CT - 1) / CT, GROW = N / RPC, PW = 256;
  const int gpw = (int)std::min<size_t>(((size_t)N * NH + PW - 1) / PW, 608);
  C* spec = reinterpret_cast<C*>(base);
  C* w0 = reinterpret_cast<C*>(base + kSpec);
  C* w1 = reinterpret_cast<C*>(base + 2 * kSpec);
  double* partE = reinterpret_cast<double*>(base + 3 * kSpec);
  double* partN = partE + 2 * 1024;
  double* partS = partN + 3 * 1024;
  const C* tw = reinterpret_cast<const C*>(base + 3 * kSpec + kPart);
  SavScal* sc = reinterpret_cast<SavScal*>(base + 3 * kSpec + kPart + kTw);
  static_assert(sizeof(SavScal) + sizeof(unsigned long long) <= kScal, "scalar record and marker must fit");
  static_assert(GROW <= 1024 && 8 * (2 * 1024 + 3 * 1024 + 608) <= kPart, "partial sums must fit");
  Slots<double> S{{spec, spec}};
  const size_t scol = (size_t)sp_len(N) * col_pitch(CT) * sizeof(C);
  const size_t srow = (size_t)RPC * (sp_len(N) + 1) * sizeof(C);
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(SavScal), st);  // p = 0, status OK
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return SPFC_ECUDA; }
  k_real_sum<<<gpw, PW, 0, st>>>(phi, (size_t)N * N, partS);
  // both "levels" are this field: zero mode of slot p and of slot 1-p
  k_scalar_op<double><<<1, 32, 0, st>>>(P, sc, SO_ZM_SLOT, partS, gpw, nullptr, 0, 0, 0.0, 0.0);
  k_scalar_op<double><<<1, 32, 0, st>>>(P, sc, SO_ZM_SLOT, partS, gpw, nullptr, 0, 1, 0.0, 0.0);
  k2d_row<double, N, E, RPC, RW_IN_REAL><<<GROW, RPC * T, srow, st>>>(P, w0, w1, partE, sc, tw,
                                                                       const_cast<double*>(phi));
  k2d_col_fwd<double, N, E, CT, CF_TO_STATE><<<GCOL, CT * T, scol, st>>>(P, S, w0, w1, nullptr, nullptr, nullptr, 0,
                                                                          sc, nullptr, tw, 0);
  k_put_zero_modes<double><<<1, 1, 0, st>>>(S, sc);
  k2d_col_inv<double, N, E, CT, CI_GRAD><<<GCOL, CT * T, 2 * scol, st>>>(P, S, nullptr, w0, w1, sc, tw, 0);
  k2d_row<double, N, E, RPC, RW_ENERGY><<<GROW, RPC * T, srow, st>>>(P, w0, w1, partE, sc, tw, nullptr);
  k2d_norms<double><<<gpw, PW, 0, st>>>(P, S, sc, partN);
  k_scalar_op<double><<<1, 32, 0, st>>>(P, sc, SO_ENERGY, partE, GROW, partN, gpw, 0, 0.0, 0.0);
  e = cudaGetLastError();
  if (e != cudaSuccess) { g_err = std::string("launch: ") + cudaGetErrorString(e); return SPFC_ECUDA; }
  SavScal h;
  e = cudaMemcpyAsync(&h, sc, sizeof(SavScal), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return SPFC_ECUDA; }
  if (h.status != DEV_OK || !std::isfinite(h.E_orig) || !std::isfinite(h.E_mod) || !std::isfinite(h.zm[0])) {
    g_err = "non-finite value in the field";
    return SPFC_ENONFINITE;
  }
  out[0] = h.E_orig;
  out[1] = h.E_mod;          // with phi^{n-1} = phi^n and r = 0: 1/2 ||L^{1/2} phi||^2
  out[2] = P.vol * h.zm[0];  // mass h^2 sum phi
  return SPFC_OK;
}

}  // namespace
}  // namespace spfc

extern "C" int spfc_field_energy_noalloc(int n, const double* L, double eps, double beta, const double* phi_dev,
                                         double* out, void* cuda_stream) {
  using namespace spfc;
  if (!L || !phi_dev || !out) { g_err = "NULL argument"; return SPFC_EINVAL; }
  if (n > NOALLOC_MAX_N) {
    g_err = "spfc_field_energy_noalloc: N exceeds the fixed scratch maximum of 256";
    return SPFC_EINVAL;
  }
  if (n != 16 && n != 32 && n != 64 && n != 128 && n != 256) {
    g_err = "spfc_field_energy_noalloc: N must be 16, 32, 64, 128 or 256";
    return SPFC_EINVAL;
  }
  if (!(L[0] > 0.0) || !(L[1] > 0.0) || !(1.0 - eps > 0.0) || !(beta > 0.0)) {
    g_err = "spfc_field_energy_noalloc: need L > 0, 1 - eps > 0, beta > 0";
    return SPFC_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return SPFC_ECUDA; }
  unsigned char* base = nullptr;
  int rc = setup_device(dev, &base);
  if (rc) return rc;
  Params P{};
  P.d = 2;
  P.N = n;
  P.NH = n / 2 + 1;
  P.kf[0] = 2.0 * M_PI / L[0];
  P.kf[1] = 2.0 * M_PI / L[1];
  P.kf[2] = 0.0;
  P.hd = (L[0] / n) * (L[1] / n);
  P.vol = L[0] * L[1];
  P.P = (double)n * n;
  P.a = 1.0 - eps;
  P.beta = beta;
  P.C = 1.0 + 1.0 / beta;
  P.dt = 1.0;
  fill_float_params(&P);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (n) {
    case 16: return run<16>(P, phi_dev, out, st, base);
    case 32: return run<32>(P, phi_dev, out, st, base);
    case 64: return run<64>(P, phi_dev, out, st, base);
    case 128: return run<128>(P, phi_dev, out, st, base);
    default: return run<256>(P, phi_dev, out, st, base);
  }
}

extern "C" const char* spfc_noalloc_last_error(void) { return spfc::g_err.c_str(); }
