// Host driver of the 2D step kernels for one run: device buffers, the launch
// sequences of init / step / diagnostics, and CUDA-graph replay of the step.
#pragma once

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "spfc_internal.h"
#include "spfc_kernels2d.cuh"
#include "spfc_step2d_persist.cuh"

namespace spfc {

#define SPFC_CK(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
      return 3;                                                                    \
    }                                                                              \
  } while (0)

// Launch shape ("schedule") per grid size: E values per FFT lane (T = N/E
// lanes per sequence), CT kx columns per column-pass block, RPC rows per
// row-pass block. Every block fills whole warps. Schedule 0 is the default;
// the others are alternatives for N >= 128 that the autotuner times:
//   1: one column per block (twice the blocks), 2: 4 values per lane
//   (twice the threads per sequence), 3: 16 values per lane, 4 columns,
//   4: 8 values per lane, 4 columns (full 32-byte sectors per row in float32),
//   5: 4 values per lane and the fewest columns that fill a warp (the most
//   blocks and threads: for the float64 path, bound by its arithmetic).
template <int N, int SCHED = 0> struct Shape2D {
  static constexpr int E = (SCHED == 2 || SCHED == 5) ? 4 : ((SCHED == 3) ? 16 : 8);  // 0, 1 and 4 use 8
  static constexpr int T = N / E;
  static constexpr int CT0 = (N >= 256) ? 2 : ((32 / T > 4) ? 32 / T : 4);
  static constexpr int CT1 = (32 / T > 1) ? 32 / T : 1;  // fewest columns that fill a warp
  static constexpr int CT = (SCHED == 1 || SCHED == 5) ? CT1 : ((SCHED == 3 || SCHED == 4) ? 4 : CT0);
  static constexpr int RPC0 = (128 / T > 1) ? 128 / T : 1;
  static constexpr int RPC = (RPC0 < N) ? RPC0 : N;
  static_assert(N % RPC == 0 && (RPC * T) % 32 == 0 && (2 * CT * T) % 32 == 0 && (CT * T) % 32 == 0,
                "tiles must divide N and fill warps");
};

// Kernel launch, optionally with programmatic stream serialization (the
// kernel may begin while its predecessor finishes; it waits with pdl_wait).
// Cooperative launch (coop) guarantees that all blocks are co-resident, as
// the grid barrier of the fused column pass requires; it fails instead of
// deadlocking when they cannot be.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                            bool coop, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (coop) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The staged twiddle table (tw_block): entry (r - 1) NS + k of block (NS, RAD)
// is exp(-2 pi i m / TW_N) with m = r k TW_N / (NS RAD), from libm in double
// precision.
template <typename R> inline void host_twiddles(std::vector<C_t<R>>& tw) {
  tw.assign(TW_LEN, C_t<R>{});
  for (int rad = 2; rad <= 8; rad *= 2)
    for (int ns = 1; ns * rad <= TW_N; ns *= 2) {
      const int b = tw_block(ns, rad);
      for (int r = 1; r < rad; ++r)
        for (int k = 0; k < ns; ++k) {
          const int m = r * k * (TW_N / (ns * rad));
          const double ang = 2.0 * M_PI * (double)m / (double)TW_N;
          tw[b + (r - 1) * ns + k].x = (R)std::cos(ang);
          tw[b + (r - 1) * ns + k].y = (R)(-std::sin(ang));
        }
    }
}

// The schedule whose steps run as one persistent cooperative kernel
// (k2d_step_persist): the last index of every grid; its start-up and
// diagnostics passes use schedule 0's tiles.
constexpr int persist_schedule(int N) { return (N >= 128) ? 6 : 1; }
// From N = 128, schedule 7: the persistent step with 4 values per FFT lane
// (twice the threads per sequence).
constexpr int persist_e4_schedule(int N) { return (N >= 128) ? 7 : -1; }
// Steps per launch of the persistent kernel (a long run is a few launches).
constexpr long long kPersistMaxSteps = 4096;

template <typename R, int N, int SCHED = 0>
class Solver2D final : public SolverBase {
  using C = C_t<R>;
  static constexpr bool PERSIST = (SCHED == persist_schedule(N) || SCHED == persist_e4_schedule(N));
  static constexpr int PEV = (SCHED == persist_e4_schedule(N)) ? 4 : 8;
  using SH = Shape2D<N, PERSIST ? 0 : SCHED>;
  using PS = PShape<R, N, PEV>;
  static constexpr int NH = N / 2 + 1;
  static constexpr int CT = SH::CT, RPC = SH::RPC, T = SH::T, E = SH::E;
  static constexpr int GCOL = (NH + CT - 1) / CT;
  static constexpr int GROW = N / RPC;
  static constexpr int PW_THREADS = 256;

 public:
  Solver2D(const Params& p, cudaStream_t s) : st_(s) {
    P = p;
    // Programmatic dependent launch measured slower for these short kernels
    // (20.5 vs 33.6 us per 512^2 step); SPFC_PDL=1 enables it for A/B timing.
    use_pdl_ = std::getenv("SPFC_PDL") != nullptr;
  }

  int setup() {
    const size_t sb = (size_t)N * NH * sizeof(C);
    spec_bytes_ = sb;
    total_ = 0;
    auto al = [&](void** ptr, size_t bytes) -> cudaError_t {
      cudaError_t e = cudaMalloc(ptr, bytes);
      if (e == cudaSuccess) total_ += bytes;
      return e;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = al((void**)&S_.s[0], sb);
    if (e == cudaSuccess) e = al((void**)&S_.s[1], sb);
    if (e == cudaSuccess) e = al((void**)&Nhat_, sb);
    if (e == cudaSuccess) e = al((void**)&W_[0], sb);
    if (e == cudaSuccess) e = al((void**)&W_[1], sb);
    if (e == cudaSuccess) e = al((void**)&real_, (size_t)N * N * sizeof(double));
    gpw_ = (int)std::min<size_t>(((size_t)N * NH + PW_THREADS - 1) / PW_THREADS, 608);
    nE_ = GROW;
    nG_ = GCOL;
    if (e == cudaSuccess) e = al((void**)&partE_, 2 * (size_t)nE_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partG_, 3 * (size_t)nG_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partN_, 4 * (size_t)gpw_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partS_, (size_t)gpw_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&sc_, sizeof(SavScal));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&hsc_, sizeof(SavScal));  // pinned: small fast reads
    if (e == cudaSuccess) e = al((void**)&counter_, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = al((void**)&sync64_, sizeof(unsigned long long));
    if (e == cudaSuccess && PERSIST) e = al((void**)&sync64p_, sizeof(unsigned long long));
    if (e == cudaSuccess && PERSIST) e = al((void**)&partP_, 5 * (size_t)PS::G * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&tw_, TW_LEN * sizeof(C));
    if (e != cudaSuccess) {
      err = std::string("device allocation failed: ") + cudaGetErrorString(e);
      return (e == cudaErrorMemoryAllocation) ? 2 : 3;
    }
    std::vector<C> tw;
    host_twiddles<R>(tw);
    SPFC_CK(cudaMemcpy(tw_, tw.data(), TW_LEN * sizeof(C), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemset(counter_, 0, 4 * sizeof(unsigned)));
    SPFC_CK(cudaMemset(sync64_, 0, sizeof(unsigned long long)));
    if (PERSIST) SPFC_CK(cudaMemset(sync64p_, 0, sizeof(unsigned long long)));
    SavScal z{};
    SPFC_CK(cudaMemcpy(sc_, &z, sizeof(SavScal), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemset(S_.s[0], 0, sb));
    SPFC_CK(cudaMemset(S_.s[1], 0, sb));
    SPFC_CK(cudaMemset(Nhat_, 0, sb));
    // opt in to > 48 KB dynamic shared memory where a tile needs it
    SPFC_CK(set_smem(k2d_col_inv<R, N, E, CT, CI_STEP>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_inv<R, N, E, CT, CI_GRAD>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_inv<R, N, E, CT, CI_FIELD>, smem_col(1)));
    SPFC_CK(set_smem(k2d_row<R, N, E, RPC, RW_NONLIN>, smem_row()));
    SPFC_CK(set_smem(k2d_row<R, N, E, RPC, RW_ENERGY>, smem_row()));
    SPFC_CK(set_smem(k2d_row<R, N, E, RPC, RW_OUT_REAL>, smem_row()));
    SPFC_CK(set_smem(k2d_row<R, N, E, RPC, RW_IN_REAL>, smem_row()));
    SPFC_CK(set_smem(k2d_col_fwd<R, N, E, CT, CF_BDF2>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_fwd<R, N, E, CT, CF_BDF1>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_fwd<R, N, E, CT, CF_NHAT>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_fwd<R, N, E, CT, CF_TO_STATE>, smem_col(1)));
    SPFC_CK(set_smem(k2d_col_fused<R, N, E, CT, false>, smem_col(2)));
    SPFC_CK(set_smem(k2d_col_fused<R, N, E, CT, true>, smem_col(2)));
    {
      // the fused pass needs all of its blocks co-resident
      int dev = 0, nsm = 0, per = 0;
      SPFC_CK(cudaGetDevice(&dev));
      SPFC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      SPFC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k2d_col_fused<R, N, E, CT, false>, CT * T,
                                                             smem_col(2)));
      if (per * nsm < GCOL) {
        err = "the fused column pass does not fit co-resident on this GPU";
        return 3;
      }
      if (PERSIST) {
        SPFC_CK(set_smem(k2d_step_persist<R, N, PEV>, PS::smem_bytes()));
        SPFC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k2d_step_persist<R, N, PEV>, PS::NT,
                                                               PS::smem_bytes()));
        if (per * nsm < PS::G) {
          err = "the persistent step does not fit co-resident on this GPU";
          return 3;
        }
      }
    }
    SPFC_CK(cudaStreamCreateWithFlags(&cap_st_, cudaStreamNonBlocking));
    return 0;
  }

  ~Solver2D() override {
    if (g1_) cudaGraphExecDestroy(g1_);
    if (g16_) cudaGraphExecDestroy(g16_);
    for (auto ev : evpool_) cudaEventDestroy(ev);
    if (cap_st_) cudaStreamDestroy(cap_st_);
    void* ptrs[] = {S_.s[0], S_.s[1], Nhat_, W_[0], W_[1], W2_, real_, partE_, partG_, partN_, partS_, sc_,
                    counter_, sync64_, sync64p_, partP_, tw_};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    if (hsc_) cudaFreeHost(hsc_);
  }

  int64_t device_bytes() const override { return (int64_t)total_; }

  // ---- init / state --------------------------------------------------------
  int init(const double* phi0, bool on_device, int mode) override {
    int rc = load_field(phi0, on_device, /*slot_rel=*/0, /*reset=*/true);
    if (rc) return rc;
    if (mode == 0 && lazy()) {  // BDF1 with the phi^4 term or the PFC model: the lazy form, completed at once
      rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
      rc = launch_row(RW_NONLIN); if (rc) return rc;
      rc = launch_col_fwd(CF_BDF1, 0); if (rc) return rc;
      rc = finalize(); if (rc) return rc;
      w_ready_ = false;
      inited = true;
      return sync();
    } else if (mode == 0) {  // BDF1: the first step, which also prepares W for the second
      rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
      rc = launch_row(RW_NONLIN); if (rc) return rc;
      rc = launch_fused(true); if (rc) return rc;
      w_ready_ = true;
      inited = true;
      return sync();
    } else if (mode == 1) {  // ghost
      rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
      rc = launch_row(RW_NONLIN); if (rc) return rc;
      rc = scalar_op(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
      rc = launch_col_fwd(CF_NHAT, 0); if (rc) return rc;
      k2d_ghost<R><<<gpw_, PW_THREADS, 0, st_>>>(P, S_, Nhat_, sc_);
      SPFC_CK(cudaGetLastError());
      rc = launch_col_inv(CI_GRAD, 1); if (rc) return rc;
      rc = launch_row(RW_ENERGY); if (rc) return rc;
      rc = scalar_op(SO_R_PREV, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
    } else if (mode == 2) {  // copy
      rc = copy_newest_to_prev(); if (rc) return rc;
      rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
      rc = launch_row(RW_ENERGY); if (rc) return rc;
      rc = scalar_op(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
      rc = scalar_op(SO_R_PREV, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
    } else {
      err = "unknown start mode";
      return 1;
    }
    w_ready_ = false;
    inited = true;
    return 0;
  }

  int set_state(const double* phi, const double* phi_prev, double r, double r_prev, bool on_device) override {
    int rc = load_field(phi, on_device, 0, true);
    if (rc) return rc;
    rc = load_field(phi_prev, on_device, 1, false);
    if (rc) return rc;
    rc = scalar_op(SO_SET_R, nullptr, 0, nullptr, 0, 0, r, r_prev);
    if (rc) return rc;
    w_ready_ = false;
    inited = true;
    return 0;
  }

  int set_stab(double A) override {
    int rc = finalize(); if (rc) return rc;
    P.stab = A;
    fill_float_params(&P);
    drop_graphs();
    w_ready_ = false;
    return 0;
  }

  // The phi^4 term's kernels carry a third work array, allocated when the
  // term is first switched on. With it on, a step is the lazy three-pass form
  // (column inverse with the pending update, row pass, column forward with
  // the scalar solve) rather than row pass + fused column pass.
  int set_gamma3(double g3) override {
    if (pfc_on()) {
      err = "the PFC model takes its phi^4 coefficient from spfc_set_pfc";
      return 1;
    }
    if (inited) { int rc = finalize(); if (rc) return rc; }
    if (g3 != 0.0 && !W2_) {
      cudaError_t e = cudaMalloc((void**)&W2_, spec_bytes_);
      if (e != cudaSuccess) {
        W2_ = nullptr;
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return (e == cudaErrorMemoryAllocation) ? 2 : 3;
      }
      total_ += spec_bytes_;
      SPFC_CK(set_smem(k2d_col_inv_g3<R, N, E, CT, CI_STEP>, smem_col(2)));
      SPFC_CK(set_smem(k2d_col_inv_g3<R, N, E, CT, CI_GRAD>, smem_col(2)));
      SPFC_CK(set_smem(k2d_row_g3<R, N, E, RPC, RW_NONLIN>, 2 * smem_row()));
      SPFC_CK(set_smem(k2d_row_g3<R, N, E, RPC, RW_ENERGY>, 2 * smem_row()));
      SPFC_CK(set_smem(k2d_col_fwd_g3<R, N, E, CT, CF_BDF2>, smem_col(2)));
      SPFC_CK(set_smem(k2d_col_fwd_g3<R, N, E, CT, CF_BDF1>, smem_col(2)));
      SPFC_CK(set_smem(k2d_col_fwd_g3<R, N, E, CT, CF_NHAT>, smem_col(2)));
    }
    P.g3 = g3;
    fill_float_params(&P);
    drop_graphs();
    w_ready_ = false;
    return 0;
  }

  // The PFC model of Sec. 1 (eq. energy-PFC) with phi^4 coefficient g3 > 0,
  // or back to the SPFC model with g3 = 0 (the optional phi^4 term then off).
  int set_pfc(double g3) override {
    if (inited) { int rc = finalize(); if (rc) return rc; }
    if (g3 > 0.0) {
      SPFC_CK(set_smem(k2d_col_inv_pfc<R, N, E, CT, CI_STEP>, smem_col(1)));
      SPFC_CK(set_smem(k2d_col_inv_pfc<R, N, E, CT, CI_GRAD>, smem_col(1)));
      SPFC_CK(set_smem(k2d_row_pfc<R, N, E, RPC, RW_NONLIN>, smem_row()));
      SPFC_CK(set_smem(k2d_row_pfc<R, N, E, RPC, RW_ENERGY>, smem_row()));
      SPFC_CK(set_smem(k2d_col_fwd_pfc<R, N, E, CT, CF_BDF2>, smem_col(1)));
      SPFC_CK(set_smem(k2d_col_fwd_pfc<R, N, E, CT, CF_BDF1>, smem_col(1)));
      SPFC_CK(set_smem(k2d_col_fwd_pfc<R, N, E, CT, CF_NHAT>, smem_col(1)));
      P.pfc = 1;
      P.g3 = g3;
      P.C = 1.0 + 1.0 / (4.0 * g3);
    } else {
      P.pfc = 0;
      P.g3 = 0.0;
      P.C = 1.0 + 1.0 / P.beta;
    }
    fill_float_params(&P);
    drop_graphs();
    w_ready_ = false;
    return 0;
  }

  int dt_change(double dt) override {
    int rc = finalize(); if (rc) return rc;
    P.dt = dt;
    fill_float_params(&P);
    drop_graphs();
    rc = copy_newest_to_prev(); if (rc) return rc;
    rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
    rc = launch_row(RW_ENERGY); if (rc) return rc;
    rc = scalar_op(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
    rc = scalar_op(SO_R_PREV, partE_, nE_, nullptr, 0, 0); if (rc) return rc;
    w_ready_ = false;
    return 0;
  }

  // ---- stepping ------------------------------------------------------------
  int step(long long n) override {
    if (n <= 0) return 0;
    if (lazy()) pend_ = true;  // the lazy three-pass steps leave their update pending
    if (!w_ready_ && !lazy()) {
      // W <- inverse DFT in y of i k~ (2 phi^n - phi^{n-1}): the first half of a step
      int rc = finalize(); if (rc) return rc;
      rc = launch_col_inv(CI_STEP, 0); if (rc) return rc;
      w_ready_ = true;
    }
    if (timing_) {
      for (long long i = 0; i < n; ++i) {
        int rc = timed_step();
        if (rc) return rc;
      }
      return 0;
    }
    if (PERSIST && !lazy()) {  // one cooperative launch per chunk of steps
      while (n > 0) {
        const long long k = n < kPersistMaxSteps ? n : kPersistMaxSteps;
        int rc = launch_persist((int)k);
        if (rc) return rc;
        n -= k;
      }
      return 0;
    }
    int rc = ensure_graphs();
    if (rc) return rc;
    long long chunks = n / 16, rest = n % 16;
    for (long long i = 0; i < chunks; ++i) SPFC_CK(cudaGraphLaunch(g16_, st_));
    for (long long i = 0; i < rest; ++i) SPFC_CK(cudaGraphLaunch(g1_, st_));
    return 0;
  }

  // ---- diagnostics ----------------------------------------------------------
  int energy(double* E_orig, double* E_mod, double* E_breve) override {
    int rc = finalize(); if (rc) return rc;
    w_ready_ = false;  // W is used as scratch below
    k2d_norms<R><<<gpw_, PW_THREADS, 0, st_>>>(P, S_, sc_, partN_);
    SPFC_CK(cudaGetLastError());
    rc = launch_col_inv(CI_GRAD, 0); if (rc) return rc;
    rc = launch_row(RW_ENERGY); if (rc) return rc;
    rc = scalar_op(SO_ENERGY, partE_, nE_, partN_, gpw_, 0); if (rc) return rc;
    SavScal h;
    rc = read_scal(&h); if (rc) return rc;
    if (E_orig) *E_orig = h.E_orig;
    if (E_mod) *E_mod = h.E_mod;
    if (E_breve) *E_breve = h.E_breve;
    return 0;
  }

  int mass(double* m, double* mean) override {
    int rc = finalize(); if (rc) return rc;
    SavScal h;
    rc = read_scal(&h); if (rc) return rc;
    if (m) *m = P.vol * h.zm[h.p];
    if (mean) *mean = h.zm[h.p];
    return 0;
  }

  int scalars(SavScal* out) override {
    int rc = finalize(); if (rc) return rc;
    return read_scal(out);
  }

  int get_field(double* out, bool on_device, int which) override {
    int rc = finalize(); if (rc) return rc;
    w_ready_ = false;  // W is used as scratch below
    rc = launch_col_inv(CI_FIELD, which); if (rc) return rc;
    rc = launch_row(RW_OUT_REAL); if (rc) return rc;
    const size_t bytes = (size_t)N * N * sizeof(double);
    SPFC_CK(cudaMemcpyAsync(out, real_, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st_));
    return sync();
  }

  int sync() override {
    SPFC_CK(cudaMemcpyAsync(hsc_, sc_, sizeof(SavScal), cudaMemcpyDeviceToHost, st_));  // after all queued work
    SPFC_CK(cudaStreamSynchronize(st_));
    SavScal h = *hsc_;
    if (h.status != DEV_OK) {
      err = "device status: non-finite value or infeasible SAV scalar system";
      return h.status;
    }
    return 0;
  }

  int dump(std::string* blob) override {
    int rc = finalize(); if (rc) return rc;
    SavScal h;
    rc = read_scal(&h); if (rc) return rc;
    blob->assign(sizeof(SavScal) + 2 * spec_bytes_, '\0');
    char* b = &(*blob)[0];
    std::memcpy(b, &h, sizeof(SavScal));
    SPFC_CK(cudaMemcpy(b + sizeof(SavScal), S_.s[h.p], spec_bytes_, cudaMemcpyDeviceToHost));
    SPFC_CK(cudaMemcpy(b + sizeof(SavScal) + spec_bytes_, S_.s[1 - h.p], spec_bytes_, cudaMemcpyDeviceToHost));
    return 0;
  }

  int restore(const std::string& blob) override {
    if (blob.size() != sizeof(SavScal) + 2 * spec_bytes_) { err = "checkpoint size mismatch"; return 1; }
    w_ready_ = false;
    SavScal h;
    std::memcpy(&h, blob.data(), sizeof(SavScal));
    const int p = h.p;
    h.p = 0;
    h.pending = PEND_NONE;
    h.status = DEV_OK;
    const double z0 = h.zm[p], z1 = h.zm[1 - p];
    h.zm[0] = z0;
    h.zm[1] = z1;
    apply_ring(&h);
    drop_graphs();
    SPFC_CK(cudaStreamSynchronize(st_));
    if (int rc = reset_barriers()) return rc;
    SPFC_CK(cudaMemcpy(S_.s[0], blob.data() + sizeof(SavScal), spec_bytes_, cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(S_.s[1], blob.data() + sizeof(SavScal) + spec_bytes_, spec_bytes_, cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(sc_, &h, sizeof(SavScal), cudaMemcpyHostToDevice));
    inited = true;
    return 0;
  }

  int set_ring(double* dev, long long cap) override {
    SPFC_CK(cudaStreamSynchronize(st_));
    ring_dev = dev;
    ring_cap = cap;
    SPFC_CK(cudaMemcpy(&sc_->ring, &ring_dev, sizeof(double*), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(&sc_->ring_cap, &ring_cap, sizeof(long long), cudaMemcpyHostToDevice));
    return 0;
  }

  int set_timing(bool on) override {
    timing_ = on;
    return 0;
  }

  int kernel_times(KernelTimes* kt) override {
    SPFC_CK(cudaStreamSynchronize(st_));
    for (auto& rec : trecs_) {
      float ms = 0.f;
      SPFC_CK(cudaEventElapsedTime(&ms, evpool_[rec.e0], evpool_[rec.e1]));
      tms_[rec.cls] += ms;
      tcount_[rec.cls] += 1;
    }
    trecs_.clear();
    evnext_ = 0;
    if (PERSIST && !lazy()) {
      kt->names = {"step"};
      kt->launches.assign(tcount_, tcount_ + 1);
      kt->ms.assign(tms_, tms_ + 1);
    } else {
      kt->names = {"row", lazy() ? "col_inv+col_fwd" : "col_fused"};
      kt->launches.assign(tcount_, tcount_ + 2);
      kt->ms.assign(tms_, tms_ + 2);
    }
    for (int i = 0; i < 3; ++i) { tcount_[i] = 0; tms_[i] = 0.0; }
    return 0;
  }

 private:
  template <typename K> static cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  static constexpr int CTP = col_pitch(CT);
  static constexpr size_t smem_col(int nf) { return (size_t)nf * sp_len(N) * CTP * sizeof(C); }
  static constexpr size_t smem_row() { return (size_t)RPC * (sp_len(N) + 1) * sizeof(C); }

  bool pfc_on() const { return P.pfc != 0; }
  bool g3_on() const { return P.g3 != 0.0 && !pfc_on(); }  // the optional phi^4 term of the SPFC model
  bool lazy() const { return g3_on() || pfc_on(); }        // steps in the lazy three-pass form

  int launch_col_inv(int mode, int which) {
    if (pfc_on() && (mode == CI_STEP || mode == CI_GRAD)) {
      if (mode == CI_STEP)
        k2d_col_inv_pfc<R, N, E, CT, CI_STEP><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, Nhat_, W_[0], sc_, tw_, which);
      else
        k2d_col_inv_pfc<R, N, E, CT, CI_GRAD><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, Nhat_, W_[0], sc_, tw_, which);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    if (g3_on() && (mode == CI_STEP || mode == CI_GRAD)) {
      if (mode == CI_STEP)
        k2d_col_inv_g3<R, N, E, CT, CI_STEP><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], W2_, sc_, tw_, which);
      else
        k2d_col_inv_g3<R, N, E, CT, CI_GRAD><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], W2_, sc_, tw_, which);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case CI_STEP:
        SPFC_CK(launch_k(k2d_col_inv<R, N, E, CT, CI_STEP>, GCOL, CT * T, smem_col(2), st_, pdl_, false, P, S_, Nhat_,
                         W_[0], W_[1], sc_, tw_, which));
        break;
      case CI_GRAD:
        k2d_col_inv<R, N, E, CT, CI_GRAD><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which);
        break;
      default:
        k2d_col_inv<R, N, E, CT, CI_FIELD><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int launch_row(int mode) {
    if (pfc_on() && (mode == RW_NONLIN || mode == RW_ENERGY)) {
      if (mode == RW_NONLIN)
        k2d_row_pfc<R, N, E, RPC, RW_NONLIN><<<GROW, RPC * T, smem_row(), st_>>>(P, W_[0], partE_, sc_, tw_);
      else
        k2d_row_pfc<R, N, E, RPC, RW_ENERGY><<<GROW, RPC * T, smem_row(), st_>>>(P, W_[0], partE_, sc_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    if (g3_on() && (mode == RW_NONLIN || mode == RW_ENERGY)) {
      if (mode == RW_NONLIN)
        k2d_row_g3<R, N, E, RPC, RW_NONLIN><<<GROW, RPC * T, 2 * smem_row(), st_>>>(P, W_[0], W_[1], W2_, partE_, sc_, tw_);
      else
        k2d_row_g3<R, N, E, RPC, RW_ENERGY><<<GROW, RPC * T, 2 * smem_row(), st_>>>(P, W_[0], W_[1], W2_, partE_, sc_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case RW_NONLIN:
        SPFC_CK(launch_k(k2d_row<R, N, E, RPC, RW_NONLIN>, GROW, RPC * T, smem_row(), st_, pdl_, false, P, W_[0], W_[1],
                         partE_, sc_, tw_, real_));
        break;
      case RW_ENERGY:
        k2d_row<R, N, E, RPC, RW_ENERGY><<<GROW, RPC * T, smem_row(), st_>>>(P, W_[0], W_[1], partE_, sc_, tw_, real_);
        break;
      case RW_OUT_REAL:
        k2d_row<R, N, E, RPC, RW_OUT_REAL><<<GROW, RPC * T, smem_row(), st_>>>(P, W_[0], W_[1], partE_, sc_, tw_, real_);
        break;
      default:
        k2d_row<R, N, E, RPC, RW_IN_REAL><<<GROW, RPC * T, smem_row(), st_>>>(P, W_[0], W_[1], partE_, sc_, tw_, real_);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int launch_col_fwd(int mode, int target) {
    if (mode == CF_BDF2 || mode == CF_BDF1) pend_ = true;  // the scalar solve leaves the update pending
    if (pfc_on() && mode != CF_TO_STATE) {
      if (mode == CF_BDF2)
        k2d_col_fwd_pfc<R, N, E, CT, CF_BDF2><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, W_[0], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      else if (mode == CF_BDF1)
        k2d_col_fwd_pfc<R, N, E, CT, CF_BDF1><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, W_[0], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      else
        k2d_col_fwd_pfc<R, N, E, CT, CF_NHAT><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, W_[0], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    if (g3_on() && mode != CF_TO_STATE) {
      if (mode == CF_BDF2)
        k2d_col_fwd_g3<R, N, E, CT, CF_BDF2><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      else if (mode == CF_BDF1)
        k2d_col_fwd_g3<R, N, E, CT, CF_BDF1><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      else
        k2d_col_fwd_g3<R, N, E, CT, CF_NHAT><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case CF_BDF2:
        SPFC_CK(launch_k(k2d_col_fwd<R, N, E, CT, CF_BDF2>, GCOL, CT * T, smem_col(2), st_, pdl_, false, P, S_, W_[0],
                         W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_, target));
        break;
      case CF_BDF1:
        k2d_col_fwd<R, N, E, CT, CF_BDF1><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_, target);
        break;
      case CF_NHAT:
        k2d_col_fwd<R, N, E, CT, CF_NHAT><<<GCOL, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_, target);
        break;
      default:
        k2d_col_fwd<R, N, E, CT, CF_TO_STATE><<<GCOL, CT * T, smem_col(1), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, partE_, nE_, sc_, counter_, tw_, target);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int scalar_op(int op, const double* a, int na, const double* b, int nb, int arg, double x0 = 0, double x1 = 0) {
    k_scalar_op<R><<<1, 32, 0, st_>>>(P, sc_, op, a, na, b, nb, arg, x0, x1);
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int read_scal(SavScal* h) {
    SPFC_CK(cudaMemcpyAsync(hsc_, sc_, sizeof(SavScal), cudaMemcpyDeviceToHost, st_));
    SPFC_CK(cudaStreamSynchronize(st_));
    *h = *hsc_;
    if (h->status != DEV_OK) {
      err = "device status: non-finite value or infeasible SAV scalar system";
      return h->status;
    }
    return 0;
  }

  // materialise a pending update (no-op otherwise). Only the lazy column
  // forward pass leaves one (the fused pass commits its update), so with no
  // such pass since the last finalize there is nothing to launch.
  int finalize() {
    if (!pend_) return 0;
    k2d_finalize<R><<<gpw_, PW_THREADS, 0, st_>>>(P, S_, Nhat_, sc_);
    SPFC_CK(cudaGetLastError());
    int rc = scalar_op(SO_FLIP, nullptr, 0, nullptr, 0, 0);
    if (!rc) pend_ = false;
    return rc;
  }

  int copy_newest_to_prev() {
    SavScal h;
    int rc = read_scal(&h);
    if (rc) return rc;
    SPFC_CK(cudaMemcpyAsync(S_.s[1 - h.p], S_.s[h.p], spec_bytes_, cudaMemcpyDeviceToDevice, st_));
    h.zm[1 - h.p] = h.zm[h.p];
    SPFC_CK(cudaMemcpyAsync(sc_, &h, sizeof(SavScal), cudaMemcpyHostToDevice, st_));
    SPFC_CK(cudaStreamSynchronize(st_));
    return 0;
  }

  // Transform a real field into slot (newest if slot_rel == 0, previous
  // otherwise). reset: clear the scalar record first (p = 0, no pending).
  int load_field(const double* f, bool on_device, int slot_rel, bool reset) {
    const size_t bytes = (size_t)N * N * sizeof(double);
    if (reset) {
      // the cleared record goes up from the pinned buffer, so the copy does not
      // synchronise the stream; the buffer is not written again before the
      // synchronisation at the end of this call
      *hsc_ = SavScal{};
      apply_ring(hsc_);
      SPFC_CK(cudaMemcpyAsync(sc_, hsc_, sizeof(SavScal), cudaMemcpyHostToDevice, st_));
      reset_barriers();
      drop_graphs();
    }
    SPFC_CK(cudaMemcpyAsync(real_, f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st_));
    k_real_sum<<<gpw_, PW_THREADS, 0, st_>>>(real_, (size_t)N * N, partS_);
    SPFC_CK(cudaGetLastError());
    int rc = scalar_op(SO_ZM_SLOT, partS_, gpw_, nullptr, 0, slot_rel);
    if (rc) return rc;
    rc = launch_row(RW_IN_REAL); if (rc) return rc;
    // slot index: p = 0 after a reset, so newest = 0 and previous = 1
    rc = launch_col_fwd(CF_TO_STATE, slot_rel == 0 ? 0 : 1); if (rc) return rc;
    k_put_zero_modes<R><<<1, 1, 0, st_>>>(S_, sc_);
    SPFC_CK(cudaGetLastError());
    SPFC_CK(cudaStreamSynchronize(st_));
    return 0;
  }

  // one step with W prepared: row pass, then the fused column pass (which
  // prepares W for the next step)
  int launch_step_kernels() {
    if (lazy()) {  // lazy three-pass form: the update stays pending between steps
      int rc = launch_col_inv(CI_STEP, 0); if (rc) return rc;
      rc = launch_row(RW_NONLIN); if (rc) return rc;
      return launch_col_fwd(CF_BDF2, 0);
    }
    int rc = launch_row(RW_NONLIN); if (rc) return rc;
    return launch_fused(false);
  }

  int launch_fused(bool bdf1) {
    if (bdf1)
      SPFC_CK(launch_k(k2d_col_fused<R, N, E, CT, true>, GCOL, CT * T, smem_col(2), st_, false, true, P, S_,
                       W_[0], W_[1], partG_, partE_, nE_, sc_, sync64_, tw_));
    else
      SPFC_CK(launch_k(k2d_col_fused<R, N, E, CT, false>, GCOL, CT * T, smem_col(2), st_, false, true, P, S_,
                       W_[0], W_[1], partG_, partE_, nE_, sc_, sync64_, tw_));
    return 0;
  }

  // The grid barriers count arrivals on monotone counters whose rounds are
  // whole multiples of the grid; a launch that stopped inside a round (a
  // latched failure) leaves a remainder, so a new start clears them.
  int reset_barriers() {
    SPFC_CK(cudaMemsetAsync(sync64_, 0, sizeof(unsigned long long), st_));
    if (PERSIST) SPFC_CK(cudaMemsetAsync(sync64p_, 0, sizeof(unsigned long long), st_));
    bar_rounds_ = 0;
    return 0;
  }

  // nsteps BDF2 steps in one cooperative launch (W prepared, nothing pending)
  int launch_persist(int nsteps) {
    const unsigned long long base = bar_rounds_ * (unsigned long long)PS::G;
    SPFC_CK(launch_k(k2d_step_persist<R, N, PEV>, PS::G, PS::NT, PS::smem_bytes(), st_, false, true, P, S_, W_[0],
                     W_[1], partP_, partP_ + 2 * PS::G, sc_, sync64p_, base, tw_, nsteps));
    bar_rounds_ += 3ull * (unsigned long long)nsteps - 1ull;  // the launch's barrier rounds
    return 0;
  }

  void drop_graphs() {
    if (g1_) { cudaGraphExecDestroy(g1_); g1_ = nullptr; }
    if (g16_) { cudaGraphExecDestroy(g16_); g16_ = nullptr; }
  }

  int capture(int nsteps, cudaGraphExec_t* out) {
    cudaStream_t keep = st_;
    st_ = cap_st_;
    pdl_ = use_pdl_;
    cudaGraph_t g = nullptr;
    SPFC_CK(cudaStreamBeginCapture(cap_st_, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int i = 0; i < nsteps && rc == 0; ++i) rc = launch_step_kernels();
    cudaError_t e = cudaStreamEndCapture(cap_st_, &g);
    st_ = keep;
    pdl_ = false;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) { err = std::string("graph capture: ") + cudaGetErrorString(e); return 3; }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { err = std::string("graph instantiate: ") + cudaGetErrorString(e); return 3; }
    return 0;
  }

  int ensure_graphs() {
    if (!g1_) { int rc = capture(1, &g1_); if (rc) return rc; }
    if (!g16_) { int rc = capture(16, &g16_); if (rc) return rc; }
    return 0;
  }

  int ev(int* idx) {
    if (evnext_ >= (int)evpool_.size()) {
      cudaEvent_t e;
      SPFC_CK(cudaEventCreate(&e));
      evpool_.push_back(e);
    }
    *idx = evnext_++;
    return 0;
  }

  int timed_step() {
    int e0, e1, e2, rc;
    if (lazy()) {  // row pass in class 0, the two column passes in class 1
      int e3;
      if ((rc = ev(&e0)) || (rc = ev(&e1)) || (rc = ev(&e2)) || (rc = ev(&e3))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e0], st_));
      if ((rc = launch_col_inv(CI_STEP, 0))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e1], st_));
      if ((rc = launch_row(RW_NONLIN))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e2], st_));
      if ((rc = launch_col_fwd(CF_BDF2, 0))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e3], st_));
      trecs_.push_back({1, e0, e1});
      trecs_.push_back({0, e1, e2});
      trecs_.push_back({1, e2, e3});
      return 0;
    }
    if (PERSIST) {
      if ((rc = ev(&e0)) || (rc = ev(&e1))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e0], st_));
      if ((rc = launch_persist(1))) return rc;
      SPFC_CK(cudaEventRecord(evpool_[e1], st_));
      trecs_.push_back({0, e0, e1});
      return 0;
    }
    if ((rc = ev(&e0)) || (rc = ev(&e1)) || (rc = ev(&e2))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e0], st_));
    if ((rc = launch_row(RW_NONLIN))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e1], st_));
    if ((rc = launch_fused(false))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e2], st_));
    trecs_.push_back({0, e0, e1});
    trecs_.push_back({1, e1, e2});
    return 0;
  }

  struct TRec { int cls, e0, e1; };

  cudaStream_t st_ = nullptr, cap_st_ = nullptr;
  Slots<R> S_{{nullptr, nullptr}};
  C* Nhat_ = nullptr;
  C* W_[2] = {nullptr, nullptr};
  C* W2_ = nullptr;                 // third work array of the phi^4 term (allocated on demand)
  double* real_ = nullptr;
  double *partE_ = nullptr, *partG_ = nullptr, *partN_ = nullptr, *partS_ = nullptr;
  SavScal* sc_ = nullptr;
  SavScal* hsc_ = nullptr;  // pinned host copy of the record
  unsigned* counter_ = nullptr;
  unsigned long long* sync64_ = nullptr;  // arrival counter of the fused pass's grid barrier
  unsigned long long* sync64p_ = nullptr; // arrival counter of the persistent step's grid barriers
  double* partP_ = nullptr;               // the persistent step's partial sums: E_1 [2][G], gamma/eta/theta [3][G]
  unsigned long long bar_rounds_ = 0;     // barrier rounds the persistent launches issued since the last reset
  C* tw_ = nullptr;
  int gpw_ = 0, nE_ = 0, nG_ = 0;
  size_t spec_bytes_ = 0, total_ = 0;
  cudaGraphExec_t g1_ = nullptr, g16_ = nullptr;
  bool timing_ = false;
  bool w_ready_ = false;            // W holds the first half of the next step
  bool pend_ = false;               // a lazy pass may have left an update pending on the device
  bool pdl_ = false;                // launch the step kernels with programmatic serialization
  bool use_pdl_ = false;
  std::vector<cudaEvent_t> evpool_;
  int evnext_ = 0;
  std::vector<TRec> trecs_;
  int64_t tcount_[3] = {0, 0, 0};
  double tms_[3] = {0, 0, 0};
};

// Number of launch schedules compiled for a 2D grid size: the tile shapes of
// the two-kernel step (six from N = 128, one below) and the persistent step.
inline int num_schedules_2d(int N) { return (N >= 128 ? persist_e4_schedule(N) : persist_schedule(N)) + 1; }

template <typename R, int N, int SCHED>
SolverBase* new_solver_2d(const Params& P, cudaStream_t st, int* status, std::string* err) {
  auto* s = new Solver2D<R, N, SCHED>(P, st);
  int rc = s->setup();
  if (rc) {
    *status = rc;
    *err = s->err;
    delete s;
    return nullptr;
  }
  s->schedule = SCHED;
  return s;
}

// Factory for one grid size N >= 256 (each in its own translation unit so
// that the build compiles them in parallel).
template <typename R, int N>
SolverBase* make_solver_2d_n(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  switch (schedule) {
    case 1: return new_solver_2d<R, N, 1>(P, st, status, err);
    case 2: return new_solver_2d<R, N, 2>(P, st, status, err);
    case 3: return new_solver_2d<R, N, 3>(P, st, status, err);
    case 4: return new_solver_2d<R, N, 4>(P, st, status, err);
    case 5: return new_solver_2d<R, N, 5>(P, st, status, err);
    case 6: return new_solver_2d<R, N, 6>(P, st, status, err);
    case 7: return new_solver_2d<R, N, 7>(P, st, status, err);
    default: return new_solver_2d<R, N, 0>(P, st, status, err);
  }
}

SolverBase* make_solver_2d_f64_128(const Params&, cudaStream_t, int, int*, std::string*);
SolverBase* make_solver_2d_f32_128(const Params&, cudaStream_t, int, int*, std::string*);
SolverBase* make_solver_2d_f64_256(const Params&, cudaStream_t, int, int*, std::string*);
SolverBase* make_solver_2d_f64_512(const Params&, cudaStream_t, int, int*, std::string*);
SolverBase* make_solver_2d_f32_256(const Params&, cudaStream_t, int, int*, std::string*);
SolverBase* make_solver_2d_f32_512(const Params&, cudaStream_t, int, int*, std::string*);

template <typename R>
SolverBase* make_solver_2d(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  const bool known = P.N == 16 || P.N == 32 || P.N == 64 || P.N == 128 || P.N == 256 || P.N == 512;
  if (!known) {
    *status = 1;
    *err = "2D grid size must be one of 16, 32, 64, 128, 256, 512";
    return nullptr;
  }
  if (schedule < 0 || schedule >= num_schedules_2d(P.N)) {
    *status = 1;
    *err = "schedule index out of range for this grid size";
    return nullptr;
  }
  constexpr bool F64 = sizeof(R) == 8;
  switch (P.N) {
    case 16: return schedule ? new_solver_2d<R, 16, 1>(P, st, status, err) : new_solver_2d<R, 16, 0>(P, st, status, err);
    case 32: return schedule ? new_solver_2d<R, 32, 1>(P, st, status, err) : new_solver_2d<R, 32, 0>(P, st, status, err);
    case 64: return schedule ? new_solver_2d<R, 64, 1>(P, st, status, err) : new_solver_2d<R, 64, 0>(P, st, status, err);
    case 128:
      return F64 ? make_solver_2d_f64_128(P, st, schedule, status, err) : make_solver_2d_f32_128(P, st, schedule, status, err);
    case 256:
      return F64 ? make_solver_2d_f64_256(P, st, schedule, status, err) : make_solver_2d_f32_256(P, st, schedule, status, err);
    default:
      return F64 ? make_solver_2d_f64_512(P, st, schedule, status, err) : make_solver_2d_f32_512(P, st, schedule, status, err);
  }
}

}  // namespace spfc
