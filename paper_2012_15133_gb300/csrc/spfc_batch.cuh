// Batched ensemble of independent 2D runs (uneven grid sizes and parameters).
//
// Runs of one grid size N form a class whose buffers are contiguous
// (run r's spectrum at offset r * N * (N/2+1)); each class steps with four
// batched launches whose blockIdx.y is the run:
//   row pass -> forward column pass (N_hat, partial sums) -> per-run scalar
//   solve (one block per run) -> inverse column pass (update, next
//   extrapolation, its gradients).
// The classes are independent branches of one CUDA graph per step. A run
// whose status latches an error stops (its blocks return early); the others
// continue. Start-up and diagnostics reuse the single-run solver on one run
// at a time.
#pragma once

#include "spfc_solver2d.cuh"

namespace spfc {

template <typename R> struct BatchView {
  C_t<R>* S0;
  C_t<R>* S1;
  C_t<R>* Nhat;
  C_t<R>* W0;
  C_t<R>* W1;
  C_t<R>* W2;   // third work array of the phi^4 term (allocated when a run of the class has one)
  double* partE;
  double* partG;
  SavScal* sc;
  const Params* P;
  size_t spec;  // complex entries per run and array
  int nE, nG;   // partial-sum blocks per run (row pass, column pass)
};

// Resident blocks per SM asked of the compiler for the batched passes (their
// many blocks hide load and shared-memory latency): 24 warps per SM on the
// float32 path (at most 85 registers per thread; 32 warps spill the row pass
// and measured slower), none on the float64 path.
template <typename R> constexpr int batch_min_blocks(int threads) {
  return sizeof(R) == 8 ? 1 : (24 * 32 + threads - 1) / threads;
}

template <typename R, int N, int E, int RPC>
__global__ void __launch_bounds__(RPC * (N / E), batch_min_blocks<R>(RPC * (N / E)))
k2b_row(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  k2d_row_body<R, N, E, RPC, RW_NONLIN>(B.P[r], B.W0 + r * B.spec, B.W1 + r * B.spec, B.partE + (size_t)r * 2 * B.nE,
                                        B.sc + r, tw, nullptr);
}

template <typename R, int N, int E, int CT>
__global__ void __launch_bounds__(CT * (N / E), batch_min_blocks<R>(CT * (N / E)))
k2b_col_fwd(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  Slots<R> S{{B.S0 + r * B.spec, B.S1 + r * B.spec}};
  k2d_col_fwd_body<R, N, E, CT, CF_PART>(B.P[r], S, B.W0 + r * B.spec, B.W1 + r * B.spec, B.Nhat + r * B.spec,
                                        B.partG + (size_t)r * 3 * B.nG, nullptr, 0, B.sc + r, nullptr, tw, 0);
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E), batch_min_blocks<R>(CT * (N / E)))
k2b_col_inv(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  Slots<R> S{{B.S0 + r * B.spec, B.S1 + r * B.spec}};
  k2d_col_inv_body<R, N, E, CT, MODE>(B.P[r], S, B.Nhat + r * B.spec, B.W0 + r * B.spec, B.W1 + r * B.spec, B.sc + r,
                                      tw, 0);
}

// The same passes with the phi^4 channel (a class with a run whose gamma3 is
// not 0; runs with gamma3 = 0 in it add zeros). No residency bound: the extra
// sequence of the row pass would not fit 85 registers.
template <typename R, int N, int E, int RPC>
__global__ void __launch_bounds__(RPC * (N / E))
k2b_row_g3(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  k2d_row_body<R, N, E, RPC, RW_NONLIN, true>(B.P[r], B.W0 + r * B.spec, B.W1 + r * B.spec,
                                              B.partE + (size_t)r * 2 * B.nE, B.sc + r, tw, nullptr,
                                              B.W2 + r * B.spec);
}

template <typename R, int N, int E, int CT>
__global__ void __launch_bounds__(CT * (N / E))
k2b_col_fwd_g3(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  Slots<R> S{{B.S0 + r * B.spec, B.S1 + r * B.spec}};
  k2d_col_fwd_body<R, N, E, CT, CF_PART, true>(B.P[r], S, B.W0 + r * B.spec, B.W1 + r * B.spec,
                                              B.Nhat + r * B.spec, B.partG + (size_t)r * 3 * B.nG, nullptr, 0,
                                              B.sc + r, nullptr, tw, 0);
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2b_col_inv_g3(BatchView<R> B, const C_t<R>* __restrict__ tw) {
  const int r = blockIdx.y;
  Slots<R> S{{B.S0 + r * B.spec, B.S1 + r * B.spec}};
  k2d_col_inv_body<R, N, E, CT, MODE, true>(B.P[r], S, B.Nhat + r * B.spec, B.W0 + r * B.spec, B.W1 + r * B.spec,
                                            B.sc + r, tw, 0, B.W2 + r * B.spec);
}

// One block per run: reduce the run's partial sums and solve its scalar
// system; the inverse column pass then applies the update into slot p.
template <typename R>
__global__ void __launch_bounds__(256)
k2b_scalar(BatchView<R> B) {
  __shared__ double red5[5][32];
  __shared__ double qres[5];
  const int r = blockIdx.x;
  SavScal* sc = B.sc + r;
  if (sc->status != DEV_OK) return;
  const double* pe = B.partE + (size_t)r * 2 * B.nE;
  const double* pg = B.partG + (size_t)r * 3 * B.nG;
  const double* arr[5] = {pe, pe + B.nE, pg, pg + B.nG, pg + 2 * B.nG};
  const int cnt[5] = {B.nE, B.nE, B.nG, B.nG, B.nG};
  block_sum_arrays<5>(arr, cnt, qres, red5);
  if (threadIdx.x == 0) {
    const SolveOut o = sav_solve(B.P[r], qres, false, RIn(sc));
    sav_commit(sc, o, 1 - sc->p, PEND_NONE);
  }
}

// A class: all runs of one grid size.
class BatchClassBase {
 public:
  virtual ~BatchClassBase() {}
  virtual int launch_step(cudaStream_t st) = 0;         // one step of every run in the class
  virtual int prepare(cudaStream_t st) = 0;             // W <- first half of the next step
  virtual int load_run(int local, const double* phi0, int mode) = 0;
  virtual int set_run_state(int local, const double* phi, const double* phi_prev, double r, double r_prev) = 0;
  virtual int run_field(int local, double* out, int which) = 0;
  virtual int run_scalars(int local, SavScal* out) = 0;
  virtual int run_energy(int local, double* e3) = 0;
  virtual int set_gamma3(int local, double g3) = 0;     // the phi^4 term of one run
  virtual int64_t device_bytes() const = 0;
  int N = 0, nruns = 0, schedule = 0;
  std::vector<int> runs;  // global run indices
  std::string err;
};

// The float32 batch uses 4-column tiles for N >= 256 (schedule 4): with many
// runs the column passes stream from HBM, and 4 float32 complex values fill a
// 32-byte sector per row. The float64 batch, bound by its arithmetic, uses the
// shapes with the most threads (schedule 5) from N = 128.
template <typename R, int N> constexpr int batch_sched() {
  return sizeof(R) == 8 ? (N >= 128 ? 5 : 0) : (N >= 256 ? 4 : 0);
}

// The tile shapes (Shape2D schedules) a batch class can be built with: from
// N = 128 the four that fill whole sectors or give the most threads (0, 2,
// 4, 5), one below. The autotuner times them per grid size and precision.
inline bool batch_schedule_valid(int N, int sched) {
  if (N < 128) return sched == 0;
  return sched == 0 || sched == 2 || sched == 4 || sched == 5;
}

template <typename R, int N_, int SCHED>
class BatchClass final : public BatchClassBase {
  using C = C_t<R>;
  using SH = Shape2D<N_, SCHED>;
  static constexpr int NH = N_ / 2 + 1;
  static constexpr int E = SH::E, T = SH::T, CT = SH::CT, RPC = SH::RPC, CTP = col_pitch(CT);
  static constexpr int GCOL = (NH + CT - 1) / CT, GROW = N_ / RPC;

 public:
  BatchClass(const std::vector<Params>& params, cudaStream_t st) : params_(params), st_(st) {
    N = N_;
    nruns = (int)params.size();
  }

  int setup() {
    const size_t spec = (size_t)N_ * NH;
    v_.spec = spec;
    v_.nE = GROW;
    v_.nG = GCOL;
    const size_t sb = spec * sizeof(C) * nruns;
    auto al = [&](void** p, size_t b) -> cudaError_t {
      cudaError_t e = cudaMalloc(p, b);
      if (e == cudaSuccess) total_ += b;
      return e;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = al((void**)&v_.S0, sb);
    if (e == cudaSuccess) e = al((void**)&v_.S1, sb);
    if (e == cudaSuccess) e = al((void**)&v_.Nhat, sb);
    if (e == cudaSuccess) e = al((void**)&v_.W0, sb);
    if (e == cudaSuccess) e = al((void**)&v_.W1, sb);
    if (e == cudaSuccess) e = al((void**)&v_.partE, (size_t)nruns * 2 * GROW * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&v_.partG, (size_t)nruns * 3 * GCOL * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&v_.sc, (size_t)nruns * sizeof(SavScal));
    if (e == cudaSuccess) e = al((void**)&Pdev_, (size_t)nruns * sizeof(Params));
    if (e == cudaSuccess) e = al((void**)&tw_, TW_LEN * sizeof(C));
    if (e != cudaSuccess) {
      err = std::string("device allocation failed: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? 2 : 3;
    }
    v_.P = Pdev_;
    std::vector<C> tw;
    host_twiddles<R>(tw);
    SPFC_CK(cudaMemcpy(tw_, tw.data(), TW_LEN * sizeof(C), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(Pdev_, params_.data(), nruns * sizeof(Params), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemset(v_.sc, 0, nruns * sizeof(SavScal)));
    auto smc = (size_t)2 * sp_len(N_) * CTP * sizeof(C);
    auto smr = (size_t)RPC * (sp_len(N_) + 1) * sizeof(C);
    SPFC_CK(cudaFuncSetAttribute(k2b_row<R, N_, E, RPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
    SPFC_CK(cudaFuncSetAttribute(k2b_col_fwd<R, N_, E, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
    SPFC_CK(cudaFuncSetAttribute(k2b_col_inv<R, N_, E, CT, CI_STEP_COMMITTED>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
    SPFC_CK(cudaFuncSetAttribute(k2b_col_inv<R, N_, E, CT, CI_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smc));
    return 0;
  }

  ~BatchClass() override {
    delete one_;
    void* ptrs[] = {v_.S0, v_.S1, v_.Nhat, v_.W0, v_.W1, v_.W2, v_.partE, v_.partG, v_.sc, Pdev_, tw_};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }

  int64_t device_bytes() const override { return (int64_t)total_; }

  int launch_step(cudaStream_t st) override {
    const size_t smc = (size_t)2 * sp_len(N_) * CTP * sizeof(C);
    const size_t smr = (size_t)RPC * (sp_len(N_) + 1) * sizeof(C);
    if (g3_) {
      k2b_row_g3<R, N_, E, RPC><<<dim3(GROW, nruns), RPC * T, 2 * smr, st>>>(v_, tw_);
      k2b_col_fwd_g3<R, N_, E, CT><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
      k2b_scalar<R><<<nruns, 256, 0, st>>>(v_);
      k2b_col_inv_g3<R, N_, E, CT, CI_STEP_COMMITTED><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    k2b_row<R, N_, E, RPC><<<dim3(GROW, nruns), RPC * T, smr, st>>>(v_, tw_);
    k2b_col_fwd<R, N_, E, CT><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
    k2b_scalar<R><<<nruns, 256, 0, st>>>(v_);
    k2b_col_inv<R, N_, E, CT, CI_STEP_COMMITTED><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
    SPFC_CK(cudaGetLastError());
    return 0;
  }

  int prepare(cudaStream_t st) override {
    const size_t smc = (size_t)2 * sp_len(N_) * CTP * sizeof(C);
    if (g3_) k2b_col_inv_g3<R, N_, E, CT, CI_STEP><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
    else k2b_col_inv<R, N_, E, CT, CI_STEP><<<dim3(GCOL, nruns), CT * T, smc, st>>>(v_, tw_);
    SPFC_CK(cudaGetLastError());
    return 0;
  }

  // Start-up of one run with the single-run solver, then its state copied in.
  int load_run(int local, const double* phi0, int mode) override {
    int rc = ensure_one(local);
    if (rc) return rc;
    rc = one_->init(phi0, false, mode);
    if (rc) {
      // the run failed at its start: latch its status so the batched kernels
      // skip it while the other runs continue
      err = one_->err;
      SavScal h{};
      h.status = (rc == 4 || rc == 5) ? rc : DEV_NONFINITE;
      SPFC_CK(cudaMemcpy(v_.sc + local, &h, sizeof(SavScal), cudaMemcpyHostToDevice));
      return rc;
    }
    return export_one(local);
  }

  // Both time levels and r of one run set directly (the single-run solver
  // transforms them, then its state is copied in).
  int set_run_state(int local, const double* phi, const double* phi_prev, double r, double r_prev) override {
    int rc = ensure_one(local);
    if (rc) return rc;
    rc = one_->set_state(phi, phi_prev, r, r_prev, false);
    if (rc) { err = one_->err; return rc; }
    return export_one(local);
  }

  int run_field(int local, double* out, int which) override {
    int rc = import_one(local);
    if (!rc) rc = one_->get_field(out, false, which);
    if (rc && err.empty()) err = one_->err;
    return rc;
  }

  int run_scalars(int local, SavScal* out) override {
    SPFC_CK(cudaMemcpy(out, v_.sc + local, sizeof(SavScal), cudaMemcpyDeviceToHost));
    return out->status;
  }

  int run_energy(int local, double* e3) override {
    int rc = import_one(local);
    if (!rc) rc = one_->energy(e3, e3 + 1, e3 + 2);
    if (rc && err.empty()) err = one_->err;
    return rc;
  }

  // The run's constants (host and device) take the term; a class with any
  // run that has it steps with the G3 passes, W2 allocated on first need.
  int set_gamma3(int local, double g3) override {
    params_[local].g3 = g3;
    fill_float_params(&params_[local]);
    SPFC_CK(cudaMemcpy(Pdev_ + local, &params_[local], sizeof(Params), cudaMemcpyHostToDevice));
    if (g3 != 0.0 && !v_.W2) {
      cudaError_t e = cudaMalloc((void**)&v_.W2, v_.spec * sizeof(C) * nruns);
      if (e != cudaSuccess) {
        v_.W2 = nullptr;
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? 2 : 3;
      }
      total_ += v_.spec * sizeof(C) * nruns;
      const size_t smc = (size_t)2 * sp_len(N_) * CTP * sizeof(C);
      const size_t smr = (size_t)RPC * (sp_len(N_) + 1) * sizeof(C);
      SPFC_CK(cudaFuncSetAttribute(k2b_row_g3<R, N_, E, RPC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(2 * smr)));
      SPFC_CK(cudaFuncSetAttribute(k2b_col_fwd_g3<R, N_, E, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smc));
      SPFC_CK(cudaFuncSetAttribute(k2b_col_inv_g3<R, N_, E, CT, CI_STEP_COMMITTED>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
      SPFC_CK(cudaFuncSetAttribute(k2b_col_inv_g3<R, N_, E, CT, CI_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smc));
    }
    g3_ = false;
    for (const Params& q : params_) g3_ = g3_ || q.g3 != 0.0;
    one_run_ = -1;  // the single-run solver takes the new constants at its next use
    return 0;
  }

 private:
  int ensure_one(int local) {
    if (one_ && one_run_ == local) return 0;
    if (!one_) {
      auto* s = new Solver2D<R, N_, 0>(params_[local], st_);
      int rc = s->setup();
      if (rc) { err = s->err; delete s; return rc; }
      one_ = s;
    }
    one_->P = params_[local];  // kernels read the per-run constants at launch
    int rc = one_->set_gamma3(params_[local].g3);  // and its phi^4 kernels their work array
    if (rc) { err = one_->err; return rc; }
    one_run_ = local;
    return 0;
  }
  // single-run solver state <-> batch slots (newest level into slot 0)
  int export_one(int local) {
    std::string blob;
    int rc = one_->dump(&blob);
    if (rc) { err = one_->err; return rc; }
    const size_t sbytes = v_.spec * sizeof(C);
    SavScal h;
    std::memcpy(&h, blob.data(), sizeof(SavScal));
    const double z0 = h.zm[h.p], z1 = h.zm[1 - h.p];
    h.p = 0;
    h.pending = PEND_NONE;
    h.zm[0] = z0;
    h.zm[1] = z1;
    SPFC_CK(cudaMemcpy(v_.S0 + local * v_.spec, blob.data() + sizeof(SavScal), sbytes, cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(v_.S1 + local * v_.spec, blob.data() + sizeof(SavScal) + sbytes, sbytes,
                       cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(v_.sc + local, &h, sizeof(SavScal), cudaMemcpyHostToDevice));
    return 0;
  }
  int import_one(int local) {
    int rc = ensure_one(local);
    if (rc) return rc;
    const size_t sbytes = v_.spec * sizeof(C);
    SPFC_CK(cudaStreamSynchronize(st_));
    SavScal h;
    SPFC_CK(cudaMemcpy(&h, v_.sc + local, sizeof(SavScal), cudaMemcpyDeviceToHost));
    std::string blob(sizeof(SavScal) + 2 * sbytes, '\0');
    std::memcpy(&blob[0], &h, sizeof(SavScal));
    const C* newest = (h.p == 0 ? v_.S0 : v_.S1) + local * v_.spec;
    const C* prev = (h.p == 0 ? v_.S1 : v_.S0) + local * v_.spec;
    SPFC_CK(cudaMemcpy(&blob[sizeof(SavScal)], newest, sbytes, cudaMemcpyDeviceToHost));
    SPFC_CK(cudaMemcpy(&blob[sizeof(SavScal) + sbytes], prev, sbytes, cudaMemcpyDeviceToHost));
    rc = one_->restore(blob);
    if (rc) err = one_->err;
    return rc;
  }

  std::vector<Params> params_;
  cudaStream_t st_;
  BatchView<R> v_{};
  Params* Pdev_ = nullptr;
  C* tw_ = nullptr;
  size_t total_ = 0;
  Solver2D<R, N_, 0>* one_ = nullptr;
  int one_run_ = -1;
  bool g3_ = false;  // some run of the class has the phi^4 term
};

template <typename R, int N, int SCHED>
BatchClassBase* new_batch_class(const std::vector<Params>& params, cudaStream_t st, int* status,
                                std::string* err) {
  auto* b = new BatchClass<R, N, SCHED>(params, st);
  const int rc = b->setup();
  if (rc) {
    *status = rc;
    *err = b->err;
    delete b;
    return nullptr;
  }
  b->schedule = SCHED;
  return b;
}

// One grid size N >= 128, every batch schedule (one translation unit per
// size and precision, compiled in parallel).
template <typename R, int N>
BatchClassBase* make_batch_class_n(int sched, const std::vector<Params>& params, cudaStream_t st, int* status,
                                   std::string* err) {
  switch (sched) {
    case 2: return new_batch_class<R, N, 2>(params, st, status, err);
    case 4: return new_batch_class<R, N, 4>(params, st, status, err);
    case 5: return new_batch_class<R, N, 5>(params, st, status, err);
    default: return new_batch_class<R, N, 0>(params, st, status, err);
  }
}

// Grids below 128 (one schedule).
template <typename R>
BatchClassBase* make_batch_class_small(int N, const std::vector<Params>& params, cudaStream_t st, int* status,
                                       std::string* err) {
  switch (N) {
    case 16: return new_batch_class<R, 16, 0>(params, st, status, err);
    case 32: return new_batch_class<R, 32, 0>(params, st, status, err);
    default: return new_batch_class<R, 64, 0>(params, st, status, err);
  }
}

}  // namespace spfc
