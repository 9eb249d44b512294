// Host driver of the 3D step kernels for one run (same contract as the 2D
// driver: device buffers, init / step / diagnostics, CUDA-graph replay).
#pragma once

#include "spfc_kernels3d.cuh"
#include "spfc_solver2d.cuh"

namespace spfc {

// Launch shape per grid size: E values per FFT lane (8 on the float32-bulk
// path; 4 on the float64 path, whose arithmetic needs the extra threads once
// one thread carries every field of its column or row pair).
template <int N, int E_ = 8> struct Shape3D {
  static constexpr int E = E_;
  static constexpr int T = N / E;
  static constexpr int CT = (32 / T > 4) ? 32 / T : 4;  // kx columns per column-pass block (>= 32 B per row)
  static constexpr int RP = 32 / T > 1 ? 32 / T : 1;    // row pairs per row-pass block
  static_assert((CT * T) % 32 == 0 && (3 * RP * T) % 32 == 0 && (RP * T) % 32 == 0, "tiles must fill warps");
};

template <typename R, int N>
class Solver3D final : public SolverBase {
  using C = C_t<R>;
  using SH = Shape3D<N, sizeof(R) == 8 ? 4 : 8>;
  static constexpr int NH = N / 2 + 1;
  static constexpr int E = SH::E, T = SH::T, CT = SH::CT, RP = SH::RP;
  static constexpr int CTP = col_pitch(CT);
  static constexpr int GX = (NH + CT - 1) / CT;          // tiles per line set
  static constexpr int GROW = N * N / (2 * RP);           // row-pass blocks
  static constexpr int PW_THREADS = 256;

 public:
  Solver3D(const Params& p, cudaStream_t s) : st_(s) { P = p; }

  int setup() {
    const size_t sb = (size_t)N * N * NH * sizeof(C);
    spec_bytes_ = sb;
    auto al = [&](void** ptr, size_t bytes) -> cudaError_t {
      cudaError_t e = cudaMalloc(ptr, bytes);
      if (e == cudaSuccess) total_ += bytes;
      return e;
    };
    gpw_ = (int)std::min<size_t>(((size_t)N * N * NH + PW_THREADS - 1) / PW_THREADS, 1216);
    nE_ = GROW;
    nG_ = GX * N;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = al((void**)&S_.s[i], sb);
    if (e == cudaSuccess) e = al((void**)&Nhat_, sb);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = al((void**)&W_[i], sb);
    if (e == cudaSuccess) e = al((void**)&real_, (size_t)N * N * N * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partE_, 2 * (size_t)nE_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partG_, 3 * (size_t)nG_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&chunk_, 5 * (size_t)kScalarBlocks * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&counter_, sizeof(unsigned));
    if (e == cudaSuccess) e = al((void**)&partN_, 3 * (size_t)gpw_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&partS_, (size_t)gpw_ * sizeof(double));
    if (e == cudaSuccess) e = al((void**)&sc_, sizeof(SavScal));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&hsc_, sizeof(SavScal));  // pinned: small fast reads
    if (e == cudaSuccess) e = al((void**)&tw_, TW_LEN * sizeof(C));
    if (e != cudaSuccess) {
      err = std::string("device allocation failed: ") + cudaGetErrorString(e);
      return (e == cudaErrorMemoryAllocation) ? 2 : 3;
    }
    std::vector<C> tw;
    host_twiddles<R>(tw);
    SPFC_CK(cudaMemcpy(tw_, tw.data(), TW_LEN * sizeof(C), cudaMemcpyHostToDevice));
    SavScal z{};
    SPFC_CK(cudaMemcpy(sc_, &z, sizeof(SavScal), cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemset(counter_, 0, sizeof(unsigned)));
    SPFC_CK(cudaMemset(S_.s[0], 0, sb));
    SPFC_CK(cudaMemset(S_.s[1], 0, sb));
    SPFC_CK(cudaMemset(Nhat_, 0, sb));
    SPFC_CK(set_smem(k3d_ypass<R, N, E, CT, Y3_FWD>, smem_col(3)));
    SPFC_CK(set_smem(k3d_ypass<R, N, E, CT, Y3_INV>, smem_col(3)));
    SPFC_CK(set_smem(k3d_ypass<R, N, E, CT, Y3_INV_FIELD>, smem_col(1)));
    SPFC_CK(set_smem(k3d_ypass<R, N, E, CT, Y3_FWD_FIELD>, smem_col(1)));
    SPFC_CK(set_smem(k3d_zfwd<R, N, E, CT, Z3F_BDF2>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zfwd<R, N, E, CT, Z3F_BDF1>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zfwd<R, N, E, CT, Z3F_NHAT>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zfwd<R, N, E, CT, Z3F_TO_STATE>, smem_col(1)));
    SPFC_CK(set_smem(k3d_zinv<R, N, E, CT, Z3I_STEP>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zinv<R, N, E, CT, Z3I_STEP_BDF1>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zinv<R, N, E, CT, Z3I_PREP>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zinv<R, N, E, CT, Z3I_GRAD>, smem_col(2)));
    SPFC_CK(set_smem(k3d_zinv<R, N, E, CT, Z3I_FIELD>, smem_col(1)));
    SPFC_CK(set_smem(k3d_row<R, N, E, RP, RW_NONLIN>, smem_row(3)));
    SPFC_CK(set_smem(k3d_row<R, N, E, RP, RW_ENERGY>, smem_row(3)));
    SPFC_CK(set_smem(k3d_row<R, N, E, RP, RW_IN_REAL>, smem_row(1)));
    SPFC_CK(set_smem(k3d_row<R, N, E, RP, RW_OUT_REAL>, smem_row(1)));
    SPFC_CK(cudaStreamCreateWithFlags(&cap_st_, cudaStreamNonBlocking));
    return 0;
  }

  ~Solver3D() override {
    if (g1_) cudaGraphExecDestroy(g1_);
    if (g8_) cudaGraphExecDestroy(g8_);
    for (auto ev : evpool_) cudaEventDestroy(ev);
    if (cap_st_) cudaStreamDestroy(cap_st_);
    void* ptrs[] = {chunk_, counter_, S_.s[0], S_.s[1], Nhat_, W_[0], W_[1], W_[2], W3_, real_, partE_, partG_, partN_, partS_, sc_,
                    tw_};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    if (hsc_) cudaFreeHost(hsc_);
  }

  int64_t device_bytes() const override { return (int64_t)total_; }

  int init(const double* phi0, bool on_device, int mode) override {
    int rc = load_field(phi0, on_device, 0, true);
    if (rc) return rc;
    if (mode == 0) {
      if ((rc = grad_to_w(0)) || (rc = row(RW_NONLIN)) || (rc = ypass(Y3_FWD)) || (rc = zfwd(Z3F_BDF1, 0)) ||
          (rc = scalar(true)) || (rc = zinv(Z3I_STEP_BDF1, 0)) || (rc = ypass(Y3_INV)))
        return rc;
      w_ready_ = true;
      inited = true;
      return sync();
    } else if (mode == 1) {
      if ((rc = grad_to_w(0)) || (rc = row(RW_NONLIN)) || (rc = sop(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0)) ||
          (rc = ypass(Y3_FWD)) || (rc = zfwd(Z3F_NHAT, 0)))
        return rc;
      k3d_ghost<R><<<gpw_, PW_THREADS, 0, st_>>>(P, S_, Nhat_, sc_);
      SPFC_CK(cudaGetLastError());
      if ((rc = grad_to_w(1)) || (rc = row(RW_ENERGY)) || (rc = sop(SO_R_PREV, partE_, nE_, nullptr, 0, 0)))
        return rc;
    } else if (mode == 2) {
      if ((rc = copy_newest_to_prev()) || (rc = grad_to_w(0)) || (rc = row(RW_ENERGY)) ||
          (rc = sop(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0)) || (rc = sop(SO_R_PREV, partE_, nE_, nullptr, 0, 0)))
        return rc;
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
    if (!rc) rc = load_field(phi_prev, on_device, 1, false);
    if (!rc) rc = sop(SO_SET_R, nullptr, 0, nullptr, 0, 0, r, r_prev);
    if (rc) return rc;
    w_ready_ = false;
    inited = true;
    return 0;
  }

  int set_stab(double A) override {
    P.stab = A;
    fill_float_params(&P);
    drop_graphs();
    w_ready_ = false;
    return 0;
  }

  // The phi^4 term's kernels carry a fourth work array (allocated when the
  // term is first switched on); the step keeps its six kernels.
  int set_gamma3(double g3) override {
    if (g3 != 0.0 && !W3_) {
      cudaError_t e = cudaMalloc((void**)&W3_, spec_bytes_);
      if (e != cudaSuccess) {
        W3_ = nullptr;
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return (e == cudaErrorMemoryAllocation) ? 2 : 3;
      }
      total_ += spec_bytes_;
      SPFC_CK(set_smem(k3d_ypass_g3<R, N, E, CT, Y3_FWD>, smem_col(3)));
      SPFC_CK(set_smem(k3d_ypass_g3<R, N, E, CT, Y3_INV>, smem_col(3)));
      SPFC_CK(set_smem(k3d_zfwd_g3<R, N, E, CT, Z3F_BDF2>, smem_col(2)));
      SPFC_CK(set_smem(k3d_zfwd_g3<R, N, E, CT, Z3F_BDF1>, smem_col(2)));
      SPFC_CK(set_smem(k3d_zfwd_g3<R, N, E, CT, Z3F_NHAT>, smem_col(2)));
      SPFC_CK(set_smem(k3d_row_g3<R, N, E, RP, RW_NONLIN>, smem_row(4)));
      SPFC_CK(set_smem(k3d_row_g3<R, N, E, RP, RW_ENERGY>, smem_row(4)));
    }
    P.g3 = g3;
    fill_float_params(&P);
    drop_graphs();
    w_ready_ = false;
    return 0;
  }

  int dt_change(double dt) override {
    P.dt = dt;
    fill_float_params(&P);
    drop_graphs();
    int rc;
    if ((rc = copy_newest_to_prev()) || (rc = grad_to_w(0)) || (rc = row(RW_ENERGY)) ||
        (rc = sop(SO_R_NEWEST, partE_, nE_, nullptr, 0, 0)) || (rc = sop(SO_R_PREV, partE_, nE_, nullptr, 0, 0)))
      return rc;
    w_ready_ = false;
    return 0;
  }

  int step(long long n) override {
    if (n <= 0) return 0;
    if (!w_ready_) {
      int rc = zinv(Z3I_PREP, 0);
      if (!rc) rc = ypass(Y3_INV);
      if (rc) return rc;
      w_ready_ = true;
    }
    if (timing_) {
      for (long long i = 0; i < n; ++i) {
        int rc = timed_step();
        if (rc) return rc;
      }
      return 0;
    }
    if (!g1_) { int rc = capture(1, &g1_); if (rc) return rc; }
    if (!g8_) { int rc = capture(8, &g8_); if (rc) return rc; }
    for (long long i = 0; i < n / 8; ++i) SPFC_CK(cudaGraphLaunch(g8_, st_));
    for (long long i = 0; i < n % 8; ++i) SPFC_CK(cudaGraphLaunch(g1_, st_));
    return 0;
  }

  int energy(double* E_orig, double* E_mod, double* E_breve) override {
    w_ready_ = false;
    k3d_norms<R><<<gpw_, PW_THREADS, 0, st_>>>(P, S_, sc_, partN_);
    SPFC_CK(cudaGetLastError());
    int rc;
    if ((rc = grad_to_w(0)) || (rc = row(RW_ENERGY)) || (rc = sop(SO_ENERGY, partE_, nE_, partN_, gpw_, 0)))
      return rc;
    SavScal h;
    if ((rc = read_scal(&h))) return rc;
    if (E_orig) *E_orig = h.E_orig;
    if (E_mod) *E_mod = h.E_mod;
    if (E_breve) *E_breve = h.E_breve;
    return 0;
  }

  int mass(double* m, double* mean) override {
    SavScal h;
    int rc = read_scal(&h);
    if (rc) return rc;
    if (m) *m = P.vol * h.zm[h.p];
    if (mean) *mean = h.zm[h.p];
    return 0;
  }

  int scalars(SavScal* out) override { return read_scal(out); }

  int get_field(double* out, bool on_device, int which) override {
    w_ready_ = false;
    int rc;
    if ((rc = zinv(Z3I_FIELD, which)) || (rc = ypass(Y3_INV_FIELD)) || (rc = row(RW_OUT_REAL))) return rc;
    SPFC_CK(cudaMemcpyAsync(out, real_, (size_t)N * N * N * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st_));
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
    kt->names = {"row", "y_fwd", "z_fwd", "scalar", "z_inv", "y_inv"};
    kt->launches.assign(tcount_, tcount_ + 6);
    kt->ms.assign(tms_, tms_ + 6);
    for (int i = 0; i < 6; ++i) { tcount_[i] = 0; tms_[i] = 0.0; }
    return 0;
  }

  int dump(std::string* blob) override {
    SavScal h;
    int rc = read_scal(&h);
    if (rc) return rc;
    blob->assign(sizeof(SavScal) + 2 * spec_bytes_, '\0');
    char* b = &(*blob)[0];
    std::memcpy(b, &h, sizeof(SavScal));
    SPFC_CK(cudaMemcpy(b + sizeof(SavScal), S_.s[h.p], spec_bytes_, cudaMemcpyDeviceToHost));
    SPFC_CK(cudaMemcpy(b + sizeof(SavScal) + spec_bytes_, S_.s[1 - h.p], spec_bytes_, cudaMemcpyDeviceToHost));
    return 0;
  }

  int restore(const std::string& blob) override {
    if (blob.size() != sizeof(SavScal) + 2 * spec_bytes_) { err = "checkpoint size mismatch"; return 1; }
    SavScal h;
    std::memcpy(&h, blob.data(), sizeof(SavScal));
    const int p = h.p;
    const double z0 = h.zm[p], z1 = h.zm[1 - p];
    h.p = 0;
    h.pending = PEND_NONE;
    h.status = DEV_OK;
    h.zm[0] = z0;
    h.zm[1] = z1;
    apply_ring(&h);
    drop_graphs();
    w_ready_ = false;
    SPFC_CK(cudaStreamSynchronize(st_));
    SPFC_CK(cudaMemcpy(S_.s[0], blob.data() + sizeof(SavScal), spec_bytes_, cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(S_.s[1], blob.data() + sizeof(SavScal) + spec_bytes_, spec_bytes_, cudaMemcpyHostToDevice));
    SPFC_CK(cudaMemcpy(sc_, &h, sizeof(SavScal), cudaMemcpyHostToDevice));
    inited = true;
    return 0;
  }

 private:
  template <typename K> static cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  static constexpr size_t smem_col(int nf) { return (size_t)nf * sp_len(N) * CTP * sizeof(C); }
  static constexpr size_t smem_row(int ns) { return (size_t)ns * RP * (sp_len(N) + 1) * sizeof(C); }

  bool g3_on() const { return P.g3 != 0.0; }

  int ypass(int mode) {
    const dim3 g(GX, N);
    if (g3_on() && (mode == Y3_FWD || mode == Y3_INV)) {
      if (mode == Y3_FWD)
        k3d_ypass_g3<R, N, E, CT, Y3_FWD><<<g, CT * T, smem_col(3), st_>>>(P, W_[0], W_[1], W_[2], W3_, sc_, tw_);
      else
        k3d_ypass_g3<R, N, E, CT, Y3_INV><<<g, CT * T, smem_col(3), st_>>>(P, W_[0], W_[1], W_[2], W3_, sc_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case Y3_FWD: k3d_ypass<R, N, E, CT, Y3_FWD><<<g, CT * T, smem_col(3), st_>>>(P, W_[0], W_[1], W_[2], sc_, tw_); break;
      case Y3_INV: k3d_ypass<R, N, E, CT, Y3_INV><<<g, CT * T, smem_col(3), st_>>>(P, W_[0], W_[1], W_[2], sc_, tw_); break;
      case Y3_INV_FIELD:
        k3d_ypass<R, N, E, CT, Y3_INV_FIELD><<<g, CT * T, smem_col(1), st_>>>(P, W_[0], W_[1], W_[2], sc_, tw_); break;
      default:
        k3d_ypass<R, N, E, CT, Y3_FWD_FIELD><<<g, CT * T, smem_col(1), st_>>>(P, W_[0], W_[1], W_[2], sc_, tw_);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int zfwd(int mode, int target) {
    const dim3 g(GX, N);
    if (g3_on() && mode != Z3F_TO_STATE) {
      if (mode == Z3F_BDF2)
        k3d_zfwd_g3<R, N, E, CT, Z3F_BDF2><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_);
      else if (mode == Z3F_BDF1)
        k3d_zfwd_g3<R, N, E, CT, Z3F_BDF1><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_);
      else
        k3d_zfwd_g3<R, N, E, CT, Z3F_NHAT><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case Z3F_BDF2:
        k3d_zfwd<R, N, E, CT, Z3F_BDF2><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_, target); break;
      case Z3F_BDF1:
        k3d_zfwd<R, N, E, CT, Z3F_BDF1><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_, target); break;
      case Z3F_NHAT:
        k3d_zfwd<R, N, E, CT, Z3F_NHAT><<<g, CT * T, smem_col(2), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_, target); break;
      default:
        k3d_zfwd<R, N, E, CT, Z3F_TO_STATE><<<g, CT * T, smem_col(1), st_>>>(P, S_, W_[0], W_[1], Nhat_, partG_, sc_, tw_, target);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int zinv(int mode, int which) {
    const dim3 g(GX, N);
    switch (mode) {
      case Z3I_STEP:
        k3d_zinv<R, N, E, CT, Z3I_STEP><<<g, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which); break;
      case Z3I_STEP_BDF1:
        k3d_zinv<R, N, E, CT, Z3I_STEP_BDF1><<<g, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which); break;
      case Z3I_PREP:
        k3d_zinv<R, N, E, CT, Z3I_PREP><<<g, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which); break;
      case Z3I_GRAD:
        k3d_zinv<R, N, E, CT, Z3I_GRAD><<<g, CT * T, smem_col(2), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which); break;
      default:
        k3d_zinv<R, N, E, CT, Z3I_FIELD><<<g, CT * T, smem_col(1), st_>>>(P, S_, Nhat_, W_[0], W_[1], sc_, tw_, which);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int row(int mode) {
    if (g3_on() && (mode == RW_NONLIN || mode == RW_ENERGY)) {
      if (mode == RW_NONLIN)
        k3d_row_g3<R, N, E, RP, RW_NONLIN><<<GROW, RP * T, smem_row(4), st_>>>(P, W_[0], W_[1], W_[2], W3_, partE_, sc_, tw_);
      else
        k3d_row_g3<R, N, E, RP, RW_ENERGY><<<GROW, RP * T, smem_row(4), st_>>>(P, W_[0], W_[1], W_[2], W3_, partE_, sc_, tw_);
      SPFC_CK(cudaGetLastError());
      return 0;
    }
    switch (mode) {
      case RW_NONLIN:
        k3d_row<R, N, E, RP, RW_NONLIN><<<GROW, RP * T, smem_row(3), st_>>>(P, W_[0], W_[1], W_[2], partE_, sc_, tw_, real_); break;
      case RW_ENERGY:
        k3d_row<R, N, E, RP, RW_ENERGY><<<GROW, RP * T, smem_row(3), st_>>>(P, W_[0], W_[1], W_[2], partE_, sc_, tw_, real_); break;
      case RW_IN_REAL:
        k3d_row<R, N, E, RP, RW_IN_REAL><<<GROW, RP * T, smem_row(1), st_>>>(P, W_[0], W_[1], W_[2], partE_, sc_, tw_, real_); break;
      default:
        k3d_row<R, N, E, RP, RW_OUT_REAL><<<GROW, RP * T, smem_row(1), st_>>>(P, W_[0], W_[1], W_[2], partE_, sc_, tw_, real_);
    }
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int scalar(bool bdf1) {
    k3d_scalar<R><<<kScalarBlocks, 256, 0, st_>>>(P, sc_, partE_, nE_, partG_, nG_, bdf1 ? 1 : 0, chunk_, counter_);
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  int sop(int op, const double* a, int na, const double* b, int nb, int arg, double x0 = 0, double x1 = 0) {
    k_scalar_op<R><<<1, 32, 0, st_>>>(P, sc_, op, a, na, b, nb, arg, x0, x1);
    SPFC_CK(cudaGetLastError());
    return 0;
  }
  // W <- the y- and z-inverse transforms of i k~_d S[which-slot] (diagnostics, starts)
  int grad_to_w(int which) {
    int rc = zinv(Z3I_GRAD, which);
    return rc ? rc : ypass(Y3_INV);
  }
  int read_scal(SavScal* h) {
    SPFC_CK(cudaMemcpyAsync(hsc_, sc_, sizeof(SavScal), cudaMemcpyDeviceToHost, st_));
    SPFC_CK(cudaStreamSynchronize(st_));
    *h = *hsc_;
    if (h->status != DEV_OK) {
      err = "device status: non-finite value, infeasible SAV scalar system or timeout";
      return h->status;
    }
    return 0;
  }
  int copy_newest_to_prev() {
    SavScal h;
    int rc = read_scal(&h);
    if (rc) return rc;
    SPFC_CK(cudaMemcpyAsync(S_.s[1 - h.p], S_.s[h.p], spec_bytes_, cudaMemcpyDeviceToDevice, st_));
    SPFC_CK(cudaMemcpyAsync(&sc_->zm[1 - h.p], &sc_->zm[h.p], sizeof(double), cudaMemcpyDeviceToDevice, st_));
    return 0;
  }
  int load_field(const double* f, bool on_device, int slot_rel, bool reset) {
    const size_t bytes = (size_t)N * N * N * sizeof(double);
    if (reset) {
      // the cleared record goes up from the pinned buffer, so the copy does not
      // synchronise the stream; the buffer is not written again before the
      // synchronisation at the end of this call
      *hsc_ = SavScal{};
      apply_ring(hsc_);
      SPFC_CK(cudaMemcpyAsync(sc_, hsc_, sizeof(SavScal), cudaMemcpyHostToDevice, st_));
      drop_graphs();
    }
    SPFC_CK(cudaMemcpyAsync(real_, f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st_));
    k_real_sum<<<gpw_, PW_THREADS, 0, st_>>>(real_, (size_t)N * N * N, partS_);
    SPFC_CK(cudaGetLastError());
    int rc = sop(SO_ZM_SLOT, partS_, gpw_, nullptr, 0, slot_rel);
    if (!rc) rc = row(RW_IN_REAL);
    if (!rc) rc = ypass(Y3_FWD_FIELD);
    if (!rc) rc = zfwd(Z3F_TO_STATE, slot_rel == 0 ? 0 : 1);
    if (rc) return rc;
    k_put_zero_modes<R><<<1, 1, 0, st_>>>(S_, sc_);
    SPFC_CK(cudaGetLastError());
    SPFC_CK(cudaStreamSynchronize(st_));
    return 0;
  }
  int launch_step() {
    int rc;
    if ((rc = row(RW_NONLIN)) || (rc = ypass(Y3_FWD)) || (rc = zfwd(Z3F_BDF2, 0)) || (rc = scalar(false)) ||
        (rc = zinv(Z3I_STEP, 0)) || (rc = ypass(Y3_INV)))
      return rc;
    return 0;
  }
  void drop_graphs() {
    if (g1_) { cudaGraphExecDestroy(g1_); g1_ = nullptr; }
    if (g8_) { cudaGraphExecDestroy(g8_); g8_ = nullptr; }
  }
  int capture(int nsteps, cudaGraphExec_t* out) {
    cudaStream_t keep = st_;
    st_ = cap_st_;
    cudaGraph_t g = nullptr;
    SPFC_CK(cudaStreamBeginCapture(cap_st_, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int i = 0; i < nsteps && rc == 0; ++i) rc = launch_step();
    cudaError_t e = cudaStreamEndCapture(cap_st_, &g);
    st_ = keep;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) { err = std::string("graph capture: ") + cudaGetErrorString(e); return 3; }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { err = std::string("graph instantiate: ") + cudaGetErrorString(e); return 3; }
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
    int e[7], rc;
    for (int i = 0; i < 7; ++i)
      if ((rc = ev(&e[i]))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[0]], st_));
    if ((rc = row(RW_NONLIN))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[1]], st_));
    if ((rc = ypass(Y3_FWD))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[2]], st_));
    if ((rc = zfwd(Z3F_BDF2, 0))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[3]], st_));
    if ((rc = scalar(false))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[4]], st_));
    if ((rc = zinv(Z3I_STEP, 0))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[5]], st_));
    if ((rc = ypass(Y3_INV))) return rc;
    SPFC_CK(cudaEventRecord(evpool_[e[6]], st_));
    for (int i = 0; i < 6; ++i) trecs_.push_back({i, e[i], e[i + 1]});
    return 0;
  }

  struct TRec { int cls, e0, e1; };
  cudaStream_t st_ = nullptr, cap_st_ = nullptr;
  Slots<R> S_{{nullptr, nullptr}};
  C* Nhat_ = nullptr;
  C* W_[3] = {nullptr, nullptr, nullptr};
  C* W3_ = nullptr;  // fourth work array of the phi^4 term (allocated on demand)
  double* real_ = nullptr;
  double *partE_ = nullptr, *partG_ = nullptr, *partN_ = nullptr, *partS_ = nullptr;
  double* chunk_ = nullptr;    // chunk sums of the spread scalar reduction
  unsigned* counter_ = nullptr; // its arrival counter (reset by the last block)
  SavScal* sc_ = nullptr;
  SavScal* hsc_ = nullptr;  // pinned host copy of the record
  C* tw_ = nullptr;
  int gpw_ = 0, nE_ = 0, nG_ = 0;
  size_t spec_bytes_ = 0, total_ = 0;
  cudaGraphExec_t g1_ = nullptr, g8_ = nullptr;
  bool timing_ = false, w_ready_ = false;
  std::vector<cudaEvent_t> evpool_;
  int evnext_ = 0;
  std::vector<TRec> trecs_;
  int64_t tcount_[6] = {0, 0, 0, 0, 0, 0};
  double tms_[6] = {0, 0, 0, 0, 0, 0};
};

template <typename R, int N>
SolverBase* new_solver_3d(const Params& P, cudaStream_t st, int* status, std::string* err) {
  auto* s = new Solver3D<R, N>(P, st);
  int rc = s->setup();
  if (rc) {
    *status = rc;
    *err = s->err;
    delete s;
    return nullptr;
  }
  return s;
}

}  // namespace spfc
