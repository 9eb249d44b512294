// 2D kernels of the BDF2-SAV Fourier pseudo-spectral step (Sec. 2.2-2.3).
//
// Layout: real fields phi[y][x] (x fastest); spectra are R2C half spectra
// F[ky][kx], kx in [0, N/2], ky in [0, N), normalised as
// F_hat = (1/P) sum_j f_j exp(-i k.x_j) (eq. spectral-coll-1 on [0,L]^2).
// Work arrays W0, W1 have the same shape and hold, between passes, data that
// is transformed along y only ([y][kx]).
//
// The step replayed in production is row -> col_fused (the fused column pass
// below: the forward half, a grid barrier with the scalar solve, then the
// update and the inverse half for the next step). The same work split into
// three separate passes, with the update left pending between steps (the
// lazy form, used by the start-up and the phi^4 term), is
// col_inv -> row -> col_fwd; the batched ensemble runs these passes with a
// separate scalar kernel between col_fwd and col_inv:
//  col_inv : phi^{n+1} = alpha b + c (lazy update of the previous step),
//            phi* = 2 phi^{n+1} - phi^n, G_d = i k~_d phi*, inverse DFT in y.
//  row     : inverse DFT in x of G_x + i G_y (one complex FFT for both real
//            gradients), s = |grad phi*|^2, E_1 partial sums, w_d = (beta s - 2) g_d,
//            forward DFT in x of w_x + i w_y, split into W_x, W_y.
//  col_fwd : forward DFT in y, N_hat = -(i k~_x W_x + i k~_y W_y), partial sums
//            of gamma = <N, A^{-1} Delta N>, eta = <N, A^{-1}(2 phi^n - phi^{n-1}/2)>,
//            theta = <N, 2 phi^n - phi^{n-1}/2>; the last block solves the scalar
//            system (eqs. solver-2, solver-4) for r^{n+1}.
#pragma once

#include "spfc_common.cuh"
#include "spfc_state.h"

namespace spfc {

// wave numbers --------------------------------------------------------------
// index i in [0,N) in DFT order; Nyquist (i = N/2) keeps its full |k| in the
// Laplacian but has first-derivative symbol 0. Evaluated in the working
// precision R (no float64 arithmetic per element on the float32 path).
template <typename R> __device__ __forceinline__ R kfull(int i, int N, R kf) {
  return (R)((i <= N / 2) ? i : i - N) * kf;
}
template <typename R> __device__ __forceinline__ R kderiv(int i, int N, R kf) {
  return (i == N / 2) ? (R)0 : (R)((i < N / 2) ? i : i - N) * kf;
}

// Per-run constants in the working precision (read, never converted, per thread).
template <typename R> struct PC;
template <> struct PC<double> {
  double kfx, kfy, kfz, dt, a, beta, invP, sdt, g3, g3b;
  int pfc;
  __device__ __forceinline__ explicit PC(const Params& P)
      : kfx(P.kf[0]), kfy(P.kf[1]), kfz(P.kf[2]), dt(P.dt), a(P.a), beta(P.beta), invP(P.invP), sdt(P.sdt),
        g3(P.g3), g3b(P.g3b), pfc(P.pfc) {}
};
template <> struct PC<float> {
  float kfx, kfy, kfz, dt, a, beta, invP, sdt, g3, g3b;
  int pfc;
  __device__ __forceinline__ explicit PC(const Params& P)
      : kfx(P.kf_f[0]), kfy(P.kf_f[1]), kfz(P.kf_f[2]), dt(P.dt_f), a(P.a_f), beta(P.beta_f), invP(P.invP_f),
        sdt(P.sdt_f), g3(P.g3_f), g3b(P.g3b_f), pfc(P.pfc) {}
};
template <typename R> __device__ __forceinline__ R read_alpha(const SavScal* sc);
template <> __device__ __forceinline__ double read_alpha<double>(const SavScal* sc) { return sc->alpha; }
template <> __device__ __forceinline__ float read_alpha<float>(const SavScal* sc) { return sc->alpha_f; }

template <typename R> struct Slots {
  C_t<R>* s[2];
  // select without dynamic indexing of the parameter array (keeps it in registers)
  __device__ __forceinline__ C_t<R>* at(int i) const { return i ? s[1] : s[0]; }
};

enum ColInvMode : int { CI_STEP = 0, CI_GRAD = 1, CI_FIELD = 2, CI_STEP_COMMITTED = 3 };
enum RowMode : int { RW_NONLIN = 0, RW_ENERGY = 1, RW_OUT_REAL = 2, RW_IN_REAL = 3 };
enum ColFwdMode : int { CF_BDF2 = 0, CF_BDF1 = 1, CF_NHAT = 2, CF_TO_STATE = 3, CF_PART = 4 };

// Explicitly rounded arithmetic for the spectral symbols and the update, so
// that every kernel that evaluates them (the lazy update in the column pass,
// the explicit finalize) produces bit-identical results regardless of how the
// compiler would contract multiply-adds.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// |k|^2 (full wave numbers, Nyquist included) of half-spectrum index (kx, ky).
template <typename R>
__device__ __forceinline__ R sym_K2(int kx, int ky, int N, const PC<R>& c) {
  const R kxx = rn_mul((R)kx, c.kfx);
  const R kyy = rn_mul((R)((ky <= N / 2) ? ky : ky - N), c.kfy);
  return rn_fma(kxx, kxx, rn_mul(kyy, kyy));
}

// Symbol of the linear operator L_N: a + |k|^4 (SPFC, Sec. 2.2), or the
// Swift-Hohenberg a + (1 - |k|^2)^2 of the PFC split.
template <typename R>
__device__ __forceinline__ R sym_L(R K2, const PC<R>& c) {
  if (c.pfc) {
    const R u = K2 - (R)1;
    return rn_fma(u, u, c.a);
  }
  return rn_fma(K2, K2, c.a);
}

// 1 / (c0 + dt |k|^2 L(k) + A dt |k|^2): inverse symbol of A_N (c0 = 3/2,
// eq. solver-1) or of the first-order operator (c0 = 1); the last term is the
// stabiliser of Sec. 5.2 (exactly zero when A = 0).
// The correctly rounded reciprocal (the value of an IEEE 1 / x, by the
// shorter reciprocal intrinsic rather than the general division).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

template <typename R>
__device__ __forceinline__ R sym_invA(R K2, R c0, const PC<R>& c) {
  const R A = rn_fma(c.sdt, K2, rn_fma(c.dt, rn_mul(K2, sym_L<R>(K2, c)), c0));
  return rcp_rn(A);
}

// Zero mode of the BDF2 update: A_0 = 3/2 and Delta_N N has no mean, so
// c_0 = (2 a - b/2) / (3/2) = a + (a - b)/3, written so that a == b gives a
// exactly (mass conservation, Theorem SPFC solvability).
__device__ __forceinline__ double zero_mode_update(double a, double b) {
  return a + (a - b) * (1.0 / 3.0);
}

// BDF2 update of one spectral coefficient (eq. solver-6 in the form
// phi^{n+1} = (dt r^{n+1}/sqrt(E1)) A^{-1} Delta N + A^{-1}(2 phi^n - phi^{n-1}/2 + s phi^n)),
// s = A dt |k|^2 the stabiliser's right-hand side (Sec. 5.2; zero when A = 0).
template <typename C, typename R>
__device__ __forceinline__ C bdf2_update(C cur, C old, C nh, R K2, R invA, R alpha, R s) {
  const R bfac = rn_mul(rn_mul(-alpha, K2), invA);
  const R vx = rn_fma(s, cur.x, rn_fma((R)2, cur.x, rn_mul((R)-0.5, old.x)));
  const R vy = rn_fma(s, cur.y, rn_fma((R)2, cur.y, rn_mul((R)-0.5, old.y)));
  return mk<C>(rn_fma(bfac, nh.x, rn_mul(vx, invA)), rn_fma(bfac, nh.y, rn_mul(vy, invA)));
}

// First-order (BDF1 start) update: phi^1 = alpha A1^{-1} Delta N + A1^{-1} (1 + s) phi^0.
template <typename C, typename R>
__device__ __forceinline__ C bdf1_update(C cur, C nh, R K2, R invA, R alpha, R s) {
  const R bfac = rn_mul(rn_mul(-alpha, K2), invA);
  const R vx = rn_fma(s, cur.x, cur.x), vy = rn_fma(s, cur.y, cur.y);
  return mk<C>(rn_fma(bfac, nh.x, rn_mul(vx, invA)), rn_fma(bfac, nh.y, rn_mul(vy, invA)));
}

// ---------------------------------------------------------------------------
// Column passes. Grid: ceil(NH/CT) blocks, each a tile of CT kx columns;
// CT * T threads, thread (lane, c) = threadIdx.x = lane * CT + c owning the
// rows y = lane + i T (i < E) of column kx0 + c, for every field of the pass
// (one warp then reads 32/CT rows of CT adjacent columns). The column FFTs
// keep their first and last stages in registers (fft_regs_multi).
// G3 (the optional phi^4 term): no third transform and no third array across
// the row pass, since k~_x is constant along a column and known in the row
// pass. The inverse pass transforms phi* and i k~_y phi* and stores Y^-1 phi*
// (W2) and G_y (W1); the row pass forms G_x = i k~_x Y^-1 phi* itself and
// returns W0 = k~_x W_x + i F_x(gamma3 phi*^3) and W1 = W_y; the forward pass
// transforms both, so that -i (Y W0 + k~_y Y W1) is N_hat with the transform of
// gamma3 phi*^3 added.
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int CT, int MODE, bool G3 = false, bool PF = false>
__device__ __forceinline__ void k2d_col_inv_body(const Params& P, Slots<R> S, const C_t<R>* __restrict__ Nhat,
                                                 C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
                                                 SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, int which,
                                                 C_t<R>* __restrict__ W2 = nullptr) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N, E>::T;
  // PF (the PFC model): the row pass needs phi* itself, not its gradients
  constexpr int NF = (MODE == CI_FIELD || PF) ? 1 : 2;
  static_assert(!G3 || MODE == CI_STEP || MODE == CI_GRAD || MODE == CI_STEP_COMMITTED,
                "the phi^4 channel is carried by the step and gradient modes");
  static_assert(!(G3 && PF), "the PFC model has its own passes");
  constexpr int NTH = CT * T;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr bool COMMITTED = (MODE == CI_STEP_COMMITTED);
  constexpr int SEQ = sp_len(N);
  static_assert(NTH % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);

  pdl_wait();
  pdl_trigger();
  if (sc->status != DEV_OK) return;
  const PC<R> pc(P);
  const int p = sc->p;
  // CI_STEP: a pending update (lazy form) is applied into slot 1-p.
  // CI_STEP_COMMITTED: the scalar solve has already flipped p; the update is
  // applied into slot p (holding phi^{n-1}) from phi^n in slot 1-p.
  const int pending = (MODE == CI_STEP) ? sc->pending : (COMMITTED ? 1 : 0);
  const R alpha = read_alpha<R>(sc);
  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c;
  const bool col = kx < NH;
  C* src_new;
  C* src_old;
  if (MODE == CI_STEP) {
    src_new = S.at(p);
    src_old = S.at(1 - p);
  } else if (COMMITTED) {
    src_new = S.at(1 - p);
    src_old = S.at(p);
  } else {
    src_new = S.at(which == 0 ? p : 1 - p);
    src_old = src_new;
  }

  // all loads first, then the pointwise spectral work in registers
  C vcur[E], vold[E], vnh[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    vcur[i] = vold[i] = vnh[i] = mk<C>(0, 0);
    if (col) {
      const size_t off = (size_t)(lane + i * T) * NH + kx;
      vcur[i] = src_new[off];
      if (MODE == CI_STEP || COMMITTED) {
        vold[i] = src_old[off];
        if (pending) vnh[i] = Nhat[off];
      }
    }
  }
  C g[NF][E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int ky = lane + i * T;
    C g0 = mk<C>(0, 0), g1 = mk<C>(0, 0);
    if (col) {
      const size_t off = (size_t)ky * NH + kx;
      C ph = vcur[i];
      if (MODE == CI_STEP || COMMITTED) {
        const C cur = vcur[i];
        C old = vold[i];
        C nw = cur;
        if (pending) {
          if (off == 0) {
            // zero mode: c_0 = phi_0^n + (phi_0^n - phi_0^{n-1})/3 (A_0 = 3/2, Delta kills N)
            const int sn = COMMITTED ? 1 - p : p;  // slot of phi^n
            const double z = zero_mode_update(sc->zm[sn], sc->zm[1 - sn]);
            sc->zm[1 - sn] = z;
            nw = mk<C>((R)z, (R)0);
          } else {
            const R K2 = sym_K2<R>(kx, ky, N, pc);
            nw = bdf2_update<C, R>(cur, old, vnh[i], K2, sym_invA<R>(K2, (R)1.5, pc), alpha, rn_mul(pc.sdt, K2));
          }
          src_old[off] = nw;  // phi^{n+1} overwrites phi^{n-1}
          old = cur;
        }
        ph = mk<C>((R)2 * nw.x - old.x, (R)2 * nw.y - old.y);  // phi* = 2 phi^{n+1} - phi^n
      }
      if (MODE == CI_FIELD || PF) {
        g0 = ph;
      } else {
        const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
        g0 = G3 ? ph : mk<C>(-ktx * ph.y, ktx * ph.x);  // i k~_x phi (G3: phi)
        g1 = mk<C>(-kty * ph.y, kty * ph.x);            // i k~_y phi
      }
    }
    g[0][i] = g0;
    if (NF == 2) g[NF - 1][i] = g1;
  }
  fft_regs_multi<C, N, E, true, NF, true>(g, sm + c, SEQ * CTP, CTP, lane, tw);
  if (col) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const size_t off = (size_t)(lane + i * T) * NH + kx;
      if constexpr (G3) W2[off] = g[0][i];  // Y^-1 phi* (the row pass forms G_x from it)
      else W0[off] = g[0][i];
      if (NF == 2) W1[off] = g[NF - 1][i];
    }
  }
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_inv(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, C_t<R>* __restrict__ W0,
            C_t<R>* __restrict__ W1, SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, int which) {
  k2d_col_inv_body<R, N, E, CT, MODE>(P, S, Nhat, W0, W1, sc, tw, which);
}

// the PFC model: W0 receives the y-inverse of phi*
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_inv_pfc(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, C_t<R>* __restrict__ W0,
                SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, int which) {
  k2d_col_inv_body<R, N, E, CT, MODE, false, true>(P, S, Nhat, W0, nullptr, sc, tw, which);
}

// with the phi^4 channel (W2 receives the y-inverse of phi*)
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_inv_g3(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, C_t<R>* __restrict__ W0,
               C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2, SavScal* __restrict__ sc,
               const C_t<R>* __restrict__ tw, int which) {
  k2d_col_inv_body<R, N, E, CT, MODE, true>(P, S, Nhat, W0, W1, sc, tw, which, W2);
}

// ---------------------------------------------------------------------------
// Row pass. Grid: N/RPC blocks, RPC rows each, T = N/E lanes per row.
// part: 2 x gridDim.x doubles: sum s^2 and sum s per block (without h^d).
// G3: each row reads Y^-1 phi* (W2) and G_y (W1), forms G_x = i k~_x Y^-1 phi*,
// also inverse-transforms phi*, adds (gamma3/beta) phi*^4 to the sum of s^2
// (E_1 takes that sum with beta/4) and, for the step, forward-transforms
// gamma3 phi*^3 and writes W0 = k~_x W_x + i F_x(gamma3 phi*^3), W1 = W_y;
// shared memory holds two sequences per row.
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int RPC, int MODE, bool G3 = false, bool PF = false>
__device__ __forceinline__ void k2d_row_body(const Params& P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
                                             double* __restrict__ part, const SavScal* __restrict__ sc,
                                             const C_t<R>* __restrict__ tw, double* __restrict__ real_io,
                                             C_t<R>* __restrict__ W2 = nullptr) {
  using C = C_t<R>;
  static_assert(!G3 || MODE == RW_NONLIN || MODE == RW_ENERGY, "the phi^4 channel is carried by the nonlinear and energy modes");
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NTH = RPC * T;
  constexpr int NH = N / 2 + 1;
  constexpr int KH = (N / 2) / T;  // half-spectrum entries per lane, Nyquist aside
  constexpr int SEQ = sp_len(N);
  static_assert(NTH % 32 == 0 && KH * T == N / 2, "rows must fill whole warps");
  using RD = Red<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ typename RD::acc red2[2][32];

  pdl_wait();
  pdl_trigger();
  // the nonlinear and energy modes check the status after issuing their W
  // loads (valid whatever the status), so that its round trip overlaps them
  constexpr bool LATE_CHECK = (MODE == RW_NONLIN || MODE == RW_ENERGY);
  if (!LATE_CHECK && sc->status != DEV_OK) return;
  const int rloc = threadIdx.x / T, lane = threadIdx.x % T;
  const int row = blockIdx.x * RPC + rloc;
  C* z = sm + rloc * (G3 ? 2 : 1) * (SEQ + 1);
  const size_t roff = (size_t)row * NH;

  if constexpr (MODE == RW_IN_REAL) {
    double v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = real_io[(size_t)row * N + lane + i * T];
#pragma unroll
    for (int i = 0; i < E; ++i) z[spr(lane + i * T)] = mk<C>((R)v[i], (R)0);
    __syncthreads();
    fft_smem<C, N, E, false>(z, 1, lane, tw);
    const R sc1 = PC<R>(P).invP;
#pragma unroll
    for (int i = 0; i < KH; ++i) W0[roff + lane + i * T] = cscale(z[spr(lane + i * T)], sc1);
    if (lane == 0) W0[roff + N / 2] = cscale(z[spr(N / 2)], sc1);
  } else if constexpr (MODE == RW_OUT_REAL) {
    C a[KH];
#pragma unroll
    for (int i = 0; i < KH; ++i) a[i] = W0[roff + lane + i * T];
    const C ny = W0[roff + N / 2];
#pragma unroll
    for (int i = 0; i < KH; ++i) {
      const int k = lane + i * T;
      z[spr(k)] = a[i];
      if (k > 0) z[spr(N - k)] = cconj(a[i]);
    }
    if (lane == 0) z[spr(N / 2)] = ny;
    __syncthreads();
    fft_smem<C, N, E, true>(z, 1, lane, tw);
#pragma unroll
    for (int i = 0; i < E; ++i) real_io[(size_t)row * N + lane + i * T] = (double)z[spr(lane + i * T)].x;
  } else if constexpr (PF) {
    // the PFC model: the row's x-spectrum of phi* (Hermitian extension loaded
    // straight into registers), inverse DFT to phi*(x), the E_1 sums
    // sum phi*^4 and sum phi*^2, w = gamma3 phi*^3 - phi*, forward DFT into W0
    const PC<R> pc(P);
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = lane + i * T;
      const bool direct = k <= N / 2;
      const C f = W0[roff + (direct ? k : N - k)];
      v[i] = direct ? f : cconj(f);
    }
    if (sc->status != DEV_OK) return;
    fft_regs<C, N, E, true>(v, z, 1, lane, tw);
    typename RD::acc acc4 = RD::zero(), acc2 = RD::zero();
    const R g3 = pc.g3;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const R ph = v[i].x, p2 = ph * ph;
      acc4 = RD::add(acc4, p2 * p2);
      acc2 = RD::add(acc2, p2);
      if (MODE == RW_NONLIN) v[i] = mk<C>(ph * (g3 * p2 - (R)1), (R)0);
    }
    if constexpr (MODE == RW_NONLIN) {
      fft_regs<C, N, E, false>(v, z, 1, lane, tw);
      const R sc1 = pc.invP;
#pragma unroll
      for (int i = 0; i < KH + 1; ++i) {
        if (i == KH && lane != 0) break;
        W0[roff + lane + i * T] = cscale(v[i], sc1);  // i == KH: the Nyquist entry N/2 (lane 0)
      }
    }
    typename RD::acc t21[2] = {acc4, acc2};
    block_red_multi<R, 2>(t21, red2);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = RD::to_double(t21[0]);
      part[gridDim.x + blockIdx.x] = RD::to_double(t21[1]);
    }
  } else if constexpr (G3) {
    // sequence 0: Z = G_x + i G_y as below, G_x = i k~_x Y^-1 phi*; sequence 1:
    // the x-spectrum of phi* (Hermitian, so its inverse is real)
    const PC<R> pc(P);
    C v[2][E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = lane + i * T;
      const bool direct = k <= N / 2;
      const int m = direct ? k : N - k;
      const C f = W2[roff + m], b = W1[roff + m];
      const R ktm = kderiv<R>(m, N, pc.kfx);
      const C a = mk<C>(-ktm * f.y, ktm * f.x);
      v[0][i] = direct ? mk<C>(a.x - b.y, a.y + b.x) : mk<C>(a.x + b.y, b.x - a.y);
      v[1][i] = direct ? f : cconj(f);
    }
    if (sc->status != DEV_OK) return;
    fft_regs_multi<C, N, E, true, 2, false>(v, z, SEQ + 1, 1, lane, tw);
    typename RD::acc acc2 = RD::zero(), acc1 = RD::zero();
    const R beta = pc.beta, g3 = pc.g3, g3b = pc.g3b;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const C g = v[0][i];
      const R s = g.x * g.x + g.y * g.y;
      const R ph = v[1][i].x, p2 = ph * ph;
      acc2 = RD::add(acc2, s * s + g3b * (p2 * p2));
      acc1 = RD::add(acc1, s);
      if (MODE == RW_NONLIN) {
        const R fac = beta * s - (R)2;
        v[0][i] = mk<C>(fac * g.x, fac * g.y);
        v[1][i] = mk<C>(g3 * p2 * ph, (R)0);
      }
    }
    if constexpr (MODE == RW_NONLIN) {
      fft_regs_multi<C, N, E, false, 2, false>(v, z, SEQ + 1, 1, lane, tw);
      fft_sync<N, E>();
#pragma unroll
      for (int i = 0; i < E; ++i) z[spr(lane + i * T)] = v[0][i];
      fft_sync<N, E>();
      const R half = (R)0.5 * pc.invP;
#pragma unroll
      for (int i = 0; i < KH + 1; ++i) {
        if (i == KH && lane != 0) break;
        const int kk = lane + i * T;
        const C zk = v[0][i], zm = cconj(z[spr((N - kk) & (N - 1))]);
        const C sx = cadd(zk, zm), dy = csub(zk, zm);
        const C f3 = cscale(v[1][i], pc.invP);  // x-spectrum of gamma3 phi*^3, k <= N/2
        const R ktk = kderiv<R>(kk, N, pc.kfx);
        W0[roff + kk] = mk<C>(ktk * sx.x * half - f3.y, ktk * sx.y * half + f3.x);  // k~_x W_x + i f3
        W1[roff + kk] = mk<C>(dy.y * half, -dy.x * half);
      }
    }
    typename RD::acc t21[2] = {acc2, acc1};
    block_red_multi<R, 2>(t21, red2);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = RD::to_double(t21[0]);
      part[gridDim.x + blockIdx.x] = RD::to_double(t21[1]);
    }
  } else {
    // Z = G_x + i G_y over the full x-spectrum, element k = lane + i T loaded
    // straight into registers: k <= N/2 from the half spectrum, k > N/2 as
    // the Hermitian mirror of N - k.
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k = lane + i * T;
      const bool direct = k <= N / 2;
      const size_t off = roff + (direct ? k : N - k);
      const C a = W0[off], b = W1[off];
      v[i] = direct ? mk<C>(a.x - b.y, a.y + b.x) : mk<C>(a.x + b.y, b.x - a.y);
    }
    if (sc->status != DEV_OK) return;
    fft_regs<C, N, E, true>(v, z, 1, lane, tw);
    // pointwise on x = lane + i T: s = g_x^2 + g_y^2, partial sums, w = (beta s - 2) g
    typename RD::acc acc2 = RD::zero(), acc1 = RD::zero();
    const PC<R> pc(P);
    const R beta = pc.beta;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const C g = v[i];
      const R s = g.x * g.x + g.y * g.y;
      acc2 = RD::add(acc2, s * s);
      acc1 = RD::add(acc1, s);
      if (MODE == RW_NONLIN) {
        const R fac = beta * s - (R)2;
        v[i] = mk<C>(fac * g.x, fac * g.y);
      }
    }
    if constexpr (MODE == RW_NONLIN) {
      fft_regs<C, N, E, false>(v, z, 1, lane, tw);
      // the split into W_x, W_y pairs k with N - k: one exchange
      fft_sync<N, E>();
#pragma unroll
      for (int i = 0; i < E; ++i) z[spr(lane + i * T)] = v[i];
      fft_sync<N, E>();
      const R half = (R)0.5 * pc.invP;
#pragma unroll
      for (int i = 0; i < KH + 1; ++i) {
        if (i == KH && lane != 0) break;
        const int kk = lane + i * T;  // i == KH: the Nyquist entry N/2 (lane 0)
        const C zk = v[i], zm = cconj(z[spr((N - kk) & (N - 1))]);
        const C sx = cadd(zk, zm), dy = csub(zk, zm);
        W0[roff + kk] = cscale(sx, half);                      // W_x = (Z_k + conj Z_{N-k}) / 2
        W1[roff + kk] = mk<C>(dy.y * half, -dy.x * half);      // W_y = (Z_k - conj Z_{N-k}) / (2i)
      }
    }
    typename RD::acc t21[2] = {acc2, acc1};
    block_red_multi<R, 2>(t21, red2);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = RD::to_double(t21[0]);
      part[gridDim.x + blockIdx.x] = RD::to_double(t21[1]);
    }
  }
}

// ---------------------------------------------------------------------------
// Scalar SAV solve (one warp): combine the partial sums in a fixed order and
// solve eqs. solver-2 / solver-4 for r^{n+1}. BDF1 is the first-order start.
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int RPC, int MODE>
__global__ void __launch_bounds__(RPC * (N / E))
k2d_row(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, double* __restrict__ part,
        const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, double* __restrict__ real_io) {
  k2d_row_body<R, N, E, RPC, MODE>(P, W0, W1, part, sc, tw, real_io);
}

// the PFC model (W0: y-inverse of phi* in, x-spectrum of gamma3 phi*^3 - phi* out)
template <typename R, int N, int E, int RPC, int MODE>
__global__ void __launch_bounds__(RPC * (N / E))
k2d_row_pfc(const Params P, C_t<R>* __restrict__ W0, double* __restrict__ part, const SavScal* __restrict__ sc,
            const C_t<R>* __restrict__ tw) {
  k2d_row_body<R, N, E, RPC, MODE, false, true>(P, W0, nullptr, part, sc, tw, nullptr);
}

// with the phi^4 channel (W2: y-inverse of phi* in; W0 out: k~_x W_x + i F_x(gamma3 phi*^3))
template <typename R, int N, int E, int RPC, int MODE>
__global__ void __launch_bounds__(RPC * (N / E))
k2d_row_g3(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2,
           double* __restrict__ part, const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw) {
  k2d_row_body<R, N, E, RPC, MODE, true>(P, W0, W1, part, sc, tw, nullptr, W2);
}

// Scalar SAV solve (eqs. solver-2, solver-4 and solver-6 reduced to scalars).
// Inputs are the grid-reduced sums q = {sum s^2, sum s (E_1), and the
// half-spectrum sums of gamma, eta, theta without |Omega|} and r of the two
// current levels; BDF1 is the first-order start (r^0 = sqrt(E_1(phi^0))).
// sav_solve computes, sav_commit writes the record.
struct SolveOut {
  double E1, S, gamma, eta, theta, denom, LHS, xi, r_new, r_prev_new, alpha;
  bool ok;
};
// r of the two current levels (float64 on both paths)
struct RIn {
  double r1, r0;
  __device__ explicit RIn(const SavScal* sc) : r1(sc->r1), r0(sc->r0) {}
  __device__ RIn() : r1(0), r0(0) {}
};

// The solve in two parts. Everything that needs only the row pass's sums
// (q[0], q[1]) and r^n, r^{n-1} -- E_1, S = sqrt(E_1), 1/S and the
// coefficients below -- is formed first (it can overlap the gamma/eta/theta
// reduction); what is left once gamma, eta, theta arrive is a chain of five
// multiply-adds and one division:
//   denom = 1 - (dt/(2 E_1)) gamma,   rho = rb - ct theta,
//   LHS = ((dt/S) rho gamma + eta) / denom,   r^{n+1} = rho + LHS/(2S),
// with rb = (4 r^n - r^{n-1})/3 and ct = 1/(3S) (eqs. solver-2 and solver-4),
// or rb = S = r^0 and ct = 1/(2S) for the first-order start.
struct SolvePre {
  double E1, S, iS;
  double dt_iS;       // dt / S
  double h;           // dt / (2 E_1)
  double rb, ct;      // rho = rb - ct theta
  double r_prev_new;  // r^n, the new level's predecessor
};

// float64 scalar algebra (both paths).
__device__ inline SolvePre sav_solve_pre(const Params& P, const double* q, bool bdf1, const RIn& rin) {
  SolvePre o;
  o.E1 = P.hd * (P.e1c4 * q[0] + P.e1c2 * q[1]) + P.C * P.vol;
  o.S = sqrt(o.E1);
  o.iS = 1.0 / o.S;
  o.dt_iS = P.dt * o.iS;
  o.h = 0.5 * P.dt * (o.iS * o.iS);
  if (bdf1) {
    o.rb = o.S;
    o.ct = 0.5 * o.iS;
    o.r_prev_new = o.S;
  } else {
    o.rb = (4.0 * rin.r1 - rin.r0) * (1.0 / 3.0);
    o.ct = o.iS * (1.0 / 3.0);
    o.r_prev_new = rin.r1;
  }
  return o;
}

__device__ inline SolveOut sav_solve_post(const Params& P, const SolvePre& pre, const double* qg) {
  SolveOut o;
  o.E1 = pre.E1;
  o.S = pre.S;
  o.gamma = P.vol * qg[0]; o.eta = P.vol * qg[1]; o.theta = P.vol * qg[2];
  o.denom = fma(-pre.h, o.gamma, 1.0);
  const double rho = fma(-pre.ct, o.theta, pre.rb);
  o.LHS = fma(pre.dt_iS * rho, o.gamma, o.eta) / o.denom;
  o.r_new = fma(0.5 * pre.iS, o.LHS, rho);
  o.r_prev_new = pre.r_prev_new;
  o.xi = o.r_new * pre.iS;
  o.alpha = pre.dt_iS * o.r_new;
  o.ok = isfinite(o.E1) && o.E1 > 0.0 && isfinite(o.gamma) && isfinite(o.eta) && isfinite(o.theta) &&
         o.denom > 0.0 && isfinite(o.r_new);
  return o;
}

__device__ inline SolveOut sav_solve(const Params& P, const double* q, bool bdf1, const RIn& rin) {
  return sav_solve_post(P, sav_solve_pre(P, q, bdf1, rin), q + 2);
}

// Write a solve into the record: r shifts, p and pending as given; alpha also
// rounded to float32 for the float32-bulk kernels.
__device__ inline void sav_commit(SavScal* sc, const SolveOut& o, int p_new, int pending) {
  sc->E1 = o.E1; sc->S = o.S; sc->gamma = o.gamma; sc->eta = o.eta; sc->theta = o.theta;
  sc->denom = o.denom; sc->LHS = o.LHS; sc->xi = o.xi;
  if (!o.ok) { sc->status = DEV_NONFINITE; return; }
  sc->r0 = o.r_prev_new;
  sc->r1 = o.r_new;
  sc->alpha = o.alpha;
  sc->alpha_f = (float)o.alpha;
  sc->p = p_new;
  sc->pending = pending;
  sc->nsteps += 1;
  if (sc->ring) {  // the step's record, written straight into pinned host memory
    double* e = sc->ring + kRingFields * (sc->nsteps % sc->ring_cap);
    e[1] = o.r_new; e[2] = o.r_prev_new; e[3] = o.xi; e[4] = o.gamma; e[5] = o.E1; e[6] = o.alpha;
    e[7] = (double)sc->status;
    e[0] = (double)sc->nsteps;
  }
}

// Lazy-update form used by the separate forward column pass: newest holds
// phi^n, the update stays pending (materialised later into slot 1-newest).
__device__ inline void sav_scalar_solve(const Params& P, SavScal* sc, const double* q, bool bdf1, int newest) {
  const SolveOut o = sav_solve(P, q, bdf1, RIn(sc));
  sav_commit(sc, o, newest, bdf1 ? PEND_BDF1 : PEND_BDF2);
}

// ---------------------------------------------------------------------------
// Column forward pass (thread layout as the inverse pass).
// partG: 3 x gridDim.x doubles (gamma, eta, theta partial sums, without |Omega|).
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int CT, int MODE, bool G3 = false, bool PF = false>
__device__ __forceinline__ void k2d_col_fwd_body(const Params& P, Slots<R> S, const C_t<R>* __restrict__ W0,
                                                 const C_t<R>* __restrict__ W1, C_t<R>* __restrict__ Nhat,
                                                 double* __restrict__ partG, const double* __restrict__ partE,
                                                 int nE, SavScal* __restrict__ sc, unsigned* __restrict__ counter,
                                                 const C_t<R>* __restrict__ tw, int target) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N, E>::T;
  // PF (the PFC model): W0 holds the x-spectrum of N itself, one field
  constexpr int NF = (MODE == CF_TO_STATE || PF) ? 1 : 2;
  static_assert(!G3 || MODE == CF_BDF2 || MODE == CF_BDF1 || MODE == CF_NHAT || MODE == CF_PART,
                "the phi^4 channel is carried by the modes that form N_hat");
  constexpr int NTH = CT * T;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr int SEQ = sp_len(N);
  static_assert(NTH % 32 == 0, "tile must fill whole warps");
  using RD = Red<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ typename RD::acc red[32];
  __shared__ double red5[5][32];
  __shared__ double qres[5];
  __shared__ bool am_last;

  pdl_wait();
  pdl_trigger();
  if (sc->status != DEV_OK) return;
  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c;
  const bool col = kx < NH;
  C v[NF][E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const size_t off = (size_t)(lane + i * T) * NH + kx;
    v[0][i] = col ? W0[off] : mk<C>(0, 0);  // G3: k~_x W_x + i F_x(gamma3 phi*^3)
    if (NF == 2) v[NF - 1][i] = col ? W1[off] : mk<C>(0, 0);
  }

  if constexpr (MODE == CF_TO_STATE) {
    fft_regs_multi<C, N, E, false, NF, true>(v, sm + c, SEQ * CTP, CTP, lane, tw);
    C* dst = S.at(target);
    if (col) {
#pragma unroll
      for (int i = 0; i < E; ++i) dst[(size_t)(lane + i * T) * NH + kx] = v[0][i];
    }
  } else {
    const PC<R> pc(P);
    const int p = sc->p;
    const int newest = (sc->pending == PEND_BDF2) ? 1 - p : p;
    const C* snew = S.at(newest);
    const C* sold = S.at(1 - newest);
    const R c0 = (MODE == CF_BDF1) ? (R)1 : (R)1.5;
    // the state is loaded before the FFT where registers allow (its latency
    // overlaps the transform), after it in the batched pass, which keeps
    // its registers low for three resident blocks per SM
    constexpr bool EARLY = (MODE != CF_PART);
    C vn[E], vo[E];
    auto load_state = [&]() {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        vn[i] = vo[i] = mk<C>(0, 0);
        if (MODE != CF_NHAT && col) {
          const size_t off = (size_t)(lane + i * T) * NH + kx;
          vn[i] = snew[off];
          if (MODE == CF_BDF2 || MODE == CF_PART) vo[i] = sold[off];
        }
      }
    };
    if (EARLY) load_state();
    fft_regs_multi<C, N, E, false, NF, true>(v, sm + c, SEQ * CTP, CTP, lane, tw);
    if (!EARLY) load_state();
    typename RD::acc ag = RD::zero(), ae = RD::zero(), at = RD::zero();
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int ky = lane + i * T;
      if (!col) continue;
      const size_t off = (size_t)ky * NH + kx;
      const C wx = v[0][i], wy = v[NF - 1][i];
      const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
      // N_hat = -i (k~_x W_x + k~_y W_y)
      C nh;
      if constexpr (PF) {
        nh = (off == 0) ? mk<C>(0, 0) : wx;  // gamma3 phi*^3 - phi*, its mean removed
      } else if constexpr (G3) {
        // -i (Y(k~_x W_x + i W2) + k~_y W_y): the transform of gamma3 phi*^3 joins
        // N_hat, whose zero mode (the mean of gamma3 phi*^3) is removed
        const R ux = wx.x + kty * wy.x, uy = wx.y + kty * wy.y;
        nh = (off == 0) ? mk<C>(0, 0) : mk<C>(uy, -ux);
      } else {
        const R ux = ktx * wx.x + kty * wy.x, uy = ktx * wx.y + kty * wy.y;
        nh = mk<C>(uy, -ux);
      }
      Nhat[off] = nh;
      if (MODE == CF_NHAT) continue;
      const R K2 = sym_K2<R>(kx, ky, N, pc);
      const R invA = sym_invA<R>(K2, c0, pc);
      C vv;
      if (MODE == CF_BDF1) {
        vv = vn[i];
      } else {
        vv = mk<C>((R)2 * vn[i].x - (R)0.5 * vo[i].x, (R)2 * vn[i].y - (R)0.5 * vo[i].y);
      }
      const R w = (kx == 0 || kx == N / 2) ? (R)1 : (R)2;  // half-spectrum Parseval weight
      const R n2 = nh.x * nh.x + nh.y * nh.y;
      const R nv = nh.x * vv.x + nh.y * vv.y;
      // eta takes the stabiliser's right-hand side s phi^n (Sec. 5.2), theta does not
      const R sK = rn_mul(pc.sdt, K2);
      const R nvs = nh.x * rn_fma(sK, vn[i].x, vv.x) + nh.y * rn_fma(sK, vn[i].y, vv.y);
      ag = RD::add(ag, w * (-K2 * invA) * n2);   // <N, A^{-1} Delta N>
      ae = RD::add(ae, w * nvs * invA);          // <N, A^{-1} v>
      at = RD::add(at, w * nv);                  // <N, v>
    }
    if constexpr (MODE != CF_NHAT) {
      const typename RD::acc tg = block_red<R>(ag, red);
      const typename RD::acc te = block_red<R>(ae, red);
      const typename RD::acc tt = block_red<R>(at, red);
      if (threadIdx.x == 0) {
        partG[blockIdx.x] = RD::to_double(tg);
        partG[gridDim.x + blockIdx.x] = RD::to_double(te);
        partG[2 * gridDim.x + blockIdx.x] = RD::to_double(tt);
        if (MODE != CF_PART) {
          __threadfence();
          const unsigned prev = atomicAdd(counter, 1u);
          am_last = (prev == gridDim.x - 1);
        } else {
          am_last = false;
        }
      }
      __syncthreads();
      if (am_last) {
        __threadfence();
        const double* arr[5] = {partE, partE + nE, partG, partG + gridDim.x, partG + 2 * gridDim.x};
        const int cnt[5] = {nE, nE, (int)gridDim.x, (int)gridDim.x, (int)gridDim.x};
        block_sum_arrays<5>(arr, cnt, qres, red5);
        if (threadIdx.x == 0) {
          sav_scalar_solve(P, sc, qres, MODE == CF_BDF1, newest);
          *counter = 0u;
        }
      }
    }
  }
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_fwd(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, const C_t<R>* __restrict__ W1,
            C_t<R>* __restrict__ Nhat, double* __restrict__ partG, const double* __restrict__ partE, int nE,
            SavScal* __restrict__ sc, unsigned* __restrict__ counter, const C_t<R>* __restrict__ tw,
            int target) {
  k2d_col_fwd_body<R, N, E, CT, MODE>(P, S, W0, W1, Nhat, partG, partE, nE, sc, counter, tw, target);
}

// the PFC model (W0 holds the x-spectrum of gamma3 phi*^3 - phi*)
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_fwd_pfc(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, C_t<R>* __restrict__ Nhat,
                double* __restrict__ partG, const double* __restrict__ partE, int nE, SavScal* __restrict__ sc,
                unsigned* __restrict__ counter, const C_t<R>* __restrict__ tw) {
  k2d_col_fwd_body<R, N, E, CT, MODE, false, true>(P, S, W0, nullptr, Nhat, partG, partE, nE, sc, counter, tw, 0);
}

// with the phi^4 channel (W0 holds k~_x W_x + i F_x(gamma3 phi*^3))
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_fwd_g3(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, const C_t<R>* __restrict__ W1,
               C_t<R>* __restrict__ Nhat, double* __restrict__ partG, const double* __restrict__ partE, int nE,
               SavScal* __restrict__ sc, unsigned* __restrict__ counter, const C_t<R>* __restrict__ tw) {
  k2d_col_fwd_body<R, N, E, CT, MODE, true>(P, S, W0, W1, Nhat, partG, partE, nE, sc, counter, tw, 0);
}

// ---------------------------------------------------------------------------
// Fused column pass: the end of step n and the start of step n+1 for one tile
// of CT kx columns, with one grid-wide barrier in between.
//   A: forward DFT in y of W (the row pass output), N_hat = -i k~ . W_hat
//      (kept in registers), partial sums of gamma, eta, theta with the state
//      (phi^n, phi^{n-1}) held in registers.
//   barrier: every block publishes its partial sums and arrives; the last
//      block reduces all of them and solves the scalar system for r^{n+1}
//      and alpha = dt r^{n+1} / sqrt(E_1); the others wait (bounded).
//   B: phi^{n+1} = alpha A^{-1} Delta N_hat + A^{-1} v (eq. solver-6) written
//      over phi^{n-1}, phi* = 2 phi^{n+1} - phi^n, i k~ phi*, inverse DFT in y
//      into W for the next row pass.
// Launched cooperatively (all blocks co-resident).
// ---------------------------------------------------------------------------
constexpr long long kSpinLimit = 1ll << 22;  // x ~100 ns sleep: about half a second

// Bounded wait until *ctr >= target (a counter other blocks advance): polls
// with a short sleep at most `limit` times. Returns false if the limit ran
// out; the caller then latches DEV_TIMEOUT and returns instead of hanging.
__device__ __forceinline__ bool wait_counter(const unsigned long long* ctr, unsigned long long target,
                                             long long limit) {
  long long it = 0;
  while (*((const volatile unsigned long long*)ctr) < target) {
    if (++it > limit) return false;
    __nanosleep(32);
  }
  return true;
}

template <typename R, int N, int E, int CT, bool BDF1>
__global__ void __launch_bounds__(CT * (N / E))
k2d_col_fused(const Params P, Slots<R> S, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
              double* __restrict__ partG, const double* __restrict__ partE, int nE, SavScal* __restrict__ sc,
              unsigned long long* __restrict__ sync64, const C_t<R>* __restrict__ tw) {
  using C = C_t<R>;
  using RD = Red<R>;
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NTH = CT * T;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr int SEQ = sp_len(N);
  static_assert(NTH % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ typename RD::acc redb[3][32];
  __shared__ double red5[5][32];
  __shared__ double qres[5];
  __shared__ int bar_ok;

  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c;
  const bool col = kx < NH;

  // ---- A: the W columns and the state of this thread's rows ky = lane + i T.
  // The W loads go out first (valid whatever the status); the status, the
  // slot index and r (one round trip) follow, then the state loads.
  C g[2][E], vn[E], vo[E], nh[E];
  R ia[E];  // A^{-1} of each row, kept for the update (the same rounded value)
#pragma unroll
  for (int i = 0; i < E; ++i) {
    g[0][i] = g[1][i] = mk<C>(0, 0);
    if (col) {
      const size_t off = (size_t)(lane + i * T) * NH + kx;
      g[0][i] = W0[off];
      g[1][i] = W1[off];
    }
  }
  if (sc->status != DEV_OK) return;
  const PC<R> pc(P);
  const int p = sc->p;  // phi^n in slot p, phi^{n-1} in slot 1-p (nothing pending)
  const RIn rin(sc);  // read before arriving at the barrier (block 0 rewrites them after it)
  C* scur = S.at(p);
  C* sold = S.at(1 - p);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    vn[i] = vo[i] = mk<C>(0, 0);
    if (col) {
      const size_t off = (size_t)(lane + i * T) * NH + kx;
      vn[i] = scur[off];
      vo[i] = sold[off];
    }
  }
  // the row pass's E_1 sums (complete before this launch), reduced while the
  // loads above are in flight; the float64 zero modes for the update
  {
    const double* arr[2] = {partE, partE + nE};
    const int cnt[2] = {nE, nE};
    block_sum_arrays<2>(arr, cnt, qres, red5);
  }
  double zm_n = 0.0, zm_o = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    zm_n = sc->zm[p];
    zm_o = sc->zm[1 - p];
  }
  fft_regs_multi<C, N, E, false, 2, true>(g, sm + c, SEQ * CTP, CTP, lane, tw);
  const R c0 = BDF1 ? (R)1 : (R)1.5;
  typename RD::acc ag = RD::zero(), ae = RD::zero(), at = RD::zero();
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int ky = lane + i * T;
    nh[i] = mk<C>(0, 0);
    ia[i] = (R)0;
    if (!col) continue;
    const C wx = g[0][i], wy = g[1][i];
    const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
    const R ux = ktx * wx.x + kty * wy.x, uy = ktx * wx.y + kty * wy.y;
    nh[i] = mk<C>(uy, -ux);  // N_hat = -i (k~_x W_x + k~_y W_y)
    const R K2 = sym_K2<R>(kx, ky, N, pc);
    const R invA = sym_invA<R>(K2, c0, pc);
    ia[i] = invA;
    C v;
    if (BDF1) v = vn[i];
    else v = mk<C>((R)2 * vn[i].x - (R)0.5 * vo[i].x, (R)2 * vn[i].y - (R)0.5 * vo[i].y);
    const R w = (kx == 0 || kx == N / 2) ? (R)1 : (R)2;  // half-spectrum Parseval weight
    const R n2 = nh[i].x * nh[i].x + nh[i].y * nh[i].y;
    const R nv = nh[i].x * v.x + nh[i].y * v.y;
    const R sK = rn_mul(pc.sdt, K2);  // stabiliser (Sec. 5.2): in eta, not in theta
    const R nvs = nh[i].x * rn_fma(sK, vn[i].x, v.x) + nh[i].y * rn_fma(sK, vn[i].y, v.y);
    ag = RD::add(ag, w * (-K2 * invA) * n2);
    ae = RD::add(ae, w * nvs * invA);
    at = RD::add(at, w * nv);
  }
  typename RD::acc t3[3] = {ag, ae, at};
  block_red_multi<R, 3>(t3, redb);

  // ---- grid barrier: publish the partial sums, arrive, wait for all blocks
  // (bounded; thread 0 takes E_1 and S meanwhile); then every block reduces
  // the gamma, eta, theta partial sums in the same fixed order and finishes
  // the scalar solve itself (identical results), and block 0 alone writes the
  // record. sync64[0] counts arrivals monotonically, so it never needs a
  // reset: this launch's target is the next multiple of the grid.
  SolvePre pre;
  if (threadIdx.x == 0) {
    partG[blockIdx.x] = RD::to_double(t3[0]);
    partG[gridDim.x + blockIdx.x] = RD::to_double(t3[1]);
    partG[2 * gridDim.x + blockIdx.x] = RD::to_double(t3[2]);
    __threadfence();
    const unsigned long long prev = atomicAdd(sync64, 1ull);
    const unsigned long long target = (prev / gridDim.x + 1ull) * gridDim.x;
    pre = sav_solve_pre(P, qres, BDF1, rin);  // E_1, S, 1/S and the rest: overlaps the wait
    const bool ok = wait_counter(sync64, target, kSpinLimit);
    if (!ok) atomicExch(&sc->status, (int)DEV_TIMEOUT);
    __threadfence();
    bar_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (!bar_ok) return;
  {
    const double* arr[3] = {partG, partG + gridDim.x, partG + 2 * gridDim.x};
    const int cnt[3] = {(int)gridDim.x, (int)gridDim.x, (int)gridDim.x};
    block_sum_arrays<3>(arr, cnt, qres + 2, red5);
  }
  __shared__ R alpha_s;
  __shared__ int solve_ok;
  if (threadIdx.x == 0) {
    const SolveOut o = sav_solve_post(P, pre, qres + 2);
    alpha_s = (R)o.alpha;
    solve_ok = o.ok;
    if (blockIdx.x == 0) sav_commit(sc, o, 1 - p, PEND_NONE);
  }
  __syncthreads();
  if (!solve_ok) return;
  const R al = alpha_s;

  // ---- B: update, next extrapolation and its gradients, inverse DFT in y
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int ky = lane + i * T;
    C g0 = mk<C>(0, 0), g1 = mk<C>(0, 0);
    if (col) {
      const size_t off = (size_t)ky * NH + kx;
      const C cur = vn[i];
      C nw;
      if (off == 0) {
        // zero mode: A_0 = c0 and Delta kills N; BDF1 keeps phi_0, BDF2 gives a + (a - b)/3
        const double z = BDF1 ? zm_n : zero_mode_update(zm_n, zm_o);
        sc->zm[1 - p] = z;
        nw = mk<C>((R)z, (R)0);
      } else {
        const R K2 = sym_K2<R>(kx, ky, N, pc);
        if (BDF1) nw = bdf1_update<C, R>(cur, nh[i], K2, ia[i], al, rn_mul(pc.sdt, K2));
        else nw = bdf2_update<C, R>(cur, vo[i], nh[i], K2, ia[i], al, rn_mul(pc.sdt, K2));
      }
      sold[off] = nw;  // phi^{n+1} over phi^{n-1}
      const C ph = mk<C>((R)2 * nw.x - cur.x, (R)2 * nw.y - cur.y);
      const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
      g0 = mk<C>(-ktx * ph.y, ktx * ph.x);
      g1 = mk<C>(-kty * ph.y, kty * ph.x);
    }
    g[0][i] = g0;
    g[1][i] = g1;
  }
  fft_regs_multi<C, N, E, true, 2, true>(g, sm + c, SEQ * CTP, CTP, lane, tw);
  if (col) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const size_t off = (size_t)(lane + i * T) * NH + kx;
      W0[off] = g[0][i];
      W1[off] = g[1][i];
    }
  }
}

// ---------------------------------------------------------------------------
// Pointwise kernels over the half spectrum (grid-stride)
// ---------------------------------------------------------------------------

// Materialise the pending update into slot 1-p (does not flip p).
template <typename R>
__global__ void k2d_finalize(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, SavScal* sc) {
  using C = C_t<R>;
  if (sc->status != DEV_OK || sc->pending == PEND_NONE) return;
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const bool bdf1 = sc->pending == PEND_BDF1;
  const R alpha = read_alpha<R>(sc);
  const PC<R> pc(P);
  C* cur = S.at(p);
  C* old = S.at(1 - p);
  const size_t total = (size_t)N * NH;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    if (off == 0) {
      const double z = bdf1 ? sc->zm[p] : zero_mode_update(sc->zm[p], sc->zm[1 - p]);
      sc->zm[1 - p] = z;
      old[0] = mk<C>((R)z, (R)0);
      continue;
    }
    const R K2 = sym_K2<R>(kx, ky, N, pc);
    const C cu = cur[off], nh = Nhat[off];
    C nw;
    if (bdf1) {
      nw = bdf1_update<C, R>(cu, nh, K2, sym_invA<R>(K2, (R)1, pc), alpha, rn_mul(pc.sdt, K2));
    } else {
      nw = bdf2_update<C, R>(cu, old[off], nh, K2, sym_invA<R>(K2, (R)1.5, pc), alpha, rn_mul(pc.sdt, K2));
    }
    old[off] = nw;
  }
}

// Ghost point (eq. scheme-SAV-initial-1): slot 1-p = phi^0 + dt |k|^2 (N_hat + (a + |k|^4) phi^0).
template <typename R>
__global__ void k2d_ghost(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, SavScal* sc) {
  using C = C_t<R>;
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const C* cur = S.at(p);
  C* dst = S.at(1 - p);
  const PC<R> pc(P);
  const size_t total = (size_t)N * NH;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    const R K2 = sym_K2<R>(kx, ky, N, pc);
    const C cu = cur[off], nh = Nhat[off];
    const R L = sym_L<R>(K2, pc);
    const R f = pc.dt * K2;
    dst[off] = mk<C>(cu.x + f * (nh.x + L * cu.x), cu.y + f * (nh.y + L * cu.y));
    if (off == 0) sc->zm[1 - p] = sc->zm[p];
  }
}

// Spectral norms of the newest level phi = slot p and psi = 2 phi - slot (1-p),
// without the zero mode (added in FP64 from zm):
// part[0..G)   = sum w |phi_k|^2, part[G..2G) = sum w |k|^4 |phi_k|^2,
// part[2G..3G) = sum w L(k) |psi_k|^2 (L the symbol of L_N), part[3G..4G) =
// sum w |k|^2 |phi_k|^2.
template <typename R>
__global__ void k2d_norms(const Params P, Slots<R> S, const SavScal* sc, double* part) {
  using C = C_t<R>;
  __shared__ double red[32];
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const C* nw = S.at(p);
  const C* ol = S.at(1 - p);
  const size_t total = (size_t)N * NH;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    if (off == 0) continue;
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    const double kxx = kx * P.kf[0], kyy = kfull<double>(ky, N, P.kf[1]);
    const double K2 = kxx * kxx + kyy * kyy;
    const double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
    const C u = nw[off], v = ol[off];
    const double n2 = (double)u.x * u.x + (double)u.y * u.y;
    const double px = 2.0 * u.x - v.x, py = 2.0 * u.y - v.y;
    const double Ls = P.pfc ? P.a + (1.0 - K2) * (1.0 - K2) : P.a + K2 * K2;
    a0 += w * n2;
    a1 += w * K2 * K2 * n2;
    a2 += w * Ls * (px * px + py * py);
    a3 += w * K2 * n2;
  }
  const double t0 = block_sum(a0, red);
  const double t1 = block_sum(a1, red);
  const double t2 = block_sum(a2, red);
  const double t3 = block_sum(a3, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = t0;
    part[gridDim.x + blockIdx.x] = t1;
    part[2 * gridDim.x + blockIdx.x] = t2;
    part[3 * gridDim.x + blockIdx.x] = t3;
  }
}

// Block partial sums of a real field (FP64).
static __global__ void k_real_sum(const double* __restrict__ f, size_t n, double* part) {
  __shared__ double red[32];
  double a = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a += f[i];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Write the FP64 zero modes into both slots.
template <typename R>
__global__ void k_put_zero_modes(Slots<R> S, const SavScal* sc) {
  using C = C_t<R>;
  const int p = sc->p;
  S.at(p)[0] = mk<C>((R)sc->zm[p], (R)0);
  S.at(1 - p)[0] = mk<C>((R)sc->zm[1 - p], (R)0);
}

enum ScalarOp : int {
  SO_FLIP = 0,        // after finalize: p = 1-p, pending = none
  SO_ZM_SLOT = 1,     // zm[slot] = sum(a)/P  (slot given by arg: 0 newest, 1 previous)
  SO_R_NEWEST = 2,    // r1 = sqrt(E1) from energy partials
  SO_R_PREV = 3,      // r0 = sqrt(E1)
  SO_ENERGY = 4,      // assemble E_N, E_mod, E_breve (a: energy partials, b: norm partials)
  SO_SET_R = 5,       // r1 = x0, r0 = x1
};

// One-warp scalar operations on the record.
// `a` holds float64 partial sums (E_1 for the ops that need them, the field
// for SO_ZM_SLOT); `b` holds float64 norm partials.
template <typename R>
__global__ void k_scalar_op(const Params P, SavScal* sc, int op, const double* a, int na, const double* b,
                            int nb, int arg, double x0, double x1) {
  const int lane = threadIdx.x;
  if (op == SO_FLIP) {
    if (lane == 0 && sc->status == DEV_OK && sc->pending != PEND_NONE) {
      sc->p = 1 - sc->p;
      sc->pending = PEND_NONE;
    }
    return;
  }
  if (op == SO_SET_R) {
    if (lane == 0) { sc->r1 = x0; sc->r0 = x1; }
    return;
  }
  if (op == SO_ZM_SLOT) {
    const double s = warp_sum_array(a, na, lane);
    if (lane == 0) sc->zm[arg == 0 ? sc->p : 1 - sc->p] = s / P.P;
    return;
  }
  const double s2 = warp_sum_array(a, na, lane);
  const double s1 = warp_sum_array(a + na, na, lane);
  if (op == SO_R_NEWEST || op == SO_R_PREV) {
    if (lane == 0) {
      const double E1 = P.hd * (P.e1c4 * s2 + P.e1c2 * s1) + P.C * P.vol;
      if (!(isfinite(E1) && E1 > 0.0)) { sc->status = DEV_NONFINITE; return; }
      if (op == SO_R_NEWEST) sc->r1 = sqrt(E1); else sc->r0 = sqrt(E1);
    }
    return;
  }
  if (op == SO_ENERGY && P.pfc) {
    // the PFC model: E_N = gamma3/4 ||phi||_4^4 + a/2 ||phi||^2 - ||grad phi||^2 + 1/2 ||Delta_N phi||^2
    // (eq. energy-PFC; s2 = sum phi^4 from the row pass), L = a + (1 + Delta)^2, whose zero-mode
    // symbol is a + 1, and E_breve = 1/2 ||L^{1/2} phi||^2 + r^2
    const double n0 = warp_sum_array(b, nb, lane);
    const double n1 = warp_sum_array(b + nb, nb, lane);
    const double n2 = warp_sum_array(b + 2 * nb, nb, lane);
    const double n3 = warp_sum_array(b + 3 * nb, nb, lane);
    if (lane == 0) {
      const int p = sc->p;
      const double z = sc->zm[p], zo = sc->zm[1 - p];
      const double phi2 = P.vol * (n0 + z * z);
      const double lap2 = P.vol * n1;
      const double grad2 = P.vol * n3;
      const double zp = 2.0 * z - zo;
      const double Lpsi = P.vol * (n2 + (P.a + 1.0) * zp * zp);
      const double Lphi = (P.a + 1.0) * phi2 - 2.0 * grad2 + lap2;
      const double r1 = sc->r1, r0 = sc->r0;
      sc->E_orig = 0.25 * P.g3 * P.hd * s2 + 0.5 * P.a * phi2 - grad2 + 0.5 * lap2;
      sc->E_mod = 0.25 * (Lphi + Lpsi) + 0.5 * (r1 * r1 + (2.0 * r1 - r0) * (2.0 * r1 - r0));
      sc->E_breve = 0.5 * Lphi + r1 * r1;
    }
    return;
  }
  if (op == SO_ENERGY) {
    const double n0 = warp_sum_array(b, nb, lane);
    const double n1 = warp_sum_array(b + nb, nb, lane);
    const double n2 = warp_sum_array(b + 2 * nb, nb, lane);
    if (lane == 0) {
      const int p = sc->p;
      const double z = sc->zm[p], zo = sc->zm[1 - p];
      const double phi2 = P.vol * (n0 + z * z);            // ||phi||^2
      const double lap2 = P.vol * n1;                       // ||Delta_N phi||^2
      const double zp = 2.0 * z - zo;
      const double Lpsi = P.vol * (n2 + P.a * zp * zp);     // ||L^{1/2} psi||^2
      const double Lphi = P.a * phi2 + lap2;
      const double grad4 = P.hd * s2, grad2 = P.hd * s1;
      const double r1 = sc->r1, r0 = sc->r0;
      sc->E_orig = 0.25 * P.beta * grad4 + 0.5 * P.a * phi2 - grad2 + 0.5 * lap2;
      sc->E_mod = 0.25 * (Lphi + Lpsi) + 0.5 * (r1 * r1 + (2.0 * r1 - r0) * (2.0 * r1 - r0));
      sc->E_breve = 0.5 * P.a * phi2 + 0.5 * lap2 + r1 * r1;
    }
  }
}

}  // namespace spfc
