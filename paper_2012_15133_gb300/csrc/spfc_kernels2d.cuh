// 2D kernels of the BDF2-SAV Fourier pseudo-spectral step (Sec. 2.2-2.3).
//
// Layout: real fields phi[y][x] (x fastest); spectra are R2C half spectra
// F[ky][kx], kx in [0, N/2], ky in [0, N), normalised as
// F_hat = (1/P) sum_j f_j exp(-i k.x_j) (eq. spectral-coll-1 on [0,L]^2).
// Work arrays W0, W1 have the same shape and hold, between passes, data that
// is transformed along y only ([y][kx]).
//
// One step = col_inv -> row -> col_fwd:
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
// Laplacian but has first-derivative symbol 0.
__device__ __forceinline__ double kfull(int i, int N, double kf) {
  return (double)((i <= N / 2) ? i : i - N) * kf;
}
__device__ __forceinline__ double kderiv(int i, int N, double kf) {
  return (i == N / 2) ? 0.0 : (double)((i < N / 2) ? i : i - N) * kf;
}

template <typename R> struct Slots {
  C_t<R>* s[2];
  // select without dynamic indexing of the parameter array (keeps it in registers)
  __device__ __forceinline__ C_t<R>* at(int i) const { return i ? s[1] : s[0]; }
};

enum ColInvMode : int { CI_STEP = 0, CI_GRAD = 1, CI_FIELD = 2 };
enum RowMode : int { RW_NONLIN = 0, RW_ENERGY = 1, RW_OUT_REAL = 2, RW_IN_REAL = 3 };
enum ColFwdMode : int { CF_BDF2 = 0, CF_BDF1 = 1, CF_NHAT = 2, CF_TO_STATE = 3 };

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
__device__ __forceinline__ R sym_K2(int kx, int ky, const Params& P) {
  const R kxx = rn_mul((R)kx, (R)P.kf[0]);
  const R kyy = (R)kfull(ky, P.N, P.kf[1]);
  return rn_fma(kxx, kxx, rn_mul(kyy, kyy));
}

// 1 / (c0 + dt |k|^2 (a + |k|^4)): inverse symbol of A_N (c0 = 3/2, eq. solver-1)
// or of the first-order operator (c0 = 1).
template <typename R>
__device__ __forceinline__ R sym_invA(R K2, R c0, const Params& P) {
  const R A = rn_fma((R)P.dt, rn_mul(K2, rn_fma(K2, K2, (R)P.a)), c0);
  return (R)1 / A;
}

// BDF2 update of one spectral coefficient (eq. solver-6 in the form
// phi^{n+1} = (dt r^{n+1}/sqrt(E1)) A^{-1} Delta N + A^{-1}(2 phi^n - phi^{n-1}/2)).
template <typename C, typename R>
__device__ __forceinline__ C bdf2_update(C cur, C old, C nh, R K2, R invA, R alpha) {
  const R bfac = rn_mul(rn_mul(-alpha, K2), invA);
  const R vx = rn_fma((R)2, cur.x, rn_mul((R)-0.5, old.x));
  const R vy = rn_fma((R)2, cur.y, rn_mul((R)-0.5, old.y));
  return mk<C>(rn_fma(bfac, nh.x, rn_mul(vx, invA)), rn_fma(bfac, nh.y, rn_mul(vy, invA)));
}

// First-order (BDF1 start) update: phi^1 = alpha A1^{-1} Delta N + A1^{-1} phi^0.
template <typename C, typename R>
__device__ __forceinline__ C bdf1_update(C cur, C nh, R K2, R invA, R alpha) {
  const R bfac = rn_mul(rn_mul(-alpha, K2), invA);
  return mk<C>(rn_fma(bfac, nh.x, rn_mul(cur.x, invA)), rn_fma(bfac, nh.y, rn_mul(cur.y, invA)));
}

// ---------------------------------------------------------------------------
// Column inverse pass. Grid: ceil(NH/CT) blocks, each a tile of CT kx columns.
// ---------------------------------------------------------------------------
template <typename R, int N, int CT, int MODE>
__global__ void __launch_bounds__((MODE == CI_FIELD ? 1 : 2) * CT * fft_shape<N>::T)
k2d_col_inv(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, C_t<R>* __restrict__ W0,
            C_t<R>* __restrict__ W1, SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, int which) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N>::T;
  constexpr int NF = (MODE == CI_FIELD) ? 1 : 2;
  constexpr int NTH = NF * CT * T;
  constexpr int CTP = CT + 1;
  constexpr int NH = N / 2 + 1;
  static_assert(NTH % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);

  if (sc->status != DEV_OK) return;
  const int p = sc->p;
  const int pending = (MODE == CI_STEP) ? sc->pending : 0;
  const R alpha = (R)sc->alpha;
  const int kx0 = blockIdx.x * CT;
  C* src_new;
  C* src_old;
  if (MODE == CI_STEP) {
    src_new = S.at(p);
    src_old = S.at(1 - p);
  } else {
    src_new = S.at(which == 0 ? p : 1 - p);
    src_old = src_new;
  }
  for (int idx = threadIdx.x; idx < N * CT; idx += NTH) {
    const int ky = idx / CT, c = idx % CT, kx = kx0 + c;
    C g0 = mk<C>(0, 0), g1 = mk<C>(0, 0);
    if (kx < NH) {
      const size_t off = (size_t)ky * NH + kx;
      const R ktx = (R)kderiv(kx, N, P.kf[0]), kty = (R)kderiv(ky, N, P.kf[1]);
      C ph;
      if (MODE == CI_STEP) {
        C cur = src_new[off], old = src_old[off];
        C nw = cur;
        if (pending) {
          if (off == 0) {
            // zero mode: c_0 = phi_0^n + (phi_0^n - phi_0^{n-1})/3 (A_0 = 3/2, Delta kills N)
            const double z = sc->zm[p] + (sc->zm[p] - sc->zm[1 - p]) / 3.0;
            sc->zm[1 - p] = z;
            nw = mk<C>((R)z, (R)0);
          } else {
            const R K2 = sym_K2<R>(kx, ky, P);
            nw = bdf2_update<C, R>(cur, old, Nhat[off], K2, sym_invA<R>(K2, (R)1.5, P), alpha);
          }
          src_old[off] = nw;  // phi^{n+1} overwrites phi^{n-1}
          old = cur;
        }
        ph = mk<C>((R)2 * nw.x - old.x, (R)2 * nw.y - old.y);  // phi* = 2 phi^{n+1} - phi^n
      } else {
        ph = src_new[off];
      }
      if (MODE == CI_FIELD) {
        g0 = ph;
      } else {
        g0 = mk<C>(-ktx * ph.y, ktx * ph.x);  // i k~_x phi
        g1 = mk<C>(-kty * ph.y, kty * ph.x);  // i k~_y phi
      }
    }
    sm[ky * CTP + c] = g0;
    if (NF == 2) sm[N * CTP + ky * CTP + c] = g1;
  }
  __syncthreads();
  {
    const int q = threadIdx.x / T, lane = threadIdx.x % T;
    const int f = q / CT, c = q % CT;
    fft_smem<C, N, true>(sm + f * N * CTP + c, CTP, lane, tw);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * CT; idx += NTH) {
    const int y = idx / CT, c = idx % CT, kx = kx0 + c;
    if (kx < NH) {
      W0[(size_t)y * NH + kx] = sm[y * CTP + c];
      if (NF == 2) W1[(size_t)y * NH + kx] = sm[N * CTP + y * CTP + c];
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass. Grid: N/RPC blocks, RPC rows each, T lanes per row.
// part: 2 x gridDim.x doubles: sum s^2 and sum s per block (without h^d).
// ---------------------------------------------------------------------------
template <typename R, int N, int RPC, int MODE>
__global__ void __launch_bounds__(RPC * fft_shape<N>::T)
k2d_row(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, double* __restrict__ part,
        const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, double* __restrict__ real_io) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N>::T;
  constexpr int NTH = RPC * T;
  constexpr int NH = N / 2 + 1;
  static_assert(NTH % 32 == 0, "rows must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ double red[32];

  if (sc->status != DEV_OK) return;
  const int rloc = threadIdx.x / T, lane = threadIdx.x % T;
  const int row = blockIdx.x * RPC + rloc;
  C* z = sm + rloc * (N + 1);
  const size_t roff = (size_t)row * NH;

  if constexpr (MODE == RW_IN_REAL) {
    for (int x = lane; x < N; x += T) z[x] = mk<C>((R)real_io[(size_t)row * N + x], (R)0);
    fft_smem<C, N, false>(z, 1, lane, tw);
    const R sc1 = (R)(1.0 / P.P);
    for (int k = lane; k < NH; k += T) W0[roff + k] = cscale(z[k], sc1);
  } else if constexpr (MODE == RW_OUT_REAL) {
    for (int k = lane; k < NH; k += T) {
      const C a = W0[roff + k];
      z[k] = a;
      if (k > 0 && k < N / 2) z[N - k] = cconj(a);
    }
    fft_smem<C, N, true>(z, 1, lane, tw);
    for (int x = lane; x < N; x += T) real_io[(size_t)row * N + x] = (double)z[x].x;
  } else {
  // pack Z = G_x + i G_y over the full x-spectrum (Hermitian extension)
  for (int k = lane; k < NH; k += T) {
    const C a = W0[roff + k], b = W1[roff + k];
    z[k] = mk<C>(a.x - b.y, a.y + b.x);
    if (k > 0 && k < N / 2) z[N - k] = mk<C>(a.x + b.y, b.x - a.y);
  }
  fft_smem<C, N, true>(z, 1, lane, tw);
  // pointwise: s = g_x^2 + g_y^2, partial sums, w = (beta s - 2) g
  R acc2 = 0, acc1 = 0;
  const R beta = (R)P.beta;
  for (int x = lane; x < N; x += T) {
    const C g = z[x];
    const R s = g.x * g.x + g.y * g.y;
    acc2 += s * s;
    acc1 += s;
    if (MODE == RW_NONLIN) {
      const R fac = beta * s - (R)2;
      z[x] = mk<C>(fac * g.x, fac * g.y);
    }
  }
  if (MODE == RW_NONLIN) {
    fft_smem<C, N, false>(z, 1, lane, tw);
    const R half = (R)(0.5 / P.P);
    for (int k = lane; k < NH; k += T) {
      const C zk = z[k], zm = cconj(z[(N - k) & (N - 1)]);
      const C sx = cadd(zk, zm), dy = csub(zk, zm);
      W0[roff + k] = cscale(sx, half);                      // W_x = (Z_k + conj Z_{N-k}) / 2
      W1[roff + k] = mk<C>(dy.y * half, -dy.x * half);      // W_y = (Z_k - conj Z_{N-k}) / (2i)
    }
  }
  const double t2 = block_sum((double)acc2, red);
  const double t1 = block_sum((double)acc1, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = t2;
    part[gridDim.x + blockIdx.x] = t1;
  }
  }
}

// ---------------------------------------------------------------------------
// Scalar SAV solve (one warp): combine the partial sums in a fixed order and
// solve eqs. solver-2 / solver-4 for r^{n+1}. BDF1 is the first-order start.
// ---------------------------------------------------------------------------
__device__ inline void sav_scalar_solve(const Params& P, SavScal* sc, const double* partE, int nE,
                                        const double* partG, int nG, bool bdf1, int newest, int lane) {
  const double s2 = warp_sum_array(partE, nE, lane);
  const double s1 = warp_sum_array(partE + nE, nE, lane);
  const double gs = warp_sum_array(partG, nG, lane);
  const double es = warp_sum_array(partG + nG, nG, lane);
  const double ts = warp_sum_array(partG + 2 * nG, nG, lane);
  if (lane != 0) return;
  const double E1 = P.hd * (0.25 * P.beta * s2 - s1) + P.C * P.vol;
  const double S = sqrt(E1);
  const double gamma = P.vol * gs, eta = P.vol * es, theta = P.vol * ts;
  const double dt = P.dt;
  double rho, r_new, r_base_prev;
  const double denom = 1.0 - dt * gamma / (2.0 * E1);
  if (bdf1) {
    const double r0 = S;  // r^0 = sqrt(E_1(phi^0))
    rho = r0 - theta / (2.0 * S);
    r_base_prev = r0;
  } else {
    rho = (4.0 * sc->r1 - sc->r0) / 3.0 - theta / (3.0 * S);
    r_base_prev = sc->r1;
  }
  const double LHS = (dt * rho * gamma / S + eta) / denom;
  r_new = rho + LHS / (2.0 * S);
  const bool ok = isfinite(E1) && E1 > 0.0 && isfinite(gamma) && isfinite(eta) && isfinite(theta) &&
                  denom > 0.0 && isfinite(r_new);
  sc->E1 = E1; sc->S = S; sc->gamma = gamma; sc->eta = eta; sc->theta = theta;
  sc->denom = denom; sc->LHS = LHS; sc->xi = r_new / S;
  if (!ok) { sc->status = DEV_NONFINITE; return; }
  sc->r0 = r_base_prev;
  sc->r1 = r_new;
  sc->alpha = dt * r_new / S;
  sc->p = newest;
  sc->pending = bdf1 ? PEND_BDF1 : PEND_BDF2;
  sc->nsteps += 1;
}

// ---------------------------------------------------------------------------
// Column forward pass. Grid: ceil(NH/CT) blocks.
// partG: 3 x gridDim.x doubles (gamma, eta, theta partial sums, without |Omega|).
// ---------------------------------------------------------------------------
template <typename R, int N, int CT, int MODE>
__global__ void __launch_bounds__((MODE == CF_TO_STATE ? 1 : 2) * CT * fft_shape<N>::T)
k2d_col_fwd(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, const C_t<R>* __restrict__ W1,
            C_t<R>* __restrict__ Nhat, double* __restrict__ partG, const double* __restrict__ partE, int nE,
            SavScal* __restrict__ sc, unsigned* __restrict__ counter, const C_t<R>* __restrict__ tw,
            int target) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N>::T;
  constexpr int NF = (MODE == CF_TO_STATE) ? 1 : 2;
  constexpr int NTH = NF * CT * T;
  constexpr int CTP = CT + 1;
  constexpr int NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ double red[32];
  __shared__ bool am_last;

  if (sc->status != DEV_OK) return;
  const int kx0 = blockIdx.x * CT;
  for (int idx = threadIdx.x; idx < N * CT; idx += NTH) {
    const int y = idx / CT, c = idx % CT, kx = kx0 + c;
    C a = mk<C>(0, 0), b = mk<C>(0, 0);
    if (kx < NH) {
      a = W0[(size_t)y * NH + kx];
      if (NF == 2) b = W1[(size_t)y * NH + kx];
    }
    sm[y * CTP + c] = a;
    if (NF == 2) sm[N * CTP + y * CTP + c] = b;
  }
  __syncthreads();
  {
    const int q = threadIdx.x / T, lane = threadIdx.x % T;
    const int f = q / CT, c = q % CT;
    fft_smem<C, N, false>(sm + f * N * CTP + c, CTP, lane, tw);
  }
  __syncthreads();

  if (MODE == CF_TO_STATE) {
    C* dst = S.at(target);
    for (int idx = threadIdx.x; idx < N * CT; idx += NTH) {
      const int ky = idx / CT, c = idx % CT, kx = kx0 + c;
      if (kx < NH) dst[(size_t)ky * NH + kx] = sm[ky * CTP + c];
    }
    return;
  }

  const int p = sc->p;
  const int newest = (sc->pending == PEND_BDF2) ? 1 - p : p;
  const C* snew = S.at(newest);
  const C* sold = S.at(1 - newest);
  const R c0 = (MODE == CF_BDF1) ? (R)1 : (R)1.5;
  R ag = 0, ae = 0, at = 0;
  for (int idx = threadIdx.x; idx < N * CT; idx += NTH) {
    const int ky = idx / CT, c = idx % CT, kx = kx0 + c;
    if (kx >= NH) continue;
    const size_t off = (size_t)ky * NH + kx;
    const C wx = sm[ky * CTP + c], wy = sm[N * CTP + ky * CTP + c];
    const R ktx = (R)kderiv(kx, N, P.kf[0]), kty = (R)kderiv(ky, N, P.kf[1]);
    // N_hat = -i (k~_x W_x + k~_y W_y)
    const R ux = ktx * wx.x + kty * wy.x, uy = ktx * wx.y + kty * wy.y;
    const C nh = mk<C>(uy, -ux);
    Nhat[off] = nh;
    if (MODE == CF_NHAT) continue;
    const R K2 = sym_K2<R>(kx, ky, P);
    const R invA = sym_invA<R>(K2, c0, P);
    C v;
    if (MODE == CF_BDF1) {
      v = snew[off];
    } else {
      const C cu = snew[off], ol = sold[off];
      v = mk<C>((R)2 * cu.x - (R)0.5 * ol.x, (R)2 * cu.y - (R)0.5 * ol.y);
    }
    const R w = (kx == 0 || kx == N / 2) ? (R)1 : (R)2;  // half-spectrum Parseval weight
    const R n2 = nh.x * nh.x + nh.y * nh.y;
    const R nv = nh.x * v.x + nh.y * v.y;
    ag += w * (-K2 * invA) * n2;   // <N, A^{-1} Delta N>
    ae += w * nv * invA;           // <N, A^{-1} v>
    at += w * nv;                  // <N, v>
  }
  if (MODE == CF_NHAT) return;
  const double tg = block_sum((double)ag, red);
  const double te = block_sum((double)ae, red);
  const double tt = block_sum((double)at, red);
  if (threadIdx.x == 0) {
    partG[blockIdx.x] = tg;
    partG[gridDim.x + blockIdx.x] = te;
    partG[2 * gridDim.x + blockIdx.x] = tt;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last && threadIdx.x < 32) {
    __threadfence();
    sav_scalar_solve(P, sc, partE, nE, partG, gridDim.x, MODE == CF_BDF1, newest, threadIdx.x);
    if (threadIdx.x == 0) *counter = 0u;
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
  const R alpha = (R)sc->alpha;
  C* cur = S.at(p);
  C* old = S.at(1 - p);
  const size_t total = (size_t)N * NH;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    if (off == 0) {
      const double z = bdf1 ? sc->zm[p] : sc->zm[p] + (sc->zm[p] - sc->zm[1 - p]) / 3.0;
      sc->zm[1 - p] = z;
      old[0] = mk<C>((R)z, (R)0);
      continue;
    }
    const R K2 = sym_K2<R>(kx, ky, P);
    const C cu = cur[off], nh = Nhat[off];
    C nw;
    if (bdf1) {
      nw = bdf1_update<C, R>(cu, nh, K2, sym_invA<R>(K2, (R)1, P), alpha);
    } else {
      nw = bdf2_update<C, R>(cu, old[off], nh, K2, sym_invA<R>(K2, (R)1.5, P), alpha);
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
  const size_t total = (size_t)N * NH;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    const R K2 = sym_K2<R>(kx, ky, P);
    const C cu = cur[off], nh = Nhat[off];
    const R L = (R)P.a + K2 * K2;
    const R f = (R)P.dt * K2;
    dst[off] = mk<C>(cu.x + f * (nh.x + L * cu.x), cu.y + f * (nh.y + L * cu.y));
    if (off == 0) sc->zm[1 - p] = sc->zm[p];
  }
}

// Spectral norms of the newest level phi = slot p and psi = 2 phi - slot (1-p),
// without the zero mode (added in FP64 from zm):
// part[0..G)   = sum w |phi_k|^2, part[G..2G) = sum w |k|^4 |phi_k|^2,
// part[2G..3G) = sum w (a + |k|^4) |psi_k|^2.
template <typename R>
__global__ void k2d_norms(const Params P, Slots<R> S, const SavScal* sc, double* part) {
  using C = C_t<R>;
  __shared__ double red[32];
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const C* nw = S.at(p);
  const C* ol = S.at(1 - p);
  const size_t total = (size_t)N * NH;
  double a0 = 0, a1 = 0, a2 = 0;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    if (off == 0) continue;
    const int ky = (int)(off / NH), kx = (int)(off % NH);
    const double kxx = kx * P.kf[0], kyy = kfull(ky, N, P.kf[1]);
    const double K2 = kxx * kxx + kyy * kyy;
    const double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
    const C u = nw[off], v = ol[off];
    const double n2 = (double)u.x * u.x + (double)u.y * u.y;
    const double px = 2.0 * u.x - v.x, py = 2.0 * u.y - v.y;
    a0 += w * n2;
    a1 += w * K2 * K2 * n2;
    a2 += w * (P.a + K2 * K2) * (px * px + py * py);
  }
  const double t0 = block_sum(a0, red);
  const double t1 = block_sum(a1, red);
  const double t2 = block_sum(a2, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = t0;
    part[gridDim.x + blockIdx.x] = t1;
    part[2 * gridDim.x + blockIdx.x] = t2;
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
static __global__ void k_scalar_op(const Params P, SavScal* sc, int op, const double* a, int na, const double* b,
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
      const double E1 = P.hd * (0.25 * P.beta * s2 - s1) + P.C * P.vol;
      if (!(isfinite(E1) && E1 > 0.0)) { sc->status = DEV_NONFINITE; return; }
      if (op == SO_R_NEWEST) sc->r1 = sqrt(E1); else sc->r0 = sqrt(E1);
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
