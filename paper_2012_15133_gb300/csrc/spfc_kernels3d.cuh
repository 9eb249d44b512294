// 3D kernels of the BDF2-SAV Fourier pseudo-spectral step (Sec. 2.2-2.3).
//
// Layout: real fields phi[z][y][x] (x fastest); half spectra F[kz][ky][kx],
// kx in [0, N/2] (NH = N/2 + 1 entries per row), PS = N * NH entries per plane.
// Work arrays W0, W1, W2 hold data that is transformed along some axes only.
//
// One step (W prepared by the previous step: the y- and z-inverse transforms
// of i k~_d phi*):
//   row    : per pair of x-rows, inverse DFT in x of the three gradients
//            (G_x + i G_y of each row, G_z of both rows packed as one complex
//            sequence), s = |grad phi*|^2, E_1 partial sums, w = (beta s - 2) g,
//            forward DFTs, split back into W_x, W_y, W_z;
//   y-fwd  : forward DFT in y; Q1 = k~_x W_x + k~_y W_y, Q2 = W_z;
//   z-fwd  : forward DFT in z; N_hat = -i (Q1 + k~_z Q2); gamma, eta, theta partial sums;
//   scalar : one block reduces all partial sums and solves for r^{n+1} (eqs. solver-2, -4);
//   z-inv  : phi^{n+1} = alpha A^{-1} Delta N_hat + A^{-1} v (eq. solver-6), phi* =
//            2 phi^{n+1} - phi^n, inverse DFT in z of phi* and of i k~_z phi*;
//   y-inv  : inverse DFT in y of i k~_y F, F and G_z; W_x = i k~_x (.) of F's.
//
// The optional phi^4 term (G3 variants) needs no further z- or y-transform
// and no further array pass: y-inv stores Y^-1 F (phi* as an x-spectrum) in W3
// instead of W_x = i k~_x Y^-1 F; the row pass forms W_x from it, carries
// phi*(row 0) + i phi*(row 1) as a fourth sequence, adds (gamma3/beta) phi*^4
// to the sum of s^2 and writes W0 = k~_x W_x + i F_x(gamma3 phi*^3) (k~_x is
// known there and constant along y and z); y-fwd then forms Q1 = Y W0 +
// k~_y Y W_y, so that -i (Q1 + k~_z Q2) gains the transform of gamma3 phi*^3;
// z-fwd removes its mean (N_hat_0 := 0).
#pragma once

#include "spfc_kernels2d.cuh"

namespace spfc {

template <typename R>
__device__ __forceinline__ R sym_K2_3d(int kx, int ky, int kz, int N, const PC<R>& c) {
  const R kxx = rn_mul((R)kx, c.kfx);
  const R kyy = rn_mul((R)((ky <= N / 2) ? ky : ky - N), c.kfy);
  const R kzz = rn_mul((R)((kz <= N / 2) ? kz : kz - N), c.kfz);
  return rn_fma(kxx, kxx, rn_fma(kyy, kyy, rn_mul(kzz, kzz)));
}

enum Y3Mode : int { Y3_FWD = 0, Y3_INV = 1, Y3_INV_FIELD = 2, Y3_FWD_FIELD = 3 };
enum Z3Mode : int { Z3F_BDF2 = 0, Z3F_BDF1 = 1, Z3F_NHAT = 2, Z3F_TO_STATE = 3 };
enum Z3IMode : int { Z3I_STEP = 0, Z3I_STEP_BDF1 = 1, Z3I_PREP = 2, Z3I_GRAD = 3, Z3I_FIELD = 4 };

template <int MODE> struct y3_nf { static constexpr int in = (MODE == Y3_FWD) ? 3 : ((MODE == Y3_INV) ? 2 : 1);
                                   static constexpr int fft = (MODE == Y3_FWD || MODE == Y3_INV) ? 3 : 1; };

// ---------------------------------------------------------------------------
// Column passes (y and z). Grid (ceil(NH/CT), N); CT * T threads, thread
// (lane, c) = threadIdx.x = lane * CT + c owning the lines lane + i T (i < E)
// of column kx0 + c for every field of the pass; the transforms keep their
// first and last stages in registers (fft_regs_multi).
// ---------------------------------------------------------------------------

// y pass: tile of CT kx columns in plane z = blockIdx.y.
template <typename R, int N, int E, int CT, int MODE, bool G3 = false>
__device__ __forceinline__ void k3d_ypass_body(const Params& P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
                                               C_t<R>* __restrict__ W2, const SavScal* __restrict__ sc,
                                               const C_t<R>* __restrict__ tw, C_t<R>* __restrict__ W3 = nullptr) {
  using C = C_t<R>;
  static_assert(!G3 || MODE == Y3_FWD || MODE == Y3_INV, "the phi^4 channel rides on the gradient passes");
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NF = y3_nf<MODE>::fft;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr int SEQ = sp_len(N);
  constexpr bool INV = (MODE == Y3_INV || MODE == Y3_INV_FIELD);
  static_assert((CT * T) % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  if (sc->status != DEV_OK) return;
  const PC<R> pc(P);
  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c;
  const bool col = kx < NH;
  const size_t base = (size_t)blockIdx.y * N * NH + kx;

  // FWD reads U_x, U_y, U_z; INV reads F, G_z and forms (i k~_y F, F, G_z); the field modes one array
  C v[NF][E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int y = lane + i * T;
    const size_t off = base + (size_t)y * NH;
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f][i] = mk<C>(0, 0);
    if (!col) continue;
    if constexpr (MODE == Y3_FWD) {
      v[0][i] = W0[off];
      v[NF - 2][i] = W1[off];
      v[NF - 1][i] = W2[off];
    } else if constexpr (MODE == Y3_INV) {
      const C F = W0[off];
      const R kty = kderiv<R>(y, N, pc.kfy);
      v[0][i] = mk<C>(-kty * F.y, kty * F.x);  // i k~_y F
      v[NF - 2][i] = F;
      v[NF - 1][i] = W1[off];                  // G_z
    } else {
      v[0][i] = W0[off];
    }
  }
  fft_regs_multi<C, N, E, INV, NF, true>(v, sm + c, SEQ * CTP, CTP, lane, tw);
  if (!col) return;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int y = lane + i * T;
    const size_t off = base + (size_t)y * NH;
    if constexpr (MODE == Y3_FWD) {
      const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(y, N, pc.kfy);
      const C a = v[0][i], b = v[NF - 2][i];
      if constexpr (G3) W0[off] = mk<C>(a.x + kty * b.x, a.y + kty * b.y);  // W0 = k~_x W_x + i F_x(gamma3 phi*^3)
      else W0[off] = mk<C>(ktx * a.x + kty * b.x, ktx * a.y + kty * b.y);  // Q1
      W1[off] = v[NF - 1][i];                                              // Q2
    } else if constexpr (MODE == Y3_INV) {
      const R ktx = kderiv<R>(kx, N, pc.kfx);
      const C Fy = v[NF - 2][i];
      if constexpr (G3) W3[off] = Fy;             // Y^-1 F: phi* as an x-spectrum (the row pass forms W_x)
      else W0[off] = mk<C>(-ktx * Fy.y, ktx * Fy.x);  // W_x = i k~_x Y^-1 F
      W1[off] = v[0][i];                          // W_y
      W2[off] = v[NF - 1][i];                     // W_z
    } else {
      W0[off] = v[0][i];
    }
  }
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k3d_ypass(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2,
          const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw) {
  k3d_ypass_body<R, N, E, CT, MODE>(P, W0, W1, W2, sc, tw);
}

// with the phi^4 channel (Y3_INV: W3 instead of W0; Y3_FWD: W0 with k~_x folded in)
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k3d_ypass_g3(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2,
             C_t<R>* __restrict__ W3, const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw) {
  k3d_ypass_body<R, N, E, CT, MODE, true>(P, W0, W1, W2, sc, tw, W3);
}

// z forward pass: tile of CT kx columns at ky = blockIdx.y.
template <typename R, int N, int E, int CT, int MODE, bool G3 = false>
__device__ __forceinline__ void k3d_zfwd_body(const Params& P, Slots<R> S, const C_t<R>* __restrict__ W0,
                                              const C_t<R>* __restrict__ W1, C_t<R>* __restrict__ Nhat,
                                              double* __restrict__ partG, const SavScal* __restrict__ sc,
                                              const C_t<R>* __restrict__ tw, int target) {
  using C = C_t<R>;
  static_assert(!G3 || MODE != Z3F_TO_STATE, "the phi^4 channel is carried by the modes that form N_hat");
  using RD = Red<R>;
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NF = (MODE == Z3F_TO_STATE) ? 1 : 2;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr int SEQ = sp_len(N);
  constexpr size_t PS = (size_t)N * NH;
  static_assert((CT * T) % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ typename RD::acc red3[3][32];
  if (sc->status != DEV_OK) return;
  const PC<R> pc(P);
  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c, ky = blockIdx.y;
  const bool col = kx < NH;
  const size_t base = (size_t)ky * NH + kx;
  C v[NF][E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const size_t off = base + (size_t)(lane + i * T) * PS;
    v[0][i] = col ? W0[off] : mk<C>(0, 0);
    if (NF == 2) v[NF - 1][i] = col ? W1[off] : mk<C>(0, 0);
  }
  if constexpr (MODE == Z3F_TO_STATE) {
    fft_regs_multi<C, N, E, false, NF, true>(v, sm + c, SEQ * CTP, CTP, lane, tw);
    C* dst = S.at(target);
    if (col) {
#pragma unroll
      for (int i = 0; i < E; ++i) dst[base + (size_t)(lane + i * T) * PS] = v[0][i];
    }
  } else {
    const int p = sc->p;
    const C* scur = S.at(p);
    const C* sold = S.at(1 - p);
    const R c0 = (MODE == Z3F_BDF1) ? (R)1 : (R)1.5;
    C vn[E], vo[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {   // issued before the FFT: their latency overlaps it
      vn[i] = vo[i] = mk<C>(0, 0);
      if (MODE != Z3F_NHAT && col) {
        const size_t off = base + (size_t)(lane + i * T) * PS;
        vn[i] = scur[off];
        if (MODE == Z3F_BDF2) vo[i] = sold[off];
      }
    }
    fft_regs_multi<C, N, E, false, NF, true>(v, sm + c, SEQ * CTP, CTP, lane, tw);
    typename RD::acc acc[3] = {RD::zero(), RD::zero(), RD::zero()};
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if (!col) continue;
      const int kz = lane + i * T;
      const size_t off = base + (size_t)kz * PS;
      const C q1 = v[0][i], q2 = v[NF - 1][i];
      const R ktz = kderiv<R>(kz, N, pc.kfz);
      const R ux = q1.x + ktz * q2.x, uy = q1.y + ktz * q2.y;
      // -i (k~_x W_x + k~_y W_y + k~_z W_z); G3: plus the transform of gamma3 phi*^3,
      // whose mean is removed (N_hat_0 := 0)
      const C nh = (G3 && off == 0) ? mk<C>(0, 0) : mk<C>(uy, -ux);
      Nhat[off] = nh;
      if (MODE == Z3F_NHAT) continue;
      const R K2 = sym_K2_3d<R>(kx, ky, kz, N, pc);
      const R invA = sym_invA<R>(K2, c0, pc);
      C vv;
      if (MODE == Z3F_BDF1) vv = vn[i];
      else vv = mk<C>((R)2 * vn[i].x - (R)0.5 * vo[i].x, (R)2 * vn[i].y - (R)0.5 * vo[i].y);
      const R w = (kx == 0 || kx == N / 2) ? (R)1 : (R)2;
      const R n2 = nh.x * nh.x + nh.y * nh.y;
      const R nv = nh.x * vv.x + nh.y * vv.y;
      const R sK = rn_mul(pc.sdt, K2);  // stabiliser (Sec. 5.2): in eta, not in theta
      const R nvs = nh.x * rn_fma(sK, vn[i].x, vv.x) + nh.y * rn_fma(sK, vn[i].y, vv.y);
      acc[0] = RD::add(acc[0], w * (-K2 * invA) * n2);
      acc[1] = RD::add(acc[1], w * nvs * invA);
      acc[2] = RD::add(acc[2], w * nv);
    }
    if constexpr (MODE != Z3F_NHAT) {
      block_red_multi<R, 3>(acc, red3);
      if (threadIdx.x == 0) {
        const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
        partG[b] = RD::to_double(acc[0]);
        partG[nb + b] = RD::to_double(acc[1]);
        partG[2 * nb + b] = RD::to_double(acc[2]);
      }
    }
  }
}

template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k3d_zfwd(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, const C_t<R>* __restrict__ W1,
         C_t<R>* __restrict__ Nhat, double* __restrict__ partG, const SavScal* __restrict__ sc,
         const C_t<R>* __restrict__ tw, int target) {
  k3d_zfwd_body<R, N, E, CT, MODE>(P, S, W0, W1, Nhat, partG, sc, tw, target);
}

// with the phi^4 channel (N_hat_0 := 0)
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k3d_zfwd_g3(const Params P, Slots<R> S, const C_t<R>* __restrict__ W0, const C_t<R>* __restrict__ W1,
            C_t<R>* __restrict__ Nhat, double* __restrict__ partG, const SavScal* __restrict__ sc,
            const C_t<R>* __restrict__ tw) {
  k3d_zfwd_body<R, N, E, CT, MODE, true>(P, S, W0, W1, Nhat, partG, sc, tw, 0);
}

// Reduce the E_1 and gamma/eta/theta partial sums and solve the scalar
// system; the update is then applied by the z-inverse pass into slot
// 1 - p_old, so p flips here. The sums are float64 (several thousand
// partials per array), spread over the grid: block b sums a fixed contiguous
// chunk of each array, and the last block to arrive (an arrival counter that
// it resets) sums the chunk sums and solves. Fixed order, so deterministic.
constexpr int kScalarBlocks = 64;

template <typename R>
__global__ void __launch_bounds__(256)
k3d_scalar(const Params P, SavScal* __restrict__ sc, const double* __restrict__ partE, int nE,
           const double* __restrict__ partG, int nG, int bdf1, double* __restrict__ chunk,
           unsigned* __restrict__ counter) {
  __shared__ double red5[5][32];
  __shared__ double qres[5];
  __shared__ bool am_last;
  if (sc->status != DEV_OK) return;
  const int nb = gridDim.x, b = blockIdx.x;
  const int cE = (nE + nb - 1) / nb, cG = (nG + nb - 1) / nb;
  const int e0 = min(b * cE, nE), g0 = min(b * cG, nG);
  const int ne = min(cE, nE - e0), ng = min(cG, nG - g0);
  {
    const double* arr[5] = {partE + e0, partE + nE + e0, partG + g0, partG + nG + g0, partG + 2 * nG + g0};
    const int cnt[5] = {ne, ne, ng, ng, ng};
    block_sum_arrays<5>(arr, cnt, qres, red5);
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) chunk[q * nb + b] = qres[q];
    __threadfence();
    am_last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  {
    const double* arr[5] = {chunk, chunk + nb, chunk + 2 * nb, chunk + 3 * nb, chunk + 4 * nb};
    const int cnt[5] = {nb, nb, nb, nb, nb};
    block_sum_arrays<5>(arr, cnt, qres, red5);
  }
  if (threadIdx.x == 0) {
    const SolveOut o = sav_solve(P, qres, bdf1 != 0, RIn(sc));
    sav_commit(sc, o, 1 - sc->p, PEND_NONE);
    *counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// z inverse pass: tile of CT kx columns at ky = blockIdx.y (thread layout as above).
// STEP: after k3d_scalar (p already points at the slot being written):
//   phi^{n+1} -> slot p, phi* = 2 phi^{n+1} - phi^n; PREP: phi* = 2 S[p] - S[1-p];
//   GRAD: phi* = S[p] (which 0) or S[1-p]; FIELD: one output, the field itself.
// Outputs: W0 = Z^-1 phi*, W1 = Z^-1 (i k~_z phi*).
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int CT, int MODE>
__global__ void __launch_bounds__(CT * (N / E))
k3d_zinv(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, C_t<R>* __restrict__ W0,
         C_t<R>* __restrict__ W1, SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw, int which) {
  using C = C_t<R>;
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NF = (MODE == Z3I_FIELD) ? 1 : 2;
  constexpr int CTP = col_pitch(CT);
  constexpr int NH = N / 2 + 1;
  constexpr int SEQ = sp_len(N);
  constexpr size_t PS = (size_t)N * NH;
  constexpr bool STEP = (MODE == Z3I_STEP || MODE == Z3I_STEP_BDF1);
  static_assert((CT * T) % 32 == 0, "tile must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  if (sc->status != DEV_OK) return;
  const PC<R> pc(P);
  const int lane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c, ky = blockIdx.y;
  const bool col = kx < NH;
  const size_t base = (size_t)ky * NH + kx;
  const int p = sc->p;
  C* A;  // STEP: phi^n; PREP: S[p]; GRAD/FIELD: the chosen slot
  C* B;  // STEP: the slot receiving phi^{n+1} (holds phi^{n-1}); PREP: S[1-p]
  if (STEP) { A = S.at(1 - p); B = S.at(p); }
  else if (MODE == Z3I_PREP) { A = S.at(p); B = S.at(1 - p); }
  else { A = S.at(which == 0 ? p : 1 - p); B = A; }
  const R al = read_alpha<R>(sc);
  C va[E], vb[E], vn[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    va[i] = vb[i] = vn[i] = mk<C>(0, 0);
    if (col) {
      const size_t off = base + (size_t)(lane + i * T) * PS;
      va[i] = A[off];
      if (STEP || MODE == Z3I_PREP) vb[i] = B[off];
      if (STEP) vn[i] = Nhat[off];
    }
  }
  C g[NF][E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int kz = lane + i * T;
    C g0 = mk<C>(0, 0), g1 = mk<C>(0, 0);
    if (col) {
      const size_t off = base + (size_t)kz * PS;
      C ph;
      if (STEP) {
        const C cur = va[i];
        C nw;
        if (off == 0) {
          const double z = (MODE == Z3I_STEP_BDF1) ? sc->zm[1 - p] : zero_mode_update(sc->zm[1 - p], sc->zm[p]);
          sc->zm[p] = z;
          nw = mk<C>((R)z, (R)0);
        } else {
          const R K2 = sym_K2_3d<R>(kx, ky, kz, N, pc);
          if (MODE == Z3I_STEP_BDF1)
            nw = bdf1_update<C, R>(cur, vn[i], K2, sym_invA<R>(K2, (R)1, pc), al, rn_mul(pc.sdt, K2));
          else
            nw = bdf2_update<C, R>(cur, vb[i], vn[i], K2, sym_invA<R>(K2, (R)1.5, pc), al, rn_mul(pc.sdt, K2));
        }
        B[off] = nw;
        ph = mk<C>((R)2 * nw.x - cur.x, (R)2 * nw.y - cur.y);
      } else if (MODE == Z3I_PREP) {
        ph = mk<C>((R)2 * va[i].x - vb[i].x, (R)2 * va[i].y - vb[i].y);
      } else {
        ph = va[i];
      }
      g0 = ph;
      const R ktz = kderiv<R>(kz, N, pc.kfz);
      g1 = mk<C>(-ktz * ph.y, ktz * ph.x);
    }
    g[0][i] = g0;
    if (NF == 2) g[NF - 1][i] = g1;
  }
  fft_regs_multi<C, N, E, true, NF, true>(g, sm + c, SEQ * CTP, CTP, lane, tw);
  if (col) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const size_t off = base + (size_t)(lane + i * T) * PS;
      W0[off] = g[0][i];
      if (NF == 2) W1[off] = g[NF - 1][i];
    }
  }
}

// ---------------------------------------------------------------------------
// x row pass over pairs of rows (flat row index z*N + y; N even, so a pair
// shares z). Grid: N*N/(2*RP) blocks of RP row pairs.
// NONLIN / ENERGY: three sequences per pair, all held by the pair's lanes:
// G_x + i G_y of each row and G_z(row 0) + i G_z(row 1), with the first and
// last FFT stages in registers. IN_REAL / OUT_REAL: one sequence per pair,
// f(row 0) + i f(row 1). T lanes per pair.
// part: 2 x gridDim.x accumulators (sum s^2, sum s).
// ---------------------------------------------------------------------------
template <typename R, int N, int E, int RP, int MODE, bool G3 = false>
__device__ __forceinline__ void k3d_row_body(const Params& P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
                                             C_t<R>* __restrict__ W2, double* __restrict__ part,
                                             const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw,
                                             double* __restrict__ real_io, C_t<R>* __restrict__ W3 = nullptr) {
  using C = C_t<R>;
  using RD = Red<R>;
  constexpr int T = fft_shape<N, E>::T;
  constexpr int NS = (MODE == RW_NONLIN || MODE == RW_ENERGY) ? (G3 ? 4 : 3) : 1;
  static_assert(!G3 || MODE == RW_NONLIN || MODE == RW_ENERGY, "the phi^4 channel is carried by the nonlinear and energy modes");
  constexpr int NTH = RP * T;
  constexpr int NH = N / 2 + 1;
  constexpr int KH = (N / 2) / T;
  constexpr int SEQ = sp_len(N);
  static_assert(NTH % 32 == 0 && KH * T == N / 2, "rows must fill whole warps");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  __shared__ typename RD::acc red2[2][32];
  if (sc->status != DEV_OK) return;
  const int pl = threadIdx.x / T, lane = threadIdx.x % T;   // local pair, lane
  const size_t row0 = 2 * ((size_t)blockIdx.x * RP + pl);
  C* z = sm + pl * NS * (SEQ + 1);                         // the pair's NS sequences

  if constexpr (MODE == RW_IN_REAL) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = lane + i * T;
      z[spr(x)] = mk<C>((R)real_io[row0 * N + x], (R)real_io[(row0 + 1) * N + x]);
    }
    __syncthreads();
    fft_smem<C, N, E, false>(z, 1, lane, tw);
    const R h = (R)0.5 * PC<R>(P).invP;
#pragma unroll
    for (int i = 0; i < KH + 1; ++i) {
      if (i == KH && lane != 0) break;
      const int k = (i == KH) ? N / 2 : lane + i * T;
      const C zk = z[spr(k)], zm = cconj(z[spr((N - k) & (N - 1))]);
      const C a = cadd(zk, zm), b = csub(zk, zm);
      W0[row0 * NH + k] = cscale(a, h);
      W0[(row0 + 1) * NH + k] = mk<C>(b.y * h, -b.x * h);
    }
  } else if constexpr (MODE == RW_OUT_REAL) {
    C a[KH], b[KH];
#pragma unroll
    for (int i = 0; i < KH; ++i) {
      a[i] = W0[row0 * NH + lane + i * T];
      b[i] = W0[(row0 + 1) * NH + lane + i * T];
    }
    const C an = W0[row0 * NH + N / 2], bn = W0[(row0 + 1) * NH + N / 2];
#pragma unroll
    for (int i = 0; i < KH; ++i) {
      const int k = lane + i * T;
      z[spr(k)] = mk<C>(a[i].x - b[i].y, a[i].y + b[i].x);
      if (k > 0) z[spr(N - k)] = mk<C>(a[i].x + b[i].y, b[i].x - a[i].y);
    }
    if (lane == 0) z[spr(N / 2)] = mk<C>(an.x - bn.y, an.y + bn.x);
    __syncthreads();
    fft_smem<C, N, E, true>(z, 1, lane, tw);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int x = lane + i * T;
      real_io[row0 * N + x] = (double)z[spr(x)].x;
      real_io[(row0 + 1) * N + x] = (double)z[spr(x)].y;
    }
  } else {
    // Z_q = A_q + i B_q over the full x-spectrum, element k = lane + i T
    // straight into registers (k > N/2 from the Hermitian mirror N - k):
    // q = 0/1: G_x + i G_y of row 0/1, q = 2: G_z(row 0) + i G_z(row 1),
    // q = 3 (G3): phi*(row 0) + i phi*(row 1); G3 forms G_x = i k~_x phi* from W3
    const PC<R> pc(P);
    C v[NS][E];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const C* Aa = (q == 3) ? W3 : ((q == 2) ? W2 : W0);
      const C* Bb = (q == 3) ? W3 : ((q == 2) ? W2 : W1);
      const size_t ra = row0 + (q == 1 ? 1 : 0);
      const size_t rb = (q >= 2) ? row0 + 1 : ra;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = lane + i * T;
        const bool direct = k <= N / 2;
        const int m = direct ? k : N - k;
        C a;
        if (G3 && q < 2) {
          const C f = W3[ra * NH + m];
          const R ktm = kderiv<R>(m, N, pc.kfx);
          a = mk<C>(-ktm * f.y, ktm * f.x);
        } else {
          a = Aa[ra * NH + m];
        }
        const C b = Bb[rb * NH + m];
        v[q][i] = direct ? mk<C>(a.x - b.y, a.y + b.x) : mk<C>(a.x + b.y, b.x - a.y);
      }
    }
    fft_regs_multi<C, N, E, true, NS, false>(v, z, SEQ + 1, 1, lane, tw);
    // pointwise on x = lane + i T for both rows of the pair
    typename RD::acc acc[2] = {RD::zero(), RD::zero()};
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const C g0 = v[0][i], g1 = v[1][i], gz = v[2][i];
      const R s0 = g0.x * g0.x + g0.y * g0.y + gz.x * gz.x;
      const R s1 = g1.x * g1.x + g1.y * g1.y + gz.y * gz.y;
      if constexpr (G3) {  // (gamma3/beta) phi*^4 joins the sum of s^2 (E_1 takes it with beta/4)
        const C ph = v[NS - 1][i];
        const R q0 = ph.x * ph.x, q1 = ph.y * ph.y;
        acc[0] = RD::add(acc[0], s0 * s0 + pc.g3b * (q0 * q0));
        acc[1] = RD::add(acc[1], s0);
        acc[0] = RD::add(acc[0], s1 * s1 + pc.g3b * (q1 * q1));
        acc[1] = RD::add(acc[1], s1);
        if (MODE == RW_NONLIN) v[NS - 1][i] = mk<C>(pc.g3 * q0 * ph.x, pc.g3 * q1 * ph.y);
      } else {
        acc[0] = RD::add(acc[0], s0 * s0);
        acc[1] = RD::add(acc[1], s0);
        acc[0] = RD::add(acc[0], s1 * s1);
        acc[1] = RD::add(acc[1], s1);
      }
      if (MODE == RW_NONLIN) {
        const R f0 = pc.beta * s0 - (R)2, f1 = pc.beta * s1 - (R)2;
        v[0][i] = mk<C>(f0 * g0.x, f0 * g0.y);
        v[1][i] = mk<C>(f1 * g1.x, f1 * g1.y);
        v[2][i] = mk<C>(f0 * gz.x, f1 * gz.y);
      }
    }
    if constexpr (MODE == RW_NONLIN) {
      fft_regs_multi<C, N, E, false, NS, false>(v, z, SEQ + 1, 1, lane, tw);
      // the split into the two signals of each sequence pairs k with N - k: one exchange
      fft_sync<N, E>();
#pragma unroll
      for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int i = 0; i < E; ++i) z[q * (SEQ + 1) + spr(lane + i * T)] = v[q][i];
      fft_sync<N, E>();
      const R h = (R)0.5 * pc.invP;
      if constexpr (G3) {
        // W0 = k~_x W_x + i F_x(gamma3 phi*^3) for both rows, W1 = W_y, W2 = W_z
#pragma unroll
        for (int i = 0; i < KH + 1; ++i) {
          if (i == KH && lane != 0) break;
          const int k = lane + i * T;  // i == KH: the Nyquist entry N/2 (lane 0)
          const int km = spr((N - k) & (N - 1));
          C sx[NS], dy[NS];
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            const C zk = v[q][i], zm = cconj(z[q * (SEQ + 1) + km]);
            sx[q] = cadd(zk, zm);
            dy[q] = csub(zk, zm);
          }
          const R ktk = kderiv<R>(k, N, pc.kfx);
          const C f0 = cscale(sx[3], h), f1 = mk<C>(dy[3].y * h, -dy[3].x * h);  // gamma3 phi*^3 of rows 0, 1
          W0[row0 * NH + k] = mk<C>(ktk * sx[0].x * h - f0.y, ktk * sx[0].y * h + f0.x);
          W1[row0 * NH + k] = mk<C>(dy[0].y * h, -dy[0].x * h);
          W0[(row0 + 1) * NH + k] = mk<C>(ktk * sx[1].x * h - f1.y, ktk * sx[1].y * h + f1.x);
          W1[(row0 + 1) * NH + k] = mk<C>(dy[1].y * h, -dy[1].x * h);
          W2[row0 * NH + k] = cscale(sx[2], h);
          W2[(row0 + 1) * NH + k] = mk<C>(dy[2].y * h, -dy[2].x * h);
        }
      } else {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          C* Oa = (q == 2) ? W2 : W0;
          C* Ob = (q == 2) ? W2 : W1;
          const size_t ra = row0 + (q == 1 ? 1 : 0);
          const size_t rb = (q == 2) ? row0 + 1 : ra;
#pragma unroll
          for (int i = 0; i < KH + 1; ++i) {
            if (i == KH && lane != 0) break;
            const int k = lane + i * T;  // i == KH: the Nyquist entry N/2 (lane 0)
            const C zk = v[q][i], zm = cconj(z[q * (SEQ + 1) + spr((N - k) & (N - 1))]);
            const C sx = cadd(zk, zm), dy = csub(zk, zm);
            Oa[ra * NH + k] = cscale(sx, h);
            Ob[rb * NH + k] = mk<C>(dy.y * h, -dy.x * h);
          }
        }
      }
    }
    block_red_multi<R, 2>(acc, red2);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = RD::to_double(acc[0]);
      part[gridDim.x + blockIdx.x] = RD::to_double(acc[1]);
    }
  }
}

template <typename R, int N, int E, int RP, int MODE>
__global__ void __launch_bounds__(RP * (N / E))
k3d_row(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2,
        double* __restrict__ part, const SavScal* __restrict__ sc, const C_t<R>* __restrict__ tw,
        double* __restrict__ real_io) {
  k3d_row_body<R, N, E, RP, MODE>(P, W0, W1, W2, part, sc, tw, real_io);
}

// with the phi^4 channel (W3: phi* as an x-spectrum in; W0 out: k~_x W_x + i F_x(gamma3 phi*^3))
template <typename R, int N, int E, int RP, int MODE>
__global__ void __launch_bounds__(RP * (N / E))
k3d_row_g3(const Params P, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1, C_t<R>* __restrict__ W2,
           C_t<R>* __restrict__ W3, double* __restrict__ part, const SavScal* __restrict__ sc,
           const C_t<R>* __restrict__ tw) {
  k3d_row_body<R, N, E, RP, MODE, true>(P, W0, W1, W2, part, sc, tw, nullptr, W3);
}

// ---------------------------------------------------------------------------
// Pointwise 3D kernels over the half spectrum (grid-stride)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void idx3(size_t off, int N, int NH, int& kx, int& ky, int& kz) {
  kx = (int)(off % NH);
  const size_t r = off / NH;
  ky = (int)(r % N);
  kz = (int)(r / N);
}

// Ghost point (eq. scheme-SAV-initial-1): slot 1-p = phi^0 + dt |k|^2 (N_hat + (a + |k|^4) phi^0).
template <typename R>
__global__ void k3d_ghost(const Params P, Slots<R> S, const C_t<R>* __restrict__ Nhat, SavScal* sc) {
  using C = C_t<R>;
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const C* cur = S.at(p);
  C* dst = S.at(1 - p);
  const PC<R> pc(P);
  const size_t total = (size_t)N * N * NH;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    int kx, ky, kz;
    idx3(off, N, NH, kx, ky, kz);
    const R K2 = sym_K2_3d<R>(kx, ky, kz, N, pc);
    const C cu = cur[off], nh = Nhat[off];
    const R L = pc.a + K2 * K2;
    const R f = pc.dt * K2;
    dst[off] = mk<C>(cu.x + f * (nh.x + L * cu.x), cu.y + f * (nh.y + L * cu.y));
    if (off == 0) sc->zm[1 - p] = sc->zm[p];
  }
}

// Spectral norms of phi = slot p and psi = 2 phi - slot (1-p), zero mode excluded.
template <typename R>
__global__ void k3d_norms(const Params P, Slots<R> S, const SavScal* sc, double* part) {
  using C = C_t<R>;
  __shared__ double red[32];
  const int N = P.N, NH = P.NH;
  const int p = sc->p;
  const C* nw = S.at(p);
  const C* ol = S.at(1 - p);
  const size_t total = (size_t)N * N * NH;
  double a0 = 0, a1 = 0, a2 = 0;
  for (size_t off = blockIdx.x * (size_t)blockDim.x + threadIdx.x; off < total;
       off += (size_t)gridDim.x * blockDim.x) {
    if (off == 0) continue;
    int kx, ky, kz;
    idx3(off, N, NH, kx, ky, kz);
    const double kxx = kx * P.kf[0], kyy = kfull<double>(ky, N, P.kf[1]), kzz = kfull<double>(kz, N, P.kf[2]);
    const double K2 = kxx * kxx + kyy * kyy + kzz * kzz;
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

}  // namespace spfc
