// Persistent 2D step: every BDF2-SAV step of a launch (Sec. 2.3, eqs.
// solver-1 .. solver-6) in one cooperative kernel whose blocks stay resident
// and meet at bounded grid barriers.
//
// On entry W0, W1 hold the inverse y-transforms of i k~_x phi* and i k~_y phi*,
// phi* = 2 phi^n - phi^{n-1} (prepared by the previous launch or by the
// column-inverse pass), the state (phi^n in slot p, phi^{n-1} in slot 1-p)
// and r^n, r^{n-1} are committed. Per step:
//   B (rows)    inverse x-DFT of G_x + i G_y, s = |grad phi*|^2, the E_1
//               partial sums, w = (beta s - 2) grad phi*, forward x-DFT, split
//               into W_x, W_y; rows stay in the block that owns them.
//   barrier
//   C (columns) forward y-DFT of W, N_hat = -i k~ . W_hat (kept in registers
//               with A^{-1} of every mode), partial sums of gamma, eta, theta;
//               the E_1 partial sums of all blocks are loaded before the
//               transform and summed in the same block reduction.
//   barrier
//   D           every block loads the gamma/eta/theta partials; while they
//               arrive thread 0 forms E_1, sqrt(E_1) and the coefficients of
//               the scalar solve; then every block sums them in the same fixed
//               order and finishes the solve in float64 (block 0 commits the
//               record); phi^{n+1} = alpha A^{-1} Delta N_hat + A^{-1} v over
//               phi^{n-1}, the next phi*, its gradients and their inverse
//               y-DFT into W.
//   barrier (only between the steps of one launch)
// A block owns the same CT kx columns in C and D of every step, so the state
// of its columns is read from global memory once per launch (staged into
// shared memory with asynchronous copies issued at entry, while the row pass
// runs) and carried in shared memory from step to step; phi^{n+1} is written
// back every step. The twiddle table is copied to shared memory at entry.
// Loads of data that other blocks wrote in this launch bypass L1 (ld.cg).
#pragma once

#include "spfc_kernels2d.cuh"

namespace spfc {

// Launch shape of the persistent step for an N x N grid: E = 8 values per FFT
// lane, T = N/E lanes per sequence; CT columns per block (at least a warp of
// threads), G = ceil((N/2+1)/CT) blocks; in the row pass each group of T
// lanes takes NSR rows at once (2 in float32; 1 in float64, for registers),
// the block RPB rows in NRR rounds.
template <typename R, int N, int EV = 8> struct PShape {
  static constexpr int E = EV;
  static constexpr int T = N / E;
  static constexpr int CT = (32 / T > 2) ? 32 / T : 2;
  static constexpr int NT = CT * T;
  static constexpr int NH = N / 2 + 1;
  static constexpr int G = (NH + CT - 1) / CT;
  static constexpr int NSR = (sizeof(R) == 8) ? 1 : 2;
  static constexpr int RPR = CT * NSR;
  static constexpr int RPB = ((N + G - 1) / G + RPR - 1) / RPR * RPR;
  static constexpr int NRR = RPB / RPR;
  static constexpr int SEQ = sp_len(N);
  static constexpr int CTP = col_pitch(CT);  // column pitch of the column-pass scratch
  // dynamic shared memory, in complex entries: twiddles, state staging
  // [2][N][CT], FFT scratch (the larger of the column and the row pass)
  // the twiddle entries its transforms read (rows and columns: one length)
  static constexpr int TW_LO = tw_lo(N, E), TW_HI = tw_hi(N, E);
  static constexpr int SM_TW = TW_HI - TW_LO;
  static constexpr int SM_ST = 2 * N * CT;
  static constexpr int SM_COL = 2 * SEQ * CTP;
  static constexpr int SM_ROW = CT * NSR * (SEQ + 1);
  static constexpr int SM_FFT = SM_COL > SM_ROW ? SM_COL : SM_ROW;
  static constexpr size_t smem_bytes() { return (size_t)(SM_TW + SM_ST + SM_FFT) * sizeof(C_t<R>); }
  static_assert(NT % 32 == 0, "a block fills whole warps");
  static_assert(G * RPB >= N, "the row rounds cover every row");
};

// Asynchronous global -> shared copies (cp.async, 8 or 16 bytes): the data
// lands in shared memory without passing through registers.
template <typename C> __device__ __forceinline__ void cp_async(C* dst_smem, const C* src_gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(C) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src_gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Grid barrier (all blocks co-resident: cooperative launch), in the usual
// release/acquire form: a block barrier, one release-add of thread 0 on a
// monotone 64-bit arrival counter (the release publishes the block's prior
// writes, which the block barrier ordered before it), acquire polls until the
// counter reaches `target`, a block barrier. The host passes each launch the
// counter's value at its start (it knows every launch's barrier count), so
// no arrival needs to read the counter back. The wait is bounded: on expiry
// it latches DEV_TIMEOUT and every thread of the block gets false.
constexpr long long kPollLimit = 1ll << 21;  // polls of at least one L2 round trip each: ~1-2 s

__device__ __forceinline__ bool wait_counter_acquire(const unsigned long long* ctr, unsigned long long target,
                                                     long long limit) {
  unsigned long long v;
  for (long long it = 0; it <= limit; ++it) {
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
  }
  return false;
}

__device__ __forceinline__ bool grid_sync(unsigned long long* ctr, unsigned long long target, SavScal* sc,
                                          int* flag_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(ctr), "l"(1ull) : "memory");
    const bool ok = wait_counter_acquire(ctr, target, kPollLimit);
    if (!ok) atomicExch(&sc->status, (int)DEV_TIMEOUT);
    *flag_smem = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag_smem != 0;
}

// Partial sums of the other blocks, loaded for a later block sum: entries
// threadIdx.x and threadIdx.x + blockDim.x of each of the NQ arrays (n <= 2
// blockDim.x entries each; L1 bypassed).
template <int NQ>
__device__ __forceinline__ void load_partials(const double* base, int n, double (*v)[NQ]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = threadIdx.x + u * blockDim.x;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[u][q] = (i < n) ? __ldcg(base + (size_t)q * n + i) : 0.0;
  }
}

// One block reduction (fixed order, results in thread 0) of three
// accumulators of precision R and ND float64 sums: shuffle trees within the
// warps, then one warp over the warps' results.
template <typename R, int ND>
__device__ __forceinline__ void block_red_mixed(typename Red<R>::acc* a, double* d,
                                                typename Red<R>::acc (*sa)[32], double (*sd)[32]) {
  using RD = Red<R>;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = RD::add2(a[k], RD::shfl(a[k], o));
#pragma unroll
    for (int k = 0; k < ND; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sa[k][wid] = a[k];
#pragma unroll
    for (int k = 0; k < ND; ++k) sd[k][wid] = d[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = (lane < nw) ? sa[k][lane] : RD::zero();
#pragma unroll
    for (int k = 0; k < ND; ++k) d[k] = (lane < nw) ? sd[k][lane] : 0.0;
    const int p2 = pow2_ceil(nw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= p2) continue;
#pragma unroll
      for (int k = 0; k < 3; ++k) a[k] = RD::add2(a[k], RD::shfl(a[k], o));
#pragma unroll
      for (int k = 0; k < ND; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
    }
  }
}

// Block sum (fixed order, result in thread 0) of NQ float64 values per thread.
template <int NQ>
__device__ __forceinline__ void block_sum_values(double* d, double (*sd)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NQ; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) sd[k][wid] = d[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) d[k] = (lane < nw) ? sd[k][lane] : 0.0;
    const int p2 = pow2_ceil(nw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= p2) continue;
#pragma unroll
      for (int k = 0; k < NQ; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
    }
  }
}

template <typename R, int N, int EV>
__global__ void __launch_bounds__(PShape<R, N, EV>::NT)
k2d_step_persist(const Params P, Slots<R> S, C_t<R>* __restrict__ W0, C_t<R>* __restrict__ W1,
                 double* __restrict__ partE, double* __restrict__ partG, SavScal* __restrict__ sc,
                 unsigned long long* __restrict__ sync64, unsigned long long bar_base,
                 const C_t<R>* __restrict__ tw_g, int nsteps) {
  using C = C_t<R>;
  using RD = Red<R>;
  using SH = PShape<R, N, EV>;
  constexpr int E = SH::E, T = SH::T, CT = SH::CT, NH = SH::NH, SEQ = SH::SEQ, CTP = SH::CTP;
  constexpr int NSR = SH::NSR, RPR = SH::RPR, RPB = SH::RPB, NRR = SH::NRR;
  constexpr int KH = (N / 2) / T;  // half-spectrum entries per lane in the row split, Nyquist aside
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw_s = reinterpret_cast<C*>(smraw);
  C* st_s = tw_s + SH::SM_TW;      // [2][N][CT]: phi^n, phi^{n-1} of this block's columns
  C* fft_s = st_s + SH::SM_ST;
  static_assert(SH::G <= 2 * SH::NT, "two partial sums per thread cover the grid");
  __shared__ typename RD::acc redb[3][32];
  __shared__ double redd[3][32];
  __shared__ R alpha_s;
  __shared__ int flag_s, ok_s;

  const int G = gridDim.x;
  const PC<R> pc(P);
  // column ownership (passes C and D)
  const int clane = threadIdx.x / CT, c = threadIdx.x % CT;
  const int kx = blockIdx.x * CT + c;
  const bool col = kx < NH;
  // row ownership (pass B)
  const int rg = threadIdx.x / T, rlane = threadIdx.x % T;
  C* zrow = fft_s + rg * NSR * (SEQ + 1);

  // Z = G_x + i G_y of the rows of round rr over the full x-spectrum
  // (Hermitian mirror for k > N/2), from W_x, W_y
  C v[NSR][E];
  int row[NSR];
  auto load_rows = [&](int rr) {
#pragma unroll
    for (int q = 0; q < NSR; ++q) {
      row[q] = blockIdx.x * RPB + rr * RPR + rg * NSR + q;
      const bool ok = row[q] < N;
      const size_t roff = (size_t)(ok ? row[q] : 0) * NH;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = rlane + i * T;
        const bool direct = k <= N / 2;
        const size_t off = roff + (direct ? k : N - k);
        C a = mk<C>(0, 0), b = mk<C>(0, 0);
        if (ok) { a = __ldcg(W0 + off); b = __ldcg(W1 + off); }
        v[q][i] = direct ? mk<C>(a.x - b.y, a.y + b.x) : mk<C>(a.x + b.y, b.x - a.y);
      }
    }
  };

  // Entry: the twiddle copies and the first rows' loads need no field of the
  // record, so they are in flight before the record is read.
  for (int m = threadIdx.x; m < SH::SM_TW; m += blockDim.x) cp_async(tw_s + m, tw_g + SH::TW_LO + m);
  cp_async_commit();
  load_rows(0);
  if (sc->status != DEV_OK) {
    cp_async_wait<0>();  // no copy may still be landing when the block leaves
    return;
  }
  int p = sc->p;
  unsigned long long bar = bar_base;     // arrival count of the last completed barrier round
  RIn rin(sc);                           // r^n, r^{n-1} (float64), carried by thread 0
  double qE[2] = {0.0, 0.0};             // the E_1 sums (thread 0)
  double zm_n = 0.0, zm_o = 0.0;          // float64 zero modes (thread 0 of block 0)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    zm_n = sc->zm[p];
    zm_o = sc->zm[1 - p];
  }
  // this block's state columns into shared memory
  {
    const C* sn = S.at(p);
    const C* so = S.at(1 - p);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int ky = clane + i * T;
      if (col) {
        const size_t off = (size_t)ky * NH + kx;
        cp_async(st_s + ky * CT + c, sn + off);
        cp_async(st_s + (N + ky) * CT + c, so + off);
      }
    }
  }
  cp_async_commit();

  for (int step = 0; step < nsteps; ++step) {
    // ---------------- B: row pass ----------------
    typename RD::acc acc2 = RD::zero(), acc1 = RD::zero();
#pragma unroll 1
    for (int rr = 0; rr < NRR; ++rr) {
      if (step > 0 || rr > 0) load_rows(rr);
      if (step == 0 && rr == 0) {
        cp_async_wait<1>();  // the twiddle group (the state may still be in flight)
        __syncthreads();
      }
      fft_regs_multi<C, N, E, true, NSR, false, TwSharedFrom<SH::TW_LO>>(v, zrow, SEQ + 1, 1, rlane, tw_s);
      const R beta = pc.beta;
#pragma unroll
      for (int q = 0; q < NSR; ++q) {
        const bool ok = row[q] < N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const C g = v[q][i];
          const R s = g.x * g.x + g.y * g.y;
          if (ok) {
            acc2 = RD::add(acc2, s * s);
            acc1 = RD::add(acc1, s);
          }
          const R fac = beta * s - (R)2;
          v[q][i] = mk<C>(fac * g.x, fac * g.y);
        }
      }
      fft_regs_multi<C, N, E, false, NSR, false, TwSharedFrom<SH::TW_LO>>(v, zrow, SEQ + 1, 1, rlane, tw_s);
      // the split into W_x, W_y pairs k with N - k: one exchange
      fft_sync<N, E>();
#pragma unroll
      for (int q = 0; q < NSR; ++q)
#pragma unroll
        for (int i = 0; i < E; ++i) zrow[q * (SEQ + 1) + spr(rlane + i * T)] = v[q][i];
      fft_sync<N, E>();
      const R half = (R)0.5 * pc.invP;
#pragma unroll
      for (int q = 0; q < NSR; ++q) {
        if (row[q] >= N) continue;
        const size_t roff = (size_t)row[q] * NH;
#pragma unroll
        for (int i = 0; i < KH + 1; ++i) {
          if (i == KH && rlane != 0) break;
          const int kk = rlane + i * T;  // i == KH: the Nyquist entry N/2 (lane 0)
          const C zk = v[q][i], zm = cconj(zrow[q * (SEQ + 1) + spr((N - kk) & (N - 1))]);
          const C sx = cadd(zk, zm), dy = csub(zk, zm);
          W0[roff + kk] = cscale(sx, half);                  // W_x = (Z_k + conj Z_{N-k}) / 2
          W1[roff + kk] = mk<C>(dy.y * half, -dy.x * half);  // W_y = (Z_k - conj Z_{N-k}) / (2i)
        }
      }
      if (NRR > 1) fft_sync<N, E>();  // zrow is reused by the next round
    }
    {
      typename RD::acc t21[2] = {acc2, acc1};
      block_red_multi<R, 2>(t21, redb);
      if (threadIdx.x == 0) {
        partE[blockIdx.x] = RD::to_double(t21[0]);
        partE[G + blockIdx.x] = RD::to_double(t21[1]);
      }
    }
    bar += G;
    if (!grid_sync(sync64, bar, sc, &flag_s)) {
      cp_async_wait<0>();  // no copy may still be landing when the block leaves
      return;
    }

    // ---------------- C: forward column pass and partial sums ----------------
    C g[2][E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      g[0][i] = g[1][i] = mk<C>(0, 0);
      if (col) {
        const size_t off = (size_t)(clane + i * T) * NH + kx;
        g[0][i] = __ldcg(W0 + off);
        g[1][i] = __ldcg(W1 + off);
      }
    }
    double pe[2][2];  // the E_1 partial sums of all blocks: loaded now, summed after the transform
    load_partials<2>(partE, G, pe);
    fft_regs_multi<C, N, E, false, 2, true, TwSharedFrom<SH::TW_LO>>(g, fft_s + c, SEQ * CTP, CTP, clane, tw_s);
    if (step == 0) cp_async_wait<0>();  // this thread's state copies have landed
    C nh[E];
    R ia[E];
    typename RD::acc ag = RD::zero(), ae = RD::zero(), at = RD::zero();
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int ky = clane + i * T;
      nh[i] = mk<C>(0, 0);
      ia[i] = (R)0;
      if (!col) continue;
      const C vn = st_s[ky * CT + c], vo = st_s[(N + ky) * CT + c];
      const C wx = g[0][i], wy = g[1][i];
      const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
      const R ux = ktx * wx.x + kty * wy.x, uy = ktx * wx.y + kty * wy.y;
      nh[i] = mk<C>(uy, -ux);  // N_hat = -i (k~_x W_x + k~_y W_y)
      const R K2 = sym_K2<R>(kx, ky, N, pc);
      const R invA = sym_invA<R>(K2, (R)1.5, pc);
      ia[i] = invA;
      const C v = mk<C>((R)2 * vn.x - (R)0.5 * vo.x, (R)2 * vn.y - (R)0.5 * vo.y);
      const R w = (kx == 0 || kx == N / 2) ? (R)1 : (R)2;  // half-spectrum Parseval weight
      const R n2 = nh[i].x * nh[i].x + nh[i].y * nh[i].y;
      const R nv = nh[i].x * v.x + nh[i].y * v.y;
      const R sK = rn_mul(pc.sdt, K2);  // stabiliser (Sec. 5.2): in eta, not in theta
      const R nvs = nh[i].x * rn_fma(sK, vn.x, v.x) + nh[i].y * rn_fma(sK, vn.y, v.y);
      ag = RD::add(ag, w * (-K2 * invA) * n2);  // <N, A^{-1} Delta N>
      ae = RD::add(ae, w * nvs * invA);         // <N, A^{-1} v>
      at = RD::add(at, w * nv);                 // <N, v>
    }
    {
      typename RD::acc t3[3] = {ag, ae, at};
      double e2[2] = {pe[0][0] + pe[1][0], pe[0][1] + pe[1][1]};
      block_red_mixed<R, 2>(t3, e2, redb, redd);
      if (threadIdx.x == 0) {
        partG[blockIdx.x] = RD::to_double(t3[0]);
        partG[G + blockIdx.x] = RD::to_double(t3[1]);
        partG[2 * G + blockIdx.x] = RD::to_double(t3[2]);
        qE[0] = e2[0];
        qE[1] = e2[1];
      }
    }
    bar += G;
    if (!grid_sync(sync64, bar, sc, &flag_s)) return;

    // ---------------- D: scalar solve, update, next extrapolation ----------------
    {
      double pg[2][3];
      load_partials<3>(partG, G, pg);
      SolvePre pre;
      if (threadIdx.x == 0) pre = sav_solve_pre(P, qE, false, rin);  // while the partial sums arrive
      double g3s[3] = {pg[0][0] + pg[1][0], pg[0][1] + pg[1][1], pg[0][2] + pg[1][2]};
      block_sum_values<3>(g3s, redd);
      if (threadIdx.x == 0) {
        const SolveOut o = sav_solve_post(P, pre, g3s);
        alpha_s = (R)o.alpha;
        ok_s = o.ok;
        if (blockIdx.x == 0) sav_commit(sc, o, 1 - p, PEND_NONE);
        rin.r0 = rin.r1;
        rin.r1 = o.r_new;
      }
    }
    __syncthreads();
    if (!ok_s) return;  // the same decision in every block (identical sums)
    const R al = alpha_s;
    C* sold = S.at(1 - p);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int ky = clane + i * T;
      C g0 = mk<C>(0, 0), g1 = mk<C>(0, 0);
      if (col) {
        const size_t off = (size_t)ky * NH + kx;
        const C cur = st_s[ky * CT + c], old = st_s[(N + ky) * CT + c];
        C nw;
        if (off == 0) {
          // zero mode: A_0 = 3/2 and Delta kills N: a + (a - b)/3 in float64
          const double z = zero_mode_update(zm_n, zm_o);
          sc->zm[1 - p] = z;
          zm_o = zm_n;
          zm_n = z;
          nw = mk<C>((R)z, (R)0);
        } else {
          const R K2 = sym_K2<R>(kx, ky, N, pc);
          nw = bdf2_update<C, R>(cur, old, nh[i], K2, ia[i], al, rn_mul(pc.sdt, K2));
        }
        sold[off] = nw;                 // phi^{n+1} over phi^{n-1}
        st_s[ky * CT + c] = nw;         // the next step's state, kept in shared memory
        st_s[(N + ky) * CT + c] = cur;
        const C ph = mk<C>((R)2 * nw.x - cur.x, (R)2 * nw.y - cur.y);  // phi* of the next step
        const R ktx = kderiv<R>(kx, N, pc.kfx), kty = kderiv<R>(ky, N, pc.kfy);
        g0 = mk<C>(-ktx * ph.y, ktx * ph.x);
        g1 = mk<C>(-kty * ph.y, kty * ph.x);
      }
      g[0][i] = g0;
      g[1][i] = g1;
    }
    fft_regs_multi<C, N, E, true, 2, true, TwSharedFrom<SH::TW_LO>>(g, fft_s + c, SEQ * CTP, CTP, clane, tw_s);
    if (col) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const size_t off = (size_t)(clane + i * T) * NH + kx;
        W0[off] = g[0][i];
        W1[off] = g[1][i];
      }
    }
    p = 1 - p;
    if (step + 1 < nsteps) {
      bar += G;
      if (!grid_sync(sync64, bar, sc, &flag_s)) return;
    }
  }
}

}  // namespace spfc
