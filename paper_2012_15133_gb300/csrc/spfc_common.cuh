// Device building blocks shared by the SPFC step kernels:
//  * complex helpers for float2 / double2,
//  * a warp-synchronous Stockham FFT in shared memory (radix 8/4/2 stages,
//    each lane owns N/T values per stage, twiddles from a table),
//  * FP64 warp / block reductions with a fixed (deterministic) order.
//
// The Fourier pseudo-spectral method of Sec. 2.1 needs only power-of-two
// complex DFTs of length 16..512; real transforms are built on top of these
// by packing two real sequences into one complex sequence.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spfc {

template <typename R> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename R> using C_t = typename cplx<R>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) re, decltype(C::x) im) {
  C c; c.x = re; c.y = im; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// In-register DFTs of length 2, 4, 8. Forward uses exp(-2 pi i q r / R),
// inverse exp(+2 pi i q r / R); outputs in natural order.
// ---------------------------------------------------------------------------
template <typename C, bool INV> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_mi<C, INV>(csub(v1, v3));
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  v1 = cadd(a1, a3);
  v3 = csub(a1, a3);
}

template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
  using R = decltype(C::x);
  const R s = (R)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<C, INV>(e0, e1, e2, e3);
  dft4<C, INV>(o0, o1, o2, o3);
  // o_q *= w^q, w = exp(-+ 2 pi i / 8)
  C t1, t2, t3;
  if (!INV) {
    t1 = mk<C>((o1.x + o1.y) * s, (o1.y - o1.x) * s);
    t2 = mk<C>(o2.y, -o2.x);
    t3 = mk<C>((o3.y - o3.x) * s, -(o3.x + o3.y) * s);
  } else {
    t1 = mk<C>((o1.x - o1.y) * s, (o1.x + o1.y) * s);
    t2 = mk<C>(-o2.y, o2.x);
    t3 = mk<C>(-(o3.x + o3.y) * s, (o3.x - o3.y) * s);
  }
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

template <typename C, int RAD, bool INV> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (RAD == 8) dft8<C, INV>(v);
  else if constexpr (RAD == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
  else dft2<C, INV>(v);
}

// Largest transform length.
constexpr int TW_N = 512;

// Staged twiddle table: one block per (span NS, radix RAD) of a Stockham
// stage (NS RAD <= TW_N), in the order RAD = 2, 4, 8 and, within a radix, NS
// ascending. Entry (r - 1) NS + k of block (NS, RAD) holds exp(-2 pi i r k /
// (NS RAD)), r = 1 .. RAD-1, k < NS: the lanes of a warp, which differ in k,
// read consecutive entries (a table indexed by r k TW_N / (NS RAD) puts them
// 64 bytes or more apart, up to eight-way shared-memory bank conflicts).
// tw_block(ns, rad) is the block's offset; with no such block, the table length.
__host__ __device__ constexpr int tw_block(int ns, int rad) {
  int off = 0;
  for (int R = 2; R <= 8; R *= 2)
    for (int st = 1; st * R <= TW_N; st *= 2) {
      if (R == rad && st == ns) return off;
      off += (R - 1) * st;
    }
  return off;
}
constexpr int TW_LEN = tw_block(0, 0);

// Radix of the stage of a length-N transform that starts with span NS, E
// values per lane (radix 8 while it divides the rest and E, then 4, then 2).
__host__ __device__ constexpr int stage_radix(int N, int E, int ns) {
  return ((N / ns) % 8 == 0 && E % 8 == 0) ? 8 : (((N / ns) % 4 == 0 && E % 4 == 0) ? 4 : 2);
}
// First and one-past-last table entry that the stages of a length-N
// transform with E values per lane read (the first stage has no twiddles).
__host__ __device__ constexpr int tw_lo(int N, int E) {
  int lo = TW_LEN;
  for (int ns = stage_radix(N, E, 1); ns < N; ns *= stage_radix(N, E, ns)) {
    const int b = tw_block(ns, stage_radix(N, E, ns));
    lo = b < lo ? b : lo;
  }
  return lo;
}
__host__ __device__ constexpr int tw_hi(int N, int E) {
  int hi = 0;
  for (int ns = stage_radix(N, E, 1); ns < N; ns *= stage_radix(N, E, ns)) {
    const int rad = stage_radix(N, E, ns);
    const int e = tw_block(ns, rad) + (rad - 1) * ns;
    hi = e > hi ? e : hi;
  }
  return hi;
}

// Where the FFT stages read the twiddle table from: global memory through the
// read-only path (TwGlobal, the default; the whole table), or a copy in
// shared memory of entries [LO, ...) of it (TwSharedFrom<LO>; a generic load,
// valid for a shared-memory pointer).
struct TwGlobal {
  template <typename C> __device__ __forceinline__ static C ld(const C* p) { return __ldg(p); }
  template <int NS, int RAD> __device__ __forceinline__ static constexpr int off() { return tw_block(NS, RAD); }
};
template <int LO> struct TwSharedFrom {
  template <typename C> __device__ __forceinline__ static C ld(const C* p) { return *p; }
  template <int NS, int RAD> __device__ __forceinline__ static constexpr int off() { return tw_block(NS, RAD) - LO; }
};

// Shared-memory position of element i of an FFT sequence: one pad slot every
// 8 elements spreads the strided writes of the first radix-8 stage over the
// banks. A sequence of length N occupies sp_len(N) slots.
__device__ __forceinline__ constexpr int sp(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int sp_len(int n) { return n + n / 8; }
// Position in a contiguous sequence (element stride 1: rows, one-column
// tiles): one pad slot every 16 elements. The strided writes of a radix-8
// stage stay spread, and 16 lanes reading consecutive elements (one 128-byte
// wavefront of 8-byte elements) no longer wrap onto the same banks as they do
// with a pad every 8 (bank model: 2.5 against 3 wavefronts per access of the
// row exchanges). Fits in sp_len(N) slots.
__device__ __forceinline__ constexpr int spr(int i) { return i + (i >> 4); }
// Slot of element i of a sequence with element stride es.
__device__ __forceinline__ int sps(int i, int es) { return es == 1 ? spr(i) : sp(i) * es; }

// Pitch (in elements) between consecutive elements of one sequence when CT
// sequences of a column tile are interleaved in shared memory (element j of
// column c at c + sp(j) * pitch; thread lane * CT + c). Bank analysis of the
// exchanges of fft_regs_multi with 8- and 16-byte elements (each group of
// lanes covering 128 bytes is one shared-memory wavefront when its words fall
// in distinct banks): the unpadded pitch CT reaches the minimum number of
// wavefronts for every tile with CT >= 2 used here, whereas an odd pitch
// CT + 1 needs up to twice as many (measured: 3.98 wavefronts per 8-byte
// access against 1.99 ideal in the 128^3 y pass).
__host__ __device__ constexpr int col_pitch(int ct) { return ct; }


// A length-N FFT is done by T = N/E lanes, each owning E values per stage.
// T <= 32: the lanes of a sequence sit in one warp (__syncwarp between
// stages); T > 32: the sequence spans warps and every thread of the block
// takes part in the same FFT call (__syncthreads between stages).
template <int N, int E> struct fft_shape {
  static constexpr int T = N / E;
  static_assert(N >= 16 && N <= TW_N && (N & (N - 1)) == 0, "FFT length must be a power of two in [16,512]");
  static_assert(E == 4 || E == 8 || E == 16, "4, 8 or 16 values per lane");
  static_assert(T >= 1 && (T <= 32 ? 32 % T == 0 : T % 32 == 0), "a sequence must not straddle warps unevenly");
};

template <int N, int E, bool BS = false> __device__ __forceinline__ void fft_sync() {
  if constexpr (N / E <= 32 && !BS) __syncwarp(); else __syncthreads();
}

// Stockham stages of radix RAD (Govindaraju et al., SC'08 formulation):
// butterfly j reads x[j + r N/RAD], twiddles by w^(r (j mod NS) N/(NS RAD)),
// transforms, and writes x[(j/NS) NS RAD + (j mod NS) + r NS].
//
// Radix of the stage that starts with span NS (the same rule for every
// caller: radix 8 while it divides the rest and E, then 4, then 2).
template <int N, int E, int NS> struct stage_rad {
  static constexpr int REM = N / NS;
  static constexpr int value = (REM % 8 == 0 && E % 8 == 0) ? 8 : ((REM % 4 == 0 && E % 4 == 0) ? 4 : 2);
};

// Span NS of the last stage.
template <int N, int E> __host__ __device__ constexpr int last_span() {
  int ns = 1;
  while (true) {
    const int rem = N / ns;
    const int rad = (rem % 8 == 0 && E % 8 == 0) ? 8 : ((rem % 4 == 0 && E % 4 == 0) ? 4 : 2);
    if (ns * rad == N) return ns;
    ns *= rad;
  }
}

// The three parts of a stage for the butterflies j = lane + m T of one lane:
// load v[m RAD + r] = x[j + r N/RAD]; twiddle and transform in registers;
// store to x[(j/NS) NS RAD + (j mod NS) + r NS].
template <typename C, int N, int E, int RAD>
__device__ __forceinline__ void stage_load(C* v, const C* s, int es, int lane) {
  constexpr int T = fft_shape<N, E>::T, NB = E / RAD, STRIDE = N / RAD;
#pragma unroll
  for (int m = 0; m < NB; ++m)
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[m * RAD + r] = s[sps(lane + m * T + r * STRIDE, es)];
}

template <typename C, int N, int E, bool INV, int NS, int RAD, class TWL = TwGlobal>
__device__ __forceinline__ void stage_compute(C* v, int lane, const C* __restrict__ tw) {
  constexpr int T = fft_shape<N, E>::T, NB = E / RAD;
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int k = (lane + m * T) & (NS - 1);
    if constexpr (NS > 1) {
      constexpr int TB = TWL::template off<NS, RAD>();
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        C w = TWL::template ld<C>(tw + TB + (r - 1) * NS + k);
        if (INV) w.y = -w.y;
        v[m * RAD + r] = cmul(v[m * RAD + r], w);
      }
    }
    dft_r<C, RAD, INV>(v + m * RAD);
  }
}

template <typename C, int N, int E, int NS, int RAD>
__device__ __forceinline__ void stage_store(const C* v, C* s, int es, int lane) {
  constexpr int T = fft_shape<N, E>::T, NB = E / RAD;
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int j = lane + m * T, k = j & (NS - 1);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) s[sps(base + r * NS, es)] = v[m * RAD + r];
  }
}

// One Stockham stage of radix RAD in shared memory, in place: all lanes of a
// sequence hold their inputs in registers across a barrier.
template <typename C, int N, int E, bool INV, int NS, int RAD>
__device__ __forceinline__ void stockham_stage(C* s, int es, int lane, const C* __restrict__ tw) {
  C v[E];
  stage_load<C, N, E, RAD>(v, s, es, lane);
  fft_sync<N, E>();
  stage_compute<C, N, E, INV, NS, RAD>(v, lane, tw);
  stage_store<C, N, E, NS, RAD>(v, s, es, lane);
  fft_sync<N, E>();
}

template <typename C, int N, int E, bool INV, int NS>
__device__ __forceinline__ void fft_stages(C* s, int es, int lane, const C* __restrict__ tw) {
  if constexpr (NS < N) {
    constexpr int RAD = stage_rad<N, E, NS>::value;
    stockham_stage<C, N, E, INV, NS, RAD>(s, es, lane, tw);
    fft_stages<C, N, E, INV, NS * RAD>(s, es, lane, tw);
  }
}

// Stages NS .. NSL (exclusive) in shared memory.
template <typename C, int N, int E, bool INV, int NS, int NSL>
__device__ __forceinline__ void fft_mid_stages(C* s, int es, int lane, const C* __restrict__ tw) {
  if constexpr (NS < NSL) {
    constexpr int RAD = stage_rad<N, E, NS>::value;
    stockham_stage<C, N, E, INV, NS, RAD>(s, es, lane, tw);
    fft_mid_stages<C, N, E, INV, NS * RAD, NSL>(s, es, lane, tw);
  }
}

// Unnormalised complex DFT of one length-N sequence held in registers: on
// entry v[i] is element lane + i T of the input, on return v[i] is element
// lane + i T of the output (T = N/E). The first stage reads its inputs from
// registers and the last leaves its outputs there (both are strided by T in
// this order), so only the middle stages and one exchange on each side go
// through shared memory (`s`, es as for fft_smem). Starts with a barrier
// (the buffer may still be read by the caller's previous use); on return
// the lanes may still be reading `s`.
template <typename C, int N, int E, bool INV>
__device__ __forceinline__ void fft_regs(C* v, C* s, int es, int lane, const C* __restrict__ tw) {
  constexpr int R1 = stage_rad<N, E, 1>::value, NB1 = E / R1;
  constexpr int NSL = last_span<N, E>();
  constexpr int RL = N / NSL, NBL = E / RL;
  static_assert(NSL > 1, "at least two stages");
  C w[E];
#pragma unroll
  for (int m = 0; m < NB1; ++m)
#pragma unroll
    for (int r = 0; r < R1; ++r) w[m * R1 + r] = v[m + r * NB1];  // element lane + T (m + r NB1)
  stage_compute<C, N, E, INV, 1, R1>(w, lane, tw);
  fft_sync<N, E>();
  stage_store<C, N, E, 1, R1>(w, s, es, lane);
  fft_sync<N, E>();
  fft_mid_stages<C, N, E, INV, R1, NSL>(s, es, lane, tw);
  stage_load<C, N, E, RL>(w, s, es, lane);
  stage_compute<C, N, E, INV, NSL, RL>(w, lane, tw);
#pragma unroll
  for (int m = 0; m < NBL; ++m)
#pragma unroll
    for (int r = 0; r < RL; ++r) v[m + r * NBL] = w[m * RL + r];  // output lane + T (m + r NBL)
}

// fft_regs for NSEQ sequences of one lane at once (sequence q in shared
// memory at s + q * qs), sharing the barriers; BS forces block-wide barriers
// (for lanes of one sequence spread over several warps).
template <typename C, int N, int E, bool INV, int NSEQ, bool BS, int NS, int NSL, class TWL = TwGlobal>
__device__ __forceinline__ void fft_mid_multi(C* s, int qs, int es, int lane, const C* __restrict__ tw) {
  if constexpr (NS < NSL) {
    constexpr int RAD = stage_rad<N, E, NS>::value;
    C v[NSEQ][E];
#pragma unroll
    for (int q = 0; q < NSEQ; ++q) stage_load<C, N, E, RAD>(v[q], s + q * qs, es, lane);
    fft_sync<N, E, BS>();
#pragma unroll
    for (int q = 0; q < NSEQ; ++q) {
      stage_compute<C, N, E, INV, NS, RAD, TWL>(v[q], lane, tw);
      stage_store<C, N, E, NS, RAD>(v[q], s + q * qs, es, lane);
    }
    fft_sync<N, E, BS>();
    fft_mid_multi<C, N, E, INV, NSEQ, BS, NS * RAD, NSL, TWL>(s, qs, es, lane, tw);
  }
}

template <typename C, int N, int E, bool INV, int NSEQ, bool BS, class TWL = TwGlobal>
__device__ __forceinline__ void fft_regs_multi(C (*v)[E], C* s, int qs, int es, int lane,
                                               const C* __restrict__ tw) {
  constexpr int R1 = stage_rad<N, E, 1>::value, NB1 = E / R1;
  constexpr int NSL = last_span<N, E>();
  constexpr int RL = N / NSL, NBL = E / RL;
  static_assert(NSL > 1, "at least two stages");
  fft_sync<N, E, BS>();
#pragma unroll
  for (int q = 0; q < NSEQ; ++q) {
    C w[E];
#pragma unroll
    for (int m = 0; m < NB1; ++m)
#pragma unroll
      for (int r = 0; r < R1; ++r) w[m * R1 + r] = v[q][m + r * NB1];
    stage_compute<C, N, E, INV, 1, R1, TWL>(w, lane, tw);
    stage_store<C, N, E, 1, R1>(w, s + q * qs, es, lane);
  }
  fft_sync<N, E, BS>();
  fft_mid_multi<C, N, E, INV, NSEQ, BS, R1, NSL, TWL>(s, qs, es, lane, tw);
#pragma unroll
  for (int q = 0; q < NSEQ; ++q) {
    C w[E];
    stage_load<C, N, E, RL>(w, s + q * qs, es, lane);
    stage_compute<C, N, E, INV, NSL, RL, TWL>(w, lane, tw);
#pragma unroll
    for (int m = 0; m < NBL; ++m)
#pragma unroll
      for (int r = 0; r < RL; ++r) v[q][m + r * NBL] = w[m * RL + r];
  }
}

// Unnormalised complex DFT of the length-N sequence whose element i is at
// s[sps(i, es)] in shared memory, in place, by the T = N/E lanes (lane = 0..T-1) of one
// sequence. Forward: exp(-2 pi i k j / N); INV: exp(+2 pi i k j / N).
// The caller has made the input visible (block or warp barrier as fft_sync);
// on return the output is visible to the sequence's lanes.
template <typename C, int N, int E, bool INV>
__device__ __forceinline__ void fft_smem(C* s, int es, int lane, const C* __restrict__ tw) {
  fft_stages<C, N, E, INV, 1>(s, es, lane, tw);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor is still running; pdl_wait()
// blocks until the predecessor grid has completed and its memory is visible,
// pdl_trigger() lets the successor grid be scheduled. Both are no-ops for a
// normal launch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `v` over the block (blockDim.x a multiple of 32, <= 1024); the
// result is returned to thread 0. `scratch` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < nw) ? scratch[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum of n values a[0..n) by one full warp, fixed order (lane-strided partial
// sums then a butterfly tree). Reads bypass L1 so that values written by
// other blocks of the same grid (before a fence) are seen.
__device__ __forceinline__ double warp_sum_array(const double* a, int n, int lane) {
  double t = 0.0;
  for (int base = 0; base < n; base += 256) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = base + lane + 32 * u;
      v[u] = (i < n) ? __ldcg(a + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) t += v[u];
  }
  return warp_sum(t);
}

// Accumulators of the SAV inner products and of E_1 (the precision split of
// the FP32-bulk path keeps these sums and everything derived from them in
// float64).
// Per thread and per block, the float64 path adds in float64. The
// float32-bulk path adds its float32 products in float-float (hi + lo,
// Knuth's two-sum on every addition): the exact sum of a thread's and then a
// block's float32 products to ~2^-48 relative, on the float32 pipes (float64
// issue is scarce on this GPU). Each block's result is stored as a float64
// (hi + lo is exact in float64: two 24-bit significands within 48 bits), and
// everything after that -- the sums over blocks, E_1, S, gamma, eta, theta,
// rho, LHS and r -- is float64 on both paths.
template <typename R> struct Red;

template <> struct Red<double> {
  using acc = double;
  __device__ static acc zero() { return 0.0; }
  __device__ static acc add(acc a, double x) { return a + x; }
  __device__ static acc add2(acc a, acc b) { return a + b; }
  __device__ static acc shfl(acc a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double to_double(acc a) { return a; }
};

template <> struct Red<float> {
  using acc = float2;   // (hi, lo)
  __device__ static acc zero() { return make_float2(0.f, 0.f); }
  __device__ static acc add(acc a, float x) {
    const float s = __fadd_rn(a.x, x);
    const float bb = __fsub_rn(s, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    return make_float2(s, __fadd_rn(a.y, err));
  }
  __device__ static acc add2(acc a, acc b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    const float lo = __fadd_rn(__fadd_rn(a.y, b.y), err);
    // renormalise (fast two-sum)
    const float h = __fadd_rn(s, lo);
    return make_float2(h, __fsub_rn(lo, __fsub_rn(h, s)));
  }
  __device__ static acc shfl(acc a, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
  }
  __device__ static double to_double(acc a) { return (double)a.x + (double)a.y; }
};

template <typename R> __device__ __forceinline__ typename Red<R>::acc warp_red(typename Red<R>::acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = Red<R>::add2(v, Red<R>::shfl(v, o));
  return v;
}

// Smallest power of two >= nw (nw >= 1). In the second stage of a block
// reduction only lanes < nw hold values; an xor-shuffle level o >= this bound
// pairs every lane below it with a zero, and adding an exact zero leaves a
// (normalised) accumulator unchanged, so those levels are skipped with the
// same result.
__device__ __forceinline__ int pow2_ceil(int nw) { return 1 << (32 - __clz(nw - 1)); }

// Block reduction of accumulators (fixed order); result valid in thread 0.
template <typename R>
__device__ __forceinline__ typename Red<R>::acc block_red(typename Red<R>::acc v, typename Red<R>::acc* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_red<R>(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  typename Red<R>::acc t = Red<R>::zero();
  if (wid == 0) {
    t = (lane < nw) ? scratch[lane] : Red<R>::zero();
    const int p2 = pow2_ceil(nw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      if (o < p2) t = Red<R>::add2(t, Red<R>::shfl(t, o));
  }
  return t;
}

// K block sums at once (the same tree as K calls of block_red, sharing the
// barriers); results in thread 0 (v overwritten).
template <typename R, int K>
__device__ __forceinline__ void block_red_multi(typename Red<R>::acc* v, typename Red<R>::acc (*scratch)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_red<R>(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k][wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
    const int p2 = pow2_ceil(nw);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (lane < nw) ? scratch[k][lane] : Red<R>::zero();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= p2) continue;
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = Red<R>::add2(v[k], Red<R>::shfl(v[k], o));
    }
  }
}

// Grid-level reduction of NQ float64 partial-sum arrays by a whole block,
// in float64, all NQ chains interleaved: thread t sums entries t,
// t + blockDim, .. of each array (L1 bypassed: the entries were written by
// other blocks of the grid), then a shuffle tree and a shared-memory tree.
// Fixed order; results in thread 0.
template <int NQ>
__device__ __forceinline__ void block_sum_arrays(const double* const* arr, const int* n, double* out,
                                                 double (*scratch)[32]) {
  double a[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) a[q] = 0.0;
  int nmax = 0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) nmax = n[q] > nmax ? n[q] : nmax;
  // two strides of loads in flight per round (the same per-thread order of
  // additions), so that a grid of up to 2 x blockDim.x blocks needs one L2
  // round trip, not two
  for (int base = 0; base < nmax; base += 2 * blockDim.x) {
    double v[2][NQ];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = base + u * blockDim.x + threadIdx.x;
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[u][q] = (i < n[q]) ? __ldcg(arr[q] + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) a[q] += v[u][q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) scratch[q][wid] = a[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] = (lane < nw) ? scratch[q][lane] : 0.0;
    const int p2 = pow2_ceil(nw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (o >= p2) continue;
#pragma unroll
      for (int q = 0; q < NQ; ++q) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) out[q] = a[q];
    }
  }
}

}  // namespace spfc
