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

// Largest twiddle table length; table[m] = exp(-2 pi i m / TW_N).
constexpr int TW_N = 512;

// Lanes per sequence for a length-N FFT: every lane owns N/T values (8 or 16).
template <int N> struct fft_shape {
  static constexpr int T = (N / 8 < 32) ? N / 8 : 32;
  static constexpr int E = N / T;
  static_assert(N >= 16 && N <= 512 && (N & (N - 1)) == 0, "FFT length must be a power of two in [16,512]");
  static_assert(32 % T == 0, "a sequence must not straddle warps");
};

// One Stockham stage of radix RAD (Govindaraju et al., SC'08 formulation):
// butterfly j reads x[j + r N/RAD], twiddles by w^(r (j mod NS) N/(NS RAD)),
// transforms, and writes x[(j/NS) NS RAD + (j mod NS) + r NS]. All lanes of a
// sequence hold their inputs in registers across a __syncwarp, so the stage
// runs in place.
template <typename C, int N, bool INV, int NS, int RAD>
__device__ __forceinline__ void stockham_stage(C* s, int es, int lane, const C* __restrict__ tw) {
  constexpr int T = fft_shape<N>::T, E = fft_shape<N>::E;
  constexpr int NB = E / RAD;
  constexpr int STRIDE = N / RAD;
  constexpr int TWS = TW_N / (NS * RAD);
  C v[E];
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int j = lane + m * T;
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[m * RAD + r] = s[(j + r * STRIDE) * es];
  }
  __syncwarp();
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    const int j = lane + m * T;
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        C w = tw[r * k * TWS];
        if (INV) w.y = -w.y;
        v[m * RAD + r] = cmul(v[m * RAD + r], w);
      }
    }
    dft_r<C, RAD, INV>(v + m * RAD);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) s[(base + r * NS) * es] = v[m * RAD + r];
  }
  __syncwarp();
}

template <typename C, int N, bool INV, int NS>
__device__ __forceinline__ void fft_stages(C* s, int es, int lane, const C* __restrict__ tw) {
  if constexpr (NS < N) {
    constexpr int E = fft_shape<N>::E;
    constexpr int REM = N / NS;
    constexpr int RAD = (REM % 8 == 0 && E % 8 == 0) ? 8 : ((REM % 4 == 0 && E % 4 == 0) ? 4 : 2);
    stockham_stage<C, N, INV, NS, RAD>(s, es, lane, tw);
    fft_stages<C, N, INV, NS * RAD>(s, es, lane, tw);
  }
}

// Unnormalised complex DFT of the length-N sequence s[0], s[es], .., s[(N-1) es]
// in shared memory, in place, by the T lanes (lane = 0..T-1) of one warp
// sub-group. Forward: exp(-2 pi i k j / N); INV: exp(+2 pi i k j / N).
// Every lane of the warp must call it (it synchronises with __syncwarp).
template <typename C, int N, bool INV>
__device__ __forceinline__ void fft_smem(C* s, int es, int lane, const C* __restrict__ tw) {
  __syncwarp();
  fft_stages<C, N, INV, 1>(s, es, lane, tw);
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reductions
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
  for (int i = lane; i < n; i += 32) t += __ldcg(a + i);
  return warp_sum(t);
}

}  // namespace spfc
