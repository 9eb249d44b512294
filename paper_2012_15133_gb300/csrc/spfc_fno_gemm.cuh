// Batched BF16 tensor-core GEMM with FP32 accumulation for the surrogate
// network: C[b] = alpha * A[b] B[b] + beta * C[b] (+ bias, GELU epilogue).
//
// Operands may be float32 or bfloat16 in memory; tiles are converted to
// bfloat16 in shared memory and multiplied with mma.sync m16n8k16 (BF16 in,
// FP32 accumulate). Every matrix index goes through a two-level stride
// (i -> (i % s) * a + (i / s) * b), which expresses the truncated-DFT layouts
// (real/imaginary halves, batch-of-rows) without copies. Split-K writes
// partial tiles to a workspace that a second kernel reduces in a fixed
// order (deterministic weight gradients).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spfc {
namespace fno {

// Index map i -> (i % s) * a + (i / s) * b. The quotient uses a multiplier
// fixed on the host (division by an invariant integer, Granlund & Montgomery
// 1994): q = (umulhi(i, m) + i) >> l with l = ceil(log2 s) and
// m = floor(2^32 (2^l - s) / s) + 1; exact for 0 <= i < 2^31 (the sum then
// stays below 2^32). m = 0 marks a one-level map (s larger than any index).
struct Ix {
  long long a = 1, b = 0;
  int s = 0x7fffffff;
  unsigned int m = 0;
  int l = 0;
  __device__ __forceinline__ long long operator()(int i) const {
    if (m == 0) return (long long)i * a;
    const int q = (int)((__umulhi((unsigned)i, m) + (unsigned)i) >> l);
    return (long long)(i - q * s) * a + (long long)q * b;
  }
};

inline Ix make_ix(long long a, int s = 0x7fffffff, long long b = 0) {
  Ix r;
  r.a = a;
  r.b = b;
  r.s = s;
  if (s != 0x7fffffff) {
    int l = 0;
    while ((1ll << l) < (long long)s) ++l;
    r.l = l;
    r.m = (unsigned int)((((unsigned long long)1 << 32) * (((unsigned long long)1 << l) - (unsigned long long)s)) /
                             (unsigned long long)s + 1ull);
  }
  return r;
}

struct Mat {
  const void* p = nullptr;
  int bf16 = 0;           // 1: __nv_bfloat16, 0: float
  Ix r, c;                // row and column index maps
  long long sb = 0;       // batch stride (elements)
};

struct Out {
  float* p = nullptr;     // FP32 output
  const float* cin = nullptr;  // C of beta * C (same addressing; p when null)
  Ix r, c;
  long long sb = 0;
  float alpha = 1.f, beta = 0.f;
  const float* bias = nullptr;  // bias[(row / bdiv) % bmod] or, if bias_col, bias[col]
  int bdiv = 1, bmod = 1 << 30, bias_col = 0;
  int act = 0;            // 1: GELU (the pre-activation goes to pre)
  float* pre = nullptr;   // optional store of the pre-activation (same addressing)
};

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

__device__ __forceinline__ float ldm(const Mat& m, long long off) {
  if (m.bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(m.p)[off]);
  return reinterpret_cast<const float*>(m.p)[off];
}

constexpr int BM = 64, BN = 64, BK = 32, GT = 128;
constexpr int SKP = BK + 8;  // padded k pitch (bf16 elements)

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Apply the epilogue to one value and store it.
__device__ __forceinline__ void store_out(const Out& o, long long base, int row, int col, float acc) {
  const long long off = base + o.r(row) + o.c(col);
  float v = o.alpha * acc;
  if (o.beta != 0.f) v += o.beta * (o.cin ? o.cin[off] : o.p[off]);
  if (o.bias) v += o.bias_col ? o.bias[col] : o.bias[(row / o.bdiv) % o.bmod];
  if (o.act == 1) {
    if (o.pre) o.pre[off] = v;
    v = gelu_f(v);
  }
  o.p[off] = v;
}

// grid: (ceil(N/BN), ceil(M/BM), batch * splits); block GT threads.
// splits > 1: raw partial sums to ws[((z * M) + row) * N + col] (z = batch * splits + split).
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, int batch, int splits, Mat A, Mat B, Out O,
                                             float* __restrict__ ws) {
  __shared__ __align__(16) __nv_bfloat16 As[BM * SKP];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN * SKP];
  const int z = blockIdx.z;
  const int bt = z / splits, split = z % splits;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kchunk = (((K + splits - 1) / splits) + BK - 1) / BK * BK;
  const int kb = split * kchunk, ke = min(K, kb + kchunk);
  const long long abase = (long long)bt * A.sb, bbase = (long long)bt * B.sb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t4 = lane & 3;
  const bool a_kfast = (A.c.a == 1 && A.c.s >= BK);   // consecutive k contiguous in A
  const bool b_nfast = (B.c.a == 1 && B.c.s >= BN);   // consecutive n contiguous in B
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  for (int k0 = kb; k0 < ke; k0 += BK) {
    // A tile (BM x BK) -> As[m][k]
#pragma unroll 4
    for (int e = 0; e < BM * BK / GT; ++e) {
      const int lin = tid + e * GT;
      int mm, kk;
      if (a_kfast) { mm = lin / BK; kk = lin % BK; } else { mm = lin % BM; kk = lin / BM; }
      const int row = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (row < M && k < ke) v = ldm(A, abase + A.r(row) + A.c(k));
      As[mm * SKP + kk] = __float2bfloat16_rn(v);
    }
    // B tile (BK x BN) -> Bs[n][k]
#pragma unroll 4
    for (int e = 0; e < BN * BK / GT; ++e) {
      const int lin = tid + e * GT;
      int nn, kk;
      if (b_nfast) { nn = lin % BN; kk = lin / BN; } else { nn = lin / BK; kk = lin % BK; }
      const int col = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (col < N && k < ke) v = ldm(B, bbase + B.r(k) + B.c(col));
      Bs[nn * SKP + kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const __nv_bfloat16* base = As + (wm + i * 16) * SKP + ks;
        af[i][0] = *reinterpret_cast<const uint32_t*>(base + g * SKP + 2 * t4);
        af[i][1] = *reinterpret_cast<const uint32_t*>(base + (g + 8) * SKP + 2 * t4);
        af[i][2] = *reinterpret_cast<const uint32_t*>(base + g * SKP + 2 * t4 + 8);
        af[i][3] = *reinterpret_cast<const uint32_t*>(base + (g + 8) * SKP + 2 * t4 + 8);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16* base = Bs + (wn + j * 8 + g) * SKP + ks;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(base + 2 * t4);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(base + 2 * t4 + 8);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
  // epilogue: acc[i][j][e]: row = wm + 16 i + g (+8 for e >= 2), col = wn + 8 j + 2 t4 + (e & 1)
  const long long obase = (long long)bt * O.sb;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + wm + 16 * i + g + ((e >= 2) ? 8 : 0);
        const int col = n0 + wn + 8 * j + 2 * t4 + (e & 1);
        if (row >= M || col >= N) continue;
        if (splits > 1) ws[((long long)z * M + row) * N + col] = acc[i][j][e];
        else store_out(O, obase, row, col, acc[i][j][e]);
      }
}

// Fixed-order reduction of the split-K partial sums, then the epilogue.
__global__ void k_gemm_reduce(int M, int N, int batch, int splits, const float* __restrict__ ws, Out O) {
  const long long total = (long long)batch * M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int bt = (int)(i / ((long long)M * N));
    const int rem = (int)(i % ((long long)M * N));
    const int row = rem / N, col = rem % N;
    float s = 0.f;
    for (int sp = 0; sp < splits; ++sp) s += ws[(((long long)bt * splits + sp) * M + row) * N + col];
    store_out(O, (long long)bt * O.sb, row, col, s);
  }
}

}  // namespace fno
}  // namespace spfc
