// Batched BF16 tensor-core GEMM with FP32 accumulation for the surrogate
// network: C[b] = alpha * A[b] B[b] + beta * C[b] (+ bias, GELU epilogue).
//
// Operands may be float32 or bfloat16 in memory; tiles are gathered,
// converted to bfloat16 in shared memory and multiplied by the fifth-
// generation tensor cores (tcgen05.mma, accumulator in tensor memory). Every
// matrix index goes through a two-level stride (i -> (i % s) * a + (i / s) * b),
// which expresses the truncated-DFT layouts (real/imaginary halves,
// batch-of-rows) without copies. Split-K writes partial tiles to a workspace
// that a second kernel reduces in a fixed order (deterministic weight
// gradients).
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

// Fixed-order reduction of the split-K partial sums, then the epilogue: one
// warp per output element, lane l summing splits l, l + 32, .. in order, then
// a fixed butterfly; lane 0 stores.
__global__ void k_gemm_reduce(int M, int N, int batch, int splits, const float* __restrict__ ws, Out O) {
  const long long total = (long long)batch * M * N;
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < total; i += nw) {
    const int bt = (int)(i / ((long long)M * N));
    const int rem = (int)(i % ((long long)M * N));
    const int row = rem / N, col = rem % N;
    float s = 0.f;
    for (int sp = lane; sp < splits; sp += 32) s += ws[(((long long)bt * splits + sp) * M + row) * N + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) store_out(O, (long long)bt * O.sb, row, col, s);
  }
}

// ---------------------------------------------------------------------------
// The tensor-core product: tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulator in tensor memory), one CTA of four warps per 128 x tn output
// tile, tn in {16, 32, 64}.
//
// The 128-row side of the tile ("X", the MMA's A operand) is whichever of M
// and N is larger; the other side ("Y", the MMA's B operand) gives the tile's
// tn columns. Both operands are gathered through their index maps (global ->
// registers -> BF16), stored K-major in the canonical no-swizzle layout of
// 8-row x 16-byte core matrices, and multiplied in K steps of 32 (two K = 16
// instructions) issued by one thread. Two shared-memory stages alternate: the
// gather of step k+1 runs while the tensor core works on step k, and a stage
// is overwritten only after the mbarrier that tcgen05.commit arrives on shows
// the instructions that read it are complete. Every wait is bounded (about a
// second of %globaltimer); a wait that runs out latches status = 1, waits
// (bounded again) for the instructions already issued, frees the tensor
// memory and leaves the tile unwritten.
//
// Epilogue: tcgen05.ld moves each warp's 32 accumulator rows to registers,
// then to shared memory (pitch tn_max + 1, conflict-free), and the tile is
// written out with consecutive threads along the output's unit-stride
// dimension (each thread keeping one tile row or one tile column), through
// the epilogue of store_out (alpha, beta * C, bias, GELU, pre-activation
// store) or, with split-K, as raw partial sums. The output offsets and the
// bias of every tile row and column are computed once, into shared memory.
// ---------------------------------------------------------------------------
constexpr int TM = 128;                  // MMA rows = tensor-memory lanes
constexpr int TNMAX = 64;                // MMA columns at most = tensor-memory columns allocated
constexpr int TK = 32;                   // K per stage
constexpr int TT = 128;                  // threads: warp w reads lanes 32w .. 32w + 31
constexpr int kXBytes = TM * TK * 2;     // one stage of X (BF16)
constexpr int kYBytes = TNMAX * TK * 2;  // one stage of Y
constexpr int kStage = kXBytes + kYBytes;
constexpr int kEpiPitch = TNMAX + 1;
constexpr int kEpiBytes = (2 * kStage > TM * kEpiPitch * 4) ? 2 * kStage : TM * kEpiPitch * 4;
constexpr int kTcSmem = kEpiBytes + (TM + TNMAX) * 8 + (TM + TNMAX) * 4;  // + per-row/column offsets and biases
constexpr long long kTcWaitNs = 1000000000ll;  // bound of one mbarrier wait

// One MMA operand: element (r, k) at sb * batch + rm(r) + km(k).
struct Opnd {
  const void* p = nullptr;
  int bf16 = 0;
  Ix rm, km;
  long long sb = 0;
  int rows = 0;      // valid rows (M or N)
  int kcontig = 0;   // 8 consecutive k from a multiple of 8 are 8 consecutive elements
  int rowfast = 0;   // consecutive rows are consecutive elements (threads laid along rows)
};

struct TcArgs {
  Opnd X, Y;
  int M = 0, N = 0, K = 0, splits = 1;
  int swap = 0;      // X holds B's columns (the tile's rows are output columns)
  int tn = 16, tn_log2 = 4;
  int ifast = 0;     // epilogue: consecutive threads along the tile's rows
  Out O;
  float* ws = nullptr;
  int* status = nullptr;
  int stall_test = 0;  // self-test of the wait bound (never set by the network)
};

__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  // kind::f16 instruction descriptor: D float32 (bits 4-5 = 1), A and B
  // bfloat16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading-
// dimension byte offset (between core matrices adjacent in K), stride byte
// offset (between 8-row groups), all >> 4; bits 46-48 hold the fixed 0b001.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

// One test of the phase; the thread may sleep until the phase completes, for
// at most the hint (1 ms), instead of spinning.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of the mbarrier phase of the given parity; false
// once kTcWaitNs have passed (or 2^24 polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((long long)(global_ns() - t0) > kTcWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp gets lane
// (taddr lane) + t, columns (taddr column) .. + 15; the wait is in the same
// statement, so no use of the registers can come before the data.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ float ldx(const Opnd& x, long long off) {
  if (x.bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(x.p)[off]);
  return reinterpret_cast<const float*>(x.p)[off];
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // lo in the low half: the lower address
  return *reinterpret_cast<const uint32_t*>(&h);
}

// k .. k+7 (k a multiple of 8) of row r, loaded into v without any use of
// the loaded values, so that the loads of every chunk of a K step are in
// flight together (a use would stall the in-order issue until its load
// lands). Returns how v holds them: 0 float32 values (zero beyond the
// operand's rows or beyond ke), 1 eight BF16 values already packed in
// v[0..3], 2 one BF16 bit pattern in the low half of each v[j].
__device__ __forceinline__ int load8(const Opnd& x, long long base, int r, int k, int ke, float (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.f;
  if (r >= x.rows) return 0;
  const long long roff = base + x.rm(r);
  if (x.kcontig && k + 8 <= ke) {
    const long long off = roff + x.km(k);
    if (x.bf16) {
      const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(x.p) + off;
      if ((reinterpret_cast<uintptr_t>(h) & 15) == 0) {
        const uint4 u = *reinterpret_cast<const uint4*>(h);
        v[0] = __uint_as_float(u.x);
        v[1] = __uint_as_float(u.y);
        v[2] = __uint_as_float(u.z);
        v[3] = __uint_as_float(u.w);
        return 1;
      }
      const unsigned short* hb = reinterpret_cast<const unsigned short*>(h);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __uint_as_float((uint32_t)hb[j]);
      return 2;
    }
    const float* f = reinterpret_cast<const float*>(x.p) + off;
    if ((reinterpret_cast<uintptr_t>(f) & 15) == 0) {
      const float4 a = reinterpret_cast<const float4*>(f)[0], b = reinterpret_cast<const float4*>(f)[1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = f[j];
    }
    return 0;
  }
  if (x.bf16) {
    const unsigned short* hb = reinterpret_cast<const unsigned short*>(x.p);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k + j < ke) v[j] = __uint_as_float((uint32_t)hb[roff + x.km(k + j)]);  // zero bits: +0
    return 2;
  }
  const float* f = reinterpret_cast<const float*>(x.p);
  if (x.km.m == 0) {  // one-level map: consecutive k a fixed stride apart
    const float* fk = f + roff + (long long)k * x.km.a;
    const long long a = x.km.a;
    if (k + 8 <= ke) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = fk[j * a];
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (k + j < ke) v[j] = fk[j * a];
    }
    return 0;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (k + j < ke) v[j] = f[roff + x.km(k + j)];
  return 0;
}

// The chunk loaded by load8 as one core-matrix row of BF16 (float32 values
// rounded to nearest even; BF16 values as they are).
__device__ __forceinline__ uint4 pack8(int mode, const float (&v)[8]) {
  uint4 u;
  if (mode == 1) {
    u.x = __float_as_uint(v[0]);
    u.y = __float_as_uint(v[1]);
    u.z = __float_as_uint(v[2]);
    u.w = __float_as_uint(v[3]);
  } else if (mode == 2) {
    u.x = __float_as_uint(v[0]) | (__float_as_uint(v[1]) << 16);
    u.y = __float_as_uint(v[2]) | (__float_as_uint(v[3]) << 16);
    u.z = __float_as_uint(v[4]) | (__float_as_uint(v[5]) << 16);
    u.w = __float_as_uint(v[6]) | (__float_as_uint(v[7]) << 16);
  } else {
    u.x = pack_bf16(v[0], v[1]);
    u.y = pack_bf16(v[2], v[3]);
    u.z = pack_bf16(v[4], v[5]);
    u.w = pack_bf16(v[6], v[7]);
  }
  return u;
}

// Byte offset of core-matrix row (r, 8 kg .. 8 kg + 7) in a stage: core
// matrix (r / 8, kg) at ((r / 8) * 4 + kg) * 128, its rows 16 bytes apart.
// So K-adjacent core matrices are 128 bytes apart (the descriptors' leading
// offset) and 8-row groups 512 (their stride offset).
__device__ __forceinline__ int core_off(int r, int kg) { return ((r >> 3) * 4 + kg) * 128 + (r & 7) * 16; }

// Chunk c of an operand tile with R rows: (row, k group). Along rows when the
// operand's rows are consecutive in memory (eight threads fill one core
// matrix either way, so the 16-byte stores are conflict-free).
__device__ __forceinline__ void chunk_rk(int rowfast, int c, int rmask, int rlog2, int& r, int& kg) {
  if (rowfast) {
    r = c & rmask;
    kg = c >> rlog2;
  } else {
    r = (c & 7) | ((c >> 5) << 3);
    kg = (c >> 3) & 3;
  }
}

// grid: (ceil(tile columns / tn), ceil(tile rows / 128), batch * splits); TT threads; kTcSmem dynamic
// shared memory. splits > 1: raw partial sums to ws[((z * M) + row) * N + col] (z = batch * splits + split).
__global__ void __launch_bounds__(TT) k_gemm_tc(const TcArgs g) {
  extern __shared__ __align__(128) uint8_t tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_s;
  __shared__ int ok_s;
  if (*(volatile const int*)g.status != 0) return;  // an earlier wait ran out: leave every tile unwritten
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z, bt = z / g.splits, split = z - bt * g.splits;
  const int p0 = blockIdx.y * TM, q0 = blockIdx.x * g.tn;
  const int kchunk = ((g.K + g.splits - 1) / g.splits + TK - 1) / TK * TK;
  const int kb = split * kchunk, ke = min(g.K, kb + kchunk);
  const int nk = ke > kb ? (ke - kb + TK - 1) / TK : 0;
  const long long xb = (long long)bt * g.X.sb, yb = (long long)bt * g.Y.sb;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(TNMAX)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  const uint32_t sbase = smem_u32(tc_smem);
  const uint32_t idesc = tc_idesc(g.tn);

  int issued = 0;  // K steps whose instructions were issued (the same in every thread)
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int k0 = kb + kt * TK;
    float xv[4][8], yv[2][8];  // every load of the step is issued before any is used
    int xo[4], yo[2], xm[4], ym[2];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int r, kg;
      chunk_rk(g.X.rowfast, tid + e * TT, TM - 1, 7, r, kg);
      xo[e] = core_off(r, kg);
      xm[e] = load8(g.X, xb, p0 + r, k0 + kg * 8, ke, xv[e]);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = tid + e * TT;
      yo[e] = -1;
      ym[e] = 0;
      if (c >= g.tn * 4) continue;
      int r, kg;
      chunk_rk(g.Y.rowfast, c, g.tn - 1, g.tn_log2, r, kg);
      yo[e] = core_off(r, kg);
      ym[e] = load8(g.Y, yb, q0 + r, k0 + kg * 8, ke, yv[e]);
    }
    const int s = kt & 1;
    if (kt >= 2) {  // stage s was read by the instructions of step kt - 2
      if (tid == 0) ok_s = mbar_wait_bounded(&mbar[s], ((kt - 2) >> 1) & 1);
      __syncthreads();
      if (!ok_s) {
        ok = false;
        break;
      }
    }
    uint8_t* xs = tc_smem + s * kStage;
    uint8_t* ys = xs + kXBytes;
#pragma unroll
    for (int e = 0; e < 4; ++e) *reinterpret_cast<uint4*>(xs + xo[e]) = pack8(xm[e], xv[e]);
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (yo[e] >= 0) *reinterpret_cast<uint4*>(ys + yo[e]) = pack8(ym[e], yv[e]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stores, before the tensor core reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t xa = sbase + s * kStage, ya = xa + kXBytes;
#pragma unroll
      for (int h = 0; h < 2; ++h)  // K = 16 each: two core matrices in K
        tc_mma(tmem, tc_sdesc(xa + h * 256, 128, 512), tc_sdesc(ya + h * 256, 128, 512), idesc, (kt | h) != 0);
      tc_commit(&mbar[s]);  // arrives once every instruction issued so far is complete
    }
    issued = kt + 1;
  }
  if (ok && issued > 0) {
    if (tid == 0) {
      ok_s = mbar_wait_bounded(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
      if (ok_s && g.stall_test)  // test of the bound: the next phase, which no instruction completes
        ok_s = mbar_wait_bounded(&mbar[(issued - 1) & 1], (((issued - 1) >> 1) + 1) & 1);
    }
    __syncthreads();
    ok = ok_s != 0;
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(g.status, 1);
      if (issued > 0) mbar_wait_bounded(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TNMAX) : "memory");
    return;
  }

  // accumulator -> shared memory (the stages are free: every instruction is complete)
  float* cs = reinterpret_cast<float*>(tc_smem);
  tc_fence_after();
  const int row = warp * 32 + lane;
  for (int cb = 0; cb < g.tn; cb += 16) {
    uint32_t r[16];
    if (issued > 0) {
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, r);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) r[j] = 0u;  // empty K range (a split past K): zero
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) cs[row * kEpiPitch + cb + j] = __uint_as_float(r[j]);
  }
  // Per tile row and per tile column: the output offset and the bias term
  // (the index maps and the bias's division once per row or column, not per
  // element). With split-K the offsets address the partial-sum workspace.
  long long* poff = reinterpret_cast<long long*>(tc_smem + kEpiBytes);
  long long* qoff = poff + TM;
  float* pbias = reinterpret_cast<float*>(qoff + TNMAX);
  float* qbias = pbias + TM;
  {
    const Out& o = g.O;
    const bool spl = g.splits > 1;
    const int p = p0 + tid;  // TT == TM: one tile row per thread
    long long po = 0;
    float pb = 0.f;
    if (p < g.X.rows) {
      if (!g.swap) {  // tile row = output row
        po = spl ? ((long long)z * g.M + p) * g.N : o.r(p);
        if (!spl && o.bias && !o.bias_col) pb = o.bias[(p / o.bdiv) % o.bmod];
      } else {        // tile row = output column
        po = spl ? (long long)p : o.c(p);
        if (!spl && o.bias && o.bias_col) pb = o.bias[p];
      }
    }
    poff[tid] = po;
    pbias[tid] = pb;
    if (tid < g.tn) {
      const int q = q0 + tid;
      long long qo = 0;
      float qb = 0.f;
      if (q < g.Y.rows) {
        if (!g.swap) {
          qo = spl ? (long long)q : o.c(q);
          if (!spl && o.bias && o.bias_col) qb = o.bias[q];
        } else {
          qo = spl ? ((long long)z * g.M + q) * g.N : o.r(q);
          if (!spl && o.bias && !o.bias_col) qb = o.bias[(q / o.bdiv) % o.bmod];
        }
      }
      qoff[tid] = qo;
      qbias[tid] = qb;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TNMAX) : "memory");

  const Out& o = g.O;
  float* const dst = g.splits > 1 ? g.ws : o.p + (long long)bt * o.sb;
  // with split-K the offsets address the workspace and k_gemm_reduce applies beta C: no C here
  const float* const cin =
      (g.splits == 1 && o.beta != 0.f) ? (o.cin ? o.cin : o.p) + (long long)bt * o.sb : nullptr;
  float* const pre = o.pre ? o.pre + (long long)bt * o.sb : nullptr;
  // raw: split-K partial sums, or an epilogue that is the identity
  const bool raw = g.splits > 1 || (o.alpha == 1.f && !cin && !o.bias && o.act != 1);
  // One output element: the epilogue in the order of store_out (alpha A B, + beta C, + bias, then GELU).
  auto emit = [&](long long off, float acc, float c, float bias) {
    if (raw) {
      dst[off] = acc;
      return;
    }
    float v = o.alpha * acc;
    if (cin) v += o.beta * c;
    if (o.bias) v += bias;  // one of the row and column terms is zero
    if (o.act == 1) {
      if (pre) pre[off] = v;
      v = gelu_f(v);
    }
    dst[off] = v;
  };
  // EG elements per thread at a time: their C loads are all in flight before the first use.
  // Consecutive threads run along the output's unit-stride dimension, so each thread keeps one
  // tile row (ifast) or one tile column for the whole tile.
  constexpr int EG = 8;
  if (g.ifast) {
    const int i = tid;  // TT == TM
    const int jn = min(g.tn, g.Y.rows - q0);
    if (p0 + i < g.X.rows) {
      const long long pi = poff[i];
      const float pb = pbias[i];
      for (int j0 = 0; j0 < jn; j0 += EG) {
        long long off[EG];
        float c[EG];
#pragma unroll
        for (int u = 0; u < EG; ++u) {
          const int j = j0 + u;
          off[u] = j < jn ? pi + qoff[j] : 0;
          c[u] = (j < jn && cin) ? cin[off[u]] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < EG; ++u) {
          const int j = j0 + u;
          if (j < jn) emit(off[u], cs[i * kEpiPitch + j], c[u], pb + qbias[j]);
        }
      }
    }
  } else {
    const int j = tid & (g.tn - 1);
    const int istep = TT >> g.tn_log2;  // rows covered by the block per pass: 8, 4 or 2
    const int in = min(TM, g.X.rows - p0);
    if (q0 + j < g.Y.rows) {
      const long long qj = qoff[j];
      const float qb = qbias[j];
      for (int i0 = tid >> g.tn_log2; i0 < in; i0 += istep * EG) {
        long long off[EG];
        float c[EG];
#pragma unroll
        for (int u = 0; u < EG; ++u) {
          const int i = i0 + u * istep;
          off[u] = i < in ? poff[i] + qj : 0;
          c[u] = (i < in && cin) ? cin[off[u]] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < EG; ++u) {
          const int i = i0 + u * istep;
          if (i < in) emit(off[u], cs[i * kEpiPitch + j], c[u], pbias[i] + qb);
        }
      }
    }
  }
}

// One operand of C = A B as the MMA sees it: rows through rm, K through km.
inline Opnd make_opnd(const Mat& m, const Ix& rm, const Ix& km, int rows) {
  Opnd o;
  o.p = m.p;
  o.bf16 = m.bf16;
  o.rm = rm;
  o.km = km;
  o.sb = m.sb;
  o.rows = rows;
  o.kcontig = (km.a == 1 && (km.m == 0 || km.s % 8 == 0)) ? 1 : 0;
  o.rowfast = (!o.kcontig && rm.a == 1) ? 1 : 0;
  return o;
}

// C[b] = alpha A[b] B[b] + beta C[b] (+ epilogue) for b < batch, A M x K, B
// K x N through their index maps; splits > 1 sums K in `splits` chunks through
// ws (batch * splits * M * N floats) in a fixed order. status: a device int
// that a wait which ran out sets to 1.
inline cudaError_t launch_gemm(int M, int N, int K, int batch, const Mat& A, const Mat& B, const Out& O, int splits,
                               float* ws, int* status, cudaStream_t st, int stall_test = 0) {
  TcArgs t;
  t.stall_test = stall_test;
  t.swap = N > M ? 1 : 0;
  if (!t.swap) {
    t.X = make_opnd(A, A.r, A.c, M);
    t.Y = make_opnd(B, B.c, B.r, N);
  } else {
    t.X = make_opnd(B, B.c, B.r, N);
    t.Y = make_opnd(A, A.r, A.c, M);
  }
  const int ps = t.swap ? N : M, qs = t.swap ? M : N;
  t.tn = qs <= 16 ? 16 : (qs <= 32 ? 32 : TNMAX);
  t.tn_log2 = t.tn == 16 ? 4 : (t.tn == 32 ? 5 : 6);
  const bool col_fast = splits > 1 || O.c.a == 1;  // the partial sums are laid out row-major
  const bool row_fast = !col_fast && O.r.a == 1;
  t.ifast = (t.swap ? col_fast : row_fast) ? 1 : 0;
  t.M = M;
  t.N = N;
  t.K = K;
  t.splits = splits;
  t.O = O;
  t.ws = ws;
  t.status = status;
  const dim3 grid((qs + t.tn - 1) / t.tn, (ps + TM - 1) / TM, batch * splits);
  k_gemm_tc<<<grid, TT, kTcSmem, st>>>(t);
  if (splits > 1) k_gemm_reduce<<<1024, 256, 0, st>>>(M, N, batch, splits, ws, O);
  return cudaGetLastError();
}

}  // namespace fno
}  // namespace spfc
