// GPU surrogate network (Fourier neural operator) for the SPFC state: forward,
// backward and Adam, all in this library's kernels. The network's definition
// (and the parameter layout) matches the float64 CPU reference used by the
// tests: lift 4 -> W, L spectral-conv layers (truncated DFT as BF16 GEMMs,
// per-mode complex channel mixing, inverse truncated DFT, plus a 1x1 conv,
// GELU between layers), projection W -> Q -> 1, output phi^n + s (d - mean d).
// Weights are held in float32 (master, for Adam) and bfloat16 (used by every
// product); accumulation is float32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cstdio>

#include "../../include/spfc.h"
#include "spfc_common.cuh"
#include "spfc_internal.h"
#include "spfc_fno_gemm.cuh"

using namespace spfc::fno;

namespace {

constexpr float kScale = 0.1f;

// --------------------------------------------------------------------------
// small kernels
// --------------------------------------------------------------------------

// Per-sample sums of x[b][0..P) in float64 and a fixed order, in two stages
// so that every SM takes part: kSampleChunks contiguous chunks per sample
// (grid (kSampleChunks, B)), then one block per sample sums its chunk
// partials.
constexpr int kSampleChunks = 64;

__global__ void k_sample_part(const float* __restrict__ x, int P, double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const int len = (P + kSampleChunks - 1) / kSampleChunks;
  const int i1 = min(P, (j + 1) * len);
  double s = 0.0;
  for (int p = j * len + threadIdx.x; p < i1; p += blockDim.x) s += (double)x[(long long)b * P + p];
  s = spfc::block_sum(s, red);
  if (threadIdx.x == 0) part[b * kSampleChunks + j] = s;
}

// mean[b] = (sum of the chunk partials of sample b) / P; kSampleChunks threads per block
__global__ void k_sample_final(const double* __restrict__ part, int P, double* __restrict__ mean) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = part[b * kSampleChunks + threadIdx.x];
  s = spfc::block_sum(s, red);
  if (threadIdx.x == 0) mean[b] = s / P;
}

// features a[b][j][p] and the lift v0[b][c][p] = sum_j Lw[c][j] a[b][j][p] + Lb[c]
__global__ void k_features_lift(int B, int P, int W, const float* __restrict__ phi_n, const float* __restrict__ phi_nm1,
                                const float* __restrict__ eps, const float* __restrict__ beta,
                                const double* __restrict__ mean, const __nv_bfloat16* __restrict__ Lw,
                                const __nv_bfloat16* __restrict__ Lb, float* __restrict__ a, float* __restrict__ v0) {
  const long long total = (long long)B * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / P), p = (int)(i % P);
    const float m = (float)mean[b];
    float f[4];
    f[0] = (phi_n[i] - m) / kScale;
    f[1] = (phi_nm1[i] - m) / kScale;
    f[2] = eps[b];
    f[3] = beta[b];
    for (int j = 0; j < 4; ++j) a[((long long)b * 4 + j) * P + p] = f[j];
    for (int c = 0; c < W; ++c) {
      float s = __bfloat162float(Lb[c]);
      for (int j = 0; j < 4; ++j) s += __bfloat162float(Lw[c * 4 + j]) * f[j];
      v0[((long long)b * W + c) * P + p] = s;
    }
  }
}

// Per-mode complex channel mixing. Vh, Oh: [b*W + ch][2*KY][m1] with the real
// part at row k and the imaginary part at row KY + k; R (bf16): Rr, Ri [i][o][KY][m1].
// One block per mode.
__global__ void k_mix_fwd(int B, int W, int KY, int m1, const float* __restrict__ Vh, const __nv_bfloat16* __restrict__ Rr,
                          const __nv_bfloat16* __restrict__ Ri, float* __restrict__ Oh) {
  extern __shared__ float sm[];
  const int mode = blockIdx.x, k = mode / m1, kx = mode % m1;
  const int nm = KY * m1;
  float* rr = sm;              // [i][o]
  float* ri = rr + W * W;
  float* vr = ri + W * W;      // [b][i]
  float* vi = vr + B * W;
  for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
    rr[t] = __bfloat162float(Rr[(long long)t * nm + mode]);
    ri[t] = __bfloat162float(Ri[(long long)t * nm + mode]);
  }
  const int rows = 2 * KY;
  for (int t = threadIdx.x; t < B * W; t += blockDim.x) {
    vr[t] = Vh[((long long)t * rows + k) * m1 + kx];
    vi[t] = Vh[((long long)t * rows + KY + k) * m1 + kx];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * W; t += blockDim.x) {
    const int b = t / W, o = t % W;
    float sr = 0.f, si = 0.f;
    for (int i = 0; i < W; ++i) {
      const float a = vr[b * W + i], c = vi[b * W + i], pr = rr[i * W + o], pi = ri[i * W + o];
      sr += a * pr - c * pi;
      si += a * pi + c * pr;
    }
    Oh[((long long)t * rows + k) * m1 + kx] = sr;
    Oh[((long long)t * rows + KY + k) * m1 + kx] = si;
  }
}

// Backward of the mixing: gVh and the gradient of (Rr, Ri) for one mode per block.
__global__ void k_mix_bwd(int B, int W, int KY, int m1, const float* __restrict__ Vh, const __nv_bfloat16* __restrict__ Rr,
                          const __nv_bfloat16* __restrict__ Ri, const float* __restrict__ gOh, float* __restrict__ gVh,
                          float* __restrict__ gRr, float* __restrict__ gRi) {
  extern __shared__ float sm[];
  const int mode = blockIdx.x, k = mode / m1, kx = mode % m1;
  const int nm = KY * m1, rows = 2 * KY;
  float* rr = sm;
  float* ri = rr + W * W;
  float* vr = ri + W * W;
  float* vi = vr + B * W;
  float* gr = vi + B * W;
  float* gi = gr + B * W;
  for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
    rr[t] = __bfloat162float(Rr[(long long)t * nm + mode]);
    ri[t] = __bfloat162float(Ri[(long long)t * nm + mode]);
  }
  for (int t = threadIdx.x; t < B * W; t += blockDim.x) {
    vr[t] = Vh[((long long)t * rows + k) * m1 + kx];
    vi[t] = Vh[((long long)t * rows + KY + k) * m1 + kx];
    gr[t] = gOh[((long long)t * rows + k) * m1 + kx];
    gi[t] = gOh[((long long)t * rows + KY + k) * m1 + kx];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * W; t += blockDim.x) {   // gVh[b][i]
    const int b = t / W, i = t % W;
    float sr = 0.f, si = 0.f;
    for (int o = 0; o < W; ++o) {
      const float a = gr[b * W + o], c = gi[b * W + o], pr = rr[i * W + o], pi = ri[i * W + o];
      sr += a * pr + c * pi;
      si += -a * pi + c * pr;
    }
    gVh[((long long)t * rows + k) * m1 + kx] = sr;
    gVh[((long long)t * rows + KY + k) * m1 + kx] = si;
  }
  for (int t = threadIdx.x; t < W * W; t += blockDim.x) {   // gR[i][o]
    const int i = t / W, o = t % W;
    float sr = 0.f, si = 0.f;
    for (int b = 0; b < B; ++b) {
      const float a = gr[b * W + o], c = gi[b * W + o], xr = vr[b * W + i], xi = vi[b * W + i];
      sr += a * xr + c * xi;
      si += c * xr - a * xi;
    }
    gRr[(long long)t * nm + mode] = sr;
    gRi[(long long)t * nm + mode] = si;
  }
}

// out = phi_n + s (d - mean d)
__global__ void k_output(int B, int P, const float* __restrict__ phi_n, const float* __restrict__ d,
                         const double* __restrict__ dmean, float* __restrict__ out) {
  const long long total = (long long)B * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    out[i] = phi_n[i] + kScale * (d[i] - (float)dmean[i / P]);
}

// Loss and dL/dd of the mean-free residual res = d - mean d - (target - phi^n) / s:
// partial sums over chunks, per-sample totals, then the gradient pass.
__device__ __forceinline__ float loss_res(const float* __restrict__ d, float dm, const float* __restrict__ phi_n,
                                          const float* __restrict__ target, long long i) {
  return d[i] - dm - (target[i] - phi_n[i]) / kScale;
}

// partial sums of the residual and its square per (chunk, sample); grid (kSampleChunks, B)
__global__ void k_loss_part(int P, const float* __restrict__ d, const double* __restrict__ dmean,
                            const float* __restrict__ phi_n, const float* __restrict__ target,
                            double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const float dm = (float)dmean[b];
  const int len = (P + kSampleChunks - 1) / kSampleChunks;
  const int i1 = min(P, (j + 1) * len);
  double s1 = 0.0, s2 = 0.0;
  for (int p = j * len + threadIdx.x; p < i1; p += blockDim.x) {
    const float res = loss_res(d, dm, phi_n, target, (long long)b * P + p);
    s1 += res;
    s2 += (double)res * res;
  }
  s1 = spfc::block_sum(s1, red);
  s2 = spfc::block_sum(s2, red);
  if (threadIdx.x == 0) {
    part[(b * kSampleChunks + j) * 2] = s1;
    part[(b * kSampleChunks + j) * 2 + 1] = s2;
  }
}

// per sample: mean residual and sum of squares from the chunk partials; kSampleChunks threads per block
__global__ void k_loss_final(int P, const double* __restrict__ part, double* __restrict__ mres,
                             double* __restrict__ loss_b) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s1 = part[(b * kSampleChunks + threadIdx.x) * 2], s2 = part[(b * kSampleChunks + threadIdx.x) * 2 + 1];
  s1 = spfc::block_sum(s1, red);
  s2 = spfc::block_sum(s2, red);
  if (threadIdx.x == 0) {
    mres[b] = s1 / P;
    loss_b[b] = s2;
  }
}

// gradient of the mean-square loss of the mean-free residual
__global__ void k_loss_grad(int B, int P, float inv_cnt, const float* __restrict__ d, const double* __restrict__ dmean,
                            const double* __restrict__ mres, const float* __restrict__ phi_n,
                            const float* __restrict__ target, float* __restrict__ gd) {
  const long long total = (long long)B * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / P);
    const float res = loss_res(d, (float)dmean[b], phi_n, target, i);
    gd[i] = 2.f * inv_cnt * (res - (float)mres[b]);
  }
}

// gz[b][q][p] = q2w[q] gd[b][p] gelu'(z[b][q][p])
// grid (x: chunks of the P points, y: b * Q + q)
__global__ void k_proj_back(int Q, int P, const float* __restrict__ gd, const __nv_bfloat16* __restrict__ q2w,
                            const float* __restrict__ z, float* __restrict__ gz) {
  const int bq = blockIdx.y, b = bq / Q, q = bq - b * Q;
  const float w = __bfloat162float(q2w[q]);
  const long long o = (long long)bq * P, ob = (long long)b * P;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    gz[o + p] = w * gd[ob + p] * gelu_grad_f(z[o + p]);
}

// g *= gelu'(u)
__global__ void k_gelu_back(long long n, const float* __restrict__ u, float* __restrict__ g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    g[i] *= gelu_grad_f(u[i]);
}

// out[c] = sum_{b,p} X[b][c][p] in two fixed-order stages: one block per
// (quarter of the points, sample, channel) into part[c][b][quarter], then
// one block per channel sums its parts.
constexpr int kBiasSplit = 4;  // blocks per (channel, sample): P / 4 contiguous points each

// grid (kBiasSplit, B, C): the sum of X[b][c][s P/4 .. (s+1) P/4) (P a
// multiple of 16, X 16-byte aligned), fixed order: each thread sums its
// float4s in four float32 partials (a few dozen values each; float64 per
// element would make the FP64 pipe the bound), then float64 across threads.
__global__ void k_bias_grad_part(int B, int C, int P, const float* __restrict__ X, double* __restrict__ part) {
  __shared__ double red[32];
  const int sp = blockIdx.x, b = blockIdx.y, c = blockIdx.z;
  const int len4 = P / (4 * kBiasSplit);
  const float4* x4 = reinterpret_cast<const float4*>(X + ((long long)b * C + c) * P) + (long long)sp * len4;
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int i = threadIdx.x; i < len4; i += blockDim.x) {
    const float4 v = x4[i];
    a.x += v.x;
    a.y += v.y;
    a.z += v.z;
    a.w += v.w;
  }
  double s = ((double)a.x + (double)a.y) + ((double)a.z + (double)a.w);
  s = spfc::block_sum(s, red);
  if (threadIdx.x == 0) part[((long long)c * B + b) * kBiasSplit + sp] = s;
}

// out[c] = the sum of channel c's B * kBiasSplit partials (<= blockDim.x), fixed order
__global__ void k_bias_grad_final(int n, const double* __restrict__ part, float* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = threadIdx.x < n ? part[(long long)c * n + threadIdx.x] : 0.0;
  s = spfc::block_sum(s, red);
  if (threadIdx.x == 0) out[c] = (float)s;
}

// Adam (Kingma & Ba) on the float32 master weights, then the bfloat16 copy.
__global__ void k_adam(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float wd, float c1, float c2,
                       __nv_bfloat16* __restrict__ wbf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] + wd * w[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wn = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wn;
    wbf[i] = __float2bfloat16_rn(wn);
  }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wbf[i] = __float2bfloat16_rn(w[i]);
}

Ix ix(long long a, int s = 0x7fffffff, long long b = 0) { return make_ix(a, s, b); }

}  // namespace

struct spfc_fno_s {
  int n, W, m1, m2, KY, L, Q, Bmax, P;
  cudaStream_t st;
  std::string err;
  // parameters (float32 master, bfloat16 copy, gradient, Adam moments)
  long long np = 0;
  float *w = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;
  __nv_bfloat16* wbf = nullptr;
  long long adam_t = 0;
  long long o_lw, o_lb, o_q1w, o_q1b, o_q2w, o_q2b;
  std::vector<long long> o_rr, o_ri, o_W, o_b;
  // tables
  float *Fx = nullptr, *Fy = nullptr, *Gy = nullptr, *Gx = nullptr;
  // activations and work
  float *a = nullptr, *z = nullptr, *q = nullptr, *d = nullptr, *Xf = nullptr, *Oh = nullptr, *Zb = nullptr;
  std::vector<float*> v, u, Vh;
  float *eps_d = nullptr, *beta_d = nullptr, *ws = nullptr, *out = nullptr;
  double *mean = nullptr, *dmean = nullptr, *lossb = nullptr, *bpart = nullptr, *spart = nullptr, *mres = nullptr;
  int* gstat = nullptr;  // set to 1 by a GEMM whose bounded wait ran out
  // gradients of activations
  float *gd = nullptr, *gz = nullptr, *gv0 = nullptr, *gv1 = nullptr, *gu = nullptr, *gXf = nullptr, *gVh = nullptr,
        *gOh = nullptr, *gZ = nullptr;
  long long ws_elems = 0;
  std::vector<void*> allocs;

  ~spfc_fno_s() {
    for (void* p : allocs) cudaFree(p);
  }

  template <typename T> int alloc(T** p, long long n_elems) {
    cudaError_t e = cudaMalloc((void**)p, (size_t)n_elems * sizeof(T));
    if (e != cudaSuccess) { err = std::string("allocation: ") + cudaGetErrorString(e); return SPFC_ENOMEM; }
    allocs.push_back(*p);
    return 0;
  }

  int ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) { err = std::string(what) + ": " + cudaGetErrorString(e); return SPFC_ECUDA; }
    return 0;
  }

  int gemm(int M, int N, int K, int batch, const Mat& A, const Mat& B, const Out& O, int splits = 1) {
    while (splits > 1 && (long long)batch * splits * M * N > ws_elems) splits /= 2;
    return ck(launch_gemm(M, N, K, batch, A, B, O, splits, ws, gstat, st), "gemm");
  }

  // The GEMMs' latched status (a bounded tensor-core wait that ran out),
  // read with the stream's work so far.
  int check_status() {
    int h = 0;
    int rc = ck(cudaMemcpyAsync(&h, gstat, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    if (!rc) rc = ck(cudaStreamSynchronize(st), "sync");
    if (!rc && h != 0) {
      err = "tensor-core GEMM: a bounded wait ran out";
      rc = SPFC_ETIMEOUT;
    }
    return rc;
  }

  Mat mf(const float* p, Ix r, Ix c, long long sb = 0) {
    Mat m;
    m.p = p;
    m.bf16 = 0;
    m.r = r;
    m.c = c;
    m.sb = sb;
    return m;
  }
  Mat mb(long long off, Ix r, Ix c) {
    Mat m;
    m.p = wbf + off;
    m.bf16 = 1;
    m.r = r;
    m.c = c;
    m.sb = 0;
    return m;
  }
  Out of(float* p, Ix r, Ix c, long long sb = 0) {
    Out o;
    o.p = p;
    o.r = r;
    o.c = c;
    o.sb = sb;
    return o;
  }

  int setup() {
    P = n * n;
    KY = 2 * m2;
    // parameter layout (same order as the CPU reference)
    long long o = 0;
    o_lw = o; o += (long long)W * 4;
    o_lb = o; o += W;
    for (int l = 0; l < L; ++l) {
      o_rr.push_back(o); o += (long long)W * W * KY * m1;
      o_ri.push_back(o); o += (long long)W * W * KY * m1;
      o_W.push_back(o); o += (long long)W * W;
      o_b.push_back(o); o += W;
    }
    o_q1w = o; o += (long long)Q * W;
    o_q1b = o; o += Q;
    o_q2w = o; o += Q;
    o_q2b = o; o += 1;
    np = o;
    int rc = 0;
    if ((rc = alloc(&w, np)) || (rc = alloc(&g, np)) || (rc = alloc(&am, np)) || (rc = alloc(&av, np)) ||
        (rc = alloc(&wbf, np)))
      return rc;
    if ((rc = ck(cudaMemset(w, 0, np * 4), "memset")) || (rc = ck(cudaMemset(g, 0, np * 4), "memset")) ||
        (rc = ck(cudaMemset(am, 0, np * 4), "memset")) || (rc = ck(cudaMemset(av, 0, np * 4), "memset")) ||
        (rc = ck(cudaMemset(wbf, 0, np * 2), "memset")))
      return rc;
    // DFT tables
    std::vector<float> fx(2LL * n * m1), fy(2LL * KY * 2 * n), gy(2LL * n * 2 * KY), gx(2LL * m1 * n);
    auto kyv = [&](int i) { return i < m2 ? i : n - KY + i; };
    const double tp = 2.0 * M_PI / n;
    for (int x = 0; x < n; ++x)
      for (int kx = 0; kx < m1; ++kx) {
        fx[(size_t)x * m1 + kx] = (float)std::cos(tp * ((long long)kx * x % n));
        fx[(size_t)n * m1 + (size_t)x * m1 + kx] = (float)-std::sin(tp * ((long long)kx * x % n));
      }
    for (int i = 0; i < KY; ++i)
      for (int y = 0; y < n; ++y) {
        const double th = tp * ((long long)kyv(i) * y % n);
        const float c = (float)std::cos(th), s = (float)std::sin(th);
        fy[(size_t)i * 2 * n + y] = c;             // Re rows: [C, S]
        fy[(size_t)i * 2 * n + n + y] = s;
        fy[(size_t)(KY + i) * 2 * n + y] = -s;     // Im rows: [-S, C]
        fy[(size_t)(KY + i) * 2 * n + n + y] = c;
        gy[(size_t)y * 2 * KY + i] = c;            // Zr = C' Or - S' Oi
        gy[(size_t)y * 2 * KY + KY + i] = -s;
        gy[(size_t)(n + y) * 2 * KY + i] = s;      // Zi = S' Or + C' Oi
        gy[(size_t)(n + y) * 2 * KY + KY + i] = c;
      }
    for (int kx = 0; kx < m1; ++kx)
      for (int x = 0; x < n; ++x) {
        const double th = tp * ((long long)kx * x % n);
        const double wgt = (kx == 0 ? 1.0 : 2.0) / ((double)n * n);
        gx[(size_t)kx * n + x] = (float)(wgt * std::cos(th));
        gx[(size_t)(m1 + kx) * n + x] = (float)(-wgt * std::sin(th));
      }
    if ((rc = alloc(&Fx, fx.size())) || (rc = alloc(&Fy, fy.size())) || (rc = alloc(&Gy, gy.size())) ||
        (rc = alloc(&Gx, gx.size())))
      return rc;
    if ((rc = ck(cudaMemcpy(Fx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice), "tables")) ||
        (rc = ck(cudaMemcpy(Fy, fy.data(), fy.size() * 4, cudaMemcpyHostToDevice), "tables")) ||
        (rc = ck(cudaMemcpy(Gy, gy.size() ? gy.data() : nullptr, gy.size() * 4, cudaMemcpyHostToDevice), "tables")) ||
        (rc = ck(cudaMemcpy(Gx, gx.data(), gx.size() * 4, cudaMemcpyHostToDevice), "tables")))
      return rc;
    // activations
    const long long BWP = (long long)Bmax * W * P, BQP = (long long)Bmax * Q * P;
    const long long spec = (long long)Bmax * W * 2 * n * m1, mix = (long long)Bmax * W * 2 * KY * m1;
    v.assign(L + 1, nullptr);
    u.assign(L, nullptr);
    Vh.assign(L, nullptr);
    for (int l = 0; l <= L; ++l)
      if ((rc = alloc(&v[l], BWP))) return rc;
    for (int l = 0; l < L; ++l)
      if ((rc = alloc(&u[l], BWP)) || (rc = alloc(&Vh[l], mix))) return rc;
    if ((rc = alloc(&a, (long long)Bmax * 4 * P)) || (rc = alloc(&z, BQP)) || (rc = alloc(&q, BQP)) ||
        (rc = alloc(&d, (long long)Bmax * P)) || (rc = alloc(&out, (long long)Bmax * P)) || (rc = alloc(&Xf, spec)) ||
        (rc = alloc(&Oh, mix)) || (rc = alloc(&Zb, spec)) || (rc = alloc(&eps_d, Bmax)) || (rc = alloc(&beta_d, Bmax)) ||
        (rc = alloc(&mean, Bmax)) || (rc = alloc(&dmean, Bmax)) || (rc = alloc(&lossb, Bmax)) ||
        (rc = alloc(&spart, 2LL * Bmax * kSampleChunks)) || (rc = alloc(&mres, Bmax)))
      return rc;
    if ((rc = alloc(&gd, (long long)Bmax * P)) || (rc = alloc(&gz, BQP)) || (rc = alloc(&gv0, BWP)) ||
        (rc = alloc(&gv1, BWP)) || (rc = alloc(&gu, BWP)) || (rc = alloc(&gXf, spec)) || (rc = alloc(&gVh, mix)) ||
        (rc = alloc(&gOh, mix)) || (rc = alloc(&gZ, spec)))
      return rc;
    ws_elems = 4LL << 20;  // split-K partial tiles of the weight-gradient GEMMs (M, N <= 64)
    if ((rc = alloc(&ws, ws_elems)) || (rc = alloc(&bpart, 64LL * 64 * kBiasSplit)) || (rc = alloc(&gstat, 1)))
      return rc;
    if ((rc = ck(cudaMemset(gstat, 0, sizeof(int)), "memset"))) return rc;
    const size_t smix = (size_t)(2 * W * W + 4 * Bmax * W) * sizeof(float);
    if (smix > 48 * 1024) {
      if ((rc = ck(cudaFuncSetAttribute(k_mix_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smix), "attr")) ||
          (rc = ck(cudaFuncSetAttribute(k_mix_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smix), "attr")))
        return rc;
    }
    return 0;
  }

  void sample_mean(int B, const float* x, double* out) {
    k_sample_part<<<dim3(kSampleChunks, B), 256, 0, st>>>(x, P, spart);
    k_sample_final<<<B, kSampleChunks, 0, st>>>(spart, P, out);
  }

  int gs(long long n_el) const { return (int)std::min<long long>((n_el + 255) / 256, 4096); }

  // forward pass for B samples already in phi_n / phi_nm1 device buffers (float)
  int forward(int B, const float* phi_n, const float* phi_nm1) {
    int rc;
    sample_mean(B, phi_n, mean);
    k_features_lift<<<gs((long long)B * P), 256, 0, st>>>(B, P, W, phi_n, phi_nm1, eps_d, beta_d, mean, wbf + o_lw,
                                                           wbf + o_lb, a, v[0]);
    if ((rc = ck(cudaGetLastError(), "lift"))) return rc;
    const long long WP = (long long)W * P, sp = 2LL * n * m1, mx = 2LL * KY * m1;
    for (int l = 0; l < L; ++l) {
      // truncated DFT along x: Xf[bc][part][y][kx] = sum_x v[bc][y][x] Fx[part][x][kx]
      if ((rc = gemm(B * W * n, 2 * m1, n, 1, mf(v[l], ix(n), ix(1)), mf(Fx, ix(m1), ix(1, m1, (long long)n * m1)),
                     of(Xf, ix(m1, n, sp), ix(1, m1, (long long)n * m1)))))
        return rc;
      // along y: Vh[bc] (2KY x m1) = Fy (2KY x 2n) Xf[bc] (2n x m1)
      if ((rc = gemm(2 * KY, m1, 2 * n, B * W, mf(Fy, ix(2 * n), ix(1)), mf(Xf, ix(m1), ix(1), sp),
                     of(Vh[l], ix(m1), ix(1), mx))))
        return rc;
      k_mix_fwd<<<KY * m1, 256, (2 * W * W + 2 * B * W) * sizeof(float), st>>>(B, W, KY, m1, Vh[l], wbf + o_rr[l],
                                                                              wbf + o_ri[l], Oh);
      if ((rc = ck(cudaGetLastError(), "mix"))) return rc;
      // inverse along y: Z[bo] (2n x m1) = Gy (2n x 2KY) Oh[bo] (2KY x m1)
      if ((rc = gemm(2 * n, m1, 2 * KY, B * W, mf(Gy, ix(2 * KY), ix(1)), mf(Oh, ix(m1), ix(1), mx),
                     of(Zb, ix(m1), ix(1), sp))))
        return rc;
      // 1x1 conv: u[b] = W_l v[b]
      if ((rc = gemm(W, P, W, B, mb(o_W[l], ix(W), ix(1)), mf(v[l], ix(P), ix(1), WP), of(u[l], ix(P), ix(1), WP))))
        return rc;
      // inverse along x accumulated onto the 1x1 conv in the epilogue, with the
      // bias (row = (b W + o) n + y): u = pre-activation, v[l+1] = gelu(u)
      // (no activation on the last layer)
      {
        Out O = of(v[l + 1], ix(n), ix(1));
        O.cin = u[l];
        O.beta = 1.f;
        O.bias = w + o_b[l];
        O.bdiv = n;
        O.bmod = W;
        if (l < L - 1) {
          O.act = 1;
          O.pre = u[l];
        }
        if ((rc = gemm(B * W * n, n, 2 * m1, 1, mf(Zb, ix(m1, n, sp), ix(1, m1, (long long)n * m1)),
                       mf(Gx, ix(n), ix(1)), O)))
          return rc;
      }
    }
    // projection
    {
      Out O1 = of(q, ix(P), ix(1), (long long)Q * P);
      O1.bias = w + o_q1b;
      O1.bdiv = 1;
      O1.bmod = Q;
      O1.act = 1;
      O1.pre = z;
      if ((rc = gemm(Q, P, W, B, mb(o_q1w, ix(W), ix(1)), mf(v[L], ix(P), ix(1), WP), O1))) return rc;
      Out O2 = of(d, ix(P), ix(1), P);
      O2.bias = w + o_q2b;
      O2.bdiv = 1;
      O2.bmod = 1;
      if ((rc = gemm(1, P, Q, B, mb(o_q2w, ix(Q), ix(1)), mf(q, ix(P), ix(1), (long long)Q * P), O2))) return rc;
    }
    sample_mean(B, d, dmean);
    return ck(cudaGetLastError(), "forward");
  }

  void bias_grad(int B, int C, const float* X, float* out) {
    k_bias_grad_part<<<dim3(kBiasSplit, B, C), 256, 0, st>>>(B, C, P, X, bpart);
    k_bias_grad_final<<<C, 256, 0, st>>>(B * kBiasSplit, bpart, out);
  }

  // dL/d(parameters) for the B samples of the last forward pass, given gd = dL/dd
  int backward(int B) {
    int rc;
    const long long WP = (long long)W * P, QP = (long long)Q * P, sp = 2LL * n * m1, mx = 2LL * KY * m1;
    const int BP = B * P;
    const int splits = std::min(1024, std::max(1, BP / 1024));
    // projection: d = q2w q + q2b, q = gelu(z), z = q1w v_L + q1b
    {
      Out O = of(g + o_q2w, ix(1), ix(1));
      if ((rc = gemm(1, Q, BP, 1, mf(gd, ix(0), ix(1)), mf(q, ix(1, P, QP), ix(P)), O, splits))) return rc;
      bias_grad(B, 1, gd, g + o_q2b);
      k_proj_back<<<dim3(std::min((P + 255) / 256, 64), B * Q), 256, 0, st>>>(Q, P, gd, wbf + o_q2w, z, gz);
      if ((rc = ck(cudaGetLastError(), "proj_back"))) return rc;
      Out O1 = of(g + o_q1w, ix(W), ix(1));
      if ((rc = gemm(Q, W, BP, 1, mf(gz, ix(P), ix(1, P, QP)), mf(v[L], ix(1, P, WP), ix(P)), O1, splits))) return rc;
      bias_grad(B, Q, gz, g + o_q1b);
      // gv = q1w^T gz
      if ((rc = gemm(W, P, Q, B, mb(o_q1w, ix(1), ix(W)), mf(gz, ix(P), ix(1), QP), of(gv0, ix(P), ix(1), WP))))
        return rc;
    }
    float* gv = gv0;
    float* gvn = gv1;
    for (int l = L - 1; l >= 0; --l) {
      // gu = gv * gelu'(u) (the last layer has no activation)
      if ((rc = ck(cudaMemcpyAsync(gu, gv, (size_t)B * WP * 4, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
      if (l < L - 1) k_gelu_back<<<gs((long long)B * WP), 256, 0, st>>>((long long)B * WP, u[l], gu);
      bias_grad(B, W, gu, g + o_b[l]);
      if ((rc = ck(cudaGetLastError(), "gelu_back"))) return rc;
      // 1x1 conv: dW = sum_b gu[b] v[b]^T; gvn = W^T gu
      if ((rc = gemm(W, W, BP, 1, mf(gu, ix(P), ix(1, P, WP)), mf(v[l], ix(1, P, WP), ix(P)),
                     of(g + o_W[l], ix(W), ix(1)), splits)))
        return rc;
      if ((rc = gemm(W, P, W, B, mb(o_W[l], ix(1), ix(W)), mf(gu, ix(P), ix(1), WP), of(gvn, ix(P), ix(1), WP))))
        return rc;
      // adjoint of the inverse along x: gZ[bo][part][y][kx] = sum_x gu[bo][y][x] Gx[part kx][x]
      if ((rc = gemm(B * W * n, 2 * m1, n, 1, mf(gu, ix(n), ix(1)), mf(Gx, ix(1), ix(n)),
                     of(gZ, ix(m1, n, sp), ix(1, m1, (long long)n * m1)))))
        return rc;
      // adjoint of the inverse along y: gOh[bo] = Gy^T gZ[bo]
      if ((rc = gemm(2 * KY, m1, 2 * n, B * W, mf(Gy, ix(1), ix(2 * KY)), mf(gZ, ix(m1), ix(1), sp),
                     of(gOh, ix(m1), ix(1), mx))))
        return rc;
      k_mix_bwd<<<KY * m1, 256, (2 * W * W + 4 * B * W) * sizeof(float), st>>>(B, W, KY, m1, Vh[l], wbf + o_rr[l],
                                                                              wbf + o_ri[l], gOh, gVh, g + o_rr[l],
                                                                              g + o_ri[l]);
      if ((rc = ck(cudaGetLastError(), "mix_bwd"))) return rc;
      // adjoint of the DFT along y: gXf[bc] = Fy^T gVh[bc]
      if ((rc = gemm(2 * n, m1, 2 * KY, B * W, mf(Fy, ix(1), ix(2 * n)), mf(gVh, ix(m1), ix(1), mx),
                     of(gXf, ix(m1), ix(1), sp))))
        return rc;
      // adjoint of the DFT along x, accumulated onto gvn: gvn[bc][y][x] += sum_j gXf[bc][j][y] Fx[j][x]
      {
        Out O = of(gvn, ix(n), ix(1));
        O.beta = 1.f;
        if ((rc = gemm(B * W * n, n, 2 * m1, 1, mf(gXf, ix(m1, n, sp), ix(1, m1, (long long)n * m1)),
                       mf(Fx, ix(1, m1, (long long)n * m1), ix(m1)), O)))
          return rc;
      }
      std::swap(gv, gvn);
    }
    // lift: v0 = Lw a + Lb
    if ((rc = gemm(W, 4, BP, 1, mf(gv, ix(P), ix(1, P, WP)), mf(a, ix(1, P, 4LL * P), ix(P)),
                   of(g + o_lw, ix(4), ix(1)), splits)))
      return rc;
    bias_grad(B, W, gv, g + o_lb);
    return ck(cudaGetLastError(), "backward");
  }

  int load_inputs(int B, const double* eps, const double* beta) {
    if (B < 1 || B > Bmax) { err = "batch size out of range"; return SPFC_EINVAL; }
    std::vector<float> e(B), bt(B);
    for (int i = 0; i < B; ++i) { e[i] = (float)eps[i]; bt[i] = (float)beta[i]; }
    int rc = ck(cudaMemcpyAsync(eps_d, e.data(), B * 4, cudaMemcpyHostToDevice, st), "eps");
    if (!rc) rc = ck(cudaMemcpyAsync(beta_d, bt.data(), B * 4, cudaMemcpyHostToDevice, st), "beta");
    if (!rc) rc = check_status();  // also reports a wait that ran out in an earlier call
    return rc;
  }
};

static thread_local std::string g_fno_err;

void spfc::fno_shape(const spfc_fno_s* f, int* n, int* max_batch, cudaStream_t* st) {
  *n = f->n;
  *max_batch = f->Bmax;
  *st = f->st;
}

// Weight file: magic, int32 {n, width, modes1, modes2, layers, proj}, int64
// parameter count, then the float32 parameters in the documented order.
static const char kFnoMagic[8] = {'S', 'P', 'F', 'C', 'F', 'N', 'O', '1'};

extern "C" {

int spfc_fno_create(int n, int width, int modes1, int modes2, int layers, int proj, int max_batch, void* stream,
                    spfc_fno_t* out) {
  if (!out) { g_fno_err = "out is NULL"; return SPFC_EINVAL; }
  *out = nullptr;
  if (n < 16 || (n & (n - 1)) || width < 1 || width > 64 || modes1 < 1 || modes1 > n / 2 || modes2 < 1 ||
      2 * modes2 > n || layers < 1 || layers > 16 || proj < 1 || proj > 64 || max_batch < 1 || max_batch > 64) {
    g_fno_err = "invalid network size (n power of two >= 16, width and proj <= 64, batch <= 64)";
    return SPFC_EINVAL;
  }
  auto* f = new spfc_fno_s();
  f->n = n; f->W = width; f->m1 = modes1; f->m2 = modes2; f->L = layers; f->Q = proj; f->Bmax = max_batch;
  f->st = (cudaStream_t)stream;
  int rc = f->setup();
  if (rc) { g_fno_err = f->err; delete f; return rc; }
  *out = f;
  return SPFC_OK;
}

int64_t spfc_fno_num_params(spfc_fno_t f) { return f ? f->np : 0; }

int spfc_fno_save(spfc_fno_t f, const char* path) {
  if (!f || !path) return SPFC_EINVAL;
  std::vector<float> w((size_t)f->np);
  int rc = spfc_fno_get_params(f, w.data());
  if (rc) return rc;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) { f->err = std::string("cannot open ") + path; return SPFC_EINVAL; }
  const int32_t hdr[6] = {f->n, f->W, f->m1, f->m2, f->L, f->Q};
  const int64_t cnt = f->np;
  bool ok = std::fwrite(kFnoMagic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 &&
            std::fwrite(&cnt, sizeof(cnt), 1, fp) == 1 && std::fwrite(w.data(), 4, w.size(), fp) == w.size();
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) { f->err = std::string("write failed: ") + path; return SPFC_EINVAL; }
  return SPFC_OK;
}

int spfc_fno_load(spfc_fno_t f, const char* path) {
  if (!f || !path) return SPFC_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) { f->err = std::string("cannot open ") + path; return SPFC_EINVAL; }
  char magic[8];
  int32_t hdr[6];
  int64_t cnt = 0;
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kFnoMagic, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, fp) == 1 && std::fread(&cnt, sizeof(cnt), 1, fp) == 1;
  const int32_t want[6] = {f->n, f->W, f->m1, f->m2, f->L, f->Q};
  if (!ok || std::memcmp(hdr, want, sizeof(hdr)) != 0 || cnt != f->np) {
    std::fclose(fp);
    f->err = "weight file does not match this network (grid size, width, modes, layers or projection)";
    return SPFC_EINVAL;
  }
  std::vector<float> w((size_t)cnt);
  ok = std::fread(w.data(), 4, w.size(), fp) == w.size();
  std::fclose(fp);
  if (!ok) { f->err = "truncated weight file"; return SPFC_EINVAL; }
  return spfc_fno_set_params(f, w.data());
}

int spfc_fno_set_params(spfc_fno_t f, const float* host) {
  if (!f || !host) return SPFC_EINVAL;
  int rc = f->ck(cudaMemcpyAsync(f->w, host, f->np * 4, cudaMemcpyHostToDevice, f->st), "set_params");
  if (rc) return rc;
  k_to_bf16<<<f->gs(f->np), 256, 0, f->st>>>(f->np, f->w, f->wbf);
  rc = f->ck(cudaMemsetAsync(f->am, 0, f->np * 4, f->st), "reset");
  if (!rc) rc = f->ck(cudaMemsetAsync(f->av, 0, f->np * 4, f->st), "reset");
  f->adam_t = 0;
  if (!rc) rc = f->ck(cudaStreamSynchronize(f->st), "sync");
  return rc;
}

int spfc_fno_get_params(spfc_fno_t f, float* host) {
  if (!f || !host) return SPFC_EINVAL;
  int rc = f->ck(cudaMemcpyAsync(host, f->w, f->np * 4, cudaMemcpyDeviceToHost, f->st), "get_params");
  if (!rc) rc = f->ck(cudaStreamSynchronize(f->st), "sync");
  return rc;
}

int spfc_fno_predict(spfc_fno_t f, int batch, const float* phi_n, const float* phi_nm1, const double* eps,
                     const double* beta, float* out) {
  if (!f || !phi_n || !phi_nm1 || !eps || !beta || !out) return SPFC_EINVAL;
  int rc = f->load_inputs(batch, eps, beta);
  if (!rc) rc = f->forward(batch, phi_n, phi_nm1);
  if (rc) return rc;
  k_output<<<f->gs((long long)batch * f->P), 256, 0, f->st>>>(batch, f->P, phi_n, f->d, f->dmean, out);
  return f->ck(cudaGetLastError(), "output");
}

int spfc_fno_loss_grad(spfc_fno_t f, int batch, const float* phi_n, const float* phi_nm1, const double* eps,
                       const double* beta, const float* target, double* loss, float* grad_host) {
  if (!f || !phi_n || !phi_nm1 || !eps || !beta || !target) return SPFC_EINVAL;
  int rc = f->load_inputs(batch, eps, beta);
  if (!rc) rc = f->forward(batch, phi_n, phi_nm1);
  if (rc) return rc;
  const float inv_cnt = 1.f / ((float)batch * f->P);
  k_loss_part<<<dim3(kSampleChunks, batch), 256, 0, f->st>>>(f->P, f->d, f->dmean, phi_n, target, f->spart);
  k_loss_final<<<batch, kSampleChunks, 0, f->st>>>(f->P, f->spart, f->mres, f->lossb);
  k_loss_grad<<<f->gs((long long)batch * f->P), 256, 0, f->st>>>(batch, f->P, inv_cnt, f->d, f->dmean, f->mres, phi_n,
                                                                  target, f->gd);
  if ((rc = f->ck(cudaGetLastError(), "loss"))) return rc;
  if ((rc = f->backward(batch))) return rc;
  std::vector<double> lb(batch);
  if ((rc = f->ck(cudaMemcpyAsync(lb.data(), f->lossb, batch * 8, cudaMemcpyDeviceToHost, f->st), "loss"))) return rc;
  if (grad_host && (rc = f->ck(cudaMemcpyAsync(grad_host, f->g, f->np * 4, cudaMemcpyDeviceToHost, f->st), "grad")))
    return rc;
  if ((rc = f->check_status())) return rc;
  double s = 0.0;
  for (double x : lb) s += x;
  if (loss) *loss = s / ((double)batch * f->P);
  return SPFC_OK;
}

int spfc_fno_adam_step(spfc_fno_t f, float lr, float beta1, float beta2, float epsilon, float weight_decay) {
  if (!f) return SPFC_EINVAL;
  f->adam_t += 1;
  const float c1 = 1.f - std::pow(beta1, (float)f->adam_t), c2 = 1.f - std::pow(beta2, (float)f->adam_t);
  k_adam<<<f->gs(f->np), 256, 0, f->st>>>(f->np, f->w, f->g, f->am, f->av, lr, beta1, beta2, epsilon, weight_decay, c1,
                                          c2, f->wbf);
  return f->ck(cudaGetLastError(), "adam");
}

void spfc_fno_destroy(spfc_fno_t f) { delete f; }

int spfc_gemm_selftest(int M, int N, int K, int batch, int splits, int flags, const float* A, const float* B,
                       float* C, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || batch < 1 || splits < 1 || splits > 1024 || (flags & ~15))
    return SPFC_EINVAL;
  const long long na = (long long)batch * M * K, nb = (long long)batch * K * N, nc = (long long)batch * M * N;
  if (na > (1ll << 26) || nb > (1ll << 26) || nc * splits > (1ll << 26)) return SPFC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const bool a_bf16 = flags & 1, a_t = flags & 2, b_t = flags & 4;
  // host copies in the requested storage: A column-major per batch (a_t), B column-major (b_t)
  std::vector<float> ha((size_t)na), hb((size_t)nb);
  for (long long b = 0; b < batch; ++b)
    for (int m = 0; m < M; ++m)
      for (int k = 0; k < K; ++k)
        ha[(size_t)(b * M * K + (a_t ? (long long)k * M + m : (long long)m * K + k))] = A[b * M * K + (long long)m * K + k];
  for (long long b = 0; b < batch; ++b)
    for (int k = 0; k < K; ++k)
      for (int n = 0; n < N; ++n)
        hb[(size_t)(b * K * N + (b_t ? (long long)n * K + k : (long long)k * N + n))] = B[b * K * N + (long long)k * N + n];
  std::vector<uint16_t> ha16;
  if (a_bf16) {  // round to nearest even, as the kernel's own conversion does
    ha16.resize(ha.size());
    for (size_t i = 0; i < ha.size(); ++i) {
      uint32_t u;
      std::memcpy(&u, &ha[i], 4);
      ha16[i] = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    }
  }
  void* da = nullptr;
  float *db = nullptr, *dc = nullptr, *ws = nullptr;
  int* status = nullptr;
  int rc = SPFC_OK;
  auto fail = [&](cudaError_t e) { return e != cudaSuccess; };
  if (fail(cudaMalloc(&da, (size_t)na * (a_bf16 ? 2 : 4))) || fail(cudaMalloc((void**)&db, (size_t)nb * 4)) ||
      fail(cudaMalloc((void**)&dc, (size_t)nc * 4)) ||
      fail(cudaMalloc((void**)&ws, (size_t)(splits > 1 ? nc * splits : 1) * 4)) ||
      fail(cudaMalloc((void**)&status, sizeof(int))))
    rc = SPFC_ENOMEM;
  int hs = 0;
  if (!rc) {
    cudaError_t e = a_bf16 ? cudaMemcpyAsync(da, ha16.data(), (size_t)na * 2, cudaMemcpyHostToDevice, st)
                           : cudaMemcpyAsync(da, ha.data(), (size_t)na * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, hb.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      Mat ma, mbm;
      ma.p = da;
      ma.bf16 = a_bf16 ? 1 : 0;
      ma.r = a_t ? make_ix(1) : make_ix(K);
      ma.c = a_t ? make_ix(M) : make_ix(1);
      ma.sb = (long long)M * K;
      mbm.p = db;
      mbm.r = b_t ? make_ix(1) : make_ix(N);
      mbm.c = b_t ? make_ix(K) : make_ix(1);
      mbm.sb = (long long)K * N;
      Out o;
      o.p = dc;
      o.r = make_ix(N);
      o.c = make_ix(1);
      o.sb = (long long)M * N;
      e = launch_gemm(M, N, K, batch, ma, mbm, o, splits, ws, status, st, (flags & 8) ? 1 : 0);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(C, dc, (size_t)nc * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = SPFC_ECUDA;
  }
  cudaFree(da);
  cudaFree(db);
  cudaFree(dc);
  cudaFree(ws);
  cudaFree(status);
  if (!rc && hs != 0) rc = SPFC_ETIMEOUT;
  return rc;
}

const char* spfc_fno_last_error(spfc_fno_t f) { return f ? f->err.c_str() : g_fno_err.c_str(); }

}  // extern "C"
