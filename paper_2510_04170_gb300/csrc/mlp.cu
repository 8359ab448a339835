// Learned warm start for Newton: a small MLP maps PDE parameters to an initial
// coefficient vector c_0 (the fallback is c_0 = 0, Alg. 1/Alg. 2's u_0).
//
// Network: x (d_in) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> W3 h2 + b3 (n).
// Arithmetic: inputs, weights and hidden activations rounded to bfloat16, all
// products accumulated in FP32; FP32 master weights updated by Adam.
// Loss (function space): L = (1/B) sum_b (y_b - t_b)^T G (y_b - t_b) with G
// block diagonal (blocks of size gblk, one per subdomain and field), the Gram
// matrix of the features at evaluation points, so the network is judged on
// u = Phi c rather than on the ill-determined coefficients; G = I when null.
//
// Kernels: a tiled FP32-accumulate product with bf16 or FP32 operands (64x64
// tiles, 16-deep K steps), fused bias + tanh + bf16 copy, the block-diagonal
// metric, tanh backward, bias reductions, Adam.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "philox.cuh"
#include "rfm_internal.cuh"

namespace {

constexpr int kLossBlocks = 4096;  // metric blocks per sample held for the loss

__device__ __forceinline__ float ld_op(const float* p) { return *p; }
__device__ __forceinline__ float ld_op(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C(m,n) = beta*C(m,n) + sum_k A(m,k) B(k,n) [+ bias(n)] [tanh]; optional bf16 copy of C.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_mm(const TA* __restrict__ A, long long sam, long long sak,
                                            const TB* __restrict__ B, long long sbk, long long sbn,
                                            float* __restrict__ C, long long scm, long long scn, int M, int N, int K,
                                            float beta, const float* __restrict__ bias, int act,
                                            __nv_bfloat16* __restrict__ Cb) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int idx = tid; idx < 16 * 64; idx += 256) {
      const int kk = idx & 15, mm = idx >> 4;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? ld_op(A + gm * sam + gk * sak) : 0.0f;
      const int nn = idx >> 4;
      const int gn = n0 + nn;
      Bs[kk][nn] = (gn < N && gk < K) ? ld_op(B + gk * sbk + gn * sbn) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty + 16 * i];
        b[i] = Bs[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= M || gn >= N) continue;
      float* cp = C + gm * scm + gn * scn;
      float v = acc[i][j];
      if (beta != 0.0f) v += beta * *cp;
      if (bias) v += bias[gn];
      if (act == 1) v = tanhf(v);
      *cp = v;
      if (Cb) Cb[gm * scm + gn * scn] = __float2bfloat16_rn(v);
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// dY = (2/B) G (Y - T) per sample, G block diagonal with blocks [nb][gblk][gblk];
// also accumulates the loss partial (1/B) sum (Y-T)^T G (Y-T) per block.
__global__ void k_metric(const float* __restrict__ Y, const float* __restrict__ T, int Bsz, int n, const float* __restrict__ G,
                         int gblk, float* __restrict__ dY, float* __restrict__ lossp) {
  // one CTA per (sample, block); thread per output row of the block
  const int b = blockIdx.x, blk = blockIdx.y;
  extern __shared__ float r[];
  const int base = blk * gblk;
  const int len = min(gblk, n - base);  // ragged last block only when G is null
  for (int i = threadIdx.x; i < len; i += blockDim.x) r[i] = Y[(size_t)b * n + base + i] - T[(size_t)b * n + base + i];
  __syncthreads();
  float lp = 0.0f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    float s = 0.0f;
    if (G) {
      const float* g = G + (size_t)blk * gblk * gblk + (size_t)i * gblk;
      for (int j = 0; j < gblk; ++j) s = fmaf(g[j], r[j], s);
    } else {
      s = r[i] / (float)n;
    }
    dY[(size_t)b * n + base + i] = 2.0f * s / (float)Bsz;
    lp += r[i] * s;
  }
  lp = warp_sum((double)lp);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lp;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    lossp[(size_t)b * gridDim.y + blk] = t / (float)Bsz;
  }
}

// dZ = dH * (1 - H^2) (tanh backward), in place on dH; optional bf16 copy.
__global__ void k_tanh_back(float* __restrict__ dH, const float* __restrict__ H, long long n,
                            __nv_bfloat16* __restrict__ dHb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float h = H[i];
    const float v = dH[i] * (1.0f - h * h);
    dH[i] = v;
    if (dHb) dHb[i] = __float2bfloat16_rn(v);
  }
}

// db[j] = sum_b dZ[b][j]
__global__ void k_colsum(const float* __restrict__ dZ, int Bsz, int n, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.0f;
  for (int b = 0; b < Bsz; ++b) s += dZ[(size_t)b * n + j];
  db[j] = s;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_init_uniform(float* __restrict__ w, long long n, float scale, uint32_t tag, uint32_t k0, uint32_t k1) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    uint32_t c[4] = {4u, tag, (uint32_t)i, 0u};
    philox4x32_10(c, k0, k1);
    w[i] = scale * (float)(2.0 * uniform53(c[0], c[1]) - 1.0);
  }
}

int blocks_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

}  // namespace

struct rfm_mlp {
  int din, H, dout;
  cudaStream_t st;
  // parameters: FP32 master, bf16 copies, Adam moments, gradients (one flat buffer each)
  long long nparam;
  float *w, *m, *v, *g;
  __nv_bfloat16* wb;
  long long off[6];  // W1, b1, W2, b2, W3, b3
  int bcap = 0;
  // activations for a batch
  float *x = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dh1 = nullptr, *dh2 = nullptr,
        *lossp = nullptr;
  __nv_bfloat16 *xb = nullptr, *h1b = nullptr, *h2b = nullptr, *dyb = nullptr, *dh2b = nullptr;
  int step = 0;
};

namespace {

template <typename TA, typename TB>
rfm_status mm(cudaStream_t st, const TA* A, long long sam, long long sak, const TB* B, long long sbk, long long sbn,
              float* C, long long scm, long long scn, int M, int N, int K, float beta, const float* bias, int act,
              __nv_bfloat16* Cb) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_mm<TA, TB><<<grid, 256, 0, st>>>(A, sam, sak, B, sbk, sbn, C, scm, scn, M, N, K, beta, bias, act, Cb);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status ensure_batch(rfm_mlp* p, int B) {
  if (B <= p->bcap) return RFM_OK;
  void** bufs[] = {(void**)&p->x,   (void**)&p->h1,  (void**)&p->h2,  (void**)&p->y,   (void**)&p->dy,
                    (void**)&p->dh1, (void**)&p->dh2, (void**)&p->lossp, (void**)&p->xb, (void**)&p->h1b,
                    (void**)&p->h2b, (void**)&p->dyb, (void**)&p->dh2b};
  for (void** b : bufs) {  // no stale pointer survives a failed reallocation
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  p->bcap = 0;
  auto al = [&](void** ptr, size_t bytes) -> bool { return cudaMalloc(ptr, bytes) == cudaSuccess; };
  const size_t fb = sizeof(float), hb = sizeof(__nv_bfloat16);
  const size_t nblk = kLossBlocks;
  bool ok = al((void**)&p->x, (size_t)B * p->din * fb) && al((void**)&p->h1, (size_t)B * p->H * fb) &&
            al((void**)&p->h2, (size_t)B * p->H * fb) && al((void**)&p->y, (size_t)B * p->dout * fb) &&
            al((void**)&p->dy, (size_t)B * p->dout * fb) && al((void**)&p->dh1, (size_t)B * p->H * fb) &&
            al((void**)&p->dh2, (size_t)B * p->H * fb) && al((void**)&p->lossp, (size_t)B * nblk * fb) &&
            al((void**)&p->xb, (size_t)B * p->din * hb) && al((void**)&p->h1b, (size_t)B * p->H * hb) &&
            al((void**)&p->h2b, (size_t)B * p->H * hb) && al((void**)&p->dyb, (size_t)B * p->dout * hb) &&
            al((void**)&p->dh2b, (size_t)B * p->H * hb);
  if (!ok) {
    rfm_set_error("mlp: batch allocation failed");
    return RFM_ENOMEM;
  }
  p->bcap = B;
  return RFM_OK;
}

// Forward for batch B from p->x (FP32): fills h1, h2, y and their bf16 copies.
rfm_status forward(rfm_mlp* p, int B) {
  cudaStream_t st = p->st;
  const int din = p->din, H = p->H, n = p->dout;
  k_to_bf16<<<blocks_for((long long)B * din), 256, 0, st>>>(p->x, (long long)B * din, p->xb);
  RFM_CHECK_LAUNCH();
  const __nv_bfloat16* W1 = p->wb + p->off[0];
  const __nv_bfloat16* W2 = p->wb + p->off[2];
  const __nv_bfloat16* W3 = p->wb + p->off[4];
  // h1[b][j] = tanh(sum_k x[b][k] W1[j][k] + b1[j])
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->xb, din, 1, W1, 1, din, p->h1, H, 1, B, H, din, 0.0f, p->w + p->off[1], 1,
             p->h1b));
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->h1b, H, 1, W2, 1, H, p->h2, H, 1, B, H, H, 0.0f, p->w + p->off[3], 1,
             p->h2b));
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->h2b, H, 1, W3, 1, H, p->y, n, 1, B, n, H, 0.0f, p->w + p->off[5], 0,
             (__nv_bfloat16*)nullptr));
  return RFM_OK;
}

// The metric's blocks must tile the output, fit the per-block shared
// residual (48 KB) and the loss-partial buffer (kLossBlocks per sample).
bool metric_ok(const rfm_mlp* p, const float* G, int gblk) {
  if (!G) return (p->dout + 1023) / 1024 <= kLossBlocks;
  return gblk > 0 && gblk <= 12288 && p->dout % gblk == 0 && p->dout / gblk <= kLossBlocks;
}

// Gradients of the loss for targets T into p->g; loss to *loss_host.
rfm_status backward(rfm_mlp* p, int B, const float* T, const float* G, int gblk, double* loss_host) {
  cudaStream_t st = p->st;
  const int din = p->din, H = p->H, n = p->dout;
  const int bs = G ? gblk : std::min(n, 1024);
  const int nblk = (n + bs - 1) / bs;
  k_metric<<<dim3(B, nblk), 256, bs * sizeof(float), st>>>(p->y, T, B, n, G, bs, p->dy, p->lossp);
  RFM_CHECK_LAUNCH();
  k_to_bf16<<<blocks_for((long long)B * n), 256, 0, st>>>(p->dy, (long long)B * n, p->dyb);
  RFM_CHECK_LAUNCH();
  float* gW1 = p->g + p->off[0];
  float* gb1 = p->g + p->off[1];
  float* gW2 = p->g + p->off[2];
  float* gb2 = p->g + p->off[3];
  float* gW3 = p->g + p->off[4];
  float* gb3 = p->g + p->off[5];
  const __nv_bfloat16* W2 = p->wb + p->off[2];
  const __nv_bfloat16* W3 = p->wb + p->off[4];
  // layer 3: gW3[i][j] = sum_b dy[b][i] h2[b][j]; gb3 = colsum(dy); dh2 = dy W3
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->dyb, 1, n, (const __nv_bfloat16*)p->h2b, H, 1, gW3, H, 1, n, H, B, 0.0f,
             (const float*)nullptr, 0, (__nv_bfloat16*)nullptr));
  k_colsum<<<(n + 255) / 256, 256, 0, st>>>(p->dy, B, n, gb3);
  RFM_CHECK_LAUNCH();
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->dyb, n, 1, W3, H, 1, p->dh2, H, 1, B, H, n, 0.0f, (const float*)nullptr, 0,
             (__nv_bfloat16*)nullptr));
  k_tanh_back<<<blocks_for((long long)B * H), 256, 0, st>>>(p->dh2, p->h2, (long long)B * H, p->dh2b);
  RFM_CHECK_LAUNCH();
  // layer 2
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->dh2b, 1, H, (const __nv_bfloat16*)p->h1b, H, 1, gW2, H, 1, H, H, B, 0.0f,
             (const float*)nullptr, 0, (__nv_bfloat16*)nullptr));
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(p->dh2, B, H, gb2);
  RFM_CHECK_LAUNCH();
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->dh2b, H, 1, W2, H, 1, p->dh1, H, 1, B, H, H, 0.0f, (const float*)nullptr, 0,
             (__nv_bfloat16*)nullptr));
  k_tanh_back<<<blocks_for((long long)B * H), 256, 0, st>>>(p->dh1, p->h1, (long long)B * H, p->dh2b);
  RFM_CHECK_LAUNCH();
  // layer 1 (dh2b now holds the bf16 copy of dh1)
  RFM_TRY(mm(st, (const __nv_bfloat16*)p->dh2b, 1, H, (const __nv_bfloat16*)p->xb, din, 1, gW1, din, 1, H, din, B,
             0.0f, (const float*)nullptr, 0, (__nv_bfloat16*)nullptr));
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(p->dh1, B, H, gb1);
  RFM_CHECK_LAUNCH();
  if (loss_host) {
    std::vector<float> lp((size_t)B * nblk);
    RFM_CUDA(cudaMemcpyAsync(lp.data(), p->lossp, lp.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    RFM_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (float v : lp) s += v;
    *loss_host = s;
  }
  return RFM_OK;
}

}  // namespace

extern "C" {

rfm_status rfm_mlp_create(int din, int hidden, int dout, uint64_t seed, void* cuda_stream, rfm_mlp** out) {
  if (!out || din <= 0 || hidden <= 0 || dout <= 0) return RFM_EINVAL;
  rfm_mlp* p = new rfm_mlp();
  p->din = din;
  p->H = hidden;
  p->dout = dout;
  p->st = (cudaStream_t)cuda_stream;
  const long long sz[6] = {(long long)hidden * din, hidden, (long long)hidden * hidden, hidden,
                           (long long)dout * hidden, dout};
  long long o = 0;
  for (int i = 0; i < 6; ++i) {
    p->off[i] = o;
    o += (sz[i] + 63) / 64 * 64;
  }
  p->nparam = o;
  bool ok = cudaMalloc((void**)&p->w, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->m, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->v, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->g, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&p->wb, o * sizeof(__nv_bfloat16)) == cudaSuccess;
  if (!ok) {
    rfm_mlp_destroy(p);  // frees whatever was allocated
    rfm_set_error("mlp: allocation failed");
    return RFM_ENOMEM;
  }
  cudaMemsetAsync(p->w, 0, o * sizeof(float), p->st);
  cudaMemsetAsync(p->g, 0, o * sizeof(float), p->st);
  cudaMemsetAsync(p->m, 0, o * sizeof(float), p->st);
  cudaMemsetAsync(p->v, 0, o * sizeof(float), p->st);
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
  // Glorot-uniform weights, zero biases
  const int fan[3][2] = {{din, hidden}, {hidden, hidden}, {hidden, dout}};
  for (int l = 0; l < 3; ++l) {
    const float sc = sqrtf(6.0f / (float)(fan[l][0] + fan[l][1]));
    k_init_uniform<<<blocks_for(sz[2 * l]), 256, 0, p->st>>>(p->w + p->off[2 * l], sz[2 * l], sc, (uint32_t)l, k0, k1);
  }
  k_to_bf16<<<blocks_for(o), 256, 0, p->st>>>(p->w, o, p->wb);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->st) != cudaSuccess) {
    rfm_mlp_destroy(p);
    rfm_set_error("mlp: initialisation failed");
    return RFM_ECUDA;
  }
  *out = p;
  return RFM_OK;
}

rfm_status rfm_mlp_destroy(rfm_mlp* p) {
  if (!p) return RFM_OK;
  cudaStreamSynchronize(p->st);
  void* bufs[] = {p->w, p->m, p->v, p->g, p->wb, p->x, p->h1, p->h2, p->y, p->dy, p->dh1, p->dh2, p->lossp,
                  p->xb, p->h1b, p->h2b, p->dyb, p->dh2b};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
  return RFM_OK;
}

int64_t rfm_mlp_num_params(const rfm_mlp* p) { return p ? p->nparam : 0; }

rfm_status rfm_mlp_params(rfm_mlp* p, float* dst_dev, const float* src_dev, int64_t* offsets_host) {
  if (!p) return RFM_EINVAL;
  if (src_dev) {
    RFM_CUDA(cudaMemcpyAsync(p->w, src_dev, p->nparam * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
    k_to_bf16<<<blocks_for(p->nparam), 256, 0, p->st>>>(p->w, p->nparam, p->wb);
    RFM_CHECK_LAUNCH();
  }
  if (dst_dev) RFM_CUDA(cudaMemcpyAsync(dst_dev, p->w, p->nparam * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  if (offsets_host)
    for (int i = 0; i < 6; ++i) offsets_host[i] = p->off[i];
  RFM_CUDA(cudaStreamSynchronize(p->st));
  return RFM_OK;
}

rfm_status rfm_mlp_forward(rfm_mlp* p, const float* x_dev, int batch, float* y_dev) {
  if (!p || !x_dev || !y_dev || batch <= 0) return RFM_EINVAL;
  RFM_TRY(ensure_batch(p, batch));
  RFM_CUDA(cudaMemcpyAsync(p->x, x_dev, (size_t)batch * p->din * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  RFM_TRY(forward(p, batch));
  RFM_CUDA(cudaMemcpyAsync(y_dev, p->y, (size_t)batch * p->dout * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  RFM_CUDA(cudaStreamSynchronize(p->st));
  return RFM_OK;
}

rfm_status rfm_mlp_gradient(rfm_mlp* p, const float* x_dev, const float* t_dev, int batch, const float* G_dev,
                            int gblk, float* grad_dev, double* loss_host) {
  if (!p || !x_dev || !t_dev || batch <= 0 || !metric_ok(p, G_dev, gblk)) return RFM_EINVAL;
  RFM_TRY(ensure_batch(p, batch));
  RFM_CUDA(cudaMemcpyAsync(p->x, x_dev, (size_t)batch * p->din * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  RFM_TRY(forward(p, batch));
  RFM_TRY(backward(p, batch, t_dev, G_dev, gblk, loss_host));
  if (grad_dev) RFM_CUDA(cudaMemcpyAsync(grad_dev, p->g, p->nparam * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  RFM_CUDA(cudaStreamSynchronize(p->st));
  return RFM_OK;
}

rfm_status rfm_mlp_train(rfm_mlp* p, const float* x_dev, const float* t_dev, int batch, const float* G_dev, int gblk,
                         int steps, float lr, double* loss_host) {
  if (!p || !x_dev || !t_dev || batch <= 0 || steps < 0 || !metric_ok(p, G_dev, gblk)) return RFM_EINVAL;
  RFM_TRY(ensure_batch(p, batch));
  RFM_CUDA(cudaMemcpyAsync(p->x, x_dev, (size_t)batch * p->din * sizeof(float), cudaMemcpyDeviceToDevice, p->st));
  for (int s = 0; s < steps; ++s) {
    RFM_TRY(forward(p, batch));
    RFM_TRY(backward(p, batch, t_dev, G_dev, gblk, (s == steps - 1) ? loss_host : nullptr));
    ++p->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)p->step), c2 = 1.0f - powf(b2, (float)p->step);
    k_adam<<<blocks_for(p->nparam), 256, 0, p->st>>>(p->w, p->g, p->m, p->v, p->nparam, lr, b1, b2, 1e-8f, c1, c2,
                                                      p->wb);
    RFM_CHECK_LAUNCH();
  }
  RFM_CUDA(cudaStreamSynchronize(p->st));
  return RFM_OK;
}

// Per-block Gram of the features at evaluation points, the metric of the
// function-space loss: G[e*fields + f] = (1/npts) sum over the points x owned
// by subdomain e of phi_{e,f}(x) phi_{e,f}(x)^T (M x M each).  The points must
// be grouped by owning subdomain: owner_start_host[e] .. owner_start_host[e+1]
// (G+1 entries) index the points of subdomain e.
rfm_status rfm_feature_gram(const rfm_problem* p, const double* pts_dev, int64_t npts, const int64_t* owner_start_host,
                            float* G_dev) {
  if (!p || !pts_dev || npts <= 0 || !owner_start_host || !G_dev) return RFM_EINVAL;
  float* Phi = nullptr;
  if (cudaMalloc((void**)&Phi, (size_t)npts * p->W * sizeof(float)) != cudaSuccess) return RFM_ENOMEM;
  rfm_status st = rfm_launch_phi_values(p, pts_dev, npts, 1.0f / sqrtf((float)npts), Phi);
  const int M = p->M, W = p->W;
  for (int e = 0; e < p->G && st == RFM_OK; ++e) {
    const long long p0 = owner_start_host[e], cnt = owner_start_host[e + 1] - owner_start_host[e];
    for (int f = 0; f < p->fields && st == RFM_OK; ++f) {
      float* Gb = G_dev + (size_t)(e * p->fields + f) * M * M;
      if (cnt <= 0) {
        if (cudaMemsetAsync(Gb, 0, (size_t)M * M * sizeof(float), p->stream) != cudaSuccess) st = RFM_ECUDA;
        continue;
      }
      const float* base = Phi + (size_t)p0 * W + (size_t)f * M;
      st = mm(p->stream, base, 1, W, base, W, 1, Gb, M, 1, M, M, (int)cnt, 0.0f, (const float*)nullptr, 0,
              (__nv_bfloat16*)nullptr);
    }
  }
  if (cudaStreamSynchronize(p->stream) != cudaSuccess && st == RFM_OK) st = RFM_ECUDA;
  cudaFree(Phi);
  return st;
}


}  // extern "C"

// ---- warm-start object: basis of training solutions + network ------------

namespace {

// per input dimension: mean and standard deviation over the training set
__global__ void k_input_stats(const double* __restrict__ P, int N, int din, float* __restrict__ mu,
                              float* __restrict__ sd) {
  const int i = threadIdx.x;
  if (i >= din) return;
  double s = 0.0, s2 = 0.0;
  for (int j = 0; j < N; ++j) s += P[(size_t)j * din + i];
  const double m = s / N;
  for (int j = 0; j < N; ++j) {
    const double d = P[(size_t)j * din + i] - m;
    s2 += d * d;
  }
  const double v = s2 / N;
  mu[i] = (float)m;
  sd[i] = v > 0.0 ? (float)sqrt(v) : 1.0f;
}

__global__ void k_normalise_inputs(const double* __restrict__ P, long long count, int din, const float* __restrict__ mu,
                                   const float* __restrict__ sd, float* __restrict__ x) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count * din;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % din);
    x[t] = ((float)P[t] - mu[i]) / sd[i];
  }
}

// t[j][k] = Z[j][k] / scale (FP32), k < rank, from Z [N][N]; also the sum of squares
__global__ void k_targets(const double* __restrict__ Z, int N, int rank, double inv, float* __restrict__ t) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)N * rank;
       q += (long long)gridDim.x * blockDim.x) {
    const long long j = q / rank, k = q - j * rank;
    t[q] = (float)(Z[(size_t)j * N + k] * inv);
  }
}

__global__ void k_sumsq_rows(const double* __restrict__ Z, int N, int rank, double* __restrict__ out) {
  // one thread per snapshot; fixed order
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int k = 0; k < rank; ++k) s += Z[(size_t)j * N + k] * Z[(size_t)j * N + k];
  out[j] = s;
}

}  // namespace

struct rfm_warmstart {
  rfm_mlp* net = nullptr;
  cudaStream_t st = nullptr;
  int din = 0, rank = 0, ntrain = 0;
  long long n = 0;
  double zscale = 1.0;
  double *mean = nullptr, *U = nullptr;
  float *mu = nullptr, *sd = nullptr, *x = nullptr, *t = nullptr, *xq = nullptr, *yq = nullptr;
  int qcap = 0;
};

namespace {
void ws_free(rfm_warmstart* w) {
  if (!w) return;
  if (w->net) rfm_mlp_destroy(w->net);
  void* b[] = {w->mean, w->U, w->mu, w->sd, w->x, w->t, w->xq, w->yq};
  for (void* q : b)
    if (q) cudaFree(q);
  delete w;
}
}  // namespace

extern "C" {

rfm_status rfm_warmstart_create(const rfm_problem* p, const double* C_dev, const double* params_dev, int N, int din,
                                const double* pts_dev, int64_t npts, double tol, int hidden, uint64_t seed,
                                rfm_warmstart** out) {
  if (!p || !C_dev || !params_dev || N < 2 || din <= 0 || din > 1024 || !pts_dev || npts <= 0 || hidden <= 0 ||
      !out) {
    rfm_set_error("rfm_warmstart_create: bad argument");
    return RFM_EINVAL;
  }
  rfm_warmstart* w = new rfm_warmstart();
  w->st = p->stream;
  w->din = din;
  w->n = p->n;
  w->ntrain = N;
  double *Uall = nullptr, *Z = nullptr, *ss = nullptr;
  rfm_status st = RFM_OK;
  auto fail = [&](rfm_status s, const char* msg) {
    if (msg) rfm_set_error(msg);
    if (Uall) cudaFree(Uall);
    if (Z) cudaFree(Z);
    if (ss) cudaFree(ss);
    ws_free(w);
    return s;
  };
  if (cudaMalloc((void**)&w->mean, (size_t)w->n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&Uall, (size_t)N * w->n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&Z, (size_t)N * N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&ss, (size_t)N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&w->mu, din * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&w->sd, din * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&w->x, (size_t)N * din * sizeof(float)) != cudaSuccess)
    return fail(RFM_ENOMEM, "rfm_warmstart_create: allocation failed");
  int rank = 0;
  st = rfm_function_basis(p, C_dev, N, pts_dev, npts, tol, w->mean, Uall, Z, &rank);
  if (st != RFM_OK) return fail(st, nullptr);
  if (rank < 1) return fail(RFM_EINVAL, "rfm_warmstart_create: the training solutions span no direction");
  w->rank = rank;
  // modes, compacted to [rank][n]
  if (cudaMalloc((void**)&w->U, (size_t)rank * w->n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&w->t, (size_t)N * rank * sizeof(float)) != cudaSuccess)
    return fail(RFM_ENOMEM, "rfm_warmstart_create: allocation failed");
  if (cudaMemcpyAsync(w->U, Uall, (size_t)rank * w->n * sizeof(double), cudaMemcpyDeviceToDevice, w->st) != cudaSuccess)
    return fail(RFM_ECUDA, "rfm_warmstart_create: copy failed");
  // coordinate scale: root mean square of the coordinates
  k_sumsq_rows<<<(N + 255) / 256, 256, 0, w->st>>>(Z, N, rank, ss);
  std::vector<double> ssh(N);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(ssh.data(), ss, N * sizeof(double), cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaStreamSynchronize(w->st) != cudaSuccess)
    return fail(RFM_ECUDA, "rfm_warmstart_create: CUDA error");
  double tot = 0.0;
  for (double v : ssh) tot += v;
  w->zscale = sqrt(tot / ((double)N * rank));
  if (!(w->zscale > 0.0)) w->zscale = 1.0;
  k_targets<<<blocks_for((long long)N * rank), 256, 0, w->st>>>(Z, N, rank, 1.0 / w->zscale, w->t);
  k_input_stats<<<1, 1024, 0, w->st>>>(params_dev, N, din, w->mu, w->sd);
  k_normalise_inputs<<<blocks_for((long long)N * din), 256, 0, w->st>>>(params_dev, N, din, w->mu, w->sd, w->x);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(w->st) != cudaSuccess)
    return fail(RFM_ECUDA, "rfm_warmstart_create: CUDA error");
  cudaFree(Uall);
  cudaFree(Z);
  cudaFree(ss);
  Uall = Z = ss = nullptr;
  st = rfm_mlp_create(din, hidden, rank, seed, (void*)w->st, &w->net);
  if (st != RFM_OK) return fail(st, nullptr);
  *out = w;
  return RFM_OK;
}

rfm_status rfm_warmstart_destroy(rfm_warmstart* w) {
  if (w) cudaStreamSynchronize(w->st);
  ws_free(w);
  return RFM_OK;
}

int rfm_warmstart_rank(const rfm_warmstart* w) { return w ? w->rank : 0; }

rfm_mlp* rfm_warmstart_network(rfm_warmstart* w) { return w ? w->net : nullptr; }

rfm_status rfm_warmstart_train(rfm_warmstart* w, int steps, float lr, double* loss_host) {
  if (!w || steps < 0 || !(lr > 0.0f)) {
    rfm_set_error("rfm_warmstart_train: bad argument");
    return RFM_EINVAL;
  }
  return rfm_mlp_train(w->net, w->x, w->t, w->ntrain, nullptr, 0, steps, lr, loss_host);
}

rfm_status rfm_warmstart_predict(rfm_warmstart* w, const double* params_dev, int batch, double* c_dev) {
  if (!w || !params_dev || batch <= 0 || !c_dev) {
    rfm_set_error("rfm_warmstart_predict: bad argument");
    return RFM_EINVAL;
  }
  if (batch > w->qcap) {
    if (w->xq) cudaFree(w->xq);
    if (w->yq) cudaFree(w->yq);
    w->xq = w->yq = nullptr;
    w->qcap = 0;
    if (cudaMalloc((void**)&w->xq, (size_t)batch * w->din * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&w->yq, (size_t)batch * w->rank * sizeof(float)) != cudaSuccess) {
      rfm_set_error("rfm_warmstart_predict: allocation failed");
      return RFM_ENOMEM;
    }
    w->qcap = batch;
  }
  k_normalise_inputs<<<blocks_for((long long)batch * w->din), 256, 0, w->st>>>(params_dev, batch, w->din, w->mu, w->sd,
                                                                              w->xq);
  RFM_CHECK_LAUNCH();
  RFM_TRY(rfm_mlp_forward(w->net, w->xq, batch, w->yq));
  return rfm_basis_combine(w->mean, w->U, w->n, w->rank, w->yq, batch, w->zscale, c_dev, (void*)w->st);
}

}  // extern "C"

