// Randomised sketch B = S_k J of the scaled Jacobian (Sec. 4.1).
//
// Count sketch: row i of J goes to bucket h(i) with sign sigma(i) (Philox
// counter (1, i, kJ, 0): h = (x0 * s) >> 32, sigma = +1 iff x1 is even).  S_k is
// never formed; buckets are built by a counting sort whose per-bucket row lists
// are then sorted, so every bucket sums its rows in increasing row order
// (deterministic).  One warp per bucket accumulates into the column-major B.
//
// Gaussian sketch: S_k[r, i] is the (r mod 2)-th Box-Muller normal of Philox
// counter (2, i, r/2, kJ), rounded to the grid 2^-4 (an integer of magnitude
// <= 137 times 2^-4, exact in bf16), stored as bf16 bits [m][s].
// B[:, block b] = S[:, rows(b)] J[rows(b), block b] for every column block b
// (the rows touching subdomain b), an FP64 GEMM with gathered operands:
// K = |rows(b)|, N = W, M = s.  Its algorithmic cost is 2 s nnz(J) flops.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "philox.cuh"
#include "rfm_internal.cuh"

namespace {

__global__ void k_hash(long long m, long long s, uint32_t kJ, uint32_t key0, uint32_t key1, int* __restrict__ hb,
                       double* __restrict__ hs, int* __restrict__ cnt) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint32_t c[4] = {1u, (uint32_t)i, kJ, 0u};
  philox4x32_10(c, key0, key1);
  const int h = (int)(((uint64_t)c[0] * (uint64_t)s) >> 32);
  hb[i] = h;
  hs[i] = (c[1] & 1u) ? -1.0 : 1.0;
  atomicAdd(cnt + h, 1);
}

// Exclusive scan of cnt[0..s) into ptr[0..s]; one CTA of 1024 threads.
__global__ void k_scan(const int* __restrict__ cnt, long long s, int* __restrict__ ptr) {
  __shared__ long long sh[1024];
  const int t = threadIdx.x;
  const long long per = (s + 1023) / 1024;
  const long long b = t * per, e = min(s, b + per);
  long long loc = 0;
  for (long long i = b; i < e; ++i) loc += cnt[i];
  sh[t] = loc;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long v = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  long long run = t ? sh[t - 1] : 0;
  for (long long i = b; i < e; ++i) {
    ptr[i] = (int)run;
    run += cnt[i];
  }
  if (t == 1023) ptr[s] = (int)sh[1023];
}

__global__ void k_fill(long long m, const int* __restrict__ hb, const int* __restrict__ ptr, int* __restrict__ cur,
                       int* __restrict__ rows) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int h = hb[i];
  const int pos = atomicAdd(cur + h, 1);
  rows[ptr[h] + pos] = (int)i;
}

__global__ void k_sort_buckets(long long s, const int* __restrict__ ptr, int* __restrict__ rows) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= s) return;
  const int beg = ptr[b], end = ptr[b + 1];
  for (int i = beg + 1; i < end; ++i) {
    const int v = rows[i];
    int j = i - 1;
    while (j >= beg && rows[j] > v) {
      rows[j + 1] = rows[j];
      --j;
    }
    rows[j + 1] = v;
  }
}

// One warp per bucket: B[bucket, cols] += sigma(i) J[i, cols] for its rows.
__global__ void k_count_scatter(long long s, const int* __restrict__ ptr, const int* __restrict__ rows,
                                const double* __restrict__ hs, const double* __restrict__ Jp,
                                const double* __restrict__ Js, const int4* __restrict__ meta, long long m_int, int W,
                                double* __restrict__ B) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long b = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); b < s; b += nw) {
    const int beg = ptr[b], end = ptr[b + 1];
    for (int t = beg; t < end; ++t) {
      const int i = rows[t];
      const double sg = hs[i];
      const int4 mt = meta[i];
      const double* row = Jp + (size_t)i * W;
      double* out = B + (size_t)mt.y * W * s + b;
      for (int j = lane; j < W; j += 32) out[(size_t)j * s] += sg * row[j];
      if ((mt.x & 0xF) == 1) {
        const double* row2 = Js + (size_t)(i - m_int) * W;
        double* out2 = B + (size_t)mt.z * W * s + b;
        for (int j = lane; j < W; j += 32) out2[(size_t)j * s] += sg * row2[j];
      }
    }
  }
}

// Gaussian sketch entries for rows i in [0, m): S[i*s + r].
__global__ void k_gauss_gen(long long m, long long s, uint32_t kJ, uint32_t key0, uint32_t key1,
                            uint16_t* __restrict__ S) {
  const long long half = s / 2;
  const long long total = m * half;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / half, q = t - i * half;
    uint32_t c[4] = {2u, (uint32_t)i, (uint32_t)q, kJ};
    philox4x32_10(c, key0, key1);
    float d0, d1;
    gauss_pair_q16(c, &d0, &d1);
    const uint16_t z0 = (uint16_t)(__float_as_uint(d0 * 0.0625f) >> 16);  // exact in bf16
    const uint16_t z1 = (uint16_t)(__float_as_uint(d1 * 0.0625f) >> 16);
    const uint32_t packed = (uint32_t)z0 | ((uint32_t)z1 << 16);
    reinterpret_cast<uint32_t*>(S + (size_t)i * s)[q] = packed;
  }
}

// B[:, b*W + col] = sum_k S[:, row_k] J[row_k, col], rows from colrows[colptr[b]..).
// Tile 128 (sketch rows) x 64 (columns), K step 16; 256 threads, 4 x 8 outputs each.
__global__ void __launch_bounds__(256) k_gauss_gemm(const uint16_t* __restrict__ S, long long s,
                                                    const double* __restrict__ Jp, const double* __restrict__ Js,
                                                    const int* __restrict__ colptr, const int* __restrict__ colrows,
                                                    long long m_int, int W, double* __restrict__ B) {
  __shared__ double As[16][128];
  __shared__ double Bs[16][64];
  __shared__ const double* rowp[16];
  __shared__ long long scol[16];
  const int b = blockIdx.z;
  const long long r0 = (long long)blockIdx.x * 128;
  const int c0 = blockIdx.y * 64;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int beg = colptr[b], end = colptr[b + 1];
  double acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[i][q] = 0.0;
  for (int k0 = beg; k0 < end; k0 += 16) {
    if (tid < 16) {
      const int k = k0 + tid;
      if (k < end) {
        const unsigned int ent = (unsigned int)colrows[k];
        const long long r = ent & 0x7fffffffu;
        rowp[tid] = (ent >> 31) ? Js + (size_t)(r - m_int) * W : Jp + (size_t)r * W;
        scol[tid] = r;
      } else {
        rowp[tid] = nullptr;
        scol[tid] = -1;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < 16 * 128; idx += 256) {
      const int kk = idx >> 7, rr = idx & 127;
      const long long gr = r0 + rr;
      const long long sc = scol[kk];
      As[kk][rr] = (sc >= 0 && gr < s) ? bf16_bits_to_double(S[(size_t)sc * s + gr]) : 0.0;
    }
    for (int idx = tid; idx < 16 * 64; idx += 256) {
      const int kk = idx >> 6, cc = idx & 63;
      const double* rp = rowp[kk];
      Bs[kk][cc] = (rp != nullptr && c0 + cc < W) ? rp[c0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 32 * i];
#pragma unroll
      for (int q = 0; q < 8; ++q) bv[q] = Bs[kk][ty + 8 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[i][q] += av[i] * bv[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int col = c0 + ty + 8 * q;
    if (col >= W) continue;
    double* out = B + ((size_t)b * W + col) * s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long gr = r0 + tx + 32 * i;
      if (gr < s) out[gr] = acc[i][q];
    }
  }
}

// Digit tiles of S for the split product (one digit per entry: d = rint(16 z),
// so S = d * 2^(3 - 7) with exponent 3), for every column block b: tiles
// [s/128][ktiles_b] starting at tile toff[b], K index = position in the block's
// row list.  Threads run along K so each warp writes within 128-byte rows.
__global__ void k_gauss_digits(long long s, long long totK, const int* __restrict__ colptr, int G,
                               const int* __restrict__ colrows, const long long* __restrict__ toff, uint32_t kJ,
                               uint32_t key0, uint32_t key1, uint16_t* __restrict__ out) {
  const long long half = s / 2;
  const long long total = half * totK;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long g = t % totK, q = t / totK;
    int lo = 0, hi = G - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (colptr[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const long long k = g - colptr[b];
    const long long kt_b = (colptr[b + 1] - colptr[b] + 63) / 64;
    const unsigned i = (unsigned)colrows[g] & 0x7fffffffu;
    uint32_t c[4] = {2u, i, (uint32_t)q, kJ};
    philox4x32_10(c, key0, key1);
    float d0, d1;
    gauss_pair_q16(c, &d0, &d1);
    const long long r = 2 * q;
    const long long mt = r >> 7;
    const int rr = (int)(r & 127);
    const long long tile = toff[b] + mt * kt_b + (k >> 6);
    uint16_t* base = out + (size_t)tile * (128 * 64);
    const int k64 = (int)(k & 63);
    base[rfm_swz128(rr, k64) >> 1] = (uint16_t)(__float_as_uint(d0) >> 16);
    base[rfm_swz128(rr + 1, k64) >> 1] = (uint16_t)(__float_as_uint(d1) >> 16);
  }
}

__global__ void k_fill_int(int* __restrict__ x, long long n, int v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

}  // namespace

rfm_status rfm_launch_count_sketch(rfm_problem* p, long long s, int kJ) {
  const uint32_t k0 = (uint32_t)(p->desc.seed & 0xffffffffull), k1 = (uint32_t)(p->desc.seed >> 32);
  int* cnt = reinterpret_cast<int*>(p->brows + p->m);  // [s] counters, then [s] cursors
  int* cur = cnt + s;
  ProfScope ps(PF_SKETCH_COUNT, p->stream);
  RFM_CUDA(cudaMemsetAsync(cnt, 0, 2 * s * sizeof(int), p->stream));
  const int g = (int)((p->m + 255) / 256);
  k_hash<<<g, 256, 0, p->stream>>>(p->m, s, (uint32_t)kJ, k0, k1, p->hbuck, p->hsign, cnt);
  RFM_CHECK_LAUNCH();
  k_scan<<<1, 1024, 0, p->stream>>>(cnt, s, p->bptr);
  RFM_CHECK_LAUNCH();
  k_fill<<<g, 256, 0, p->stream>>>(p->m, p->hbuck, p->bptr, cur, p->brows);
  RFM_CHECK_LAUNCH();
  k_sort_buckets<<<(int)((s + 255) / 256), 256, 0, p->stream>>>(s, p->bptr, p->brows);
  RFM_CHECK_LAUNCH();
  RFM_CUDA(cudaMemsetAsync(p->B, 0, (size_t)s * p->n * sizeof(double), p->stream));
  long long nb = (s + 7) / 8;
  if (nb > 152 * 32) nb = 152 * 32;
  k_count_scatter<<<(int)nb, 256, 0, p->stream>>>(s, p->bptr, p->brows, p->hsign, p->Jp, p->Js, p->rmeta, p->m_int,
                                                 p->W, p->B);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_gauss_sketch(rfm_problem* p, long long s, int kJ) {
  const uint32_t k0 = (uint32_t)(p->desc.seed & 0xffffffffull), k1 = (uint32_t)(p->desc.seed >> 32);
  {
    ProfScope ps(PF_SKETCH_GEN, p->stream);
    k_gauss_gen<<<152 * 16, 256, 0, p->stream>>>(p->m, s, (uint32_t)kJ, k0, k1, p->Sg);
    RFM_CHECK_LAUNCH();
  }
  ProfScope ps(PF_SKETCH_GEMM, p->stream);
  dim3 grid((unsigned)((s + 127) / 128), (unsigned)((p->W + 63) / 64), (unsigned)p->G);
  rfm_prof_work(PF_SKETCH_GEMM, 2.0 * (double)s * (double)(p->m + p->m_iface) * p->W);  // FP64 flops
  k_gauss_gemm<<<grid, 256, 0, p->stream>>>(p->Sg, s, p->Jp, p->Js, p->colptr, p->colrows, p->m_int, p->W, p->B);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

// B[:, block b] = S[:, rows(b)] J[rows(b), block b] with the product emulated to
// FP64 accuracy on the bf16 tensor cores: S is one exact digit per entry,
// each Jacobian column block is split into 8 digits.
rfm_status rfm_launch_gauss_sketch_tc(rfm_problem* p, long long s, int kJ) {
  const uint32_t k0 = (uint32_t)(p->desc.seed & 0xffffffffull), k1 = (uint32_t)(p->desc.seed >> 32);
  const int G = p->G;
  const long long mtiles = (s + 127) / 128;
  std::vector<long long> toff(G + 1, 0);
  long long maxK = 0;
  for (int b = 0; b < G; ++b) {
    const long long K = p->colptr_h[b + 1] - p->colptr_h[b];
    maxK = std::max(maxK, K);
    toff[b + 1] = toff[b] + mtiles * ((K + 63) / 64);
  }
  const long long sbytes = toff[G] * 128 * 64 * 2;
  const long long jbytes = rfm_oz_digit_bytes(p->W, maxK, 8, 64);
  auto grow = [&](void** ptr, long long* cap, long long need) -> rfm_status {
    if (need <= *cap) return RFM_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (cudaMalloc(ptr, (size_t)need) != cudaSuccess) {
      rfm_set_error("tensor-core sketch: allocation of " + std::to_string(need) + " bytes failed");
      return RFM_ENOMEM;
    }
    *cap = need;
    return RFM_OK;
  };
  RFM_TRY(grow((void**)&p->sdig, &p->sdig_bytes, sbytes));
  RFM_TRY(grow((void**)&p->jdig, &p->jdig_bytes, jbytes));
  RFM_TRY(grow((void**)&p->oz_e, &p->oz_e_cap, (s + p->W + 64) * (long long)sizeof(int)));
  if (!p->oz_toff) {
    if (cudaMalloc(&p->oz_toff, (size_t)(G + 1) * sizeof(long long)) != cudaSuccess) return RFM_ENOMEM;
  }
  RFM_CUDA(cudaMemcpyAsync(p->oz_toff, toff.data(), (G + 1) * sizeof(long long), cudaMemcpyHostToDevice, p->stream));
  int* es = p->oz_e;
  int* ej = p->oz_e + s;
  {
    ProfScope ps(PF_SKETCH_GEN, p->stream);
    RFM_CUDA(cudaMemsetAsync(p->sdig, 0, (size_t)sbytes, p->stream));
    const long long totK = p->colptr_h[G];
    k_gauss_digits<<<152 * 16, 256, 0, p->stream>>>(s, totK, p->colptr, G, p->colrows, p->oz_toff, (uint32_t)kJ, k0, k1,
                                                   p->sdig);
    RFM_CHECK_LAUNCH();
    k_fill_int<<<64, 256, 0, p->stream>>>(es, s, 3);
    RFM_CHECK_LAUNCH();
  }
  ProfScope ps(PF_SKETCH_GEMM, p->stream);
  for (int b = 0; b < G; ++b) {
    const long long K = p->colptr_h[b + 1] - p->colptr_h[b];
    if (K == 0) continue;
    RFM_TRY(rfm_oz_slice_jblock(p->Jp, p->Js, p->colrows + p->colptr_h[b], K, p->m_int, p->W, 8, ej, p->jdig,
                                p->stream));
    RFM_TRY(rfm_oz_gemm(p->sdig + (size_t)toff[b] * 128 * 64, 1, es, p->jdig, 8, ej, s, p->W, K, 9,
                        p->B + (size_t)b * p->W * s, s, 0, p->sync + SYNC_ERR, p->stream));
  }
  return RFM_OK;
}
