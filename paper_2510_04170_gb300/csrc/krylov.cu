// Matrix-vector kernels of the LSQR inner solve on J R^{-1} (Alg. 1 steps 3-4).
//
//  * k_jmv:   y = s1 * J x + s2 * y.  One warp per row; a row is W contiguous
//             doubles of its primary block (and W more of the secondary block
//             for interface rows), read once, coalesced.
//  * k_jtmv:  y = J^T x.  One CTA per (column block, 64-column chunk); the
//             rows touching the block are walked in a fixed order and the
//             eight warps' partial sums are combined in a fixed order, so the
//             result is deterministic.
//  * k_trsv:  x = R^{-1} b or x = R^{-T} b for the upper-triangular
//             preconditioner R (column-major, leading dimension ldr), in one
//             launch: 64-row blocks are claimed through a ticket counter in
//             dependency order, each block waits (bounded) on the per-block
//             flags of the blocks it needs, accumulates their contribution
//             with coalesced column reads of R, solves its diagonal block in
//             one warp and publishes its part of x with a release flag.
//  * k_partial_* / k_finish_*: deterministic two-stage norms and dots.
#include "rfm_internal.cuh"

namespace {

constexpr int TB = 64;  // triangular block

__global__ void __launch_bounds__(256) k_jmv(const double* __restrict__ Jp, const double* __restrict__ Js,
                                             const int4* __restrict__ meta, long long m, long long m_int, int W,
                                             const double* __restrict__ x, double s1, double s2,
                                             const double* __restrict__ s2dev, const int* __restrict__ skip,
                                             double* __restrict__ y) {
  if (skip && *skip) return;
  if (s2dev) s2 *= s2dev[0];
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
    const int4 mt = meta[i];
    const double* row = Jp + (size_t)i * W;
    const double* xb = x + (size_t)mt.y * W;
    double acc = 0.0;
    for (int j = lane; j < W; j += 32) acc += row[j] * xb[j];
    if ((mt.x & 0xF) == 1) {
      const double* row2 = Js + (size_t)(i - m_int) * W;
      const double* xb2 = x + (size_t)mt.z * W;
      for (int j = lane; j < W; j += 32) acc += row2[j] * xb2[j];
    }
    acc = warp_sum(acc);
    if (lane == 0) y[i] = s2 == 0.0 ? s1 * acc : s1 * acc + s2 * y[i];
  }
}

__global__ void __launch_bounds__(256) k_jtmv(const double* __restrict__ Jp, const double* __restrict__ Js,
                                              const int* __restrict__ colptr, const int* __restrict__ colrows,
                                              long long m_int, int W, const double* __restrict__ x,
                                              const int* __restrict__ skip, double* __restrict__ y) {
  if (skip && *skip) return;
  const int b = blockIdx.x;
  const int c0 = blockIdx.y * 64;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ca = c0 + lane, cb = c0 + 32 + lane;
  double acc0 = 0.0, acc1 = 0.0;
  const int beg = colptr[b], end = colptr[b + 1];
  for (int t = beg + w; t < end; t += 8) {
    const unsigned int ent = (unsigned int)colrows[t];
    const long long r = ent & 0x7fffffffu;
    const double* row = (ent >> 31) ? Js + (size_t)(r - m_int) * W : Jp + (size_t)r * W;
    const double xr = x[r];
    if (ca < W) acc0 += row[ca] * xr;
    if (cb < W) acc1 += row[cb] * xr;
  }
  __shared__ double sh[8][64];
  sh[w][lane] = acc0;
  sh[w][32 + lane] = acc1;
  __syncthreads();
  if (threadIdx.x < 64) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += sh[k][threadIdx.x];
    const int col = c0 + threadIdx.x;
    if (col < W) y[(size_t)b * W + col] = s;
  }
}

// x = R^{-1} b (TRANS = 0) or R^{-T} b (TRANS = 1).
template <int TRANS>
__global__ void __launch_bounds__(256) k_trsv(const double* __restrict__ R, long long ldr, int n,
                                              const double* __restrict__ rhs, double* __restrict__ x,
                                              unsigned int* __restrict__ flags, const unsigned int* __restrict__ epoch_dev,
                                              unsigned int* __restrict__ ticket, unsigned int* __restrict__ err,
                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const unsigned int epoch = *epoch_dev;  // set by k_trsv_prep, which ran before this launch
  __shared__ double sdiag[TB][TB + 1];
  __shared__ double sacc[8][TB];
  __shared__ double srec[TB];
  __shared__ int sblk;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nblk = (n + TB - 1) / TB;
  if (tid == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    sblk = TRANS == 0 ? nblk - 1 - (int)t : (int)t;
  }
  __syncthreads();
  const int k = sblk;
  const int r0 = k * TB;
  const int rows = min(TB, n - r0);
  // diagonal tile (column-major in R)
  for (int idx = tid; idx < TB * TB; idx += 256) {
    const int rr = idx % TB, cc = idx / TB;
    sdiag[rr][cc] = (rr < rows && cc < rows) ? R[(size_t)(r0 + cc) * ldr + r0 + rr] : 0.0;
  }
  // reciprocals of the block's pivots, taken in parallel before any wait so the
  // dependency chain below only multiplies
  if (tid < TB) srec[tid] = tid < rows ? 1.0 / R[(size_t)(r0 + tid) * ldr + r0 + tid] : 0.0;
  double a0 = 0.0, a1 = 0.0;          // TRANS 0: rows lane, lane+32 of the block
  double pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // TRANS 1: columns w + 8 t of the block, partial over lanes
  if (TRANS == 0) {
    for (int j = nblk - 1; j > k; --j) {
      if (tid == 0) wait_flag(flags + j, epoch, err);
      __syncthreads();
      const int c0 = j * TB, cols = min(TB, n - c0);
      for (int cc = w; cc < cols; cc += 8) {
        const double xc = __ldcg(x + c0 + cc);
        const double* col = R + (size_t)(c0 + cc) * ldr + r0;
        if (lane < rows) a0 += col[lane] * xc;
        if (lane + 32 < rows) a1 += col[lane + 32] * xc;
      }
    }
    sacc[w][lane] = a0;
    sacc[w][lane + 32] = a1;
  } else {
    for (int j = 0; j < k; ++j) {
      if (tid == 0) wait_flag(flags + j, epoch, err);
      __syncthreads();
      const int q0 = j * TB;  // full block: j < k < nblk
      const double z0 = __ldcg(x + q0 + lane), z1 = __ldcg(x + q0 + 32 + lane);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int cc = w + 8 * t;
        if (cc < rows) {
          const double* col = R + (size_t)(r0 + cc) * ldr + q0;
          pc[t] += col[lane] * z0 + col[lane + 32] * z1;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const double v = warp_sum(pc[t]);
      if (lane == 0) sacc[0][w + 8 * t] = v;
    }
  }
  __syncthreads();
  if (w == 0) {
    double acc[2];
    for (int h = 0; h < 2; ++h) {
      const int rr = lane + 32 * h;
      double s = 0.0;
      if (TRANS == 0) {
        for (int q = 0; q < 8; ++q) s += sacc[q][rr];
      } else {
        s = sacc[0][rr];
      }
      acc[h] = rr < rows ? rhs[r0 + rr] - s : 0.0;
    }
    // solve the diagonal block in registers: lane owns entries lane, lane+32
    double xv[2] = {0.0, 0.0};
    if (TRANS == 0) {
      for (int i = rows - 1; i >= 0; --i) {
        const int h = i >> 5, ln = i & 31;
        const double num = __shfl_sync(0xffffffffu, acc[h], ln);
        const double xi = num * srec[i];
        if (lane == ln) xv[h] = xi;
        if (lane < i) acc[0] -= sdiag[lane][i] * xi;
        if (lane + 32 < i) acc[1] -= sdiag[lane + 32][i] * xi;
      }
    } else {
      for (int i = 0; i < rows; ++i) {
        const int h = i >> 5, ln = i & 31;
        const double num = __shfl_sync(0xffffffffu, acc[h], ln);
        const double xi = num * srec[i];
        if (lane == ln) xv[h] = xi;
        if (lane > i) acc[0] -= sdiag[i][lane] * xi;
        if (lane + 32 > i) acc[1] -= sdiag[i][lane + 32] * xi;
      }
    }
    if (lane < rows) x[r0 + lane] = xv[0];
    if (lane + 32 < rows) x[r0 + lane + 32] = xv[1];
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + k, epoch);
  }
}

// Next epoch for the block flags (never 0, the initial flag value) and a fresh
// ticket counter; runs before every k_trsv so that replays of a captured graph
// see a new epoch each time.
__global__ void k_trsv_prep(unsigned int* __restrict__ epoch, unsigned int* __restrict__ ticket) {
  unsigned int e = *epoch + 1u;
  *epoch = e == 0u ? 1u : e;
  *ticket = 0u;
}

__global__ void k_partial_dot(const double* __restrict__ a, const double* __restrict__ b, long long n,
                              double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

__global__ void k_finish(const double* __restrict__ partial, int np, int take_sqrt, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) acc += partial[i];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[0] = take_sqrt ? sqrt(acc) : acc;
}

constexpr int kRedBlocks = 304;

}  // namespace

rfm_status rfm_norm2(cudaStream_t st, const double* x, long long n, double* partial, double* out_dev) {
  k_partial_dot<<<kRedBlocks, 256, 0, st>>>(x, x, n, partial);
  RFM_CHECK_LAUNCH();
  k_finish<<<1, 32, 0, st>>>(partial, kRedBlocks, 1, out_dev);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_dot(cudaStream_t st, const double* x, const double* y, long long n, double* partial,
                   double* out_dev) {
  k_partial_dot<<<kRedBlocks, 256, 0, st>>>(x, y, n, partial);
  RFM_CHECK_LAUNCH();
  k_finish<<<1, 32, 0, st>>>(partial, kRedBlocks, 0, out_dev);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_jmv(rfm_problem* p, const double* x, double* y) {
  ProfScope ps(PF_JMV, p->stream);
  rfm_prof_work(PF_JMV, 8.0 * ((double)(p->m + p->m_iface) * p->W + p->m + p->n));
  long long g = (p->m + 7) / 8;
  if (g > 152 * 64) g = 152 * 64;
  k_jmv<<<(int)g, 256, 0, p->stream>>>(p->Jp, p->Js, p->rmeta, p->m, p->m_int, p->W, x, 1.0, 0.0, nullptr, p->skip,
                                       y);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_jmv_axpby(rfm_problem* p, const double* x, double s1, double s2, double* y,
                                const double* s2dev) {
  ProfScope ps(PF_JMV, p->stream);
  rfm_prof_work(PF_JMV, 8.0 * ((double)(p->m + p->m_iface) * p->W + 2.0 * p->m + p->n));
  long long g = (p->m + 7) / 8;
  if (g > 152 * 64) g = 152 * 64;
  k_jmv<<<(int)g, 256, 0, p->stream>>>(p->Jp, p->Js, p->rmeta, p->m, p->m_int, p->W, x, s1, s2, s2dev, p->skip, y);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_jtmv(rfm_problem* p, const double* x, double* y) {
  dim3 grid(p->G, (p->W + 63) / 64);
  ProfScope ps(PF_JTMV, p->stream);
  rfm_prof_work(PF_JTMV, 8.0 * ((double)(p->m + p->m_iface) * p->W + p->m + p->n));
  k_jtmv<<<grid, 256, 0, p->stream>>>(p->Jp, p->Js, p->colptr, p->colrows, p->m_int, p->W, x, p->skip, y);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_trsv(rfm_problem* p, int trans, const double* b, double* x) {
  const int n = (int)p->n;
  const int nblk = (n + TB - 1) / TB;
  if (nblk > RFM_SYNC_WORDS - SYNC_FLAGS) {
    rfm_set_error("trsv: too many blocks");
    return RFM_EINVAL;
  }
  k_trsv_prep<<<1, 1, 0, p->stream>>>(p->sync + SYNC_EPOCH, p->sync + SYNC_TICKET);
  RFM_CHECK_LAUNCH();
  ProfScope ps(PF_TRSV, p->stream);
  rfm_prof_work(PF_TRSV, 8.0 * (double)n * (n + 1) / 2 + 16.0 * n);  // R read once, b and x
  if (trans == 0)
    k_trsv<0><<<nblk, 256, 0, p->stream>>>(p->R, p->ldr, n, b, x, p->sync + SYNC_FLAGS, p->sync + SYNC_EPOCH,
                                           p->sync + SYNC_TICKET, p->sync + SYNC_ERR, p->skip);
  else
    k_trsv<1><<<nblk, 256, 0, p->stream>>>(p->R, p->ldr, n, b, x, p->sync + SYNC_FLAGS, p->sync + SYNC_EPOCH,
                                           p->sync + SYNC_TICKET, p->sync + SYNC_ERR, p->skip);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}
