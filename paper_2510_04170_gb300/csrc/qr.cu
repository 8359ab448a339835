// Householder QR of the sketch B = S_k J (Sec. 4.1, "thin QR B = Q R") giving
// the right preconditioner R.  Blocked right-looking Householder with the
// compact-WY trailing update (Schreiber & Van Loan):
//
//   for each panel of NB columns:
//     k_panel   (cooperative, one CTA per SM slice of rows): the panel's rows
//               stay in shared memory; per column one bounded grid barrier
//               combines the column norm below the pivot and the products of
//               the unscaled column with the rest of the panel, from which
//               every CTA forms v^T A (details at the kernel).  Reflector
//               H = I - tau v v^T, v_0 = 1, beta = -sign(alpha) ||x||.  At the
//               end T (NB x NB, upper) with T_jj = tau_j,
//               T_{:j,j} = -tau_j T_{:j,:j} V_{:,:j}^T v_j.
//     k_vta     W_z = V^T A_trail over a K-slice z (split K, deterministic)
//     k_wt      W2 = T^T sum_z W_z
//     k_update  A_trail -= V W2
//   k_normalise: flip rows of R to a positive diagonal, floor pivots below
//               1e-14 max_j R_jj (rank guard; flag raised).
//
// All sums are reduced in a fixed order, so repeated runs give identical bits.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "rfm_internal.cuh"

namespace {

constexpr int NB = 32;

struct PanelArgs {
  double* A;
  long long lda;
  long long s;
  long long j0;
  int nbw;           // columns in this panel (<= NB)
  int P;             // CTAs (<= 256)
  int chunk;         // rows per CTA
  double* part;      // two buffers of [512][NB + 2] partials (row 511 of each: the pivot row)
  double* gram;      // [P][NB*NB]
  double* tau;       // [n]
  double* T;         // [NB][NB] (row-major T[i][j])
  unsigned int* bar;  // [2]: count, generation
  unsigned int* err;
};

// Grid-wide barrier: an arrival counter bar[0] and a generation word
// bar[BAR_GEN], on different 128-byte lines so that the CTAs polling the
// generation do not contend with the arrivals' atomics.
constexpr int BAR_GEN = 32;

__device__ __forceinline__ void grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned int* err) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(bar + BAR_GEN);
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      st_release(bar + BAR_GEN, g + 1);
    } else {
      wait_flag(bar + BAR_GEN, g + 1, err, 32);
    }
  }
  __syncthreads();
}

// Sum over the P CTAs of partial value idx (stride NB + 2 per CTA) in a fixed
// order: each lane loads its CTAs' values (all loads issued before the adds),
// then the lanes are combined by the warp's butterfly.  Every CTA obtains
// bitwise the same result.
__device__ __forceinline__ double sum_partials(const double* part, int P, int idx, int lane) {
  double t[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = lane + 32 * u;
    t[u] = q < P ? __ldcg(part + q * (NB + 2) + idx) : 0.0;
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += t[u];
  return warp_sum(s);
}

// One grid-wide barrier per column.  Before it, every CTA contributes, for
// its rows below the pivot row j, sigma = sum x_r^2 and p_k = sum x_r A_rk for
// the remaining panel columns k (x = column j, not yet scaled); the CTA that
// holds row j also publishes alpha = A_jj and the pivot row A_jk.  After it,
// every CTA forms beta, tau, 1/(alpha - beta) and
//     w_k = v^T A_k = A_jk + p_k / (alpha - beta)     (v_j = 1, v_r = x_r / (alpha - beta)),
// the same quantities the two-barrier form obtains by reducing v^T A_k after
// scaling.  The partials alternate between two buffers, so a CTA that runs
// ahead into column j + 1 never overwrites values another CTA still reads.
__global__ void __launch_bounds__(256) k_panel(PanelArgs a) {
  extern __shared__ double sp[];  // [NB][chunk] column-major panel slice
  __shared__ double sw[NB];       // w_k, then tau w_k
  __shared__ double sv[NB + 2];   // reduced sigma and p_k
  const int c = blockIdx.x;
  const long long rbeg = a.j0 + (long long)c * a.chunk;
  const long long rend = min(a.s, rbeg + a.chunk);
  const int nr = rbeg < rend ? (int)(rend - rbeg) : 0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int chunk = a.chunk;
  for (int jj = 0; jj < a.nbw; ++jj) {
    const double* col = a.A + (size_t)(a.j0 + jj) * a.lda + rbeg;
    for (int r = tid; r < nr; r += blockDim.x) sp[jj * chunk + r] = col[r];
  }
  __syncthreads();
  for (int jj = 0; jj < a.nbw; ++jj) {
    const long long j = a.j0 + jj;  // pivot row
    double* v = sp + jj * chunk;
    const int rest = a.nbw - jj - 1;
    double* part = a.part + (size_t)(jj & 1) * 512 * (NB + 2);  // [P][NB + 2] this column's partials
    double* piv = part + (size_t)511 * (NB + 2);                 // alpha, A_jk of the pivot row
    // local partials: slot 0 sigma (kk = -1), slot 1 + kk p_k; one warp per slot
    for (int kk = w - 1; kk < rest; kk += (blockDim.x >> 5)) {
      const double* ck = kk < 0 ? v : sp + (jj + 1 + kk) * chunk;
      double acc = 0.0;
      for (int r = lane; r < nr; r += 32)
        if (rbeg + r > j) acc += v[r] * ck[r];
      acc = warp_sum(acc);
      if (lane == 0) part[c * (NB + 2) + 1 + kk] = acc;
    }
    if (j >= rbeg && j < rend && tid <= rest) piv[tid] = sp[(jj + tid) * chunk + (j - rbeg)];
    grid_barrier(a.bar, a.P, a.err);
    for (int idx = w; idx <= rest; idx += (blockDim.x >> 5)) {
      const double sm = sum_partials(part, a.P, idx, lane);
      if (lane == 0) sv[idx] = sm;
    }
    __syncthreads();
    const double sigma = sv[0], alpha = __ldcg(piv);
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (sigma != 0.0) {
      const double nrm = sqrt(alpha * alpha + sigma);
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    if (tid < rest) sw[tid] = tau * (__ldcg(piv + 1 + tid) + scale * sv[1 + tid]);  // tau w_k
    // v_r = x_r / (alpha - beta) below the pivot, v_j = 1
    if (tau != 0.0)
      for (int r = tid; r < nr; r += blockDim.x)
        if (rbeg + r > j) v[r] *= scale;
    __syncthreads();
    if (tau != 0.0) {
      for (int kk = 0; kk < rest; ++kk) {
        const double f = sw[kk];
        double* ck = sp + (jj + 1 + kk) * chunk;
        for (int r = tid; r < nr; r += blockDim.x) {
          const long long gr = rbeg + r;
          if (gr >= j) ck[r] -= (gr == j ? 1.0 : v[r]) * f;
        }
      }
    }
    __syncthreads();
    if (tid == 0 && j >= rbeg && j < rend) v[j - rbeg] = beta;
    if (c == 0 && tid == 0) a.tau[j] = tau;
    __syncthreads();
  }
  // partial Gram V^T V of this CTA's rows (v_j = 1 on the pivot, 0 above)
  for (int pq = tid; pq < a.nbw * a.nbw; pq += blockDim.x) {
    const int p = pq / a.nbw, q = pq % a.nbw;
    double acc = 0.0;
    if (p <= q) {
      for (int r = 0; r < nr; ++r) {
        const long long gr = rbeg + r;
        const double vp = gr < a.j0 + p ? 0.0 : (gr == a.j0 + p ? 1.0 : sp[p * chunk + r]);
        const double vq = gr < a.j0 + q ? 0.0 : (gr == a.j0 + q ? 1.0 : sp[q * chunk + r]);
        acc += vp * vq;
      }
    }
    a.gram[(size_t)c * NB * NB + pq] = acc;
  }
  // write the panel back (R entries on and above the diagonal, v below)
  for (int jj = 0; jj < a.nbw; ++jj) {
    double* col = a.A + (size_t)(a.j0 + jj) * a.lda + rbeg;
    for (int r = tid; r < nr; r += blockDim.x) col[r] = sp[jj * chunk + r];
  }
  grid_barrier(a.bar, a.P, a.err);
  if (c == 0) {
    __shared__ double G[NB][NB + 1];
    __shared__ double Ts[NB][NB + 1];
    for (int pq = tid; pq < a.nbw * a.nbw; pq += blockDim.x) {
      // sum over CTAs in increasing order, eight loads in flight
      double s = 0.0;
      int q = 0;
      for (; q + 8 <= a.P; q += 8) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = __ldcg(a.gram + (size_t)(q + u) * NB * NB + pq);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += t[u];
      }
      for (; q < a.P; ++q) s += __ldcg(a.gram + (size_t)q * NB * NB + pq);
      G[pq / a.nbw][pq % a.nbw] = s;
    }
    for (int pq = tid; pq < NB * (NB + 1); pq += blockDim.x) Ts[pq / (NB + 1)][pq % (NB + 1)] = 0.0;
    __syncthreads();
    // T column by column (compact WY: T[:j, j] = -tau_j T[:j, :j] G[:j, j]); rows in parallel
    for (int jj = 0; jj < a.nbw; ++jj) {
      const double tj = __ldcg(a.tau + a.j0 + jj);
      if (tid < jj) {
        double s = 0.0;
        for (int l = tid; l < jj; ++l) s += Ts[tid][l] * G[l][jj];
        Ts[tid][jj] = -tj * s;
      } else if (tid == jj) {
        Ts[jj][jj] = tj;
      }
      __syncthreads();
    }
    for (int pq = tid; pq < NB * NB; pq += blockDim.x) {
      const int p = pq / NB, q = pq % NB;
      a.T[pq] = (p < a.nbw && q < a.nbw) ? Ts[p][q] : 0.0;
    }
  }
}

// Vector of panel column p at global row gr (unit pivot, zero above).
__device__ __forceinline__ double vval(const double* A, long long lda, long long j0, int p, long long gr) {
  const long long piv = j0 + p;
  if (gr < piv) return 0.0;
  if (gr == piv) return 1.0;
  return A[(size_t)(j0 + p) * lda + gr];
}

// Wp[z][p][col] = sum_{r in K-slice z} v_p(r) A[r, j1 + col]
__global__ void __launch_bounds__(256) k_vta(const double* __restrict__ A, long long lda, long long s, long long j0,
                                             int nbw, long long j1, long long nt, long long kchunk,
                                             double* __restrict__ Wp) {
  __shared__ double Vs[32][NB + 1];
  __shared__ double As[32][64 + 1];
  const int tid = threadIdx.x;
  const long long col0 = (long long)blockIdx.x * 64;
  const int z = blockIdx.y;
  const long long kb = j0 + (long long)z * kchunk;
  const long long ke = min(s, kb + kchunk);
  const int ay = tid >> 4, cx = tid & 15;
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (long long r0 = kb; r0 < ke; r0 += 32) {
    for (int idx = tid; idx < 32 * NB; idx += 256) {
      const int rr = idx & 31, p = idx >> 5;
      const long long gr = r0 + rr;
      Vs[rr][p] = (gr < ke && p < nbw) ? vval(A, lda, j0, p, gr) : 0.0;
    }
    for (int idx = tid; idx < 32 * 64; idx += 256) {
      const int rr = idx & 31, cc = idx >> 5;
      const long long gr = r0 + rr, gc = col0 + cc;
      As[rr][cc] = (gr < ke && gc < nt) ? A[(size_t)(j1 + gc) * lda + gr] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const double v0 = Vs[rr][ay], v1 = Vs[rr][ay + 16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double av = As[rr][cx + 16 * q];
        acc[0][q] += v0 * av;
        acc[1][q] += v1 * av;
      }
    }
    __syncthreads();
  }
  for (int h = 0; h < 2; ++h)
    for (int q = 0; q < 4; ++q) {
      const long long gc = col0 + cx + 16 * q;
      const int p = ay + 16 * h;
      if (gc < nt) Wp[((size_t)z * NB + p) * nt + gc] = acc[h][q];
    }
}

// W2[p][col] = sum_q T[q][p] sum_z Wp[z][q][col]
__global__ void k_wt(const double* __restrict__ Wp, int nz, const double* __restrict__ T, int nbw, long long nt,
                     double* __restrict__ W2) {
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= nt) return;
  double wv[NB];
  for (int q = 0; q < NB; ++q) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += Wp[((size_t)z * NB + q) * nt + col];
    wv[q] = s;
  }
  for (int p = 0; p < NB; ++p) {
    double s = 0.0;
    for (int q = 0; q <= p && q < nbw; ++q) s += T[q * NB + p] * wv[q];
    W2[(size_t)p * nt + col] = p < nbw ? s : 0.0;
  }
}

// A[r, j1 + col] -= sum_p v_p(r) W2[p][col] for r in [j0, s)
__global__ void __launch_bounds__(256) k_update(double* __restrict__ A, long long lda, long long s, long long j0,
                                                int nbw, long long j1, long long nt, const double* __restrict__ W2) {
  __shared__ double Vs[NB][128];
  __shared__ double Ws[NB][64];
  const int tid = threadIdx.x;
  const long long r0 = j0 + (long long)blockIdx.x * 128;
  const long long c0 = (long long)blockIdx.y * 64;
  for (int idx = tid; idx < NB * 128; idx += 256) {
    const int rr = idx & 127, p = idx >> 7;
    const long long gr = r0 + rr;
    Vs[p][rr] = (gr < s && p < nbw) ? vval(A, lda, j0, p, gr) : 0.0;
  }
  for (int idx = tid; idx < NB * 64; idx += 256) {
    const int cc = idx & 63, p = idx >> 6;
    const long long gc = c0 + cc;
    Ws[p][cc] = gc < nt ? W2[(size_t)p * nt + gc] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 31, ty = tid >> 5;
  double acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[i][q] = 0.0;
#pragma unroll 4
  for (int p = 0; p < NB; ++p) {
    double vv[4], ww[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) vv[i] = Vs[p][tx + 32 * i];
#pragma unroll
    for (int q = 0; q < 8; ++q) ww[q] = Ws[p][ty + 8 * q];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[i][q] += vv[i] * ww[q];
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long gc = c0 + ty + 8 * q;
    if (gc >= nt) continue;
    double* colp = A + (size_t)(j1 + gc) * lda;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long gr = r0 + tx + 32 * i;
      if (gr < s) colp[gr] -= acc[i][q];
    }
  }
}

__global__ void k_diag(const double* __restrict__ A, long long lda, long long n, double* __restrict__ dg) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dg[i] = A[(size_t)i * lda + i];
}

// Flip row i of R when R_ii < 0 (upper triangle only).
__global__ void k_flip(double* __restrict__ A, long long lda, long long n, const double* __restrict__ dg) {
  const long long col = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= col; i += (long long)gridDim.x * blockDim.x)
    if (dg[i] < 0.0) A[(size_t)col * lda + i] = -A[(size_t)col * lda + i];
}

__global__ void k_floor(double* __restrict__ A, long long lda, long long n, unsigned int* flag) {
  __shared__ double sh[40];
  double mx = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, A[(size_t)i * lda + i]);
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) sh[32] = v;
  }
  __syncthreads();
  const double fl = 1e-14 * sh[32];
  for (long long i = threadIdx.x; i < n; i += blockDim.x)
    if (A[(size_t)i * lda + i] < fl) {
      A[(size_t)i * lda + i] = fl;
      atomicExch(flag, 1u);
    }
}

struct QrScratch {
  double* part;
  double* gram;
  double* tau;
  double* T;
  double* Wp;
  double* W2;
  double* dg;
};

}  // namespace

long long rfm_householder_scratch(long long s, long long n) {
  const long long P = 1024;
  const long long maxz = 64;
  return P * (NB + 2) + P * NB * NB + n + NB * NB + maxz * NB * n + NB * n + n + 64;
}

namespace {

QrScratch carve(double* scratch, long long n) {
  QrScratch q;
  double* w = scratch;
  q.part = w; w += 1024 * (NB + 2);
  q.gram = w; w += 1024LL * NB * NB;
  q.tau = w; w += n;
  q.T = w; w += NB * NB;
  q.Wp = w; w += 64LL * NB * n;
  q.W2 = w; w += (long long)NB * n;
  q.dg = w;
  return q;
}

rfm_status qr_init_device() {
  const cudaError_t attr = rfm_smem_attr((const void*)k_panel, 200 * 1024);  // once per device
  if (attr != cudaSuccess || rfm_num_sms() == 0) {
    rfm_set_error("householder: device set-up failed");
    return RFM_ECUDA;
  }
  return RFM_OK;
}

// Householder factorisation of columns [c0, c1) (rows c0..s) in NB-wide
// panels; the FP64 compact-WY update of each panel is applied to the columns
// up to cend (cend >= c1).
rfm_status factor_range(double* A, long long s, long long lda, long long c0, long long c1, long long cend,
                        cudaStream_t st, const QrScratch& q, unsigned int* sync, int panel_cap) {
  unsigned int* bar = sync + SYNC_BAR;
  unsigned int* err = sync + SYNC_ERR;
  const int nsm = rfm_num_sms();
  for (long long j0 = c0; j0 < c1; j0 += NB) {
    const int nbw = (int)std::min<long long>(NB, c1 - j0);
    const long long rows = s - j0;
    // rows per CTA: at least 64, at most what fits in 200 KB of shared memory
    const long long maxchunk = (200LL * 1024) / (NB * (long long)sizeof(double));
    const long long cap = panel_cap > 0 ? std::min(panel_cap, nsm) : nsm;
    long long P = std::min<long long>(std::min<long long>((rows + 63) / 64, cap), 256);  // k_panel sums <= 256 partials
    if (P < 1) P = 1;
    long long chunk = (rows + P - 1) / P;
    if (chunk > maxchunk && cap < nsm) {  // the cap would overflow shared memory: take the fewest CTAs that fit
      P = std::min<long long>((rows + maxchunk - 1) / maxchunk, nsm);
      chunk = (rows + P - 1) / P;
    }
    if (chunk > maxchunk) {
      rfm_set_error("householder: sketch too tall for the panel kernel");
      return RFM_EINVAL;
    }
    PanelArgs a;
    a.A = A; a.lda = lda; a.s = s; a.j0 = j0; a.nbw = nbw; a.P = (int)P; a.chunk = (int)chunk;
    a.part = q.part; a.gram = q.gram; a.tau = q.tau; a.T = q.T; a.bar = bar; a.err = err;
    void* args[] = {&a};
    const size_t smem = (size_t)NB * chunk * sizeof(double);
    {
      ProfScope ps(PF_QR_PANEL, st);
      RFM_CUDA(cudaLaunchCooperativeKernel((const void*)k_panel, dim3((unsigned)P), dim3(256), args, smem, st));
      rfm_count_launch();
    }
    const long long j1 = j0 + nbw;
    const long long nt = cend - j1;
    if (nt <= 0) continue;
    const long long ctiles = (nt + 63) / 64;
    long long nz = (2LL * nsm + ctiles - 1) / ctiles;
    nz = std::max<long long>(1, std::min<long long>(nz, std::min<long long>(64, (rows + 255) / 256)));
    const long long kchunk = (rows + nz - 1) / nz;
    nz = (rows + kchunk - 1) / kchunk;
    {
      ProfScope ps(PF_QR_VTA, st);
      rfm_prof_work(PF_QR_VTA, 2.0 * nbw * (double)nt * (double)rows);  // FP64 flops
      k_vta<<<dim3((unsigned)ctiles, (unsigned)nz), 256, 0, st>>>(A, lda, s, j0, nbw, j1, nt, kchunk, q.Wp);
      RFM_CHECK_LAUNCH();
      k_wt<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(q.Wp, (int)nz, q.T, nbw, nt, q.W2);
      RFM_CHECK_LAUNCH();
    }
    ProfScope psu(PF_QR_UPDATE, st);
    rfm_prof_work(PF_QR_UPDATE, 2.0 * nbw * (double)nt * (double)rows);  // FP64 flops
    k_update<<<dim3((unsigned)((rows + 127) / 128), (unsigned)ctiles), 256, 0, st>>>(A, lda, s, j0, nbw, j1, nt, q.W2);
    RFM_CHECK_LAUNCH();
  }
  return RFM_OK;
}

// Positive diagonal and pivot floor; reads back the rank flag and the error word.
rfm_status finish_r(double* A, long long n, long long lda, cudaStream_t st, const QrScratch& q, unsigned int* sync,
                    int* rank_flag_host) {
  k_diag<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, n, q.dg);
  RFM_CHECK_LAUNCH();
  k_flip<<<dim3((unsigned)std::min<long long>(64, (n + 255) / 256), (unsigned)n), 256, 0, st>>>(A, lda, n, q.dg);
  RFM_CHECK_LAUNCH();
  RFM_CUDA(cudaMemsetAsync(sync + SYNC_BAR + 2, 0, sizeof(unsigned int), st));
  k_floor<<<1, 1024, 0, st>>>(A, lda, n, sync + SYNC_BAR + 2);
  RFM_CHECK_LAUNCH();
  if (rank_flag_host) {
    unsigned int hv[2] = {0, 0};
    RFM_CUDA(cudaMemcpyAsync(hv, sync + SYNC_BAR + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    RFM_CUDA(cudaMemcpyAsync(hv + 1, sync + SYNC_ERR, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    RFM_CUDA(cudaStreamSynchronize(st));
    *rank_flag_host = (int)hv[0];
    if (hv[1]) {
      rfm_set_error("householder: a bounded device wait timed out (code " + std::to_string(hv[1]) + ")");
      return RFM_ETIMEOUT;
    }
  }
  return RFM_OK;
}

}  // namespace

rfm_status rfm_householder_inplace(double* A, long long s, long long n, long long lda, cudaStream_t st,
                                   double* scratch, long long scratch_len, unsigned int* sync, int* rank_flag_host,
                                   int panel_cap, long long ncols) {
  if (s < n || n <= 0) {
    rfm_set_error("householder: need s >= n > 0");
    return RFM_EINVAL;
  }
  if (scratch_len < rfm_householder_scratch(s, n)) {
    rfm_set_error("householder: scratch too small");
    return RFM_EINVAL;
  }
  RFM_TRY(qr_init_device());
  const QrScratch q = carve(scratch, n);
  RFM_CUDA(cudaMemsetAsync(sync + SYNC_BAR, 0, 2 * sizeof(unsigned int), st));
  const long long c1 = ncols < 0 ? n : std::min<long long>(n, ((ncols + NB - 1) / NB) * NB);
  RFM_TRY(factor_range(A, s, lda, 0, c1, n, st, q, sync, panel_cap));
  return finish_r(A, n, lda, st, q, sync, rank_flag_host);
}

// ---------------------------------------------------------------------------
// Allocation-free Householder R.
//
// Same computation as rfm_householder_r, for callers that must not allocate
// device memory while they run: services that reserve all device memory up
// front through their own pool (where a cudaMalloc fails or implicitly
// synchronises the device and stalls other streams), or loops with fixed
// latency budgets.  The QR scratch lives in file-scope device arrays of fixed
// size (17.2 MB of scratch + 16 KB of barrier words per GPU that loads the
// library, held until the process exits), sized for n <= 512 columns.
// Every call shares these arrays and they keep the last call's contents;
// calls that overlap on the GPU (two streams, or two host threads) race on
// them and must be serialised by the caller.
#define RFM_NOALLOC_MAX_N 512
#define RFM_NOALLOC_MAX_DEVICES 64

namespace {
constexpr long long kNoallocScratch = 1024LL * (NB + 2) + 1024LL * NB * NB + RFM_NOALLOC_MAX_N + NB * NB +
                                      64LL * NB * RFM_NOALLOC_MAX_N + (long long)NB * RFM_NOALLOC_MAX_N +
                                      RFM_NOALLOC_MAX_N + 64;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratch];
static __device__ __align__(256) unsigned int g_noalloc_sync[RFM_SYNC_WORDS];

namespace {

struct NoallocDev {
  double* scratch = nullptr;
  unsigned int* sync = nullptr;
};
NoallocDev g_noalloc_dev[RFM_NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

__global__ void k_noalloc_copy_r(const double* __restrict__ A, long long lda, long long n, double* __restrict__ R) {
  const long long col = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    R[(size_t)col * n + i] = i <= col ? A[(size_t)col * lda + i] : 0.0;
}

// Device addresses of the fixed arrays for the current device, resolved once
// per device (host code must not pass the arrays' host-side names to kernels).
rfm_status noalloc_setup(NoallocDev* out) {
  int dev = 0;
  RFM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= RFM_NOALLOC_MAX_DEVICES) {
    rfm_set_error("rfm_householder_r_noalloc: device ordinal out of range");
    return RFM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocDev& d = g_noalloc_dev[dev];
  if (!d.scratch) {
    void* ps = nullptr;
    void* py = nullptr;
    cudaError_t e1 = cudaGetSymbolAddress(&ps, g_noalloc_scratch);
    if (e1 != cudaSuccess) {
      rfm_set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e1));
      return RFM_ECUDA;
    }
    cudaError_t e2 = cudaGetSymbolAddress(&py, g_noalloc_sync);
    if (e2 != cudaSuccess) {
      rfm_set_error(std::string("cudaGetSymbolAddress(sync): ") + cudaGetErrorString(e2));
      return RFM_ECUDA;
    }
    d.scratch = static_cast<double*>(ps);
    d.sync = static_cast<unsigned int*>(py);
  }
  *out = d;
  return RFM_OK;
}

}  // namespace

extern "C" rfm_status rfm_householder_r_noalloc(double* A_dev, int64_t s, int64_t n, void* cuda_stream,
                                                double* R_dev, int* rank_flag_host) {
  if (!A_dev || !R_dev || n <= 0 || s < n) {
    rfm_set_error("rfm_householder_r_noalloc: need A, R and s >= n > 0");
    return RFM_EINVAL;
  }
  if (n > RFM_NOALLOC_MAX_N) {
    rfm_set_error("rfm_householder_r_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                  std::to_string(RFM_NOALLOC_MAX_N) + " columns; use rfm_householder_r");
    return RFM_EINVAL;
  }
  NoallocDev d;
  RFM_TRY(noalloc_setup(&d));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // barrier counters, flags and the error word must start at zero
  RFM_CUDA(cudaMemsetAsync(d.sync, 0, RFM_SYNC_WORDS * sizeof(unsigned int), st));
  int flag = 0;
  RFM_TRY(rfm_householder_inplace(A_dev, s, n, s, st, d.scratch, kNoallocScratch, d.sync, &flag));
  dim3 grid((unsigned)std::min<long long>(64, (n + 255) / 256), (unsigned)n);
  k_noalloc_copy_r<<<grid, 256, 0, st>>>(A_dev, s, n, R_dev);
  RFM_CHECK_LAUNCH();
  RFM_CUDA(cudaStreamSynchronize(st));
  if (rank_flag_host) *rank_flag_host = flag;
  return RFM_OK;
}

// ---------------------------------------------------------------------------
// Householder QR with the trailing update on the tensor cores.
//
// Outer blocks of QB = 128 columns: inside a block the 32-wide panels and their
// FP64 updates run as above; the block's reflectors V (rows x 128, unit
// diagonal) then update the trailing matrix in compact-WY form
//     W = V^T A_t,  W2 = T^T W,  A_t -= V W2
// with both products on the emulated-FP64 tensor-core GEMM (digit splitting,
// exact level accumulation).  T (128 x 128) comes from the Gram V^T V, which
// the first product returns next to W, and the reflector coefficients,
// T_jj = tau_j, T_{:j,j} = -tau_j T_{:j,:j} G_{:j,j}.

rfm_status rfm_oz_slice_house_vt(const double* A, long long lda, long long j0, long long nb, long long K, int ndig,
                                 int* e, uint16_t* out, cudaStream_t st);
rfm_status rfm_oz_slice_house_v(const double* A, long long lda, long long j0, long long rows, long long nb, int ndig,
                                int* e, uint16_t* out, cudaStream_t st);
// Digit slices written into row tiles rt0 .. of planes holding plane_rtiles row
// tiles each, so that several slices form one GEMM operand.
rfm_status rfm_oz_slice_strided_at(const double* base, long long si, long long sk, long long R, long long K, int ndig,
                                   int tile_rows, int* e, uint16_t* out, long long plane_rtiles, long long rt0,
                                   cudaStream_t st);
rfm_status rfm_oz_slice_house_vt_at(const double* A, long long lda, long long j0, long long nb, long long K, int ndig,
                                    int tile_rows, int* e, uint16_t* out, long long plane_rtiles, long long rt0,
                                    cudaStream_t st);

namespace {

constexpr int QB = 128;
constexpr int QDIG = 8;

// T from G and tau, column by column.  One CTA of QB threads; T is kept in
// dynamic shared memory (QB x (QB+1) doubles).
__global__ void k_block_t(const double* __restrict__ G, const double* __restrict__ tau, int nbw,
                          double* __restrict__ T) {
  extern __shared__ double Ts[];  // [QB][QB + 1]
  for (int idx = threadIdx.x; idx < QB * (QB + 1); idx += blockDim.x) Ts[idx] = 0.0;
  __syncthreads();
  const int i = threadIdx.x;
  for (int j = 0; j < nbw; ++j) {
    const double tj = tau[j];
    double v = 0.0;
    if (i < j) {
      for (int l = i; l < j; ++l) v += Ts[i * (QB + 1) + l] * G[l * QB + j];
      v = -tj * v;
    }
    __syncthreads();
    if (i < j) Ts[i * (QB + 1) + j] = v;
    if (i == j) Ts[j * (QB + 1) + j] = tj;
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < QB * QB; idx += blockDim.x) T[idx] = Ts[(idx / QB) * (QB + 1) + idx % QB];
}


}  // namespace

long long rfm_householder_emulated_bytes(long long s, long long n) {
  long long b = 0;
  b += rfm_oz_digit_bytes(QB, s, QDIG, 128);  // V^T
  b += rfm_oz_digit_bytes(n + QB, s, QDIG, 64);  // [V, A_t]: the Gram and V^T A_t in one product
  b += rfm_oz_digit_bytes(s, QB, QDIG, 128);  // V
  b += rfm_oz_digit_bytes(n, QB, QDIG, 64);   // W2
  b += 8LL * (2LL * QB * (n + QB) + QB * QB);  // [G, W], W2, T
  b += 8LL * 8 * QB * (n + QB);  // split-K partials of V^T [V, A_t]
  b += 4LL * (QB + n + QB + s + n) + 4096;
  return b;
}

rfm_status rfm_householder_emulated(double* A, long long s, long long n, long long lda, cudaStream_t st,
                                    double* scratch, long long scratch_len, unsigned int* sync, void* emu,
                                    long long emu_bytes, int* rank_flag_host, int panel_cap, long long ncols) {
  if (s < n || n <= 0) {
    rfm_set_error("householder: need s >= n > 0");
    return RFM_EINVAL;
  }
  if (scratch_len < rfm_householder_scratch(s, n) || emu_bytes < rfm_householder_emulated_bytes(s, n)) {
    rfm_set_error("householder: scratch too small");
    return RFM_EINVAL;
  }
  RFM_TRY(qr_init_device());
  const cudaError_t t_attr = rfm_smem_attr((const void*)k_block_t, (int)(QB * (QB + 1) * sizeof(double)));
  if (t_attr != cudaSuccess) {
    rfm_set_error("householder: k_block_t shared-memory attribute");
    return RFM_ECUDA;
  }
  const QrScratch q = carve(scratch, n);
  char* w = static_cast<char*>(emu);
  auto take = [&](long long bytes) {
    char* r = w;
    w += (bytes + 255) & ~255LL;
    return r;
  };
  uint16_t* d_vt = reinterpret_cast<uint16_t*>(take(rfm_oz_digit_bytes(QB, s, QDIG, 128)));
  uint16_t* d_at = reinterpret_cast<uint16_t*>(take(rfm_oz_digit_bytes(n + QB, s, QDIG, 64)));
  uint16_t* d_v = reinterpret_cast<uint16_t*>(take(rfm_oz_digit_bytes(s, QB, QDIG, 128)));
  uint16_t* d_w2 = reinterpret_cast<uint16_t*>(take(rfm_oz_digit_bytes(n, QB, QDIG, 64)));
  double* Wm = reinterpret_cast<double*>(take(8LL * QB * (n + QB)));  // [G, W] = V^T [V, A_t]
  double* W2 = reinterpret_cast<double*>(take(8LL * QB * n));
  double* T = reinterpret_cast<double*>(take(8LL * QB * QB));
  const long long part_elems = 8LL * QB * (n + QB);
  double* part = reinterpret_cast<double*>(take(8LL * part_elems));
  int* e_vt = reinterpret_cast<int*>(take(4LL * QB));
  int* e_at = reinterpret_cast<int*>(take(4LL * (n + QB)));
  int* e_v = reinterpret_cast<int*>(take(4LL * s));
  int* e_w2 = reinterpret_cast<int*>(take(4LL * n));
  unsigned int* err = sync + SYNC_ERR;
  RFM_CUDA(cudaMemsetAsync(sync + SYNC_BAR, 0, 2 * sizeof(unsigned int), st));
  const long long cstop = ncols < 0 ? n : std::min<long long>(n, ncols);
  for (long long J0 = 0; J0 < cstop; J0 += QB) {
    const long long c1 = std::min<long long>(n, J0 + QB);
    const int nbw = (int)(c1 - J0);
    const long long rows = s - J0;
    const long long nt = n - c1;
    RFM_TRY(factor_range(A, s, lda, J0, c1, c1, st, q, sync, panel_cap));
    if (nt <= 0) break;
    {
      // One emulated product gives the block's Gram and V^T A_t: its B operand
      // is [V, A_t] (V^T as the first two 64-row tiles, then the trailing
      // columns), so C = [G, W] with G = V^T V (exactly symmetric: the digit
      // pairs (p, q) and (q, p) give the same integer level sums).  T then
      // comes from G and tau, T_jj = tau_j, T_{:j,j} = -tau_j T_{:j,:j} G_{:j,j}.
      ProfScope ps(PF_QR_VTA, st);
      const long long prt = 2 + (nt + 63) / 64;  // row tiles of the B operand
      RFM_TRY(rfm_oz_slice_house_vt(A, lda, J0, nbw, rows, QDIG, e_vt, d_vt, st));
      RFM_TRY(rfm_oz_slice_house_vt_at(A, lda, J0, nbw, rows, QDIG, 64, e_at, d_at, prt, 0, st));
      RFM_TRY(rfm_oz_slice_strided_at(A + (size_t)c1 * lda + J0, lda, 1, nt, rows, QDIG, 64, e_at + QB, d_at, prt, 2,
                                      st));
      RFM_TRY(rfm_oz_gemm_part(d_vt, QDIG, e_vt, d_at, QDIG, e_at, nbw, QB + nt, rows, QDIG + 1, Wm, QB, 0, err, st,
                               part, part_elems));
      k_block_t<<<1, QB, QB * (QB + 1) * sizeof(double), st>>>(Wm, q.tau + J0, nbw, T);
      RFM_CHECK_LAUNCH();
      // W2 = T^T W on the emulated GEMM as well (M = K = 128, N = nt): the
      // digit buffers of V^T and of W2 are free at this point of the stream.
      // T is stored row-major, T(q, p) = T[q QB + p], so T^T(p, q) = T[p + q QB].
      RFM_TRY(rfm_oz_slice_strided(T, 1, QB, nbw, nbw, QDIG, 128, e_vt, d_vt, st));
      RFM_TRY(rfm_oz_slice_strided(Wm + (size_t)QB * QB, QB, 1, nt, nbw, QDIG, 64, e_w2, d_w2, st));
      RFM_TRY(rfm_oz_gemm(d_vt, QDIG, e_vt, d_w2, QDIG, e_w2, nbw, nt, nbw, QDIG + 1, W2, QB, 0, err, st));
    }
    {
      ProfScope ps(PF_QR_UPDATE, st);
      RFM_TRY(rfm_oz_slice_house_v(A, lda, J0, rows, nbw, QDIG, e_v, d_v, st));
      RFM_TRY(rfm_oz_slice_strided(W2, QB, 1, nt, nbw, QDIG, 64, e_w2, d_w2, st));
      RFM_TRY(rfm_oz_gemm(d_v, QDIG, e_v, d_w2, QDIG, e_w2, rows, nt, nbw, QDIG + 1, A + (size_t)c1 * lda + J0, lda,
                          1, err, st));
    }
  }
  return finish_r(A, n, lda, st, q, sync, rank_flag_host);
}
