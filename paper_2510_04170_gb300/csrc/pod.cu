// Function-space basis of converged solutions for the learned warm start.
//
// Coefficient vectors of RFM solutions cancel heavily (|c| is many orders of
// magnitude above |u| = |Phi c|), so a network cannot regress c directly.  The
// snapshots c_j are centred (c_j - cbar) and orthonormalised in the L2 inner
// product of u over a set of evaluation points (sum over points of u(x) v(x),
// divided by their number) by modified Gram-Schmidt with column pivoting
// (Businger-Golub: at every step the remaining snapshot of largest norm).  The
// same column operations carried on the coefficient vectors give modes U_k
// with u(U_k) orthonormal, and every snapshot gets coordinates Z_j with
// c_j - cbar = sum_k Z_jk U_k up to the truncation tolerance; the network
// learns x -> Z, and c_0 = cbar + sum_k z_k U_k is formed in FP64.
//
// Layout: snapshots row-major [N][n] (one snapshot contiguous), point values
// [N][len] with len = npts * fields, Z [N][N] with Z[j][k] the coordinate of
// snapshot j on mode k.  Every reduction is a fixed-order block tree
// (deterministic).
#include <math.h>
#include <stdint.h>

#include <vector>

#include "rfm_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// cbar[i] = (1/N) sum_j C[j][i]; D[j][i] = C[j][i] - cbar[i]
__global__ void k_centre(const double* __restrict__ C, int N, long long n, double* __restrict__ mean,
                         double* __restrict__ D) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += C[(size_t)j * n + i];
    const double m = s / N;
    mean[i] = m;
    for (int j = 0; j < N; ++j) D[(size_t)j * n + i] = C[(size_t)j * n + i] - m;
  }
}

// sq[cols[b]] = sum_q V[cols[b]][q]^2, one block per listed column
__global__ void k_colsq(const double* __restrict__ V, long long len, const int* __restrict__ cols,
                        double* __restrict__ sq) {
  __shared__ double sh[32];
  const int j = cols[blockIdx.x];
  const double* v = V + (size_t)j * len;
  double s = 0.0;
  for (long long q = threadIdx.x; q < len; q += blockDim.x) s += v[q] * v[q];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) sq[j] = s;
}

// Normalise pivot column p by rkk: V_p /= rkk, D_p /= rkk; copy D_p to U_k.
__global__ void k_normalise(double* __restrict__ V, long long len, double* __restrict__ D, long long n, int p,
                            double rkk, double* __restrict__ Uk) {
  const double inv = 1.0 / rkk;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < len; q += (long long)gridDim.x * blockDim.x)
    V[(size_t)p * len + q] *= inv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = D[(size_t)p * n + i] * inv;
    D[(size_t)p * n + i] = d;
    Uk[i] = d;
  }
}

// For each listed column j: r = <V_p, V_j>; V_j -= r V_p; D_j -= r D_p; Z[j][k] = r.
__global__ void k_project(double* __restrict__ V, long long len, double* __restrict__ D, long long n, int p,
                          const int* __restrict__ cols, double* __restrict__ Z, int N, int k) {
  __shared__ double sh[32];
  __shared__ double r_sh;
  const int j = cols[blockIdx.x];
  const double* q = V + (size_t)p * len;
  double* v = V + (size_t)j * len;
  double s = 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) s += q[t] * v[t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    r_sh = s;
    Z[(size_t)j * N + k] = s;
  }
  __syncthreads();
  const double r = r_sh;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) v[t] -= r * q[t];
  const double* u = D + (size_t)p * n;
  double* d = D + (size_t)j * n;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) d[i] -= r * u[i];
}

// c[b][i] = mean[i] + scale * sum_k y[b][k] U[k][i]
__global__ void k_combine(const double* __restrict__ mean, const double* __restrict__ U, long long n, int r,
                          const float* __restrict__ y, int batch, double scale, double* __restrict__ c) {
  const long long total = (long long)batch * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n, i = t - b * n;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += (double)y[b * r + k] * U[(size_t)k * n + i];
    c[t] = mean[i] + scale * s;
  }
}

int blocks_for(long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

}  // namespace

extern "C" {

rfm_status rfm_function_basis(const rfm_problem* p, const double* C_dev, int N, const double* pts_dev, int64_t npts,
                              double tol, double* mean_dev, double* U_dev, double* Z_dev, int* rank_host) {
  if (!p || !C_dev || N <= 0 || !pts_dev || npts <= 0 || !(tol >= 0.0) || !mean_dev || !U_dev || !Z_dev ||
      !rank_host) {
    rfm_set_error("rfm_function_basis: bad argument");
    return RFM_EINVAL;
  }
  cudaStream_t st = p->stream;
  const long long n = p->n, len = npts * p->fields;
  double *D = nullptr, *V = nullptr, *sq = nullptr;
  int* cols = nullptr;
  rfm_status res = RFM_OK;
  if (cudaMalloc((void**)&D, (size_t)N * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&V, (size_t)N * len * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&sq, (size_t)N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&cols, (size_t)N * sizeof(int)) != cudaSuccess) {
    rfm_set_error("rfm_function_basis: allocation failed");
    res = RFM_ENOMEM;
  }
  std::vector<int> rest(N);
  std::vector<double> sqh(N);
  for (int j = 0; j < N; ++j) rest[j] = j;
  const double scale = 1.0 / sqrt((double)npts);
  int rank = 0;
  if (res == RFM_OK) {
    k_centre<<<blocks_for(n), kThreads, 0, st>>>(C_dev, N, n, mean_dev, D);
    if (cudaGetLastError() != cudaSuccess) res = RFM_ECUDA;
    if (cudaMemsetAsync(Z_dev, 0, (size_t)N * N * sizeof(double), st) != cudaSuccess) res = RFM_ECUDA;
    // V_j = values of u(D_j) at the points, scaled so that sum_q V^2 is the mean square
    for (int j = 0; j < N && res == RFM_OK; ++j) res = rfm_launch_eval(p, D + (size_t)j * n, pts_dev, npts,
                                                                       V + (size_t)j * len);
  }
  for (int j = 0; j < N && res == RFM_OK; ++j) {  // V_j *= 1/sqrt(npts) (k_normalise with rkk = sqrt(npts))
    k_normalise<<<blocks_for(len), kThreads, 0, st>>>(V, len, D, 0, j, 1.0 / scale, nullptr);
    if (cudaGetLastError() != cudaSuccess) res = RFM_ECUDA;
  }
  double norm0 = 0.0;
  for (int k = 0; k < N && res == RFM_OK; ++k) {
    const int m = N - k;
    if (cudaMemcpyAsync(cols, rest.data() + k, m * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      res = RFM_ECUDA;
      break;
    }
    k_colsq<<<m, kThreads, 0, st>>>(V, len, cols, sq);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(sqh.data(), sq, N * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      res = RFM_ECUDA;
      break;
    }
    int best = k;
    for (int t = k + 1; t < N; ++t)
      if (sqh[rest[t]] > sqh[rest[best]]) best = t;
    const double rkk = sqrt(sqh[rest[best]]);
    if (k == 0) norm0 = rkk;
    if (!(rkk > tol * norm0) || rkk == 0.0) break;
    std::swap(rest[k], rest[best]);
    const int piv = rest[k];
    k_normalise<<<blocks_for(len > n ? len : n), kThreads, 0, st>>>(V, len, D, n, piv, rkk, U_dev + (size_t)k * n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(Z_dev + (size_t)piv * N + k, &rkk, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      res = RFM_ECUDA;
      break;
    }
    rank = k + 1;
    if (m > 1) {
      if (cudaMemcpyAsync(cols, rest.data() + k + 1, (m - 1) * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        res = RFM_ECUDA;
        break;
      }
      k_project<<<m - 1, kThreads, 0, st>>>(V, len, D, n, piv, cols, Z_dev, N, k);
      if (cudaGetLastError() != cudaSuccess) {
        res = RFM_ECUDA;
        break;
      }
    }
    // the host copies above read pageable memory; keep them ordered with the kernels
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      res = RFM_ECUDA;
      break;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && res == RFM_OK) res = RFM_ECUDA;
  if (D) cudaFree(D);
  if (V) cudaFree(V);
  if (sq) cudaFree(sq);
  if (cols) cudaFree(cols);
  if (res == RFM_ECUDA) rfm_set_error("rfm_function_basis: CUDA error");
  *rank_host = rank;
  return res;
}

rfm_status rfm_basis_combine(const double* mean_dev, const double* U_dev, int64_t n, int rank, const float* y_dev,
                             int batch, double scale, double* c_dev, void* cuda_stream) {
  if (!mean_dev || (rank > 0 && (!U_dev || !y_dev)) || n <= 0 || rank < 0 || batch <= 0 || !c_dev) {
    rfm_set_error("rfm_basis_combine: bad argument");
    return RFM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_combine<<<blocks_for((long long)batch * n), kThreads, 0, st>>>(mean_dev, U_dev, n, rank, y_dev, batch, scale, c_dev);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    rfm_set_error("rfm_basis_combine: CUDA error");
    return RFM_ECUDA;
  }
  return RFM_OK;
}

}  // extern "C"
