// C ABI of librfm: problem set-up, the individual hot-path steps and the IPN /
// AMIPN drivers (Alg. 1, Alg. 2 of arXiv 2510.04170).  All numerical work runs
// in kernels (here and in assemble.cu, sketch.cu, qr.cu, oz.cu, krylov.cu);
// LSQR's scalar recurrences run on the device too.  The host code sequences
// launches and evaluates the golden-section bracket and the Newton stopping
// tests.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rfm_internal.cuh"

rfm_status rfm_launch_jmv_axpby(rfm_problem* p, const double* x, double s1, double s2, double* y,
                                const double* s2dev = nullptr);

namespace {

thread_local std::string g_err;

// ---------------------------------------------------------------- vector kernels
__global__ void k_scale_by(double* __restrict__ x, long long n, const double* __restrict__ s, int inv,
                           const int* __restrict__ skip = nullptr) {
  if (skip && *skip) return;
  const double sv = s[0];
  if (sv == 0.0) return;
  const double f = inv ? 1.0 / sv : sv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = inv ? x[i] / sv : x[i] * f;
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, long long n, double a, double b) {
  // y = a x + b y
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : a * x[i] + b * y[i];
}

__global__ void k_neg_copy(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = -x[i];
}

__global__ void k_sub(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                      long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a[i] - b[i];
}

// ---------------------------------------------------------------- LSQR scalars
// Paige-Saunders LSQR (Alg. 1 step 4 solves J R^{-1} y = -F with it) keeps
// its scalar recurrences on the device: the norms land in sc[0] (beta, ||u||)
// and sc[1] (alpha, ||v||); the state below carries the rest between
// iterations, and the convergence flag *done makes the iteration's kernels
// return at once, so a fixed chunk of iterations can be replayed as one graph.
enum LsqrSlot {
  LS_ALPHA, LS_RHOBAR, LS_PHIBAR, LS_SUMSQ, LS_DD, LS_NORMB, LS_ETA, LS_CONLIM, LS_LIMIT, LS_ITN, LS_ISTOP, LS_SLOTS
};

struct Rot {
  double rho, c, s, theta, rhobar, phi, phibar;
};

// One plane rotation of the bidiagonal (beta, alpha the new norms).
__device__ __forceinline__ Rot lsqr_rot(const double* st, const double* sc) {
  Rot r;
  const double beta = sc[0], alpha = sc[1];
  r.rho = hypot(st[LS_RHOBAR], beta);
  r.c = st[LS_RHOBAR] / r.rho;
  r.s = beta / r.rho;
  r.theta = r.s * alpha;
  r.rhobar = -r.c * alpha;
  r.phi = r.c * st[LS_PHIBAR];
  r.phibar = r.s * st[LS_PHIBAR];
  return r;
}

// After u_1 = b / beta_1 and v_1 = R^-T J^T u_1 / alpha_1: initial state; a
// zero right-hand side or a zero first alpha ends LSQR with x = 0.
__global__ void k_lsqr_init(double* __restrict__ st, const double* __restrict__ sc, double eta, double conlim,
                            double limit, int* __restrict__ done) {
  const double beta = sc[0], alpha = sc[1];
  st[LS_ALPHA] = alpha;
  st[LS_RHOBAR] = alpha;
  st[LS_PHIBAR] = beta;
  st[LS_SUMSQ] = 0.0;
  st[LS_DD] = 0.0;
  st[LS_NORMB] = beta;
  st[LS_ETA] = eta;
  st[LS_CONLIM] = conlim;
  st[LS_LIMIT] = limit;
  st[LS_ITN] = 0.0;
  st[LS_ISTOP] = 7.0;
  *done = (beta > 0.0 && alpha > 0.0 && limit > 0.0) ? 0 : 1;
  if (!(beta > 0.0 && alpha > 0.0)) st[LS_ISTOP] = 0.0;
}

// y = a x + b y with b = bscale * bdev[0]
__global__ void k_axpby_dev(double* __restrict__ y, const double* __restrict__ x, long long n, double a,
                            const double* __restrict__ bdev, double bscale, const int* __restrict__ skip) {
  if (*skip) return;
  const double b = bscale * bdev[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// LSQR update with the old w: dk = w / rho; x += phi dk; w = v - (theta/rho) w;
// partial sums of ||dk||^2 and ||x||^2 per block.  Every block derives the
// rotation from the same device scalars.
__global__ void k_lsqr_update(double* __restrict__ x, double* __restrict__ w, const double* __restrict__ v, long long n,
                              const double* __restrict__ lst, const double* __restrict__ sc,
                              double* __restrict__ partial, const int* __restrict__ skip) {
  if (*skip) return;
  const Rot r = lsqr_rot(lst, sc);
  const double rho = r.rho, phi = r.phi, theta = r.theta;
  double sd = 0.0, sx = 0.0;
  const double tr = theta / rho;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double dk = w[i] / rho;
    const double xi = x[i] + phi * dk;
    x[i] = xi;
    w[i] = v[i] - tr * w[i];
    sd += dk * dk;
    sx += xi * xi;
  }
  __shared__ double sh[2][32];
  sd = warp_sum(sd);
  sx = warp_sum(sx);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = sd;
    sh[1][threadIdx.x >> 5] = sx;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < (blockDim.x >> 5) ? sh[0][threadIdx.x] : 0.0;
    double b = threadIdx.x < (blockDim.x >> 5) ? sh[1][threadIdx.x] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
      partial[2 * blockIdx.x] = a;
      partial[2 * blockIdx.x + 1] = b;
    }
  }
}

// End of an LSQR iteration (one warp): reduces ||dk||^2 and ||x||^2, advances
// the state and applies the stopping tests (istop 1: ||r|| small, 2: ||A^T r||
// small, 3: cond(A) above conlim, 7: iteration limit).
__global__ void k_lsqr_finish(const double* __restrict__ partial, int np, double* __restrict__ st,
                              const double* __restrict__ sc, int* __restrict__ done) {
  if (*done) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (threadIdx.x != 0) return;
  const Rot r = lsqr_rot(st, sc);
  const double beta = sc[0], alpha = sc[1];
  st[LS_SUMSQ] += st[LS_ALPHA] * st[LS_ALPHA] + beta * beta;  // ||B_k||_F^2: alpha_i with beta_{i+1}
  st[LS_ALPHA] = alpha;
  st[LS_RHOBAR] = r.rhobar;
  st[LS_PHIBAR] = r.phibar;
  st[LS_DD] += a;
  st[LS_ITN] += 1.0;
  const double eta = st[LS_ETA];
  const double normx = sqrt(b);
  const double normA = sqrt(st[LS_SUMSQ]);
  const double condA = normA * sqrt(st[LS_DD]);
  const double normr = r.phibar;
  const double normar = r.phibar * alpha * fabs(r.c);
  int istop = 7;
  if (normr <= eta * st[LS_NORMB] + eta * normA * normx) istop = 1;
  else if (normar <= eta * normA * normr) istop = 2;
  else if (condA >= st[LS_CONLIM]) istop = 3;
  st[LS_ISTOP] = (double)istop;
  if (istop != 7 || st[LS_ITN] >= st[LS_LIMIT]) *done = 1;
}

__global__ void k_copy_r(const double* __restrict__ A, long long lda, long long n, double* __restrict__ R) {
  const long long col = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    R[(size_t)col * n + i] = i <= col ? A[(size_t)col * lda + i] : 0.0;
}

constexpr int kVecBlocks = 304;

int vgrid(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, kVecBlocks));
}

// ---------------------------------------------------------------- helpers
template <class T>
rfm_status dalloc(T** ptr, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    g_err = std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes: " + cudaGetErrorString(e);
    return RFM_ENOMEM;
  }
  return RFM_OK;
}

void dfree(void* ptr) {
  if (ptr) cudaFree(ptr);
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  double* acc;
  Timer(cudaStream_t s, double* acc_) : st(s), acc(acc_) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  ~Timer() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (acc) *acc += ms;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// work-vector slots inside p->work
enum { WV_U, WV_V, WV_W, WV_X, WV_TN, WV_TN2, WV_TM, WV_D, WV_Z, WV_FPREV, WV_FNEW, WV_P0, WV_P1, WV_UU, WV_VV, WV_B,
       WV_COUNT };

// Doubles per work-vector slot: an m-vector of per-row quantities (the
// line-search split stores `fields` values per row, or the 10-entry 2-jet of
// u for PDE kinds 4-6) or an n-vector.
long long vec_stride(const rfm_problem* p) {
  const long long per_row = p->desc.pde_kind >= 4 ? 10 : std::max(1, p->fields);
  return std::max(p->m * per_row, p->n) + 64;
}

double* wv(rfm_problem* p, int slot) { return p->work + (size_t)slot * vec_stride(p); }

rfm_status read_scalars(rfm_problem* p, const double* dev, int count, double* host) {
  RFM_CUDA(cudaMemcpyAsync(p->hostbuf, dev, count * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  memcpy(host, p->hostbuf, count * sizeof(double));
  return RFM_OK;
}

// Clears the device error word at the start of a public call, so a wait that
// gave up in an earlier call is not reported again.
rfm_status clear_err(rfm_problem* p) {
  RFM_CUDA(cudaMemsetAsync(p->sync + SYNC_ERR, 0, sizeof(unsigned int), p->stream));
  return RFM_OK;
}

rfm_status check_timeout(rfm_problem* p) {
  unsigned int e = 0;
  RFM_CUDA(cudaMemcpyAsync(&e, p->sync + SYNC_ERR, sizeof(unsigned int), cudaMemcpyDeviceToHost, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  if (e) {
    g_err = "a bounded device wait timed out";
    return RFM_ETIMEOUT;
  }
  return RFM_OK;
}

// ---------------------------------------------------------------- problem build
rfm_status build_tables(rfm_problem* p, std::vector<RowSeg>& segs, std::vector<double>& Xh,
                        std::vector<double>& muh, std::vector<double>& sgh) {
  const rfm_problem_desc& d = p->desc;
  const int D = p->d;
  p->nmaxbp = 1;
  for (int b = 0; b < D; ++b) p->nmaxbp = std::max(p->nmaxbp, p->N[b] + 1);
  Xh.assign(3 * p->nmaxbp + 6, 0.0);
  for (int b = 0; b < D; ++b) {
    for (int j = 0; j <= p->N[b]; ++j) {
      double x = d.lo[b] + ((d.hi[b] - d.lo[b]) * (double)j) / (double)p->N[b];
      if (j == 0) x = d.lo[b];
      if (j == p->N[b]) x = d.hi[b];
      Xh[b * p->nmaxbp + j] = x;
    }
    Xh[3 * p->nmaxbp + b] = d.lo[b];
    Xh[3 * p->nmaxbp + 3 + b] = d.hi[b];
  }
  auto sub_index = [&](int e, int* idx) {
    for (int b = D - 1; b >= 0; --b) {
      idx[b] = e % p->N[b];
      e /= p->N[b];
    }
  };
  auto sub_id = [&](const int* idx) {
    int e = 0;
    for (int b = 0; b < D; ++b) e = e * p->N[b] + idx[b];
    return e;
  };
  muh.assign(4 * p->G, 0.0);
  sgh.assign(4 * p->G, 1.0);
  for (int e = 0; e < p->G; ++e) {
    int idx[3];
    sub_index(e, idx);
    for (int b = 0; b < D; ++b) {
      const double a = Xh[b * p->nmaxbp + idx[b]], c = Xh[b * p->nmaxbp + idx[b] + 1];
      muh[4 * e + b] = 0.5 * (a + c);
      sgh[4 * e + b] = 0.5 * (c - a);
    }
  }
  long long row = 0;
  auto add = [&](int kind, int e0, int e1, int axis, int sord, int field, int side, const int* q) {
    RowSeg s;
    memset(&s, 0, sizeof(s));
    s.kind = kind; s.e0 = e0; s.e1 = e1; s.axis = axis; s.sord = sord; s.field = field; s.side = side;
    long long cnt = 1;
    for (int b = 0; b < 3; ++b) {
      s.q[b] = (b < D && !(kind != 0 && b == axis)) ? q[b] : 1;
      cnt *= s.q[b];
    }
    s.row0 = row;
    s.count = cnt;
    row += cnt;
    segs.push_back(s);
  };
  for (int e = 0; e < p->G; ++e)
    for (int f = 0; f < p->fields; ++f) add(0, e, -1, -1, 0, f, 0, d.q_int);
  p->m_int = row;
  for (int a = 0; a < D; ++a)
    for (int e = 0; e < p->G; ++e) {
      int idx[3];
      sub_index(e, idx);
      if (idx[a] >= p->N[a] - 1) continue;
      int nb[3] = {idx[0], idx[1], idx[2]};
      nb[a] += 1;
      const int e2 = sub_id(nb);
      for (int f = 0; f < p->fields; ++f)
        for (int s = 0; s < d.cont_order; ++s) add(1, e, e2, a, s, f, 0, d.q_iface);
    }
  p->m_iface = row - p->m_int;
  for (int a = 0; a < D; ++a)
    for (int side = 0; side < 2; ++side)
      for (int e = 0; e < p->G; ++e) {
        int idx[3];
        sub_index(e, idx);
        if (idx[a] != (side == 0 ? 0 : p->N[a] - 1)) continue;
        for (int f = 0; f < p->fields; ++f) add(2, e, -1, a, 0, f, side, d.q_bdy);
      }
  p->m = row;
  p->m_bdy = p->m - p->m_int - p->m_iface;
  return RFM_OK;
}

// Row tables of the unit-ball geometry (Sec. 6.2, diffusion-reaction on the
// unit ball): the interior grid of every subdomain and the face grids of every
// interface, in the order of the box layout, keeping the points with
// x^2 + y^2 + z^2 < 1; then Dirichlet rows at the Fibonacci points of the unit
// sphere, z_i = 1 - (2i + 1)/N, radius sqrt(1 - z_i^2), azimuth
// i pi (3 - sqrt 5), grouped by the subdomain that contains them (floor of
// the scaled coordinate, clamped).  pts [m][4], meta as in k_points.
void build_ball_rows(rfm_problem* p, const std::vector<double>& Xh, std::vector<double>& pts,
                     std::vector<int4>& meta) {
  const rfm_problem_desc& d = p->desc;
  const int nbp = p->nmaxbp;
  auto grid_pt = [&](int b, int j, int pp, int q) {
    const double a = Xh[b * nbp + j], c = Xh[b * nbp + j + 1];
    if (pp == 0) return a;
    if (pp == q - 1) return c;
    return a + ((c - a) * (double)pp) / (double)(q - 1);
  };
  auto inside = [](const double* x) { return (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2] < 1.0; };
  auto idx_of = [&](int e, int* idx) {
    for (int b = 2; b >= 0; --b) {
      idx[b] = e % p->N[b];
      e /= p->N[b];
    }
  };
  auto push = [&](const double* x, int kind, int field, int axis, int sord, int e0, int e1) {
    pts.insert(pts.end(), {x[0], x[1], x[2], 0.0});
    const int code = kind | (field << 4) | ((axis & 0xF) << 8) | (sord << 12);
    meta.push_back(make_int4(code, e0, e1, 0));
  };
  for (int e = 0; e < p->G; ++e) {
    int idx[3];
    idx_of(e, idx);
    for (int f = 0; f < p->fields; ++f)
      for (int i0 = 0; i0 < d.q_int[0]; ++i0)
        for (int i1 = 0; i1 < d.q_int[1]; ++i1)
          for (int i2 = 0; i2 < d.q_int[2]; ++i2) {
            const double x[3] = {grid_pt(0, idx[0], i0, d.q_int[0]), grid_pt(1, idx[1], i1, d.q_int[1]),
                                 grid_pt(2, idx[2], i2, d.q_int[2])};
            if (inside(x)) push(x, 0, f, -1, 0, e, -1);
          }
  }
  p->m_int = (long long)meta.size();
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < p->G; ++e) {
      int idx[3];
      idx_of(e, idx);
      if (idx[a] >= p->N[a] - 1) continue;
      int nb[3] = {idx[0], idx[1], idx[2]};
      nb[a] += 1;
      const int e2 = (nb[0] * p->N[1] + nb[1]) * p->N[2] + nb[2];
      const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;  // the two axes along the face, in order
      for (int f = 0; f < p->fields; ++f)
        for (int so = 0; so < d.cont_order; ++so)
          for (int i0 = 0; i0 < d.q_iface[b0]; ++i0)
            for (int i1 = 0; i1 < d.q_iface[b1]; ++i1) {
              double x[3];
              x[a] = Xh[a * nbp + idx[a] + 1];
              x[b0] = grid_pt(b0, idx[b0], i0, d.q_iface[b0]);
              x[b1] = grid_pt(b1, idx[b1], i1, d.q_iface[b1]);
              if (inside(x)) push(x, 1, f, a, so, e, e2);
            }
    }
  p->m_iface = (long long)meta.size() - p->m_int;
  const long long N = d.n_sphere;
  const double ga = 3.141592653589793 * (3.0 - sqrt(5.0));
  std::vector<std::vector<long long>> by_owner(p->G);
  std::vector<double> F(3 * N);
  for (long long i = 0; i < N; ++i) {
    const double z = 1.0 - (2.0 * (double)i + 1.0) / (double)N;
    const double r = sqrt(1.0 - z * z);
    const double th = (double)i * ga;
    F[3 * i] = r * cos(th);
    F[3 * i + 1] = r * sin(th);
    F[3 * i + 2] = z;
    int e = 0;
    for (int b = 0; b < 3; ++b) {
      long long t = (long long)floor((F[3 * i + b] - d.lo[b]) / (d.hi[b] - d.lo[b]) * (double)p->N[b]);
      t = std::min<long long>(std::max<long long>(t, 0), p->N[b] - 1);
      e = e * p->N[b] + (int)t;
    }
    by_owner[e].push_back(i);
  }
  for (int e = 0; e < p->G; ++e)
    for (int f = 0; f < p->fields; ++f)
      for (long long i : by_owner[e]) push(&F[3 * i], 2, f, -1, 0, e, -1);
  p->m = (long long)meta.size();
  p->m_bdy = p->m - p->m_int - p->m_iface;
}

rfm_status ensure_sketch(rfm_problem* p, long long s, int kind) {
  if (s < p->n) {
    g_err = "sketch rows must be >= n";
    return RFM_EINVAL;
  }
  if (kind == RFM_SKETCH_GAUSS && (s % 2)) {
    g_err = "Gaussian sketch needs an even row count";
    return RFM_EINVAL;
  }
  if (s > p->s_cap) {
    dfree(p->B);
    p->B = nullptr;
    p->s_cap = 0;
    RFM_TRY(dalloc(&p->B, (size_t)s * p->n));
    p->s_cap = s;
  }
  if (kind == RFM_SKETCH_COUNT && s + 1 > p->bptr_cap) {
    dfree(p->bptr);
    dfree(p->brows);
    p->bptr = nullptr;
    p->brows = nullptr;
    p->bptr_cap = 0;
    RFM_TRY(dalloc(&p->bptr, (size_t)s + 1));
    RFM_TRY(dalloc(&p->brows, (size_t)p->m + 2 * s + 2));
    p->bptr_cap = s + 1;
  }
  if (kind == RFM_SKETCH_GAUSS && p->precision == 0 && s > p->sg_cap) {
    dfree(p->Sg);
    p->Sg = nullptr;
    p->sg_cap = 0;
    RFM_TRY(dalloc(&p->Sg, (size_t)s * p->m));
    p->sg_cap = s;
  }
  return RFM_OK;
}

// FP64 panel scratch of the Householder QR, owned by the problem (problems on
// different streams or host threads never share it).
rfm_status ensure_qr_scratch(rfm_problem* p, long long s, long long n) {
  const long long need = rfm_householder_scratch(s, n);
  if (need > p->qr_scratch_len) {
    dfree(p->qr_scratch);
    p->qr_scratch = nullptr;
    p->qr_scratch_len = 0;
    RFM_TRY(dalloc(&p->qr_scratch, (size_t)need));
    p->qr_scratch_len = need;
  }
  return RFM_OK;
}

rfm_status do_sketch(rfm_problem* p, int kind, long long s, int kJ) {
  if (!p->have_j) {
    g_err = "no Jacobian assembled";
    return RFM_EINVAL;
  }
  RFM_TRY(ensure_sketch(p, s, kind));
  p->s = s;
  if (kind == RFM_SKETCH_COUNT) return rfm_launch_count_sketch(p, s, kJ);
  if (kind == RFM_SKETCH_GAUSS)
    return p->precision >= 1 ? rfm_launch_gauss_sketch_tc(p, s, kJ) : rfm_launch_gauss_sketch(p, s, kJ);
  g_err = "unknown sketch kind";
  return RFM_EINVAL;
}

rfm_status do_qr(rfm_problem* p) {
  RFM_TRY(ensure_qr_scratch(p, p->s, p->n));
  int flag = 0;
  if (p->precision >= 2) {
    const long long need = rfm_householder_emulated_bytes(p->s, p->n);
    if (need > p->qr_emu_bytes) {
      dfree(p->qr_emu);
      p->qr_emu = nullptr;
      p->qr_emu_bytes = 0;
      char* buf = nullptr;
      RFM_TRY(dalloc(&buf, (size_t)need));
      p->qr_emu = buf;
      p->qr_emu_bytes = need;
    }
    RFM_TRY(rfm_householder_emulated(p->B, p->s, p->n, p->s, p->stream, p->qr_scratch, p->qr_scratch_len, p->sync,
                                     p->qr_emu, p->qr_emu_bytes, &flag, p->qr_panel_cap));
  } else {
    RFM_TRY(
        rfm_householder_inplace(p->B, p->s, p->n, p->s, p->stream, p->qr_scratch, p->qr_scratch_len, p->sync, &flag,
                                p->qr_panel_cap));
  }
  p->R = p->B;
  p->ldr = p->s;
  p->have_r = true;
  p->rank_flag = flag;
  return rfm_trsv_prepare(p);
}

// ---------------------------------------------------------------- LSQR
struct LsqrOut {
  int itn, istop;
};

constexpr int kLsqrChunk = 16;  // iterations per replayed graph

// One chunk of kLsqrChunk iterations, every kernel guarded by the done flag.
rfm_status lsqr_chunk(rfm_problem* p, double* lst, int* done) {
  const long long m = p->m, n = p->n;
  cudaStream_t st = p->stream;
  double* u = wv(p, WV_U);
  double* v = wv(p, WV_V);
  double* w = wv(p, WV_W);
  double* x = wv(p, WV_X);
  double* tn = wv(p, WV_TN);
  double* tn2 = wv(p, WV_TN2);
  double* sc = p->red + 1024;
  for (int it = 0; it < kLsqrChunk; ++it) {
    // beta u = J R^{-1} v - alpha u
    RFM_TRY(rfm_launch_trsv(p, 0, v, tn));
    RFM_TRY(rfm_launch_jmv_axpby(p, tn, 1.0, -1.0, u, lst + LS_ALPHA));
    RFM_TRY(rfm_norm2(st, u, m, p->red, sc));
    k_scale_by<<<vgrid(m), 256, 0, st>>>(u, m, sc, 1, done);
    RFM_CHECK_LAUNCH();
    // alpha v = R^{-T} J^T u - beta v
    RFM_TRY(rfm_launch_jtmv(p, u, tn));
    RFM_TRY(rfm_launch_trsv(p, 1, tn, tn2));
    k_axpby_dev<<<vgrid(n), 256, 0, st>>>(v, tn2, n, 1.0, sc, -1.0, done);
    RFM_CHECK_LAUNCH();
    RFM_TRY(rfm_norm2(st, v, n, p->red, sc + 1));
    k_scale_by<<<vgrid(n), 256, 0, st>>>(v, n, sc + 1, 1, done);
    RFM_CHECK_LAUNCH();
    k_lsqr_update<<<kVecBlocks, 256, 0, st>>>(x, w, v, n, lst, sc, p->red, done);
    RFM_CHECK_LAUNCH();
    k_lsqr_finish<<<1, 32, 0, st>>>(p->red, kVecBlocks, lst, sc, done);
    RFM_CHECK_LAUNCH();
  }
  return RFM_OK;
}

void drop_lsqr_graph(rfm_problem* p) {
  if (p->lsqr_graph) cudaGraphExecDestroy((cudaGraphExec_t)p->lsqr_graph);
  p->lsqr_graph = nullptr;
  p->lsqr_graph_key = 0;
}

// Captures one chunk into a graph (once per problem and preconditioner
// storage), or rebuilds it when R moved.
rfm_status lsqr_graph(rfm_problem* p, double* lst, int* done) {
  // everything the captured launches bake in: R and the vector workspace
  unsigned long long key = 1469598103934665603ull;
  for (unsigned long long v : {(unsigned long long)(uintptr_t)p->R, (unsigned long long)p->ldr,
                               (unsigned long long)(uintptr_t)p->work, (unsigned long long)p->work_cap,
                               (unsigned long long)(uintptr_t)p->Jp, (unsigned long long)(uintptr_t)p->Js})
    key = (key ^ v) * 1099511628211ull;
  if (p->lsqr_graph && p->lsqr_graph_key == key) return RFM_OK;
  drop_lsqr_graph(p);
  // capture on a private stream (the problem's may be the legacy default
  // stream, which cannot be captured); the graph is replayed on p->stream
  if (!p->cap_stream) RFM_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaStream_t home = p->stream;
  p->stream = p->cap_stream;
  rfm_count_pause(true);  // captured launches do not run; this thread stops counting them
  cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
  rfm_status r = e == cudaSuccess ? lsqr_chunk(p, lst, done) : RFM_ECUDA;
  if (e == cudaSuccess) e = cudaStreamEndCapture(p->stream, &g);
  rfm_count_pause(false);
  p->stream = home;
  if (r != RFM_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) {
    g_err = std::string("lsqr graph capture: ") + cudaGetErrorString(e);
    return RFM_ECUDA;
  }
  // kernels per replay, counted on the captured graph itself
  size_t nodes = 0;
  long long kernels = 0;
  if (cudaGraphGetNodes(g, nullptr, &nodes) == cudaSuccess && nodes > 0) {
    std::vector<cudaGraphNode_t> list(nodes);
    if (cudaGraphGetNodes(g, list.data(), &nodes) == cudaSuccess)
      for (size_t i = 0; i < nodes; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(list[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    g_err = std::string("lsqr graph instantiate: ") + cudaGetErrorString(e);
    return RFM_ECUDA;
  }
  p->lsqr_graph = ex;
  p->lsqr_graph_key = key;
  p->lsqr_graph_launches = kernels;
  return RFM_OK;
}

rfm_status lsqr(rfm_problem* p, const double* b, double eta, double conlim, long long iter_lim, double* d_out,
                LsqrOut* out) {
  const long long m = p->m, n = p->n;
  cudaStream_t st = p->stream;
  double* u = wv(p, WV_U);
  double* v = wv(p, WV_V);
  double* w = wv(p, WV_W);
  double* x = wv(p, WV_X);
  double* tn = wv(p, WV_TN);
  double* sc = p->red + 1024;  // device scalars
  double* lst = p->red + 2048;  // LSQR state
  int* done = (int*)(p->sync + SYNC_LSQR_DONE);
  out->itn = 0;
  out->istop = 0;
  // u_1 = b / beta_1, v_1 = R^{-T} J^T u_1 / alpha_1, w_1 = v_1, x_0 = 0
  RFM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
  RFM_CUDA(cudaMemcpyAsync(u, b, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  RFM_TRY(rfm_norm2(st, u, m, p->red, sc));
  k_scale_by<<<vgrid(m), 256, 0, st>>>(u, m, sc, 1);
  RFM_CHECK_LAUNCH();
  RFM_TRY(rfm_launch_jtmv(p, u, tn));
  RFM_TRY(rfm_launch_trsv(p, 1, tn, v));
  RFM_TRY(rfm_norm2(st, v, n, p->red, sc + 1));
  k_scale_by<<<vgrid(n), 256, 0, st>>>(v, n, sc + 1, 1);
  RFM_CHECK_LAUNCH();
  RFM_CUDA(cudaMemcpyAsync(w, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  k_lsqr_init<<<1, 1, 0, st>>>(lst, sc, eta, conlim, (double)iter_lim, done);
  RFM_CHECK_LAUNCH();
  // chunks of iterations until the device sets done; replayed from a graph
  // unless LSQR's own kernels are being timed (event timing needs eager launches)
  bool graph = !p->lsqr_eager &&
               !rfm_prof_active((1u << PF_TRSV) | (1u << PF_JMV) | (1u << PF_JTMV) | (1u << PF_VECTOR));
  p->skip = done;
  rfm_status r = RFM_OK;
  if (graph) {
    r = lsqr_graph(p, lst, done);
    if (r != RFM_OK) {  // capture or instantiation refused: run the same kernels eagerly from now on
      cudaGetLastError();
      p->lsqr_eager = true;
      graph = false;
      r = RFM_OK;
    }
  }
  int* hflag = (int*)p->hostbuf;
  for (long long chunks = 0; r == RFM_OK; ++chunks) {
    if (graph) {
      if (cudaGraphLaunch((cudaGraphExec_t)p->lsqr_graph, st) != cudaSuccess) {
        g_err = "lsqr graph launch failed";
        r = RFM_ECUDA;
        break;
      }
      rfm_count_launches(p->lsqr_graph_launches);
    } else {
      r = lsqr_chunk(p, lst, done);
      if (r != RFM_OK) break;
    }
    if (cudaMemcpyAsync(hflag, done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      g_err = "lsqr: CUDA error";
      r = RFM_ECUDA;
      break;
    }
    if (*hflag) break;
    if (chunks * kLsqrChunk > iter_lim + kLsqrChunk) {  // the device stops at iter_lim; guard the host loop too
      g_err = "lsqr: iteration limit not honoured";
      r = RFM_ECUDA;
      break;
    }
  }
  p->skip = nullptr;
  RFM_TRY(r);
  double hs[2];
  RFM_TRY(read_scalars(p, lst + LS_ITN, 2, hs));
  out->itn = (int)hs[0];
  out->istop = (int)hs[1];
  RFM_TRY(rfm_launch_trsv(p, 0, x, d_out));
  return check_timeout(p);
}

// ---------------------------------------------------------------- line search
const double kGold = 0.6180339887498949;  // (sqrt(5) - 1) / 2

rfm_status linesearch(rfm_problem* p, const double* c, const double* dvec, double f0, double* alpha_out,
                      double* fbest_out) {
  double* P0 = wv(p, WV_P0);
  double* P1 = wv(p, WV_P1);
  double* U = wv(p, WV_UU);
  double* V = wv(p, WV_VV);
  RFM_TRY(rfm_launch_ls_precompute(p, c, dvec, P0, P1, U, V));
  double* sc = p->red + 1024 + 8;
  auto phi = [&](double a, double* out) -> rfm_status {
    RFM_TRY(rfm_launch_ls_eval(p, P0, P1, U, V, a, sc));
    return read_scalars(p, sc, 1, out);
  };
  double a = 0.0, b = 1.0;
  double x1 = b - kGold * (b - a), x2 = a + kGold * (b - a);
  double f1, f2;
  RFM_TRY(phi(x1, &f1));
  RFM_TRY(phi(x2, &f2));
  std::vector<std::pair<double, double>> pts = {{x1, f1}, {x2, f2}};
  while (b - a > 1e-3) {
    if (f1 < f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - kGold * (b - a);
      RFM_TRY(phi(x1, &f1));
      pts.push_back({x1, f1});
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + kGold * (b - a);
      RFM_TRY(phi(x2, &f2));
      pts.push_back({x2, f2});
    }
  }
  double fone;
  RFM_TRY(phi(1.0, &fone));
  pts.push_back({1.0, fone});
  double fmin = pts[0].second;
  for (auto& q : pts) fmin = std::min(fmin, q.second);
  double best = -1.0, fbest = 0.0;
  for (auto& q : pts)
    if (q.second <= fmin * (1.0 + 1e-12) && q.first > best) best = q.first;
  fbest = INFINITY;
  for (auto& q : pts)
    if (q.first == best) fbest = std::min(fbest, q.second);
  if (!(fbest < f0)) {
    *alpha_out = 0.0;
    *fbest_out = f0;
  } else {
    *alpha_out = best;
    *fbest_out = fbest;
  }
  return RFM_OK;
}

long long sketch_rows_for(const rfm_problem* p, const rfm_solve_opts* o) {
  long long s = o->sketch_rows > 0 ? o->sketch_rows : (long long)ceil(o->gamma * (double)p->n);
  if (o->sketch_kind == RFM_SKETCH_GAUSS && (s % 2)) s += 1;
  return s;
}

rfm_status linearise(rfm_problem* p, const rfm_solve_opts* o, const double* c, int kJ, rfm_solve_info* info) {
  {
    Timer t(p->stream, &info->t_assemble);
    RFM_TRY(rfm_launch_assemble(p, c, o->row_scale_c, true, nullptr, p->F));
    p->have_j = true;
  }
  {
    Timer t(p->stream, &info->t_sketch);
    RFM_TRY(do_sketch(p, o->sketch_kind, sketch_rows_for(p, o), kJ));
  }
  {
    Timer t(p->stream, &info->t_qr);
    RFM_TRY(do_qr(p));
  }
  info->rank_flag |= p->rank_flag;
  info->n_jac += 1;
  return RFM_OK;
}

rfm_status direction(rfm_problem* p, const rfm_solve_opts* o, const double* rhs, double* d, rfm_solve_info* info) {
  Timer t(p->stream, &info->t_lsqr);
  LsqrOut lo;
  const long long lim = o->lsqr_max_iter > 0 ? o->lsqr_max_iter : 2 * p->n;
  RFM_TRY(lsqr(p, rhs, o->eta, o->conlim, lim, d, &lo));
  info->lsqr_iters_total += lo.itn;
  info->lsqr_iters_max = std::max(info->lsqr_iters_max, lo.itn);
  return RFM_OK;
}

rfm_status scaled_residual_norm(rfm_problem* p, const double* c, double* Fout, double* norm) {
  RFM_TRY(rfm_launch_assemble(p, c, 0.0, false, p->lam, Fout));
  RFM_TRY(rfm_norm2(p->stream, Fout, p->m, p->red, p->red + 1024 + 16));
  return read_scalars(p, p->red + 1024 + 16, 1, norm);
}

// R (upper triangle of the s x n column-major A) into R_dev [n][n]
// column-major, zeros below; synchronises the stream.  Errors are returned,
// never thrown past the caller's frees.
rfm_status copy_r_out(const double* A, long long lda, long long n, double* R_dev, cudaStream_t st) {
  dim3 grid((unsigned)std::min<long long>(64, (n + 255) / 256), (unsigned)n);
  k_copy_r<<<grid, 256, 0, st>>>(A, lda, n, R_dev);
  rfm_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    g_err = std::string("householder: ") + cudaGetErrorString(e);
    return RFM_ECUDA;
  }
  return RFM_OK;
}

bool validate_opts(const rfm_solve_opts* o) {
  return o && (o->sketch_kind == RFM_SKETCH_COUNT || o->sketch_kind == RFM_SKETCH_GAUSS) && o->eta > 0 &&
         o->precision >= 0 && o->precision <= 2 &&
         o->max_outer > 0 && o->m_max > 0 && o->row_scale_c > 0 && (o->sketch_rows > 0 || o->gamma >= 1.0);
}

}  // namespace

void rfm_set_error(const std::string& msg) { g_err = msg; }

extern "C" {

const char* rfm_last_error(void) { return g_err.c_str(); }

void rfm_default_opts(rfm_solve_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->sketch_kind = RFM_SKETCH_COUNT;
  o->gamma = 3.0;
  o->sketch_rows = 0;
  o->eta = 1e-6;
  o->eps = 1e-10;
  o->max_outer = 50;
  o->m_max = 3;
  o->tau_rel = 1e-3;
  o->row_scale_c = 100.0;
  o->precision = 0;
  o->lsqr_max_iter = 0;
  o->conlim = 1e8;
}

rfm_status rfm_problem_create(const rfm_problem_desc* desc, void* cuda_stream, rfm_problem** out) {
  if (!desc || !out) {
    g_err = "null argument";
    return RFM_EINVAL;
  }
  *out = nullptr;
  const int D = desc->dim;
  if (D < 2 || D > 3 || desc->M <= 0 || desc->fields < 1 || desc->fields > RFM_MAX_FIELDS ||
      desc->cont_order < 1 || desc->cont_order > 2 || desc->fields * desc->M > RFM_MAX_WIDTH ||
      desc->pde_kind < 0 || desc->pde_kind > 7 || (desc->pde_kind == 1 && (desc->fields != 2 || D != 3)) ||
      (desc->pde_kind >= 4 && D != 3) || (desc->pde_kind != 1 && desc->fields != 1) || desc->geometry < 0 ||
      desc->geometry > 1 || (desc->geometry == 1 && (D != 3 || desc->n_sphere <= 0 || desc->n_sphere > (1 << 26)))) {
    g_err = "invalid problem description";
    return RFM_EINVAL;
  }
  for (int b = 0; b < D; ++b)
    if (desc->nsub[b] <= 0 || desc->q_int[b] < 2 || desc->q_bdy[b] < 2 || desc->q_iface[b] < 2 ||
        !(desc->hi[b] > desc->lo[b])) {
      g_err = "invalid subdomain grid, point counts or box";
      return RFM_EINVAL;
    }
  rfm_problem* p = new rfm_problem();
  p->desc = *desc;
  p->stream = (cudaStream_t)cuda_stream;
  p->d = D;
  p->M = desc->M;
  p->fields = desc->fields;
  p->W = desc->fields * desc->M;
  p->G = 1;
  for (int b = 0; b < 3; ++b) p->N[b] = b < D ? desc->nsub[b] : 1;
  for (int b = 0; b < D; ++b) p->G *= p->N[b];
  p->n = (long long)p->G * p->W;
  std::vector<RowSeg> segs;
  std::vector<double> Xh, muh, sgh;
  build_tables(p, segs, Xh, muh, sgh);
  p->nseg = (int)segs.size();
  std::vector<double> ball_pts;
  std::vector<int4> ball_meta;
  if (desc->geometry == 1) {
    build_ball_rows(p, Xh, ball_pts, ball_meta);
    p->explicit_rows = true;
  }
  // transposed block structure for J^T and the Gaussian sketch
  std::vector<int> colptr(p->G + 1, 0), colrows;
  {
    std::vector<std::vector<int>> lists(p->G);
    if (p->explicit_rows) {
      for (long long r = 0; r < p->m; ++r) {
        const int4 mt = ball_meta[r];
        lists[mt.y].push_back((int)r);
        if ((mt.x & 0xF) == 1) lists[mt.z].push_back((int)(r | 0x80000000u));
      }
    } else {
      for (const RowSeg& s : segs)
        for (long long r = s.row0; r < s.row0 + s.count; ++r) {
          lists[s.e0].push_back((int)r);
          if (s.kind == 1) lists[s.e1].push_back((int)(r | 0x80000000u));
        }
    }
    for (int b = 0; b < p->G; ++b) {
      std::sort(lists[b].begin(), lists[b].end(),
                [](int x, int y) { return (unsigned)(x & 0x7fffffff) < (unsigned)(y & 0x7fffffff); });
      colptr[b + 1] = colptr[b] + (int)lists[b].size();
      colrows.insert(colrows.end(), lists[b].begin(), lists[b].end());
    }
  }
  p->colptr_h = colptr;
  rfm_status st = RFM_OK;
#define TRYA(x)                       \
  do {                                \
    st = (x);                         \
    if (st != RFM_OK) goto fail;      \
  } while (0)
  {
    const long long nfeat = (long long)p->G * p->fields * p->M;
    TRYA(dalloc(&p->X, Xh.size()));
    TRYA(dalloc(&p->mu, muh.size()));
    TRYA(dalloc(&p->sig, sgh.size()));
    TRYA(dalloc(&p->feat, 4 * nfeat));
    TRYA(dalloc(&p->segs, segs.size()));
    TRYA(dalloc(&p->pts, 4 * p->m));
    TRYA(dalloc(&p->rmeta, p->m));
    TRYA(dalloc(&p->rhs, p->m));
    TRYA(dalloc(&p->Jp, (size_t)p->m * p->W));
    TRYA(dalloc(&p->Js, (size_t)std::max(1LL, p->m_iface) * p->W));
    TRYA(dalloc(&p->lam, p->m));
    TRYA(dalloc(&p->F, p->m));
    TRYA(dalloc(&p->colptr, colptr.size()));
    TRYA(dalloc(&p->colrows, colrows.size()));
    TRYA(dalloc(&p->hbuck, p->m));
    TRYA(dalloc(&p->hsign, p->m));
    TRYA(dalloc(&p->red, 4096));
    TRYA(dalloc(&p->trsv_acc, (size_t)((p->n + 63) / 64) * 64));
    TRYA(dalloc(&p->dinv, (size_t)((p->n + 63) / 64) * 64 * 64));
    TRYA(dalloc(&p->sync, RFM_SYNC_WORDS));
    p->work_cap = vec_stride(p) * WV_COUNT;
    TRYA(dalloc(&p->work, p->work_cap));
    if (cudaMallocHost((void**)&p->hostbuf, 64 * sizeof(double)) != cudaSuccess) {
      g_err = "cudaMallocHost failed";
      st = RFM_ENOMEM;
      goto fail;
    }
    cudaStream_t s0 = p->stream;
#define CPY(dst, src, cnt)                                                                          \
  if (cudaMemcpyAsync(dst, src, (cnt) * sizeof(*(src)), cudaMemcpyHostToDevice, s0) != cudaSuccess) { \
    g_err = "upload failed";                                                                        \
    st = RFM_ECUDA;                                                                                 \
    goto fail;                                                                                      \
  }
    CPY(p->X, Xh.data(), Xh.size());
    CPY(p->mu, muh.data(), muh.size());
    CPY(p->sig, sgh.data(), sgh.size());
    CPY(p->segs, segs.data(), segs.size());
    CPY(p->colptr, colptr.data(), colptr.size());
    CPY(p->colrows, colrows.data(), colrows.size());
    if (p->explicit_rows) {
      CPY(p->pts, ball_pts.data(), ball_pts.size());
      CPY(p->rmeta, ball_meta.data(), ball_meta.size());
    }
#undef CPY
    if (cudaMemsetAsync(p->sync, 0, RFM_SYNC_WORDS * sizeof(unsigned int), s0) != cudaSuccess) {
      st = RFM_ECUDA;
      goto fail;
    }
    TRYA(rfm_launch_setup(p));
    if (cudaStreamSynchronize(s0) != cudaSuccess) {
      g_err = std::string("problem setup: ") + cudaGetErrorString(cudaGetLastError());
      st = RFM_ECUDA;
      goto fail;
    }
  }
  *out = p;
  return RFM_OK;
fail:
  rfm_problem_destroy(p);
  return st;
#undef TRYA
}

rfm_status rfm_problem_destroy(rfm_problem* p) {
  if (!p) return RFM_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  void* bufs[] = {p->X, p->mu, p->sig, p->feat, p->segs, p->pts, p->rmeta, p->rhs, p->Jp, p->Js, p->lam, p->F,
                  p->colptr, p->colrows, p->B, p->Sg, p->hbuck, p->hsign, p->bptr, p->brows, p->Rown, p->work,
                  p->red, p->sync, p->sdig, p->jdig, p->oz_e, p->oz_toff, p->qr_emu, p->qr_scratch,
                  p->trsv_acc, p->dinv};
  drop_lsqr_graph(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (void* b : bufs) dfree(b);
  if (p->hostbuf) cudaFreeHost(p->hostbuf);
  delete p;
  return RFM_OK;
}

rfm_status rfm_problem_sizes(const rfm_problem* p, int64_t* m, int64_t* n, int64_t* W, int64_t* G, int64_t* m_int,
                             int64_t* m_iface, int64_t* nnz) {
  if (!p) return RFM_EINVAL;
  if (nnz) *nnz = (p->m + p->m_iface) * (int64_t)p->W;
  if (m) *m = p->m;
  if (n) *n = p->n;
  if (W) *W = p->W;
  if (G) *G = p->G;
  if (m_int) *m_int = p->m_int;
  if (m_iface) *m_iface = p->m_iface;
  return RFM_OK;
}

rfm_status rfm_get_features(const rfm_problem* p, double* feat_dev) {
  if (!p || !feat_dev) return RFM_EINVAL;
  RFM_CUDA(cudaMemcpyAsync(feat_dev, p->feat, 4 * (size_t)p->G * p->fields * p->M * sizeof(double),
                           cudaMemcpyDeviceToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_get_points(const rfm_problem* p, double* pts_dev) {
  if (!p || !pts_dev) return RFM_EINVAL;
  RFM_CUDA(cudaMemcpyAsync(pts_dev, p->pts, 4 * (size_t)p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_assemble(rfm_problem* p, const double* c_dev, double c_scale, double* F_dev, double* lam_dev) {
  if (!p || !c_dev || !(c_scale > 0)) {
    g_err = "rfm_assemble: bad argument";
    return RFM_EINVAL;
  }
  RFM_TRY(rfm_launch_assemble(p, c_dev, c_scale, true, nullptr, p->F));
  p->have_j = true;
  p->have_r = false;
  p->dinv_of = nullptr;
  if (F_dev) RFM_CUDA(cudaMemcpyAsync(F_dev, p->F, p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  if (lam_dev) RFM_CUDA(cudaMemcpyAsync(lam_dev, p->lam, p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_get_jacobian(const rfm_problem* p, double* Jp_dev, double* Js_dev, int32_t* blk_dev) {
  if (!p || !p->have_j) {
    g_err = "no Jacobian assembled";
    return RFM_EINVAL;
  }
  if (Jp_dev)
    RFM_CUDA(cudaMemcpyAsync(Jp_dev, p->Jp, (size_t)p->m * p->W * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  if (Js_dev && p->m_iface)
    RFM_CUDA(cudaMemcpyAsync(Js_dev, p->Js, (size_t)p->m_iface * p->W * sizeof(double), cudaMemcpyDeviceToDevice,
                             p->stream));
  if (blk_dev)
    RFM_CUDA(cudaMemcpy2DAsync(blk_dev, 2 * sizeof(int32_t), reinterpret_cast<const char*>(p->rmeta) + 4,
                               sizeof(int4), 2 * sizeof(int32_t), p->m, cudaMemcpyDeviceToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_residual(rfm_problem* p, const double* c_dev, double* F_dev, double* norm_host) {
  if (!p || !c_dev || !p->have_j) {
    g_err = "rfm_residual: needs c and stored row scales";
    return RFM_EINVAL;
  }
  double* Fo = F_dev ? F_dev : wv(p, WV_TM);
  RFM_TRY(rfm_launch_assemble(p, c_dev, 0.0, false, p->lam, Fo));
  double nv = 0.0;
  RFM_TRY(rfm_norm2(p->stream, Fo, p->m, p->red, p->red + 1024 + 16));
  RFM_TRY(read_scalars(p, p->red + 1024 + 16, 1, &nv));
  if (norm_host) *norm_host = nv;
  return RFM_OK;
}

rfm_status rfm_set_rhs(rfm_problem* p, const double* rhs_dev) {
  if (!p || !rhs_dev) {
    g_err = "rfm_set_rhs: null argument";
    return RFM_EINVAL;
  }
  RFM_CUDA(cudaMemcpyAsync(p->rhs, rhs_dev, (size_t)p->m * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  if (p->m_iface)  // interface rows have no data: keep them at zero
    RFM_CUDA(cudaMemsetAsync(p->rhs + p->m_int, 0, (size_t)p->m_iface * sizeof(double), p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_set_wait_limit(rfm_problem* p, int64_t polls) {
  if (!p) {
    g_err = "rfm_set_wait_limit: null problem";
    return RFM_EINVAL;
  }
  const int v = polls < 0 ? -1 : (int)std::min<int64_t>(polls, 0x7fffffff);
  RFM_CUDA(cudaMemcpyAsync(p->sync + SYNC_WAITLIM, &v, sizeof(int), cudaMemcpyHostToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_set_precision(rfm_problem* p, int precision) {
  if (!p || precision < 0 || precision > 2) {
    g_err = "rfm_set_precision: precision must be 0, 1 or 2";
    return RFM_EINVAL;
  }
  p->precision = precision;
  return RFM_OK;
}

rfm_status rfm_sketch(rfm_problem* p, int kind, int64_t s, int kJ, double* B_dev) {
  if (!p) return RFM_EINVAL;
  RFM_TRY(clear_err(p));
  RFM_TRY(do_sketch(p, kind, s, kJ));
  p->have_r = false;
  p->dinv_of = nullptr;
  if (B_dev) RFM_CUDA(cudaMemcpyAsync(B_dev, p->B, (size_t)s * p->n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_qr(rfm_problem* p, double* R_dev) {
  if (!p || p->s <= 0) {
    g_err = "rfm_qr: no sketch";
    return RFM_EINVAL;
  }
  RFM_TRY(clear_err(p));
  RFM_TRY(do_qr(p));
  if (R_dev) {
    dim3 grid((unsigned)std::min<long long>(64, (p->n + 255) / 256), (unsigned)p->n);
    k_copy_r<<<grid, 256, 0, p->stream>>>(p->R, p->ldr, p->n, R_dev);
    RFM_CHECK_LAUNCH();
  }
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return p->rank_flag ? RFM_ERANK : RFM_OK;
}

rfm_status rfm_set_r(rfm_problem* p, const double* R_dev) {
  if (!p || !R_dev) return RFM_EINVAL;
  if (!p->Rown) RFM_TRY(dalloc(&p->Rown, (size_t)p->n * p->n));
  RFM_CUDA(cudaMemcpyAsync(p->Rown, R_dev, (size_t)p->n * p->n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  p->R = p->Rown;
  p->ldr = p->n;
  p->have_r = true;
  RFM_TRY(rfm_trsv_prepare(p));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_householder_r(double* A_dev, int64_t s, int64_t n, void* cuda_stream, double* R_dev,
                             int* rank_flag_host) {
  if (!A_dev || !R_dev || s < n || n <= 0) {
    g_err = "rfm_householder_r: bad argument";
    return RFM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long qs = rfm_householder_scratch(s, n);
  double* scratch = nullptr;
  unsigned int* sync = nullptr;
  RFM_TRY(dalloc(&scratch, (size_t)qs));
  rfm_status r = dalloc(&sync, RFM_SYNC_WORDS);
  int flag = 0;
  if (r == RFM_OK && cudaMemsetAsync(sync, 0, RFM_SYNC_WORDS * sizeof(unsigned int), st) != cudaSuccess) r = RFM_ECUDA;
  if (r == RFM_OK) r = rfm_householder_inplace(A_dev, s, n, s, st, scratch, qs, sync, &flag);
  if (r == RFM_OK) r = copy_r_out(A_dev, s, n, R_dev, st);
  cudaStreamSynchronize(st);
  dfree(sync);
  dfree(scratch);
  if (rank_flag_host) *rank_flag_host = flag;
  return r;
}

rfm_status rfm_householder_r_tc(double* A_dev, int64_t s, int64_t n, void* cuda_stream, double* R_dev,
                                int* rank_flag_host) {
  if (!A_dev || !R_dev || s < n || n <= 0) {
    g_err = "rfm_householder_r_tc: bad argument";
    return RFM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long qs = rfm_householder_scratch(s, n);
  double* scratch = nullptr;
  unsigned int* sync = nullptr;
  char* emu = nullptr;
  const long long eb = rfm_householder_emulated_bytes(s, n);
  RFM_TRY(dalloc(&scratch, (size_t)qs));
  rfm_status r = dalloc(&sync, RFM_SYNC_WORDS);
  if (r == RFM_OK) r = dalloc(&emu, (size_t)eb);
  int flag = 0;
  if (r == RFM_OK && cudaMemsetAsync(sync, 0, RFM_SYNC_WORDS * sizeof(unsigned int), st) != cudaSuccess) r = RFM_ECUDA;
  if (r == RFM_OK) r = rfm_householder_emulated(A_dev, s, n, s, st, scratch, qs, sync, emu, eb, &flag);
  if (r == RFM_OK) r = copy_r_out(A_dev, s, n, R_dev, st);
  cudaStreamSynchronize(st);
  dfree(sync);
  dfree(emu);
  dfree(scratch);
  if (rank_flag_host) *rank_flag_host = flag;
  return r;
}

rfm_status rfm_jmv(rfm_problem* p, int trans, const double* x_dev, double* y_dev) {
  if (!p || !p->have_j || !x_dev || !y_dev) return RFM_EINVAL;
  RFM_TRY(trans ? rfm_launch_jtmv(p, x_dev, y_dev) : rfm_launch_jmv(p, x_dev, y_dev));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

rfm_status rfm_trsv(rfm_problem* p, int trans, const double* b_dev, double* x_dev) {
  if (!p || !p->have_r || !b_dev || !x_dev) return RFM_EINVAL;
  RFM_TRY(clear_err(p));
  RFM_TRY(rfm_launch_trsv(p, trans, b_dev, x_dev));
  return check_timeout(p);
}

rfm_status rfm_lsqr(rfm_problem* p, const double* b_dev, double eta, double conlim, int64_t max_iter, double* d_dev,
                    int* iters_host, int* istop_host) {
  if (!p || !p->have_j || !p->have_r || !b_dev || !d_dev || !(eta > 0)) return RFM_EINVAL;
  RFM_TRY(clear_err(p));
  LsqrOut lo;
  RFM_TRY(lsqr(p, b_dev, eta, conlim, max_iter > 0 ? max_iter : 2 * p->n, d_dev, &lo));
  if (iters_host) *iters_host = lo.itn;
  if (istop_host) *istop_host = lo.istop;
  return RFM_OK;
}

rfm_status rfm_linesearch(rfm_problem* p, const double* c_dev, const double* d_dev, double f0, double* alpha_host,
                          double* fbest_host) {
  if (!p || !p->have_j || !c_dev || !d_dev) return RFM_EINVAL;
  double a = 0, fb = 0;
  RFM_TRY(linesearch(p, c_dev, d_dev, f0, &a, &fb));
  if (alpha_host) *alpha_host = a;
  if (fbest_host) *fbest_host = fb;
  return RFM_OK;
}

rfm_status rfm_ipn_solve(rfm_problem* p, const rfm_solve_opts* opts, double* c_dev, rfm_solve_info* info_out) {
  if (!p || !c_dev || !validate_opts(opts)) {
    g_err = "rfm_ipn_solve: bad argument";
    return RFM_EINVAL;
  }
  rfm_solve_info info;
  memset(&info, 0, sizeof(info));
  p->precision = opts->precision;
  RFM_TRY(clear_err(p));
  const long long n = p->n, m = p->m;
  double* b = wv(p, WV_B);
  double* d = wv(p, WV_D);
  rfm_status st = RFM_ENOCONV;
  {
    Timer total(p->stream, &info.t_total);
    for (int k = 0; k < opts->max_outer; ++k) {
      RFM_TRY(linearise(p, opts, c_dev, k, &info));
      double f0 = 0.0;
      RFM_TRY(rfm_norm2(p->stream, p->F, m, p->red, p->red + 1024 + 16));
      RFM_TRY(read_scalars(p, p->red + 1024 + 16, 1, &f0));
      k_neg_copy<<<vgrid(m), 256, 0, p->stream>>>(b, p->F, m);
      RFM_CHECK_LAUNCH();
      RFM_TRY(direction(p, opts, b, d, &info));
      double alpha = 0, f1 = f0;
      {
        Timer t(p->stream, &info.t_linesearch);
        RFM_TRY(linesearch(p, c_dev, d, f0, &alpha, &f1));
      }
      k_axpby<<<vgrid(n), 256, 0, p->stream>>>(c_dev, d, n, alpha, 1.0);
      RFM_CHECK_LAUNCH();
      info.outer_iters = k + 1;
      info.final_resid = f1;
      if (!std::isfinite(f1)) {
        st = RFM_ENONFINITE;
        break;
      }
      if (fabs(f1 - f0) < opts->eps) {
        st = RFM_OK;
        break;
      }
    }
  }
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  info.status = st;
  if (info_out) *info_out = info;
  if (st == RFM_ENOCONV) g_err = "IPN reached max_outer";
  return st;
}

rfm_status rfm_amipn_solve(rfm_problem* p, const rfm_solve_opts* opts, double* c_dev, rfm_solve_info* info_out) {
  if (!p || !c_dev || !validate_opts(opts)) {
    g_err = "rfm_amipn_solve: bad argument";
    return RFM_EINVAL;
  }
  rfm_solve_info info;
  memset(&info, 0, sizeof(info));
  p->precision = opts->precision;
  RFM_TRY(clear_err(p));
  const long long n = p->n, m = p->m;
  double* d = wv(p, WV_D);
  double* z = wv(p, WV_Z);
  double* Fprev = wv(p, WV_FPREV);
  double* Fnew = wv(p, WV_FNEW);
  double* diff = wv(p, WV_TM);
  double* sc = p->red + 1024 + 24;
  rfm_status st = RFM_ENOCONV;
  {
    Timer total(p->stream, &info.t_total);
    int kJ = 0;
    RFM_TRY(linearise(p, opts, c_dev, kJ, &info));
    for (int k = 0; k < opts->max_outer; ++k) {
      // F_{k,0} = -W F(u_k)
      double nk0 = 0.0;
      RFM_TRY(scaled_residual_norm(p, c_dev, Fprev, &nk0));
      k_neg_copy<<<vgrid(m), 256, 0, p->stream>>>(Fprev, Fprev, m);
      RFM_CHECK_LAUNCH();
      RFM_CUDA(cudaMemcpyAsync(z, c_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
      bool flag = true;
      double nk1 = nk0;
      for (int i = 0; i < opts->m_max; ++i) {
        RFM_TRY(direction(p, opts, Fprev, d, &info));
        double f0 = 0.0;
        RFM_TRY(rfm_norm2(p->stream, Fprev, m, p->red, sc));
        RFM_TRY(read_scalars(p, sc, 1, &f0));
        double alpha = 0, fb = 0;
        {
          Timer t(p->stream, &info.t_linesearch);
          RFM_TRY(linesearch(p, z, d, f0, &alpha, &fb));
        }
        k_axpby<<<vgrid(n), 256, 0, p->stream>>>(z, d, n, alpha, 1.0);
        RFM_CHECK_LAUNCH();
        double nn = 0.0;
        RFM_TRY(scaled_residual_norm(p, z, Fnew, &nn));
        k_neg_copy<<<vgrid(m), 256, 0, p->stream>>>(Fnew, Fnew, m);
        RFM_CHECK_LAUNCH();
        k_sub<<<vgrid(m), 256, 0, p->stream>>>(diff, Fnew, Fprev, m);
        RFM_CHECK_LAUNCH();
        double dn = 0.0;
        RFM_TRY(rfm_norm2(p->stream, diff, m, p->red, sc + 1));
        RFM_TRY(read_scalars(p, sc + 1, 1, &dn));
        std::swap(Fprev, Fnew);
        nk1 = nn;
        if (dn < opts->tau_rel * nk0) {
          flag = false;
          break;
        }
      }
      RFM_CUDA(cudaMemcpyAsync(c_dev, z, n * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
      info.outer_iters = k + 1;
      info.final_resid = nk1;
      if (!std::isfinite(nk1)) {
        st = RFM_ENONFINITE;
        break;
      }
      if (fabs(nk1 - nk0) < opts->eps) {
        st = RFM_OK;
        break;
      }
      if (flag) {
        ++kJ;
        RFM_TRY(linearise(p, opts, c_dev, kJ, &info));
      }
    }
  }
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  info.status = st;
  if (info_out) *info_out = info;
  if (st == RFM_ENOCONV) g_err = "AMIPN reached max_outer";
  return st;
}

rfm_status rfm_eval(const rfm_problem* p, const double* c_dev, const double* pts_dev, int64_t npts, double* u_dev) {
  if (!p || !c_dev || npts < 0) {
    g_err = "rfm_eval: bad argument";
    return RFM_EINVAL;
  }
  if (npts == 0) return RFM_OK;  // empty query set: nothing to read or write
  if (!pts_dev || !u_dev) {
    g_err = "rfm_eval: null points or output";
    return RFM_EINVAL;
  }
  RFM_TRY(rfm_launch_eval(p, c_dev, pts_dev, npts, u_dev));
  RFM_CUDA(cudaStreamSynchronize(p->stream));
  return RFM_OK;
}

}  // extern "C"
