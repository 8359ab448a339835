// Assembly kernels of the RFM nonlinear least-squares system.
//
//  * k_features: k, b ~ U[-R, R] from Philox4x32-10 (Sec. 2.2, Eq. 2.6).
//  * k_points:   collocation points and right-hand sides f / g of every row
//                (Sec. 5: interior grids, interface faces Eqs. con:1-3,
//                boundary faces Eqs. bdy:1-3).
//  * k_assemble: residual F and Jacobian J of Alg. 3 steps 1-4, with the row
//                rescaling lambda_i = c / max_j |J_ij| (Sec. 5) fused into the
//                epilogue.  One warp per row: the tanh features of the row's
//                subdomain are evaluated once, staged in shared memory, and
//                the warp writes the scaled row (W contiguous doubles).
//  * k_ls_pre / k_ls_eval: the golden-section objective
//                phi(alpha) = ||W F(c + alpha d)|| (Alg. 1 step 5) in O(m) per
//                alpha after one pass that splits every row into its linear
//                part and the field values entering the nonlinearity.
//  * k_eval:     u_n(x) on the owning subdomain (Eq. 2.7, indicator PoU).
//
// Features: phi = tanh(z), z = sum_b k_b (x_b - mu_b)/sigma_b + b;
//   d phi/dx_b = (1 - t^2) k_b/sigma_b,  d^2 phi/dx_b^2 = -2 t (1 - t^2) (k_b/sigma_b)^2.
#include <math.h>

#include "philox.cuh"
#include "rfm_internal.cuh"

namespace {

constexpr double kPi = 3.141592653589793;

struct PdeConst {
  int kind, d, fields, M, W;
  double p[8];
};

__global__ void k_features(double* __restrict__ feat, long long nfeat, int d, double R, uint32_t key0,
                           uint32_t key1) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= nfeat) return;
  double v[4];
  const int npair = (d + 2) / 2;
  for (int r = 0; r < npair; ++r) {
    uint32_t c[4] = {0u, (uint32_t)g, (uint32_t)r, 0u};
    philox4x32_10(c, key0, key1);
    v[2 * r] = uniform53(c[0], c[1]);
    v[2 * r + 1] = uniform53(c[2], c[3]);
  }
  double out[4] = {0, 0, 0, 0};
  for (int t = 0; t <= d; ++t) out[t] = R * (2.0 * v[t] - 1.0);
  *reinterpret_cast<double4*>(feat + 4 * g) = make_double4(out[0], out[1], out[2], out[3]);
}

__device__ __forceinline__ double grid_pt(const double* X, int nbp, int b, int j, int p, int q) {
  const double a = X[b * nbp + j], c = X[b * nbp + j + 1];
  if (p == 0) return a;
  if (p == q - 1) return c;
  return a + ((c - a) * (double)p) / (double)(q - 1);
}

// Value, gradient and Hessian (H00 H11 H22 H01 H02 H12) of the manufactured
// solutions of the 3D examples of Sec. 6.2 (kinds 4-6), each a product of
// one-variable factors differentiated by hand:
//   kind 4  u = (2 + x^2 + y^2 + z^2) sin(pi x) sin(pi y) sin(pi z)
//   kind 5  u = (x + y + z) sin(pi x) sin(pi y) cos(pi z)
//   kind 6  u = sin(x(1-x)) sin(y(1-y)) e^(z + 1/2)
//   kind 7  u = (x^2 + y^2 + z^2) sin(pi x) sin(pi y) sin(pi z)
__device__ void exact_jet3(int kind, const double* x, double& u, double* g, double* h) {
  double f[3][3];  // factor b: value, first, second derivative
  if (kind == 6) {
    for (int b = 0; b < 2; ++b) {
      const double w = x[b] * (1.0 - x[b]), sw = sin(w), cw = cos(w), dw = 1.0 - 2.0 * x[b];
      f[b][0] = sw;
      f[b][1] = cw * dw;
      f[b][2] = -sw * dw * dw - 2.0 * cw;
    }
    const double e = exp(x[2] + 0.5);
    f[2][0] = f[2][1] = f[2][2] = e;
  } else {
    for (int b = 0; b < 3; ++b) {
      const double sn = sin(kPi * x[b]), cs = cos(kPi * x[b]);
      if (kind == 5 && b == 2) {
        f[b][0] = cs;
        f[b][1] = -kPi * sn;
        f[b][2] = -kPi * kPi * cs;
      } else {
        f[b][0] = sn;
        f[b][1] = kPi * cs;
        f[b][2] = -kPi * kPi * sn;
      }
    }
  }
  // P = f0 f1 f2 and its derivatives
  const double P = f[0][0] * f[1][0] * f[2][0];
  const double dP[3] = {f[0][1] * f[1][0] * f[2][0], f[0][0] * f[1][1] * f[2][0], f[0][0] * f[1][0] * f[2][1]};
  const double hP[6] = {f[0][2] * f[1][0] * f[2][0], f[0][0] * f[1][2] * f[2][0], f[0][0] * f[1][0] * f[2][2],
                        f[0][1] * f[1][1] * f[2][0], f[0][1] * f[1][0] * f[2][1], f[0][0] * f[1][1] * f[2][1]};
  if (kind == 6) {
    u = P;
    for (int b = 0; b < 3; ++b) g[b] = dP[b];
    for (int k = 0; k < 6; ++k) h[k] = hP[k];
    return;
  }
  // u = r P with r = 2 + |x|^2 (kind 4) or x + y + z (kind 5)
  double r, dr[3], hr;
  if (kind == 4 || kind == 7) {
    r = (kind == 4 ? 2.0 : 0.0) + x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    for (int b = 0; b < 3; ++b) dr[b] = 2.0 * x[b];
    hr = 2.0;  // diagonal of Hess r; off-diagonal 0
  } else {
    r = x[0] + x[1] + x[2];
    for (int b = 0; b < 3; ++b) dr[b] = 1.0;
    hr = 0.0;
  }
  u = r * P;
  for (int b = 0; b < 3; ++b) g[b] = dr[b] * P + r * dP[b];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k) {
    const int a = ia[k], b = ib[k];
    h[k] = (k < 3 ? hr * P : 0.0) + dr[a] * dP[b] + dP[a] * dr[b] + r * hP[k];
  }
}

// Residual of an interior row of kinds 4-6 from the 2-jet Q = (u, grad u,
// Hess u as H00 H11 H22 H01 H02 H12) of the solution at the point, and its
// partial derivatives C = dR/dQ (the Jacobian row is then
// sum_k C_k (2-jet of phi_j)_k):
//   kind 4  R = Lap u + p0 u + p1 cosh(u)                       (Sec. 6.2, Helmholtz)
//   kind 5  R = -(1 + u^2) Lap u - 2 u |grad u|^2               (-div((1 + u^2) grad u))
//   kind 6  R = -(1 + |g|^2) Lap u - 2 g^T H g                  (-div((1 + |grad u|^2) grad u))
//   kind 7  kind 5 plus the reaction u^3 - u + e^u              (diffusion-reaction on the unit ball)
__device__ __forceinline__ double jet_residual(const PdeConst& pc, const double* Q, double* C) {
  const double u = Q[0], g0 = Q[1], g1 = Q[2], g2 = Q[3];
  const double H00 = Q[4], H11 = Q[5], H22 = Q[6], H01 = Q[7], H02 = Q[8], H12 = Q[9];
  const double lap = H00 + H11 + H22;
#pragma unroll
  for (int k = 0; k < 10; ++k) C[k] = 0.0;
  if (pc.kind == 4) {
    C[0] = pc.p[0] + pc.p[1] * sinh(u);
    C[4] = C[5] = C[6] = 1.0;
    return lap + pc.p[0] * u + pc.p[1] * cosh(u);
  }
  const double gg = g0 * g0 + g1 * g1 + g2 * g2;
  if (pc.kind == 5 || pc.kind == 7) {
    const double L = 1.0 + u * u;
    C[0] = -2.0 * u * lap - 2.0 * gg;
    C[1] = -4.0 * u * g0;
    C[2] = -4.0 * u * g1;
    C[3] = -4.0 * u * g2;
    C[4] = C[5] = C[6] = -L;
    double R = -L * lap - 2.0 * u * gg;
    if (pc.kind == 7) {  // reaction u^3 - u + e^u
      const double eu = exp(u);
      C[0] += 3.0 * u * u - 1.0 + eu;
      R += u * u * u - u + eu;
    }
    return R;
  }
  const double L = 1.0 + gg;
  const double Hg0 = H00 * g0 + H01 * g1 + H02 * g2;
  const double Hg1 = H01 * g0 + H11 * g1 + H12 * g2;
  const double Hg2 = H02 * g0 + H12 * g1 + H22 * g2;
  C[1] = -2.0 * g0 * lap - 4.0 * Hg0;
  C[2] = -2.0 * g1 * lap - 4.0 * Hg1;
  C[3] = -2.0 * g2 * lap - 4.0 * Hg2;
  C[4] = -L - 2.0 * g0 * g0;
  C[5] = -L - 2.0 * g1 * g1;
  C[6] = -L - 2.0 * g2 * g2;
  C[7] = -4.0 * g0 * g1;
  C[8] = -4.0 * g0 * g2;
  C[9] = -4.0 * g1 * g2;
  return -L * lap - 2.0 * (g0 * Hg0 + g1 * Hg1 + g2 * Hg2);
}

__device__ double exact_field(const PdeConst& pc, const double* x, int f) {
  if (pc.kind == 3) return 0.0;
  if (pc.kind >= 4) {
    double u, g[3], h[6];
    exact_jet3(pc.kind, x, u, g, h);
    return u;
  }
  if (pc.kind == 1 && f == 0) {
    const double ax = x[0] * (1.0 - x[0]), ay = x[1] * (1.0 - x[1]);
    return sin(ax) * sin(ay) * exp(x[2]);
  }
  double s = 1.0;
  for (int b = 0; b < pc.d; ++b) s = s * sin(kPi * x[b]);
  return s;
}

__device__ double source_term(const PdeConst& pc, const double* x, int f) {
  const int d = pc.d;
  const double pi = kPi;
  if (pc.kind == 0) {
    const double u = exact_field(pc, x, 0);
    return d * pi * pi * u + pc.p[0] * (u * u * u);
  }
  if (pc.kind == 2) {
    const double u = exact_field(pc, x, 0);
    const double a = 1.0 + 0.5 * sin(2.0 * pi * x[0]);
    const double ax = pi * cos(2.0 * pi * x[0]);
    double ux = pi * cos(pi * x[0]);
    for (int b = 1; b < d; ++b) ux = ux * sin(pi * x[b]);
    return a * d * pi * pi * u - ax * ux + pc.p[0] * (u * u * u);
  }
  if (pc.kind == 3) {
    double s = 1.0;
    for (int b = 0; b < d; ++b) s = s * sin(pc.p[2] * pi * x[b]);
    return pc.p[1] * s;
  }
  if (pc.kind >= 4) {
    double Q[10], C[10];
    exact_jet3(pc.kind, x, Q[0], Q + 1, Q + 4);
    return jet_residual(pc, Q, C);
  }
  // kind 1: Gray-Scott with u = sin(x(1-x)) sin(y(1-y)) e^z, v = prod sin(pi x_b)
  const double eu = pc.p[0], ev = pc.p[1], Fc = pc.p[2], kk = pc.p[3];
  const double X0 = x[0], Y0 = x[1], Z0 = x[2];
  const double ax = X0 * (1 - X0), ay = Y0 * (1 - Y0);
  const double sx = sin(ax), cx = cos(ax), sy = sin(ay), cy = cos(ay), ez = exp(Z0);
  const double u = sx * sy * ez;
  const double uxx = (-sx * ((1 - 2 * X0) * (1 - 2 * X0)) - 2 * cx) * sy * ez;
  const double uyy = sx * (-sy * ((1 - 2 * Y0) * (1 - 2 * Y0)) - 2 * cy) * ez;
  const double lap_u = uxx + uyy + u;
  const double v = sin(pi * X0) * sin(pi * Y0) * sin(pi * Z0);
  const double lap_v = -3 * pi * pi * v;
  if (f == 0) return -eu * lap_u + u * v * v - Fc * (1 - u);
  return -ev * lap_v - u * v * v + (Fc + kk) * v;
}

__global__ void k_points(const RowSeg* __restrict__ segs, int nseg, const double* __restrict__ X, int nbp,
                         PdeConst pc, int N0, int N1, int N2, const double* __restrict__ lo,
                         double* __restrict__ pts, int4* __restrict__ meta, double* __restrict__ rhs,
                         long long m) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int lo_s = 0, hi_s = nseg - 1;
  while (lo_s < hi_s) {
    const int mid = (lo_s + hi_s + 1) / 2;
    if (segs[mid].row0 <= i) lo_s = mid; else hi_s = mid - 1;
  }
  const RowSeg sg = segs[lo_s];
  long long li = i - sg.row0;
  const int d = pc.d;
  const int Ns[3] = {N0, N1, N2};
  int idx[3];
  {
    int e = sg.e0;
    for (int b = d - 1; b >= 0; --b) {
      idx[b] = e % Ns[b];
      e /= Ns[b];
    }
  }
  double x[3] = {0, 0, 0};
  for (int b = d - 1; b >= 0; --b) {
    if (sg.kind != 0 && b == sg.axis) continue;
    const int q = sg.q[b];
    const int pcoord = (int)(li % q);
    li /= q;
    x[b] = grid_pt(X, nbp, b, idx[b], pcoord, q);
  }
  if (sg.kind == 1) x[sg.axis] = X[sg.axis * nbp + idx[sg.axis] + 1];
  if (sg.kind == 2) x[sg.axis] = sg.side == 0 ? X[sg.axis * nbp] : X[sg.axis * nbp + Ns[sg.axis]];
  *reinterpret_cast<double4*>(pts + 4 * i) = make_double4(x[0], x[1], x[2], 0.0);
  const int code = sg.kind | (sg.field << 4) | ((sg.axis & 0xF) << 8) | (sg.sord << 12) | ((sg.side & 1) << 16);
  meta[i] = make_int4(code, sg.e0, sg.e1, 0);
  double r = 0.0;
  if (sg.kind == 0) r = source_term(pc, x, sg.field);
  else if (sg.kind == 2) r = exact_field(pc, x, sg.field);
  rhs[i] = r;
}

// Right-hand sides of rows whose points and metadata the host built (masked
// geometries): the source f on interior rows, the Dirichlet data g on
// boundary rows, 0 on interface rows.
__global__ void k_rows_rhs(PdeConst pc, const double* __restrict__ pts, const int4* __restrict__ meta,
                           double* __restrict__ rhs, long long m) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int code = meta[i].x, kind = code & 0xF, f = (code >> 4) & 0xF;
  const double x[3] = {pts[4 * i], pts[4 * i + 1], pts[4 * i + 2]};
  rhs[i] = kind == 0 ? source_term(pc, x, f) : (kind == 2 ? exact_field(pc, x, f) : 0.0);
}

// Nonlinear term N_f(u) of the row's field and its partial derivatives
// coef[g] = dN_f / du_g.
__device__ __forceinline__ double nonlinear(const PdeConst& pc, int f, const double* u, double* coef) {
  if (pc.kind == 1) {
    const double Fc = pc.p[2], kk = pc.p[3];
    const double uu = u[0], vv = u[1];
    if (f == 0) {
      coef[0] = vv * vv + Fc;
      coef[1] = 2.0 * uu * vv;
      return uu * vv * vv - Fc * (1.0 - uu);
    }
    coef[0] = -(vv * vv);
    coef[1] = -2.0 * uu * vv + (Fc + kk);
    return -uu * vv * vv + (Fc + kk) * vv;
  }
  const double k3 = pc.p[0];
  coef[0] = 3.0 * k3 * (u[0] * u[0]);
  coef[1] = 0.0;
  return k3 * (u[0] * u[0] * u[0]);
}

struct RowGeo {
  double l[3];    // l_e(x)
  double is[3];   // 1 / sigma_e  (used as k_b / sigma_b)
  double sg[3];
};

__device__ __forceinline__ RowGeo row_geo(const double* mu, const double* sig, int e, const double* x, int d) {
  RowGeo g;
  for (int b = 0; b < 3; ++b) {
    if (b < d) {
      const double s = sig[4 * e + b];
      g.sg[b] = s;
      g.l[b] = (x[b] - mu[4 * e + b]) / s;
    } else {
      g.sg[b] = 1.0;
      g.l[b] = 0.0;
    }
  }
  return g;
}

// tanh feature at the row point: t, 1 - t^2 and the feature vector k.
__device__ __forceinline__ void feature_at(const double4 kb, const RowGeo& g, int d, double& t, double& s1) {
  double z = g.l[0] * kb.x;
  if (d > 1) z = z + g.l[1] * kb.y;
  if (d > 2) z = z + g.l[2] * kb.z;
  z = z + (d == 2 ? kb.z : kb.w);
  t = tanh(z);
  s1 = 1.0 - t * t;
}

__device__ __forceinline__ double kcomp(const double4 kb, int b) { return b == 0 ? kb.x : (b == 1 ? kb.y : kb.z); }

// Linear-operator part L(phi_j) of an interior row of field f (Alg. 3 step 1).
__device__ __forceinline__ double linear_part(const PdeConst& pc, int f, const double4 kb, const RowGeo& g,
                                              double t, double s1, double a, double ax) {
  double lap = 0.0;
  for (int b = 0; b < pc.d; ++b) {
    const double ks = kcomp(kb, b) / g.sg[b];
    lap = lap + (-2.0 * t * s1) * (ks * ks);
  }
  if (pc.kind == 0) return -lap;
  if (pc.kind == 1) return -(f == 0 ? pc.p[0] : pc.p[1]) * lap;
  const double gx = s1 * (kb.x / g.sg[0]);
  return -a * lap - ax * gx;
}

enum { MODE_JF = 0, MODE_RES = 1, MODE_LS = 2 };

// One warp per row.  MODE_JF: scaled J row + scaled F + lambda.  MODE_RES:
// lambda-scaled F only (lambda given).  MODE_LS: line-search split of the row
// at the two vectors c and dv.
template <int MODE>
__global__ void __launch_bounds__(128) k_assemble(PdeConst pc, const double* __restrict__ pts,
                                                  const int4* __restrict__ meta, const double* __restrict__ rhs,
                                                  const double* __restrict__ feat, const double* __restrict__ mu,
                                                  const double* __restrict__ sig, const double* __restrict__ c,
                                                  const double* __restrict__ dv, long long m, long long m_int,
                                                  double cscale, const double* __restrict__ lam_in,
                                                  double* __restrict__ Jp, double* __restrict__ Js,
                                                  double* __restrict__ lam_out, double* __restrict__ Fout,
                                                  double* __restrict__ P1, double* __restrict__ U,
                                                  double* __restrict__ V) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = pc.W, M = pc.M, d = pc.d, fields = pc.fields;
  double* sA = smem + (size_t)wib * 2 * W;   // phi values of all fields (or e0 values)
  double* sB = sA + W;                        // linear part of the row field (or e1 values)
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + wib; i < m; i += nwarps) {
    const int4 mt = meta[i];
    const int kind = mt.x & 0xF, f = (mt.x >> 4) & 0xF, axis = (mt.x >> 8) & 0xF, sord = (mt.x >> 12) & 0xF;
    const int e0 = mt.y, e1 = mt.z;
    const double4 xp = *reinterpret_cast<const double4*>(pts + 4 * i);
    const double x[3] = {xp.x, xp.y, xp.z};
    double Fi = 0.0, Fd = 0.0;
    double rowmax = 0.0;
    if (kind == 0 && pc.kind >= 4) {
      // kinds 4-6 (one field, 3D): the residual is a function of the 2-jet
      // of u at the point.  Pass 1 accumulates the jet, the residual gives
      // the coefficients C = dR/dQ, pass 2 forms J_j = sum_k C_k jet_k(phi_j).
      const RowGeo g = row_geo(mu, sig, e0, x, d);
      const long long fb = (long long)e0 * M;
      double Q[10], Qd[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        Q[k] = 0.0;
        Qd[k] = 0.0;
      }
      for (int j = lane; j < M; j += 32) {
        const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * (fb + j));
        double t, s1;
        feature_at(kb, g, d, t, s1);
        const double k0 = kb.x / g.sg[0], k1 = kb.y / g.sg[1], k2 = kb.z / g.sg[2];
        const double h = -2.0 * t * s1;
        const double jt[10] = {t, s1 * k0, s1 * k1, s1 * k2, h * k0 * k0, h * k1 * k1, h * k2 * k2,
                               h * k0 * k1, h * k0 * k2, h * k1 * k2};
        const double cj = c[fb + j];
#pragma unroll
        for (int k = 0; k < 10; ++k) Q[k] += cj * jt[k];
        if (MODE == MODE_LS) {
          const double dj = dv[fb + j];
#pragma unroll
          for (int k = 0; k < 10; ++k) Qd[k] += dj * jt[k];
        }
        if (MODE == MODE_JF) {
          sA[j] = t;
          sB[j] = s1;
        }
      }
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        Q[k] = warp_sum(Q[k]);
        if (MODE == MODE_LS) Qd[k] = warp_sum(Qd[k]);
      }
      if (MODE == MODE_LS) {
        if (lane == 0) {
          Fout[i] = -rhs[i];
          P1[i] = 0.0;
#pragma unroll
          for (int k = 0; k < 10; ++k) {
            U[i * 10 + k] = Q[k];
            V[i * 10 + k] = Qd[k];
          }
        }
        continue;
      }
      double C[10];
      Fi = jet_residual(pc, Q, C) - rhs[i];
      if (MODE == MODE_JF) {
        __syncwarp();
        for (int j = lane; j < M; j += 32) {
          const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * (fb + j));
          const double k0 = kb.x / g.sg[0], k1 = kb.y / g.sg[1], k2 = kb.z / g.sg[2];
          const double t = sA[j], s1 = sB[j], h = -2.0 * t * s1;
          const double Jv = C[0] * t + s1 * (C[1] * k0 + C[2] * k1 + C[3] * k2) +
                            h * (C[4] * k0 * k0 + C[5] * k1 * k1 + C[6] * k2 * k2 + C[7] * k0 * k1 +
                                 C[8] * k0 * k2 + C[9] * k1 * k2);
          sA[j] = Jv;
          rowmax = fmax(rowmax, fabs(Jv));
        }
      }
    } else if (kind == 0) {
      const RowGeo g = row_geo(mu, sig, e0, x, d);
      double a = 0.0, ax = 0.0;
      if (pc.kind >= 2) {
        a = 1.0 + 0.5 * sin(2.0 * kPi * x[0]);
        ax = kPi * cos(2.0 * kPi * x[0]);
      }
      double u[RFM_MAX_FIELDS] = {0, 0}, ud[RFM_MAX_FIELDS] = {0, 0};
      double lu = 0.0, lud = 0.0;
      for (int ff = 0; ff < fields; ++ff) {
        const long long fb = ((long long)e0 * fields + ff) * M;
        for (int j = lane; j < M; j += 32) {
          const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * (fb + j));
          double t, s1;
          feature_at(kb, g, d, t, s1);
          const double cj = c[fb + j];
          u[ff] += t * cj;
          if (MODE == MODE_LS) ud[ff] += t * dv[fb + j];
          if (MODE == MODE_JF) sA[ff * M + j] = t;
          if (ff == f) {
            const double L = linear_part(pc, f, kb, g, t, s1, a, ax);
            lu += L * cj;
            if (MODE == MODE_LS) lud += L * dv[fb + j];
            if (MODE == MODE_JF) sB[j] = L;
          }
        }
      }
      for (int ff = 0; ff < fields; ++ff) {
        u[ff] = warp_sum(u[ff]);
        if (MODE == MODE_LS) ud[ff] = warp_sum(ud[ff]);
      }
      lu = warp_sum(lu);
      if (MODE == MODE_LS) lud = warp_sum(lud);
      double coef[2];
      const double N = nonlinear(pc, f, u, coef);
      Fi = lu + N - rhs[i];
      if (MODE == MODE_LS) {
        if (lane == 0) {
          Fout[i] = lu - rhs[i];
          P1[i] = lud;
          for (int ff = 0; ff < fields; ++ff) {
            U[i * fields + ff] = u[ff];
            V[i * fields + ff] = ud[ff];
          }
        }
        continue;
      }
      if (MODE == MODE_JF) {
        __syncwarp();
        for (int ff = 0; ff < fields; ++ff)
          for (int j = lane; j < M; j += 32) {
            const double Jv = (ff == f ? sB[j] : 0.0) + coef[ff] * sA[ff * M + j];
            sA[ff * M + j] = Jv;
            rowmax = fmax(rowmax, fabs(Jv));
          }
      }
    } else {
      // interface (C^0 / C^1 rows, Eqs. con:1-3) or boundary (Eqs. bdy:1-3)
      const bool iface = kind == 1;
      double acc = 0.0, accd = 0.0;
      for (int side = 0; side < (iface ? 2 : 1); ++side) {
        const int e = side == 0 ? e0 : e1;
        const double sgn = side == 0 ? 1.0 : -1.0;
        const RowGeo g = row_geo(mu, sig, e, x, d);
        const long long fb = ((long long)e * fields + f) * M;
        double* dst = side == 0 ? sA : sB;
        for (int j = lane; j < M; j += 32) {
          const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * (fb + j));
          double t, s1;
          feature_at(kb, g, d, t, s1);
          double val = t;
          if (iface && sord == 1) val = s1 * (kcomp(kb, axis) / g.sg[axis]);
          val = sgn * val;
          acc += val * c[fb + j];
          if (MODE == MODE_LS) accd += val * dv[fb + j];
          if (MODE == MODE_JF) {
            dst[j] = val;
            rowmax = fmax(rowmax, fabs(val));
          }
        }
      }
      acc = warp_sum(acc);
      if (MODE == MODE_LS) accd = warp_sum(accd);
      Fi = acc - (kind == 2 ? rhs[i] : 0.0);
      Fd = accd;
      if (MODE == MODE_LS) {
        if (lane == 0) {
          Fout[i] = Fi;
          P1[i] = Fd;
        }
        continue;
      }
    }
    if (MODE == MODE_RES) {
      if (lane == 0) Fout[i] = lam_in[i] * Fi;
      continue;
    }
    // MODE_JF epilogue: lambda_i = c / max_j |J_ij| (zero row keeps 1)
    rowmax = warp_max(rowmax);
    const double lam = rowmax > 0.0 ? cscale / rowmax : 1.0;
    __syncwarp();
    double* jrow = Jp + (size_t)i * W;
    if (kind == 0) {
      for (int col = lane; col < W; col += 32) jrow[col] = lam * sA[col];
    } else {
      for (int col = lane; col < W; col += 32) {
        const int ff = col / M, j = col - ff * M;
        jrow[col] = ff == f ? lam * sA[j] : 0.0;
      }
      if (kind == 1) {
        double* srow = Js + (size_t)(i - m_int) * W;
        for (int col = lane; col < W; col += 32) {
          const int ff = col / M, j = col - ff * M;
          srow[col] = ff == f ? lam * sB[j] : 0.0;
        }
      }
    }
    if (lane == 0) {
      lam_out[i] = lam;
      Fout[i] = lam * Fi;
    }
    __syncwarp();
  }
}

// phi(alpha)^2 partial sums: sum_i (lambda_i (P0 + alpha P1 + N_f(U + alpha V)))^2.
__global__ void k_ls_eval(PdeConst pc, const int4* __restrict__ meta, const double* __restrict__ lam,
                          const double* __restrict__ P0, const double* __restrict__ P1,
                          const double* __restrict__ U, const double* __restrict__ V, long long m,
                          double alpha, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    double val = P0[i] + alpha * P1[i];
    const int kind = meta[i].x & 0xF;
    if (kind == 0 && pc.kind >= 4) {
      double q[10], C[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) q[k] = U[i * 10 + k] + alpha * V[i * 10 + k];
      val += jet_residual(pc, q, C);
    } else if (kind == 0) {
      const int f = (meta[i].x >> 4) & 0xF;
      double u[2] = {0, 0}, coef[2];
      for (int ff = 0; ff < pc.fields; ++ff) u[ff] = U[i * pc.fields + ff] + alpha * V[i * pc.fields + ff];
      val += nonlinear(pc, f, u, coef);
    }
    const double r = lam[i] * val;
    acc += r * r;
  }
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

__global__ void k_sum_sqrt(const double* __restrict__ partial, int np, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) acc += partial[i];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[0] = sqrt(acc);
}

// u_n(x) at query points: one warp per point, lanes over features.
__global__ void k_eval(PdeConst pc, const double* __restrict__ feat, const double* __restrict__ mu,
                       const double* __restrict__ sig, const double* __restrict__ lo, const double* __restrict__ hi,
                       int N0, int N1, int N2, const double* __restrict__ c, const double* __restrict__ pts,
                       long long npts, double* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const int Ns[3] = {N0, N1, N2};
  for (long long q = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); q < npts; q += nwarps) {
    double x[3] = {0, 0, 0};
    int e = 0;
    for (int b = 0; b < pc.d; ++b) {
      x[b] = pts[q * pc.d + b];
      int t = (int)floor((x[b] - lo[b]) / (hi[b] - lo[b]) * Ns[b]);
      t = t < 0 ? 0 : (t > Ns[b] - 1 ? Ns[b] - 1 : t);
      e = e * Ns[b] + t;
    }
    const RowGeo g = row_geo(mu, sig, e, x, pc.d);
    for (int ff = 0; ff < pc.fields; ++ff) {
      const long long fb = ((long long)e * pc.fields + ff) * pc.M;
      double acc = 0.0;
      for (int j = lane; j < pc.M; j += 32) {
        const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * (fb + j));
        double t, s1;
        feature_at(kb, g, pc.d, t, s1);
        acc += t * c[fb + j];
      }
      acc = warp_sum(acc);
      if (lane == 0) u[q * pc.fields + ff] = acc;
    }
  }
}

// Phi[q][col] = scale * phi_col(x_q) for the W = fields*M features of the
// owning subdomain of point q (FP32 output).  One warp per point.
__global__ void k_phi_values(PdeConst pc, const double* __restrict__ feat, const double* __restrict__ mu,
                             const double* __restrict__ sig, const double* __restrict__ lo,
                             const double* __restrict__ hi, int N0, int N1, int N2, const double* __restrict__ pts,
                             long long npts, float scale, float* __restrict__ Phi) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const int Ns[3] = {N0, N1, N2};
  for (long long q = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); q < npts; q += nwarps) {
    double x[3] = {0, 0, 0};
    int e = 0;
    for (int b = 0; b < pc.d; ++b) {
      x[b] = pts[q * pc.d + b];
      int t = (int)floor((x[b] - lo[b]) / (hi[b] - lo[b]) * Ns[b]);
      t = t < 0 ? 0 : (t > Ns[b] - 1 ? Ns[b] - 1 : t);
      e = e * Ns[b] + t;
    }
    const RowGeo g = row_geo(mu, sig, e, x, pc.d);
    for (int col = lane; col < pc.W; col += 32) {
      const long long fb = (long long)e * pc.W + col;
      const double4 kb = *reinterpret_cast<const double4*>(feat + 4 * fb);
      double t, s1;
      feature_at(kb, g, pc.d, t, s1);
      Phi[(size_t)q * pc.W + col] = scale * (float)t;
    }
  }
}

PdeConst make_pc(const rfm_problem* p) {
  PdeConst pc;
  pc.kind = p->desc.pde_kind;
  pc.d = p->d;
  pc.fields = p->fields;
  pc.M = p->M;
  pc.W = p->W;
  for (int i = 0; i < 8; ++i) pc.p[i] = p->desc.pde_params[i];
  return pc;
}

int grid_for(long long work, int per_block, int cap) {
  long long g = (work + per_block - 1) / per_block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

size_t asm_smem(const rfm_problem* p) { return (size_t)4 * 2 * p->W * sizeof(double); }

}  // namespace

rfm_status rfm_launch_setup(rfm_problem* p) {
  const long long nfeat = (long long)p->G * p->fields * p->M;
  const uint32_t k0 = (uint32_t)(p->desc.seed & 0xffffffffull), k1 = (uint32_t)(p->desc.seed >> 32);
  k_features<<<grid_for(nfeat, 256, 1 << 30), 256, 0, p->stream>>>(p->feat, nfeat, p->d, p->desc.feat_range, k0,
                                                                     k1);
  RFM_CHECK_LAUNCH();
  PdeConst pc = make_pc(p);
  if (p->explicit_rows)  // points and metadata uploaded by the host: right-hand sides only
    k_rows_rhs<<<grid_for(p->m, 256, 1 << 30), 256, 0, p->stream>>>(pc, p->pts, p->rmeta, p->rhs, p->m);
  else
    k_points<<<grid_for(p->m, 256, 1 << 30), 256, 0, p->stream>>>(
        p->segs, p->nseg, p->X, p->nmaxbp, pc, p->N[0], p->N[1], p->N[2], nullptr, p->pts, p->rmeta, p->rhs, p->m);
  RFM_CHECK_LAUNCH();
  {  // once per device
    const int bytes = 4 * 2 * RFM_MAX_WIDTH * (int)sizeof(double);
    RFM_CUDA(rfm_smem_attr((const void*)k_assemble<MODE_JF>, bytes));
    RFM_CUDA(rfm_smem_attr((const void*)k_assemble<MODE_RES>, bytes));
    RFM_CUDA(rfm_smem_attr((const void*)k_assemble<MODE_LS>, bytes));
  }
  return RFM_OK;
}

rfm_status rfm_launch_assemble(rfm_problem* p, const double* c, double cscale, bool want_j, const double* lam_in,
                               double* Fout) {
  PdeConst pc = make_pc(p);
  const int grid = grid_for(p->m, 4, 152 * 16);
  ProfScope ps(want_j ? PF_ASSEMBLE : PF_RESIDUAL, p->stream);
  if (want_j) rfm_prof_work(PF_ASSEMBLE, 8.0 * ((double)(p->m + p->m_iface) * p->W + 2.0 * p->m));
  if (want_j) {
    k_assemble<MODE_JF><<<grid, 128, asm_smem(p), p->stream>>>(pc, p->pts, p->rmeta, p->rhs, p->feat, p->mu, p->sig, c,
                                                               nullptr, p->m, p->m_int, cscale, nullptr, p->Jp, p->Js,
                                                               p->lam, Fout, nullptr, nullptr, nullptr);
  } else {
    k_assemble<MODE_RES><<<grid, 128, asm_smem(p), p->stream>>>(pc, p->pts, p->rmeta, p->rhs, p->feat, p->mu, p->sig,
                                                                c, nullptr, p->m, p->m_int, cscale, lam_in, nullptr,
                                                                nullptr, nullptr, Fout, nullptr, nullptr, nullptr);
  }
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_ls_precompute(rfm_problem* p, const double* c, const double* dvec, double* P0, double* P1,
                                    double* U, double* V) {
  PdeConst pc = make_pc(p);
  const int grid = grid_for(p->m, 4, 152 * 16);
  ProfScope ps(PF_LS_PRE, p->stream);
  k_assemble<MODE_LS><<<grid, 128, asm_smem(p), p->stream>>>(pc, p->pts, p->rmeta, p->rhs, p->feat, p->mu, p->sig, c,
                                                             dvec, p->m, p->m_int, 0.0, nullptr, nullptr, nullptr,
                                                             nullptr, P0, P1, U, V);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_ls_eval(rfm_problem* p, const double* P0, const double* P1, const double* U, const double* V,
                              double alpha, double* out_dev) {
  PdeConst pc = make_pc(p);
  const int nb = 304;
  ProfScope ps(PF_LS_EVAL, p->stream);
  k_ls_eval<<<nb, 256, 0, p->stream>>>(pc, p->rmeta, p->lam, P0, P1, U, V, p->m, alpha, p->red);
  RFM_CHECK_LAUNCH();
  k_sum_sqrt<<<1, 32, 0, p->stream>>>(p->red, nb, out_dev);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_eval(const rfm_problem* p, const double* c, const double* pts, long long npts, double* u) {
  PdeConst pc = make_pc(p);
  double* lohi = p->work;  // caller guarantees no concurrent use
  (void)lohi;
  // lo/hi live in the first 6 doubles after the breakpoint table (see api.cu)
  const double* lo = p->X + 3 * p->nmaxbp;
  const double* hi = lo + 3;
  ProfScope ps(PF_EVAL, p->stream);
  k_eval<<<grid_for(npts, 8, 152 * 32), 256, 0, p->stream>>>(pc, p->feat, p->mu, p->sig, lo, hi, p->N[0], p->N[1],
                                                             p->N[2], c, pts, npts, u);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_launch_phi_values(const rfm_problem* p, const double* pts, long long npts, float scale, float* Phi) {
  PdeConst pc = make_pc(p);
  const double* lo = p->X + 3 * p->nmaxbp;
  const double* hi = lo + 3;
  k_phi_values<<<grid_for(npts, 8, 152 * 32), 256, 0, p->stream>>>(pc, p->feat, p->mu, p->sig, lo, hi, p->N[0],
                                                                   p->N[1], p->N[2], pts, npts, scale, Phi);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}
