// Matrix-vector kernels of the LSQR inner solve on J R^{-1} (Alg. 1 steps 3-4).
//
//  * k_jmv:   y = s1 * J x + s2 * y.  One warp per row; a row is W contiguous
//             doubles of its primary block (and W more of the secondary block
//             for interface rows), read once, coalesced.
//  * k_jtmv:  y = J^T x.  One CTA per (column block, 64-column chunk); the
//             rows touching the block are walked in a fixed order and the
//             eight warps' partial sums are combined in a fixed order, so the
//             result is deterministic.
//  * k_trsv_chain: x = R^{-1} b or x = R^{-T} b for the upper-triangular
//             preconditioner R (column-major, leading dimension ldr), in one
//             cooperative launch: one chain CTA solves the 64 x 64 diagonal
//             blocks in dependency order from tiles it prefetched into shared
//             memory, and helper CTAs stream the rest of R once, each adding
//             the contributions of published blocks to the blocks it owns
//             (details at the kernel).
//  * k_trsv:  the same solve for sizes with more blocks than the helpers can
//             own: 64-row blocks are claimed through a ticket counter in
//             dependency order, each block waits (bounded) on the per-block
//             flags of the blocks it needs, accumulates their contribution
//             with coalesced column reads of R, solves its diagonal block in
//             one warp and publishes its part of x with a release flag.
//  * k_partial_* / k_finish_*: deterministic two-stage norms and dots.
#include <algorithm>

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

// ---------------------------------------------------------------------------
// Triangular solve as one chain CTA plus helper CTAs (cooperative launch, all
// CTAs co-resident).  The 64-row blocks are solved in dependency order
// t = 0, 1, ... (block nblk-1-t for R^{-1}, block t for R^{-T}).  The chain
// CTA solves the diagonal blocks one after another, with the inverse Z_k of
// each 64 x 64 diagonal block, computed once per factorisation
// (k_trsv_dinv): x_k = Z_k (b_k - sum_j R_kj x_j), two dense products and no
// dependent substitution.  It holds Z_k and the tiles coupling block k to the
// two blocks solved just before (order distance 1 and 2) in shared memory
// (cp.async, issued ahead), so its step reads no global memory except the
// right-hand side and one partial sum.  The helper CTAs add the
// contributions of all earlier blocks (distance >= 3) as soon as each block
// is published: helper h owns the targets t = 3 + (h - 1) + H m, streams
// their tiles of R (each read once), and publishes each target's partial sum
// three steps before the chain needs it.  All sums are in a fixed order, so
// results are deterministic.  Waits are bounded (wait_flag).
constexpr int TLD = TB + 2;            // leading dimension of a shared-memory tile (doubles; 16-byte rows)
constexpr int TTILE = TB * TLD;        // doubles per shared-memory tile
constexpr int CHAIN_NEAR = 3;          // the chain applies distances 1 .. CHAIN_NEAR-1 itself
constexpr int HMAXT = 4;               // targets per helper CTA

__host__ __device__ constexpr size_t chain_smem_bytes() {
  return (size_t)(2 * 3 * TTILE + 3 * TB + TB + 2 * TB + 2 * TB) * sizeof(double);
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(double* dst, const double* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Tile of R with row block a and column block b into shared memory,
// column-major with leading dimension TLD: T[cc * TLD + rr] = R(a*64 + rr, b*64 + cc).
// Entries outside the n x n triangle's index range are zero.
__device__ __forceinline__ void load_tile(double* T, const double* __restrict__ R, long long ldr, int n, int a,
                                          int b, int first, int stride) {
  // pairs of rows: one 16-byte copy when both lie inside (R's leading
  // dimension and row offsets are even, so the source is 16-byte aligned)
  const bool even = (ldr & 1) == 0;
  for (int idx = first; idx < TB * TB / 2; idx += stride) {
    const int rr = (idx & (TB / 2 - 1)) * 2, cc = idx >> 5;
    const int gr = a * TB + rr, gc = b * TB + cc;
    double* dst = T + cc * TLD + rr;
    const double* src = R + (size_t)gc * ldr + gr;
    if (gc < n && gr + 1 < n && even) {
      cp_async16(dst, src);
    } else {
      if (gc < n && gr < n) cp_async8(dst, src);
      else dst[0] = 0.0;
      if (gc < n && gr + 1 < n) cp_async8(dst + 1, src + 1);
      else dst[1] = 0.0;
    }
  }
}

template <int TRANS>
__device__ __forceinline__ int chain_block(int t, int nblk) { return TRANS == 0 ? nblk - 1 - t : t; }

// Inverse of each 64 x 64 diagonal block of R, block k stored column-major at
// Z + k * 4096: Z[k][c * 64 + r] = (R_kk^{-1})(r, c).  Entries below the
// diagonal and, in a ragged last block, rows and columns past n are zero.
// Column c solves R_kk z = e_c by back substitution (one warp per column,
// rows on the lanes, IEEE division by each pivot).
__global__ void __launch_bounds__(256) k_trsv_dinv(const double* __restrict__ R, long long ldr, int n,
                                                   double* __restrict__ Z) {
  __shared__ double D[TB * TLD];
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = k * TB, rows = min(TB, n - r0);
  for (int idx = tid; idx < TB * TB; idx += blockDim.x) {
    const int r = idx & (TB - 1), c = idx >> 6;
    D[c * TLD + r] = (r <= c && c < rows) ? R[(size_t)(r0 + c) * ldr + r0 + r] : 0.0;
  }
  __syncthreads();
  double* out = Z + (size_t)k * TB * TB;
  for (int j = w; j < TB; j += 8) {
    double acc0 = lane == j ? 1.0 : 0.0, acc1 = lane + 32 == j ? 1.0 : 0.0;
    double z0 = 0.0, z1 = 0.0;
    if (j < rows) {
      for (int i = j; i >= 0; --i) {
        const double zi = __shfl_sync(0xffffffffu, i < 32 ? acc0 : acc1, i & 31) / D[i * TLD + i];
        if (i < 32 && lane == i) z0 = zi;
        if (i >= 32 && lane == i - 32) z1 = zi;
        if (lane < i) acc0 -= D[i * TLD + lane] * zi;
        if (lane + 32 < i) acc1 -= D[i * TLD + lane + 32] * zi;
      }
    }
    out[j * TB + lane] = z0;
    out[j * TB + lane + 32] = z1;
  }
}

// A helper's partial sum is published by overwriting this value, which the
// chain polls for: a signalling NaN with a fixed payload, which no
// arithmetic result has (operations on NaN return the canonical quiet NaN).
constexpr unsigned long long ACC_EMPTY = 0x7FF4A5A5A5A5A5A5ull;
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_b64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Before each chain launch: the progress counter at 0 and every helper
// partial sum at ACC_EMPTY.
__global__ void k_trsv_chain_prep(unsigned int* __restrict__ prog, double* __restrict__ accbuf, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *prog = 0u;
  if (i < count) reinterpret_cast<unsigned long long*>(accbuf)[i] = ACC_EMPTY;
}

struct ChainArgs {
  const double* R;
  const double* Z;            // inverses of the diagonal blocks (k_trsv_dinv)
  long long ldr;
  int n, nblk, H;
  const double* rhs;
  double* x;
  double* accbuf;             // [nblk][64] helper partial sums, ACC_EMPTY until published
  unsigned int* prog;         // number of blocks the chain has published (reset by k_trsv_chain_prep)
  unsigned int* err;
  const int* skip;
};

template <int TRANS>
__global__ void __launch_bounds__(256, 1) k_trsv_chain(ChainArgs a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) double csm[];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nblk = a.nblk, n = a.n;
  const int wlim = (int)__ldcg(a.err + (SYNC_WAITLIM - SYNC_ERR));
  const unsigned int wlimit = wlim == 0 ? (1u << 22) : (unsigned int)wlim;
  if (blockIdx.x == 0) {
    // ------------------------------------------------------------ chain
    // Warps 0-3 take step t's critical path: y = base_t - C1_t x_{t-1}, then
    // x_t = Z_k y, two threads per row (each a fixed half of the terms), with
    // base_t = b_k - (helper sum) - (distance-2 sum) prepared one step ahead.
    // Warps 4-7 meanwhile publish x_{t-1}, issue the copies of Z and C1 for
    // step t + 2, form the distance-2 sum of step t + 1 (C2_{t+1} x_{t-1},
    // with C2_{t+1} fetched into registers one step earlier), fetch C2_{t+2},
    // acquire the helpers' sum of step t + 1 and form base_{t+1}.
    double* Zb = csm;                          // [3] inverse diagonal tiles
    double* C1b = Zb + 3 * TTILE;              // [3] coupling to the previous block
    double* xh = C1b + 3 * TTILE;              // x of the last three steps [3][64]
    double* ys = xh + 3 * TB;                  // [64] right-hand side of the diagonal block
    double* base = ys + TB;                    // [2][64]
    double* d2p = base + 2 * TB;               // [2][64] halves of the distance-2 sum
    const bool crit = w < 4;
    const int ct = crit ? tid : tid - 128;     // thread index within its group of 128
    const int r = ct >> 1, hh = ct & 1;        // row and half (critical path)
    const int q64 = ct & 63, qh = ct >> 6;     // distance-2 layout
    // Term i (0..31) of half hh: the column index of a tile row.  The order
    // keeps a warp's shared-memory reads on distinct banks: T[term * TLD + r]
    // for TRANS 0, T[r * TLD + term] for TRANS 1.
    auto term = [&](int i) { return TRANS == 0 ? (i & 3) + 8 * (i >> 2) + 4 * hh : 2 * i + hh; };
    auto tile_dot = [&](const double* T, const double* v, int i0, int i1) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int i = i0; i < i1; i += 4) {
        const int y0 = term(i), y1 = term(i + 1), y2 = term(i + 2), y3 = term(i + 3);
        if (TRANS == 0) {
          s0 += T[y0 * TLD + r] * v[y0];
          s1 += T[y1 * TLD + r] * v[y1];
          s2 += T[y2 * TLD + r] * v[y2];
          s3 += T[y3 * TLD + r] * v[y3];
        } else {
          s0 += T[r * TLD + y0] * v[y0];
          s1 += T[r * TLD + y1] * v[y1];
          s2 += T[r * TLD + y2] * v[y2];
          s3 += T[r * TLD + y3] * v[y3];
        }
      }
      const double s = (s0 + s1) + (s2 + s3);
      return s + __shfl_xor_sync(0xffffffffu, s, 1);
    };
    auto issue_zc1 = [&](int tt) {             // Z_tt and C1_tt
      const int k = chain_block<TRANS>(tt, nblk);
      const double* src = a.Z + (size_t)k * TB * TB;
      double* dst = Zb + (tt % 3) * TTILE;
      for (int idx = ct; idx < TB * TB / 2; idx += 128) {
        const int rr = (idx & (TB / 2 - 1)) * 2, cc = idx >> 5;
        cp_async16(dst + cc * TLD + rr, src + cc * TB + rr);
      }
      if (tt >= 1) {
        const int j = chain_block<TRANS>(tt - 1, nblk);
        if (TRANS == 0) load_tile(C1b + (tt % 3) * TTILE, a.R, a.ldr, n, k, j, ct, 128);
        else load_tile(C1b + (tt % 3) * TTILE, a.R, a.ldr, n, j, k, ct, 128);
      }
    };
    // C2_tt in registers: thread (q64, qh) holds the 32 entries of output
    // row q64 of block k against the source rows 32 qh .. 32 qh + 31 of
    // block j.  TRANS 0: R(k*64 + q64, j*64 + 32 qh + i), one column of R per
    // entry, the lanes of a warp on consecutive rows; TRANS 1 (the coupling
    // of R^T): R(j*64 + 32 qh + i, k*64 + q64), 32 consecutive entries of one
    // column of R per thread.
    double c2v[32];
    auto fetch_c2 = [&](int tt) {
      const int k = chain_block<TRANS>(tt, nblk), j = chain_block<TRANS>(tt - 2, nblk);
      const int go = k * TB + q64, gs = j * TB + 32 * qh;  // output index, first source index
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const bool ok = go < n && gs + i < n;
        if (TRANS == 0) c2v[i] = ok ? __ldg(a.R + (size_t)(gs + i) * a.ldr + go) : 0.0;
        else c2v[i] = ok ? __ldg(a.R + (size_t)go * a.ldr + gs + i) : 0.0;
      }
    };
    // the half qh of C2 x_{t-2} for output q64, into d2p[2][64]
    auto dist2 = [&](const double* xv) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
      for (int i = 0; i < 32; i += 4) {
        s0 += c2v[i] * xv[32 * qh + i];
        s1 += c2v[i + 1] * xv[32 * qh + i + 1];
        s2 += c2v[i + 2] * xv[32 * qh + i + 2];
        s3 += c2v[i + 3] * xv[32 * qh + i + 3];
      }
      d2p[qh * TB + q64] = (s0 + s1) + (s2 + s3);
    };
    // x = Z y with the triangle balanced over the threads: rows g and 63 - g
    // share four threads (s = ct & 3), whose terms are the positions p = s,
    // s + 4, ... of the pair's 65 terms (row A = g first, then row B = 63 - g).
    const int zg = ct >> 2, zs = ct & 3;
    const int zA = zg, zB = TB - 1 - zg;
    const int znA = TRANS == 0 ? TB - zg : zg + 1;  // terms of row A
    auto zdot = [&](const double* Zt, const double* yv, double& xa, double& xb) {
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll
      for (int i = 0; i < 17; ++i) {
        const int pos = zs + 4 * i;
        if (pos > TB) break;  // 65 terms per pair
        const bool inA = pos < znA;
        // column of the term: TRANS 0 row A columns g .. 63, row B 63-g .. 63;
        // TRANS 1 row A columns 0 .. g, row B 0 .. 63-g
        const int c = TRANS == 0 ? (inA ? zg + pos : pos - 1) : (inA ? pos : pos - znA);
        const int row = inA ? zA : zB;
        const double zv = TRANS == 0 ? Zt[c * TLD + row] : Zt[row * TLD + c];
        const double prod = zv * yv[c];
        if (inA) {
          if (i & 1) a1 += prod; else a0 += prod;
        } else {
          if (i & 1) b1 += prod; else b0 += prod;
        }
      }
      double sa = a0 + a1, sb = b0 + b1;
      sa += __shfl_xor_sync(0xffffffffu, sa, 1);
      sb += __shfl_xor_sync(0xffffffffu, sb, 1);
      sa += __shfl_xor_sync(0xffffffffu, sa, 2);
      sb += __shfl_xor_sync(0xffffffffu, sb, 2);
      xa = sa;
      xb = sb;
    };
    if (!crit) {
      issue_zc1(0);
      cp_async_commit();
      if (nblk > 1) issue_zc1(1);
      cp_async_commit();
      if (ct < TB) {
        const int r0 = chain_block<TRANS>(0, nblk) * TB;
        base[ct] = r0 + ct < n ? a.rhs[r0 + ct] : 0.0;
      }
      cp_async_wait1();
    }
    __syncthreads();
    for (int t = 0; t < nblk; ++t) {
      if (crit) {
        const int k = chain_block<TRANS>(t, nblk);
        const int r0 = k * TB, rows = min(TB, n - r0);
        const double bs = base[(t & 1) * TB + r];
        const double p = t >= 1 ? tile_dot(C1b + (t % 3) * TTILE, xh + ((t + 2) % 3) * TB, 0, 32) : 0.0;
        if (hh == 0) ys[r] = bs - p;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        double xa, xb;
        zdot(Zb + (t % 3) * TTILE, ys, xa, xb);
        if (zs == 0) {
          xh[(t % 3) * TB + zA] = xa;
          if (zA < rows) a.x[r0 + zA] = xa;
        } else if (zs == 1) {
          xh[(t % 3) * TB + zB] = xb;
          if (zB < rows) a.x[r0 + zB] = xb;
        }
      } else {
        const bool more = t + 1 < nblk;
        const int r1 = more ? chain_block<TRANS>(t + 1, nblk) * TB : 0;
        const double rb = more && ct < TB && r1 + ct < n ? a.rhs[r1 + ct] : 0.0;
        if (ct == 96 && t >= 1) {  // blocks 0 .. t-1 are in a.x (barrier at the end of step t-1)
          __threadfence();
          st_release(a.prog, (unsigned int)t);
        }
        if (t + 2 < nblk) issue_zc1(t + 2);
        cp_async_commit();
        if (more) {
          if (t + 1 >= 2) {
            dist2(xh + ((t + 2) % 3) * TB);
          } else if (ct < TB) {
            d2p[ct] = 0.0;
            d2p[TB + ct] = 0.0;
          }
          if (t + 2 < nblk) fetch_c2(t + 2);
        }
        // the helpers' sum of step t + 1: poll the entry until it is published
        double acc = 0.0;
        if (more && ct < TB && t + 1 >= CHAIN_NEAR) {
          const double* src = a.accbuf + (size_t)r1 + ct;
          unsigned long long v = ld_relaxed_b64(src);
          unsigned int spins = 0;
          while (v == ACC_EMPTY) {
            if (wlim < 0 || ++spins > wlimit) {
              atomicExch(a.err, 1u);
              v = 0ull;
              break;
            }
            if (spins > (1u << 16)) __nanosleep(128);
            v = ld_relaxed_b64(src);
          }
          acc = __longlong_as_double((long long)v);
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (more && ct < TB) base[((t + 1) & 1) * TB + ct] = (rb - acc) - (d2p[ct] + d2p[TB + ct]);
        cp_async_wait1();  // Z_{t+1} and C1_{t+1}
      }
      __syncthreads();
    }
    if (!crit && ct == 96) {
      __threadfence();
      st_release(a.prog, (unsigned int)nblk);
    }
    cp_async_wait0();
    return;
  }
  // -------------------------------------------------------------- helper
  const int h = blockIdx.x - 1;
  int tg[HMAXT], nt = 0;
#pragma unroll
  for (int m = 0; m < HMAXT; ++m) {
    const int t = CHAIN_NEAR + h + a.H * m;
    tg[m] = t < nblk ? t : -1;
    if (t < nblk) nt = m + 1;
  }
  if (nt == 0) return;
  const int tmax = tg[nt - 1];
  double* sred = csm;                    // [8][64]
  __shared__ unsigned int seen_s;        // progress counter as last read
  double pa[HMAXT][2];   // TRANS 0: partial sums of target rows lane, lane+32 over this warp's sources
  double ptp[HMAXT][8];  // TRANS 1: partial sums of target rows w + 8 q over this lane's sources
#pragma unroll
  for (int m = 0; m < HMAXT; ++m) {
    pa[m][0] = pa[m][1] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) ptp[m][q] = 0.0;
  }
  unsigned int seen = 0;
  for (int u = 0; u + CHAIN_NEAR <= tmax; ++u) {
    const int j = chain_block<TRANS>(u, nblk);
    const int c0 = j * TB;
    // this step's tile entries into registers first (they do not depend on
    // x): TRANS 0 rows lane, lane+32 of R(k, j), columns w + 8 q; TRANS 1
    // rows w + 8 q of R(j, k) (columns of block k), read along j's rows
    double tv[HMAXT][16];
#pragma unroll
    for (int m = 0; m < HMAXT; ++m) {
      const bool live = m < nt && tg[m] >= u + CHAIN_NEAR;
      const int k = live ? chain_block<TRANS>(tg[m], nblk) : 0;
      const int r0 = k * TB;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int y = w + 8 * q;
        if (TRANS == 0) {  // R(r0 + lane (+32), c0 + y)
          const bool ok = live && c0 + y < n;
          const double* col = a.R + (size_t)(c0 + y) * a.ldr + r0;
          tv[m][2 * q] = ok && r0 + lane < n ? __ldg(col + lane) : 0.0;
          tv[m][2 * q + 1] = ok && r0 + lane + 32 < n ? __ldg(col + lane + 32) : 0.0;
        } else {           // R(c0 + lane (+32), r0 + y): target row y
          const bool ok = live && r0 + y < n;
          const double* col = a.R + (size_t)(r0 + y) * a.ldr + c0;
          tv[m][2 * q] = ok ? __ldg(col + lane) : 0.0;
          tv[m][2 * q + 1] = ok ? __ldg(col + lane + 32) : 0.0;
        }
      }
    }
    // block u published?  (the counter only grows; read it again only when needed)
    if (seen < (unsigned int)(u + 1)) {
      if (tid == 0) {
        unsigned int v = ld_acquire(a.prog), spins = 0;
        while (v < (unsigned int)(u + 1)) {
          if (wlim < 0 || ++spins > wlimit) {
            atomicExch(a.err, 1u);
            v = (unsigned int)(u + 1);
            break;
          }
          if (spins > (1u << 16)) __nanosleep(128);
          v = ld_acquire(a.prog);
        }
        seen_s = v;
      }
      __syncthreads();
      seen = seen_s;
    }
    double xv[8], z0 = 0.0, z1 = 0.0;
    if (TRANS == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int y = w + 8 * q;
        xv[q] = c0 + y < n ? __ldcg(a.x + c0 + y) : 0.0;
      }
    } else {
      z0 = __ldcg(a.x + c0 + lane);
      z1 = __ldcg(a.x + c0 + lane + 32);
    }
    // The target due now (its last helper source) first, then published;
    // then the targets still live.  Slots past their target (or empty) do no
    // arithmetic.
#pragma unroll
    for (int m = 0; m < HMAXT; ++m) {
      if (!(m < nt && tg[m] == u + CHAIN_NEAR)) continue;
      if (TRANS == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          pa[m][0] += tv[m][2 * q] * xv[q];
          pa[m][1] += tv[m][2 * q + 1] * xv[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) ptp[m][q] = fma(tv[m][2 * q + 1], z1, fma(tv[m][2 * q], z0, ptp[m][q]));
      }
      const int k = chain_block<TRANS>(tg[m], nblk);
      double* out = a.accbuf + (size_t)k * TB;
      if (TRANS == 0) {
        sred[w * TB + lane] = pa[m][0];
        sred[w * TB + lane + 32] = pa[m][1];
        __syncthreads();
        if (w == 0) {
          for (int hh = 0; hh < 2; ++hh) {
            double sm = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) sm += sred[q * TB + lane + 32 * hh];
            st_relaxed_f64(out + lane + 32 * hh, sm);
          }
        }
      } else {
        // sum of ptp[m][q] over the lanes, lane q (< 8) ends with entry q
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = ptp[m][q];
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int q = 0; q < o; ++q) {
            const double send = up ? v[q] : v[q + o];
            const double keep = up ? v[q + o] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
        // lanes L and L ^ 8, L ^ 16, L ^ 24 hold partial sums of entry L & 7
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 8);
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
        if (lane < 8) st_relaxed_f64(out + w + 8 * lane, v[0]);
      }
      __syncthreads();  // sred is rewritten by the next publication
    }
#pragma unroll
    for (int m = 0; m < HMAXT; ++m) {
      if (!(m < nt && tg[m] > u + CHAIN_NEAR)) continue;
      if (TRANS == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          pa[m][0] += tv[m][2 * q] * xv[q];
          pa[m][1] += tv[m][2 * q + 1] * xv[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) ptp[m][q] = fma(tv[m][2 * q + 1], z1, fma(tv[m][2 * q], z0, ptp[m][q]));
      }
    }
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

rfm_status rfm_trsv_prepare(rfm_problem* p) {
  if (!p->dinv || !p->R) return RFM_OK;
  const int n = (int)p->n;
  k_trsv_dinv<<<(n + TB - 1) / TB, 256, 0, p->stream>>>(p->R, p->ldr, n, p->dinv);
  RFM_CHECK_LAUNCH();
  p->dinv_of = p->R;
  return RFM_OK;
}

rfm_status rfm_launch_trsv(rfm_problem* p, int trans, const double* b, double* x) {
  const int n = (int)p->n;
  const int nblk = (n + TB - 1) / TB;
  if (nblk > RFM_SYNC_WORDS - SYNC_FLAGS) {
    rfm_set_error("trsv: too many blocks");
    return RFM_EINVAL;
  }
  if (p->dinv && p->dinv_of != p->R) RFM_TRY(rfm_trsv_prepare(p));
  ProfScope ps(PF_TRSV, p->stream);
  rfm_prof_work(PF_TRSV, 8.0 * (double)n * (n + 1) / 2 + 16.0 * n);  // R read once, b and x
  // chain + helpers when every target past distance 2 has a helper slot
  const int nsm = rfm_num_sms();
  const int H = nblk > CHAIN_NEAR ? std::min(nsm - 1, nblk - CHAIN_NEAR) : 0;
  if (p->trsv_acc && p->dinv && nsm > 1 && nblk - CHAIN_NEAR <= HMAXT * H) {
    k_trsv_chain_prep<<<(nblk * TB + 255) / 256, 256, 0, p->stream>>>(p->sync + SYNC_TICKET, p->trsv_acc, nblk * TB);
    RFM_CHECK_LAUNCH();
    ChainArgs a;
    a.R = p->R; a.Z = p->dinv; a.ldr = p->ldr; a.n = n; a.nblk = nblk; a.H = H; a.rhs = b; a.x = x;
    a.accbuf = p->trsv_acc; a.prog = p->sync + SYNC_TICKET;
    a.err = p->sync + SYNC_ERR; a.skip = p->skip;
    const void* fn = trans == 0 ? (const void*)k_trsv_chain<0> : (const void*)k_trsv_chain<1>;
    RFM_CUDA(rfm_smem_attr(fn, (int)chain_smem_bytes()));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(1 + H));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = chain_smem_bytes();
    cfg.stream = p->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident: helpers and the chain wait on each other
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (trans == 0) RFM_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_chain<0>, a));
    else RFM_CUDA(cudaLaunchKernelEx(&cfg, k_trsv_chain<1>, a));
    RFM_CHECK_LAUNCH();
    return RFM_OK;
  }
  k_trsv_prep<<<1, 1, 0, p->stream>>>(p->sync + SYNC_EPOCH, p->sync + SYNC_TICKET);
  RFM_CHECK_LAUNCH();
  if (trans == 0)
    k_trsv<0><<<nblk, 256, 0, p->stream>>>(p->R, p->ldr, n, b, x, p->sync + SYNC_FLAGS, p->sync + SYNC_EPOCH,
                                           p->sync + SYNC_TICKET, p->sync + SYNC_ERR, p->skip);
  else
    k_trsv<1><<<nblk, 256, 0, p->stream>>>(p->R, p->ldr, n, b, x, p->sync + SYNC_FLAGS, p->sync + SYNC_EPOCH,
                                           p->sync + SYNC_TICKET, p->sync + SYNC_ERR, p->skip);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}
