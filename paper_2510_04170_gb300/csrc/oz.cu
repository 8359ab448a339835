// FP64-accurate matrix products on the bf16 tensor cores (tcgen05), for the
// dense contractions of the preconditioner: the sketch B = S_k J and the QR
// trailing update (Sec. 4.1).
//
// Splitting (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012):
// every row i of A (over K) is scaled by 2^-e_i with max_k |A_ik| < 2^e_i and
// written as digits  A_ik = 2^e_i sum_p a_p(i,k) 2^(-beta p)  with integers
// |a_1| <= 2^beta, |a_p| <= 2^(beta-1) (nearest rounding, beta = 7), each exact
// in bfloat16; B likewise per column.  Then
//     (A B)_ij = 2^(e_i + f_j) sum_l 2^(-beta l) L_l(i,j),
//     L_l = sum over digit pairs with p + q = l of a_p b_q,
// and every L_l of the leading levels accumulated over a K-chunk of 512 is an
// integer below 2^24, so its FP32 tensor-core accumulation is exact.  Per
// chunk the four leading levels combine exactly into the int64
// L_0 2^21 + L_1 2^14 + L_2 2^7 + L_3 and the four trailing ones into
// L_4 2^21 + L_5 2^14 + L_6 2^7 + L_7 (their accumulators may pass 2^24 and
// round there, ~2^-49 of the leading term's unit at level 7), both summed over
// chunks in int64; at the end the 128-bit fixed-point value is rounded once
// to FP64 with integer operations, so the epilogue issues one FP64
// instruction per element (the C update).  Pairs with p + q > Lmax are
// dropped (their weight is below 2^(-beta (Lmax+1)) relative to
// max|A_i.| max|B_.j|).
//
// Kernel layout: persistent, one CTA per SM looping over 128 x 64 output
// tiles, 18 warps.
//   warp 0  producer: cp.async.bulk of pre-tiled digit tiles (16 KB A, 8 KB B)
//           into shared memory, completion on mbarriers (expect_tx)
//   warp 1  owns the 512-column TMEM allocation; lane 0 issues tcgen05.mma
//           (kind::f16, bf16 x bf16 -> f32, M=128, N=64 w, K=16), one MMA for
//           w digit pairs that share an A digit, into the TMEM accumulators
//           of their levels (64 columns each), and commits to mbarriers
//   warps 2-17 epilogue: tcgen05.ld the levels of each chunk, combine them
//           into two int64 running sums per element (four warps per TMEM
//           lane quarter, 16 columns each), then round once to FP64, scale
//           and write (or subtract from) C; C is prefetched into L2 at the
//           start of the tile and read-modify-written four columns at a time
// Digit tiles are K-major with 128-byte rows in the 128B-swizzle pattern so a
// tile is one contiguous bulk copy and the UMMA shared-memory descriptor reads
// it directly.  Every wait is bounded; on timeout an error word is set, the
// CTA drains its copies (bounded), frees TMEM and exits.
#include <stdint.h>

#include <algorithm>

#include "rfm_internal.cuh"

namespace {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int ATILE = BM * BK * 2;  // 16384 bytes
constexpr int BTILE = BN * BK * 2;  // 8192 bytes
constexpr int MAXD = 8;             // digits per operand
constexpr int ASTAGES = 6;
constexpr int EPI_WARPS = 16;       // four warps per TMEM lane quarter, 16 columns each
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);
constexpr int EPI_GRP = 4;          // C elements loaded per round trip in the final update
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int KCHUNK = 8;           // k-tiles per exact chunk (8 * 64 = 512)
constexpr int BETA = 7;
constexpr unsigned long long kWaitNs = 2000000000ull;  // give up after 2 s

__device__ __forceinline__ int swz128(int r, int k) { return rfm_swz128(r, k); }

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for completion of the phase with the given parity: gives up
// after kWaitNs of wall time and records `code` in *err.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* err, unsigned code) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 0 && gtimer() - t0 > kWaitNs) break;
  }
  atomicCAS(err, 0u, code);
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ uint64_t umma_desc(const void* smem_tile) {
  const uint64_t addr = smem_u32(smem_tile);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;          // start address
  d |= (uint64_t)1 << 16;                // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset: 8-row groups 1024 B apart
  d |= (uint64_t)1 << 46;                // descriptor version
  d |= (uint64_t)2 << 61;                // 128-byte swizzle
  return d;
}
// kind::f16 instruction descriptor: bf16 A and B (K-major), f32 accumulate,
// M=128, N = 64 w (w = 1, 2 or 4 consecutive B digit tiles).
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Levels l0 .. l0+3 of 8 columns (levels >= nlev read as 0) combined exactly,
// L_l0 2^(3 BETA) + L_(l0+1) 2^(2 BETA) + L_(l0+2) 2^BETA + L_(l0+3), and
// added to acc[0..7].  (Eighteen warps leave 96 registers a thread, which the
// accumulators largely fill, so one level is loaded per wait.)
__device__ __forceinline__ void tmem_levels4(uint32_t cbase, int l0, int nlev, long long* acc) {
  float v[8];
  long long I[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (l0 + q < nlev) {  // warp-uniform
      tmem_ld8(cbase + (uint32_t)((l0 + q) * BN), v);
#pragma unroll
      for (int i = 0; i < 8; ++i) I[i] = (q == 0 ? 0 : I[i] << BETA) + (long long)__float2int_rn(v[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) I[i] = q == 0 ? 0 : I[i] << BETA;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] += I[i];
}

// (ah 2^28 + al) 2^k rounded to the nearest double (ties to even) with integer
// operations only: the 128-bit two's-complement sum, its leading bit, a 53-bit
// mantissa with round and sticky bits, and the exponent field; ldexp of the
// rounded mantissa where the result leaves the normal range.  |ah| < 2^63
// keeps the leading bit below 2^91, so every shift below stays under 64.
__device__ __forceinline__ double fix_to_double(long long ah, long long al, int k) {
  long long h = ah >> 36;
  const unsigned long long l0 = (unsigned long long)ah << 28;
  const unsigned long long l = l0 + (unsigned long long)al;
  h += (al >> 63) + (l < l0 ? 1 : 0);
  const bool neg = h < 0;
  unsigned long long H = (unsigned long long)h, L = l;
  if (neg) {
    L = ~L + 1ull;
    H = ~H + (L == 0 ? 1ull : 0ull);
  }
  if ((H | L) == 0) return 0.0;
  int msb = H ? 127 - __clzll((long long)H) : 63 - __clzll((long long)L);
  const int sh = msb - 52;
  unsigned long long mant;
  bool up = false;
  if (sh <= 0) {
    mant = L << (-sh);
  } else {
    mant = (L >> sh) | (H << (64 - sh));
    const unsigned long long rbit = (L >> (sh - 1)) & 1ull;
    const bool sticky = (L & ((1ull << (sh - 1)) - 1ull)) != 0;
    up = rbit && (sticky || (mant & 1ull));
  }
  if (up) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++msb;
    }
  }
  const int e = msb + k + 1023;
  if (e > 0 && e < 2047)
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)e << 52) |
                                            (mant & ((1ull << 52) - 1ull))));
  const double mv = (double)mant;  // exact: mant < 2^53
  return ldexp(neg ? -mv : mv, msb - 52 + k);
}

// ---------------------------------------------------------------- GEMM kernel
struct OzArgs {
  const uint16_t* A;  // digit tiles [pA][mtiles][ktiles][ATILE/2]
  const uint16_t* B;  // digit tiles [pB][ntiles][ktiles][BTILE/2]
  int pA, pB, Lmax;   // digits; keep pairs with p + q <= Lmax (p, q from 1)
  int mtiles, ntiles, ktiles;
  const int* ea;      // per row of A: exponent e_i
  const int* eb;      // per column of B: exponent f_j
  double* C;          // column-major, C[i + j * ldc]
  long long ldc, M, N;
  int mode;           // 0: C = AB, 1: C -= AB
  unsigned* err;
  // split K (mode 0): tile t covers the chunks [kz cps, (kz+1) cps) of its
  // output tile, kz = t mod ksplit, and writes its FP64 partial to
  // part[kz][i + j M] (summed in order by k_split_sum)
  int ksplit, cps;
  double* part;
};

// Tile order: groups of TGM M-tiles, N-tiles swept inside a group with the
// group's M-tiles fastest, so the CTAs in flight share a few A tiles (the
// group's, kept in L2) instead of each N-tile re-reading all of A.
constexpr int TGM = 16;
__device__ __forceinline__ void tile_coords(int t, const OzArgs& g, int& mt, int& nt, int& kz) {
  kz = t % g.ksplit;
  t /= g.ksplit;
  const int per = TGM * g.ntiles;
  const int grp = t / per, in = t - grp * per;
  const int gsz = min(TGM, g.mtiles - grp * TGM);
  mt = grp * TGM + in % gsz;
  nt = in / gsz;
}

struct __align__(8) OzBars {
  uint64_t a_full[ASTAGES], a_empty[ASTAGES], b_full[2], b_empty[2], acc_full, acc_empty, fin;
  uint32_t tmem_base;
};

__global__ void __launch_bounds__(NTHREADS, 1) k_oz_gemm(OzArgs g) {
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* abuf = smem;                          // ASTAGES * ATILE
  unsigned char* bbuf = abuf + ASTAGES * ATILE;        // 2 * MAXD * BTILE
  OzBars* bars = reinterpret_cast<OzBars*>(bbuf + 2 * MAXD * BTILE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nlev = min(g.Lmax - 1, g.pA + g.pB - 1);
  const int nchunks = (g.ktiles + KCHUNK - 1) / KCHUNK;
  const int ntiles_total = g.mtiles * g.ntiles * g.ksplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ASTAGES; ++s) {
      mbar_init(&bars->a_full[s], 1);
      mbar_init(&bars->a_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars->b_full[b], 1);
      mbar_init(&bars->b_empty[b], 1);
    }
    mbar_init(&bars->acc_full, 1);
    mbar_init(&bars->acc_empty, EPI_WARPS);
    mbar_init(&bars->fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  // Persistent: tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (tile_coords).
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer
      unsigned aidx = 0, kglob = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles_total && ok; t += gridDim.x) {
        int mt, nt, kz;
        tile_coords(t, g, mt, nt, kz);
        const int kt1 = min(g.ktiles, (kz + 1) * g.cps * KCHUNK);
        for (int kt = kz * g.cps * KCHUNK; kt < kt1 && ok; ++kt) {
          const int b = kglob & 1;
          const unsigned use_b = kglob >> 1;
          if (use_b > 0) ok = mbar_wait(&bars->b_empty[b], (use_b - 1) & 1, g.err, 2);
          if (!ok) break;
          mbar_expect_tx(&bars->b_full[b], (unsigned)(g.pB * BTILE));
          ++kglob;
          for (int q = 0; q < g.pB; ++q) {
            const uint16_t* src = g.B + (((size_t)q * g.ntiles + nt) * g.ktiles + kt) * (BTILE / 2);
            bulk_g2s(bbuf + (size_t)(b * MAXD + q) * BTILE, src, BTILE, &bars->b_full[b]);
          }
          for (int p = 0; p < g.pA && ok; ++p) {
            const int s = aidx % ASTAGES;
            const unsigned use = aidx / ASTAGES;
            if (use > 0) ok = mbar_wait(&bars->a_empty[s], (use - 1) & 1, g.err, 3);
            if (!ok) break;
            mbar_expect_tx(&bars->a_full[s], (unsigned)ATILE);
            const uint16_t* src = g.A + (((size_t)p * g.mtiles + mt) * g.ktiles + kt) * (ATILE / 2);
            bulk_g2s(abuf + (size_t)s * ATILE, src, ATILE, &bars->a_full[s]);
            ++aidx;
          }
        }
      }
      // drain: no copy may still be writing shared memory at exit
      for (unsigned t = (aidx > ASTAGES ? aidx - ASTAGES : 0); t < aidx; ++t)
        mbar_wait(&bars->a_full[t % ASTAGES], (t / ASTAGES) & 1, g.err, 4);
      for (unsigned k = (kglob > 2 ? kglob - 2 : 0); k < kglob; ++k)
        mbar_wait(&bars->b_full[k & 1], (k >> 1) & 1, g.err, 5);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      unsigned aidx = 0, kglob = 0, cglob = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles_total && ok; t += gridDim.x) {
        const int kz = t % g.ksplit;
        const int c1 = min(nchunks, (kz + 1) * g.cps);
        for (int c = kz * g.cps; c < c1 && ok; ++c) {
          if (cglob > 0) {
            ok = mbar_wait(&bars->acc_empty, (cglob - 1) & 1, g.err, 6);
            tc_fence_after();
            if (!ok) break;
          }
          unsigned initmask = 0;
          const int kend = min(g.ktiles, (c + 1) * KCHUNK);
          for (int kt = c * KCHUNK; kt < kend && ok; ++kt) {
            const int b = kglob & 1;
            ok = mbar_wait(&bars->b_full[b], (kglob >> 1) & 1, g.err, 7);
            if (!ok) break;
            for (int p = 0; p < g.pA && ok; ++p) {
              const int s = aidx % ASTAGES;
              ok = mbar_wait(&bars->a_full[s], (aidx / ASTAGES) & 1, g.err, 8);
              if (!ok) break;
              tc_fence_after();
              const uint64_t ad = umma_desc(abuf + (size_t)s * ATILE);
              // Pairs (p, q) with p + q + 2 <= Lmax.  The B digit tiles q, q+1, ...
              // are consecutive in shared memory and their levels p+q, p+q+1, ...
              // are consecutive 64-column TMEM accumulators, so w of them form one
              // MMA with N = 64 w: one read of the A tile serves w pairs.  Each
              // level receives its pairs in the same order as one MMA per pair.
              // A group's levels are all fresh (first write) or all started.
              const int qmax = min(g.pB - 1, g.Lmax - 2 - p);
              for (int q = 0; q <= qmax;) {
                const int l = p + q;
                int w = 4;
                while (w > 1) {
                  const unsigned m = ((1u << w) - 1u) << l;
                  const unsigned fresh = ~initmask & m;
                  if (q + w - 1 <= qmax && (fresh == 0u || fresh == m)) break;
                  w >>= 1;
                }
                const uint64_t bd = umma_desc(bbuf + (size_t)(b * MAXD + q) * BTILE);
                const uint32_t started = (initmask >> l) & 1u;
                const uint32_t idesc = idesc_n(BN * w);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  umma_bf16(tmem + (uint32_t)(l * BN), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                            (started || kk > 0) ? 1u : 0u);
                initmask |= ((1u << w) - 1u) << l;
                q += w;
              }
              umma_commit(&bars->a_empty[s]);
              ++aidx;
            }
            umma_commit(&bars->b_empty[b]);
            ++kglob;
          }
          umma_commit(&bars->acc_full);
          ++cglob;
        }
      }
      // every MMA this thread issued has completed once `fin` fires
      umma_commit(&bars->fin);
      mbar_wait(&bars->fin, 0, g.err, 10);
    }
  } else {
    // ---------------- epilogue (warps 2..9): TMEM lane quarter = warp % 4,
    // column slice = (warp - 2) / 4
    const int quarter = warp & 3;
    const int col0 = ((warp - 2) >> 2) * EPI_COLS;
    const int row = quarter * 32 + lane;
    const uint32_t tlane = (uint32_t)(quarter * 32) << 16;
    unsigned cglob = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles_total && alive; t += gridDim.x) {
      int mt, nt, kz;
      tile_coords(t, g, mt, nt, kz);
      if (g.mode != 0) {  // C is read in the final update: start bringing it into L2 now
        const long long gi = (long long)mt * BM + row;
        if (gi < g.M)
#pragma unroll 4
          for (int j = 0; j < EPI_COLS; ++j) {
            const long long gj = (long long)nt * BN + col0 + j;
            if (gj < g.N) asm volatile("prefetch.global.L2 [%0];" ::"l"(g.C + gi + gj * g.ldc));
          }
      }
      long long ai[EPI_COLS];  // levels 0-3, in units of level 3
      long long al[EPI_COLS];  // levels 4-7, in units of level 7
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) {
        ai[j] = 0;
        al[j] = 0;
      }
      const int c1 = min(nchunks, (kz + 1) * g.cps);
      for (int c = kz * g.cps; c < c1; ++c) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars->acc_full, cglob & 1, g.err, 9));
        tc_fence_after();
        if (!ok) {
          alive = false;
          break;
        }
#pragma unroll
        for (int grp = 0; grp < EPI_COLS / 8; ++grp) {
          const uint32_t cbase = tmem + tlane + (uint32_t)(col0 + grp * 8);
          // leading levels: exact integers below 2^24 (32-bit conversions),
          // combined exactly in int64
          tmem_levels4(cbase, 0, nlev, ai + grp * 8);
          // remaining levels, combined the same way in int64 (their FP32
          // accumulators may exceed 2^24 and round there, far below the
          // result's last bit; the values stay integers below 2^31)
          if (nlev > 4) tmem_levels4(cbase, 4, nlev, al + grp * 8);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->acc_empty);
        ++cglob;
      }
      if (!alive) break;
      const long long gi = (long long)mt * BM + row;
      if (gi < g.M) {
        const int ei = g.ea[gi];
        // EPI_GRP columns at a time: their exponents and (mode 1) C values are
        // loaded together, so one memory round trip serves EPI_GRP elements
#pragma unroll
        for (int j0 = 0; j0 < EPI_COLS; j0 += EPI_GRP) {
          double cv[EPI_GRP];
          int eb[EPI_GRP];
#pragma unroll
          for (int i = 0; i < EPI_GRP; ++i) {
            const long long gj = (long long)nt * BN + col0 + j0 + i;
            const bool in = gj < g.N;
            eb[i] = in ? __ldg(g.eb + gj) : 0;
            cv[i] = (in && g.mode != 0) ? __ldcg(g.C + gi + gj * g.ldc) : 0.0;
          }
#pragma unroll
          for (int i = 0; i < EPI_GRP; ++i) {
            const long long gj = (long long)nt * BN + col0 + j0 + i;
            if (gj < g.N) {
              // value = 2^(e+f-9 BETA) (ai 2^(4 BETA) + al), one rounding to FP64
              const double val = fix_to_double(ai[j0 + i], al[j0 + i], ei + eb[i] - 9 * BETA);
              if (g.ksplit > 1) g.part[(size_t)kz * g.M * g.N + gi + gj * g.M] = val;
              else g.C[gi + gj * g.ldc] = g.mode == 0 ? val : cv[i] - val;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- slicing
// Accessors give X(i, k) for row i (the M or N index) and reduction index k.
struct AccStrided {  // X(i, k) = base[i * si + k * sk]
  const double* base;
  long long si, sk;
  __device__ double operator()(long long i, long long k) const { return base[i * si + k * sk]; }
};
struct AccHouseVt {  // row i = Householder vector i of the panel at j0, k = row offset from j0
  const double* A;
  long long lda, j0;
  __device__ double operator()(long long i, long long k) const {
    if (k < i) return 0.0;
    if (k == i) return 1.0;
    return A[(size_t)(j0 + i) * lda + j0 + k];
  }
};
struct AccHouseV {  // row i = matrix row j0 + i, k = panel column
  const double* A;
  long long lda, j0;
  __device__ double operator()(long long i, long long k) const {
    if (i < k) return 0.0;
    if (i == k) return 1.0;
    return A[(size_t)(j0 + k) * lda + j0 + i];
  }
};

struct AccJBlock {  // row j = column j of a Jacobian column block, k = k-th row touching the block
  const double* Jp;
  const double* Js;
  const int* rows;
  long long m_int;
  int W;
  __device__ double operator()(long long j, long long k) const {
    const unsigned ent = (unsigned)rows[k];
    const long long r = ent & 0x7fffffffu;
    const double* row = (ent >> 31) ? Js + (size_t)(r - m_int) * W : Jp + (size_t)r * W;
    return row[j];
  }
};

// e[i] = exponent with max_k |X(i,k)| < 2^e[i] (0 for a zero row), from the
// largest biased exponent field of the row (integer work only).  One warp per row.
template <class Acc>
__global__ void k_rowexp(Acc X, long long R, long long K, int* __restrict__ e) {
  const int lane = threadIdx.x & 31;
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < R;
       i += (long long)gridDim.x * (blockDim.x >> 5)) {
    unsigned mx = 0;
    bool nz = false;
    long long k = lane;
    for (; k + 96 < K; k += 128) {  // four independent loads in flight per lane
      const unsigned long long b0 = (unsigned long long)__double_as_longlong(X(i, k));
      const unsigned long long b1 = (unsigned long long)__double_as_longlong(X(i, k + 32));
      const unsigned long long b2 = (unsigned long long)__double_as_longlong(X(i, k + 64));
      const unsigned long long b3 = (unsigned long long)__double_as_longlong(X(i, k + 96));
      mx = max(max(mx, (unsigned)((b0 >> 52) & 0x7FF)), (unsigned)((b1 >> 52) & 0x7FF));
      mx = max(max(mx, (unsigned)((b2 >> 52) & 0x7FF)), (unsigned)((b3 >> 52) & 0x7FF));
      nz |= ((b0 | b1 | b2 | b3) << 1) != 0;
    }
    for (; k < K; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(X(i, k));
      mx = max(mx, (unsigned)((b >> 52) & 0x7FF));
      nz |= (b << 1) != 0;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) e[i] = nz ? (mx == 0 ? -1022 : (int)mx - 1022) : 0;
  }
}

// Balanced base-2^7 digits of x 2^-e (|x| < 2^e): V = round(x 2^(7 ndig - e))
// as an integer built from the mantissa bits; the ndig-1 low digits lie in
// [-64, 63] and d_1 takes the rest (|d_1| <= 128).  Adding the bias
// 64 (1 + 2^7 + ... + 2^(7(ndig-2))) to V turns every low digit into the
// plain 7-bit field (digit + 64) of U = V + bias, so each digit is one field
// extract, and the top digit is U >> 7(ndig-1) (the same digits as peeling
// V from its low end with nearest remainders).
__device__ __forceinline__ long long biased_of(double x, int e, int ndig) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & ((1ull << 52) - 1);
  if (E != 0) m |= 1ull << 52;
  const int sh = (E == 0 ? 1 : E) - 1075 - e + 7 * ndig;
  long long V;
  if (sh >= 0) V = (long long)(m << sh);
  else if (sh > -63) V = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else V = 0;
  if (b >> 63) V = -V;
  // bias = 64 (128^(ndig-1) - 1) / 127: ndig-1 seven-bit fields of value 64
  const long long bias = (long long)(0x0001020408102040ull >> (7 * (MAXD - ndig)));
  return V + bias;
}

// bf16 bits of digit dd (0 = the top one) of the biased integer U: the top
// digit is U >> 7(ndig-1) (|d_1| <= 128), digit dd >= 1 the 7-bit field
// 7(ndig-1-dd) of U minus 64; small integers, exact in bf16.
__device__ __forceinline__ uint32_t digit_bits(long long U, int dd, int ndig) {
  float v;
  if (dd == 0) {
    v = (float)(int)(U >> (7 * (ndig - 1)));
  } else {
    const int bit = 7 * (ndig - 1 - dd);
    const unsigned lo = (unsigned)U, hi = (unsigned)((unsigned long long)U >> 32);
    const unsigned f = (bit < 32 ? __funnelshift_r(lo, hi, bit) : hi >> (bit - 32)) & 127u;
    // exact float of f - 64: 2^23 + f minus (2^23 + 64)
    v = __int_as_float((int)(0x4B000000u | f)) - 8388672.0f;
  }
  return __float_as_uint(v) >> 16;
}

// Digit tiles: out[d][rtile][ktile][tile], tile = TR rows x 64 k in the 128B
// swizzle.  One thread per 16-byte chunk (row r, 8 consecutive k): it reads 8
// values and writes one 16-byte chunk per digit plane.
// The tiles go to row-tile positions rt0 .. rt0 + rtiles - 1 of digit planes
// that hold plane_rtiles row tiles each (several slices can share one operand).
template <class Acc, int TR>
__global__ void k_digits(Acc X, long long R, long long K, const int* __restrict__ e, int ndig, long long rtiles,
                         long long ktiles, uint16_t* __restrict__ out, long long plane_rtiles, long long rt0) {
  const long long total = rtiles * TR * ktiles * 8;
  const size_t plane = (size_t)plane_rtiles * ktiles * TR * 64;  // elements per digit plane
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c8 = (int)(t & 7);
    long long rest = t >> 3;
    const int r = (int)(rest % TR);
    rest /= TR;
    const long long kt = rest % ktiles;
    const long long rt = rest / ktiles;
    const long long i = rt * TR + r, k0 = kt * 64 + c8 * 8;
    // the 8 values' biased integers first, then one digit plane at a time
    // (few registers: no digits are held for all planes at once)
    long long U[8];
    const int ei = i < R ? e[i] : 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) U[j] = biased_of((i < R && k0 + j < K) ? X(i, k0 + j) : 0.0, ei, ndig);
    const size_t base = ((size_t)(rt + rt0) * ktiles + kt) * (TR * 64) + (size_t)(swz128(r, c8 * 8) >> 1);
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
      if (d < ndig)
        *reinterpret_cast<uint4*>(out + (size_t)d * plane + base) =
            make_uint4(digit_bits(U[0], d, ndig) | (digit_bits(U[1], d, ndig) << 16),
                       digit_bits(U[2], d, ndig) | (digit_bits(U[3], d, ndig) << 16),
                       digit_bits(U[4], d, ndig) | (digit_bits(U[5], d, ndig) << 16),
                       digit_bits(U[6], d, ndig) | (digit_bits(U[7], d, ndig) << 16));
  }
}


size_t oz_smem_bytes() { return (size_t)ASTAGES * ATILE + 2 * MAXD * BTILE + sizeof(OzBars) + 1024; }

}  // namespace

// ---------------------------------------------------------------- host side
long long rfm_oz_digit_bytes(long long rows, long long K, int ndig, int tile_rows) {
  const long long rt = (rows + tile_rows - 1) / tile_rows, kt = (K + 63) / 64;
  return (long long)ndig * rt * kt * tile_rows * 64 * 2;
}

template <class Acc>
static rfm_status slice(Acc X, long long R, long long K, int ndig, int tile_rows, int* e, uint16_t* out,
                        cudaStream_t st, long long plane_rtiles = 0, long long rt0 = 0) {
  ProfScope ps(PF_OZ_SLICE, st);
  const int g1 = (int)std::min<long long>((R + 7) / 8, 152LL * 32);
  k_rowexp<<<std::max(1, g1), 256, 0, st>>>(X, R, K, e);
  RFM_CHECK_LAUNCH();
  const long long rt = (R + tile_rows - 1) / tile_rows, kt = (K + 63) / 64;
  const long long prt = plane_rtiles > 0 ? plane_rtiles : rt;
  const long long total = rt * tile_rows * kt * 8;
  const int g2 = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
  if (tile_rows == BM)
    k_digits<Acc, BM><<<std::max(1, g2), 256, 0, st>>>(X, R, K, e, ndig, rt, kt, out, prt, rt0);
  else
    k_digits<Acc, BN><<<std::max(1, g2), 256, 0, st>>>(X, R, K, e, ndig, rt, kt, out, prt, rt0);
  RFM_CHECK_LAUNCH();
  return RFM_OK;
}

rfm_status rfm_oz_slice_strided(const double* base, long long si, long long sk, long long R, long long K, int ndig,
                                int tile_rows, int* e, uint16_t* out, cudaStream_t st) {
  return slice(AccStrided{base, si, sk}, R, K, ndig, tile_rows, e, out, st);
}
rfm_status rfm_oz_slice_house_vt(const double* A, long long lda, long long j0, long long nb, long long K, int ndig,
                                 int* e, uint16_t* out, cudaStream_t st) {
  return slice(AccHouseVt{A, lda, j0}, nb, K, ndig, BM, e, out, st);
}
rfm_status rfm_oz_slice_strided_at(const double* base, long long si, long long sk, long long R, long long K, int ndig,
                                   int tile_rows, int* e, uint16_t* out, long long plane_rtiles, long long rt0,
                                   cudaStream_t st) {
  return slice(AccStrided{base, si, sk}, R, K, ndig, tile_rows, e, out, st, plane_rtiles, rt0);
}
rfm_status rfm_oz_slice_house_vt_at(const double* A, long long lda, long long j0, long long nb, long long K, int ndig,
                                    int tile_rows, int* e, uint16_t* out, long long plane_rtiles, long long rt0,
                                    cudaStream_t st) {
  return slice(AccHouseVt{A, lda, j0}, nb, K, ndig, tile_rows, e, out, st, plane_rtiles, rt0);
}
rfm_status rfm_oz_slice_house_v(const double* A, long long lda, long long j0, long long rows, long long nb, int ndig,
                                int* e, uint16_t* out, cudaStream_t st) {
  return slice(AccHouseV{A, lda, j0}, rows, nb, ndig, BM, e, out, st);
}

rfm_status rfm_oz_slice_jblock(const double* Jp, const double* Js, const int* rows, long long K, long long m_int,
                               int W, int ndig, int* e, uint16_t* out, cudaStream_t st) {
  return slice(AccJBlock{Jp, Js, rows, m_int, W}, W, K, ndig, BN, e, out, st);
}

namespace {
// C[i + j ldc] = sum over z = 0 .. Z-1, in that order, of part[z][i + j M]
__global__ void k_split_sum(const double* __restrict__ part, int Z, long long M, long long N, double* __restrict__ C,
                            long long ldc) {
  const long long MN = M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < MN;
       idx += (long long)gridDim.x * blockDim.x) {
    double v = part[idx];
    for (int z = 1; z < Z; ++z) v += part[(size_t)z * MN + idx];
    const long long i = idx % M, j = idx / M;
    C[i + j * ldc] = v;
  }
}
}  // namespace

rfm_status rfm_oz_gemm(const uint16_t* Ad, int pA, const int* ea, const uint16_t* Bd, int pB, const int* eb,
                       long long M, long long N, long long K, int Lmax, double* C, long long ldc, int mode,
                       unsigned* err, cudaStream_t st) {
  return rfm_oz_gemm_part(Ad, pA, ea, Bd, pB, eb, M, N, K, Lmax, C, ldc, mode, err, st, nullptr, 0);
}

rfm_status rfm_oz_gemm_part(const uint16_t* Ad, int pA, const int* ea, const uint16_t* Bd, int pB, const int* eb,
                            long long M, long long N, long long K, int Lmax, double* C, long long ldc, int mode,
                            unsigned* err, cudaStream_t st, double* part, long long part_elems) {
  if (pA < 1 || pB < 1 || pA > MAXD || pB > MAXD || Lmax < 2 || Lmax - 1 > 8) {
    rfm_set_error("oz_gemm: bad digit counts");
    return RFM_EINVAL;
  }
  RFM_CUDA(rfm_smem_attr((const void*)k_oz_gemm, (int)oz_smem_bytes()));  // once per device
  OzArgs a;
  a.A = Ad; a.B = Bd; a.pA = pA; a.pB = pB; a.Lmax = Lmax;
  a.mtiles = (int)((M + BM - 1) / BM);
  a.ntiles = (int)((N + BN - 1) / BN);
  a.ktiles = (int)((K + BK - 1) / BK);
  a.ea = ea; a.eb = eb; a.C = C; a.ldc = ldc; a.M = M; a.N = N; a.mode = mode; a.err = err;
  if (a.ktiles == 0) return RFM_OK;
  ProfScope ps(PF_OZ_GEMM, st);
  {
    int pairs = 0;
    for (int p = 0; p < pA; ++p)
      for (int q = 0; q < pB; ++q)
        if (p + q + 2 <= Lmax) ++pairs;
    rfm_prof_work(PF_OZ_GEMM, 2.0 * pairs * (double)M * (double)N * (double)K);  // bf16 tensor flops
  }
  const int nsm = rfm_num_sms();
  if (nsm == 0) {
    rfm_set_error("oz_gemm: cannot query the device");
    return RFM_ECUDA;
  }
  const long long tiles = (long long)a.mtiles * a.ntiles;
  // Split K when the output tiles leave the last wave of CTAs partly idle
  // (mode 0, a workspace for the partials, at least two 512-deep chunks per
  // split): the split count with the best fill of whole waves, ties to fewer.
  const int nchunks = (a.ktiles + KCHUNK - 1) / KCHUNK;
  a.ksplit = 1;
  a.cps = nchunks;
  a.part = part;
  if (mode == 0 && part && tiles < 4LL * nsm && nchunks >= 4) {
    double best = (double)tiles / (double)(nsm * ((tiles + nsm - 1) / nsm));
    for (int z = 2; z <= 8 && nchunks / z >= 2; ++z) {
      const int cps = (nchunks + z - 1) / z;
      const int zz = (nchunks + cps - 1) / cps;  // no empty split
      if ((long long)zz * M * N > part_elems) break;
      const long long u = tiles * zz;
      const double fill = (double)u / (double)(nsm * ((u + nsm - 1) / nsm));
      if (fill > best + 0.02) {
        best = fill;
        a.ksplit = zz;
        a.cps = cps;
      }
    }
  }
  k_oz_gemm<<<(unsigned)std::min<long long>(tiles * a.ksplit, nsm), NTHREADS, oz_smem_bytes(), st>>>(a);
  RFM_CHECK_LAUNCH();
  if (a.ksplit > 1) {
    const long long MN = M * N;
    k_split_sum<<<(unsigned)std::min<long long>((MN + 255) / 256, 152LL * 16), 256, 0, st>>>(part, a.ksplit, M, N, C,
                                                                                            ldc);
    RFM_CHECK_LAUNCH();
  }
  return RFM_OK;
}

// C (M x N, col-major ldc) = A (M x K, col-major lda) * B (K x N, col-major ldb)
// emulated to FP64 accuracy with `digits` digits per operand.
extern "C" rfm_status rfm_emulated_dgemm(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                         int64_t ldc, int64_t M, int64_t N, int64_t K, int digits,
                                         void* cuda_stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || digits < 1 || digits > MAXD || lda < M || ldb < K || ldc < M) {
    rfm_set_error("rfm_emulated_dgemm: bad argument");
    return RFM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long abytes = rfm_oz_digit_bytes(M, K, digits, BM);
  const long long bbytes = rfm_oz_digit_bytes(N, K, digits, BN);
  char* buf = nullptr;
  const size_t total = (size_t)abytes + bbytes + (size_t)(M + N + 64) * sizeof(int) + 64;
  if (cudaMalloc(&buf, total) != cudaSuccess) {
    rfm_set_error("rfm_emulated_dgemm: allocation failed");
    return RFM_ENOMEM;
  }
  uint16_t* Ad = reinterpret_cast<uint16_t*>(buf);
  uint16_t* Bd = reinterpret_cast<uint16_t*>(buf + abytes);
  int* ea = reinterpret_cast<int*>(buf + abytes + bbytes);
  int* eb = ea + M;
  unsigned* err = reinterpret_cast<unsigned*>(eb + N);
  rfm_status s = RFM_OK;
  if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess) s = RFM_ECUDA;
  // A rows over k: A[i + k*lda];  B columns over k: B[k + j*ldb]
  if (s == RFM_OK) s = rfm_oz_slice_strided(A, 1, lda, M, K, digits, BM, ea, Ad, st);
  if (s == RFM_OK) s = rfm_oz_slice_strided(B, ldb, 1, N, K, digits, BN, eb, Bd, st);
  if (s == RFM_OK) s = rfm_oz_gemm(Ad, digits, ea, Bd, digits, eb, M, N, K, digits + 1, C, ldc, 0, err, st);
  unsigned herr = 0;
  if (s == RFM_OK) {
    if (cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rfm_set_error(std::string("rfm_emulated_dgemm: ") + cudaGetErrorString(cudaGetLastError()));
      s = RFM_ECUDA;
    } else if (herr) {
      rfm_set_error("rfm_emulated_dgemm: a bounded wait timed out (code " + std::to_string(herr) + ")");
      s = RFM_ETIMEOUT;
    }
  }
  cudaFree(buf);
  return s;
}
