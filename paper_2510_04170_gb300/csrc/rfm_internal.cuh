// Internal declarations shared by the CUDA translation units of librfm.
// Hot-path kernels for the random feature method with the IPN / AMIPN solvers
// (arXiv 2510.04170): assembly (Alg. 3), sketch + QR preconditioner (Sec. 4.1),
// LSQR on J R^{-1} and the golden-section line search (Alg. 1, Alg. 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rfm.h"

#define RFM_MAX_FIELDS 2
#define RFM_MAX_WIDTH 2048

// One run of rows that share a point grid (Sec. 5): an interior grid of a
// subdomain, or a face grid on an interface or a boundary face.
struct RowSeg {
  int kind;     // 0 interior, 1 interface, 2 boundary
  int e0, e1;   // subdomain (left / own) and right neighbour (interface only)
  int axis;     // normal axis of a face (-1 interior)
  int sord;     // derivative order across an interface (0: C^0, 1: C^1)
  int field;
  int side;     // boundary side 0 lo, 1 hi
  int q[3];     // points per axis (face grids: along the axes != axis)
  int pad;
  long long row0;
  long long count;
};

struct rfm_problem {
  rfm_problem_desc desc;
  cudaStream_t stream;
  int d, G, M, fields, W, nmaxbp;
  int N[3];
  long long n, m, m_int, m_iface, m_bdy;
  // device tables
  double* X = nullptr;      // breakpoints [3][nmaxbp]
  double* mu = nullptr;     // [G][4]
  double* sig = nullptr;    // [G][4]
  double* feat = nullptr;   // [G*fields*M][4]
  RowSeg* segs = nullptr;
  int nseg = 0;
  bool explicit_rows = false;  // geometry with masked grids: points and row metadata built on the host
  double* pts = nullptr;    // [m][4]
  int4* rmeta = nullptr;    // per row: {kind|field<<4|axis<<8|sord<<12|side<<16, e0, e1, 0}
  double* rhs = nullptr;    // [m] source f (interior) or boundary data g
  // Jacobian (scaled) and residual
  double* Jp = nullptr;     // [m][W]
  double* Js = nullptr;     // [m_iface][W]
  double* lam = nullptr;    // [m]
  double* F = nullptr;      // [m]
  bool have_j = false;
  int* colptr = nullptr;    // [G+1] transposed block structure
  int* colrows = nullptr;   // row | (secondary << 31)
  // sketch / QR
  long long s = 0, s_cap = 0;
  double* B = nullptr;      // s x n column-major (R in its upper triangle after QR)
  uint16_t* Sg = nullptr;   // Gaussian sketch, bf16 bits, [m][s]
  long long sg_cap = 0;
  int* hbuck = nullptr;     // count sketch buckets [m]
  double* hsign = nullptr;  // [m]
  int* bptr = nullptr;      // [s+1]
  int* brows = nullptr;     // [m]
  long long bptr_cap = 0;
  double* R = nullptr;      // points into B (ld = ldr) or into Rown
  double* Rown = nullptr;
  long long ldr = 0;
  bool have_r = false;
  int rank_flag = 0;
  // tensor-core (emulated FP64) paths
  int precision = 0;        // 0 FP64, 1 + tensor-core sketch, 2 + tensor-core QR update
  std::vector<int> colptr_h;
  uint16_t* sdig = nullptr;  // S digit tiles of all column blocks
  long long sdig_bytes = 0;
  uint16_t* jdig = nullptr;  // J digit tiles of one column block
  long long jdig_bytes = 0;
  int* oz_e = nullptr;       // exponents: [s] for S (all 3) then [W] for J
  long long oz_e_cap = 0;
  long long* oz_toff = nullptr;
  void* qr_emu = nullptr;
  long long qr_emu_bytes = 0;
  // scratch
  double* work = nullptr;   // general vectors
  long long work_cap = 0;
  double* red = nullptr;    // reduction partials
  unsigned int* sync = nullptr;  // counters / flags / error words
  double* hostbuf = nullptr;     // pinned host scalars
  // LSQR iterations run from device-resident scalars; while they run, the
  // iteration's kernels return at once once *skip (the convergence flag) is set
  const int* skip = nullptr;
  void* lsqr_graph = nullptr;    // cudaGraphExec_t of one chunk of iterations
  cudaStream_t cap_stream = nullptr;  // private stream the chunk is captured on
  unsigned long long lsqr_graph_key = 0;
  long long lsqr_graph_launches = 0;  // kernels per chunk (launch accounting)
  bool lsqr_eager = false;        // graph capture failed once: replay the chunk's kernels eagerly
  int qr_panel_cap = 0;           // most CTAs per panel factorisation (0: one per SM)
  double* trsv_acc = nullptr;     // [ceil(n/64)][64] partial sums of the triangular solve's helpers
  double* dinv = nullptr;         // [ceil(n/64)][64 x 64] inverses of R's diagonal blocks (column-major)
  const double* dinv_of = nullptr;  // the R that dinv was computed from (nullptr: stale)
  // per-problem QR scratch (FP64 panel buffers)
  double* qr_scratch = nullptr;
  long long qr_scratch_len = 0;
};

// ---- error handling --------------------------------------------------------
void rfm_set_error(const std::string& msg);
#define RFM_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      rfm_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
      return RFM_ECUDA;                                                         \
    }                                                                           \
  } while (0)
void rfm_count_launch();
void rfm_count_launches(long long k);  // kernels run by one replay of a captured graph
void rfm_count_pause(bool paused);     // this thread's launches are being captured, not run
long long rfm_launches_now();
bool rfm_prof_active(unsigned int families);  // are any of these families (bit masks) being timed?
int rfm_num_sms();  // SMs of the current device (0 if it cannot be queried), cached per device
// Sets a kernel's dynamic shared-memory limit once per (device, kernel); the
// attribute belongs to the current device's context.
cudaError_t rfm_smem_attr(const void* func, int bytes);
#define RFM_CHECK_LAUNCH()                                                      \
  do {                                                                          \
    rfm_count_launch();                                                         \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess) {                                                    \
      rfm_set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));   \
      return RFM_ECUDA;                                                         \
    }                                                                           \
  } while (0)
#define RFM_TRY(x)                 \
  do {                             \
    rfm_status s_ = (x);           \
    if (s_ != RFM_OK) return s_;   \
  } while (0)

// ---- optional per-kernel-family timing (prof.cu) -----------------------------
enum {
  PF_ASSEMBLE = 0, PF_RESIDUAL, PF_SKETCH_COUNT, PF_SKETCH_GEN, PF_SKETCH_GEMM, PF_QR_PANEL, PF_QR_VTA,
  PF_QR_UPDATE, PF_TRSV, PF_JMV, PF_JTMV, PF_LS_PRE, PF_LS_EVAL, PF_VECTOR, PF_EVAL, PF_OZ_GEMM, PF_OZ_SLICE,
  RFM_PROF_FAMILIES
};
void* rfm_prof_begin(int fam, cudaStream_t st);
// Adds `units` of algorithmic work (bytes or flops, per family) when family
// `fam` is being profiled.
void rfm_prof_work(int fam, double units);
void rfm_prof_end(void* h, cudaStream_t st);
struct ProfScope {
  void* h;
  cudaStream_t st;
  ProfScope(int fam, cudaStream_t s) : h(rfm_prof_begin(fam, s)), st(s) {}
  ~ProfScope() { rfm_prof_end(h, st); }
};

// ---- launchers implemented in the .cu files -----------------------------------
rfm_status rfm_launch_setup(rfm_problem* p);                        // features, points, rhs
rfm_status rfm_launch_assemble(rfm_problem* p, const double* c, double cscale, bool want_j,
                               const double* lam_in, double* Fout);
rfm_status rfm_launch_ls_precompute(rfm_problem* p, const double* c, const double* dvec, double* P0,
                                    double* P1, double* U, double* V);
rfm_status rfm_launch_ls_eval(rfm_problem* p, const double* P0, const double* P1, const double* U,
                              const double* V, double alpha, double* out_dev);
rfm_status rfm_launch_eval(const rfm_problem* p, const double* c, const double* pts, long long npts,
                           double* u);
rfm_status rfm_launch_phi_values(const rfm_problem* p, const double* pts, long long npts, float scale, float* Phi);
rfm_status rfm_launch_jmv(rfm_problem* p, const double* x, double* y);
rfm_status rfm_launch_jtmv(rfm_problem* p, const double* x, double* y);
rfm_status rfm_launch_trsv(rfm_problem* p, int trans, const double* b, double* x);
rfm_status rfm_trsv_prepare(rfm_problem* p);  // inverts R's diagonal blocks (after every change of R)
rfm_status rfm_launch_count_sketch(rfm_problem* p, long long s, int kJ);
rfm_status rfm_launch_gauss_sketch(rfm_problem* p, long long s, int kJ);
rfm_status rfm_launch_gauss_sketch_tc(rfm_problem* p, long long s, int kJ);
rfm_status rfm_householder_emulated(double* A, long long s, long long n, long long lda, cudaStream_t st,
                                    double* scratch, long long scratch_len, unsigned int* sync, void* emu,
                                    long long emu_bytes, int* rank_flag_host, int panel_cap = 0,
                                    long long ncols = -1);
long long rfm_householder_emulated_bytes(long long s, long long n);
rfm_status rfm_oz_slice_jblock(const double* Jp, const double* Js, const int* rows, long long K, long long m_int,
                               int W, int ndig, int* e, uint16_t* out, cudaStream_t st);
rfm_status rfm_oz_gemm(const uint16_t* Ad, int pA, const int* ea, const uint16_t* Bd, int pB, const int* eb,
                       long long M, long long N, long long K, int Lmax, double* C, long long ldc, int mode,
                       unsigned* err, cudaStream_t st);
// rfm_oz_gemm that may split K over several CTAs per output tile (mode 0,
// when the tiles alone leave the last wave of CTAs partly idle): the partial
// products go to part (part_elems doubles; up to 8 M N) and are summed in a
// fixed order into C.  part = nullptr never splits.
rfm_status rfm_oz_gemm_part(const uint16_t* Ad, int pA, const int* ea, const uint16_t* Bd, int pB, const int* eb,
                            long long M, long long N, long long K, int Lmax, double* C, long long ldc, int mode,
                            unsigned* err, cudaStream_t st, double* part, long long part_elems);
rfm_status rfm_oz_slice_strided(const double* base, long long si, long long sk, long long R, long long K, int ndig,
                                int tile_rows, int* e, uint16_t* out, cudaStream_t st);
long long rfm_oz_digit_bytes(long long rows, long long K, int ndig, int tile_rows);
rfm_status rfm_householder_inplace(double* A, long long s, long long n, long long lda,
                                   cudaStream_t st, double* scratch, long long scratch_len,
                                   unsigned int* sync, int* rank_flag_host, int panel_cap = 0,
                                   long long ncols = -1);
// panel_cap: most CTAs of one panel factorisation (0: one per SM); ncols >= 0
// stops after the blocks that cover the first ncols columns (timing probes).
long long rfm_householder_scratch(long long s, long long n);
// deterministic norms / dots: result written to out_dev[0]
rfm_status rfm_norm2(cudaStream_t st, const double* x, long long n, double* partial, double* out_dev);
rfm_status rfm_dot(cudaStream_t st, const double* x, const double* y, long long n, double* partial,
                   double* out_dev);

#define RFM_SYNC_WORDS 4096
// layout of p->sync
#define SYNC_ERR 0
#define SYNC_TICKET 8
#define SYNC_EPOCH 9
#define SYNC_LSQR_DONE 10
#define SYNC_WAITLIM 11
#define SYNC_BAR 16
#define SYNC_FLAGS 64

// ---- device helpers ------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait until *flag == want.  Polls without sleeping first (a sleep's
// granularity is far coarser than the expected wait), then backs off; gives up
// after a poll limit and records the failure in *err, so a missing producer
// never hangs the GPU.  `err` is word SYNC_ERR of a sync block whose word
// SYNC_WAITLIM holds the limit: 0 the default of 2^22 polls (well under a
// second of sleeping), a positive count that many polls, a negative value
// "give up at once" (a host-side test setting, rfm_set_wait_limit).
// `pause_ns` > 0 sleeps that long between polls from the start (many waiters
// on one line leave the L2 slice free for the write they wait for).
__device__ __forceinline__ bool wait_flag(const unsigned int* flag, unsigned int want,
                                          unsigned int* err, unsigned int pause_ns = 0) {
  const int lim = (int)__ldcg(err + (SYNC_WAITLIM - SYNC_ERR));
  if (lim < 0) {
    atomicExch(err, 1u);
    return false;
  }
  const unsigned int limit = lim == 0 ? (1u << 22) : (unsigned int)lim;
  unsigned int spins = 0;
  while (ld_acquire(flag) != want) {
    if (++spins > limit) {
      atomicExch(err, 1u);
      return false;
    }
    if (pause_ns) __nanosleep(pause_ns);
    else if (spins > (1u << 16)) __nanosleep(128);
  }
  return true;
}
#endif

// Byte offset of element (row r, column k < 64) of a K-major tile with 128-byte
// rows in the 128-byte swizzle pattern (16-byte chunk c of row r stored at
// chunk c ^ (r mod 8); 8-row groups 1024 bytes apart), 2-byte elements.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int rfm_swz128(int r, int k) {
  const int chunk = k >> 3;
  return (r >> 3) * 1024 + (r & 7) * 128 + (((chunk ^ (r & 7)) & 7) << 4) + ((k & 7) << 1);
}


