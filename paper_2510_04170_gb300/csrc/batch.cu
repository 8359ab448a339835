// Batched solves: many independent RFM problems (instances of one PDE family
// with different subdomain grids, features per subdomain and coefficients)
// solved concurrently on one GPU.
//
// Instances are independent units, so the batch needs no exchange between
// them: a pool of host workers, one CUDA stream each, takes instances from a
// queue ordered by decreasing cost (largest n^2 s first, so the long solves
// start first and the short ones fill the tail), and each solve keeps its own
// workspace, QR scratch and captured LSQR graph.  Small instances cannot fill
// 152 SMs alone (their panel factorisations use rows/64 CTAs, their matvecs a
// few hundred); running several at once fills the GPU.  After its solve an
// instance releases its sketch/QR buffers, so device memory holds only the
// workspaces of the instances in flight.
//
// The autotuner picks, per sketch size (s, n), the QR configuration: FP64
// panels with the FP64 trailing update, or the tensor-core (emulated FP64)
// trailing update, each with the panel factorisation spread over at most 16,
// 32, 64 or all SMs (fewer CTAs make the two grid barriers per column cheaper,
// more CTAs share the panel's rows; shared memory bounds the rows per CTA).
// Each candidate factors the first 128 columns of a seeded random s x n
// matrix (updating all n columns), timed with CUDA events after one warm-up;
// the fastest is cached per (s, n) for the process.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rfm_internal.cuh"

namespace {

// uniform [-1, 1) from a 64-bit mix of the index (SplitMix64 finaliser)
__global__ void k_fill_probe(double* __restrict__ A, long long count, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    A[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

constexpr int kCaps = 4;              // panel CTA caps tried: 16, 32, 64, all SMs
constexpr int kCands = 2 * kCaps;     // x {FP64 update, tensor-core update}

struct QrChoice {
  int precision = 0;
  int panel_cap = 0;
  double ms[kCands] = {};
};

std::mutex g_tune_mu;
std::map<std::pair<long long, long long>, QrChoice> g_tune;

rfm_status probe_qr(long long s, long long n, cudaStream_t st, QrChoice* out) {
  const int nsm = rfm_num_sms();
  if (nsm == 0) {
    rfm_set_error("autotune: cannot query the device");
    return RFM_ECUDA;
  }
  const long long qs = rfm_householder_scratch(s, n);
  const long long eb = rfm_householder_emulated_bytes(s, n);
  double *A = nullptr, *scratch = nullptr;
  unsigned int* sync = nullptr;
  void* emu = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rfm_status r = RFM_OK;
  if (cudaMalloc((void**)&A, (size_t)s * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&scratch, (size_t)qs * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&sync, RFM_SYNC_WORDS * sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&emu, (size_t)eb) != cudaSuccess) {
    rfm_set_error("autotune: allocation failed");
    r = RFM_ENOMEM;
  }
  if (r == RFM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) r = RFM_ECUDA;
  const int caps[kCaps] = {std::min(16, nsm), std::min(32, nsm), std::min(64, nsm), nsm};
  const long long ncols = std::min<long long>(n, 128);
  for (int c = 0; c < kCands && r == RFM_OK; ++c) {
    const int prec = c < kCaps ? 0 : 2, cap = caps[c % kCaps];
    float best = 1e30f;
    for (int rep = 0; rep < 2 && r == RFM_OK; ++rep) {  // first run warms up
      k_fill_probe<<<(unsigned)std::min<long long>((s * n + 255) / 256, 152 * 16), 256, 0, st>>>(A, s * n, 12345ull);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemsetAsync(sync, 0, RFM_SYNC_WORDS * sizeof(unsigned int), st) != cudaSuccess ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        r = RFM_ECUDA;
        break;
      }
      int flag = 0;
      r = prec == 0 ? rfm_householder_inplace(A, s, n, s, st, scratch, qs, sync, &flag, cap, ncols)
                    : rfm_householder_emulated(A, s, n, s, st, scratch, qs, sync, emu, eb, &flag, cap, ncols);
      if (r != RFM_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        r = RFM_ECUDA;
        break;
      }
      if (rep > 0) best = std::min(best, ms);
    }
    out->ms[c] = best;
  }
  if (r == RFM_OK) {
    int arg = 0;
    for (int c = 1; c < kCands; ++c)
      if (out->ms[c] < out->ms[arg]) arg = c;
    out->precision = arg < kCaps ? 0 : 2;
    out->panel_cap = caps[arg % kCaps];
  }
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (A) cudaFree(A);
  if (scratch) cudaFree(scratch);
  if (sync) cudaFree(sync);
  if (emu) cudaFree(emu);
  if (r == RFM_ECUDA) rfm_set_error("autotune: CUDA error");
  return r;
}

rfm_status tuned_qr(long long s, long long n, cudaStream_t st, QrChoice* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);  // one probe at a time; later callers hit the cache
  auto it = g_tune.find({s, n});
  if (it != g_tune.end()) {
    *out = it->second;
    return RFM_OK;
  }
  QrChoice c;
  RFM_TRY(probe_qr(s, n, st, &c));
  g_tune[{s, n}] = c;
  *out = c;
  return RFM_OK;
}

long long sketch_rows_of(const rfm_problem* p, const rfm_solve_opts* o) {
  return o->sketch_rows > 0 ? o->sketch_rows : (long long)ceil(o->gamma * (double)p->n);
}

// Frees the sketch, QR and digit buffers of a finished instance (they are
// re-created on its next solve).
void release_workspace(rfm_problem* p) {
  void** bufs[] = {(void**)&p->B, (void**)&p->Sg, (void**)&p->qr_emu, (void**)&p->qr_scratch, (void**)&p->sdig,
                   (void**)&p->jdig, (void**)&p->Rown};
  for (void** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  p->s_cap = p->sg_cap = 0;
  p->qr_emu_bytes = p->qr_scratch_len = p->sdig_bytes = p->jdig_bytes = 0;
  p->R = nullptr;
  p->have_r = false;
  p->dinv_of = nullptr;
  if (p->lsqr_graph) cudaGraphExecDestroy((cudaGraphExec_t)p->lsqr_graph);
  p->lsqr_graph = nullptr;
  p->lsqr_graph_key = 0;
}

}  // namespace

struct rfm_batch {
  std::vector<rfm_problem*> probs;
  std::vector<cudaStream_t> streams;
  std::vector<QrChoice> choice;  // per instance, filled by the autotuner
};

extern "C" {

rfm_status rfm_autotune_qr(int64_t s, int64_t n, void* cuda_stream, int* precision_out, int* panel_cap_out,
                           double* ms8_out) {
  if (s < n || n <= 0) {
    rfm_set_error("rfm_autotune_qr: need s >= n > 0");
    return RFM_EINVAL;
  }
  QrChoice c;
  RFM_TRY(tuned_qr(s, n, (cudaStream_t)cuda_stream, &c));
  if (precision_out) *precision_out = c.precision;
  if (panel_cap_out) *panel_cap_out = c.panel_cap;
  if (ms8_out)
    for (int i = 0; i < kCands; ++i) ms8_out[i] = c.ms[i];
  return RFM_OK;
}

rfm_status rfm_batch_create(const rfm_problem_desc* descs, int count, int streams, rfm_batch** out) {
  if (!descs || count <= 0 || streams <= 0 || streams > 64 || !out) {
    rfm_set_error("rfm_batch_create: bad argument");
    return RFM_EINVAL;
  }
  rfm_batch* b = new rfm_batch();
  rfm_status r = RFM_OK;
  for (int w = 0; w < std::min(streams, count) && r == RFM_OK; ++w) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      rfm_set_error("rfm_batch_create: stream creation failed");
      r = RFM_ECUDA;
    } else {
      b->streams.push_back(s);
    }
  }
  for (int i = 0; i < count && r == RFM_OK; ++i) {
    rfm_problem* p = nullptr;
    r = rfm_problem_create(&descs[i], (void*)b->streams[i % b->streams.size()], &p);
    if (r == RFM_OK) b->probs.push_back(p);
  }
  if (r != RFM_OK) {
    rfm_batch_destroy(b);
    return r;
  }
  *out = b;
  return RFM_OK;
}

rfm_status rfm_batch_destroy(rfm_batch* b) {
  if (!b) return RFM_OK;
  for (rfm_problem* p : b->probs) rfm_problem_destroy(p);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  delete b;
  return RFM_OK;
}

int rfm_batch_size(const rfm_batch* b) { return b ? (int)b->probs.size() : 0; }

rfm_problem* rfm_batch_problem(rfm_batch* b, int i) {
  return (b && i >= 0 && i < (int)b->probs.size()) ? b->probs[i] : nullptr;
}

rfm_status rfm_batch_solve(rfm_batch* b, const rfm_solve_opts* opts, int solver, double* const* c_dev,
                           rfm_solve_info* infos, int* tuned_precision_out) {
  if (!b || !opts || !c_dev || !infos || (solver != 0 && solver != 1)) {
    rfm_set_error("rfm_batch_solve: bad argument");
    return RFM_EINVAL;
  }
  const int count = (int)b->probs.size();
  for (int i = 0; i < count; ++i)
    if (!c_dev[i]) {
      rfm_set_error("rfm_batch_solve: null coefficient vector");
      return RFM_EINVAL;
    }
  // autotune: one probe per distinct (s, n), precision -1 selects per instance
  const bool autosel = opts->precision < 0;
  b->choice.assign(count, QrChoice());
  for (int i = 0; i < count; ++i) {
    rfm_problem* p = b->probs[i];
    if (autosel) RFM_TRY(tuned_qr(sketch_rows_of(p, opts), p->n, b->streams[0], &b->choice[i]));
    else b->choice[i].precision = opts->precision;
    if (tuned_precision_out) tuned_precision_out[i] = b->choice[i].precision;
  }
  // longest first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const double cx = (double)b->probs[x]->n * b->probs[x]->n * sketch_rows_of(b->probs[x], opts);
    const double cy = (double)b->probs[y]->n * b->probs[y]->n * sketch_rows_of(b->probs[y], opts);
    return cx > cy;
  });
  std::atomic<int> next{0};
  std::vector<rfm_status> status(count, RFM_OK);
  std::vector<std::string> errs(count);
  auto worker = [&](int w) {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = order[k];
      rfm_problem* p = b->probs[i];
      p->stream = b->streams[w];
      p->qr_panel_cap = b->choice[i].panel_cap;
      rfm_solve_opts o = *opts;
      o.precision = b->choice[i].precision;
      rfm_status st = solver == 0 ? rfm_ipn_solve(p, &o, c_dev[i], &infos[i]) : rfm_amipn_solve(p, &o, c_dev[i], &infos[i]);
      if (st != RFM_OK && st != RFM_ENOCONV) errs[i] = rfm_last_error();
      status[i] = st;
      cudaStreamSynchronize(p->stream);
      release_workspace(p);
    }
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < (int)b->streams.size(); ++w) pool.emplace_back(worker, w);
  for (std::thread& t : pool) t.join();
  rfm_status worst = RFM_OK;
  for (int i = 0; i < count; ++i) {
    if (status[i] != RFM_OK && status[i] != RFM_ENOCONV) {
      rfm_set_error("instance " + std::to_string(i) + ": " + errs[i]);
      return status[i];
    }
    if (status[i] == RFM_ENOCONV) worst = RFM_ENOCONV;
  }
  return worst;
}

}  // extern "C"
