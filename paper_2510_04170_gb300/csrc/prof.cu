// Optional per-kernel-family timing with CUDA events recorded on the stream
// each kernel is launched on.  Disabled by default (zero overhead beyond one
// branch per launch); a benchmark enables it, runs, then reads the totals.
#include <atomic>
#include <mutex>
#include <vector>

#include "rfm_internal.cuh"

namespace {

const char* kNames[RFM_PROF_FAMILIES] = {"assemble",  "residual", "sketch_count", "sketch_gauss_gen", "sketch_gemm",
                                         "qr_panel",  "qr_vta",   "qr_update",    "trsv",             "jmv",
                                         "jtmv",      "ls_pre",   "ls_eval",      "vector",           "eval",
                                         "oz_gemm",   "oz_slice"};

struct Rec {
  int fam;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
unsigned int g_mask = 0;
std::atomic<long long> g_launches{0};
std::vector<Rec> g_recs;
double g_ms[RFM_PROF_FAMILIES];
double g_work[RFM_PROF_FAMILIES];
long long g_cnt[RFM_PROF_FAMILIES];

void drain_locked() {
  for (Rec& r : g_recs) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    g_ms[r.fam] += ms;
    g_cnt[r.fam] += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
}

}  // namespace

void rfm_prof_work(int fam, double units) {
  if (!g_on || !((g_mask >> fam) & 1u)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_work[fam] += units;
}

namespace {
thread_local bool t_count_paused = false;
}  // namespace

void rfm_count_pause(bool paused) { t_count_paused = paused; }
void rfm_count_launch() {
  if (!t_count_paused) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void rfm_count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long rfm_launches_now() { return g_launches.load(std::memory_order_relaxed); }
bool rfm_prof_active(unsigned int families) { return g_on && (g_mask & families) != 0; }

// Per-device settings: the SM count and the dynamic shared-memory attributes
// of kernels belong to one device's context, so they are cached per device
// ordinal (a process may drive several GPUs from one library instance).
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
int g_sms[kMaxDevices];
struct AttrSet {
  int dev;
  const void* func;
  int bytes;
};
std::vector<AttrSet> g_attrs;
}  // namespace

int rfm_num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    g_sms[dev] = v;
  }
  return g_sms[dev];
}

cudaError_t rfm_smem_attr(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  for (const AttrSet& a : g_attrs)
    if (a.dev == dev && a.func == func && a.bytes >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attrs.push_back({dev, func, bytes});
  return e;
}

void* rfm_prof_begin(int fam, cudaStream_t st) {
  if (!g_on || !((g_mask >> fam) & 1u)) return nullptr;
  Rec* r = new Rec;
  r->fam = fam;
  cudaEventCreate(&r->a);
  cudaEventCreate(&r->b);
  cudaEventRecord(r->a, st);
  return r;
}

void rfm_prof_end(void* h, cudaStream_t st) {
  if (!h) return;
  Rec* r = static_cast<Rec*>(h);
  cudaEventRecord(r->b, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(*r);
  delete r;
  if (g_recs.size() > 4096) drain_locked();
}

extern "C" {

rfm_status rfm_profile_enable(int mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  for (int i = 0; i < RFM_PROF_FAMILIES; ++i) {
    g_ms[i] = 0.0;
    g_cnt[i] = 0;
    g_work[i] = 0.0;
  }
  g_mask = (unsigned int)mask;
  g_on = mask != 0;
  return RFM_OK;
}

int64_t rfm_launch_count(void) { return g_launches.load(); }

rfm_status rfm_profile_work(int family, double* units) {
  if (family < 0 || family >= RFM_PROF_FAMILIES || !units) return RFM_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  *units = g_work[family];
  return RFM_OK;
}

int rfm_profile_count(void) { return RFM_PROF_FAMILIES; }

const char* rfm_profile_name(int family) {
  return (family >= 0 && family < RFM_PROF_FAMILIES) ? kNames[family] : "";
}

rfm_status rfm_profile_read(int family, double* ms, int64_t* launches) {
  if (family < 0 || family >= RFM_PROF_FAMILIES) return RFM_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  if (ms) *ms = g_ms[family];
  if (launches) *launches = g_cnt[family];
  return RFM_OK;
}

}  // extern "C"
