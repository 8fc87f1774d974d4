// runtime.cu -- host runtime and C ABI of libpsc (declared in include/psc.h).
//
// A context owns one device's resident state: scanners, material tables,
// phantoms (packed voxels, alias table, per-phantom Woodcock majorant),
// LUTs, sensitivity / normalisation sinograms and int64 accumulators.  Calls
// validate their arguments, never throw across the ABI, and enqueue kernels
// on the caller's stream.
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <climits>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <string>
#include <unordered_map>
#include <vector>
#include <map>
#include <algorithm>

#include <sys/mman.h>
#include <unistd.h>

#include "psc.h"
#include "psc_internal.h"

using namespace psc;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(PSC_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

namespace psc {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace psc

namespace {

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
  } while (0)

constexpr int kCounterSlots = 4096;

enum Kind { kScannerObj = 1, kMaterialsObj, kPhantomObj, kLutObj, kSinoObj, kAccObj };

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool own = true;  // false: caller-owned memory (psc_acc_wrap), not freed
  ~DevBuf() {
    if (p && own) cudaFree(p);
  }
};

struct Object {
  int kind;
  size_t bytes = 0;
  explicit Object(int k) : kind(k) {}
  virtual ~Object() = default;
};

struct ScannerObj : Object {
  psc_scanner_desc desc;
  ScannerParams params{};
  long long n_bins = 0, n_lor = 0;
  ScannerObj() : Object(kScannerObj) {}
};

struct MaterialsObj : Object {
  int n_mat = 0, n_e = 0;
  std::vector<double> comp, rayl, phot, kappa;
  MaterialsObj() : Object(kMaterialsObj) {}
};

struct PhantomObj : Object {
  psc_phantom_desc desc;  // host pointers cleared
  int n_mat = 0, n_e = 0;
  long long n_vox = 0;
  DevBuf vox, alias, xs, maj, kappa;
  // completes after every transport launch so far that reads this phantom
  // (each launch's record first waits for the previous one)
  std::mutex use_mu;
  cudaEvent_t last_use = nullptr;
  PhantomObj() : Object(kPhantomObj) {}
  ~PhantomObj() override {
    if (last_use) cudaEventDestroy(last_use);
  }
};

struct LutObj : Object {
  psc_lut_desc desc;
  DevBuf data;
  LutParams params;
  LutObj() : Object(kLutObj) {}
};

struct SinoObj : Object {
  int32_t scanner = 0;
  int per_lor = 0;
  long long n = 0;
  DevBuf data, data32, recip;  // FP64 values, FP32 copy, FP64 reciprocal (made on first use)
  SinoObj() : Object(kSinoObj) {}
};

struct AccObj : Object {
  int32_t scanner = 0;
  long long n = 0;
  DevBuf data;
  AccObj() : Object(kAccObj) {}
};

// device guard: make the context's device current for the call
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace psc {
// launch schedule of a batched transport launch: CTA size and count (0:
// as many as fit), work items per CTA and request, and the largest work item
struct Sched {
  int block = 0, grid = 0;
  int chunks_per_cta = 2;
  unsigned long long max_chunk = 65536;
};
}  // namespace psc

struct psc_ctx {
  int device = 0;
  int sms = 0;
  int max_smem_optin = 0;
  uint64_t budget = 0;
  uint64_t resident = 0;
  std::mutex mu;
  int32_t next_id = 1;
  std::unordered_map<int32_t, std::shared_ptr<Object>> objs;
  // finalize working buffer (FP32, sinogram-sized), grown on demand; its
  // users are ordered on the GPU through scratch_done (the last smoothing
  // pass that wrote it), so calls on different streams never overlap on it
  std::mutex scratch_mu;
  DevBuf scratch;
  cudaEvent_t scratch_done = nullptr;
  // statistics counters of psc_simulate (used only when stats are requested)
  std::mutex stats_mu;
  DevBuf stats;
  // work counters of the persistent transport launches: a ring of slots,
  // each zeroed on the launch's stream before use
  DevBuf counters;
  DevBuf dbg;                     // bounds-check record (DebugRecord) of the debug build
  // host-mapped word the axial pass sets when a bounded wait for its tile
  // copies ran out (reported by the next finalize call), or nullptr
  int* status_host = nullptr;
  int* status_dev = nullptr;
  unsigned long long counter_next = 0;
  // slot fields the transport kernel keeps in global memory, grown on
  // demand; launches on different streams are ordered through cold_done
  std::mutex cold_mu;
  DevBuf cold;
  cudaEvent_t cold_done = nullptr;
  cudaStream_t upload = nullptr;  // non-blocking stream of alias-table uploads
  // the batched-launch autotuner's choices, per request mix (scanner,
  // phantom, LUT of each request, sorted): the schedule and its probed rate
  std::map<std::vector<std::tuple<int, int, int>>, std::pair<psc::Sched, double>> tuned;
};

// True while stream s is being captured into a CUDA graph.  Calls captured
// on one stream take their order from the graph: they skip the events that
// order the context's shared buffers (slot buffer, smoothing scratch) and
// phantoms across streams, and they cannot allocate or wait, so their
// buffers must exist from an earlier call outside the capture.
static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st == cudaStreamCaptureStatusActive;
}

// Debug builds: after a call's launches, wait for them and fail with
// PSC_EDEVICE if a bounds check caught an index (the record is then cleared).
static int debug_check(psc_ctx* ctx, cudaStream_t s, const char* what) {
#if PSC_DEBUG
  if (capturing(s)) return PSC_OK;  // checked when a launch outside a capture waits
  static const char* const kSites[] = {"self-test", "alias table", "voxel", "material id", "Rayleigh kappa",
                                       "LUT tap", "accumulator bin", "per-history output", "slot",
                                       "finalize bin", "finalize LOR factor", "smoothing column"};
  psc::DebugRecord r;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&r, ctx->dbg.p, sizeof r, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(PSC_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
  if (r.count) {
    cudaMemset(ctx->dbg.p, 0, sizeof r);
    return fail(PSC_EDEVICE, "bounds check failed in %s: %llu accesses out of range, the first at %s (index %llu, bound %llu)",
                what, r.count, r.site < 12 ? kSites[r.site] : "?", r.index, r.bound);
  }
#else
  (void)ctx;
  (void)s;
  (void)what;
#endif
  return PSC_OK;
}

namespace {

int dev_alloc(psc_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->budget && ctx->resident + bytes > ctx->budget)
      return fail(PSC_ENOMEM, "device memory budget exceeded (%llu + %llu > %llu bytes)",
                  (unsigned long long)ctx->resident, (unsigned long long)bytes,
                  (unsigned long long)ctx->budget);
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(PSC_ENOMEM, "cudaMalloc(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return PSC_OK;
}

int32_t add_object(psc_ctx* ctx, std::shared_ptr<Object> o) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  const int32_t id = ctx->next_id++;
  ctx->resident += o->bytes;
  ctx->objs.emplace(id, std::move(o));
  return id;
}

template <class T>
std::shared_ptr<T> get(psc_ctx* ctx, int32_t id, int kind) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->objs.find(id);
  if (it == ctx->objs.end() || it->second->kind != kind) return nullptr;
  return std::static_pointer_cast<T>(it->second);
}

const char* kind_name(int k) {
  switch (k) {
    case kScannerObj: return "scanner";
    case kMaterialsObj: return "materials";
    case kPhantomObj: return "phantom";
    case kLutObj: return "lut";
    case kSinoObj: return "sinogram";
    case kAccObj: return "accumulator";
  }
  return "object";
}

#define GET(T, var, id, kind)                                                     \
  auto var = get<T>(ctx, id, kind);                                               \
  if (!var) return fail(PSC_ENOTFOUND, "no %s with id %d", kind_name(kind), (int)(id))

// ---------------------------------------------------------------------------
// Vose's alias method (Vose 1991) in FP64 with a fixed work-list order:
// scaled weights n * a_i / sum, indices pushed in ascending order onto a
// "small" (< 1) or "large" stack, pairs popped from the tops; leftovers get
// probability 1.
// ---------------------------------------------------------------------------
int build_alias(const float* a, long long n, std::vector<double>& prob, std::vector<int32_t>& alias) {
  double sum = 0.0;
  for (long long i = 0; i < n; ++i) {
    const double v = (double)a[i];
    if (!(v >= 0.0) || !std::isfinite(v)) return fail(PSC_EINVAL, "activity[%lld] is negative or not finite", i);
    sum += v;
  }
  if (!(sum > 0.0) || !std::isfinite(sum)) return fail(PSC_EINVAL, "activity has no positive finite sum");
  prob.assign((size_t)n, 0.0);
  alias.assign((size_t)n, 0);
  std::vector<double> p((size_t)n);
  std::vector<int32_t> small, large;
  small.reserve((size_t)n);
  large.reserve((size_t)n);
  for (long long i = 0; i < n; ++i) {
    p[i] = ((double)a[i] * (double)n) / sum;
    (p[i] < 1.0 ? small : large).push_back((int32_t)i);
  }
  while (!small.empty() && !large.empty()) {
    const int32_t s = small.back();
    small.pop_back();
    const int32_t l = large.back();
    large.pop_back();
    prob[s] = p[s];
    alias[s] = l;
    p[l] = (p[l] + p[s]) - 1.0;
    (p[l] < 1.0 ? small : large).push_back(l);
  }
  while (!large.empty()) {
    const int32_t l = large.back();
    large.pop_back();
    prob[l] = 1.0;
    alias[l] = l;
  }
  while (!small.empty()) {
    const int32_t s = small.back();
    small.pop_back();
    prob[s] = 1.0;
    alias[s] = s;
  }
  return PSC_OK;
}

float round_up_f32(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

int check_scanner(const psc_scanner_desc* d) {
  if (!d) return fail(PSC_EINVAL, "scanner desc is NULL");
  if (d->n_crystals < 4 || (d->n_crystals & 1)) return fail(PSC_EINVAL, "n_crystals must be even and >= 4");
  if (d->n_rings < 1 || d->n_tof < 1) return fail(PSC_EINVAL, "n_rings and n_tof must be >= 1");
  if (d->n_rad < 1 || d->n_rad > d->n_crystals - 1 || ((d->n_crystals - 1 - d->n_rad) & 1))
    return fail(PSC_EINVAL, "n_rad must be in [1, n_crystals-1] with n_crystals-1-n_rad even");
  if (!(d->radius > 0) || !(d->ring_pitch > 0) || !(d->tof_bin_mm > 0) || !(d->tof_sigma_mm >= 0))
    return fail(PSC_EINVAL, "radius, ring_pitch, tof_bin_mm must be > 0 and tof_sigma_mm >= 0");
  if (d->module_t < 1 || d->module_a < 1) return fail(PSC_EINVAL, "module sizes must be >= 1");
  if (!(d->e_hi >= d->e_lo) || !(d->e_lo >= 0)) return fail(PSC_EINVAL, "bad energy window");
  if (!(d->e_res_fwhm >= 0.0 && d->e_res_fwhm < 1.0)) return fail(PSC_EINVAL, "e_res_fwhm must be in [0, 1)");
  if (d->gap_mode < 0 || d->gap_mode > 2) return fail(PSC_EINVAL, "gap_mode must be 0, 1 or 2");
  if (d->gap_mode) {
    if (d->n_crystals % d->module_t || d->n_rings % d->module_a)
      return fail(PSC_EINVAL, "with gaps, module_t must divide n_crystals and module_a n_rings");
    if (!(d->gap_t_mm >= 0) || !(d->gap_a_mm >= 0) || !(d->crystal_depth_mm > 0) || !(d->doi_mm >= 0) ||
        !(d->mu_block >= 0))
      return fail(PSC_EINVAL, "gap widths, crystal depth, doi and mu_block must be >= 0 (depth > 0)");
    if (!(d->gap_t_mm < 2.0 * M_PI * d->radius * d->module_t / d->n_crystals) ||
        !(d->gap_a_mm < d->n_rings * d->ring_pitch * d->module_a / d->n_rings))
      return fail(PSC_EINVAL, "a gap must be narrower than its module or block");
  }
  return PSC_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* psc_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// error reporting for the library's other translation units
int psc::psc_set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

extern "C" {

#if PSC_DEBUG
// a known violation per lane (index 5 of 3): the record must count 32 and keep one
__global__ void debug_selftest_kernel(DebugRecord* r) { (void)dbg_idx(r, kSiteSelfTest, 5, 3); }
#endif

int psc_create(psc_ctx** out, int32_t device, uint64_t mem_budget_bytes) {
  if (!out) return fail(PSC_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(PSC_EINVAL, "device %d out of range (%d devices)", device, n);
  psc_ctx* ctx = new (std::nothrow) psc_ctx();
  if (!ctx) return fail(PSC_ENOMEM, "host allocation failed");
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaGetDeviceProperties");
  }
  ctx->sms = prop.multiProcessorCount;
  ctx->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
  e = cudaMalloc(&ctx->stats.p, sizeof(unsigned long long) * kStatCount);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaMalloc(stats)");
  }
  ctx->stats.bytes = sizeof(unsigned long long) * kStatCount;
  e = cudaMalloc(&ctx->counters.p, sizeof(unsigned long long) * kCounterSlots);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaMalloc(counters)");
  }
  ctx->counters.bytes = sizeof(unsigned long long) * kCounterSlots;
  e = cudaMalloc(&ctx->dbg.p, sizeof(DebugRecord));
  if (e == cudaSuccess) e = cudaMemset(ctx->dbg.p, 0, sizeof(DebugRecord));
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaMalloc(debug record)");
  }
  ctx->dbg.bytes = sizeof(DebugRecord);
#if PSC_DEBUG
  {  // the checks record what they catch: a known violation, then a clean record
    DebugRecord r;
    debug_selftest_kernel<<<1, 32>>>((DebugRecord*)ctx->dbg.p);
    e = cudaMemcpy(&r, ctx->dbg.p, sizeof r, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->dbg.p, 0, sizeof(DebugRecord));
    if (e != cudaSuccess || r.count != 32 || r.site != kSiteSelfTest || r.index != 5 || r.bound != 3) {
      delete ctx;
      return e != cudaSuccess ? cuda_fail(e, "debug self-test") : fail(PSC_EDEVICE, "debug self-test: record not kept");
    }
  }
#endif
  e = cudaEventCreateWithFlags(&ctx->scratch_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->cold_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->upload, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (ctx->scratch_done) cudaEventDestroy(ctx->scratch_done);
    if (ctx->cold_done) cudaEventDestroy(ctx->cold_done);
    delete ctx;
    return cuda_fail(e, "cudaEventCreate");
  }
  if (cudaHostAlloc((void**)&ctx->status_host, sizeof(int), cudaHostAllocMapped) == cudaSuccess) {
    *ctx->status_host = 0;
    if (cudaHostGetDevicePointer((void**)&ctx->status_dev, ctx->status_host, 0) != cudaSuccess) {
      cudaGetLastError();
      ctx->status_dev = nullptr;
    }
  } else {
    cudaGetLastError();
    ctx->status_host = nullptr;
  }
  *out = ctx;
  return PSC_OK;
}

void psc_destroy(psc_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->scratch_done) cudaEventDestroy(ctx->scratch_done);
  if (ctx->cold_done) cudaEventDestroy(ctx->cold_done);
  if (ctx->upload) cudaStreamDestroy(ctx->upload);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  delete ctx;
}

uint64_t psc_resident_bytes(const psc_ctx* ctx) { return ctx ? ctx->resident : 0; }

}  // extern "C"

namespace {

std::mutex g_host_mu;
std::unordered_map<void*, size_t> g_host;  // buffer -> mapped bytes

// the kernel's transparent huge page size (2 MB where it does not say)
size_t huge_page_bytes() {
  size_t hp = 2u << 20;
  if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long v = 0;
    if (std::fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) hp = (size_t)v;
    std::fclose(f);
  }
  return hp;
}

}  // namespace

extern "C" {

#ifdef MADV_COLLAPSE
constexpr int kMadvCollapse = MADV_COLLAPSE;
#else
constexpr int kMadvCollapse = 25;  // Linux's value for MADV_COLLAPSE
#endif

int psc_host_alloc(uint64_t bytes, void** ptr) {
  if (!ptr) return fail(PSC_EINVAL, "ptr is NULL");
  *ptr = nullptr;
  if (bytes == 0) return fail(PSC_EINVAL, "zero bytes");
  const size_t hp = huge_page_bytes();
  if (bytes > SIZE_MAX - 2 * hp) return fail(PSC_EOVERFLOW, "%llu bytes", (unsigned long long)bytes);
  const size_t len = (size_t)((bytes + hp - 1) / hp * hp);
  // map one huge page more than needed, then trim to a huge-page-aligned range
  void* raw = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return fail(PSC_ENOMEM, "mapping %zu bytes of host memory failed", len + hp);
  const uintptr_t a = ((uintptr_t)raw + hp - 1) & ~(uintptr_t)(hp - 1);
  const size_t head = a - (uintptr_t)raw;
  if (head) munmap(raw, head);
  if (hp - head) munmap((char*)a + len, hp - head);
  char* p = (char*)a;
  madvise(p, len, MADV_HUGEPAGE);  // advice only: without it the buffer still works, on base pages
  const long pg = sysconf(_SC_PAGESIZE);
  const size_t step = pg > 0 ? (size_t)pg : 4096;
  // fault in now, as huge pages where possible, with one nonzero byte per
  // base page: the kernel may split huge pages whose base pages are all
  // zero (its underused-huge-page shrinker); the contents are unspecified
  for (size_t i = 0; i < len; i += step) p[i] = 1;
  // where a fault found no free huge page (fragmented memory), collapse each
  // huge-page block now (Linux 6.1+): a block that fails is released and
  // faulted in again, then collapsed once more.  A registered buffer with
  // base pages scattered through it read back at a quarter of the host
  // link's rate in measurements; where the kernel cannot collapse, the
  // buffer stays as faulted.
  for (size_t off = 0; off < len; off += hp) {
    char* b = p + off;
    for (int attempt = 0; attempt < 3; ++attempt) {
      if (madvise(b, hp, kMadvCollapse) == 0) break;
      if (errno == EINVAL) {  // no MADV_COLLAPSE in this kernel
        off = len;
        break;
      }
      if (attempt == 1) {     // give the block's memory back and fault it in again
        madvise(b, hp, MADV_DONTNEED);
        for (size_t i = 0; i < hp; i += step) b[i] = 1;
      }
    }
  }
  const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterPortable);
  if (e != cudaSuccess) {
    cudaGetLastError();
    munmap(p, len);
    return cuda_fail(e, "registering host buffer");
  }
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host[p] = len;
  }
  *ptr = p;
  return PSC_OK;
}

int psc_host_free(void* ptr) {
  size_t len = 0;
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    auto it = g_host.find(ptr);
    if (it == g_host.end()) return fail(PSC_EINVAL, "%p is not a buffer of psc_host_alloc", ptr);
    len = it->second;
    g_host.erase(it);
  }
  const cudaError_t e = cudaHostUnregister(ptr);
  munmap(ptr, len);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "unregistering host buffer");
  }
  return PSC_OK;
}

int psc_load_scanner(psc_ctx* ctx, const psc_scanner_desc* d, int32_t* id) {
  if (!ctx || !id) return fail(PSC_EINVAL, "ctx or id is NULL");
  int rc = check_scanner(d);
  if (rc) return rc;
  auto o = std::make_shared<ScannerObj>();
  o->desc = *d;
  ScannerParams& s = o->params;
  s.radius = (float)d->radius;
  s.r2 = (float)(d->radius * d->radius);
  s.half_len = (float)(0.5 * d->n_rings * d->ring_pitch);
  s.inv_pitch = (float)(1.0 / d->ring_pitch);
  s.e_lo = (float)d->e_lo;
  s.e_hi = (float)d->e_hi;
  // FWHM e_res * 511 keV at 511 keV, scaling as sqrt(E); photons more than
  // 5 sigma below the window after a Compton event are dropped
  const double fwhm_to_sigma = 2.0 * std::sqrt(2.0 * std::log(2.0));
  s.e_res_k = (float)(d->e_res_fwhm * std::sqrt(511.0) / fwhm_to_sigma);
  s.escape_words = (d->e_res_fwhm > 0.0 ? 2 : 0) + (d->gap_mode == 2 ? 2 : 0);
  s.gap_mode = d->gap_mode;
  if (d->gap_mode) {
    s.n_mod = d->n_crystals / d->module_t;
    s.n_blk = d->n_rings / d->module_a;
    const double mod_phi = 2.0 * M_PI / s.n_mod, blk_pitch = d->n_rings * d->ring_pitch / s.n_blk;
    s.mod_phi = (float)mod_phi;
    s.inv_mod_phi = (float)(1.0 / mod_phi);
    s.gap_gamma = (float)(d->gap_t_mm / d->radius);
    s.inv_crys_phi = (float)(d->module_t / (mod_phi - d->gap_t_mm / d->radius));
    s.blk_pitch = (float)blk_pitch;
    s.inv_blk_pitch = (float)(1.0 / blk_pitch);
    s.gap_a = (float)d->gap_a_mm;
    s.inv_ring_w = (float)(d->module_a / (blk_pitch - d->gap_a_mm));
    s.gap_t_mm = (float)d->gap_t_mm;
    s.depth = (float)d->crystal_depth_mm;
    s.doi = (float)d->doi_mm;
    s.mu = (float)d->mu_block;
  }
  s.e_kill = d->e_res_fwhm > 0.0
                 ? (float)std::max(0.0, d->e_lo - 5.0 * d->e_res_fwhm * std::sqrt(511.0 * d->e_lo) / fwhm_to_sigma)
                 : (float)d->e_lo;
  s.crystals_per_radian = (float)(d->n_crystals / (2.0 * M_PI));
  s.inv_tof_bin = (float)(1.0 / d->tof_bin_mm);
  s.tof_half = (float)(0.5 * d->n_tof);
  s.tof_sigma = (float)d->tof_sigma_mm;
  s.n_crystals = d->n_crystals;
  s.n_rings = d->n_rings;
  s.module_t = d->module_t;
  s.module_a = d->module_a;
  s.n_tof = d->n_tof;
  s.n_rad = d->n_rad;
  s.n_views = d->n_crystals / 2;
  s.rad_off = (d->n_crystals - 1 - d->n_rad) / 2;
  o->n_lor = (long long)d->n_rings * d->n_rings * s.n_views * d->n_rad;
  o->n_bins = o->n_lor * d->n_tof;
  *id = add_object(ctx, o);
  return PSC_OK;
}

int psc_load_materials(psc_ctx* ctx, const psc_materials_desc* d, int32_t* id) {
  if (!ctx || !id || !d) return fail(PSC_EINVAL, "NULL argument");
  if (d->n_mat < 1 || d->n_mat > kMaxMaterials) return fail(PSC_EINVAL, "n_mat must be in [1, %d]", kMaxMaterials);
  if (d->n_e < 512) return fail(PSC_EINVAL, "n_e must be >= 512 (nodes 0..511 keV at least)");
  if (!d->compton || !d->rayleigh || !d->photo || !d->kappa) return fail(PSC_EINVAL, "NULL table");
  auto o = std::make_shared<MaterialsObj>();
  const size_t n = (size_t)d->n_mat * d->n_e;
  o->n_mat = d->n_mat;
  o->n_e = d->n_e;
  o->comp.assign(d->compton, d->compton + n);
  o->rayl.assign(d->rayleigh, d->rayleigh + n);
  o->phot.assign(d->photo, d->photo + n);
  o->kappa.assign(d->kappa, d->kappa + d->n_mat);
  for (size_t i = 0; i < n; ++i)
    if (!(o->comp[i] >= 0) || !(o->rayl[i] >= 0) || !(o->phot[i] >= 0) || !std::isfinite(o->comp[i] + o->rayl[i] + o->phot[i]))
      return fail(PSC_EINVAL, "cross-section table entry %zu negative or not finite", i);
  for (int m = 0; m < d->n_mat; ++m)
    if (!(o->kappa[m] >= 0) || !std::isfinite(o->kappa[m])) return fail(PSC_EINVAL, "kappa[%d] invalid", m);
  *id = add_object(ctx, o);
  return PSC_OK;
}

// Alias acceptance as an integer threshold: a uniform u = (2k + 1) 2^-24,
// k = x >> 9, satisfies u < p exactly when k < ceil((p 2^24 - 1) / 2), so the
// kernel decides with one integer compare what the FP64 comparison decides.
static uint32_t alias_threshold(double p) {
  const double t = std::ceil((std::ldexp(p, 24) - 1.0) / 2.0);
  if (!(t > 0.0)) return 0u;
  return t >= 8388608.0 ? 8388608u : (uint32_t)t;
}

}  // extern "C"

namespace psc {

int alias_table(const float* activity, long long n_vox, std::vector<uint2>& tab) {
  std::vector<double> prob;
  std::vector<int32_t> alias;
  int rc = build_alias(activity, n_vox, prob, alias);
  if (rc) return rc;
  tab.resize((size_t)n_vox);
  for (long long i = 0; i < n_vox; ++i) tab[i] = make_uint2(alias_threshold(prob[i]), (uint32_t)alias[i]);
  return PSC_OK;
}

}  // namespace psc

namespace {

// waits for the launches still reading the phantom's current table, then
// uploads on the context's own non-blocking stream (so work on other
// streams keeps running)
int put_alias_obj(psc_ctx* ctx, PhantomObj* o, const uint2* tab) {
  std::lock_guard<std::mutex> lk(o->use_mu);
  if (o->last_use) CK(cudaEventSynchronize(o->last_use), "wait for launches reading the phantom");
  CK(cudaMemcpyAsync(o->alias.p, tab, sizeof(uint2) * o->n_vox, cudaMemcpyHostToDevice, ctx->upload),
     "upload alias");
  CK(cudaStreamSynchronize(ctx->upload), "upload alias");
  return PSC_OK;
}

int upload_alias(psc_ctx* ctx, PhantomObj* o, const float* activity) {
  std::vector<uint2> tab;
  int rc = psc::alias_table(activity, o->n_vox, tab);
  return rc ? rc : put_alias_obj(ctx, o, tab.data());
}

}  // namespace

namespace psc {

int put_alias(psc_ctx* ctx, int32_t phantom, const uint2* tab, long long n_vox) {
  GET(PhantomObj, ph, phantom, kPhantomObj);
  if (ph->n_vox != n_vox) return fail(PSC_EINVAL, "alias table of %lld entries for a phantom of %lld voxels", n_vox,
                                      ph->n_vox);
  DeviceGuard g(ctx->device);
  return put_alias_obj(ctx, ph.get(), tab);
}

}  // namespace psc

extern "C" {

int psc_load_phantom(psc_ctx* ctx, const psc_phantom_desc* d, int32_t materials, int32_t* id) {
  if (!ctx || !id || !d) return fail(PSC_EINVAL, "NULL argument");
  GET(MaterialsObj, mat, materials, kMaterialsObj);
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(PSC_EINVAL, "phantom dims must be >= 1");
  const long long nv = (long long)d->nx * d->ny * d->nz;
  if (nv > (1LL << 31) - 1) return fail(PSC_EOVERFLOW, "phantom has more than 2^31-1 voxels");
  if (!(d->dx > 0) || !(d->dy > 0) || !(d->dz > 0)) return fail(PSC_EINVAL, "voxel sizes must be > 0");
  if (!d->material || !d->density || !d->activity) return fail(PSC_EINVAL, "NULL phantom array");
  DeviceGuard g(ctx->device);
  auto o = std::make_shared<PhantomObj>();
  o->desc = *d;
  o->desc.material = nullptr;
  o->desc.density = nullptr;
  o->desc.activity = nullptr;
  o->n_vox = nv;
  o->n_mat = mat->n_mat;
  o->n_e = mat->n_e;
  // packed voxels and the densest voxel per material
  std::vector<float2> vox((size_t)nv);
  std::vector<double> rho_max((size_t)mat->n_mat, 0.0);
  for (long long v = 0; v < nv; ++v) {
    const int m = d->material[v];
    const float r = d->density[v];
    if (m >= mat->n_mat) return fail(PSC_EINVAL, "material[%lld] = %d >= n_mat", v, m);
    if (!(r >= 0.0f) || !std::isfinite(r)) return fail(PSC_EINVAL, "density[%lld] invalid", v);
    int bits = m;
    float fm;
    std::memcpy(&fm, &bits, sizeof fm);
    vox[v] = make_float2(r, fm);
    if ((double)r > rho_max[m]) rho_max[m] = (double)r;
  }
  // cumulative cross sections (mm^-1 per g/cm^3) and the Woodcock majorant
  const int ne = mat->n_e;
  std::vector<float4> xs((size_t)mat->n_mat * ne);
  std::vector<float> maj((size_t)ne);
  for (int m = 0; m < mat->n_mat; ++m)
    for (int k = 0; k < ne; ++k) {
      const double c = mat->comp[(size_t)m * ne + k], r = mat->rayl[(size_t)m * ne + k],
                   p = mat->phot[(size_t)m * ne + k];
      xs[(size_t)m * ne + k] = make_float4((float)(c / 10.0), (float)((c + r) / 10.0), (float)((c + r + p) / 10.0), 0.0f);
    }
  for (int k = 0; k < ne; ++k) {
    double best = 0.0;
    for (int m = 0; m < mat->n_mat; ++m) {
      const double tot = mat->comp[(size_t)m * ne + k] + mat->rayl[(size_t)m * ne + k] + mat->phot[(size_t)m * ne + k];
      const double mu = rho_max[m] * tot / 10.0;
      if (mu > best) best = mu;
    }
    maj[k] = round_up_f32(best);
  }
  std::vector<float> kap(kMaxMaterials, 0.0f);
  for (int m = 0; m < mat->n_mat; ++m) kap[m] = (float)mat->kappa[m];
  int rc;
  if ((rc = dev_alloc(ctx, o->vox, sizeof(float2) * nv))) return rc;
  if ((rc = dev_alloc(ctx, o->alias, sizeof(uint2) * nv))) return rc;
  if ((rc = dev_alloc(ctx, o->xs, sizeof(float4) * xs.size()))) return rc;
  if ((rc = dev_alloc(ctx, o->maj, sizeof(float) * ne))) return rc;
  if ((rc = dev_alloc(ctx, o->kappa, sizeof(float) * kMaxMaterials))) return rc;
  o->bytes = o->vox.bytes + o->alias.bytes + o->xs.bytes + o->maj.bytes + o->kappa.bytes;
  CK(cudaMemcpy(o->vox.p, vox.data(), sizeof(float2) * nv, cudaMemcpyHostToDevice), "upload voxels");
  CK(cudaMemcpy(o->xs.p, xs.data(), sizeof(float4) * xs.size(), cudaMemcpyHostToDevice), "upload tables");
  CK(cudaMemcpy(o->maj.p, maj.data(), sizeof(float) * ne, cudaMemcpyHostToDevice), "upload majorant");
  CK(cudaMemcpy(o->kappa.p, kap.data(), sizeof(float) * kMaxMaterials, cudaMemcpyHostToDevice), "upload kappa");
  if ((rc = upload_alias(ctx, o.get(), d->activity))) return rc;
  *id = add_object(ctx, o);
  return PSC_OK;
}

int64_t psc_phantom_voxels(psc_ctx* ctx, int32_t phantom) {
  if (!ctx) return fail(PSC_EINVAL, "ctx is NULL");
  GET(PhantomObj, ph, phantom, kPhantomObj);
  return ph->n_vox;
}

int psc_update_activity(psc_ctx* ctx, int32_t phantom, const float* activity) {
  if (!ctx || !activity) return fail(PSC_EINVAL, "NULL argument");
  GET(PhantomObj, ph, phantom, kPhantomObj);
  DeviceGuard g(ctx->device);
  return upload_alias(ctx, ph.get(), activity);
}

int psc_phantom_alias(psc_ctx* ctx, int32_t phantom, uint32_t* threshold, int32_t* alias) {
  if (!ctx || !threshold || !alias) return fail(PSC_EINVAL, "NULL argument");
  GET(PhantomObj, ph, phantom, kPhantomObj);
  DeviceGuard g(ctx->device);
  std::vector<uint2> tab((size_t)ph->n_vox);
  CK(cudaMemcpy(tab.data(), ph->alias.p, sizeof(uint2) * ph->n_vox, cudaMemcpyDeviceToHost), "read alias");
  for (long long i = 0; i < ph->n_vox; ++i) {
    threshold[i] = tab[i].x;
    alias[i] = (int32_t)tab[i].y;
  }
  return PSC_OK;
}

int psc_load_lut(psc_ctx* ctx, const psc_lut_desc* d, int32_t* id) {
  if (!ctx || !id || !d) return fail(PSC_EINVAL, "NULL argument");
  if (d->n_e < 1 || d->n_a < 1 || d->n_b < 1 || d->n_tpos < 1 || d->n_apos < 1)
    return fail(PSC_EINVAL, "LUT axis sizes must be >= 1");
  if (!(d->e_max > d->e_min) || !(d->a_max > d->a_min) || !(d->b_max > d->b_min))
    return fail(PSC_EINVAL, "LUT axis ranges must be increasing");
  if (d->dtype < PSC_LUT_F32 || d->dtype > PSC_LUT_BF16) return fail(PSC_EINVAL, "unknown LUT dtype %d", d->dtype);
  const long long n = (long long)d->n_e * d->n_a * d->n_b * d->n_tpos * d->n_apos;
  DeviceGuard g(ctx->device);
  auto o = std::make_shared<LutObj>();
  o->desc = *d;
  o->desc.data = nullptr;
  const size_t esz = d->dtype == PSC_LUT_F32 ? 4 : 2;
  std::vector<unsigned char> host((size_t)n * esz);
  for (long long i = 0; i < n; ++i) {
    const float v = d->data ? d->data[i] : 1.0f;
    if (!(v >= 0.0f && v <= 1.0f)) return fail(PSC_EINVAL, "LUT value %lld = %g outside [0, 1]", i, (double)v);
    if (d->dtype == PSC_LUT_F32) {
      std::memcpy(&host[(size_t)i * 4], &v, 4);
    } else if (d->dtype == PSC_LUT_F16) {
      const __half h = __float2half_rn(v);
      std::memcpy(&host[(size_t)i * 2], &h, 2);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      std::memcpy(&host[(size_t)i * 2], &h, 2);
    }
  }
  int rc;
  if ((rc = dev_alloc(ctx, o->data, host.size()))) return rc;
  o->bytes = o->data.bytes;
  CK(cudaMemcpy(o->data.p, host.data(), host.size(), cudaMemcpyHostToDevice), "upload LUT");
  LutParams& L = o->params;
  L.data = o->data.p;
  L.dtype = d->dtype;
  L.n_e = d->n_e;
  L.n_a = d->n_a;
  L.n_b = d->n_b;
  L.n_tpos = d->n_tpos;
  L.n_apos = d->n_apos;
  L.e_min = (float)d->e_min;
  L.e_scale = (float)(d->n_e / (d->e_max - d->e_min));
  L.a_min = (float)d->a_min;
  L.a_scale = (float)(d->n_a / (d->a_max - d->a_min));
  L.b_min = (float)d->b_min;
  L.b_scale = (float)(d->n_b / (d->b_max - d->b_min));
  const long long block = (long long)d->n_e * d->n_a * d->n_b;
  L.t_stride = d->n_tpos > 1 ? block : 0;
  L.a_stride = d->n_apos > 1 ? block * d->n_tpos : 0;
  L.size = block * d->n_tpos * d->n_apos;
  *id = add_object(ctx, o);
  return PSC_OK;
}

int psc_load_sinogram(psc_ctx* ctx, int32_t scanner, const double* host, int32_t per_lor, int32_t* id) {
  if (!ctx || !id || !host) return fail(PSC_EINVAL, "NULL argument");
  GET(ScannerObj, sc, scanner, kScannerObj);
  DeviceGuard g(ctx->device);
  auto o = std::make_shared<SinoObj>();
  o->scanner = scanner;
  o->per_lor = per_lor ? 1 : 0;
  o->n = per_lor ? sc->n_lor : sc->n_bins;
  int rc;
  if ((rc = dev_alloc(ctx, o->data, sizeof(double) * o->n))) return rc;
  if ((rc = dev_alloc(ctx, o->data32, sizeof(float) * o->n))) return rc;
  o->bytes = o->data.bytes + o->data32.bytes;
  CK(cudaMemcpy(o->data.p, host, sizeof(double) * o->n, cudaMemcpyHostToDevice), "upload sinogram");
  CK(launch_narrow((const double*)o->data.p, (float*)o->data32.p, o->n, ctx->sms, 0), "FP32 copy of the sinogram");
  CK(cudaStreamSynchronize(0), "FP32 copy of the sinogram");
  *id = add_object(ctx, o);
  return PSC_OK;
}

int psc_acc_create(psc_ctx* ctx, int32_t scanner, int32_t* id) {
  if (!ctx || !id) return fail(PSC_EINVAL, "NULL argument");
  GET(ScannerObj, sc, scanner, kScannerObj);
  DeviceGuard g(ctx->device);
  auto o = std::make_shared<AccObj>();
  o->scanner = scanner;
  o->n = sc->n_bins;
  int rc;
  if ((rc = dev_alloc(ctx, o->data, sizeof(long long) * o->n))) return rc;
  o->bytes = o->data.bytes;
  CK(cudaMemset(o->data.p, 0, sizeof(long long) * o->n), "zero accumulator");
  *id = add_object(ctx, o);
  return PSC_OK;
}

int psc_acc_wrap(psc_ctx* ctx, int32_t scanner, int64_t* device, int32_t* id) {
  if (!ctx || !id || !device) return fail(PSC_EINVAL, "NULL argument");
  if ((uintptr_t)device % 8) return fail(PSC_EINVAL, "accumulator memory must be 8-byte aligned");
  GET(ScannerObj, sc, scanner, kScannerObj);
  DeviceGuard g(ctx->device);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, device) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
      at.device != ctx->device) {
    cudaGetLastError();
    return fail(PSC_EINVAL, "accumulator memory is not device memory of the context's device");
  }
  auto o = std::make_shared<AccObj>();
  o->scanner = scanner;
  o->n = sc->n_bins;
  o->data.p = device;
  o->data.bytes = sizeof(long long) * (size_t)o->n;
  o->data.own = false;
  o->bytes = 0;
  *id = add_object(ctx, o);
  return PSC_OK;
}

int psc_acc_zero(psc_ctx* ctx, int32_t acc, psc_stream stream) {
  if (!ctx) return fail(PSC_EINVAL, "ctx is NULL");
  GET(AccObj, a, acc, kAccObj);
  DeviceGuard g(ctx->device);
  CK(cudaMemsetAsync(a->data.p, 0, sizeof(long long) * a->n, (cudaStream_t)stream), "zero accumulator");
  return PSC_OK;
}

int psc_acc_read(psc_ctx* ctx, int32_t acc, int64_t* out, psc_stream stream) {
  if (!ctx || !out) return fail(PSC_EINVAL, "NULL argument");
  GET(AccObj, a, acc, kAccObj);
  DeviceGuard g(ctx->device);
  CK(cudaMemcpyAsync(out, a->data.p, sizeof(long long) * a->n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "read accumulator");
  return PSC_OK;
}

int psc_acc_write(psc_ctx* ctx, int32_t acc, const int64_t* in, psc_stream stream) {
  if (!ctx || !in) return fail(PSC_EINVAL, "NULL argument");
  GET(AccObj, a, acc, kAccObj);
  DeviceGuard g(ctx->device);
  CK(cudaMemcpyAsync(a->data.p, in, sizeof(long long) * a->n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "write accumulator");
  return PSC_OK;
}

int psc_unload(psc_ctx* ctx, int32_t id) {
  if (!ctx) return fail(PSC_EINVAL, "ctx is NULL");
  std::shared_ptr<Object> o;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->objs.find(id);
    if (it == ctx->objs.end()) return fail(PSC_ENOTFOUND, "no object with id %d", (int)id);
    o = it->second;
    ctx->objs.erase(it);
    ctx->resident -= o->bytes;
  }
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();  // no kernel may still read it
  o.reset();
  return PSC_OK;
}

// validate one request and describe it as a kernel job
static int make_job(psc_ctx* ctx, const psc_sim_args* a, Job& jb, int& lut_dtype) {
  GET(ScannerObj, sc, a->scanner, kScannerObj);
  GET(PhantomObj, ph, a->phantom, kPhantomObj);
  GET(AccObj, acc, a->acc, kAccObj);
  std::shared_ptr<LutObj> lut;
  if (a->lut != 0) {
    lut = get<LutObj>(ctx, a->lut, kLutObj);
    if (!lut) return fail(PSC_ENOTFOUND, "no lut with id %d", (int)a->lut);
    const psc_scanner_desc& sd = sc->desc;
    const int nt = sd.gap_mode ? sd.module_t + 2 : sd.module_t;
    const int na = sd.gap_mode ? (sd.n_rings / sd.module_a) * (sd.module_a + 2) : sd.module_a;
    if ((lut->desc.n_tpos != nt && lut->desc.n_tpos != 1) || (lut->desc.n_apos != na && lut->desc.n_apos != 1))
      return fail(PSC_EINVAL, "LUT positions (%d, %d) match neither the scanner's (%d, %d) nor 1", lut->desc.n_tpos,
                  lut->desc.n_apos, nt, na);
  }
  if (acc->scanner != a->scanner) return fail(PSC_EINVAL, "accumulator belongs to scanner %d", (int)acc->scanner);
  if (a->first_history + a->n_histories < a->first_history) return fail(PSC_EOVERFLOW, "history range wraps");
  if (a->bin_mask < 0 || a->bin_mask > 3) return fail(PSC_EINVAL, "bin_mask must be in [0, 3]");
  if (a->block < 0 || a->block > 512 || (a->block % 32) || a->grid < 0)
    return fail(PSC_EINVAL, "block must be a multiple of 32 in [32, 512], grid >= 0");
  const psc_phantom_desc& pd = ph->desc;
  const double R2 = sc->desc.radius * sc->desc.radius;
  for (int i = 0; i < 4; ++i) {
    const double x = pd.ox + ((i & 1) ? pd.nx * pd.dx : 0.0), y = pd.oy + ((i & 2) ? pd.ny * pd.dy : 0.0);
    if (!(x * x + y * y < R2)) return fail(PSC_EINVAL, "phantom grid reaches outside the detector cylinder");
  }
  std::memset(&jb, 0, sizeof jb);
  jb.sc = sc->params;
  PhantomParams& q = jb.ph;
  q.nx = pd.nx;
  q.m_nx = pd.nx > 1 ? (uint32_t)((1ull << 32) / (unsigned long long)pd.nx) : 0xffffffffu;
  q.m_nxy = (long long)pd.nx * pd.ny > 1 ? (uint32_t)((1ull << 32) / ((unsigned long long)pd.nx * pd.ny))
                                         : 0xffffffffu;
  q.ny = pd.ny;
  q.nz = pd.nz;
  q.n_mat = ph->n_mat;
  q.n_e = ph->n_e;
  // staged table nodes: from just below the lowest energy a tracked photon can have
  q.e0 = std::max(0, std::min((int)std::floor(sc->params.e_kill) - 1, ph->n_e - 2));
  q.n_tab = ph->n_e - q.e0;
  q.n_vox = ph->n_vox;
  q.ox = (float)pd.ox;
  q.oy = (float)pd.oy;
  q.oz = (float)pd.oz;
  q.dx = (float)pd.dx;
  q.dy = (float)pd.dy;
  q.dz = (float)pd.dz;
  q.inv_dx = (float)(1.0 / pd.dx);
  q.inv_dy = (float)(1.0 / pd.dy);
  q.inv_dz = (float)(1.0 / pd.dz);
  q.vox = (const float2*)ph->vox.p;
  q.alias = (const uint2*)ph->alias.p;
  q.xs = (const float4*)ph->xs.p;
  q.maj = (const float*)ph->maj.p;
  q.kappa = (const float*)ph->kappa.p;
  if (lut) {
    jb.lut = lut->params;
  } else {
    jb.lut.dtype = -1;
  }
  lut_dtype = jb.lut.dtype;
  jb.seed = a->seed;
  jb.first = a->first_history;
  jb.n = a->n_histories;
  jb.bin_mask = a->bin_mask ? a->bin_mask : PSC_BIN_SCATTER;
  jb.acc = (unsigned long long*)acc->data.p;
  jb.cls_out = a->cls_out;
  jb.key_out = (long long*)a->key_out;
  jb.q_out = (long long*)a->q_out;
  if (a->lm_out && !a->lm_count) return fail(PSC_EINVAL, "lm_out needs lm_count");
  return PSC_OK;
}

using psc::Sched;

static int batch_impl(psc_ctx* ctx, const psc_sim_args* args, int32_t n, psc_stats* stats, psc_stream stream,
                      const Sched& sc_in) {
  if (!ctx || (!args && n > 0) || n < 0) return fail(PSC_EINVAL, "NULL argument or negative count");
  std::vector<Job> jobs;
  std::vector<ListmodeOut> lms;
  std::vector<int> dts;
  std::vector<std::shared_ptr<PhantomObj>> phs;
  jobs.reserve(n);
  for (int i = 0; i < n; ++i) {
    Job jb;
    int dt;
    int rc = make_job(ctx, &args[i], jb, dt);
    if (rc) return rc;
    if (jb.n == 0) continue;
    jobs.push_back(jb);
    lms.push_back(ListmodeOut{args[i].lm_out, args[i].lm_out ? (unsigned long long*)args[i].lm_count : nullptr,
                              args[i].lm_out ? args[i].lm_capacity : 0});
    dts.push_back(dt);
    phs.push_back(get<PhantomObj>(ctx, args[i].phantom, kPhantomObj));
  }
  if (stats) std::memset(stats, 0, sizeof *stats);
  if (jobs.empty()) return PSC_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int block = sc_in.block ? sc_in.block : (n > 0 && args[0].block ? args[0].block : 512);
  const bool cap = capturing(s);
  if (cap && stats) return fail(PSC_EINVAL, "statistics wait for the stream: not in a stream capture");
  std::unique_lock<std::mutex> lk(ctx->stats_mu, std::defer_lock);
  unsigned long long* dstats = nullptr;
  if (stats) {
    lk.lock();
    dstats = (unsigned long long*)ctx->stats.p;
    CK(cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * kStatCount, s), "zero stats");
  }
  // one launch per LUT storage type, at most kMaxJobs jobs each
  std::vector<bool> done(jobs.size(), false);
  int last_grid = 0;
  for (size_t i0 = 0; i0 < jobs.size(); ++i0) {
    if (done[i0]) continue;
    BatchParams bp;
    std::memset(&bp, 0, sizeof bp);
    size_t smem = 0;
    unsigned long long total = 0;
    const int dt = dts[i0];
    std::vector<PhantomObj*> used;
    for (size_t i = i0; i < jobs.size() && bp.n_jobs < kMaxJobs; ++i) {
      if (done[i] || dts[i] != dt) continue;
      done[i] = true;
      used.push_back(phs[i].get());
      bp.jobs[bp.n_jobs] = jobs[i];
      bp.lm[bp.n_jobs] = lms[i];
      smem = std::max(smem, transport_smem_bytes(jobs[i].ph, block));
      ++bp.n_jobs;
    }
    if ((int)smem > ctx->max_smem_optin) return fail(PSC_EINVAL, "material tables need %zu bytes of shared memory", smem);
    int grid = sc_in.grid ? sc_in.grid : (n > 0 ? args[0].grid : 0);
    if (grid == 0) {
      int per_sm = 0;
      CK(transport_occupancy(dt, block, smem, &per_sm), "occupancy");
      grid = ctx->sms * std::max(per_sm, 1);
    }
    // work items: chunks sized so every CTA gets chunks_per_cta of each job,
    // within [1024, max_chunk] histories
    for (int j = 0; j < bp.n_jobs; ++j) {
      Job& jb = bp.jobs[j];
      const unsigned long long parts = (unsigned long long)sc_in.chunks_per_cta * (unsigned long long)grid;
      const unsigned long long per = (jb.n + parts - 1) / parts;
      jb.chunk = std::min<unsigned long long>(std::max<unsigned long long>(1024, sc_in.max_chunk),
                                              std::max<unsigned long long>(1024, per));
      total += (jb.n + jb.chunk - 1) / jb.chunk;
      bp.chunk_end[j] = total;
    }
    if ((unsigned long long)grid > total) grid = (int)total;
    unsigned long long* counter = (unsigned long long*)ctx->counters.p + (ctx->counter_next++ % kCounterSlots);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s), "zero work counter");
    bp.next_chunk = counter;
    bp.stats = dstats;
    bp.dbg = (DebugRecord*)ctx->dbg.p;
    std::lock_guard<std::mutex> cl(ctx->cold_mu);
    const size_t cold_bytes = sizeof(uint32_t) * transport_cold_words(grid, block);
    if (ctx->cold.bytes < cold_bytes) {
      if (cap)
        return fail(PSC_EINVAL, "the transport's slot buffer grows outside a capture: run the call once first");
      CK(cudaEventSynchronize(ctx->cold_done), "wait for the slot buffer's last user");
      if (ctx->cold.p) {
        cudaFree(ctx->cold.p);
        ctx->cold.p = nullptr;
        ctx->cold.bytes = 0;
      }
      cudaError_t e = cudaMalloc(&ctx->cold.p, cold_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->cold.p = nullptr;
        return fail(PSC_ENOMEM, "transport slot buffer of %zu bytes: %s", cold_bytes, cudaGetErrorString(e));
      }
      ctx->cold.bytes = cold_bytes;
    }
    bp.cold = (uint32_t*)ctx->cold.p;
    if (!cap) CK(cudaStreamWaitEvent(s, ctx->cold_done, 0), "order slot buffer users");
    CK(launch_transport(bp, dt, grid, block, smem, s), "transport kernel launch");
    last_grid = grid;
    if (cap) continue;  // a captured launch takes its order from the graph
    CK(cudaEventRecord(ctx->cold_done, s), "order slot buffer users");
    for (PhantomObj* ph : used) {  // activity updates wait for this launch
      std::lock_guard<std::mutex> ul(ph->use_mu);
      if (!ph->last_use) CK(cudaEventCreateWithFlags(&ph->last_use, cudaEventDisableTiming), "phantom event");
      else CK(cudaStreamWaitEvent(s, ph->last_use, 0), "order phantom users");
      CK(cudaEventRecord(ph->last_use, s), "phantom event");
    }
  }
  {
    const int rc = debug_check(ctx, s, "the transport kernel");
    if (rc) return rc;
  }
  if (stats) {
    unsigned long long h[kStatCount];
    CK(cudaMemcpyAsync(h, dstats, sizeof h, cudaMemcpyDeviceToHost, s), "read stats");
    CK(cudaStreamSynchronize(s), "transport kernel");
    for (int k = 0; k < 8; ++k) stats->class_counts[k] = h[k];
    stats->steps = h[kStatSteps];
    stats->compton = h[kStatCompton];
    stats->rayleigh = h[kStatRayleigh];
    stats->photo = h[kStatPhoto];
    stats->binned = h[kStatBinned];
    stats->weight_sum = h[kStatWeight];
    stats->rng_blocks = h[kStatRng];
    stats->tries = h[kStatTries];
    stats->detected = h[kStatDetected];
    stats->atomics = h[kStatAtomics];
    stats->grid = last_grid;
    stats->block = block;
  }
  return PSC_OK;
}

int psc_simulate_batch(psc_ctx* ctx, const psc_sim_args* args, int32_t n, psc_stats* stats,
                       psc_stream stream) {
  return batch_impl(ctx, args, n, stats, stream, Sched{});
}

// The autotuner of batched launches.  Candidate schedules run on
// consecutive slices of every request's own histories (each slice a fixed
// fraction of each request's budget, so every probe sees the request mix),
// timed with events; the fastest runs the rest.  Every history is simulated
// exactly once into its request's accumulator, and the accumulators do not
// depend on the schedule (counter-based streams, integer sums), so the
// result equals psc_simulate_batch's bit for bit.  The choice is cached per
// request mix (the requests' scanner, phantom and LUT objects).
static const Sched kTuneCandidates[] = {
    {512, 0, 2, 65536}, {512, 0, 8, 65536}, {512, 0, 2, 16384}, {512, 0, 16, 8192},
    {256, 0, 2, 65536}, {256, 0, 8, 16384}};
constexpr int kTuneSlices = 48;  // a probe takes 1/48 of every request's histories

int psc_simulate_batch_tuned(psc_ctx* ctx, const psc_sim_args* args, int32_t n, psc_schedule* chosen,
                             psc_stream stream) {
  if (!ctx || (!args && n > 0) || n < 0) return fail(PSC_EINVAL, "NULL argument or negative count");
  for (int i = 0; i < n; ++i)
    if (args[i].lm_out || args[i].cls_out || args[i].key_out || args[i].q_out)
      return fail(PSC_EINVAL, "the tuned batch takes no per-history outputs");
  std::vector<std::tuple<int, int, int>> key;
  for (int i = 0; i < n; ++i) key.emplace_back(args[i].scanner, args[i].phantom, args[i].lut);
  std::sort(key.begin(), key.end());
  std::vector<psc_sim_args> rest(args, args + n);
  Sched best;
  double best_rate = 0.0;
  int probed = 0;
  auto cached = ctx->tuned.find(key);
  if (cached == ctx->tuned.end() && capturing((cudaStream_t)stream))
    return fail(PSC_EINVAL, "the autotuner's probes wait for the stream: tune this request mix outside a capture");
  if (cached != ctx->tuned.end()) {
    best = cached->second.first;
    best_rate = cached->second.second;
  } else {
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    int rc = PSC_OK;
    for (const Sched& c : kTuneCandidates) {
      std::vector<psc_sim_args> slice(rest);
      unsigned long long hist = 0;
      for (int i = 0; i < n; ++i) {
        const unsigned long long take = std::min<unsigned long long>(
            rest[i].n_histories, std::max<unsigned long long>(1024, args[i].n_histories / kTuneSlices));
        slice[i].n_histories = take;
        rest[i].first_history += take;
        rest[i].n_histories -= take;
        hist += take;
      }
      if (hist == 0) break;
      if ((rc = cudaEventRecord(e0, s) != cudaSuccess ? fail(PSC_EDEVICE, "event") : PSC_OK)) break;
      if ((rc = batch_impl(ctx, slice.data(), n, nullptr, stream, c))) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(PSC_EDEVICE, "probe timing");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = ms > 0.0f ? (double)hist / (ms * 1e-3) : 0.0;
      if (rate > best_rate) {
        best_rate = rate;
        best = c;
      }
      ++probed;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (probed == (int)(sizeof(kTuneCandidates) / sizeof(kTuneCandidates[0]))) ctx->tuned[key] = {best, best_rate};
  }
  if (chosen) {
    chosen->block = best.block;
    chosen->grid = best.grid;
    chosen->chunks_per_cta = best.chunks_per_cta;
    chosen->max_chunk = (int32_t)best.max_chunk;
    chosen->rate = best_rate;
    chosen->probed = probed;
  }
  return batch_impl(ctx, rest.data(), n, nullptr, stream, best);
}

int psc_simulate(psc_ctx* ctx, const psc_sim_args* a, psc_stats* stats, psc_stream stream) {
  if (!ctx || !a) return fail(PSC_EINVAL, "NULL argument");
  return psc_simulate_batch(ctx, a, 1, stats, stream);
}

// Copies of finished parts of the estimate to host memory, for
// psc_finalize_host: after each part is written on stream s, copy stream c
// waits for it and copies it.  One event per part, released when done.
struct HostCopy {
  double* host = nullptr;
  cudaStream_t c = nullptr;
};

static int copy_planes_2d(double* host, const double* dev, long long plane_elems, long long first_plane,
                          long long pitch_planes, long long rows, cudaStream_t c) {
  const size_t width = sizeof(double) * (size_t)plane_elems;
  const size_t pitch = width * (size_t)pitch_planes;
  const size_t off = (size_t)first_plane * (size_t)plane_elems;
  if (rows == 1) {
    CK(cudaMemcpyAsync(host + off, dev + off, width, cudaMemcpyDeviceToHost, c), "copy to host");
  } else if (pitch <= (size_t)INT32_MAX) {
    CK(cudaMemcpy2DAsync(host + off, pitch, dev + off, pitch, width, (size_t)rows, cudaMemcpyDeviceToHost, c),
       "copy to host");
  } else {
    for (long long r = 0; r < rows; ++r)
      CK(cudaMemcpyAsync(host + off + (size_t)r * pitch_planes * plane_elems, dev + off + (size_t)r * pitch_planes *
                         plane_elems, width, cudaMemcpyDeviceToHost, c), "copy to host");
  }
  return PSC_OK;
}

// stream c waits for the work enqueued on s so far
static int join(cudaStream_t c, cudaStream_t s) {
  if (c == s) return PSC_OK;
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  cudaError_t e = cudaEventRecord(ev, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c, ev, 0);
  cudaEventDestroy(ev);  // released once the wait is satisfied
  CK(e, "order the copy stream");
  return PSC_OK;
}

static int finalize_launches(psc_ctx* ctx, const psc_finalize_args* a, double* out, psc_stream stream, int divide,
                             const HostCopy* hc);

static int finalize_impl(psc_ctx* ctx, const psc_finalize_args* a, double* out, psc_stream stream, int divide,
                         const HostCopy* hc = nullptr) {
  const int rc = finalize_launches(ctx, a, out, stream, divide, hc);
  return rc ? rc : debug_check(ctx, (cudaStream_t)stream, "finalize");
}

static int finalize_launches(psc_ctx* ctx, const psc_finalize_args* a, double* out, psc_stream stream, int divide,
                             const HostCopy* hc) {
  if (!ctx || !a || !out) return fail(PSC_EINVAL, "NULL argument");
  GET(AccObj, acc, a->acc, kAccObj);
  GET(ScannerObj, sc, acc->scanner, kScannerObj);
  std::shared_ptr<SinoObj> sens, norm;
  if (a->sens) {
    sens = get<SinoObj>(ctx, a->sens, kSinoObj);
    if (!sens) return fail(PSC_ENOTFOUND, "no sinogram with id %d", (int)a->sens);
    if (sens->scanner != acc->scanner) return fail(PSC_EINVAL, "sensitivity sinogram belongs to another scanner");
  }
  if (a->norm) {
    norm = get<SinoObj>(ctx, a->norm, kSinoObj);
    if (!norm) return fail(PSC_ENOTFOUND, "no sinogram with id %d", (int)a->norm);
    if (norm->scanner != acc->scanner) return fail(PSC_EINVAL, "normalisation sinogram belongs to another scanner");
  }
  if (!std::isfinite(a->scale)) return fail(PSC_EINVAL, "scale must be finite");
  if (ctx->status_host && __atomic_exchange_n(ctx->status_host, 0, __ATOMIC_ACQ_REL))
    return fail(PSC_EDEVICE, "an earlier smoothing call on this context stopped: its shared-memory tile copies did "
                             "not complete within the bounded wait, so that estimate is incomplete");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool cap = capturing(s);
  FinParams p;
  std::memset(&p, 0, sizeof p);
  const psc_scanner_desc& d = sc->desc;
  p.acc = (const long long*)acc->data.p;
  p.out = out;
  p.sens = sens ? (const double*)sens->data.p : nullptr;
  p.sens32 = sens ? (const float*)sens->data32.p : nullptr;
  p.sens_per_lor = sens ? sens->per_lor : 0;
  p.c = std::ldexp(a->scale, -32);
  p.n_bins = sc->n_bins;
  p.n_rings = d.n_rings;
  p.V = d.n_crystals / 2;
  p.R = d.n_rad;
  p.T = d.n_tof;
  p.smooth = a->smooth ? 1 : 0;
  p.sens_first = a->sens_first ? 1 : 0;
  p.divide_acc = divide;
  p.dbg = (DebugRecord*)ctx->dbg.p;
  p.status = ctx->status_dev;
  if (a->seg_lo != a->seg_hi) {
    if (a->seg_lo < 0 || a->seg_hi > 2 * d.n_rings - 1 || a->seg_lo > a->seg_hi)
      return fail(PSC_EINVAL, "segment range [%d, %d) outside [0, %d)", (int)a->seg_lo, (int)a->seg_hi,
                  2 * d.n_rings - 1);
    p.seg_lo = a->seg_lo;
    p.seg_hi = a->seg_hi;
  }
  p.magic_T = p.T == 1 ? 0u : (unsigned)(((1ULL << 32) + p.T - 1) / p.T);
  if ((long long)p.V * p.R * p.T * p.T >= (1LL << 32))
    return fail(PSC_EOVERFLOW, "a sinogram plane is too large");
  const int nr = d.n_rings;
  const bool all_planes = p.seg_hi <= p.seg_lo;
  const int s_lo = all_planes ? 0 : p.seg_lo, s_hi = all_planes ? 2 * nr - 1 : p.seg_hi;
  const int n_planes = finalize_planes(p);
  const long long J = (long long)p.V * p.R * p.T;  // bins per plane
  auto seg_len = [&](int sg) { return nr - std::abs(sg - (nr - 1)); };
  // parts of the estimate copied as they finish: groups of whole segments of
  // about equal size (plane ranges when every plane is finalized without
  // smoothing), about kHostParts of them; a group's planes are the rows
  // ra (n + 1) + d of the layout
  constexpr int kHostParts = 8;
  auto for_groups = [&](auto&& run_group) -> int {
    int lo = s_lo, idx = 0;
    long long done = 0;
    for (int k = 1; k <= kHostParts && lo < s_hi; ++k) {
      const long long target = (long long)n_planes * k / kHostParts;
      int hi = lo, n_idx = 0;
      while (hi < s_hi && (done < target || hi == lo)) {
        done += seg_len(hi);
        n_idx += seg_len(hi);
        ++hi;
      }
      if (k == kHostParts)
        while (hi < s_hi) n_idx += seg_len(hi++);
      int rc = run_group(lo, hi, idx, idx + n_idx);
      if (!rc) rc = join(hc->c, (cudaStream_t)stream);
      for (int sg = lo; sg < hi && !rc; ++sg) {
        const int dd = sg - (nr - 1), ra0 = std::max(0, -dd);
        rc = copy_planes_2d(hc->host, out, J, (long long)ra0 * (nr + 1) + dd, nr + 1, seg_len(sg), hc->c);
      }
      if (rc) return rc;
      lo = hi;
      idx += n_idx;
    }
    return PSC_OK;
  };
  if (!p.smooth) {
    if (!hc) {
      CK(launch_finalize(p, ctx->sms, s), "finalize");
      return PSC_OK;
    }
    if (all_planes) {
      for (int k = 0; k < kHostParts; ++k) {
        const int lo = (int)((long long)n_planes * k / kHostParts), hi = (int)((long long)n_planes * (k + 1) / kHostParts);
        if (hi <= lo) continue;
        CK(launch_finalize_planes(p, lo, hi, ctx->sms, s), "finalize");
        int rc;
        if ((rc = join(hc->c, s))) return rc;
        // planes [lo, hi) are contiguous: one copy of (hi - lo) J elements at plane lo
        CK(cudaMemcpyAsync(hc->host + (size_t)lo * (size_t)J, out + (size_t)lo * (size_t)J,
                           sizeof(double) * (size_t)J * (size_t)(hi - lo), cudaMemcpyDeviceToHost, hc->c),
           "copy to host");
      }
      return PSC_OK;
    }
    return for_groups([&](int, int, int i_lo, int i_hi) -> int {
      CK(launch_finalize_planes(p, i_lo, i_hi, ctx->sms, s), "finalize");
      return PSC_OK;
    });
  }
  {
    const int rc = finalize_plan(p, a->sigma);
    if (rc) return rc;
  }
  if (norm) {
    p.norm = (const double*)norm->data.p;
    p.norm_per_lor = norm->per_lor;
    if (!norm->recip.p) {
      if (cap) return fail(PSC_EINVAL, "the normalisation's reciprocal is made outside a capture: run the call once first");
      int rc;
      if ((rc = dev_alloc(ctx, norm->recip, sizeof(double) * norm->n))) return rc;
      norm->bytes += norm->recip.bytes;
      CK(launch_reciprocal((const double*)norm->data.p, (double*)norm->recip.p, nullptr, norm->n, ctx->sms, s),
         "reciprocal");
    }
    p.rnorm = (const double*)norm->recip.p;
    p.norm32 = (const float*)norm->data32.p;
  }
  if (cap && hc && hc->c != s)
    return fail(PSC_EINVAL, "in a stream capture the copies to host memory run on the capturing stream");
  {
    std::lock_guard<std::mutex> lk(ctx->scratch_mu);
    const size_t need = sizeof(float) * (size_t)p.n_bins;
    if (ctx->scratch.bytes < need) {
      if (cap) return fail(PSC_EINVAL, "the smoothing scratch grows outside a capture: run the call once first");
      cudaStreamSynchronize(s);
      cudaDeviceSynchronize();
      if (ctx->scratch.p) {
        cudaFree(ctx->scratch.p);
        ctx->scratch.p = nullptr;
        ctx->scratch.bytes = 0;
      }
      cudaError_t e = cudaMalloc(&ctx->scratch.p, need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->scratch.p = nullptr;
        return fail(PSC_ENOMEM, "finalize scratch of %zu bytes: %s", need, cudaGetErrorString(e));
      }
      ctx->scratch.bytes = need;
    }
    p.scratch = (float*)ctx->scratch.p;
    if (!cap) CK(cudaStreamWaitEvent(s, ctx->scratch_done, 0), "order scratch users");
    if (!hc) {
      CK(launch_finalize(p, ctx->sms, s), "finalize");
    } else {
      // the axial pass in groups of whole segments, each copied when written
      CK(launch_smooth_front(p, s), "finalize");
      const int rc = for_groups([&](int lo, int hi, int, int) -> int {
        CK(launch_smooth_axial(p, lo, hi, s), "finalize");
        return PSC_OK;
      });
      if (rc) return rc;
    }
    if (!cap) CK(cudaEventRecord(ctx->scratch_done, s), "order scratch users");
  }
  return PSC_OK;
}

int psc_finalize(psc_ctx* ctx, const psc_finalize_args* a, double* out, psc_stream stream) {
  return finalize_impl(ctx, a, out, stream, 0);
}

int psc_finalize_host(psc_ctx* ctx, const psc_finalize_args* a, double* work, double* out_host, psc_stream stream,
                      psc_stream copy_stream) {
  if (!out_host) return fail(PSC_EINVAL, "out_host is NULL");
  HostCopy hc;
  hc.host = out_host;
  hc.c = (cudaStream_t)copy_stream;
  return finalize_impl(ctx, a, work, stream, 0, &hc);
}

int psc_norm_sinogram(psc_ctx* ctx, int32_t acc, const double* sigma, double* out, psc_stream stream) {
  if (!sigma) return fail(PSC_EINVAL, "sigma is NULL: the normalisation sinogram is a smoothed ratio");
  psc_finalize_args a;
  std::memset(&a, 0, sizeof a);
  a.acc = acc;
  a.smooth = 1;
  for (int i = 0; i < 3; ++i) a.sigma[i] = sigma[i];
  a.scale = 1.0;
  return finalize_impl(ctx, &a, out, stream, 1);
}

int psc_acc_span(psc_ctx* ctx, int32_t acc, int32_t span, int64_t* out, int64_t* out_planes, psc_stream stream) {
  if (!ctx) return fail(PSC_EINVAL, "ctx is NULL");
  GET(AccObj, a, acc, kAccObj);
  GET(ScannerObj, sc, a->scanner, kScannerObj);
  const psc_scanner_desc& d = sc->desc;
  if (span < 1 || !(span & 1)) return fail(PSC_EINVAL, "span %d must be odd and >= 1", (int)span);
  const int planes = span_planes(d.n_rings, span);
  if (out_planes) *out_planes = planes;
  if (!out) return PSC_OK;
  DeviceGuard g(ctx->device);
  CK(launch_span((const long long*)a->data.p, (long long*)out, d.n_rings, span,
                 (long long)(d.n_crystals / 2) * d.n_rad * d.n_tof, ctx->sms, (cudaStream_t)stream),
     "span mashing");
  return PSC_OK;
}

int psc_acc_mash(psc_ctx* ctx, int32_t acc, int32_t view_factor, int32_t tof_factor, int64_t* out,
                 psc_stream stream) {
  if (!ctx || !out) return fail(PSC_EINVAL, "NULL argument");
  GET(AccObj, a, acc, kAccObj);
  GET(ScannerObj, sc, a->scanner, kScannerObj);
  const psc_scanner_desc& d = sc->desc;
  const int V = d.n_crystals / 2;
  if (view_factor < 1 || tof_factor < 1 || V % view_factor || d.n_tof % tof_factor)
    return fail(PSC_EINVAL, "mashing factors (%d, %d) must divide %d views and %d TOF bins", view_factor, tof_factor,
                V, d.n_tof);
  DeviceGuard g(ctx->device);
  CK(launch_mash((const long long*)a->data.p, (long long*)out, d.n_rings * d.n_rings, V, d.n_rad, d.n_tof,
                 view_factor, tof_factor, (cudaStream_t)stream),
     "mash");
  return PSC_OK;
}

int psc_acc_rotate_sum(psc_ctx* ctx, int32_t acc, int32_t step, int32_t out_acc, psc_stream stream) {
  if (!ctx) return fail(PSC_EINVAL, "ctx is NULL");
  GET(AccObj, a, acc, kAccObj);
  GET(AccObj, o, out_acc, kAccObj);
  GET(ScannerObj, sc, a->scanner, kScannerObj);
  if (acc == out_acc) return fail(PSC_EINVAL, "the rotation sum needs a separate output accumulator");
  if (o->scanner != a->scanner) return fail(PSC_EINVAL, "output accumulator belongs to another scanner");
  const psc_scanner_desc& d = sc->desc;
  if (step < 1 || d.n_crystals % step) return fail(PSC_EINVAL, "step %d must divide %d crystals", step, d.n_crystals);
  if (d.n_rings > 255) return fail(PSC_EINVAL, "at most 255 rings");
  DeviceGuard g(ctx->device);
  CK(launch_rotate_sum((const long long*)a->data.p, (long long*)o->data.p, d.n_crystals, d.n_rings, d.n_rad,
                       d.n_tof, step, (cudaStream_t)stream),
     "rotation sum");
  return PSC_OK;
}

}  // extern "C"
