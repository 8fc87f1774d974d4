// server.cu -- continuous-batching request loop for scatter requests
// (the joint activity/scatter estimation of Sec. 2.3.3 issues one request
// per iteration: same phantom and attenuation, new activity image).
//
// A host thread owns the device work of all requests:
//   admission  waiting requests become active when an accumulator for their
//              scanner can be taken from the pool or allocated within the
//              context's memory budget (and, for a new activity image, when
//              no active request still uses that phantom);
//   epochs     one batched transport launch per epoch covers the next slice
//              of every active request, so requests that arrive while others
//              run join at the next epoch and share the GPU with them;
//   finalize   a request whose histories are all simulated is finalized on a
//              second stream, overlapping the next epoch's transport; its
//              accumulator returns to the pool when that work has completed.
// Each request's accumulator receives exactly its own histories, so its
// result is the same as when it runs alone.  Built on the public C ABI.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "psc.h"
#include "psc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { kWaiting = 0, kActive = 1, kFinalizing = 2, kDoneState = 3, kFailed = 4 };

struct Request {
  uint64_t ticket = 0;
  psc_request r{};
  std::vector<uint2> alias;      // alias table of the new activity image (empty: keep)
  uint64_t next = 0;             // histories already launched
  int32_t acc = 0;
  int state = kWaiting;
  int error = 0;
  std::string message;
  double t_submit = 0, t_start = 0, t_done = 0;
  cudaEvent_t fin = nullptr;
};

struct Server {
  psc_ctx* ctx = nullptr;
  psc_server_config cfg{};
  int device = 0;
  cudaStream_t sc = nullptr, sf = nullptr;  // transport / finalize streams
  cudaEvent_t epoch_ev[2] = {nullptr, nullptr};
  int epoch_i = 0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  Clock::time_point t0;
  std::deque<std::shared_ptr<Request>> waiting;
  std::vector<std::shared_ptr<Request>> active, finalizing;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::map<int32_t, std::vector<int32_t>> pool;  // scanner -> free accumulators

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  void fail(const std::shared_ptr<Request>& q, int code);
};

std::mutex g_servers_mu;
std::unordered_map<psc_ctx*, std::unique_ptr<Server>> g_servers;

Server* server_of(psc_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_servers_mu);
  auto it = g_servers.find(ctx);
  return it == g_servers.end() ? nullptr : it->second.get();
}

void Server::fail(const std::shared_ptr<Request>& q, int code) {
  q->state = kFailed;
  q->error = code;
  q->message = psc_last_error();
  q->t_done = now();
  if (q->acc) pool[q->r.scanner].push_back(q->acc);
  q->acc = 0;
}

void Server::run() {
  cudaSetDevice(device);
  for (;;) {
    // ---- take admissible requests off the queue (FIFO) ----
    std::vector<std::shared_ptr<Request>> cand;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (stop && waiting.empty() && active.empty() && finalizing.empty()) break;
      while (!waiting.empty() && (int)(active.size() + cand.size()) < cfg.max_active) {
        auto q = waiting.front();
        bool busy = false;
        if (!q->alias.empty()) {
          for (auto& a : active) busy |= a->r.phantom == q->r.phantom;
          for (auto& a : finalizing) busy |= a->r.phantom == q->r.phantom;
          for (auto& a : cand) busy |= a->r.phantom == q->r.phantom;
        }
        if (busy) break;
        waiting.pop_front();
        cand.push_back(q);
      }
    }
    // ---- admission: accumulator from the pool or the memory budget ----
    for (size_t i = 0; i < cand.size(); ++i) {
      auto& q = cand[i];
      int32_t acc = 0;
      auto& free_accs = pool[q->r.scanner];
      int rc = PSC_OK;
      if (!free_accs.empty()) {
        acc = free_accs.back();
        free_accs.pop_back();
      } else {
        rc = psc_acc_create(ctx, q->r.scanner, &acc);
        if (rc == PSC_ENOMEM && (!active.empty() || !finalizing.empty())) {
          // no memory until a running request completes: requeue in order
          std::lock_guard<std::mutex> lk(mu);
          for (size_t k = cand.size(); k > i; --k) waiting.push_front(cand[k - 1]);
          break;
        }
      }
      q->acc = acc;
      if (!rc && !q->alias.empty()) rc = psc::put_alias(ctx, q->r.phantom, q->alias.data(), (long long)q->alias.size());
      if (!rc) rc = psc_acc_zero(ctx, acc, sc);
      std::lock_guard<std::mutex> lk(mu);
      if (rc) {
        fail(q, rc);
        cv_done.notify_all();
        continue;
      }
      q->state = kActive;
      q->t_start = now();
      active.push_back(q);
    }
    // ---- one epoch over every active request ----
    if (!active.empty()) {
      const uint64_t quota = std::max<uint64_t>(cfg.min_slice, cfg.epoch_histories / active.size());
      std::vector<psc_sim_args> args;
      std::vector<std::shared_ptr<Request>> ending, still;
      for (auto& q : active) {
        const uint64_t k = std::min<uint64_t>(quota, q->r.n_histories - q->next);
        psc_sim_args a;
        std::memset(&a, 0, sizeof a);
        a.seed = q->r.seed;
        a.first_history = q->r.first_history + q->next;
        a.n_histories = k;
        a.scanner = q->r.scanner;
        a.phantom = q->r.phantom;
        a.lut = q->r.lut;
        a.acc = q->acc;
        a.bin_mask = PSC_BIN_SCATTER;
        args.push_back(a);
        q->next += k;
        (q->next >= q->r.n_histories ? ending : still).push_back(q);
      }
      // keep at most two epochs queued on the device
      cudaEvent_t ev = epoch_ev[epoch_i++ & 1];
      cudaEventSynchronize(ev);
      const int rc = psc_simulate_batch(ctx, args.data(), (int32_t)args.size(), nullptr, sc);
      if (rc) {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& q : active) fail(q, rc);
        active.clear();
        cv_done.notify_all();
        continue;
      }
      cudaEventRecord(ev, sc);
      for (auto& q : ending) {
        psc_finalize_args f;
        std::memset(&f, 0, sizeof f);
        f.acc = q->acc;
        f.sens = q->r.sens;
        f.norm = q->r.norm;
        f.smooth = q->r.smooth;
        std::memcpy(f.sigma, q->r.sigma, sizeof f.sigma);
        f.scale = q->r.scale;
        f.sens_first = q->r.sens_first;
        int frc = cudaStreamWaitEvent(sf, ev, 0) == cudaSuccess ? PSC_OK : PSC_EDEVICE;
        if (!frc) frc = psc_finalize(ctx, &f, q->r.out, sf);
        if (!frc && cudaEventRecord(q->fin, sf) != cudaSuccess) frc = PSC_EDEVICE;
        std::lock_guard<std::mutex> lk(mu);
        if (frc) {
          fail(q, frc);
          cv_done.notify_all();
          continue;
        }
        q->state = kFinalizing;
        finalizing.push_back(q);
      }
      active.swap(still);
    }
    // ---- completions ----
    for (size_t i = 0; i < finalizing.size();) {
      auto q = finalizing[i];
      const cudaError_t e = cudaEventQuery(q->fin);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      std::lock_guard<std::mutex> lk(mu);
      if (e == cudaSuccess) {
        q->state = kDoneState;
        q->t_done = now();
        pool[q->r.scanner].push_back(q->acc);
        q->acc = 0;
      } else {
        fail(q, PSC_EDEVICE);
      }
      finalizing.erase(finalizing.begin() + i);
      cv_done.notify_all();
    }
    if (active.empty()) {
      std::unique_lock<std::mutex> lk(mu);
      if (waiting.empty() || !finalizing.empty()) cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

}  // namespace

extern "C" {

int psc_server_start(psc_ctx* ctx, const psc_server_config* cfg) {
  if (!ctx || !cfg) return psc::psc_set_error(PSC_EINVAL, "NULL argument");
  if (cfg->max_active < 1 || cfg->epoch_histories < 1)
    return psc::psc_set_error(PSC_EINVAL, "max_active and epoch_histories must be >= 1");
  if (server_of(ctx)) return psc::psc_set_error(PSC_EINVAL, "a server already runs on this context");
  auto s = std::make_unique<Server>();
  s->ctx = ctx;
  s->cfg = *cfg;
  if (s->cfg.min_slice == 0) s->cfg.min_slice = 65536;
  cudaGetDevice(&s->device);
  if (cudaStreamCreateWithFlags(&s->sc, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->sf, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->epoch_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->epoch_ev[1], cudaEventDisableTiming) != cudaSuccess)
    return psc::psc_set_error(PSC_EDEVICE, "server streams/events");
  s->t0 = Clock::now();
  Server* raw = s.get();
  {
    std::lock_guard<std::mutex> lk(g_servers_mu);
    g_servers[ctx] = std::move(s);
  }
  raw->th = std::thread([raw] { raw->run(); });
  return PSC_OK;
}

int psc_server_stop(psc_ctx* ctx) {
  std::unique_ptr<Server> s;
  {
    std::lock_guard<std::mutex> lk(g_servers_mu);
    auto it = g_servers.find(ctx);
    if (it == g_servers.end()) return psc::psc_set_error(PSC_ENOTFOUND, "no server on this context");
    s = std::move(it->second);
    g_servers.erase(it);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->th.join();
  cudaStreamSynchronize(s->sc);
  cudaStreamSynchronize(s->sf);
  for (auto& kv : s->all)
    if (kv.second->fin) cudaEventDestroy(kv.second->fin);
  for (auto& kv : s->pool)
    for (int32_t a : kv.second) psc_unload(ctx, a);
  cudaEventDestroy(s->epoch_ev[0]);
  cudaEventDestroy(s->epoch_ev[1]);
  cudaStreamDestroy(s->sc);
  cudaStreamDestroy(s->sf);
  return PSC_OK;
}

int psc_submit(psc_ctx* ctx, const psc_request* r, uint64_t* ticket) {
  Server* s = server_of(ctx);
  if (!s) return psc::psc_set_error(PSC_ENOTFOUND, "no server on this context");
  if (!r || !ticket || !r->out) return psc::psc_set_error(PSC_EINVAL, "NULL argument");
  if (r->n_histories == 0 || r->first_history + r->n_histories < r->first_history)
    return psc::psc_set_error(PSC_EINVAL, "history range must be non-empty and not wrap");
  auto q = std::make_shared<Request>();
  q->r = *r;
  if (r->activity) {
    // the alias table is built now, on the caller's thread (the caller's
    // buffer may change before admission, and the server thread only uploads)
    const int64_t nv = psc_phantom_voxels(ctx, r->phantom);
    if (nv <= 0) return psc::psc_set_error(PSC_ENOTFOUND, "no phantom with id %d", (int)r->phantom);
    const int rc = psc::alias_table(r->activity, nv, q->alias);
    if (rc) return rc;
  }
  if (cudaEventCreateWithFlags(&q->fin, cudaEventDisableTiming) != cudaSuccess)
    return psc::psc_set_error(PSC_EDEVICE, "cudaEventCreate");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    s->waiting.push_back(q);
    s->all[q->ticket] = q;
    *ticket = q->ticket;
  }
  s->cv_work.notify_all();
  return PSC_OK;
}

int psc_poll(psc_ctx* ctx, uint64_t ticket, psc_request_status* st) {
  Server* s = server_of(ctx);
  if (!s) return psc::psc_set_error(PSC_ENOTFOUND, "no server on this context");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return psc::psc_set_error(PSC_ENOTFOUND, "unknown ticket");
  const auto& q = it->second;
  if (st) {
    st->state = q->state;
    st->error = q->error;
    st->t_submit = q->t_submit;
    st->t_start = q->t_start;
    st->t_done = q->t_done;
  }
  return PSC_OK;
}

int psc_wait(psc_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
  Server* s = server_of(ctx);
  if (!s) return psc::psc_set_error(PSC_ENOTFOUND, "no server on this context");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return psc::psc_set_error(PSC_ENOTFOUND, "unknown ticket");
  auto q = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us), [&] {
    return q->state == kDoneState || q->state == kFailed;
  });
  if (!ok) return psc::psc_set_error(PSC_ETIMEOUT, "request %llu not done within %lld us",
                                     (unsigned long long)ticket, (long long)timeout_us);
  if (q->state == kFailed) return psc::psc_set_error(q->error, "request failed: %s", q->message.c_str());
  return PSC_OK;
}

}  // extern "C"
