// server.cpp -- request server with continuous batching (gnss_server_*).
//
// The paper's deployment runs many instances of the receiver per cloud
// server and measures throughput as "effective running time" (Section 4),
// and it names fewer, larger GPU operations as the cure for the GPU's
// serialisation of small per-thread requests (Section 5, Listing 3b).  This
// server is that idea for one GPU: clients submit recordings at any time;
// a dispatcher thread admits queued requests while their device memory fits
// the budget, groups every admitted request into one batched launch
// (gnss_acquire_batch), and keeps several batches in flight on separate
// streams so that new requests overlap with running ones.
//
//   submit: copy the recording into a pinned host arena (the caller may free
//           its buffer on return); plans are created once per descriptor and
//           kept resident with their code spectra.
//   dispatch: FIFO admission by device bytes (recording + scratch + records),
//           one device allocation per batch, H2D copies, batched kernels,
//           D2H of the records, completion through cudaLaunchHostFunc.
//   poll / wait: results are handed out once and released.
//   admission bound (optional): a submission whose projected wait -- the work
//           queued and in flight ahead of it plus its own, over the
//           throughput achieved while busy -- exceeds max_queue_wait_ms is
//           refused with GNSS_EBUSY, so that latency past saturation stays
//           bounded instead of growing with the queue.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace gnss {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one pinned host buffer.
class PinnedArena {
 public:
  bool init(size_t bytes) {
    if (cudaHostAlloc(&base_, bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  ~PinnedArena() {
    if (base_) cudaFreeHost(base_);
  }
  unsigned char* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, left = it->second - bytes;
        free_.erase(it);
        if (left) free_[off + bytes] = left;
        used_[off] = bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(unsigned char* p) {
    if (!p) return;
    const size_t off = (size_t)(p - base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }

 private:
  unsigned char* base_ = nullptr;
  size_t size_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;
};

enum class St { Queued, Running, Done, Failed, Cancelled };

struct Req {
  uint64_t ticket = 0;
  gnss_plan_desc desc;
  size_t n_samples = 0;
  size_t rec_bytes = 0;
  unsigned char* staging = nullptr;  // pinned copy of the recording
  St state = St::Queued;
  bool cancel_requested = false;
  gnss_status status = GNSS_OK;
  std::string error;
  std::vector<gnss_detection> result;
  Clock::time_point t_submit, t_done;
  double work = 0.0;  // algorithmic FLOPs of the acquisition (admission bound)
};

struct Batch;

}  // namespace
}  // namespace gnss

struct gnss_server {
  gnss_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;  // dispatcher wake-ups and waiters
  std::deque<std::shared_ptr<gnss::Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<gnss::Req>> reqs;  // every request not yet handed out
  std::map<std::string, gnss_plan*> plans;
  gnss::PinnedArena arena;
  std::vector<cudaStream_t> streams;
  size_t next_stream = 0;
  size_t reserved = 0;    // device bytes of batches in flight
  int in_flight = 0;      // batches in flight
  uint64_t next_ticket = 1;
  bool stop = false;
  int inject_alloc_fail = -1;  // fail the k-th next device allocation (testing hook)
  // throughput while busy, for the admission bound: work completed and time
  // with at least one batch in flight, both weighted toward recent batches
  // (each completion scales the sums by kRateDecay); busy_mark is the start
  // of the busy time not yet added
  double work_in_flight = 0.0, work_done = 0.0, busy_s = 0.0;
  std::chrono::steady_clock::time_point busy_mark;
  gnss_server_stats stats;
  std::thread dispatcher;
};

namespace gnss {
namespace {

struct Batch {
  gnss_server* srv;
  std::vector<std::shared_ptr<Req>> reqs;
  size_t bytes = 0;
  double work = 0.0;  // sum of its requests' work
  void* dev = nullptr;
  gnss_detection* host_out = nullptr;  // pinned records of the whole batch (in the arena)
  std::vector<size_t> out_off;         // record offset per request
  std::vector<int> n_prn;
  cudaStream_t stream = nullptr;
  cudaError_t error = cudaSuccess;
};

size_t rec_bytes_of(uint32_t format, size_t n) { return format == GNSS_FMT_I8_IQ ? 2 * n : (n + 1) / 2; }
size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device bytes one request holds while in flight: recording, records,
// surfaces-free scratch of the batched kernels.
size_t device_need(const gnss_plan* plan, size_t n_samples) {
  const size_t L = (size_t)plan->desc.coh_ms * plan->N;
  size_t B = n_samples / L;
  if (plan->desc.noncoh && B > plan->desc.noncoh) B = plan->desc.noncoh;
  AcqShape s;
  memset(&s, 0, sizeof(s));
  s.N = plan->N;
  s.B = (int)B;
  s.D = plan->D;
  s.G = plan->G;
  s.C = plan->C;  // shared spectra (0: one per bin, the upper bound)
  s.P = plan->P;
  s.sets = plan->sets;
  return al256(rec_bytes_of(plan->desc.format, n_samples)) + al256(sizeof(gnss_detection) * plan->P) +
         scratch_layout(s).total + 1024;
}

// Algorithmic FLOPs of one acquisition (5 N log2 N per complex FFT, 6 per
// complex product): per (bin, block) the wipe-off and fold of L samples and a
// forward FFT, per (PRN, bin, block) the conj-multiply, IFFT, |.|^2 and sum.
double acquisition_work(const gnss_plan* plan, size_t n_samples) {
  const size_t L = (size_t)plan->desc.coh_ms * plan->N;
  size_t B = n_samples / L;
  if (plan->desc.noncoh && B > plan->desc.noncoh) B = plan->desc.noncoh;
  const double N = plan->N, lg = std::log2(N);
  return (double)plan->D * (double)B * (8.0 * (double)L + 5.0 * N * lg) +
         (double)plan->P * plan->D * (double)B * (5.0 * N * lg + 10.0 * N);
}

// Weight of the earlier batches in the throughput estimate, per completion
// (about the last 20 batches count).
constexpr double kRateDecay = 0.95;

// Achieved throughput (FLOP/s) while at least one batch was in flight,
// weighted toward recent batches; 0 before the first batch completes.
// Caller holds srv->mu.
double busy_rate(const gnss_server* srv, Clock::time_point now) {
  double t = srv->busy_s;
  if (srv->in_flight > 0) t += std::chrono::duration<double>(now - srv->busy_mark).count();
  return (srv->work_done > 0.0 && t > 0.0) ? srv->work_done / t : 0.0;
}

// A batch completed (caller holds srv->mu, in_flight still counts it).
void account_completion(gnss_server* srv, double work, Clock::time_point now) {
  srv->busy_s = kRateDecay * srv->busy_s + std::chrono::duration<double>(now - srv->busy_mark).count();
  srv->work_done = kRateDecay * srv->work_done + work;
  srv->busy_mark = now;
}

void CUDART_CB on_batch_done(void* arg) {
  Batch* b = static_cast<Batch*>(arg);
  gnss_server* srv = b->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    const auto now = Clock::now();
    for (size_t k = 0; k < b->reqs.size(); ++k) {
      Req& r = *b->reqs[k];
      srv->arena.release(r.staging);
      r.staging = nullptr;
      if (r.cancel_requested) {
        r.state = St::Cancelled;
        r.status = GNSS_ECANCELLED;
      } else {
        r.result.assign(b->host_out + b->out_off[k], b->host_out + b->out_off[k] + b->n_prn[k]);
        r.state = St::Done;
        r.status = GNSS_OK;
        for (const gnss_detection& d : r.result)
          if (d.flags & GNSS_DET_TIMEOUTS) r.status = GNSS_ETIMEOUT;  // records kept, call reported
        if (r.status == GNSS_OK) srv->stats.completed++;
        else srv->stats.failed++;
      }
      r.t_done = now;
    }
    srv->arena.release(reinterpret_cast<unsigned char*>(b->host_out));
    srv->reserved -= b->bytes;
    srv->work_in_flight -= b->work;
    account_completion(srv, b->work, now);
    srv->in_flight--;
  }
  srv->cv.notify_all();
  delete b;
}

void fail_requests(gnss_server* srv, std::vector<std::shared_ptr<Req>>& rs, gnss_status st, const std::string& msg) {
  // caller holds srv->mu
  for (auto& r : rs) {
    srv->arena.release(r->staging);
    r->staging = nullptr;
    r->state = St::Failed;
    r->status = st;
    r->error = msg;
    r->t_done = Clock::now();
    srv->stats.failed++;
  }
}

std::string plan_key(const gnss_plan_desc& d) { return std::string(reinterpret_cast<const char*>(&d), sizeof(d)); }

gnss_plan* find_plan(gnss_server* srv, const gnss_plan_desc& d) {
  // caller holds srv->mu
  auto it = srv->plans.find(plan_key(d));
  return it == srv->plans.end() ? nullptr : it->second;
}

// Create the plans that the first max_batch queued requests still lack.  No
// CUDA call may run under srv->mu: plan creation allocates and synchronises,
// which waits for streams whose completion callbacks take srv->mu.  So the
// lock is released around the creation.  Returns true when it created (or
// failed to create) anything, i.e. when the queue must be looked at again.
bool create_missing_plans(gnss_server* srv, std::unique_lock<std::mutex>& lk) {
  std::vector<gnss_plan_desc> missing;
  size_t seen = 0;
  for (auto& r : srv->queue) {
    if (seen++ >= srv->cfg.max_batch) break;
    if (find_plan(srv, r->desc)) continue;
    bool dup = false;
    for (auto& m : missing) dup = dup || plan_key(m) == plan_key(r->desc);
    if (!dup) missing.push_back(r->desc);
  }
  if (missing.empty()) return false;
  std::vector<gnss_plan*> made(missing.size(), nullptr);
  std::vector<gnss_status> st(missing.size(), GNSS_OK);
  std::vector<std::string> err(missing.size());
  lk.unlock();
  for (size_t k = 0; k < missing.size(); ++k) {
    st[k] = gnss_plan_create(&missing[k], &made[k]);
    if (st[k] != GNSS_OK) err[k] = gnss_last_error();
  }
  lk.lock();
  for (size_t k = 0; k < missing.size(); ++k) {
    if (st[k] == GNSS_OK) {
      srv->plans[plan_key(missing[k])] = made[k];
      continue;
    }
    std::vector<std::shared_ptr<Req>> bad;
    for (auto it = srv->queue.begin(); it != srv->queue.end();) {
      if (plan_key((*it)->desc) == plan_key(missing[k])) {
        bad.push_back(*it);
        it = srv->queue.erase(it);
      } else {
        ++it;
      }
    }
    fail_requests(srv, bad, st[k], "plan creation failed: " + err[k]);
  }
  srv->cv.notify_all();
  return true;
}

// Dispatcher: admit, launch, repeat until the server stops.
void dispatch_loop(gnss_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    // queue timeout (watchdog for requests that wait too long to be admitted)
    if (srv->cfg.queue_timeout_ms) {
      const auto now = Clock::now();
      for (auto it = srv->queue.begin(); it != srv->queue.end();) {
        if (now - (*it)->t_submit > std::chrono::milliseconds(srv->cfg.queue_timeout_ms)) {
          std::vector<std::shared_ptr<Req>> one{*it};
          fail_requests(srv, one, GNSS_ETIMEOUT, "request waited longer than the queue timeout");
          it = srv->queue.erase(it);
          srv->cv.notify_all();
        } else {
          ++it;
        }
      }
    }
    if (srv->queue.empty() || srv->in_flight >= (int)srv->streams.size() * 2) {
      srv->cv.wait_for(lk, std::chrono::milliseconds(srv->cfg.queue_timeout_ms ? 5 : 50));
      continue;
    }
    if (create_missing_plans(srv, lk)) continue;
    // admit FIFO while memory fits (every plan needed exists now)
    Batch* b = new Batch;
    b->srv = srv;
    std::vector<gnss_plan*> plans;
    while (!srv->queue.empty() && b->reqs.size() < srv->cfg.max_batch) {
      std::shared_ptr<Req> r = srv->queue.front();
      gnss_plan* plan = find_plan(srv, r->desc);
      if (!plan) break;  // beyond the section whose plans were made; next round
      const size_t need = device_need(plan, r->n_samples);
      if (srv->reserved + b->bytes + need > srv->cfg.device_mem_budget) break;
      b->bytes += need;
      b->work += r->work;
      b->reqs.push_back(r);
      plans.push_back(plan);
      srv->queue.pop_front();
    }
    if (b->reqs.empty()) {  // head does not fit until running batches finish
      delete b;
      srv->cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // pinned records of the batch
    size_t n_rec = 0;
    for (auto* p : plans) n_rec += p->P;
    b->host_out = reinterpret_cast<gnss_detection*>(srv->arena.alloc(sizeof(gnss_detection) * n_rec));
    if (!b->host_out) {  // host arena full: put the requests back and wait
      for (auto it = b->reqs.rbegin(); it != b->reqs.rend(); ++it) srv->queue.push_front(*it);
      delete b;
      srv->cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    for (auto& r : b->reqs) r->state = St::Running;
    srv->reserved += b->bytes;
    srv->work_in_flight += b->work;
    if (srv->in_flight++ == 0) srv->busy_mark = Clock::now();
    srv->stats.batches++;
    b->stream = srv->streams[srv->next_stream++ % srv->streams.size()];
    const bool inject = srv->inject_alloc_fail == 0;
    if (srv->inject_alloc_fail >= 0) srv->inject_alloc_fail--;
    lk.unlock();

    // --- device work, outside the lock ---
    cudaStream_t st = b->stream;
    cudaError_t e = inject ? cudaErrorMemoryAllocation : cudaSuccess;
    size_t rec_total = 0;
    for (size_t k = 0; k < b->reqs.size(); ++k) rec_total += al256(b->reqs[k]->rec_bytes) + al256(sizeof(gnss_detection) * plans[k]->P);
    char* dev = nullptr;
    if (e == cudaSuccess && scratch_alloc(srv->device, rec_total, st, (void**)&dev) != GNSS_OK) {
      e = cudaErrorMemoryAllocation;
      dev = nullptr;
    }
    std::vector<gnss_request> gr(b->reqs.size());
    size_t off = 0, rec_off = 0;
    for (size_t k = 0; k < b->reqs.size() && e == cudaSuccess; ++k) {
      Req& r = *b->reqs[k];
      char* d_smp = dev + off;
      off += al256(r.rec_bytes);
      gnss_detection* d_out = reinterpret_cast<gnss_detection*>(dev + off);
      off += al256(sizeof(gnss_detection) * plans[k]->P);
      e = cudaMemcpyAsync(d_smp, r.staging, r.rec_bytes, cudaMemcpyHostToDevice, st);
      gr[k].plan = plans[k];
      gr[k].samples_dev = d_smp;
      gr[k].n_samples = r.n_samples;
      gr[k].out_dev = d_out;
      gr[k].surface_dev = nullptr;
      b->out_off.push_back(rec_off);
      b->n_prn.push_back(plans[k]->P);
      rec_off += plans[k]->P;
    }
    gnss_status bst = GNSS_OK;
    std::string bmsg;
    if (e == cudaSuccess) {
      bst = gnss_acquire_batch(gr.data(), gr.size(), srv->cfg.device_mem_budget, st);
      if (bst != GNSS_OK) bmsg = gnss_last_error();
    }
    for (size_t k = 0; k < gr.size() && e == cudaSuccess && bst == GNSS_OK; ++k)
      e = cudaMemcpyAsync(b->host_out + b->out_off[k], gr[k].out_dev, sizeof(gnss_detection) * b->n_prn[k],
                          cudaMemcpyDeviceToHost, st);
    if (dev) cudaFreeAsync(dev, st);
    if (e == cudaSuccess && bst == GNSS_OK) e = cudaLaunchHostFunc(st, on_batch_done, b);
    lk.lock();
    if (e != cudaSuccess || bst != GNSS_OK) {
      // the batch never reached the completion callback: release it here
      cudaGetLastError();
      const gnss_status fs = bst != GNSS_OK ? bst : (e == cudaErrorMemoryAllocation ? GNSS_ENOMEM : GNSS_ECUDA);
      const std::string msg = bst != GNSS_OK ? bmsg : std::string(cudaGetErrorString(e));
      lk.unlock();
      cudaStreamSynchronize(st);  // copies that did start read the staging buffers
      lk.lock();
      fail_requests(srv, b->reqs, fs, msg);
      srv->arena.release(reinterpret_cast<unsigned char*>(b->host_out));
      srv->reserved -= b->bytes;
      srv->work_in_flight -= b->work;
      account_completion(srv, 0.0, Clock::now());  // its busy time, no work
      srv->in_flight--;
      delete b;
      srv->cv.notify_all();
    }
  }
}

void fill_result(Req& r, gnss_detection* out, size_t cap, size_t* n) {
  const size_t k = r.result.size() < cap ? r.result.size() : cap;
  if (out && k) memcpy(out, r.result.data(), k * sizeof(gnss_detection));
  if (n) *n = r.result.size();
}

}  // namespace
}  // namespace gnss

using namespace gnss;

extern "C" {

gnss_status gnss_server_create(const gnss_server_config* cfg, gnss_server** out) {
  if (!out) return fail_status(GNSS_EINVAL, "NULL argument");
  *out = nullptr;
  std::unique_ptr<gnss_server> s(new (std::nothrow) gnss_server);
  if (!s) return fail_status(GNSS_ENOMEM, "host allocation failed");
  memset(&s->cfg, 0, sizeof(s->cfg));
  if (cfg) s->cfg = *cfg;
  if (!s->cfg.device_mem_budget) s->cfg.device_mem_budget = (size_t)16 << 30;
  if (!s->cfg.host_staging_bytes) s->cfg.host_staging_bytes = (size_t)1 << 30;
  if (!s->cfg.max_batch) s->cfg.max_batch = 64;
  if (!s->cfg.streams) s->cfg.streams = 2;
  if (s->cfg.streams > 16) return fail_status(GNSS_EINVAL, "at most 16 streams");
  memset(&s->stats, 0, sizeof(s->stats));
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (!s->arena.init(s->cfg.host_staging_bytes)) return fail_status(GNSS_ENOMEM, "pinned host staging allocation failed");
  for (uint32_t k = 0; k < s->cfg.streams; ++k) {
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      return cuda_status(e, "cudaStreamCreate");
    }
    s->streams.push_back(st);
  }
  gnss_server* raw = s.release();
  raw->dispatcher = std::thread(dispatch_loop, raw);
  *out = raw;
  return GNSS_OK;
}

gnss_status gnss_server_destroy(gnss_server* srv) {
  if (!srv) return GNSS_OK;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    // fail what is still queued, let running batches finish
    std::vector<std::shared_ptr<Req>> q(srv->queue.begin(), srv->queue.end());
    fail_requests(srv, q, GNSS_ECANCELLED, "server destroyed");
    srv->queue.clear();
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->dispatcher.joinable()) srv->dispatcher.join();
  for (auto st : srv->streams) cudaStreamSynchronize(st);
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv.wait(lk, [&] { return srv->in_flight == 0; });
  }
  for (auto st : srv->streams) cudaStreamDestroy(st);
  for (auto& kv : srv->plans) gnss_plan_destroy(kv.second);
  delete srv;
  return GNSS_OK;
}

gnss_status gnss_submit(gnss_server* srv, const gnss_plan_desc* desc, const void* host_samples, size_t n_samples,
                        uint64_t* ticket) {
  if (!srv || !desc || !host_samples || !ticket) return fail_status(GNSS_EINVAL, "NULL argument");
  double work = 0.0;
  if (desc->flags & GNSS_SECOND_WHOLE) return fail_status(GNSS_EINVAL, "GNSS_SECOND_WHOLE needs surfaces; not served");
  if (desc->fs_hz == 0 || desc->fs_hz % 1000 || !supported_fft_size((int)(desc->fs_hz / 1000)) || desc->coh_ms < 1 ||
      desc->n_dopp < 1 || desc->n_dopp > 100000 || desc->format > GNSS_FMT_2BIT_IQ || (desc->prn_mask & 0xFFFFFFFFull) == 0 ||
      (desc->prn_mask >> 32))
    return fail_status(GNSS_EINVAL, "invalid descriptor");
  const size_t N = desc->fs_hz / 1000;
  if (n_samples < (size_t)desc->coh_ms * N) return fail_status(GNSS_EINVAL, "n_samples is shorter than one coherent block");
  // a request larger than the whole device budget could never be admitted
  {
    gnss_plan probe;
    memset(&probe, 0, sizeof(probe));
    probe.desc = *desc;
    probe.N = (int)N;
    probe.D = (int)desc->n_dopp;
    std::vector<int> group, gkey, cls;
    probe.G = fold_groups(*desc, group, gkey);  // the plan's own fold groups and spectrum classes
    probe.C = (desc->flags & GNSS_CODE_DOPPLER) ? 0 : spectrum_classes(*desc, group, cls);
    if (probe.C >= probe.D) probe.C = 0;
    probe.P = __builtin_popcountll(desc->prn_mask);
    probe.sets = (desc->flags & GNSS_HALF_BIT) ? 2 : 1;
    if (device_need(&probe, n_samples) > srv->cfg.device_mem_budget)
      return fail_status(GNSS_EBUSY, "request needs more device memory than the server budget");
    work = acquisition_work(&probe, n_samples);
  }
  auto r = std::make_shared<Req>();
  r->desc = *desc;
  r->n_samples = n_samples;
  r->rec_bytes = rec_bytes_of(desc->format, n_samples);
  r->work = work;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (srv->stop) return fail_status(GNSS_ECANCELLED, "server is shutting down");
  if (srv->cfg.max_queue_wait_ms) {
    // projected wait: the work queued and in flight ahead of this request,
    // plus its own, at the throughput achieved while busy
    const double rate = busy_rate(srv, Clock::now());
    if (rate > 0.0) {
      double ahead = srv->work_in_flight + work;
      for (const auto& q : srv->queue) ahead += q->work;
      const double wait_ms = 1e3 * ahead / rate;
      if (wait_ms > (double)srv->cfg.max_queue_wait_ms) {
        if (srv->stats.refused < 0xFFFFFFFFu) srv->stats.refused++;
        return fail_status(GNSS_EBUSY, "projected wait " + std::to_string((long long)wait_ms) +
                                           " ms exceeds the admission bound of " +
                                           std::to_string(srv->cfg.max_queue_wait_ms) + " ms");
      }
    }
  }
  r->staging = srv->arena.alloc(r->rec_bytes);
  if (!r->staging) return fail_status(GNSS_EBUSY, "host staging full: too many queued recordings");
  memcpy(r->staging, host_samples, r->rec_bytes);
  r->ticket = srv->next_ticket++;
  r->t_submit = Clock::now();
  srv->reqs[r->ticket] = r;
  srv->queue.push_back(r);
  srv->stats.submitted++;
  *ticket = r->ticket;
  lk.unlock();
  srv->cv.notify_all();
  return GNSS_OK;
}

static gnss_status take_result(gnss_server* srv, uint64_t ticket, gnss_detection* out, size_t cap, size_t* n,
                               std::unique_lock<std::mutex>& lk, bool* pending) {
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail_status(GNSS_EINVAL, "unknown ticket");
  Req& r = *it->second;
  *pending = (r.state == St::Queued || r.state == St::Running);
  if (*pending) return GNSS_EAGAIN;
  gnss_status st = r.status;
  if (r.state == St::Done) fill_result(r, out, cap, n);
  else if (!r.error.empty()) set_error(r.error);
  srv->reqs.erase(it);
  (void)lk;
  return st;
}

gnss_status gnss_poll(gnss_server* srv, uint64_t ticket, gnss_detection* out, size_t cap, size_t* n) {
  if (!srv) return fail_status(GNSS_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  bool pending = false;
  return take_result(srv, ticket, out, cap, n, lk, &pending);
}

gnss_status gnss_wait(gnss_server* srv, uint64_t ticket, uint32_t timeout_ms, gnss_detection* out, size_t cap,
                      size_t* n) {
  if (!srv) return fail_status(GNSS_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    bool pending = false;
    gnss_status st = take_result(srv, ticket, out, cap, n, lk, &pending);
    if (!pending) return st;
    if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      st = take_result(srv, ticket, out, cap, n, lk, &pending);
      if (!pending) return st;
      return fail_status(GNSS_ETIMEOUT, "request not finished within the wait time");
    }
  }
}

gnss_status gnss_cancel(gnss_server* srv, uint64_t ticket) {
  if (!srv) return fail_status(GNSS_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail_status(GNSS_EINVAL, "unknown ticket");
  Req& r = *it->second;
  if (r.state == St::Queued) {
    for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
      if ((*q)->ticket == ticket) {
        srv->queue.erase(q);
        break;
      }
    srv->arena.release(r.staging);
    r.staging = nullptr;
    r.state = St::Cancelled;
    r.status = GNSS_ECANCELLED;
  } else if (r.state == St::Running) {
    r.cancel_requested = true;  // results are discarded when its batch completes
  }
  lk.unlock();
  srv->cv.notify_all();
  return GNSS_OK;
}

gnss_status gnss_server_get_stats(gnss_server* srv, gnss_server_stats* out) {
  if (!srv || !out) return fail_status(GNSS_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->stats;
  out->queued = srv->queue.size();
  out->batches_in_flight = (uint32_t)srv->in_flight;
  out->device_bytes_reserved = srv->reserved;
  return GNSS_OK;
}

gnss_status gnss_server_inject_alloc_failure(gnss_server* srv, int k) {
  if (!srv) return fail_status(GNSS_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->inject_alloc_fail = k;
  return GNSS_OK;
}

}  // extern "C"
