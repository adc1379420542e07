// Serving loop: continuous batching of encode/decode requests on one GPU.
//
// Callers submit jobs (ec_server_submit) from any thread.  A request is
// admitted only while the block bytes of all admitted, unfinished requests
// stay within an HBM budget; otherwise EC_EBUSY tells the caller to retry.
// One scheduler thread forms a batch from every request that arrived while
// earlier batches were on the GPU, writes its stripe descriptors and block
// table into the pinned staging of a free slot, copies them to the slot's
// device tables and launches the batched pipeline (one persistent launch
// per compiled module, the dense bitmatrix executor for programs without one) on the
// slot's stream.  Several slots are in flight at once, so their work
// overlaps on the device; a slot returns to the pool when its completion
// event fires, which also timestamps every request in it (latency =
// submission to observed completion) and frees its admitted bytes.  No
// device memory is allocated per batch.
//
// Every slot has its own status word in host memory that the GPU writes
// directly (mapped pinned memory), cleared before each dispatch: a bounded
// wait of the slot's kernels that times out sets it, and the scheduler reads
// it when the slot's event fires, so every request of that batch completes
// with EC_ETIMEOUT (its outputs are incomplete) without a copy on the
// latency path.  A dispatch that fails completes its requests with the
// failure (after the work it did enqueue has finished) and returns their
// admitted bytes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_set>
#include <tuple>
#include <vector>

#include "internal.h"

using xorec::Program;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
  uint64_t ticket = 0;
  Program* prog = nullptr;
  void* mod = nullptr;          // compiled module that runs it, or nullptr = the dense executor
  std::vector<uint64_t> ptrs;
  long long S = 0, tiles = 0;
  int T = 0;                    // tile bytes per strip its items were counted in
  size_t bytes = 0;
  long long bytes_in = 0, bytes_out = 0;
  Clock::time_point t0;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Req> reqs;
  int* h_status = nullptr;      // the slot's status word (mapped pinned host memory)
  int* d_status = nullptr;      // the same word as the kernels address it
  int fail_status = EC_OK;      // the dispatch failed after enqueuing work: the
                                // requests complete with this status
  // one device table per slot and its pinned staging copy, laid out per
  // dispatch as [work-queue heads][stripe descriptors][block pointers], so
  // that one copy carries a whole batch's tables
  xk::u8* d_tab = nullptr;
  xk::u8* h_tab = nullptr;
  size_t cap = 0;   // bytes
};

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

struct ec_server {
  int device = -1;
  size_t budget = 0;
  int max_batch = 0;
  int chunk = 2;
  std::chrono::microseconds idle_spin{1000};
  xorec::DeviceInfo di;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> pending;
  std::atomic<size_t> n_pending{0};   // pending.size(), readable without the lock
  size_t admitted = 0;
  std::vector<Slot> slots;
  struct Done {
    uint64_t ticket;
    double latency_us;
    int status;
  };
  std::vector<Done> done;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  int error = EC_OK;
  std::thread th;
  ec_server_stats stats{};
  // launch shapes by (module, max_in, max_slots, dense words, dense form)
  std::map<std::tuple<void*, int, int, int, int>, std::pair<size_t, int>> shapes;
  // background compilation of programs that arrive without a compiled module
  bool background_compile = true;
  std::thread compiler;
  std::mutex cmu;
  std::condition_variable ccv;
  std::vector<std::pair<ec_plan*, Program*>> to_compile;
  std::unordered_set<Program*> queued;
  bool cstop = false;
};

namespace {

void free_slot(Slot& s) {
  if (s.st) cudaStreamDestroy(s.st);
  if (s.done) cudaEventDestroy(s.done);
  if (s.d_tab) cudaFree(s.d_tab);
  if (s.h_tab) cudaFreeHost(s.h_tab);
  if (s.h_status) cudaFreeHost(s.h_status);
  s = Slot();
}

// The slot's status word: pinned host memory mapped into the device's
// address space, so kernels write it directly and the host reads it.
bool alloc_status(Slot& s) {
  if (xorec::host_malloc_mapped(&s.h_status, 64) != cudaSuccess) {
    cudaGetLastError();
    s.h_status = nullptr;
    return false;
  }
  *reinterpret_cast<volatile int*>(s.h_status) = 0;
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&s.d_status), s.h_status, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Capacity of the slot's table (bytes); contents are rewritten per dispatch.
bool grow_table(Slot& s, size_t need) {
  if (need <= s.cap) return true;
  const size_t cap = std::max(need, 2 * s.cap);
  if (s.d_tab) cudaFree(s.d_tab);
  if (s.h_tab) cudaFreeHost(s.h_tab);
  s.d_tab = nullptr;
  s.h_tab = nullptr;
  s.cap = 0;
  if (xorec::dev_malloc(&s.d_tab, cap) != cudaSuccess ||
      xorec::host_malloc_pinned(&s.h_tab, cap) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s.cap = cap;
  return true;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Launch one batch of requests on a free slot.  On success the requests
// move into the slot.  On failure *enqueued tells whether some of their
// work is already on the slot's stream.
ec_status dispatch(ec_server* sv, Slot& sl, std::vector<Req>& reqs, bool* enqueued) {
  *enqueued = false;
  xorec::TraceRange trace_("xorec serve dispatch");
  // group by launch target: compiled module of this block size, or the dense
  // executor (by the tile its items were counted in)
  auto target = [&](const Req& r) { return std::make_pair(r.mod, r.T); };
  std::stable_sort(reqs.begin(), reqs.end(),
                   [&](const Req& a, const Req& b) { return target(a) < target(b); });
  size_t n_blocks = 0, n_launches = 0;
  for (size_t i = 0; i < reqs.size(); ++i) {
    n_blocks += reqs[i].ptrs.size();
    if (i == 0 || target(reqs[i]) != target(reqs[i - 1])) ++n_launches;
  }
  const int dense_form = xorec::dense_form();
  const size_t desc_off = align_up(n_launches * sizeof(xk::u64), 64);
  const size_t block_off = desc_off + reqs.size() * sizeof(xk::StripeDesc);
  const size_t bytes = block_off + n_blocks * sizeof(xk::u64);
  if (!grow_table(sl, bytes)) return fail(EC_ENOMEM, "allocation of a serving slot's table failed");
  std::memset(sl.h_tab, 0, n_launches * sizeof(xk::u64));   // work-queue heads
  auto* h_descs = reinterpret_cast<xk::StripeDesc*>(sl.h_tab + desc_off);
  auto* h_blocks = reinterpret_cast<xk::u64*>(sl.h_tab + block_off);
  auto* d_queues = reinterpret_cast<xk::u64*>(sl.d_tab);
  auto* d_descs = reinterpret_cast<xk::StripeDesc*>(sl.d_tab + desc_off);
  auto* d_blocks = reinterpret_cast<xk::u64*>(sl.d_tab + block_off);
  struct L { void* mod; int threads, T, begin, n; long long items; int max_in, max_slots; };
  std::vector<L> launches;
  size_t off = 0;
  for (size_t i = 0; i < reqs.size(); ++i) {
    const Req& r = reqs[i];
    void* mod = r.mod;
    if (launches.empty() || launches.back().mod != mod || launches.back().T != r.T)
      launches.push_back(L{mod, xorec::launch_threads(mod), r.T, static_cast<int>(i), 0, 0, 0, 0});
    L& l = launches.back();
    xk::StripeDesc& d = h_descs[i];
    std::memset(&d, 0, sizeof(d));
    d.blocks = d_blocks + off;
    d.S = r.S;
    d.item_base = l.items;
    d.n_inblk = r.prog->n_in / 8;
    d.n_outblk = r.prog->n_out / 8;
    d.prog = r.prog->mod_index;
    d.code = r.prog->d_code;
    d.code_len = static_cast<int>(r.prog->chunks.size() / 8);
    d.n_slots = r.prog->interp_slots;
    std::memcpy(h_blocks + off, r.ptrs.data(), r.ptrs.size() * sizeof(xk::u64));
    off += r.ptrs.size();
    l.n += 1;
    l.items += r.tiles;
    l.max_in = std::max(l.max_in, r.prog->n_in);
    if (!mod) l.max_slots = std::max(l.max_slots, r.prog->interp_slots);
  }
  // the slot is free: none of its kernels can write the word now
  *reinterpret_cast<volatile int*>(sl.h_status) = 0;
  if (cudaMemcpyAsync(sl.d_tab, sl.h_tab, bytes, cudaMemcpyHostToDevice, sl.st) != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "copy of a serving slot's table failed");
  }
  *enqueued = true;
  if (xorec::take_injected_timeout() &&
      !xorec::launch_selftest_wait_to(sl.st, sv->di.status, sl.d_status))
    return EC_ECUDA;
  for (size_t li = 0; li < launches.size(); ++li) {
    const L& l = launches[li];
    const int dense_w = l.T / (4 * xorec::kDenseThreads);
    auto key = std::make_tuple(l.mod, l.max_in, l.max_slots, dense_w, dense_form);
    auto it = sv->shapes.find(key);
    if (it == sv->shapes.end()) {
      size_t smem = 0;
      int per_sm = 1;
      if (!xorec::batch_launch_shape(l.mod, false, l.max_in, l.max_slots, l.threads,
                                     sv->di.smem_optin, &smem, &per_sm, dense_w, dense_form))
        return fail(EC_ENOTSUP, "a program needs more shared memory than one CTA can hold");
      it = sv->shapes.emplace(key, std::make_pair(smem, per_sm)).first;
    }
    xk::BatchParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.stripes = d_descs + l.begin;
    bp.n_stripes = l.n;
    bp.chunk = sv->chunk;
    bp.queue = d_queues + li;
    xorec::set_ranges(&bp, l.items, 1);
    bp.n_items = l.items;
    bp.T = l.T;
    bp.max_in = l.max_in;
    bp.status = sv->di.status;
    bp.local_status = sl.d_status;
    const long long full = static_cast<long long>(sv->di.sms) * it->second.second;
    const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(full, l.items)));
    const bool ok = xorec::batch_launch(l.mod, false, bp, l.threads, grid, it->second.first,
                                        sl.st, dense_w, dense_form);
    if (!ok) return EC_ECUDA;
  }
  if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "cudaEventRecord on a serving slot failed");
  }
  sl.reqs = std::move(reqs);
  sl.fail_status = EC_OK;
  sl.busy = true;
  return EC_OK;
}

// Return requests to their callers with `status` (caller holds sv->mu).
void complete_locked(ec_server* sv, const std::vector<Req>& reqs, int status,
                     Clock::time_point now) {
  for (const Req& r : reqs) {
    sv->done.push_back({r.ticket, std::chrono::duration<double, std::micro>(now - r.t0).count(),
                        status});
    sv->admitted -= r.bytes;
    sv->stats.completed += 1;
    if (status == EC_OK) {
      sv->stats.bytes_in += r.bytes_in;
      sv->stats.bytes_out += r.bytes_out;
    } else {
      sv->stats.failed += 1;
    }
  }
}

void scheduler(ec_server* sv) {
  cudaSetDevice(sv->device);
  auto last_active = Clock::now();
  for (;;) {
    bool worked = false;
    for (Slot& sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const auto now = Clock::now();
      int status = sl.fail_status;
      if (q != cudaSuccess) {
        cudaGetLastError();
        status = EC_ECUDA;
      } else if (status == EC_OK &&
                 *reinterpret_cast<volatile int*>(sl.h_status) == xk::XK_STATUS_TIMEOUT) {
        status = EC_ETIMEOUT;
      }
      std::lock_guard<std::mutex> lk(sv->mu);
      if (q != cudaSuccess) sv->error = EC_ECUDA;
      complete_locked(sv, sl.reqs, status, now);
      sl.reqs.clear();
      sl.fail_status = EC_OK;
      sl.busy = false;
      worked = true;
    }
    Slot* free_slot_p = nullptr;
    int busy = 0;
    for (Slot& sl : sv->slots) {
      if (sl.busy) ++busy;
      else if (!free_slot_p) free_slot_p = &sl;
    }
    std::vector<Req> take;
    const bool has_pending = sv->n_pending.load(std::memory_order_acquire) > 0;
    const bool stopping = sv->stop.load(std::memory_order_acquire);
    const bool can_launch = free_slot_p && has_pending;
    const bool may_sleep = !worked && busy == 0 && Clock::now() - last_active >= sv->idle_spin;
    if (!can_launch && !stopping && !may_sleep) {
      // nothing to launch: poll the slots and the queue again without
      // taking the lock, so that submitters never wait for the scheduler
      // and a request that arrives while idle starts without a wake-up
      if (worked || busy > 0) last_active = Clock::now();
      if (!worked) std::this_thread::yield();
      continue;
    }
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->stats.slots_busy = busy;
      if (sv->stop && sv->pending.empty() && busy == 0) return;
      if (free_slot_p && !sv->pending.empty()) {
        while (!sv->pending.empty() && static_cast<int>(take.size()) < sv->max_batch) {
          take.push_back(std::move(sv->pending.front()));
          sv->pending.pop_front();
          sv->n_pending.fetch_sub(1, std::memory_order_relaxed);
        }
      } else if (!worked && busy == 0) {
        // idle for longer than the polling window: sleep until a
        // submission notifies
        sv->cv.wait_for(lk, std::chrono::microseconds(200));
        continue;
      }
    }
    if (!take.empty()) {
      const size_t n = take.size();
      Slot& sl = *free_slot_p;
      bool enqueued = false;
      const ec_status ds = dispatch(sv, sl, take, &enqueued);
      if (ds == EC_OK) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stats.batches += 1;
        sv->stats.max_batch_seen = std::max<long long>(sv->stats.max_batch_seen, n);
      } else if (enqueued && cudaEventRecord(sl.done, sl.st) == cudaSuccess) {
        // part of the batch is on the GPU: its requests fail once it is done
        sl.reqs = std::move(take);
        sl.fail_status = ds;
        sl.busy = true;
      } else {
        if (enqueued) {
          cudaGetLastError();
          cudaStreamSynchronize(sl.st);
          cudaGetLastError();
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        complete_locked(sv, take, ds, Clock::now());
      }
      worked = true;
    }
    if (worked || busy > 0) last_active = Clock::now();
    if (!worked) std::this_thread::yield();
  }
}

// Compiles, in the background, the programs that requests found without a
// compiled module; the dense executor runs them meanwhile.  New programs that
// arrive together are compiled into shared modules.
void compiler_loop(ec_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<std::pair<ec_plan*, Program*>> want;
    {
      std::unique_lock<std::mutex> lk(sv->cmu);
      sv->ccv.wait(lk, [&] { return sv->cstop || !sv->to_compile.empty(); });
      if (sv->cstop) return;
      // a short gathering window, so that a burst of new patterns shares
      // one module compile
      sv->ccv.wait_for(lk, std::chrono::milliseconds(5), [&] { return sv->cstop; });
      if (sv->cstop) return;
      want.swap(sv->to_compile);
    }
    xorec::compile_modules(want, false, nullptr);
    long long n = 0;
    for (auto& w : want) {
      std::lock_guard<std::mutex> lk(w.first->mu);
      if (w.second->mod) ++n;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stats.compiled_in_background += n;
  }
}

}  // namespace

extern "C" {

ec_status ec_server_create(const ec_server_opts* opts, ec_server** out) {
  if (!out) return fail(EC_EINVAL, "out is NULL");
  *out = nullptr;
  auto sv = new ec_server();
  if (!xorec::device_info(&sv->di)) {
    delete sv;
    return EC_ECUDA;
  }
  sv->device = sv->di.device;
  sv->budget = opts && opts->hbm_budget ? opts->hbm_budget : (static_cast<size_t>(32) << 30);
  sv->max_batch = opts && opts->max_batch > 0 ? opts->max_batch : 512;
  const int n_slots = opts && opts->slots > 0 ? opts->slots : 4;
  if (opts && opts->idle_spin_us != 0)
    sv->idle_spin = std::chrono::microseconds(std::max(0, opts->idle_spin_us));
  sv->chunk = std::max(1, env_int("EC_BATCH_CHUNK", 2));
  sv->background_compile = !(opts && opts->no_background_compile) && xorec::jit_available();
  sv->slots.resize(n_slots);
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        !alloc_status(sl) ||
        !grow_table(sl, static_cast<size_t>(sv->max_batch) *
                            (sizeof(xk::u64) + sizeof(xk::StripeDesc) + 16 * sizeof(xk::u64)))) {
      cudaGetLastError();
      for (Slot& s2 : sv->slots) free_slot(s2);
      delete sv;
      return fail(EC_ENOMEM, "allocation of the serving slots failed");
    }
  }
  sv->th = std::thread(scheduler, sv);
  if (sv->background_compile) sv->compiler = std::thread(compiler_loop, sv);
  *out = sv;
  return EC_OK;
}

ec_status ec_server_warm(ec_server* sv, ec_plan* plan, int max_erasures) {
  if (!sv || !plan) return fail(EC_EINVAL, "NULL argument");
  const int n = plan->k + plan->m;
  max_erasures = std::min(max_erasures, plan->m);
  std::vector<std::vector<int>> sets;
  for (int e = 1; e <= max_erasures; ++e) {
    std::vector<int> idx(e);
    for (int i = 0; i < e; ++i) idx[i] = i;
    for (;;) {
      sets.push_back(idx);
      int i = e - 1;
      while (i >= 0 && idx[i] == n - e + i) --i;
      if (i < 0) break;
      ++idx[i];
      for (int j = i + 1; j < e; ++j) idx[j] = idx[j - 1] + 1;
    }
  }
  std::vector<int> flat, counts;
  for (auto& s : sets) {
    flat.insert(flat.end(), s.begin(), s.end());
    counts.push_back(static_cast<int>(s.size()));
  }
  ec_status st = ec_decode_prepare(plan, flat.data(), counts.data(), static_cast<int>(sets.size()), 0);
  if (st != EC_OK) return st;
  std::vector<std::pair<ec_plan*, Program*>> want;
  want.emplace_back(plan, plan->enc.get());
  for (auto& s : sets) {
    Program* p = nullptr;
    st = get_decode_program(plan, s, &p);
    if (st != EC_OK) return st;
    want.emplace_back(plan, p);
  }
  if (!xorec::jit_available()) return EC_OK;   // the dense executor serves everything
  return xorec::compile_modules(want, false, nullptr);
}

ec_status ec_server_submit(ec_server* sv, const ec_job* job, uint64_t* ticket) {
  if (!sv || !job) return fail(EC_EINVAL, "NULL argument");
  Req r;
  std::vector<int> er;
  ec_status s = xorec::resolve_job(*job, &r.prog, &er, &r.ptrs);
  if (s != EC_OK) return s;
  {
    // launch target fixed at submission: the program's compiled module
    // (modules live as long as their plan; a launch takes its module's
    // block size), else the dense executor
    std::lock_guard<std::mutex> lk(job->plan->mu);
    r.mod = r.prog->mod;
    if (!r.mod && !xorec::ensure_device_code(r.prog)) return EC_ECUDA;
  }
  if (!r.mod && sv->background_compile) {
    std::lock_guard<std::mutex> lk(sv->cmu);
    if (sv->queued.insert(r.prog).second) {
      sv->to_compile.emplace_back(job->plan, r.prog);
      sv->ccv.notify_one();
    }
  }
  const size_t B = job->block_bytes;
  r.T = xorec::launch_tile(r.mod, false, xorec::launch_threads(r.mod));
  r.S = static_cast<long long>(B / 8);
  r.tiles = (r.S + r.T - 1) / r.T;
  r.bytes_in = static_cast<long long>(r.prog->n_in / 8) * static_cast<long long>(B);
  r.bytes_out = static_cast<long long>(r.prog->n_out / 8) * static_cast<long long>(B);
  r.bytes = static_cast<size_t>(r.bytes_in + r.bytes_out);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return fail(EC_EINVAL, "server is shutting down");
  if (sv->admitted + r.bytes > sv->budget) {
    sv->stats.rejected += 1;
    return EC_EBUSY;
  }
  r.ticket = sv->next_ticket++;
  r.t0 = Clock::now();
  if (ticket) *ticket = r.ticket;
  sv->admitted += r.bytes;
  sv->stats.submitted += 1;
  sv->pending.push_back(std::move(r));
  sv->n_pending.fetch_add(1, std::memory_order_release);
  sv->cv.notify_one();
  return EC_OK;
}

ec_status ec_server_cancel(ec_server* sv, uint64_t ticket) {
  if (!sv) return fail(EC_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (ticket == 0 || ticket >= sv->next_ticket) return fail(EC_EINVAL, "unknown ticket");
  for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
    if (it->ticket != ticket) continue;
    sv->admitted -= it->bytes;
    sv->stats.cancelled += 1;
    sv->pending.erase(it);
    sv->n_pending.fetch_sub(1, std::memory_order_relaxed);
    return EC_OK;
  }
  return EC_EBUSY;   // launched or finished
}

ec_status ec_server_poll_ex(ec_server* sv, uint64_t* tickets, double* latency_us, int* status,
                            int max, int* n_done) {
  if (!sv || !n_done || max < 0) return fail(EC_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  const int n = std::min<int>(max, static_cast<int>(sv->done.size()));
  for (int i = 0; i < n; ++i) {
    if (tickets) tickets[i] = sv->done[i].ticket;
    if (latency_us) latency_us[i] = sv->done[i].latency_us;
    if (status) status[i] = sv->done[i].status;
  }
  sv->done.erase(sv->done.begin(), sv->done.begin() + n);
  *n_done = n;
  return sv->error == EC_OK ? EC_OK : fail(static_cast<ec_status>(sv->error), "a batch failed on the GPU");
}

ec_status ec_server_poll(ec_server* sv, uint64_t* tickets, double* latency_us, int max,
                         int* n_done) {
  if (!sv || !n_done || max < 0) return fail(EC_EINVAL, "bad argument");
  std::vector<int> st(static_cast<size_t>(max));
  const ec_status s = ec_server_poll_ex(sv, tickets, latency_us, st.data(), max, n_done);
  if (s != EC_OK) return s;
  for (int i = 0; i < *n_done; ++i)
    if (st[i] != EC_OK)
      return fail(static_cast<ec_status>(st[i]), "a returned request failed; its outputs are incomplete");
  return EC_OK;
}

ec_status ec_server_stats_get(ec_server* sv, ec_server_stats* out) {
  if (!sv || !out) return fail(EC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->admitted_bytes = static_cast<long long>(sv->admitted);
  out->pending = static_cast<long long>(sv->pending.size());
  return EC_OK;
}

void ec_server_destroy(ec_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_one();
  }
  if (sv->th.joinable()) sv->th.join();
  {
    std::lock_guard<std::mutex> lk(sv->cmu);
    sv->cstop = true;
    sv->ccv.notify_one();
  }
  if (sv->compiler.joinable()) sv->compiler.join();
  for (Slot& s : sv->slots) free_slot(s);
  delete sv;
}

}  // extern "C"
