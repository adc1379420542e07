// Batched execution: many stripes with mixed codes, block sizes and
// encode/decode programs in a few persistent launches.
//
// ec_batch_create builds every program the jobs need (decode programs in
// parallel host threads, Sec. 1 inversion + Sec. 4-6 optimisation), compiles
// the ones without a compiled form into multi-program modules (one module
// per plan and input width, NVRTC, in parallel), and lays out in device
// memory one descriptor per stripe (work items are tiles of every strip of
// a stripe, numbered stripe after stripe).  ec_batch_run then only
// launches: one persistent launch per module plus one launch of the dense
// bitmatrix executor (the interpreter in batches created with
// EC_EXEC_INTERP) for programs without a module; it allocates nothing and
// can be captured in a CUDA graph.  Items are ordered stripe by stripe,
// largest stripes first inside each launch, and CTAs take them round robin.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.h"

using xorec::Program;
using xorec::kDenseThreads;

namespace {


int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

// Threads per CTA of batched launches (tile = 4 * threads bytes per strip)
// and the occupancy the compiled modules are built for.
int batch_threads() { return env_int("EC_BATCH_THREADS", 128); }
// Default module shape for programs of n_in input strips: EC_BATCH_THREADS,
// else 128 threads halved while two CTAs' tiles do not fit.
int batch_threads_for(int n_in) {
  const int th = env_int("EC_BATCH_THREADS", 0);
  return th > 0 ? th : xorec::tile_threads_for_inputs(n_in, 128);
}
int batch_minb_for(int n_in) {
  return env_int("EC_BATCH_MINB", xorec::default_minb(batch_threads_for(n_in), n_in));
}

struct Launch {
  void* mod = nullptr;                 // compiled module, or nullptr: the dense
                                       // executor (the interpreter if `interp`)
  bool interp = false;
  int dense_w = 4;                     // the dense executor's words per column
  int dense_form = 1;                  // and form (table)
  int threads = 128;                   // threads per CTA that own a column
  int T = 512;                         // tile bytes per strip
  int stripe_begin = 0, n_stripes = 0; // the launch's stripes in the descriptor array
  long long n_items = 0;
  int max_in = 0, max_slots = 0;
  size_t smem = 0;
  int grid = 0;
  int n_ranges = 1;                    // per-SM item ranges (work-queue heads)
};

template <class F>
void parallel_for(size_t n, F f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(n, hw);
  std::atomic<size_t> next{0};
  std::vector<std::thread> pool;
  for (size_t t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        const size_t i = next.fetch_add(1);
        if (i >= n) return;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

}  // namespace

struct ec_batch {
  int device = -1;
  std::vector<Launch> launches;
  // launches fan out over these streams (fork/join through events) so that
  // the tail of one persistent launch overlaps the start of the next
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  int chunk = 8;
  int queue_stride = 1;                // work-queue heads per launch (its item ranges)
  xk::u64* d_queues = nullptr;         // queue_stride heads per launch, then the status word
  int* d_status = nullptr;             // the batch's own status word (set on a timeout)
  xk::StripeDesc* d_descs = nullptr;
  xk::u64* d_blocks = nullptr;
  xk::TensorMap* d_maps = nullptr;     // per-block tensor maps of the stripes' inputs
  int* status = nullptr;
  ec_batch_info info{};
};

namespace {

struct Entry {
  const ec_job* job;
  ec_plan* plan;
  Program* prog = nullptr;
  std::vector<int> er;                 // sorted erasures (decode)
  std::vector<uint64_t> ptrs;          // inputs then outputs (program order)
  long long S = 0, tiles = 0;
  int launch = -1;
};

ec_status check_job(const ec_job& j) {
  if (!j.plan || !j.blocks || !j.out) return fail(EC_EINVAL, "job with NULL plan, blocks or out");
  if (j.op != EC_OP_ENCODE && j.op != EC_OP_DECODE) return fail(EC_EINVAL, "bad job op");
  if (j.block_bytes == 0 || j.block_bytes % 128 != 0)
    return fail(EC_EINVAL, "block_bytes must be a positive multiple of 128");
  return EC_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Block pointer list in program order (the same order ec_encode/ec_decode use).
ec_status job_pointers(Entry* e) {
  const ec_job& j = *e->job;
  const int k = e->plan->k, m = e->plan->m;
  if (j.op == EC_OP_ENCODE) {
    for (int i = 0; i < k; ++i) {
      if (!j.blocks[i] || !aligned16(j.blocks[i])) return fail(EC_EINVAL, "data block NULL or not 16-byte aligned");
      e->ptrs.push_back(reinterpret_cast<uint64_t>(j.blocks[i]));
    }
    for (int i = 0; i < m; ++i) {
      if (!j.out[i] || !aligned16(j.out[i])) return fail(EC_EINVAL, "parity block NULL or not 16-byte aligned");
      e->ptrs.push_back(reinterpret_cast<uint64_t>(j.out[i]));
    }
    return EC_OK;
  }
  for (int id = 0, x = 0; id < k + m && static_cast<int>(e->ptrs.size()) < k; ++id) {
    if (x < static_cast<int>(e->er.size()) && e->er[x] == id) { ++x; continue; }
    if (!j.blocks[id] || !aligned16(j.blocks[id]))
      return fail(EC_EINVAL, "surviving block NULL or not 16-byte aligned");
    e->ptrs.push_back(reinterpret_cast<uint64_t>(j.blocks[id]));
  }
  for (int id : e->er) {
    const int pos = static_cast<int>(std::find(j.erasures, j.erasures + j.n_erasures, id) - j.erasures);
    if (!j.out[pos] || !aligned16(j.out[pos])) return fail(EC_EINVAL, "output block NULL or not 16-byte aligned");
    e->ptrs.push_back(reinterpret_cast<uint64_t>(j.out[pos]));
  }
  return EC_OK;
}

void free_batch(ec_batch* b) {
  for (cudaStream_t st : b->lanes) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_queues) cudaFree(b->d_queues);
  if (b->d_blocks) cudaFree(b->d_blocks);
  if (b->d_maps) cudaFree(b->d_maps);
  delete b;
}

}  // namespace

namespace xorec {

// Program, sorted erasures and block pointers (program order) of one job.
ec_status resolve_job(const ec_job& j, Program** prog, std::vector<int>* er,
                      std::vector<uint64_t>* ptrs) {
  ec_status s = check_job(j);
  if (s != EC_OK) return s;
  Entry e;
  e.job = &j;
  e.plan = j.plan;
  if (j.op == EC_OP_DECODE) {
    s = canon_erasures(j.plan, j.erasures, j.n_erasures, &e.er);
    if (s != EC_OK) return s;
    s = get_decode_program(j.plan, e.er, &e.prog);
    if (s != EC_OK) return s;
  } else {
    e.prog = j.plan->enc.get();
  }
  s = job_pointers(&e);
  if (s != EC_OK) return s;
  *prog = e.prog;
  *er = e.er;
  *ptrs = e.ptrs;
  return EC_OK;
}


// Launch shape of a plan's compiled modules: the autotuner's choice for the
// plan (threads per CTA, hence the strip tile of 4 x threads bytes, and
// resident CTAs per SM, hence the register cap), else the defaults.
int plan_module_threads(const ec_plan* p, int n_in) {
  return p->tuned_threads > 0 ? p->tuned_threads : batch_threads_for(n_in);
}

// A tuned shape keeps its occupancy in batch modules down to a 128-register
// cap: a tighter cap leaves the batched pipeline no registers of its own
// beside the program's values (the autotuned RS(6,3) shape, register budget
// 96 at 5 CTAs/SM, spilled 40 B in a module at its 96-register cap).
int plan_module_minb(const ec_plan* p, int n_in) {
  if (!(p->tuned_threads > 0 && p->tuned_minb > 0)) return batch_minb_for(n_in);
  const int floor_cap = env_int("EC_MODULE_MIN_CAP", 128);
  if (floor_cap <= 0) return p->tuned_minb;
  return std::max(1, std::min(p->tuned_minb, 65536 / (p->tuned_threads * floor_cap)));
}

// Threads per CTA that own a column in a batched launch of `mod`: the
// module's, or (no module) the dense executor's.
int launch_threads(void* mod) { return mod ? jit_module_threads(mod) : kDenseThreads; }

// Tile bytes per strip of a batched launch: 4 x threads for modules and the
// interpreter (interp: a batch created with EC_EXEC_INTERP), the dense
// executor's words per thread otherwise.
int launch_tile(void* mod, bool interp, int threads) {
  return mod || interp ? 4 * threads : 4 * dense_words() * kDenseThreads;
}

// One batched launch on its target (dense_w, dense_form: the dense
// executor's form its shape was computed for).
bool batch_launch(void* mod, bool interp, const xk::BatchParams& bp, int threads, int grid,
                  size_t smem, cudaStream_t st, int dense_w, int dense_form) {
  if (mod) return jit_module_launch(mod, bp, grid, smem, st);
  if (interp) return launch_interp_batch(bp, threads, grid, smem, st);
  xk::BatchParams dp = bp;
  dp.win = kDenseWin;
  return launch_dense_batch(dp, dense_w, dense_form, grid, smem, st);
}

// A program of one group of rows that the windowed pipeline runs (its
// modules hold a ring of windows, not a stage of every input strip).
static bool window_program(const Program* p) {
  int w, nw, np;
  return windowed(*p) && window_layout(*p, &w, &nw, &np, nullptr) && np == nw;
}

// Threads that own a column in the module that runs `prog`: the plan's
// tuned shape, else window_threads(true) for windowed programs and the default
// module shape otherwise.
int module_threads(const ec_plan* plan, const Program* prog) {
  if (plan->tuned_threads > 0) return plan->tuned_threads;
  return window_program(prog) ? window_threads(true) : plan_module_threads(plan, prog->n_in);
}

// Such a module fits one CTA: a ring of windows (windowed programs) or a
// stage of every input strip, and code small enough to compile quickly.
static bool module_fits(const Program* prog, int threads, size_t smem_optin) {
  if (window_program(prog))
    return 128 + static_cast<size_t>(xk::kWinRing) * prog->stats.window * 4 * threads <= smem_optin &&
           prog->stats.fused.mem <= kMaxCompiledMemOps;
  return compiled_tier_fits(prog, threads, smem_optin);
}

// Compile every program of `want` that has no module of its plan's launch
// shape into multi-program modules (per plan and input width, NVRTC, in
// parallel host threads).  Modules belong to their plan.  Each group is cut
// into as few modules as keep every module within EC_BATCH_MODULE_SIZE
// programs (default 256) and EC_BATCH_MODULE_MEM memory operations of
// straight-line code (default 256 K), programs spread evenly over them: a
// batch then runs few long launches (every launch starts each SM on a
// program whose code is not yet in its instruction cache), at the price of
// fewer, longer compiles
// (RS(10,4) decode over 231 erasure sets: two modules of at most 128
// programs, 0.936 of the measured copy bandwidth, batch built in 12.5 s; one
// module, 0.954, 26.5 s).
ec_status compile_modules(const std::vector<std::pair<ec_plan*, Program*>>& want, bool must,
                          int* built) {
  const long module_size = std::max(1, env_int("EC_BATCH_MODULE_SIZE", 256));
  const long module_mem = std::max(1024, env_int("EC_BATCH_MODULE_MEM", 262144));
  DeviceInfo di;
  if (!device_info(&di)) return EC_ECUDA;
  // modules per plan, input width and pipeline (windowed or not)
  std::map<std::tuple<ec_plan*, int, bool>, std::vector<Program*>> pending;
  std::vector<Program*> seen;
  for (const auto& w : want) {
    const int threads = module_threads(w.first, w.second);
    if (!module_fits(w.second, threads, di.smem_optin)) continue;   // dense executor
    std::lock_guard<std::mutex> lk(w.first->mu);
    if ((w.second->mod && jit_module_threads(w.second->mod) == threads) ||
        std::find(seen.begin(), seen.end(), w.second) != seen.end())
      continue;
    seen.push_back(w.second);
    pending[{w.first, w.second->n_in, window_program(w.second)}].push_back(w.second);
  }
  std::vector<std::pair<ec_plan*, std::vector<Program*>>> to_compile;
  for (auto& kv : pending) {
    const std::vector<Program*>& ps = kv.second;
    long mem = 0;
    for (const Program* p : ps) mem += p->stats.fused.mem;
    const long n = static_cast<long>(ps.size());
    const long n_mod = std::max({1L, (n + module_size - 1) / module_size,
                                 std::min(n, (mem + module_mem - 1) / module_mem)});
    for (long m = 0; m < n_mod; ++m)
      to_compile.emplace_back(std::get<0>(kv.first),
                              std::vector<Program*>(ps.begin() + n * m / n_mod,
                                                    ps.begin() + n * (m + 1) / n_mod));
  }
  std::vector<std::string> errs(to_compile.size());
  std::vector<void*> mods(to_compile.size(), nullptr);
  parallel_for(to_compile.size(), [&](size_t i) {
    std::vector<const Program*> ps(to_compile[i].second.begin(), to_compile[i].second.end());
    ec_plan* plan = to_compile[i].first;
    const int n_in = ps.front()->n_in;
    mods[i] = jit_compile_module(ps, module_threads(plan, ps.front()), plan_module_minb(plan, n_in),
                                 &errs[i], env_int("EC_MODULE_NO_SPILL", 0) != 0);
  });
  if (built) *built = static_cast<int>(to_compile.size());
  for (size_t i = 0; i < to_compile.size(); ++i) {
    ec_plan* plan = to_compile[i].first;
    std::lock_guard<std::mutex> lk(plan->mu);
    if (!mods[i]) {
      if (must) {
        for (size_t j = i; j < mods.size(); ++j) jit_module_release(mods[j]);
        return fail(EC_ECUDA, "module compile failed: " + errs[i]);
      }
      continue;   // these programs stay with the dense executor
    }
    plan->modules.push_back(mods[i]);
    for (size_t j = 0; j < to_compile[i].second.size(); ++j) {
      to_compile[i].second[j]->mod = mods[i];
      to_compile[i].second[j]->mod_index = static_cast<int>(j);
    }
  }
  return EC_OK;
}

// Shared memory and resident CTAs per SM of a batched launch (module, dense
// executor, or interpreter).
bool batch_launch_shape(void* mod, bool interp, int max_in, int max_slots, int threads,
                        size_t smem_optin, size_t* smem, int* per_sm, int dense_w,
                        int dense_form) {
  const int T = 4 * threads;
  if (!mod && !interp) {
    // the dense executor: a ring of windows of kDenseWin strips (and its
    // tables)
    *smem = dense_smem_bytes(4 * dense_w * kDenseThreads, dense_form);
    if (*smem > smem_optin) return false;
    *per_sm = std::max(1, dense_max_ctas_per_sm(dense_w, dense_form, true, *smem));
    return true;
  }
  int win = 0, n_win = 0;
  if (mod && jit_module_window(mod, &win, &n_win)) {
    *smem = 128 + static_cast<size_t>(xk::kWinRing) * win * T;
    *per_sm = std::max(1, jit_module_ctas_per_sm(mod, *smem));
    return true;
  }
  if (mod) {
    *smem = xk::kBatchHeader + static_cast<size_t>(max_in) * T;
    *per_sm = std::max(1, jit_module_ctas_per_sm(mod, *smem));
    return true;
  }
  *smem = interp_batch_smem_bytes(max_in, max_slots, T);
  if (*smem > smem_optin) return false;
  *per_sm = std::max(1, interp_batch_max_ctas_per_sm(threads, *smem));
  return true;
}

// A launch's items split into n_ranges contiguous ranges (BatchParams).
void set_ranges(xk::BatchParams* bp, long long n_items, int n_ranges) {
  bp->n_ranges = std::max(1, n_ranges);
  bp->range_len = n_items / bp->n_ranges;
  bp->range_rem = static_cast<int>(n_items % bp->n_ranges);
}

// Item ranges of a batched launch (one work-queue head each, see
// run_batch_pipeline): one per SM when every SM's range holds at least four
// chunks per resident CTA and the programs preload their inputs, else a
// single queue.  Programs with more input strips are far larger than an SM's
// instruction cache, so ranges gain nothing there, and their tiles are short
// (256 B of each of hundreds of strips): with a single queue all CTAs read
// neighbouring tiles, which keeps DRAM rows open (RS(100,4) decode: 0.39 of
// the copy bandwidth with one queue, 0.20 with per-SM ranges).
// The dense executor's code is small and shared by every stripe: one
// queue.  EC_BATCH_RANGES overrides (1 = a single queue).
int batch_ranges(long long n_items, int sms, int per_sm, int chunk, int max_in, bool dense) {
  const int forced = env_int("EC_BATCH_RANGES", 0);
  if (forced > 0) return std::min(forced, std::max(1, sms));
  if (dense || max_in > kPreloadMaxInputs) return 1;
  const long long per_range = 4ll * std::max(1, per_sm) * std::max(1, chunk);
  return n_items >= per_range * sms ? std::max(1, sms) : 1;
}

}  // namespace xorec

extern "C" {

ec_status ec_batch_create(const ec_job* jobs, int n_jobs, int executor, ec_batch** out) {
  xorec::TraceRange trace_("xorec batch create");
  if (!out) return fail(EC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(EC_EINVAL, "bad job list");
  if (executor < EC_EXEC_AUTO || executor > EC_EXEC_DENSE) return fail(EC_EINVAL, "bad executor");
  const auto t0 = std::chrono::steady_clock::now();
  xorec::DeviceInfo di;
  if (!xorec::device_info(&di)) return EC_ECUDA;

  // 1. validate, canonicalise erasures
  std::vector<Entry> ents(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    ec_status s = check_job(jobs[i]);
    if (s != EC_OK) return s;
    ents[i].job = &jobs[i];
    ents[i].plan = jobs[i].plan;
    if (jobs[i].op == EC_OP_DECODE) {
      s = canon_erasures(jobs[i].plan, jobs[i].erasures, jobs[i].n_erasures, &ents[i].er);
      if (s != EC_OK) return s;
    }
  }
  // 2. programs (decode programs built in parallel, cached by the plan)
  std::map<std::pair<ec_plan*, std::vector<int>>, Program*> dec;
  for (auto& e : ents)
    if (e.job->op == EC_OP_DECODE) dec[{e.plan, e.er}] = nullptr;
  std::vector<std::pair<ec_plan*, std::vector<int>>> keys;
  for (auto& kv : dec) keys.push_back(kv.first);
  std::vector<Program*> built(keys.size(), nullptr);
  std::atomic<int> rc{EC_OK};
  parallel_for(keys.size(), [&](size_t i) {
    Program* p = nullptr;
    const ec_status s = get_decode_program(keys[i].first, keys[i].second, &p);
    if (s != EC_OK) rc.store(s);
    built[i] = p;
  });
  if (rc.load() != EC_OK) return static_cast<ec_status>(rc.load());
  for (size_t i = 0; i < keys.size(); ++i) dec[keys[i]] = built[i];
  for (auto& e : ents) {
    e.prog = e.job->op == EC_OP_ENCODE ? e.plan->enc.get() : dec[{e.plan, e.er}];
    ec_status s = job_pointers(&e);
    if (s != EC_OK) return s;
    e.S = static_cast<long long>(e.job->block_bytes / 8);
  }

  // 3. tiers: compile programs without a module (per plan, per input width)
  bool compiled =
      (executor == EC_EXEC_AUTO || executor == EC_EXEC_COMPILED) && xorec::jit_available();
  if (executor == EC_EXEC_COMPILED && !compiled)
    return fail(EC_ENOTSUP, "no run-time compiler available");
  int modules_built = 0;
  if (compiled) {
    std::vector<std::pair<ec_plan*, Program*>> want;
    for (auto& e : ents) want.emplace_back(e.plan, e.prog);
    const ec_status cs = xorec::compile_modules(want, executor == EC_EXEC_COMPILED, &modules_built);
    if (cs != EC_OK) return cs;
  }

  // 4. launches: one per module in use, one for the dense executor (or the
  // interpreter)
  auto b = new ec_batch();
  b->device = di.device;
  b->status = di.status;
  b->chunk = std::max(1, env_int("EC_BATCH_CHUNK", 2));
  b->queue_stride = std::max(1, di.sms);
  std::map<void*, int> launch_of;
  for (auto& e : ents) {
    void* mod = compiled ? e.prog->mod : nullptr;
    auto it = launch_of.find(mod);
    if (it == launch_of.end()) {
      it = launch_of.emplace(mod, static_cast<int>(b->launches.size())).first;
      Launch L;
      L.mod = mod;
      L.interp = !mod && executor == EC_EXEC_INTERP;
      L.dense_w = xorec::dense_words();
      L.dense_form = xorec::dense_form();
      L.threads = L.interp ? batch_threads() : xorec::launch_threads(mod);
      b->launches.push_back(L);
    }
    e.launch = it->second;
    Launch& L = b->launches[e.launch];
    L.max_in = std::max(L.max_in, e.prog->n_in);
    if (!mod) L.max_slots = std::max(L.max_slots, e.prog->interp_slots);
  }
  // the interpreter's tile shrinks (down to 32 threads, 128 bytes per strip)
  // until its stage of every input strip and its slots fit one CTA
  for (auto& L : b->launches) {
    while (L.interp && L.threads > 32 &&
           xorec::interp_batch_smem_bytes(L.max_in, L.max_slots, 4 * L.threads) > di.smem_optin)
      L.threads /= 2;
    L.T = L.mod || L.interp ? 4 * L.threads : 4 * L.dense_w * kDenseThreads;
  }
  for (auto& e : ents) {
    const Launch& L = b->launches[e.launch];
    e.tiles = (e.S + L.T - 1) / L.T;
  }
  // programs without a module need their streams and masks on the device
  for (auto& e : ents)
    if (!(compiled && e.prog->mod) && !xorec::ensure_device_code(e.prog)) {
      free_batch(b);
      return EC_ECUDA;
    }

  // 5. host layout: stripes grouped by launch, largest first
  std::vector<int> order(ents.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    if (ents[a].launch != ents[c].launch) return ents[a].launch < ents[c].launch;
    return ents[a].S > ents[c].S;
  });
  std::vector<xk::StripeDesc> descs(ents.size());
  std::vector<xk::u64> blocks;
  // tensor maps of every input block (one tiled copy per block and tile);
  // map_at[stripe] = index of its first map, -1 = one 1-D copy per strip
  std::vector<xk::TensorMap> maps;
  std::vector<long long> map_at(ents.size(), -1);
  long long bytes_in = 0, bytes_out = 0, total_items = 0;
  int cur = -1;
  long long launch_items = 0;
  for (size_t oi = 0; oi < order.size(); ++oi) {
    Entry& e = ents[order[oi]];
    if (e.launch != cur) {
      cur = e.launch;
      launch_items = 0;
      b->launches[cur].stripe_begin = static_cast<int>(oi);
    }
    Launch& L = b->launches[cur];
    xk::StripeDesc& d = descs[oi];
    std::memset(&d, 0, sizeof(d));
    d.blocks = reinterpret_cast<const xk::u64*>(blocks.size() * sizeof(xk::u64));  // offset for now
    d.S = e.S;
    d.item_base = launch_items;
    d.n_inblk = e.prog->n_in / 8;
    d.n_outblk = e.prog->n_out / 8;
    d.prog = e.prog->mod_index;
    d.code = e.prog->d_code;
    d.code_len = static_cast<int>(e.prog->chunks.size() / 8);
    d.n_slots = e.prog->interp_slots;
    for (uint64_t p : e.ptrs) blocks.push_back(p);
    {
      bool ok = true;
      for (int j = 0; j < d.n_inblk && ok; ++j)
        ok = xorec::block_tensor_map_allowed(reinterpret_cast<const void*>(e.ptrs[j]), e.S, L.T);
      if (ok) {
        map_at[oi] = static_cast<long long>(maps.size());
        maps.resize(maps.size() + d.n_inblk);
      }
    }
    launch_items += e.tiles;
    L.n_items = launch_items;
    L.n_stripes += 1;
    total_items += e.tiles;
    bytes_in += static_cast<long long>(d.n_inblk) * static_cast<long long>(e.job->block_bytes);
    bytes_out += static_cast<long long>(d.n_outblk) * static_cast<long long>(e.job->block_bytes);
  }

  // encode the tensor maps in parallel host threads (each with the device's
  // context current); a stripe whose maps the driver refuses falls back to
  // one copy per strip
  {
    std::vector<char> refused(order.size(), 0);
    parallel_for(order.size(), [&](size_t oi) {
      if (map_at[oi] < 0) return;
      thread_local int current = -1;
      if (current != di.device) {
        if (cudaSetDevice(di.device) != cudaSuccess) {
          cudaGetLastError();
          refused[oi] = 1;
          return;
        }
        current = di.device;
      }
      const Entry& e = ents[order[oi]];
      const int T = b->launches[e.launch].T;
      for (int j = 0; j < descs[oi].n_inblk; ++j)
        if (!xorec::block_tensor_map(reinterpret_cast<const void*>(e.ptrs[j]), e.S, T,
                                     &maps[map_at[oi] + j]))
          refused[oi] = 1;
    });
    for (size_t oi = 0; oi < order.size(); ++oi)
      if (refused[oi]) map_at[oi] = -1;
  }

  // 6. device copies (owned by the batch)
  if (!ents.empty()) {
    if (xorec::dev_malloc(&b->d_descs, descs.size() * sizeof(xk::StripeDesc)) != cudaSuccess ||
        xorec::dev_malloc(&b->d_queues,
                          (b->launches.size() * b->queue_stride + 1) * sizeof(xk::u64)) !=
            cudaSuccess ||
        xorec::dev_malloc(&b->d_blocks, std::max<size_t>(1, blocks.size()) * sizeof(xk::u64)) !=
            cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ENOMEM, "device allocation of the batch tables failed");
    }
    if (!maps.empty() &&
        xorec::dev_malloc(&b->d_maps, maps.size() * sizeof(xk::TensorMap)) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ENOMEM, "device allocation of the batch tensor maps failed");
    }
    b->d_status = reinterpret_cast<int*>(b->d_queues + b->launches.size() * b->queue_stride);
    if (cudaMemset(b->d_status, 0, sizeof(xk::u64)) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ECUDA, "clearing the batch status word failed");
    }
    for (auto& d : descs)
      d.blocks = b->d_blocks + reinterpret_cast<uintptr_t>(d.blocks) / sizeof(xk::u64);
    for (size_t i = 0; i < descs.size(); ++i)
      descs[i].maps = map_at[i] >= 0 ? b->d_maps + map_at[i] : nullptr;
    if (!maps.empty() && cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(xk::TensorMap),
                                    cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ECUDA, "upload of the batch tensor maps failed");
    }
    if (cudaMemcpy(b->d_descs, descs.data(), descs.size() * sizeof(xk::StripeDesc),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_blocks, blocks.data(), blocks.size() * sizeof(xk::u64),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ECUDA, "upload of the batch tables failed");
    }
  }

  // 7. launch shapes: persistent grids; launches of different modules are
  // spread over a few lanes so that their tails overlap
  int n_modules = 0, n_compiled_progs = 0;
  for (auto& L : b->launches) {
    int per_sm = 1;
    if (L.mod) ++n_modules;
    if (!xorec::batch_launch_shape(L.mod, L.interp, L.max_in, L.max_slots, L.threads,
                                   di.smem_optin, &L.smem, &per_sm, L.dense_w,
                                   L.dense_form)) {
      free_batch(b);
      return fail(EC_ENOTSUP, "a program needs more shared memory than one CTA can hold");
    }
    const long long grid = static_cast<long long>(di.sms) * std::max(1, per_sm);
    L.grid = static_cast<int>(std::min<long long>(grid, std::max<long long>(1, L.n_items)));
    L.n_ranges = xorec::batch_ranges(L.n_items, di.sms, per_sm, b->chunk, L.max_in,
                                     !L.mod && !L.interp);
    if (env_int("XOREC_LOG", 0))
      std::fprintf(stderr, "[xorec] batch launch: %s items=%lld max_in=%d smem=%zu ctas/sm=%d grid=%d regs=%d ranges=%d\n",
                   L.mod ? "module" : L.interp ? "interp" : "dense", L.n_items, L.max_in, L.smem, per_sm, L.grid,
                   L.mod ? xorec::jit_module_regs(L.mod) : 0, L.n_ranges);
  }
  // largest launches first; lanes for concurrent launches
  std::stable_sort(b->launches.begin(), b->launches.end(),
                   [](const Launch& x, const Launch& y) { return x.n_items > y.n_items; });
  const int n_lanes = std::min<int>(static_cast<int>(b->launches.size()),
                                    std::max(1, env_int("EC_BATCH_LANES", 4)));
  if (n_lanes > 1) {
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_batch(b);
      return fail(EC_ECUDA, "cudaEventCreate failed");
    }
    for (int i = 0; i < n_lanes; ++i) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return fail(EC_ECUDA, "stream or event creation failed");
      }
      b->lanes.push_back(st);
      b->done.push_back(ev);
    }
  }
  std::vector<Program*> progs;
  for (auto& e : ents)
    if (std::find(progs.begin(), progs.end(), e.prog) == progs.end()) {
      progs.push_back(e.prog);
      if (compiled && e.prog->mod) ++n_compiled_progs;
    }
  b->info.stripes = static_cast<long long>(ents.size());
  b->info.items = total_items;
  b->info.bytes_in = bytes_in;
  b->info.bytes_out = bytes_out;
  b->info.programs = static_cast<int>(progs.size());
  b->info.compiled_programs = n_compiled_progs;
  b->info.launches = static_cast<int>(b->launches.size());
  b->info.modules_built = modules_built;
  b->info.prepare_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = b;
  return EC_OK;
}

ec_status ec_batch_run(ec_batch* b, void* stream) {
  xorec::TraceRange trace_("xorec batch run");
  if (!b) return fail(EC_EINVAL, "NULL batch");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (b->launches.empty()) return EC_OK;
  if (cudaMemsetAsync(b->d_queues, 0, b->launches.size() * b->queue_stride * sizeof(xk::u64),
                      caller) != cudaSuccess)
    return fail(EC_ECUDA, "resetting the work queues failed");
  if (xorec::take_injected_timeout() &&
      !xorec::launch_selftest_wait_to(caller, b->status, b->d_status))
    return EC_ECUDA;
  const bool fan = !b->lanes.empty();
  if (fan) {
    if (cudaEventRecord(b->fork, caller) != cudaSuccess) return fail(EC_ECUDA, "cudaEventRecord failed");
    for (cudaStream_t ln : b->lanes)
      if (cudaStreamWaitEvent(ln, b->fork, 0) != cudaSuccess) return fail(EC_ECUDA, "cudaStreamWaitEvent failed");
  }
  for (size_t li = 0; li < b->launches.size(); ++li) {
    const Launch& L = b->launches[li];
    cudaStream_t st = fan ? b->lanes[li % b->lanes.size()] : caller;
    if (L.n_items == 0) continue;
    xk::BatchParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.stripes = b->d_descs + L.stripe_begin;
    bp.n_stripes = L.n_stripes;
    bp.chunk = b->chunk;
    bp.queue = b->d_queues + li * b->queue_stride;
    xorec::set_ranges(&bp, L.n_items, L.n_ranges);
    bp.n_items = L.n_items;
    bp.T = L.T;
    bp.max_in = L.max_in;
    bp.status = b->status;
    bp.local_status = b->d_status;
    const bool ok = xorec::batch_launch(L.mod, L.interp, bp, L.threads, L.grid, L.smem, st,
                                        L.dense_w, L.dense_form);
    if (!ok) return EC_ECUDA;
  }
  if (fan) {
    for (size_t i = 0; i < b->lanes.size(); ++i) {
      if (cudaEventRecord(b->done[i], b->lanes[i]) != cudaSuccess ||
          cudaStreamWaitEvent(caller, b->done[i], 0) != cudaSuccess)
        return fail(EC_ECUDA, "joining the batch lanes failed");
    }
  }
  return EC_OK;
}

ec_status ec_plan_module_source(ec_plan* plan, const int* sets, const int* counts, int n_sets,
                                char* buf, size_t len, size_t* need) {
  if (!plan || (n_sets > 0 && (!sets || !counts)) || n_sets < 0)
    return fail(EC_EINVAL, "bad argument");
  std::vector<const Program*> progs;
  if (n_sets == 0) progs.push_back(plan->enc.get());
  size_t off = 0;
  for (int i = 0; i < n_sets; ++i) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, sets + off, counts[i], &er);
    if (s != EC_OK) return s;
    off += counts[i];
    Program* p = nullptr;
    s = get_decode_program(plan, er, &p);
    if (s != EC_OK) return s;
    progs.push_back(p);
  }
  const int n_in = progs.front()->n_in;
  for (const Program* p : progs)
    if (p->n_in != n_in) return fail(EC_EINVAL, "programs of one module share their input count");
  const std::string src = xorec::jit_module_source(progs, xorec::module_threads(plan, progs.front()),
                                                   xorec::plan_module_minb(plan, n_in));
  if (need) *need = src.size() + 1;
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, src.size());
    std::memcpy(buf, src.data(), n);
    buf[n] = '\0';
  }
  return EC_OK;
}

ec_status ec_batch_status(ec_batch* b, int* status, int reset) {
  if (!b || !status) return fail(EC_EINVAL, "NULL argument");
  *status = 0;
  if (!b->d_status) return EC_OK;   // an empty batch launches nothing
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "cudaDeviceSynchronize failed");
  }
  int v = 0;
  if (cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "reading the batch status word failed");
  }
  if (reset && cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "resetting the batch status word failed");
  }
  *status = v == xk::XK_STATUS_TIMEOUT ? EC_ETIMEOUT : 0;
  return EC_OK;
}

ec_status ec_batch_info_get(const ec_batch* b, ec_batch_info* out) {
  if (!b || !out) return fail(EC_EINVAL, "NULL argument");
  *out = b->info;
  return EC_OK;
}

void ec_batch_destroy(ec_batch* b) {
  if (b) free_batch(b);
}

ec_status ec_run_batch(const ec_job* jobs, int n_jobs, void* stream) {
  ec_batch* b = nullptr;
  ec_status s = ec_batch_create(jobs, n_jobs, EC_EXEC_AUTO, &b);
  if (s != EC_OK) return s;
  s = ec_batch_run(b, stream);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && s == EC_OK) {
    cudaGetLastError();
    s = fail(EC_ECUDA, "batch execution failed");
  }
  if (s == EC_OK && b->d_status) {
    int v = 0;
    if (cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      s = fail(EC_ECUDA, "reading the batch status word failed");
    } else if (v == xk::XK_STATUS_TIMEOUT) {
      s = fail(EC_ETIMEOUT, "a bounded wait of the batch timed out; its outputs are incomplete");
    }
  }
  ec_batch_destroy(b);
  return s;
}

}  // extern "C"
