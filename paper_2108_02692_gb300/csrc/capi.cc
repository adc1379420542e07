// C ABI of the library (declared in include/xorec.h).
#include <cuda.h>   // tensor-map types; the encoder is taken from the driver at run time
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/xorec.h"
#include "gf.h"
#include "internal.h"

using xorec::Program;

namespace xorec {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

std::atomic<int> g_fail_allocs{0};

bool take_injected_alloc_failure() {
  int v = g_fail_allocs.load(std::memory_order_relaxed);
  while (v > 0)
    if (g_fail_allocs.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
  return false;
}

std::atomic<int> g_inject_timeouts{0};

bool take_injected_timeout() {
  int v = g_inject_timeouts.load(std::memory_order_relaxed);
  while (v > 0)
    if (g_inject_timeouts.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return true;
  return false;
}

static std::mutex g_dev_mu;
static DeviceInfo g_dev[64];

bool device_info(DeviceInfo* out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    set_error("no CUDA device");
    return false;
  }
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo& d = g_dev[dev];
  if (d.device < 0) {
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
      cudaGetLastError();
      set_error("cudaDeviceGetAttribute failed");
      return false;
    }
    int* st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess || cudaMemset(st, 0, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      set_error("cannot allocate the device status word");
      return false;
    }
    d.sms = sms;
    d.smem_optin = static_cast<size_t>(optin);
    d.status = st;
    d.device = dev;
  }
  *out = d;
  return true;
}

// Device buffer of a program: its chunk stream (16-byte chunks), then the
// dense executor's control words (column masks, then row words).
bool ensure_device_code(Program* p) {
  if (p->d_code) return true;
  const size_t code_bytes = p->chunks.size() * sizeof(uint16_t);
  const size_t mask_bytes = p->masks.size() * sizeof(uint32_t);
  const size_t row_bytes = p->rowbits.size() * sizeof(uint32_t);
  const size_t bytes = std::max<size_t>(16, code_bytes + mask_bytes + row_bytes);
  uint16_t* d = nullptr;
  if (dev_malloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of the program failed");
    return false;
  }
  if ((code_bytes && cudaMemcpy(d, p->chunks.data(), code_bytes, cudaMemcpyHostToDevice) !=
                         cudaSuccess) ||
      (mask_bytes && cudaMemcpy(reinterpret_cast<uint8_t*>(d) + code_bytes, p->masks.data(),
                                mask_bytes, cudaMemcpyHostToDevice) != cudaSuccess) ||
      (row_bytes && cudaMemcpy(reinterpret_cast<uint8_t*>(d) + code_bytes + mask_bytes,
                               p->rowbits.data(), row_bytes, cudaMemcpyHostToDevice) !=
                        cudaSuccess)) {
    cudaGetLastError();
    cudaFree(d);
    set_error("upload of the program failed");
    return false;
  }
  p->d_code = d;
  return true;
}

static int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

static std::mutex g_jit_mu;

// The compiled tier runs a program only when one tile of all its input
// strips fits a CTA's shared memory and the straight-line code stays small
// enough to compile quickly (kMaxCompiledMemOps); everything else goes to
// the interpreter.

// Shared memory a CTA may use on sm_103 (opt-in limit).
constexpr size_t kSmemOptin = 232448;

int tile_threads_for_inputs(int n_in, int threads) {
  while (threads > 64 &&
         2 * (static_cast<size_t>(n_in) * 4 * threads + xk::kBatchHeader) > kSmemOptin)
    threads /= 2;
  return threads;
}

int default_minb(int threads, int n_in) {
  const bool wide_preload = n_in > kPreloadCap128Inputs && n_in <= kPreloadMaxInputs;
  return minb_for(threads, wide_preload ? 168 : 128);
}

int program_threads(const Program* p) {
  if (p->threads > 0) return p->threads;
  const int th = env_int("EC_JIT_THREADS", 0);
  if (th > 0) return th;
  // windowed programs keep a ring of a few windows, not a tile of every strip
  return windowed(*p) ? window_threads(false) : tile_threads_for_inputs(p->n_in, 128);
}

// Consumer threads of a windowed kernel (one 4-byte column each; the
// producer warp comes on top): a multiple of 32 from 64 to 512.  Single
// launches take one CTA of 320 per SM, whose warps all run the same phase
// of the program and so share its instruction-cache lines (encode, 128
// stripes x 1 MiB, of measured HBM, 128 -> 320 threads: RS(48,4) 0.96 ->
// 1.03, RS(100,4) 0.97 -> 1.02, RS(128,4) 0.43 -> 0.50).  Batch modules
// keep three CTAs of 128: their CTAs pop items one by one, and wider CTAs
// lost (RS(48,4) decode 1.00 -> 0.96, RS(100,4) 0.78 -> 0.73 at 320).
// EC_WIN_THREADS and EC_WIN_MODULE_THREADS override.
int window_threads(bool module) {
  const int dflt = module ? 128 : 320;
  const int th = env_int(module ? "EC_WIN_MODULE_THREADS" : "EC_WIN_THREADS", dflt);
  return th >= 64 && th <= 512 && th % 32 == 0 ? th : dflt;
}

bool compiled_tier_fits(const Program* p, int threads, size_t smem_optin) {
  const size_t smem = 128 + static_cast<size_t>(p->n_in) * 4 * threads + xk::kBatchHeader;
  return smem <= smem_optin && p->stats.fused.mem <= kMaxCompiledMemOps;
}

// Shared memory of a windowed program's single launch: barriers and the
// ring of kWinRing windows.
static size_t window_smem_bytes(const Program* p, int threads) {
  return 128 + static_cast<size_t>(xk::kWinRing) * p->stats.window * 4 * threads;
}

bool single_launch_fits(const Program* p, int threads, size_t smem_optin) {
  if (windowed(*p))
    return window_smem_bytes(p, threads) <= smem_optin &&
           p->stats.fused.mem <= kMaxCompiledMemOps;
  return compiled_tier_fits(p, threads, smem_optin);
}

// Compile p's straight-line kernel once.  The compile itself runs without
// the lock so that several programs can compile at the same time.
bool jit_ensure(Program* p, int threads, std::string* err) {
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    if (p->jit) return true;
  }
  if (!jit_available()) {
    *err = "no run-time compiler";
    return false;
  }
  Program tmp;   // compile into a scratch holder, then publish
  tmp.fused = p->fused;
  tmp.sched = p->sched;
  tmp.load_group = p->load_group;
  tmp.n_in = p->n_in;
  tmp.n_out = p->n_out;
  tmp.minb = p->minb;
  tmp.stats = p->stats;
  if (!jit_compile(&tmp, threads, err)) return false;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (p->jit) {
    jit_release(&tmp);   // another thread won
  } else {
    p->jit = tmp.jit;
  }
  return true;
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return static_cast<EncodeTiledFn>(nullptr);
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

}  // namespace

int input_tensor_map(const xk::IoDesc& io, int n_in, int T, xk::TensorMap* out, int box_rows) {
  static_assert(sizeof(xk::TensorMap) == sizeof(CUtensorMap), "tensor map size");
  if (env_int("EC_TMA_TENSOR", 1) == 0) return 0;
  if (io.tab || !io.in_base || io.n_stripes < 1) return 0;
  const long long S = io.S;
  const uint64_t base = reinterpret_cast<uint64_t>(io.in_base);
  // strips equally spaced by S across the stripe's blocks; 16-byte rules
  if (n_in < 8 || n_in % 8 != 0 || n_in != 8 * io.n_inblk) return 0;
  const int es = 1 << xk::tmap_elem_shift(T);    // element bytes
  if (T % 16 != 0 || T / es < 4 || T / es > 256) return 0;
  if (S <= 0 || S % 16 != 0 || base % 16 != 0 || io.in_bstride != 8 * S) return 0;
  const long long plane = static_cast<long long>(n_in) * S;
  const long long sstride = io.n_stripes > 1 ? io.in_sstride : plane;
  if (sstride % 16 != 0 || sstride < plane || sstride >= (1ll << 40)) return 0;
  if (S / 4 > 0xffffffffll || io.n_stripes > 0xffffffffll) return 0;
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return 0;
  // box rows: the largest multiple of 8 strips that divides n_in and fits
  // a box dimension (256), so that the boxes tile the stage exactly; or the
  // window of a windowed program (rows past n_in are zero-filled)
  int rows = 8;
  for (int r = 256; r >= 8; r -= 8)
    if (n_in % r == 0) {
      rows = r;
      break;
    }
  if (box_rows > 0) {
    if (box_rows % 8 != 0 || box_rows > 256) return 0;
    rows = box_rows;
  }
  const cuuint64_t dim[3] = {static_cast<cuuint64_t>(S / es), static_cast<cuuint64_t>(n_in),
                             static_cast<cuuint64_t>(io.n_stripes)};
  const cuuint64_t stride[2] = {static_cast<cuuint64_t>(S), static_cast<cuuint64_t>(sstride)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(T / es), static_cast<cuuint32_t>(rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r =
      enc(reinterpret_cast<CUtensorMap*>(out),
          es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
          const_cast<uint8_t*>(io.in_base), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? rows : 0;
}

bool block_tensor_map_allowed(const void* block, long long S, int T) {
  if (env_int("EC_TMA_TENSOR", 1) == 0) return false;
  const uint64_t base = reinterpret_cast<uint64_t>(block);
  if (!block || base % 16 != 0 || S <= 0 || S % 16 != 0 || S / 4 > 0xffffffffll) return false;
  const int es = 1 << xk::tmap_elem_shift(T);
  if (T % 16 != 0 || T / es < 4 || T / es > 256) return false;
  return tensor_map_encoder() != nullptr;
}

bool block_tensor_map(const void* block, long long S, int T, xk::TensorMap* out) {
  if (!block_tensor_map_allowed(block, S, T)) return false;
  const EncodeTiledFn enc = tensor_map_encoder();
  const int es = 1 << xk::tmap_elem_shift(T);
  const cuuint64_t dim[2] = {static_cast<cuuint64_t>(S / es), 8};
  const cuuint64_t stride[1] = {static_cast<cuuint64_t>(S)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(T / es), 8};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      enc(reinterpret_cast<CUtensorMap*>(out),
          es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
          const_cast<void*>(block), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool launch_program(Program* p, const xk::IoDesc& io, int executor, cudaStream_t stream) {
  DeviceInfo di;
  if (!device_info(&di)) return false;
  if (io.n_stripes == 0 || io.S == 0) return true;
  bool compiled = false;
  int threads = 0, nstage = 0;
  if (executor == EC_EXEC_AUTO || executor == EC_EXEC_COMPILED) {
    threads = program_threads(p);
    nstage = env_int("EC_JIT_NSTAGE", 1);
    std::string err = "program too large for the compiled tier";
    compiled = single_launch_fits(p, threads, di.smem_optin) && jit_ensure(p, threads, &err);
    if (!compiled && executor == EC_EXEC_COMPILED) {
      set_error("compiled tier unavailable: " + err);
      return false;
    }
  }
  xk::LaunchParams lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.io = io;
  lp.n_in = p->n_in;
  lp.n_out = p->n_out;
  lp.status = di.status;
  size_t smem = 0;
  int per_sm = 0;
  const bool win = compiled && jit_is_windowed(p);
  if (compiled && win) {
    int w = 0, n_win = 0, n_phases = 0;
    window_layout(*p, &w, &n_win, &n_phases, nullptr);
    lp.T = 4 * threads;
    lp.win = w;
    lp.n_win = n_win;
    lp.n_phases = n_phases;
    smem = window_smem_bytes(p, threads);
    per_sm = jit_max_ctas_per_sm(p, threads, smem);
  } else if (compiled) {
    lp.T = 4 * threads;
    for (;; --nstage) {
      smem = interp_smem_bytes(p->n_in, 0, lp.T, nstage);
      if (smem <= di.smem_optin || nstage == 1) break;
    }
    if (smem > di.smem_optin) {
      compiled = false;   // too many inputs for the compiled tile: interpret
    } else {
      per_sm = jit_max_ctas_per_sm(p, threads, smem);
    }
  }
  const bool dense = !compiled && executor != EC_EXEC_INTERP;
  int dense_w = 0;
  int dense_form = 0;
  if (dense) {
    // the dense bitmatrix executor: windows of one block stream through a
    // ring; all output rows' accumulators in registers, in groups of 32
    if (!ensure_device_code(p)) return false;
    dense_w = dense_words();
    dense_form = xorec::dense_form();
    lp.T = 4 * dense_w * kDenseThreads;
    lp.win = kDenseWin;
    lp.n_win = p->n_in / kDenseWin;
    lp.n_phases = lp.n_win * ((p->n_out + 31) / 32);
    lp.code = p->d_code;
    lp.code_len = static_cast<int>(p->chunks.size() / 8);
    nstage = 1;
    smem = dense_smem_bytes(lp.T, dense_form);
    per_sm = dense_max_ctas_per_sm(dense_w, dense_form, false, smem);
  } else if (!compiled) {
    if (!ensure_device_code(p)) return false;
    // one stage (more resident CTAs hide more latency than a second stage
    // of the same CTA) and 8 bytes per thread and strip, halving per byte
    // the work of fetching and addressing each operand; the tile shrinks
    // (words, then threads) while it does not fit
    int words = env_int("EC_INTERP_WORDS", 2) == 1 ? 1 : 2;
    threads = env_int("EC_INTERP_THREADS", words == 2 ? 64 : 128);
    nstage = env_int("EC_INTERP_NSTAGE", 1);
    for (;;) {
      lp.T = 4 * words * threads;
      smem = interp_smem_bytes(p->n_in, p->interp_slots, lp.T, nstage);
      if (smem <= di.smem_optin) break;
      if (nstage > 1) { --nstage; continue; }
      if (words > 1) { words = 1; continue; }
      if (threads > 32) { threads /= 2; continue; }
      set_error("program needs more shared memory than one CTA can hold");
      return false;
    }
    lp.code = p->d_code;
    lp.code_len = static_cast<int>(p->chunks.size() / 8);
    lp.n_slots = p->interp_slots;
    per_sm = interp_max_ctas_per_sm(threads, smem, lp.T);
  }
  lp.nstage = nstage;
  lp.tiles_per_strip = (io.S + lp.T - 1) / lp.T;
  lp.n_items = io.n_stripes * lp.tiles_per_strip;
  if (per_sm < 1) per_sm = 1;
  long long grid = static_cast<long long>(di.sms) * per_sm;
  const int grid_env = env_int("EC_GRID", 0);
  if (grid_env > 0) grid = grid_env;
  if (grid > lp.n_items) grid = lp.n_items;
  if (compiled) {
    xk::TensorMap tm;
    lp.tmap = input_tensor_map(io, p->n_in, lp.T, &tm, win ? lp.win : 0);
    return jit_launch(p, lp, lp.tmap ? &tm : nullptr, threads, static_cast<int>(grid), smem,
                      stream);
  }
  if (dense) {
    xk::TensorMap tm;
    lp.tmap = input_tensor_map(io, p->n_in, lp.T, &tm, kDenseWin);
    return launch_dense(lp, lp.tmap ? &tm : nullptr, dense_w, dense_form,
                        static_cast<int>(grid),
                        smem, stream);
  }
  xk::TensorMap tm;
  lp.tmap = input_tensor_map(io, p->n_in, lp.T, &tm, 0);
  return launch_interp(lp, lp.tmap ? &tm : nullptr, threads, static_cast<int>(grid), smem, stream);
}

}  // namespace xorec

// ------------------------------------------------------------------ helpers

namespace {

}  // namespace

ec_status fail(ec_status s, const std::string& msg) {
  xorec::set_error(msg);
  return s;
}

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

ec_status check_block_bytes(size_t B) {
  if (B == 0 || B % 128 != 0) return fail(EC_EINVAL, "block_bytes must be a positive multiple of 128");
  return EC_OK;
}

// Upload a per-call pointer table with a stream-ordered allocation and run.
ec_status run_with_table(Program* p, const std::vector<uint64_t>& tab, int n_inblk, int n_outblk,
                         long long n_stripes, size_t B, int executor, cudaStream_t st) {
  const size_t bytes = tab.size() * sizeof(uint64_t);
  void* d = nullptr;
  if (xorec::dev_malloc_async(&d, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ENOMEM, "cudaMallocAsync of the block table failed");
  }
  if (cudaMemcpyAsync(d, tab.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(d, st);
    return fail(EC_ECUDA, "copy of the block table failed");
  }
  xk::IoDesc io;
  std::memset(&io, 0, sizeof(io));
  io.tab = static_cast<const xk::u64*>(d);
  io.n_inblk = n_inblk;
  io.n_outblk = n_outblk;
  io.S = static_cast<long long>(B / 8);
  io.n_stripes = n_stripes;
  const bool ok = xorec::launch_program(p, io, executor, st);
  cudaFreeAsync(d, st);
  return ok ? EC_OK : EC_ECUDA;
}

}  // namespace

// Decode program for a sorted erasure set (built on first use).
ec_status get_decode_program(ec_plan* plan, const std::vector<int>& er, Program** out) {
  xorec::TraceRange trace_("xorec plan decoder");
  {
    std::lock_guard<std::mutex> lk(plan->mu);
    auto it = plan->dec.find(er);
    if (it != plan->dec.end()) {
      *out = it->second.get();
      return EC_OK;
    }
  }
  const int k = plan->k, m = plan->m;
  std::vector<int> S;
  for (int id = 0, j = 0; id < k + m && static_cast<int>(S.size()) < k; ++id) {
    if (j < static_cast<int>(er.size()) && er[j] == id) { ++j; continue; }
    S.push_back(id);
  }
  std::vector<uint8_t> R;
  if (!xorec::decode_matrix(k, m, plan->P.data(), er, S, &R))
    return fail(EC_ESINGULAR, "survivor submatrix is singular for this erasure set");
  // Decoders run mostly inside batch modules, whose pipeline keeps about
  // eight registers of its own beside the program's values: their budget
  // stays that far below the register cap of the plan's module shape, so
  // that modules compile without spills.
  xorec::PlanOptions o = plan->opts;
  const int margin = xorec::env_int("EC_DECODE_REG_MARGIN", 8);
  if (8 * k <= xorec::kPreloadMaxInputs && margin > 0) {
    const int th = xorec::plan_module_threads(plan, 8 * k);
    const int minb = xorec::plan_module_minb(plan, 8 * k);
    const int cap = std::min(255, 65536 / (th * minb)) & ~7;
    o.reg_budget = std::max(32, std::min(o.reg_budget, cap - margin));
  }
  auto prog = std::make_unique<Program>();
  std::string err;
  if (!xorec::build_program(static_cast<int>(er.size()), k, R.data(), o, prog.get(), &err))
    return fail(EC_EINVAL, err);
  prog->threads = plan->tuned_threads;
  prog->minb = plan->tuned_minb;
  std::lock_guard<std::mutex> lk(plan->mu);
  auto it = plan->dec.find(er);
  if (it == plan->dec.end()) it = plan->dec.emplace(er, std::move(prog)).first;
  *out = it->second.get();
  return EC_OK;
}

ec_status canon_erasures(const ec_plan* plan, const int* erasures, int n, std::vector<int>* out) {
  if (n < 1) return fail(EC_EINVAL, "at least one erasure is required");
  if (n > plan->m) return fail(EC_ETOOMANY, "more erasures than parity blocks");
  if (!erasures) return fail(EC_EINVAL, "erasures is NULL");
  std::vector<int> e(erasures, erasures + n);
  for (int x : e)
    if (x < 0 || x >= plan->k + plan->m) return fail(EC_EINVAL, "erasure id out of range");
  std::sort(e.begin(), e.end());
  if (std::adjacent_find(e.begin(), e.end()) != e.end())
    return fail(EC_EINVAL, "duplicate erasure id");
  *out = e;
  return EC_OK;
}

namespace {

void release_program(Program* p) {
  if (!p) return;
  if (p->d_code) cudaFree(p->d_code);
  p->d_code = nullptr;
}

}  // namespace


// -------------------------------------------------------------- plan API

extern "C" {

const char* ec_last_error(void) { return xorec::g_last_error.c_str(); }

ec_status ec_program_check(const uint16_t* code, size_t len, int n_in, int n_out, int n_slots) {
  if ((!code && len) || n_in < 0 || n_out < 0 || n_slots < 0)
    return fail(EC_EINVAL, "bad argument");
  std::string err;
  if (!xorec::check_program_stream(code, len, n_in, n_out, n_slots, &err)) return fail(EC_EINVAL, err);
  return EC_OK;
}

ec_status ec_debug_fail_alloc(int n) {
  xorec::g_fail_allocs.store(std::max(0, n));
  return EC_OK;
}

ec_status ec_debug_inject_timeout(int n) {
  xorec::g_inject_timeouts.store(std::max(0, n));
  return EC_OK;
}

const char* ec_version(void) { return "xorec 0.1 (sm_103a)"; }

ec_status ec_plan_create_ex(int k, int m, int matrix_kind, const uint8_t* matrix,
                            const ec_plan_opts* opts, ec_plan** out) {
  xorec::TraceRange trace_("xorec plan create");
  if (!out) return fail(EC_EINVAL, "out is NULL");
  *out = nullptr;
  if (k < 1 || m < 1 || k + m > 256) return fail(EC_EINVAL, "need 1 <= k, 1 <= m, k + m <= 256");
  auto plan = std::make_unique<ec_plan>();
  plan->k = k;
  plan->m = m;
  plan->matrix_kind = matrix_kind;
  switch (matrix_kind) {
    case EC_MATRIX_CAUCHY: plan->P = xorec::cauchy_parity(k, m); break;
    case EC_MATRIX_POWER: plan->P = xorec::power_parity(k, m); break;
    case EC_MATRIX_CAUCHY_MIN: plan->P = xorec::cauchy_min_parity(k, m); break;
    case EC_MATRIX_USER:
      if (!matrix) return fail(EC_EINVAL, "EC_MATRIX_USER needs a matrix");
      plan->P.assign(matrix, matrix + static_cast<size_t>(k) * m);
      break;
    default: return fail(EC_EINVAL, "unknown matrix kind");
  }
  if (opts) {
    if (opts->opt_level < EC_OPT_RAW || opts->opt_level > EC_OPT_TRIPLE)
      return fail(EC_EINVAL, "bad opt_level");
    if (opts->sched != EC_SCHED_DFS && opts->sched != EC_SCHED_GREEDY)
      return fail(EC_EINVAL, "bad sched");
    if (opts->executor < EC_EXEC_AUTO || opts->executor > EC_EXEC_DENSE)
      return fail(EC_EINVAL, "bad executor");
    plan->opts.opt_level = opts->opt_level;
    plan->opts.sched = opts->sched;
    plan->opts.greedy_cap = opts->greedy_cap > 0 ? opts->greedy_cap : 128;
    plan->executor = opts->executor;
    if (opts->max_temps < -2) return fail(EC_EINVAL, "bad max_temps");
    plan->opts.max_temps = opts->max_temps;
    if (opts->reg_budget != 0 && (opts->reg_budget < 32 || opts->reg_budget > 255))
      return fail(EC_EINVAL, "reg_budget must be 0 or in [32, 255]");
    plan->opts.reg_budget = opts->reg_budget > 0 ? opts->reg_budget : 128;
    if (opts->stream_window < -1) return fail(EC_EINVAL, "bad stream_window");
    plan->opts.stream_window = opts->stream_window;
    if (opts->stream_temps < -1) return fail(EC_EINVAL, "bad stream_temps");
    plan->opts.stream_temps = opts->stream_temps;
  }
  plan->enc = std::make_unique<Program>();
  std::string err;
  if (!xorec::build_program(m, k, plan->P.data(), plan->opts, plan->enc.get(), &err))
    return fail(EC_EINVAL, err);
  if (plan->opts.reg_budget > 128) {
    // a register budget above the default cap of 128 registers also raises
    // the compiled kernels' cap (fewer resident CTAs per SM), as
    // ec_plan_set_launch does; smaller budgets keep the default cap
    const int th = xorec::program_threads(plan->enc.get());
    plan->tuned_threads = th;
    plan->tuned_minb = xorec::minb_for(th, plan->opts.reg_budget);
    plan->enc->threads = th;
    plan->enc->minb = plan->tuned_minb;
  }
  *out = plan.release();
  return EC_OK;
}

ec_status ec_plan_create(int k, int m, const uint8_t* matrix, ec_plan** out) {
  return ec_plan_create_ex(k, m, matrix ? EC_MATRIX_USER : EC_MATRIX_CAUCHY, matrix, nullptr, out);
}

void ec_plan_destroy(ec_plan* plan) {
  if (!plan) return;
  xorec::host_io_release(plan->hostio);
  for (void* mod : plan->modules) xorec::jit_module_release(mod);
  release_program(plan->enc.get());
  xorec::jit_release(plan->enc.get());
  for (auto& kv : plan->dec) {
    release_program(kv.second.get());
    xorec::jit_release(kv.second.get());
  }
  for (auto& p : plan->retired) {
    release_program(p.get());
    xorec::jit_release(p.get());
  }
  delete plan;
}

ec_status ec_plan_matrix(const ec_plan* plan, uint8_t* out) {
  if (!plan || !out) return fail(EC_EINVAL, "NULL argument");
  std::memcpy(out, plan->P.data(), plan->P.size());
  return EC_OK;
}

ec_status ec_plan_set_executor(ec_plan* plan, int executor) {
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  if (executor < EC_EXEC_AUTO || executor > EC_EXEC_DENSE) return fail(EC_EINVAL, "bad executor");
  if (executor == EC_EXEC_COMPILED && !xorec::jit_available())
    return fail(EC_ENOTSUP, "no run-time compiler available");
  plan->executor = executor;
  return EC_OK;
}

static void fill_stats(const xorec::SlpMetrics& m, ec_slp_stats* s) {
  s->xors = m.xors;
  s->mem = m.mem;
  s->nvar = m.nvar;
  s->stmts = m.stmts;
}

ec_status ec_plan_info(ec_plan* plan, const int* erasures, int n_erasures, ec_program_info* out) {
  if (!plan || !out) return fail(EC_EINVAL, "NULL argument");
  Program* p = plan->enc.get();
  if (erasures) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, erasures, n_erasures, &er);
    if (s != EC_OK) return s;
    s = get_decode_program(plan, er, &p);
    if (s != EC_OK) return s;
  }
  std::memset(out, 0, sizeof(*out));
  out->n_in = p->n_in;
  out->n_out = p->n_out;
  out->slots = p->n_slots;
  out->stmts = p->n_stmts;
  out->code_words = static_cast<int>(p->code.size());
  out->sched_nvar = p->stats.sched_nvar;
  fill_stats(p->stats.raw, &out->raw);
  fill_stats(p->stats.compressed, &out->compressed);
  fill_stats(p->stats.fused, &out->fused);
  out->compiled = p->jit != nullptr;
  out->regs = xorec::jit_regs(p);
  out->temps = p->stats.temps;
  out->max_live = p->stats.max_live;
  out->threads = xorec::program_threads(p);
  out->lop3 = static_cast<int>(p->stats.lop3);
  out->loads = static_cast<int>(p->stats.loads);
  out->window = p->stats.window;
  out->window_temps = p->stats.window_temps;
  return EC_OK;
}

ec_status ec_plan_program(ec_plan* plan, const int* erasures, int n_erasures, uint16_t* buf,
                          size_t len, size_t* need) {
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  Program* p = plan->enc.get();
  if (erasures) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, erasures, n_erasures, &er);
    if (s != EC_OK) return s;
    s = get_decode_program(plan, er, &p);
    if (s != EC_OK) return s;
  }
  if (need) *need = p->code.size();
  if (buf) std::memcpy(buf, p->code.data(), std::min(len, p->code.size()) * sizeof(uint16_t));
  return EC_OK;
}

ec_status ec_plan_dense_words(ec_plan* plan, const int* erasures, int n_erasures, uint32_t* buf,
                              size_t len, size_t* need) {
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  Program* p = plan->enc.get();
  if (erasures) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, erasures, n_erasures, &er);
    if (s != EC_OK) return s;
    s = get_decode_program(plan, er, &p);
    if (s != EC_OK) return s;
  }
  const size_t n = p->masks.size() + p->rowbits.size();
  if (need) *need = n;
  if (buf) {
    const size_t a = std::min(len, p->masks.size());
    std::memcpy(buf, p->masks.data(), a * sizeof(uint32_t));
    if (len > a)
      std::memcpy(buf + a, p->rowbits.data(), std::min(len - a, p->rowbits.size()) * sizeof(uint32_t));
  }
  return EC_OK;
}

ec_status ec_plan_kernel_source(ec_plan* plan, const int* erasures, int n_erasures, char* buf,
                                size_t len, size_t* need) {
  if (!plan) return fail(EC_EINVAL, "NULL plan");
  Program* p = plan->enc.get();
  if (erasures) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, erasures, n_erasures, &er);
    if (s != EC_OK) return s;
    s = get_decode_program(plan, er, &p);
    if (s != EC_OK) return s;
  }
  const std::string src = xorec::jit_source(*p, xorec::program_threads(p));
  if (need) *need = src.size() + 1;
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, src.size());
    std::memcpy(buf, src.data(), n);
    buf[n] = '\0';
  }
  return EC_OK;
}

ec_status ec_encode(ec_plan* plan, const uint8_t* const* data, uint8_t* const* parity,
                    size_t block_bytes, void* stream) {
  xorec::TraceRange trace_("xorec encode");
  if (!plan || !data || !parity) return fail(EC_EINVAL, "NULL argument");
  ec_status s = check_block_bytes(block_bytes);
  if (s != EC_OK) return s;
  std::vector<uint64_t> tab;
  for (int j = 0; j < plan->k; ++j) {
    if (!data[j] || !aligned16(data[j])) return fail(EC_EINVAL, "data block NULL or not 16-byte aligned");
    tab.push_back(reinterpret_cast<uint64_t>(data[j]));
  }
  for (int i = 0; i < plan->m; ++i) {
    if (!parity[i] || !aligned16(parity[i])) return fail(EC_EINVAL, "parity block NULL or not 16-byte aligned");
    tab.push_back(reinterpret_cast<uint64_t>(parity[i]));
  }
  return run_with_table(plan->enc.get(), tab, plan->k, plan->m, 1, block_bytes, plan->executor,
                        static_cast<cudaStream_t>(stream));
}

ec_status ec_encode_strided(ec_plan* plan, const uint8_t* data, size_t data_stripe_stride,
                            size_t data_block_stride, uint8_t* parity, size_t par_stripe_stride,
                            size_t par_block_stride, int n_stripes, size_t block_bytes,
                            void* stream) {
  xorec::TraceRange trace_("xorec encode strided");
  if (!plan || !data || !parity) return fail(EC_EINVAL, "NULL argument");
  if (n_stripes < 0) return fail(EC_EINVAL, "negative stripe count");
  ec_status s = check_block_bytes(block_bytes);
  if (s != EC_OK) return s;
  if (!aligned16(data) || !aligned16(parity) || data_stripe_stride % 16 || data_block_stride % 16 ||
      par_stripe_stride % 16 || par_block_stride % 16)
    return fail(EC_EINVAL, "bases and strides must be multiples of 16 bytes");
  if (n_stripes == 0) return EC_OK;
  xk::IoDesc io;
  std::memset(&io, 0, sizeof(io));
  io.in_base = data;
  io.in_sstride = static_cast<long long>(data_stripe_stride);
  io.in_bstride = static_cast<long long>(data_block_stride);
  io.out_base = parity;
  io.out_sstride = static_cast<long long>(par_stripe_stride);
  io.out_bstride = static_cast<long long>(par_block_stride);
  io.n_inblk = plan->k;
  io.n_outblk = plan->m;
  io.S = static_cast<long long>(block_bytes / 8);
  io.n_stripes = n_stripes;
  return xorec::launch_program(plan->enc.get(), io, plan->executor,
                               static_cast<cudaStream_t>(stream))
             ? EC_OK
             : EC_ECUDA;
}

ec_status ec_decode(ec_plan* plan, const int* erasures, int n_erasures,
                    const uint8_t* const* blocks, uint8_t* const* out, size_t block_bytes,
                    void* stream) {
  xorec::TraceRange trace_("xorec decode");
  if (!plan || !blocks || !out) return fail(EC_EINVAL, "NULL argument");
  std::vector<int> er;
  ec_status s = canon_erasures(plan, erasures, n_erasures, &er);
  if (s != EC_OK) return s;
  s = check_block_bytes(block_bytes);
  if (s != EC_OK) return s;
  Program* p = nullptr;
  s = get_decode_program(plan, er, &p);
  if (s != EC_OK) return s;
  const int k = plan->k, m = plan->m;
  std::vector<uint64_t> tab;
  for (int id = 0, j = 0; id < k + m && static_cast<int>(tab.size()) < k; ++id) {
    if (j < static_cast<int>(er.size()) && er[j] == id) { ++j; continue; }
    if (!blocks[id] || !aligned16(blocks[id]))
      return fail(EC_EINVAL, "surviving block NULL or not 16-byte aligned");
    tab.push_back(reinterpret_cast<uint64_t>(blocks[id]));
  }
  for (int e : er) {   // program outputs follow the sorted erasure order
    const int pos = static_cast<int>(std::find(erasures, erasures + n_erasures, e) - erasures);
    if (!out[pos] || !aligned16(out[pos])) return fail(EC_EINVAL, "output block NULL or not 16-byte aligned");
    tab.push_back(reinterpret_cast<uint64_t>(out[pos]));
  }
  return run_with_table(p, tab, k, static_cast<int>(er.size()), 1, block_bytes, plan->executor,
                        static_cast<cudaStream_t>(stream));
}

ec_status ec_decode_prepare(ec_plan* plan, const int* sets, const int* counts, int n_sets,
                            int n_threads) {
  if (!plan || (n_sets > 0 && (!sets || !counts))) return fail(EC_EINVAL, "NULL argument");
  std::vector<std::vector<int>> todo;
  size_t off = 0;
  for (int i = 0; i < n_sets; ++i) {
    std::vector<int> er;
    ec_status s = canon_erasures(plan, sets + off, counts[i], &er);
    if (s != EC_OK) return s;
    off += counts[i];
    todo.push_back(er);
  }
  if (n_threads <= 0) n_threads = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  std::atomic<size_t> next{0};
  std::atomic<int> rc{EC_OK};
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        const size_t i = next.fetch_add(1);
        if (i >= todo.size()) return;
        Program* p = nullptr;
        const ec_status s = get_decode_program(plan, todo[i], &p);
        if (s != EC_OK) rc.store(s);
      }
    });
  for (auto& th : pool) th.join();
  return static_cast<ec_status>(rc.load());
}

ec_status ec_plan_compile(ec_plan* plan, const int* sets, const int* counts, int n_sets,
                          int n_threads) {
  if (!plan || (n_sets > 0 && (!sets || !counts))) return fail(EC_EINVAL, "NULL argument");
  if (!xorec::jit_available()) return fail(EC_ENOTSUP, "no run-time compiler available");
  std::vector<Program*> progs;
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
    if (std::find(progs.begin(), progs.end(), p) == progs.end()) progs.push_back(p);
  }
  xorec::DeviceInfo di;
  if (!xorec::device_info(&di)) return EC_ECUDA;
  progs.erase(std::remove_if(progs.begin(), progs.end(),
                             [&](Program* p) {
                               return !xorec::single_launch_fits(p, xorec::program_threads(p),
                                                                 di.smem_optin);
                             }),
              progs.end());
  if (n_threads <= 0) n_threads = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  std::atomic<size_t> next{0};
  std::atomic<int> rc{EC_OK};
  std::string first_err;
  std::mutex err_mu;
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t)
    pool.emplace_back([&]() {
      for (;;) {
        const size_t i = next.fetch_add(1);
        if (i >= progs.size()) return;
        std::string err;
        if (!xorec::jit_ensure(progs[i], xorec::program_threads(progs[i]), &err)) {
          rc.store(EC_ECUDA);
          std::lock_guard<std::mutex> lk(err_mu);
          if (first_err.empty()) first_err = err;
        }
      }
    });
  for (auto& th : pool) th.join();
  if (rc.load() != EC_OK) return fail(EC_ECUDA, "compile failed: " + first_err);
  return EC_OK;
}

ec_status ec_device_status(int* status, int reset) {
  if (!status) return fail(EC_EINVAL, "NULL argument");
  xorec::DeviceInfo di;
  if (!xorec::device_info(&di)) return EC_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(EC_ECUDA, "cudaDeviceSynchronize failed");
  }
  int v = 0;
  if (cudaMemcpy(&v, di.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(EC_ECUDA, "reading the status word failed");
  if (reset && cudaMemset(di.status, 0, sizeof(int)) != cudaSuccess)
    return fail(EC_ECUDA, "resetting the status word failed");
  // the allocation-free encoder keeps its own word in its static scratch
  int w = 0;
  if (xorec::noalloc_status(di.device, &w, reset != 0) && w == xk::XK_STATUS_TIMEOUT)
    v = w;
  *status = v == xk::XK_STATUS_TIMEOUT ? EC_ETIMEOUT : 0;
  return EC_OK;
}

ec_status ec_selftest_wait_timeout(void* stream) {
  return xorec::launch_selftest_wait(static_cast<cudaStream_t>(stream)) ? EC_OK : EC_ECUDA;
}

ec_status ec_synth_fill(uint8_t* dst, size_t n, uint64_t seed, uint64_t offset, void* stream) {
  if (!dst && n) return fail(EC_EINVAL, "NULL destination");
  return xorec::launch_synth_fill(dst, n, seed, offset, static_cast<cudaStream_t>(stream))
             ? EC_OK
             : EC_ECUDA;
}

// ---------------------------------------------------------------- SLP API

struct ec_slp {
  xorec::Slp p;
};

static ec_status wrap(const xorec::Slp& p, ec_slp** out) {
  if (!out) return fail(EC_EINVAL, "out is NULL");
  *out = new ec_slp{p};
  return EC_OK;
}

ec_status ec_slp_parse(const char* text, ec_slp** out) {
  if (!text) return fail(EC_EINVAL, "NULL text");
  xorec::Slp p;
  std::string err;
  if (!xorec::parse_slp(text, &p, &err)) return fail(EC_EINVAL, err);
  return wrap(p, out);
}

ec_status ec_slp_from_matrix(int rows, int cols, const uint8_t* A, int form, ec_slp** out) {
  if (rows < 1 || cols < 1 || !A || (form != 0 && form != 1)) return fail(EC_EINVAL, "bad arguments");
  std::vector<xorec::Bits> R = xorec::bitmatrix_rows(rows, cols, A);
  std::vector<int> order;
  for (int i = 0; i < rows; ++i)
    for (int s = 7; s >= 0; --s) order.push_back(8 * i + s);
  return wrap(form == 0 ? xorec::slp_rows_fused(8 * cols, R, order)
                        : xorec::slp_rows_chains(8 * cols, R, order),
              out);
}

ec_status ec_slp_repair(const ec_slp* in, int xor_cancel, ec_slp** out) {
  if (!in) return fail(EC_EINVAL, "NULL program");
  return wrap(xorec::repair(in->p, xor_cancel != 0), out);
}

static bool single_assignment(const xorec::Slp& p) {
  std::vector<char> seen(p.n_var, 0);
  for (const auto& s : p.body) {
    if (seen[s.dst - p.n_const]) return false;
    seen[s.dst - p.n_const] = 1;
  }
  return true;
}

ec_status ec_slp_fuse(const ec_slp* in, int cancel_pairs, ec_slp** out) {
  if (!in) return fail(EC_EINVAL, "NULL program");
  if (!single_assignment(in->p)) return fail(EC_EINVAL, "fusion needs a single-assignment program");
  return wrap(xorec::fuse(in->p, cancel_pairs != 0), out);
}

ec_status ec_slp_schedule(const ec_slp* in, int kind, int cap, ec_slp** out) {
  if (!in) return fail(EC_EINVAL, "NULL program");
  if (!single_assignment(in->p)) return fail(EC_EINVAL, "scheduling needs a single-assignment program");
  xorec::Schedule s = kind == EC_SCHED_GREEDY ? xorec::schedule_greedy(in->p, cap, true)
                                              : xorec::schedule_dfs(in->p, true);
  return wrap(xorec::schedule_to_slp(in->p, s), out);
}

ec_status ec_slp_stats_get(const ec_slp* p, ec_slp_stats* out) {
  if (!p || !out) return fail(EC_EINVAL, "NULL argument");
  fill_stats(xorec::metrics(p->p), out);
  return EC_OK;
}

long ec_slp_iocost(const ec_slp* p, int cap) {
  if (!p || cap < 1) return -1;
  return xorec::lru_iocost(p->p, cap, nullptr);
}

int ec_slp_ccap(const ec_slp* p) { return p ? xorec::ccap(p->p) : -1; }

ec_status ec_slp_equivalent(const ec_slp* a, const ec_slp* b, int* eq) {
  if (!a || !b || !eq) return fail(EC_EINVAL, "NULL argument");
  *eq = xorec::equivalent(a->p, b->p) ? 1 : 0;
  return EC_OK;
}

ec_status ec_slp_to_text(const ec_slp* p, char* buf, size_t len, size_t* need) {
  if (!p) return fail(EC_EINVAL, "NULL program");
  const std::string s = xorec::slp_to_text(p->p);
  if (need) *need = s.size() + 1;
  if (buf && len) {
    const size_t n = std::min(len - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = '\0';
  }
  return EC_OK;
}

void ec_slp_destroy(ec_slp* p) { delete p; }

}  // extern "C"
