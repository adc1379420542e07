// Host-side internals shared by the C ABI, the executors and the compiled
// tier.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/xorec.h"
#include "plan.h"
#include "tile_pipeline.cuh"

struct xorec_host_io;   // host-memory encode lanes (hostio.cc)

struct ec_plan {
  int k = 0, m = 0;
  int matrix_kind = 0;
  std::vector<uint8_t> P;                    // m x k parity rows
  xorec::PlanOptions opts;
  int executor = 0;                          // EC_EXEC_*
  std::unique_ptr<xorec::Program> enc;
  std::mutex mu;                             // guards dec and modules
  std::map<std::vector<int>, std::unique_ptr<xorec::Program>> dec;  // key: sorted erasures
  std::vector<void*> modules;                // compiled multi-program modules (batches)
  xorec_host_io* hostio = nullptr;           // lanes and staging of ec_encode_host_strided
  std::mutex hostio_mu;                      // one host-memory encode enqueues at a time
  int tuned_threads = 0, tuned_minb = 0;     // compiled-tier launch shape from the autotuner
  std::vector<std::unique_ptr<xorec::Program>> retired;  // encoders replaced by the autotuner
};

// Shared by the C ABI translation units.
ec_status fail(ec_status s, const std::string& msg);
ec_status canon_erasures(const ec_plan* plan, const int* erasures, int n, std::vector<int>* out);
ec_status get_decode_program(ec_plan* plan, const std::vector<int>& er, xorec::Program** out);

namespace xorec {

void set_error(const std::string& msg);

// Device and pinned-host allocations of the library.  ec_debug_fail_alloc
// makes the n-th one from now fail as if memory ran out (host-side fault
// injection for the tests; no GPU fault is involved).
bool take_injected_alloc_failure();
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  if (take_injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t st) {
  if (take_injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, st);
}
template <class T>
cudaError_t host_malloc_pinned(T** p, size_t bytes) {
  if (take_injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}
// Pinned host memory that kernels address directly (cudaHostGetDevicePointer).
template <class T>
cudaError_t host_malloc_mapped(T** p, size_t bytes) {
  if (take_injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(reinterpret_cast<void**>(p), bytes, cudaHostAllocMapped);
}

// NVTX range for the duration of a scope (plan, compile, encode, decode,
// batch and serving steps show up on an nsys or ncu timeline).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Host check of an interpreter stream before it is uploaded or compiled:
// every statement well formed, operands below n_in + n_slots, slots written
// before they are read, output strips below n_out.  The format is the one
// Program documents.
bool check_program_stream(const uint16_t* code, size_t len, int n_in, int n_out, int n_slots,
                          std::string* err);

// Per-device state: SM count, status word.
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  size_t smem_optin = 0;
  int* status = nullptr;     // device word written by kernels on timeout
};
bool device_info(DeviceInfo* out);

// Upload the program's interpreter stream to the device (once).
bool ensure_device_code(Program* p);

struct LaunchShape {
  int threads = 128;   // threads per CTA; T = 4 * threads
  int nstage = 2;
  int grid = 0;        // 0 = one persistent wave
};

// Fill `io`-addressed launch parameters and run the interpreter or the
// compiled kernel of `p` over n_stripes stripes of strip length S.
bool launch_program(Program* p, const xk::IoDesc& io, int executor, cudaStream_t stream);

// Interpreter launch (executor.cu).
bool launch_interp(const xk::LaunchParams& lp, const xk::TensorMap* tm, int threads, int grid,
                   size_t smem, cudaStream_t stream);
size_t interp_smem_bytes(int n_in, int n_slots, int T, int nstage);
int interp_max_ctas_per_sm(int threads, size_t smem, int T);

// Batched interpreter (executor.cu).
size_t interp_batch_smem_bytes(int max_in, int max_slots, int T);
int interp_batch_max_ctas_per_sm(int threads, size_t smem);
bool launch_interp_batch(const xk::BatchParams& bp, int threads, int grid, size_t smem,
                         cudaStream_t stream);

// Dense bitmatrix executor (executor.cu): words per consumer thread and
// strip, mask or table form, shared memory of a launch with tiles of T
// bytes, resident CTAs, single and batched launches (kDenseThreads
// consumers, windows of kDenseWin strips; the control words follow the
// chunk stream in the program's device buffer).
constexpr int kDenseThreads = 128;
constexpr int kDenseWin = 8;
int dense_words();
int dense_form();
size_t dense_smem_bytes(int T, int form);
int dense_max_ctas_per_sm(int W, int form, bool batch, size_t smem);
bool launch_dense(const xk::LaunchParams& lp, const xk::TensorMap* tm, int W, int form,
                  int grid, size_t smem, cudaStream_t stream);
bool launch_dense_batch(const xk::BatchParams& bp, int W, int form, int grid, size_t smem,
                        cudaStream_t stream);

// Compiled tier (jit.cc).
bool jit_available();
bool jit_ensure(Program* p, int threads, std::string* err);
bool compiled_tier_fits(const Program* p, int threads, size_t smem_optin);
// A single launch of `p` fits the compiled tier: its shared memory (the
// windowed ring, or a stage of every input strip) and its code size.
bool single_launch_fits(const Program* p, int threads, size_t smem_optin);
// Threads per CTA of a launch whose tile holds n_in input strips when no
// shape was chosen: `threads`, halved (not below 64) while two CTAs' tiles
// do not fit one CTA's shared memory, so that an SM keeps at least two CTAs
// and overlaps one's copies with the other's XORs.
int tile_threads_for_inputs(int n_in, int threads);
// Threads per CTA of p's compiled tier: the tuned or pinned shape, else
// EC_JIT_THREADS, else tile_threads_for_inputs(n_in, 128).
int program_threads(const Program* p);
// Consumer threads of a windowed single launch, or of a windowed batch module.
int window_threads(bool module);
// Resident CTAs per SM (the __launch_bounds__ minimum) that leave each of
// `threads` threads reg_budget registers of the SM's 65,536.
int minb_for(int threads, int reg_budget);
// Resident CTAs per SM of a compiled kernel with no tuned shape: a
// 128-register cap, or 168 for preloaded programs of more than
// kPreloadCap128Inputs input strips.
int default_minb(int threads, int n_in);
bool jit_compile(Program* p, int threads, std::string* err);
// Two-level programs that stream their inputs window by window through a
// small ring (run_window_pipeline): the layout of their phases (jit.cc).
bool window_layout(const Program& p, int* win, int* n_win, int* n_phases,
                   std::vector<int>* phase);
// The compiled tier runs `p` with the windowed pipeline (EC_WINDOWED=0
// turns it off).
bool windowed(const Program& p);
// The compiled kernel of `p` exists and is the windowed form (its launch
// follows the kernel, whatever EC_WINDOWED says later).
bool jit_is_windowed(const Program* p);
// A module of `progs` takes the batched windowed pipeline (jit.cc): its
// window and windows per item.
bool window_module(const std::vector<const Program*>& progs, int* win, int* n_win);
// The module is windowed: its window and windows per item.
bool jit_module_window(void* mod, int* win, int* n_win);
bool jit_launch(Program* p, const xk::LaunchParams& lp, const xk::TensorMap* tm, int threads,
                int grid, size_t smem, cudaStream_t stream);
// Tensor map of a strided launch's inputs as [stripe][input strip][element]
// (4-byte elements, 8-byte ones for tiles over 1 KiB: xk::tmap_elem_shift)
// with a box of one tile of up to 256 input strips; returns the strips per
// box (a multiple of 8 that divides n_in), or 0 (no map) when the layout or
// the driver does not allow one.
int input_tensor_map(const xk::IoDesc& io, int n_in, int T, xk::TensorMap* out, int box_rows);
// Tensor map of one block as [strip][element] (8 strips S bytes apart)
// with a box of one tile of its 8 strips; false when not allowed.
bool block_tensor_map(const void* block, long long S, int T, xk::TensorMap* out);
bool block_tensor_map_allowed(const void* block, long long S, int T);
int jit_max_ctas_per_sm(Program* p, int threads, size_t smem);
void jit_release(Program* p);
int jit_regs(const Program* p);
std::string jit_source(const Program& p, int threads);
void* jit_compile_module(const std::vector<const Program*>& progs, int threads, int minb,
                         std::string* err, bool no_spill);
std::string jit_module_source(const std::vector<const Program*>& progs, int threads, int minb);
int jit_module_ctas_per_sm(void* mod, size_t smem);
bool jit_module_launch(void* mod, const xk::BatchParams& bp, int grid, size_t smem,
                       cudaStream_t stream);
void jit_module_release(void* mod);
int jit_module_regs(void* mod);
int jit_module_threads(void* mod);

void host_io_release(xorec_host_io* h);

// Batch helpers (batch.cc), shared with the serving loop.
ec_status resolve_job(const ec_job& j, Program** prog, std::vector<int>* er,
                      std::vector<uint64_t>* ptrs);
int launch_threads(void* mod);
int launch_tile(void* mod, bool interp, int threads);
bool batch_launch(void* mod, bool interp, const xk::BatchParams& bp, int threads, int grid,
                  size_t smem, cudaStream_t st, int dense_w, int dense_form);
// Launch shape of a plan's batch modules for programs of n_in input strips:
// the autotuner's (or ec_plan_set_launch's) shape, else the defaults.
int plan_module_threads(const ec_plan* p, int n_in);
int plan_module_minb(const ec_plan* p, int n_in);
ec_status compile_modules(const std::vector<std::pair<ec_plan*, Program*>>& want, bool must,
                          int* built);
bool batch_launch_shape(void* mod, bool interp, int max_in, int max_slots, int threads,
                        size_t smem_optin, size_t* smem, int* per_sm, int dense_w,
                        int dense_form);
int batch_ranges(long long n_items, int sms, int per_sm, int chunk, int max_in, bool dense);
// Split a launch's items into n_ranges contiguous ranges (BatchParams).
void set_ranges(xk::BatchParams* bp, long long n_items, int n_ranges);

// Bounded-wait self-test (executor.cu): a one-thread kernel whose wait
// gives up after its limit and records the timeout in `status` (the
// device's word) and, when not null, `also` (a batch's, slot's or the
// allocation-free encoder's own word).
bool launch_selftest_wait(cudaStream_t stream);
bool launch_selftest_wait_to(cudaStream_t stream, int* status, int* also);
// ec_debug_inject_timeout: true (once per count) when the next batched run,
// serving dispatch or allocation-free encode should be preceded by the
// self-test wait on its status words.
bool take_injected_timeout();

// Status word of the allocation-free encoder on device `dev` (noalloc.cu):
// false when that device has not run it yet; reset clears the word.
bool noalloc_status(int dev, int* value, bool reset);

// Synthetic input generator (executor.cu).
bool launch_synth_fill(uint8_t* dst, size_t n, uint64_t seed, uint64_t offset,
                       cudaStream_t stream);

}  // namespace xorec
