// Encode entry point that allocates nothing (ec_encode_noalloc).
//
// Why: some callers cannot allocate device memory at the moment they need
// to encode, for example code that runs inside another runtime's memory
// allocator or under a fixed, pre-planned device-memory budget where any
// cudaMalloc (or stream-ordered allocation) is forbidden or could fail.
// ec_encode allocates a small block table per call; this variant instead
// keeps its scratch (status word, block table, instruction stream) in one
// file-scope device array that every GPU loading the library holds until
// the process exits.
//
// The array is shared by every call: each call overwrites the table and
// the instruction stream, so calls whose work overlaps on the GPU (on
// different streams, or from different host threads) race with each other.
// The first call on a device does the set-up for that device (looks up the
// array's device address and clears the status word); make that first call
// before any stream capture.  Uses the interpreter executor, which is part
// of this library, so no module is loaded either.  A bounded wait of its
// kernel that times out is recorded in the array's status word, which
// ec_device_status reads (and clears on request) beside the device's own
// word.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/xorec.h"
#include "internal.h"

namespace {

constexpr size_t kStatusBytes = 256;
constexpr size_t kTableBytes = static_cast<size_t>(EC_NOALLOC_MAX_BLOCKS) * sizeof(uint64_t);
constexpr size_t kCodeBytes = static_cast<size_t>(EC_NOALLOC_MAX_CODE_WORDS) * sizeof(uint16_t);
constexpr size_t kScratchBytes = kStatusBytes + kTableBytes + kCodeBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_ptr[64] = {nullptr};

// Per-device set-up, with that device current: the host-side name of the
// array is only a stand-in, so the device address is looked up here.
ec_status scratch_for_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      xorec::set_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                       cudaGetErrorString(e));
      return EC_ECUDA;
    }
    if (cudaMemset(p, 0, kStatusBytes) != cudaSuccess) {
      cudaGetLastError();
      xorec::set_error("clearing the scratch status word failed");
      return EC_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return EC_OK;
}

}  // namespace

namespace xorec {

// Read (and optionally clear) the status word at the start of the scratch
// array of device `dev`; the kernels of ec_encode_noalloc write their
// timeouts there.  Plain copies, no allocation.
bool noalloc_status(int dev, int* value, bool reset) {
  unsigned char* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64 || !g_scratch_ptr[dev]) return false;
    p = g_scratch_ptr[dev];
  }
  int v = 0;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (reset && cudaMemset(p, 0, sizeof(int)) != cudaSuccess) cudaGetLastError();
  *value = v;
  return true;
}

}  // namespace xorec

namespace {

ec_status bad(ec_status s, const char* msg) {
  xorec::set_error(msg);
  return s;
}

}  // namespace

extern "C" ec_status ec_encode_noalloc(ec_plan* plan, const uint8_t* const* data,
                                       uint8_t* const* parity, size_t block_bytes,
                                       void* stream) {
  if (!plan || !data || !parity) return bad(EC_EINVAL, "NULL argument");
  if (block_bytes == 0 || block_bytes % 128 != 0)
    return bad(EC_EINVAL, "block_bytes must be a positive multiple of 128");
  const xorec::Program* p = plan->enc.get();
  const int nblk = plan->k + plan->m;
  if (nblk > EC_NOALLOC_MAX_BLOCKS)
    return bad(EC_EINVAL, "k + m exceeds the no-allocation block limit");
  if (p->chunks.size() > static_cast<size_t>(EC_NOALLOC_MAX_CODE_WORDS))
    return bad(EC_EINVAL, "encoding program exceeds the no-allocation limit of 32768 words");
  uint64_t tab[EC_NOALLOC_MAX_BLOCKS];
  for (int j = 0; j < plan->k; ++j) {
    if (!data[j] || (reinterpret_cast<uintptr_t>(data[j]) & 15u))
      return bad(EC_EINVAL, "data block NULL or not 16-byte aligned");
    tab[j] = reinterpret_cast<uint64_t>(data[j]);
  }
  for (int i = 0; i < plan->m; ++i) {
    if (!parity[i] || (reinterpret_cast<uintptr_t>(parity[i]) & 15u))
      return bad(EC_EINVAL, "parity block NULL or not 16-byte aligned");
    tab[plan->k + i] = reinterpret_cast<uint64_t>(parity[i]);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return bad(EC_ECUDA, "no CUDA device");
  }
  unsigned char* scratch = nullptr;
  ec_status s = scratch_for_device(dev, &scratch);
  if (s != EC_OK) return s;
  int sms = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return bad(EC_ECUDA, "cudaDeviceGetAttribute failed");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint64_t* d_tab = reinterpret_cast<uint64_t*>(scratch + kStatusBytes);
  uint16_t* d_code = reinterpret_cast<uint16_t*>(scratch + kStatusBytes + kTableBytes);
  if (cudaMemcpyAsync(d_tab, tab, nblk * sizeof(uint64_t), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      (!p->chunks.empty() &&
       cudaMemcpyAsync(d_code, p->chunks.data(), p->chunks.size() * sizeof(uint16_t),
                       cudaMemcpyHostToDevice, st) != cudaSuccess)) {
    cudaGetLastError();
    return bad(EC_ECUDA, "copy into the scratch array failed");
  }
  xk::LaunchParams lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.io.tab = reinterpret_cast<const xk::u64*>(d_tab);
  lp.io.n_inblk = plan->k;
  lp.io.n_outblk = plan->m;
  lp.io.S = static_cast<long long>(block_bytes / 8);
  lp.io.n_stripes = 1;
  lp.n_in = p->n_in;
  lp.n_out = p->n_out;
  lp.code = d_code;
  lp.code_len = static_cast<int>(p->chunks.size() / 8);
  lp.n_slots = p->interp_slots;
  lp.status = reinterpret_cast<int*>(scratch);
  // the interpreter's shape for single launches: one stage, 8 bytes per
  // thread and strip at 64 threads; the tile shrinks while it does not fit
  int threads = 64, words = 2;
  const int nstage = 1;
  size_t smem = 0;
  for (;;) {
    lp.T = 4 * words * threads;
    smem = xorec::interp_smem_bytes(p->n_in, p->interp_slots, lp.T, nstage);
    if (smem <= static_cast<size_t>(optin)) break;
    if (words > 1) { words = 1; continue; }
    if (threads > 32) { threads /= 2; continue; }
    return bad(EC_EINVAL, "program needs more shared memory than one CTA can hold");
  }
  lp.nstage = nstage;
  if (xorec::take_injected_timeout() &&
      !xorec::launch_selftest_wait_to(st, nullptr, lp.status))
    return EC_ECUDA;
  lp.tiles_per_strip = (lp.io.S + lp.T - 1) / lp.T;
  lp.n_items = lp.tiles_per_strip;
  int per_sm = xorec::interp_max_ctas_per_sm(threads, smem, lp.T);
  if (per_sm < 1) per_sm = 1;
  long long grid = static_cast<long long>(sms) * per_sm;
  if (grid > lp.n_items) grid = lp.n_items;
  return xorec::launch_interp(lp, nullptr, threads, static_cast<int>(grid), smem, st) ? EC_OK
                                                                                      : EC_ECUDA;
}
