// Encoding from host memory: chunks of stripes go host -> device, are
// encoded and their parity comes back, on a few lanes (streams) so that
// both copy directions and the kernels overlap.  Each lane owns a device
// staging buffer that it reuses in stream order; the buffers belong to the
// plan and grow when a larger chunk is requested.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int kLanes = 3;

}  // namespace

struct xorec_host_io {
  int device = -1;
  cudaStream_t lane[kLanes] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t done[kLanes] = {};
  uint8_t* dbuf[kLanes] = {};
  size_t cap = 0;                       // bytes per lane buffer
};

namespace xorec {

void host_io_release(xorec_host_io* h) {
  if (!h) return;
  for (int i = 0; i < kLanes; ++i) {
    if (h->lane[i]) cudaStreamDestroy(h->lane[i]);
    if (h->done[i]) cudaEventDestroy(h->done[i]);
    if (h->dbuf[i]) cudaFree(h->dbuf[i]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  delete h;
}

}  // namespace xorec

namespace {

ec_status ensure_io(ec_plan* plan, size_t bytes, xorec_host_io** out) {
  std::lock_guard<std::mutex> lk(plan->mu);
  xorec_host_io*& h = plan->hostio;
  if (!h) {
    h = new xorec_host_io();
    cudaGetDevice(&h->device);
    if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(EC_ECUDA, "cudaEventCreate failed");
    }
    for (int i = 0; i < kLanes; ++i)
      if (cudaStreamCreateWithFlags(&h->lane[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->done[i], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(EC_ECUDA, "stream creation failed");
      }
  }
  if (bytes > h->cap) {
    for (int i = 0; i < kLanes; ++i) {
      if (h->dbuf[i]) {
        cudaStreamSynchronize(h->lane[i]);
        cudaFree(h->dbuf[i]);
        h->dbuf[i] = nullptr;
      }
      if (xorec::dev_malloc(&h->dbuf[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        h->cap = 0;
        return fail(EC_ENOMEM, "device staging allocation failed");
      }
    }
    h->cap = bytes;
  }
  *out = h;
  return EC_OK;
}

}  // namespace

extern "C" ec_status ec_encode_host_strided(ec_plan* plan, const uint8_t* data,
                                            size_t data_stripe_stride, size_t data_block_stride,
                                            uint8_t* parity, size_t par_stripe_stride,
                                            size_t par_block_stride, int n_stripes,
                                            size_t block_bytes, int chunk_stripes, void* stream) {
  xorec::TraceRange trace_("xorec encode from host");
  if (!plan || !data || !parity) return fail(EC_EINVAL, "NULL argument");
  if (n_stripes < 0) return fail(EC_EINVAL, "negative stripe count");
  if (block_bytes == 0 || block_bytes % 128 != 0)
    return fail(EC_EINVAL, "block_bytes must be a positive multiple of 128");
  if (n_stripes == 0) return EC_OK;
  // the plan's lanes, staging and fork/join events are shared: enqueue one
  // call at a time (the lanes' stream order then keeps staging reuse safe)
  std::lock_guard<std::mutex> io_lock(plan->hostio_mu);
  const int k = plan->k, m = plan->m;
  const int chunk = chunk_stripes > 0 ? std::min(chunk_stripes, n_stripes) : std::min(16, n_stripes);
  const size_t din = static_cast<size_t>(k) * block_bytes;    // device data per stripe
  const size_t dout = static_cast<size_t>(m) * block_bytes;
  xorec_host_io* h = nullptr;
  ec_status s = ensure_io(plan, static_cast<size_t>(chunk) * (din + dout), &h);
  if (s != EC_OK) return s;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (cudaEventRecord(h->fork, caller) != cudaSuccess) return fail(EC_ECUDA, "cudaEventRecord failed");
  for (int i = 0; i < kLanes; ++i)
    if (cudaStreamWaitEvent(h->lane[i], h->fork, 0) != cudaSuccess)
      return fail(EC_ECUDA, "cudaStreamWaitEvent failed");
  const bool dense_in = data_block_stride == block_bytes && data_stripe_stride == din;
  const bool dense_out = par_block_stride == block_bytes && par_stripe_stride == dout;
  int li = 0;
  for (int c0 = 0; c0 < n_stripes; c0 += chunk, li = (li + 1) % kLanes) {
    const int n = std::min(chunk, n_stripes - c0);
    cudaStream_t st = h->lane[li];
    uint8_t* d_in = h->dbuf[li];
    uint8_t* d_out = h->dbuf[li] + static_cast<size_t>(chunk) * din;
    // host -> device: the chunk's data blocks, packed [stripe][block][B]
    if (dense_in) {
      if (cudaMemcpyAsync(d_in, data + static_cast<size_t>(c0) * din, n * din,
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(EC_ECUDA, "host to device copy failed");
    } else {
      for (int i = 0; i < n; ++i)
        if (cudaMemcpy2DAsync(d_in + i * din, block_bytes,
                              data + static_cast<size_t>(c0 + i) * data_stripe_stride,
                              data_block_stride, block_bytes, k, cudaMemcpyHostToDevice,
                              st) != cudaSuccess)
          return fail(EC_ECUDA, "host to device copy failed");
    }
    xk::IoDesc io;
    std::memset(&io, 0, sizeof(io));
    io.in_base = d_in;
    io.in_sstride = static_cast<long long>(din);
    io.in_bstride = static_cast<long long>(block_bytes);
    io.out_base = d_out;
    io.out_sstride = static_cast<long long>(dout);
    io.out_bstride = static_cast<long long>(block_bytes);
    io.n_inblk = k;
    io.n_outblk = m;
    io.S = static_cast<long long>(block_bytes / 8);
    io.n_stripes = n;
    if (!xorec::launch_program(plan->enc.get(), io, plan->executor, st)) return EC_ECUDA;
    // device -> host: the chunk's parity blocks
    if (dense_out) {
      if (cudaMemcpyAsync(parity + static_cast<size_t>(c0) * dout, d_out, n * dout,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail(EC_ECUDA, "device to host copy failed");
    } else {
      for (int i = 0; i < n; ++i)
        if (cudaMemcpy2DAsync(parity + static_cast<size_t>(c0 + i) * par_stripe_stride,
                              par_block_stride, d_out + i * dout, block_bytes, block_bytes, m,
                              cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return fail(EC_ECUDA, "device to host copy failed");
    }
  }
  for (int i = 0; i < kLanes; ++i)
    if (cudaEventRecord(h->done[i], h->lane[i]) != cudaSuccess ||
        cudaStreamWaitEvent(caller, h->done[i], 0) != cudaSuccess)
      return fail(EC_ECUDA, "joining the copy lanes failed");
  return EC_OK;
}
