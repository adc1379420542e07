// Device-side tile pipeline shared by the SLP interpreter (compiled into the
// library) and the straight-line SLP kernels compiled per plan at run time.
// This header includes nothing so that it compiles both under nvcc and NVRTC.
//
// Work decomposition (blocking, Sec. 6.1, retargeted): every stripe's strips
// are cut into tiles of T bytes; one work item = (stripe, tile).  A CTA walks
// items blockIdx.x, blockIdx.x + gridDim.x, ...; for each item one warp
// stages every input strip's tile in shared memory with TMA (one tiled
// tensor copy per item for strided inputs, one per input block in batches,
// else one 1-D bulk copy per strip), completion is tracked by an mbarrier
// with a transaction count, and every thread then runs the XOR program on
// its own 4-byte column of the tile.  `nstage` stages form a ring so that the copies of the next
// items overlap the computation of the current one.  Every input byte is
// read from HBM once and every output byte written once.
//
// Waits are bounded: an mbarrier wait that exceeds ~2 s of %globaltimer sets
// the status word to XK_STATUS_TIMEOUT (batched launches also set their
// batch's or serving slot's own word), waits (bounded again) for the CTA's
// copies still in flight and returns.
#pragma once

namespace xk {

typedef unsigned char u8;
typedef unsigned short u16;
typedef unsigned int u32;
typedef unsigned long long u64;
typedef long long i64;

enum { XK_STATUS_OK = 0, XK_STATUS_TIMEOUT = 1 };

// Block addressing for a launch.  Either a device table with, per stripe,
// n_inblk input block addresses followed by n_outblk output block
// addresses, or (tab == 0) strided bases.
struct IoDesc {
  const u64* tab;
  const u8* in_base;
  i64 in_sstride, in_bstride;
  u8* out_base;
  i64 out_sstride, out_bstride;
  int n_inblk, n_outblk;
  i64 S;          // strip bytes (block bytes / 8)
  i64 n_stripes;
};

// Opaque TMA tensor map (the driver's 128-byte descriptor), passed to
// kernels as a __grid_constant__ parameter.
struct alignas(64) TensorMap {
  u64 opaque[16];
};

struct LaunchParams {
  IoDesc io;
  int n_in, n_out;       // input / output strips (8 per block)
  int T;                 // tile bytes per strip (multiple of 16)
  int nstage;            // stages in the shared-memory ring
  int tmap;              // > 0: the kernel's tensor map describes the inputs
                         // as [stripe][input strip][4-byte word] with boxes
                         // of tmap strips (tmap divides n_in), and n_in/tmap
                         // 3-D copies fill a stage; 0: per-strip copies
  i64 tiles_per_strip;
  i64 n_items;
  const u16* code;       // interpreter stream (unused by compiled kernels)
  int code_len;
  int n_slots;
  int* status;
  // windowed programs (run_window_pipeline): input strips per window, windows
  // per group of rows, phases per item (groups x windows); 0 otherwise
  int win, n_win, n_phases, pad_;
};

// Window slots in the shared-memory ring of windowed programs.
constexpr int kWinRing = 4;

// Tensor maps address a strip in 4-byte elements, or in 8-byte elements
// when a tile is wider than a box dimension (at most 256 elements) of
// 4-byte elements holds: log2 of the element size for tiles of T bytes.
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
__host__ __device__
#endif
constexpr int tmap_elem_shift(int T) { return T > 1024 ? 3 : 2; }

// Batched launches: every stripe has its own program, strip length and
// blocks.  Work items are (stripe, tile) pairs listed in `items`.
struct StripeDesc {
  const u64* blocks;     // n_inblk input block addresses, then n_outblk outputs
  i64 S;                 // strip bytes (block bytes / 8)
  i64 item_base;         // index of the stripe's first item in the launch
  const u16* code;       // interpreter stream of the stripe's program
  int code_len;
  int n_slots;
  int n_inblk, n_outblk;
  int prog;              // program index inside a compiled module
  int pad_;
  const TensorMap* maps; // n_inblk tensor maps (input block j as [strip][element],
                         // box = one tile of its 8 strips), or null:
                         // one 1-D copy per strip
};

struct BatchParams {
  const StripeDesc* stripes;   // the launch's stripes; item_base is increasing
  int n_stripes;
  int chunk;                   // consecutive items a CTA takes from the queue at a time
  u64* queue;                  // n_ranges work-queue heads (chunks handed out), zero at launch
  i64 n_items;
  int T;                   // tile bytes per strip
  int max_in;              // largest n_in (strips) of the launch: stage size
  int* status;             // the device's status word
  int n_ranges;            // items split into this many contiguous ranges, one
                           // per SM (<= 1: one queue for all items)
  int range_rem;           // n_items % n_ranges
  i64 range_len;           // n_items / n_ranges
  int* local_status;       // the batch's or serving slot's own status word, or null
  // windowed modules (run_batch_window_pipeline): input strips per window,
  // windows per item (= phases: the programs have one group of rows); 0
  // otherwise
  int win, n_win;
};

// Shared-memory header of batched launches: the mbarrier (bytes 0..7), the
// item ring (64..95), warp 0's work-queue state (128..191) and the table of
// the next item's source addresses (one per strip, from byte 256).
constexpr int kMaxPrepared = 128;
constexpr int kBatchHeader = 256 + 8 * kMaxPrepared;
constexpr int kRing = 4;

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)

__device__ __forceinline__ const u8* in_block(const IoDesc& io, i64 s, int b) {
  if (io.tab) return reinterpret_cast<const u8*>(io.tab[s * (io.n_inblk + io.n_outblk) + b]);
  return io.in_base + s * io.in_sstride + b * io.in_bstride;
}

__device__ __forceinline__ u8* out_block(const IoDesc& io, i64 s, int b) {
  if (io.tab)
    return reinterpret_cast<u8*>(io.tab[s * (io.n_inblk + io.n_outblk) + io.n_inblk + b]);
  return io.out_base + s * io.out_sstride + b * io.out_bstride;
}

__device__ __forceinline__ u32 smem_addr(const void* p) {
  u32 r;
  asm("{ .reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t; }" : "=r"(r) : "l"(p));
  return r;
}

__device__ __forceinline__ u64 now_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(u32 bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u32 bar, u32 bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }"
               ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_1d(u32 dst, const void* src, u32 bytes, u32 bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// One tiled 2-D TMA copy (box given by the tensor map) into shared memory;
// coordinates in elements, innermost first.
__device__ __forceinline__ void tma_load_2d(u32 dst, const TensorMap* tm, int x, int y, u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<u64>(tm)), "r"(x), "r"(y), "r"(bar) : "memory");
}

// One tiled 3-D TMA copy (box given by the tensor map) into shared memory;
// coordinates in elements, innermost first.
__device__ __forceinline__ void tma_load_3d(u32 dst, const TensorMap* tm, int x, int y, int z,
                                            u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<u64>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u32 bar, u32 parity) {
  u32 ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase with `parity` completed, false after
// about two seconds.
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const u64 t0 = now_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (now_ns() - t0 > 2000000000ull) return false;
  }
}

// Warp 0 issues the copies of one work item into stage `dst`: one tiled
// copy of every input strip's tile when the launch has a tensor map (the
// box is n_in x T bytes; past the end of a strip it is zero-filled and still
// counts in full), else one 1-D bulk copy per strip.
__device__ __forceinline__ void issue_item(const LaunchParams& p, const TensorMap* tm, i64 item,
                                           u8* dst, u32 bar) {
  const i64 s = item / p.tiles_per_strip;
  const i64 c0 = (item % p.tiles_per_strip) * p.T;
  const int lane = threadIdx.x & 31;
  if (p.tmap == p.n_in) {
    if (lane == 0) {
      mbar_arrive_expect_tx(bar, static_cast<u32>(p.n_in) * static_cast<u32>(p.T));
      tma_load_3d(smem_addr(dst), tm, static_cast<int>(c0 >> tmap_elem_shift(p.T)), 0,
                  static_cast<int>(s), bar);
    }
    return;
  }
  if (p.tmap > 0) {
    // more strips than one box holds: one copy per box of tmap strips,
    // spread over the warp's lanes
    if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<u32>(p.n_in) * static_cast<u32>(p.T));
    __syncwarp();
    for (int y = lane * p.tmap; y < p.n_in; y += 32 * p.tmap)
      tma_load_3d(smem_addr(dst + static_cast<i64>(y) * p.T), tm,
                  static_cast<int>(c0 >> tmap_elem_shift(p.T)), y,
                  static_cast<int>(s), bar);
    return;
  }
  const i64 rest = p.io.S - c0;
  const int len = rest < p.T ? static_cast<int>(rest) : p.T;
  if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<u32>(p.n_in) * static_cast<u32>(len));
  __syncwarp();
  for (int c = lane; c < p.n_in; c += 32) {
    const u8* src = in_block(p.io, s, c >> 3) + static_cast<i64>(c & 7) * p.io.S + c0;
    tma_load_1d(smem_addr(dst + static_cast<i64>(c) * p.T), src, static_cast<u32>(len), bar);
  }
}

// Shared memory: [mbarriers, 128 B][nstage stages of n_in * T][slots].
// A Body either reads its operands from the stage while it computes
// (kEarlyRelease = false):
//   void operator()(const LaunchParams&, i64 stripe, i64 c0, int len,
//                   const u8* stage, u8* slots) const
// or first copies its column of every input strip into registers and
// computes from there (kEarlyRelease = true), which frees the stage for the
// next copy before the XOR work starts:
//   void load(const LaunchParams&, int len, const u8* stage, Regs&) const
//   void compute(const LaunchParams&, i64 stripe, i64 c0, int len, Regs&) const
template <class Body>
__device__ __forceinline__ void run_pipeline(const LaunchParams& p, u8* smem, const Body& body,
                                             const TensorMap* tm) {
  u64* bars = reinterpret_cast<u64*>(smem);
  u8* stages = smem + 128;
  const i64 stage_bytes = static_cast<i64>(p.n_in) * p.T;
  u8* slots = stages + p.nstage * stage_bytes;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < p.nstage; ++s) mbar_init(smem_addr(&bars[s]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  const i64 first = blockIdx.x, step = gridDim.x;
  if (tid < 32) {
    for (int s = 0; s < p.nstage; ++s) {
      const i64 it = first + s * step;
      if (it < p.n_items) issue_item(p, tm, it, stages + s * stage_bytes, smem_addr(&bars[s]));
    }
  }
  for (i64 i = 0;; ++i) {
    const i64 item = first + i * step;
    if (item >= p.n_items) break;
    const int st = static_cast<int>(i % p.nstage);
    const u32 par = static_cast<u32>((i / p.nstage) & 1);
    const bool ok = mbar_wait(smem_addr(&bars[st]), par);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(p.status, XK_STATUS_TIMEOUT);
        for (int d = 0; d < p.nstage; ++d) {
          const i64 j = i + d;
          if (first + j * step < p.n_items)
            mbar_wait(smem_addr(&bars[j % p.nstage]), static_cast<u32>((j / p.nstage) & 1));
        }
      }
      return;
    }
    const i64 s = item / p.tiles_per_strip;
    const i64 c0 = (item % p.tiles_per_strip) * p.T;
    const i64 rest = p.io.S - c0;
    const int len = rest < p.T ? static_cast<int>(rest) : p.T;
    const i64 nxt = item + p.nstage * step;
    if constexpr (Body::kEarlyRelease) {
      // Copy this thread's input words into registers, hand the stage back
      // to the copy engine at once, then run the program from registers.
      typename Body::Regs r;
      body.load(p, len, stages + st * stage_bytes, r);
      __syncthreads();
      if (tid < 32 && nxt < p.n_items) {
        if (tid == 0) fence_proxy_async();
        __syncwarp();
        issue_item(p, tm, nxt, stages + st * stage_bytes, smem_addr(&bars[st]));
      }
      body.compute(p, s, c0, len, r);
    } else {
      body(p, s, c0, len, stages + st * stage_bytes, slots);
      __syncthreads();
      if (tid < 32 && nxt < p.n_items) {
        if (tid == 0) fence_proxy_async();
        __syncwarp();
        issue_item(p, tm, nxt, stages + st * stage_bytes, smem_addr(&bars[st]));
      }
    }
  }
}

// Windowed pipeline, for two-level programs whose inputs stream through in
// windows (the multilevel pebble game: registers hold the partial sums of a
// group of rows, shared memory one window of input strips at a time).  The
// program reads the windows in a fixed order of phases: for every group of
// rows, every window of `win` input strips in turn.  Instead of a stage
// holding a tile of all n_in strips, shared memory holds a ring of kWinRing
// window slots (win x T bytes each), so several CTAs fit an SM even for codes
// of hundreds of strips.  Warp 0 produces: for each of the CTA's items and
// each phase it waits until the phase's slot is free, then copies the
// phase's window into it (one tiled tensor copy of `win` strips when the
// launch has a tensor map, else one 1-D bulk copy per strip).  The other
// warps consume: the program waits for each phase's slot, reads its operands
// from it, and releases it (one arrival per consumer thread).  A group of
// rows after the first reads the windows again; they come from L2.
//
// Shared memory: [full barriers][empty barriers] (128 B), then the ring.
// Consumer-side view of the ring.  Phase q of the CTA's running phase count
// uses slot q % kWinRing, in round q / kWinRing.
struct WindowView {
  u8* ring;
  u32 full0, empty0;     // shared addresses of the barrier arrays
  i64 slot_bytes;
  // Wait for phase q's window; the slot's address, or null after a wait
  // that timed out.
  __device__ __forceinline__ const u8* begin(i64 q) const {
    const int slot = static_cast<int>(q % kWinRing);
    if (!mbar_wait(full0 + 8u * slot, static_cast<u32>((q / kWinRing) & 1))) return nullptr;
    return ring + slot * slot_bytes;
  }
  // This thread is done with phase q's window.
  __device__ __forceinline__ void end(i64 q) const {
    const int slot = static_cast<int>(q % kWinRing);
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }"
                 ::"r"(empty0 + 8u * slot) : "memory");
  }
};

// Warp 0: copy window w of `item` into `dst`; completion on `bar`.
__device__ __forceinline__ void issue_window(const LaunchParams& p, const TensorMap* tm, i64 item,
                                             int w, u8* dst, u32 bar) {
  const i64 s = item / p.tiles_per_strip;
  const i64 c0 = (item % p.tiles_per_strip) * p.T;
  const int lane = threadIdx.x & 31;
  const int y0 = w * p.win;
  if (p.tmap > 0) {
    // one box of `win` strips; rows past n_in are zero-filled and counted
    if (lane == 0) {
      mbar_arrive_expect_tx(bar, static_cast<u32>(p.win) * static_cast<u32>(p.T));
      tma_load_3d(smem_addr(dst), tm, static_cast<int>(c0 >> tmap_elem_shift(p.T)), y0,
                  static_cast<int>(s), bar);
    }
    return;
  }
  const i64 rest = p.io.S - c0;
  const int len = rest < p.T ? static_cast<int>(rest) : p.T;
  const int n = p.n_in - y0 < p.win ? p.n_in - y0 : p.win;
  if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<u32>(n) * static_cast<u32>(len));
  __syncwarp();
  for (int c = lane; c < n; c += 32) {
    const int strip = y0 + c;
    const u8* src = in_block(p.io, s, strip >> 3) + static_cast<i64>(strip & 7) * p.io.S + c0;
    tma_load_1d(smem_addr(dst + static_cast<i64>(c) * p.T), src, static_cast<u32>(len), bar);
  }
}

// Body (windowed programs; each consumer owns kColBytes bytes of every
// strip of the tile):
//   bool compute(const LaunchParams&, const WindowView&, i64 q0, i64 stripe,
//                i64 c0, int len, int col) const
// runs the program on column `col` of the item whose first phase is the
// CTA's phase q0 (col may lie past len: its results are not stored, but it
// takes part in every phase); false when a wait timed out.
template <class Body, int kColBytes = 4>
__device__ __forceinline__ void run_window_pipeline(const LaunchParams& p, u8* smem,
                                                    const Body& body, const TensorMap* tm) {
  u64* full = reinterpret_cast<u64*>(smem);
  u64* empty = reinterpret_cast<u64*>(smem + 64);
  const int tid = threadIdx.x;
  const int n_cons = static_cast<int>(blockDim.x) - 32;
  WindowView v;
  v.ring = smem + 128;
  v.full0 = smem_addr(full);
  v.empty0 = smem_addr(empty);
  v.slot_bytes = static_cast<i64>(p.win) * p.T;
  if (tid == 0) {
    for (int r = 0; r < kWinRing; ++r) {
      mbar_init(smem_addr(&full[r]), 1);
      mbar_init(smem_addr(&empty[r]), static_cast<u32>(n_cons));
    }
    fence_mbar_init();
  }
  __syncthreads();
  const i64 first = blockIdx.x, step = gridDim.x;
  if (tid < 32) {
    // producer: a fresh empty barrier counts its phase before phase 0 as
    // complete, so the first round of slots needs no release
    i64 q = 0;
    bool ok = true;
    for (i64 item = first; ok && item < p.n_items; item += step)
      for (int ph = 0; ph < p.n_phases; ++ph, ++q) {
        const int slot = static_cast<int>(q % kWinRing);
        if (tid == 0) ok = mbar_wait(smem_addr(&empty[slot]), static_cast<u32>(((q / kWinRing) & 1) ^ 1));
        ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
        if (!ok) break;
        if (tid == 0) fence_proxy_async();
        __syncwarp();
        issue_window(p, tm, item, ph % p.n_win, v.ring + slot * v.slot_bytes,
                     smem_addr(&full[slot]));
      }
    if (!ok && tid == 0) {
      // a release never came: record it and let the copies in flight land
      // (bounded) before the CTA ends
      atomicExch(p.status, XK_STATUS_TIMEOUT);
      for (i64 d = q - kWinRing; d < q; ++d)
        if (d >= 0) mbar_wait(smem_addr(&full[d % kWinRing]), static_cast<u32>((d / kWinRing) & 1));
    }
    return;
  }
  const int col = (tid - 32) * kColBytes;
  i64 q0 = 0;
  for (i64 item = first; item < p.n_items; item += step, q0 += p.n_phases) {
    const i64 s = item / p.tiles_per_strip;
    const i64 c0 = (item % p.tiles_per_strip) * p.T;
    const i64 rest = p.io.S - c0;
    const int len = rest < p.T ? static_cast<int>(rest) : p.T;
    if (!body.compute(p, v, q0, s, c0, len, col)) {
      atomicExch(p.status, XK_STATUS_TIMEOUT);
      return;
    }
  }
}

// Batched pipeline: the same single-stage, early-release ring as
// run_pipeline, but each item names its stripe, whose descriptor gives the
// program, the strip length and the block addresses.  Body (for batches):
//   kEarlyRelease == true:
//     void load(const StripeDesc&, int len, const u8* stage, Regs&) const
//     void compute(const StripeDesc&, i64 c0, int len, Regs&) const
//   kEarlyRelease == false:
//     void operator()(const StripeDesc&, i64 c0, int len, const u8* stage,
//                     u8* slots, int T) const
// Item -> stripe.  A CTA mostly visits consecutive items, so each caller
// keeps a cursor into the stripe list and moves it to the next stripe, or
// searches when the CTA has moved to another range of items.
__device__ __forceinline__ int find_stripe(const BatchParams& p, i64 item);

__device__ __forceinline__ void batch_item_geom(const BatchParams& p, i64 item, int& cursor,
                                                const StripeDesc*& d, i64& c0, int& len) {
  // the cursor's stripe, else the next one, else a binary search (a CTA
  // that moves to another range of items jumps)
  if (p.stripes[cursor].item_base > item) {
    cursor = find_stripe(p, item);
  } else if (cursor + 1 < p.n_stripes && p.stripes[cursor + 1].item_base <= item) {
    ++cursor;
    if (cursor + 1 < p.n_stripes && p.stripes[cursor + 1].item_base <= item)
      cursor = find_stripe(p, item);
  }
  d = &p.stripes[cursor];
  c0 = (item - d->item_base) * p.T;
  const i64 rest = d->S - c0;
  len = rest < p.T ? static_cast<int>(rest) : p.T;
}

// Source addresses of one batched item, computed by warp 0 ahead of the
// copy into a small shared table (strip c -> src[c]), so that the copy can
// be issued without waiting on descriptor loads.  Codes wider than
// kMaxPrepared strips are addressed at issue time instead.
struct NextCopy {
  u32 bytes;     // expected transaction bytes
  u32 len;
  int n_in;
  int x;                    // tensor copies: first word of the tile
  const TensorMap* maps;    // tensor copies: the stripe's block maps, or null
};

// First stripe cursor for `item` (binary search over item_base).
__device__ __forceinline__ int find_stripe(const BatchParams& p, i64 item) {
  int lo = 0, hi = p.n_stripes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.stripes[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void prepare_batch_item(const BatchParams& p, i64 item, int& cursor,
                                                   NextCopy& nc, const u8** src) {
  const StripeDesc* d;
  i64 c0;
  int len;
  batch_item_geom(p, item, cursor, d, c0, len);
  const int n_in = 8 * d->n_inblk;
  const int lane = threadIdx.x & 31;
  nc.len = static_cast<u32>(len);
  nc.n_in = n_in;
  nc.maps = d->maps;
  if (nc.maps) {
    // one tiled copy per input block: the full box lands (zero-filled past
    // the end of the strips) and counts in full
    nc.x = static_cast<int>(c0 >> tmap_elem_shift(p.T));
    nc.bytes = static_cast<u32>(n_in) * static_cast<u32>(p.T);
    return;
  }
  if (n_in <= kMaxPrepared)
    for (int c = lane; c < n_in; c += 32)
      src[c] = reinterpret_cast<const u8*>(d->blocks[c >> 3]) + static_cast<i64>(c & 7) * d->S + c0;
  nc.bytes = static_cast<u32>(n_in) * static_cast<u32>(len);
}

__device__ __forceinline__ void issue_batch_prepared(const BatchParams& p, i64 item, int cursor,
                                                     const NextCopy& nc, const u8* const* src,
                                                     u8* dst, u32 bar) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) mbar_arrive_expect_tx(bar, nc.bytes);
  __syncwarp();
  if (nc.maps) {
    for (int j = lane; 8 * j < nc.n_in; j += 32)
      tma_load_2d(smem_addr(dst + static_cast<i64>(8 * j) * p.T), nc.maps + j, nc.x, 0, bar);
    return;
  }
  if (nc.n_in <= kMaxPrepared) {
    for (int c = lane; c < nc.n_in; c += 32)
      tma_load_1d(smem_addr(dst + static_cast<i64>(c) * p.T), src[c], nc.len, bar);
    return;
  }
  const StripeDesc* d;
  i64 c0;
  int len;
  batch_item_geom(p, item, cursor, d, c0, len);
  for (int c = lane; c < nc.n_in; c += 32) {
    const u8* s = reinterpret_cast<const u8*>(d->blocks[c >> 3]) + static_cast<i64>(c & 7) * d->S + c0;
    tma_load_1d(smem_addr(dst + static_cast<i64>(c) * p.T), s, nc.len, bar);
  }
}

// Warp 0's work-queue state, kept in shared memory between items so that
// none of it occupies registers while the XOR program runs.
struct QueueState {
  i64 q_pos, q_end;   // current chunk [q_pos, q_end)
  int cur_r;          // range popped from, -1 when every range is empty
  int home;           // range of the SM the CTA runs on
  int prep_cur;       // stripe cursor of the prepared item
  int pad_;
  NextCopy nc;        // the prepared copy
};

// Items are split into n_ranges contiguous ranges: the first range_rem
// ranges hold range_len + 1 items, the others range_len.
__device__ __forceinline__ i64 range_lo(const BatchParams& p, int r) {
  return p.range_len * r + (r < p.range_rem ? r : p.range_rem);
}

// Warp 0 (all lanes): the nearest range, from `home` on, whose queue head
// still has items; -1 when none has.  Heads only grow, so a range seen
// empty stays empty; a range seen non-empty may empty before the pop, which
// then fails and the scan runs again.
__device__ __forceinline__ int next_range(const BatchParams& p, int home, int R, i64 C) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < R; base += 32) {
    bool left = false;
    if (base + lane < R) {
      int r = home + base + lane;
      if (r >= R) r -= R;
      const u64 h = *reinterpret_cast<volatile const u64*>(p.queue + r);
      left = range_lo(p, r) + static_cast<i64>(h) * C < range_lo(p, r + 1);
    }
    const u32 b = __ballot_sync(0xffffffffu, left);
    if (b) {
      const int r = home + base + __ffs(b) - 1;
      return r >= R ? r - R : r;
    }
  }
  return -1;
}

// Warp 0 (all lanes): next item of this CTA, -1 at the end.
__device__ __forceinline__ i64 batch_pop(const BatchParams& p, QueueState& q) {
  const int R = p.n_ranges > 1 ? p.n_ranges : 1;
  const i64 C = p.chunk > 0 ? p.chunk : 1;
  while (q.q_pos >= q.q_end) {
    if (q.cur_r < 0) return -1;
    u64 c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(p.queue + q.cur_r, 1ull);
    c = __shfl_sync(0xffffffffu, c, 0);
    const i64 lo = range_lo(p, q.cur_r) + static_cast<i64>(c) * C;
    const i64 hi = range_lo(p, q.cur_r + 1);
    if (lo < hi) {
      q.q_pos = lo;
      q.q_end = lo + C < hi ? lo + C : hi;
      break;
    }
    q.cur_r = next_range(p, q.home, R, C);
  }
  return q.q_pos++;
}

template <class Body>
__device__ __forceinline__ void run_batch_pipeline(const BatchParams& p, u8* smem, const Body& body,
                                                   u8* slots) {
  u64* bar = reinterpret_cast<u64*>(smem);
  volatile i64* ring = reinterpret_cast<volatile i64*>(smem + 64);
  QueueState* qs = reinterpret_cast<QueueState*>(smem + 128);
  const u8** src = reinterpret_cast<const u8**>(smem + 256);
  u8* stage = smem + kBatchHeader;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_addr(bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Work queue: warp 0 pops chunks of `chunk` consecutive items (consecutive
  // items mostly share a stripe, whose descriptor stays in L1, and each CTA
  // streams long runs of every strip; popping on demand balances stripes of
  // different cost).  The items are split into n_ranges contiguous ranges,
  // one per SM, each with its own queue head: a CTA pops from the range of
  // the SM it runs on, so the CTAs of one SM work on the same stripe, hence
  // the same program, and an SM runs only the few programs of its range
  // (straight-line programs of many decode patterns otherwise compete for
  // the SM's instruction cache).  When its range is empty, a CTA takes
  // chunks from the nearest range that still has items (a warp-wide scan of
  // the heads); it returns only when every range is empty, so every item is
  // processed exactly once whichever SMs the CTAs land on.  Warp 0 works
  // two items ahead: it publishes item indices in a ring in shared memory
  // and keeps the source table of the next copy prepared, so that neither
  // the queue nor the descriptors delay the barrier.
  if (tid < 32) {
    QueueState q;
    q.q_pos = q.q_end = 0;
    q.home = 0;
    if (p.n_ranges > 1) {
      u32 sm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
      q.home = static_cast<int>(sm % static_cast<u32>(p.n_ranges));
    }
    q.cur_r = q.home;
    q.prep_cur = 0;
    q.pad_ = 0;
    const i64 a = batch_pop(p, q);
    const i64 b2 = a >= 0 ? batch_pop(p, q) : -1;
    if (tid == 0) {
      ring[0] = a;
      ring[1] = b2;
    }
    if (a >= 0) {
      q.prep_cur = find_stripe(p, a);
      prepare_batch_item(p, a, q.prep_cur, q.nc, src);
      __syncwarp();
      issue_batch_prepared(p, a, q.prep_cur, q.nc, src, stage, smem_addr(bar));
      __syncwarp();
      if (b2 >= 0) prepare_batch_item(p, b2, q.prep_cur, q.nc, src);
    }
    __syncwarp();
    if (tid == 0) *qs = q;
  }
  __syncthreads();
  int cur;   // stripe cursor of the current item
  {
    const i64 a = ring[0];
    cur = a >= 0 ? find_stripe(p, a) : 0;
  }
  for (i64 i = 0;; ++i) {
    const i64 item = ring[i % kRing];
    if (item < 0) break;
    const i64 nxt = ring[(i + 1) % kRing];
    const StripeDesc* d;
    i64 c0;
    int len;
    batch_item_geom(p, item, cur, d, c0, len);
    const bool ok = mbar_wait(smem_addr(bar), static_cast<u32>(i & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(p.status, XK_STATUS_TIMEOUT);
        if (p.local_status) *reinterpret_cast<volatile int*>(p.local_status) = XK_STATUS_TIMEOUT;
        mbar_wait(smem_addr(bar), static_cast<u32>(i & 1));
      }
      return;
    }
    // warp 0, once the stage is free: issue the copy of the next item
    // (prepared one item earlier) ...
    auto issue_next = [&]() {
      if (tid < 32 && nxt >= 0) {
        if (tid == 0) fence_proxy_async();
        __syncwarp();
        issue_batch_prepared(p, nxt, qs->prep_cur, qs->nc, src, stage, smem_addr(bar));
        __syncwarp();
      }
    };
    // ... and, after its own share of the work (no input words are held in
    // registers then), pop the item after it and prepare its sources.  The
    // ring entry it writes is read by the other warps only after the next
    // iteration's barrier.
    auto prepare_after = [&]() {
      if (tid < 32) {
        QueueState q = *qs;
        const i64 after = nxt >= 0 ? batch_pop(p, q) : -1;
        if (tid == 0) ring[(i + 2) % kRing] = after;
        if (after >= 0) prepare_batch_item(p, after, q.prep_cur, q.nc, src);
        __syncwarp();
        if (tid == 0) *qs = q;
      }
    };
    if constexpr (Body::kEarlyRelease) {
      typename Body::Regs r;
      body.load(*d, len, stage, r);
      __syncthreads();
      issue_next();
      body.compute(*d, c0, len, r);
      prepare_after();
    } else {
      body(*d, c0, len, stage, slots, p.T);
      __syncthreads();
      issue_next();
      prepare_after();
    }
  }
}

// Batched form of the windowed pipeline, for modules of single-group
// windowed programs (one phase per window).  Warp 0 pops items from the work
// queue (chunks of consecutive items; one queue) and, per item and window,
// waits for a free slot, copies the window (one 2-D tensor copy per input
// block of the window, or one 1-D copy per strip) and, in the item's first
// slot, leaves the item's index for the consumers; a last slot holding -1
// ends the launch.  The consumers take the item from its first slot and run
// its program window by window.  Each consumer owns kColBytes bytes of
// every strip of the tile (T = kColBytes x consumers).  With kStripePhases
// (the dense bitmatrix executor) an item's windows and phases follow its
// stripe, so one launch mixes codes of any width.
// Shared memory: [full barriers (0)][empty barriers (64)][slot items (96)],
// then the ring from byte 128.
// Body (windowed modules):
//   bool compute(const StripeDesc&, const WindowView&, i64 q0, i64 c0, int len,
//                int col) const
//   int groups(const StripeDesc&) const      (kStripePhases only)
__device__ __forceinline__ void issue_batch_window(const BatchParams& p, const StripeDesc* d,
                                                   i64 c0, int len, int w, u8* dst, u32 bar) {
  const int lane = threadIdx.x & 31;
  const int n_in = 8 * d->n_inblk;
  const int y0 = w * p.win;
  const int n = n_in - y0 < p.win ? n_in - y0 : p.win;
  if (d->maps) {
    // one box of a block's 8 strips per block; past the end of the strips it
    // is zero-filled and counts in full
    const int b0 = y0 >> 3, nb = n >> 3;
    if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<u32>(n) * static_cast<u32>(p.T));
    __syncwarp();
    for (int j = lane; j < nb; j += 32)
      tma_load_2d(smem_addr(dst + static_cast<i64>(8 * j) * p.T), d->maps + b0 + j,
                  static_cast<int>(c0 >> tmap_elem_shift(p.T)), 0, bar);
    return;
  }
  if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<u32>(n) * static_cast<u32>(len));
  __syncwarp();
  for (int c = lane; c < n; c += 32) {
    const int strip = y0 + c;
    const u8* src = reinterpret_cast<const u8*>(d->blocks[strip >> 3]) +
                    static_cast<i64>(strip & 7) * d->S + c0;
    tma_load_1d(smem_addr(dst + static_cast<i64>(c) * p.T), src, static_cast<u32>(len), bar);
  }
}

// Windows and phases of one item: the launch's (windowed modules), or,
// with kStripePhases, the stripe's own (windows of p.win strips over its
// inputs, read once per group of rows: Body::groups(const StripeDesc&)).
template <bool kStripePhases>
__device__ __forceinline__ int item_windows(const BatchParams& p, const StripeDesc& d) {
  return kStripePhases ? (8 * d.n_inblk + p.win - 1) / p.win : p.n_win;
}
template <bool kStripePhases, class Body>
__device__ __forceinline__ int item_phases(const BatchParams& p, const StripeDesc& d,
                                           const Body& body) {
  if constexpr (kStripePhases) return item_windows<true>(p, d) * body.groups(d);
  else return p.n_win;
}

template <class Body, int kColBytes = 4, bool kStripePhases = false>
__device__ __forceinline__ void run_batch_window_pipeline(const BatchParams& p, u8* smem,
                                                          const Body& body) {
  u64* full = reinterpret_cast<u64*>(smem);
  u64* empty = reinterpret_cast<u64*>(smem + 64);
  volatile i64* slot_item = reinterpret_cast<volatile i64*>(smem + 96);
  const int tid = threadIdx.x;
  const int n_cons = static_cast<int>(blockDim.x) - 32;
  WindowView v;
  v.ring = smem + 128;
  v.full0 = smem_addr(full);
  v.empty0 = smem_addr(empty);
  v.slot_bytes = static_cast<i64>(p.win) * p.T;
  if (tid == 0) {
    for (int r = 0; r < kWinRing; ++r) {
      mbar_init(smem_addr(&full[r]), 1);
      mbar_init(smem_addr(&empty[r]), static_cast<u32>(n_cons));
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid < 32) {
    // producer: a fresh empty barrier counts its phase before phase 0 as
    // complete, so the first round of slots needs no release
    QueueState qs;
    qs.q_pos = qs.q_end = 0;
    qs.cur_r = 0;
    qs.home = 0;
    qs.prep_cur = 0;
    qs.pad_ = 0;
    int cursor = 0;
    i64 q = 0;
    bool ok = true;
    for (bool done = false; ok && !done;) {
      const i64 item = batch_pop(p, qs);
      const StripeDesc* d = nullptr;
      i64 c0 = 0;
      int len = 0;
      if (item >= 0) batch_item_geom(p, item, cursor, d, c0, len);
      const int phases = item >= 0 ? item_phases<kStripePhases>(p, *d, body) : 1;
      const int nw = item >= 0 ? item_windows<kStripePhases>(p, *d) : 1;
      for (int ph = 0; ph < phases; ++ph, ++q) {
        const int slot = static_cast<int>(q % kWinRing);
        if (tid == 0)
          ok = mbar_wait(smem_addr(&empty[slot]), static_cast<u32>(((q / kWinRing) & 1) ^ 1));
        ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
        if (!ok) break;
        if (ph == 0 && tid == 0) slot_item[slot] = item;
        if (item < 0) {
          // the end: an arrival without copies completes the slot's phase
          if (tid == 0)
            asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }"
                         ::"r"(smem_addr(&full[slot])) : "memory");
          done = true;
          break;
        }
        if (tid == 0) fence_proxy_async();
        __syncwarp();
        issue_batch_window(p, d, c0, len, ph % nw, v.ring + slot * v.slot_bytes,
                           smem_addr(&full[slot]));
      }
    }
    if (!ok && tid == 0) {
      // a release never came: record it and let the copies in flight land
      // (bounded) before the CTA ends
      atomicExch(p.status, XK_STATUS_TIMEOUT);
      if (p.local_status) *reinterpret_cast<volatile int*>(p.local_status) = XK_STATUS_TIMEOUT;
      for (i64 x = q - kWinRing; x < q; ++x)
        if (x >= 0) mbar_wait(smem_addr(&full[x % kWinRing]), static_cast<u32>((x / kWinRing) & 1));
    }
    return;
  }
  const int col = (tid - 32) * kColBytes;
  int cursor = 0;
  for (i64 q0 = 0;;) {
    const int slot = static_cast<int>(q0 % kWinRing);
    if (!mbar_wait(v.full0 + 8u * slot, static_cast<u32>((q0 / kWinRing) & 1))) {
      atomicExch(p.status, XK_STATUS_TIMEOUT);
      if (p.local_status) *reinterpret_cast<volatile int*>(p.local_status) = XK_STATUS_TIMEOUT;
      return;
    }
    const i64 item = slot_item[slot];
    if (item < 0) return;
    const StripeDesc* d;
    i64 c0;
    int len;
    batch_item_geom(p, item, cursor, d, c0, len);
    if (!body.compute(*d, v, q0, c0, len, col)) {
      atomicExch(p.status, XK_STATUS_TIMEOUT);
      if (p.local_status) *reinterpret_cast<volatile int*>(p.local_status) = XK_STATUS_TIMEOUT;
      return;
    }
    q0 += item_phases<kStripePhases>(p, *d, body);
  }
}

#endif  // __CUDACC__ || __CUDACC_RTC__

}  // namespace xk
