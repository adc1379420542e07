// GPU executors compiled into the library: the SLP interpreter, the dense
// bitmatrix executor (programs without a compiled kernel) and the synthetic
// input generator.
//
// The interpreter runs the instruction stream of a scheduled, fused SLP
// (Sec. 4-6 of the paper; the stream format is described in plan.h) over
// the tiles staged by the shared pipeline (tile_pipeline.cuh).  Each thread
// owns one 4-byte column of every strip of the tile: for each statement it
// XORs its operands (input strips of the stage or pebble slots, both in
// shared memory) in registers, stores the result into its slot when a later
// statement reads it, and writes it to each output strip it is returned as.
// Threads touch only their own column, so statements need no barrier.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tile_pipeline.cuh"

namespace {

using namespace xk;

// Shared-memory accesses by 32-bit shared-window address.  Volatile so
// that a statement's reads of a slot stay after the earlier statement's
// write of it (the same thread, the same address).
template <int W> struct Words { u32 v[W]; };

template <int W>
__device__ __forceinline__ Words<W> lds(u32 a) {
  Words<W> r;
  if constexpr (W == 1) {
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r.v[0]) : "r"(a));
  } else if constexpr (W == 2) {
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.v[0]), "=r"(r.v[1]) : "r"(a));
  } else {
    static_assert(W == 4, "one, two or four words");
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]) : "r"(a));
  }
  return r;
}

template <int W>
__device__ __forceinline__ void sts(u32 a, const Words<W>& x) {
  if constexpr (W == 1) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(x.v[0]) : "memory");
  } else if constexpr (W == 2) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(x.v[0]), "r"(x.v[1]) : "memory");
  } else {
    static_assert(W == 4, "one, two or four words");
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x.v[0]), "r"(x.v[1]),
                 "r"(x.v[2]), "r"(x.v[3])
                 : "memory");
  }
}

template <int W>
__device__ __forceinline__ void stg(u8* p, const Words<W>& x) {
  if constexpr (W == 1) {
    *reinterpret_cast<u32*>(p) = x.v[0];
  } else if constexpr (W == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(x.v[0], x.v[1]);
  } else {
    static_assert(W == 4, "one, two or four words");
    *reinterpret_cast<uint4*>(p) = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
  }
}

template <int W>
__device__ __forceinline__ void xor_in(Words<W>& acc, const Words<W>& x) {
#pragma unroll
  for (int w = 0; w < W; ++w) acc.v[w] ^= x.v[w];
}

// Runs a program for one thread's column of a tile: W 4-byte words of
// every strip (bytes [col, col + 4W) of the tile).  code: the program's
// device stream of n_chunks 16-byte chunks (Program::chunks: per statement a
// header chunk, ceil(a/8) chunks of operand ids, then chunks of the outputs
// beyond five), read warp-uniformly one chunk ahead of its use, so a chunk's
// eight operand loads wait only for the shared memory.  in_col: shared
// address of the column in input strip 0 of the stage (strip c at
// in_col + c*T); slot_col: shared address of the column in slot 0 (slot s
// at slot_col + s*T); out(r): global address of output strip r at this
// column.  Operand ids below n_in are input strips, the others slots.
template <int W, bool kGap, class OutAddr>
__device__ __forceinline__ void interpret_run(const u16* __restrict__ code, int n_chunks, int n_in,
                                              u32 T, u32 in_col, u32 slot_col, const OutAddr& out) {
  // operand o at in_col + o*T, plus `gap` for slots when they do not
  // directly follow the input strips (kGap)
  const u32 gap = slot_col - (in_col + static_cast<u32>(n_in) * T);
  auto addr = [&](u32 o) -> u32 {
    if constexpr (kGap) return in_col + o * T + (o >= static_cast<u32>(n_in) ? gap : 0u);
    return in_col + o * T;
  };
  const uint4* chunk = reinterpret_cast<const uint4*>(code);
  int at = 0;
  uint4 ahead = n_chunks > 0 ? __ldg(chunk) : make_uint4(0, 0, 0, 0);
  auto take = [&]() -> uint4 {   // the next chunk; starts the load of the one after
    const uint4 c = ahead;
    if (++at < n_chunks) ahead = __ldg(chunk + at);
    return c;
  };
  while (at < n_chunks) {
    const uint4 h = take();
    const int na = static_cast<int>(h.x & 0xffffu);
    const int no = static_cast<int>(h.x >> 16);
    const u32 slot = h.y & 0xffffu;
    Words<W> acc;
#pragma unroll
    for (int w = 0; w < W; ++w) acc.v[w] = 0;
    for (int left = na; left > 0; left -= 8) {
      const uint4 c = take();
      const u32 id[8] = {c.x & 0xffffu, c.x >> 16, c.y & 0xffffu, c.y >> 16,
                         c.z & 0xffffu, c.z >> 16, c.w & 0xffffu, c.w >> 16};
      if (left >= 8) {
        Words<W> x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = lds<W>(addr(id[q]));
#pragma unroll
        for (int q = 0; q < 8; ++q) xor_in(acc, x[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 7; ++q)
          if (q < left) xor_in(acc, lds<W>(addr(id[q])));
      }
    }
    if (slot != 0xffffu) sts<W>(slot_col + slot * T, acc);
    const u32 first[5] = {h.y >> 16, h.z & 0xffffu, h.z >> 16, h.w & 0xffffu, h.w >> 16};
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (q < no) stg<W>(out(static_cast<int>(first[q])), acc);
    for (int left = no - 5; left > 0; left -= 8) {
      const uint4 c = take();
      const u32 id[8] = {c.x & 0xffffu, c.x >> 16, c.y & 0xffffu, c.y >> 16,
                         c.z & 0xffffu, c.z >> 16, c.w & 0xffffu, c.w >> 16};
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < left) stg<W>(out(static_cast<int>(id[q])), acc);
    }
  }
}

template <int W, class OutAddr>
__device__ __forceinline__ void interpret(const u16* __restrict__ code, int n_chunks, int n_in,
                                          u32 T, u32 in_col, u32 slot_col, const OutAddr& out) {
  // single launches with one stage keep the slots right after the inputs
  if (slot_col == in_col + static_cast<u32>(n_in) * T)
    interpret_run<W, false>(code, n_chunks, n_in, T, in_col, slot_col, out);
  else
    interpret_run<W, true>(code, n_chunks, n_in, T, in_col, slot_col, out);
}

template <int W>
struct InterpBody {
  static constexpr bool kEarlyRelease = false;
  __device__ __forceinline__ void operator()(const LaunchParams& p, i64 s, i64 c0, int len,
                                             const u8* stg_base, u8* slots) const {
    const int col = threadIdx.x * 4 * W;
    if (col >= len) return;
    auto out = [&](int r) {
      return out_block(p.io, s, r >> 3) + static_cast<i64>(r & 7) * p.io.S + c0 + col;
    };
    interpret<W>(p.code, p.code_len, p.n_in, static_cast<u32>(p.T), smem_addr(stg_base + col),
                 smem_addr(slots + col), out);
  }
};

struct InterpBatchBody {
  static constexpr bool kEarlyRelease = false;
  __device__ __forceinline__ void operator()(const StripeDesc& d, i64 c0, int len, const u8* stg,
                                             u8* slots, int T) const {
    const int col = threadIdx.x * 4;
    if (col >= len) return;
    const u64* outs = d.blocks + d.n_inblk;
    auto out = [&](int r) {
      return reinterpret_cast<u8*>(outs[r >> 3]) + static_cast<i64>(r & 7) * d.S + c0 + col;
    };
    interpret<1>(d.code, d.code_len, 8 * d.n_inblk, static_cast<u32>(T), smem_addr(stg + col),
                 smem_addr(slots + col), out);
  }
};

// Single-launch interpreter: each thread owns W 4-byte words per strip
// (tile T = 4 * W * threads bytes).
// Shared memory, not registers, bounds its resident CTAs (the stage and the
// slots of a program take tens of KB), so the register cap is left loose.
template <int W>
__global__ void __launch_bounds__(256, 1)
    interp_kernel(LaunchParams p, const __grid_constant__ TensorMap tm) {
  extern __shared__ __align__(128) u8 smem[];
  run_pipeline(p, smem, InterpBody<W>(), &tm);
}

// Batched interpreter: shared memory = [header][stage: max_in * T]
// [slots: the largest slot count of the launch * T].
__global__ void __launch_bounds__(256, 1) interp_batch_kernel(BatchParams p) {
  extern __shared__ __align__(128) u8 smem[];
  u8* slots = smem + kBatchHeader + static_cast<i64>(p.max_in) * p.T;
  run_batch_pipeline(p, smem, InterpBatchBody(), slots);
}

// ------------------------------------------------ dense bitmatrix executor
// Runs a program without a compiled kernel by evaluating its bitmatrix
// (Sec. 1, property (ii): output strip r is the XOR of the input strips c
// whose bit (r, c) is set), the linear map every SLP of the program
// computes.  On the GPU this beats interpreting the optimised SLP: the
// interpreter fetches, decodes and addresses every operand, while here the
// control is a few uniform words per window and every input word is read
// from shared memory once.
//
// The inputs stream through the windowed pipeline (tile_pipeline.cuh) in
// windows of kDenseWin strips (one block); consumers own W 4-byte words of
// every strip.  Output rows go in groups of up to 32: per group, every
// window is read once (a group after the first reads them again, from L2)
// and XORed into the group's register accumulators; at the end of the group
// each accumulator is written to its output strip.  Two forms:
//   masks: per input strip, XOR it into the accumulators of the rows whose
//     bit is set (a uniform test and W XORs per row and strip);
//   tables (the method of four Russians, Arlazarov, Dinic, Kronrod and
//     Faradzev): per window, each consumer writes the XORs of all 16 subsets
//     of strips 0-3 and of strips 4-7 of its column into two tables in
//     shared memory (15 XORs each, in Gray-code order so one entry is live at
//     a time); a row then takes two table entries, chosen by its 8 bits of
//     the window: per row and strip, a quarter of a table read and about a
//     third of the masks' integer work.
// Control words follow the program's chunk stream in its device buffer:
// n_groups * n_in masks (group g's mask of input strip c is word g*n_in + c,
// bit r for output strip 32 g + r), then as many row words (group g, window
// w: words g*n_in + 8 w + j hold the window's bits of rows 4j .. 4j+3, one
// byte per row, bit i for strip 8 w + i).
using xorec::kDenseThreads;
using xorec::kDenseWin;

// Forms.  A third form, tables for 24 rows of a group and masks for 8 (the
// masks' integer work beside the tables' shared-memory traffic), ran RS(10,4)
// encode at 0.417 of the copy bandwidth against 0.521 for tables alone and
// was dropped.
enum { kMaskForm = 0, kTableForm = 1 };

template <int W>
struct DenseTile {
  static constexpr u32 T = 4u * W * kDenseThreads;   // tile bytes per strip
};

// One group of kRows output rows (rows <= kRows of them real): every window
// of the item, then the stores.  q: the CTA's phase counter; masks, rowb: the
// group's masks and row words; tbl: shared address of this consumer's column
// in entry 0 of table 0 (entries T bytes apart).
template <int W, int kForm, int kRows, class OutAddr>
__device__ __forceinline__ bool dense_group(const WindowView& v, i64& q, int n_win, int col,
                                            bool store, const u32* __restrict__ masks,
                                            const u32* __restrict__ rowb, u32 tbl, int rows,
                                            const OutAddr& out) {
  constexpr u32 T = DenseTile<W>::T;
  // rows [0, kTab) from the tables, [kTab, kRows) from the masks
  constexpr int kTab = kForm == kMaskForm ? 0 : kRows;
  Words<W> acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int w = 0; w < W; ++w) acc[r].v[w] = 0;
  if constexpr (kTab > 0) {
    Words<W> z;
#pragma unroll
    for (int w = 0; w < W; ++w) z.v[w] = 0;
    sts<W>(tbl, z);
    sts<W>(tbl + 16 * T, z);
  }
  for (int w = 0; w < n_win; ++w, ++q) {
    const u8* slot = v.begin(q);
    if (!slot) return false;
    u32 mk[kDenseWin], rb[kDenseWin];
    if constexpr (kTab < kRows) {
      const uint4 m0 = __ldg(reinterpret_cast<const uint4*>(masks + kDenseWin * w));
      const uint4 m1 = __ldg(reinterpret_cast<const uint4*>(masks + kDenseWin * w) + 1);
      mk[0] = m0.x; mk[1] = m0.y; mk[2] = m0.z; mk[3] = m0.w;
      mk[4] = m1.x; mk[5] = m1.y; mk[6] = m1.z; mk[7] = m1.w;
    }
    if constexpr (kTab > 0) {
      const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(rowb + kDenseWin * w));
      const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(rowb + kDenseWin * w) + 1);
      rb[0] = r0.x; rb[1] = r0.y; rb[2] = r0.z; rb[3] = r0.w;
      rb[4] = r1.x; rb[5] = r1.y; rb[6] = r1.z; rb[7] = r1.w;
    }
    const u32 a = smem_addr(slot) + static_cast<u32>(col);
    Words<W> x[kDenseWin];
#pragma unroll
    for (int c = 0; c < kDenseWin; ++c) x[c] = lds<W>(a + static_cast<u32>(c) * T);
    v.end(q);   // the window now lives in registers (and the tables)
    if constexpr (kTab > 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        Words<W> cur = x[4 * h];
        sts<W>(tbl + (16 * h + 1) * T, cur);
#pragma unroll
        for (int i = 2; i < 16; ++i) {
          // Gray code i ^ (i >> 1) differs from the previous one in the
          // lowest set bit of i
          xor_in(cur, x[4 * h + ((i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : 3)]);
          sts<W>(tbl + (16 * h + (i ^ (i >> 1))) * T, cur);
        }
      }
#pragma unroll
      for (int r = 0; r < kTab; ++r) {
        const u32 b = (rb[r >> 2] >> (8 * (r & 3))) & 0xffu;
        const Words<W> lo = lds<W>(tbl + (b & 15u) * T);
        const Words<W> hi = lds<W>(tbl + (16u + (b >> 4)) * T);
#pragma unroll
        for (int k = 0; k < W; ++k) acc[r].v[k] ^= lo.v[k] ^ hi.v[k];
      }
    }
#pragma unroll
    for (int c = 0; c < kDenseWin; ++c)
#pragma unroll
      for (int r = kTab; r < kRows; ++r)
        if ((mk[c] >> r) & 1u) xor_in(acc[r], x[c]);
  }
  if (store) {
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (r < rows) stg<W>(out(r), acc[r]);
  }
  return true;
}

__device__ __forceinline__ int dense_groups(int n_out) { return (n_out + 31) / 32; }

// All groups of one item.  n_in: input strips (a multiple of kDenseWin);
// masks: the program's control words (masks, then row words).
template <int W, int kForm, class OutAddr>
__device__ __forceinline__ bool dense_item(const WindowView& v, i64 q0, int n_in, int n_out,
                                           int col, bool store, const u32* masks,
                                           const OutAddr& out) {
  constexpr u32 T = DenseTile<W>::T;
  i64 q = q0;
  const int n_win = n_in / kDenseWin;
  const u32* rowb = masks + static_cast<i64>(dense_groups(n_out)) * n_in;
  const u32 tbl = smem_addr(v.ring) + static_cast<u32>(xk::kWinRing * kDenseWin) * T +
                  static_cast<u32>(col);
  for (int g = 0; 32 * g < n_out; ++g) {
    const int rows = n_out - 32 * g < 32 ? n_out - 32 * g : 32;
    const i64 off = static_cast<i64>(g) * n_in;
    auto og = [&](int r) { return out(32 * g + r); };
    const bool ok =
        rows <= 8 ? dense_group<W, kForm, 8>(v, q, n_win, col, store, masks + off, rowb + off, tbl,
                                             rows, og)
        : rows <= 16
            ? dense_group<W, kForm, 16>(v, q, n_win, col, store, masks + off, rowb + off, tbl,
                                        rows, og)
            : dense_group<W, kForm, 32>(v, q, n_win, col, store, masks + off, rowb + off, tbl,
                                        rows, og);
    if (!ok) return false;
  }
  return true;
}

template <int W, int kForm>
struct DenseBody {
  __device__ __forceinline__ bool compute(const LaunchParams& p, const WindowView& v, i64 q0,
                                          i64 s, i64 c0, int len, int col) const {
    const u32* masks = reinterpret_cast<const u32*>(p.code + 8 * static_cast<i64>(p.code_len));
    auto out = [&](int r) {
      return out_block(p.io, s, r >> 3) + static_cast<i64>(r & 7) * p.io.S + c0 + col;
    };
    return dense_item<W, kForm>(v, q0, p.n_in, p.n_out, col, col < len, masks, out);
  }
};

template <int W, int kForm>
struct DenseBatchBody {
  __device__ __forceinline__ int groups(const StripeDesc& d) const {
    return dense_groups(8 * d.n_outblk);
  }
  __device__ __forceinline__ bool compute(const StripeDesc& d, const WindowView& v, i64 q0, i64 c0,
                                          int len, int col) const {
    const u32* masks = reinterpret_cast<const u32*>(d.code + 8 * static_cast<i64>(d.code_len));
    const u64* outs = d.blocks + d.n_inblk;
    auto out = [&](int r) {
      return reinterpret_cast<u8*>(outs[r >> 3]) + static_cast<i64>(r & 7) * d.S + c0 + col;
    };
    return dense_item<W, kForm>(v, q0, 8 * d.n_inblk, 8 * d.n_outblk, col, col < len, masks,
                                out);
  }
};

// Single launches and batches: kDenseThreads consumer threads and the
// producer warp.  Register caps: three CTAs per SM hold 32 accumulators of
// two words (about 120 registers), two CTAs 32 of four.
template <int W, int kForm>
__global__ void __launch_bounds__(kDenseThreads + 32, W == 4 ? 2 : 3)
    dense_kernel(LaunchParams p, const __grid_constant__ TensorMap tm) {
  extern __shared__ __align__(128) u8 smem[];
  run_window_pipeline<DenseBody<W, kForm>, 4 * W>(p, smem, DenseBody<W, kForm>(), &tm);
}

template <int W, int kForm>
__global__ void __launch_bounds__(kDenseThreads + 32, W == 4 ? 2 : 3)
    dense_batch_kernel(BatchParams p) {
  extern __shared__ __align__(128) u8 smem[];
  run_batch_window_pipeline<DenseBatchBody<W, kForm>, 4 * W, true>(p, smem,
                                                                   DenseBatchBody<W, kForm>());
}

// Self-test of the bounded waits: one thread waits, with the pipeline's
// mbar_wait, on an mbarrier whose phase nothing completes; the wait gives
// up after its limit, the kernel records the timeout like the pipelines do
// and returns.
// `also` (may be null) is a second status word, written the way batched
// launches write their batch's or slot's own word.
__global__ void selftest_wait_kernel(int* status, int* also) {
  __shared__ __align__(8) u64 bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_addr(&bar), 1);
  fence_mbar_init();
  if (!mbar_wait(smem_addr(&bar), 0)) {
    if (status) atomicExch(status, XK_STATUS_TIMEOUT);
    if (also) *reinterpret_cast<volatile int*>(also) = XK_STATUS_TIMEOUT;
  }
}

// SplitMix64 (Steele, Lea, Flood 2014) in counter form: byte n of stream
// `seed` is byte n % 8 (little-endian) of mix(seed + (n/8 + 1) * gamma).
__device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void synth_kernel(u8* dst, u64 n, u64 seed, u64 offset) {
  const u64 gamma = 0x9E3779B97F4A7C15ull;
  const u64 stride = static_cast<u64>(gridDim.x) * blockDim.x;
  // aligned fast path: whole 8-byte words of the stream
  if ((offset & 7) == 0 && (reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
    const u64 w0 = offset >> 3;
    const u64 nw = n >> 3;
    u64* d = reinterpret_cast<u64*>(dst);
    for (u64 i = blockIdx.x * static_cast<u64>(blockDim.x) + threadIdx.x; i < nw; i += stride)
      d[i] = mix64(seed + (w0 + i + 1) * gamma);
    for (u64 i = (nw << 3) + blockIdx.x * static_cast<u64>(blockDim.x) + threadIdx.x; i < n;
         i += stride) {
      const u64 b = offset + i;
      dst[i] = static_cast<u8>(mix64(seed + ((b >> 3) + 1) * gamma) >> (8 * (b & 7)));
    }
    return;
  }
  for (u64 i = blockIdx.x * static_cast<u64>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const u64 b = offset + i;
    dst[i] = static_cast<u8>(mix64(seed + ((b >> 3) + 1) * gamma) >> (8 * (b & 7)));
  }
}

}  // namespace

namespace xorec {

size_t interp_smem_bytes(int n_in, int n_slots, int T, int nstage) {
  return 128 + static_cast<size_t>(nstage) * n_in * T + static_cast<size_t>(n_slots) * T;
}

// The kernel instance for a tile of T bytes per strip at `threads` threads:
// 4 bytes per thread (W = 1) or 8 (W = 2).
static const void* interp_kernel_for(int threads, int T) {
  return T == 8 * threads ? reinterpret_cast<const void*>(&interp_kernel<2>)
                          : reinterpret_cast<const void*>(&interp_kernel<1>);
}

int interp_max_ctas_per_sm(int threads, size_t smem, int T) {
  const void* k = interp_kernel_for(threads, T);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

bool launch_interp(const xk::LaunchParams& lp, const xk::TensorMap* tm, int threads, int grid,
                   size_t smem, cudaStream_t stream) {
  if (lp.T != 4 * threads && lp.T != 8 * threads) {
    set_error("interpreter tile must be 4 or 8 bytes per thread");
    return false;
  }
  const void* k = interp_kernel_for(threads, lp.T);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    set_error("cudaFuncSetAttribute(interp) failed");
    return false;
  }
  xk::TensorMap map;
  if (tm) map = *tm;
  else std::memset(&map, 0, sizeof(map));
  if (lp.T == 8 * threads)
    interp_kernel<2><<<grid, threads, smem, stream>>>(lp, map);
  else
    interp_kernel<1><<<grid, threads, smem, stream>>>(lp, map);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("interpreter launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

// Dense bitmatrix executor: 128 consumer threads and the producer warp, the
// form (EC_DENSE_KIND: table or mask) and W words per consumer and
// strip (EC_DENSE_WORDS: 2 or 4).  RS(10,4) encode, 256 stripes x 1 MiB,
// fraction of the measured copy bandwidth: tables 0.521 with two words (3
// CTAs per SM, bound by shared-memory bandwidth), 0.387 with four (their
// tables leave room for one CTA per SM); masks 0.265 with two words, 0.366
// with four (bound by the integer pipe: four words halve the tests per
// byte).
int dense_form() {
  const char* v = std::getenv("EC_DENSE_KIND");
  return v && std::strcmp(v, "mask") == 0 ? kMaskForm : kTableForm;
}

int dense_words() {
  const char* v = std::getenv("EC_DENSE_WORDS");
  if (v && *v) return std::atoi(v) == 2 ? 2 : 4;
  return dense_form() == kMaskForm ? 4 : 2;
}

size_t dense_smem_bytes(int T, int form) {
  return 128 + static_cast<size_t>(xk::kWinRing) * kDenseWin * T +
         (form != kMaskForm ? static_cast<size_t>(32) * T : 0);
}

namespace {

template <int W, int kForm>
struct DenseEntry {
  static const void* single() { return reinterpret_cast<const void*>(&dense_kernel<W, kForm>); }
  static const void* batch() { return reinterpret_cast<const void*>(&dense_batch_kernel<W, kForm>); }
};

const void* dense_kernel_for(int W, int form, bool batch) {
  static const void* const table[2][2][2] = {
      {{DenseEntry<2, kMaskForm>::single(), DenseEntry<2, kMaskForm>::batch()},
       {DenseEntry<2, kTableForm>::single(), DenseEntry<2, kTableForm>::batch()}},
      {{DenseEntry<4, kMaskForm>::single(), DenseEntry<4, kMaskForm>::batch()},
       {DenseEntry<4, kTableForm>::single(), DenseEntry<4, kTableForm>::batch()}}};
  if (form != kMaskForm && form != kTableForm) return nullptr;
  return table[W == 4 ? 1 : 0][form][batch ? 1 : 0];
}

}  // namespace

int dense_max_ctas_per_sm(int W, int form, bool batch, size_t smem) {
  const void* k = dense_kernel_for(W, form, batch);
  if (!k || cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kDenseThreads + 32, smem) !=
      cudaSuccess)
    return 0;
  return n;
}

bool launch_dense(const xk::LaunchParams& lp, const xk::TensorMap* tm, int W, int form,
                  int grid, size_t smem, cudaStream_t stream) {
  const void* k = dense_kernel_for(W, form, false);
  if (!k || lp.T != 4 * W * kDenseThreads || lp.win != kDenseWin || lp.n_in % kDenseWin != 0 ||
      smem < dense_smem_bytes(lp.T, form)) {
    set_error("dense executor: bad launch shape");
    return false;
  }
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    set_error("cudaFuncSetAttribute(dense) failed");
    return false;
  }
  xk::TensorMap map;
  if (tm) map = *tm;
  else std::memset(&map, 0, sizeof(map));
  xk::LaunchParams lpc = lp;
  void* args[] = {&lpc, &map};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kDenseThreads + 32), args, smem,
                                         stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("dense executor launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

bool launch_dense_batch(const xk::BatchParams& bp, int W, int form, int grid, size_t smem,
                        cudaStream_t stream) {
  const void* k = dense_kernel_for(W, form, true);
  if (!k || bp.T != 4 * W * kDenseThreads || bp.win != kDenseWin ||
      smem < dense_smem_bytes(bp.T, form)) {
    set_error("dense executor: bad batch launch shape");
    return false;
  }
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    set_error("cudaFuncSetAttribute(dense batch) failed");
    return false;
  }
  xk::BatchParams bpc = bp;
  void* args[] = {&bpc};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kDenseThreads + 32), args, smem,
                                         stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("batched dense executor launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

size_t interp_batch_smem_bytes(int max_in, int max_slots, int T) {
  return xk::kBatchHeader + static_cast<size_t>(max_in) * T + static_cast<size_t>(max_slots) * T;
}

int interp_batch_max_ctas_per_sm(int threads, size_t smem) {
  if (cudaFuncSetAttribute(interp_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, interp_batch_kernel, threads, smem) !=
      cudaSuccess)
    return 0;
  return n;
}

bool launch_interp_batch(const xk::BatchParams& bp, int threads, int grid, size_t smem,
                         cudaStream_t stream) {
  if (cudaFuncSetAttribute(interp_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    set_error("cudaFuncSetAttribute(interp batch) failed");
    return false;
  }
  interp_batch_kernel<<<grid, threads, smem, stream>>>(bp);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("batched interpreter launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

bool launch_selftest_wait(cudaStream_t stream) {
  DeviceInfo di;
  if (!device_info(&di)) return false;
  return launch_selftest_wait_to(stream, di.status, nullptr);
}

bool launch_selftest_wait_to(cudaStream_t stream, int* status, int* also) {
  selftest_wait_kernel<<<1, 32, 0, stream>>>(status, also);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("self-test launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

bool launch_synth_fill(uint8_t* dst, size_t n, uint64_t seed, uint64_t offset,
                       cudaStream_t stream) {
  if (n == 0) return true;
  DeviceInfo di;
  if (!device_info(&di)) return false;
  const u64 words = (n + 7) / 8;
  u64 blocks = (words + 255) / 256;
  const u64 cap = static_cast<u64>(di.sms) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  synth_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(dst, n, seed, offset);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("synth launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

}  // namespace xorec
