// Compiled tier: the scheduled, fused SLP of a plan is emitted as a
// straight-line CUDA body (one SSA register per statement, operands read
// from the shared-memory stage) and compiled for sm_103a with NVRTC when the
// plan is built.  The pebble schedule (Sec. 6.6) orders the statements so
// that each value dies soon after it is produced, which bounds the registers
// the compiler needs; temporaries never leave the register file.  The tile
// pipeline around the body is the same one the interpreter uses.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace {

const char* kPipelineSrc =
#include "tile_pipeline_src.inc"
    ;

// XORs of two-level programs as inline PTX: the compiler front end would
// otherwise reassociate each row's chain of partial sums (its intermediate
// values have one use) into one expression over all of the row's inputs and
// load every input at once, which is the register pressure the grouping
// avoids.
const char* kOpaqueXorSrc = R"XKSRC(
__device__ __forceinline__ xk::u32 xk_x3(xk::u32 a, xk::u32 b, xk::u32 c) {
  xk::u32 d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ xk::u32 xk_x2(xk::u32 a, xk::u32 b) {
  xk::u32 d;
  asm("xor.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
)XKSRC";

struct JitKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  int threads = 0;          // threads that own a column of the tile
  int block = 0;            // threads per CTA (a producer warp more for windowed programs)
  int win = 0, n_win = 0;   // windowed modules: strips per window, windows per item
  int regs = 0;
  size_t smem_set = 0;
  int device = -1;
};

// Straight-line statements of a scheduled program: one SSA register per
// statement, stores to output strip t of output block b through O(b, t, v)
// as soon as a returned value is ready.  Inputs come from I(c); a two-level
// program (load groups) reads each input word once per group, into a
// register named for the input and the group, at its first use there.
void emit_statements(std::ostringstream& os, const xorec::Program& p) {
  const xorec::Slp& q = p.fused;
  const int nc = q.n_const;
  const bool grouped = !p.load_group.empty();
  std::vector<int> loaded(nc, -1);
  std::vector<std::vector<int>> outs_of(q.n_var);
  for (int r = 0; r < static_cast<int>(q.ret.size()); ++r)
    if (q.ret[r] >= nc) outs_of[q.ret[r] - nc].push_back(r);
  for (size_t k = 0; k < p.sched.steps.size(); ++k) {
    const auto& st = p.sched.steps[k];
    const int g = grouped ? p.load_group[k] : 0;
    if (grouped)
      for (int a : st.args)
        if (a < nc && loaded[a] != g) {
          os << "    const xk::u32 i" << a << "_" << g << " = I(" << a << ");\n";
          loaded[a] = g;
        }
    os << "    const xk::u32 v" << st.node << " = ";
    if (grouped && st.args.size() >= 2 && st.args.size() <= 3) {
      os << (st.args.size() == 3 ? "xk_x3(" : "xk_x2(");
      for (size_t i = 0; i < st.args.size(); ++i) {
        const int a = st.args[i];
        if (i) os << ", ";
        if (a < nc) os << "i" << a << "_" << g;
        else os << "v" << (a - nc);
      }
      os << ");\n";
    } else {
      if (st.args.empty()) os << "0u";
      for (size_t i = 0; i < st.args.size(); ++i) {
        const int a = st.args[i];
        if (i) os << " ^ ";
        if (a < nc && grouped) os << "i" << a << "_" << g;
        else if (a < nc) os << "I(" << a << ")";
        else os << "v" << (a - nc);
      }
      os << ";\n";
    }
    for (int r : outs_of[st.node]) os << "    O(" << (r >> 3) << ", " << (r & 7) << ", v" << st.node << ");\n";
  }
  for (int r = 0; r < static_cast<int>(q.ret.size()); ++r) {
    const int t = q.ret[r];
    if (t < 0) os << "    O(" << (r >> 3) << ", " << (r & 7) << ", 0u);\n";
    else if (t < nc) os << "    O(" << (r >> 3) << ", " << (r & 7) << ", I(" << t << "));\n";
  }
}

// The statements of a windowed program in phases of (group of rows, window
// of inputs), after the output pointers ob<b>, `keep`, `S`, `v`, `q0` and
// `col` are in scope: each phase waits for its ring slot, redefines I(c) to
// read from it and releases it at its end; outputs that are zero are written
// after the last phase.
void emit_window_statements(std::ostringstream& os, const xorec::Program& p, int threads) {
  int win = 0, n_win = 0, n_phases = 0;
  std::vector<int> phase;
  xorec::window_layout(p, &win, &n_win, &n_phases, &phase);
  const xorec::Slp& q = p.fused;
  const int nc = q.n_const;
  const int T = 4 * threads;
  os << "#define O(b, t, v) if (keep) *reinterpret_cast<xk::u32*>(ob##b + (t) * S) = (v)\n";
  std::vector<int> loaded(nc, -1);
  std::vector<std::vector<int>> outs_of(q.n_var);
  for (int r = 0; r < static_cast<int>(q.ret.size()); ++r)
    if (q.ret[r] >= nc) outs_of[q.ret[r] - nc].push_back(r);
  int open = -1;   // phase whose slot is held
  auto enter = [&](int ph) {
    while (open < ph) {
      if (open >= 0) os << "    v.end(q0 + " << open << ");\n";
      ++open;
      const int c0w = (open % n_win) * win;
      os << "    const xk::u8* in" << open << " = v.begin(q0 + " << open << ");\n"
         << "    if (!in" << open << ") return false;\n"
         << "    in" << open << " += col;\n"
         << "#undef I\n#define I(c) (*reinterpret_cast<const xk::u32*>(in" << open << " + ((c) - "
         << c0w << ") * " << T << "))\n";
    }
  };
  for (size_t k = 0; k < p.sched.steps.size(); ++k) {
    const auto& st = p.sched.steps[k];
    const int g = p.load_group[k];
    enter(phase[k]);
    for (int a : st.args)
      if (a < nc && loaded[a] != g) {
        os << "    const xk::u32 i" << a << "_" << g << " = I(" << a << ");\n";
        loaded[a] = g;
      }
    os << "    const xk::u32 v" << st.node << " = ";
    if (st.args.size() >= 2 && st.args.size() <= 3) {
      os << (st.args.size() == 3 ? "xk_x3(" : "xk_x2(");
      for (size_t i = 0; i < st.args.size(); ++i) {
        const int a = st.args[i];
        if (i) os << ", ";
        if (a < nc) os << "i" << a << "_" << g;
        else os << "v" << (a - nc);
      }
      os << ");\n";
    } else {
      if (st.args.empty()) os << "0u";
      for (size_t i = 0; i < st.args.size(); ++i) {
        const int a = st.args[i];
        if (i) os << " ^ ";
        if (a < nc) os << "i" << a << "_" << g;
        else os << "v" << (a - nc);
      }
      os << ";\n";
    }
    for (int r : outs_of[st.node]) os << "    O(" << (r >> 3) << ", " << (r & 7) << ", v" << st.node << ");\n";
  }
  enter(n_phases - 1);   // phases without statements still take and free their slot
  os << "    v.end(q0 + " << (n_phases - 1) << ");\n";
  for (int r = 0; r < static_cast<int>(q.ret.size()); ++r)
    if (q.ret[r] < 0) os << "    O(" << (r >> 3) << ", " << (r & 7) << ", 0u);\n";
  os << "#undef I\n#undef O\n";
}

// Windowed single-launch body (run_window_pipeline).
std::string gen_window_body(const xorec::Program& p, int threads) {
  std::ostringstream os;
  os << "struct SlpBody {\n"
        "  __device__ __forceinline__ bool compute(const xk::LaunchParams& p, const xk::WindowView& v,\n"
        "      xk::i64 q0, xk::i64 s, xk::i64 c0, int len, int col) const {\n"
        "    const bool keep = col < len;\n"
        "    const xk::i64 S = p.io.S;\n";
  for (int b = 0; b < p.n_out / 8; ++b)
    os << "    xk::u8* ob" << b << " = xk::out_block(p.io, s, " << b << ") + c0 + col;\n";
  emit_window_statements(os, p, threads);
  os << "    return true;\n  }\n};\n";
  return os.str();
}

// Windowed multi-program module (run_batch_window_pipeline): every program
// has one group of rows and the same windows.
std::string gen_window_module_source(const std::vector<const xorec::Program*>& progs, int threads,
                                     int minb) {
  std::ostringstream os;
  os << kPipelineSrc << "\n" << kOpaqueXorSrc;
  for (size_t i = 0; i < progs.size(); ++i) {
    os << "__device__ __forceinline__ bool prog_" << i
       << "(const xk::StripeDesc& d, const xk::WindowView& v, xk::i64 q0, xk::i64 c0, int col,\n"
          "    bool keep) {\n"
          "    const xk::i64 S = d.S;\n";
    for (int b = 0; b < progs[i]->n_out / 8; ++b)
      os << "    xk::u8* ob" << b << " = reinterpret_cast<xk::u8*>(d.blocks[d.n_inblk + " << b
         << "]) + c0 + col;\n";
    emit_window_statements(os, *progs[i], threads);
    os << "    return true;\n}\n";
  }
  os << "struct ModBody {\n"
        "  __device__ __forceinline__ bool compute(const xk::StripeDesc& d, const xk::WindowView& v,\n"
        "      xk::i64 q0, xk::i64 c0, int len, int col) const {\n"
        "    const bool keep = col < len;\n"
        "    switch (d.prog) {\n";
  for (size_t i = 0; i < progs.size(); ++i)
    os << "      case " << i << ": return prog_" << i << "(d, v, q0, c0, col, keep);\n";
  os << "      default: return false;\n"
        "    }\n"
        "  }\n"
        "};\n";
  os << "extern \"C\" __global__ void __launch_bounds__(" << threads + 32 << ", " << minb
     << ") xorec_mod(xk::BatchParams p) {\n"
        "  extern __shared__ __align__(128) xk::u8 smem[];\n"
        "  xk::run_batch_window_pipeline(p, smem, ModBody());\n"
        "}\n";
  return os.str();
}

// Single-program body.  Narrow programs (n_in <= kPreloadMaxInputs):
// load() copies each thread's 4-byte column of every input strip from the
// stage into registers and compute() runs the statements from registers.
// Wide programs run from the stage (kEarlyRelease = false).
std::string gen_body(const xorec::Program& p, int threads) {
  const int nc = p.fused.n_const;
  const int T = 4 * threads;
  std::ostringstream os;
  if (nc > xorec::kPreloadMaxInputs) {
    os << "struct SlpBody {\n"
          "  static constexpr bool kEarlyRelease = false;\n"
          "  __device__ __forceinline__ void operator()(const xk::LaunchParams& p, xk::i64 s,\n"
          "      xk::i64 c0, int len, const xk::u8* stg, xk::u8*) const {\n"
          "    const int col = threadIdx.x * 4;\n"
          "    if (col >= len) return;\n"
          "    const xk::u8* in = stg + col;\n"
          "    const xk::i64 S = p.io.S;\n";
    for (int b = 0; b < p.n_out / 8; ++b)
      os << "    xk::u8* ob" << b << " = xk::out_block(p.io, s, " << b << ") + c0 + col;\n";
    os << "#define I(c) (*reinterpret_cast<const xk::u32*>(in + (c) * " << T << "))\n";
    os << "#define O(b, t, v) *reinterpret_cast<xk::u32*>(ob##b + (t) * S) = (v)\n";
    emit_statements(os, p);
    os << "#undef I\n#undef O\n  }\n};\n";
    return os.str();
  }
  os << "struct SlpBody {\n"
        "  static constexpr bool kEarlyRelease = true;\n"
        "  struct Regs { xk::u32 x[" << (nc > 0 ? nc : 1) << "]; };\n"
        "  __device__ __forceinline__ void load(const xk::LaunchParams&, int len,\n"
        "      const xk::u8* stg, Regs& r) const {\n"
        "    const int col = threadIdx.x * 4;\n"
        "    if (col >= len) return;\n"
        "    const xk::u8* in = stg + col;\n";
  for (int c = 0; c < nc; ++c)
    os << "    r.x[" << c << "] = *reinterpret_cast<const xk::u32*>(in + " << c * T << ");\n";
  os << "  }\n"
        "  __device__ __forceinline__ void compute(const xk::LaunchParams& p, xk::i64 s,\n"
        "      xk::i64 c0, int len, Regs& r) const {\n"
        "    const int col = threadIdx.x * 4;\n"
        "    if (col >= len) return;\n"
        "    const xk::i64 S = p.io.S;\n";
  for (int b = 0; b < p.n_out / 8; ++b)
    os << "    xk::u8* ob" << b << " = xk::out_block(p.io, s, " << b << ") + c0 + col;\n";
  os << "#define I(c) r.x[c]\n";
  os << "#define O(b, t, v) *reinterpret_cast<xk::u32*>(ob##b + (t) * S) = (v)\n";
  emit_statements(os, p);
  os << "#undef I\n#undef O\n  }\n};\n";
  return os.str();
}

// Multi-program module for batched launches: all programs share n_in; the
// stripe descriptor names the program (d.prog) and the output blocks.
std::string gen_module_source(const std::vector<const xorec::Program*>& progs, int threads,
                              int minb) {
  const int nc = progs.front()->n_in;
  const int T = 4 * threads;
  std::ostringstream os;
  os << kPipelineSrc << "\n";
  for (size_t i = 0; i < progs.size(); ++i) {
    os << "__device__ __forceinline__ void prog_" << i
       << "(const xk::StripeDesc& d, xk::i64 c0, int col, const xk::u32* x) {\n"
          "    const xk::i64 S = d.S;\n";
    for (int b = 0; b < progs[i]->n_out / 8; ++b)
      os << "    xk::u8* ob" << b << " = reinterpret_cast<xk::u8*>(d.blocks[d.n_inblk + " << b
         << "]) + c0 + col;\n";
    os << "#define I(c) x[c]\n";
    os << "#define O(b, t, v) *reinterpret_cast<xk::u32*>(ob##b + (t) * S) = (v)\n";
    emit_statements(os, *progs[i]);
    os << "#undef I\n#undef O\n}\n";
  }
  if (nc > xorec::kPreloadMaxInputs) {
    // wide programs: operands from the stage at each use
    std::ostringstream ws;
    ws << kPipelineSrc << "\n";
    if (std::any_of(progs.begin(), progs.end(),
                    [](const xorec::Program* q) { return !q->load_group.empty(); }))
      ws << kOpaqueXorSrc;
    for (size_t i = 0; i < progs.size(); ++i) {
      ws << "__device__ __forceinline__ void prog_" << i
         << "(const xk::StripeDesc& d, xk::i64 c0, int col, const xk::u8* in) {\n"
            "    const xk::i64 S = d.S;\n";
      for (int b = 0; b < progs[i]->n_out / 8; ++b)
        ws << "    xk::u8* ob" << b << " = reinterpret_cast<xk::u8*>(d.blocks[d.n_inblk + " << b
           << "]) + c0 + col;\n";
      ws << "#define I(c) (*reinterpret_cast<const xk::u32*>(in + (c) * " << T << "))\n";
      ws << "#define O(b, t, v) *reinterpret_cast<xk::u32*>(ob##b + (t) * S) = (v)\n";
      emit_statements(ws, *progs[i]);
      ws << "#undef I\n#undef O\n}\n";
    }
    ws << "struct ModBody {\n"
          "  static constexpr bool kEarlyRelease = false;\n"
          "  __device__ __forceinline__ void operator()(const xk::StripeDesc& d, xk::i64 c0, int len,\n"
          "      const xk::u8* stg, xk::u8*, int) const {\n"
          "    const int col = threadIdx.x * 4;\n"
          "    if (col >= len) return;\n"
          "    switch (d.prog) {\n";
    for (size_t i = 0; i < progs.size(); ++i)
      ws << "      case " << i << ": prog_" << i << "(d, c0, col, stg + col); break;\n";
    ws << "      default: break;\n"
          "    }\n"
          "  }\n"
          "};\n";
    ws << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", " << minb
       << ") xorec_mod(xk::BatchParams p) {\n"
          "  extern __shared__ __align__(128) xk::u8 smem[];\n"
          "  xk::run_batch_pipeline(p, smem, ModBody(), nullptr);\n"
          "}\n";
    return ws.str();
  }
  os << "struct ModBody {\n"
        "  static constexpr bool kEarlyRelease = true;\n"
        "  struct Regs { xk::u32 x[" << nc << "]; };\n"
        "  __device__ __forceinline__ void load(const xk::StripeDesc&, int len, const xk::u8* stg,\n"
        "                                       Regs& r) const {\n"
        "    const int col = threadIdx.x * 4;\n"
        "    if (col >= len) return;\n"
        "    const xk::u8* in = stg + col;\n";
  for (int c = 0; c < nc; ++c)
    os << "    r.x[" << c << "] = *reinterpret_cast<const xk::u32*>(in + " << c * T << ");\n";
  os << "  }\n"
        "  __device__ __forceinline__ void compute(const xk::StripeDesc& d, xk::i64 c0, int len,\n"
        "                                          Regs& r) const {\n"
        "    const int col = threadIdx.x * 4;\n"
        "    if (col >= len) return;\n"
        "    switch (d.prog) {\n";
  for (size_t i = 0; i < progs.size(); ++i)
    os << "      case " << i << ": prog_" << i << "(d, c0, col, r.x); break;\n";
  os << "      default: break;\n"
        "    }\n"
        "  }\n"
        "};\n";
  os << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", " << minb
     << ") xorec_mod(xk::BatchParams p) {\n"
        "  extern __shared__ __align__(128) xk::u8 smem[];\n"
        "  xk::run_batch_pipeline(p, smem, ModBody(), nullptr);\n"
        "}\n";
  return os.str();
}

int env_or(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

// minb > 0 overrides the resident CTAs per SM the kernel is built for.
std::string gen_source(const xorec::Program& p, int threads, int minb = 0) {
  std::ostringstream os;
  os << kPipelineSrc << "\n";
  if (!p.load_group.empty()) os << kOpaqueXorSrc;
  if (xorec::windowed(p)) {
    const int block = threads + 32;
    os << gen_window_body(p, threads);
    os << "extern \"C\" __global__ void __launch_bounds__(" << block << ", "
       << (minb > 0 ? minb : p.minb > 0 ? p.minb : xorec::minb_for(block, 128))
       << ") xorec_slp(xk::LaunchParams p, const __grid_constant__ xk::TensorMap tm) {\n"
          "  extern __shared__ __align__(128) xk::u8 smem[];\n"
          "  xk::run_window_pipeline(p, smem, SlpBody(), &tm);\n"
          "}\n";
    return os.str();
  }
  os << gen_body(p, threads);
  os << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", "
     << (p.minb > 0 ? p.minb : env_or("EC_JIT_MINB", xorec::default_minb(threads, p.n_in)))
     << ") xorec_slp(xk::LaunchParams p, const __grid_constant__ xk::TensorMap tm) {\n"
        "  extern __shared__ __align__(128) xk::u8 smem[];\n"
        "  xk::run_pipeline(p, smem, SlpBody(), &tm);\n"
        "}\n";
  return os.str();
}

}  // namespace

namespace xorec {

// Phases of a two-level program read window by window: window `win` (the
// program's input window, a multiple of 8 strips), n_win windows per group,
// one phase per (group, window) in that order; phase[k] is the phase of
// schedule step k (a step with input operands belongs to their window, one
// without to the phase before it).  False when the program does not have
// that form (not two-level, or an output that is an input strip itself).
bool window_layout(const Program& p, int* win, int* n_win, int* n_phases, std::vector<int>* phase) {
  if (p.load_group.empty() || p.stats.window <= 0 || p.stats.window % 8 != 0) return false;
  const int nc = p.fused.n_const;
  if (p.load_group.size() != p.sched.steps.size() || p.sched.steps.empty()) return false;
  for (int t : p.fused.ret)
    if (t >= 0 && t < nc) return false;
  const int w = p.stats.window;
  const int nw = (p.n_in + w - 1) / w;
  int groups = 0;
  for (int g : p.load_group) groups = std::max(groups, g + 1);
  std::vector<int> ph(p.sched.steps.size(), 0);
  int cur = 0;
  for (size_t k = 0; k < p.sched.steps.size(); ++k) {
    int x = -1;
    for (int a : p.sched.steps[k].args)
      if (a < nc) {
        const int y = p.load_group[k] * nw + a / w;
        if (x >= 0 && y != x) return false;   // operands from two windows
        x = y;
      }
    if (x < 0) x = cur;
    if (x < cur) return false;                // phases must not go back
    ph[k] = cur = x;
  }
  *win = w;
  *n_win = nw;
  *n_phases = groups * nw;
  if (phase) *phase = std::move(ph);
  return true;
}

// Measured on GB300 (encode, 128 stripes x 1 MiB, fraction of the copy
// bandwidth, full-stage kernel -> windowed): RS(100,4) 0.45 -> 0.93,
// RS(48,4) 0.75 -> 0.98, RS(32,4) 0.93 -> 0.98 (scaled Cauchy matrix 1.03 ->
// 0.99), RS(16,4) 1.02 -> 0.98, RS(24,8) (two groups) 0.78 -> 0.68.  The
// full-stage kernel keeps several CTAs per SM up to 256 input strips, and a
// second group of rows reads every window again, so the windowed pipeline is
// taken for single-group programs of more than 256 input strips.
// EC_WINDOWED=1 takes it for every program of the form, 0 for none.
bool windowed(const Program& p) {
  const char* e = std::getenv("EC_WINDOWED");
  const int force = e && *e ? std::atoi(e) : -1;
  if (force == 0) return false;
  int win, n_win, n_phases;
  if (!window_layout(p, &win, &n_win, &n_phases, nullptr)) return false;
  return force == 1 || (n_phases == n_win && p.n_in > 256);
}

// A module of these programs takes the batched windowed pipeline: every
// program is windowed, with one group of rows (one phase per window), and
// all have the same windows.
bool window_module(const std::vector<const Program*>& progs, int* win, int* n_win) {
  int w0 = -1, nw0 = -1;
  for (const Program* p : progs) {
    int w, nw, np;
    if (!windowed(*p) || !window_layout(*p, &w, &nw, &np, nullptr) || np != nw) return false;
    if (w0 >= 0 && (w != w0 || nw != nw0)) return false;
    w0 = w;
    nw0 = nw;
  }
  if (w0 < 0) return false;
  *win = w0;
  *n_win = nw0;
  return true;
}

bool jit_module_window(void* mod, int* win, int* n_win) {
  auto* jk = static_cast<JitKernel*>(mod);
  if (!jk || jk->win <= 0) return false;
  *win = jk->win;
  *n_win = jk->n_win;
  return true;
}

bool jit_available() {
  int major = 0, minor = 0;
  return nvrtcVersion(&major, &minor) == NVRTC_SUCCESS;
}

static bool jit_set_smem(JitKernel* jk, size_t smem) {
  if (jk->smem_set >= smem) return true;
  if (cudaKernelSetAttributeForDevice(jk->kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem), jk->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  jk->smem_set = smem;
  return true;
}

// Largest "N bytes spill stores" figure of a ptxas report (0 if none).
static long spill_stores(const std::string& log) {
  long most = 0;
  const std::string key = " bytes spill stores";
  for (size_t at = log.find(key); at != std::string::npos; at = log.find(key, at + 1)) {
    size_t b = at;
    while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
    if (b < at) most = std::max(most, std::strtol(log.c_str() + b, nullptr, 10));
  }
  return most;
}

// NVRTC: source -> cubin for the current device -> loaded kernel `name`.
// With spill_bytes, ptxas also reports and *spill_bytes receives the bytes
// it spilled per thread.
static JitKernel* compile_and_load(const std::string& src, const char* name, int threads,
                                   std::string* err, long* spill_bytes = nullptr, int block = 0) {
  xorec::TraceRange trace_("xorec nvrtc compile");
  DeviceInfo di;
  if (!device_info(&di)) {
    *err = "no CUDA device";
    return nullptr;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, di.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, di.device) != cudaSuccess) {
    *err = "cudaDeviceGetAttribute failed";
    return nullptr;
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "xorec_slp.cu", 0, nullptr, nullptr) !=
      NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return nullptr;
  }
  char arch[64];
  std::snprintf(arch, sizeof(arch), "-arch=sm_%d%da", major, minor);
  const char* opts[] = {arch, "-std=c++17", "-default-device", "--extra-device-vectorization",
                        "--ptxas-options=-v"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, spill_bytes ? 5 : 4, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    *err = "NVRTC compile failed: " + log.substr(0, 2000);
    return nullptr;
  }
  if (spill_bytes) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    *spill_bytes = spill_stores(log);
  }
  size_t nbin = 0;
  nvrtcGetCUBINSize(prog, &nbin);
  std::vector<char> cubin(nbin);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  auto* jk = new JitKernel();
  if (cudaLibraryLoadData(&jk->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
          cudaSuccess ||
      cudaLibraryGetKernel(&jk->kern, jk->lib, name) != cudaSuccess) {
    cudaGetLastError();
    delete jk;
    *err = "loading the compiled SLP kernel failed";
    return nullptr;
  }
  jk->threads = threads;
  jk->block = block > 0 ? block : threads;
  jk->device = di.device;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(jk->kern)) == cudaSuccess)
    jk->regs = fa.numRegs;
  else
    cudaGetLastError();
  return jk;
}

static void jit_release_kernel(JitKernel* jk) {
  cudaLibraryUnload(jk->lib);
  delete jk;
}

// Compile `p` for the current device's architecture.  Stores a JitKernel in
// p->jit on success.
bool jit_compile(Program* p, int threads, std::string* err) {
  if (p->jit) return true;
  if (windowed(*p) && p->minb <= 0) {
    // the register cap of three resident CTAs is too tight for the partial
    // sums and window inputs of the widest programs: ptxas spills there, and
    // the kernel is compiled again for two CTAs per SM
    int minb = minb_for(threads + 32, 128);
    for (;;) {
      long spill = 0;
      JitKernel* jk = compile_and_load(gen_source(*p, threads, minb), "xorec_slp", threads, err,
                                       &spill, threads + 32);
      if (!jk) return false;
      if (spill == 0 || minb <= 2) {
        p->jit = jk;
        return true;
      }
      jit_release_kernel(jk);
      --minb;
    }
  }
  JitKernel* jk = compile_and_load(gen_source(*p, threads), "xorec_slp", threads, err, nullptr,
                                   windowed(*p) ? threads + 32 : threads);
  if (!jk) return false;
  p->jit = jk;
  return true;
}

// A module of programs sharing n_in (batched launches).  With
// no_spill, a module that ptxas reports spilling is compiled again with one
// resident CTA per SM fewer (a higher register cap), down to one.
void* jit_compile_module(const std::vector<const Program*>& progs, int threads, int minb,
                         std::string* err, bool no_spill) {
  if (progs.empty()) {
    *err = "empty module";
    return nullptr;
  }
  // modules of windowed programs take the batched windowed pipeline, built
  // for three CTAs per SM, or two when ptxas spills at three
  int win = 0, n_win = 0;
  if (window_module(progs, &win, &n_win)) {
    for (int mb = minb_for(threads + 32, 128);; --mb) {
      long spill = 0;
      JitKernel* jk = compile_and_load(gen_window_module_source(progs, threads, mb), "xorec_mod",
                                       threads, err, &spill, threads + 32);
      if (!jk) return nullptr;
      jk->win = win;
      jk->n_win = n_win;
      if (spill == 0 || mb <= 2) return jk;
      jit_release_kernel(jk);
    }
  }
  for (;;) {
    long spill = 0;
    JitKernel* jk = compile_and_load(gen_module_source(progs, threads, minb), "xorec_mod", threads,
                                     err, no_spill ? &spill : nullptr);
    if (!jk || spill == 0 || minb <= 1) return jk;
    jit_module_release(jk);
    --minb;
  }
}

std::string jit_module_source(const std::vector<const Program*>& progs, int threads, int minb) {
  if (progs.empty()) return std::string();
  int win = 0, n_win = 0;
  if (window_module(progs, &win, &n_win))
    return gen_window_module_source(progs, threads, minb_for(threads + 32, 128));
  return gen_module_source(progs, threads, minb);
}

int jit_module_ctas_per_sm(void* mod, size_t smem) {
  auto* jk = static_cast<JitKernel*>(mod);
  if (!jk || !jit_set_smem(jk, smem)) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, reinterpret_cast<const void*>(jk->kern),
                                                    jk->block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

bool jit_module_launch(void* mod, const xk::BatchParams& bp, int grid, size_t smem,
                       cudaStream_t stream) {
  auto* jk = static_cast<JitKernel*>(mod);
  if (!jk || !jit_set_smem(jk, smem)) {
    set_error("compiled module missing or shared memory size refused");
    return false;
  }
  xk::BatchParams copy = bp;
  copy.win = jk->win;
  copy.n_win = jk->n_win;
  void* args[] = {&copy};
  const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(jk->kern), dim3(grid),
                                         dim3(jk->block), args, smem, stream);
  if (e != cudaSuccess) {
    set_error(std::string("compiled module launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

void jit_module_release(void* mod) {
  auto* jk = static_cast<JitKernel*>(mod);
  if (!jk) return;
  cudaLibraryUnload(jk->lib);
  delete jk;
}

int jit_module_threads(void* mod) {
  auto* jk = static_cast<JitKernel*>(mod);
  return jk ? jk->threads : 0;
}

int jit_module_regs(void* mod) {
  auto* jk = static_cast<JitKernel*>(mod);
  return jk ? jk->regs : 0;
}

int jit_max_ctas_per_sm(Program* p, int threads, size_t smem) {
  auto* jk = static_cast<JitKernel*>(p->jit);
  if (!jk || !jit_set_smem(jk, smem)) return 0;
  (void)threads;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, reinterpret_cast<const void*>(jk->kern),
                                                    jk->block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

bool jit_launch(Program* p, const xk::LaunchParams& lp, const xk::TensorMap* tm, int threads,
                int grid, size_t smem, cudaStream_t stream) {
  auto* jk = static_cast<JitKernel*>(p->jit);
  if (!jk || jk->threads != threads) {
    set_error("compiled kernel missing or built for another block size");
    return false;
  }
  if (!jit_set_smem(jk, smem)) {
    set_error("cannot set shared memory size of the compiled kernel");
    return false;
  }
  xk::LaunchParams copy = lp;
  xk::TensorMap map;
  if (tm) map = *tm;
  else std::memset(&map, 0, sizeof(map));
  void* args[] = {&copy, &map};
  const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(jk->kern), dim3(grid),
                                         dim3(jk->block), args, smem, stream);
  if (e != cudaSuccess) {
    set_error(std::string("compiled kernel launch failed: ") + cudaGetErrorString(e));
    return false;
  }
  return true;
}

// Source of the straight-line kernel (for inspection and tests).
std::string jit_source(const Program& p, int threads) { return gen_source(p, threads); }

void jit_release(Program* p) {
  auto* jk = static_cast<JitKernel*>(p ? p->jit : nullptr);
  if (!jk) return;
  cudaLibraryUnload(jk->lib);
  delete jk;
  p->jit = nullptr;
}

bool jit_is_windowed(const Program* p) {
  const auto* jk = static_cast<const JitKernel*>(p ? p->jit : nullptr);
  return jk && jk->block != jk->threads;
}

int jit_regs(const Program* p) {
  const auto* jk = static_cast<const JitKernel*>(p ? p->jit : nullptr);
  return jk ? jk->regs : 0;
}

}  // namespace xorec
