// Plan construction: coding matrix -> bitmatrix -> SLP -> optimiser passes
// -> executable program for the GPU executors (host side).
#pragma once
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "slp.h"

namespace xorec {

// Bitmatrix of a rows x cols matrix over GF(2^8): row 8i+s, column 8j+t is
// bit s of A[i][j] * 2^t (Sec. 1, property (ii)).
std::vector<Bits> bitmatrix_rows(int rows, int cols, const uint8_t* A);

// Programs with more input strips than this do not preload every input word
// into registers: their compiled body reads operands from the shared-memory
// stage.
constexpr int kPreloadMaxInputs = 96;
// Preloaded programs with more input strips than this need more than 128
// registers per thread (the input words plus the pipeline's own state):
// ptxas spills 16-68 bytes at a 128-register cap for every code of 11 or 12
// data blocks, and none at 168, while no code of up to 10 spills at 128.
constexpr int kPreloadCap128Inputs = 80;
// Largest program (#_M memory operations) the compiled tier takes, so that
// NVRTC compiles it in seconds.
constexpr long kMaxCompiledMemOps = 65536;

enum OptLevel { kOptRaw = 0, kOptRePair = 1, kOptXorRePair = 2, kOptTriple = 3 };
enum SchedKind { kSchedDfs = 0, kSchedGreedy = 1 };

struct PipelineStats {
  SlpMetrics raw, compressed, fused;
  int raw_ccap = 0;
  int sched_nvar = 0;      // pebbles of the paper's game (goals hold)
  int slots = 0;           // pebbles when outputs stream out (GPU setting)
  int temps = 0;           // temporaries kept by (Xor)RePair
  int max_live = 0;        // registers with all inputs preloaded
  long lop3 = 0;           // three-input XOR instructions of the fused program
  long loads = 0;          // input words a thread loads from the stage per tile
  int window = 0;          // input window of a two-level program (0 = not one)
  int window_temps = 0;    // XorRePair temporals per window of a two-level program
};

// An executable program for one linear map from n_in input strips to n_out
// output strips.  `code` is the interpreter's instruction stream:
//   word 0: number of arguments a
//   word 1: number of outputs o | (has_slot << 15)
//   [slot]               if has_slot
//   out_0 .. out_{o-1}   output strip indices
//   arg_0 .. arg_{a-1}   operand ids: < n_in input strip, else slot + n_in
// `sched` keeps the scheduled fused program for code generation.
//
// `chunks` is the stream the interpreter runs on the device, in 16-byte
// chunks of eight 16-bit words, so that one 128-bit load brings eight
// operand ids.  Per statement: a header chunk (a, o, slot or 0xffff, the
// first five output strips, unused ones 0xffff), ceil(a/8) chunks of
// operand ids (the last padded with 0xffff), then, when o > 5, chunks of
// the remaining output strips (padded with 0xffff).  For programs of up to
// kPreloadMaxInputs inputs it is the unoptimised fused program's stream (no
// slots: the interpreter's occupancy is bounded by the shared memory its
// slots take), with interp_slots = 0; otherwise the program's own.
struct Program {
  int n_in = 0, n_out = 0, n_slots = 0, n_stmts = 0;
  std::vector<uint16_t> code;
  std::vector<uint16_t> chunks;
  int interp_slots = 0;      // slots of the stream in `chunks`
  // column masks of the program's bitmatrix for the dense executor: word
  // g * n_in + c, bit r is bit (32 g + r, c) (output strip 32 g + r reads
  // input strip c); ceil(n_out / 32) groups
  std::vector<uint32_t> masks;
  // row words of the dense executor's table form: word g * n_in + 8 w + j
  // holds the bits of window w (input strips 8 w .. 8 w + 7, bit i for strip
  // 8 w + i) of output strips 32 g + 4 j .. 32 g + 4 j + 3, one byte each
  std::vector<uint32_t> rowbits;
  PipelineStats stats;
  Slp fused;                 // single-assignment fused program
  Schedule sched;            // GPU schedule of `fused`
  // two-level programs (slp_rows_stream): load group of each schedule step;
  // the compiled body loads an input word at its first use in a group.
  // Empty: inputs preloaded (narrow) or read at every use (wide).
  std::vector<int> load_group;
  uint64_t hash = 0;         // content hash of the fused program
  // device copy of `chunks` followed by `masks` and `rowbits` (owned; freed
  // by the plan)
  uint16_t* d_code = nullptr;
  // compiled tier (set once a straight-line kernel exists for this program)
  void* jit = nullptr;
  // multi-program module holding this program (batched launches)
  void* mod = nullptr;
  int mod_index = -1;
  // launch shape of the compiled tier chosen by the autotuner (0 = default)
  int threads = 0;
  int minb = 0;
};

struct PlanOptions {
  int opt_level = kOptXorRePair;
  int sched = kSchedDfs;
  int greedy_cap = 128;
  bool cancel_pairs = true;
  // Temporaries budget of (Xor)RePair: -1 = none (the paper's full run),
  // -2 = automatic (largest budget whose schedule needs at most reg_budget
  // registers with all inputs preloaded), >= 0 = explicit.
  int max_temps = -2;
  int reg_budget = 128;
  // Programs with more than kPreloadMaxInputs inputs and automatic
  // temporaries: input window of the two-level program (0 = automatic,
  // -1 = off: one fused statement per row, operands read at every use).
  int stream_window = 0;
  // XorRePair temporals per window of a two-level program (0 = automatic,
  // -1 = none, > 0 = explicit).
  int stream_temps = 0;
};

// The device form of an interpreter stream (Program::chunks).
std::vector<uint16_t> chunk_stream(const std::vector<uint16_t>& code);

// Build the program for the linear map A (rows x cols over GF(2^8)).
bool build_program(int rows, int cols, const uint8_t* A, const PlanOptions& o,
                   Program* out, std::string* err);

}  // namespace xorec
