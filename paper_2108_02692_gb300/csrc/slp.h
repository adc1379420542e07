// Straight-line programs over XOR and the optimiser passes of the paper,
// retargeted to a GPU executor (host side).
//
//   SLP / MultiSLP and set semantics ........ Sec. 4.1, Sec. 5.1
//   RePair, XorRePair (Rebuild) .............. Sec. 4.3, Sec. 4.4
//   XOR fusion (deforestation) ............... Sec. 5.2
//   abstract LRU cache, CCap, IOcost ......... Sec. 6.2
//   pebble game, DFS and greedy schedulers ... Sec. 6.4, Sec. 6.6
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace xorec {

// Growable bitset used for set semantics (sets of constants) and for
// "which originals contain this term" indices.
struct Bits {
  std::vector<uint64_t> w;
  Bits() = default;
  explicit Bits(int n) : w((n + 63) / 64, 0) {}
  void set(int i) { w[i >> 6] |= (1ull << (i & 63)); }
  void flip(int i) { w[i >> 6] ^= (1ull << (i & 63)); }
  bool test(int i) const { return (w[i >> 6] >> (i & 63)) & 1ull; }
  int count() const;
  int xor_count(const Bits& o) const;   // |this (+) o|
  int and_count(const Bits& o) const;   // |this & o|
  Bits& operator^=(const Bits& o);
  bool operator==(const Bits& o) const { return w == o.w; }
  bool any() const;
};

// A statement dst <- XOR(args).  Terms are ints: constants are
// [0, n_const), variables are [n_const, n_const + n_var).  A variable may
// be assigned more than once (register-allocated programs such as P_reg or
// pebble strategies); RePair and fusion require single assignment.
struct Stmt {
  int dst;
  std::vector<int> args;
};

struct Slp {
  int n_const = 0;
  int n_var = 0;
  std::vector<Stmt> body;
  std::vector<int> ret;   // returned terms; -1 = the zero array
  std::vector<std::string> const_names;
  std::vector<std::string> var_names;
  bool is_const(int t) const { return t >= 0 && t < n_const; }
};

struct SlpMetrics {
  long xors;   // sum over statements of (arity - 1)                [Sec. 4.1]
  long mem;    // #_M: sum over statements of (arity + 1)            [Sec. 5.1]
  int nvar;    // number of distinct assigned variables              [Sec. 4.1]
  int stmts;   // number of statements (the paper's #XOR after fusion)
};

// Set semantics: the value of each returned term as a set of constants.
std::vector<Bits> semantics(const Slp& p);
bool equivalent(const Slp& a, const Slp& b);
SlpMetrics metrics(const Slp& p);

// Abstract LRU cache (Sec. 6.2): for each statement, access the arguments
// in order (load on miss, else move to most-recent), then allocate or
// update the destination; evict the least recently used element when full.
// IOcost = loads + evictions.  reloads counts loads of evicted elements.
long lru_iocost(const Slp& p, int cap, long* reloads = nullptr);
// CCap: minimum capacity with no reload.
int ccap(const Slp& p);

// Text form (for the paper's worked examples and debugging):
//   const a b c d
//   v1 = a b
//   v2 = b c d
//   ret v2 v3 v1
bool parse_slp(const std::string& text, Slp* out, std::string* err);
std::string slp_to_text(const Slp& p);

// One statement per row: v_r <- XOR(columns set in row r), in column order.
Slp slp_rows_fused(int n_const, const std::vector<Bits>& rows,
                   const std::vector<int>& row_order);
// Binary left-to-right chains per row (v <- c1 + c2; v <- v + c3; ...),
// the unoptimised program whose counts the paper prints (Sec. 7.5).
Slp slp_rows_chains(int n_const, const std::vector<Bits>& rows,
                    const std::vector<int>& row_order);

// Two-level program for rows whose input words do not all fit the
// registers: the multilevel pebble game named as future work in Sec. 8, with
// the registers as the first level and the shared-memory tile of the inputs
// (Sec. 6.1's blocking) as the second.  Rows are taken in groups of
// group_rows partial sums and the inputs in windows of `window` columns; for
// each group and window, every row of the group adds the window's inputs it
// contains, two per statement (acc <- acc + a + b, one three-input XOR; a
// row's first statement takes up to three inputs).  Within a group every
// input is needed in one window only, so it is loaded once per group.
// Single assignment, not fused (fusion would merge each row back into one
// statement that needs all its inputs at once).  stmt_group receives the
// group of each statement.
// window_temps > 0: the group's rows restricted to each window are first
// shortened by XorRePair (RePair when xor_cancel is false) with at most
// window_temps temporals, and fusion (Sec. 4.3-4.4, Sec. 5.2); temporals live
// within their window, and a row's fused window part is added into its
// partial sum.
Slp slp_rows_stream(int n_const, const std::vector<Bits>& rows, int window, int group_rows,
                    std::vector<int>* stmt_group, int window_temps = 0,
                    bool xor_cancel = true);

// RePair (xor_cancel = false) or XorRePair (true) on the flattened
// semantics of p.  Returns a single-assignment program of binary
// temporals; returned terms become the temporal, constant or zero that
// each original reduces to (Sec. 4.3, Sec. 4.4).
// max_temps >= 0 stops after that many temporals (the most frequent pairs
// come first, so a budget keeps the most valuable ones); definitions not yet
// reduced stay as n-ary statements.
Slp repair(const Slp& p, bool xor_cancel, int max_temps = -1);

// A complete (Xor)RePair run from which the program under any temporaries
// budget can be taken: each iteration adds one temporal, so budget b is the
// first b iterations of the run.
class RepairTrace {
 public:
  // max_temps >= 0 stops the run after that many temporals (the run is
  // deterministic, so this is a prefix of the complete run); complete()
  // says whether the run ended on its own.
  RepairTrace(const Slp& p, bool xor_cancel, int max_temps = -1);
  int n_temps() const { return static_cast<int>(tdef_.size()); }
  bool complete() const { return complete_; }
  Slp at(int b) const;   // program after b temporals (b >= n_temps: all)

 private:
  int nc_ = 0, n_orig_ = 0;
  std::vector<std::string> const_names_;
  std::vector<std::vector<int>> init_;                        // initial definitions
  std::vector<std::pair<int, int>> tdef_;                     // temporal i = (x, y)
  std::vector<std::vector<std::pair<int, std::vector<int>>>> changes_;  // per iteration
  bool complete_ = true;
};

// Triple compression: the RePair idea (Sec. 4.3) with triples of terms in
// place of pairs, for an executor whose XOR instruction takes three inputs
// (LOP3): a statement of n arguments costs ceil((n-1)/2) instructions, so a
// temporal t = a + b + c costs one instruction and removes one from every
// definition it replaces, where a pair temporal removes one argument
// (half an instruction on average).  Each iteration replaces the most
// frequent triple (ties: the smallest triple of term ids; terms are
// constants, then temporals in creation order) in every original that
// contains it, while some triple occurs at least twice.  Like RepairTrace,
// budget b is the first b iterations of one run.
class TripleTrace {
 public:
  explicit TripleTrace(const Slp& p);
  int n_temps() const { return static_cast<int>(tdef_.size()); }
  Slp at(int b) const;

 private:
  int nc_ = 0, n_orig_ = 0;
  std::vector<std::string> const_names_;
  std::vector<std::vector<int>> init_;        // initial definitions (sorted constants)
  std::vector<std::vector<int>> tdef_;        // temporal i = XOR of three terms
};

// Instructions of a fused program on a three-input XOR unit:
// sum over statements of ceil((arity - 1) / 2).
long lop3_count(const Slp& p);

// XOR fusion: repeatedly unfold variables used exactly once into their
// user; dead variables are dropped.  cancel_pairs removes arguments that
// occur twice in one fused statement (x + x = 0).  Requires single
// assignment (Sec. 5.2).
Slp fuse(const Slp& p, bool cancel_pairs);

// Pebble-game schedules of a single-assignment MultiSLP (Sec. 6.4, 6.6).
// goals_hold: goal nodes keep their pebble to the end (the paper's game);
// otherwise a goal's pebble is freed after its last use, which is the GPU
// setting where outputs stream to memory as soon as they are computed.
struct Schedule {
  struct Step {
    int node;                 // variable id in the input program
    int pebble;               // pebble (register or slot) receiving it
    std::vector<int> args;    // constants, or variable ids of the input
  };
  std::vector<Step> steps;
  int n_pebbles = 0;
};
Schedule schedule_dfs(const Slp& p, bool goals_hold);
Schedule schedule_greedy(const Slp& p, int cap, bool goals_hold);
// Registers a thread needs to run schedule s of q when every input word is
// loaded into a register first: inputs live until their last use, values
// from their statement until their last use (Sec. 6.2's cache capacity with
// the register file as the cache and no reloading).
int max_live_preloaded(const Slp& q, const Schedule& s);

// The schedule that computes p's statements in program order (p single
// assignment), pebbles assigned as in schedule_dfs.
Schedule schedule_in_order(const Slp& p, bool goals_hold);
// Registers a thread needs to run schedule s of q when an input word is
// loaded at its first use in each group (group[i] = group of step i) and kept
// until its last use in that group; *loads receives the number of input
// loads.  With one group this is the single-level game with inputs loaded on
// first use and never evicted.
int max_live_grouped(const Slp& q, const Schedule& s, const std::vector<int>& group,
                     long* loads);

// The program of a schedule, with variables renamed to pebbles.  Requires
// goals_hold schedules so that returned values are still on their pebble.
Slp schedule_to_slp(const Slp& p, const Schedule& s);

}  // namespace xorec
