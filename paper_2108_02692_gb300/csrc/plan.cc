#include "plan.h"

#include <algorithm>
#include <memory>

#include "gf.h"

namespace xorec {

std::vector<Bits> bitmatrix_rows(int rows, int cols, const uint8_t* A) {
  std::vector<Bits> R(static_cast<size_t>(8) * rows, Bits(8 * cols));
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j)
      for (int t = 0; t < 8; ++t) {
        const uint8_t c = gf_mul(A[static_cast<size_t>(i) * cols + j], static_cast<uint8_t>(1u << t));
        for (int s = 0; s < 8; ++s)
          if ((c >> s) & 1u) R[8 * i + s].set(8 * j + t);
      }
  return R;
}

namespace {

uint64_t fnv1a(uint64_t h, uint64_t v) {
  for (int i = 0; i < 8; ++i) {
    h ^= (v >> (8 * i)) & 0xff;
    h *= 0x100000001b3ull;
  }
  return h;
}

// Lower a GPU schedule of the fused program into the interpreter stream.
bool lower(const Slp& q, const Schedule& s, int n_in, int n_out, Program* p,
           std::string* err) {
  const int nc = q.n_const;
  std::vector<std::vector<int>> outs_of(q.n_var);
  std::vector<int> copy_rows, zero_rows;
  for (int r = 0; r < static_cast<int>(q.ret.size()); ++r) {
    const int t = q.ret[r];
    if (t < 0) zero_rows.push_back(r);
    else if (t < nc) copy_rows.push_back(r);
    else outs_of[t - nc].push_back(r);
  }
  std::vector<int> slot_of(q.n_var, -1);
  std::vector<uint16_t> code;
  int n_stmts = 0;
  auto emit = [&](const std::vector<int>& args, const std::vector<int>& outs, int slot) {
    if (args.size() > 0x7fff || outs.size() > 0x7fff) return false;
    code.push_back(static_cast<uint16_t>(args.size()));
    code.push_back(static_cast<uint16_t>(outs.size() | (slot >= 0 ? 0x8000u : 0u)));
    if (slot >= 0) code.push_back(static_cast<uint16_t>(slot));
    for (int o : outs) code.push_back(static_cast<uint16_t>(o));
    for (int a : args) code.push_back(static_cast<uint16_t>(a));
    ++n_stmts;
    return true;
  };
  for (const auto& st : s.steps) {
    std::vector<int> args;
    for (int a : st.args) {
      if (a < nc) {
        args.push_back(a);
      } else {
        const int sl = slot_of[a - nc];
        if (sl < 0) { *err = "schedule reads a value that holds no slot"; return false; }
        args.push_back(n_in + sl);
      }
    }
    slot_of[st.node] = st.pebble;
    if (!emit(args, outs_of[st.node], st.pebble)) { *err = "statement too large"; return false; }
  }
  for (int r : copy_rows)
    if (!emit({q.ret[r]}, {r}, -1)) return false;
  for (int r : zero_rows)
    if (!emit({}, {r}, -1)) return false;
  if (n_in + s.n_pebbles > 0xffff) { *err = "program too large"; return false; }
  p->code = code;
  p->n_in = n_in;
  p->n_out = n_out;
  p->n_slots = s.n_pebbles;
  p->n_stmts = n_stmts;
  uint64_t h = 0xcbf29ce484222325ull;
  h = fnv1a(h, static_cast<uint64_t>(n_in) << 32 | static_cast<uint32_t>(n_out));
  for (uint16_t w : code) h = fnv1a(h, w);
  p->hash = h;
  return true;
}

}  // namespace

std::vector<uint16_t> chunk_stream(const std::vector<uint16_t>& code) {
  std::vector<uint16_t> out;
  auto pad = [&]() {
    while (out.size() % 8) out.push_back(0xffff);
  };
  size_t pc = 0;
  while (pc < code.size()) {
    const uint16_t na = code[pc];
    const uint16_t w1 = code[pc + 1];
    pc += 2;
    const uint16_t no = w1 & 0x7fff;
    const uint16_t slot = (w1 & 0x8000) ? code[pc++] : 0xffff;
    const size_t outs = pc, args = pc + no;
    pc = args + na;
    out.push_back(na);
    out.push_back(no);
    out.push_back(slot);
    for (int q = 0; q < 5; ++q) out.push_back(q < no ? code[outs + q] : 0xffff);
    for (size_t a = 0; a < na; ++a) out.push_back(code[args + a]);
    pad();
    for (size_t q = 5; q < no; ++q) out.push_back(code[outs + q]);
    pad();
  }
  return out;
}

bool check_program_stream(const uint16_t* code, size_t len, int n_in, int n_out, int n_slots,
                          std::string* err) {
  std::vector<char> written(static_cast<size_t>(std::max(0, n_slots)), 0);
  size_t pc = 0;
  auto bad = [&](const char* what) {
    *err = std::string("instruction stream: ") + what + " at word " + std::to_string(pc);
    return false;
  };
  while (pc < len) {
    if (pc + 2 > len) return bad("truncated statement header");
    const int na = code[pc];
    const int w1 = code[pc + 1];
    const int no = w1 & 0x7fff;
    const bool has_slot = (w1 & 0x8000) != 0;
    size_t q = pc + 2;
    int slot = -1;
    if (has_slot) {
      if (q >= len) return bad("truncated slot");
      slot = code[q++];
      if (slot >= n_slots) return bad("slot out of range");
    }
    if (q + static_cast<size_t>(no) + static_cast<size_t>(na) > len) return bad("truncated statement");
    for (int o = 0; o < no; ++o)
      if (code[q + o] >= n_out) return bad("output strip out of range");
    q += no;
    for (int a = 0; a < na; ++a) {
      const int id = code[q + a];
      if (id >= n_in + n_slots) return bad("operand out of range");
      if (id >= n_in && !written[id - n_in]) return bad("slot read before it is written");
    }
    if (slot >= 0) written[slot] = 1;
    pc = q + na;
  }
  return true;
}

bool build_program(int rows, int cols, const uint8_t* A, const PlanOptions& o,
                   Program* out, std::string* err) {
  const int n_in = 8 * cols, n_out = 8 * rows;
  std::vector<Bits> R = bitmatrix_rows(rows, cols, A);
  std::vector<int> order;
  for (int i = 0; i < rows; ++i)
    for (int s = 7; s >= 0; --s) order.push_back(8 * i + s);
  Slp chains = slp_rows_chains(n_in, R, order);
  Program p;
  p.stats.raw = metrics(chains);
  // the dense executor's control words (plan.h): bit (r, c) of the
  // bitmatrix, by input strip and by output strip
  p.masks.assign(static_cast<size_t>((n_out + 31) / 32) * n_in, 0u);
  p.rowbits.assign(p.masks.size(), 0u);
  for (int r = 0; r < n_out; ++r)
    for (int c = 0; c < n_in; ++c)
      if (R[r].test(c)) {
        const size_t g = static_cast<size_t>(r / 32) * n_in;
        const int rr = r % 32;
        p.masks[g + c] |= 1u << rr;
        p.rowbits[g + 8 * (c / 8) + rr / 4] |= 1u << (8 * (rr % 4) + c % 8);
      }
  Slp fused;
  // Two-level program for wide codes (inputs do not fit the registers):
  // groups of partial sums as large as the register budget allows.
  bool two_level = false;
  Schedule stream_sched;
  if (n_in > kPreloadMaxInputs && o.stream_window >= 0 &&
      (o.opt_level == kOptRaw || o.max_temps == -2)) {
    const int window = o.stream_window > 0 ? o.stream_window : 32;
    // candidates: temporals per window x rows per group (halved from all
    // rows); each keeps the values live within reg_budget - 32 (addresses
    // and loop state need the rest), and the cheapest by three-input XORs
    // plus twice the shared-memory loads (the narrower pipe) wins
    // (the unoptimised level keeps every window uncompressed)
    std::vector<int> temps_c;
    if (o.opt_level == kOptRaw || o.stream_temps < 0) temps_c = {0};
    else if (o.stream_temps > 0) temps_c = {o.stream_temps};
    else temps_c = {0, 8, 16, 32};
    long best_cost = -1;
    for (int wt : temps_c) {
      for (int rows_per_group = n_out;; rows_per_group = (rows_per_group + 1) / 2) {
        std::vector<int> group;
        long loads = 0;
        Slp st = slp_rows_stream(n_in, R, window, rows_per_group, &group, wt,
                                 o.opt_level != kOptRePair);
        Schedule sc = schedule_in_order(st, false);
        const int live = max_live_grouped(st, sc, group, &loads);
        if (live + 32 <= o.reg_budget || rows_per_group <= 8) {
          const long cost = lop3_count(st) + 2 * loads;
          if (metrics(st).mem <= kMaxCompiledMemOps && (best_cost < 0 || cost < best_cost)) {
            best_cost = cost;
            two_level = true;
            fused = std::move(st);
            stream_sched = std::move(sc);
            p.load_group = std::move(group);
            p.stats.max_live = live;
            p.stats.loads = loads;
            p.stats.window = window;
            p.stats.window_temps = wt;
          }
          break;
        }
      }
    }
  }
  if (two_level) {
    p.stats.compressed = p.stats.raw;
  } else if (o.opt_level == kOptRaw) {
    fused = slp_rows_fused(n_in, R, order);
    p.stats.compressed = p.stats.raw;
  } else if (o.max_temps == -2 && n_in >= o.reg_budget) {
    // the inputs alone exceed the register budget: no temporaries
    fused = slp_rows_fused(n_in, R, order);
    p.stats.compressed = p.stats.raw;
  } else {
    // compression trace: (Xor)RePair pairs, or triples when enumerating the
    // rows' triples stays small
    long triples = 0;
    for (const auto& r : R) {
      const long n = r.count();
      triples += n * (n - 1) * (n - 2) / 6;
    }
    const bool use_triples = o.opt_level == kOptTriple && triples <= 8000000;
    std::unique_ptr<RepairTrace> rt;
    std::unique_ptr<TripleTrace> tt;
    if (use_triples) {
      tt = std::make_unique<TripleTrace>(chains);
    } else {
      // With the automatic budget only the first temporals can fit the
      // register budget: run a prefix of reg_budget temporals first (the run
      // is deterministic, so it is the complete run's prefix) and the
      // complete run only if every temporal of the prefix fits.
      const bool xc = o.opt_level != kOptRePair;
      const int cap = o.max_temps == -2 ? o.reg_budget : (o.max_temps >= 0 ? o.max_temps : -1);
      rt = std::make_unique<RepairTrace>(chains, xc, cap);
      if (!rt->complete() && o.max_temps == -2) {
        Slp f = fuse(rt->at(rt->n_temps()), o.cancel_pairs);
        if (max_live_preloaded(f, schedule_dfs(f, false)) <= o.reg_budget)
          rt = std::make_unique<RepairTrace>(chains, xc);
      }
    }
    auto at = [&](int x) { return use_triples ? tt->at(x) : rt->at(x); };
    int b = use_triples ? tt->n_temps() : rt->n_temps();
    const int all = b;
    if (o.max_temps >= 0) {
      b = std::min(o.max_temps, all);
    } else if (o.max_temps == -2) {
      // largest budget whose DFS schedule fits the register budget
      auto live_at = [&](int x) {
        Slp f = fuse(at(x), o.cancel_pairs);
        return max_live_preloaded(f, schedule_dfs(f, false));
      };
      if (live_at(b) > o.reg_budget) {
        int lo = 0, hi = b;   // live_at(lo) assumed to fit, live_at(hi) does not
        while (hi - lo > 1) {
          const int mid = (lo + hi) / 2;
          if (live_at(mid) <= o.reg_budget) lo = mid; else hi = mid;
        }
        b = lo;
      }
    }
    Slp co = at(b);
    p.stats.temps = b;
    p.stats.compressed = metrics(co);
    fused = fuse(co, o.cancel_pairs);
  }
  p.stats.fused = metrics(fused);
  p.stats.lop3 = lop3_count(fused);
  if (!equivalent(chains, fused)) {
    *err = "internal: optimised program is not equivalent to the bitmatrix";
    return false;
  }
  Schedule gpu;
  if (two_level) {
    // the statements are already in the order of the two-level game
    p.stats.sched_nvar = schedule_in_order(fused, true).n_pebbles;
    gpu = std::move(stream_sched);
  } else {
    Schedule paper = o.sched == kSchedGreedy ? schedule_greedy(fused, o.greedy_cap, true)
                                             : schedule_dfs(fused, true);
    p.stats.sched_nvar = paper.n_pebbles;
    gpu = o.sched == kSchedGreedy ? schedule_greedy(fused, o.greedy_cap, false)
                                  : schedule_dfs(fused, false);
    p.stats.max_live = max_live_preloaded(fused, gpu);
    // inputs preloaded once, or (wide programs) read at every use
    if (n_in <= kPreloadMaxInputs) {
      p.stats.loads = n_in;
    } else {
      for (const auto& st : fused.body)
        for (int a : st.args) p.stats.loads += a < n_in;
    }
  }
  p.stats.slots = gpu.n_pebbles;
  if (!lower(fused, gpu, n_in, n_out, &p, err)) return false;
  if (!check_program_stream(p.code.data(), p.code.size(), n_in, n_out, p.n_slots, err))
    return false;
  p.chunks = chunk_stream(p.code);
  p.interp_slots = p.n_slots;
  if (!two_level && n_in <= kPreloadMaxInputs && p.n_slots > 0) {
    // The interpreter keeps every input strip and every slot of its tile in
    // shared memory, so slots cost it resident warps: it runs the
    // unoptimised fused program instead (one statement per output strip, no
    // slots), the paper's P^{+F}; more XORs, twice the resident warps.
    Slp plain = slp_rows_fused(n_in, R, order);
    Program ip;
    if (!lower(plain, schedule_dfs(plain, false), n_in, n_out, &ip, err)) return false;
    if (!check_program_stream(ip.code.data(), ip.code.size(), n_in, n_out, ip.n_slots, err))
      return false;
    p.chunks = chunk_stream(ip.code);
    p.interp_slots = ip.n_slots;
  }
  p.fused = fused;
  p.sched = gpu;
  *out = std::move(p);
  return true;
}

}  // namespace xorec
