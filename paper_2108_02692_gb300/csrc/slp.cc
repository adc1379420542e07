#include "slp.h"

#include <algorithm>
#include <functional>
#include <list>
#include <map>
#include <queue>
#include <sstream>
#include <unordered_map>

namespace xorec {

// ------------------------------------------------------------------ Bits

int Bits::count() const {
  int c = 0;
  for (uint64_t x : w) c += __builtin_popcountll(x);
  return c;
}
int Bits::xor_count(const Bits& o) const {
  int c = 0;
  for (size_t i = 0; i < w.size(); ++i) c += __builtin_popcountll(w[i] ^ o.w[i]);
  return c;
}
int Bits::and_count(const Bits& o) const {
  int c = 0;
  for (size_t i = 0; i < w.size(); ++i) c += __builtin_popcountll(w[i] & o.w[i]);
  return c;
}
Bits& Bits::operator^=(const Bits& o) {
  for (size_t i = 0; i < w.size(); ++i) w[i] ^= o.w[i];
  return *this;
}
bool Bits::any() const {
  for (uint64_t x : w)
    if (x) return true;
  return false;
}

// ------------------------------------------------------ semantics, metrics

std::vector<Bits> semantics(const Slp& p) {
  std::vector<Bits> val(p.n_var, Bits(p.n_const));
  auto value_of = [&](int t) {
    if (p.is_const(t)) {
      Bits b(p.n_const);
      b.set(t);
      return b;
    }
    return val[t - p.n_const];
  };
  for (const Stmt& s : p.body) {
    Bits acc(p.n_const);
    for (int a : s.args) acc ^= value_of(a);
    val[s.dst - p.n_const] = acc;
  }
  std::vector<Bits> out;
  out.reserve(p.ret.size());
  for (int r : p.ret) out.push_back(r < 0 ? Bits(p.n_const) : value_of(r));
  return out;
}

bool equivalent(const Slp& a, const Slp& b) {
  if (a.n_const != b.n_const) return false;
  return semantics(a) == semantics(b);
}

SlpMetrics metrics(const Slp& p) {
  SlpMetrics m{0, 0, 0, 0};
  std::vector<char> seen(p.n_var, 0);
  for (const Stmt& s : p.body) {
    const long n = static_cast<long>(s.args.size());
    m.xors += n > 0 ? n - 1 : 0;
    m.mem += n + 1;
    m.stmts += 1;
    if (!seen[s.dst - p.n_const]) {
      seen[s.dst - p.n_const] = 1;
      m.nvar += 1;
    }
  }
  return m;
}

// ------------------------------------------------------------- LRU cache

namespace {

struct Lru {
  int cap;
  std::list<int> order;  // front = least recently used
  std::unordered_map<int, std::list<int>::iterator> pos;
  std::vector<char> evicted;
  long io = 0, reloads = 0;
  Lru(int c, int universe) : cap(c), evicted(universe, 0) {}
  bool has(int x) const { return pos.count(x) != 0; }
  void touch(int x) {
    order.erase(pos[x]);
    order.push_back(x);
    pos[x] = std::prev(order.end());
  }
  void make_room() {
    if (static_cast<int>(order.size()) >= cap && !order.empty()) {
      const int v = order.front();
      order.pop_front();
      pos.erase(v);
      evicted[v] = 1;
      ++io;
    }
  }
  void insert(int x) {
    order.push_back(x);
    pos[x] = std::prev(order.end());
  }
  // Argument access: load on miss.
  void use(int x) {
    if (has(x)) {
      touch(x);
      return;
    }
    make_room();
    ++io;
    if (evicted[x]) ++reloads;
    insert(x);
  }
  // Destination: allocate on miss (no transfer), else update position.
  void def(int x) {
    if (has(x)) {
      touch(x);
      return;
    }
    make_room();
    insert(x);
  }
};

}  // namespace

long lru_iocost(const Slp& p, int cap, long* reloads) {
  Lru c(cap, p.n_const + p.n_var);
  for (const Stmt& s : p.body) {
    for (int a : s.args) c.use(a);
    c.def(s.dst);
  }
  if (reloads) *reloads = c.reloads;
  return c.io;
}

int ccap(const Slp& p) {
  const int hi = p.n_const + p.n_var + 1;
  for (int cap = 1; cap <= hi; ++cap) {
    long rel = 0;
    lru_iocost(p, cap, &rel);
    if (rel == 0) return cap;
  }
  return hi;
}

// --------------------------------------------------------------- text I/O

bool parse_slp(const std::string& text, Slp* out, std::string* err) {
  Slp p;
  std::map<std::string, int> cid, vid;
  std::vector<std::pair<std::string, std::vector<std::string>>> stmts;
  std::vector<std::string> ret;
  std::istringstream in(text);
  std::string line;
  while (std::getline(in, line)) {
    for (char& ch : line)
      if (ch == ';' || ch == ',' || ch == '(' || ch == ')' || ch == '^' || ch == '+') ch = ' ';
    std::istringstream ls(line);
    std::vector<std::string> tok;
    std::string t;
    while (ls >> t) tok.push_back(t);
    if (tok.empty() || tok[0][0] == '#') continue;
    if (tok[0] == "const") {
      for (size_t i = 1; i < tok.size(); ++i) {
        if (cid.count(tok[i])) { *err = "duplicate constant " + tok[i]; return false; }
        const int id = static_cast<int>(cid.size());
        cid[tok[i]] = id;
        p.const_names.push_back(tok[i]);
      }
    } else if (tok[0] == "ret") {
      ret.assign(tok.begin() + 1, tok.end());
    } else {
      if (tok.size() < 2 || (tok[1] != "=" && tok[1] != "<-")) {
        *err = "bad statement: " + line;
        return false;
      }
      std::vector<std::string> args(tok.begin() + 2, tok.end());
      if (!args.empty() && args[0] == "xor") args.erase(args.begin());
      stmts.emplace_back(tok[0], args);
    }
  }
  p.n_const = static_cast<int>(cid.size());
  for (auto& st : stmts) {
    if (cid.count(st.first)) { *err = "assignment to constant " + st.first; return false; }
    if (!vid.count(st.first)) {
      const int id = static_cast<int>(vid.size());
      vid[st.first] = id;
      p.var_names.push_back(st.first);
    }
  }
  p.n_var = static_cast<int>(vid.size());
  auto term = [&](const std::string& s, int* t) {
    if (cid.count(s)) { *t = cid[s]; return true; }
    if (vid.count(s)) { *t = p.n_const + vid[s]; return true; }
    if (s == "0") { *t = -1; return true; }
    *err = "unknown name " + s;
    return false;
  };
  for (auto& st : stmts) {
    Stmt s;
    s.dst = p.n_const + vid[st.first];
    for (auto& a : st.second) {
      int t;
      if (!term(a, &t) || t < 0) { if (err->empty()) *err = "bad argument"; return false; }
      s.args.push_back(t);
    }
    p.body.push_back(s);
  }
  for (auto& r : ret) {
    int t;
    if (!term(r, &t)) return false;
    p.ret.push_back(t);
  }
  *out = p;
  return true;
}

std::string slp_to_text(const Slp& p) {
  auto name = [&](int t) -> std::string {
    if (t < 0) return "0";
    if (p.is_const(t))
      return t < static_cast<int>(p.const_names.size()) ? p.const_names[t] : "c" + std::to_string(t);
    const int v = t - p.n_const;
    return v < static_cast<int>(p.var_names.size()) ? p.var_names[v] : "v" + std::to_string(v);
  };
  std::ostringstream os;
  os << "const";
  for (int c = 0; c < p.n_const; ++c) os << ' ' << name(c);
  os << '\n';
  for (const Stmt& s : p.body) {
    os << name(s.dst) << " =";
    for (int a : s.args) os << ' ' << name(a);
    os << '\n';
  }
  os << "ret";
  for (int r : p.ret) os << ' ' << name(r);
  os << '\n';
  return os.str();
}

// ------------------------------------------------------- raw programs

Slp slp_rows_fused(int n_const, const std::vector<Bits>& rows,
                   const std::vector<int>& row_order) {
  Slp p;
  p.n_const = n_const;
  p.n_var = static_cast<int>(rows.size());
  p.ret.assign(rows.size(), -1);
  for (int r : row_order) {
    Stmt s;
    s.dst = n_const + r;
    for (int c = 0; c < n_const; ++c)
      if (rows[r].test(c)) s.args.push_back(c);
    if (s.args.empty()) continue;      // zero row: returns the zero array
    p.ret[r] = s.dst;
    p.body.push_back(s);
  }
  return p;
}

Slp slp_rows_chains(int n_const, const std::vector<Bits>& rows,
                    const std::vector<int>& row_order) {
  Slp p;
  p.n_const = n_const;
  p.n_var = static_cast<int>(rows.size());
  p.ret.assign(rows.size(), -1);
  for (int r : row_order) {
    std::vector<int> cols;
    for (int c = 0; c < n_const; ++c)
      if (rows[r].test(c)) cols.push_back(c);
    if (cols.empty()) continue;
    const int v = n_const + r;
    p.ret[r] = v;
    if (cols.size() == 1) {
      p.body.push_back(Stmt{v, {cols[0]}});
      continue;
    }
    p.body.push_back(Stmt{v, {cols[0], cols[1]}});
    for (size_t i = 2; i < cols.size(); ++i) p.body.push_back(Stmt{v, {v, cols[i]}});
  }
  return p;
}

Slp slp_rows_stream(int n_const, const std::vector<Bits>& rows, int window, int group_rows,
                    std::vector<int>* stmt_group, int window_temps, bool xor_cancel) {
  Slp p;
  p.n_const = n_const;
  const int n_rows = static_cast<int>(rows.size());
  p.ret.assign(n_rows, -1);
  stmt_group->clear();
  if (window < 1) window = 1;
  if (group_rows < 1) group_rows = 1;
  std::vector<int> acc(n_rows, -1);   // current partial sum of each row
  auto add = [&](int g, std::vector<int> args) {
    const int v = n_const + p.n_var++;
    p.body.push_back(Stmt{v, std::move(args)});
    stmt_group->push_back(g);
    return v;
  };
  // acc <- acc + XOR(args) as a chain of three-input statements; a row's
  // first statement (acc < 0) takes up to three arguments
  auto chain = [&](int g, const std::vector<int>& args, int start) {
    size_t i = 0;
    int cur = start;
    if (cur < 0) {
      const size_t n = std::min<size_t>(3, args.size());
      cur = add(g, std::vector<int>(args.begin(), args.begin() + n));
      i = n;
    }
    for (; i < args.size(); i += 2) {
      std::vector<int> a{cur, args[i]};
      if (i + 1 < args.size()) a.push_back(args[i + 1]);
      cur = add(g, a);
    }
    return cur;
  };
  for (int g = 0, r0 = 0; r0 < n_rows; ++g, r0 += group_rows) {
    const int r1 = std::min(n_rows, r0 + group_rows);
    for (int c0 = 0; c0 < n_const; c0 += window) {
      const int c1 = std::min(n_const, c0 + window);
      if (window_temps > 0) {
        // the group's rows restricted to the window form a small MultiSLP;
        // XorRePair (at most window_temps temporals) and fusion shorten it
        const int wn = c1 - c0;
        std::vector<int> rid;
        std::vector<Bits> sub;
        for (int r = r0; r < r1; ++r) {
          Bits b(wn);
          bool any = false;
          for (int c = c0; c < c1; ++c)
            if (rows[r].test(c)) {
              b.set(c - c0);
              any = true;
            }
          if (any) {
            rid.push_back(r);
            sub.push_back(b);
          }
        }
        if (rid.empty()) continue;
        std::vector<int> ord(rid.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = static_cast<int>(i);
        RepairTrace rt(slp_rows_chains(wn, sub, ord), xor_cancel, window_temps);
        const Slp f = fuse(rt.at(rt.n_temps()), true);
        std::vector<int> val(f.n_var, -1), users(f.n_var, 0), n_goal(f.n_var, 0),
            goal_row(f.n_var, -1);
        for (const Stmt& st : f.body)
          for (int a : st.args)
            if (a >= wn) users[a - wn] += 1;
        for (size_t i = 0; i < f.ret.size(); ++i)
          if (f.ret[i] >= wn) {
            n_goal[f.ret[i] - wn] += 1;
            goal_row[f.ret[i] - wn] = rid[i];
          }
        auto folded = [&](int v) { return n_goal[v] == 1 && users[v] == 0; };
        for (const Stmt& st : f.body) {
          const int v = st.dst - wn;
          std::vector<int> args;
          for (int a : st.args) args.push_back(a < wn ? c0 + a : val[a - wn]);
          if (folded(v)) {
            // one row's part with no other use: straight into its partial sum
            const int r = goal_row[v];
            acc[r] = chain(g, args, acc[r]);
          } else {
            val[v] = chain(g, args, -1);
          }
        }
        for (size_t i = 0; i < f.ret.size(); ++i) {
          const int t = f.ret[i], r = rid[i];
          if (t < 0 || (t >= wn && folded(t - wn))) continue;
          const int term = t < wn ? c0 + t : val[t - wn];
          acc[r] = acc[r] < 0 && t >= wn ? term : chain(g, {term}, acc[r]);
        }
        continue;
      }
      for (int r = r0; r < r1; ++r) {
        std::vector<int> cs;
        for (int c = c0; c < c1; ++c)
          if (rows[r].test(c)) cs.push_back(c);
        size_t i = 0;
        if (acc[r] < 0 && !cs.empty()) {
          // the first statement of a row takes up to three inputs
          const size_t n = std::min<size_t>(3, cs.size());
          acc[r] = add(g, std::vector<int>(cs.begin(), cs.begin() + n));
          i = n;
        }
        for (; i < cs.size(); i += 2) {
          std::vector<int> args{acc[r], cs[i]};
          if (i + 1 < cs.size()) args.push_back(cs[i + 1]);
          acc[r] = add(g, args);
        }
      }
    }
  }
  for (int r = 0; r < n_rows; ++r) p.ret[r] = acc[r];
  return p;
}

// --------------------------------------------------- RePair / XorRePair

namespace {

// Term order (Sec. 4.3): temporals in generation order precede constants;
// constants are in index order.  Term ids: constant c -> c, temporal i ->
// n_const + i.
struct Ranker {
  int nc;
  long rank(int t) const { return t < nc ? (1L << 40) + t : static_cast<long>(t - nc); }
};

}  // namespace

// One run of (Xor)RePair to completion.  Every iteration adds exactly one
// temporal, so the program after b temporals (a budget) is a prefix of this
// run; the run records the definition changes of every iteration so that
// any prefix can be rebuilt without running the algorithm again.
RepairTrace::RepairTrace(const Slp& in, bool xor_cancel, int max_temps)
    : nc_(in.n_const), const_names_(in.const_names) {
  const int nc = nc_;
  const Ranker rk{nc};
  const std::vector<Bits> goal = semantics(in);
  n_orig_ = static_cast<int>(goal.size());
  const int n_orig = n_orig_;

  std::vector<std::vector<int>> def(n_orig);
  std::vector<char> active(n_orig, 0);
  for (int o = 0; o < n_orig; ++o) {
    for (int c = 0; c < nc; ++c)
      if (goal[o].test(c)) def[o].push_back(c);
    active[o] = def[o].size() >= 2;
  }
  init_ = def;
  std::vector<Bits> tval;
  std::vector<Bits> occ;  // term -> active originals containing it
  auto ensure_occ = [&](int t) {
    if (static_cast<int>(occ.size()) <= t) occ.resize(t + 1, Bits(n_orig));
  };
  auto value_of = [&](int t) {
    if (t < nc) {
      Bits b(nc);
      b.set(t);
      return b;
    }
    return tval[t - nc];
  };
  auto sort_def = [&](std::vector<int>& d) {
    std::sort(d.begin(), d.end(), [&](int x, int y) { return rk.rank(x) < rk.rank(y); });
  };
  auto attach = [&](int o) {
    for (int t : def[o]) { ensure_occ(t); occ[t].set(o); }
  };
  auto detach = [&](int o) {
    for (int t : def[o]) { ensure_occ(t); if (occ[t].test(o)) occ[t].flip(o); }
  };
  for (int o = 0; o < n_orig; ++o)
    if (active[o]) attach(o);

  // Rebuild(v) (Sec. 4.4): greedily XOR existing temporals into
  // rem = [[v]] while that strictly shrinks rem; ties go to the earliest
  // temporal.  The greedy path of every original is cached: a temporal
  // created later changes the path only at the first step where it is
  // strictly better than the choice made there, so the path is recomputed
  // from that step on, which gives the same result as starting over.
  struct Path {
    std::vector<int> pick;   // temporal chosen at each step
    std::vector<Bits> rem;   // rem before each step; back() = final rem
  };
  std::vector<Path> path(n_orig);
  for (int o = 0; o < n_orig; ++o) path[o].rem.push_back(goal[o]);
  auto extend = [&](Path& P, size_t k) {
    P.pick.resize(k);
    P.rem.resize(k + 1);
    Bits rem = P.rem[k];
    int size = rem.count();
    for (;;) {
      int best = -1, best_size = size;
      for (size_t t = 0; t < tval.size(); ++t) {
        const int sz = rem.xor_count(tval[t]);
        if (sz < best_size) { best_size = sz; best = static_cast<int>(t); }
      }
      if (best < 0) break;
      rem ^= tval[best];
      size = best_size;
      P.pick.push_back(best);
      P.rem.push_back(rem);
    }
  };
  auto note_new_temporal = [&](Path& P, int t) {
    for (size_t k = 0; k < P.rem.size(); ++k) {
      const int cand = P.rem[k].xor_count(tval[t]);
      const int cur = k < P.pick.size() ? P.rem[k + 1].count() : P.rem[k].count();
      if (cand < cur) {
        extend(P, k);
        return;
      }
    }
  };
  auto rebuilt_def = [&](const Path& P) {
    std::vector<char> in_s(tval.size(), 0);
    for (int t : P.pick) in_s[t] ^= 1;
    std::vector<int> d;
    for (size_t t = 0; t < in_s.size(); ++t)
      if (in_s[t]) d.push_back(nc + static_cast<int>(t));
    for (int c = 0; c < nc; ++c)
      if (P.rem.back().test(c)) d.push_back(c);
    sort_def(d);
    return d;
  };

  for (;;) {
    bool any = false;
    for (int o = 0; o < n_orig; ++o) any |= active[o] != 0;
    if (!any) break;
    if (max_temps >= 0 && static_cast<int>(tdef_.size()) >= max_temps) {
      complete_ = false;
      break;
    }
    // Terms present in active definitions, in term order.
    std::vector<int> present;
    for (int t = 0; t < static_cast<int>(occ.size()); ++t)
      if (occ[t].any()) present.push_back(t);
    std::sort(present.begin(), present.end(),
              [&](int x, int y) { return rk.rank(x) < rk.rank(y); });
    // Most frequent pair; the first maximum in lexicographic order wins.
    int bx = -1, by = -1, bf = 0;
    for (size_t i = 0; i < present.size(); ++i)
      for (size_t j = i + 1; j < present.size(); ++j) {
        const int f = occ[present[i]].and_count(occ[present[j]]);
        if (f > bf) { bf = f; bx = present[i]; by = present[j]; }
      }
    if (bx < 0) break;  // cannot happen: an active definition has >= 2 terms
    // Pair(bx, by)
    std::vector<std::pair<int, std::vector<int>>> changes;
    const int t = nc + static_cast<int>(tdef_.size());
    tdef_.emplace_back(bx, by);
    Bits v = value_of(bx);
    v ^= value_of(by);
    tval.push_back(v);
    ensure_occ(t);
    Bits both = occ[bx];
    for (size_t i = 0; i < both.w.size(); ++i) both.w[i] &= occ[by].w[i];
    for (int o = 0; o < n_orig; ++o) {
      if (!both.test(o)) continue;
      detach(o);
      std::vector<int> nd;
      for (int x : def[o])
        if (x != bx && x != by) nd.push_back(x);
      nd.push_back(t);
      sort_def(nd);
      def[o] = nd;
      active[o] = def[o].size() >= 2;
      if (active[o]) attach(o);
      changes.emplace_back(o, nd);
    }
    if (xor_cancel) {
      for (int o = 0; o < n_orig; ++o) {
        if (!active[o]) continue;
        note_new_temporal(path[o], t - nc);
        std::vector<int> nd = rebuilt_def(path[o]);
        if (nd.size() < def[o].size()) {
          detach(o);
          def[o] = nd;
          active[o] = def[o].size() >= 2;
          if (active[o]) attach(o);
          changes.emplace_back(o, nd);
        }
      }
    }
    changes_.push_back(std::move(changes));
  }
}

Slp RepairTrace::at(int b) const {
  const int nc = nc_;
  const int T = std::max(0, std::min(b, n_temps()));
  std::vector<std::vector<int>> def = init_;
  for (int i = 0; i < T; ++i)
    for (const auto& ch : changes_[i]) def[ch.first] = ch.second;
  Slp out;
  out.n_const = nc;
  out.const_names = const_names_;
  out.n_var = T;
  for (int i = 0; i < T; ++i) {
    out.body.push_back(Stmt{nc + i, {tdef_[i].first, tdef_[i].second}});
    out.var_names.push_back("t" + std::to_string(i + 1));
  }
  out.ret.resize(n_orig_);
  for (int o = 0; o < n_orig_; ++o) {
    if (def[o].size() <= 1) {
      out.ret[o] = def[o].empty() ? -1 : def[o][0];
      continue;
    }
    // budget reached: the remaining definition becomes one n-ary statement
    const int v = nc + out.n_var++;
    out.var_names.push_back("o" + std::to_string(o));
    out.body.push_back(Stmt{v, def[o]});
    out.ret[o] = v;
  }
  return out;
}

// ------------------------------------------------------ triple compression

namespace {

// Triple key of terms x < y < z (each below 2^21).
uint64_t triple_key(int x, int y, int z) {
  return (static_cast<uint64_t>(x) << 42) | (static_cast<uint64_t>(y) << 21) |
         static_cast<uint64_t>(z);
}

}  // namespace

TripleTrace::TripleTrace(const Slp& in) : nc_(in.n_const), const_names_(in.const_names) {
  const int nc = nc_;
  const std::vector<Bits> goal = semantics(in);
  n_orig_ = static_cast<int>(goal.size());
  std::vector<std::vector<int>> def(n_orig_);
  for (int o = 0; o < n_orig_; ++o)
    for (int c = 0; c < nc; ++c)
      if (goal[o].test(c)) def[o].push_back(c);
  init_ = def;

  // count[key] = originals containing the triple; a lazy max-heap of
  // (count, -key) finds the most frequent (stale entries are skipped)
  std::unordered_map<uint64_t, int> count;
  std::priority_queue<std::pair<int, int64_t>> heap;
  auto bump = [&](int x, int y, int z, int d) {
    const uint64_t k = triple_key(x, y, z);
    int& c = count[k];
    c += d;
    if (d > 0 && c >= 2) heap.emplace(c, -static_cast<int64_t>(k));
  };
  // the triples of sorted row r that contain its term t
  auto touch = [&](const std::vector<int>& r, int t, int d) {
    const int n = static_cast<int>(r.size());
    for (int i = 0; i < n; ++i) {
      if (r[i] == t) continue;
      for (int j = i + 1; j < n; ++j) {
        if (r[j] == t) continue;
        int v[3] = {r[i], r[j], t};
        std::sort(v, v + 3);
        bump(v[0], v[1], v[2], d);
      }
    }
  };
  for (const auto& r : def) {
    const int n = static_cast<int>(r.size());
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        for (int k = j + 1; k < n; ++k) bump(r[i], r[j], r[k], 1);
  }
  for (;;) {
    int best = 0;
    uint64_t key = 0;
    while (!heap.empty()) {
      const auto top = heap.top();
      const uint64_t k = static_cast<uint64_t>(-top.second);
      auto it = count.find(k);
      if (it == count.end() || it->second != top.first) {
        heap.pop();
        continue;
      }
      best = top.first;
      key = k;
      break;
    }
    if (best < 2) break;
    const int x = static_cast<int>(key >> 42), y = static_cast<int>((key >> 21) & 0x1fffff),
              z = static_cast<int>(key & 0x1fffff);
    const int t = nc + static_cast<int>(tdef_.size());
    if (t >= (1 << 21)) break;   // term ids must fit the key
    tdef_.push_back({x, y, z});
    for (auto& r : def) {
      if (!std::binary_search(r.begin(), r.end(), x) || !std::binary_search(r.begin(), r.end(), y) ||
          !std::binary_search(r.begin(), r.end(), z))
        continue;
      // drop the triples through x, y or z (each once), then the three terms
      std::vector<int> rest;
      for (int v : r)
        if (v != x && v != y && v != z) rest.push_back(v);
      touch(r, x, -1);
      {
        std::vector<int> r2;
        for (int v : r)
          if (v != x) r2.push_back(v);
        touch(r2, y, -1);
        std::vector<int> r3;
        for (int v : r2)
          if (v != y) r3.push_back(v);
        touch(r3, z, -1);
      }
      // add the temporal (it is larger than every term so far)
      rest.push_back(t);
      touch(rest, t, 1);
      r.swap(rest);
    }
  }
}

Slp TripleTrace::at(int b) const {
  const int nc = nc_;
  const int T = std::max(0, std::min(b, n_temps()));
  std::vector<std::vector<int>> def = init_;
  for (int i = 0; i < T; ++i) {
    const auto& td = tdef_[i];
    for (auto& r : def) {
      if (!std::binary_search(r.begin(), r.end(), td[0]) ||
          !std::binary_search(r.begin(), r.end(), td[1]) ||
          !std::binary_search(r.begin(), r.end(), td[2]))
        continue;
      std::vector<int> rest;
      for (int v : r)
        if (v != td[0] && v != td[1] && v != td[2]) rest.push_back(v);
      rest.push_back(nc + i);
      r.swap(rest);
    }
  }
  Slp out;
  out.n_const = nc;
  out.const_names = const_names_;
  out.n_var = T;
  for (int i = 0; i < T; ++i) {
    out.body.push_back(Stmt{nc + i, tdef_[i]});
    out.var_names.push_back("t" + std::to_string(i + 1));
  }
  out.ret.resize(n_orig_);
  for (int o = 0; o < n_orig_; ++o) {
    if (def[o].size() <= 1) {
      out.ret[o] = def[o].empty() ? -1 : def[o][0];
      continue;
    }
    const int v = nc + out.n_var++;
    out.var_names.push_back("o" + std::to_string(o));
    out.body.push_back(Stmt{v, def[o]});
    out.ret[o] = v;
  }
  return out;
}

long lop3_count(const Slp& p) {
  long n = 0;
  for (const auto& s : p.body)
    if (s.args.size() >= 2) n += static_cast<long>(s.args.size()) / 2;
  return n;
}

Slp repair(const Slp& in, bool xor_cancel, int max_temps) {
  RepairTrace tr(in, xor_cancel);
  return tr.at(max_temps < 0 ? tr.n_temps() : max_temps);
}

// ------------------------------------------------------------ XOR fusion

Slp fuse(const Slp& p, bool cancel_pairs) {
  const int nc = p.n_const;
  std::vector<int> def_idx(p.n_var, -1);
  for (size_t i = 0; i < p.body.size(); ++i) def_idx[p.body[i].dst - nc] = static_cast<int>(i);
  // Live variables: reachable from the returned terms.
  std::vector<char> live(p.n_var, 0), in_ret(p.n_var, 0);
  std::vector<int> stack;
  for (int r : p.ret)
    if (r >= nc) {
      in_ret[r - nc] = 1;
      if (!live[r - nc]) { live[r - nc] = 1; stack.push_back(r - nc); }
    }
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    for (int a : p.body[def_idx[v]].args)
      if (a >= nc && !live[a - nc]) { live[a - nc] = 1; stack.push_back(a - nc); }
  }
  std::vector<int> uses(p.n_var, 0);
  for (const Stmt& s : p.body)
    if (live[s.dst - nc])
      for (int a : s.args)
        if (a >= nc) uses[a - nc] += 1;
  for (int r : p.ret)
    if (r >= nc) uses[r - nc] += 1;
  std::vector<char> keep(p.n_var, 0);
  for (int v = 0; v < p.n_var; ++v) keep[v] = live[v] && (uses[v] != 1 || in_ret[v]);

  std::function<void(int, std::vector<int>&)> expand = [&](int t, std::vector<int>& out) {
    if (t < nc || keep[t - nc]) { out.push_back(t); return; }
    for (int a : p.body[def_idx[t - nc]].args) expand(a, out);
  };
  Slp q;
  q.n_const = nc;
  q.n_var = p.n_var;
  q.const_names = p.const_names;
  q.var_names = p.var_names;
  q.ret = p.ret;
  for (const Stmt& s : p.body) {
    if (!keep[s.dst - nc]) continue;
    std::vector<int> args;
    for (int a : s.args) expand(a, args);
    if (cancel_pairs) {
      std::unordered_map<int, int> cnt;
      for (int a : args) cnt[a] += 1;
      std::vector<int> kept;
      for (int a : args) {
        auto it = cnt.find(a);
        if (it != cnt.end() && (it->second & 1)) kept.push_back(a);
        if (it != cnt.end()) cnt.erase(it);
      }
      args.swap(kept);
    }
    q.body.push_back(Stmt{s.dst, args});
  }
  return q;
}

// ------------------------------------------------------- pebble schedules

namespace {

struct Graph {
  int nc = 0;
  int nv = 0;
  std::vector<int> def_idx;              // var -> statement
  std::vector<std::vector<int>> kids;    // var -> ordered children (terms)
  std::vector<int> n_parents;            // distinct parent statements
  std::vector<char> goal;
};

Graph build_graph(const Slp& p) {
  Graph g;
  g.nc = p.n_const;
  g.nv = p.n_var;
  g.def_idx.assign(p.n_var, -1);
  g.kids.assign(p.n_var, {});
  g.n_parents.assign(p.n_var, 0);
  g.goal.assign(p.n_var, 0);
  for (size_t i = 0; i < p.body.size(); ++i) {
    const int v = p.body[i].dst - p.n_const;
    g.def_idx[v] = static_cast<int>(i);
    std::vector<int> k = p.body[i].args;
    // children in term order: variables (generation order) then constants
    std::stable_sort(k.begin(), k.end(), [&](int a, int b) {
      const bool va = a >= p.n_const, vb = b >= p.n_const;
      if (va != vb) return va;
      return a < b;
    });
    g.kids[v] = k;
    std::vector<int> seen;
    for (int a : k)
      if (a >= p.n_const && std::find(seen.begin(), seen.end(), a) == seen.end()) {
        seen.push_back(a);
        g.n_parents[a - p.n_const] += 1;
      }
  }
  for (int r : p.ret)
    if (r >= p.n_const) g.goal[r - p.n_const] = 1;
  return g;
}

std::vector<int> distinct_vars(const std::vector<int>& args, int nc) {
  std::vector<int> out;
  for (int a : args)
    if (a >= nc && std::find(out.begin(), out.end(), a) == out.end()) out.push_back(a);
  return out;
}

}  // namespace

// Pebbles for the statements of g taken in `order`: a pebble is given back
// when the last parent of its node has been computed (goals keep theirs when
// goals_hold), and a new node takes the pebble of the most recently computed
// dead node.
static Schedule assign_pebbles(const Graph& g, const std::vector<int>& order, bool goals_hold) {
  const int nc = g.nc;
  Schedule s;
  std::vector<int> remaining = g.n_parents, pebble(g.nv, -1), when(g.nv, -1);
  std::vector<std::pair<int, int>> free_list;  // (time its node was computed, pebble)
  for (size_t i = 0; i < order.size(); ++i) {
    const int n = order[i];
    // children whose last parent is n give their pebble back
    for (int c : distinct_vars(g.kids[n], nc)) {
      const int cv = c - nc;
      if (--remaining[cv] == 0 && !(g.goal[cv] && goals_hold) && pebble[cv] >= 0)
        free_list.emplace_back(when[cv], pebble[cv]);
    }
    int peb = -1;
    const bool needs = goals_hold ? true : (g.n_parents[n] > 0);
    if (needs) {
      if (!free_list.empty()) {
        // reuse the pebble of the most recently computed dead node
        auto it = std::max_element(free_list.begin(), free_list.end());
        peb = it->second;
        free_list.erase(it);
      } else {
        peb = s.n_pebbles++;
      }
    }
    pebble[n] = peb;
    when[n] = static_cast<int>(i);
    s.steps.push_back(Schedule::Step{n, peb, g.kids[n]});
  }
  return s;
}

Schedule schedule_dfs(const Slp& p, bool goals_hold) {
  Graph g = build_graph(p);
  const int nc = g.nc;
  std::vector<int> order;
  std::vector<char> visited(g.nv, 0);
  std::function<void(int)> visit = [&](int v) {
    if (visited[v]) return;
    visited[v] = 1;
    for (int a : g.kids[v])
      if (a >= nc) visit(a - nc);
    order.push_back(v);
  };
  for (int v = 0; v < g.nv; ++v)  // roots in term order
    if (g.def_idx[v] >= 0 && g.n_parents[v] == 0) visit(v);
  return assign_pebbles(g, order, goals_hold);
}

Schedule schedule_in_order(const Slp& p, bool goals_hold) {
  Graph g = build_graph(p);
  std::vector<int> order;
  for (const auto& st : p.body) order.push_back(st.dst - p.n_const);
  return assign_pebbles(g, order, goals_hold);
}

Schedule schedule_greedy(const Slp& p, int cap, bool goals_hold) {
  Graph g = build_graph(p);
  const int nc = g.nc;
  // The cache holds constants (ids [0,nc)) and pebbles (ids nc + pebble).
  Lru cache(cap, nc + g.nv + 1);
  std::vector<int> remaining = g.n_parents, pebble(g.nv, -1), kids_left(g.nv, 0);
  std::vector<char> done(g.nv, 0);
  int total = 0;
  for (int v = 0; v < g.nv; ++v)
    if (g.def_idx[v] >= 0) {
      ++total;
      kids_left[v] = static_cast<int>(distinct_vars(g.kids[v], nc).size());
    }
  std::vector<int> parents_of_count;
  std::vector<std::vector<int>> parents(g.nv);
  for (int v = 0; v < g.nv; ++v)
    if (g.def_idx[v] >= 0)
      for (int c : distinct_vars(g.kids[v], nc)) parents[c - nc].push_back(v);
  std::vector<int> free_peb;  // pebbles of dead nodes: (node id) owners
  std::vector<int> owner;     // pebble -> node currently on it
  Schedule s;
  auto block_of = [&](int t) { return t < nc ? t : nc + pebble[t - nc]; };
  for (int step = 0; step < total; ++step) {
    int best = -1;
    long bh = -1, bc = 1;
    for (int v = 0; v < g.nv; ++v) {
      if (g.def_idx[v] < 0 || done[v] || kids_left[v] != 0) continue;
      std::vector<int> C;
      for (int a : g.kids[v])
        if (std::find(C.begin(), C.end(), a) == C.end()) C.push_back(a);
      long h = 0;
      for (int a : C) h += cache.has(block_of(a)) ? 1 : 0;
      const long c = C.empty() ? 1 : static_cast<long>(C.size());
      if (C.empty()) h = 1;
      if (best < 0 || h * bc > bh * c) { best = v; bh = h; bc = c; }
    }
    const int n = best;
    std::vector<int> C, H, M;
    for (int a : g.kids[n])
      if (std::find(C.begin(), C.end(), a) == C.end()) C.push_back(a);
    for (int a : C) (cache.has(block_of(a)) ? H : M).push_back(a);
    for (int a : H) cache.use(block_of(a));
    for (int a : M) cache.use(block_of(a));
    std::vector<int> args = H;
    args.insert(args.end(), M.begin(), M.end());
    // children whose last parent is n become movable
    for (int c : distinct_vars(g.kids[n], nc)) {
      const int cv = c - nc;
      if (--remaining[cv] == 0 && !(g.goal[cv] && goals_hold) && pebble[cv] >= 0)
        free_peb.push_back(cv);
    }
    int peb = -1;
    const bool needs = goals_hold ? true : (g.n_parents[n] > 0);
    if (needs) {
      // prefer a movable pebble that is cached, then any movable one; ties by
      // node order; else a fresh pebble
      int pick = -1;
      for (int pass = 0; pass < 2 && pick < 0; ++pass) {
        int bestv = -1;
        for (int v : free_peb) {
          if (pass == 0 && !cache.has(nc + pebble[v])) continue;
          if (bestv < 0 || v < bestv) bestv = v;
        }
        pick = bestv;
      }
      if (pick >= 0) {
        peb = pebble[pick];
        free_peb.erase(std::find(free_peb.begin(), free_peb.end(), pick));
      } else {
        peb = s.n_pebbles++;
      }
    }
    pebble[n] = peb;
    if (peb >= 0) cache.def(nc + peb);
    done[n] = 1;
    for (int par : parents[n]) kids_left[par] -= 1;
    // map args to input ids (constants or variable ids of p)
    s.steps.push_back(Schedule::Step{n, peb, args});
  }
  return s;
}

int max_live_preloaded(const Slp& q, const Schedule& s) {
  const int nc = q.n_const;
  std::vector<int> last_in(nc, -1), last_v(q.n_var, -1);
  for (size_t i = 0; i < s.steps.size(); ++i)
    for (int a : s.steps[i].args) {
      if (a < nc) last_in[a] = static_cast<int>(i);
      else last_v[a - nc] = static_cast<int>(i);
    }
  int live = 0;
  for (int c = 0; c < nc; ++c) live += last_in[c] >= 0;
  int peak = live;
  for (size_t i = 0; i < s.steps.size(); ++i) {
    const int n = s.steps[i].node;
    const bool kept = last_v[n] > static_cast<int>(i);
    peak = std::max(peak, live + 1);   // the result is written while operands are live
    if (kept) ++live;
    for (int a : s.steps[i].args) {
      if (a < nc) {
        if (last_in[a] == static_cast<int>(i)) { --live; last_in[a] = -2; }
      } else if (last_v[a - nc] == static_cast<int>(i)) {
        --live;
        last_v[a - nc] = -2;
      }
    }
  }
  return peak;
}

int max_live_grouped(const Slp& q, const Schedule& s, const std::vector<int>& group,
                     long* loads) {
  const int nc = q.n_const;
  const size_t n = s.steps.size();
  // an input is live from its first to its last use within a group; a
  // variable from its statement to its last use
  std::vector<int> last_v(q.n_var, -1);
  std::vector<std::vector<int>> in_end(n);   // inputs whose group-range ends at step i
  std::vector<int> in_start(n, 0);
  std::vector<int> first(nc, -1), last(nc, -1), seen_group(nc, -1);
  long nload = 0;
  auto close = [&](int c) {
    if (first[c] >= 0) in_end[last[c]].push_back(c);
    first[c] = last[c] = -1;
  };
  for (size_t i = 0; i < n; ++i) {
    const int g = i < group.size() ? group[i] : 0;
    for (int a : s.steps[i].args) {
      if (a >= nc) {
        last_v[a - nc] = static_cast<int>(i);
        continue;
      }
      if (seen_group[a] != g) {
        close(a);
        seen_group[a] = g;
        first[a] = static_cast<int>(i);
        ++in_start[i];
        ++nload;
      }
      last[a] = static_cast<int>(i);
    }
  }
  for (int c = 0; c < nc; ++c) close(c);
  int live = 0, peak = 0;
  for (size_t i = 0; i < n; ++i) {
    live += in_start[i];
    const int v = s.steps[i].node;
    peak = std::max(peak, live + 1);   // the result is written while operands are live
    if (last_v[v] > static_cast<int>(i)) ++live;
    live -= static_cast<int>(in_end[i].size());
    for (int a : distinct_vars(s.steps[i].args, nc))
      if (last_v[a - nc] == static_cast<int>(i)) --live;
  }
  if (loads) *loads = nload;
  return peak;
}

Slp schedule_to_slp(const Slp& p, const Schedule& s) {
  const int nc = p.n_const;
  Slp q;
  q.n_const = nc;
  q.const_names = p.const_names;
  q.n_var = s.n_pebbles;
  for (int i = 0; i < s.n_pebbles; ++i) q.var_names.push_back("p" + std::to_string(i + 1));
  std::vector<int> pebble(p.n_var, -1);
  for (const auto& st : s.steps) {
    Stmt x;
    x.dst = nc + st.pebble;
    for (int a : st.args) x.args.push_back(a < nc ? a : nc + pebble[a - nc]);
    pebble[st.node] = st.pebble;
    q.body.push_back(x);
  }
  for (int r : p.ret) q.ret.push_back(r < nc ? r : nc + pebble[r - nc]);
  return q;
}

}  // namespace xorec
