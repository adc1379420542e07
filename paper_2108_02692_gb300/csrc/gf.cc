#include "gf.h"

#include <cstring>

namespace xorec {
namespace {

struct Tables {
  uint8_t exp[510];
  uint8_t log[256];
  Tables() {
    // 2^i by repeated multiplication by x with reduction by 0x11d.
    uint8_t v = 1;
    for (int i = 0; i < 255; ++i) {
      exp[i] = v;
      exp[i + 255] = v;
      log[v] = static_cast<uint8_t>(i);
      const uint8_t carry = static_cast<uint8_t>(v >> 7);
      v = static_cast<uint8_t>((v << 1) ^ (carry ? 0x1d : 0x00));
    }
    log[0] = 0;
  }
};

const Tables& tabs() {
  static const Tables t;
  return t;
}

}  // namespace

uint8_t gf_mul(uint8_t a, uint8_t b) {
  if (!a || !b) return 0;
  const Tables& t = tabs();
  return t.exp[t.log[a] + t.log[b]];
}

uint8_t gf_inv(uint8_t a) {
  if (!a) return 0;
  const Tables& t = tabs();
  return t.exp[(255 - t.log[a]) % 255];
}

uint8_t gf_exp2(unsigned e) { return tabs().exp[e % 255]; }

std::vector<uint8_t> cauchy_parity(int k, int m) {
  std::vector<uint8_t> P(static_cast<size_t>(k) * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j)
      P[static_cast<size_t>(i) * k + j] = gf_inv(static_cast<uint8_t>((k + i) ^ j));
  return P;
}

int bitmatrix_ones(uint8_t a) {
  int n = 0;
  for (int t = 0; t < 8; ++t) n += __builtin_popcount(gf_mul(a, static_cast<uint8_t>(1u << t)));
  return n;
}

std::vector<uint8_t> cauchy_min_parity(int k, int m) {
  std::vector<uint8_t> P = cauchy_parity(k, m);
  auto at = [&](int i, int j) -> uint8_t& { return P[static_cast<size_t>(i) * k + j]; };
  for (int j = 0; j < k; ++j) {
    const uint8_t s = gf_inv(at(0, j));
    for (int i = 0; i < m; ++i) at(i, j) = gf_mul(at(i, j), s);
  }
  for (int i = 1; i < m; ++i) {
    int best_ones = -1;
    uint8_t best = 1;
    for (int c = 0; c < k; ++c) {
      const uint8_t d = at(i, c);
      const uint8_t s = gf_inv(d);
      int ones = 0;
      for (int j = 0; j < k; ++j) ones += bitmatrix_ones(gf_mul(at(i, j), s));
      if (best_ones < 0 || ones < best_ones || (ones == best_ones && d < best)) {
        best_ones = ones;
        best = d;
      }
    }
    const uint8_t s = gf_inv(best);
    for (int j = 0; j < k; ++j) at(i, j) = gf_mul(at(i, j), s);
  }
  return P;
}

std::vector<uint8_t> power_parity(int k, int m) {
  std::vector<uint8_t> P(static_cast<size_t>(k) * m);
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < k; ++j)
      P[static_cast<size_t>(r) * k + j] = gf_exp2(static_cast<unsigned>(r * j));
  return P;
}

void generator_row(int k, const uint8_t* P, int r, uint8_t* row) {
  if (r < k) {
    std::memset(row, 0, k);
    row[r] = 1;
  } else {
    std::memcpy(row, P + static_cast<size_t>(r - k) * k, k);
  }
}

bool gf_invert(int n, const uint8_t* M, uint8_t* out) {
  std::vector<uint8_t> a(M, M + static_cast<size_t>(n) * n);
  std::memset(out, 0, static_cast<size_t>(n) * n);
  for (int i = 0; i < n; ++i) out[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    while (piv < n && !a[static_cast<size_t>(piv) * n + c]) ++piv;
    if (piv == n) return false;
    if (piv != c) {
      for (int x = 0; x < n; ++x) {
        std::swap(a[static_cast<size_t>(c) * n + x], a[static_cast<size_t>(piv) * n + x]);
        std::swap(out[c * n + x], out[piv * n + x]);
      }
    }
    const uint8_t s = gf_inv(a[static_cast<size_t>(c) * n + c]);
    for (int x = 0; x < n; ++x) {
      a[static_cast<size_t>(c) * n + x] = gf_mul(a[static_cast<size_t>(c) * n + x], s);
      out[c * n + x] = gf_mul(out[c * n + x], s);
    }
    for (int r = 0; r < n; ++r) {
      const uint8_t f = a[static_cast<size_t>(r) * n + c];
      if (r == c || !f) continue;
      for (int x = 0; x < n; ++x) {
        a[static_cast<size_t>(r) * n + x] ^= gf_mul(f, a[static_cast<size_t>(c) * n + x]);
        out[r * n + x] ^= gf_mul(f, out[c * n + x]);
      }
    }
  }
  return true;
}

bool decode_matrix(int k, int m, const uint8_t* P, const std::vector<int>& E,
                   const std::vector<int>& S, std::vector<uint8_t>* R) {
  (void)m;
  std::vector<uint8_t> M(static_cast<size_t>(k) * k), Minv(static_cast<size_t>(k) * k);
  for (int i = 0; i < k; ++i) generator_row(k, P, S[i], &M[static_cast<size_t>(i) * k]);
  if (!gf_invert(k, M.data(), Minv.data())) return false;
  R->assign(E.size() * static_cast<size_t>(k), 0);
  std::vector<uint8_t> row(k);
  for (size_t i = 0; i < E.size(); ++i) {
    generator_row(k, P, E[i], row.data());
    for (int c = 0; c < k; ++c) {
      uint8_t acc = 0;
      for (int x = 0; x < k; ++x) acc ^= gf_mul(row[x], Minv[static_cast<size_t>(x) * k + c]);
      (*R)[i * k + c] = acc;
    }
  }
  return true;
}

}  // namespace xorec
