/*
 * Plain CPU oracle for XOR-based Reed-Solomon coding over bit-sliced strips.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU baseline of the
 * benchmark use it.  It shares no code, table or constant generator with the
 * CUDA path.  It is written to be slow and obviously correct: every result is
 * the plain definition, evaluated element by element with GF(2^8) log/antilog
 * tables.
 *
 * Definitions followed (paper sections in brackets):
 *   - GF(2^8) = GF(2)[x]/(x^8+x^4+x^3+x^2+1), i.e. polynomial 0x11d, with the
 *     primitive element 2 [Sec. 7.1].  Bit b of a byte is the coefficient of
 *     x^b.
 *   - RS(n,p) encoding is the matrix product b = V d over GF(2^8) with a
 *     systematic generator [I ; P]; the stored blocks are the n data blocks
 *     followed by the p parity blocks [Sec. 1].
 *   - Decoding picks n surviving rows, forms the n x n submatrix M of the
 *     generator and applies M^{-1} [Sec. 1].
 *   - The byte <-> bit-vector isomorphism and the 8x8 GF(2) matrix of a
 *     constant: column t of x~ holds the bits of x * 2^t, so that
 *     x*y = B^{-1}(x~ . B(y)) [Sec. 1, properties (i) and (ii)].
 *   - Blocks are split into 8 strips ("8 x n arrays of N/(8n) bytes")
 *     [Sec. 6.1, Sec. 7.6].  Strip t of a block of B bytes is the byte range
 *     [t*B/8, (t+1)*B/8).  Bit t of field element e is bit (e mod 8) of byte
 *     floor(e/8) of strip t.  A block of B bytes therefore holds B elements.
 *
 * Parity status: every function here is pinned by tests that do not re-run
 * its own formula (field axioms checked exhaustively, spot values, a
 * hand-worked RS(2,1) example, unit vectors, linearity, brute-force MDS
 * recovery, the paper's printed XOR counts 755 and 1368).  The scaled
 * Cauchy matrix is pinned by structure (a row and column scaling of the
 * Cauchy matrix, all-ones single parity row), by full rank of every survivor
 * submatrix of RS(10,4) computed with carry-less arithmetic, by brute-force
 * recovery, and by its bitmatrix ones counted from carry-less products.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_POLY 0x11d

static uint8_t orc_exp_tab[512];
static uint8_t orc_log_tab[256];
static int orc_ready = 0;

/* Log/antilog tables of GF(2^8) with polynomial 0x11d and generator 2
 * [Sec. 7.1].  exp[i] = 2^i; the table is doubled so exp[a+b] needs no
 * reduction modulo 255.  log[0] is unused. */
static void orc_init(void) {
  if (orc_ready) return;
  unsigned v = 1;
  for (int i = 0; i < 255; i++) {
    orc_exp_tab[i] = (uint8_t)v;
    orc_log_tab[v] = (uint8_t)i;
    v <<= 1;                         /* multiply by x */
    if (v & 0x100) v ^= ORC_POLY;    /* reduce by x^8+x^4+x^3+x^2+1 */
  }
  for (int i = 255; i < 512; i++) orc_exp_tab[i] = orc_exp_tab[i - 255];
  orc_log_tab[0] = 0;
  orc_ready = 1;
}

void orc_gf_tables(uint8_t *exp_out, uint8_t *log_out) {
  orc_init();
  memcpy(exp_out, orc_exp_tab, 512);
  memcpy(log_out, orc_log_tab, 256);
}

/* Field product by tables [Sec. 1]. */
uint8_t orc_gf_mul(uint8_t a, uint8_t b) {
  orc_init();
  if (a == 0 || b == 0) return 0;
  return orc_exp_tab[orc_log_tab[a] + orc_log_tab[b]];
}

/* Multiplicative inverse; 0 has none and maps to 0. */
uint8_t orc_gf_inv(uint8_t a) {
  orc_init();
  if (a == 0) return 0;
  return orc_exp_tab[255 - orc_log_tab[a]];
}

/* 2^e for e >= 0. */
uint8_t orc_gf_pow2(long e) {
  orc_init();
  return orc_exp_tab[e % 255];
}

/* Cauchy parity rows: P[i][j] = 1 / (x_i + y_j) with x_i = k + i and
 * y_j = j (field addition is XOR).  The m values x_i and the k values y_j
 * are distinct field elements and no x_i equals a y_j, so every x_i + y_j is
 * nonzero, every square submatrix is nonsingular and [I ; P] is MDS.
 * Requires k + m <= 256.  Returns 0 on success, -1 on bad sizes. */
int orc_cauchy(int k, int m, uint8_t *P) {
  if (k < 1 || m < 1 || k + m > 256) return -1;
  for (int i = 0; i < m; i++)
    for (int j = 0; j < k; j++)
      P[i * k + j] = orc_gf_inv((uint8_t)((k + i) ^ j));
  return 0;
}

/* Number of ones in the 8x8 GF(2) matrix of multiplication by a: column t
 * holds the bits of a * 2^t [Sec. 1, property (ii)]. */
static int orc_ones(uint8_t a) {
  int n = 0;
  for (int t = 0; t < 8; t++) {
    uint8_t col = orc_gf_mul(a, (uint8_t)(1u << t));
    for (int b = 0; b < 8; b++) n += (col >> b) & 1;
  }
  return n;
}

/* Cauchy parity rows scaled to few bitmatrix ones.  The XOR count of a
 * bitmatrix program is its number of ones minus one per row, and two
 * matrices of one size can differ a lot in it [Sec. 7.6].  Multiplying a
 * row or a column of P by a nonzero constant multiplies every square
 * submatrix's determinant by a nonzero constant, so the code stays MDS.
 * Steps: start from orc_cauchy; divide each column by its row-0 entry;
 * then, for each row r >= 1 in turn, among the entries of row r choose the
 * divisor that leaves the row with the fewest ones (on a tie the smallest
 * entry) and divide the row by it. */
int orc_cauchy_min(int k, int m, uint8_t *P) {
  if (orc_cauchy(k, m, P) != 0) return -1;
  for (int j = 0; j < k; j++) {
    uint8_t top = P[j];
    for (int i = 0; i < m; i++) P[i * k + j] = orc_gf_mul(P[i * k + j], orc_gf_inv(top));
  }
  for (int r = 1; r < m; r++) {
    int best_ones = 1 << 30;
    uint8_t best_div = 0;
    for (int c = 0; c < k; c++) {
      uint8_t div = P[r * k + c];
      int ones = 0;
      for (int j = 0; j < k; j++) ones += orc_ones(orc_gf_mul(P[r * k + j], orc_gf_inv(div)));
      if (ones < best_ones || (ones == best_ones && div < best_div)) {
        best_ones = ones;
        best_div = div;
      }
    }
    for (int j = 0; j < k; j++) P[r * k + j] = orc_gf_mul(P[r * k + j], orc_gf_inv(best_div));
  }
  return 0;
}

/* Power parity rows P[r][j] = 2^(r*j): the parity part of the systematic
 * encoding matrix whose bitmatrix gives the XOR counts the paper prints for
 * RS(10,4) [Sec. 7.1, Sec. 7.5].  Not MDS for every (k, m). */
int orc_power(int k, int m, uint8_t *P) {
  if (k < 1 || m < 1 || k + m > 256) return -1;
  for (int r = 0; r < m; r++)
    for (int j = 0; j < k; j++)
      P[r * k + j] = orc_gf_pow2((long)r * (long)j);
  return 0;
}

/* Element e of a bit-sliced block of B bytes [Sec. 6.1 layout]. */
uint8_t orc_get_elem(const uint8_t *block, size_t B, size_t e) {
  size_t S = B / 8;
  uint8_t v = 0;
  for (int t = 0; t < 8; t++) {
    uint8_t byte = block[(size_t)t * S + e / 8];
    v |= (uint8_t)(((byte >> (e % 8)) & 1u) << t);
  }
  return v;
}

void orc_set_elem(uint8_t *block, size_t B, size_t e, uint8_t v) {
  size_t S = B / 8;
  for (int t = 0; t < 8; t++) {
    uint8_t *byte = &block[(size_t)t * S + e / 8];
    uint8_t mask = (uint8_t)(1u << (e % 8));
    if ((v >> t) & 1u) *byte |= mask; else *byte &= (uint8_t)~mask;
  }
}

/* out_i = sum_j A[i][j] * in_j over GF(2^8), element by element, for a
 * rows x cols matrix A (row-major) and blocks of B bytes (B % 8 == 0).
 * Each input block is un-sliced element by element, multiplied with the
 * tables and the result sliced back [Sec. 1]. */
int orc_apply(int rows, int cols, const uint8_t *A,
              const uint8_t *const *in, uint8_t *const *out, size_t B) {
  if (rows < 0 || cols < 0 || B % 8 != 0) return -1;
  for (int i = 0; i < rows; i++) {
    for (size_t e = 0; e < B; e++) {
      uint8_t acc = 0;
      for (int j = 0; j < cols; j++)
        acc ^= orc_gf_mul(A[i * cols + j], orc_get_elem(in[j], B, e));
      orc_set_elem(out[i], B, e, acc);
    }
  }
  return 0;
}

/* Encoding: parity_i = sum_j P[i][j] d_j for the generator [I ; P]
 * [Sec. 1, Sec. 7.1]. */
int orc_encode(int k, int m, const uint8_t *P, const uint8_t *const *data,
               uint8_t *const *parity, size_t B) {
  return orc_apply(m, k, P, data, parity, B);
}

/* Gauss-Jordan inversion of an n x n matrix over GF(2^8) (row-major).
 * Returns 0 on success, 1 if singular, -1 on bad size. */
int orc_invert(int n, const uint8_t *M, uint8_t *Minv) {
  if (n < 1) return -1;
  uint8_t *a = (uint8_t *)malloc((size_t)n * n);
  if (!a) return -1;
  memcpy(a, M, (size_t)n * n);
  memset(Minv, 0, (size_t)n * n);
  for (int i = 0; i < n; i++) Minv[i * n + i] = 1;
  for (int c = 0; c < n; c++) {
    int piv = -1;
    for (int r = c; r < n; r++)
      if (a[r * n + c]) { piv = r; break; }
    if (piv < 0) { free(a); return 1; }
    if (piv != c) {
      for (int x = 0; x < n; x++) {
        uint8_t t = a[c * n + x]; a[c * n + x] = a[piv * n + x]; a[piv * n + x] = t;
        t = Minv[c * n + x]; Minv[c * n + x] = Minv[piv * n + x]; Minv[piv * n + x] = t;
      }
    }
    uint8_t s = orc_gf_inv(a[c * n + c]);
    for (int x = 0; x < n; x++) {
      a[c * n + x] = orc_gf_mul(a[c * n + x], s);
      Minv[c * n + x] = orc_gf_mul(Minv[c * n + x], s);
    }
    for (int r = 0; r < n; r++) {
      if (r == c || a[r * n + c] == 0) continue;
      uint8_t f = a[r * n + c];
      for (int x = 0; x < n; x++) {
        a[r * n + x] ^= orc_gf_mul(f, a[c * n + x]);
        Minv[r * n + x] ^= orc_gf_mul(f, Minv[c * n + x]);
      }
    }
  }
  free(a);
  return 0;
}

/* Row r of the systematic generator [I ; P] (k columns). */
static void orc_gen_row(int k, const uint8_t *P, int r, uint8_t *row) {
  if (r < k) {
    memset(row, 0, (size_t)k);
    row[r] = 1;
  } else {
    memcpy(row, P + (size_t)(r - k) * k, (size_t)k);
  }
}

/* Decoding used only to check the oracle itself (MDS recovery): the n
 * surviving rows S are the first k block ids that are not erased, in
 * ascending order; D = M^{-1} B recovers the data and erased parity is
 * re-encoded from it [Sec. 1].  blocks[] is indexed by block id (k + m
 * entries, erased ones ignored); out[i] receives block erasures[i].
 * Returns 0, 1 if M is singular, -1 on bad arguments. */
int orc_decode(int k, int m, const uint8_t *P, const int *erasures, int ne,
               const uint8_t *const *blocks, uint8_t *const *out, size_t B) {
  if (k < 1 || m < 1 || ne < 0 || ne > m || B % 8 != 0) return -1;
  int n = k + m;
  char *erased = (char *)calloc((size_t)n, 1);
  int *surv = (int *)malloc(sizeof(int) * (size_t)k);
  uint8_t *M = (uint8_t *)malloc((size_t)k * k);
  uint8_t *Minv = (uint8_t *)malloc((size_t)k * k);
  uint8_t *R = (uint8_t *)malloc((size_t)(ne ? ne : 1) * k);
  uint8_t *row = (uint8_t *)malloc((size_t)k);
  const uint8_t **sb = (const uint8_t **)malloc(sizeof(uint8_t *) * (size_t)k);
  int rc = -1;
  if (!erased || !surv || !M || !Minv || !R || !row || !sb) goto done;
  for (int i = 0; i < ne; i++) {
    if (erasures[i] < 0 || erasures[i] >= n || erased[erasures[i]]) goto done;
    erased[erasures[i]] = 1;
  }
  {
    int c = 0;
    for (int id = 0; id < n && c < k; id++)
      if (!erased[id]) surv[c++] = id;
    if (c < k) goto done;
  }
  for (int i = 0; i < k; i++) {
    orc_gen_row(k, P, surv[i], M + (size_t)i * k);
    sb[i] = blocks[surv[i]];
  }
  rc = orc_invert(k, M, Minv);
  if (rc != 0) goto done;
  /* R = G[E] * M^{-1} */
  for (int i = 0; i < ne; i++) {
    orc_gen_row(k, P, erasures[i], row);
    for (int c = 0; c < k; c++) {
      uint8_t acc = 0;
      for (int x = 0; x < k; x++) acc ^= orc_gf_mul(row[x], Minv[x * k + c]);
      R[(size_t)i * k + c] = acc;
    }
  }
  rc = orc_apply(ne, k, R, sb, out, B);
done:
  free(erased); free(surv); free(M); free(Minv); free(R); free(row); free(sb);
  return rc;
}

/* Bitmatrix of a rows x cols matrix A over GF(2^8): a (8 rows) x (8 cols)
 * 0/1 matrix, entry [8i+s][8j+t] = bit s of A[i][j] * 2^t
 * [Sec. 1, property (ii)].  bits is row-major, one byte per entry. */
void orc_bitmatrix(int rows, int cols, const uint8_t *A, uint8_t *bits) {
  int W = 8 * cols;
  for (int i = 0; i < rows; i++)
    for (int j = 0; j < cols; j++)
      for (int t = 0; t < 8; t++) {
        uint8_t col = orc_gf_mul(A[i * cols + j], (uint8_t)(1u << t));
        for (int s = 0; s < 8; s++)
          bits[(size_t)(8 * i + s) * W + 8 * j + t] = (uint8_t)((col >> s) & 1u);
      }
}

/* Matrix product over GF(2) as array XORs [Sec. 1]: output strip (i,s) is
 * the XOR of the input strips (j,t) whose bitmatrix entry is 1.  Blocks of
 * B bytes, strips of B/8 bytes. */
int orc_apply_bitmatrix(int rows, int cols, const uint8_t *bits,
                        const uint8_t *const *in, uint8_t *const *out, size_t B) {
  if (B % 8 != 0) return -1;
  size_t S = B / 8;
  int W = 8 * cols;
  for (int i = 0; i < rows; i++)
    for (int s = 0; s < 8; s++) {
      uint8_t *dst = out[i] + (size_t)s * S;
      memset(dst, 0, S);
      for (int j = 0; j < cols; j++)
        for (int t = 0; t < 8; t++) {
          if (!bits[(size_t)(8 * i + s) * W + 8 * j + t]) continue;
          const uint8_t *src = in[j] + (size_t)t * S;
          for (size_t w = 0; w < S; w++) dst[w] ^= src[w];
        }
    }
  return 0;
}
