// GF(2^8) arithmetic and coding matrices for the planner (host side).
//
// Field: GF(2)[x] / (x^8 + x^4 + x^3 + x^2 + 1), polynomial 0x11d, primitive
// element 2 (Sec. 7.1).  Bit b of a byte is the coefficient of x^b.
#pragma once
#include <cstdint>
#include <vector>

namespace xorec {

uint8_t gf_mul(uint8_t a, uint8_t b);
uint8_t gf_inv(uint8_t a);          // inv(0) = 0
uint8_t gf_exp2(unsigned e);        // 2^e

// Parity rows of the systematic generator [I ; P] (m x k, row-major).
// Cauchy: P[i][j] = 1 / ((k + i) XOR j); MDS for k + m <= 256.
std::vector<uint8_t> cauchy_parity(int k, int m);
// Cauchy rows and columns scaled by nonzero constants so that the bitmatrix
// has few ones (the XOR count of an unoptimised program depends on the
// matrix, Sec. 7.6): every column is divided by its entry in row 0 (row 0
// becomes all ones), then every other row is divided by the entry of that
// row that leaves the row with the fewest bitmatrix ones (ties: the smallest
// entry).  Scaling rows and columns keeps every square submatrix
// nonsingular, so the code stays MDS.
std::vector<uint8_t> cauchy_min_parity(int k, int m);
// Ones in the 8 x 8 GF(2) matrix of multiplication by a (Sec. 1, (ii)).
int bitmatrix_ones(uint8_t a);
// Power rows P[r][j] = 2^(r*j): the matrix that reproduces the XOR counts the
// paper prints for RS(10,4) (Sec. 7.1, Sec. 7.5).  Not MDS in general.
std::vector<uint8_t> power_parity(int k, int m);

// Row r of [I ; P] (k entries).
void generator_row(int k, const uint8_t* P, int r, uint8_t* row);

// Gauss-Jordan inverse of an n x n matrix; false if singular.
bool gf_invert(int n, const uint8_t* M, uint8_t* out);

// Decode matrix R = G[E] * G[S]^{-1} (|E| x k) for erasures E and the
// survivor list S (k ids).  Returns false if G[S] is singular (Sec. 1).
bool decode_matrix(int k, int m, const uint8_t* P, const std::vector<int>& E,
                   const std::vector<int>& S, std::vector<uint8_t>* R);

}  // namespace xorec
