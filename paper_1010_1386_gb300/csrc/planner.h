// Host-side planning of one resultant: trimmed degrees, the degree bound D,
// the Hadamard bit bound, the prime count and the output limb count.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/rs.h"

struct PolyInfo {
  bool zero = true;
  int my = -1;     // y-degree (largest j with f_j != 0)
  int mx = -1;     // x-degree
  int tdeg = -1;   // total degree
  int L = 1;       // limbs per coefficient
  int stride = 1;  // row stride of the input array (deg_y extent + 1)
  int nc = 0;      // coefficients kept: sum_j (dx_j + 1)
  std::vector<int> dx;  // x-degree of f_j, j = 0..my (-1 for f_j = 0)
  double log2_rownorm2 = 0.0;  // log2 of a bound on max_{|x|=1} sum_j |f_j(x)|^2 (rounded up)
};

struct PairPlan {
  int status = RS_OK;
  bool trivial_zero = false;  // f == 0 or g == 0: R = 0, no device work
  PolyInfo f, g;
  int D = 0;      // degree bound of R
  int N = 0;      // points = D + 1
  int bits = 0;   // |coef R| < 2^bits
  int K = 0;      // primes (images are taken for the first K)
  int Kcrt = 0;   // primes R's Chinese remaindering uses (0: all K); a square-free
                  // batch draws more primes than R needs, for its factors
  int Lout = 0;   // output limbs
  int cap = 0;    // compiled register capacity class for G1
  int staged = 0; // shared-memory words G1 stages per tile
};

// Analyse and plan; returns RS_OK or an error code (also stored in plan.status).
// `log2p` lists log2 of the primes of the table in order (may be empty for
// a bound-only query, in which case K is estimated from 31-bit primes).
int rs_plan_pair(const rs_bipoly *f, const rs_bipoly *g, const std::vector<double> &log2p,
                 PairPlan &plan, const char **why);

// Shared-memory words one G1 tile of `threads` points stages for plan p in
// register-capacity class C: per-j x-degrees, chirp-scaled coefficients of
// f and g ([x-degree + 1][C] each) and the window of q^{C(t,2)}.
inline int rs_g1_staged_words(const PairPlan &p, int C, int threads) {
  const int meta = (2 * (p.f.my + p.g.my + 2) + 7) & ~7;
  const int dx = p.f.mx > p.g.mx ? p.f.mx : p.g.mx;
  return meta + (p.f.mx + 1) * C + (p.g.mx + 1) * C + threads + dx;
}

// Primes in (2^31 - 2^20, 2^31), descending, by a sieve of Eratosthenes.
std::vector<uint32_t> rs_prime_table(int count);
