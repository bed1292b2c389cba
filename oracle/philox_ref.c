/*
 * MACH oracle, C part: the Bernoulli coin of MACH (Section 3, Remark 1;
 * Algorithm 1 and Algorithm 2, "toss a coin ... with probability p of
 * keeping it") driven by the counter-based generator Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
 * SC'11).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the plain, slow CPU oracle.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load it.  It shares no code with the CUDA path and must never be linked
 * into it.
 *
 * Coin definition (the reading this project fixes, so that the kept index set
 * is reproducible bit for bit on any machine):
 *   - linear index l of entry (i_1..i_d) is its zero-based C-order offset;
 *   - Philox4x32-10 with key (seed mod 2^32, seed div 2^32) is evaluated at
 *     counter (q mod 2^32, q div 2^32, 0, 0), q = l div 4, giving 4 words;
 *   - word w = out[l mod 4];  the entry is kept iff w < T, where
 *     T = floor(p * 2^32) is an integer computed once on the host
 *     (T = 2^32 when p = 1, so every entry is kept).
 * The coin depends on l only, never on the value.
 *
 * Philox4x32-10 as published: ten rounds; each round multiplies words 0 and 2
 * by the two round multipliers (full 32x32->64 products), and the new state
 * is (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)).  The
 * key is bumped by the two Weyl constants before every round but the first.
 * The Weyl constants are the 32-bit fractional parts of the golden ratio and
 * of sqrt(3); the tests recompute them from those closed forms.
 */
#include <stdint.h>

#define ORACLE_PHILOX_M0 0xD2511F53u
#define ORACLE_PHILOX_M1 0xCD9E8D57u
#define ORACLE_PHILOX_W0 0x9E3779B9u
#define ORACLE_PHILOX_W1 0xBB67AE85u

void oracle_philox_constants(uint32_t out[4]) {
  out[0] = ORACLE_PHILOX_M0;
  out[1] = ORACLE_PHILOX_M1;
  out[2] = ORACLE_PHILOX_W0;
  out[3] = ORACLE_PHILOX_W1;
}

/* One Philox4x32 evaluation with a configurable round count (10 is the
 * published Philox4x32-10; other counts exist only so the tests can show
 * that fewer rounds fail the avalanche test that 10 rounds pass). */
void oracle_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds,
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int r;
  for (r = 0; r < rounds; ++r) {
    uint64_t prod0, prod1;
    uint32_t n0, n1, n2, n3;
    if (r > 0) {
      k0 += ORACLE_PHILOX_W0;
      k1 += ORACLE_PHILOX_W1;
    }
    prod0 = (uint64_t)ORACLE_PHILOX_M0 * (uint64_t)x0;
    prod1 = (uint64_t)ORACLE_PHILOX_M1 * (uint64_t)x2;
    n0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    n1 = (uint32_t)prod1;
    n2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    n3 = (uint32_t)prod0;
    x0 = n0;
    x1 = n1;
    x2 = n2;
    x3 = n3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* Philox4x32-10 over a batch of counters q (words 2 and 3 of the counter are
 * zero): out receives 4*n words. */
void oracle_philox_batch(const uint64_t* q, int64_t n, uint64_t seed, uint32_t* out) {
  uint32_t key[2];
  int64_t i;
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
  for (i = 0; i < n; ++i) {
    uint32_t ctr[4];
    ctr[0] = (uint32_t)(q[i] & 0xffffffffu);
    ctr[1] = (uint32_t)(q[i] >> 32);
    ctr[2] = 0;
    ctr[3] = 0;
    oracle_philox4x32(ctr, key, 10, out + 4 * i);
  }
}

/* The MACH coin for one linear index l: 1 if kept, 0 if zeroed. */
int oracle_keep(int64_t l, uint64_t seed, uint64_t T) {
  uint32_t ctr[4], key[2], w[4];
  uint64_t q = (uint64_t)l >> 2;
  ctr[0] = (uint32_t)(q & 0xffffffffu);
  ctr[1] = (uint32_t)(q >> 32);
  ctr[2] = 0;
  ctr[3] = 0;
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
  oracle_philox4x32(ctr, key, 10, w);
  return (uint64_t)w[l & 3] < T;
}

/* Every kept linear index in [l0, l1), in increasing order.  Writes at most
 * cap indices to idx_out and returns the total number kept (which may exceed
 * cap; the caller then retries with a larger buffer). */
int64_t oracle_kept_indices(int64_t l0, int64_t l1, uint64_t seed, uint64_t T,
                            int64_t* idx_out, int64_t cap) {
  int64_t count = 0, l;
  for (l = l0; l < l1; ++l) {
    if (oracle_keep(l, seed, T)) {
      if (count < cap) idx_out[count] = l;
      ++count;
    }
  }
  return count;
}
