/*
 * Seeded synthetic graph inputs, shared by the CPU oracle and the CUDA library.
 *
 * This header holds no BFS arithmetic. It defines counter-based random draws
 * and the two graph generators built on them:
 *
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004), the generator family of
 *     the Graph500 workloads the paper measures on (Sec. 4, "Workloads"):
 *     undirected pair k is drawn by `scale` independent quadrant choices with
 *     probabilities A, B, C, D, then both endpoints are relabelled by a seeded
 *     bijection of [0, 2^scale) so vertex IDs carry no degree information.
 *   - Chung-Lu (Chung & Lu, 2002): each endpoint is drawn with probability
 *     proportional to a per-vertex weight, by an integer inverse-CDF search.
 *
 * Every function is a pure function of integer arguments, so host code (gcc)
 * and device code (nvcc) produce identical results bit for bit. Probabilities
 * enter only as integer thresholds computed once on the host.
 */
#ifndef DOBFS_INPUTS_GEN_H
#define DOBFS_INPUTS_GEN_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GEN_HD static __host__ __device__ __forceinline__
#else
#define GEN_HD static inline
#endif

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014): adds the
 * golden-ratio increment, then two xor-shift-multiply rounds. A bijection of
 * 64-bit integers; used here as a counter-based generator: draw c of stream
 * `key` is gen_mix64(key ^ c). */
GEN_HD uint64_t gen_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Stream keys derived from the user seed: one for R-MAT quadrant draws, one
 * for the relabelling bijection, one for Chung-Lu endpoint draws. */
GEN_HD uint64_t gen_key_pairs(uint64_t seed) { return gen_mix64(seed ^ 0x52A7D00D00000001ull); }
GEN_HD uint64_t gen_key_perm(uint64_t seed) { return gen_mix64(seed ^ 0x9E3A7B1500000002ull); }

/* High 64 bits of the 128-bit product a*b. */
GEN_HD uint64_t gen_mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

/* Seeded bijection of [0, 2^bits), bits in [0, 32]: four rounds of
 * (multiply by an odd constant, add a constant) mod 2^bits followed by a
 * right xor-shift by ceil(bits/2). Each step is invertible on bits-wide
 * values, so the composition is a permutation. */
GEN_HD uint32_t gen_perm_pow2(uint32_t x, int bits, uint64_t pkey) {
  if (bits <= 0) return 0;
  const uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
  const int sh = (bits + 1) / 2;
  uint64_t y = (uint64_t)x & mask;
  for (int r = 0; r < 4; ++r) {
    const uint64_t m = gen_mix64(pkey + (uint64_t)r);
    y = (y * (m | 1ull) + (m >> 32)) & mask;
    y ^= y >> sh;
  }
  return (uint32_t)y;
}

/* Seeded bijection of [0, n) for any n >= 1: the power-of-two permutation
 * of the enclosing range, with cycle walking until the value lands in
 * [0, n). For n a power of two no walking happens. */
GEN_HD uint32_t gen_perm(uint32_t x, uint32_t n, uint64_t pkey) {
  int bits = 0;
  while (bits < 32 && (1ull << bits) < (uint64_t)n) ++bits;
  uint32_t y = gen_perm_pow2(x, bits, pkey);
  while (y >= n) y = gen_perm_pow2(y, bits, pkey);
  return y;
}

/* R-MAT pair k at `scale` (<= 31), before relabelling. Bit i of both
 * endpoints comes from one 32-bit draw x: quadrant q = [x>=t_a] + [x>=t_ab]
 * + [x>=t_abc] in {0:A, 1:B, 2:C, 3:D}; the source bit is q>>1 (set in C, D)
 * and the destination bit is q&1 (set in B, D). Draws come two per 64-bit
 * counter value (k<<4 | i/2), low half first. */
GEN_HD void gen_rmat_pair_raw(uint64_t k, int scale, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                              uint64_t kpairs, uint32_t* u_out, uint32_t* v_out) {
  uint32_t u = 0, v = 0;
  for (int i = 0; i < scale; i += 2) {
    const uint64_t r = gen_mix64(kpairs ^ ((k << 4) | (uint64_t)(i >> 1)));
    for (int h = 0; h < 2 && i + h < scale; ++h) {
      const uint32_t x = (uint32_t)(r >> (32 * h));
      const uint32_t q = (uint32_t)(x >= t_a) + (uint32_t)(x >= t_ab) + (uint32_t)(x >= t_abc);
      u |= (q >> 1) << (i + h);
      v |= (q & 1u) << (i + h);
    }
  }
  *u_out = u;
  *v_out = v;
}

/* R-MAT pair k, relabelled: the published vertex IDs. */
GEN_HD void gen_rmat_pair(uint64_t k, int scale, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                          uint64_t kpairs, uint64_t kperm, uint32_t* u_out, uint32_t* v_out) {
  uint32_t u, v;
  gen_rmat_pair_raw(k, scale, t_a, t_ab, t_abc, kpairs, &u, &v);
  *u_out = gen_perm_pow2(u, scale, kperm);
  *v_out = gen_perm_pow2(v, scale, kperm);
}

/* Index drawn from an inclusive cumulative integer weight table cdf[0..n-1]
 * (non-decreasing, cdf[n-1] > 0): t = floor(r * total / 2^64) lies in
 * [0, total); the result is the first i with cdf[i] > t, so index i is drawn
 * with probability (cdf[i] - cdf[i-1]) / total. */
GEN_HD uint32_t gen_cdf_pick(uint64_t r, const uint64_t* cdf, uint32_t n) {
  const uint64_t t = gen_mulhi64(r, cdf[n - 1]);
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (cdf[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* Chung-Lu pair k: both endpoints drawn from the weight table, then
 * relabelled by the seeded bijection of [0, n). */
GEN_HD void gen_chunglu_pair(uint64_t k, const uint64_t* cdf, uint32_t n, uint64_t kpairs,
                             uint64_t kperm, uint32_t* u_out, uint32_t* v_out) {
  const uint32_t a = gen_cdf_pick(gen_mix64(kpairs ^ (2ull * k)), cdf, n);
  const uint32_t b = gen_cdf_pick(gen_mix64(kpairs ^ (2ull * k + 1ull)), cdf, n);
  *u_out = gen_perm(a, n, kperm);
  *v_out = gen_perm(b, n, kperm);
}

#endif /* DOBFS_INPUTS_GEN_H */
