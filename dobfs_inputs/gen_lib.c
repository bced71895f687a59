/*
 * Host-side batch entry points over gen.h, loaded from Python by
 * dobfs_inputs/__init__.py. Seeded input generation only.
 */
#include <stdint.h>
#include <stdlib.h>
#include "gen.h"

uint64_t gen_c_mix64(uint64_t z) { return gen_mix64(z); }

uint32_t gen_c_perm(uint32_t x, uint32_t n, uint64_t seed) { return gen_perm(x, n, gen_key_perm(seed)); }

/* Pairs k0 .. k0+count-1 of an R-MAT stream into src/dst (relabelled IDs). */
void gen_c_rmat_pairs(int scale, uint32_t t_a, uint32_t t_ab, uint32_t t_abc, uint64_t seed,
                      uint64_t k0, int64_t count, int32_t* src, int32_t* dst) {
  const uint64_t kp = gen_key_pairs(seed), kq = gen_key_perm(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    uint32_t u, v;
    gen_rmat_pair(k0 + (uint64_t)i, scale, t_a, t_ab, t_abc, kp, kq, &u, &v);
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}

/* Same, without the relabelling (used only to test quadrant frequencies). */
void gen_c_rmat_pairs_raw(int scale, uint32_t t_a, uint32_t t_ab, uint32_t t_abc, uint64_t seed,
                          uint64_t k0, int64_t count, int32_t* src, int32_t* dst) {
  const uint64_t kp = gen_key_pairs(seed);
  for (int64_t i = 0; i < count; ++i) {
    uint32_t u, v;
    gen_rmat_pair_raw(k0 + (uint64_t)i, scale, t_a, t_ab, t_abc, kp, &u, &v);
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}

/* Pairs k0 .. k0+count-1 of a Chung-Lu stream over the weight table
 * cdf[0..n-1]. The draws are those of gen_chunglu_pair; only the search is
 * faster: a table B of 2^24 buckets over t = floor(r * total / 2^64) holds
 * B[b] = the first index i with cdf[i] > b << shift, and since that first
 * index is non-decreasing in t, the answer for t in bucket b lies in
 * [B[b], B[b+1]], where a binary search finds it. `plain` != 0 uses
 * gen_cdf_pick itself (for testing that both agree). */
static uint32_t first_above(const uint64_t* cdf, uint32_t lo, uint32_t hi, uint64_t t) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (cdf[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

void gen_c_chunglu_pairs(const uint64_t* cdf, uint32_t n, uint64_t seed, uint64_t k0, int64_t count,
                         int32_t* src, int32_t* dst, int plain) {
  const uint64_t kp = gen_key_pairs(seed), kq = gen_key_perm(seed);
  const uint64_t total = cdf[n - 1];
  int sh = 0;
  while ((total >> sh) >= (1ull << 24)) ++sh;
  const uint64_t nb = (total >> sh) + 1;
  uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nb + 1));
  for (uint64_t b = 0; b <= nb; ++b) {
    const uint64_t t = b << sh;
    B[b] = (t >= total) ? n - 1 : first_above(cdf, 0, n - 1, t);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    const uint64_t k = k0 + (uint64_t)i;
    uint32_t ab[2];
    for (int h = 0; h < 2; ++h) {
      const uint64_t r = gen_mix64(kp ^ (2ull * k + (uint64_t)h));
      if (plain) {
        ab[h] = gen_cdf_pick(r, cdf, n);
      } else {
        const uint64_t t = gen_mulhi64(r, total);
        const uint64_t b = t >> sh;
        ab[h] = first_above(cdf, B[b], B[b + 1], t);
      }
    }
    src[i] = (int32_t)gen_perm(ab[0], n, kq);
    dst[i] = (int32_t)gen_perm(ab[1], n, kq);
  }
  free(B);
}
