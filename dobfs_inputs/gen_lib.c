/*
 * Host-side batch entry points over gen.h, loaded from Python by
 * dobfs_inputs/__init__.py. Seeded input generation only.
 */
#include <stdint.h>
#include "gen.h"

uint64_t gen_c_mix64(uint64_t z) { return gen_mix64(z); }

uint32_t gen_c_perm(uint32_t x, uint32_t n, uint64_t seed) { return gen_perm(x, n, gen_key_perm(seed)); }

/* Pairs k0 .. k0+count-1 of an R-MAT stream into src/dst (relabelled IDs). */
void gen_c_rmat_pairs(int scale, uint32_t t_a, uint32_t t_ab, uint32_t t_abc, uint64_t seed,
                      uint64_t k0, int64_t count, int32_t* src, int32_t* dst) {
  const uint64_t kp = gen_key_pairs(seed), kq = gen_key_perm(seed);
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

/* Pairs k0 .. k0+count-1 of a Chung-Lu stream over the weight table cdf[0..n-1]. */
void gen_c_chunglu_pairs(const uint64_t* cdf, uint32_t n, uint64_t seed, uint64_t k0, int64_t count,
                         int32_t* src, int32_t* dst) {
  const uint64_t kp = gen_key_pairs(seed), kq = gen_key_perm(seed);
  for (int64_t i = 0; i < count; ++i) {
    uint32_t u, v;
    gen_chunglu_pair(k0 + (uint64_t)i, cdf, n, kp, kq, &u, &v);
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}
