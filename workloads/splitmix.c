/*
 * Seeded synthetic inputs: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw number i (0-based) of seed s is mix64(s + (i + 1) * GAMMA).
 *
 * This file holds no part of the spin-summation arithmetic. Both the oracle
 * side and the GPU side read their inputs from here, so both see the same
 * bytes. Built as a small shared library with OpenMP for large tensors.
 */
#include <stdint.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GAMMA); }

/* raw 64-bit draws start .. start+n-1 */
void wl_draw_u64(uint64_t seed, uint64_t start, int64_t n, uint64_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) out[i] = draw(seed, start + (uint64_t)i);
}

/* uniform in [-1, 1): the top 53 bits as a fraction of 2^53, times 2, minus 1 */
void wl_uniform_f64(uint64_t seed, uint64_t start, int64_t n, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    uint64_t x = draw(seed, start + (uint64_t)i);
    out[i] = (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

/* integer-valued doubles in {-3, ..., 3}: ((x >> 32) mod 7) - 3 */
void wl_int7_f64(uint64_t seed, uint64_t start, int64_t n, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    uint64_t x = draw(seed, start + (uint64_t)i);
    out[i] = (double)((int64_t)((x >> 32) % 7) - 3);
  }
}
