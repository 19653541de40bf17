/* Seeded synthetic inputs for the ESMP2 workloads: a counter-based generator.
 *
 * Every value is a pure function of (seed, stream, counter), so any block of the
 * two-electron integral tensor can be produced on its own, in any order, by any
 * number of threads, and the same numbers come out every time.
 *
 *   mix64      : the SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
 *   draw(k, n) : mix64(k + (n + 1) * 0x9E3779B97F4A7C15)   -- n-th output of stream k
 *   normal     : Box-Muller (cosine branch) from draws 2n and 2n+1.
 *
 * Streams: 1 = Fock matrix, 2 = two-electron integrals, 3 = CI-singles matrix G.
 * Integrals (pq|rs) are real with 8-fold permutational symmetry: the counter is
 * the rank of the canonical index (P >= R with P = pair(p,q), R = pair(r,s),
 * pair(p,q) = max(max+1)/2 + min).
 *
 * This file holds input generation only; it contains none of the method's
 * arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * 0x9E3779B97F4A7C15ULL + mix64(stream + 1));
}

static inline uint64_t draw(uint64_t key, uint64_t n) {
  return mix64(key + (n + 1) * 0x9E3779B97F4A7C15ULL);
}

static inline double unif(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

static inline double normal(uint64_t key, uint64_t n) {
  double u1 = ((double)(draw(key, 2 * n) >> 11) + 1.0) * 0x1.0p-53; /* (0,1] */
  double u2 = (double)(draw(key, 2 * n + 1) >> 11) * 0x1.0p-53;     /* [0,1) */
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

static inline uint64_t pair_rank(uint64_t p, uint64_t q) {
  uint64_t hi = p > q ? p : q, lo = p > q ? q : p;
  return hi * (hi + 1) / 2 + lo;
}

static inline double eri(uint64_t key, double sigma, int p, int q, int r, int s) {
  uint64_t P = pair_rank((uint64_t)p, (uint64_t)q), R = pair_rank((uint64_t)r, (uint64_t)s);
  uint64_t n = P >= R ? P * (P + 1) / 2 + R : R * (R + 1) / 2 + P;
  return sigma * normal(key, n);
}

/* Scalar access for tests. */
double synth_eri(uint64_t seed, double sigma, int p, int q, int r, int s) {
  return eri(synth_stream_key(seed, 2), sigma, p, q, r, s);
}

double synth_normal(uint64_t seed, uint64_t stream, uint64_t n) {
  return normal(synth_stream_key(seed, stream), n);
}

double synth_uniform(uint64_t seed, uint64_t stream, uint64_t n) {
  return unif(draw(synth_stream_key(seed, stream), n));
}

/* kind 0: ovov[i][a][j][b] = (i a|j b)      (No*Nv*No*Nv)
 * kind 1: ooov[i][j][k][a] = (i j|k a)      (No*No*No*Nv)
 * kind 2: ovvv[i][a][b][c] = (i a|b c)      (No*Nv*Nv*Nv)
 * kind 3: full[p][q][r][s], p..s < No+Nv    (N^4, small systems only)
 * Virtual orbital a is spatial orbital No + a. */
int synth_eri_block(int kind, int No, int Nv, uint64_t seed, double sigma, double *out) {
  const uint64_t key = synth_stream_key(seed, 2);
  const int N = No + Nv;
  int64_t d0, d1, d2, d3;
  int o0, o1, o2, o3;
  switch (kind) {
    case 0: d0 = No; d1 = Nv; d2 = No; d3 = Nv; o0 = 0; o1 = No; o2 = 0; o3 = No; break;
    case 1: d0 = No; d1 = No; d2 = No; d3 = Nv; o0 = 0; o1 = 0; o2 = 0; o3 = No; break;
    case 2: d0 = No; d1 = Nv; d2 = Nv; d3 = Nv; o0 = 0; o1 = No; o2 = No; o3 = No; break;
    case 3: d0 = N; d1 = N; d2 = N; d3 = N; o0 = o1 = o2 = o3 = 0; break;
    default: return -1;
  }
  const int64_t outer = d0 * d1;
#pragma omp parallel for schedule(static)
  for (int64_t pq = 0; pq < outer; ++pq) {
    const int p = (int)(pq / d1) + o0, q = (int)(pq % d1) + o1;
    double *dst = out + pq * d2 * d3;
    for (int64_t r = 0; r < d2; ++r)
      for (int64_t s = 0; s < d3; ++s)
        dst[r * d3 + s] = eri(key, sigma, p, q, (int)r + o2, (int)s + o3);
  }
  return 0;
}

/* Symmetric N x N Fock-like matrix: occupied diagonal U[-2,-0.3], virtual
 * diagonal U[0.2,3], every off-diagonal element N(0, sigma_off). */
void synth_fock(int No, int Nv, uint64_t seed, double sigma_off, double *F) {
  const uint64_t key = synth_stream_key(seed, 1);
  const int N = No + Nv;
  for (int q = 0; q < N; ++q)
    for (int p = 0; p <= q; ++p) {
      const uint64_t n = (uint64_t)q * (q + 1) / 2 + (uint64_t)p;
      double v;
      if (p == q) {
        const double u = unif(draw(key, 2 * n));
        v = (p < No) ? (-2.0 + 1.7 * u) : (0.2 + 2.8 * u);
      } else {
        v = sigma_off * normal(key, n);
      }
      F[(size_t)p * N + q] = v;
      F[(size_t)q * N + p] = v;
    }
}

/* G[i][a] ~ N(0,1), No x Nv. */
void synth_gauss_matrix(int No, int Nv, uint64_t seed, double *G) {
  const uint64_t key = synth_stream_key(seed, 3);
  for (int i = 0; i < No; ++i)
    for (int a = 0; a < Nv; ++a)
      G[(size_t)i * Nv + a] = normal(key, (uint64_t)i * Nv + a);
}
