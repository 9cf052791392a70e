/*
 * codec_oracle.c — plain CPU reference of the error-bounded array codec.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg); the
 * library never uses it and it shares no code with the CUDA codec.
 *
 * The workflow of "A workflow for seismic imaging with quantified
 * uncertainty" (arXiv 2001.06444) compresses velocity models, images and
 * seismograms between its stages with a fixed-accuracy block codec (§3,
 * §4.2, Tables 1-2; Lindstrom et al. 2016).  This codec follows the same
 * published architecture, in its own concrete form:
 *   1. 4 x 4 blocks (edge blocks padded by repeating their last row/column);
 *   2. a common block exponent e (max |x| = f 2^e, f in [0.5, 1));
 *   3. fixed point q = rint(x 2^(28 - e));
 *   4. an exactly reversible integer transform: a two-level S-transform
 *      (d = b - a, s = a + floor(d/2)) on each row, then on each column;
 *   5. coefficients in order of frequency level, coded as sign-magnitude bit
 *      planes from plane 30 down to kmin, coefficients that are not yet
 *      significant being coded by run-style group tests;
 *   6. kmin, the lowest plane kept: the largest k >= 1 with
 *      16 2^k + 21.5 <= tol 2^(28 - e), else 0 (all planes).
 * Every element then decodes within max(tol, 2^(e - 23)) of its input: the
 * dropped planes (coefficient error below 2^kmin) and the rounding of the
 * inverse transform contribute at most (16 2^kmin + 5.5) 2^(e - 28) (the
 * inverse of one 4-point transform turns input errors E into at most 4E + 1),
 * and rounding the result to float at most 2^(e - 24).
 *
 * Stream layout (little endian): 48-byte header {u32 magic "RTMZ", u32
 * version 1, i64 n0, i64 n1, f64 tol, u64 stream bits, u32 blocks per chunk
 * (16), u32 0}; u64 bit offset of every chunk of 16 blocks; u32 words of
 * the bit stream, bits taken least significant first.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CZ_P 28
#define CZ_CHUNK 16
#define CZ_HEADER 48
#define CZ_BLOCK_MAX_BITS 576

/* coefficient (row*4 + col) order by level lev(row) + lev(col), lev = 0,1,2,2 */
static const int PERM[16] = {0, 1, 4, 2, 3, 5, 8, 12, 6, 7, 9, 13, 10, 11, 14, 15};

typedef struct {
  uint32_t *w;
  uint64_t pos;
} bitw;

typedef struct {
  const uint32_t *w;
  uint64_t pos;
} bitr;

static void put(bitw *b, int bit) {
  if (b->w && bit) b->w[b->pos >> 5] |= 1u << (b->pos & 31);
  b->pos++;
}

static void putn(bitw *b, uint32_t v, int n) {
  for (int i = 0; i < n; ++i) put(b, (v >> i) & 1u);
}

static int get(bitr *b) {
  const int bit = (b->w[b->pos >> 5] >> (b->pos & 31)) & 1u;
  b->pos++;
  return bit;
}

static uint32_t getn(bitr *b, int n) {
  uint32_t v = 0;
  for (int i = 0; i < n; ++i) v |= (uint32_t)get(b) << i;
  return v;
}

/* floor(v / 2) for any sign */
static int32_t half_floor(int32_t v) { return (int32_t)floor((double)v / 2.0); }

/* two-level S-transform of (a, b, c, d) at stride s -> (ss, dd, d1, d2) */
static void fwd4(int32_t *v, int s) {
  int32_t a = v[0], b = v[s], c = v[2 * s], d = v[3 * s];
  int32_t d1 = b - a, s1 = a + half_floor(d1);
  int32_t d2 = d - c, s2 = c + half_floor(d2);
  int32_t dd = s2 - s1, ss = s1 + half_floor(dd);
  v[0] = ss;
  v[s] = dd;
  v[2 * s] = d1;
  v[3 * s] = d2;
}

static void inv4(int32_t *v, int s) {
  int32_t ss = v[0], dd = v[s], d1 = v[2 * s], d2 = v[3 * s];
  int32_t s1 = ss - half_floor(dd), s2 = dd + s1;
  int32_t a = s1 - half_floor(d1), b = d1 + a;
  int32_t c = s2 - half_floor(d2), d = d2 + c;
  v[0] = a;
  v[s] = b;
  v[2 * s] = c;
  v[3 * s] = d;
}

/* lowest bit plane kept for tolerance tol and block exponent e */
int oracle_codec_kmin(double tol, int e) {
  const double T = ldexp(tol, CZ_P - e);
  int k = 0;
  while (k < 30 && 16.0 * ldexp(1.0, k + 1) + 21.5 <= T) k++;
  return k;
}

/* exposed for the tests: forward then inverse transform of a 4 x 4 block */
void oracle_codec_transform(const int32_t *in, int32_t *fwd, int32_t *back) {
  int32_t q[16];
  memcpy(q, in, sizeof(q));
  for (int r = 0; r < 4; ++r) fwd4(q + 4 * r, 1);
  for (int c = 0; c < 4; ++c) fwd4(q + c, 4);
  memcpy(fwd, q, sizeof(q));
  for (int c = 0; c < 4; ++c) inv4(q + c, 4);
  for (int r = 0; r < 4; ++r) inv4(q + 4 * r, 1);
  memcpy(back, q, sizeof(q));
}

static void encode_block(const float *x, double tol, bitw *bw) {
  double mx = 0.0;
  for (int i = 0; i < 16; ++i) mx = fabs((double)x[i]) > mx ? fabs((double)x[i]) : mx;
  if (mx == 0.0) {
    put(bw, 0);
    return;
  }
  put(bw, 1);
  int e;
  frexp(mx, &e);
  putn(bw, (uint32_t)(e + 150), 9);
  int32_t q[16];
  for (int i = 0; i < 16; ++i) q[i] = (int32_t)rint(ldexp((double)x[i], CZ_P - e));
  for (int r = 0; r < 4; ++r) fwd4(q + 4 * r, 1);
  for (int c = 0; c < 4; ++c) fwd4(q + c, 4);
  const int kmin = oracle_codec_kmin(tol, e);
  uint32_t m[16];
  int neg[16], sig[16];
  for (int i = 0; i < 16; ++i) {
    const int32_t c = q[PERM[i]];
    neg[i] = c < 0;
    m[i] = (uint32_t)(c < 0 ? -(int64_t)c : c);
    sig[i] = 0;
  }
  for (int k = 30; k >= kmin; --k) {
    int R[16], nr = 0;
    for (int i = 0; i < 16; ++i) {
      if (sig[i])
        put(bw, (m[i] >> k) & 1u);
      else
        R[nr++] = i;
    }
    int pos = 0;
    while (pos < nr) {
      int g = 0;
      for (int t = pos; t < nr; ++t) g |= (m[R[t]] >> k) & 1u;
      put(bw, g);
      if (!g) break;
      for (;;) {
        const int i = R[pos++];
        const int b = (m[i] >> k) & 1u;
        put(bw, b);
        if (b) {
          put(bw, neg[i]);
          sig[i] = 1;
          break;
        }
      }
    }
  }
}

static void decode_block(bitr *br, double tol, float *x) {
  if (!get(br)) {
    for (int i = 0; i < 16; ++i) x[i] = 0.0f;
    return;
  }
  const int e = (int)getn(br, 9) - 150;
  const int kmin = oracle_codec_kmin(tol, e);
  uint32_t m[16] = {0};
  int neg[16] = {0}, sig[16] = {0};
  for (int k = 30; k >= kmin; --k) {
    int R[16], nr = 0;
    for (int i = 0; i < 16; ++i) {
      if (sig[i]) {
        if (get(br)) m[i] |= 1u << k;
      } else {
        R[nr++] = i;
      }
    }
    int pos = 0;
    while (pos < nr) {
      if (!get(br)) break;
      for (;;) {
        const int i = R[pos++];
        if (get(br)) {
          m[i] |= 1u << k;
          neg[i] = get(br);
          sig[i] = 1;
          break;
        }
      }
    }
  }
  int32_t q[16];
  for (int i = 0; i < 16; ++i) {
    int64_t c = 0;
    if (sig[i]) {
      c = (int64_t)m[i] + (kmin > 0 ? ((int64_t)1 << (kmin - 1)) : 0); /* midpoint */
      if (neg[i]) c = -c;
    }
    q[PERM[i]] = (int32_t)c;
  }
  for (int c = 0; c < 4; ++c) inv4(q + c, 4);
  for (int r = 0; r < 4; ++r) inv4(q + 4 * r, 1);
  for (int i = 0; i < 16; ++i) x[i] = (float)ldexp((double)q[i], e - CZ_P);
}

static void gather_block(const float *data, int64_t n0, int64_t n1, int64_t bi, int64_t bj,
                         float *x) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      int64_t i = 4 * bi + r, j = 4 * bj + c;
      if (i > n0 - 1) i = n0 - 1;
      if (j > n1 - 1) j = n1 - 1;
      x[4 * r + c] = data[i * n1 + j];
    }
}

/* upper bound of the compressed size in bytes */
uint64_t oracle_codec_bound(int64_t n0, int64_t n1) {
  const uint64_t nb = (uint64_t)((n0 + 3) / 4) * (uint64_t)((n1 + 3) / 4);
  const uint64_t nchunk = (nb + CZ_CHUNK - 1) / CZ_CHUNK;
  return CZ_HEADER + 8 * nchunk + 4 * ((nb * CZ_BLOCK_MAX_BITS + 31) / 32);
}

/* Compress data [n0][n1]; returns the byte count written to out (zeroed by
 * the call; capacity >= oracle_codec_bound), or 0 on bad arguments. */
uint64_t oracle_codec_compress(const float *data, int64_t n0, int64_t n1, double tol,
                               unsigned char *out, uint64_t capacity) {
  if (n0 < 1 || n1 < 1 || !(tol > 0) || capacity < oracle_codec_bound(n0, n1)) return 0;
  memset(out, 0, capacity);
  const int64_t nb0 = (n0 + 3) / 4, nb1 = (n1 + 3) / 4, nb = nb0 * nb1;
  const int64_t nchunk = (nb + CZ_CHUNK - 1) / CZ_CHUNK;
  uint64_t *index = (uint64_t *)(out + CZ_HEADER);
  uint32_t *words = (uint32_t *)(out + CZ_HEADER + 8 * nchunk);
  bitw bw = {words, 0};
  float x[16];
  for (int64_t b = 0; b < nb; ++b) {
    if (b % CZ_CHUNK == 0) index[b / CZ_CHUNK] = bw.pos;
    gather_block(data, n0, n1, b / nb1, b % nb1, x);
    encode_block(x, tol, &bw);
  }
  const uint32_t magic = 0x5A4D5452u, version = 1, chunk = CZ_CHUNK, zero = 0;
  memcpy(out + 0, &magic, 4);
  memcpy(out + 4, &version, 4);
  memcpy(out + 8, &n0, 8);
  memcpy(out + 16, &n1, 8);
  memcpy(out + 24, &tol, 8);
  memcpy(out + 32, &bw.pos, 8);
  memcpy(out + 40, &chunk, 4);
  memcpy(out + 44, &zero, 4);
  return CZ_HEADER + 8 * (uint64_t)nchunk + 4 * ((bw.pos + 31) / 32);
}

/* Decompress into data [n0][n1]; returns 0 on success. */
int oracle_codec_decompress(const unsigned char *in, uint64_t nbytes, float *data, int64_t n0,
                            int64_t n1) {
  uint32_t magic;
  int64_t m0, m1;
  double tol;
  uint64_t bits;
  if (nbytes < CZ_HEADER) return -1;
  memcpy(&magic, in, 4);
  memcpy(&m0, in + 8, 8);
  memcpy(&m1, in + 16, 8);
  memcpy(&tol, in + 24, 8);
  memcpy(&bits, in + 32, 8);
  if (magic != 0x5A4D5452u || m0 != n0 || m1 != n1) return -2;
  const int64_t nb0 = (n0 + 3) / 4, nb1 = (n1 + 3) / 4, nb = nb0 * nb1;
  const int64_t nchunk = (nb + CZ_CHUNK - 1) / CZ_CHUNK;
  bitr br = {(const uint32_t *)(in + CZ_HEADER + 8 * nchunk), 0};
  float x[16];
  for (int64_t b = 0; b < nb; ++b) {
    decode_block(&br, tol, x);
    const int64_t bi = b / nb1, bj = b % nb1;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        const int64_t i = 4 * bi + r, j = 4 * bj + c;
        if (i < n0 && j < n1) data[i * n1 + j] = x[4 * r + c];
      }
  }
  return br.pos == bits ? 0 : -3;
}
