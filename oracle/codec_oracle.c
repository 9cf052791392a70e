/*
 * codec_oracle.c — plain CPU reference of the error-bounded array codec.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg); the
 * library never uses it and it shares no code with the CUDA codec.
 *
 * The workflow of "A workflow for seismic imaging with quantified
 * uncertainty" (arXiv 2001.06444) compresses velocity models, images and
 * seismograms between its stages with a transform block codec, in a
 * fixed-accuracy (absolute tolerance) mode and a lossless mode (§3, §4.2,
 * Tables 1-2; the codec architecture is Lindstrom 2014/2016).  This codec
 * follows that published architecture in its own concrete form:
 *   1. 4 x 4 blocks (edge blocks padded by repeating their last row/column);
 *   2. fixed accuracy: a common block exponent e (max |x| = f 2^e, f in
 *      [0.5, 1)) and fixed point q = rint(x 2^(28 - e));
 *      lossless: q = the float's bits read as an order-preserving integer
 *      (sign-magnitude to two's complement);
 *   3. an exactly reversible integer transform: a two-level S-transform
 *      (d = b - a, s = a + floor(d/2)) on each row, then on each column;
 *   4. coefficients in order of frequency level; their magnitudes coded by
 *      bit plane from the top plane (30; lossless 32) down to kmin with
 *      prefix significance: a run-style group test per plane asks whether
 *      any coefficient outside the significant prefix has its bit set, and
 *      a scan then moves the prefix up to that coefficient;
 *   5. the bits of each significant coefficient below the plane at which it
 *      entered the prefix, lowest plane first, then a sign bit (1 for a
 *      negative coefficient whose kept magnitude is not zero, else 0), after
 *      the significance section of the block: every member carries a sign
 *      bit, so the significance section alone fixes the length of the
 *      refinement section;
 *   6. kmin, the lowest plane kept: the largest k >= 1 with
 *      16 2^k + 21.5 <= tol 2^(28 - e), else 0 (all planes); lossless 0.
 * Fixed accuracy decodes every element within max(tol, 2^(e - 23)) of its
 * input: dropped planes leave each coefficient within 2^kmin, the inverse
 * transform (with its floor rounding) turns that into at most
 * (16 2^kmin + 5.5) 2^(e - 28), and rounding to float adds at most
 * 2^(e - 24).  Lossless decoding returns the input bits exactly.
 *
 * Stream of one array (little endian): 64-byte header {u32 magic "RTMZ",
 * u32 version 3, u32 mode (0 fixed accuracy, 1 lossless), u32 blocks per
 * chunk (32), i64 n0, i64 n1, f64 tol, u64 words of the bit section, u64
 * chunks, u64 0}; the u32 word offset of every chunk of 32 blocks, padded
 * with zeros to a multiple of four entries; the bit section as u32 words,
 * bits taken least significant first.  Every chunk starts on a word.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CZ_P 28
#define CZ_CHUNK 32
#define CZ_HEADER 64
#define CZ_BLOCK_MAX_BITS 640

/* coefficient (row*4 + col) order by level lev(row) + lev(col), lev = 0,1,2,2 */
static const int PERM[16] = {0, 1, 4, 2, 3, 5, 8, 12, 6, 7, 9, 13, 10, 11, 14, 15};

typedef struct {
  uint32_t *w;
  uint64_t pos;
} bitw;

typedef struct {
  const uint32_t *w;
  uint64_t nbits;
  uint64_t pos;
  int bad; /* read past the end */
} bitr;

static void put(bitw *b, int bit) {
  if (bit) b->w[b->pos >> 5] |= 1u << (b->pos & 31);
  b->pos++;
}

static void putn(bitw *b, uint32_t v, int n) {
  for (int i = 0; i < n; ++i) put(b, (v >> i) & 1u);
}

static int get(bitr *b) {
  if (b->pos >= b->nbits) {
    b->bad = 1;
    return 0;
  }
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
static int64_t half_floor(int64_t v) { return (int64_t)floor((double)v / 2.0); }

/* two-level S-transform of (a, b, c, d) at stride s -> (ss, dd, d1, d2) */
static void fwd4(int64_t *v, int s) {
  int64_t a = v[0], b = v[s], c = v[2 * s], d = v[3 * s];
  int64_t d1 = b - a, s1 = a + half_floor(d1);
  int64_t d2 = d - c, s2 = c + half_floor(d2);
  int64_t dd = s2 - s1, ss = s1 + half_floor(dd);
  v[0] = ss;
  v[s] = dd;
  v[2 * s] = d1;
  v[3 * s] = d2;
}

static void inv4(int64_t *v, int s) {
  int64_t ss = v[0], dd = v[s], d1 = v[2 * s], d2 = v[3 * s];
  int64_t s1 = ss - half_floor(dd), s2 = dd + s1;
  int64_t a = s1 - half_floor(d1), b = d1 + a;
  int64_t c = s2 - half_floor(d2), d = d2 + c;
  v[0] = a;
  v[s] = b;
  v[2 * s] = c;
  v[3 * s] = d;
}

static void forward(int64_t *q) {
  for (int r = 0; r < 4; ++r) fwd4(q + 4 * r, 1);
  for (int c = 0; c < 4; ++c) fwd4(q + c, 4);
}

static void inverse(int64_t *q) {
  for (int c = 0; c < 4; ++c) inv4(q + c, 4);
  for (int r = 0; r < 4; ++r) inv4(q + 4 * r, 1);
}

/* lowest bit plane kept for tolerance tol and block exponent e */
int oracle_codec_kmin(double tol, int e) {
  const double T = ldexp(tol, CZ_P - e);
  int k = 0;
  while (k < 30 && 16.0 * ldexp(1.0, k + 1) + 21.5 <= T) k++;
  return k;
}

/* exposed for the tests: forward then inverse transform of a 4 x 4 block */
void oracle_codec_transform(const int64_t *in, int64_t *fwd, int64_t *back) {
  int64_t q[16];
  memcpy(q, in, sizeof(q));
  forward(q);
  memcpy(fwd, q, sizeof(q));
  inverse(q);
  memcpy(back, q, sizeof(q));
}

/* order-preserving integer of a float's bits, and back */
static int64_t float_to_ordered(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return (u >> 31) ? -1 - (int64_t)(u & 0x7fffffffu) : (int64_t)u;
}

static float ordered_to_float(int64_t i) {
  const uint32_t u = i < 0 ? 0x80000000u | (uint32_t)(-1 - i) : (uint32_t)i;
  float x;
  memcpy(&x, &u, 4);
  return x;
}

/* Significance and refinement coding of 16 magnitudes (coding order),
 * planes top..kmin. */
static void encode_planes(const uint64_t *m, const int *neg, int top, int kmin, bitw *bw) {
  int entry[16];
  int n = 0;
  for (int k = top; k >= kmin; --k) {
    while (n < 16) {
      int g = 0;
      for (int i = n; i < 16; ++i) g |= (int)((m[i] >> k) & 1u);
      put(bw, g);
      if (!g) break;
      int b;
      do {
        b = (int)((m[n] >> k) & 1u);
        put(bw, b);
        entry[n] = k;
        n++;
      } while (!b);
    }
  }
  for (int i = 0; i < n; ++i) {
    for (int k = kmin; k < entry[i]; ++k) put(bw, (int)((m[i] >> k) & 1u));
    put(bw, (m[i] >> kmin) ? neg[i] : 0);
  }
}

/* returns 0, or -1 on a malformed block */
static int decode_planes(bitr *br, uint64_t *m, int *neg, int top, int kmin) {
  int entry[16];
  int n = 0;
  for (int i = 0; i < 16; ++i) m[i] = 0, neg[i] = 0;
  for (int k = top; k >= kmin; --k) {
    while (n < 16) {
      if (!get(br)) break;
      int b;
      do {
        if (n > 15 || br->bad) return -1;
        b = get(br);
        entry[n] = k;
        if (b) m[n] |= (uint64_t)1 << k;
        n++;
      } while (!b);
    }
  }
  for (int i = 0; i < n; ++i) {
    for (int k = kmin; k < entry[i]; ++k)
      if (get(br)) m[i] |= (uint64_t)1 << k;
    const int sg = get(br);
    if (m[i] >> kmin) neg[i] = sg;
  }
  return br->bad ? -1 : 0;
}

static void encode_block(const float *x, double tol, bitw *bw) {
  int64_t q[16];
  int top, kmin;
  if (tol > 0) {
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
    for (int i = 0; i < 16; ++i) q[i] = (int64_t)rint(ldexp((double)x[i], CZ_P - e));
    top = 30;
    kmin = oracle_codec_kmin(tol, e);
  } else {
    int any = 0;
    for (int i = 0; i < 16; ++i) {
      q[i] = float_to_ordered(x[i]);
      any |= q[i] != 0;
    }
    put(bw, any);
    if (!any) return;
    top = 32;
    kmin = 0;
  }
  forward(q);
  uint64_t m[16];
  int neg[16];
  for (int i = 0; i < 16; ++i) {
    const int64_t c = q[PERM[i]];
    neg[i] = c < 0;
    m[i] = (uint64_t)(c < 0 ? -c : c);
  }
  encode_planes(m, neg, top, kmin, bw);
}

static int decode_block(bitr *br, double tol, float *x) {
  if (!get(br)) {
    for (int i = 0; i < 16; ++i) x[i] = 0.0f;
    return br->bad ? -1 : 0;
  }
  int e = 0, top = 32, kmin = 0;
  if (tol > 0) {
    e = (int)getn(br, 9) - 150;
    top = 30;
    kmin = oracle_codec_kmin(tol, e);
  }
  uint64_t m[16];
  int neg[16];
  if (decode_planes(br, m, neg, top, kmin)) return -1;
  int64_t q[16];
  for (int i = 0; i < 16; ++i) {
    int64_t c = 0;
    if (m[i]) {
      c = (int64_t)m[i] + (kmin > 0 ? ((int64_t)1 << (kmin - 1)) : 0); /* midpoint */
      if (neg[i]) c = -c;
    }
    q[PERM[i]] = c;
  }
  inverse(q);
  for (int i = 0; i < 16; ++i)
    x[i] = tol > 0 ? (float)ldexp((double)q[i], e - CZ_P) : ordered_to_float(q[i]);
  return 0;
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

static int64_t nchunks(int64_t n0, int64_t n1) {
  const int64_t nb = ((n0 + 3) / 4) * ((n1 + 3) / 4);
  return (nb + CZ_CHUNK - 1) / CZ_CHUNK;
}

/* upper bound of the compressed size in bytes */
uint64_t oracle_codec_bound(int64_t n0, int64_t n1) {
  const uint64_t nb = (uint64_t)((n0 + 3) / 4) * (uint64_t)((n1 + 3) / 4);
  const uint64_t nc = (uint64_t)nchunks(n0, n1);
  return CZ_HEADER + 16 * ((nc + 3) / 4) + 4 * (nb * CZ_BLOCK_MAX_BITS / 32);
}

/* Compress data [n0][n1] with absolute tolerance tol (> 0), or losslessly
 * (tol == 0).  Returns the byte count written to out (zeroed by the call;
 * capacity >= oracle_codec_bound), or 0 on bad arguments or, with tol > 0,
 * a non-finite value. */
uint64_t oracle_codec_compress(const float *data, int64_t n0, int64_t n1, double tol,
                               unsigned char *out, uint64_t capacity) {
  if (n0 < 1 || n1 < 1 || !(tol >= 0) || !isfinite(tol) || capacity < oracle_codec_bound(n0, n1))
    return 0;
  if (tol > 0)
    for (int64_t i = 0; i < n0 * n1; ++i)
      if (!isfinite(data[i])) return 0;
  memset(out, 0, capacity);
  const int64_t nb1 = (n1 + 3) / 4, nb = ((n0 + 3) / 4) * nb1, nc = nchunks(n0, n1);
  uint32_t *index = (uint32_t *)(out + CZ_HEADER);
  uint32_t *words = (uint32_t *)(out + CZ_HEADER + 16 * ((nc + 3) / 4));
  bitw bw = {words, 0};
  float x[16];
  for (int64_t b = 0; b < nb; ++b) {
    if (b % CZ_CHUNK == 0) {
      bw.pos = (bw.pos + 31) / 32 * 32; /* chunks start on a word */
      index[b / CZ_CHUNK] = (uint32_t)(bw.pos / 32);
    }
    gather_block(data, n0, n1, b / nb1, b % nb1, x);
    encode_block(x, tol, &bw);
  }
  const uint64_t nwords = (bw.pos + 31) / 32;
  const uint32_t head[4] = {0x5A4D5452u, 3u, tol > 0 ? 0u : 1u, CZ_CHUNK};
  const uint64_t tail[3] = {nwords, (uint64_t)nc, 0};
  memcpy(out + 0, head, 16);
  memcpy(out + 16, &n0, 8);
  memcpy(out + 24, &n1, 8);
  memcpy(out + 32, &tol, 8);
  memcpy(out + 40, tail, 24);
  return CZ_HEADER + 16 * ((uint64_t)(nc + 3) / 4) + 4 * nwords;
}

/* Decompress into data [n0][n1]; returns 0 on success, < 0 on a stream that
 * is malformed or does not match n0 x n1. */
int oracle_codec_decompress(const unsigned char *in, uint64_t nbytes, float *data, int64_t n0,
                            int64_t n1) {
  uint32_t head[4];
  int64_t m0, m1;
  double tol;
  uint64_t tail[2];
  if (nbytes < CZ_HEADER || n0 < 1 || n1 < 1) return -1;
  memcpy(head, in, 16);
  memcpy(&m0, in + 16, 8);
  memcpy(&m1, in + 24, 8);
  memcpy(&tol, in + 32, 8);
  memcpy(tail, in + 40, 16);
  const int64_t nb1 = (n1 + 3) / 4, nb = ((n0 + 3) / 4) * nb1, nc = nchunks(n0, n1);
  if (head[0] != 0x5A4D5452u || head[1] != 3u || head[3] != CZ_CHUNK || m0 != n0 || m1 != n1 ||
      tail[1] != (uint64_t)nc || (head[2] == 0) != (tol > 0) || head[2] > 1)
    return -2;
  const uint64_t start = CZ_HEADER + 16 * ((uint64_t)(nc + 3) / 4);
  if (start > nbytes || tail[0] > (nbytes - start) / 4) return -2;
  const uint32_t *index = (const uint32_t *)(in + CZ_HEADER);
  bitr br = {(const uint32_t *)(in + start), tail[0] * 32, 0, 0};
  float x[16];
  for (int64_t b = 0; b < nb; ++b) {
    if (b % CZ_CHUNK == 0) {
      br.pos = (br.pos + 31) / 32 * 32;
      if (index[b / CZ_CHUNK] != br.pos / 32) return -3;
    }
    if (decode_block(&br, tol, x)) return -3;
    const int64_t bi = b / nb1, bj = b % nb1;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        const int64_t i = 4 * bi + r, j = 4 * bj + c;
        if (i < n0 && j < n1) data[i * n1 + j] = x[4 * r + c];
      }
  }
  return (br.pos + 31) / 32 == tail[0] ? 0 : -3;
}
