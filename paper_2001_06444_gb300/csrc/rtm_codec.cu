// rtm_codec.cu — error-bounded compression of velocity models, images and
// seismograms on the device (§3, §4.2, Tables 1-2: a transform block codec
// used in fixed-accuracy and lossless modes between the workflow's stages).
//
// Stream of one array (little endian): a 64-byte header {u32 magic "RTMZ",
// u32 version 2, u32 mode (0 fixed accuracy, 1 lossless), u32 blocks per
// chunk (32), i64 n0, i64 n1, f64 tol, u64 words of the bit section, u64
// chunks, u64 0}; the u32 word offset of every chunk of 32 blocks (zero
// padded to a multiple of four entries); the bit section, u32 words, bits
// least significant first.  Each chunk starts on a word.
//
// Per 4 x 4 block (blocks row-major; edge blocks repeat their last row and
// column): a flag (0: all zero); fixed accuracy: 9 bits of e + 150 (block
// exponent, max |x| = f 2^e, f in [0.5, 1)), fixed point q = rint(x 2^(28-e));
// lossless: q = the float's bits as an order-preserving integer.  A
// two-level S-transform on rows then columns, coefficients in frequency
// order, magnitudes coded from plane 30 (lossless 32) down to kmin with
// prefix significance (a group test per plane, a scan to the next
// significant coefficient), then, per significant coefficient, its bits
// below the plane where it entered the prefix (lowest first) and its sign.
// kmin is the largest k >= 1 with 16 2^k + 21.5 <= tol 2^(28-e), else 0.
//
// Encoding: one warp per chunk, one lane per block.  Each lane computes its
// block's coded length in closed form (events of the plane scan are the
// suffix maxima of the coefficients' top planes), a warp scan places the
// blocks, the lanes write their bits into shared memory, and each tile of 8
// chunks finds its place in the output by a single-pass decoupled look-back
// over the tiles before it (dynamic tile order, so every wait is on a tile
// that is already running; each wait is bounded by the global timer).
// Decoding: one thread per chunk, the chunk index giving its start.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "rtm_engine.h"

namespace {

using u32 = uint32_t;
using u64 = unsigned long long;

constexpr int kP = 28;
constexpr int kChunk = 32;               // blocks per chunk = lanes of a warp
constexpr int kWarps = 8;                // chunks per tile
constexpr int kTile = kChunk * kWarps;   // blocks per tile (one CTA)
constexpr int kBlockWords = 20;          // 640 bits bound one coded block
constexpr int kHeader = 64;
constexpr u32 kMagic = 0x5A4D5452u;
constexpr int kTab = 288;                // kmin by e + 150, e in [-150, 137]
constexpr u64 kAgg = 1ull << 62, kIncl = 2ull << 62, kNonFinite = 1ull << 61,
              kPoison = 1ull << 60, kValMask = (1ull << 40) - 1;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

__host__ __device__ constexpr int perm(int i) {
  // coefficient (row*4 + col) in coding order: by lev(row) + lev(col),
  // lev = 0, 1, 2, 2
  return i == 0 ? 0 : i == 1 ? 1 : i == 2 ? 4 : i == 3 ? 2 : i == 4 ? 3 : i == 5 ? 5
       : i == 6 ? 8 : i == 7 ? 12 : i == 8 ? 6 : i == 9 ? 7 : i == 10 ? 9 : i == 11 ? 13
       : i == 12 ? 10 : i == 13 ? 11 : i == 14 ? 14 : 15;
}

struct EncArgs {
  const float *data;
  long long n0, n1, nb1, nb, tiles, nchunk;
  unsigned char *out;
  u64 stride, index_bytes;
  u64 *sizes;
  u64 *status;
  u64 *ticket;
  int *err;
  double tol;
};

struct DecArgs {
  const unsigned char *in;
  float *out;
  long long n0, n1, nb1, nb, nchunk;
  u64 stride, index_bytes;
  int *err;  // [0] malformed flag, [1] first malformed array
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// kmin for every block exponent of a tolerance: the largest k in [1, 30]
// with 16 2^k <= T - 21.5, T = tol 2^(28 - e), else 0.  T - 21.5 is exact
// for T < 2^52, and above that k is 30 whatever the rounding.
__device__ void fill_kmin(unsigned char *tab, double tol) {
  for (int i = threadIdx.x; i < kTab; i += blockDim.x) {
    const double r = ldexp(tol, kP - (i - 150)) - 21.5;
    const int k = r >= 32.0 ? ilogb(r) - 4 : 0;
    tab[i] = (unsigned char)min(k, 30);
  }
}

// rint(x 2^(28 - e)) from the float's bits, for |x| < 2^e
__device__ __forceinline__ int fixed_point(u32 bits, int e) {
  const u32 E = (bits >> 23) & 0xffu;
  const u32 M = (bits & 0x7fffffu) | (E ? 0x800000u : 0u);
  const int s = (E ? (int)E : 1) - 122 - e;  // x 2^(28-e) = M 2^s
  u32 q;
  if (s >= 0) {
    q = M << s;
  } else if (-s > 25) {
    q = 0;
  } else {
    const int r = -s;
    q = M >> r;
    const u32 rem = M & ((1u << r) - 1u), half = 1u << (r - 1);
    q += (rem > half) | ((rem == half) & (q & 1u));
  }
  return (bits >> 31) ? -(int)q : (int)q;
}

__device__ __forceinline__ u64 rne_shift(u64 a, int r) {
  if (r <= 0) return a;
  if (r >= 64) return 0;
  const u64 q = a >> r, rem = a & ((1ull << r) - 1ull), half = 1ull << (r - 1);
  return q + ((rem > half) | ((rem == half) & (q & 1ull)));
}

// q 2^(e - 28) rounded once to float (nearest, ties to even)
__device__ __forceinline__ float fixed_to_float(long long q, int e) {
  if (q == 0) return 0.0f;
  const u32 sign = q < 0 ? 0x80000000u : 0u;
  const u64 a = q < 0 ? (u64)(-q) : (u64)q;
  const int L = 63 - __clzll((long long)a);
  int X = L + e - kP;  // exponent of the leading bit
  u32 bits;
  if (X >= -126) {
    u64 mant = L <= 23 ? a << (23 - L) : rne_shift(a, L - 23);
    if (mant >> 24) {
      mant >>= 1;
      X++;
    }
    bits = X > 127 ? 0x7f800000u : ((u32)(X + 127) << 23) | ((u32)mant & 0x7fffffu);
  } else {
    const int sh = e - kP + 149;  // units of 2^-149
    bits = (u32)(sh >= 0 ? a << sh : rne_shift(a, -sh));
  }
  return __uint_as_float(bits | sign);
}

// ---------------------------------------------------------------- encode --

// Magnitudes and signs of one block's coefficients in coding order, its
// coded length, and what emission needs.
template <bool LL>
struct Coded {
  using U = typename std::conditional<LL, u64, u32>::type;
  U m[16];
  u32 neg = 0;   // bit i: coefficient i negative
  int top[16];   // highest set plane, -1 for zero
  int s[16];     // plane at which coefficient i entered the prefix
  int kmin = 0, e = 0, cur = 0, len = 1;
  bool zero = true, nonfinite = false;
};

template <bool LL>
__device__ __forceinline__ void analyse(const float (&x)[16], const unsigned char *ktab,
                                        Coded<LL> &c) {
  constexpr int Ktop = LL ? 32 : 30;
  u32 bits[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) bits[i] = __float_as_uint(x[i]);
  using S = typename std::conditional<LL, long long, int>::type;
  S q[16];
  if (LL) {
    u32 any = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      any |= bits[i];
      q[i] = (bits[i] >> 31) ? (S)(-1ll - (long long)(bits[i] & 0x7fffffffu)) : (S)bits[i];
    }
    if (!any) return;
  } else {
    u32 mx = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) mx = max(mx, bits[i] & 0x7fffffffu);
    if (!mx) return;
    c.nonfinite = mx >= 0x7f800000u;
    const u32 E = mx >> 23;
    c.e = E ? (int)E - 126 : (31 - __clz(mx)) - 148;
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = fixed_point(bits[i], c.e);
    c.kmin = ktab[c.e + 150];
  }
  c.zero = false;
  // two-level S-transform: rows, then columns (floor(d/2) = d >> 1)
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int o = pass ? l : 4 * l, st = pass ? 4 : 1;
      const S a = q[o], b = q[o + st], cc = q[o + 2 * st], d = q[o + 3 * st];
      const S d1 = b - a, s1 = a + (d1 >> 1);
      const S d2 = d - cc, s2 = cc + (d2 >> 1);
      const S dd = s2 - s1, ss = s1 + (dd >> 1);
      q[o] = ss;
      q[o + st] = dd;
      q[o + 2 * st] = d1;
      q[o + 3 * st] = d2;
    }
  }
  int sfx = -1;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const S v = q[perm(i)];
    c.neg |= (v < 0 ? 1u : 0u) << i;
    c.m[i] = (typename Coded<LL>::U)(v < 0 ? -v : v);
    if (LL)
      c.top[i] = c.m[i] ? 63 - __clzll((long long)c.m[i]) : -1;
    else
      c.top[i] = c.m[i] ? 31 - __clz((int)c.m[i]) : -1;
  }
#pragma unroll
  for (int i = 15; i >= 0; --i) {
    sfx = max(sfx, c.top[i]);
    c.s[i] = sfx;
  }
  // prefix members: s >= kmin; events (found coefficients): top == s
  int cur = 0, nev = 0, refine = 0, plast = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (c.s[i] >= c.kmin) {
      cur = i + 1;
      plast = c.s[i];
      nev += c.top[i] == c.s[i];
      refine += c.s[i] - c.kmin + ((c.m[i] >> c.kmin) != 0);
    }
  }
  c.cur = cur;
  int sig;
  if (cur == 0) {
    sig = Ktop - c.kmin + 1;
  } else {
    sig = nev + cur + (Ktop - plast) + (cur < 16 ? plast - c.kmin + 1 : 0);
  }
  c.len = 1 + (LL ? 0 : 9) + sig + refine;
}

__device__ __forceinline__ void put(u32 *buf, u32 pos, u64 v) {
  if (!v) return;
  const u64 x = v << (pos & 31);
  atomicOr(buf + (pos >> 5), (u32)x);
  if (x >> 32) atomicOr(buf + (pos >> 5) + 1, (u32)(x >> 32));
}

template <bool LL>
__device__ __forceinline__ void emit(const Coded<LL> &c, u32 *buf, u32 pos) {
  constexpr int Ktop = LL ? 32 : 30;
  if (c.zero) return;  // the flag bit is 0
  put(buf, pos, 1);
  pos += 1;
  if (!LL) {
    put(buf, pos, (u64)(c.e + 150));
    pos += 9;
  }
  int k = Ktop, nxt = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (c.s[i] >= c.kmin && c.top[i] == c.s[i]) {
      pos += k - c.s[i];   // failed group tests of the planes in between
      put(buf, pos, 1);    // group test succeeds
      pos += 1 + (i - nxt);  // scanned coefficients without the bit
      put(buf, pos, 1);    // the coefficient found
      pos += 1;
      nxt = i + 1;
      k = c.s[i];
    }
  }
  if (c.cur < 16) pos += k - c.kmin + 1;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i < c.cur) {
      const int w = c.s[i] - c.kmin;
      const u64 t = (u64)(c.m[i] >> c.kmin);
      put(buf, pos, t & ((1ull << w) - 1ull));
      pos += w;
      if (t) {
        put(buf, pos, (c.neg >> i) & 1u);
        pos += 1;
      }
    }
  }
}

template <bool LL>
__global__ void __launch_bounds__(kTile) k_cz_encode(const EncArgs a) {
  __shared__ u32 sbuf[kWarps][kChunk * kBlockWords];
  __shared__ u32 s_words[kWarps];
  __shared__ unsigned char s_kmin[kTab];
  __shared__ u64 s_tile, s_prefix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(a.ticket, 1ull);
  if (!LL) fill_kmin(s_kmin, a.tol);
  __syncthreads();
  const long long T = (long long)s_tile;
  const long long arr = T / a.tiles, lt = T % a.tiles;
  const long long b = lt * kTile + threadIdx.x;
  const float *src = a.data + arr * a.n0 * a.n1;

  Coded<LL> c;
  if (b < a.nb) {
    const long long bi = b / a.nb1, bj = b % a.nb1;
    float x[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float *row = src + min(4 * bi + r, a.n0 - 1) * a.n1;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) x[4 * r + cc] = row[min(4 * bj + cc, a.n1 - 1)];
    }
    analyse<LL>(x, s_kmin, c);
  } else {
    c.len = 0;
  }
  // place the blocks of this chunk
  int incl = c.len;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const int chunk_bits = __shfl_sync(0xffffffffu, incl, 31);
  const u32 nw = (u32)(chunk_bits + 31) >> 5;
  u32 *buf = sbuf[warp];
  for (u32 i = lane; i < nw; i += 32) buf[i] = 0;
  __syncwarp();
  if (c.len) emit<LL>(c, buf, (u32)(incl - c.len));
  __syncwarp();
  if (lane == 0) s_words[warp] = nw;
  const int nf = __syncthreads_or(c.nonfinite);

  // words before this tile: decoupled look-back over the array's tiles
  if (warp == 0) {
    u32 agg = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) agg += s_words[w];
    const u64 mine = (u64)agg | (nf ? kNonFinite : 0ull);
    volatile u64 *st = a.status + arr * a.tiles;
    if (lane == 0) st[lt] = (lt == 0 ? kIncl : kAgg) | mine;
    u64 prefix = 0, flags = 0;
    if (lt > 0) {
      long long j = lt - 1;
      const unsigned long long t0 = now_ns();
      for (;;) {
        const long long idx = j - lane;
        const u64 s = idx >= 0 ? (u64)st[idx] : (u64)kIncl;
        const u32 notready = __ballot_sync(0xffffffffu, (s >> 62) == 0);
        const u32 inc = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        const u32 need = inc ? (u32)(((u64)(inc & (0u - inc)) << 1) - 1ull) : 0xffffffffu;
        if (notready & need) {
          if (now_ns() - t0 > kWaitNs) {
            flags |= kPoison;
            if (lane == 0) atomicExch(a.err, 1);
            break;
          }
          continue;
        }
        const bool use = (need >> lane) & 1u;
        u64 v = use ? (s & kValMask) : 0ull, f = use ? (s & (kNonFinite | kPoison)) : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          v += __shfl_xor_sync(0xffffffffu, v, d);
          f |= __shfl_xor_sync(0xffffffffu, f, d);
        }
        prefix += v;
        flags |= f;
        if (inc) break;
        j -= 32;
      }
      if (lane == 0) st[lt] = kIncl | ((prefix + agg) & kValMask) | flags | (mine & kNonFinite);
    }
    if (lane == 0) s_prefix = prefix | (flags & ~kValMask) | (mine & kNonFinite);
  }
  __syncthreads();
  const u64 pre = s_prefix;
  if (pre & kPoison) return;  // a wait gave up: nothing is written
  unsigned char *slot = a.out + arr * a.stride;
  u32 *index = reinterpret_cast<u32 *>(slot + kHeader);
  u32 *words = reinterpret_cast<u32 *>(slot + kHeader + a.index_bytes);
  u64 start = pre & kValMask;
  for (int w = 0; w < warp; ++w) start += s_words[w];
  const long long chunk = lt * kWarps + warp;
  if (chunk < a.nchunk) {
    if (lane == 0) index[chunk] = (u32)start;
    for (u32 i = lane; i < nw; i += 32) words[start + i] = buf[i];
  }
  if (lt == a.tiles - 1 && threadIdx.x == 0) {
    u64 total = start;
    for (int w = warp; w < kWarps; ++w) total += s_words[w];
    const bool bad = (pre & kNonFinite) && !LL;
    for (long long i = a.nchunk; i < (long long)(a.index_bytes / 4); ++i) index[i] = 0;
    u32 *h = reinterpret_cast<u32 *>(slot);
    h[0] = bad ? 0u : kMagic;
    h[1] = 2u;
    h[2] = LL ? 1u : 0u;
    h[3] = kChunk;
    long long *hl = reinterpret_cast<long long *>(slot + 16);
    hl[0] = a.n0;
    hl[1] = a.n1;
    *reinterpret_cast<double *>(slot + 32) = LL ? 0.0 : a.tol;
    u64 *hu = reinterpret_cast<u64 *>(slot + 40);
    hu[0] = total;
    hu[1] = (u64)a.nchunk;
    hu[2] = 0;
    a.sizes[arr] = bad ? 0ull : kHeader + a.index_bytes + 4 * total;
  }
}

// ---------------------------------------------------------------- decode --

struct Reader {
  const u32 *w;
  u64 nw, widx, pos, end;
  u64 buf;
  int avail;
  __device__ void init(const u32 *words, u64 nwords, u64 start) {
    w = words;
    nw = nwords;
    widx = start;
    pos = start * 32;
    end = nwords * 32;
    buf = 0;
    avail = 0;
    refill();
  }
  __device__ __forceinline__ void refill() {
    while (avail <= 32) {
      const u32 v = widx < nw ? __ldg(w + widx) : 0u;
      buf |= (u64)v << avail;
      avail += 32;
      widx++;
    }
  }
  __device__ __forceinline__ void skip(int n) {  // n <= 32
    buf >>= n;
    avail -= n;
    pos += n;
    refill();
  }
  __device__ __forceinline__ u32 get(int n) {  // n <= 32
    const u32 v = n ? (u32)buf & (0xffffffffu >> (32 - n)) : 0u;
    skip(n);
    return v;
  }
  // zero bits before the next one, at most lim (which are consumed)
  __device__ __forceinline__ int zeros(int lim) {
    int z = 0;
    while (z < lim) {
      const u32 v = (u32)buf;
      int c = v ? __ffs(v) - 1 : 32;
      c = min(c, lim - z);
      skip(c);
      z += c;
      if (c < 32) break;
    }
    return z;
  }
  __device__ bool overrun() const { return pos > end; }
};

template <bool LL>
__device__ __forceinline__ bool decode_block(Reader &rd, const unsigned char *ktab,
                                             unsigned char *sfx, float (&x)[16]) {
  constexpr int Ktop = LL ? 32 : 30;
  if (!rd.get(1)) {
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = 0.0f;
    return true;
  }
  int e = 0, kmin = 0;
  if (!LL) {
    const int eb = (int)rd.get(9);
    if (eb >= kTab) return false;
    e = eb - 150;
    kmin = ktab[eb];
  }
  // significance section
  u32 found = 0;
  int n = 0, k = Ktop;
  while (k >= kmin && n < 16) {
    const int lim = k - kmin + 1;
    const int z = rd.zeros(lim);  // failed group tests
    if (z == lim) break;
    k -= z;
    rd.skip(1);  // the group test that succeeds
    const int g = rd.zeros(16 - n);
    if (g == 16 - n) return false;
    rd.skip(1);
    const int p = n + g;
    for (int i = n; i <= p; ++i) sfx[i * blockDim.x] = (unsigned char)k;
    found |= 1u << p;
    n = p + 1;
  }
  // refinement: magnitudes and signs, back in block order
  using S = long long;
  S q[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    S v = 0;
    if (i < n) {
      const int w = sfx[i * blockDim.x] - kmin;
      u64 t = w > 32 ? 0ull : (u64)rd.get(min(w, 32));
      if ((found >> i) & 1u) t |= 1ull << w;
      if (t) {
        const bool ng = rd.get(1);
        v = (S)((t << kmin) + (kmin > 0 ? (1ull << (kmin - 1)) : 0ull));
        if (ng) v = -v;
      }
    }
    q[perm(i)] = v;
  }
  // inverse transform: columns, then rows
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int o = pass ? 4 * l : l, st = pass ? 1 : 4;
      const S ss = q[o], dd = q[o + st], d1 = q[o + 2 * st], d2 = q[o + 3 * st];
      const S s1 = ss - (dd >> 1), s2 = dd + s1;
      const S a0 = s1 - (d1 >> 1), b0 = d1 + a0;
      const S c0 = s2 - (d2 >> 1), e0 = d2 + c0;
      q[o] = a0;
      q[o + st] = b0;
      q[o + 2 * st] = c0;
      q[o + 3 * st] = e0;
    }
  }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (LL) {
      ok &= q[i] >= -2147483648ll && q[i] <= 2147483647ll;
      const u32 u = q[i] < 0 ? 0x80000000u | (u32)(-1ll - q[i]) : (u32)q[i];
      x[i] = __uint_as_float(u);
    } else {
      x[i] = fixed_to_float(q[i], e);
    }
  }
  return ok;
}

template <bool LL>
__device__ void decode_chunk(const DecArgs &a, const unsigned char *slot, long long arr,
                             const unsigned char *ktab, unsigned char *sfx) {
  const long long ch = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= a.nchunk) return;
  const u64 nwords = *reinterpret_cast<const u64 *>(slot + 40);
  const u32 *index = reinterpret_cast<const u32 *>(slot + kHeader);
  const u32 *words = reinterpret_cast<const u32 *>(slot + kHeader + a.index_bytes);
  const u64 start = index[ch];
  const u64 next = ch + 1 < a.nchunk ? (u64)index[ch + 1] : nwords;
  bool ok = start <= next && next <= nwords && (ch > 0 || start == 0);
  float *dst = a.out + arr * a.n0 * a.n1;
  if (ok) {
    Reader rd;
    rd.init(words, next, start);
    const long long b0 = ch * kChunk, b1 = min(b0 + kChunk, a.nb);
    for (long long b = b0; b < b1 && ok; ++b) {
      float x[16];
      ok = decode_block<LL>(rd, ktab, sfx, x);
      const long long bi = b / a.nb1, bj = b % a.nb1;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long i = 4 * bi + r;
        if (i < a.n0) {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const long long j = 4 * bj + cc;
            if (j < a.n1) dst[i * a.n1 + j] = x[4 * r + cc];
          }
        }
      }
    }
    ok = ok && !rd.overrun() && (rd.pos + 31) / 32 == next;
  }
  if (!ok) {
    atomicExch(a.err, 1);
    atomicMin(a.err + 1, (int)arr);
  }
}

__global__ void __launch_bounds__(128) k_cz_decode(const DecArgs a) {
  __shared__ unsigned char s_kmin[kTab];
  __shared__ unsigned char s_sfx[16 * 128];
  __shared__ int s_ok;
  const long long arr = blockIdx.y;
  const unsigned char *slot = a.in + arr * a.stride;
  if (threadIdx.x == 0) {
    const u32 *h = reinterpret_cast<const u32 *>(slot);
    const long long *hl = reinterpret_cast<const long long *>(slot + 16);
    const u64 *hu = reinterpret_cast<const u64 *>(slot + 40);
    const double tol = *reinterpret_cast<const double *>(slot + 32);
    const u64 cap = (a.stride - kHeader - a.index_bytes) / 4;
    s_ok = h[0] == kMagic && h[1] == 2u && h[2] <= 1u && h[3] == (u32)kChunk &&
           hl[0] == a.n0 && hl[1] == a.n1 && hu[1] == (u64)a.nchunk && hu[0] <= cap &&
           (h[2] ? tol == 0.0 : (tol > 0.0 && tol < 1e300));
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
      atomicExch(a.err, 1);
      atomicMin(a.err + 1, (int)arr);
    }
    return;
  }
  const double tol = *reinterpret_cast<const double *>(slot + 32);
  const int mode = reinterpret_cast<const u32 *>(slot)[2];
  if (!mode) fill_kmin(s_kmin, tol);
  __syncthreads();
  if (mode)
    decode_chunk<true>(a, slot, arr, s_kmin, s_sfx + threadIdx.x);
  else
    decode_chunk<false>(a, slot, arr, s_kmin, s_sfx + threadIdx.x);
}

}  // namespace

namespace rtm {

bool codec_shape(long long n0, long long n1, long long *nb1, long long *nb, long long *nchunk,
                 u64 *index_bytes, u64 *bound) {
  if (n0 < 1 || n1 < 1 || n0 > (1ll << 40) || n1 > (1ll << 40)) return false;
  const long long b1 = (n1 + 3) / 4, b0 = (n0 + 3) / 4;
  if (b0 > (1ll << 31) / b1) return false;
  const long long n = b0 * b1;
  if ((u64)n * kBlockWords >= (1ull << 32)) return false;  // word offsets are u32
  const long long nc = (n + kChunk - 1) / kChunk;
  const u64 ib = 16ull * (u64)((nc + 3) / 4);
  if (nb1) *nb1 = b1;
  if (nb) *nb = n;
  if (nchunk) *nchunk = nc;
  if (index_bytes) *index_bytes = ib;
  if (bound) *bound = kHeader + ib + 4ull * kBlockWords * (u64)n;
  return true;
}

cudaError_t launch_cz_encode(const float *data, long long count, long long n0, long long n1,
                             double tol, unsigned char *out, u64 stride, u64 *sizes, u64 *scratch,
                             int *err, cudaStream_t st) {
  EncArgs a{};
  u64 bound = 0;
  if (!codec_shape(n0, n1, &a.nb1, &a.nb, &a.nchunk, &a.index_bytes, &bound))
    return cudaErrorInvalidValue;
  a.data = data;
  a.n0 = n0;
  a.n1 = n1;
  a.tiles = (a.nb + kTile - 1) / kTile;
  a.out = out;
  a.stride = stride;
  a.sizes = sizes;
  a.ticket = scratch;
  a.status = scratch + 1;
  a.err = err;
  a.tol = tol;
  const long long grid = count * a.tiles;
  if (grid > 0x7fffffffll) return cudaErrorInvalidValue;
  if (tol > 0)
    k_cz_encode<false><<<(unsigned)grid, kTile, 0, st>>>(a);
  else
    k_cz_encode<true><<<(unsigned)grid, kTile, 0, st>>>(a);
  return cudaGetLastError();
}

u64 codec_scratch_words(long long count, long long n0, long long n1) {
  long long nb = 0;
  if (!codec_shape(n0, n1, nullptr, &nb, nullptr, nullptr, nullptr)) return 0;
  return 1 + (u64)count * (u64)((nb + kTile - 1) / kTile);
}

cudaError_t launch_cz_decode(const unsigned char *in, u64 stride, long long count, long long n0,
                             long long n1, float *out, int *err, cudaStream_t st) {
  DecArgs a{};
  if (!codec_shape(n0, n1, &a.nb1, &a.nb, &a.nchunk, &a.index_bytes, nullptr))
    return cudaErrorInvalidValue;
  a.in = in;
  a.out = out;
  a.n0 = n0;
  a.n1 = n1;
  a.stride = stride;
  a.err = err;
  if (count > 65535 || (a.nchunk + 127) / 128 > 0x7fffffffll) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((a.nchunk + 127) / 128), (unsigned)count);
  k_cz_decode<<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rtm

// ------------------------------------------------------------------ ABI --

using namespace rtm;

namespace {

#define CZ_CU(x)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

// Device time of one codec launch, recorded while profiling is on.
struct CodecTimer {
  rtm_ctx *ctx;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CodecTimer(rtm_ctx *c, cudaStream_t s) : ctx(c), st(s) {
    if (ctx->prof && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      e0 = e1 = nullptr;
  }
  ~CodecTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  void start() {
    if (e0) cudaEventRecord(e0, st);
  }
  void stop() {
    if (e1) cudaEventRecord(e1, st);
  }
  // after the stream was synchronised
  void account(double bytes) {
    float ms = 0.f;
    if (e0 && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 0.f;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats.launches += 1;
    if (e0) {
      ctx->stats.codec_launches += 1;
      ctx->stats.codec_ms += ms;
      ctx->stats.codec_bytes += bytes;
    }
  }
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

uint64_t rtm_compress_bound(long long n0, long long n1) {
  u64 b = 0;
  return codec_shape(n0, n1, nullptr, nullptr, nullptr, nullptr, &b) ? b : 0;
}

int rtm_compress(rtm_ctx *ctx, const float *data, long long count, long long n0, long long n1,
                 double tol, void *out, uint64_t out_stride, uint64_t *out_bytes,
                 void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  if (!data || !out || !out_bytes) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  u64 bound = 0;
  if (!codec_shape(n0, n1, nullptr, nullptr, nullptr, nullptr, &bound))
    return fail(ctx, RTM_ERR_ARG, "unsupported shape %lld x %lld", n0, n1);
  if (count < 1 || !(tol >= 0) || !std::isfinite(tol) || tol > 1e300)
    return fail(ctx, RTM_ERR_ARG, "need count >= 1 and a finite tol >= 0");
  if (out_stride < bound || out_stride % 16 || !aligned16(out))
    return fail(ctx, RTM_ERR_ARG, "out_stride %llu must be >= %llu and a multiple of 16, out "
                "16-byte aligned", (unsigned long long)out_stride, bound);
  if ((u64)count > ~0ull / out_stride) return fail(ctx, RTM_ERR_ARG, "count * out_stride overflows");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "cudaSetDevice");
  if (is_device_ptr(out_bytes)) return fail(ctx, RTM_ERR_ARG, "out_bytes must be host memory");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nbytes_in = (size_t)count * n0 * n1 * 4;
  DevBuf din, dout, scratch;
  const float *d_data = data;
  if (!is_device_ptr(data)) {
    CZ_CU(din.alloc(ctx, nbytes_in, st));
    CZ_CU(cudaMemcpyAsync(din.p, data, nbytes_in, cudaMemcpyHostToDevice, st));
    d_data = din.as<float>();
  }
  const bool out_dev = is_device_ptr(out);
  unsigned char *d_out = static_cast<unsigned char *>(out);
  if (!out_dev) {
    CZ_CU(dout.alloc(ctx, (size_t)count * out_stride, st));
    d_out = dout.as<unsigned char>();
  }
  const u64 nw = codec_scratch_words(count, n0, n1);
  const size_t sbytes = nw * 8 + (size_t)count * 8 + 16;
  CZ_CU(scratch.alloc(ctx, sbytes, st));
  CZ_CU(cudaMemsetAsync(scratch.p, 0, sbytes, st));
  u64 *ticket = scratch.as<u64>();
  u64 *sizes = ticket + nw;
  int *err = reinterpret_cast<int *>(sizes + count);
  CodecTimer tm(ctx, st);
  tm.start();
  CZ_CU(launch_cz_encode(d_data, count, n0, n1, tol, d_out, out_stride, sizes, ticket, err, st));
  tm.stop();
  int herr = 0;
  CZ_CU(cudaMemcpyAsync(out_bytes, sizes, (size_t)count * 8, cudaMemcpyDeviceToHost, st));
  CZ_CU(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  CZ_CU(cudaStreamSynchronize(st));
  double total = 0;
  long long bad = 0, first_bad = -1;
  for (long long i = 0; i < count; ++i) {
    total += (double)out_bytes[i];
    if (!out_bytes[i] && first_bad < 0) first_bad = i;
    bad += !out_bytes[i];
  }
  tm.account((double)nbytes_in + total);
  if (herr) {
    for (long long i = 0; i < count; ++i) out_bytes[i] = 0;
    return fail(ctx, RTM_ERR_TIMEOUT, "a device-side wait of the encoder gave up");
  }
  if (!out_dev) {
    for (long long i = 0; i < count; ++i)
      if (out_bytes[i])
        CZ_CU(cudaMemcpyAsync(static_cast<unsigned char *>(out) + i * out_stride,
                              d_out + i * out_stride, out_bytes[i], cudaMemcpyDeviceToHost, st));
    CZ_CU(cudaStreamSynchronize(st));
  }
  if (bad)
    return fail(ctx, RTM_ERR_ARG, "%lld array(s) hold a NaN or an infinity (first: %lld); use tol "
                "= 0 (lossless) for them", bad, first_bad);
  return RTM_OK;
}

int rtm_decompress(rtm_ctx *ctx, const void *in, uint64_t in_stride, long long count,
                   long long n0, long long n1, float *data, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  if (!in || !data) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  u64 ib = 0;
  if (!codec_shape(n0, n1, nullptr, nullptr, nullptr, &ib, nullptr))
    return fail(ctx, RTM_ERR_ARG, "unsupported shape %lld x %lld", n0, n1);
  if (count < 1 || count > 65535) return fail(ctx, RTM_ERR_ARG, "need 1 <= count <= 65535");
  if (in_stride < kHeader + ib || in_stride % 16 || !aligned16(in))
    return fail(ctx, RTM_ERR_ARG, "in_stride %llu must be >= %llu and a multiple of 16, in "
                "16-byte aligned", (unsigned long long)in_stride, kHeader + ib);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nbytes_out = (size_t)count * n0 * n1 * 4;
  DevBuf din, dout, scratch;
  const unsigned char *d_in = static_cast<const unsigned char *>(in);
  if (!is_device_ptr(in)) {
    CZ_CU(din.alloc(ctx, (size_t)count * in_stride, st));
    CZ_CU(cudaMemcpyAsync(din.p, in, (size_t)count * in_stride, cudaMemcpyHostToDevice, st));
    d_in = din.as<unsigned char>();
  }
  const bool out_dev = is_device_ptr(data);
  float *d_data = data;
  if (!out_dev) {
    CZ_CU(dout.alloc(ctx, nbytes_out, st));
    d_data = dout.as<float>();
  }
  CZ_CU(scratch.alloc(ctx, 16, st));
  const int init[4] = {0, 0x7fffffff, 0, 0};
  CZ_CU(cudaMemcpyAsync(scratch.p, init, 16, cudaMemcpyHostToDevice, st));
  CodecTimer tm(ctx, st);
  tm.start();
  CZ_CU(launch_cz_decode(d_in, in_stride, count, n0, n1, d_data, scratch.as<int>(), st));
  tm.stop();
  int herr[2] = {0, 0};
  CZ_CU(cudaMemcpyAsync(herr, scratch.p, 8, cudaMemcpyDeviceToHost, st));
  if (!out_dev) CZ_CU(cudaMemcpyAsync(data, d_data, nbytes_out, cudaMemcpyDeviceToHost, st));
  CZ_CU(cudaStreamSynchronize(st));
  double sbytes = 0;  // stream bytes read: header, index and words of every stream
  if (ctx->prof) {
    std::vector<u64> words((size_t)count);
    for (long long i = 0; i < count; ++i)
      CZ_CU(cudaMemcpyAsync(&words[i], d_in + i * in_stride + 40, 8, cudaMemcpyDeviceToHost, st));
    CZ_CU(cudaStreamSynchronize(st));
    for (u64 w : words) sbytes += (double)(kHeader + ib + 4 * w);
  }
  tm.account((double)nbytes_out + sbytes);
  if (herr[0])
    return fail(ctx, RTM_ERR_ARG, "stream %d is malformed or was not made for %lld x %lld", herr[1],
                n0, n1);
  return RTM_OK;
}

}  // extern "C"
