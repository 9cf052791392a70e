// rtm_codec.cu — error-bounded compression of velocity models, images and
// seismograms on the device (§3, §4.2, Tables 1-2: a transform block codec
// used in fixed-accuracy and lossless modes between the workflow's stages).
//
// Stream of one array (little endian): a 64-byte header {u32 magic "RTMZ",
// u32 version 3, u32 mode (0 fixed accuracy, 1 lossless), u32 blocks per
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
// below the plane where it entered the prefix (lowest first) and a sign bit
// (0 when its kept magnitude is zero): the significance section alone fixes
// the length of the refinement section.
// kmin is the largest k >= 1 with 16 2^k + 21.5 <= tol 2^(28-e), else 0.
//
// Encoding, in three passes with no device-side waiting:
//   1. one CTA per tile of 128 blocks (4 chunks), one warp per chunk, one lane
//      per block.  Each lane computes its block's coded length in closed form
//      (the events of the plane scan are the suffix maxima of the
//      coefficients' top planes), a warp scan places the blocks, the lanes
//      write their bits into shared memory, and the tile is copied to a
//      staging slot of the maximum tile size;
//   2. per array, an exclusive scan of the tiles' word counts, the header and
//      the stream's byte count;
//   3. one CTA per tile copies its words to their offset and writes the
//      offsets of its chunks.
// Decoding, per group of arrays, in two passes with no device-side waiting:
//   1. the walk: one thread per chunk (a CTA's chunks ordered by size first)
//      finds the bit offset and the cost class (events, members) of every
//      block; the CTA lists its blocks that are not all zero in class order
//      (a segment of the decode's list) and writes its all-zero blocks to
//      the output, row by row;
//   2. the decode: a CTA per segment, one block per thread in list order,
//      so that the lanes of a warp run the same loops for as many trips.
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
constexpr int kWarps = 4;                // chunks per encoder tile
constexpr int kTile = kChunk * kWarps;   // blocks per encoder tile (one CTA)
constexpr int kBlockWords = 20;          // 640 bits bound one coded block
constexpr int kChunkWords = kChunk * kBlockWords;
constexpr int kTileWords = kTile * kBlockWords;
constexpr int kWalk = 128;               // decoder's walk: chunks per CTA, one per thread
constexpr int kWalkKeys = 64;            // size classes the walk orders chunks by
constexpr int kSeg = kWalk * kChunk;     // blocks of a walk CTA: a segment of the decode's list
constexpr int kClasses = 256;            // decode cost classes (0: all-zero blocks)
constexpr int kDec = 256;                // decoder: threads per CTA, one block per thread
constexpr u64 kGroupBlocks = 1ull << 24; // list entries per group of arrays
static_assert(kClasses % kWalk == 0 && kWalk % 32 == 0 && kWalk >= 64,
              "class counts spread evenly over the walk threads");
static_assert(kSeg <= (1 << 13), "a segment's block index takes 13 bits of a list entry");
constexpr int kHeader = 64;
constexpr u32 kMagic = 0x5A4D5452u;
constexpr u32 kVersion = 3;
constexpr int kTab = 288;                // kmin by e + 150, e in [-150, 137]

__host__ __device__ constexpr int perm(int i) {
  // coefficient (row*4 + col) in coding order: by lev(row) + lev(col),
  // lev = 0, 1, 2, 2
  return i == 0 ? 0 : i == 1 ? 1 : i == 2 ? 4 : i == 3 ? 2 : i == 4 ? 3 : i == 5 ? 5
       : i == 6 ? 8 : i == 7 ? 12 : i == 8 ? 6 : i == 9 ? 7 : i == 10 ? 9 : i == 11 ? 13
       : i == 12 ? 10 : i == 13 ? 11 : i == 14 ? 14 : 15;
}

// perm(i) for a run-time i: the 16 values as nibbles of one constant
constexpr u64 kPermPack = 0xfebad976c8532410ull;
__host__ __device__ constexpr bool perm_pack_ok(int i = 0) {
  return i == 16 || ((int)((kPermPack >> (4 * i)) & 15u) == perm(i) && perm_pack_ok(i + 1));
}
static_assert(perm_pack_ok(), "packed coefficient order");
__device__ __forceinline__ int perm_rt(int i) { return (int)((kPermPack >> (4 * i)) & 15u); }

struct EncArgs {
  const float *data;
  long long n0, n1;
  u32 nb1, nb, tiles, nchunk;
  unsigned char *out;
  u64 stride, index_bytes;
  u64 *sizes;             // [count] stream bytes
  u32 *stage;             // [count * tiles][kTileWords] coded tiles
  u32 *chunk_words;       // [count * tiles][kWarps]
  u64 *tile_off;          // [count * tiles] word offset of each tile
  u32 *nonfinite;         // [count] array holds a NaN or an infinity
  const unsigned char *kmin;  // [kTab]
  double tol;
};

struct DecArgs {
  const unsigned char *in;
  float *out;
  long long n0, n1;
  u32 nb1, nb, nchunk;
  u64 stride, index_bytes;
  const unsigned char *kmin;  // [count][kTab]
  int *err;  // [0] malformed flag, [1] first malformed array
  u32 arr0;       // first array of this group (error reports)
  u32 count;      // arrays in this group
  u32 nseg;       // segments (kWalk chunks, kSeg blocks) per array
  u32 *list;      // [count][nseg][kSeg] per segment: its blocks not all zero, in class
                  // order: index in the segment << 15 | bit offset in the chunk
  u32 *segcount;  // [count][nseg] entries of each segment's list
};

// kmin for every block exponent of a tolerance: the largest k in [1, 30]
// with 16 2^k <= T - 21.5, T = tol 2^(28 - e), else 0.  T - 21.5 is exact
// for T < 2^52, and above that k is 30 whatever the rounding.  One CTA per
// array, one thread per exponent; the tolerance comes from the stream header
// (decoding) or from tol (encoding, in == nullptr).
__global__ void k_cz_kmin(const unsigned char *in, u64 stride, double tol, unsigned char *tab) {
  if (in) tol = *reinterpret_cast<const double *>(in + blockIdx.x * stride + 32);
  const int i = threadIdx.x;
  if (i >= kTab) return;
  int k = 0;
  if (tol > 0.0 && tol < 1e300) {
    const double r = ldexp(tol, kP - (i - 150)) - 21.5;
    k = r >= 32.0 ? ilogb(r) - 4 : 0;
  }
  tab[blockIdx.x * kTab + i] = (unsigned char)min(k, 30);
}

// rint(x 2^(28 - e)) from the float's bits, for |x| < 2^e (any e)
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

// q 2^(e - 28) rounded once to float (nearest, ties to even), any e
__device__ __forceinline__ float fixed_to_float_slow(long long q, int e) {
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

// Bits appended at a running position of a zeroed shared-memory chunk: a
// 64-bit accumulator whose whole words are OR-ed into place (the first and
// last word of a block are shared with its neighbours).
struct BitWriter {
  u32 *buf;
  u32 w;
  int n;
  u64 acc;
  __device__ __forceinline__ BitWriter(u32 *b, u32 pos) : buf(b), w(pos >> 5), n(pos & 31), acc(0) {}
  // v < 2^k, k <= 32
  __device__ __forceinline__ void put(u64 v, int k) {
    acc |= v << n;
    n += k;
    if (n >= 32) {
      if ((u32)acc) atomicOr(buf + w, (u32)acc);
      acc >>= 32;
      n -= 32;
      w++;
    }
  }
  __device__ __forceinline__ void flush() {
    if ((u32)acc) atomicOr(buf + w, (u32)acc);
  }
};

// One block: analysis (coded length) and emission.
template <bool LL>
struct Block {
  using S = typename std::conditional<LL, long long, int>::type;
  using U = typename std::conditional<LL, u64, u32>::type;
  static constexpr int Ktop = LL ? 32 : 30;
  U m[16];
  int s[16];      // plane at which coefficient i entered the prefix
  u32 neg = 0;    // bit i: coefficient i negative
  u32 ev = 0;     // bit i: coefficient i found by a scan (its top plane is s[i])
  u32 nz = 0;     // bit i: kept magnitude of coefficient i is not zero
  int kmin = 0, e = 0, cur = 0, len = 1;
  bool zero = true, nonfinite = false;

  __device__ __forceinline__ void analyse(const u32 (&bits)[16], const unsigned char *ktab) {
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
      nonfinite = mx >= 0x7f800000u;
      const u32 E = mx >> 23;
      e = E ? (int)E - 126 : (31 - __clz(mx)) - 148;
      kmin = ktab[e + 150];
      if (nonfinite) {
#pragma unroll
        for (int i = 0; i < 16; ++i) q[i] = 0;  // refused later; keep the length bounded
      } else if (e >= -99) {
        // x 2^(28-e) is exact (or below 1/2 when it underflows), 2^(28-e) a float
        const float scale = __uint_as_float((u32)(28 - e + 127) << 23);
#pragma unroll
        for (int i = 0; i < 16; ++i) q[i] = __float2int_rn(__fmul_rn(__uint_as_float(bits[i]), scale));
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) q[i] = fixed_point(bits[i], e);
      }
    }
    zero = false;
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
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const S v = q[perm(i)];
      neg |= (v < 0 ? 1u : 0u) << i;
      m[i] = (U)(v < 0 ? -v : v);
    }
    int sfx = -1;
#pragma unroll
    for (int i = 15; i >= 0; --i) {
      const int top = LL ? 63 - __clzll((long long)m[i]) : 31 - __clz((int)m[i]);  // -1 for 0
      sfx = max(sfx, top);
      s[i] = sfx;
      ev |= (u32)(top == sfx && top >= kmin) << i;
      nz |= (u32)(top >= kmin) << i;
    }
    // prefix members: s >= kmin (a prefix, as s does not increase)
    int refine = 0, plast = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const bool mem = s[i] >= kmin;
      cur += mem;
      refine += mem ? s[i] - kmin : 0;
      plast = mem ? s[i] : plast;
    }
    refine += cur;  // a sign bit per member
    const int nev = __popc(ev);
    const int sig = cur == 0 ? Ktop - kmin + 1
                             : nev + cur + (Ktop - plast) + (cur < 16 ? plast - kmin + 1 : 0);
    len = 1 + (LL ? 0 : 9) + sig + refine;
  }

  __device__ __forceinline__ void emit(u32 *buf, u32 pos) const {
    if (zero) return;  // the flag bit is 0
    BitWriter bw(buf, pos);
    if (LL)
      bw.put(1, 1);
    else
      bw.put(1u | ((u32)(e + 150) << 1), 10);
    int k = Ktop, nxt = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if ((ev >> i) & 1u) {
        bw.put(0, k - s[i]);  // failed group tests of the planes in between
        const int gap = i - nxt;  // scanned coefficients without the bit
        bw.put(1u | (1u << (gap + 1)), gap + 2);
        nxt = i + 1;
        k = s[i];
      }
    }
    if (cur < 16) {
      const int z = k - kmin + 1;  // up to 33
      bw.put(0, z - (z > 32));
      if (z > 32) bw.put(0, 1);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (i < cur) {
        const int w = s[i] - kmin;
        const u64 t = (u64)(m[i] >> kmin);
        const u64 field = t & ((1ull << w) - 1ull);
        const u64 sg = (neg >> i) & 1u;
        const u64 sgk = sg & (nz >> i);  // the sign of a zero kept magnitude is 0
        if (LL) {
          bw.put(field, w);
          bw.put(sgk, 1);
        } else {
          bw.put(field | (sgk << w), w + 1);
        }
      }
    }
    bw.flush();
  }

  // Fixed accuracy, the same bits with rolled loops over the events and the
  // prefix members only (sparse blocks skip the rest): s[i] and m[i] are read
  // back from this lane's shared-memory slots ss[i * stride], ms[i * stride].
  __device__ __forceinline__ void emit_rolled(u32 *buf, u32 pos, const unsigned char *ss,
                                              const u32 *ms, int stride) const {
    static_assert(!LL, "fixed accuracy only");
    if (zero) return;
    BitWriter bw(buf, pos);
    bw.put(1u | ((u32)(e + 150) << 1), 10);
    int k = Ktop, nxt = 0;
#pragma unroll 1
    for (u32 b = ev; b; b &= b - 1u) {
      const int i = __ffs(b) - 1;
      const int si = ss[i * stride];
      bw.put(0, k - si);  // failed group tests of the planes in between (<= 30)
      const int gap = i - nxt;
      bw.put(1u | (1u << (gap + 1)), gap + 2);
      nxt = i + 1;
      k = si;
    }
    if (cur < 16) bw.put(0, k - kmin + 1);  // <= 31
#pragma unroll 1
    for (int i = 0; i < cur; ++i) {
      const int w = ss[i * stride] - kmin;  // <= 30
      const u32 t = ms[i * stride] >> kmin;
      const u32 field = t & ((1u << w) - 1u);
      bw.put(field | (((neg & nz) >> i & 1u) << w), w + 1);
    }
    bw.flush();
  }
};

// Pass 1: code one tile (128 blocks, 4 chunks) into its staging slot of
// kTileWords words and record the words of each chunk.
template <bool LL>
__global__ void __launch_bounds__(kTile, LL ? 4 : 6) k_cz_encode(const __grid_constant__ EncArgs a) {
  __shared__ u32 sbuf[kWarps][kChunkWords];
  __shared__ u32 s_words[kWarps];
  __shared__ unsigned char s_kmin[kTab];
  __shared__ unsigned char s_s[LL ? 1 : 16][kTile];  // entry planes (fixed accuracy)
  __shared__ u32 s_m[LL ? 1 : 16][kTile];            // magnitudes (fixed accuracy)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kTab; i += blockDim.x) s_kmin[i] = a.kmin[i];
  __syncthreads();
  const u64 T = blockIdx.x;  // tile over all arrays
  const u32 arr = (u32)(T / a.tiles), lt = (u32)(T % a.tiles);
  const u32 b = lt * kTile + threadIdx.x;
  const float *src = a.data + (long long)arr * a.n0 * a.n1;

  Block<LL> c;
  if (b < a.nb) {
    const u32 bi = b / a.nb1, bj = b - bi * a.nb1;
    u32 bits[16];
    long long col[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) col[cc] = min((long long)(4 * bj + cc), a.n1 - 1);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float *row = src + min((long long)(4 * bi + r), a.n0 - 1) * a.n1;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) bits[4 * r + cc] = __float_as_uint(row[col[cc]]);
    }
    c.analyse(bits, s_kmin);
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
  if (lane == 0) s_words[warp] = nw;
  __syncwarp();
  // fixed accuracy: warps of dense blocks keep the unrolled emission, the
  // others take the rolled loops (the vote is warp-uniform)
  const bool dense = LL || __all_sync(0xffffffffu, c.len == 0 || c.zero || c.cur >= 12);
  if (c.len) {
    if (dense) {
      c.emit(buf, (u32)(incl - c.len));
    } else if constexpr (!LL) {
      if (!c.zero) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          s_s[i][threadIdx.x] = (unsigned char)max(c.s[i], 0);
          s_m[i][threadIdx.x] = c.m[i];
        }
      }
      c.emit_rolled(buf, (u32)(incl - c.len), &s_s[0][threadIdx.x], &s_m[0][threadIdx.x], kTile);
    }
  }
  const int nf = __syncthreads_or(c.nonfinite);
  u32 off = 0;
  for (int w = 0; w < warp; ++w) off += s_words[w];
  u32 *stage = a.stage + T * kTileWords;
  for (u32 i = lane; i < nw; i += 32) stage[off + i] = buf[i];
  if (lane == 0) a.chunk_words[T * kWarps + warp] = nw;
  if (threadIdx.x == 0 && nf) atomicOr(a.nonfinite + arr, 1u);
}

// Pass 2: per array, the word offset of every tile (exclusive scan of the
// tiles' words), the header and the stream's byte count.
template <bool LL>
__global__ void __launch_bounds__(1024) k_cz_scan(const __grid_constant__ EncArgs a) {
  __shared__ u32 s_warp[32];
  __shared__ u64 s_carry;
  const u32 arr = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const u32 *cw = a.chunk_words + (u64)arr * a.tiles * kWarps;
  u64 *toff = a.tile_off + (u64)arr * a.tiles;
  for (u32 base = 0; base < a.tiles; base += blockDim.x) {
    const u32 t = base + threadIdx.x;
    u32 v = 0;
    if (t < a.tiles) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) v += cw[(u64)t * kWarps + w];
    }
    u32 incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u32 y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u32 before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      before += w < warp ? s_warp[w] : 0u;
      total += s_warp[w];
    }
    const u64 carry = s_carry;
    if (t < a.tiles) toff[t] = carry + before + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const u64 words = s_carry;
    unsigned char *slot = a.out + (u64)arr * a.stride;
    const bool bad = !LL && a.nonfinite[arr];
    u32 *index = reinterpret_cast<u32 *>(slot + kHeader);
    for (u32 i = a.nchunk; i < (u32)(a.index_bytes / 4); ++i) index[i] = 0;
    u32 *h = reinterpret_cast<u32 *>(slot);
    h[0] = bad ? 0u : kMagic;
    h[1] = kVersion;
    h[2] = LL ? 1u : 0u;
    h[3] = kChunk;
    long long *hl = reinterpret_cast<long long *>(slot + 16);
    hl[0] = a.n0;
    hl[1] = a.n1;
    *reinterpret_cast<double *>(slot + 32) = LL ? 0.0 : a.tol;
    u64 *hu = reinterpret_cast<u64 *>(slot + 40);
    hu[0] = words;
    hu[1] = (u64)a.nchunk;
    hu[2] = 0;
    a.sizes[arr] = bad ? 0ull : kHeader + a.index_bytes + 4 * words;
  }
}

// Pass 3: copy each tile's words from its staging slot to its offset and
// write the offsets of its chunks.
__global__ void __launch_bounds__(kTile) k_cz_place(const __grid_constant__ EncArgs a) {
  const u64 T = blockIdx.x;
  const u32 arr = (u32)(T / a.tiles), lt = (u32)(T % a.tiles);
  const u32 *cw = a.chunk_words + T * kWarps;
  u32 tw = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) tw += cw[w];
  const u64 base = a.tile_off[T];
  unsigned char *slot = a.out + (u64)arr * a.stride;
  u32 *index = reinterpret_cast<u32 *>(slot + kHeader);
  u32 *words = reinterpret_cast<u32 *>(slot + kHeader + a.index_bytes);
  const u32 *stage = a.stage + T * kTileWords;
  for (u32 i = threadIdx.x; i < tw; i += blockDim.x) words[base + i] = stage[i];
  if (threadIdx.x < kWarps) {
    const u32 chunk = lt * kWarps + threadIdx.x;
    u32 off = 0;
    for (int w = 0; w < (int)threadIdx.x; ++w) off += cw[w];
    if (chunk < a.nchunk) index[chunk] = (u32)(base + off);
  }
}

// ---------------------------------------------------------------- decode --

// Sequential reader over the words of one chunk in global memory (the walk);
// positions count bits from the chunk's first bit, reads past its end see
// zeros.  At least 32 bits are buffered after every call, and the word after
// the buffered ones is already loading.
struct GReader {
  const u32 *w;
  u32 nw, widx, pos;
  int avail;
  u64 buf;
  u32 nxt;  // word widx - 1
  __device__ __forceinline__ void init(const u32 *words, u32 nwords) {
    w = words;
    nw = nwords;
    buf = nw > 0 ? __ldg(w) : 0u;
    nxt = nw > 1 ? __ldg(w + 1) : 0u;
    avail = 32;
    widx = 2;
    pos = 0;
  }
  // start at bit `bit` of the chunk (the decode)
  __device__ __forceinline__ void init_at(const u32 *words, u32 nwords, u32 bit) {
    w = words;
    nw = nwords;
    const u32 wi = bit >> 5;
    const u32 a0 = wi < nw ? __ldg(w + wi) : 0u, a1 = wi + 1 < nw ? __ldg(w + wi + 1) : 0u;
    buf = (((u64)a1 << 32) | a0) >> (bit & 31);
    avail = 64 - (int)(bit & 31);
    nxt = wi + 2 < nw ? __ldg(w + wi + 2) : 0u;
    widx = wi + 3;
    pos = bit;
  }
  __device__ __forceinline__ void refill() {
    if (avail <= 32) {
      buf |= (u64)nxt << avail;
      avail += 32;
      nxt = widx < nw ? __ldg(w + widx) : 0u;
      widx++;
    }
  }
  __device__ __forceinline__ u32 peek() const { return (u32)buf; }
  __device__ __forceinline__ void skip(int n) {  // n <= 32
    buf >>= n;
    avail -= n;
    pos += (u32)n;
    refill();
  }
  __device__ __forceinline__ void advance(u32 n) {  // any n
    if (n <= 32)
      skip((int)n);
    else
      init_at(w, nw, pos + n);
  }
  __device__ bool overrun() const { return pos > nw * 32u; }
};

template <class R>
__device__ __forceinline__ u32 getbits(R &rd, int n) {  // n <= 32
  const u32 v = n ? rd.peek() & (0xffffffffu >> (32 - n)) : 0u;
  rd.skip(n);
  return v;
}

// zero bits before the next one, at most lim (all consumed)
template <class R>
__device__ __forceinline__ int zeros(R &rd, int lim) {
  int z = 0;
  while (z < lim) {
    const u32 v = rd.peek();
    const int c = min(v ? __ffs(v) - 1 : 32, lim - z);
    rd.skip(c);
    z += c;
    if (c < 32) break;
  }
  return z;
}

// The significance section of a nonzero block: per event, the failed group
// tests of the planes before it, the successful test, the scanned
// coefficients without the bit and the one found.  Sets bit p of found for
// every coefficient found and sfx[p * sstride] to the plane it was found at.
// Returns false on a malformed section.
template <bool LL, class R>
__device__ __forceinline__ bool significance(R &rd, int kmin, unsigned char *sfx, int sstride,
                                             u32 &found) {
  constexpr int Ktop = LL ? 32 : 30;
  found = 0;
  int n = 0, k = Ktop;
  while (k >= kmin && n < 16) {
    const int lim = k - kmin + 1;
    const u32 v = rd.peek();
    const int z = v ? __ffs(v) - 1 : 32;
    int g;
    if (z < lim && z < 31) {
      const u32 v2 = v >> (z + 1);  // 31 - z valid bits
      g = v2 ? __ffs(v2) - 1 : 32;
      if (g < 31 - z && g < 16 - n) {
        rd.skip(z + g + 2);
      } else {
        rd.skip(z + 1);
        g = zeros(rd, 16 - n);
        if (g == 16 - n) return false;
        rd.skip(1);
      }
      k -= z;
    } else {
      const int zz = zeros(rd, lim);
      if (zz == lim) break;
      k -= zz;
      rd.skip(1);
      g = zeros(rd, 16 - n);
      if (g == 16 - n) return false;
      rd.skip(1);
    }
    const int p = n + g;
    sfx[p * sstride] = (unsigned char)k;
    found |= 1u << p;
    n = p + 1;
  }
  return true;
}

// The walk of one chunk: the bit offset of each of its first nblk blocks
// that is not all zero into offs, and its cost class (1 + 16 min(events, 14)
// + min(members, 15): the trip counts of the decode's two loops) into cls;
// both arrays come zeroed, and class 0 marks an all-zero block.  Every
// iteration consumes one token: a run of all-zero blocks, a block's head, or
// one event of its significance section (failed group tests, the successful
// one, the scan, the coefficient found).  Every member of the prefix
// carries w bits and a sign, w the plane above kmin of the next coefficient
// found, so the refinement section is skipped in one step with the token
// that ends the significance section.  The lanes of a warp, each on its own
// chunk, move one token per iteration whatever their blocks look like, and
// a warp takes as many iterations as its longest chunk has tokens.  Returns
// false on a malformed chunk.
template <bool LL>
__device__ bool walk_chunk(GReader &rd, u32 nblk, const unsigned char *ktab, unsigned short *offs,
                           unsigned char *cls) {
  constexpr int Ktop = LL ? 32 : 30;
  int phase = 0;  // 0 a block's head, 1 an event, 3 a scan past the window
  int k = 0, kmin = 0, n = 0, g = 0, ne = 0;
  u32 blk = 0, refine = 0;
  bool ok = true;
  while (blk < nblk && ok) {
    const u32 v = rd.peek();
    u32 adv = 0;
    bool event = false;  // an event ends in this token: coefficient n + g at plane k
    bool done = false;   // the significance section ends with this token
    if (phase == 0) {
      if (!(v & 1u)) {  // a run of all-zero blocks (one flag bit each)
        adv = (u32)min(v ? __ffs(v) - 1 : 32, (int)(nblk - blk));
        blk += adv;
      } else {
        offs[blk] = (unsigned short)rd.pos;  // < 2^16: a chunk holds at most 640 words
        if (LL) {
          adv = 1;
        } else {
          const int eb = (int)((v >> 1) & 511u);
          ok = eb < kTab;
          kmin = ok ? ktab[eb] : 0;
          adv = 10;
        }
        phase = 1;
        k = Ktop;
        n = 0;
        ne = 0;
        refine = 0;
      }
    } else if (phase == 1) {
      const int lim = k - kmin + 1;
      const int z = v ? __ffs(v) - 1 : 32;
      if (z >= lim) {  // every remaining plane fails
        adv = (u32)lim;
        done = true;
      } else if (z == 32) {  // (lossless) 32 failed tests, planes left
        adv = 32;
        k -= 32;
      } else {
        k -= z;
        const u32 v2 = z < 31 ? v >> (z + 1) : 0u;  // 31 - z valid bits
        g = v2 ? __ffs(v2) - 1 : 32;
        if (g < 31 - z) {
          adv = (u32)(z + g + 2);
          event = true;
        } else {  // the scan goes on past the window
          adv = 32;
          g = 31 - z;
          phase = 3;
        }
        ok = g < 16 - n;
      }
    } else {
      const int zz = v ? __ffs(v) - 1 : 32;
      g += zz;
      ok = zz < 32 && g < 16 - n;
      adv = (u32)(zz + 1);
      event = true;
      phase = 1;
    }
    if (event && ok) {  // members n .. n + g enter the prefix at plane k
      refine += (u32)(g + 1) * (u32)(k - kmin + 1);
      n += g + 1;
      ++ne;
      done = n == 16;
    }
    if (done && ok) {
      cls[blk] = (unsigned char)(1 + min(ne, 14) * 16 + min(n, 15));
      adv += refine;
      phase = 0;
      ++blk;
    }
    rd.advance(adv);
  }
  return ok;
}

// Decode one block into x (the decode).  Returns false on a malformed block.
template <bool LL, class R>
__device__ __forceinline__ bool decode_block(R &rd, const unsigned char *ktab,
                                             unsigned char *sfx, int *qs, int sstride,
                                             float (&x)[16]) {
  if (!getbits(rd, 1)) {
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = 0.0f;
    return true;
  }
  int e = 0, kmin = 0;
  if (!LL) {
    const int eb = (int)getbits(rd, 9);
    if (eb >= kTab) return false;
    e = eb - 150;
    kmin = ktab[eb];
  }
  u32 found;
  if (!significance<LL>(rd, kmin, sfx, sstride, found)) return false;
  // refinement: magnitudes and signs, in coding order, each at the midpoint
  // of its kept interval.  Fixed accuracy takes a rolled loop over the
  // members (one trip per member, so lanes with as many members stay in
  // step), the coefficients through this thread's shared-memory slots qs[j *
  // sstride], j in block order; lossless keeps the unrolled register form
  // (its 64-bit slots would cost occupancy).
  using S = typename std::conditional<LL, long long, int>::type;
  S q[16];
  long long qw[16];
  const u64 half = kmin > 0 ? (1ull << (kmin - 1)) : 0ull;
  const int n = found ? 32 - __clz(found) : 0;  // members: up to the last coefficient found
  if constexpr (!LL) {
#pragma unroll
    for (int j = 0; j < 16; ++j) qs[j * sstride] = 0;
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
      const int w = sfx[(i + __ffs(found >> i) - 1) * sstride] - kmin;  // 0 .. 30
      const u32 fs = getbits(rd, w + 1);  // w bits, then the sign
      u64 t = fs & ((1u << w) - 1u);
      if ((found >> i) & 1u) t |= 1ull << w;
      if (t) {
        const long long v = (long long)((t << kmin) + half);
        qs[perm_rt(i) * sstride] = (int)((fs >> w) ? -v : v);
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      q[j] = (S)qs[j * sstride];
      qw[j] = (long long)qs[j * sstride];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      long long v = 0;
      if (i < n) {
        const int w = sfx[(i + __ffs(found >> i) - 1) * sstride] - kmin;
        u64 t = w > 32 ? 0ull : (u64)getbits(rd, min(w, 32));
        if ((found >> i) & 1u) t |= 1ull << w;
        const bool ng = getbits(rd, 1);
        if (t) {
          v = (long long)((t << kmin) + half);
          if (ng) v = -v;
        }
      }
      q[perm(i)] = (S)v;
      qw[perm(i)] = v;
    }
  }
  const bool wide = !LL && kmin > 26;  // fixed accuracy with kmin > 26 reconstructs in 64 bits
  bool ok = true;
  if (LL || !wide) {
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
    if (LL) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const long long v = (long long)q[i];
        ok &= v >= -2147483648ll && v <= 2147483647ll;
        x[i] = __uint_as_float(v < 0 ? 0x80000000u | (u32)(-1ll - v) : (u32)v);
      }
    } else if (e >= -98 && e <= 120) {
      // every nonzero value is a normal float: one rounding in the conversion,
      // then an exact scaling by 2^(e-28)
      const float scale = __uint_as_float((u32)(e - kP + 127) << 23);
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = __fmul_rn(__int2float_rn((int)q[i]), scale);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = fixed_to_float_slow((long long)q[i], e);
    }
  } else {
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int o = pass ? 4 * l : l, st = pass ? 1 : 4;
        const long long ss = qw[o], dd = qw[o + st], d1 = qw[o + 2 * st], d2 = qw[o + 3 * st];
        const long long s1 = ss - (dd >> 1), s2 = dd + s1;
        const long long a0 = s1 - (d1 >> 1), b0 = d1 + a0;
        const long long c0 = s2 - (d2 >> 1), e0 = d2 + c0;
        qw[o] = a0;
        qw[o + st] = b0;
        qw[o + 2 * st] = c0;
        qw[o + 3 * st] = e0;
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = fixed_to_float_slow(qw[i], e);
  }
  return ok;
}


// The stream header of array arr checked against the call (one thread).
__device__ __forceinline__ bool header_ok(const DecArgs &a, const unsigned char *slot) {
  const u32 *h = reinterpret_cast<const u32 *>(slot);
  const long long *hl = reinterpret_cast<const long long *>(slot + 16);
  const u64 *hu = reinterpret_cast<const u64 *>(slot + 40);
  const double tol = *reinterpret_cast<const double *>(slot + 32);
  const u64 cap = (a.stride - kHeader - a.index_bytes) / 4;
  return h[0] == kMagic && h[1] == kVersion && h[2] <= 1u && h[3] == (u32)kChunk && hl[0] == a.n0 &&
         hl[1] == a.n1 && hu[1] == (u64)a.nchunk && hu[0] <= cap &&
         (h[2] ? tol == 0.0 : (tol > 0.0 && tol < 1e300));
}

// The words [start, next) of chunk c, checked against the index and the bit
// section; false for a malformed index.
__device__ __forceinline__ bool chunk_words(const DecArgs &a, const unsigned char *slot, u32 c,
                                            u32 &start, u32 &next) {
  const u64 nwords = *reinterpret_cast<const u64 *>(slot + 40);
  const u32 *index = reinterpret_cast<const u32 *>(slot + kHeader);
  start = index[c];
  next = c + 1 < a.nchunk ? index[c + 1] : (u32)min(nwords, (u64)0xffffffffu);
  return start <= next && next <= nwords && next - start <= (u32)kChunkWords &&
         (c > 0 || start == 0);
}

__device__ __forceinline__ void report_bad(const DecArgs &a, u32 arr) {
  atomicExch(a.err, 1);
  atomicMin(a.err + 1, (int)(a.arr0 + arr));
}

// Chunk size classes by which a walk CTA orders its chunks: word counts
// below 48 one by one, then in steps of 16 words.
__device__ __forceinline__ int walk_key(u32 nw) {
  return nw < 48u ? (int)nw : min(48 + (int)((nw - 48u) >> 4), kWalkKeys - 1);
}

// Pass 1 of decoding: one thread per chunk, one segment (kWalk chunks) per
// CTA.  The CTA's chunks are first ordered by size class (a counting sort in
// shared memory), so that a warp walks chunks of similar length: the walk
// moves one token per iteration and a warp takes as many iterations as its
// longest chunk.  The bit offsets and cost classes of the blocks stay in
// shared memory; the CTA then writes the segment's list (its blocks that are
// not all zero, ordered by class with a second counting sort) and its count,
// and writes the all-zero blocks to the output.  One kernel per mode; each
// skips the other mode's streams, and the fixed-accuracy one reports bad
// headers.
template <bool LL>
__global__ void __launch_bounds__(kWalk) k_cz_walk(const __grid_constant__ DecArgs a) {
  __shared__ unsigned short s_offs[kWalk][kChunk + 1];
  __shared__ unsigned char s_cls[kWalk][kChunk + 4];
  __shared__ unsigned char s_kmin[kTab];
  __shared__ int s_cnt[kClasses];
  __shared__ unsigned short s_order[kWalk];
  __shared__ int s_wsum[kWalk / 32];
  __shared__ u32 s_nnz;
  __shared__ int s_ok;
  const u32 arr = blockIdx.y;
  const int tid = threadIdx.x;
  const unsigned char *slot = a.in + (u64)arr * a.stride;
  if (tid == 0) s_ok = header_ok(a, slot);
  for (int i = tid; i < kClasses; i += kWalk) s_cnt[i] = 0;
  for (int i = tid; i < kTab; i += kWalk) s_kmin[i] = a.kmin[arr * kTab + i];
  __syncthreads();
  if (!s_ok) {
    if (!LL && tid == 0 && blockIdx.x == 0) report_bad(a, arr);
    return;
  }
  if ((reinterpret_cast<const u32 *>(slot)[2] != 0) != LL) return;
  const u32 *words = reinterpret_cast<const u32 *>(slot + kHeader + a.index_bytes);
  const u32 c0 = blockIdx.x * kWalk;
  const u32 rows = min((u32)kWalk, a.nchunk - c0);
  // order the chunks by size class
  {
    u32 start = 0, next = 0;
    const bool ok = (u32)tid < rows && chunk_words(a, slot, c0 + tid, start, next);
    const int key = walk_key(ok ? next - start : 0u);
    const int rank = atomicAdd(&s_cnt[key], 1);
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the class counts, two per lane
      const int x0 = s_cnt[2 * tid], x1 = s_cnt[2 * tid + 1];
      int inc = x0 + x1;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (tid >= d) inc += y;
      }
      const int exc = inc - x0 - x1;
      s_cnt[2 * tid] = exc;
      s_cnt[2 * tid + 1] = exc + x0;
    }
    __syncthreads();
    s_order[s_cnt[key] + rank] = (unsigned short)tid;
    __syncthreads();
    for (int i = tid; i < kClasses; i += kWalk) s_cnt[i] = 0;  // (now the class histogram)
  }
  const int r = s_order[tid];  // the chunk this thread walks
  bool bad = false;
  if ((u32)r < rows) {
    const u32 c = c0 + r;
    u32 start, next;
    bool ok = chunk_words(a, slot, c, start, next);
    const u32 nblk = min((u32)kChunk, a.nb - c * kChunk);
    for (u32 k = 0; k < (u32)kChunk; ++k) {  // (blocks not reached stay all zero)
      s_offs[r][k] = 0;
      s_cls[r][k] = 0;
    }
    if (ok) {
      GReader rd;
      rd.init(words + start, next - start);
      ok = walk_chunk<LL>(rd, nblk, s_kmin, s_offs[r], s_cls[r]);
      ok = ok && !rd.overrun() && (rd.pos + 31) / 32 == next - start;
    }
    bad = !ok;
  }
  __syncthreads();
  // the segment's list: its blocks that are not all zero, in class order,
  // each entry the block's index in the segment (13 bits) over its bit
  // offset in its chunk (15 bits: a chunk holds at most 640 words)
  const u32 B0 = c0 * kChunk, nblocks = min(rows * kChunk, a.nb - B0);
  for (u32 i = tid; i < nblocks; i += kWalk) {
    const unsigned q = s_cls[i >> 5][i & 31];
    if (q) atomicAdd(&s_cnt[q], 1);
  }
  __syncthreads();
  {  // exclusive scan of the class counts, kPerT consecutive ones per thread
    constexpr int kPerT = kClasses / kWalk;
    const int lane = tid & 31, warp = tid >> 5;
    int x[kPerT], sum = 0;
#pragma unroll
    for (int j = 0; j < kPerT; ++j) {
      x[j] = s_cnt[tid * kPerT + j];
      sum += x[j];
    }
    int inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += y;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    int run = inc - sum;
#pragma unroll
    for (int w = 0; w < kWalk / 32; ++w) run += w < warp ? s_wsum[w] : 0;
#pragma unroll
    for (int j = 0; j < kPerT; ++j) {
      s_cnt[tid * kPerT + j] = run;
      run += x[j];
    }
    if (tid == kWalk - 1) s_nnz = (u32)run;
  }
  __syncthreads();
  const u64 seg = (u64)arr * a.nseg + blockIdx.x;
  u32 *list = a.list + seg * kSeg;
  for (u32 i = tid; i < nblocks; i += kWalk) {
    const unsigned q = s_cls[i >> 5][i & 31];
    if (q) list[atomicAdd(&s_cnt[q], 1)] = (i << 15) | s_offs[i >> 5][i & 31];
  }
  if (tid == 0) a.segcount[seg] = s_nnz;
  // the segment's all-zero blocks to the output, row by row: a warp per row,
  // 32 consecutive floats per store
  {
    const u32 B1 = B0 + nblocks, bi0 = B0 / a.nb1, bi1 = (B1 - 1) / a.nb1;
    const u32 r1 = min(4 * bi1 + 4, (u32)a.n0), lane = tid & 31;
    for (u32 i = 4 * bi0 + (tid >> 5); i < r1; i += kWalk / 32) {
      const u32 rb = (i >> 2) * a.nb1;  // first block of this row's block row
      const u32 lo = max(B0, rb), hi = min(B1, rb + a.nb1);
      const u32 j1 = min(4 * (hi - rb), (u32)a.n1);
      float *row = a.out + ((u64)arr * a.n0 + i) * a.n1;
      for (u32 j = 4 * (lo - rb) + lane; j < j1; j += 32) {
        const u32 l = rb + (j >> 2) - B0;  // the block's index in the segment
        if (s_cls[l >> 5][l & 31] == 0) row[j] = 0.0f;
      }
    }
  }
  if (bad) report_bad(a, arr);
}

// The 4 x 4 block b of array arr to the output (edge blocks clipped).
__device__ __forceinline__ void store_block(const DecArgs &a, u32 arr, u32 b, const float (&x)[16]) {
  const u32 bi = b / a.nb1, bj = b - bi * a.nb1;
  float *p0 = a.out + ((long long)arr * a.n0 + 4ll * bi) * a.n1 + 4ll * bj;
  if (4ll * bi + 3 < a.n0 && 4ll * bj + 3 < a.n1) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) p0[cc] = x[4 * r + cc];
      p0 += a.n1;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (4ll * bi + r < a.n0) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          if (4ll * bj + cc < a.n1) p0[cc] = x[4 * r + cc];
      }
      p0 += a.n1;
    }
  }
}

// Pass 2: decode the listed blocks of one mode, a CTA per segment (a
// grid-stride loop over one resident wave of CTAs), a thread per entry in
// list order, so that the lanes of a warp hold blocks of one class and run
// the decode's loops for as many trips.  Each thread reads its block's bits
// from global memory, bounded by its chunk.
template <bool LL>
__global__ void __launch_bounds__(kDec) k_cz_decode(const __grid_constant__ DecArgs a) {
  __shared__ unsigned char s_sfx[16][kDec];
  __shared__ int s_q[LL ? 1 : 16][kDec];  // coefficient slots (fixed accuracy)
  __shared__ u32 s_n;
  const int tid = threadIdx.x;
  const u64 nseg = (u64)a.count * a.nseg;
  for (u64 seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
    const u32 arr = (u32)(seg / a.nseg), sj = (u32)(seg - (u64)arr * a.nseg);
    const unsigned char *slot = a.in + (u64)arr * a.stride;
    if (tid == 0)
      s_n = header_ok(a, slot) && (reinterpret_cast<const u32 *>(slot)[2] != 0) == LL
                ? a.segcount[seg]
                : 0u;
    __syncthreads();
    const u32 n = s_n;
    const u32 *list = a.list + seg * kSeg;
    const u32 *words = reinterpret_cast<const u32 *>(slot + kHeader + a.index_bytes);
    for (u32 p = tid; p < n; p += kDec) {
      const u32 e = list[p];
      const u32 b = sj * kSeg + (e >> 15);
      u32 start, next;
      if (!chunk_words(a, slot, b / kChunk, start, next)) continue;  // (reported by the walk)
      GReader rd;
      rd.init_at(words + start, next - start, e & 0x7fffu);
      float x[16];
      const bool ok = decode_block<LL>(rd, a.kmin + (u64)arr * kTab, &s_sfx[0][tid],
                                       &s_q[0][tid], kDec, x) &&
                      !rd.overrun();
      if (!ok) report_bad(a, arr);
      store_block(a, arr, b, x);
    }
    __syncthreads();  // (s_n is set again for the next segment)
  }
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

// device scratch of one compression, in bytes
u64 codec_scratch_bytes(long long count, long long n0, long long n1) {
  long long nb = 0;
  if (!codec_shape(n0, n1, nullptr, &nb, nullptr, nullptr, nullptr)) return 0;
  const u64 tiles = (u64)count * (u64)((nb + kTile - 1) / kTile);
  return tiles * (4ull * kTileWords + 4ull * kWarps + 8ull) + 4ull * (u64)count + 512;
}

cudaError_t launch_cz_encode(const float *data, long long count, long long n0, long long n1,
                             double tol, unsigned char *out, u64 stride, u64 *sizes,
                             unsigned char *scratch, cudaStream_t st) {
  EncArgs a{};
  long long nb1, nb, nchunk;
  if (!codec_shape(n0, n1, &nb1, &nb, &nchunk, &a.index_bytes, nullptr))
    return cudaErrorInvalidValue;
  a.nb1 = (u32)nb1;
  a.nb = (u32)nb;
  a.nchunk = (u32)nchunk;
  a.data = data;
  a.n0 = n0;
  a.n1 = n1;
  a.tiles = (u32)((nb + kTile - 1) / kTile);
  const u64 tiles = (u64)count * a.tiles;
  if (tiles > 0x7fffffffull || count > 0xffffffffll) return cudaErrorInvalidValue;
  a.out = out;
  a.stride = stride;
  a.sizes = sizes;
  // scratch: stage | tile_off | chunk_words | nonfinite | kmin; every word but
  // the non-finite flags is written before it is read
  a.stage = reinterpret_cast<u32 *>(scratch);
  a.tile_off = reinterpret_cast<u64 *>(scratch + tiles * 4ull * kTileWords);
  a.chunk_words = reinterpret_cast<u32 *>(scratch + tiles * (4ull * kTileWords + 8ull));
  a.nonfinite = a.chunk_words + tiles * kWarps;
  unsigned char *tab = reinterpret_cast<unsigned char *>(a.nonfinite + count);
  a.kmin = tab;
  a.tol = tol;
  cudaError_t e = cudaMemsetAsync(a.nonfinite, 0, 4ull * (u64)count, st);
  if (e != cudaSuccess) return e;
  k_cz_kmin<<<1, kTab, 0, st>>>(nullptr, 0, tol, tab);
  if (tol > 0) {
    k_cz_encode<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
    k_cz_scan<false><<<(unsigned)count, 1024, 0, st>>>(a);
  } else {
    k_cz_encode<true><<<(unsigned)tiles, kTile, 0, st>>>(a);
    k_cz_scan<true><<<(unsigned)count, 1024, 0, st>>>(a);
  }
  k_cz_place<<<(unsigned)tiles, kTile, 0, st>>>(a);
  return cudaGetLastError();
}

// Arrays decoded per group: at most kGroupBlocks list entries (kSeg per
// segment), at least one array; the groups of a call are made as even as that
// allows.
static long long decode_group(long long count, long long nchunk) {
  const long long per = (nchunk + kWalk - 1) / kWalk * kSeg;
  const long long most = std::max(1ll, std::min(count, (long long)(kGroupBlocks / (u64)per)));
  const long long groups = (count + most - 1) / most;
  return (count + groups - 1) / groups;
}

// device scratch of one decompression, in bytes: the 16-byte error record,
// the kmin tables (count x kTab bytes, padded to 16), then for a group of
// arrays the segment counts (4 bytes per segment, padded to 16) and lists
// (4 bytes per block slot)
u64 codec_decode_scratch_bytes(long long count, long long n0, long long n1) {
  long long nchunk = 0;
  if (!codec_shape(n0, n1, nullptr, nullptr, &nchunk, nullptr, nullptr)) return 0;
  const u64 nseg = (u64)((nchunk + kWalk - 1) / kWalk), G = (u64)decode_group(count, nchunk);
  return 16 + ((u64)count * kTab + 15) / 16 * 16 + (4 * G * nseg + 15) / 16 * 16 +
         4ull * kSeg * G * nseg;
}

// scratch: codec_decode_scratch_bytes(count, n0, n1) bytes, 16-byte aligned;
// its first 8 bytes must hold {0, 0x7fffffff} (the error record)
cudaError_t launch_cz_decode(const unsigned char *in, u64 stride, long long count, long long n0,
                             long long n1, float *out, unsigned char *scratch, cudaStream_t st) {
  DecArgs a{};
  long long nb1, nb, nchunk;
  if (!codec_shape(n0, n1, &nb1, &nb, &nchunk, &a.index_bytes, nullptr))
    return cudaErrorInvalidValue;
  if (count < 1 || count > 65535) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0, per_sm[2] = {0, 0};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_cz_decode<false>, kDec, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_cz_decode<true>, kDec, 0);
  if (e != cudaSuccess) return e;
  a.nb1 = (u32)nb1;
  a.nb = (u32)nb;
  a.nchunk = (u32)nchunk;
  a.nseg = (u32)((nchunk + kWalk - 1) / kWalk);
  a.n0 = n0;
  a.n1 = n1;
  a.stride = stride;
  a.err = reinterpret_cast<int *>(scratch);
  unsigned char *tab = scratch + 16, *p = tab + ((u64)count * kTab + 15) / 16 * 16;
  const long long G = decode_group(count, nchunk);
  a.segcount = reinterpret_cast<u32 *>(p);
  a.list = reinterpret_cast<u32 *>(p + (4ull * G * a.nseg + 15) / 16 * 16);
  k_cz_kmin<<<(unsigned)count, kTab, 0, st>>>(in, stride, 0.0, tab);
  for (long long g0 = 0; g0 < count; g0 += G) {
    const long long g = std::min(G, count - g0);
    a.arr0 = (u32)g0;
    a.count = (u32)g;
    a.in = in + (u64)g0 * stride;
    a.out = out + (u64)g0 * (u64)n0 * (u64)n1;
    a.kmin = tab + (u64)g0 * kTab;
    const dim3 gwalk(a.nseg, (unsigned)g);
    // the decode loops over the group's segments with one resident wave of CTAs
    const u64 nseg = (u64)g * a.nseg;
    const unsigned gd0 = (unsigned)std::min<u64>(nseg, (u64)std::max(1, per_sm[0]) * nsm);
    const unsigned gd1 = (unsigned)std::min<u64>(nseg, (u64)std::max(1, per_sm[1]) * nsm);
    k_cz_walk<false><<<gwalk, kWalk, 0, st>>>(a);
    k_cz_walk<true><<<gwalk, kWalk, 0, st>>>(a);
    k_cz_decode<false><<<gd0, kDec, 0, st>>>(a);
    k_cz_decode<true><<<gd1, kDec, 0, st>>>(a);
  }
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
  const u64 stage_bytes = codec_scratch_bytes(count, n0, n1);
  DevBuf dsizes;
  CZ_CU(scratch.alloc(ctx, stage_bytes, st));
  CZ_CU(dsizes.alloc(ctx, (size_t)count * 8, st));
  u64 *sizes = dsizes.as<u64>();
  CodecTimer tm(ctx, st);
  tm.start();
  CZ_CU(launch_cz_encode(d_data, count, n0, n1, tol, d_out, out_stride, sizes,
                         scratch.as<unsigned char>(), st));
  tm.stop();
  CZ_CU(cudaMemcpyAsync(out_bytes, sizes, (size_t)count * 8, cudaMemcpyDeviceToHost, st));
  CZ_CU(cudaStreamSynchronize(st));
  double total = 0;
  long long bad = 0, first_bad = -1;
  for (long long i = 0; i < count; ++i) {
    total += (double)out_bytes[i];
    if (!out_bytes[i] && first_bad < 0) first_bad = i;
    bad += !out_bytes[i];
  }
  tm.account((double)nbytes_in + total);
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
  CZ_CU(scratch.alloc(ctx, codec_decode_scratch_bytes(count, n0, n1), st));
  const int init[4] = {0, 0x7fffffff, 0, 0};
  CZ_CU(cudaMemcpyAsync(scratch.p, init, 16, cudaMemcpyHostToDevice, st));
  CodecTimer tm(ctx, st);
  tm.start();
  CZ_CU(launch_cz_decode(d_in, in_stride, count, n0, n1, d_data, scratch.as<unsigned char>(), st));
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
