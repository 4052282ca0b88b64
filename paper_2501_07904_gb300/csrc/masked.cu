// Masked TT evaluation x(i) = G_1[i_1] G_2[:, i_2, :] ... G_d[:, i_d] at a set
// Omega of row-major linear indices, and its core gradients: the observation
// operator P_Omega of the completion experiment (Sec. 4.2.2) and the
// derivative of sum_e gout_e x(i_e) with respect to every core.
//
// Plan (built once per index set, reused by every call):
//  * every index is range-checked and decoded into its mode indices;
//  * for each core k the entries are ordered stably by (i_k, i_nb), nb the
//    neighbouring core whose slice enters the costlier interface product, by
//    LSD radix passes over 8-bit digits (a stable counting sort per digit);
//  * per chunk of kChunk consecutive positions of each order, three bits say
//    whether its first slice continues from the previous chunk, whether its
//    last slice continues into the next one, and whether it holds one slice.
//
// Evaluation, per chunk of one order (kChunk entries, one CTA):
//  * the left interface L = G_1[i_1] .. G_{k-1}[i_{k-1}] (length r_{k-1}) and
//    the right interface R = G_{k+1}[i_{k+1}] .. G_d[i_d] (length r_k) of
//    every entry are recomputed, step by step, by thread groups that keep the
//    current core slice's column (or row) in registers and reload it only
//    when the slice index changes between consecutive entries (the sort makes
//    runs of equal neighbour slices);
//  * forward (k = the pivot core, largest r_{k-1} r_k): the slice G_k[:, i, :]
//    of each run of equal i_k is staged in shared memory once and
//    x = L^T G_k[:, i, :] R is formed per entry in registers;
//  * backward (one pass per core k): dG_k[:, i, :] += sum_e L_e (gout_e R_e)^T
//    over the entries of slice i, summed by fixed thread groups in 4 x 4
//    register tiles and folded in group order.  A slice wholly inside the
//    chunk is added to the gradient by that CTA alone; a slice that straddles
//    chunk boundaries leaves one partial per chunk, and a fix-up pass adds
//    those partials in chunk order.  No floating-point atomics are used, so a
//    plan gives bitwise-equal gradients on every call.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ttutv.h"
#include "internal.h"

namespace ttk {
namespace {

constexpr int kEvalMaxD = TT_MAXD;
constexpr int kEvalMaxR = 64;
constexpr int kChunk = 128;        // entries per chunk of an order (one CTA)
constexpr int kEvalThreads = 128;  // threads of the evaluation CTA (one per chunk entry)
constexpr int kSortTile = 2048;    // entries per radix tile (256 threads x 8 rounds)
static_assert(kChunk == kEvalThreads, "the forward contraction runs one thread per entry");

__device__ __forceinline__ int round4_dev(int x) { return (x + 3) & ~3; }

// Two FP32 fused multiply-adds in one packed instruction (each lane rounded
// to nearest, as fmaf).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// smallest power of two >= x, and >= 4 (the width of a chain-step lane group)
__device__ __forceinline__ int group_width(int x) {
  const int p = x <= 1 ? 1 : 1 << (32 - __clz(x - 1));
  return p < 4 ? 4 : p;
}

int round4(int x) { return (x + 3) & ~3; }
int bits_of(int64_t x) {  // number of bits of x >= 0
  int b = 0;
  while (x > 0) {
    ++b;
    x >>= 1;
  }
  return b;
}
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------ plan build

struct DecodeArgs {
  int d;
  int64_t dims[kEvalMaxD];
  int64_t total;
};

// ix[k][e] = i_k of entry e; an index outside [0, prod(dims)) sets bit 0 of *err
// and decodes as 0 in every mode, so later passes stay in bounds.
__global__ void decode_kernel(const int64_t* __restrict__ idx, int64_t n, DecodeArgs a,
                              int32_t* __restrict__ ix, int32_t* __restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t lin = idx[e];
    const bool bad = lin < 0 || lin >= a.total;
    if (bad) {
      atomicOr(err, 1);
      lin = 0;
    }
    for (int k = a.d - 1; k >= 0; --k) {
      ix[(int64_t)k * n + e] = (int32_t)(lin % a.dims[k]);
      lin /= a.dims[k];
    }
  }
}

// One stable counting-sort pass on the 8-bit digit (key[v] >> shift) & 255 of
// the entry ids v = in[p] (in == null: v = p).  Tile t covers positions
// [t*2048, (t+1)*2048) in 8 rounds of 256 consecutive positions; inside a
// round a warp ranks equal digits with a match mask and the warps are
// offset by the counts of the warps before them, so equal digits keep their
// input order.  count pass: hist[digit * ntiles + t] = the tile's counts;
// scatter pass: hist holds their exclusive scan (digit-major), and each id
// goes to out[hist[digit][t] + rank].
__global__ void __launch_bounds__(256) radix_kernel(const int32_t* __restrict__ in,
                                                    int32_t* __restrict__ out, int64_t n,
                                                    const int32_t* __restrict__ key, int shift,
                                                    int32_t* __restrict__ hist, int64_t ntiles,
                                                    int scatter, int32_t* __restrict__ err) {
  __shared__ int wcnt[8][256];
  __shared__ int run[256];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * kSortTile;
  run[t] = scatter ? hist[(int64_t)t * ntiles + tile] : 0;
#pragma unroll
  for (int ww = 0; ww < 8; ++ww) wcnt[ww][t] = 0;
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  for (int j = 0; j < kSortTile / 256; ++j) {
    const int64_t p = base + (int64_t)j * 256 + t;
    const bool valid = p < n;
    int v = 0, dig = 256;
    if (valid) {
      v = in ? in[p] : (int)p;
      dig = (key[v] >> shift) & 255;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rk = __popc(peers & below);
    if (valid && rk == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    if (valid && scatter) {
      int pos = run[dig] + rk;
      for (int ww = 0; ww < w; ++ww) pos += wcnt[ww][dig];
      if (pos >= 0 && pos < n)
        out[pos] = v;
      else
        atomicOr(err, 2);  // inconsistent counts: skip the store
    }
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) {
      s += wcnt[ww][t];
      wcnt[ww][t] = 0;
    }
    run[t] += s;
    __syncthreads();
  }
  if (!scatter) hist[(int64_t)t * ntiles + tile] = run[t];
}

// In-place exclusive scan of m non-negative counts whose total fits int32
// (one CTA; each thread scans a contiguous range).
__global__ void __launch_bounds__(1024) scan_kernel(int32_t* __restrict__ a, int64_t m) {
  __shared__ int64_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t lo = m * t / 1024, hi = m * (t + 1) / 1024;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  int64_t x = s;  // inclusive warp scan
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t v = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  int64_t run = x - s + (w > 0 ? wsum[w - 1] : 0);
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t v = a[i];
    a[i] = (int32_t)run;
    run += v;
  }
}

// Chunk bits of core k's order: 1 = the first slice continues from the
// previous chunk, 2 = the last slice continues into the next chunk, 4 = one
// slice only.
// A chunk holding the start of a slice that continues past it (its "head")
// also gets the last chunk of that slice in head_end (found by binary search
// on the sorted keys); other chunks get -1.
__global__ void chunk_info_kernel(const int32_t* __restrict__ keyk, const int32_t* __restrict__ perm,
                                  int64_t n, int64_t nchunks, uint8_t* __restrict__ info,
                                  int32_t* __restrict__ head_end) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t first = c * kChunk, last = min(n, first + kChunk) - 1;
    const int32_t kf = keyk[perm[first]], kl = keyk[perm[last]];
    uint8_t b = 0;
    if (c > 0 && keyk[perm[first - 1]] == kf) b |= 1;
    if (last + 1 < n && keyk[perm[last + 1]] == kl) b |= 2;
    if (kf == kl) b |= 4;
    info[c] = b;
    int32_t he = -1;
    if ((b & 2) && !((b & 4) && (b & 1))) {
      int64_t lo = last + 1, hi = n;  // first position past the slice lies in (last, n]
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (keyk[perm[mid]] == kl)
          lo = mid + 1;
        else
          hi = mid;
      }
      he = (int32_t)((lo - 1) / kChunk);
    }
    head_end[c] = he;
  }
}

// pos[perm[p]] = p: an entry's position in an order.
__global__ void inverse_perm_kernel(const int32_t* __restrict__ perm, int64_t n,
                                    int32_t* __restrict__ pos) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    pos[perm[p]] = (int32_t)p;
}

// ------------------------------------------------------------------ evaluation

struct PassArgs {
  int d, k;            // number of cores, the core of this order
  int backward;        // 0: forward (x), 1: gradient of core k
  int64_t n, nchunks;
  int dims[kEvalMaxD];
  int ranks[kEvalMaxD + 1];
  // cores left of core k (and core k in the forward and in the left row of
  // mode 1) come from `cores`, those right of it from `rcores`; the plain
  // backward passes the same set twice
  const float* cores[kEvalMaxD];
  const float* rcores[kEvalMaxD];
  const int32_t* ix;   // [d][n]
  const int32_t* perm; // [n] order of core k
  const uint8_t* info; // [nchunks]
  const int32_t* head_end;  // [nchunks]
  const float* gout;   // [n] (backward)
  float* grad;         // core k's gradient (backward)
  float* slots;        // [2 * nchunks][slot_elems] (backward)
  int slot_elems;
  float* out;          // [n] (forward)
  // d = 3 backward: the middle core's pass (mode 1) writes, per entry,
  // gout (G_2[:, i_2, :] G_3[:, i_3, 0]) at the entry's position in core 1's
  // order (rows1, r_1 wide) and gout G_1[0, i_1, :] G_2[:, i_2, :] at its
  // position in core 3's order (rows3, r_2 wide); the outer cores' passes
  // read those rows as their interface (mode 2: right side given, core 1;
  // mode 3: left side given, core 3).  Mode 0: interfaces from chains.
  int mode;
  int accumulate;      // forward: out += x (the tangent evaluation's passes) instead of out = x
  const int32_t* pos1;  // [n] entry -> position in core 1's order (mode 1)
  const int32_t* pos3;  // [n] entry -> position in core 3's order (mode 1)
  float* rows1;         // [n][r_1]
  float* rows3;         // [n][r_2]
  // shared-memory carve-up (in 4-byte words)
  int sL, sR, sT;      // row strides of the L, R and scratch buffers (0: buffer unused)
  int off_L, off_R, off_T, off_U;
  int off_U2;          // mode 1 with two core sets: core k's slice from rcores (else -1)
};

// Left chain step over the chunk: out[p][b] = sum_q in[p][q] G[(q*I + i_p) r1 + b]
// for p < cnt, b < r1 (in == null: the vector [1]).  Groups of W lanes own
// contiguous entry ranges; lane o keeps column o of the current slice in
// registers (NI >= round4(r0) of them) and reloads it when i_p changes.
// Padding lanes o in [r1, round4(r1)) write zeros.
template <int NI>
__device__ void left_step(const float* __restrict__ G, int I, int r0, int r1,
                          const int32_t* __restrict__ iv, const float* in, int sin, float* out,
                          int sout, int cnt) {
  const int W = group_width(r1);
  const int groups = kEvalThreads / W, E = kChunk / groups;
  const int t = threadIdx.x, g = t / W, o = t % W;
  if (o >= round4_dev(r1)) return;
  const bool live = o < r1;
  float2 col[NI / 2];  // (col[2h], col[2h+1]) = rows 2h, 2h+1 of column o
#pragma unroll
  for (int h = 0; h < NI / 2; ++h) col[h] = make_float2(0.0f, 0.0f);
  int cur = -1;
  const int p1 = min(cnt, (g + 1) * E);
  for (int p = g * E; p < p1; ++p) {
    const int i = iv[p];
    if (live && i != cur) {
      cur = i;
      const float* gp = G + (int64_t)i * r1 + o;
      const int64_t rs = (int64_t)I * r1;
#pragma unroll
      for (int h = 0; h < NI / 2; ++h) {
        if (2 * h < r0) col[h].x = __ldg(gp + 2 * h * rs);
        if (2 * h + 1 < r0) col[h].y = __ldg(gp + (2 * h + 1) * rs);
      }
    }
    // rows 4h, 4h+1, 4h+2, 4h+3 go to four running sums, added at the end
    float2 acc = make_float2(0.0f, 0.0f), acc2 = make_float2(0.0f, 0.0f);
    if (live) {
      const float* vp = in + p * sin;
#pragma unroll
      for (int q4 = 0; q4 < NI; q4 += 4) {
        if (q4 < r0) {
          const float4 v = *reinterpret_cast<const float4*>(vp + q4);
          acc = ffma2(make_float2(v.x, v.y), col[q4 / 2], acc);
          acc2 = ffma2(make_float2(v.z, v.w), col[q4 / 2 + 1], acc2);
        }
      }
    }
    out[p * sout + o] = (acc.x + acc.y) + (acc2.x + acc2.y);
  }
}

// Right chain step: out[p][q] = s_p sum_b G[(q*I + i_p) r1 + b] in[p][b] for
// q < r0, s_p = scale[p] (1 when scale is null).  Lane o keeps row o of the
// current slice (NI >= round4(r1) values).
template <int NI>
__device__ void right_step(const float* __restrict__ G, int I, int r0, int r1,
                           const int32_t* __restrict__ iv, const float* in, int sin, float* out,
                           int sout, int cnt, const float* scale) {
  const int W = group_width(r0);
  const int groups = kEvalThreads / W, E = kChunk / groups;
  const int t = threadIdx.x, g = t / W, o = t % W;
  if (o >= round4_dev(r0)) return;
  const bool live = o < r0;
  float2 row[NI / 2];  // (row[2h], row[2h+1]) = columns 2h, 2h+1 of row o
#pragma unroll
  for (int h = 0; h < NI / 2; ++h) row[h] = make_float2(0.0f, 0.0f);
  int cur = -1;
  const int p1 = min(cnt, (g + 1) * E);
  for (int p = g * E; p < p1; ++p) {
    const int i = iv[p];
    if (live && i != cur) {
      cur = i;
      const float* gp = G + ((int64_t)o * I + i) * r1;
#pragma unroll
      for (int h = 0; h < NI / 2; ++h) {
        if (2 * h < r1) row[h].x = __ldg(gp + 2 * h);
        if (2 * h + 1 < r1) row[h].y = __ldg(gp + 2 * h + 1);
      }
    }
    float2 acc = make_float2(0.0f, 0.0f), acc2 = make_float2(0.0f, 0.0f);
    if (live) {
      const float* vp = in + p * sin;
#pragma unroll
      for (int b4 = 0; b4 < NI; b4 += 4) {
        if (b4 < r1) {
          const float4 v = *reinterpret_cast<const float4*>(vp + b4);
          acc = ffma2(row[b4 / 2], make_float2(v.x, v.y), acc);
          acc2 = ffma2(row[b4 / 2 + 1], make_float2(v.z, v.w), acc2);
        }
      }
    }
    const float y = (acc.x + acc.y) + (acc2.x + acc2.y);
    out[p * sout + o] = scale ? y * scale[p] : y;
  }
}

// First step of a chain (the input is the vector [1]): a gather, spread over
// (entry, element) so every load is independent.  Left: the row
// G_1[0, i_p, :]; right: the column G_d[:, i_p, 0]; times scale[p] when
// scale is set.  Padding is zeroed.
template <bool LEFT>
__device__ void copy_step(const float* __restrict__ G, int I, int r, const int32_t* __restrict__ iv,
                          float* out, int sout, int cnt, const float* scale) {
  const int W = group_width(r), lw = __ffs(W) - 1, groups = kEvalThreads >> lw;
  const int t = threadIdx.x, o = t & (W - 1);
  if (o >= round4_dev(r)) return;
  const bool live = o < r;
  // eight gathers in flight per thread before their stores
  for (int pb = t >> lw; pb < cnt; pb += 8 * groups) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = pb + u * groups;
      v[u] = 0.0f;
      if (live && p < cnt) {
        const int64_t i = iv[p];
        v[u] = __ldg(LEFT ? G + i * r + o : G + (int64_t)o * I + i);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = pb + u * groups;
      if (p < cnt) out[p * sout + o] = scale ? v[u] * scale[p] : v[u];
    }
  }
}

// Stage the zero-padded slice G[:, i, :] (r0 x r1) as U[rLp][rRp], eight
// loads in flight per thread.
__device__ __forceinline__ void stage_slice(const float* __restrict__ G, int I, int i, int r0,
                                            int r1, float* U) {
  const int rLp = round4_dev(r0), rRp = round4_dev(r1), m = rLp * rRp;
  for (int eb = threadIdx.x; eb < m; eb += 8 * kEvalThreads) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = eb + u * kEvalThreads;
      const int q = e / rRp, b = e - q * rRp;
      v[u] = (e < m && q < r0 && b < r1) ? __ldg(G + ((int64_t)q * I + i) * r1 + b) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = eb + u * kEvalThreads;
      if (e < m) U[e] = v[u];
    }
  }
}

// Stage cnt given rows (rows[p][0..r), contiguous) as dst[p][0..round4(r)),
// zero padded; vector loads when r is a multiple of 4.
__device__ __forceinline__ void stage_rows(const float* __restrict__ rows, int r, int cnt,
                                           float* dst, int sd) {
  const int t = threadIdx.x;
  if ((r & 3) == 0) {
    const int r4 = r >> 2, m = cnt * r4;
    const float4* src = reinterpret_cast<const float4*>(rows);
    for (int fb = t; fb < m; fb += 8 * kEvalThreads) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int f = fb + u * kEvalThreads;
        v[u] = f < m ? __ldg(src + f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int f = fb + u * kEvalThreads;
        if (f < m) {
          const int p = f / r4, o = (f - p * r4) * 4;
          *reinterpret_cast<float4*>(dst + p * sd + o) = v[u];
        }
      }
    }
  } else {
    const int rp = round4_dev(r), m = cnt * rp;
    for (int eb = t; eb < m; eb += 8 * kEvalThreads) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = eb + u * kEvalThreads;
        const int p = e / rp, o = e - p * rp;
        v[u] = (e < m && o < r) ? __ldg(rows + (int64_t)p * r + o) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = eb + u * kEvalThreads;
        if (e < m) {
          const int p = e / rp, o = e - p * rp;
          dst[p * sd + o] = v[u];
        }
      }
    }
  }
}

// scale: per-entry factor applied to the step's output (null: none; left
// chains take it on their first copy only).
template <bool LEFT>
__device__ __forceinline__ void chain_step(const float* G, int I, int r0, int r1, const int32_t* iv,
                                           const float* in, int sin, float* out, int sout,
                                           int cnt, const float* scale) {
  if (in == nullptr) {
    if (LEFT)
      copy_step<true>(G, I, r1, iv, out, sout, cnt, scale);
    else
      copy_step<false>(G, I, r0, iv, out, sout, cnt, scale);
    return;
  }
  const int nin = LEFT ? r0 : r1;
  if (nin <= 4) {
    LEFT ? left_step<4>(G, I, r0, r1, iv, in, sin, out, sout, cnt)
         : right_step<4>(G, I, r0, r1, iv, in, sin, out, sout, cnt, scale);
  } else if (nin <= 8) {
    LEFT ? left_step<8>(G, I, r0, r1, iv, in, sin, out, sout, cnt)
         : right_step<8>(G, I, r0, r1, iv, in, sin, out, sout, cnt, scale);
  } else if (nin <= 16) {
    LEFT ? left_step<16>(G, I, r0, r1, iv, in, sin, out, sout, cnt)
         : right_step<16>(G, I, r0, r1, iv, in, sin, out, sout, cnt, scale);
  } else if (nin <= 32) {
    LEFT ? left_step<32>(G, I, r0, r1, iv, in, sin, out, sout, cnt)
         : right_step<32>(G, I, r0, r1, iv, in, sin, out, sout, cnt, scale);
  } else {
    LEFT ? left_step<64>(G, I, r0, r1, iv, in, sin, out, sout, cnt)
         : right_step<64>(G, I, r0, r1, iv, in, sin, out, sout, cnt, scale);
  }
}

// Mode 1 (d = 3, middle core, backward) for entry p: with L = gout a (Ls),
// c (Rs) and M staged in U (rLp x rRp, zero padded),
//   T[q][p] = gout sum_b M[q][b] c[b]       (core 1's row; row stride kChunk + 1)
//   rows3[pos3] = sum_q L[q] M[q][:]        (core 3's row)
// c and the running w stay in registers (NB >= round4(rR)).
template <int NB, bool DO_U, bool DO_W>
__device__ void emit_entry(const PassArgs& a, int p, const float* Ls, const float* Rs, float* Ts,
                           const float* U, float g, int pos3, int rL, int rR) {
  const int rLp = round4_dev(rL), rRp = round4_dev(rR);
  float2 cr[NB / 2], w[NB / 2];
  const float* rp = Rs + p * a.sR;
#pragma unroll
  for (int b4 = 0; b4 < NB; b4 += 4) {
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (DO_U && b4 < rRp) v = *reinterpret_cast<const float4*>(rp + b4);
    cr[b4 / 2] = make_float2(v.x, v.y);
    cr[b4 / 2 + 1] = make_float2(v.z, v.w);
    w[b4 / 2] = w[b4 / 2 + 1] = make_float2(0.0f, 0.0f);
  }
  const float* lp = Ls + p * a.sL;
  float* tp = Ts + p;  // u of entry p at Ts[q * (kChunk + 1) + p]
  for (int q4 = 0; q4 < rLp; q4 += 4) {
    float4 l = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (DO_W) l = *reinterpret_cast<const float4*>(lp + q4);
    const float lq[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const float* mrow = U + (q4 + qq) * rRp;
      const float2 ll = make_float2(lq[qq], lq[qq]);
      float2 ua = make_float2(0.0f, 0.0f), ub = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int b4 = 0; b4 < NB; b4 += 4) {
        if (b4 < rRp) {
          const float4 m = *reinterpret_cast<const float4*>(mrow + b4);
          const float2 m01 = make_float2(m.x, m.y), m23 = make_float2(m.z, m.w);
          if (DO_U) {
            ua = ffma2(m01, cr[b4 / 2], ua);
            ub = ffma2(m23, cr[b4 / 2 + 1], ub);
          }
          if (DO_W) {
            w[b4 / 2] = ffma2(ll, m01, w[b4 / 2]);
            w[b4 / 2 + 1] = ffma2(ll, m23, w[b4 / 2 + 1]);
          }
        }
      }
      if (DO_U) tp[(q4 + qq) * (kChunk + 1)] = ((ua.x + ua.y) + (ub.x + ub.y)) * g;
    }
  }
  if (!DO_W) return;
  float* dst = a.rows3 + (int64_t)pos3 * rR;
  if ((rR & 3) == 0) {
#pragma unroll
    for (int b4 = 0; b4 < NB; b4 += 4)
      if (b4 < rR)
        *reinterpret_cast<float4*>(dst + b4) =
            make_float4(w[b4 / 2].x, w[b4 / 2].y, w[b4 / 2 + 1].x, w[b4 / 2 + 1].y);
  } else {
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < rR) dst[b] = (b & 1) ? w[b / 2].y : w[b / 2].x;
  }
}

// One chunk of core k's order: interfaces, then the forward contraction or
// the gradient accumulation of core k.
__global__ void __launch_bounds__(kEvalThreads, 5) eval_pass_kernel(PassArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int segs[kChunk + 1];
  __shared__ int nseg;
  __shared__ int wstarts[kEvalThreads / 32];
  int32_t* ixs = reinterpret_cast<int32_t*>(sm);  // [d][kChunk] mode indices
  float* gs = sm + a.d * kChunk;                   // [kChunk] gout (backward)
  float* Ls = sm + a.off_L;
  float* Rs = sm + a.off_R;
  float* Ts = sm + a.off_T;
  float* U = sm + a.off_U;
  float* U2 = a.off_U2 >= 0 ? sm + a.off_U2 : U;
  const int t = threadIdx.x, k = a.k, d = a.d;
  const int64_t c = blockIdx.x, p0 = c * kChunk;
  const int cnt = (int)min((int64_t)kChunk, a.n - p0);
  int32_t* posA = reinterpret_cast<int32_t*>(gs + kChunk);  // [kChunk] (mode 1)
  int32_t* posB = posA + kChunk;                              // [kChunk] (mode 1)
  // (bounds-checked build: an entry id, mode index or position read from the
  // plan outside its range is counted and replaced by 0, so every later
  // access of the pass stays inside its buffer)
  for (int p = t; p < cnt; p += kEvalThreads) {
    int e = a.perm[p0 + p];
    if (!TT_IN(e, a.n)) e = 0;
    if (a.mode >= 2) {  // the given rows replace the chains: only i_k is needed
      const int v = a.ix[(int64_t)k * a.n + e];
      ixs[k * kChunk + p] = TT_IN(v, a.dims[k]) ? v : 0;
    } else {
      for (int j = 0; j < d; ++j) {
        const int v = a.ix[(int64_t)j * a.n + e];
        ixs[j * kChunk + p] = TT_IN(v, a.dims[j]) ? v : 0;
      }
      if (a.backward) gs[p] = a.gout[e];
      if (a.mode == 1) {
        const int pa = a.pos1[e], pb = a.pos3[e];
        posA[p] = TT_IN(pa, a.n) ? pa : 0;
        posB[p] = TT_IN(pb, a.n) ? pb : 0;
      }
    }
  }
  __syncthreads();
  {  // runs of equal i_k: starts found by warp ballots, listed in order
    const int32_t* key = ixs + k * kChunk;
    const bool start = t < cnt && (t == 0 || key[t] != key[t - 1]);
    const unsigned m = __ballot_sync(0xffffffffu, start);
    if ((t & 31) == 0) wstarts[t >> 5] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < kEvalThreads / 32; ++w) {
      off += w < (t >> 5) ? wstarts[w] : 0;
      tot += wstarts[w];
    }
    if (start) segs[off + __popc(m & ((1u << (t & 31)) - 1u))] = t;
    if (t == 0) {
      segs[tot] = cnt;
      nseg = tot;
    }
  }
  if (a.mode >= 2) {
    // interfaces given: the stored rows of this order on one side, [1] on the other
    const bool right = a.mode == 2;
    const float* rows = right ? a.rows1 : a.rows3;
    const int r = right ? a.ranks[1] : a.ranks[d - 1];
    float* dst = right ? Rs : Ls;
    float* one = right ? Ls : Rs;
    const int sd = right ? a.sR : a.sL, so = right ? a.sL : a.sR;
    stage_rows(rows + p0 * r, r, cnt, dst, sd);
    for (int p = t; p < cnt; p += kEvalThreads) {
      one[p * so] = 1.0f;
      one[p * so + 1] = one[p * so + 2] = one[p * so + 3] = 0.0f;
    }
  }
  // left interface over cores 0 .. k-1; step j writes Ls when k-1-j is even
  // (mode 1 scales it by gout)
  if (a.mode < 2 && k == 0) {
    for (int p = t; p < cnt; p += kEvalThreads) {
      Ls[p * a.sL] = 1.0f;
      Ls[p * a.sL + 1] = Ls[p * a.sL + 2] = Ls[p * a.sL + 3] = 0.0f;
    }
  }
  for (int j = 0; a.mode < 2 && j < k; ++j) {
    const bool toL = ((k - 1 - j) & 1) == 0;
    float* dst = toL ? Ls : Ts;
    const float* src = j == 0 ? nullptr : (toL ? Ts : Ls);
    chain_step<true>(a.cores[j], a.dims[j], a.ranks[j], a.ranks[j + 1], ixs + j * kChunk, src,
                     toL ? a.sT : a.sL, dst, toL ? a.sL : a.sT, cnt,
                     (a.mode == 1 && j == k - 1) ? gs : nullptr);
    __syncthreads();
  }
  // right interface over cores d-1 .. k+1; step s (core d-1-s) writes Rs when nR-1-s is even
  const int nR = a.mode < 2 ? d - 1 - k : 0;
  if (a.mode < 2 && nR == 0) {  // R = [1] (times gout in the backward)
    for (int p = t; p < cnt; p += kEvalThreads) {
      Rs[p * a.sR] = a.backward ? gs[p] : 1.0f;
      Rs[p * a.sR + 1] = Rs[p * a.sR + 2] = Rs[p * a.sR + 3] = 0.0f;
    }
  }
  for (int s = 0; s < nR; ++s) {
    const int j = d - 1 - s;
    const bool toR = ((nR - 1 - s) & 1) == 0;
    float* dst = toR ? Rs : Ts;
    const float* src = s == 0 ? nullptr : (toR ? Ts : Rs);
    // the backward's last right step folds in gout (mode 1: the left side has it)
    chain_step<false>(a.rcores[j], a.dims[j], a.ranks[j], a.ranks[j + 1], ixs + j * kChunk, src,
                      toR ? a.sT : a.sR, dst, toR ? a.sR : a.sT, cnt,
                      (a.backward && a.mode == 0 && s == nR - 1) ? gs : nullptr);
    __syncthreads();
  }
  const int rL = a.ranks[k], rR = a.ranks[k + 1], rLp = round4_dev(rL), rRp = round4_dev(rR);
  const float* Gk = a.cores[k];
  const int I = a.dims[k];
  __syncthreads();

  if (!a.backward) {
    // x_p = L_p^T G_k[:, i, :] R_p, the slice staged once per run of equal i_k
    for (int s = 0; s < nseg; ++s) {
      const int s0 = segs[s], s1 = segs[s + 1];
      const int i = ixs[k * kChunk + s0];
      stage_slice(Gk, I, i, rL, rR, U);
      __syncthreads();
      const int p = t;
      if (p >= s0 && p < s1) {
        const float* lp = Ls + p * a.sL;
        const float* rp = Rs + p * a.sR;
        float x = 0.0f;
        for (int bc = 0; bc < rRp; bc += 16) {
          float2 u[8];  // u[b] = sum_q L[q] M[q][bc + b], pairs of b
#pragma unroll
          for (int j = 0; j < 8; ++j) u[j] = make_float2(0.0f, 0.0f);
          for (int q4 = 0; q4 < rLp; q4 += 4) {
            const float4 l = *reinterpret_cast<const float4*>(lp + q4);
            const float lq[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float* mrow = U + (q4 + qq) * rRp + bc;
              const float2 ll = make_float2(lq[qq], lq[qq]);
#pragma unroll
              for (int j4 = 0; j4 < 4; ++j4) {
                if (bc + 4 * j4 < rRp) {
                  const float4 m = *reinterpret_cast<const float4*>(mrow + 4 * j4);
                  u[2 * j4] = ffma2(ll, make_float2(m.x, m.y), u[2 * j4]);
                  u[2 * j4 + 1] = ffma2(ll, make_float2(m.z, m.w), u[2 * j4 + 1]);
                }
              }
            }
          }
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            if (bc + 4 * j4 < rRp) {
              const float4 r = *reinterpret_cast<const float4*>(rp + bc + 4 * j4);
              x = fmaf(u[2 * j4].x, r.x, x);
              x = fmaf(u[2 * j4].y, r.y, x);
              x = fmaf(u[2 * j4 + 1].x, r.z, x);
              x = fmaf(u[2 * j4 + 1].y, r.w, x);
            }
          }
        }
        const int o = a.perm[p0 + p];
        if (TT_IN(o, a.n)) a.out[o] = a.accumulate ? a.out[o] + x : x;
      }
      __syncthreads();
    }
    return;
  }

  if (a.mode == 1) {
    // per run of equal i_2: stage M = G_2[:, i_2, :]; per entry (L = gout a,
    // R = c): u = M c -> gout u into the scratch rows, w = L^T M -> rows3
    // (two core sets: u takes the right set's slice, w the left set's)
    for (int s = 0; s < nseg; ++s) {
      const int s0 = segs[s], s1 = segs[s + 1];
      const int i = ixs[k * kChunk + s0];
      stage_slice(Gk, I, i, rL, rR, U);
      if (U2 != U) stage_slice(a.rcores[k], I, i, rL, rR, U2);
      __syncthreads();
      if (t >= s0 && t < s1) {
        // u = M c takes the right set's slice, w = L^T M the left set's: with
        // two sets the entry is emitted in two halves
        if (U2 != U) {
          if (rRp <= 8) {
            emit_entry<8, true, false>(a, t, Ls, Rs, Ts, U2, gs[t], posB[t], rL, rR);
            emit_entry<8, false, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
          } else if (rRp <= 16) {
            emit_entry<16, true, false>(a, t, Ls, Rs, Ts, U2, gs[t], posB[t], rL, rR);
            emit_entry<16, false, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
          } else {
            emit_entry<32, true, false>(a, t, Ls, Rs, Ts, U2, gs[t], posB[t], rL, rR);
            emit_entry<32, false, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
          }
        } else if (rRp <= 4) {
          emit_entry<4, true, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
        } else if (rRp <= 8) {
          emit_entry<8, true, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
        } else if (rRp <= 16) {
          emit_entry<16, true, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
        } else {
          emit_entry<32, true, true>(a, t, Ls, Rs, Ts, U, gs[t], posB[t], rL, rR);
        }
      }
      __syncthreads();
    }
    // the u rows, coalesced, to their positions in core 1's order
    {
      const int W = group_width(rL), lw = __ffs(W) - 1, groups = kEvalThreads >> lw;
      const int o = t & (W - 1);
      if (o < rL)
        for (int p = t >> lw; p < cnt; p += groups)
          a.rows1[(int64_t)posA[p] * rL + o] = Ts[o * (kChunk + 1) + p];
    }
    __syncthreads();
  }

  // backward (R_p already carries gout_p; mode 1: L_p does):
  // dG_k[:, i, :] += sum_p L_p R_p^T per run, in 4 x 4 tiles: group g of
  // ntiles threads takes entries s0 + g, s0 + g + G, ...; groups fold in order.
  const int tb = rRp / 4, ntiles = (rLp / 4) * tb;
  const int G = ntiles >= kEvalThreads ? 1 : kEvalThreads / ntiles;
  const int grp = ntiles >= kEvalThreads ? 0 : t / ntiles;
  const bool active = t < G * min(ntiles, kEvalThreads);
  const int nt = ntiles > kEvalThreads ? 2 : 1;  // tiles per thread (ntiles <= 256)
  int tq0[2], tb0[2];
  bool own[2];
  for (int u = 0; u < 2; ++u) {
    const int tile = ntiles > kEvalThreads ? t + u * kEvalThreads : t % ntiles;
    own[u] = active && u < nt && tile < ntiles;
    tq0[u] = own[u] ? (tile / tb) * 4 : 0;
    tb0[u] = own[u] ? (tile % tb) * 4 : 0;
  }
  const uint8_t inf = a.info[c];
  float* F = a.mode == 1 ? Ts : U;  // mode 1: the scratch rows are written out by now
  for (int s = 0; s < nseg; ++s) {
    const int s0 = segs[s], s1 = segs[s + 1];
    const int i = ixs[k * kChunk + s0];
    float acc[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[u][j] = 0.0f;
    if (active) {
      for (int p = s0 + grp; p < s1; p += G) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (own[u]) {
            const float4 l = *reinterpret_cast<const float4*>(Ls + p * a.sL + tq0[u]);
            const float4 r = *reinterpret_cast<const float4*>(Rs + p * a.sR + tb0[u]);
            const float lv[4] = {l.x, l.y, l.z, l.w};
            const float2 r01 = make_float2(r.x, r.y), r23 = make_float2(r.z, r.w);
#pragma unroll
            for (int qa = 0; qa < 4; ++qa) {
              const float2 ll = make_float2(lv[qa], lv[qa]);
              float2 a01 = make_float2(acc[u][qa * 4], acc[u][qa * 4 + 1]);
              float2 a23 = make_float2(acc[u][qa * 4 + 2], acc[u][qa * 4 + 3]);
              a01 = ffma2(ll, r01, a01);
              a23 = ffma2(ll, r23, a23);
              acc[u][qa * 4] = a01.x;
              acc[u][qa * 4 + 1] = a01.y;
              acc[u][qa * 4 + 2] = a23.x;
              acc[u][qa * 4 + 3] = a23.y;
            }
          }
        }
      }
    }
    const bool shared = (s == 0 && (inf & 1)) || (s == nseg - 1 && (inf & 2));
    float* slot = a.slots + (2 * c + (s == 0 ? 0 : 1)) * (int64_t)a.slot_elems;
    if (G > 1) {
      // fold the G group partials of every tile element in group order, one
      // element per thread; F[j][group][tile] keeps both sides conflict-free
      const int GN = G * ntiles;
      if (active) {
#pragma unroll
        for (int j = 0; j < 16; ++j) F[j * GN + t] = acc[0][j];
      }
      __syncthreads();
      for (int e = t; e < ntiles * 16; e += kEvalThreads) {
        const int tile = e % ntiles, j = e / ntiles;
        float v = 0.0f;
        for (int g = 0; g < G; ++g) v += F[j * GN + g * ntiles + tile];
        const int q = (tile / tb) * 4 + (j >> 2), b = (tile % tb) * 4 + (j & 3);
        if (shared)
          slot[q * rRp + b] = v;
        else if (q < rL && b < rR)
          a.grad[((int64_t)q * I + i) * rR + b] += v;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!own[u]) continue;
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const int q = tq0[u] + qa, b = tb0[u] + bb;
            if (shared)
              slot[q * rRp + b] = acc[u][qa * 4 + bb];
            else if (q < rL && b < rR)
              a.grad[((int64_t)q * I + i) * rR + b] += acc[u][qa * 4 + bb];
          }
      }
    }
    __syncthreads();
  }
}

// Slices of core k that straddle chunk boundaries: the chunk holding a
// slice's start (its "head") adds the slice's partials in chunk order.
__global__ void eval_fixup_kernel(PassArgs a) {
  const int64_t c = blockIdx.x;
  const int64_t cend = a.head_end[c];
  if (cend < 0) return;
  const bool single = a.info[c] & 4;
  const int k = a.k, rL = a.ranks[k], rR = a.ranks[k + 1], rRp = round4_dev(rR);
  const int rLp = round4_dev(rL), I = a.dims[k];
  const int64_t last = min(a.n, (c + 1) * kChunk) - 1;
  int el = a.perm[last];
  if (!TT_IN(el, a.n)) el = 0;
  int i = a.ix[(int64_t)k * a.n + el];
  if (!TT_IN(i, I)) i = 0;
  for (int e = threadIdx.x; e < rLp * rRp; e += blockDim.x) {
    const int q = e / rRp, b = e % rRp;
    if (q >= rL || b >= rR) continue;
    float v = a.slots[(2 * c + (single ? 0 : 1)) * (int64_t)a.slot_elems + e];
#pragma unroll 8
    for (int64_t cc = c + 1; cc <= cend; ++cc) v += a.slots[2 * cc * (int64_t)a.slot_elems + e];
    a.grad[((int64_t)q * I + i) * rR + b] += v;
  }
}

// ------------------------------------------------------------------ tangent gauge
//
// For an m x r left unfolding U with orthonormal columns and the increment Y
// of the same shape: Y <- Y - U (U^T Y).  S = U^T Y is summed by row blocks
// (gauge_gram_kernel: block b takes rows [b*rows, (b+1)*rows) and writes its
// partial; products in FP32 over 32-row tiles, the tiles' sums added in
// FP64, since GB300 issues FP64 at 1/64 of the FP32 rate), the partials in
// block order (gauge_reduce_kernel), then every row is updated from S in
// FP64 (gauge_apply_kernel).

constexpr int kGaugeThreads = 256;
constexpr int kGaugeRows = 128;     // rows per partial sum
constexpr int kGaugeMaxBlocks = 152;
constexpr int kGaugeTile = 32;      // rows staged per round

int gauge_blocks(int64_t m) {
  return (int)std::min<int64_t>(kGaugeMaxBlocks, (m + kGaugeRows - 1) / kGaugeRows);
}

__global__ void __launch_bounds__(kGaugeThreads) gauge_gram_kernel(const float* __restrict__ U,
                                                                   const float* __restrict__ Y,
                                                                   int64_t m, int r, int64_t rows,
                                                                   double* __restrict__ part) {
  __shared__ float us[kGaugeTile * kEvalMaxR], ys[kGaugeTile * kEvalMaxR];
  const int t = threadIdx.x, rr = r * r;
  const int64_t i0 = blockIdx.x * rows, i1 = min(m, i0 + rows);
  double acc[kEvalMaxR * kEvalMaxR / kGaugeThreads];
#pragma unroll
  for (int j = 0; j < kEvalMaxR * kEvalMaxR / kGaugeThreads; ++j) acc[j] = 0.0;
  for (int64_t ib = i0; ib < i1; ib += kGaugeTile) {
    const int nr = (int)min((int64_t)kGaugeTile, i1 - ib);
    __syncthreads();
    for (int e = t; e < nr * r; e += kGaugeThreads) {
      us[e] = U[ib * r + e];
      ys[e] = Y[ib * r + e];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kEvalMaxR * kEvalMaxR / kGaugeThreads; ++j) {
      const int e = t + j * kGaugeThreads;
      if (e < rr) {
        const int a = e / r, b = e - a * r;
        float v = 0.0f;
        for (int q = 0; q < nr; ++q) v = fmaf(us[q * r + a], ys[q * r + b], v);
        acc[j] += (double)v;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kEvalMaxR * kEvalMaxR / kGaugeThreads; ++j) {
    const int e = t + j * kGaugeThreads;
    if (e < rr) part[(int64_t)blockIdx.x * rr + e] = acc[j];
  }
}

__global__ void gauge_reduce_kernel(const double* __restrict__ part, int nblk, int rr,
                                    double* __restrict__ S) {
  for (int e = threadIdx.x; e < rr; e += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += part[(int64_t)b * rr + e];
    S[e] = v;
  }
}

__global__ void __launch_bounds__(kGaugeThreads) gauge_apply_kernel(const float* __restrict__ U,
                                                                    float* __restrict__ Y,
                                                                    int64_t m, int r,
                                                                    const double* __restrict__ S) {
  __shared__ double ss[kEvalMaxR * kEvalMaxR];
  for (int e = threadIdx.x; e < r * r; e += kGaugeThreads) ss[e] = S[e];
  __syncthreads();
  const int64_t total = m * r;
  for (int64_t e = (int64_t)blockIdx.x * kGaugeThreads + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kGaugeThreads) {
    const int64_t i = e / r;
    const int b = (int)(e - i * r);
    const float* ui = U + i * r;
    double v = 0.0;
    for (int a = 0; a < r; ++a) v = fma((double)ui[a], ss[a * r + b], v);
    Y[e] = (float)((double)Y[e] - v);
  }
}

}  // namespace

// Byte layout of a plan's device block (computed from d, dims, ranks, n).
struct Layout {
  int64_t nchunks = 0, ntiles = 0;
  int slot_elems = 0;
  int pivot = 0;
  int nb[kEvalMaxD];
  bool fast3 = false;  // d = 3 with round4(r_2) <= 32: the backward stores per-entry rows
  size_t off_err = 0, off_ix = 0, off_perm = 0, off_info = 0, off_head = 0, off_slots = 0,
         off_pos = 0, off_rows1 = 0, off_rows3 = 0, off_tmp = 0, off_hist = 0, off_gauge = 0,
         total = 0;
};

bool valid_shape(int d, const int64_t* dims, const int64_t* ranks, int64_t n, const char** why) {
  if (d < 1 || d > kEvalMaxD) return *why = "d must be in [1, 16]", false;
  if (n < 0 || n > INT32_MAX) return *why = "n must be in [0, 2^31)", false;
  int64_t total = 1;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > INT32_MAX) return *why = "dims must be in [1, 2^31)", false;
    if (total > INT64_MAX / dims[k]) return *why = "prod(dims) overflows int64", false;
    total *= dims[k];
  }
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > kEvalMaxR) return *why = "ranks must be in [1, 64]", false;
  if (ranks[0] != 1 || ranks[d] != 1) return *why = "r_0 = r_d = 1", false;
  return true;
}

Layout layout_of(int d, const int64_t* dims, const int64_t* ranks, int64_t n) {
  Layout L;
  L.nchunks = (n + kChunk - 1) / kChunk;
  L.ntiles = (n + kSortTile - 1) / kSortTile;
  int64_t best = -1;
  for (int k = 0; k < d; ++k) {
    const int64_t cost = ranks[k] * ranks[k + 1];
    L.slot_elems = std::max<int>(L.slot_elems, round4((int)ranks[k]) * round4((int)ranks[k + 1]));
    if (cost > best) best = cost, L.pivot = k;
    int nb = -1;
    int64_t nc = -1;
    if (k > 0) nb = k - 1, nc = ranks[k - 1] * ranks[k];
    if (k + 1 < d && ranks[k + 1] * ranks[k + 2] > nc) nb = k + 1;
    L.nb[k] = nb;
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.off_err = take(sizeof(int32_t));
  L.off_ix = take((size_t)d * n * sizeof(int32_t));
  L.off_perm = take((size_t)d * n * sizeof(int32_t));
  L.off_info = take((size_t)d * L.nchunks);
  L.off_head = take((size_t)d * L.nchunks * sizeof(int32_t));
  L.off_slots = take((size_t)2 * L.nchunks * L.slot_elems * sizeof(float));
  L.fast3 = d == 3 && round4((int)ranks[2]) <= 32;
  if (L.fast3) {
    L.off_pos = take((size_t)2 * n * sizeof(int32_t));
    L.off_rows1 = take((size_t)n * ranks[1] * sizeof(float));
    L.off_rows3 = take((size_t)n * ranks[2] * sizeof(float));
  }
  L.off_tmp = take((size_t)n * sizeof(int32_t));
  L.off_hist = take((size_t)256 * L.ntiles * sizeof(int32_t));
  // tangent projection: the FP64 partials of U_k^T Y_k (k < d-1), then S
  size_t gauge = 0;
  for (int k = 0; k + 1 < d; ++k)
    gauge = std::max(gauge, (size_t)(gauge_blocks(ranks[k] * dims[k]) + 1) * ranks[k + 1] *
                                ranks[k + 1] * sizeof(double));
  L.off_gauge = take(gauge);
  L.total = o;
  return L;
}

// Shared-memory carve-up of core k's pass (words) and its byte size.
size_t pass_smem(PassArgs& a, const int64_t* ranks) {
  int rmax = 1;
  for (int j = 0; j <= a.d; ++j) rmax = std::max<int>(rmax, (int)ranks[j]);
  const int rL = (int)ranks[a.k], rR = (int)ranks[a.k + 1];
  // the left buffer holds every output of the left chain (lengths ranks[1..k];
  // its steps alternate with the scratch buffer), the right one every output
  // of the right chain (ranks[k+1..d-1])
  int mL = 1, mR = 1;
  for (int j = 1; j <= a.k; ++j) mL = std::max<int>(mL, (int)ranks[j]);
  for (int j = a.k + 1; j < a.d; ++j) mR = std::max<int>(mR, (int)ranks[j]);
  a.sL = round4(mL) + 4;
  a.sR = round4(mR) + 4;
  // scratch: chains of two or more steps; mode 1 keeps its u rows there
  const bool needT = a.mode == 1 || (a.mode == 0 && (a.k >= 2 || a.d - 1 - a.k >= 2));
  a.sT = needT ? round4(rmax) + 4 : 0;
  if (a.mode == 1) a.sT = std::max(a.sT, 16);  // also the fold buffer (128 x 16 words)
  a.off_L = (a.d + 3) * kChunk;  // mode indices, gout and two position lists first
  a.off_R = a.off_L + kChunk * a.sL;
  a.off_T = a.off_R + kChunk * a.sR;
  const int usz = a.mode == 1 ? round4(rL) * round4(rR)
                              : std::max(round4(rL) * round4(rR), kEvalThreads * 16);
  // the staging / fold buffer is only used after the chains: it shares the
  // scratch buffer when that is large enough
  a.off_U2 = -1;
  if (a.mode != 1 && a.sT > 0 && kChunk * a.sT >= usz) {
    a.off_U = a.off_T;
    return (size_t)(a.off_T + kChunk * a.sT) * sizeof(float);
  }
  a.off_U = a.off_T + kChunk * a.sT;
  if (a.mode == 1 && a.rcores[a.k] != a.cores[a.k]) {
    a.off_U2 = a.off_U + usz;  // usz is a multiple of 16 words: float4-aligned
    return (size_t)(a.off_U2 + usz) * sizeof(float);
  }
  return (size_t)(a.off_U + usz) * sizeof(float);
}

int radix_digits(int64_t extent) { return (bits_of(extent - 1) + 7) / 8; }

cudaError_t configure_once() {
  static cudaError_t st = [] {
    return cudaFuncSetAttribute(eval_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                160 * 1024);
  }();
  return st;
}

TT_BOUNDS_READER(bounds_masked)

}  // namespace ttk

struct tt_eval_plan {
  int32_t d;
  int64_t n;
  int64_t dims[TT_MAXD];
  int64_t ranks[TT_MAXD + 1];
  char* base;
  tt_free_fn free_fn;  // null: base came from cudaMallocAsync
  void* alloc_ctx;
  ttk::Layout L;
};

namespace {

tt_status plan_fail(tt_status s, const char* msg) {
  ttk::set_last_error(msg);
  return s;
}

tt_status plan_cuda_fail(cudaError_t e, const char* what) {
  static thread_local char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  ttk::set_last_error(buf);
  return TT_ECUDA;
}

#define EV_CK(expr, what)                          \
  do {                                             \
    const cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return plan_cuda_fail(e_, what); \
  } while (0)

ttk::PassArgs pass_args(const tt_eval_plan* P, const float* const* cores,
                        const float* const* rcores, int k, int backward) {
  ttk::PassArgs a;
  std::memset(&a, 0, sizeof a);
  a.d = P->d;
  a.k = k;
  a.backward = backward;
  a.n = P->n;
  a.nchunks = P->L.nchunks;
  for (int j = 0; j < P->d; ++j) {
    a.dims[j] = (int)P->dims[j];
    a.cores[j] = cores[j];
    a.rcores[j] = rcores[j];
  }
  for (int j = 0; j <= P->d; ++j) a.ranks[j] = (int)P->ranks[j];
  a.ix = reinterpret_cast<const int32_t*>(P->base + P->L.off_ix);
  a.perm = reinterpret_cast<const int32_t*>(P->base + P->L.off_perm) + (int64_t)k * P->n;
  a.info = reinterpret_cast<const uint8_t*>(P->base + P->L.off_info) + (int64_t)k * P->L.nchunks;
  a.head_end = reinterpret_cast<const int32_t*>(P->base + P->L.off_head) + (int64_t)k * P->L.nchunks;
  a.slots = reinterpret_cast<float*>(P->base + P->L.off_slots);
  a.slot_elems = P->L.slot_elems;
  if (P->L.fast3) {
    a.pos1 = reinterpret_cast<const int32_t*>(P->base + P->L.off_pos);
    a.pos3 = a.pos1 + P->n;
    a.rows1 = reinterpret_cast<float*>(P->base + P->L.off_rows1);
    a.rows3 = reinterpret_cast<float*>(P->base + P->L.off_rows3);
  }
  return a;
}

}  // namespace

extern "C" {

tt_status tt_eval_plan_create(int32_t d, const int64_t* dims, const int64_t* ranks,
                              const int64_t* idx, int64_t n, tt_alloc_fn alloc, tt_free_fn free_fn,
                              void* alloc_ctx, void* stream, tt_eval_plan** out) {
  ttk::set_last_error("");
  if (!out) return plan_fail(TT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dims || !ranks || (n > 0 && !idx)) return plan_fail(TT_EINVAL, "NULL argument");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return plan_fail(TT_EINVAL, "give both alloc and free_fn, or neither");
  const char* why = "";
  if (!ttk::valid_shape(d, dims, ranks, n, &why)) return plan_fail(TT_EINVAL, why);
  cudaStream_t st = (cudaStream_t)stream;
  EV_CK(ttk::configure_once(), "masked evaluation setup");
  tt_eval_plan* P = new tt_eval_plan();
  P->d = d;
  P->n = n;
  for (int k = 0; k < d; ++k) P->dims[k] = dims[k];
  for (int k = 0; k <= d; ++k) P->ranks[k] = ranks[k];
  P->L = ttk::layout_of(d, dims, ranks, n);
  P->free_fn = free_fn;
  P->alloc_ctx = alloc_ctx;
  void* base = nullptr;
  if (alloc) {
    base = alloc(P->L.total, stream, alloc_ctx);
    if (!base) {
      delete P;
      return plan_fail(TT_ENOMEM, "plan allocation failed");
    }
  } else {
    const cudaError_t e = cudaMallocAsync(&base, P->L.total, st);
    if (e != cudaSuccess) {
      delete P;
      return plan_cuda_fail(e, "plan allocation");
    }
  }
  P->base = (char*)base;
  auto bail = [&](tt_status s) {
    tt_eval_plan_destroy(P, stream);
    return s;
  };
  int32_t* err = reinterpret_cast<int32_t*>(P->base + P->L.off_err);
  int32_t* ix = reinterpret_cast<int32_t*>(P->base + P->L.off_ix);
  int32_t* perm = reinterpret_cast<int32_t*>(P->base + P->L.off_perm);
  uint8_t* info = reinterpret_cast<uint8_t*>(P->base + P->L.off_info);
  int32_t* tmp = reinterpret_cast<int32_t*>(P->base + P->L.off_tmp);
  int32_t* hist = reinterpret_cast<int32_t*>(P->base + P->L.off_hist);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return bail(plan_cuda_fail(e, "plan setup"));
  if (n > 0) {
    ttk::DecodeArgs da;
    da.d = d;
    da.total = 1;
    for (int k = 0; k < d; ++k) da.dims[k] = dims[k], da.total *= dims[k];
    ttk::count_launch();
    ttk::decode_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(idx, n, da,
                                                                                    ix, err);
    for (int k = 0; k < d && e == cudaSuccess; ++k) {
      // LSD passes: digits of i_nb first, then of i_k (at least one pass)
      struct Pass { int mode, shift; };
      std::vector<Pass> passes;
      const int nb = P->L.nb[k];
      if (nb >= 0)
        for (int g = 0; g < ttk::radix_digits(dims[nb]); ++g) passes.push_back({nb, 8 * g});
      const int dk = std::max(1, ttk::radix_digits(dims[k]));
      for (int g = 0; g < dk; ++g) passes.push_back({k, 8 * g});
      const int np = (int)passes.size();
      int32_t* pk = perm + (int64_t)k * n;
      const int32_t* src = nullptr;
      for (int s = 0; s < np && e == cudaSuccess; ++s) {
        int32_t* dst = ((np - 1 - s) % 2 == 0) ? pk : tmp;
        const int32_t* key = ix + (int64_t)passes[s].mode * n;
        const unsigned g = (unsigned)P->L.ntiles;
        ttk::count_launch(3);
        ttk::radix_kernel<<<g, 256, 0, st>>>(src, dst, n, key, passes[s].shift, hist, P->L.ntiles, 0,
                                            err);
        ttk::scan_kernel<<<1, 1024, 0, st>>>(hist, 256 * P->L.ntiles);
        ttk::radix_kernel<<<g, 256, 0, st>>>(src, dst, n, key, passes[s].shift, hist, P->L.ntiles, 1,
                                            err);
        e = cudaGetLastError();
        src = dst;
      }
      ttk::count_launch();
      ttk::chunk_info_kernel<<<(int)std::min<int64_t>((P->L.nchunks + 255) / 256, 4096), 256, 0, st>>>(
          ix + (int64_t)k * n, pk, n, P->L.nchunks, info + (int64_t)k * P->L.nchunks,
          reinterpret_cast<int32_t*>(P->base + P->L.off_head) + (int64_t)k * P->L.nchunks);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess && P->L.fast3) {
      int32_t* pos = reinterpret_cast<int32_t*>(P->base + P->L.off_pos);
      const int g = (int)std::min<int64_t>((n + 255) / 256, 4096);
      ttk::count_launch(2);
      ttk::inverse_perm_kernel<<<g, 256, 0, st>>>(perm, n, pos);
      ttk::inverse_perm_kernel<<<g, 256, 0, st>>>(perm + 2 * n, n, pos + n);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bail(plan_cuda_fail(e, "plan build"));
  }
  int32_t bad = 0;
  e = cudaMemcpyAsync(&bad, err, sizeof bad, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(plan_cuda_fail(e, "plan build"));
  if (bad & 1) return bail(plan_fail(TT_EINVAL, "an index lies outside [0, prod(dims))"));
  if (bad) return bail(plan_fail(TT_ECUDA, "plan build: inconsistent sort counts"));
  *out = P;
  return TT_OK;
}

void tt_eval_plan_destroy(tt_eval_plan* plan, void* stream) {
  if (!plan) return;
  if (plan->base) {
    if (plan->free_fn)
      plan->free_fn(plan->base, stream, plan->alloc_ctx);
    else
      cudaFreeAsync(plan->base, (cudaStream_t)stream);
  }
  delete plan;
}

size_t tt_eval_plan_device_bytes(const tt_eval_plan* plan) { return plan ? plan->L.total : 0; }

tt_status tt_eval_plan_at(const tt_eval_plan* plan, const float* const* cores, float* out,
                          void* stream) {
  ttk::set_last_error("");
  if (!plan || !cores || (plan->n > 0 && !out)) return plan_fail(TT_EINVAL, "NULL argument");
  for (int k = 0; k < plan->d; ++k)
    if (!cores[k]) return plan_fail(TT_EINVAL, "NULL core");
  if (plan->n == 0) return TT_OK;
  ttk::PassArgs a = pass_args(plan, cores, cores, plan->L.pivot, 0);
  a.out = out;
  const size_t sm = ttk::pass_smem(a, plan->ranks);
  ttk::count_launch();
  ttk::eval_pass_kernel<<<(unsigned)plan->L.nchunks, ttk::kEvalThreads, sm, (cudaStream_t)stream>>>(a);
  EV_CK(cudaGetLastError(), "masked evaluation");
  return TT_OK;
}

tt_status tt_eval_plan_backward(tt_eval_plan* plan, const float* const* cores, const float* gout,
                                float* const* grads, void* stream) {
  return tt_eval_plan_backward_mixed(plan, cores, cores, gout, grads, stream);
}

tt_status tt_eval_plan_backward_mixed(tt_eval_plan* plan, const float* const* left,
                                      const float* const* right, const float* gout,
                                      float* const* grads, void* stream) {
  ttk::set_last_error("");
  if (!plan || !left || !right || !grads || (plan->n > 0 && !gout))
    return plan_fail(TT_EINVAL, "NULL argument");
  for (int k = 0; k < plan->d; ++k)
    if (!left[k] || !right[k] || !grads[k]) return plan_fail(TT_EINVAL, "NULL core or gradient");
  if (plan->n == 0) return TT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // d = 3: the middle core's pass first (it writes the outer cores' rows)
  const int order3[3] = {1, 0, 2};
  for (int kk = 0; kk < plan->d; ++kk) {
    const int k = plan->L.fast3 ? order3[kk] : kk;
    ttk::PassArgs a = pass_args(plan, left, right, k, 1);
    a.gout = gout;
    a.grad = grads[k];
    if (plan->L.fast3) a.mode = k == 1 ? 1 : (k == 0 ? 2 : 3);
    const size_t sm = ttk::pass_smem(a, plan->ranks);
    ttk::count_launch(2);
    ttk::eval_pass_kernel<<<(unsigned)plan->L.nchunks, ttk::kEvalThreads, sm, st>>>(a);
    ttk::eval_fixup_kernel<<<(unsigned)plan->L.nchunks, ttk::kEvalThreads, 0, st>>>(a);
    EV_CK(cudaGetLastError(), "masked evaluation backward");
  }
  return TT_OK;
}

tt_status tt_tangent_project(tt_eval_plan* plan, const float* const* U, const float* const* V,
                             const float* z, float* const* dU, void* stream) {
  ttk::set_last_error("");
  if (!plan || !U || !V || !dU || (plan->n > 0 && !z)) return plan_fail(TT_EINVAL, "NULL argument");
  for (int k = 0; k < plan->d; ++k)
    if (!U[k] || !V[k] || !dU[k]) return plan_fail(TT_EINVAL, "NULL core or increment");
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < plan->d; ++k)
    EV_CK(cudaMemsetAsync(dU[k], 0,
                          (size_t)plan->ranks[k] * plan->dims[k] * plan->ranks[k + 1] * sizeof(float),
                          st),
          "tangent projection");
  if (plan->n == 0) return TT_OK;
  const tt_status s = tt_eval_plan_backward_mixed(plan, U, V, z, dU, stream);
  if (s != TT_OK) return s;
  double* part = reinterpret_cast<double*>(plan->base + plan->L.off_gauge);
  for (int k = 0; k + 1 < plan->d; ++k) {
    const int64_t m = plan->ranks[k] * plan->dims[k];
    const int r = (int)plan->ranks[k + 1];
    const int nblk = ttk::gauge_blocks(m);
    const int64_t rows = (m + nblk - 1) / nblk;
    double* S = part + (int64_t)nblk * r * r;
    const int napply = (int)std::min<int64_t>((m * r + ttk::kGaugeThreads - 1) / ttk::kGaugeThreads,
                                              1024);
    ttk::count_launch(3);
    ttk::gauge_gram_kernel<<<nblk, ttk::kGaugeThreads, 0, st>>>(U[k], dU[k], m, r, rows, part);
    ttk::gauge_reduce_kernel<<<1, ttk::kGaugeThreads, 0, st>>>(part, nblk, r * r, S);
    ttk::gauge_apply_kernel<<<napply, ttk::kGaugeThreads, 0, st>>>(U[k], dU[k], m, r, S);
    EV_CK(cudaGetLastError(), "tangent projection");
  }
  return TT_OK;
}

tt_status tt_tangent_eval(const tt_eval_plan* plan, const float* const* U, const float* const* V,
                          const float* const* dU, float* out, void* stream) {
  ttk::set_last_error("");
  if (!plan || !U || !V || !dU || (plan->n > 0 && !out)) return plan_fail(TT_EINVAL, "NULL argument");
  for (int k = 0; k < plan->d; ++k)
    if (!U[k] || !V[k] || !dU[k]) return plan_fail(TT_EINVAL, "NULL core");
  if (plan->n == 0) return TT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // pass k: the forward contraction with U left of core k, dU_k in its place
  // and V right of it, in core k's order, added to out (pass 0 writes it)
  for (int k = 0; k < plan->d; ++k) {
    const float* left[TT_MAXD];
    for (int j = 0; j < plan->d; ++j) left[j] = j == k ? dU[k] : U[j];
    ttk::PassArgs a = pass_args(plan, left, V, k, 0);
    a.out = out;
    a.accumulate = k > 0 ? 1 : 0;
    const size_t sm = ttk::pass_smem(a, plan->ranks);
    ttk::count_launch();
    ttk::eval_pass_kernel<<<(unsigned)plan->L.nchunks, ttk::kEvalThreads, sm, st>>>(a);
    EV_CK(cudaGetLastError(), "tangent evaluation");
  }
  return TT_OK;
}

tt_status tt_eval_at(int32_t d, const int64_t* dims, const int64_t* ranks,
                     const float* const* cores, const int64_t* idx, int64_t n, float* out,
                     void* stream) {
  tt_eval_plan* P = nullptr;
  tt_status s = tt_eval_plan_create(d, dims, ranks, idx, n, nullptr, nullptr, nullptr, stream, &P);
  if (s != TT_OK) return s;
  s = tt_eval_plan_at(P, cores, out, stream);
  tt_eval_plan_destroy(P, stream);
  return s;
}

tt_status tt_eval_at_backward(int32_t d, const int64_t* dims, const int64_t* ranks,
                              const float* const* cores, const int64_t* idx, int64_t n,
                              const float* gout, float* const* grads, void* stream) {
  tt_eval_plan* P = nullptr;
  tt_status s = tt_eval_plan_create(d, dims, ranks, idx, n, nullptr, nullptr, nullptr, stream, &P);
  if (s != TT_OK) return s;
  s = tt_eval_plan_backward(P, cores, gout, grads, stream);
  tt_eval_plan_destroy(P, stream);
  return s;
}

}  // extern "C"
