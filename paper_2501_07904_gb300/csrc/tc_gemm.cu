// Tensor-core (tcgen05) products for the mixed-precision sweep: D = A B with
// FP32 data, TF32 operands rounded to nearest, FP32 accumulation.
//
// One persistent CTA per SM, sixteen warps with fixed roles (a warp runs on
// scheduler warp % 4; the converters stay off the MMA issuer's scheduler):
//   warp 0     TMA producer: 2-D tensor-map copies of the FP32 operand
//              slabs (128 rows of A and n_mma rows of B by one k-block: 32 k,
//              or 64 k for an unsplit product) into a staging ring;
//   warp 1     allocates tensor memory; one lane issues tcgen05.mma;
//   warps 2-4, 6-8, 10, 11  converters: round the staged FP32 values to TF32
//              (and, for a split operand, keep the remainder x - hi, whose
//              low bits the MMA ignores), writing K-major 128-byte-swizzled
//              operand tiles;
//   warps 5, 9 idle;
//   warps 12-15 epilogue: after every chunk of k-blocks the
//              accumulator is read back and added into a running FP32 sum
//              kept in spare TMEM columns, which bounds the rounding drift of
//              the tensor-core accumulation; at the end of a work segment the
//              sum goes to the output (through a per-warp staging buffer, so
//              that every store writes whole 128-byte row segments) or to a
//              partial.
// A split operand x = hi + lo (both TF32) makes the product accurate to
// ~2^-22 relative: the main term hi*hi accumulates in its own TMEM columns
// and the small cross terms (hi*lo, lo*hi) in a second set, so only the main
// term's accumulation drift bounds the chunk length.  With a split B the
// MMA hi * [B_hi | B_lo] (N = 2 n_mma) gives the main term and one cross
// term at once; a split product wider than 102 columns keeps one cross-term
// region per work segment (two main-term buffers then fit in TMEM).
// Work is scheduled stream-K: the (tile, k-block) sequence is cut into one
// contiguous range per CTA, so a few output tiles over a long K (Gram
// matrices, sketches) still occupy every SM.  Tiles covered by several CTAs
// are finished by a fix-up kernel that adds the partials in CTA order
// (deterministic).
//
// Every mbarrier wait is bounded (tc_common.cuh): a stall sets the error
// word, the roles unwind, in-flight copies and MMAs are drained and the
// tensor memory is released before the kernel returns.
#include <cuda.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace ttk {
namespace {

using namespace tc;

constexpr int kThreads = 512;
constexpr int kConv = 256;     // converter threads (eight warps)
constexpr int kBM = 128;       // rows of an output tile (MMA M)
constexpr int kBK = 32;        // k per 128-byte swizzle atom row of TF32 (a k-block holds 1 or 2)
// The tensor-core accumulation drifts toward zero by up to about one FP32
// ulp per accumulate step, so the epilogue drains TMEM into a running
// round-to-nearest FP32 sum after at most kChunkMMA MMAs (a chunk of
// TcArgs::chunk_kb k-blocks); three accumulator buffers let the MMAs run
// ahead of the drains.
constexpr int kChunkMMA = 16;
constexpr int kAccBufs = 3;
constexpr int kMaxStages = 8;
constexpr int kSmemBudget = 225 * 1024;

struct TcArgs {
  int64_t M, N, K;
  int kb;            // k-blocks per tile
  int natoms;        // swizzle atoms (32 k each) per k-block: 2 for unsplit products, else 1
  int ntm, ntn;      // tile grid (rows, cols of tiles)
  int ntiles;
  int64_t total;     // ntiles * kb
  int G;             // CTAs
  int n_mma;         // MMA N (multiple of 16, <= NREG; of 32 for a split operand)
  int split;         // a_split || b_split: cross terms accumulate at column n_mma
  int merge;         // hi*[B_hi | B_lo] in one MMA of N = 2 n_mma (B tile rows contiguous)
  int nacc;          // TMEM accumulator buffers (<= kAccBufs)
  int acc_stride;    // TMEM columns per buffer
  int xshared;       // split, n_mma > 102: one cross-term region per work segment
  int cross_col;     // its first TMEM column (xshared)
  int sum_col;       // first TMEM column of the running sum
  int a_kmajor, b_kmajor;  // source layouts (1: contiguous along k)
  int a_split, b_split;
  int sym;           // Gram: upper tiles only, diagonal tiles use A for B
  int all_partial;   // every segment writes a partial (FP64 output / mirroring)
  int round_out;     // round FP32 outputs to TF32
  int S_st, S_op;    // ring depths
  int chunk_kb;      // k-blocks per TMEM chunk
  int res_b;         // B converted once per CTA and kept in shared memory
  uint32_t res_b_bytes;  // its size per k-block (hi [+ lo])
  const float* bptr; // B source for the resident copy
  int64_t ldb;
  uint32_t stage_bytes, a_box_bytes, b_box_bytes, op_bytes;
  float* out;
  int64_t ldo;
  float* part;       // [G][2][128][NREG]
  double* sq_part;   // [G] (sum of squares of directly written outputs) or null
  int* err;
};

__device__ __forceinline__ int64_t seg_beg(const TcArgs& a, int c) {
  return (int64_t)c * a.total / a.G;
}

// Tile t -> (row tile, col tile); a Gram enumerates the upper triangle row by row.
__host__ __device__ __forceinline__ void tile_coords(int t, int ntm, int ntn, int sym, int& mt,
                                                     int& nt) {
  if (!sym) {
    mt = t / ntn;
    nt = t % ntn;
    return;
  }
  mt = 0;
  int row_len = ntn;
  while (t >= row_len) {
    t -= row_len;
    ++mt;
    --row_len;
  }
  nt = mt + t;
}

// Position in the (tile, k-block) sequence, advanced without divisions.
struct Cursor {
  int t, kbi, mt, nt;
  __device__ __forceinline__ void init(const TcArgs& a, int64_t pos) {
    t = (int)(pos / a.kb);
    kbi = (int)(pos % a.kb);
    tile_coords(t, a.ntm, a.ntn, a.sym, mt, nt);
  }
  __device__ __forceinline__ void next_tile(const TcArgs& a) {
    kbi = 0;
    ++t;
    if (++nt == a.ntn) {
      ++mt;
      nt = a.sym ? mt : 0;
    }
  }
  __device__ __forceinline__ void next(const TcArgs& a) {
    if (++kbi == a.kb) next_tile(a);
  }
};

// Convert one staged FP32 slab into a K-major SW128 TF32 tile of R rows
// (R a multiple of 16, at most 128); hi/lo are shared addresses, lo = 0 for
// an unsplit operand.  A thread owns the 16-byte chunks idx = ct + 256 j of a
// K-major source (row idx / 8, chunk idx % 8), or half of row ct % 128 of an
// MN-major one; all of its loads are issued before the first conversion.
//   K-major source:  staging [R][32]  (one float4 per chunk)
//   MN-major source: staging [32][R]  (four floats, stride R, per chunk)
__device__ __forceinline__ void store_chunk(uint32_t hi, uint32_t lo, uint32_t off, float4 v) {
  const uint32_t h0 = to_tf32(v.x), h1 = to_tf32(v.y), h2 = to_tf32(v.z), h3 = to_tf32(v.w);
  sts128(hi + off, h0, h1, h2, h3);
  if (lo)
    sts128(lo + off, __float_as_uint(v.x - __uint_as_float(h0)), __float_as_uint(v.y - __uint_as_float(h1)),
           __float_as_uint(v.z - __uint_as_float(h2)), __float_as_uint(v.w - __uint_as_float(h3)));
}

template <int NA>
__device__ __forceinline__ void convert_slab(uint32_t stg, int kmajor, int R, uint32_t hi,
                                             uint32_t lo, int ct) {
  // NA atoms of 32 k: atom t of the destination at hi + t * R * 128; a thread
  // converts four chunks per group (group g: chunks ct + kConv (4 g + j))
  constexpr int kPer = 1024 / kConv;  // chunks per thread and group for R = 128
  if (kmajor) {
    const int nchunks = R * 8 * NA;
#pragma unroll
    for (int g = 0; g < NA; ++g) {
      float4 v[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int idx = ct + kConv * (kPer * g + j);
        if (idx < nchunks) v[j] = lds128(stg + (uint32_t)idx * 16u);  // row idx/(8 NA), chunk idx%(8 NA)
      }
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int idx = ct + kConv * (kPer * g + j);
        if (idx < nchunks) {
          const uint32_t row = (uint32_t)(idx / (8 * NA)), ch = (uint32_t)(idx % (8 * NA));
          const uint32_t at = (ch >> 3) * (uint32_t)R * 128u;
          store_chunk(hi + at, lo ? lo + at : 0u, sw128_off(row, (ch & 7u) * 4u), v[j]);
        }
      }
    }
  } else {
    // thread ct owns row ct % 128, chunks q = kPer NA (ct / 128) ... + kPer NA - 1
    const int row = ct & 127, q0 = (ct >> 7) * kPer * NA;
    if (row >= R) return;
    const uint32_t p0 = stg + (uint32_t)row * 4u;
#pragma unroll
    for (int g = 0; g < NA; ++g) {
      float4 v[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const uint32_t p = p0 + (uint32_t)((q0 + kPer * g + j) * 4 * R) * 4u;
        v[j].x = lds32(p);
        v[j].y = lds32(p + 4u * R);
        v[j].z = lds32(p + 8u * R);
        v[j].w = lds32(p + 12u * R);
      }
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const uint32_t q = (uint32_t)(q0 + kPer * g + j), at = (q >> 3) * (uint32_t)R * 128u;
        store_chunk(hi + at, lo ? lo + at : 0u, sw128_off((uint32_t)row, (q & 7u) * 4u), v[j]);
      }
    }
  }
}

__device__ __forceinline__ float round_tf32(float x) { return __uint_as_float(to_tf32(x)); }

// NA: swizzle atoms per k-block (a compile-time copy of TcArgs::natoms)
template <int NREG, int NA>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the tiles (SW128 atoms) is established by hand.
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)smem;  // 64 barriers
  uint64_t* full = bars;
  uint64_t* empty = bars + kMaxStages;
  uint64_t* opfull = bars + 2 * kMaxStages;
  uint64_t* opempty = bars + 3 * kMaxStages;
  uint64_t* accfull = bars + 4 * kMaxStages;
  uint64_t* accempty = accfull + kAccBufs;
  uint64_t* finalbar = accfull + 2 * kAccBufs;
  uint64_t* crossfree = finalbar + 1;  // the epilogue has read a segment's cross terms
  uint32_t* tmem_slot = (uint32_t*)(bars + 48);
  double* red = (double*)(bars + 56);  // 4 doubles
  uint8_t* stage_base = smem + 1024;
  uint8_t* op_base = stage_base + (size_t)a.S_st * a.stage_bytes;
  uint8_t* resb_base = op_base + (size_t)a.S_op * a.op_bytes;
  // epilogue store staging, 2 KB per epilogue warp, after the resident B
  const uint32_t stg0 = smem_u32(resb_base) + (a.res_b ? (uint32_t)a.kb * a.res_b_bytes : 0u);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x;

  if (tid == 0) {
    for (int s = 0; s < a.S_st; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConv);
    }
    for (int t = 0; t < a.S_op; ++t) {
      mbar_init(&opfull[t], kConv);
      mbar_init(&opempty[t], 1);
    }
    for (int b = 0; b < a.nacc; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 128);
    }
    mbar_init(finalbar, 1);
    mbar_init(crossfree, 128);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  if (a.res_b) {
    // resident B: every thread converts chunks (k-block, row j, k quad q) of
    // B straight from global memory (it is small and L2-resident)
    const uint32_t rb = smem_u32(resb_base);
    const int nchunks = a.kb * a.n_mma * 8;
    for (int idx = tid; idx < nchunks; idx += kThreads) {
      const int kbi = idx / (a.n_mma * 8), w = idx % (a.n_mma * 8);
      const int j = w % a.n_mma, q = w / a.n_mma;
      float4 v;
      float* vv = &v.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t k = (int64_t)kbi * kBK + q * 4 + e;
        vv[e] = (k < a.K && j < a.N) ? (a.b_kmajor ? a.bptr[k + (int64_t)j * a.ldb] : a.bptr[k * a.ldb + j])
                                     : 0.f;
      }
      const uint32_t hi = rb + (uint32_t)kbi * a.res_b_bytes;
      store_chunk(hi, a.b_split ? hi + (uint32_t)a.n_mma * 128u : 0u, sw128_off((uint32_t)j, (uint32_t)q * 4u), v);
    }
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t beg = seg_beg(a, c), end = seg_beg(a, c + 1);
  const int first_tile = (int)(beg / a.kb);

  if (warp == 0) {
    // ---------------- TMA producer (warp-wide loop, one elected issuer) ----------------
    int s = 0;
    uint32_t ph = 0;
    uint32_t issued = 0u, issued_ph = 0u;  // per-stage bits
    bool ok = true;
    Cursor cur;
    cur.init(a, beg);
    for (int64_t pos = beg; pos < end; ++pos, cur.next(a)) {
      const bool same = (a.sym && cur.mt == cur.nt) || a.res_b;  // no B slab to load
      ok = __all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, a.err));
      if (!ok) break;
      if (elect_one()) {
        uint8_t* st = stage_base + (size_t)s * a.stage_bytes;
        mbar_arrive_expect_tx(&full[s], a.a_box_bytes + (same ? 0u : a.b_box_bytes));
        const int k0 = cur.kbi * kBK * NA;
        if (a.a_kmajor)
          tma_load_2d(st, &mapA, k0, cur.mt * kBM, &full[s]);
        else
          tma_load_2d(st, &mapA, cur.mt * kBM, k0, &full[s]);
        if (!same) {
          const int n0 = cur.nt * NREG;
          if (a.b_kmajor)
            tma_load_2d(st + a.a_box_bytes, &mapB, k0, n0, &full[s]);
          else
            tma_load_2d(st + a.a_box_bytes, &mapB, n0, k0, &full[s]);
        }
      }
      __syncwarp();
      issued |= 1u << s;
      issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
      if (++s == a.S_st) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (!ok) {
      // drain copies still in flight before the CTA's shared memory goes away
      for (int i = 0; i < a.S_st; ++i) {
        if (!((issued >> i) & 1u)) continue;
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(&full[i], (issued_ph >> i) & 1u) &&
               globaltimer_ns() - t0 < kWaitLimitNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (warp-wide loop, one elected issuer) ----------------
    const uint32_t idesc = idesc_tf32(kBM, a.n_mma);
    const uint32_t idesc2 = idesc_tf32(kBM, 2 * a.n_mma);
    const uint32_t op0 = smem_u32(op_base);
    int t_op = 0;
    uint32_t ph_op = 0;
    uint32_t fills[kAccBufs] = {0u, 0u, 0u};
    uint32_t nseg = 0;
    int buf = 0;
    bool ok = true;
    int64_t pos = beg;
    Cursor cur;
    cur.init(a, beg);
    while (pos < end && ok) {
      const int kstart = cur.kbi;
      const int kend = (int)std::min<int64_t>((int64_t)a.kb, kstart + (end - pos));
      const bool same = a.sym && cur.mt == cur.nt;
      if (a.xshared) {
        // the previous segment's cross terms must have been read
        ok = __all_sync(0xffffffffu, mbar_wait(crossfree, (nseg & 1u) ^ 1u, a.err));
        if (!ok) break;
        ++nseg;
      }
      for (int kbi = kstart; kbi < kend; ++kbi) {
        const int local = kbi - kstart;
        const bool chunk_start = (local % a.chunk_kb) == 0;
        if (chunk_start) {
          ok = __all_sync(0xffffffffu, mbar_wait(&accempty[buf], (fills[buf] & 1u) ^ 1u, a.err));
          if (!ok) break;
        }
        ok = __all_sync(0xffffffffu, mbar_wait(&opfull[t_op], ph_op, a.err));
        if (!ok) break;
        const uint32_t a_hi = op0 + (uint32_t)t_op * a.op_bytes;
        const uint32_t a_lo = a_hi + 16384u;
        uint32_t b_hi = same ? a_hi : a_hi + (a.a_split || NA == 2 ? 32768u : 16384u);
        if (a.res_b) b_hi = smem_u32(resb_base) + (uint32_t)kbi * a.res_b_bytes;
        const uint32_t b_lo = same ? a_lo : b_hi + (uint32_t)a.n_mma * 128u;
        const uint32_t d = tmem + (uint32_t)(buf * a.acc_stride);
        // cross terms of a split product: beside the main term, or one
        // region for the whole segment
        const uint32_t dc = a.xshared ? tmem + (uint32_t)a.cross_col : d + (uint32_t)a.n_mma;
        const uint32_t acc_x0 = a.xshared ? (kbi == kstart ? 0u : 1u) : (chunk_start ? 0u : 1u);
        const bool chunk_end = (local % a.chunk_kb == a.chunk_kb - 1) || (kbi == kend - 1);
        if (elect_one()) {
          // a TMEM buffer handed back by the epilogue is written only after
          // its reads (tcgen05.ld before the epilogue's arrive)
          if (chunk_start) tc_fence_after();
          // a k-step of 8 TF32 moves the start address by 32 bytes (2 in the
          // descriptor's 16-byte units) inside the swizzle atom
          const uint64_t dah = make_sw128_desc(a_hi), dbh = make_sw128_desc(b_hi);
          const uint64_t dal = make_sw128_desc(a_lo), dbl = make_sw128_desc(b_lo);
          // the main term hi*hi accumulates at d, the small cross terms
          // hi*lo and lo*hi at dc: the chunk length bounds the drift of the
          // main term only
          const bool merge = a.merge && !(same && a.n_mma != kBM);
          if (NA == 2) {
            // an unsplit product, two atoms per k-block: atom t of A at
            // + t * 16 KB, of B at + t * n_mma * 128 bytes (16-byte units)
            const uint64_t tb = same ? 1024u : (uint64_t)a.n_mma * 8u;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const uint32_t acc = (chunk_start && kk == 0) ? 0u : 1u;
              const uint64_t k4 = 2u * (uint64_t)(kk & 3);
              mma_tf32(d, dah + k4 + (kk >> 2) * 1024u, dbh + k4 + (kk >> 2) * tb, idesc, acc);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t acc = (chunk_start && kk == 0) ? 0u : 1u;
              const uint32_t accx = (kk == 0) ? acc_x0 : 1u;
              const uint64_t o = 2u * (uint64_t)kk;
              if (merge) {
                mma_tf32(d, dah + o, dbh + o, idesc2, acc);  // [hi*hi | hi*lo]
              } else {
                mma_tf32(d, dah + o, dbh + o, idesc, acc);
                if (a.b_split) mma_tf32(dc, dah + o, dbl + o, idesc, accx);
              }
              if (a.a_split) mma_tf32(dc, dal + o, dbh + o, idesc, a.b_split ? 1u : accx);
            }
          }
          mma_commit(&opempty[t_op]);
          if (chunk_end) mma_commit(&accfull[buf]);
        }
        __syncwarp();
        if (++t_op == a.S_op) {
          t_op = 0;
          ph_op ^= 1u;
        }
        if (chunk_end) {
          ++fills[buf];
          if (++buf == a.nacc) buf = 0;
        }
      }
      pos += kend - kstart;
      cur.next_tile(a);
    }
    // every MMA issued so far has completed once this barrier flips
    if (elect_one()) mma_commit(finalbar);
    __syncwarp();
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(finalbar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
    }
  } else if (warp < 12 && warp != 5 && warp != 9) {
    // ---------------- converters ----------------
    const int ci = warp - 2 - (warp > 5 ? 1 : 0) - (warp > 9 ? 1 : 0);
    const int ct = ci * 32 + lane;  // 0 .. kConv-1
    int s = 0, t_op = 0;
    uint32_t ph = 0, ph_op = 0;
    Cursor cur;
    cur.init(a, beg);
    for (int64_t pos = beg; pos < end; ++pos, cur.next(a)) {
      const bool same = (a.sym && cur.mt == cur.nt) || a.res_b;  // no B slab to convert
      bool ok = mbar_wait(&full[s], ph, a.err);
      ok = ok && mbar_wait(&opempty[t_op], ph_op ^ 1u, a.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      const uint32_t st = smem_u32(stage_base) + (uint32_t)s * a.stage_bytes;
      const uint32_t op = smem_u32(op_base) + (uint32_t)t_op * a.op_bytes;
      if (NA == 2) {
        // unsplit operands only
        convert_slab<2>(st, a.a_kmajor, kBM, op, 0u, ct);
        if (!same) convert_slab<2>(st + a.a_box_bytes, a.b_kmajor, a.n_mma, op + 32768u, 0u, ct);
      } else {
        convert_slab<1>(st, a.a_kmajor, kBM, op, a.a_split ? op + 16384u : 0u, ct);
        if (!same) {
          const uint32_t bh = op + (a.a_split ? 32768u : 16384u);
          convert_slab<1>(st + a.a_box_bytes, a.b_kmajor, a.n_mma, bh,
                          a.b_split ? bh + (uint32_t)a.n_mma * 128u : 0u, ct);
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&opfull[t_op]);
      mbar_arrive(&empty[s]);
      if (++s == a.S_st) {
        s = 0;
        ph ^= 1u;
      }
      if (++t_op == a.S_op) {
        t_op = 0;
        ph_op ^= 1u;
      }
    }
  } else if (warp >= 12) {
    // ---------------- epilogue ----------------
    // TMEM: nacc accumulator buffers of acc_stride columns (a split product's
    // cross terms at column n_mma of each), then NREG columns holding the
    // running FP32 sum of the current segment's drained chunks.
    const int q = warp & 3;               // TMEM lane quarter of this warp
    const int row = q * 32 + lane;        // tile row owned by this thread
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t sum_addr = lane_addr + (uint32_t)a.sum_col;
    double sq = 0.0;
    int buf = 0;
    uint32_t drains[kAccBufs] = {0u, 0u, 0u};
    bool ok = true;
    int64_t pos = beg;
    Cursor cur;
    cur.init(a, beg);
    while (pos < end && ok) {
      const int t = cur.t, kstart = cur.kbi, mt = cur.mt, nt = cur.nt;
      const int kend = (int)std::min<int64_t>((int64_t)a.kb, kstart + (end - pos));
      const int nchunks = (kend - kstart + a.chunk_kb - 1) / a.chunk_kb;
      const bool direct = (kstart == 0 && kend == a.kb) && !a.all_partial;
      const int64_t m = (int64_t)mt * kBM + row;
      const int64_t n0 = (int64_t)nt * NREG;
      const int ncols = (int)std::min<int64_t>((int64_t)NREG, a.N - n0);
      float* o = a.out + m * a.ldo + n0;
      const bool vec = ((a.ldo & 3) == 0) && ((((uintptr_t)a.out) & 15) == 0);
      float* pp = a.part + (((size_t)c * 2 + ((t == first_tile) ? 0 : 1)) * kBM + row) * NREG;
      float rs = 0.f;
      for (int ch = 0; ch < nchunks; ++ch) {
        bool w = mbar_wait(&accfull[buf], drains[buf] & 1u, a.err);
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool last = (ch == nchunks - 1);
#pragma unroll 1
        for (int c32 = 0; c32 < NREG / 32; ++c32) {
          float v[32];
          {
            const uint32_t ab = lane_addr + (uint32_t)(buf * a.acc_stride + c32 * 32);
            // main part (and a split product's cross part), then the running
            // sum: one 32-column load in flight at a time (register budget)
            tmem_ld32(ab, v);
            if (a.split && (!a.xshared || last)) {
              // a shared cross region is complete (and read) at the
              // segment's last chunk only
              float u[32];
              tmem_ld32(a.xshared ? lane_addr + (uint32_t)(a.cross_col + c32 * 32) : ab + (uint32_t)a.n_mma, u);
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] += u[j];
            }
            if (ch > 0) {
              float u[32];
              tmem_ld32(sum_addr + (uint32_t)(c32 * 32), u);
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] += u[j];
            }
          }
          if (!last) {
            tmem_st32(sum_addr + (uint32_t)(c32 * 32), v);
            continue;
          }
          if (direct) {
            const int jb = c32 * 32;
            if (a.round_out) {
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] = round_tf32(v[j]);
            }
            if (vec && jb + 32 <= ncols) {
              // a full 32-column chunk: the warp passes its 32 rows through
              // its 2 KB staging buffer, 16 rows at a time (chunk positions
              // swizzled by row), so that every store writes four whole
              // 128-byte row segments
              if (m < a.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) rs += v[j] * v[j];
              }
              const uint32_t sbuf = stg0 + (uint32_t)q * 2048u;
              const int64_t gr0 = (int64_t)mt * kBM + q * 32;  // this warp's first row
              float* const ob = a.out + n0 + jb + 4 * (lane & 7);
#pragma unroll 1
              for (int h = 0; h < 2; ++h) {
                if ((lane >> 4) == h) {
                  const uint32_t r = (uint32_t)(lane & 15);
#pragma unroll
                  for (int jc = 0; jc < 8; ++jc)
                    sts128(sbuf + r * 128u + ((((uint32_t)jc ^ (r & 7u)) << 4)), __float_as_uint(v[4 * jc]),
                           __float_as_uint(v[4 * jc + 1]), __float_as_uint(v[4 * jc + 2]),
                           __float_as_uint(v[4 * jc + 3]));
                }
                __syncwarp();
#pragma unroll
                for (int pq = 0; pq < 4; ++pq) {
                  const uint32_t r = (uint32_t)(lane >> 3) + 4u * pq, jc = (uint32_t)(lane & 7);
                  const float4 x = lds128(sbuf + r * 128u + ((jc ^ (r & 7u)) << 4));
                  const int64_t gm = gr0 + 16 * h + (int)r;
                  if (gm < a.M) *reinterpret_cast<float4*>(ob + gm * a.ldo) = x;
                }
                __syncwarp();
              }
            } else if (m < a.M) {
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                const float v0 = v[j], v1 = v[j + 1], v2 = v[j + 2], v3 = v[j + 3];
                const int jj = jb + j;
                if (jj + 3 < ncols) {
                  if (vec) {
                    *reinterpret_cast<float4*>(o + jj) = make_float4(v0, v1, v2, v3);
                  } else {
                    o[jj] = v0;
                    o[jj + 1] = v1;
                    o[jj + 2] = v2;
                    o[jj + 3] = v3;
                  }
                  rs += v0 * v0 + v1 * v1 + v2 * v2 + v3 * v3;
                } else {
                  if (jj < ncols) { o[jj] = v0; rs += v0 * v0; }
                  if (jj + 1 < ncols) { o[jj + 1] = v1; rs += v1 * v1; }
                  if (jj + 2 < ncols) { o[jj + 2] = v2; rs += v2 * v2; }
                }
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(pp + c32 * 32 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          }
        }
        tc_fence_before();
        mbar_arrive(&accempty[buf]);
        if (a.xshared && last) mbar_arrive(crossfree);
        ++drains[buf];
        if (++buf == a.nacc) buf = 0;
      }
      sq += (double)rs;
      pos += kend - kstart;
      cur.next_tile(a);
    }
    if (a.sq_part) {
      for (int o2 = 16; o2 > 0; o2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o2);
      if (lane == 0) red[q] = sq;
      named_barrier(1, 128);
      if (tid == 12 * 32) a.sq_part[c] = red[0] + red[1] + red[2] + red[3];
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// Finish tiles covered by more than one CTA (or every tile when all_partial):
// the FP32 partials are added in CTA order with compensated (Kahan) FP32
// sums -- accurate to about one ulp of the result, without FP64 adds, which
// GB300 issues at a small fraction of the FP32 rate -- and mirrored for a
// Gram.  blockIdx.y selects kBM / gridDim.y rows of the tile (one row per
// block for the few tiles of a Gram, more where most blocks find no split
// tile).

template <int NREG>
__global__ void tc_fixup_kernel(TcArgs a, double* __restrict__ out64, double* __restrict__ fix_sq) {
  __shared__ double red[32];
  __shared__ uint32_t slot_off[1024];  // per contributing CTA: offset of its partial (in floats)
  int t;
  if (a.all_partial) {
    t = blockIdx.x;
  } else {
    // block b finishes the tile in which CTA b's range starts, when that
    // start lies strictly inside a tile and no earlier CTA start does
    const int b = blockIdx.x;
    t = -1;
    if (b >= 1 && b < a.G) {
      const int64_t pb = seg_beg(a, b);
      const int tt = (int)(pb / a.kb);
      if (pb % a.kb != 0 && seg_beg(a, b - 1) <= (int64_t)tt * a.kb) t = tt;
    }
  }
  float sqf = 0.f;
  if (t >= 0) {
    int mt, nt;
    tile_coords(t, a.ntm, a.ntn, a.sym, mt, nt);
    const int64_t p_lo = (int64_t)t * a.kb, p_hi = p_lo + a.kb - 1;
    const int c_lo = (int)(((p_lo + 1) * a.G - 1) / a.total);
    const int c_hi = (int)(((p_hi + 1) * a.G - 1) / a.total);
    const int64_t m0 = (int64_t)mt * kBM, n0 = (int64_t)nt * NREG;
    const int ncc = c_hi - c_lo + 1;  // <= G <= the SM count
    for (int q = threadIdx.x; q < ncc; q += blockDim.x) {
      const int cc = c_lo + q;
      const int slot = (seg_beg(a, cc) / a.kb == t) ? 0 : 1;
      slot_off[q] = (uint32_t)(((size_t)cc * 2 + slot) * kBM * NREG);
    }
    __syncthreads();
    const int rows = kBM / gridDim.y;
    const int i0 = blockIdx.y * rows;
    for (int e = threadIdx.x; e < rows * NREG; e += blockDim.x) {
      const int i = i0 + e / NREG, j = e % NREG;
      const int64_t m = m0 + i, n = n0 + j;
      if (m >= a.M || n >= a.N) continue;
      float sum = 0.f, comp = 0.f;
      const float* pe = a.part + (size_t)i * NREG + j;
      for (int q = 0; q < ncc; ++q) {
        const float y = pe[slot_off[q]] - comp;
        const float tsum = sum + y;
        comp = (tsum - sum) - y;
        sum = tsum;
      }
      const bool mirror = a.sym && mt != nt;
      if (out64) {
        const double s = (double)sum - (double)comp;
        out64[m * a.N + n] = s;
        if (mirror) out64[n * a.N + m] = s;
      }
      if (a.out) {
        float v = sum - comp;
        if (a.round_out) v = round_tf32(v);
        a.out[m * a.ldo + n] = v;
        sqf += v * v;
        if (mirror) {
          a.out[n * a.ldo + m] = v;
          sqf += v * v;
        }
      }
    }
  }
  if (fix_sq) {
    const double sq = block_sum((double)sqf, red);
    if (threadIdx.x == 0) fix_sq[(size_t)blockIdx.x * gridDim.y + blockIdx.y] = sq;
  }
}

__global__ void tc_sumsq_kernel(const double* __restrict__ a, int na, const double* __restrict__ b,
                                int nb, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < na; i += blockDim.x) s += a[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += b[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct DevInfo {
  int sms = 0;
  bool attr_set[4] = {false, false, false, false};
};

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
std::vector<DevInfo> g_dev;

cudaError_t dev_info(DevInfo** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
    g_encode = (EncodeTiledFn)fn;
  }
  if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
  DevInfo& d = g_dev[dev];
  if (d.sms == 0) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  *out = &d;
  return cudaSuccess;
}

struct Plan {
  TcArgs a;
  int nreg;
  size_t smem;
  size_t part_bytes, sq_bytes, fix_bytes;
  int fix_blocks;
};

int64_t ceil_div(int64_t x, int64_t y) { return (x + y - 1) / y; }

bool make_plan(int64_t M, int64_t N, int64_t K, bool sym, bool out64, bool a_split, bool b_split,
               int sms, Plan& p) {
  memset(&p, 0, sizeof(p));
  TcArgs& a = p.a;
  const int64_t nw = std::min<int64_t>(N, 128);
  p.nreg = nw <= 32 ? 32 : (nw <= 64 ? 64 : 128);
  a.M = M;
  a.N = N;
  a.K = K;
  // a split product keeps its cross terms at column n_mma: 32-aligned for the
  // epilogue's 32-column TMEM loads
  a.split = (a_split || b_split) ? 1 : 0;
  a.n_mma = (int)std::min<int64_t>(p.nreg, ceil_div(nw, a.split ? 32 : 16) * (a.split ? 32 : 16));
  a.merge = b_split ? 1 : 0;
  a.acc_stride = a.split ? 2 * a.n_mma : p.nreg;
  a.nacc = std::min(kAccBufs, (512 - a.n_mma) / a.acc_stride);
  a.xshared = 0;
  if (a.split && a.nacc < 2) {
    // two main-term buffers, one cross region per work segment, the sum
    a.xshared = 1;
    a.merge = 0;
    a.acc_stride = a.n_mma;
    a.nacc = 2;
    a.cross_col = 2 * a.n_mma;
  }
  a.sum_col = a.xshared ? 3 * a.n_mma : a.nacc * a.acc_stride;
  if (a.nacc < 1 || a.sum_col + p.nreg > 512) return false;
  // an unsplit product takes two swizzle atoms (64 k) per k-block: half the
  // per-k-block hand-offs for the same bytes
  a.natoms = (!a_split && !b_split && p.nreg == 128) ? 2 : 1;
  a.kb = (int)ceil_div(K, (int64_t)kBK * a.natoms);
  a.ntm = (int)ceil_div(M, kBM);
  a.ntn = (int)ceil_div(N, p.nreg);
  if (sym) {
    if (M != N || p.nreg != 128 && a.ntm != 1) return false;
    if (a.ntm != a.ntn) return false;
    a.ntiles = a.ntm * (a.ntm + 1) / 2;
  } else {
    a.ntiles = a.ntm * a.ntn;
  }
  a.sym = sym ? 1 : 0;
  a.total = (int64_t)a.ntiles * a.kb;
  a.all_partial = (sym || out64) ? 1 : 0;
  int64_t G = std::min<int64_t>((int64_t)sms, std::max<int64_t>(1, ceil_div(a.total, 4)));
  if (a.all_partial) {
    // Every CTA leaves a kBM x nreg partial for the fix-up to sum: at least
    // 8 k-blocks per CTA, so that a short product (a Cholesky-QR Gram of a
    // few MB) writes and re-reads fewer partials than it reads operands
    // (16 k-blocks per CTA was slower: the split operand's conversion bounds
    // a CTA's rate)
    G = std::min<int64_t>(G, std::max<int64_t>(1, ceil_div(a.total, 8)));
    // each CTA range no longer than a tile: at most two tiles (partial slots) per CTA
    G = std::max<int64_t>(G, a.ntiles);
    if (G > sms) return false;
    G = std::min<int64_t>(G, a.total);
  }
  a.G = (int)G;
  a.a_split = a_split ? 1 : 0;
  a.b_split = b_split ? 1 : 0;
  a.chunk_kb = std::max(1, kChunkMMA / (4 * a.natoms));  // main-term MMAs per k-block
  a.a_box_bytes = kBM * kBK * 4 * a.natoms;
  a.b_box_bytes = (uint32_t)a.n_mma * kBK * 4 * a.natoms;
  // a Gram's off-diagonal tiles load B; diagonal ones reuse A.  A B operand
  // of one column tile and at most 8 k-blocks (64 KB converted) stays
  // resident: converted once per CTA instead of once per row tile.
  a.res_b_bytes = (uint32_t)a.n_mma * 128u * (b_split ? 2u : 1u);
  a.res_b = (a.natoms == 1 && !sym && a.ntn == 1 && a.kb <= 8 &&
             (size_t)a.kb * a.res_b_bytes <= 65536u && a.ntm >= 8) ? 1 : 0;
  const size_t res_bytes = a.res_b ? (size_t)a.kb * a.res_b_bytes : 0;
  const bool any_b = (!sym || a.ntm > 1) && !a.res_b;
  a.stage_bytes = a.a_box_bytes + (any_b ? a.b_box_bytes : 0u);
  a.stage_bytes = (a.stage_bytes + 1023u) & ~1023u;
  a.op_bytes = 16384u * (uint32_t)a.natoms * (a_split ? 2u : 1u) +
               (any_b ? (uint32_t)a.n_mma * 128u * (uint32_t)a.natoms * (b_split ? 2u : 1u) : 0u);
  a.op_bytes = (a.op_bytes + 1023u) & ~1023u;
  // barriers, alignment slack, resident B, epilogue store staging
  const size_t fixed = 2048 + 1024 + res_bytes + 8192;
  a.S_op = 2;
  if (fixed + 4 * (size_t)a.stage_bytes + 3 * (size_t)a.op_bytes <= (size_t)kSmemBudget) a.S_op = 3;
  const size_t left = kSmemBudget - fixed - (size_t)a.S_op * a.op_bytes;
  a.S_st = (int)std::min<size_t>(kMaxStages, left / a.stage_bytes);
  if (a.S_st < 2) return false;
  p.smem = fixed + (size_t)a.S_st * a.stage_bytes + (size_t)a.S_op * a.op_bytes;
  p.part_bytes = ((size_t)G * 2 * kBM * p.nreg * sizeof(float) + 255) & ~(size_t)255;
  p.sq_bytes = ((size_t)G * sizeof(double) + 255) & ~(size_t)255;
  p.fix_blocks = a.all_partial ? a.ntiles : (int)G;
  p.fix_bytes = ((size_t)p.fix_blocks * kBM * sizeof(double) + 255) & ~(size_t)255;
  return true;
}

// Tensor map of an FP32 operand: rows R (the M or N side) by K.
bool encode(CUtensorMap* map, const float* p, int64_t ld, bool kmajor, int64_t R, int64_t K,
            int box_rows, int box_k) {
  cuuint64_t dims[2], strides[1];
  cuuint32_t box[2], estr[2] = {1, 1};
  if (kmajor) {
    dims[0] = (cuuint64_t)K;
    dims[1] = (cuuint64_t)R;
    box[0] = (cuuint32_t)box_k;
    box[1] = (cuuint32_t)box_rows;
  } else {
    dims[0] = (cuuint64_t)R;
    dims[1] = (cuuint64_t)K;
    box[0] = (cuuint32_t)box_rows;
    box[1] = (cuuint32_t)box_k;
  }
  strides[0] = (cuuint64_t)ld * sizeof(float);
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)p, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int NREG, int NA>
cudaError_t launch(const Plan& p, const CUtensorMap& ma, const CUtensorMap& mb, DevInfo* d,
                   int slot, cudaStream_t st) {
  if (!d->attr_set[slot]) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<NREG, NA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
    if (e != cudaSuccess) return e;
    d->attr_set[slot] = true;
  }
  tc_gemm_kernel<NREG, NA><<<p.a.G, kThreads, p.smem, st>>>(ma, mb, p.a);
  return cudaGetLastError();
}

}  // namespace

bool tc_gemm_eligible(Mat<float> A, Mat<float> B, int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if ((A.ld & 3) || (B.ld & 3) || (((uintptr_t)A.p) & 15) || (((uintptr_t)B.p) & 15)) return false;
  if (K > INT32_MAX - 64 || M > INT32_MAX - 256 || N > INT32_MAX - 256) return false;
  // TMA strides below 2^40 bytes
  if ((uint64_t)A.ld * 4 >= (1ull << 40) || (uint64_t)B.ld * 4 >= (1ull << 40)) return false;
  return true;
}

size_t tc_gemm_ws_bytes(int64_t M, int64_t N, int64_t K, bool sym, bool out64, bool a_split,
                        bool b_split) {
  DevInfo* d = nullptr;
  int sms = 152;
  if (dev_info(&d) == cudaSuccess) sms = d->sms;
  Plan p;
  if (!make_plan(M, N, K, sym, out64, a_split, b_split, sms, p)) return 0;
  return p.part_bytes + p.sq_bytes + p.fix_bytes + 256;
}

cudaError_t tc_gemm(Mat<float> A, Mat<float> B, int64_t M, int64_t N, int64_t K, float* out,
                    int64_t ldo, double* out64, bool sym, double* sumsq, void* ws, cudaStream_t st,
                    TcOpts o) {
  if (!tc_gemm_eligible(A, B, M, N, K)) return cudaErrorNotSupported;
  if (!out && !out64) return cudaErrorInvalidValue;
  if (sumsq && !out) return cudaErrorInvalidValue;
  if (!o.err) return cudaErrorInvalidValue;
  DevInfo* d = nullptr;
  cudaError_t e = dev_info(&d);
  if (e != cudaSuccess) return e;
  Plan p;
  if (!make_plan(M, N, K, sym, out64 != nullptr, o.a_split, o.b_split, d->sms, p))
    return cudaErrorNotSupported;
  TcArgs& a = p.a;
  a.a_kmajor = A.row ? 1 : 0;   // A(i,k) = p[i*ld + k]
  a.b_kmajor = B.row ? 0 : 1;   // B(k,j) = p[k + j*ld]
  a.bptr = B.p;
  a.ldb = B.ld;
  a.round_out = o.round_out ? 1 : 0;
  a.out = out;
  a.ldo = ldo;
  a.err = o.err;
  char* w = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  a.part = (float*)w;
  double* sq_part = (double*)(w + p.part_bytes);
  double* fix_sq = (double*)(w + p.part_bytes + p.sq_bytes);
  a.sq_part = sumsq ? sq_part : nullptr;

  CUtensorMap ma, mb;
  if (!encode(&ma, A.p, A.ld, a.a_kmajor != 0, M, K, kBM, kBK * a.natoms)) return cudaErrorInvalidValue;
  if (!encode(&mb, B.p, B.ld, a.b_kmajor != 0, N, K, a.n_mma, kBK * a.natoms)) return cudaErrorInvalidValue;

  const int slot = a.natoms == 2 ? 3 : (p.nreg == 32 ? 0 : (p.nreg == 64 ? 1 : 2));
  int nl = 1;
  if (a.natoms == 2)
    e = launch<128, 2>(p, ma, mb, d, slot, st);
  else if (p.nreg == 32)
    e = launch<32, 1>(p, ma, mb, d, slot, st);
  else if (p.nreg == 64)
    e = launch<64, 1>(p, ma, mb, d, slot, st);
  else
    e = launch<128, 1>(p, ma, mb, d, slot, st);
  if (e != cudaSuccess) return e;
  // without FP64 output or a Gram, the fix-up only sums tiles that a CTA
  // boundary splits: none when every boundary falls on a tile edge
  bool split_tile = false;
  for (int b = 1; b < a.G && !split_tile; ++b)
    split_tile = ((int64_t)b * a.total / a.G) % a.kb != 0;
  const bool need_fix = a.all_partial || (a.G > 1 && split_tile);
  const unsigned fg_y = a.all_partial ? kBM : 16;
  if (need_fix) {
    ++nl;
    const dim3 fg((unsigned)p.fix_blocks, fg_y);
    if (p.nreg == 32)
      tc_fixup_kernel<32><<<fg, 256, 0, st>>>(a, out64, sumsq ? fix_sq : nullptr);
    else if (p.nreg == 64)
      tc_fixup_kernel<64><<<fg, 256, 0, st>>>(a, out64, sumsq ? fix_sq : nullptr);
    else
      tc_fixup_kernel<128><<<fg, 256, 0, st>>>(a, out64, sumsq ? fix_sq : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (sumsq) {
    ++nl;
    tc_sumsq_kernel<<<1, 256, 0, st>>>(sq_part, a.G, fix_sq,
                                       need_fix ? p.fix_blocks * (int)fg_y : 0, sumsq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  count_launch(nl);
  return cudaSuccess;
}


namespace {
// The bounded wait of the tensor-core kernels on an mbarrier of one arrival,
// which lane 0 completes (arrive) or nothing does; the wait then runs out
// after limit_ns and sets the error word.
__global__ void wait_selftest_kernel(int arrive, uint64_t limit_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
  mbar_wait(&bar, 0, err, limit_ns);
}
}  // namespace

cudaError_t wait_selftest(bool arrive, uint64_t limit_ns, int* err, cudaStream_t st) {
  count_launch();
  wait_selftest_kernel<<<1, 32, 0, st>>>(arrive ? 1 : 0, limit_ns, err);
  return cudaGetLastError();
}

TT_BOUNDS_READER(bounds_tc_gemm)

}  // namespace ttk
