// Tiled SIMT GEMM for the sweep's Gram, sketch, projection and carry
// products (FP32 or FP64 data).  D = A B with either operand row- or
// column-major, so every product of the sweep (C^T C, C C^T, C^T Omega,
// C W, Z^T C, ...) is a view of the stored matrices with no transposition
// pass.  Long inner products are summed hierarchically (see internal.h);
// split-K partials are FP64 and reduced in a fixed order (deterministic).
#include <algorithm>
#include <type_traits>

#include "dfloat.cuh"
#include "internal.h"

namespace ttk {
namespace {

constexpr int BK = 16, NT = 256;
constexpr int FLUSH_TILES = 32;  // FP32 tile sums folded into FP64 every 32 k-tiles (512 products)
constexpr int FLUSH_DF = 8;      // compensated sums folded into FP64 every 8 k-tiles (128 products)
constexpr int kTargetBlocks = 152 * 8;

// Accumulation modes.
//   kF32: FP32 products summed in FP32 over one k-tile, those sums in FP32
//         over FLUSH_TILES tiles, then in FP64;
//   kF64: FP64 data, FP64 products and sums;
//   kDF:  FP32 data, each product split exactly into p + e (e by an FMA:
//         a b - p is representable) and summed by Knuth's TwoSum into a
//         running (hi, lo) pair of FP32 words (Ogita, Rump and Oishi's
//         compensated dot product, "Dot2"), folded into FP64 every FLUSH_DF
//         tiles.  Over a window of n = 128 products the error is at most
//         ~n u^2 sum|a b| (u = 2^-24), i.e. below 5e-13 of sum|a b| -- the
//         order of an FP64 sum of exact products over the same split-K chunk
//         -- at FP32 instruction rates (FP64 runs at a small fraction of them
//         on this part).  The error-free transformations (dfloat.cuh) use
//         the _rn intrinsics, which the compiler never contracts into FMAs.
enum AccMode { kF32 = 0, kF64 = 1, kDF = 2 };

__device__ __forceinline__ void two_prod_sum(float a, float b, float& hi, float& lo) {
  float p, e, s, q;
  two_prod(a, b, p, e);  // a b = p + e exactly (no underflow)
  two_sum(hi, p, s, q);  // hi + p = s + q exactly
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(q, e));
}

// One BMX x BMX output tile per block (16 x 16 threads, TMX x TMX each).
template <typename T, int MODE, int BMX, bool AR, bool BR>
__global__ void __launch_bounds__(NT) gemm_tile_kernel(const T* __restrict__ A, int64_t lda,
                                                       const T* __restrict__ B, int64_t ldb,
                                                       int64_t M, int64_t N, int64_t K,
                                                       int64_t kchunk, bool sym,
                                                       T* __restrict__ out, int64_t ldo,
                                                       double* __restrict__ part,
                                                       double* __restrict__ sq_part, bool swap) {
  constexpr int BM = BMX, BN = BMX, TM = BMX / 16, TN = BMX / 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ double red[32];
  // grid.x walks the (possibly huge) row-tile range, grid.y the column tiles;
  // swapped when the column tiles are the ones above grid.y's 65535 limit
  const unsigned bx = swap ? blockIdx.y : blockIdx.x, by = swap ? blockIdx.x : blockIdx.y;
  const unsigned gny = swap ? gridDim.x : gridDim.y;
  const int64_t m0 = (int64_t)bx * BM, n0 = (int64_t)by * BN;
  // Gram: tiles strictly below the diagonal are mirrored, not computed.
  const bool skip = sym && (by < bx);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);

  using Acc = typename std::conditional<MODE == kF64, double, float>::type;
  Acc acc[TM][TN];
  float lo[TM][TN];
  double acc64[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[i][j] = Acc(0);
      lo[i][j] = 0.0f;
      acc64[i][j] = 0.0;
    }

  if (!skip) {
    int tiles = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
      for (int e = threadIdx.x; e < BM * BK; e += NT) {
        int i, kk;
        if (AR) {
          i = e / BK;
          kk = e % BK;
        } else {
          kk = e / BM;
          i = e % BM;
        }
        const int64_t m = m0 + i, k = k0 + kk;
        T v = T(0);
        if (m < M && k < ke) v = AR ? A[m * lda + k] : A[m + k * lda];
        As[kk][i] = v;
      }
      for (int e = threadIdx.x; e < BN * BK; e += NT) {
        int j, kk;
        if (BR) {
          kk = e / BN;
          j = e % BN;
        } else {
          j = e / BK;
          kk = e % BK;
        }
        const int64_t n = n0 + j, k = k0 + kk;
        T v = T(0);
        if (n < N && k < ke) v = BR ? B[k * ldb + n] : B[k + n * ldb];
        Bs[kk][j] = v;
      }
      __syncthreads();
      if constexpr (MODE == kF32) {
        float t[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) t[i][j] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          T a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) t[i][j] = fma(a[i], b[j], t[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] += t[i][j];
        if (++tiles == FLUSH_TILES) {
          tiles = 0;
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              acc64[i][j] += (double)acc[i][j];
              acc[i][j] = 0.0f;
            }
        }
      } else if constexpr (MODE == kDF) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          float a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) two_prod_sum(a[i], b[j], acc[i][j], lo[i][j]);
        }
        if (++tiles == FLUSH_DF) {
          tiles = 0;
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              acc64[i][j] += (double)acc[i][j] + (double)lo[i][j];
              acc[i][j] = 0.0f;
              lo[i][j] = 0.0f;
            }
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          Acc a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = (Acc)As[kk][ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = (Acc)Bs[kk][tx * TN + j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc64[i][j] += (double)acc[i][j] + (double)lo[i][j];
  }

  double sq = 0.0;
  if (!skip) {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t m = m0 + ty * TM + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t n = n0 + tx * TN + j;
        if (n >= N) continue;
        if (part) {
          part[((int64_t)blockIdx.z * M + m) * N + n] = acc64[i][j];
        } else {
          const T v = (T)acc64[i][j];
          out[m * ldo + n] = v;
          sq += (double)v * (double)v;
        }
      }
    }
  }
  if (sq_part) {
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) sq_part[(int64_t)bx * gny + by] = sq;
  }
}

// Sum the split-K partials in order z = 0..S-1; mirror Gram tiles.
template <typename T>
__global__ void reduce_partials_kernel(const double* __restrict__ part, int S, int64_t M,
                                       int64_t N, bool sym, int bt, T* __restrict__ out, int64_t ldo,
                                       double* __restrict__ out64, double* __restrict__ sq_part) {
  __shared__ double red[32];
  double sq = 0.0;
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    int64_t si = i, sj = j;
    if (sym && (j / bt) < (i / bt)) {
      si = j;
      sj = i;
    }
    double s = 0.0;
    for (int z = 0; z < S; ++z) s += part[((int64_t)z * M + si) * N + sj];
    if (out64) out64[e] = s;
    if (out) {
      const T v = (T)s;
      out[i * ldo + j] = v;
      sq += (double)v * (double)v;
    }
  }
  if (sq_part) {
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) sq_part[blockIdx.x] = sq;
  }
}

// Fixed-order sum of per-block partials into one FP64 scalar.
__global__ void sum_scalars_kernel(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

struct Plan {
  int bt;  // square output tile: 64 (kF32, kF64) or 32 (kDF)
  int64_t gm, gn;
  int S;
  int64_t kchunk;
  int reduce_blocks;
};

Plan make_plan(int64_t M, int64_t N, int64_t K, int bt) {
  Plan p;
  p.bt = bt;
  p.gm = (M + bt - 1) / bt;
  p.gn = (N + bt - 1) / bt;
  const int64_t tiles = p.gm * p.gn;
  int64_t S = 1;
  if (tiles < kTargetBlocks / 2) {
    S = (kTargetBlocks + tiles - 1) / tiles;
    S = std::min<int64_t>(S, std::max<int64_t>(1, K / (BK * 8)));
    // keep the FP64 partials within 256 MiB
    const int64_t cap = std::max<int64_t>(1, ((int64_t)256 << 20) / (8 * std::max<int64_t>(1, M * N)));
    S = std::max<int64_t>(1, std::min<int64_t>(S, cap));
    S = std::min<int64_t>(S, 65535);
  }
  p.S = (int)S;
  int64_t kc = (K + S - 1) / S;
  kc = ((kc + BK - 1) / BK) * BK;
  p.kchunk = std::max<int64_t>(kc, BK);
  p.reduce_blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (M * N + 255) / 256));
  return p;
}

template <typename T, bool AR, bool BR>
void launch_tiles(dim3 grid, cudaStream_t st, Mat<T> A, Mat<T> B, int64_t M, int64_t N, int64_t K,
                  int64_t kchunk, bool sym, T* out, int64_t ldo, double* part, double* sqp,
                  bool accurate, bool swap) {
  if constexpr (std::is_same<T, double>::value) {
    gemm_tile_kernel<double, kF64, 64, AR, BR><<<grid, NT, 0, st>>>(A.p, A.ld, B.p, B.ld, M, N, K,
                                                                   kchunk, sym, out, ldo, part, sqp, swap);
  } else {
    if (accurate)
      gemm_tile_kernel<float, kDF, 32, AR, BR><<<grid, NT, 0, st>>>(A.p, A.ld, B.p, B.ld, M, N, K,
                                                                   kchunk, sym, out, ldo, part, sqp, swap);
    else
      gemm_tile_kernel<float, kF32, 64, AR, BR><<<grid, NT, 0, st>>>(A.p, A.ld, B.p, B.ld, M, N, K,
                                                                    kchunk, sym, out, ldo, part, sqp, swap);
  }
}

}  // namespace

template <typename T>
size_t gemm_ws_bytes(int64_t M, int64_t N, int64_t K, bool fp64_out_or_sym) {
  size_t best = 0;
  for (int bt : {64, 32}) {
    const Plan p = make_plan(M, N, K, bt);
    size_t b = 0;
    if (p.S > 1 || fp64_out_or_sym) b += (size_t)p.S * M * N * sizeof(double);
    b += (size_t)std::max<int64_t>(p.gm * p.gn, p.reduce_blocks) * sizeof(double) + 512;
    best = std::max(best, b);
  }
  return best;
}

template <typename T>
cudaError_t gemm(Mat<T> A, Mat<T> B, int64_t M, int64_t N, int64_t K, T* out, int64_t ldo,
                 double* out64, bool sym, double* sumsq, void* ws, cudaStream_t st, bool accurate) {
  if (M <= 0 || N <= 0) {
    if (sumsq) return cudaMemsetAsync(sumsq, 0, sizeof(double), st);
    return cudaSuccess;
  }
  const bool df = accurate && std::is_same<T, float>::value;
  const Plan p = make_plan(M, N, K, df ? 32 : 64);
  const bool use_part = (p.S > 1) || (out64 != nullptr) || sym;
  double* part = (double*)ws;
  double* sq_part = (double*)((char*)ws + (use_part ? (size_t)p.S * M * N * sizeof(double) : 0));
  sq_part = (double*)(((uintptr_t)sq_part + 255) & ~(uintptr_t)255);
  if (K <= 0) {
    // empty inner dimension: the product is zero
    if (out) {
      cudaError_t e = cudaMemset2DAsync(out, ldo * sizeof(T), 0, N * sizeof(T), M, st);
      if (e != cudaSuccess) return e;
    }
    if (out64) {
      cudaError_t e = cudaMemsetAsync(out64, 0, M * N * sizeof(double), st);
      if (e != cudaSuccess) return e;
    }
    if (sumsq) return cudaMemsetAsync(sumsq, 0, sizeof(double), st);
    return cudaSuccess;
  }
  // grid.y holds at most 65535 tiles: a very wide product puts its column
  // tiles on grid.x instead
  const bool swap = p.gn > 65535;
  if (swap && p.gm > 65535) return cudaErrorInvalidConfiguration;
  count_launch(1 + (use_part ? 1 : 0) + (sumsq ? 1 : 0));
  dim3 grid(swap ? (unsigned)p.gn : (unsigned)p.gm, swap ? (unsigned)p.gm : (unsigned)p.gn, (unsigned)p.S);
  double* sqp = (!use_part && sumsq) ? sq_part : nullptr;
if (A.row && B.row)
    launch_tiles<T, true, true>(grid, st, A, B, M, N, K, p.kchunk, sym, out, ldo,
                                use_part ? part : nullptr, sqp, accurate, swap);
  else if (A.row && !B.row)
    launch_tiles<T, true, false>(grid, st, A, B, M, N, K, p.kchunk, sym, out, ldo,
                                 use_part ? part : nullptr, sqp, accurate, swap);
  else if (!A.row && B.row)
    launch_tiles<T, false, true>(grid, st, A, B, M, N, K, p.kchunk, sym, out, ldo,
                                 use_part ? part : nullptr, sqp, accurate, swap);
  else
    launch_tiles<T, false, false>(grid, st, A, B, M, N, K, p.kchunk, sym, out, ldo,
                                  use_part ? part : nullptr, sqp, accurate, swap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (use_part) {
    reduce_partials_kernel<T><<<p.reduce_blocks, 256, 0, st>>>(
        part, p.S, M, N, sym, p.bt, out, ldo, out64, (sumsq && out) ? sq_part : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (sumsq) {
      if (out) {
        sum_scalars_kernel<<<1, 1024, 0, st>>>(sq_part, p.reduce_blocks, sumsq);
      } else {
        return cudaErrorInvalidValue;  // sum of squares needs the rounded T output
      }
    }
  } else if (sumsq) {
    sum_scalars_kernel<<<1, 1024, 0, st>>>(sq_part, p.gm * p.gn, sumsq);
  }
  return cudaGetLastError();
}

template size_t gemm_ws_bytes<float>(int64_t, int64_t, int64_t, bool);
template size_t gemm_ws_bytes<double>(int64_t, int64_t, int64_t, bool);
template cudaError_t gemm<float>(Mat<float>, Mat<float>, int64_t, int64_t, int64_t, float*,
                                 int64_t, double*, bool, double*, void*, cudaStream_t, bool);
template cudaError_t gemm<double>(Mat<double>, Mat<double>, int64_t, int64_t, int64_t, double*,
                                  int64_t, double*, bool, double*, void*, cudaStream_t, bool);

TT_BOUNDS_READER(bounds_gemm)

}  // namespace ttk
