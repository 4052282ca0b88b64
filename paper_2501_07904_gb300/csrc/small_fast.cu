// Register-resident single-CTA small factorizations: the fast path of
// small_factor() for the sweep's pivoted QLP (SM_QLP) and shifted
// Cholesky-QR (SM_ORTH), for n <= 128 in FP32 and n <= 64 in FP64 or in
// double-float (an FP32 pair, dfloat.cuh: FP64-grade tails at FP32 issue
// rates, selected by SmallParams::df_math).
//
// The symmetric n x n matrix is held in registers, a TI x TJ tile per thread
// (256 threads: FP32 8 x 8 tiles cover 128 x 128, FP64 4 x 4 tiles 64 x 64).
// Every Cholesky factorization is right-looking on these tiles.  Pivoted
// (chol_rl): one pivot per step, the 16 threads holding the pivot row write
// row j of R to shared memory, one barrier, then every thread applies the
// rank-1 update to its tile; each warp keeps its own copy of the remaining
// diagonal and so chooses the next pivot without a further barrier.  Column
// order (chol_col4): the same, four columns per barrier.  Pivoting is virtual
// (nothing is swapped): R's rows come out in step order and its columns keep
// the original coordinates.  The same row operations applied to an identity
// tile give E = L^{-1} P (row j of E belongs to step j), so R^{-1} = E^T comes
// out of the factorization with no triangular inverse.
//
// Pivoted QLP (Stewart's rank-revealing UTV, cited in Sec. 2.2):
//   1. pivoted Cholesky of G = X^T X gives R_1 (the R of column-pivoted QR of X);
//   2. the column-pivoted QR of R_1^T is computed as the pivoted Cholesky of
//      R_1 R_1^T, which makes the same pivot choices and gives the same R_2;
//   3. Q_2(:, 1:r) = R_1^T(:, pivots) R_2,11^{-1} = R_1^T E(1:r, :)^T: the
//      Cholesky-QR factor of the pivoted columns, i.e. the Householder basis
//      up to column signs; in FP32 one more Cholesky-QR pass restores
//      orthonormality.
// R_1's columns carry original coordinates, so Z_1 = Pi_1 Q_2(:, 1:r) comes out
// directly.  Truncation error of rank j: tail(j) = mu^2 + s_1 + trace of the
// Schur complement of R_1 R_1^T after j pivots = sum_{i>j} ||L(:, i)||^2.
#include <math.h>

#include "dfloat.cuh"
#include "internal.h"

namespace ttk {
namespace {

constexpr int FT = 256;  // threads: 8 warps

// Tile rows (I) and columns (J) per thread; ty = tid / 16 and tx = tid % 16
// take 16 values each, so the tiles cover NT = 16 I = 16 J rows and columns.
template <typename T>
struct Tile;
template <>
struct Tile<float> {
  static constexpr int I = 8, J = 8;
};
template <>
struct Tile<double> {
  static constexpr int I = 4, J = 4;
};
template <>
struct Tile<df32> {
  static constexpr int I = 4, J = 4;
};
template <typename T>
constexpr int tile_n() {
  return 16 * Tile<T>::I;
}

struct Scal {
  double trace;
  int kept;
};

// Register tile of a thread: rows r = I ty + i, columns c = tx + 16 jj.  A
// thread's rows are contiguous (16-byte loads fetch its row multipliers); the
// strided columns make the column-side shared-memory reads of a warp hit 16
// distinct banks.
template <typename T>
__device__ __forceinline__ int tile_r(int i) {
  return Tile<T>::I * (int)(threadIdx.x / 16) + i;
}
__device__ __forceinline__ int tile_c(int jj) { return (int)(threadIdx.x % 16) + 16 * jj; }

// Arithmetic of the working type: FP32, FP64 or double-float (dfloat.cuh).
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ df32 tfma(df32 a, df32 b, df32 c) { return fma_df(a, b, c); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ df32 tmax(df32 a, df32 b) { return fmax_df(a, b); }
__device__ __forceinline__ float tshfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double tshfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df32 tshfl_xor(df32 v, int o) {
  return df32(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}
__device__ __forceinline__ float tshfl(unsigned m, float v, int src) { return __shfl_sync(m, v, src); }
__device__ __forceinline__ double tshfl(unsigned m, double v, int src) { return __shfl_sync(m, v, src); }
__device__ __forceinline__ df32 tshfl(unsigned m, df32 v, int src) {
  return df32(__shfl_sync(m, v.h, src), __shfl_sync(m, v.l, src));
}
__device__ __forceinline__ float tinv_sqrt(float x) { return 1.0f / sqrtf(x); }
__device__ __forceinline__ double tinv_sqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ df32 tinv_sqrt(df32 x) { return rsqrt_df(x, rsqrtf(x.h)); }

// K consecutive shared-memory elements (K sizeof(T) a multiple of 16 bytes,
// 16-byte aligned) to and from v[o .. o + K)
template <int K, int N>
__device__ __forceinline__ void vload(const float* p, float (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 x = reinterpret_cast<const float4*>(p)[q];
    v[o + 4 * q] = x.x;
    v[o + 4 * q + 1] = x.y;
    v[o + 4 * q + 2] = x.z;
    v[o + 4 * q + 3] = x.w;
  }
}
template <int K, int N>
__device__ __forceinline__ void vload(const double* p, double (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 2; ++q) {
    const double2 x = reinterpret_cast<const double2*>(p)[q];
    v[o + 2 * q] = x.x;
    v[o + 2 * q + 1] = x.y;
  }
}
template <int K, int N>
__device__ __forceinline__ void vload(const df32* p, df32 (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 2; ++q) {
    const float4 x = reinterpret_cast<const float4*>(p)[q];
    v[o + 2 * q] = df32(x.x, x.y);
    v[o + 2 * q + 1] = df32(x.z, x.w);
  }
}
template <int K, int N>
__device__ __forceinline__ void vstore(float* p, const float (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 4; ++q)
    reinterpret_cast<float4*>(p)[q] =
        make_float4(v[o + 4 * q], v[o + 4 * q + 1], v[o + 4 * q + 2], v[o + 4 * q + 3]);
}
template <int K, int N>
__device__ __forceinline__ void vstore(double* p, const double (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 2; ++q)
    reinterpret_cast<double2*>(p)[q] = make_double2(v[o + 2 * q], v[o + 2 * q + 1]);
}

template <int K, int N>
__device__ __forceinline__ void vstore(df32* p, const df32 (&v)[N], int o) {
#pragma unroll
  for (int q = 0; q < K / 2; ++q)
    reinterpret_cast<float4*>(p)[q] =
        make_float4(v[o + 2 * q].h, v[o + 2 * q].l, v[o + 2 * q + 1].h, v[o + 2 * q + 1].l);
}

// Column-permuted position of column c = tx + 16 jj in a row: the CW =
// 16 / sizeof(T) columns of a thread that share jj / CW are contiguous, so a
// thread reads its TJ columns with TJ / CW 16-byte loads.
template <typename T>
__device__ __forceinline__ int cperm(int c) {
  constexpr int CW = 16 / (int)sizeof(T);
  const int tx = c & 15, jj = c >> 4;
  return (jj / CW) * 16 * CW + tx * CW + jj % CW;
}

template <typename T, int TI>
__device__ __forceinline__ T sel_vec(const T (&d)[TI], int m) {
  T v = d[0];
#pragma unroll
  for (int k = 1; k < TI; ++k) v = (m == k) ? d[k] : v;
  return v;
}

template <typename T, int TI, int TJ>
__device__ void load_regs(T (&a)[TI][TJ], const double* G, int n) {
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) {
      const int r = tile_r<T>(i), c = tile_c(jj);
      a[i][jj] = (r < n && c < n) ? (T)G[r * n + c] : T(0);
    }
}

// a[r][c] = sum_{q < qn} A(r, q) B(c, q) over the thread's tile (r < mr, c < mc).
template <typename T, int TI, int TJ, typename FA, typename FB>
__device__ __forceinline__ void tile_product(T (&a)[TI][TJ], int mr, int mc, int qn, FA fa, FB fb) {
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) a[i][jj] = T(0);
#pragma unroll 2
  for (int q = 0; q < qn; ++q) {
    T ra[TI], cb[TJ];
#pragma unroll
    for (int i = 0; i < TI; ++i) ra[i] = tile_r<T>(i) < mr ? fa(tile_r<T>(i), q) : T(0);
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) cb[jj] = tile_c(jj) < mc ? fb(tile_c(jj), q) : T(0);
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj) a[i][jj] = tfma(ra[i], cb[jj], a[i][jj]);
  }
}

template <typename T, int TI, int TJ>
__device__ __forceinline__ void store_tile(const T (&a)[TI][TJ], T* S, int ld, int mr, int mc) {
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj)
      if (tile_r<T>(i) < mr && tile_c(jj) < mc) S[tile_r<T>(i) * ld + tile_c(jj)] = a[i][jj];
}

// Warp argmax of non-negative candidates, lowest index on ties; 'has' marks
// a lane's candidate.  Returns (index or -1, value).
__device__ __forceinline__ int warp_argmax(bool has, float v, int idx, float& best) {
  const unsigned key = has ? __float_as_uint(v > 0.f ? v : 0.f) : 0u;
  const unsigned mx = __reduce_max_sync(0xffffffffu, key);
  const bool any = __any_sync(0xffffffffu, has);
  const unsigned cand = (has && key == mx) ? (unsigned)idx : 0xffffffffu;
  const unsigned pi = __reduce_min_sync(0xffffffffu, cand);
  best = __uint_as_float(mx);
  return any ? (int)pi : -1;
}
__device__ __forceinline__ int warp_argmax(bool has, double v, int idx, double& best) {
  double b = has ? v : -1.0;
  int bi = has ? idx : 0x7fffffff;
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, b, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > b || (ob == b && oi < bi)) {
      b = ob;
      bi = oi;
    }
  }
  best = b;
  return bi == 0x7fffffff ? -1 : bi;
}

__device__ __forceinline__ int warp_argmax(bool has, df32 v, int idx, df32& best) {
  df32 b = has ? v : df32(-1);
  int bi = has ? idx : 0x7fffffff;
  for (int o = 16; o > 0; o >>= 1) {
    const df32 ob = tshfl_xor(b, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > b || (ob == b && oi < bi)) {
      b = ob;
      bi = oi;
    }
  }
  best = b;
  return bi == 0x7fffffff ? -1 : bi;
}

// rs = 1/sqrt(x) (0 when drop).  FP32: the hardware reciprocal square root
// refined by one Newton step, rs (3 - x rs^2) / 2.
__device__ __forceinline__ float recip_sqrt(float x, bool drop) {
  float r = rsqrtf(x);
  r = r * (1.5f - 0.5f * x * r * r);
  return drop ? 0.f : r;
}
__device__ __forceinline__ double recip_sqrt(double x, bool drop) {
  return drop ? 0.0 : 1.0 / sqrt(x);
}
__device__ __forceinline__ df32 recip_sqrt(df32 x, bool drop) {
  return drop ? df32(0) : tinv_sqrt(x);
}

// Sum of the warp's copy of the remaining diagonal over the entries not yet
// eliminated; the xor butterfly leaves the same value in every lane (and, as
// every warp holds the same copy, in every warp), clamped at 0.
template <typename T, int DM>
__device__ __forceinline__ T remaining_trace(const T (&d)[DM], unsigned dmask) {
  T s = T(0);
#pragma unroll
  for (int m = 0; m < DM; ++m)
    if (!((dmask >> m) & 1u)) s += d[m];
  for (int o = 16; o > 0; o >>= 1) s += tshfl_xor(s, o);
  return s > T(0) ? s : T(0);
}

// Row p of the Schur complement (held by the 16 threads with ty = p / TI as
// tile row IP = p % TI) scaled into row j of R, and row p of the identity
// tile b into row j of E: R's row in natural order (rN) and column-permuted
// (rC), E's row column-permuted (eC).  Eliminated columns give zeros in R
// through the keep multipliers (kC, column-permuted, 0 once eliminated).
template <bool AUG, int IP, typename T, int TI, int TJ>
__device__ __forceinline__ void emit_row(const T (&a)[TI][TJ], const T (&b)[TI][TJ], int p, T dp,
                                         T rs, T* rN, T* rC, T* eC, const T* kC) {
  constexpr int CW = 16 / (int)sizeof(T), HW = 16 * CW;
  const int tx = threadIdx.x & 15;
  T v[TJ], w[TJ], kp[TJ];
#pragma unroll
  for (int h = 0; h < TJ / CW; ++h) vload<CW>(kC + h * HW + tx * CW, kp, h * CW);
#pragma unroll
  for (int jj = 0; jj < TJ; ++jj) {
    const int c = tile_c(jj);
    v[jj] = a[IP][jj] * rs * kp[jj];
    if (c == p) v[jj] = dp * rs;
    rN[c] = v[jj];
    if (AUG) w[jj] = b[IP][jj] * rs;
  }
#pragma unroll
  for (int h = 0; h < TJ / CW; ++h) {
    vstore<CW>(rC + h * HW + tx * CW, v, h * CW);
    if (AUG) vstore<CW>(eC + h * HW + tx * CW, w, h * CW);
  }
}

// Pivoted Cholesky of the symmetric n x n matrix held in the register tiles
// a: largest remaining diagonal first (lowest index on ties), stopping at a
// pivot not above tol * (largest initial diagonal) or as stop_mode says:
//   stop_mode  0: tolerance only;
//              1: first j >= 1 with base + trace <= delta2;
//              2: j == r_stop;
//   kmax       at most this many steps.
// Row j of R belongs to step j and has original-coordinate columns; it is
// stored (ld ld) if R != null.  tails[j] = base + remaining trace before
// step j (if tails != null).  AUG: the same row operations applied to the
// identity (tile b) give row j of E (ld ld, columns < n) = row j of L^{-1} P,
// a dropped step leaving a zero row, so R^{-1} = E^T.  Returns the number of
// steps; sc.trace = the remaining Schur trace (>= 0), sc.kept = steps not
// dropped.  Scratch: ring (7 NT entries, 16-byte aligned), trace_j (n + 1),
// dsm (n).
//
// One step: the owners of the pivot row write row j of R (and E) to a
// double-buffered ring slot, one barrier, every thread applies the rank-1
// update to its tile.  Each warp keeps its own copy of the remaining diagonal
// (DM = NT / 32 entries a lane) and so chooses the next pivot without a
// further barrier.  (Column order: chol_col4.)
template <bool AUG, typename T, int TI, int TJ>
__device__ int chol_rl(T (&a)[TI][TJ], T (&b)[TI][TJ], int n, double tol, int stop_mode,
                       double base, double delta2, int r_stop, int kmax, T* R, T* E, int ld,
                       T* ring, T* trace_j, T* dsm, double* tails, Scal& sc) {
  constexpr int NT = 16 * TI;  // rows and columns the tiles cover
  constexpr int CW = 16 / (int)sizeof(T), HW = 16 * CW, NH = TJ / CW;
  constexpr int DM = NT / 32;  // diagonal entries a lane keeps
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ty = tid >> 4, tx = tid & 15;
  const bool need_trace = stop_mode == 1 || tails != nullptr;
  T* kC = ring + 6 * NT;
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) {
      const int r = tile_r<T>(i), c = tile_c(jj);
      if (AUG) b[i][jj] = (r == c && r < n) ? T(1) : T(0);
      if (r == c && r < n) dsm[r] = a[i][jj];
    }
  if (tid < NT) kC[cperm<T>(tid)] = tid < n ? T(1) : T(0);
  __syncthreads();
  // this warp's copy of the remaining diagonal, d[m] = entry DM lane + m;
  // bit m of dmask is set once that entry is eliminated (or lies beyond n)
  T d[DM];
  unsigned dmask = 0u;
  T dmax = T(0);
#pragma unroll
  for (int m = 0; m < DM; ++m) {
    const int t = DM * lane + m;
    d[m] = t < n ? dsm[t] : T(0);
    if (t >= n) dmask |= 1u << m;
    dmax = tmax(dmax, d[m]);
  }
  for (int o = 16; o > 0; o >>= 1) dmax = tmax(dmax, tshfl_xor(dmax, o));
  // tol_abs >= 0, so dp > tol_abs also means dp > 0 (and is false for NaN)
  const T tol_abs = (T)(tol * (double)dmax);
  const T stop_trace = (T)(delta2 - base);
  int jlim = min(kmax, n);
  if (stop_mode == 2 && r_stop >= 0) jlim = min(jlim, r_stop);
  const int wr0 = 2 * TI * warp;  // this warp's rows: wr0 .. wr0 + 2 TI - 1
  const bool warp_rows = wr0 < n;

  int j = 0, kept = 0;
  for (;; ++j) {
    T* rN = ring + (j & 1) * NT;
    T* rC = ring + 2 * NT + (j & 1) * NT;
    T* eC = ring + 4 * NT + (j & 1) * NT;
    const T trt = need_trace ? remaining_trace(d, dmask) : T(0);
    int p;
    T dp;
    {
      bool has = false;
      T bv = T(0);
      int bi = 0;
#pragma unroll
      for (int m = 0; m < DM; ++m)
        if (!((dmask >> m) & 1u)) {
          const T v = d[m] > T(0) ? d[m] : T(0);
          if (!has || v > bv) {
            has = true;
            bv = v;
            bi = DM * lane + m;
          }
        }
      p = warp_argmax(has, bv, bi, dp);
    }
    const bool stop = j >= jlim || p < 0 || (stop_mode == 1 && j >= 1 && trt <= stop_trace) ||
                      !(dp > tol_abs);
    if (need_trace && tid == 0) trace_j[j] = trt;
    if (stop) break;
    ++kept;
    const T rs = recip_sqrt(dp, false);
    if (tid == 0) kC[cperm<T>(p)] = T(0);
    if (ty == (unsigned)p / TI) {
      switch ((unsigned)p % TI) {
#define TT_EMIT(K)                                                          \
  case K:                                                                   \
    emit_row<AUG, K % TI>(a, b, p, dp, rs, rN, rC, eC, kC);               \
    break;
        TT_EMIT(0) TT_EMIT(1) TT_EMIT(2) TT_EMIT(3) TT_EMIT(4) TT_EMIT(5) TT_EMIT(6) TT_EMIT(7)
#undef TT_EMIT
      }
    }
    __syncthreads();
    // the step's row loads all go out at once
    T l[DM], lr[TI], lc[TJ], le[TJ];
    vload<DM>(rN + DM * lane, l, 0);
    vload<TI>(rN + TI * ty, lr, 0);
    if (R != nullptr && tid < n) R[j * ld + tid] = rN[tid];
    if (AUG && tid < n) E[j * ld + tid] = eC[cperm<T>(tid)];
    // rank-1 update of every tile column below n
    if (warp_rows) {
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int clo = h * HW;
        if (clo < n) {
          vload<CW>(rC + clo + tx * CW, lc, h * CW);
#pragma unroll
          for (int i = 0; i < TI; ++i)
#pragma unroll
            for (int k = 0; k < CW; ++k)
              a[i][h * CW + k] = tfma(-lr[i], lc[h * CW + k], a[i][h * CW + k]);
        }
        if (AUG && clo < n) {
          vload<CW>(eC + clo + tx * CW, le, h * CW);
#pragma unroll
          for (int i = 0; i < TI; ++i)
#pragma unroll
            for (int k = 0; k < CW; ++k)
              b[i][h * CW + k] = tfma(-lr[i], le[h * CW + k], b[i][h * CW + k]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < DM; ++m) d[m] = tfma(-l[m], l[m], d[m]);
    if ((unsigned)p / DM == (unsigned)lane) dmask |= 1u << ((unsigned)p % DM);
  }
  const T trend = remaining_trace(d, dmask);
  __syncthreads();  // trace_j[j] was written after the last barrier
  if (tails)
    for (int q = tid; q <= j; q += FT) tails[q] = base + (double)trace_j[q];
  if (tid == 0) {
    sc.trace = (double)trend;
    sc.kept = kept;
  }
  __syncthreads();
  return j;
}

// The four rows j0 .. j0 + kb - 1 (kb <= 4) of a column-order block, held by
// this thread as tile rows I0 .. I0 + 3: row s of R (and of E) from the block
// factor (Lt = the block's rows of R inside the block, rs = the pivots'
// reciprocal square roots) and the thread's columns, published to the ring
// slots slot + s * 3 NT (natural order, column-permuted, E column-permuted).
template <bool AUG, int I0, typename T, int TI, int TJ>
__device__ __forceinline__ void publish_block4(const T (&a)[TI][TJ], const T (&b)[TI][TJ],
                                               const T (&Lt)[4][4], const T (&rs)[4], int j0,
                                               int kb, T* slot) {
  constexpr int NT = 16 * TI, CW = 16 / (int)sizeof(T), HW = 16 * CW, NH = TJ / CW;
  const int tx = threadIdx.x & 15;
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    T rv[4][CW], ev[4][CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      const int jj = h * CW + k, c = tile_c(jj);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        T x = a[I0 + s][jj];
        T ex = AUG ? b[I0 + s][jj] : T(0);
#pragma unroll
        for (int u = 0; u < s; ++u) {
          x = tfma(-Lt[u][s], rv[u][k], x);
          if (AUG) ex = tfma(-Lt[u][s], ev[u][k], ex);
        }
        rv[s][k] = c > j0 + s ? x * rs[s] : (c == j0 + s ? Lt[s][s] : T(0));
        ev[s][k] = ex * rs[s];
        if (s < kb) slot[s * 3 * NT + c] = rv[s][k];
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < kb) {
        vstore<CW>(slot + s * 3 * NT + NT + h * HW + tx * CW, rv[s], 0);
        if (AUG) vstore<CW>(slot + s * 3 * NT + 2 * NT + h * HW + tx * CW, ev[s], 0);
      }
  }
}

// Column-order Cholesky (no pivoting, all columns up to kmax) blocked by four
// columns: the same fused multiply-adds in the same order as a right-looking
// elimination with one column per barrier, so the same results.  A pivot not
// above tol * (largest initial diagonal) is dropped (zero row of R and E, no
// elimination); R^{-1} = E^T (rows of E stored, ld ld, columns < n); sc.kept
// counts the pivots kept.  The 16 threads holding rows j0 .. j0 + 3 (consecutive
// rows of one tile-row group) gather the block's 4 x 4 upper triangle by
// shuffles, factor it (every one of them, identically), form the block's rows
// of R and E for their columns and publish them; after one barrier every
// thread applies the four rank-1 updates in order.  One barrier per four
// columns instead of one per column.  Ring: two sets of four row slots
// (24 NT entries).
template <bool AUG, typename T, int TI, int TJ>
__device__ void chol_col4(T (&a)[TI][TJ], T (&b)[TI][TJ], int n, double tol, int kmax, T* E,
                          int ld, T* ring, T* dsm, Scal& sc) {
  constexpr int NT = 16 * TI;
  constexpr int CW = 16 / (int)sizeof(T), HW = 16 * CW, NH = TJ / CW;
  constexpr int DM = NT / 32;
  static_assert(TI % 4 == 0, "a tile-row group must hold whole blocks of four rows");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ty = tid >> 4, tx = tid & 15;
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) {
      const int r = tile_r<T>(i), c = tile_c(jj);
      if (AUG) b[i][jj] = (r == c && r < n) ? T(1) : T(0);
      if (r == c && r < n) dsm[r] = a[i][jj];
    }
  __syncthreads();
  T dmax = T(0);
#pragma unroll
  for (int m = 0; m < DM; ++m) {
    const int t = DM * lane + m;
    dmax = tmax(dmax, t < n ? dsm[t] : T(0));
  }
  for (int o = 16; o > 0; o >>= 1) dmax = tmax(dmax, tshfl_xor(dmax, o));
  // tol_abs >= 0, so dd > tol_abs also means dd > 0 (and is false for NaN)
  const T tol_abs = (T)(tol * (double)dmax);
  const int jlim = min(kmax, n);
  const int wr0 = 2 * TI * warp;  // this warp's rows: wr0 .. wr0 + 2 TI - 1
  int kept = 0;
  for (int j0 = 0, blk = 0; j0 < jlim; j0 += 4, ++blk) {
    const int kb = min(4, jlim - j0);
    T* slot = ring + (blk & 1) * 12 * NT;
    if (ty == j0 / TI) {
      // the block's upper triangle U[s][t] = A(j0 + s, j0 + t), s <= t, from
      // the threads holding columns j0 .. j0 + 3 (all in column block jb)
      const unsigned hm = 0xFFFFu << (lane & 16);
      const int i0 = j0 % TI, jb = j0 / 16;
      T colv[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        T rowv[TJ];
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj) rowv[jj] = a[s][jj];
#pragma unroll
        for (int o = 4; o < TI; o += 4)
#pragma unroll
          for (int jj = 0; jj < TJ; ++jj) rowv[jj] = (i0 == o) ? a[o + s][jj] : rowv[jj];
        colv[s] = sel_vec(rowv, jb);
      }
      T U[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int src = (lane & 16) | ((j0 + t) & 15);
#pragma unroll
        for (int s = 0; s < 4; ++s) U[s][t] = tshfl(hm, colv[s], src);
      }
      // its factor: Lt[s][t] = R(j0 + s, j0 + t), t >= s
      T Lt[4][4], rs[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        T dd = U[s][s];
#pragma unroll
        for (int u = 0; u < s; ++u) dd = tfma(-Lt[u][s], Lt[u][s], dd);
        const bool drop = (s >= kb) || !(dd > tol_abs);
        rs[s] = recip_sqrt(dd, drop);
        Lt[s][s] = drop ? T(0) : dd * rs[s];
#pragma unroll
        for (int t = s + 1; t < 4; ++t) {
          T x = U[s][t];
#pragma unroll
          for (int u = 0; u < s; ++u) x = tfma(-Lt[u][s], Lt[u][t], x);
          Lt[s][t] = x * rs[s];
        }
      }
      if (i0 == 0)
        publish_block4<AUG, 0>(a, b, Lt, rs, j0, kb, slot);
      else
        publish_block4<AUG, 4 % TI>(a, b, Lt, rs, j0, kb, slot);
    }
    __syncthreads();
    if (tid == 0)
      for (int s = 0; s < kb; ++s) kept += (slot[s * 3 * NT + j0 + s] != T(0)) ? 1 : 0;
    // the block's rank-1 updates in order; a warp whose rows are all
    // eliminated skips, column halves as in chol_rl's column order
    for (int s = 0; s < kb; ++s) {
      const int j = j0 + s;
      const T* rN = slot + s * 3 * NT;
      if (AUG && tid < n) E[j * ld + tid] = rN[2 * NT + cperm<T>(tid)];
      if (wr0 + 2 * TI - 1 > j) {
        T lr[TI], lc[TJ], le[TJ];
        vload<TI>(rN + TI * ty, lr, 0);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const int clo = h * HW, chi = clo + HW - 1;
          if (clo < n && chi > j && chi >= wr0) {
            vload<CW>(rN + NT + clo + tx * CW, lc, h * CW);
#pragma unroll
            for (int i = 0; i < TI; ++i)
#pragma unroll
              for (int k = 0; k < CW; ++k)
                a[i][h * CW + k] = tfma(-lr[i], lc[h * CW + k], a[i][h * CW + k]);
          }
          if (AUG && clo < n && clo <= j) {
            vload<CW>(rN + 2 * NT + clo + tx * CW, le, h * CW);
#pragma unroll
            for (int i = 0; i < TI; ++i)
#pragma unroll
              for (int k = 0; k < CW; ++k)
                b[i][h * CW + k] = tfma(-lr[i], le[h * CW + k], b[i][h * CW + k]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    sc.kept = kept;
    sc.trace = 0.0;
  }
  __syncthreads();
}

template <typename T, typename ZT>
__global__ void __launch_bounds__(FT, 1) small_fast_kernel(const double* __restrict__ G,
                                                           SmallParams prm, ZT* __restrict__ Z,
                                                           int ldz, StepInfo* __restrict__ info,
                                                           T* __restrict__ gws) {
  constexpr int TI = Tile<T>::I, TJ = Tile<T>::J, NT = tile_n<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = prm.n, tid = threadIdx.x;
  const int nn = ((n + 31) / 32) * 32, ld = nn + 1;
  T* ring = (T*)smem_raw;          // 24 NT: rows of R and E in flight, keep multipliers
  T* trj = ring + 24 * NT;         // NT + 1 (padded to NT + 4): traces per step
  T* dsm = trj + NT + 4;           // NT: initial diagonal, completion vector
  T* R1 = dsm + NT;                // nn x ld
  T* R2 = R1 + nn * ld;            // nn x ld
  T* X = R2 + nn * ld;             // nn x ld: E of the latest factorization
  __shared__ Scal sc;
  __shared__ double redd[32];
  T a[TI][TJ], b[TI][TJ];

  // the register tile's loads go out first; the FP64 trace and the scalars
  // load meanwhile
  const bool gw = prm.mode == SM_QLP && prm.Gw != nullptr;
  load_regs(a, gw ? prm.Gw : G, n);
  const double x2_in = prm.x2_dev ? *prm.x2_dev : 0.0;
  const double nA_in = (prm.normA2_dev && !prm.normA2_is_trace) ? *prm.normA2_dev : 0.0;
  double tr = 0.0;
  for (int i = tid; i < n; i += FT) tr += G[i * n + i];
  tr = block_sum(tr, redd);
  const double x2 = prm.x2_dev ? x2_in : tr;
  double normA2 = -1.0, delta2 = prm.delta2;
  if (prm.normA2_dev) {
    normA2 = prm.normA2_is_trace ? tr : nA_in;
    delta2 = prm.delta2_scale * normA2;
  }
  const bool finite = isfinite(tr) && isfinite(x2) && (normA2 < 0.0 || isfinite(normA2));
  if (tid == 0) {
    info->x2 = x2;
    info->trace = tr;
    info->delta2 = delta2;
    info->normA2 = normA2;
    info->status = finite ? 0 : 1;
  }
  if (!finite) {
    for (int e = tid; e < n * ldz; e += FT) Z[e] = ZT(0);
    if (tid == 0) {
      info->r = 1;
      info->k1 = 0;
      info->nsteps = 0;
      info->mu2 = 0.0;
      info->s1 = 0.0;
      info->tail = 0.0;
    }
    return;
  }

  if (prm.mode == SM_ORTH) {
    if (prm.shift_rel > 0.0) {
      const T sh = (T)(prm.shift_rel * tr);
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj)
          if (tile_r<T>(i) == tile_c(jj) && tile_r<T>(i) < n) a[i][jj] += sh;
    }
    chol_col4<true>(a, b, n, prm.piv_tol, n, X, ld, ring, dsm, sc);
    // Z = R^{-1} = E^T: warp w writes rows w, w + 8, ...
    for (int i = tid >> 5; i < n; i += FT / 32)
      for (int c = tid & 31; c < ldz; c += 32) Z[(size_t)i * ldz + c] = (c < n) ? (ZT)X[c * ld + i] : ZT(0);
    if (tid == 0) {
      info->r = sc.kept;
      info->k1 = sc.kept;
      info->nsteps = n;
      info->mu2 = 0.0;
      info->s1 = 0.0;
      info->tail = 0.0;
    }
    return;
  }

  // ---- SM_QLP ----------------------------------------------------------
  T* Tw = gws;  // E of the whitening factor (global scratch, nn x ld)
  if (gw) {
    // W^T W = T^T T; factor A = T^{-T} G T^{-1}, the Gram of X Q for Q = W T^{-1}
    // (T^{-1} = E^T: T^{-1}(k, c) = E(c, k), upper triangular)
    chol_col4<true>(a, b, n, 0.0, n, X, ld, ring, dsm, sc);
    for (int e = tid; e < nn * ld; e += FT) Tw[e] = X[e];
    for (int e = tid; e < n * n; e += FT) R2[(e / n) * ld + e % n] = (T)G[e];
    __syncthreads();
    // G T^{-1}, back into R2
    tile_product(a, n, n, n, [&](int r, int k) { return R2[r * ld + k]; },
                 [&](int c, int k) { return k <= c ? X[c * ld + k] : T(0); });
    __syncthreads();
    store_tile(a, R2, ld, n, n);
    __syncthreads();
    // a = T^{-T} (G T^{-1})
    tile_product(a, n, n, n, [&](int r, int k) { return k <= r ? X[r * ld + k] : T(0); },
                 [&](int c, int k) { return R2[k * ld + c]; });
    double t2 = 0.0;
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj)
        if (tile_r<T>(i) == tile_c(jj)) t2 += (double)a[i][jj];
    tr = block_sum(t2, redd);
  }
  // range miss mu^2 = ||X||^2 - ||X P_W||^2; zero by construction when W
  // spans the whole row space (Omega = I), where the difference is rounding
  const double mu2 = (prm.x2_dev && !prm.range_exact) ? fmax(0.0, x2 - tr) : 0.0;

  // phase 1: pivoted Cholesky of G
  const int k1 = chol_rl<false>(a, b, n, prm.piv_tol, 0, 0.0, 0.0, 0, n, R1, (T*)nullptr,
                                      ld, ring, trj, dsm, nullptr, sc);
  const double s1 = sc.trace;
  // phase 2: pivoted Cholesky of M = R_1 R_1^T, with E
  tile_product(a, k1, k1, n, [&](int r, int q) { return R1[r * ld + q]; },
               [&](int c, int q) { return R1[c * ld + q]; });
  const bool fixed = prm.r_fixed >= 1;
  const int rt = fixed ? min(prm.r_fixed, prm.r_cap) : -1;
  const int r2 = chol_rl<true>(a, b, k1, 0.0, fixed ? 2 : 1, mu2 + s1, delta2, rt,
                                     min(k1, prm.r_cap), (T*)nullptr, X, ld, ring, trj, dsm,
                                     info->tails, sc);
  const int r = fixed ? rt : max(1, r2);
  const int rz = min(r, r2);  // columns produced by the factorization

  // Zs = R_1^T E(1:rz, :)^T (n x rz), into R2
  tile_product(a, n, rz, k1, [&](int i, int q) { return R1[q * ld + i]; },
               [&](int c, int q) { return X[c * ld + q]; });
  store_tile(a, R2, ld, n, rz);
  __syncthreads();
  if (sizeof(T) == 4 && rz > 0) {
    // one more Cholesky-QR pass: Zs <- Zs R^{-1}, R^T R = Zs^T Zs, R^{-1} = E^T
    tile_product(a, rz, rz, n, [&](int rr, int q) { return R2[q * ld + rr]; },
                 [&](int c, int q) { return R2[q * ld + c]; });
    chol_col4<true>(a, b, rz, 0.0, rz, X, ld, ring, dsm, sc);
    tile_product(a, n, rz, rz, [&](int i, int q) { return R2[i * ld + q]; },
                 [&](int c, int q) { return q <= c ? X[c * ld + q] : T(0); });
    __syncthreads();
    store_tile(a, R2, ld, n, rz);
    __syncthreads();
  }
  // fixed rank above the numerical rank: complete with unit vectors
  // orthogonalized (twice) against the columns already formed
  if (r > rz && tid < 32) {
    const int lane = tid;
    T* v = dsm;
    int cand = 0;
    for (int c = rz; c < r; ++c) {
      for (; cand < n; ++cand) {
        for (int i = lane; i < n; i += 32) v[i] = (i == cand) ? T(1) : T(0);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int bcol = 0; bcol < c; ++bcol) {
            T dot = T(0);
            for (int i = lane; i < n; i += 32) dot += R2[i * ld + bcol] * v[i];
            for (int o = 16; o > 0; o >>= 1) dot += tshfl_xor(dot, o);
            for (int i = lane; i < n; i += 32) v[i] -= dot * R2[i * ld + bcol];
            __syncwarp();
          }
        }
        T nv = T(0);
        for (int i = lane; i < n; i += 32) nv += v[i] * v[i];
        for (int o = 16; o > 0; o >>= 1) nv += tshfl_xor(nv, o);
        if (nv > T(0.25)) {
          const T s = tinv_sqrt(nv);
          for (int i = lane; i < n; i += 32) R2[i * ld + c] = v[i] * s;
          __syncwarp();
          ++cand;
          break;
        }
      }
    }
  }
  __syncthreads();
  // output (whitened: Z_1 = T^{-1} Zs, the whitening E brought back into X)
  if (gw) {
    for (int e = tid; e < nn * ld; e += FT) X[e] = Tw[e];
    __syncthreads();
    tile_product(a, n, r, n, [&](int i, int k) { return k >= i ? X[k * ld + i] : T(0); },
                 [&](int c, int k) { return R2[k * ld + c]; });
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
      for (int jj = 0; jj < TJ; ++jj)
        if (tile_r<T>(i) < n && tile_c(jj) < r) Z[(size_t)tile_r<T>(i) * ldz + tile_c(jj)] = (ZT)a[i][jj];
  } else {
    for (int i = tid >> 5; i < n; i += FT / 32)
      for (int c = tid & 31; c < r; c += 32) Z[(size_t)i * ldz + c] = (ZT)R2[i * ld + c];
  }
  if (tid == 0) {
    info->r = r;
    info->k1 = k1;
    info->nsteps = r2;
    info->mu2 = mu2;
    info->s1 = s1;
    info->tail = info->tails[min(r, r2)];
  }
}

template <typename T>
size_t fast_smem_bytes(int n) {
  constexpr int NT = tile_n<T>();
  const int nn = ((n + 31) / 32) * 32, ld = nn + 1;
  return (size_t)(3 * nn * ld + 26 * NT + 4) * sizeof(T);
}

template <typename T, typename ZT>
cudaError_t launch_fast(const double* G, SmallParams prm, void* Z, int ldz, void* ws,
                        StepInfo* info, cudaStream_t st) {
  const size_t sm = fast_smem_bytes<T>(prm.n);
  auto kern = small_fast_kernel<T, ZT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  count_launch();
  kern<<<1, FT, sm, st>>>(G, prm, (ZT*)Z, ldz, info, (T*)ws);
  return cudaGetLastError();
}

}  // namespace

bool small_fast_eligible(const SmallParams& prm, bool fp64) {
  if (prm.mode != SM_QLP && prm.mode != SM_ORTH) return false;
  if (prm.l11) return false;
  const int lim = fp64 ? tile_n<double>() : tile_n<float>();
  return prm.n >= 1 && prm.n <= lim;
}

cudaError_t small_factor_fast(const double* G, SmallParams prm, bool fp64_math, void* Z,
                              bool z_fp64, int ldz, void* ws, StepInfo* info, cudaStream_t st) {
  if (fp64_math && prm.df_math)
    return z_fp64 ? launch_fast<df32, double>(G, prm, Z, ldz, ws, info, st)
                  : launch_fast<df32, float>(G, prm, Z, ldz, ws, info, st);
  if (fp64_math)
    return z_fp64 ? launch_fast<double, double>(G, prm, Z, ldz, ws, info, st)
                  : launch_fast<double, float>(G, prm, Z, ldz, ws, info, st);
  return z_fp64 ? launch_fast<float, double>(G, prm, Z, ldz, ws, info, st)
                : launch_fast<float, float>(G, prm, Z, ldz, ws, info, st);
}

TT_BOUNDS_READER(bounds_small_fast)

}  // namespace ttk
