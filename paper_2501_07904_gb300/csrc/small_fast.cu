// Register-resident single-CTA small factorizations: the fast path of
// small_factor() for the sweep's pivoted QLP (SM_QLP) and shifted
// Cholesky-QR (SM_ORTH), for n <= 128 in FP32 and n <= 64 in FP64.
//
// The symmetric n x n matrix is held in registers, a 4 x 8 tile per thread
// (512 threads cover 128 x 128).  The Cholesky factorizations are blocked by
// panels of 32 steps: one warp factors a panel from a shared-memory copy of
// the Schur complement (pivot by warp reductions, left-looking column
// updates), then every thread applies the panel's rank-32 update to its
// tile.  Pivoting is virtual (nothing is swapped): the factor's rows come out
// in pivot order and its columns keep the original coordinates.
//
// Pivoted QLP (Stewart's rank-revealing UTV, cited in Sec. 2.2):
//   1. pivoted Cholesky of G = X^T X gives R_1 (the R of column-pivoted QR of X);
//   2. the column-pivoted QR of R_1^T is computed as the pivoted Cholesky of
//      R_1 R_1^T, which makes the same pivot choices and gives the same R_2;
//   3. Q_2(:, 1:r) = R_1^T(:, pivots) R_2,11^{-1}: the Cholesky-QR factor of the
//      pivoted columns, i.e. the Householder basis up to column signs; in FP32
//      one more Cholesky-QR pass restores orthonormality.
// R_1's columns carry original coordinates, so Z_1 = Pi_1 Q_2(:, 1:r) comes out
// directly.  Truncation error of rank j: tail(j) = mu^2 + s_1 + trace of the
// Schur complement of R_1 R_1^T after j pivots = sum_{i>j} ||L(:, i)||^2.
#include <math.h>

#include "internal.h"

namespace ttk {
namespace {

constexpr int FT = 512;  // threads
constexpr int NP = 128;  // the register tiles cover NP x NP

struct Scal {
  int p, stop;
  double dp, trace;
};

// Register tile of a thread: rows r = ty + 32 i (i < 4), columns c = tx + 16 jj
// (jj < 8) with ty = tid / 16, tx = tid % 16.  The strided columns make the
// column-side shared-memory reads of a warp hit 16 distinct banks.
__device__ __forceinline__ int tile_r(int i) { return (int)(threadIdx.x / 16) + 32 * i; }
__device__ __forceinline__ int tile_c(int jj) { return (int)(threadIdx.x % 16) + 16 * jj; }

template <typename T>
__device__ __forceinline__ T sel4(const T (&a)[4][8], int i, int jj) {
  return i == 0 ? a[0][jj] : (i == 1 ? a[1][jj] : (i == 2 ? a[2][jj] : a[3][jj]));
}

template <typename T>
__device__ void load_regs(T (&a)[4][8], const double* G, int n) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int r = tile_r(i), c = tile_c(jj);
      a[i][jj] = (r < n && c < n) ? (T)G[r * n + c] : T(0);
    }
}

// a[r][c] = sum_{q < qn} A(r, q) B(c, q) over the thread's tile (r < mr, c < mc).
template <typename T, typename FA, typename FB>
__device__ __forceinline__ void tile_product(T (&a)[4][8], int mr, int mc, int qn, FA fa, FB fb) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) a[i][jj] = T(0);
#pragma unroll 4
  for (int q = 0; q < qn; ++q) {
    T ra[4], cb[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) ra[i] = tile_r(i) < mr ? fa(tile_r(i), q) : T(0);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) cb[jj] = tile_c(jj) < mc ? fb(tile_c(jj), q) : T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) a[i][jj] = fma(ra[i], cb[jj], a[i][jj]);
  }
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

// rs = 1/sqrt(x) and inv = 1/x (both 0 when drop).  FP32: the hardware
// reciprocal square root refined by one Newton step, rs (3 - x rs^2) / 2.
__device__ __forceinline__ void recip_sqrt(float x, bool drop, float& rs, float& inv) {
  float r = rsqrtf(x);
  r = r * (1.5f - 0.5f * x * r * r);
  rs = drop ? 0.f : r;
  inv = drop ? 0.f : r * r;
}
__device__ __forceinline__ void recip_sqrt(double x, bool drop, double& rs, double& inv) {
  rs = drop ? 0.0 : 1.0 / sqrt(x);
  inv = drop ? 0.0 : 1.0 / x;
}

// Cholesky of the symmetric n x n matrix held in the register tiles a.
//   pivot      largest remaining diagonal first (lowest index on ties); else
//              column order, a column whose remaining diagonal is not above
//              tol * (largest initial diagonal) being dropped (zero row of R,
//              no elimination);
//   stop_mode  0: tolerance (pivoted) or all columns (column order);
//              1: first j >= 1 with base + trace <= delta2;
//              2: j == r_stop;
//   kmax       at most this many steps.
// Rows of R (ld ldr) in step order with original-coordinate columns;
// perm[j] = column eliminated at step j; tails[j] = base + remaining trace
// before step j (if tails != null).  Returns the number of steps; sc.trace =
// the remaining Schur trace (>= 0).
//
// Left-looking on the factor itself: the matrix is copied once to shared S
// (ld lds) and the pivot column of step j is S(p, i) - sum_{q<j} R(q, p)
// R(q, i), so no Schur complement is ever written back.  Four threads share
// row i (= tid / 4) and split the sum over q by q mod 4; each keeps the
// row's remaining diagonal.  A step takes one barrier, after row j of R and
// the next step's per-warp pivot and trace partials are written.  Pivoting
// is virtual.
template <typename T>
__device__ int pchol(T (&a)[4][8], int n, bool pivot, double tol, int stop_mode, double base,
                     double delta2, int r_stop, int kmax, T* R, int ldr, int* perm, T* S, int lds,
                     T* part_v, int* part_i, T* trace_j, double* tails, Scal& sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row = tid >> 2, sub = tid & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int r = tile_r(i), c = tile_c(jj);
      if (r < n && c < n) S[r * lds + c] = a[i][jj];
    }
  __syncthreads();
  bool done = row >= n;
  T d = done ? T(0) : S[row * lds + row];
  // largest initial diagonal
  double d0;
  {
    T m = (sub == 0 && !done) ? d : T(0);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) part_v[warp] = m;
    __syncthreads();
    T mm = T(0);
    for (int w = 0; w < FT / 32; ++w) mm = fmax(mm, part_v[w]);
    d0 = (double)mm;
    __syncthreads();
  }
  // The step loop runs in T only (FP64 issues at a small fraction of the FP32
  // rate): thresholds are formed once, traces kept in trace_j[] and turned
  // into FP64 tails after the loop.
  const T tol_abs = (T)(tol * d0);
  const T stop_trace = (T)(delta2 - base);
  // Per-warp partials of step jn (pivot candidate, trace, and row jn's
  // diagonal for column order), double-buffered by step parity so that one
  // barrier per step suffices.
  auto partials = [&](int jn, int par) {
    const bool cand = (sub == 0) && !done;
    T tr = cand ? d : T(0);
    tr += __shfl_xor_sync(0xffffffffu, tr, 4);  // the row sums sit on lanes 4k
    tr += __shfl_xor_sync(0xffffffffu, tr, 8);
    tr += __shfl_xor_sync(0xffffffffu, tr, 16);
    T bv;
    const int bi = warp_argmax(cand, cand ? d : T(0), row, bv);
    if (lane == 0) {
      part_v[par * 64 + warp] = bv;
      part_v[par * 64 + 16 + warp] = tr;
      part_i[par * 32 + warp] = bi;
    }
    if (sub == 0 && row == jn) part_v[par * 64 + 32] = d;
  };
  partials(0, 0);
  __syncthreads();
  int j = 0;
  for (;; ++j) {
    const int par = j & 1;
    // every warp combines the FT/32 partials, one per lane (warps are in row
    // order, so the lowest row wins a tie as within a warp)
    T cv = T(0), ct = T(0);
    int ci = -1;
    if (lane < FT / 32) {
      ci = part_i[par * 32 + lane];
      cv = part_v[par * 64 + lane];
      ct = part_v[par * 64 + 16 + lane];
    }
    // full butterfly: every lane (and so every warp) holds the same trace and
    // takes the same stop decision
    for (int o = 16; o > 0; o >>= 1) ct += __shfl_xor_sync(0xffffffffu, ct, o);
    T bv;
    const int bi = warp_argmax(ci >= 0, cv, ci, bv);
    int p;
    T dp;
    if (pivot) {
      p = bi;
      dp = bv;
    } else {
      p = j < n ? j : -1;
      dp = (p >= 0) ? part_v[par * 64 + 32] : T(0);
    }
    const T trt = ct > T(0) ? ct : T(0);
    int stop = 0;
    bool drop = false;
    if (j >= kmax || j >= n || p < 0) stop = 1;  // every step eliminates or drops a row
    if (!stop && stop_mode == 1 && j >= 1 && trt <= stop_trace) stop = 1;
    if (!stop && stop_mode == 2 && j == r_stop) stop = 1;
    if (!stop) {
      const bool ok = (dp > T(0)) && (dp > tol_abs);
      if (pivot && !ok) stop = 1;
      if (!pivot && !ok) drop = true;
    }
    if (tid == 0) trace_j[j] = trt;
    if (stop) break;
    // column p of the Schur complement for this thread's row: four
    // independent partial sums over q = sub, sub + 4, ... keep loads in flight
    T acc = T(0);
    if (!done && !drop) {
      const T* rp = R + p;
      const T* rr = R + row;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int q = sub;
      for (; q + 12 < j; q += 16) {
        a0 += rp[q * ldr] * rr[q * ldr];
        a1 += rp[(q + 4) * ldr] * rr[(q + 4) * ldr];
        a2 += rp[(q + 8) * ldr] * rr[(q + 8) * ldr];
        a3 += rp[(q + 12) * ldr] * rr[(q + 12) * ldr];
      }
      for (; q < j; q += 4) a0 += rp[q * ldr] * rr[q * ldr];
      acc = (a0 + a1) + (a2 + a3);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    const T u = (done || drop) ? T(0) : ((row == p) ? dp : S[p * lds + row] - acc);
    T rs, inv;
    recip_sqrt(dp, drop, rs, inv);
    if (sub == 0 && row < ldr) R[j * ldr + row] = u * rs;
    if (tid < ldr - NP) R[j * ldr + NP + tid] = T(0);
    if (!done) d -= u * u * inv;
    if (row == p) done = true;
    if (tid == 0) perm[j] = p;
    partials(j + 1, par ^ 1);
    __syncthreads();
  }
  __syncthreads();
  if (tails)
    for (int q = tid; q <= j; q += FT) tails[q] = base + (double)trace_j[q];
  if (tid == 0) sc.trace = (double)trace_j[j];
  __syncthreads();
  return j;
}

// Column-order Cholesky (no pivoting, stop_mode 0, kmax = n) of the
// symmetric n x n matrix in the register tiles a, blocked right-looking by
// 32 columns in shared S (ld lds, lower triangle overwritten by L):
//   1. warp 0 factors the 32 x 32 diagonal block (one row per lane, __syncwarp
//      between columns); a column whose remaining diagonal is not above
//      tol * (largest initial diagonal) is dropped (zero column of L);
//   2. one thread per row below solves its panel row against that block;
//   3. every thread applies the rank-32 update to 4 x 4 blocks of the
//      trailing lower triangle.
// Three barriers per block of 32 columns.  R = L^T (ld ldr) and perm[j] = j
// as pchol() gives them for this mode; returns n.  rsb: 32 scratch entries.
template <typename T>
__device__ int chol_blocked(const T (&a)[4][8], int n, double tol, T* R, int ldr, int* perm, T* S,
                            int lds, T* rsb, Scal& sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int r = tile_r(i), c = tile_c(jj);
      if (r < n && c < n) S[r * lds + c] = a[i][jj];
    }
  __syncthreads();
  T tol_abs;
  {
    T m = T(0);
    for (int i = lane; i < n; i += 32) m = fmax(m, S[i * lds + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    tol_abs = (T)(tol * (double)m);
  }
  for (int kb = 0; kb < n; kb += 32) {
    const int nb = min(32, n - kb);
    // 1. diagonal block, by warp 0 in shared memory, four columns per step:
    //    every lane factors the 4 x 4 pivot block in registers (the same
    //    drop rule, column by column), the lanes below solve their rows
    //    against it, then each lane applies the rank-4 update to its row.
    if (warp == 0) {
      for (int k0 = 0; k0 < nb; k0 += 4) {
        const int kw = min(4, nb - k0);
        T L4[4][4], rs4[4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            L4[a][b] = (b <= a && a < kw) ? S[(kb + k0 + a) * lds + kb + k0 + b] : T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T dcc = L4[c][c];
#pragma unroll
          for (int t = 0; t < c; ++t) dcc -= L4[c][t] * L4[c][t];
          const bool drop = (c >= kw) || !(dcc > tol_abs);
          T rsc, invc;
          recip_sqrt(dcc, drop, rsc, invc);
          rs4[c] = rsc;
          L4[c][c] = drop ? T(0) : dcc * rsc;
#pragma unroll
          for (int a = c + 1; a < 4; ++a) {
            T v = L4[a][c];
#pragma unroll
            for (int t = 0; t < c; ++t) v -= L4[a][t] * L4[c][t];
            L4[a][c] = v * rsc;
          }
        }
        const int i = lane;
        T x[4] = {T(0), T(0), T(0), T(0)};
        if (i >= k0 + kw && i < nb) {
          T* Si = S + (kb + i) * lds + kb + k0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            T v = (c < kw) ? Si[c] : T(0);
#pragma unroll
            for (int t = 0; t < c; ++t) v -= x[t] * L4[c][t];
            x[c] = v * rs4[c];
          }
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c < kw) Si[c] = x[c];
        } else if (i >= k0 && i < k0 + kw) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c <= i - k0) S[(kb + i) * lds + kb + k0 + c] = L4[i - k0][c];
          rsb[i] = rs4[i - k0];
        }
        __syncwarp();
        if (i >= k0 + kw && i < nb) {
          T* row = S + (kb + i) * lds + kb;
          const T* Lg = S + kb * lds + kb + k0;  // L(kb + j, kb + k0 + t) = Lg[j * lds + t]
          int j = k0 + kw;
          for (; j + 1 <= i; j += 2) {
            const T* l0 = Lg + j * lds;
            const T* l1 = l0 + lds;
            const T r0 = row[j], r1 = row[j + 1];
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              if (t < kw) {
                s0 += x[t] * l0[t];
                s1 += x[t] * l1[t];
              }
            }
            row[j] = r0 - s0;
            row[j + 1] = r1 - s1;
          }
          if (j <= i) {
            const T* l0 = Lg + j * lds;
            T s0 = T(0);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (t < kw) s0 += x[t] * l0[t];
            row[j] -= s0;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // 2. panel rows below the block, one thread per row, in registers:
    //    L(r, kb+c) = (S(r, kb+c) - sum_{c'<c} L(r, kb+c') L(kb+c, kb+c')) / L(kb+c, kb+c)
    const int r0 = kb + nb;
    if (tid < n - r0) {
      const int r = r0 + tid;
      T* Sr = S + r * lds + kb;
      T x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < nb) {
          const T* Lc = S + (kb + c) * lds + kb;
          T acc = Sr[c];
#pragma unroll
          for (int cp = 0; cp < c; ++cp) acc -= x[cp] * Lc[cp];
          x[c] = acc * rsb[c];
        } else {
          x[c] = T(0);
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < nb) Sr[c] = x[c];
    }
    __syncthreads();
    // 3. trailing update of the lower triangle, 4 x 4 blocks per thread
    const int m2 = n - r0;
    if (m2 > 0) {
      const int nt = (m2 + 3) / 4;
      for (int blk = tid; blk < nt * nt; blk += FT) {
        const int bi = blk / nt, bj = blk % nt;
        if (bj > bi) continue;
        T acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
        const int i0 = r0 + 4 * bi, j0 = r0 + 4 * bj;
        for (int c = 0; c < nb; ++c) {
          T li[4], lj[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            li[x] = (i0 + x < n) ? S[(i0 + x) * lds + kb + c] : T(0);
            lj[x] = (j0 + x < n) ? S[(j0 + x) * lds + kb + c] : T(0);
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += li[x] * lj[y];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y)
            if (i0 + x < n && j0 + y <= i0 + x) S[(i0 + x) * lds + j0 + y] -= acc[x][y];
      }
    }
    __syncthreads();
  }
  // R = L^T, zero below the diagonal and beyond n
  for (int e = tid; e < n * ldr; e += FT) {
    const int j = e / ldr, c = e % ldr;
    R[e] = (c < n && c >= j) ? S[c * lds + j] : T(0);
  }
  for (int j = tid; j < n; j += FT) perm[j] = j;
  if (tid == 0) sc.trace = 0.0;
  __syncthreads();
  return n;
}

// X = U^{-1} for the upper-triangular m x m U (ld ld); a row/column with
// U_kk == 0 is treated as dropped (zero in X).  Blocked by 32: one warp per
// diagonal block (a thread per column), then X_IJ = -X_II sum_K U_IK X_KJ by
// block distance.  tmp: (m/32) * 1024 entries.
template <typename T>
__device__ void tri_inverse(const T* U, int m, int ld, T* X, T* tmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (m + 31) / 32;
  for (int e = tid; e < m * ld; e += FT) X[e] = T(0);
  __syncthreads();
  // diagonal blocks: warp w inverts block w; lane c keeps column c of X in
  // registers (back substitution with the block's reciprocal diagonal)
  if (warp < nb) {
    const int b0 = warp * 32, c = lane, mb = min(32, m - b0);
    T* dinv = tmp + warp * 32;  // (the off-diagonal phase rewrites tmp later)
    if (c < mb) {
      const T u = U[(b0 + c) * ld + b0 + c];
      dinv[c] = (u != T(0)) ? T(1) / u : T(0);
    }
    __syncwarp();
    T x[32];
#pragma unroll
    for (int r = 31; r >= 0; --r) {
      if (r > c || r >= mb || c >= mb) {
        x[r] = T(0);
      } else if (r == c) {
        x[r] = dinv[r];
      } else {
        T sacc = T(0);
#pragma unroll
        for (int k = r + 1; k < 32; ++k)
          if (k <= c) sacc += U[(b0 + r) * ld + b0 + k] * x[k];
        x[r] = -sacc * dinv[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (r <= c && c < mb) X[(b0 + r) * ld + b0 + c] = x[r];
  }
  __syncthreads();
  for (int dist = 1; dist < nb; ++dist) {
    const int nblk = nb - dist;
    for (int e = tid; e < nblk * 1024; e += FT) {
      const int bI = e / 1024, w = e % 1024;
      const int i = bI * 32 + w / 32, c = (bI + dist) * 32 + w % 32;
      T s = T(0);
      if (i < m && c < m)
        for (int k = (bI + 1) * 32; k <= c; ++k) s += U[i * ld + k] * X[k * ld + c];
      tmp[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < nblk * 1024; e += FT) {
      const int bI = e / 1024, w = e % 1024;
      const int i = bI * 32 + w / 32, c = (bI + dist) * 32 + w % 32;
      if (i >= m || c >= m) continue;
      T s = T(0);
      for (int k = i; k < (bI + 1) * 32 && k < m; ++k)
        s += X[i * ld + k] * tmp[bI * 1024 + (k - bI * 32) * 32 + w % 32];
      X[i * ld + c] = -s;
    }
    __syncthreads();
  }
}

// out[i][c] = sum_{k <= c} A[i][k] B[k][c] for B upper triangular (n x m).
template <typename T>
__device__ void mul_upper(const T* A, int lda, const T* B, int ldb, int n, int m, T* out,
                          int ldo) {
  for (int e = threadIdx.x; e < n * m; e += FT) {
    const int i = e / m, c = e % m;
    T s = T(0);
    for (int k = 0; k <= c; ++k) s += A[i * lda + k] * B[k * ldb + c];
    out[i * ldo + c] = s;
  }
  __syncthreads();
}

template <typename T, typename ZT>
__global__ void __launch_bounds__(FT, 1) small_fast_kernel(const double* __restrict__ G,
                                                           SmallParams prm, ZT* __restrict__ Z,
                                                           int ldz, StepInfo* __restrict__ info,
                                                           T* __restrict__ gws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = prm.n, tid = threadIdx.x;
  const int nn = ((n + 31) / 32) * 32, ld = nn + 1;
  T* R1 = (T*)smem_raw;            // nn x ld
  T* R2 = R1 + nn * ld;            // nn x ld
  T* X = R2 + nn * ld;             // nn x ld
  T* tmp = X + nn * ld;            // (nn/32) * 1024
  T* dbuf = tmp + (nn / 32) * 1024;  // 2 NP
  T* Lbuf = dbuf + 2 * NP;         // 2 NP
  int* dn = (int*)(Lbuf + 2 * NP); // 2 NP
  int* perm1 = dn + 2 * NP;        // NP
  int* perm2 = perm1 + NP;         // NP
  __shared__ Scal sc;
  __shared__ double redd[32];
  T a[4][8];

  double tr = 0.0;
  for (int i = tid; i < n; i += FT) tr += G[i * n + i];
  tr = block_sum(tr, redd);
  const double x2 = prm.x2_dev ? *prm.x2_dev : tr;
  double normA2 = -1.0, delta2 = prm.delta2;
  if (prm.normA2_dev) {
    normA2 = prm.normA2_is_trace ? tr : *prm.normA2_dev;
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
    load_regs(a, G, n);
    if (prm.shift_rel > 0.0) {
      const T sh = (T)(prm.shift_rel * tr);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (tile_r(i) == tile_c(jj) && tile_r(i) < n) a[i][jj] += sh;
    }
    chol_blocked(a, n, prm.piv_tol, R1, ld, perm1, X, ld, dbuf, sc);
    tri_inverse(R1, n, ld, X, tmp);
    for (int e = tid; e < n * ldz; e += FT) {
      const int i = e / ldz, c = e % ldz;
      Z[e] = (c < n) ? (ZT)X[i * ld + c] : ZT(0);
    }
    if (tid == 0) {
      int kept = 0;
      for (int i = 0; i < n; ++i) kept += (R1[i * ld + i] != T(0));
      info->r = kept;
      info->k1 = kept;
      info->nsteps = n;
      info->mu2 = 0.0;
      info->s1 = 0.0;
      info->tail = 0.0;
    }
    return;
  }

  // ---- SM_QLP ----------------------------------------------------------
  T* Tw = gws;  // whitening factor T^{-1} (global scratch, nn x ld)
  if (prm.Gw) {
    // W^T W = T^T T; factor A = T^{-T} G T^{-1}, the Gram of X Q for Q = W T^{-1}
    load_regs(a, prm.Gw, n);
    chol_blocked(a, n, 0.0, R1, ld, perm1, X, ld, dbuf, sc);
    tri_inverse(R1, n, ld, X, tmp);
    for (int e = tid; e < nn * ld; e += FT) Tw[e] = X[e];
    for (int e = tid; e < n * n; e += FT) R2[(e / n) * ld + e % n] = (T)G[e];
    __syncthreads();
    // G T^{-1} (T^{-1} upper triangular), back into R2
    tile_product(a, n, n, n, [&](int r, int k) { return R2[r * ld + k]; },
                 [&](int c, int k) { return k <= c ? X[k * ld + c] : T(0); });
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (tile_r(i) < n && tile_c(jj) < n) R2[tile_r(i) * ld + tile_c(jj)] = a[i][jj];
    __syncthreads();
    // a = T^{-T} (G T^{-1})
    tile_product(a, n, n, n, [&](int r, int k) { return k <= r ? X[k * ld + r] : T(0); },
                 [&](int c, int k) { return R2[k * ld + c]; });
    double t2 = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (tile_r(i) == tile_c(jj)) t2 += (double)a[i][jj];
    tr = block_sum(t2, redd);
  } else {
    load_regs(a, G, n);
  }
  const double mu2 = prm.x2_dev ? fmax(0.0, x2 - tr) : 0.0;

  // phase 1: pivoted Cholesky of G
  const int k1 = pchol(a, n, true, prm.piv_tol, 0, 0.0, 0.0, 0, n, R1, ld, perm1, X, ld, dbuf, dn, Lbuf,
                       nullptr, sc);
  const double s1 = sc.trace;
  // phase 2: pivoted Cholesky of M = R_1 R_1^T
  tile_product(a, k1, k1, n, [&](int r, int q) { return R1[r * ld + q]; },
               [&](int c, int q) { return R1[c * ld + q]; });
  const bool fixed = prm.r_fixed >= 1;
  const int rt = fixed ? min(prm.r_fixed, prm.r_cap) : -1;
  const int r2 = pchol(a, k1, true, 0.0, fixed ? 2 : 1, mu2 + s1, delta2, rt, min(k1, prm.r_cap),
                       R2, ld, perm2, X, ld, dbuf, dn, Lbuf, info->tails, sc);
  const int r = fixed ? rt : max(1, r2);
  const int rz = min(r, r2);  // columns produced by the factorization

  // R2_11[a][b] = R2[a][perm2[b]] (b >= a), compacted into R2
  for (int e = tid; e < rz * rz; e += FT) {
    const int aa = e / rz, b = e % rz;
    X[aa * ld + b] = (b >= aa) ? R2[aa * ld + perm2[b]] : T(0);
  }
  __syncthreads();
  for (int e = tid; e < rz * rz; e += FT) R2[(e / rz) * ld + e % rz] = X[(e / rz) * ld + e % rz];
  __syncthreads();
  tri_inverse(R2, rz, ld, X, tmp);
  // Zs = R_1^T(:, perm2) R2_11^{-1} (n x rz), into R2
  tile_product(a, n, rz, rz, [&](int i, int q) { return R1[perm2[q] * ld + i]; },
               [&](int c, int q) { return q <= c ? X[q * ld + c] : T(0); });
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (tile_r(i) < n && tile_c(jj) < rz) R2[tile_r(i) * ld + tile_c(jj)] = a[i][jj];
  __syncthreads();
  if (sizeof(T) == 4 && rz > 0) {
    // one more Cholesky-QR pass: Zs <- Zs chol(Zs^T Zs)^{-1}
    tile_product(a, rz, rz, n, [&](int rr, int q) { return R2[q * ld + rr]; },
                 [&](int c, int q) { return R2[q * ld + c]; });
    chol_blocked(a, rz, 0.0, R1, ld, perm1, X, ld, dbuf, sc);
    tri_inverse(R1, rz, ld, X, tmp);
    tile_product(a, n, rz, rz, [&](int i, int q) { return R2[i * ld + q]; },
                 [&](int c, int q) { return q <= c ? X[q * ld + c] : T(0); });
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (tile_r(i) < n && tile_c(jj) < rz) R2[tile_r(i) * ld + tile_c(jj)] = a[i][jj];
    __syncthreads();
  }
  // fixed rank above the numerical rank: complete with unit vectors
  // orthogonalized (twice) against the columns already formed
  if (r > rz && tid < 32) {
    const int lane = tid;
    T* v = Lbuf;
    int cand = 0;
    for (int c = rz; c < r; ++c) {
      for (; cand < n; ++cand) {
        for (int i = lane; i < n; i += 32) v[i] = (i == cand) ? T(1) : T(0);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int b = 0; b < c; ++b) {
            T dot = T(0);
            for (int i = lane; i < n; i += 32) dot += R2[i * ld + b] * v[i];
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            for (int i = lane; i < n; i += 32) v[i] -= dot * R2[i * ld + b];
            __syncwarp();
          }
        }
        T nv = T(0);
        for (int i = lane; i < n; i += 32) nv += v[i] * v[i];
        for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
        if (nv > T(0.25)) {
          const T s = T(1) / sqrt(nv);
          for (int i = lane; i < n; i += 32) R2[i * ld + c] = v[i] * s;
          __syncwarp();
          ++cand;
          break;
        }
      }
    }
  }
  __syncthreads();
  // output (whitened: Z_1 = T^{-1} Zs, T^{-1} brought back into X)
  if (prm.Gw) {
    for (int e = tid; e < nn * ld; e += FT) X[e] = Tw[e];
    __syncthreads();
    tile_product(a, n, r, n, [&](int i, int k) { return k >= i ? X[i * ld + k] : T(0); },
                 [&](int c, int k) { return R2[k * ld + c]; });
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (tile_r(i) < n && tile_c(jj) < r) Z[(size_t)tile_r(i) * ldz + tile_c(jj)] = (ZT)a[i][jj];
  } else {
    for (int e = tid; e < n * r; e += FT) {
      const int i = e / r, c = e % r;
      Z[(size_t)i * ldz + c] = (ZT)R2[i * ld + c];
    }
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
  const int nn = ((n + 31) / 32) * 32, ld = nn + 1;
  return (size_t)(3 * nn * ld + (nn / 32) * 1024 + 4 * NP) * sizeof(T) + 4 * NP * sizeof(int);
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
  const int lim = fp64 ? 64 : 128;
  return prm.n >= 1 && prm.n <= lim;
}

cudaError_t small_factor_fast(const double* G, SmallParams prm, bool fp64_math, void* Z,
                              bool z_fp64, int ldz, void* ws, StepInfo* info, cudaStream_t st) {
  if (fp64_math)
    return z_fp64 ? launch_fast<double, double>(G, prm, Z, ldz, ws, info, st)
                  : launch_fast<double, float>(G, prm, Z, ldz, ws, info, st);
  return z_fp64 ? launch_fast<float, double>(G, prm, Z, ldz, ws, info, st)
                : launch_fast<float, float>(G, prm, Z, ldz, ws, info, st);
}

}  // namespace ttk
