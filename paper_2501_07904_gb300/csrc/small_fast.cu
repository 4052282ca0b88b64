// Register-resident single-CTA small factorizations: the fast path of
// small_factor() for the sweep's pivoted QLP (SM_QLP) and shifted
// Cholesky-QR (SM_ORTH), for n <= 128 in FP32 and n <= 64 in FP64.
//
// The symmetric n x n matrix is held in registers, a 4 x 8 tile per thread
// (512 threads cover 128 x 128).  One Cholesky step is: one warp picks the
// pivot p (largest remaining diagonal, lowest index on ties), the owners of
// row p publish it to shared memory, every thread applies the rank-one update
// to its own entries -- two barriers per step.  Pivoting is virtual (nothing
// is swapped): the factor's rows come out in pivot order and its columns keep
// the original coordinates.
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
  int p, stop, drop;
  double dp, trace;
};

template <typename T>
__device__ __forceinline__ T sel4(const T (&a)[4][8], int i, int jj) {
  return i == 0 ? a[0][jj] : (i == 1 ? a[1][jj] : (i == 2 ? a[2][jj] : a[3][jj]));
}

template <typename T>
__device__ void load_regs(T (&a)[4][8], const double* G, int n) {
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int r = 4 * ty + i, c = 8 * tx + jj;
      a[i][jj] = (r < n && c < n) ? (T)G[r * n + c] : T(0);
    }
}

// Cholesky of the symmetric matrix in registers (see file comment).
//   pivot      largest remaining diagonal first; else column order, a column
//              whose remaining diagonal is not above tol * (largest initial
//              diagonal) being dropped (zero row of R);
//   stop_mode  0: tolerance (pivoted) or all columns (column order);
//              1: first j >= 1 with base + trace <= delta2;
//              2: j == r_stop;
//   kmax       at most this many steps.
// Rows of R (ld ldr) in step order, perm[j] = column eliminated at step j;
// tails[j] = base + remaining trace before step j (if tails != null).
// Returns the number of steps; sc.trace = remaining Schur trace (>= 0, FP64).
template <typename T>
__device__ int pchol(T (&a)[4][8], int n, bool pivot, double tol, int stop_mode, double base,
                     double delta2, int r_stop, int kmax, T* R, int ldr, int* perm, T* d, T* Lraw,
                     int* done, double* tails, Scal& sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid / 16, tx = tid % 16;
  for (int i = tid; i < NP; i += FT) done[i] = (i >= n) ? 1 : 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (4 * ty + i == 8 * tx + jj) d[4 * ty + i] = a[i][jj];
  __syncthreads();
  double d0 = 0.0;
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m = fmax(m, (double)d[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    d0 = m;
  }
  int j = 0;
  for (;; ++j) {
    if (warp == 0) {
      double tr = 0.0;
      T best = lowest_value<T>();
      int bi = 0x7fffffff;
      for (int i = lane; i < NP; i += 32) {
        if (done[i]) continue;
        tr += (double)d[i];
        if (d[i] > best || (d[i] == best && i < bi)) {
          best = d[i];
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        tr = fmax(tr, 0.0);
        if (tails) tails[j] = base + tr;
        int stop = 0, drop = 0, p = bi;
        double dp = (double)best;
        if (!pivot) {
          p = j;
          dp = (j < n) ? (double)d[j] : 0.0;
        }
        if (j >= kmax) stop = 1;
        if (!stop && stop_mode == 1 && j >= 1 && base + tr <= delta2) stop = 1;
        if (!stop && stop_mode == 2 && j == r_stop) stop = 1;
        if (!stop) {
          const bool ok = (dp > 0.0) && (dp > tol * d0);
          if (pivot && !ok) stop = 1;
          if (!pivot && !ok) drop = 1;
        }
        sc.p = p;
        sc.dp = dp;
        sc.stop = stop;
        sc.drop = drop;
        sc.trace = tr;
      }
    }
    __syncthreads();
    if (sc.stop) break;
    const int p = sc.p;
    if (sc.drop) {
      for (int c = tid; c < ldr; c += FT) R[j * ldr + c] = T(0);
      if (tid == 0) {
        done[p] = 1;
        perm[j] = p;
      }
      continue;
    }
    if (ty == p / 4) {
      const int pi = p % 4;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int c = 8 * tx + jj;
        Lraw[c] = done[c] ? T(0) : sel4(a, pi, jj);
      }
    }
    __syncthreads();
    const T dp = (T)sc.dp;
    const T inv = T(1) / dp;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T lr = Lraw[4 * ty + i] * inv;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) a[i][jj] -= lr * Lraw[8 * tx + jj];
    }
    if (warp == 0) {
      const T s = sqrt(dp);
      for (int c = lane; c < ldr; c += 32) {
        const T l = (c < NP) ? Lraw[c] : T(0);
        R[j * ldr + c] = l / s;
        if (c < NP && !done[c]) d[c] -= l * l * inv;
      }
      __syncwarp();
      if (lane == 0) {
        done[p] = 1;
        perm[j] = p;
        d[p] = T(0);
      }
    }
  }
  __syncthreads();
  return j;
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
  if (warp < nb) {
    const int b0 = warp * 32, c = b0 + lane;
    if (c < m && U[c * ld + c] != T(0)) {
      X[c * ld + c] = T(1) / U[c * ld + c];
      for (int i = c - 1; i >= b0; --i) {
        if (U[i * ld + i] == T(0)) continue;
        T s = T(0);
        for (int k = i + 1; k <= c; ++k) s += U[i * ld + k] * X[k * ld + c];
        X[i * ld + c] = -s / U[i * ld + i];
      }
    }
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
  const int ty = tid / 16, tx = tid % 16;
  const int nn = ((n + 31) / 32) * 32, ld = nn + 1;
  T* R1 = (T*)smem_raw;            // nn x ld
  T* R2 = R1 + nn * ld;            // nn x ld
  T* X = R2 + nn * ld;             // nn x ld
  T* tmp = X + nn * ld;            // (nn/32) * 1024
  T* d = tmp + (nn / 32) * 1024;   // NP
  T* Lraw = d + NP;                // NP
  int* done = (int*)(Lraw + NP);   // NP
  int* perm1 = done + NP;          // NP
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
          if (4 * ty + i == 8 * tx + jj && 4 * ty + i < n) a[i][jj] += sh;
    }
    pchol(a, n, false, prm.piv_tol, 0, 0.0, 0.0, 0, n, R1, ld, perm1, d, Lraw, done, nullptr, sc);
    tri_inverse(R1, n, ld, X, tmp);
    int kept = 0;
    if (tid == 0)
      for (int i = 0; i < n; ++i) kept += (R1[i * ld + i] != T(0));
    for (int e = tid; e < n * ldz; e += FT) {
      const int i = e / ldz, c = e % ldz;
      Z[e] = (c < n) ? (ZT)X[i * ld + c] : ZT(0);
    }
    if (tid == 0) {
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
    pchol(a, n, false, 0.0, 0, 0.0, 0.0, 0, n, R1, ld, perm1, d, Lraw, done, nullptr, sc);
    tri_inverse(R1, n, ld, X, tmp);
    for (int e = tid; e < nn * ld; e += FT) Tw[e] = X[e];
    for (int e = tid; e < n * n; e += FT) {  // R2 = G T^{-1}
      const int i = e / n, c = e % n;
      double s = 0.0;
      for (int k = 0; k <= c; ++k) s += G[i * n + k] * (double)X[k * ld + c];
      R2[i * ld + c] = (T)s;
    }
    __syncthreads();
    double t2 = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int r = 4 * ty + i, c = 8 * tx + jj;
        T s = T(0);
        if (r < n && c < n)
          for (int k = 0; k <= r; ++k) s += X[k * ld + r] * R2[k * ld + c];
        a[i][jj] = s;
        if (r == c) t2 += (double)s;
      }
    tr = block_sum(t2, redd);
  } else {
    load_regs(a, G, n);
  }
  const double mu2 = prm.x2_dev ? fmax(0.0, x2 - tr) : 0.0;

  // phase 1: pivoted Cholesky of G
  const int k1 = pchol(a, n, true, prm.piv_tol, 0, 0.0, 0.0, 0, n, R1, ld, perm1, d, Lraw, done,
                       nullptr, sc);
  const double s1 = sc.trace;
  // phase 2: pivoted Cholesky of M = R_1 R_1^T
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int r = 4 * ty + i, c = 8 * tx + jj;
      T s = T(0);
      if (r < k1 && c < k1)
        for (int q = 0; q < n; ++q) s += R1[r * ld + q] * R1[c * ld + q];
      a[i][jj] = s;
    }
  const bool fixed = prm.r_fixed >= 1;
  const int rt = fixed ? min(prm.r_fixed, prm.r_cap) : -1;
  const int r2 = pchol(a, k1, true, 0.0, fixed ? 2 : 1, mu2 + s1, delta2, rt, min(k1, prm.r_cap),
                       R2, ld, perm2, d, Lraw, done, info->tails, sc);
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
  // Zs = R_1^T(:, perm2) R2_11^{-1}  (n x rz) into R2
  for (int e = tid; e < n * rz; e += FT) {
    const int i = e / rz, c = e % rz;
    T s = T(0);
    for (int aa = 0; aa <= c; ++aa) s += R1[perm2[aa] * ld + i] * X[aa * ld + c];
    R2[i * ld + c] = s;
  }
  __syncthreads();
  if (sizeof(T) == 4 && rz > 0) {
    // one more Cholesky-QR pass: Zs <- Zs chol(Zs^T Zs)^{-1}
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int rr = 4 * ty + i, c = 8 * tx + jj;
        T s = T(0);
        if (rr < rz && c < rz)
          for (int q = 0; q < n; ++q) s += R2[q * ld + rr] * R2[q * ld + c];
        a[i][jj] = s;
      }
    pchol(a, rz, false, 0.0, 0, 0.0, 0.0, 0, rz, R1, ld, perm1, d, Lraw, done, nullptr, sc);
    tri_inverse(R1, rz, ld, X, tmp);
    mul_upper(R2, ld, X, ld, n, rz, R1, ld);  // R1 = Zs X
    for (int e = tid; e < n * rz; e += FT) R2[(e / rz) * ld + e % rz] = R1[(e / rz) * ld + e % rz];
    __syncthreads();
  }
  // fixed rank above the numerical rank: complete with unit vectors
  // orthogonalized (twice) against the columns already formed
  if (r > rz && tid < 32) {
    const int lane = tid;
    int cand = 0;
    for (int c = rz; c < r; ++c) {
      for (; cand < n; ++cand) {
        // v = e_cand - Z Z^T e_cand, twice
        for (int i = lane; i < n; i += 32) Lraw[i] = (i == cand) ? T(1) : T(0);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int b = 0; b < c; ++b) {
            T dot = T(0);
            for (int i = lane; i < n; i += 32) dot += R2[i * ld + b] * Lraw[i];
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            for (int i = lane; i < n; i += 32) Lraw[i] -= dot * R2[i * ld + b];
            __syncwarp();
          }
        }
        T nv = T(0);
        for (int i = lane; i < n; i += 32) nv += Lraw[i] * Lraw[i];
        for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
        if (nv > T(0.25)) {
          const T s = T(1) / sqrt(nv);
          for (int i = lane; i < n; i += 32) R2[i * ld + c] = Lraw[i] * s;
          __syncwarp();
          ++cand;
          break;
        }
      }
    }
  }
  __syncthreads();
  // output (whitened: Z_1 = T^{-1} Zs)
  for (int e = tid; e < n * r; e += FT) {
    const int i = e / r, c = e % r;
    T z;
    if (prm.Gw) {
      z = T(0);
      for (int k = i; k < n; ++k) z += Tw[i * ld + k] * R2[k * ld + c];
    } else {
      z = R2[i * ld + c];
    }
    Z[(size_t)i * ldz + c] = (ZT)z;
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
  return (size_t)(3 * nn * ld + (nn / 32) * 1024 + 2 * NP) * sizeof(T) + 3 * NP * sizeof(int);
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
