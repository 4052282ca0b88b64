// Single-CTA factorizations of the small (n <= 256) Gram matrix of each
// sweep step, in FP32 or FP64.
//
//  SM_QLP     rank-revealing UTV of the factored matrix X through its Gram
//             G = X^T X: pivoted Cholesky (= the R factor of column-pivoted
//             QR of X, the rank-revealing QR the paper lists as a UTV, Sec. 2.2),
//             then Stewart's pivoted QLP step -- column-pivoted Householder QR
//             of R_1^T, L = R_2^T, Z = Pi_1 Q_2 -- with the truncation error
//             of rank j read off as the trailing Frobenius norm after j
//             Householder steps (= sum_{i>j} ||L(:,i)||^2, the ||[R12;R22]||
//             of Eq. urv / ||[L21 L22]|| of Eq. ulv).  The rank is the smallest
//             j >= 1 with error <= delta^2 (Alg. 2, step 5), or fixed.
//  SM_JACOBI  TT-SVD: cyclic Jacobi eigen-decomposition of G; the error of
//             rank j is the sum of the dropped eigenvalues.
//  SM_ORTH    one pass of (shifted) Cholesky-QR of a sketch Y from
//             G = Y^T Y: R = chol(G + shift I) in column order, S = R^{-1},
//             so that Y S spans Y[:, :j] for every j -- the basis Householder
//             QR of Y gives, up to signs.  With a shift of a few n u ||G||
//             the factorization cannot break down; two further unshifted
//             passes make the columns orthonormal to working precision
//             (shifted Cholesky-QR3).  A column with no positive pivot even
//             then (an exactly dependent column) is dropped: zero in S.
//  SM_USVP    USV-plus-style deflation (the inner factor the paper runs in
//             TT-ULV, Sec. 4): basis vectors one at a time, each from the
//             column of largest norm of the deflated matrix D = X (I - V V^T)
//             followed by q power iterations v <- D^T D v / ||.||, then
//             re-orthogonalized twice against V.  D^T D is kept explicitly
//             (the Gram, deflated after each vector by a rank-two update), so
//             the error of rank i is mu^2 + trace(D^T D).  Stops at the
//             fixed rank, or at the first i >= 1 with error <= delta^2.
//  SM_LURV    low-rank revealing URV with Givens rotations (the Fierro-Hansen
//             family the paper runs inside TT-URV in Sec. 4), warm-started
//             from the pivoted QR X Pi = Q R (the pivoted Cholesky of G), V =
//             Pi.  Vector i: the dominant right singular vector v of the
//             trailing block R(i:, i:) is estimated (start from the block's
//             column of largest norm, then q power iterations), rotated onto
//             e_i by column Givens rotations (pairs (c, c+1), c from n-2 down
//             to i, on R and V), and the subdiagonal fill each leaves is
//             chased away by a row rotation of the same pair; the error of
//             keeping i+1 vectors is mu^2 + s1 + ||R(:, i+1:)||_F^2.
#include <math.h>

#include "internal.h"

namespace ttk {
namespace {

constexpr int NT = 512;

template <typename T>
__device__ __forceinline__ void swap_vals(T& a, T& b) {
  T t = a;
  a = b;
  b = t;
}

// Block-cooperative pivoted Cholesky of the symmetric n x n matrix A (full
// storage, row-major, leading dimension lda >= n; 0 means n).  Pivot = largest remaining diagonal (lowest index on
// ties); stops when it is not above tol_rel * (largest initial diagonal).
// On return rows 0..k1-1 of A hold R_1 (upper trapezoidal, columns in pivot
// order), everything else is zero; perm[i] = original index of position i;
// rem = remaining Schur-complement diagonal (clamped at 0), in FP64.
template <typename T>
__device__ int pivoted_cholesky(T* A, int n, int* perm, double tol_rel, double& rem, T* redt,
                                int* redi, double* redd, int lda = 0) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (lda < n) lda = n;
  for (int i = tid; i < n; i += nt) perm[i] = i;
  T v = lowest_value<T>();
  int idx = 0x7fffffff;
  for (int i = tid; i < n; i += nt) {
    const T a = A[i * lda + i];
    if (a > v) {
      v = a;
      idx = i;
    }
  }
  T d0;
  int i0;
  block_argmax(v, idx, redt, redi, d0, i0);
  (void)i0;
  int j = 0;
  for (; j < n; ++j) {
    v = lowest_value<T>();
    idx = 0x7fffffff;
    for (int i = j + tid; i < n; i += nt) {
      const T a = A[i * lda + i];
      if (a > v) {
        v = a;
        idx = i;
      }
    }
    T dp;
    int p;
    block_argmax(v, idx, redt, redi, dp, p);
    if (!(dp > T(0)) || !((double)dp > tol_rel * (double)d0)) break;
    if (p != j) {
      for (int c = tid; c < n; c += nt) swap_vals(A[j * lda + c], A[p * lda + c]);
      __syncthreads();
      for (int r = tid; r < n; r += nt) swap_vals(A[r * lda + j], A[r * lda + p]);
      if (tid == 0) swap_vals(perm[j], perm[p]);
      __syncthreads();
    }
    const T rjj = sqrt(A[j * lda + j]);
    __syncthreads();
    for (int c = j + tid; c < n; c += nt) A[j * lda + c] = (c == j) ? rjj : A[j * lda + c] / rjj;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int r = j + 1 + e / m, c = j + 1 + e % m;
      A[r * lda + c] -= A[j * lda + r] * A[j * lda + c];
    }
    __syncthreads();
  }
  const int k1 = j;
  double s = 0.0;
  for (int i = k1 + tid; i < n; i += nt) {
    const double a = (double)A[i * lda + i];
    s += a > 0.0 ? a : 0.0;
  }
  rem = block_sum(s, redd);
  for (int e = tid; e < n * n; e += nt) {
    const int r = e / n, c = e % n;
    if (r >= k1 || c < r) A[r * lda + c] = T(0);
  }
  __syncthreads();
  return k1;
}

// Cholesky of the symmetric n x n matrix A in column order (no pivoting),
// skipping every column whose remaining diagonal is not above
// tol_rel * (largest initial diagonal).  Kept rows of A then hold R (upper);
// keep[j] marks the kept columns.  Returns the number kept.
template <typename T>
__device__ int cholesky_drop(T* A, int n, int* keep, double tol_rel, T* redt, int* redi) {
  const int tid = threadIdx.x, nt = blockDim.x;
  T v = lowest_value<T>();
  int idx = 0x7fffffff;
  for (int i = tid; i < n; i += nt) {
    const T a = A[i * n + i];
    if (a > v) {
      v = a;
      idx = i;
    }
  }
  T d0;
  int i0;
  block_argmax(v, idx, redt, redi, d0, i0);
  (void)i0;
  int kept = 0;
  for (int j = 0; j < n; ++j) {
    const T djj = A[j * n + j];
    const bool k = (djj > T(0)) && ((double)djj > tol_rel * (double)d0);
    __syncthreads();
    if (!k) {
      for (int c = j + tid; c < n; c += nt) A[j * n + c] = T(0);
      if (tid == 0) keep[j] = 0;
      __syncthreads();
      continue;
    }
    ++kept;
    const T rjj = sqrt(djj);
    for (int c = j + tid; c < n; c += nt) A[j * n + c] = (c == j) ? rjj : A[j * n + c] / rjj;
    if (tid == 0) keep[j] = 1;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int r = j + 1 + e / m, c = j + 1 + e % m;
      A[r * n + c] -= A[j * n + r] * A[j * n + c];
    }
    __syncthreads();
  }
  return kept;
}

template <typename T, typename ZT>
__global__ void __launch_bounds__(NT, 1) small_kernel(const double* __restrict__ G, SmallParams prm,
                                                   T* __restrict__ work, int* __restrict__ iwork,
                                                   ZT* __restrict__ Z, int ldz,
                                                   StepInfo* __restrict__ info) {
  __shared__ T redt[32];
  __shared__ int redi[32];
  __shared__ double redd[32];
  __shared__ T rc[kMaxSmall / 2], rs[kMaxSmall / 2];
  __shared__ int rp[kMaxSmall / 2], rq[kMaxSmall / 2];
  __shared__ int order[kMaxSmall];

  const int n = prm.n, tid = threadIdx.x, nt = blockDim.x;
  T* A = work;
  T* Mq = work + (size_t)n * n;
  T* Qe = work + (size_t)2 * n * n;
  T* cn = work + (size_t)3 * n * n;
  T* tau = cn + n;
  T* Ti = tau + n;                 // n x n: T^{-1} of the whitening (prm.Gw)
  int* perm1 = iwork;

  double tr = 0.0;
  if (prm.Gw) {
    // Whitening: G_W = W^T W = T^T T (Cholesky, column order); factor
    // T^{-T} G T^{-1}, the Gram of X Q for the orthonormal Q = W T^{-1}.
    for (int e = tid; e < n * n; e += nt) Mq[e] = (T)prm.Gw[e];
    __syncthreads();
    const int kw = cholesky_drop(Mq, n, iwork + n, 0.0, redt, redi);
    (void)kw;
    for (int c = tid; c < n; c += nt) {
      for (int i = c + 1; i < n; ++i) Ti[i * n + c] = T(0);
      if (!iwork[n + c]) {
        for (int i = 0; i <= c; ++i) Ti[i * n + c] = T(0);
        continue;
      }
      Ti[c * n + c] = T(1) / Mq[c * n + c];
      for (int i = c - 1; i >= 0; --i) {
        T acc = T(0);
        if (iwork[n + i])
          for (int k = i + 1; k <= c; ++k) acc += Mq[i * n + k] * Ti[k * n + c];
        Ti[i * n + c] = iwork[n + i] ? -acc / Mq[i * n + i] : T(0);
      }
    }
    __syncthreads();
    // Qe = G T^{-1}, then A = T^{-T} Qe
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, c = e % n;
      T acc = T(0);
      for (int k = 0; k <= c; ++k) acc += (T)G[i * n + k] * Ti[k * n + c];
      Qe[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, c = e % n;
      T acc = T(0);
      for (int k = 0; k <= i; ++k) acc += Ti[k * n + i] * Qe[k * n + c];
      A[e] = acc;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) tr += (double)A[i * n + i];
  } else {
    for (int e = tid; e < n * n; e += nt) A[e] = (T)G[e];
    for (int i = tid; i < n; i += nt) tr += G[i * n + i];
  }
  tr = block_sum(tr, redd);
  const double x2 = prm.x2_dev ? *prm.x2_dev : tr;
  double normA2 = -1.0, delta2 = prm.delta2;
  if (prm.normA2_dev) {
    normA2 = prm.normA2_is_trace ? tr : *prm.normA2_dev;
    delta2 = prm.delta2_scale * normA2;
  }
  // range miss mu^2 = ||X||^2 - ||X P_W||^2; zero by construction when W
  // spans the whole row space (Omega = I), where the difference is rounding
  const double mu2 = (prm.x2_dev && !prm.range_exact) ? fmax(0.0, x2 - tr) : 0.0;
  const bool finite = isfinite(tr) && isfinite(x2) && (normA2 < 0.0 || isfinite(normA2));
  if (tid == 0) {
    info->x2 = x2;
    info->trace = tr;
    info->mu2 = mu2;
    info->delta2 = delta2;
    info->normA2 = normA2;
    info->status = finite ? 0 : 1;
  }
  __syncthreads();
  if (!finite) {
    for (int e = tid; e < n * ldz; e += nt) Z[e] = ZT(0);
    if (tid == 0) {
      info->r = 1;
      info->k1 = 0;
      info->nsteps = 0;
      info->s1 = 0.0;
      info->tail = 0.0;
    }
    return;
  }

  if (prm.mode == SM_ORTH) {
    int* keep = iwork;
    if (prm.shift_rel > 0.0) {
      const T sh = (T)(prm.shift_rel * tr);
      for (int i = tid; i < n; i += nt) A[i * n + i] += sh;
      __syncthreads();
    }
    const int kept = cholesky_drop(A, n, keep, prm.piv_tol, redt, redi);
    // Qe = R^{-1} on the kept columns, one column per thread (back substitution).
    for (int c = tid; c < n; c += nt) {
      if (!keep[c]) {
        for (int i = 0; i < n; ++i) Qe[i * n + c] = T(0);
        continue;
      }
      for (int i = c + 1; i < n; ++i) Qe[i * n + c] = T(0);
      Qe[c * n + c] = T(1) / A[c * n + c];
      for (int i = c - 1; i >= 0; --i) {
        if (!keep[i]) {
          Qe[i * n + c] = T(0);
          continue;
        }
        T s = T(0);
        for (int k = i + 1; k <= c; ++k)
          if (keep[k]) s += A[i * n + k] * Qe[k * n + c];
        Qe[i * n + c] = -s / A[i * n + i];
      }
    }
    __syncthreads();
    for (int e = tid; e < n * ldz; e += nt) {
      const int j = e / ldz, c = e % ldz;
      Z[(size_t)j * ldz + c] = (c < n) ? (ZT)Qe[j * n + c] : ZT(0);
    }
    if (tid == 0) {
      info->r = kept;
      info->k1 = kept;
      info->nsteps = n;
      info->s1 = 0.0;
      info->tail = 0.0;
    }
    return;
  }

  const bool fixed = prm.r_fixed >= 1;
  const int rt = fixed ? min(prm.r_fixed, prm.r_cap) : -1;

  if (prm.mode == SM_JACOBI) {
    T* V = Mq;
    for (int e = tid; e < n * n; e += nt) V[e] = (e / n == e % n) ? T(1) : T(0);
    const int nn = n + (n & 1);
    const int npairs = nn / 2;
    const double eps_t = sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920929e-07;
    int sweep = 0;
    bool conv = false;
    const int max_sweeps = prm.jacobi_sweeps > 0 ? prm.jacobi_sweeps : 60;
    for (; sweep < max_sweeps; ++sweep) {
      double off = 0.0, dg = 0.0;
      for (int e = tid; e < n * n; e += nt) {
        const double a = (double)A[e];
        if (e / n == e % n)
          dg += a * a;
        else
          off += a * a;
      }
      off = block_sum(off, redd);
      dg = block_sum(dg, redd);
      if (off <= (double)n * n * eps_t * eps_t * dg) {
        conv = true;
        break;
      }
      for (int t = 0; t < nn - 1; ++t) {
        for (int i = tid; i < npairs; i += nt) {
          const int x = (i == 0) ? 0 : 1 + ((i - 1 + t) % (nn - 1));
          const int y = 1 + ((nn - 2 - i + t) % (nn - 1));
          const int p = min(x, y), q = max(x, y);
          T c = T(1), s = T(0);
          if (q < n) {
            const T apq = A[p * n + q];
            if (apq != T(0)) {
              const T tt = (A[q * n + q] - A[p * n + p]) / (T(2) * apq);
              const T sg = tt >= T(0) ? T(1) : T(-1);
              const T t1 = sg / (fabs(tt) + sqrt(T(1) + tt * tt));
              c = T(1) / sqrt(T(1) + t1 * t1);
              s = t1 * c;
            }
          }
          rc[i] = c;
          rs[i] = s;
          rp[i] = p;
          rq[i] = q < n ? q : -1;
        }
        __syncthreads();
        for (int e = tid; e < npairs * n; e += nt) {
          const int i = e / n, k = e % n;
          const int p = rp[i], q = rq[i];
          if (q < 0 || rs[i] == T(0)) continue;
          const T c = rc[i], s = rs[i];
          const T ap = A[p * n + k], aq = A[q * n + k];
          A[p * n + k] = c * ap - s * aq;
          A[q * n + k] = s * ap + c * aq;
        }
        __syncthreads();
        // columns p, q of every row k: consecutive threads take the pairs of
        // one row, so a warp's loads fall in that row's few cache lines
        for (int e = tid; e < npairs * n; e += nt) {
          const int k = e / npairs, i = e % npairs;
          const int p = rp[i], q = rq[i];
          if (q < 0 || rs[i] == T(0)) continue;
          const T c = rc[i], s = rs[i];
          const T ap = A[k * n + p], aq = A[k * n + q];
          A[k * n + p] = c * ap - s * aq;
          A[k * n + q] = s * ap + c * aq;
          const T vp = V[k * n + p], vq = V[k * n + q];
          V[k * n + p] = c * vp - s * vq;
          V[k * n + q] = s * vp + c * vq;
        }
        __syncthreads();
      }
    }
    // order eigenvalues descending (stable: lower index first on ties)
    for (int i = tid; i < n; i += nt) {
      const T li = A[i * n + i];
      int rank = 0;
      for (int k = 0; k < n; ++k) {
        const T lk = A[k * n + k];
        if (lk > li || (lk == li && k < i)) ++rank;
      }
      order[rank] = i;
    }
    __syncthreads();
    if (tid == 0) {
      double acc = mu2;
      info->tails[n] = acc;
      for (int k = n - 1; k >= 0; --k) {
        const double l = (double)A[order[k] * n + order[k]];
        acc += l > 0.0 ? l : 0.0;
        info->tails[k] = acc;
      }
      int r;
      if (fixed) {
        r = rt;
      } else {
        r = prm.r_cap;
        for (int k = 1; k <= prm.r_cap; ++k)
          if (info->tails[k] <= delta2) {
            r = k;
            break;
          }
      }
      info->r = r;
      info->k1 = n;
      info->nsteps = sweep;
      info->s1 = 0.0;
      info->tail = info->tails[r];
      if (!conv) info->status |= 2;
    }
    __syncthreads();
    const int r = info->r;
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, c = e % r;
      T z;
      if (prm.Gw) {
        z = T(0);
        for (int k = i; k < n; ++k) z += Ti[i * n + k] * V[k * n + order[c]];
      } else {
        z = V[i * n + order[c]];
      }
      Z[(size_t)i * ldz + c] = (ZT)z;
    }
    return;
  }

  if (prm.mode == SM_USVP) {
    __shared__ T sv[kMaxSmall];
    T* Vb = Mq;            // basis, column c at Vb[i * n + c]
    T* w = Qe;             // n
    T* cf = Qe + n;        // n
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int rmax = fixed ? rt : min(prm.r_cap, n);
    const int q = max(0, prm.usvp_iters);
    // w = A v (A: the deflated Gram, global; v in sv), one warp per row
    auto matvec = [&]() {
      for (int i = warp; i < n; i += nwarps) {
        T acc = T(0);
        for (int c = lane; c < n; c += 32) acc += A[i * n + c] * sv[c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) w[i] = acc;
      }
      __syncthreads();
    };
    // sv <- src / ||src|| (returns ||src||^2)
    auto normalize_from = [&](const T* src) -> T {
      T s = T(0);
      for (int i = tid; i < n; i += nt) s += src[i] * src[i];
      s = block_sum(s, redt);
      const T inv = s > T(0) ? T(1) / sqrt(s) : T(0);
      for (int i = tid; i < n; i += nt) sv[i] = src[i] * inv;
      __syncthreads();
      return s;
    };
    // sv <- sv - V (V^T sv), twice, for the first r basis columns
    auto reorth = [&](int r) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int c = tid; c < r; c += nt) {
          T acc = T(0);
          for (int i = 0; i < n; ++i) acc += Vb[i * n + c] * sv[i];
          cf[c] = acc;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
          T acc = sv[i];
          for (int c = 0; c < r; ++c) acc -= Vb[i * n + c] * cf[c];
          w[i] = acc;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) sv[i] = w[i];
        __syncthreads();
      }
    };
    double tail = mu2 + tr;
    if (tid == 0) info->tails[0] = tail;
    int r = 0;
    while (r < rmax) {
      if (!fixed && r >= 1 && tail <= delta2) break;
      T best = lowest_value<T>();
      int bi = 0x7fffffff;
      for (int i = tid; i < n; i += nt) {
        const T a = A[i * n + i];
        if (a > best) {
          best = a;
          bi = i;
        }
      }
      T dmax;
      int j;
      block_argmax(best, bi, redt, redi, dmax, j);
      bool ok = dmax > T(0);
      if (ok) {
        // start: D^T D e_j (row j of the symmetric deflated Gram)
        for (int i = tid; i < n; i += nt) w[i] = A[j * n + i];
        __syncthreads();
        ok = normalize_from(w) > T(0);
        for (int it = 0; ok && it < q; ++it) {
          matvec();
          if (!(normalize_from(w) > T(0))) {
            // D^T D v = 0: keep the previous v (restored from the basis-free copy)
            for (int i = tid; i < n; i += nt) w[i] = A[j * n + i];
            __syncthreads();
            normalize_from(w);
            break;
          }
        }
        if (ok) {
          reorth(r);
          for (int i = tid; i < n; i += nt) w[i] = sv[i];
          __syncthreads();
          ok = normalize_from(w) > T(0);
        }
      }
      if (!ok) {
        if (!fixed) break;  // nothing left to capture
        // complete the fixed rank with unit vectors orthogonal to V
        bool found = false;
        for (int cand = 0; cand < n && !found; ++cand) {
          for (int i = tid; i < n; i += nt) sv[i] = (i == cand) ? T(1) : T(0);
          __syncthreads();
          reorth(r);
          for (int i = tid; i < n; i += nt) w[i] = sv[i];
          __syncthreads();
          found = normalize_from(w) > T(0.25);
        }
        if (!found) break;
      }
      // deflate: u = A v, lam = v^T u, A <- A - v u^T - u v^T + lam v v^T
      matvec();
      T lam = T(0);
      for (int i = tid; i < n; i += nt) lam += sv[i] * w[i];
      lam = block_sum(lam, redt);
      for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, c = e % n;
        A[e] = A[e] - sv[i] * w[c] - w[i] * sv[c] + lam * sv[i] * sv[c];
      }
      for (int i = tid; i < n; i += nt) Vb[i * n + r] = sv[i];
      __syncthreads();
      double t2 = 0.0;
      for (int i = tid; i < n; i += nt) t2 += (double)A[i * n + i];
      t2 = block_sum(t2, redd);
      tail = mu2 + fmax(t2, 0.0);
      ++r;
      if (tid == 0) info->tails[r] = tail;
    }
    if (r == 0) {  // a zero matrix: one unit vector (rank >= 1)
      for (int i = tid; i < n; i += nt) Vb[i * n] = (i == 0) ? T(1) : T(0);
      r = 1;
      if (tid == 0) info->tails[1] = tail;
    }
    __syncthreads();
    for (int e = tid; e < n * ldz; e += nt) {
      const int i = e / ldz, c = e % ldz;
      T z = T(0);
      if (c < r) {
        if (prm.Gw)
          for (int k = i; k < n; ++k) z += Ti[i * n + k] * Vb[k * n + c];
        else
          z = Vb[i * n + c];
      }
      Z[(size_t)i * ldz + c] = (ZT)z;
    }
    if (tid == 0) {
      info->r = r;
      info->k1 = r;
      info->nsteps = r;
      info->s1 = 0.0;
      info->tail = tail;
    }
    return;
  }

  if (prm.mode == SM_LURV) {
    // The whole chase of one vector is R <- Qr R G with G the column rotations
    // (fixed by v alone) and Qr the row rotations.  The row-rotation angles
    // follow from one scalar recurrence: at pair (p, p+1) the rotation zeroes
    // s_p rho_{p+1} against y_p = c_p R(p,p) + s_p R(p,p+1) (row p seen through
    // the column rotations right of it), giving rho_p^2 = y_p^2 + s_p^2
    // rho_{p+1}^2.  So the column rotations run first (one thread per row of
    // R and of V), the recurrence next (a warp scan of affine maps), and the
    // row rotations last (one thread per column); the product equals the
    // interleaved chase, and the entries below the diagonal, zero in exact
    // arithmetic, are set to zero.  R (and V) live in shared memory when they
    // fit, row-major R and column-major V with an odd leading dimension (both
    // the row-wise and the column-wise walks are then free of bank conflicts);
    // else column-major in the global work area.
    __shared__ T lva[kMaxSmall], lvb[kMaxSmall], lw[kMaxSmall], lcn[kMaxSmall];
    __shared__ T lcs[kMaxSmall], lsn[kMaxSmall], lcr[kMaxSmall], lsr[kMaxSmall];
    __shared__ T ldg[kMaxSmall], ly[kMaxSmall];
    __shared__ double lq[kMaxSmall];
    __shared__ T wpart[32];
    extern __shared__ __align__(16) unsigned char small_dyn[];
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5, half = nt >> 1;
    const unsigned full = 0xffffffffu;
    double s1;
    const int lds = n | 1;
    T* Rb;     // R(p, c) at Rb[p * rsp + c * rsc]
    T* Vb;     // V(p, c) at Vb[p + c * vsc]
    int rsp, rsc, vsc;
    int k1;
    if (prm.lurv_smem) {
      Rb = reinterpret_cast<T*>(small_dyn);
      rsp = lds;
      rsc = 1;
      for (int e = tid; e < n * n; e += nt) Rb[(e / n) * lds + e % n] = A[e];
      __syncthreads();
      k1 = pivoted_cholesky(Rb, n, perm1, prm.piv_tol, s1, redt, redi, redd, lds);
    } else {
      k1 = pivoted_cholesky(A, n, perm1, prm.piv_tol, s1, redt, redi, redd);
      Rb = Mq;
      rsp = 1;
      rsc = n;
      for (int e = tid; e < n * n; e += nt) Mq[e] = A[(e % n) * n + e / n];
    }
    if (prm.lurv_smem == 2) {
      Vb = Rb + (size_t)n * lds;
      vsc = lds;
    } else {
      Vb = Qe;
      vsc = n;
    }
    auto R_ = [&](int p, int c) -> T& { return Rb[p * rsp + c * rsc]; };
    for (int e = tid; e < n * n; e += nt) {
      const int c = e / n, p = e % n;
      Vb[p + c * vsc] = perm1[c] == p ? T(1) : T(0);
    }
    __syncthreads();
    const int rmax = max(1, fixed ? rt : min(prm.r_cap, n));
    const int q = max(0, prm.usvp_iters);
    const double base = mu2 + s1;
    // lcn[c] = ||R(i0:k1, c)||^2 for c >= i0; returns sum_{c >= i0} ||R(:, c)||^2
    auto col_sums = [&](int i0) -> double {
      double part = 0.0;
      for (int c = i0 + warp; c < n; c += nwarps) {
        T sa = T(0), st = T(0);
        const int pe = min(c + 1, k1);
        for (int p = lane; p < pe; p += 32) {
          const T x = R_(p, c);
          sa += x * x;
          if (p >= i0) st += x * x;
        }
        for (int o = 16; o > 0; o >>= 1) {
          sa += __shfl_xor_sync(full, sa, o);
          st += __shfl_xor_sync(full, st, o);
        }
        if (lane == 0) {
          lcn[c] = st;
          part += (double)sa;
        }
      }
      return block_sum(part, redd);
    };
    // dst[c] = sum_p R(p, c) src[p] over rows [i0, min(c + 1, k1)), columns
    // c >= i0: four threads per column, each a quarter of the rows, combined
    // by shuffles; returns ||dst||^2 (every thread, the warps' partial sums
    // added in one order)
    auto rt_mv = [&](T* dst, const T* src, int i0) -> T {
      const int cols = n - i0, qr = (k1 - i0 + 3) >> 2;
      T part = T(0);
      for (int b0 = 0; b0 < 4 * cols; b0 += nt) {
        const int t = b0 + tid, pc = t >> 2, q4 = t & 3;
        T acc = T(0);
        if (pc < cols) {
          const int c = i0 + pc;
          const int p0 = i0 + q4 * qr, p1 = min(min(c + 1, k1), p0 + qr);
          for (int p = p0; p < p1; ++p) acc += R_(p, c) * src[p];
        }
        acc += __shfl_xor_sync(full, acc, 1);
        acc += __shfl_xor_sync(full, acc, 2);
        if (pc < cols && q4 == 0) {
          dst[i0 + pc] = acc;
          part += acc * acc;
        }
      }
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(full, part, o);
      if (lane == 0) wpart[warp] = part;
      __syncthreads();
      T s = T(0);
      for (int w = 0; w < nwarps; ++w) s += wpart[w];
      return s;
    };
    // dst[p] = scale * sum_c R(p, c) src[c] over rows [i0, k1), columns
    // c >= p: four threads per row, each a quarter of the columns, combined
    // by shuffles
    auto r_mv = [&](T* dst, const T* src, T scale, int i0) {
      const int rows = k1 - i0, qc = (n - i0 + 3) >> 2;
      for (int b0 = 0; b0 < 4 * rows; b0 += nt) {
        const int t = b0 + tid, pr = t >> 2, q4 = t & 3;
        T acc = T(0);
        if (pr < rows) {
          const int p = i0 + pr;
          const int c0 = i0 + q4 * qc, c1 = min(n, c0 + qc);
          for (int c = max(c0, p); c < c1; ++c) acc += R_(p, c) * src[c];
        }
        acc += __shfl_xor_sync(full, acc, 1);
        acc += __shfl_xor_sync(full, acc, 2);
        if (pr < rows && q4 == 0) dst[i0 + pr] = acc * scale;
      }
      __syncthreads();
    };
    double tail = base + col_sums(0);
    if (tid == 0) info->tails[0] = tail;
    int i = 0;
    while (i < rmax) {
      if (fixed ? i >= rt : (i >= 1 && tail <= delta2)) break;
      bool rot = false;
      T* pv = lva;
      if (i < k1) {
        T best = lowest_value<T>();
        int bi = 0x7fffffff;
        for (int c = i + tid; c < n; c += nt)
          if (lcn[c] > best) {
            best = lcn[c];
            bi = c;
          }
        T cmax;
        int j0;
        block_argmax(best, bi, redt, redi, cmax, j0);
        if (cmax > T(0)) {
          // v ~ T^T T e_j0, then q power iterations v <- T^T T v; v is kept
          // unnormalized (the rotation angles depend on its direction only)
          // and the next product takes the scale 1 / ||v||
          for (int p = i + tid; p < k1; p += nt) lw[p] = R_(p, j0);
          __syncthreads();
          const T nv = rt_mv(lva, lw, i);
          rot = nv > T(0);
          if (rot) {
            T* pt = lvb;
            T scale = T(1) / sqrt(nv);
            for (int it = 0; it < q; ++it) {
              r_mv(lw, pv, scale, i);
              const T nw = rt_mv(pt, lw, i);
              if (!(nw > T(0))) break;  // T^T T v = 0: keep v
              T* t = pv;
              pv = pt;
              pt = t;
              scale = T(1) / sqrt(nw);
            }
          }
        }
      }
      if (rot) {
        // column rotations: (c_c, s_c) rotates (v_c, ||v(c+1:)||) onto
        // (||v(c:)||, 0); the last pair takes v_{n-1} itself.  Suffix sums of
        // squares by one warp: a serial run per lane, then a shuffle scan.
        if (warp == 0) {
          const int m = n - i, per = (m + 31) / 32;
          const int b0 = i + lane * per, b1 = min(b0 + per, n);
          double loc = 0.0;
          for (int t = b1 - 1; t >= b0; --t) loc += (double)pv[t] * (double)pv[t];
          double suf = loc;  // sum over lanes >= lane
          for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_down_sync(full, suf, o);
            if (lane + o < 32) suf += y;
          }
          double acc = __shfl_down_sync(full, suf, 1);
          if (lane == 31) acc = 0.0;
          for (int t = b1 - 1; t >= b0; --t) {
            acc += (double)pv[t] * (double)pv[t];
            lq[t] = acc;
          }
        }
        __syncthreads();
        for (int c = i + tid; c < n - 1; c += nt) {
          const double h = sqrt(lq[c]);
          const double b = c == n - 2 ? (double)pv[n - 1] : sqrt(lq[c + 1]);
          lcs[c] = h > 0.0 ? (T)((double)pv[c] / h) : T(1);
          lsn[c] = h > 0.0 ? (T)(b / h) : T(0);
        }
        __syncthreads();
        // threads [0, half): rows of R; [half, nt): rows of V
        const bool onR = tid < half;
        T* M = onR ? Rb : Vb;
        const int msp = onR ? rsp : 1, msc = onR ? rsc : vsc;
        const int rows = onR ? k1 : n;
        for (int p = onR ? tid : tid - half; p < rows; p += half) {
          T* row = M + (size_t)p * msp;  // entry c at row[c * msc]
          if (onR) ldg[p] = row[p * msc];
          T carry = row[(n - 1) * msc];
          for (int c0 = n - 2; c0 >= i; c0 -= 8) {
            T a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = c0 - u >= i ? row[(c0 - u) * msc] : T(0);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int c = c0 - u;
              if (c >= i) {
                const T cs = lcs[c], sn = lsn[c];
                const T na = cs * a[u] + sn * carry;
                if (onR && c == p) ly[p] = na;
                row[(c + 1) * msc] = -sn * a[u] + cs * carry;
                carry = na;
              }
            }
          }
          row[i * msc] = carry;
        }
        __syncthreads();
        // row rotations on (p, p+1), p from P0 down to i (rows below k1 only)
        const int P0 = min(n - 2, k1 - 2);
        if (P0 >= i) {
          const double rc0 = P0 + 1 <= n - 2 ? (double)ly[P0 + 1] : (double)ldg[P0 + 1];
          if (warp == 0) {
            // rho_p^2 = a_p x + b_p applied to x = rho_{p+1}^2, from x = rc0^2;
            // lane L composes the maps of its run of p (descending), then an
            // exclusive shuffle scan gives the value entering the run
            const int m = P0 - i + 1, per = (m + 31) / 32;
            const int t0 = lane * per, t1 = min(t0 + per, m);  // t = P0 - p
            double ca = 1.0, cb = 0.0;  // composed map x -> ca x + cb
            for (int t = t0; t < t1; ++t) {
              const int p = P0 - t;
              const double sp = (double)lsn[p], yp = (double)ly[p];
              const double a = sp * sp, b = yp * yp;
              cb = fma(a, cb, b);
              ca = a * ca;
            }
            // inclusive scan over lanes: G_L = F_L o ... o F_0
            double ga = ca, gb = cb;
            for (int o = 1; o < 32; o <<= 1) {
              const double pa = __shfl_up_sync(full, ga, o), pb = __shfl_up_sync(full, gb, o);
              if (lane >= o) {
                gb = fma(ga, pb, gb);
                ga = ga * pa;
              }
            }
            double ea = __shfl_up_sync(full, ga, 1), eb = __shfl_up_sync(full, gb, 1);
            if (lane == 0) {
              ea = 1.0;
              eb = 0.0;
            }
            double x = fma(ea, rc0 * rc0, eb);
            for (int t = t0; t < t1; ++t) {
              const int p = P0 - t;
              const double sp = (double)lsn[p], yp = (double)ly[p];
              x = fma(sp * sp, x, yp * yp);
              lq[p] = x;
            }
          }
          __syncthreads();
          for (int p = i + tid; p <= P0; p += nt) {
            const double rho = sqrt(lq[p]);
            const double prev = p == P0 ? rc0 : sqrt(lq[p + 1]);
            const double b = (double)lsn[p] * prev;
            lcr[p] = rho > 0.0 ? (T)((double)ly[p] / rho) : T(1);
            lsr[p] = rho > 0.0 ? (T)(b / rho) : T(0);
          }
          __syncthreads();
          for (int c = i + tid; c < n; c += nt) {
            T* col = Rb + (size_t)c * rsc;  // entry p at col[p * rsp]
            T carry = col[(P0 + 1) * rsp];
            for (int p0 = P0; p0 >= i; p0 -= 8) {
              T a[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) a[u] = p0 - u >= i ? col[(p0 - u) * rsp] : T(0);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int p = p0 - u;
                if (p >= i) {
                  const T cr = lcr[p], sr = lsr[p];
                  col[(p + 1) * rsp] = -sr * a[u] + cr * carry;
                  carry = cr * a[u] + sr * carry;
                }
              }
            }
            col[i * rsp] = carry;
            for (int p = max(c + 1, i); p < k1; ++p) col[p * rsp] = T(0);
          }
          __syncthreads();
        }
      }
      ++i;
      tail = base + col_sums(i);
      if (tid == 0) info->tails[i] = tail;
    }
    const int r = i;
    __syncthreads();
    for (int e = tid; e < n * ldz; e += nt) {
      const int row = e / ldz, c = e % ldz;
      T z = T(0);
      if (c < r) {
        if (prm.Gw)
          for (int k = row; k < n; ++k) z += Ti[row * n + k] * Vb[k + c * vsc];
        else
          z = Vb[row + c * vsc];
      }
      Z[(size_t)row * ldz + c] = (ZT)z;
    }
    if (tid == 0) {
      info->r = r;
      info->k1 = k1;
      info->nsteps = r;
      info->s1 = s1;
      info->tail = tail;
      if (prm.lurv_smem) info->status |= 4 * prm.lurv_smem;
    }
    return;
  }

  // ---- SM_QLP ----
  // (with prm.l11, the appendix's Alg. 4 keeping L_11 alone: order[] records
  // the second pivoting, d2[] the diagonal of R_2, and the error of rank j is
  // mu^2 + s1 + ||L||^2 - ||L(0:j, 0:j)||^2)
  __shared__ T d2[kMaxSmall];
  double s1;
  const int k1 = pivoted_cholesky(A, n, perm1, prm.piv_tol, s1, redt, redi, redd);
  // M = R_1^T (n x k1): rows are pivoted columns of X, columns the Cholesky rows.
  for (int e = tid; e < n * k1; e += nt) {
    const int i = e / k1, c = e % k1;
    Mq[i * n + c] = A[c * n + i];
  }
  for (int c = tid; c < n; c += nt) order[c] = c;
  __syncthreads();
  double totL2 = 0.0, l11sq = 0.0;
  if (prm.l11) {
    double part = 0.0;
    for (int e = tid; e < n * k1; e += nt) {
      const double x = (double)Mq[(e / k1) * n + e % k1];
      part += x * x;
    }
    totL2 = block_sum(part, redd);
  }
  const int kk = min(n, k1);
  int j = 0, r = 1;
  for (;; ++j) {
    double part = 0.0;
    for (int c = j + tid; c < k1; c += nt) {
      T s = T(0);
      for (int i = j; i < n; ++i) {
        const T x = Mq[i * n + c];
        s += x * x;
      }
      cn[c] = s;
      part += (double)s;
    }
    const double trail = block_sum(part, redd);
    double tj = mu2 + s1 + trail;
    if (prm.l11) {
      if (j >= 1) {  // column j-1 of R_2 is final: its part above and on the diagonal
        double pc = 0.0;
        for (int i = tid; i < j - 1; i += nt) {
          const double x = (double)Mq[i * n + (j - 1)];
          pc += x * x;
        }
        pc = block_sum(pc, redd);
        l11sq += pc + (double)d2[j - 1] * (double)d2[j - 1];
      }
      tj = mu2 + s1 + fmax(totL2 - l11sq, 0.0);
    }
    if (tid == 0) info->tails[j] = tj;
    if (fixed) {
      if (j == rt || j >= kk) {
        r = rt;
        break;
      }
    } else {
      if (j >= 1 && tj <= delta2) {
        r = min(j, prm.r_cap);
        break;
      }
      if (j >= kk || j >= prm.r_cap) {
        r = max(1, min(j, prm.r_cap));
        break;
      }
    }
    // pivot: largest remaining column norm
    T v = lowest_value<T>();
    int idx = 0x7fffffff;
    for (int c = j + tid; c < k1; c += nt) {
      if (cn[c] > v) {
        v = cn[c];
        idx = c;
      }
    }
    T cq;
    int q;
    block_argmax(v, idx, redt, redi, cq, q);
    if (q != j) {
      for (int i = tid; i < n; i += nt) swap_vals(Mq[i * n + j], Mq[i * n + q]);
      if (tid == 0) swap_vals(order[j], order[q]);
    }
    __syncthreads();
    const T alpha = sqrt(cq > T(0) ? cq : T(0));
    const T x0 = Mq[j * n + j];
    const T sg = x0 >= T(0) ? T(1) : T(-1);
    if (tid == 0) d2[j] = -sg * alpha;
    // tau = 2 / ||v||^2 from the stored v itself (FP64 sum): the reflector is
    // then orthogonal to working precision even when the column norm used for
    // alpha carries FP32 summation error.
    double rest = 0.0;
    for (int i = j + 1 + tid; i < n; i += nt) {
      const double x = (double)Mq[i * n + j];
      rest += x * x;
    }
    rest = block_sum(rest, redd);
    const double v0 = (double)(x0 + sg * alpha);
    const double vtv = v0 * v0 + rest;
    const T tj_ = vtv > 0.0 ? (T)(2.0 / vtv) : T(0);
    __syncthreads();
    if (tid == 0) {
      Mq[j * n + j] = x0 + sg * alpha;
      tau[j] = tj_;
    }
    __syncthreads();
    for (int c = j + 1 + tid; c < k1; c += nt) {
      T w = T(0);
      for (int i = j; i < n; ++i) w += Mq[i * n + j] * Mq[i * n + c];
      w *= tj_;
      for (int i = j; i < n; ++i) Mq[i * n + c] -= w * Mq[i * n + j];
    }
    __syncthreads();
  }
  const int nref = j;  // reflectors 0..nref-1 were formed
  // Z_1 = Pi_1 Q_2(:, 0:r): apply H_0 ... H_{nref-1} to the unit vectors.
  for (int c = tid; c < r; c += nt) {
    for (int i = 0; i < n; ++i) Qe[i * n + c] = (i == c) ? T(1) : T(0);
    for (int h = min(nref - 1, c); h >= 0; --h) {
      T w = T(0);
      for (int i = h; i < n; ++i) w += Mq[i * n + h] * Qe[i * n + c];
      w *= tau[h];
      for (int i = h; i < n; ++i) Qe[i * n + c] -= w * Mq[i * n + h];
    }
  }
  __syncthreads();
  if (prm.l11) {
    // B T = U_1 L_11 with T = Pi_1 R_11^{-1} E_J L_11: U_1 = Q_1(:, J) for the
    // rows J = order[0..rr) of R_1 taken first by the second pivoting, Q_1 =
    // B Pi_1 R_11^{-1}, and L_11 = R_1(J, :) Q_2(:, 0:r) (= R_2(0:r, 0:r)^T).
    // One thread per column t: the right-hand side E_J L_11(:, t) in Mq(:, t)
    // (pivot order), then back substitution with R_11 in place.
    const int rr = min(r, nref);
    for (int t = tid; t < r; t += nt) {
      for (int i = 0; i < k1; ++i) Mq[i * n + t] = T(0);
      for (int s2 = 0; s2 < rr; ++s2) {
        const int row = order[s2];
        T acc = T(0);
        for (int i = row; i < n; ++i) acc += A[row * n + i] * Qe[i * n + t];
        Mq[row * n + t] = acc;
      }
      for (int i = k1 - 1; i >= 0; --i) {
        T acc = Mq[i * n + t];
        for (int k = i + 1; k < k1; ++k) acc -= A[i * n + k] * Mq[k * n + t];
        Mq[i * n + t] = acc / A[i * n + i];
      }
    }
    __syncthreads();
    // Pi_1 Y into A (R_1 is no longer needed)
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, t = e % r;
      A[perm1[i] * n + t] = i < k1 ? Mq[i * n + t] : T(0);
    }
    __syncthreads();
    ZT* Tl = reinterpret_cast<ZT*>(prm.Tl);
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, t = e % r;
      T v;
      if (prm.Gw) {
        v = T(0);
        for (int k = i; k < n; ++k) v += Ti[i * n + k] * A[k * n + t];
      } else {
        v = A[i * n + t];
      }
      Tl[(size_t)i * ldz + t] = (ZT)v;
    }
    __syncthreads();
  }
  if (prm.Gw) {
    // Z_1 = T^{-1} Pi_1 Q_2(:, 0:r) (Mq is free again: hold Pi_1 Q_2 there)
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, c = e % r;
      Mq[perm1[i] * n + c] = Qe[i * n + c];
    }
    __syncthreads();
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, c = e % r;
      T acc = T(0);
      for (int k = i; k < n; ++k) acc += Ti[i * n + k] * Mq[k * n + c];
      Z[(size_t)i * ldz + c] = (ZT)acc;
    }
  } else {
    for (int e = tid; e < n * r; e += nt) {
      const int i = e / r, c = e % r;
      Z[(size_t)perm1[i] * ldz + c] = (ZT)Qe[i * n + c];
    }
  }
  if (tid == 0) {
    info->r = r;
    info->k1 = k1;
    info->nsteps = j;
    info->s1 = s1;
    info->tail = info->tails[min(r, j)];
  }
}

template <typename T, typename ZT>
cudaError_t launch_small(const double* G, SmallParams prm, void* Z, int ldz, void* ws,
                         StepInfo* info, cudaStream_t st) {
  const int n = prm.n;
  T* work = (T*)ws;
  size_t off = ((size_t)(4 * n * n + 2 * n) * sizeof(T) + 255) & ~(size_t)255;
  int* iwork = (int*)((char*)ws + off);
  size_t dyn = 0;
  prm.lurv_smem = 0;
  if (prm.mode == SM_LURV) {
    // R (and V) in shared memory when they fit beside the kernel's static
    // arrays; the opt-in limit is raised once
    // (per device: each device holds its own copy of the kernel's attributes)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
    static int room_p1[64];  // 1 + the room found on each device; 0: not yet
    int room = (dev >= 0 && dev < 64) ? room_p1[dev] - 1 : -1;
    if (room < 0) {
      int optin = 0;
      cudaFuncAttributes fa;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
              cudaSuccess ||
          cudaFuncGetAttributes(&fa, small_kernel<T, ZT>) != cudaSuccess)
        return cudaGetLastError();
      room = max(0, optin - (int)fa.sharedSizeBytes);
      if (room > 0 && cudaFuncSetAttribute(small_kernel<T, ZT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           room) != cudaSuccess) {
        (void)cudaGetLastError();
        room = 0;
      }
      if (dev >= 0 && dev < 64) room_p1[dev] = room + 1;
    }
    // R, then V, each n x (n | 1)
    const size_t need = (size_t)n * (n | 1) * sizeof(T);
    if (2 * need <= (size_t)room) {
      dyn = 2 * need;
      prm.lurv_smem = 2;
    } else if (need <= (size_t)room) {
      dyn = need;
      prm.lurv_smem = 1;
    }
  }
  count_launch();
  small_kernel<T, ZT><<<1, NT, dyn, st>>>(G, prm, work, iwork, (ZT*)Z, ldz, info);
  return cudaGetLastError();
}

}  // namespace

size_t small_ws_bytes(int n, bool fp64) {
  const size_t el = fp64 ? 8 : 4;
  const size_t nn = ((size_t)n + 31) / 32 * 32;
  size_t off = ((4 * nn * (nn + 1) + 2 * nn) * el + 255) & ~(size_t)255;
  return off + (size_t)2 * nn * sizeof(int) + 256;
}

cudaError_t small_factor(const double* G, SmallParams prm, bool fp64_math, void* Z, bool z_fp64,
                         int ldz, void* ws, StepInfo* info, cudaStream_t st) {
  if (prm.n < 1 || prm.n > kMaxSmall) return cudaErrorInvalidValue;
  if (small_fast_eligible(prm, fp64_math))
    return small_factor_fast(G, prm, fp64_math, Z, z_fp64, ldz, ws, info, st);
  if (fp64_math)
    return z_fp64 ? launch_small<double, double>(G, prm, Z, ldz, ws, info, st)
                  : launch_small<double, float>(G, prm, Z, ldz, ws, info, st);
  return z_fp64 ? launch_small<float, double>(G, prm, Z, ldz, ws, info, st)
                : launch_small<float, float>(G, prm, Z, ldz, ws, info, st);
}

TT_BOUNDS_READER(bounds_small)

}  // namespace ttk
