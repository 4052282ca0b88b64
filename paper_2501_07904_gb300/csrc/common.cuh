// Shared device-side definitions of the TT-UTV library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ttk {

constexpr int kMaxSmall = 256;  // largest Gram / sketch side factored by one CTA

// Bounds-checked build (-DTT_BOUNDS_CHECK): TT_IN(i, n) is false when i lies
// outside [0, n), and then counts the violation (and the source line of the
// first one) in this translation unit's device words; the caller skips the
// access, so the kernel goes on and the host reads the count through
// tt_bounds_violations.  Without the flag TT_IN is the constant true.
#ifdef TT_BOUNDS_CHECK
static __device__ unsigned int g_bc_count;
static __device__ int g_bc_line;
__device__ __forceinline__ bool bc_in(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_bc_count, 1u) == 0u) g_bc_line = line;
  return false;
}
#define TT_IN(i, n) (::ttk::bc_in((long long)(i), (long long)(n), __LINE__))
// This translation unit's count (and first line); reset zeroes it.
static inline unsigned int bc_read_tu(int* line, bool reset) {
  unsigned int c = 0;
  int l = 0;
  cudaMemcpyFromSymbol(&c, g_bc_count, sizeof c);
  cudaMemcpyFromSymbol(&l, g_bc_line, sizeof l);
  if (reset) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_bc_count, &z, sizeof z);
  }
  if (line) *line = l;
  return c;
}
#define TT_BOUNDS_READER(name) \
  unsigned int name(int* line, bool reset) { return bc_read_tu(line, reset); }
#else
#define TT_IN(i, n) true
#define TT_BOUNDS_READER(name)                    \
  unsigned int name(int* line, bool /*reset*/) {  \
    if (line) *line = 0;                          \
    return 0u;                                    \
  }
#endif

// Result of one small factorization, written by the single-CTA kernels and
// copied to the host once per sweep step (the next step's shapes need r).
struct StepInfo {
  int32_t r;         // chosen rank (or numerical rank k1 for the orthonormalization kernel)
  int32_t status;    // bit 0: non-finite input, bit 1: Jacobi not converged;
                     // bits 2-3 (Givens URV): R, or R and V, held in shared memory
  int32_t k1;        // steps taken by the pivoted Cholesky (numerical rank of the Gram)
  int32_t nsteps;    // QLP / Jacobi steps or sweeps done
  double x2;         // ||X||_F^2 of the factored matrix
  double trace;      // trace of the Gram matrix passed in
  double mu2;        // range miss x2 - trace (sketch path), 0 on the exact path
  double s1;         // energy left in the Schur complement when the pivoted Cholesky stopped
  double delta2;     // tolerance used for the rank decision
  double normA2;     // ||A||_F^2 seen by this step
  double tail;       // Gram-based truncation error ||E||_F^2 at rank r
  double tails[kMaxSmall + 1];  // tail(j) for j = 0..nsteps
};

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the multiply/xor round
// function with Weyl-sequence key bumps between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Sign of the Rademacher sketch entry Omega(i, j) of sweep step `step`:
// counter (i, j/128, step, purpose 0), key (seed lo, seed hi); bit j%128 of the
// 128-bit output, word (j%128)/32, bit j%32; +1 if the bit is 0.
__device__ __forceinline__ float sketch_sign(uint64_t i, uint64_t j, uint64_t seed, uint32_t step) {
  uint32_t c[4] = {(uint32_t)i, (uint32_t)(j >> 7), step, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t b = (uint32_t)(j & 127);
  const uint32_t w = c[b >> 5];
  return ((w >> (b & 31)) & 1u) ? -1.0f : 1.0f;
}

// Block-wide reductions (blockDim.x a multiple of 32, <= 1024).  `red` is
// shared scratch of at least 32 entries; every thread receives the result.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T s = (lane < nw) ? red[lane] : T(0);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <typename T> __device__ __forceinline__ T lowest_value();
template <> __device__ __forceinline__ float lowest_value<float>() { return -3.402823466e38f; }
template <> __device__ __forceinline__ double lowest_value<double>() { return -1.7976931348623157e308; }

// Argmax with the lowest index winning ties; non-candidates pass
// v = lowest_value<T>() and idx = INT_MAX.
template <typename T>
__device__ __forceinline__ void block_argmax(T v, int idx, T* redv, int* redi, T& best, int& bidx) {
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    redv[wid] = v;
    redi[wid] = idx;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T w = (lane < nw) ? redv[lane] : lowest_value<T>();
  int wi = (lane < nw) ? redi[lane] : 0x7fffffff;
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, w, o);
    const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
    if (ov > w || (ov == w && oi < wi)) {
      w = ov;
      wi = oi;
    }
  }
  best = w;
  bidx = wi;
}

}  // namespace ttk
