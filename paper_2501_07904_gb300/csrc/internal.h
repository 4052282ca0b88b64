// Host-side launchers shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace ttk {

// Set the thread-local message returned by tt_last_error().
void set_last_error(const char* msg);

// Process-wide count of kernels launched by this library.
void count_launch(int n = 1);
uint64_t launches();

// Matrix operand: element (i, j) is p[i*ld + j] (row) or p[i + j*ld] (!row).
template <typename T>
struct Mat {
  const T* p;
  int64_t ld;
  bool row;
};

// D (M x N) = A (M x K) B (K x N), FP32 or FP64 data.  FP32 products are
// summed in FP32 over 16 products, those sums in FP32 over 32 tiles, and the
// result in FP64, so an output carries no more than ~1e-6 relative rounding
// from long inner products.  When the M x N tile grid cannot fill the GPU the
// K range is split and the FP64 partials are summed in a fixed order.
//   out     T output (ld ldo), may be null when out64 is given;
//   out64   FP64 output (ld N), may be null;
//   sym     A = B^T (a Gram matrix): only tiles on or above the diagonal are
//           computed and the result is mirrored;
//   sumsq   if non-null, receives sum of squares of the T-rounded outputs (FP64);
//   accurate FP32 data only: each product split exactly into two FP32 words
//           and summed with TwoSum compensation, folded into FP64 every 128
//           products (error ~1e-13 of sum |a b|), for Gram matrices whose
//           truncation errors must be resolved below FP32 rounding.
// Scratch comes from `ws` (gemm_ws_bytes); returns the first launch error.
template <typename T>
size_t gemm_ws_bytes(int64_t M, int64_t N, int64_t K, bool fp64_out_or_sym);
template <typename T>
cudaError_t gemm(Mat<T> A, Mat<T> B, int64_t M, int64_t N, int64_t K, T* out, int64_t ldo,
                 double* out64, bool sym, double* sumsq, void* ws, cudaStream_t st,
                 bool accurate = false);

// Tensor-core product (tc_gemm.cu): same contract as gemm<float> for FP32
// data, computed with tcgen05 MMAs on TF32 operands rounded to nearest and
// FP32 accumulation.  A split operand is carried as hi + lo (both TF32),
// which makes its products accurate to ~2^-22 relative; round_out rounds the
// FP32 result to TF32 (so it is exact as a later TF32 operand).  err is a
// device int set to 1 when a bounded wait in the kernel ran out.
// tc_gemm returns cudaErrorNotSupported for shapes or layouts it does not
// take (leading dimensions not a multiple of 4, unaligned pointers, too many
// Gram tiles); callers then use gemm<float>.
struct TcOpts {
  bool a_split = false;
  bool b_split = false;
  bool round_out = false;
  int* err = nullptr;
};
bool tc_gemm_eligible(Mat<float> A, Mat<float> B, int64_t M, int64_t N, int64_t K);
size_t tc_gemm_ws_bytes(int64_t M, int64_t N, int64_t K, bool sym, bool out64, bool a_split,
                        bool b_split);
cudaError_t tc_gemm(Mat<float> A, Mat<float> B, int64_t M, int64_t N, int64_t K, float* out,
                    int64_t ldo, double* out64, bool sym, double* sumsq, void* ws, cudaStream_t st,
                    TcOpts o);

// Diagnostic: the tensor-core kernels' bounded mbarrier wait on a barrier
// that is (arrive) or is not completed; err (device int) is set to 1 when the
// wait runs out after limit_ns.
cudaError_t wait_selftest(bool arrive, uint64_t limit_ns, int* err, cudaStream_t st);

// Small single-CTA factorizations of an n x n FP64 Gram matrix (n <= 256).
enum SmallMode { SM_QLP = 0, SM_JACOBI = 1, SM_ORTH = 2, SM_USVP = 3, SM_LURV = 4 };
struct SmallParams {
  int n;                  // Gram size
  int mode;               // SmallMode
  int r_fixed;            // -1: rank by tolerance
  int r_cap;              // largest admissible rank
  double delta2;          // tolerance (used when normA2_dev == null)
  const double* normA2_dev;  // if set: delta2 = delta2_scale * (*normA2_dev or trace)
  int normA2_is_trace;    // 1: ||A||^2 is this Gram's trace (first exact step)
  double delta2_scale;
  const double* x2_dev;   // ||X||^2 of the factored matrix, null on the exact path (x2 = trace)
  double piv_tol;         // relative pivot tolerance of the (pivoted) Cholesky
  double shift_rel;       // SM_ORTH: diagonal shift, relative to trace(G)
  const double* Gw;       // QLP/Jacobi on a sketch: W^T W of the range basis, or null
  int range_exact;        // 1: the sketch is the identity, so W spans X's row space (mu^2 = 0)
  int df_math;            // with fp64_math: run the fast path in double-float (n <= 64)
  int usvp_iters;         // SM_USVP / SM_LURV: power iterations per vector
  // SM_QLP, appendix Alg. 4 with L_11 kept alone: rank by the error
  // mu^2 + ||L||^2 - ||L_11||^2, and Tl (n x r, ld = ldz, Z's type) receives
  // T with B T = U_1 L_11 (runs on the generic kernel)
  int l11;
  void* Tl;
  int jacobi_sweeps;      // SM_JACOBI sweep cap (0: the default 60)
  int lurv_smem;          // SM_LURV, set by the launcher: 1 R, 2 R and V in dynamic shared memory
};
size_t small_ws_bytes(int n, bool fp64);
// Register-resident fast path (small_fast.cu) for SM_QLP / SM_ORTH with
// n <= 128 (FP32) or n <= 64 (FP64); small_factor() dispatches to it.
bool small_fast_eligible(const SmallParams& prm, bool fp64);
cudaError_t small_factor_fast(const double* G, SmallParams prm, bool fp64_math, void* Z,
                              bool z_fp64, int ldz, void* ws, StepInfo* info, cudaStream_t st);
// Z (n x ldz, written as T_out = float/double per zfp64) receives the basis Z_1
// (QLP/Jacobi) or the orthonormalizing factor S (ORTH).
cudaError_t small_factor(const double* G, SmallParams prm, bool fp64_math, void* Z, bool z_fp64,
                         int ldz, void* ws, StepInfo* info, cudaStream_t st);

// Elementwise helpers.
// Rows of the sketch: local row i is global row (i / blk) * stride + off + i % blk
// (blk <= 0: the identity mapping), the rows a slab of a partitioned unfolding owns.
cudaError_t fill_sketch(void* out, bool fp64, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t step, bool identity, cudaStream_t st, int64_t blk = 0,
                        int64_t stride = 0, int64_t off = 0);
cudaError_t cast_copy(const void* in, bool in64, void* out, bool out64, int64_t n, cudaStream_t st);
// Gathered column blocks [P][rows][outer * blk] of a partitioned unfolding
// (rank p: blk consecutive columns of each outer group) back to
// [rows][outer * P * blk] in column order.
cudaError_t unshard_cols(const void* in, void* out, bool fp64, int P, int64_t rows, int64_t outer,
                         int64_t blk, cudaStream_t st);
cudaError_t copy2d(const void* in, int64_t ldi, bool trans, void* out, int64_t ldo, int64_t rows,
                   int64_t cols, bool fp64, cudaStream_t st);
size_t sumsq_ws_bytes(int64_t n);
cudaError_t sumsq(const void* x, bool fp64, int64_t n, double* out, void* ws, cudaStream_t st);
// out = in with its d modes in reverse order (dims are in's mode sizes).
cudaError_t reverse_modes(const void* in, void* out, bool fp64, int d, const int64_t* dims,
                          cudaStream_t st);
// out[b][i][a] = in[a][i][b] for an [A][I][B] array.
cudaError_t swap_outer(const void* in, void* out, bool fp64, int64_t A, int64_t I, int64_t B,
                       cudaStream_t st);
// Streamed ||A - X||^2 and ||A||^2 in FP64 over slabs: part (diff_sumsq_parts_bytes())
// is started by the first slab (first = true) and accumulated by the later ones;
// sum_pairs writes the two totals to out[0], out[1].
size_t diff_sumsq_parts_bytes();
cudaError_t diff_sumsq(const void* a, const void* x, bool fp64, int64_t n, double* part,
                       bool first, cudaStream_t st);
cudaError_t sum_pairs(const double* part, double* out, cudaStream_t st);

// Bounds-check counters of each translation unit (zero without -DTT_BOUNDS_CHECK).
unsigned int bounds_driver(int* line, bool reset);
unsigned int bounds_gemm(int* line, bool reset);
unsigned int bounds_masked(int* line, bool reset);
unsigned int bounds_misc(int* line, bool reset);
unsigned int bounds_small(int* line, bool reset);
unsigned int bounds_small_fast(int* line, bool reset);
unsigned int bounds_tc_gemm(int* line, bool reset);

}  // namespace ttk
