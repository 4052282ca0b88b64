// Elementwise kernels of the sweep (sketch matrix, casts, core copies,
// sums of squares).
#include <algorithm>
#include <atomic>

#include "internal.h"

namespace ttk {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kGrid = 152 * 8;
constexpr int kMaxModes = 16;
constexpr int TT_MAXD_INTERNAL = 18;

// Row i of the local block is row (i / blk) * stride + off + i % blk of the
// whole sketch (a slab of a partitioned unfolding draws the rows the whole
// unfolding would: blk = rows, off = 0 for an unpartitioned one).
template <typename T>
__global__ void fill_sketch_kernel(T* __restrict__ out, int64_t rows, int64_t cols, uint64_t seed,
                                   uint32_t step, bool identity, int64_t blk, int64_t stride,
                                   int64_t off) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    const int64_t gi = (i / blk) * stride + off + i % blk;
    T v;
    if (identity)
      v = (gi == j) ? T(1) : T(0);
    else
      v = (T)sketch_sign((uint64_t)gi, (uint64_t)j, seed, step);
    out[e] = v;
  }
}

template <typename TI, typename TO>
__global__ void cast_kernel(const TI* __restrict__ in, TO* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (TO)in[e];
}

template <typename T>
__global__ void copy2d_kernel(const T* __restrict__ in, int64_t ldi, bool trans,
                              T* __restrict__ out, int64_t ldo, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    out[i * ldo + j] = trans ? in[j * ldi + i] : in[i * ldi + j];
  }
}

template <typename T>
__global__ void sumsq_kernel(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[e];
    s += v * v;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_parts_kernel(const double* __restrict__ v, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// Columns of a partitioned unfolding back in order: `in` holds P rank blocks
// [P][rows][outer * blk] (rank p's columns are its slab of the fastest mode:
// blk of them per outer index), `out` is [rows][outer * P * blk] with column
// (o, p, t) at o * P * blk + p * blk + t.
template <typename T>
__global__ void unshard_cols_kernel(const T* __restrict__ in, T* __restrict__ out, int P, int64_t rows,
                                    int64_t outer, int64_t blk) {
  const int64_t nl = outer * blk, total = (int64_t)P * rows * nl;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e % blk, o = (e / blk) % outer, i = (e / nl) % rows, p = e / (nl * rows);
    const int64_t dst = i * (outer * P * blk) + o * P * blk + p * blk + t;
    if (TT_IN(dst, total)) out[dst] = in[e];
  }
}

// ---- mode reversal (the index-reversed tensor of the Remark after Thm 3.2)
struct RevArgs {
  int nmid;                 // middle modes 1 .. d-2
  int64_t i1, id;           // sizes of the first and last mode
  int64_t mid_dims[kMaxModes];
  int64_t mid_in[kMaxModes];   // input stride of each middle mode
  int64_t mid_out[kMaxModes];  // output stride of each middle mode
  int64_t s_in1, s_outd;       // input stride of mode 1, output stride of mode d
  int64_t nmidtot, t1, td;     // middle index count; tiles along modes 1 and d
  int64_t total;               // elements of the tensor (bounds-checked build)
};

// out[i_d, ..., i_1] = in[i_1, ..., i_d], both row-major.  A block moves one
// 32 x 32 tile of (i_1, i_d) for one middle index: it reads rows of i_d
// (contiguous in the input) and writes rows of i_1 (contiguous in the output).
template <typename T>
__global__ void __launch_bounds__(256) reverse_modes_kernel(const T* __restrict__ in,
                                                            T* __restrict__ out, RevArgs a) {
  __shared__ T tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t ntiles = a.nmidtot * a.t1 * a.td;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t tdi = t % a.td, rest = t / a.td;
    const int64_t t1i = rest % a.t1, mid = rest / a.t1;
    int64_t mi = 0, mo = 0, r = mid;
    for (int k = a.nmid - 1; k >= 0; --k) {
      const int64_t ik = r % a.mid_dims[k];
      r /= a.mid_dims[k];
      mi += ik * a.mid_in[k];
      mo += ik * a.mid_out[k];
    }
    for (int q = ty; q < 32; q += 8) {
      const int64_t i1 = t1i * 32 + q, id = tdi * 32 + tx;
      const int64_t src = i1 * a.s_in1 + mi + id;
      if (i1 < a.i1 && id < a.id && TT_IN(src, a.total)) tile[q][tx] = in[src];
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int64_t id = tdi * 32 + q, i1 = t1i * 32 + tx;
      const int64_t dst = id * a.s_outd + mo + i1;
      if (i1 < a.i1 && id < a.id && TT_IN(dst, a.total)) out[dst] = tile[tx][q];
    }
    __syncthreads();
  }
}

// out[b][i][a] = in[a][i][b] for an [A][I][B] array (a core of the reversed
// tensor read back as a core of the original one).
template <typename T>
__global__ void swap_outer_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t A,
                                  int64_t I, int64_t B) {
  const int64_t total = A * I * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % A, rest = e / A;
    const int64_t i = rest % I, b = rest / I;
    const int64_t src = (a * I + i) * B + b;
    if (TT_IN(src, total)) out[e] = in[src];
  }
}

// ---- streamed reconstruction error
// part[2 b] (+)= sum (a - x)^2 and part[2 b + 1] (+)= sum a^2 over block b's
// grid-stride share, in FP64; `first` starts the sums (slabs are processed in
// order on one stream, so the totals are deterministic).
template <typename T>
__global__ void diff_sumsq_kernel(const T* __restrict__ a, const T* __restrict__ x, int64_t n,
                                  double* __restrict__ part, bool first) {
  __shared__ double red[32];
  double s = 0.0, q = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double av = (double)a[e], dv = av - (double)x[e];
    s += dv * dv;
    q += av * av;
  }
  s = block_sum(s, red);
  q = block_sum(q, red);
  if (threadIdx.x == 0) {
    if (first) {
      part[2 * blockIdx.x] = s;
      part[2 * blockIdx.x + 1] = q;
    } else {
      part[2 * blockIdx.x] += s;
      part[2 * blockIdx.x + 1] += q;
    }
  }
}

__global__ void sum_pairs_kernel(const double* __restrict__ v, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s += v[2 * i];
    q += v[2 * i + 1];
  }
  s = block_sum(s, red);
  q = block_sum(q, red);
  if (threadIdx.x == 0) {
    out[0] = s;
    out[1] = q;
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > kGrid) b = kGrid;
  return (int)b;
}

}  // namespace

cudaError_t fill_sketch(void* out, bool fp64, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t step, bool identity, cudaStream_t st, int64_t blk, int64_t stride,
                        int64_t off) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (blk <= 0) blk = rows;
  count_launch(1);
  const int g = grid_for(rows * cols, 256);
  if (fp64)
    fill_sketch_kernel<double><<<g, 256, 0, st>>>((double*)out, rows, cols, seed, step, identity, blk,
                                                  stride, off);
  else
    fill_sketch_kernel<float><<<g, 256, 0, st>>>((float*)out, rows, cols, seed, step, identity, blk,
                                                 stride, off);
  return cudaGetLastError();
}

cudaError_t unshard_cols(const void* in, void* out, bool fp64, int P, int64_t rows, int64_t outer,
                         int64_t blk, cudaStream_t st) {
  const int64_t total = (int64_t)P * rows * outer * blk;
  if (total <= 0) return cudaSuccess;
  count_launch();
  const int g = grid_for(total, 256);
  if (fp64)
    unshard_cols_kernel<double><<<g, 256, 0, st>>>((const double*)in, (double*)out, P, rows, outer, blk);
  else
    unshard_cols_kernel<float><<<g, 256, 0, st>>>((const float*)in, (float*)out, P, rows, outer, blk);
  return cudaGetLastError();
}

cudaError_t cast_copy(const void* in, bool in64, void* out, bool out64, int64_t n,
                      cudaStream_t st) {
  const int g = grid_for(n, 256);
  if (in64 != out64) count_launch();
  if (in64 && !out64)
    cast_kernel<double, float><<<g, 256, 0, st>>>((const double*)in, (float*)out, n);
  else if (!in64 && out64)
    cast_kernel<float, double><<<g, 256, 0, st>>>((const float*)in, (double*)out, n);
  else
    return cudaMemcpyAsync(out, in, n * (in64 ? 8 : 4), cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

cudaError_t copy2d(const void* in, int64_t ldi, bool trans, void* out, int64_t ldo, int64_t rows,
                   int64_t cols, bool fp64, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int g = grid_for(rows * cols, 256);
  count_launch();
  if (fp64)
    copy2d_kernel<double><<<g, 256, 0, st>>>((const double*)in, ldi, trans, (double*)out, ldo,
                                             rows, cols);
  else
    copy2d_kernel<float><<<g, 256, 0, st>>>((const float*)in, ldi, trans, (float*)out, ldo, rows,
                                            cols);
  return cudaGetLastError();
}

size_t sumsq_ws_bytes(int64_t) { return (size_t)kGrid * sizeof(double) + 256; }

cudaError_t sumsq(const void* x, bool fp64, int64_t n, double* out, void* ws, cudaStream_t st) {
  count_launch(2);
  const int g = grid_for(n, 256);
  double* part = (double*)ws;
  if (fp64)
    sumsq_kernel<double><<<g, 256, 0, st>>>((const double*)x, n, part);
  else
    sumsq_kernel<float><<<g, 256, 0, st>>>((const float*)x, n, part);
  sum_parts_kernel<<<1, 1024, 0, st>>>(part, g, out);
  return cudaGetLastError();
}

cudaError_t reverse_modes(const void* in, void* out, bool fp64, int d, const int64_t* dims,
                          cudaStream_t st) {
  if (d < 2 || d - 2 > kMaxModes) return cudaErrorInvalidValue;
  RevArgs a;
  a.nmid = d - 2;
  a.i1 = dims[0];
  a.id = dims[d - 1];
  // input strides: S_k = prod dims[k+1 ..]; output (modes reversed): prod dims[.. k-1]
  int64_t sin[TT_MAXD_INTERNAL], sout[TT_MAXD_INTERNAL];
  sin[d - 1] = 1;
  for (int k = d - 2; k >= 0; --k) sin[k] = sin[k + 1] * dims[k + 1];
  sout[0] = 1;
  for (int k = 1; k < d; ++k) sout[k] = sout[k - 1] * dims[k - 1];
  a.nmidtot = 1;
  for (int k = 1; k < d - 1; ++k) {
    a.mid_dims[k - 1] = dims[k];
    a.mid_in[k - 1] = sin[k];
    a.mid_out[k - 1] = sout[k];
    a.nmidtot *= dims[k];
  }
  a.s_in1 = sin[0];
  a.s_outd = sout[d - 1];
  a.t1 = (a.i1 + 31) / 32;
  a.td = (a.id + 31) / 32;
  a.total = a.i1 * a.nmidtot * a.id;
  const int64_t ntiles = a.nmidtot * a.t1 * a.td;
  if (ntiles <= 0) return cudaSuccess;
  const int g = (int)std::min<int64_t>(ntiles, (int64_t)kGrid * 2);
  count_launch(1);
  if (fp64)
    reverse_modes_kernel<double><<<g, 256, 0, st>>>((const double*)in, (double*)out, a);
  else
    reverse_modes_kernel<float><<<g, 256, 0, st>>>((const float*)in, (float*)out, a);
  return cudaGetLastError();
}

cudaError_t swap_outer(const void* in, void* out, bool fp64, int64_t A, int64_t I, int64_t B,
                       cudaStream_t st) {
  const int64_t n = A * I * B;
  if (n <= 0) return cudaSuccess;
  count_launch(1);
  const int g = grid_for(n, 256);
  if (fp64)
    swap_outer_kernel<double><<<g, 256, 0, st>>>((const double*)in, (double*)out, A, I, B);
  else
    swap_outer_kernel<float><<<g, 256, 0, st>>>((const float*)in, (float*)out, A, I, B);
  return cudaGetLastError();
}

size_t diff_sumsq_parts_bytes() { return (size_t)2 * kGrid * sizeof(double); }

cudaError_t diff_sumsq(const void* a, const void* x, bool fp64, int64_t n, double* part,
                       bool first, cudaStream_t st) {
  count_launch(1);
  // every slab launches the full grid so each block's slot is written by
  // the first slab and accumulated by the later ones
  if (fp64)
    diff_sumsq_kernel<double><<<kGrid, 256, 0, st>>>((const double*)a, (const double*)x, n, part, first);
  else
    diff_sumsq_kernel<float><<<kGrid, 256, 0, st>>>((const float*)a, (const float*)x, n, part, first);
  return cudaGetLastError();
}

cudaError_t sum_pairs(const double* part, double* out, cudaStream_t st) {
  count_launch(1);
  sum_pairs_kernel<<<1, 1024, 0, st>>>(part, kGrid, out);
  return cudaGetLastError();
}

TT_BOUNDS_READER(bounds_misc)

}  // namespace ttk
