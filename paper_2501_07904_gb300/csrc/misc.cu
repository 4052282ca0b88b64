// Elementwise kernels of the sweep (sketch matrix, casts, core copies,
// sums of squares) and the masked TT evaluation with its gradient.
#include <atomic>

#include "internal.h"

namespace ttk {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kGrid = 152 * 8;

template <typename T>
__global__ void fill_sketch_kernel(T* __restrict__ out, int64_t rows, int64_t cols, uint64_t seed,
                                   uint32_t step, bool identity) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    T v;
    if (identity)
      v = (i == j) ? T(1) : T(0);
    else
      v = (T)sketch_sign((uint64_t)i, (uint64_t)j, seed, step);
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

constexpr int kEvalMaxD = 16;
constexpr int kEvalMaxR = 64;

struct EvalArgs {
  int d;
  int64_t dims[kEvalMaxD];
  int ranks[kEvalMaxD + 1];
  const float* cores[kEvalMaxD];
  float* grads[kEvalMaxD];
};

__device__ __forceinline__ void decode(const EvalArgs& a, int64_t lin, int* ix) {
  for (int k = a.d - 1; k >= 0; --k) {
    ix[k] = (int)(lin % a.dims[k]);
    lin /= a.dims[k];
  }
}

// x = G_1[i_1] ... G_d[i_d], left to right, one entry per thread.
__global__ void eval_kernel(EvalArgs a, const int64_t* __restrict__ idx, int64_t n,
                            float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ix[kEvalMaxD];
    decode(a, idx[e], ix);
    float v[kEvalMaxR], w[kEvalMaxR];
    v[0] = 1.0f;
    for (int k = 0; k < a.d; ++k) {
      const int r0 = a.ranks[k], r1 = a.ranks[k + 1];
      const float* g = a.cores[k] + (int64_t)ix[k] * r1;  // G_k[a, i_k, b] at (a*I_k + i_k)*r1 + b
      const int64_t sa = a.dims[k] * r1;
      for (int b = 0; b < r1; ++b) w[b] = 0.0f;
      for (int q = 0; q < r0; ++q) {
        const float vq = v[q];
        const float* gr = g + q * sa;
        for (int b = 0; b < r1; ++b) w[b] = fmaf(vq, gr[b], w[b]);
      }
      for (int b = 0; b < r1; ++b) v[b] = w[b];
    }
    out[e] = v[0];
  }
}

// dG_k[:, i_k, :] += gout * left_k^T right_k^T, interfaces recomputed per core.
__global__ void eval_backward_kernel(EvalArgs a, const int64_t* __restrict__ idx, int64_t n,
                                     const float* __restrict__ gout) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ix[kEvalMaxD];
    decode(a, idx[e], ix);
    const float g = gout[e];
    for (int k = 0; k < a.d; ++k) {
      float left[kEvalMaxR], right[kEvalMaxR], w[kEvalMaxR];
      // left = G_1[i_1] ... G_{k-1}[i_{k-1}]  (1 x r_{k-1})
      left[0] = 1.0f;
      for (int t = 0; t < k; ++t) {
        const int r0 = a.ranks[t], r1 = a.ranks[t + 1];
        const float* gg = a.cores[t] + (int64_t)ix[t] * r1;
        const int64_t sa = a.dims[t] * r1;
        for (int b = 0; b < r1; ++b) w[b] = 0.0f;
        for (int q = 0; q < r0; ++q)
          for (int b = 0; b < r1; ++b) w[b] = fmaf(left[q], gg[q * sa + b], w[b]);
        for (int b = 0; b < r1; ++b) left[b] = w[b];
      }
      // right = G_{k+1}[i_{k+1}] ... G_d[i_d]  (r_k x 1)
      right[0] = 1.0f;
      for (int t = a.d - 1; t > k; --t) {
        const int r0 = a.ranks[t], r1 = a.ranks[t + 1];
        const float* gg = a.cores[t] + (int64_t)ix[t] * r1;
        const int64_t sa = a.dims[t] * r1;
        for (int q = 0; q < r0; ++q) {
          float s = 0.0f;
          for (int b = 0; b < r1; ++b) s = fmaf(gg[q * sa + b], right[b], s);
          w[q] = s;
        }
        for (int q = 0; q < r0; ++q) right[q] = w[q];
      }
      const int r0 = a.ranks[k], r1 = a.ranks[k + 1];
      float* gk = a.grads[k] + (int64_t)ix[k] * r1;
      const int64_t sa = a.dims[k] * r1;
      for (int q = 0; q < r0; ++q) {
        const float lq = g * left[q];
        for (int b = 0; b < r1; ++b) atomicAdd(gk + q * sa + b, lq * right[b]);
      }
    }
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > kGrid) b = kGrid;
  return (int)b;
}

bool fill_eval_args(EvalArgs& a, int d, const int64_t* dims, const int64_t* ranks,
                    const float* const* cores, float* const* grads) {
  if (d < 1 || d > kEvalMaxD) return false;
  a.d = d;
  for (int k = 0; k < d; ++k) {
    a.dims[k] = dims[k];
    a.cores[k] = cores[k];
    a.grads[k] = grads ? grads[k] : nullptr;
  }
  for (int k = 0; k <= d; ++k) {
    if (ranks[k] < 1 || ranks[k] > kEvalMaxR) return false;
    a.ranks[k] = (int)ranks[k];
  }
  return a.ranks[0] == 1 && a.ranks[d] == 1;
}

}  // namespace

cudaError_t fill_sketch(void* out, bool fp64, int64_t rows, int64_t cols, uint64_t seed,
                        uint32_t step, bool identity, cudaStream_t st) {
  count_launch(1);
  const int g = grid_for(rows * cols, 256);
  if (fp64)
    fill_sketch_kernel<double><<<g, 256, 0, st>>>((double*)out, rows, cols, seed, step, identity);
  else
    fill_sketch_kernel<float><<<g, 256, 0, st>>>((float*)out, rows, cols, seed, step, identity);
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

cudaError_t eval_at(int d, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                    const int64_t* idx, int64_t n, float* out, cudaStream_t st) {
  EvalArgs a;
  if (!fill_eval_args(a, d, dims, ranks, cores, nullptr)) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  count_launch();
  eval_kernel<<<grid_for(n, 128), 128, 0, st>>>(a, idx, n, out);
  return cudaGetLastError();
}

cudaError_t eval_at_backward(int d, const int64_t* dims, const int64_t* ranks,
                             const float* const* cores, const int64_t* idx, int64_t n,
                             const float* gout, float* const* grads, cudaStream_t st) {
  EvalArgs a;
  if (!fill_eval_args(a, d, dims, ranks, cores, grads)) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  count_launch();
  eval_backward_kernel<<<grid_for(n, 128), 128, 0, st>>>(a, idx, n, gout);
  return cudaGetLastError();
}

}  // namespace ttk
